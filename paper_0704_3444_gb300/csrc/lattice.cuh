// lattice.cuh -- D2Q9 lattice, storage precisions and kernel parameters shared by
// every kernel of the library.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "mclb_internal.h"

namespace mclb {

// D2Q9 velocities v_i and weights w_i (c_s^2 = 1/3), in the order
// (0,0), (1,0), (0,1), (-1,0), (0,-1), (1,1), (-1,1), (-1,-1), (1,-1).
__host__ __device__ __forceinline__ constexpr int vx(int i)
{
    return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
// Index of the opposite velocity, v_opp9(i) = -v_i.
__host__ __device__ __forceinline__ constexpr int opp9(int i)
{
    return i == 0 ? 0 : (i <= 4 ? (i <= 2 ? i + 2 : i - 2) : (i <= 6 ? i + 2 : i - 2));
}

__host__ __device__ __forceinline__ constexpr int vy(int i)
{
    return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
template <typename C>
__host__ __device__ __forceinline__ constexpr C wq(int i)
{
    return i == 0 ? C(4.0 / 9.0) : (i < 5 ? C(1.0 / 9.0) : C(1.0 / 36.0));
}
// FP32 weights whose exact sum is 1.  The floats nearest to 4/9, 1/9 and 1/36 sum to
// 1 + 7.45e-9, and every step would add that fraction of each site's mass through the
// equilibria (sum_i f^e_i = rho^s sum_i w_i, Sec. 3) and, in the 16-bit formats, again
// when the populations are rebuilt from the reference density: a steady drift of the
// component masses (3e-4 after 40 000 steps).  Taking w_5..8 one unit in the last place
// below the nearest float to 1/36 (14913080 * 2^-29) makes w_0 + 4 w_1 + 4 w_5 = 1
// exactly, with w_0 and w_1 the nearest floats.
template <>
__host__ __device__ __forceinline__ constexpr float wq<float>(int i)
{
    return i == 0 ? float(4.0 / 9.0) : (i < 5 ? float(1.0 / 9.0) : 14913080.0f * 0x1p-29f);
}

// Storage precisions.  C is the arithmetic type.  The 16-bit formats ("shifted") hold,
// per site and component, the deviations f_i - w_i R in 16 bits and the reference
// density R in FP32 (a separate line per component row), so that the few mantissa
// bits describe the departure from the local equilibrium-like part rather than f
// itself; R is chosen so that the stored site mass sum_i f_i is exact in FP32.
template <typename T>
struct Storage;

template <>
struct Storage<double> {
    using C = double;
    static constexpr bool shifted = false;
    __device__ __forceinline__ static C load(const double* p) { return __ldg(p); }
    __device__ __forceinline__ static void store(double* p, C v) { *p = v; }
    __device__ __forceinline__ static C round(C v) { return v; }
};

template <>
struct Storage<float> {
    using C = float;
    static constexpr bool shifted = false;
    __device__ __forceinline__ static C load(const float* p) { return __ldg(p); }
    __device__ __forceinline__ static void store(float* p, C v) { *p = v; }
    __device__ __forceinline__ static C round(C v) { return v; }
};

template <>
struct Storage<__nv_bfloat16> {
    using C = float;
    static constexpr bool shifted = true;
    __device__ __forceinline__ static C load(const __nv_bfloat16* p)
    {
        return __bfloat162float(__ldg(p));
    }
    __device__ __forceinline__ static void store(__nv_bfloat16* p, C v)
    {
        *p = __float2bfloat16_rn(v);
    }
    __device__ __forceinline__ static C round(C v) { return __bfloat162float(__float2bfloat16_rn(v)); }
    __device__ __forceinline__ static __nv_bfloat16 pack(C v) { return __float2bfloat16_rn(v); }
};

template <>
struct Storage<__half> {
    using C = float;
    static constexpr bool shifted = true;
    __device__ __forceinline__ static C load(const __half* p) { return __half2float(__ldg(p)); }
    __device__ __forceinline__ static void store(__half* p, C v) { *p = __float2half_rn(v); }
    __device__ __forceinline__ static C round(C v) { return __half2float(__float2half_rn(v)); }
    __device__ __forceinline__ static __half pack(C v) { return __float2half_rn(v); }
};

// Kernel parameters in the arithmetic type.  Built on the host from a Problem.
template <typename C>
struct StepParams {
    int nx, ny;
    int nz;               // layers (D3Q19), 1 otherwise
    long long S;
    int hx;               // ghost columns per side
    long long pitch;      // elements per (row, velocity) line
    long long plane;      // elements per component (ny * 9 * pitch)
    long long rbytes;     // byte offset of the FP32 density lines in a buffer (16-bit formats)
    C omega;              // 1 / tau
    C fcoef;              // 1 - 1/(2 tau), Eq. definef
    C gx, gy, gz;         // body acceleration
    C kappa, theta;
    C log_floor;          // floor of rho^s / rho inside a logarithm
    int bary;             // 1: barycentric u in the forcing's second moment, 0: u^s (Eq. ff3)
    int gd;               // 1: Gibbs-Duhem total force (kappa = 0), 0: Eq. definef as printed
    int walls;            // 1: solid walls below row 0 and above row ny - 1 (D2Q9)
    long long band;       // staged launches: 0 = every site; > 0 = the first and the last
                          // `band` sites only (the rows next to the walls)
    C chi[NMAX * NMAX];
    C th_m[NMAX];         // theta / m^s
    C logc[NMAX];         // theta / m^s - 1/3: coefficient of ln rho^s in nu^s
    C m_inv_m1[NMAX];     // 1/m^s - 1
    C inv_m[NMAX];        // 1/m^s
    C m[NMAX];
    unsigned int log_mask; // bit s set when logc[s] != 0
    int withhold;          // test hook: the single-pass kernel issues no copies
    unsigned int* status;
};

template <typename C>
inline StepParams<C> make_params(const Problem& P, unsigned int* status)
{
    StepParams<C> p{};
    p.nx = P.nx;
    p.ny = P.ny;
    p.nz = P.nz > 0 ? P.nz : 1;
    p.S = P.S;
    p.hx = P.hx;
    p.pitch = P.pitch;
    p.plane = P.plane;
    p.rbytes = P.rbytes;
    p.omega = C(1.0 / P.tau);
    p.fcoef = C(1.0 - 1.0 / (2.0 * P.tau));
    p.gx = C(P.gx);
    p.gy = C(P.gy);
    p.gz = C(P.gz);
    p.kappa = C(P.kappa);
    p.theta = C(P.theta);
    p.log_floor = C(1e-12);
    p.bary = P.forcing_velocity;
    p.gd = P.force_form;
    p.walls = P.walls;
    p.band = 0;
    p.log_mask = 0;
    for (int a = 0; a < P.N; ++a) {
        for (int b = 0; b < P.N; ++b) p.chi[a * P.N + b] = C(P.chi[a * P.N + b]);
        double c = P.theta / P.m[a] - 1.0 / 3.0;
        p.th_m[a] = C(P.theta / P.m[a]);
        p.logc[a] = C(c);
        if (c != 0.0) p.log_mask |= 1u << a;
        p.m_inv_m1[a] = C(1.0 / P.m[a] - 1.0);
        p.inv_m[a] = C(1.0 / P.m[a]);
        p.m[a] = C(P.m[a]);
    }
    p.withhold = P.withhold;
    p.status = status;
    return p;
}

// a + d mod n for |d| <= n
__device__ __forceinline__ int wrap_add(int a, int d, int n)
{
    a += d;
    a += (a < 0) ? n : 0;
    a -= (a >= n) ? n : 0;
    return a;
}

// Offset of the start (ghosts included) of the line of component s, row y, velocity i.
template <typename C>
__device__ __forceinline__ long long line_off(const StepParams<C>& p, int s, int y, int i)
{
    return ((long long)s * p.ny + y) * (Q * p.pitch) + (long long)i * p.pitch;
}

// Element offset of (s, i, y, x) with 0 <= x < nx in the ghost-padded layout.
template <typename C>
__device__ __forceinline__ long long fidx(const StepParams<C>& p, int s, int i, int y, int x)
{
    return line_off(p, s, y, i) + p.hx + x;
}

// Store one distribution value at column x of a line (row points at the line start,
// ghosts included) and at every ghost column that repeats column x.
template <typename T, typename C>
__device__ __forceinline__ void store_row(T* row, int x, int nx, int hx, C v)
{
    Storage<T>::store(row + hx + x, v);
    if (x < hx)
        for (int g = nx + x; g < nx + hx; g += nx) Storage<T>::store(row + hx + g, v);
    if (x >= nx - hx)
        for (int g = x - nx; g >= -hx; g -= nx) Storage<T>::store(row + hx + g, v);
}

// Start (ghosts included) of the FP32 density line of component s, row y (16-bit formats).
template <typename T, typename C>
__device__ __forceinline__ float* rho_line(T* f, const StepParams<C>& p, int s, int y)
{
    return reinterpret_cast<float*>(reinterpret_cast<char*>(f) + p.rbytes) +
           ((long long)s * p.ny + y) * p.pitch;
}
template <typename T, typename C>
__device__ __forceinline__ const float* rho_line(const T* f, const StepParams<C>& p, int s, int y)
{
    return reinterpret_cast<const float*>(reinterpret_cast<const char*>(f) + p.rbytes) +
           ((long long)s * p.ny + y) * p.pitch;
}

// Store the nine post-collision values of component s at column x of row y, ghosts
// included.  In the 16-bit formats the values become deviations d_i = f_i - w_i M
// (M = sum_i f_i) rounded to 16 bits, and the FP32 reference R = M - sum_i d_i, so that
// sum_i (d_i + w_i R) = M: every site keeps its mass to FP32 rounding.
template <typename T, typename C>
__device__ __forceinline__ void store_site(T* f, const StepParams<C>& p, int s, int y, int x,
                                           const C (&out)[Q])
{
    if constexpr (!Storage<T>::shifted) {
#pragma unroll
        for (int i = 0; i < Q; ++i) store_row(f + line_off(p, s, y, i), x, p.nx, p.hx, out[i]);
    } else {
        C M = C(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) M += out[i];
        C dsum = C(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const C d = Storage<T>::round(out[i] - wq<C>(i) * M);
            dsum += d;
            store_row(f + line_off(p, s, y, i), x, p.nx, p.hx, d);
        }
        store_row(rho_line(f, p, s, y), x, p.nx, p.hx, M - dsum);
    }
}

}  // namespace mclb
