// cube.cuh -- the D3Q19 lattice: the staged timestep (three launches) and the diagnostics.
//
// The method's equations are written for any lattice whose weights give the Sec. 3
// moments; D3Q19 (the rest velocity, weight 1/3; six axis directions, 1/18; twelve face
// diagonals, 1/36; c_s^2 = 1/3) is isotropic to fourth order, so the equilibrium and
// forcing polynomials of the D2Q9 path, with three-component dot products, keep the
// Sec. 3 and Eqs. ff1-ff3 moments.  The stages are those of the D2Q9 staged schedule
// (staged.cuh), with the discrete operators over the nineteen velocities:
//   k19_density    rho^s = sum_i f^s_i(r - v_i)                     (Eq. ssLB streaming)
//   k19_potential  nu^s = mu^s/m^s - kappa lap rho^s - (1/3) ln rho^s (Eq. lgf, Eq. definef)
//   k19_collide    pull again, j^s, u, a^s = -(1 - 1/2tau) grad nu^s + g, f^e, F, BGK
// lap g = 6 sum_i w_i (g(r + v_i) - g(r)), grad g = 3 sum_i w_i v_i g(r + v_i); periodic
// in x, y and z; the per-site chemistry (site_nu, site_mu, site_psi) is shared with D2Q9.
//
// Layout: component s, layer z, row y, velocity i, column x at
//   (((s * nz + z) * ny + y) * 19 + i) * nx + x
// (the nineteen velocity lines of one (z, y) row adjacent; no ghost columns), holding
// post-collision values: the pre-collision f^s_i(r) is the value stored at r - v_i.
// Velocity order: 0; (+-1,0,0), (0,+-1,0), (0,0,+-1); (1,1,0), (-1,-1,0), (1,-1,0),
// (-1,1,0), (1,0,1), (-1,0,-1), (1,0,-1), (-1,0,1), (0,1,1), (0,-1,-1), (0,1,-1),
// (0,-1,1).  FP64 and FP32 storage.
#pragma once

#include "staged.cuh"

namespace mclb {

constexpr int Q19 = 19;

// Component d (0: x, 1: y, 2: z) of velocity i.
__host__ __device__ __forceinline__ constexpr int c19(int i, int d)
{
    return d == 0 ? ((i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1
                     : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0)
         : d == 1 ? ((i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1
                     : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0)
                  : ((i == 5 || i == 11 || i == 14 || i == 15 || i == 18) ? 1
                     : (i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0);
}

// Weights.  FP32: w0 = 2796203 * 2^-23, w1 = 1864135 * 2^-25 (axis), w2 = 1864135 * 2^-26
// (diagonal), whose sum w0 + 6 w1 + 12 w2 is exactly 1 (with the rounded 1/3, 1/18 and
// 1/36 it is 1 + 1.5e-8, a fixed-sign bias of every site's equilibrium mass).
template <typename C>
__host__ __device__ __forceinline__ constexpr C w19(int i);
template <>
__host__ __device__ __forceinline__ constexpr double w19<double>(int i)
{
    return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
}
template <>
__host__ __device__ __forceinline__ constexpr float w19<float>(int i)
{
    return i == 0 ? 2796203.0f * 0x1p-23f : (i <= 6 ? 1864135.0f * 0x1p-25f : 1864135.0f * 0x1p-26f);
}

// Site coordinates of a linear site index (z * ny + y) * nx + x (< 2^31: one 32-bit
// division per thread, none per neighbour).
struct Site3 {
    int x, y, z;
};
template <typename C>
__device__ __forceinline__ Site3 site3(const StepParams<C>& p, long long site)
{
    const unsigned t = (unsigned)site, nx = (unsigned)p.nx, ny = (unsigned)p.ny;
    const unsigned row = t / nx;
    Site3 c;
    c.x = (int)(t - row * nx);
    c.z = (int)(row / ny);
    c.y = (int)(row - (unsigned)c.z * ny);
    return c;
}

// A neighbour (x + dx, y + dy, z + dz), periodic, as its row z * ny + y and column x.
struct Nb3 {
    int row, x;
};
template <typename C>
__device__ __forceinline__ Nb3 nb3(const StepParams<C>& p, const Site3& c, int dx, int dy, int dz)
{
    Nb3 n;
    n.x = wrap_add(c.x, dx, p.nx);
    n.row = wrap_add(c.z, dz, p.nz) * p.ny + wrap_add(c.y, dy, p.ny);
    return n;
}

// Per-thread neighbourhood: the three wrapped columns x - 1, x, x + 1 and, for a (dy, dz)
// row offset, the start of that row in the stored layout (in units of elements: row *
// 19 * nx) and in an N * S field (row * nx).  Each (dy, dz) pair is shared by one to
// three velocities, so the compiler forms each row base once.
struct Hood3 {
    int xw[3];
};
template <typename C>
__device__ __forceinline__ Hood3 hood3(const StepParams<C>& p, const Site3& c)
{
    Hood3 h;
    h.xw[0] = wrap_add(c.x, -1, p.nx);
    h.xw[1] = c.x;
    h.xw[2] = wrap_add(c.x, 1, p.nx);
    return h;
}
template <typename C>
__device__ __forceinline__ int row3(const StepParams<C>& p, const Site3& c, int dy, int dz)
{
    return wrap_add(c.z, dz, p.nz) * p.ny + wrap_add(c.y, dy, p.ny);
}
// stored element (component 0) of velocity i pulled by the site: (row, x) of r - v_i
template <typename C>
__device__ __forceinline__ long long src19(const StepParams<C>& p, const Site3& c, const Hood3& h,
                                           int i)
{
    const long long rb = (long long)row3(p, c, -c19(i, 1), -c19(i, 2)) * (Q19 * (long long)p.nx);
    return rb + (long long)i * p.nx + h.xw[1 - c19(i, 0)];
}
// field index of the neighbour r + v_i
template <typename C>
__device__ __forceinline__ long long fnb3(const StepParams<C>& p, const Site3& c, const Hood3& h,
                                         int i)
{
    return (long long)row3(p, c, c19(i, 1), c19(i, 2)) * p.nx + h.xw[1 + c19(i, 0)];
}

// Linear site index of a neighbour (index into an N * S field: s * S + nbr3(...)).
template <typename C>
__device__ __forceinline__ long long nbr3(const StepParams<C>& p, const Site3& c, int dx, int dy,
                                          int dz)
{
    const Nb3 n = nb3(p, c, dx, dy, dz);
    return (long long)n.row * p.nx + n.x;
}

// Stored element (component 0, velocity i) of the site at (row, x); component s is
// s * 19 * S further.
template <typename C>
__device__ __forceinline__ long long at19(const StepParams<C>& p, int i, int row, int x)
{
    return ((long long)row * Q19 + i) * p.nx + x;
}

// Pre-collision f^s_i at site c: the post-collision value stored at c - v_i.
template <typename T>
__device__ __forceinline__ typename Storage<T>::C pull19(const T* __restrict__ f,
                                                         const StepParams<typename Storage<T>::C>& p,
                                                         int s, int i, const Site3& c)
{
    const Nb3 n = nb3(p, c, -c19(i, 0), -c19(i, 1), -c19(i, 2));
    return Storage<T>::load(f + (long long)s * Q19 * p.S + at19(p, i, n.row, n.x));
}

// rho^s and, when js is given, the momenta j^s = sum_i f^s_i v_i ([s][d][site]) that the
// collision would otherwise pull the populations a second time to form.
template <typename T, int N>
__global__ void __launch_bounds__(SITE_THREADS)
k19_density(const T* __restrict__ f, typename Storage<T>::C* __restrict__ rs,
            typename Storage<T>::C* __restrict__ js,
            const __grid_constant__ StepParams<typename Storage<T>::C> p)
{
    using C = typename Storage<T>::C;
    const long long site = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (site >= p.S) return;
    const Site3 c = site3(p, site);
    const Hood3 h = hood3(p, c);
    C r[N], j[N][3];
#pragma unroll
    for (int s = 0; s < N; ++s) r[s] = j[s][0] = j[s][1] = j[s][2] = C(0);
#pragma unroll
    for (int i = 0; i < Q19; ++i) {
        const T* src = f + src19(p, c, h, i);
#pragma unroll
        for (int s = 0; s < N; ++s) {
            const C v = Storage<T>::load(src + (long long)s * Q19 * p.S);
            r[s] += v;
#pragma unroll
            for (int d = 0; d < 3; ++d)
                if (c19(i, d)) j[s][d] += C(c19(i, d)) * v;
        }
    }
#pragma unroll
    for (int s = 0; s < N; ++s) rs[s * p.S + site] = r[s];
    if (js)
#pragma unroll
        for (int s = 0; s < N; ++s)
#pragma unroll
            for (int d = 0; d < 3; ++d) js[(s * 3 + d) * p.S + site] = j[s][d];
}

// lap g = 6 sum_i w_i (g(r + v_i) - g(r)) of every component's density field (each
// neighbour's index formed once for all components).
template <typename C, int N>
__device__ __forceinline__ void laplacians19(const C* __restrict__ rs, const StepParams<C>& p,
                                             const Site3& c, const C (&r)[N], C (&lap)[N])
{
    C acc[N];
    const Hood3 h = hood3(p, c);
#pragma unroll
    for (int s = 0; s < N; ++s) acc[s] = C(0);
#pragma unroll
    for (int i = 1; i < Q19; ++i) {
        const long long t = fnb3(p, c, h, i);
#pragma unroll
        for (int s = 0; s < N; ++s) acc[s] += w19<C>(i) * (rs[s * p.S + t] - r[s]);
    }
#pragma unroll
    for (int s = 0; s < N; ++s) lap[s] = C(6) * acc[s];
}

template <typename C, int N>
__global__ void __launch_bounds__(SITE_THREADS)
k19_potential(const C* __restrict__ rs, C* __restrict__ nu, const __grid_constant__ StepParams<C> p)
{
    const long long site = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (site >= p.S) return;
    const Site3 c = site3(p, site);
    C r[N], lap[N], out[N];
#pragma unroll
    for (int s = 0; s < N; ++s) r[s] = rs[s * p.S + site];
    laplacians19<C, N>(rs, p, c, r, lap);
    site_nu<C, N>(p, r, lap, out);
#pragma unroll
    for (int s = 0; s < N; ++s) nu[s * p.S + site] = out[s];
}

// grad g = 3 sum_i w_i v_i g(r + v_i) of one scalar field.
template <typename C>
__device__ __forceinline__ void grad19(const C* __restrict__ g, const StepParams<C>& p,
                                       const Site3& c, C (&gr)[3])
{
    C a0 = C(0), a1 = C(0), a2 = C(0);
#pragma unroll
    for (int i = 1; i < Q19; ++i) {
        const C v = w19<C>(i) * g[nbr3(p, c, c19(i, 0), c19(i, 1), c19(i, 2))];
        if (c19(i, 0)) a0 += C(c19(i, 0)) * v;
        if (c19(i, 1)) a1 += C(c19(i, 1)) * v;
        if (c19(i, 2)) a2 += C(c19(i, 2)) * v;
    }
    gr[0] = C(3) * a0;
    gr[1] = C(3) * a1;
    gr[2] = C(3) * a2;
}

// grad g = 3 sum_i w_i v_i g(r + v_i) of N fields g + s * S at once.
template <typename C, int N>
__device__ __forceinline__ void grads19(const C* __restrict__ g, const StepParams<C>& p,
                                        const Site3& c, C (&gr)[N][3])
{
    const Hood3 h = hood3(p, c);
#pragma unroll
    for (int s = 0; s < N; ++s) gr[s][0] = gr[s][1] = gr[s][2] = C(0);
#pragma unroll
    for (int i = 1; i < Q19; ++i) {
        const long long t = fnb3(p, c, h, i);
#pragma unroll
        for (int s = 0; s < N; ++s) {
            const C v = w19<C>(i) * g[s * p.S + t];
#pragma unroll
            for (int d = 0; d < 3; ++d)
                if (c19(i, d)) gr[s][d] += C(c19(i, d)) * v;
        }
    }
#pragma unroll
    for (int s = 0; s < N; ++s)
#pragma unroll
        for (int d = 0; d < 3; ++d) gr[s][d] *= C(3);
}

// Accelerations a^s (Eq. definef plus the body force; with p.gd the Gibbs-Duhem shift
// (A_c - A)/rho of every component, A = sum_s rho^s (a^s - g), A_c = (1 - 1/2tau)
// (1/3) grad rho).  r: the site's rho^s, rho their sum.
template <typename C, int N>
__device__ __forceinline__ void accel19(const C* __restrict__ rs, const C* __restrict__ nu,
                                        const StepParams<C>& p, const Site3& c, const C (&r)[N],
                                        C rho, C (&a)[N][3])
{
    const C g[3] = {p.gx, p.gy, p.gz};
    grads19<C, N>(nu, p, c, a);
#pragma unroll
    for (int s = 0; s < N; ++s)
#pragma unroll
        for (int d = 0; d < 3; ++d) a[s][d] = -p.fcoef * a[s][d] + g[d];
    if (p.gd) {
        C grt[3] = {C(0), C(0), C(0)};
        C gs[N][3];
        grads19<C, N>(rs, p, c, gs);
#pragma unroll
        for (int s = 0; s < N; ++s)
#pragma unroll
            for (int d = 0; d < 3; ++d) grt[d] += gs[s][d];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            C A = C(0);
#pragma unroll
            for (int s = 0; s < N; ++s) A += r[s] * (a[s][d] - g[d]);
            const C sh = (p.fcoef * grt[d] / C(3) - A) / rho;
#pragma unroll
            for (int s = 0; s < N; ++s) a[s][d] += sh;
        }
    }
}

// rs, js: the densities and momenta k19_density wrote for fin (the same sums, in the same
// order, as pulling the populations here would form)
template <typename T, int N>
__global__ void __launch_bounds__(SITE_THREADS, 2)
k19_collide(const T* __restrict__ fin, T* __restrict__ fout,
            const typename Storage<T>::C* __restrict__ rs,
            const typename Storage<T>::C* __restrict__ js,
            const typename Storage<T>::C* __restrict__ nu,
            const __grid_constant__ StepParams<typename Storage<T>::C> p)
{
    using C = typename Storage<T>::C;
    const long long site = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (site >= p.S) return;
    const Site3 c = site3(p, site);
    const Hood3 h = hood3(p, c);
    const long long cstride = (long long)Q19 * p.S;   // one component's stored values
    C r[N], j[N][3];
#pragma unroll
    for (int s = 0; s < N; ++s) {
        r[s] = rs[s * p.S + site];
#pragma unroll
        for (int d = 0; d < 3; ++d) j[s][d] = js[(s * 3 + d) * p.S + site];
    }
    C rho = C(0), jt[3] = {C(0), C(0), C(0)};
#pragma unroll
    for (int s = 0; s < N; ++s) {
        rho += r[s];
#pragma unroll
        for (int d = 0; d < 3; ++d) jt[d] += j[s][d];
    }
    const C inv = C(1) / rho;
    const C u[3] = {jt[0] * inv, jt[1] * inv, jt[2] * inv};
    const C base = C(-1.5) * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    C a[N][3];
    accel19<C, N>(rs, nu, p, c, r, rho, a);
    // f* = f (1 - 1/tau) + (rho^s/tau) e_i + w_i [3 rho^s (v.a) + 9 (v.a)(v.J) - 3 a.J
    // + rho^s/tau], e_i = w_i (3 v.u + 9/2 (v.u)^2 - 3/2 u.u), J = j^s or rho^s u (Eq. ff3);
    // J is kept in j, and the per-component constants are formed once
    C r3[N], omr[N], m3aj[N];
#pragma unroll
    for (int s = 0; s < N; ++s) {
        if (p.bary)
#pragma unroll
            for (int d = 0; d < 3; ++d) j[s][d] = r[s] * u[d];
        r3[s] = C(3) * r[s];
        omr[s] = p.omega * r[s];
        m3aj[s] = fma(C(-3), a[s][0] * j[s][0] + a[s][1] * j[s][1] + a[s][2] * j[s][2], omr[s]);
    }
    const C keep = C(1) - p.omega;
    const Nb3 here = nb3(p, c, 0, 0, 0);
    T* dst = fout + at19(p, 0, here.row, here.x);
#pragma unroll
    for (int i = 0; i < Q19; ++i) {
        C cu = C(0);
#pragma unroll
        for (int d = 0; d < 3; ++d)
            if (c19(i, d)) cu += C(c19(i, d)) * u[d];
        const C e = (i == 0) ? w19<C>(0) * base : w19<C>(i) * fma(cu, fma(C(4.5), cu, C(3)), base);
        const T* src = fin + src19(p, c, h, i);
#pragma unroll
        for (int s = 0; s < N; ++s) {
            C ca = C(0), cj = C(0);
#pragma unroll
            for (int d = 0; d < 3; ++d)
                if (c19(i, d)) {
                    ca += C(c19(i, d)) * a[s][d];
                    cj += C(c19(i, d)) * j[s][d];
                }
            const C F = (i == 0) ? w19<C>(0) * m3aj[s]
                                 : w19<C>(i) * fma(ca, fma(C(9), cj, r3[s]), m3aj[s]);
            const C v = Storage<T>::load(src + s * cstride);
            dst[s * cstride + (long long)i * p.nx] = T(fma(keep, v, fma(omr[s], e, F)));
        }
    }
    if (!(rho > C(0)) || !isfinite(rho)) atomicOr(p.status, STATUS_NONFINITE);
}

// ---------------------------------------------------------------- diagnostics

// Stored so that pulling yields f^e_i(rho^s, u) at every site: the value of velocity i at
// site r is the equilibrium at r + v_i (u: 3 * S values, or null for rest).
template <typename T, int N>
__global__ void __launch_bounds__(SITE_THREADS)
k19_init(const double* __restrict__ rho, const double* __restrict__ u, T* __restrict__ f,
         const __grid_constant__ StepParams<typename Storage<T>::C> p)
{
    using C = typename Storage<T>::C;
    const long long site = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (site >= p.S) return;
    const Site3 c = site3(p, site);
#pragma unroll
    for (int i = 0; i < Q19; ++i) {
        const long long t = nbr3(p, c, c19(i, 0), c19(i, 1), c19(i, 2));
        C uu = C(0), cu = C(0);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const C ud = u ? C(u[d * p.S + t]) : C(0);
            uu += ud * ud;
            cu += C(c19(i, d)) * ud;
        }
        const Nb3 h = nb3(p, c, 0, 0, 0);
#pragma unroll
        for (int s = 0; s < N; ++s)
            f[(long long)s * Q19 * p.S + at19(p, i, h.row, h.x)] =
                T(w19<C>(i) * C(rho[s * p.S + t]) * (C(1) + C(3) * cu + C(4.5) * cu * cu - C(1.5) * uu));
    }
}

template <typename T, int N>
__global__ void __launch_bounds__(SITE_THREADS)
k19_get_state(const T* __restrict__ f, double* __restrict__ out,
              const __grid_constant__ StepParams<typename Storage<T>::C> p)
{
    const long long site = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (site >= p.S) return;
    const Site3 c = site3(p, site);
#pragma unroll
    for (int s = 0; s < N; ++s)
#pragma unroll
        for (int i = 0; i < Q19; ++i) out[(s * Q19 + i) * p.S + site] = (double)pull19(f, p, s, i, c);
}

template <typename T, int N>
__global__ void __launch_bounds__(SITE_THREADS)
k19_set_state(const double* __restrict__ in, T* __restrict__ f,
              const __grid_constant__ StepParams<typename Storage<T>::C> p)
{
    using C = typename Storage<T>::C;
    const long long site = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (site >= p.S) return;
    const Site3 c = site3(p, site);
#pragma unroll
    for (int i = 0; i < Q19; ++i) {
        const long long t = nbr3(p, c, c19(i, 0), c19(i, 1), c19(i, 2));
        const Nb3 h = nb3(p, c, 0, 0, 0);
#pragma unroll
        for (int s = 0; s < N; ++s)
            f[(long long)s * Q19 * p.S + at19(p, i, h.row, h.x)] = T(C(in[(s * Q19 + i) * p.S + t]));
    }
}

// Output fields (after k19_density and k19_potential of the same state): rho^s; U (3 * S)
// = u + (sum_s rho^s a^s)/(2 rho) (Eq. scon); mu^s; P (6 * S: xx, xy, xz, yy, yz, zz) =
// (sum_s rho^s mu^s - psi) I + kappa sum_s grad rho^s grad rho^s (Eq. ppp, diagnostic).
template <typename T, int N>
__global__ void __launch_bounds__(SITE_THREADS)
k19_moments(const T* __restrict__ f, const typename Storage<T>::C* __restrict__ rs,
            const typename Storage<T>::C* __restrict__ nu, double* __restrict__ rho_out,
            double* __restrict__ U, double* __restrict__ mu_out, double* __restrict__ P,
            const __grid_constant__ StepParams<typename Storage<T>::C> p)
{
    using C = typename Storage<T>::C;
    const long long site = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (site >= p.S) return;
    const Site3 c = site3(p, site);
    C r[N];
    C rho = C(0);
#pragma unroll
    for (int s = 0; s < N; ++s) {
        r[s] = rs[s * p.S + site];
        rho += r[s];
    }
    if (rho_out)
#pragma unroll
        for (int s = 0; s < N; ++s) rho_out[s * p.S + site] = (double)r[s];
    if (U) {
        C jt[3] = {C(0), C(0), C(0)}, ft[3] = {C(0), C(0), C(0)};
        C a[N][3];
        accel19<C, N>(rs, nu, p, c, r, rho, a);
#pragma unroll
        for (int s = 0; s < N; ++s) {
#pragma unroll
            for (int i = 0; i < Q19; ++i) {
                const C v = pull19(f, p, s, i, c);
#pragma unroll
                for (int d = 0; d < 3; ++d) jt[d] += v * C(c19(i, d));
            }
#pragma unroll
            for (int d = 0; d < 3; ++d) ft[d] += r[s] * a[s][d];
        }
#pragma unroll
        for (int d = 0; d < 3; ++d) U[d * p.S + site] = (double)(jt[d] / rho + C(0.5) * ft[d] / rho);
    }
    if (mu_out || P) {
        C lap[N], mu[N];
        laplacians19<C, N>(rs, p, c, r, lap);
        site_mu<C, N>(p, r, lap, mu);
        if (mu_out)
#pragma unroll
            for (int s = 0; s < N; ++s) mu_out[s * p.S + site] = (double)mu[s];
        if (P) {
            const C psi = site_psi<C, N>(p, r);
            C rmu = C(0), gg = C(0), t[6] = {C(0), C(0), C(0), C(0), C(0), C(0)};
#pragma unroll
            for (int s = 0; s < N; ++s) {
                C g[3];
                grad19(rs + s * p.S, p, c, g);
                rmu += r[s] * mu[s];
                gg += C(0.5) * p.kappa * (g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
                t[0] += p.kappa * g[0] * g[0];
                t[1] += p.kappa * g[0] * g[1];
                t[2] += p.kappa * g[0] * g[2];
                t[3] += p.kappa * g[1] * g[1];
                t[4] += p.kappa * g[1] * g[2];
                t[5] += p.kappa * g[2] * g[2];
            }
            const C iso = rmu - (psi + gg);
            P[site] = (double)(iso + t[0]);
            P[p.S + site] = (double)t[1];
            P[2 * p.S + site] = (double)t[2];
            P[3 * p.S + site] = (double)(iso + t[3]);
            P[4 * p.S + site] = (double)t[4];
            P[5 * p.S + site] = (double)(iso + t[5]);
        }
    }
}

// Conservation sums (after k19_density and k19_potential): mass^s, momentum (3), force
// sum_s rho^s a^s (3), as per-block FP64 partials (fixed grid, fixed tree).
template <typename T, int N>
__global__ void __launch_bounds__(SITE_THREADS)
k19_conservation(const T* __restrict__ f, const typename Storage<T>::C* __restrict__ rs,
                 const typename Storage<T>::C* __restrict__ nu, double* __restrict__ partial,
                 const __grid_constant__ StepParams<typename Storage<T>::C> p)
{
    using C = typename Storage<T>::C;
    constexpr int K = N + 6;
    double acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = 0.0;
    for (long long site = (long long)blockIdx.x * blockDim.x + threadIdx.x; site < p.S;
         site += (long long)gridDim.x * blockDim.x) {
        const Site3 c = site3(p, site);
        C rl[N], a[N][3];
        C rho = C(0);
#pragma unroll
        for (int s = 0; s < N; ++s) {
            rl[s] = rs[s * p.S + site];
            rho += rl[s];
        }
        accel19<C, N>(rs, nu, p, c, rl, rho, a);
#pragma unroll
        for (int s = 0; s < N; ++s) {
            acc[s] += (double)rl[s];
            double j[3] = {0.0, 0.0, 0.0};
#pragma unroll
            for (int i = 0; i < Q19; ++i) {
                const double v = (double)pull19(f, p, s, i, c);
#pragma unroll
                for (int d = 0; d < 3; ++d) j[d] += v * c19(i, d);
            }
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                acc[N + d] += j[d];
                acc[N + 3 + d] += (double)rl[s] * (double)a[s][d];
            }
        }
    }
    block_reduce_store<K>(acc, partial);
}

// FP64 compositions phi^s = rho^s / rho and a bulk flag (1 where every |grad phi^s| < tol).
template <typename T, int N>
__global__ void __launch_bounds__(SITE_THREADS)
k19_compositions(const typename Storage<T>::C* __restrict__ rs, double* __restrict__ phi,
                 double* __restrict__ bulk, double tol,
                 const __grid_constant__ StepParams<typename Storage<T>::C> p)
{
    const long long site = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (site >= p.S) return;
    const Site3 c = site3(p, site);
    double g[N][3];
#pragma unroll
    for (int s = 0; s < N; ++s) g[s][0] = g[s][1] = g[s][2] = 0.0;
#pragma unroll
    for (int i = 1; i < Q19; ++i) {
        const long long t = nbr3(p, c, c19(i, 0), c19(i, 1), c19(i, 2));
        double rho = 0.0;
#pragma unroll
        for (int s = 0; s < N; ++s) rho += (double)rs[s * p.S + t];
#pragma unroll
        for (int s = 0; s < N; ++s) {
            const double ph = (double)rs[s * p.S + t] / rho;
#pragma unroll
            for (int d = 0; d < 3; ++d) g[s][d] += 3.0 * w19<double>(i) * c19(i, d) * ph;
        }
    }
    double rho = 0.0, g2max = 0.0;
#pragma unroll
    for (int s = 0; s < N; ++s) rho += (double)rs[s * p.S + site];
#pragma unroll
    for (int s = 0; s < N; ++s) {
        phi[s * p.S + site] = (double)rs[s * p.S + site] / rho;
        const double g2 = g[s][0] * g[s][0] + g[s][1] * g[s][1] + g[s][2] * g[s][2];
        g2max = g2 > g2max ? g2 : g2max;
    }
    bulk[site] = (g2max < tol * tol) ? 1.0 : 0.0;
}

}  // namespace mclb
