// line3.cuh -- the D1Q3 lattice of the paper's own simulations (Sec. 4): velocities
// v = 0, +1, -1, weights 2/3, 1/6, 1/6, one periodic line of nx sites.
//
// The same timestep as the D2Q9 kernels (Eq. ssLB with the Eq. definef force, Eq. lgf
// potentials, Sec. 3 equilibria, Eqs. ff1-ff3 forcing) with the discrete operators
// built from the D1Q3 weights: grad g = (g(x+1) - g(x-1)) / 2, lap g = g(x+1) + g(x-1)
// - 2 g(x).  Storage: post-collision values f*[(s * 3 + i) * nx + x] (pull scheme: the
// pre-collision population f_i(x) is the value stored at x - v_i), FP64 or FP32.
//
// Two schedules:
//   - k_line3_resident: one CTA owns a whole line (nx <= L3_MAX_SITES, one site per
//     thread) and advances it by K steps in shared memory before writing it back, so a
//     line crosses HBM once per launch instead of once per step.  A batch launches one
//     CTA per line (every line of the same N in one launch).  Three CTA barriers per
//     step, no other waits.
//   - k_line3_tile: one launch per step for longer lines; a CTA pulls L3_TILE sites
//     (252 written, two halo sites on each side for the radius-2 stencil of the force).
#pragma once

#include "staged.cuh"

namespace mclb {

constexpr int L3_MAX_SITES = 1024;  // longest line the resident kernel holds
constexpr int L3_TILE = 256;        // threads (sites) of a tile CTA, 4 of them halo
constexpr int L3_CHUNK = LINE3_CHUNK;  // most steps one resident launch advances

__host__ __device__ __forceinline__ constexpr int v3(int i) { return i == 0 ? 0 : (i == 1 ? 1 : -1); }

// D1Q3 weights; in FP32 w_+- is one unit in the last place below the float nearest to
// 1/6 (11184810 * 2^-26), so that 2/3 rounded plus twice it is exactly 1 (the nearest
// floats sum to 1 + 3e-8, a mass drift of that size per step).
template <typename C>
__host__ __device__ __forceinline__ constexpr C w3(int i)
{
    return i == 0 ? C(2.0 / 3.0) : C(1.0 / 6.0);
}
template <>
__host__ __device__ __forceinline__ constexpr float w3<float>(int i)
{
    return i == 0 ? float(2.0 / 3.0) : 11184810.0f * 0x1p-26f;
}

__device__ __forceinline__ int wrap1(int a, int n)
{
    a %= n;
    return a < 0 ? a + n : a;
}

// Post-collision populations of one component at one site: f (1 - 1/tau) + (rho^s/tau)
// w_i (1 + 3 v u + 9/2 v^2 u^2 - 3/2 u^2) + w_i (3 rho^s v a + 9 v^2 a j - 3 a j), with
// the constant w_i rho^s/tau carried in the forcing bracket so that 1 - 3/2 u^2 is never
// rounded (that rounding biases the FP32 masses).
template <typename C>
__device__ __forceinline__ void collide3(const StepParams<C>& p, const C (&f)[3], C r, C j, C u,
                                         C a, C (&out)[3])
{
    const C base = C(-1.5) * u * u;
    const C uu45 = C(4.5) * u * u;
    const C keep = C(1) - p.omega, omr = p.omega * r;
    const C m3aj = C(-3) * a * j + omr;
    const C e0 = w3<C>(0) * base;
    const C ep = w3<C>(1) * (base + uu45 + C(3) * u);
    const C em = w3<C>(2) * (base + uu45 - C(3) * u);
    const C ar3 = C(3) * r * a, aj9 = C(9) * a * j;
    const C F0 = w3<C>(0) * m3aj;
    const C Fp = w3<C>(1) * (ar3 + aj9 + m3aj);
    const C Fm = w3<C>(2) * (-ar3 + aj9 + m3aj);
    out[0] = keep * f[0] + (omr * e0 + F0);
    out[1] = keep * f[1] + (omr * ep + Fp);
    out[2] = keep * f[2] + (omr * em + Fm);
}

// rho^s of component s at site x (pull of the three populations).
template <typename T>
__device__ __forceinline__ typename Storage<T>::C pull_rho3(const T* __restrict__ f, int nx, int s,
                                                            int x)
{
    using C = typename Storage<T>::C;
    C r = C(0);
#pragma unroll
    for (int i = 0; i < 3; ++i) r += C(f[(long long)(s * 3 + i) * nx + wrap1(x - v3(i), nx)]);
    return r;
}

// nu^s at site x from rho^s at x - 1, x, x + 1 (each rho array holds all N components).
template <typename C, int N>
__device__ __forceinline__ void nu3(const StepParams<C>& p, const C (&rl)[N], const C (&rc)[N],
                                    const C (&rr)[N], C (&nu)[N])
{
    C lap[N];
#pragma unroll
    for (int s = 0; s < N; ++s) lap[s] = (rr[s] + rl[s]) - C(2) * rc[s];
    site_nu<C, N>(p, rc, lap, nu);
}

// Gibbs-Duhem reading of the sum of the component forces (kappa = 0) on D1Q3: every a^s
// shifted by (A_c - A) / rho, A = sum_s rho^s (a^s - g), A_c = (1 - 1/(2 tau)) (1/3) d_x rho.
template <typename C, int N>
__device__ __forceinline__ void gibbs_duhem3(const StepParams<C>& p, const C (&r)[N], C rho,
                                             C grad_rho, C (&a)[N])
{
    C A = C(0);
#pragma unroll
    for (int s = 0; s < N; ++s) A += r[s] * (a[s] - p.gx);
    const C d = (p.fcoef * grad_rho / C(3) - A) / rho;
#pragma unroll
    for (int s = 0; s < N; ++s) a[s] += d;
}

// One instance of a resident launch: buffers and parameters.
template <typename T>
struct Line3Item {
    StepParams<typename Storage<T>::C> p;
    T* f[2];
};

template <typename T, int N>
struct Line3Smem {
    using C = typename Storage<T>::C;
    // per site: 3N post-collision populations, N densities, N potentials
    static constexpr size_t bytes(int nx) { return (size_t)(5 * N) * nx * sizeof(C); }
};

// K steps of one line per CTA, in shared memory: reads items[b].f[parity], writes
// items[b].f[parity ^ 1].  blockDim.x >= the longest nx of the launch.
template <typename T, int N>
__global__ void __launch_bounds__(L3_MAX_SITES)
k_line3_resident(const Line3Item<T>* __restrict__ items, int parity, int nsteps)
{
    using C = typename Storage<T>::C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ StepParams<C> p;
    if (threadIdx.x == 0) p = items[blockIdx.x].p;
    __syncthreads();
    const int nx = p.nx;
    C* A = reinterpret_cast<C*>(smem_raw);  // [3N][nx] post-collision
    C* R = A + 3 * N * nx;                  // [N][nx]
    C* NU = R + N * nx;                     // [N][nx]
    const T* fin = items[blockIdx.x].f[parity];
    T* fout = items[blockIdx.x].f[parity ^ 1];
    for (int k = threadIdx.x; k < 3 * N * nx; k += blockDim.x) A[k] = C(fin[k]);
    __syncthreads();
    const int x = threadIdx.x;
    const bool act = x < nx;
    const int xl = act ? wrap1(x - 1, nx) : 0, xr = act ? wrap1(x + 1, nx) : 0;
    bool bad = false;
    for (int t = 0; t < nsteps; ++t) {
        C f[N][3], r[N], j[N];
        C u = C(0);
        if (act) {
            C rho = C(0), jt = C(0);
#pragma unroll
            for (int s = 0; s < N; ++s) {
                f[s][0] = A[(s * 3 + 0) * nx + x];
                f[s][1] = A[(s * 3 + 1) * nx + xl];
                f[s][2] = A[(s * 3 + 2) * nx + xr];
                r[s] = (f[s][0] + f[s][1]) + f[s][2];
                j[s] = f[s][1] - f[s][2];
                rho += r[s];
                jt += j[s];
                R[s * nx + x] = r[s];
            }
            u = jt / rho;
            bad = bad || !(rho > C(0)) || !isfinite(rho);
        }
        __syncthreads();
        if (act) {
            C rl[N], rc[N], rr[N], nu[N];
#pragma unroll
            for (int s = 0; s < N; ++s) {
                rl[s] = R[s * nx + xl];
                rc[s] = R[s * nx + x];
                rr[s] = R[s * nx + xr];
            }
            nu3<C, N>(p, rl, rc, rr, nu);
#pragma unroll
            for (int s = 0; s < N; ++s) NU[s * nx + x] = nu[s];
        }
        __syncthreads();
        if (act) {
            C a[N], rho = C(0);
#pragma unroll
            for (int s = 0; s < N; ++s) {
                a[s] = -p.fcoef * (C(0.5) * (NU[s * nx + xr] - NU[s * nx + xl])) + p.gx;
                rho += r[s];
            }
            if (p.gd) {
                C rl = C(0), rr = C(0);
#pragma unroll
                for (int s = 0; s < N; ++s) {
                    rl += R[s * nx + xl];
                    rr += R[s * nx + xr];
                }
                gibbs_duhem3<C, N>(p, r, rho, C(0.5) * (rr - rl), a);
            }
#pragma unroll
            for (int s = 0; s < N; ++s) {
                const C jf = p.bary ? r[s] * u : j[s];
                C out[3];
                collide3(p, f[s], r[s], jf, u, a[s], out);
#pragma unroll
                for (int i = 0; i < 3; ++i) A[(s * 3 + i) * nx + x] = out[i];
            }
        }
        __syncthreads();
    }
    if (bad) atomicOr(p.status, STATUS_NONFINITE);
    for (int k = threadIdx.x; k < 3 * N * nx; k += blockDim.x) fout[k] = T(A[k]);
}

// One step of a line of any length: CTA b covers written sites [x0, x0 + L3_TILE - 4),
// thread t the site x0 - 2 + t (indices wrap, so lines shorter than a tile work too).
template <typename T, int N>
__global__ void __launch_bounds__(L3_TILE)
k_line3_tile(const T* __restrict__ fin, T* __restrict__ fout,
             const __grid_constant__ StepParams<typename Storage<T>::C> p)
{
    using C = typename Storage<T>::C;
    __shared__ C R[N][L3_TILE];
    __shared__ C NU[N][L3_TILE];
    const int nx = p.nx;
    const int t = threadIdx.x;
    const int x0 = blockIdx.x * (L3_TILE - 4);
    const int x = wrap1(x0 - 2 + t, nx);
    C f[N][3], r[N], j[N];
    C rho = C(0), jt = C(0);
#pragma unroll
    for (int s = 0; s < N; ++s) {
#pragma unroll
        for (int i = 0; i < 3; ++i) f[s][i] = C(fin[(long long)(s * 3 + i) * nx + wrap1(x - v3(i), nx)]);
        r[s] = (f[s][0] + f[s][1]) + f[s][2];
        j[s] = f[s][1] - f[s][2];
        rho += r[s];
        jt += j[s];
        R[s][t] = r[s];
    }
    const C u = jt / rho;
    __syncthreads();
    if (t >= 1 && t < L3_TILE - 1) {
        C rl[N], rc[N], rr[N], nu[N];
#pragma unroll
        for (int s = 0; s < N; ++s) {
            rl[s] = R[s][t - 1];
            rc[s] = r[s];
            rr[s] = R[s][t + 1];
        }
        nu3<C, N>(p, rl, rc, rr, nu);
#pragma unroll
        for (int s = 0; s < N; ++s) NU[s][t] = nu[s];
    }
    __syncthreads();
    const int xo = x0 - 2 + t;
    if (t >= 2 && t < L3_TILE - 2 && xo < nx) {
        if (!(rho > C(0)) || !isfinite(rho)) atomicOr(p.status, STATUS_NONFINITE);
        C a[N];
#pragma unroll
        for (int s = 0; s < N; ++s) a[s] = -p.fcoef * (C(0.5) * (NU[s][t + 1] - NU[s][t - 1])) + p.gx;
        if (p.gd) {
            C rl = C(0), rr = C(0);
#pragma unroll
            for (int s = 0; s < N; ++s) {
                rl += R[s][t - 1];
                rr += R[s][t + 1];
            }
            gibbs_duhem3<C, N>(p, r, rho, C(0.5) * (rr - rl), a);
        }
#pragma unroll
        for (int s = 0; s < N; ++s) {
            const C jf = p.bary ? r[s] * u : j[s];
            C out[3];
            collide3(p, f[s], r[s], jf, u, a[s], out);
#pragma unroll
            for (int i = 0; i < 3; ++i) fout[(long long)(s * 3 + i) * nx + xo] = T(out[i]);
        }
    }
}

// f*_i(x) such that the pull at x + v_i yields f^e_i(rho(x + v_i), u(x + v_i)).
template <typename T, int N>
__global__ void __launch_bounds__(SITE_THREADS)
k_line3_init(const double* __restrict__ rho, const double* __restrict__ u, T* __restrict__ f,
             const __grid_constant__ StepParams<typename Storage<T>::C> p)
{
    using C = typename Storage<T>::C;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= p.nx) return;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const int xs = wrap1(x + v3(i), p.nx);
        const C uu = u ? C(u[xs]) : C(0);
        const C cu = C(v3(i)) * uu;
#pragma unroll
        for (int s = 0; s < N; ++s)
            f[(long long)(s * 3 + i) * p.nx + x] =
                T(w3<C>(i) * C(rho[(long long)s * p.nx + xs]) *
                  (C(1) + C(3) * cu + C(4.5) * cu * cu - C(1.5) * uu * uu));
    }
}

template <typename T, int N>
__global__ void __launch_bounds__(SITE_THREADS)
k_line3_get_state(const T* __restrict__ f, double* __restrict__ out,
                  const __grid_constant__ StepParams<typename Storage<T>::C> p)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= p.nx) return;
#pragma unroll
    for (int s = 0; s < N; ++s)
#pragma unroll
        for (int i = 0; i < 3; ++i)
            out[(long long)(s * 3 + i) * p.nx + x] =
                (double)f[(long long)(s * 3 + i) * p.nx + wrap1(x - v3(i), p.nx)];
}

template <typename T, int N>
__global__ void __launch_bounds__(SITE_THREADS)
k_line3_set_state(const double* __restrict__ in, T* __restrict__ f,
                  const __grid_constant__ StepParams<typename Storage<T>::C> p)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= p.nx) return;
#pragma unroll
    for (int s = 0; s < N; ++s)
#pragma unroll
        for (int i = 0; i < 3; ++i)
            f[(long long)(s * 3 + i) * p.nx + x] =
                T(in[(long long)(s * 3 + i) * p.nx + wrap1(x + v3(i), p.nx)]);
}

// rho^s at x - 2 .. x + 2, nu^s at x - 1 .. x + 1 and the site's own moments.
template <typename T, int N>
struct Line3Site {
    using C = typename Storage<T>::C;
    C r[5][N];
    C nu[3][N];
    C j[N];
    C rho, u;
    __device__ __forceinline__ Line3Site(const T* __restrict__ f, const StepParams<C>& p, int x)
    {
#pragma unroll
        for (int d = 0; d < 5; ++d)
#pragma unroll
            for (int s = 0; s < N; ++s) r[d][s] = pull_rho3(f, p.nx, s, x - 2 + d);
#pragma unroll
        for (int d = 0; d < 3; ++d) nu3<C, N>(p, r[d], r[d + 1], r[d + 2], nu[d]);
        rho = C(0);
        C jt = C(0);
#pragma unroll
        for (int s = 0; s < N; ++s) {
            j[s] = C(f[(long long)(s * 3 + 1) * p.nx + wrap1(x - 1, p.nx)]) -
                   C(f[(long long)(s * 3 + 2) * p.nx + wrap1(x + 1, p.nx)]);
            rho += r[2][s];
            jt += j[s];
        }
        u = jt / rho;
        // Gibbs-Duhem reading: the common shift of every a^s
        shift = C(0);
        if (p.gd) {
            C A = C(0), rl = C(0), rr = C(0);
#pragma unroll
            for (int s = 0; s < N; ++s) {
                A += r[2][s] * (-p.fcoef * (C(0.5) * (nu[2][s] - nu[0][s])));
                rl += r[1][s];
                rr += r[3][s];
            }
            shift = (p.fcoef * (C(0.5) * (rr - rl)) / C(3) - A) / rho;
        }
    }
    C shift;
    __device__ __forceinline__ C accel(const StepParams<C>& p, int s) const
    {
        return -p.fcoef * (C(0.5) * (nu[2][s] - nu[0][s])) + p.gx + shift;
    }
};

// Output fields in the shapes of a D2Q9 lattice with ny = 1: rho^s; U = (u + a/2, 0);
// mu^s/m^s with the gradient term; P = (iso + kappa sum (d_x rho)^2, 0, iso).
template <typename T, int N>
__global__ void __launch_bounds__(SITE_THREADS)
k_line3_moments(const T* __restrict__ f, double* __restrict__ rho_out, double* __restrict__ U,
                double* __restrict__ mu_out, double* __restrict__ P,
                const __grid_constant__ StepParams<typename Storage<T>::C> p)
{
    using C = typename Storage<T>::C;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= p.nx) return;
    const Line3Site<T, N> q(f, p, x);
    const int nx = p.nx;
    if (rho_out)
#pragma unroll
        for (int s = 0; s < N; ++s) rho_out[(long long)s * nx + x] = (double)q.r[2][s];
    if (U) {
        C fx = C(0);
#pragma unroll
        for (int s = 0; s < N; ++s) fx += q.r[2][s] * q.accel(p, s);
        U[x] = (double)(q.u + C(0.5) * fx / q.rho);
        U[nx + x] = 0.0;
    }
    if (mu_out || P) {
        C lap[N], mu[N];
#pragma unroll
        for (int s = 0; s < N; ++s) lap[s] = (q.r[3][s] + q.r[1][s]) - C(2) * q.r[2][s];
        site_mu<C, N>(p, q.r[2], lap, mu);
        if (mu_out)
#pragma unroll
            for (int s = 0; s < N; ++s) mu_out[(long long)s * nx + x] = (double)mu[s];
        if (P) {
            const C psi = site_psi<C, N>(p, q.r[2]);
            C rmu = C(0), gg = C(0), pxx = C(0);
#pragma unroll
            for (int s = 0; s < N; ++s) {
                const C gx = C(0.5) * (q.r[3][s] - q.r[1][s]);
                rmu += q.r[2][s] * mu[s];
                gg += C(0.5) * p.kappa * gx * gx;
                pxx += p.kappa * gx * gx;
            }
            const C iso = rmu - (psi + gg);
            P[x] = (double)(iso + pxx);
            P[nx + x] = 0.0;
            P[2 * nx + x] = (double)iso;
        }
    }
}

// Conservation sums (FP64, fixed-grid block partials): mass^s, momentum (x, 0), force (x, 0).
template <typename T, int N>
__global__ void __launch_bounds__(SITE_THREADS)
k_line3_conservation(const T* __restrict__ f, double* __restrict__ partial,
                     const __grid_constant__ StepParams<typename Storage<T>::C> p)
{
    constexpr int K = N + 4;
    double acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = 0.0;
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < p.nx; x += gridDim.x * blockDim.x) {
        const Line3Site<T, N> q(f, p, x);
#pragma unroll
        for (int s = 0; s < N; ++s) {
            acc[s] += (double)q.r[2][s];
            acc[N] += (double)q.j[s];
            acc[N + 2] += (double)q.r[2][s] * (double)q.accel(p, s);
        }
    }
    block_reduce_store<K>(acc, partial);
}

// FP64 compositions and bulk flags (|d_x phi^s| < tol for every s).
template <typename T, int N>
__global__ void __launch_bounds__(SITE_THREADS)
k_line3_compositions(const T* __restrict__ f, double* __restrict__ phi, double* __restrict__ bulk,
                     double tol, const __grid_constant__ StepParams<typename Storage<T>::C> p)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= p.nx) return;
    double ph[3][N];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        double rho = 0.0, r[N];
#pragma unroll
        for (int s = 0; s < N; ++s) {
            r[s] = (double)pull_rho3(f, p.nx, s, x - 1 + d);
            rho += r[s];
        }
#pragma unroll
        for (int s = 0; s < N; ++s) ph[d][s] = r[s] / rho;
    }
    double gmax = 0.0;
#pragma unroll
    for (int s = 0; s < N; ++s) {
        phi[(long long)s * p.nx + x] = ph[1][s];
        const double g = fabs(0.5 * (ph[2][s] - ph[0][s]));
        gmax = g > gmax ? g : gmax;
    }
    bulk[x] = gmax < tol ? 1.0 : 0.0;
}

}  // namespace mclb
