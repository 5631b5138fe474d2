// staged.cuh -- the three-launch timestep and the diagnostic kernels.
//
// Staged schedule (one thread per site, periodic neighbours by index arithmetic):
//   k_density    rho^s = sum_i f^s_i(r - v_i)           pull streaming + zeroth moment
//   k_potential  nu^s  = mu^s/m^s - kappa lap rho^s - (1/3) ln rho^s
//   k_collide    pull f again, first moments, barycentric u, a^s = -(1 - 1/2tau) grad nu^s + g,
//                f^e, F, BGK (Eq. ssLB), store post-collision values in place (pull scheme)
// The density and potential fields live in handle-owned scratch memory.
#pragma once

#include "physics.cuh"

namespace mclb {

constexpr int SITE_THREADS = 256;

// The site functions below take a compile-time flag E: with E = true they handle solid
// walls in y (p.walls), with E = false they assume a periodic neighbourhood.  The timestep
// kernels use E = false on every row that no wall touches (all rows of a periodic
// lattice, rows 1 .. ny - 2 between walls), so the periodic path is free of wall tests.

// Pre-collision value f^s_i(x, y) = post-collision value stored at (x - v_i, y - v_i).
// With walls (p.walls), a population whose source row lies beyond a wall is the site's
// own post-collision value of the opposite velocity (halfway bounce-back).
template <bool E = true, typename T>
__device__ __forceinline__ typename Storage<T>::C pull(const T* __restrict__ f,
                                                       const StepParams<typename Storage<T>::C>& p,
                                                       int s, int i, int x, int y)
{
    using C = typename Storage<T>::C;
    int xs = wrap_add(x, -vx(i), p.nx), ys = wrap_add(y, -vy(i), p.ny), is = i;
    if constexpr (E) {
        const int yb = y - vy(i);
        if (p.walls && (yb < 0 || yb >= p.ny)) {
            xs = x;
            ys = y;
            is = opp9(i);
        }
    }
    C v = Storage<T>::load(f + fidx(p, s, is, ys, xs));
    if constexpr (Storage<T>::shifted) v += wq<C>(i) * __ldg(rho_line(f, p, s, ys) + p.hx + xs);
    return v;
}

// Row y + dy as a stencil sees it: periodic, or with walls the mirror image of the row
// next to the wall (rows -1 and ny read rows 0 and ny - 1: zero normal gradient).
template <bool E = true, typename C>
__device__ __forceinline__ int stencil_row(const StepParams<C>& p, int y, int dy)
{
    if constexpr (E) {
        if (p.walls) {
            const int yy = y + dy;
            return yy < 0 ? 0 : (yy >= p.ny ? p.ny - 1 : yy);
        }
    }
    return wrap_add(y, dy, p.ny);
}

// Site of thread t in a band launch (BAND = true): every site, or with p.band > 0 the first
// and the last p.band sites (rows next to the walls); -1 for a thread beyond them.  The
// full-lattice launches (BAND = false) index sites directly.
template <typename C>
__device__ __forceinline__ long long site_of(const StepParams<C>& p, long long t)
{
    if (p.band == 0) return t < p.S ? t : -1;
    return t < p.band ? t : (t < 2 * p.band ? p.S - 2 * p.band + t : -1);
}

// True where a timestep kernel must take the wall-aware (E = true) path.
template <typename C>
__device__ __forceinline__ bool wall_row(const StepParams<C>& p, long long site)
{
    if (!p.walls) return false;
    const int y = (int)(site / p.nx);
    return y == 0 || y == p.ny - 1;
}

// Velocity whose stored value at (x, y) the site (x + v_i, y + v_i) pulls as f_i, or,
// when that site lies beyond a wall, the velocity the site (x, y) itself pulls it as.
template <typename C>
__device__ __forceinline__ bool bounced(const StepParams<C>& p, int y, int i)
{
    const int yy = y + vy(i);
    return p.walls && (yy < 0 || yy >= p.ny);
}

// rho^s at one site (pull streaming + zeroth moment).
template <typename T, int N, bool E = true>
__device__ __forceinline__ void density_site(const T* __restrict__ f,
                                             typename Storage<T>::C* __restrict__ rs,
                                             const StepParams<typename Storage<T>::C>& p, long long site)
{
    using C = typename Storage<T>::C;
    const int y = (int)(site / p.nx), x = (int)(site - (long long)y * p.nx);
#pragma unroll
    for (int s = 0; s < N; ++s) {
        C r = C(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) r += pull<E>(f, p, s, i, x, y);
        rs[s * p.S + site] = r;
    }
}

template <typename T, int N, bool BAND = false>
__global__ void __launch_bounds__(SITE_THREADS)
k_density(const T* __restrict__ f, typename Storage<T>::C* __restrict__ rs,
          const __grid_constant__ StepParams<typename Storage<T>::C> p)
{
    long long site = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if constexpr (BAND) {
        site = site_of(p, site);
        if (site < 0) return;
    } else if (site >= p.S) {
        return;
    }
    if (wall_row(p, site))
        density_site<T, N, true>(f, rs, p, site);
    else
        density_site<T, N, false>(f, rs, p, site);
}

template <typename C, int N, bool E = true>
__device__ __forceinline__ void neighbour_laplacians(const C* __restrict__ rs,
                                                     const StepParams<C>& p, int x, int y,
                                                     const C (&r)[N], C (&lap)[N])
{
    // lap g = 6 sum_i w_i (g(r + v_i) - g(r))
#pragma unroll
    for (int s = 0; s < N; ++s) {
        C acc = C(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int xx = wrap_add(x, vx(i), p.nx), yy = stencil_row<E>(p, y, vy(i));
            acc += wq<C>(i) * (rs[s * p.S + (long long)yy * p.nx + xx] - r[s]);
        }
        lap[s] = C(6) * acc;
    }
}

// nu^s at one site from the density fields.
template <typename C, int N, bool E = true>
__device__ __forceinline__ void potential_site(const C* __restrict__ rs, C* __restrict__ nu,
                                               const StepParams<C>& p, long long site)
{
    const int y = (int)(site / p.nx), x = (int)(site - (long long)y * p.nx);
    C r[N], lap[N], out[N];
#pragma unroll
    for (int s = 0; s < N; ++s) r[s] = rs[s * p.S + site];
    neighbour_laplacians<C, N, E>(rs, p, x, y, r, lap);
    site_nu<C, N>(p, r, lap, out);
#pragma unroll
    for (int s = 0; s < N; ++s) nu[s * p.S + site] = out[s];
}

template <typename C, int N, bool BAND = false>
__global__ void __launch_bounds__(SITE_THREADS)
k_potential(const C* __restrict__ rs, C* __restrict__ nu, const __grid_constant__ StepParams<C> p)
{
    long long site = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if constexpr (BAND) {
        site = site_of(p, site);
        if (site < 0) return;
    } else if (site >= p.S) {
        return;
    }
    if (wall_row(p, site))
        potential_site<C, N, true>(rs, nu, p, site);
    else
        potential_site<C, N, false>(rs, nu, p, site);
}

// grad g = 3 sum_i w_i v_i g(r + v_i) of one component's field
template <bool E = true, typename C>
__device__ __forceinline__ void field_grad(const C* __restrict__ g, const StepParams<C>& p, int x,
                                           int y, C& gx, C& gy)
{
    C ax = C(0), ay = C(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int xx = wrap_add(x, vx(i), p.nx), yy = stencil_row<E>(p, y, vy(i));
        const C v = g[(long long)yy * p.nx + xx];
        ax += wq<C>(i) * C(vx(i)) * v;
        ay += wq<C>(i) * C(vy(i)) * v;
    }
    gx = C(3) * ax;
    gy = C(3) * ay;
}

// grad rho = 3 sum_i w_i v_i rho(r + v_i) of the total density, from the N density fields
template <typename C, int N, bool E = true>
__device__ __forceinline__ void rho_grad(const C* __restrict__ rs, const StepParams<C>& p, int x,
                                         int y, C& gx, C& gy)
{
    C ax = C(0), ay = C(0);
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const int xx = wrap_add(x, vx(i), p.nx), yy = stencil_row<E>(p, y, vy(i));
        C r = C(0);
#pragma unroll
        for (int s = 0; s < N; ++s) r += rs[s * p.S + (long long)yy * p.nx + xx];
        ax += wq<C>(i) * C(vx(i)) * r;
        ay += wq<C>(i) * C(vy(i)) * r;
    }
    gx = C(3) * ax;
    gy = C(3) * ay;
}

// Accelerations a^s at (x, y) from the potential fields (Eq. definef plus the body force;
// with p.gd the Gibbs-Duhem shift).  r: the site's rho^s, rho their sum.
template <typename C, int N, bool E = true>
__device__ __forceinline__ void site_accel(const C* __restrict__ rs, const C* __restrict__ nu,
                                           const StepParams<C>& p, int x, int y, const C (&r)[N],
                                           C rho, C (&ax)[N], C (&ay)[N])
{
#pragma unroll
    for (int s = 0; s < N; ++s) {
        C gx, gy;
        field_grad<E>(nu + s * p.S, p, x, y, gx, gy);
        ax[s] = -p.fcoef * gx + p.gx;
        ay[s] = -p.fcoef * gy + p.gy;
    }
    if (p.gd) {
        C grx, gry;
        rho_grad<C, N, E>(rs, p, x, y, grx, gry);
        gibbs_duhem_shift<C, N>(p, r, rho, grx, gry, ax, ay);
    }
}

// Collision at one site from the pulled populations and the potential fields; the
// post-collision values are stored in place (pull scheme), ghosts included.
template <typename T, int N, bool E = true>
__device__ __forceinline__ void collide_site(const T* __restrict__ fin, T* __restrict__ fout,
                                             const typename Storage<T>::C* __restrict__ rs,
                                             const typename Storage<T>::C* __restrict__ nu,
                                             const StepParams<typename Storage<T>::C>& p,
                                             long long site)
{
    using C = typename Storage<T>::C;
    const int y = (int)(site / p.nx), x = (int)(site - (long long)y * p.nx);
    C f[N][Q];
    C r[N], jx[N], jy[N];
    C rho = C(0), jxt = C(0), jyt = C(0);
#pragma unroll
    for (int s = 0; s < N; ++s) {
        C a = C(0), bx = C(0), by = C(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const C v = pull<E>(fin, p, s, i, x, y);
            f[s][i] = v;
            a += v;
            bx += v * C(vx(i));
            by += v * C(vy(i));
        }
        r[s] = a;
        jx[s] = bx;
        jy[s] = by;
        rho += a;
        jxt += bx;
        jyt += by;
    }
    const C inv = C(1) / rho;
    const C ux = jxt * inv, uy = jyt * inv;
    C e[Q];
    eq_weights(ux, uy, e);
    C ax[N], ay[N];
    site_accel<C, N, E>(rs, nu, p, x, y, r, rho, ax, ay);
#pragma unroll
    for (int s = 0; s < N; ++s) {
        C out[Q], fjx, fjy;
        forcing_momentum(p, r[s], jx[s], jy[s], ux, uy, fjx, fjy);
        collide(p, f[s], e, r[s], fjx, fjy, ax[s], ay[s], out);
        store_site(fout, p, s, y, x, out);
    }
    if (!(rho > C(0)) || !isfinite(rho)) atomicOr(p.status, STATUS_NONFINITE);
}

template <typename T, int N, bool BAND = false>
__global__ void __launch_bounds__(SITE_THREADS)
k_collide(const T* __restrict__ fin, T* __restrict__ fout,
          const typename Storage<T>::C* __restrict__ rs,
          const typename Storage<T>::C* __restrict__ nu,
          const __grid_constant__ StepParams<typename Storage<T>::C> p)
{
    long long site = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if constexpr (BAND) {
        site = site_of(p, site);
        if (site < 0) return;
    } else if (site >= p.S) {
        return;
    }
    if (wall_row(p, site))
        collide_site<T, N, true>(fin, fout, rs, nu, p, site);
    else
        collide_site<T, N, false>(fin, fout, rs, nu, p, site);
}

// ---------------------------------------------------------------- diagnostics

// f^s_i stored at (x, y) so that pulling yields f^e_i(rho^s, u) at (x + v_i, y + v_i).
template <typename T, int N>
__global__ void __launch_bounds__(SITE_THREADS)
k_init(const double* __restrict__ rho, const double* __restrict__ u, T* __restrict__ f,
       const __grid_constant__ StepParams<typename Storage<T>::C> p)
{
    using C = typename Storage<T>::C;
    const long long site = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (site >= p.S) return;
    const int y = (int)(site / p.nx), x = (int)(site - (long long)y * p.nx);
    C v[N][Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        // the site that pulls this value, and as which velocity (itself, as the opposite
        // velocity, when the value is bounced back from a wall)
        const bool bb = bounced(p, y, i);
        const int ie = bb ? opp9(i) : i;
        const int xx = bb ? x : wrap_add(x, vx(i), p.nx), yy = bb ? y : wrap_add(y, vy(i), p.ny);
        const long long t = (long long)yy * p.nx + xx;
        const C ux = u ? C(u[t]) : C(0), uy = u ? C(u[p.S + t]) : C(0);
        const C uu = ux * ux + uy * uy;
        const C cu = C(vx(ie)) * ux + C(vy(ie)) * uy;
#pragma unroll
        for (int s = 0; s < N; ++s)
            v[s][i] = wq<C>(i) * C(rho[s * p.S + t]) *
                      (C(1) + C(3) * cu + C(4.5) * cu * cu - C(1.5) * uu);
    }
#pragma unroll
    for (int s = 0; s < N; ++s) store_site(f, p, s, y, x, v[s]);
}

template <typename T, int N>
__global__ void __launch_bounds__(SITE_THREADS)
k_get_state(const T* __restrict__ f, double* __restrict__ out,
            const __grid_constant__ StepParams<typename Storage<T>::C> p)
{
    const long long site = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (site >= p.S) return;
    const int y = (int)(site / p.nx), x = (int)(site - (long long)y * p.nx);
#pragma unroll
    for (int s = 0; s < N; ++s)
#pragma unroll
        for (int i = 0; i < Q; ++i) out[(s * Q + i) * p.S + site] = (double)pull(f, p, s, i, x, y);
}

template <typename T, int N>
__global__ void __launch_bounds__(SITE_THREADS)
k_set_state(const double* __restrict__ in, T* __restrict__ f,
            const __grid_constant__ StepParams<typename Storage<T>::C> p)
{
    using C = typename Storage<T>::C;
    const long long site = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (site >= p.S) return;
    const int y = (int)(site / p.nx), x = (int)(site - (long long)y * p.nx);
    C v[N][Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const bool bb = bounced(p, y, i);
        const int ie = bb ? opp9(i) : i;
        const int xx = bb ? x : wrap_add(x, vx(i), p.nx), yy = bb ? y : wrap_add(y, vy(i), p.ny);
        const long long t = (long long)yy * p.nx + xx;
#pragma unroll
        for (int s = 0; s < N; ++s) v[s][i] = C(in[(s * Q + ie) * p.S + t]);
    }
#pragma unroll
    for (int s = 0; s < N; ++s) store_site(f, p, s, y, x, v[s]);
}

// Output fields: rho^s, U = u + (sum_s rho^s a^s)/(2 rho), mu^s, P (needs k_density and
// k_potential to have filled the scratch fields for the same state).
template <typename T, int N>
__global__ void __launch_bounds__(SITE_THREADS)
k_moments(const T* __restrict__ f, const typename Storage<T>::C* __restrict__ rs,
          const typename Storage<T>::C* __restrict__ nu, double* __restrict__ rho_out,
          double* __restrict__ U, double* __restrict__ mu_out, double* __restrict__ P,
          const __grid_constant__ StepParams<typename Storage<T>::C> p)
{
    using C = typename Storage<T>::C;
    const long long site = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (site >= p.S) return;
    const int y = (int)(site / p.nx), x = (int)(site - (long long)y * p.nx);
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
        C jxt = C(0), jyt = C(0), fx = C(0), fy = C(0);
        C ax[N], ay[N];
        site_accel<C, N>(rs, nu, p, x, y, r, rho, ax, ay);
#pragma unroll
        for (int s = 0; s < N; ++s) {
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const C v = pull(f, p, s, i, x, y);
                jxt += v * C(vx(i));
                jyt += v * C(vy(i));
            }
            fx += r[s] * ax[s];
            fy += r[s] * ay[s];
        }
        U[site] = (double)(jxt / rho + C(0.5) * fx / rho);
        U[p.S + site] = (double)(jyt / rho + C(0.5) * fy / rho);
    }
    if (mu_out || P) {
        C lap[N], mu[N];
        neighbour_laplacians<C, N>(rs, p, x, y, r, lap);
        site_mu<C, N>(p, r, lap, mu);
        if (mu_out)
#pragma unroll
            for (int s = 0; s < N; ++s) mu_out[s * p.S + site] = (double)mu[s];
        if (P) {
            const C psi = site_psi<C, N>(p, r);
            C rmu = C(0), gg = C(0), pxx = C(0), pxy = C(0), pyy = C(0);
#pragma unroll
            for (int s = 0; s < N; ++s) {
                C gx, gy;
                field_grad(rs + s * p.S, p, x, y, gx, gy);
                rmu += r[s] * mu[s];
                gg += C(0.5) * p.kappa * (gx * gx + gy * gy);
                pxx += p.kappa * gx * gx;
                pxy += p.kappa * gx * gy;
                pyy += p.kappa * gy * gy;
            }
            const C iso = rmu - (psi + gg);
            P[site] = (double)(iso + pxx);
            P[p.S + site] = (double)pxy;
            P[2 * p.S + site] = (double)(iso + pyy);
        }
    }
}

// Deterministic FP64 block reduction of K values per thread into partial[block * K + k].
template <int K>
__device__ __forceinline__ void block_reduce_store(double (&v)[K], double* partial)
{
    __shared__ double red[SITE_THREADS];
    for (int k = 0; k < K; ++k) {
        red[threadIdx.x] = v[k];
        __syncthreads();
        for (int w = SITE_THREADS / 2; w > 0; w >>= 1) {
            if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) partial[blockIdx.x * K + k] = red[0];
        __syncthreads();
    }
}

// Conservation sums over the sites [s0, s1) (row-major, so a range of whole rows is a
// y band): mass^s, total momentum sum_s j^s, force sum_s rho^s a^s.
template <typename T, int N>
__global__ void __launch_bounds__(SITE_THREADS)
k_conservation(const T* __restrict__ f, const typename Storage<T>::C* __restrict__ rs,
               const typename Storage<T>::C* __restrict__ nu, double* __restrict__ partial,
               long long s0, long long s1,
               const __grid_constant__ StepParams<typename Storage<T>::C> p)
{
    using C = typename Storage<T>::C;
    constexpr int K = N + 4;
    double acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = 0.0;
    for (long long site = s0 + (long long)blockIdx.x * blockDim.x + threadIdx.x; site < s1;
         site += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(site / p.nx), x = (int)(site - (long long)y * p.nx);
        C rl[N], ax[N], ay[N];
        C rho = C(0);
#pragma unroll
        for (int s = 0; s < N; ++s) {
            rl[s] = rs[s * p.S + site];
            rho += rl[s];
        }
        site_accel<C, N>(rs, nu, p, x, y, rl, rho, ax, ay);
#pragma unroll
        for (int s = 0; s < N; ++s) {
            const C r = rl[s];
            acc[s] += (double)r;
            double jx = 0.0, jy = 0.0;
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const double v = (double)pull(f, p, s, i, x, y);
                jx += v * vx(i);
                jy += v * vy(i);
            }
            acc[N] += jx;
            acc[N + 1] += jy;
            acc[N + 2] += (double)r * (double)ax[s];
            acc[N + 3] += (double)r * (double)ay[s];
        }
    }
    block_reduce_store<K>(acc, partial);
}

// Sum the per-block partials in a fixed order: out[k] = sum_b partial[b * K + k].
static __global__ void k_reduce_partials(const double* __restrict__ partial, int nblocks, int K,
                                  double* __restrict__ out)
{
    __shared__ double red[SITE_THREADS];
    for (int k = 0; k < K; ++k) {
        double a = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += blockDim.x) a += partial[b * K + k];
        red[threadIdx.x] = a;
        __syncthreads();
        for (int w = SITE_THREADS / 2; w > 0; w >>= 1) {
            if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[k] = red[0];
        __syncthreads();
    }
}

// FP64 compositions phi^s = rho^s / rho and a bulk flag (1 where every |grad phi^s| < tol).
template <typename T, int N>
__global__ void __launch_bounds__(SITE_THREADS)
k_compositions(const typename Storage<T>::C* __restrict__ rs, double* __restrict__ phi,
               double* __restrict__ bulk, double tol,
               const __grid_constant__ StepParams<typename Storage<T>::C> p)
{
    const long long site = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (site >= p.S) return;
    const int y = (int)(site / p.nx), x = (int)(site - (long long)y * p.nx);
    double g2max = 0.0;
    double here[N];
    {
        double rho = 0.0;
#pragma unroll
        for (int s = 0; s < N; ++s) rho += (double)rs[s * p.S + site];
#pragma unroll
        for (int s = 0; s < N; ++s) here[s] = (double)rs[s * p.S + site] / rho;
    }
    double gx[N], gy[N];
#pragma unroll
    for (int s = 0; s < N; ++s) gx[s] = gy[s] = 0.0;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const int xx = wrap_add(x, vx(i), p.nx), yy = stencil_row(p, y, vy(i));
        const long long t = (long long)yy * p.nx + xx;
        double rho = 0.0;
#pragma unroll
        for (int s = 0; s < N; ++s) rho += (double)rs[s * p.S + t];
#pragma unroll
        for (int s = 0; s < N; ++s) {
            const double ph = (double)rs[s * p.S + t] / rho;
            gx[s] += 3.0 * wq<double>(i) * vx(i) * ph;
            gy[s] += 3.0 * wq<double>(i) * vy(i) * ph;
        }
    }
#pragma unroll
    for (int s = 0; s < N; ++s) {
        phi[s * p.S + site] = here[s];
        const double g2 = gx[s] * gx[s] + gy[s] * gy[s];
        g2max = g2 > g2max ? g2 : g2max;
    }
    bulk[site] = (g2max < tol * tol) ? 1.0 : 0.0;
}

}  // namespace mclb
