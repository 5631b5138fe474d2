// cube_march.cuh -- the D3Q19 timestep in two launches: the density pass (k19_density,
// cube.cuh) and a z-plane march over x-y tiles that forms nu^s in shared memory and collides.
//
// The march does what k19_potential and k19_collide do, with the same per-site arithmetic
// in the same order (the result equals the staged schedule's bit for bit), without writing
// nu^s and j^s to HBM and reading them back (2 x 16 N B fewer per site in FP32), and with
// the 18-neighbour Laplacian and gradient gathers from shared memory.  A CTA owns a tile of M3_OUT_X columns x M3_OUT_Y rows
// and a segment of z planes.  Lane l of every warp holds column x0 - 2 + l (two halo
// columns each side); the tile's rows carry two halo rows each side.  Iteration k of the
// march, lead plane m = z0 - 2 + k:
//   A  rho^s(m), read from the density pass's field, on the whole tile with its halo, into
//      a ring of three density planes in shared memory;
//   B  nu^s(m - 1) (Eq. lgf with the -kappa lap rho^s term of Eq. definef and the -(1/3) ln
//      rho^s of the forcing) on the tile and a halo of one; the D3Q19 Laplacian reads the
//      density planes m - 2, m - 1, m; into a ring of three potential planes;
//   C  the collision of plane m - 2 on the tile: the 19 N populations pulled, rho^s and j^s
//      from them, grad nu^s from the potential planes m - 3 .. m - 1, Eq. ssLB with the
//      forcing of Eqs. ff1-ff3, stored in place (pull scheme).
// Two CTA barriers per plane: between A and B, and between B and C.  C reads no density
// plane (it sums the pulled values again, the same sum the density pass formed), so the
// next iteration's A may overwrite the density slot of plane m - 2 while C runs; the next
// B writes the potential slot of plane m - 3 only after every warp has passed the next
// barrier, i.e. finished C.  No CTA waits on another: there is no spin-wait.
#pragma once

#include <utility>

#include "cube.cuh"

namespace mclb {

constexpr int M3_WARPS = 4;
constexpr int M3_RC = 2;                     // rows each warp collides (one at a time)
constexpr int M3_THREADS = 32 * M3_WARPS;
constexpr int M3_OUT_X = 28;                 // written columns of the 32 a warp holds
constexpr int M3_OUT_Y = M3_RC * M3_WARPS;   // written rows
constexpr int M3_ROWS = M3_OUT_Y + 4;        // rows with the two-row halo each side
constexpr int M3_NMAX = 4;                   // components the march takes

// Bytes of shared memory: the density and potential rings, three planes each.
template <typename C, int N>
constexpr size_t m3_smem_bytes() { return (size_t)2 * 3 * N * M3_ROWS * 32 * sizeof(C); }

__device__ __forceinline__ int pmod(int a, int n)
{
    a %= n;
    return a < 0 ? a + n : a;
}
__device__ __forceinline__ int dec_wrap(int a, int n) { return a == 0 ? n - 1 : a - 1; }
__device__ __forceinline__ int inc_wrap(int a, int n) { return a == n - 1 ? 0 : a + 1; }

// The wrapped rows y - 1, y, y + 1 of a site (its planes z - 1, z, z + 1 travel as zz[3]);
// the start of the stored row (z', y') of component 0 is ((z' ny + y') * 19) nx (32-bit:
// 19 S < 2^31).
struct M3Rows {
    int y[3];
};

__device__ __forceinline__ M3Rows m3_rows(int y, int ny)
{
    M3Rows r;
    r.y[1] = pmod(y, ny);
    r.y[0] = dec_wrap(r.y[1], ny);
    r.y[2] = inc_wrap(r.y[1], ny);
    return r;
}

__device__ __forceinline__ unsigned m3_rowbase(int z, int y, int ny, int nx)
{
    return ((unsigned)(z * ny + y) * 19u) * (unsigned)nx;
}

// Stored offset (component 0) of the value that site (x, y[1], zz[1]) pulls as velocity i:
// the post-collision value of velocity i at (x - c_x, y - c_y, z - c_z).
template <int I>
__device__ __forceinline__ unsigned m3_src(const int (&xw)[3], const M3Rows& r, const int (&zz)[3],
                                           int ny, int nx)
{
    return m3_rowbase(zz[1 - c19(I, 2)], r.y[1 - c19(I, 1)], ny, nx) + (unsigned)(I * nx) +
           (unsigned)xw[1 - c19(I, 0)];
}

// Index of tile row r, lane l, component s, ring slot q in a ring of three planes.
template <int N>
__device__ __forceinline__ int m3_at(int q, int s, int r, int l)
{
    return ((q * N + s) * M3_ROWS + r) * 32 + l;
}

template <int I, typename T, int N>
__device__ __forceinline__ void m3_pull_one(const T* __restrict__ f, unsigned cst, const int (&xw)[3],
                                            const M3Rows& rw, const int (&zz)[3], int ny, int nx,
                                            typename Storage<T>::C (&v)[N][Q19])
{
    const unsigned o = m3_src<I>(xw, rw, zz, ny, nx);
#pragma unroll
    for (int s = 0; s < N; ++s) v[s][I] = Storage<T>::load(f + (size_t)s * cst + o);
}

template <typename T, int N, int... I>
__device__ __forceinline__ void m3_pull_all(const T* __restrict__ f, unsigned cst, const int (&xw)[3],
                                            const M3Rows& rw, const int (&zz)[3], int ny, int nx,
                                            typename Storage<T>::C (&v)[N][Q19],
                                            std::integer_sequence<int, I...>)
{
    (m3_pull_one<I, T, N>(f, cst, xw, rw, zz, ny, nx, v), ...);
}

// The 19 N pre-collision values of a site.
template <typename T, int N>
__device__ __forceinline__ void m3_pull(const T* __restrict__ f, unsigned cst, const int (&xw)[3],
                                        const M3Rows& rw, const int (&zz)[3], int ny, int nx,
                                        typename Storage<T>::C (&v)[N][Q19])
{
    m3_pull_all<T, N>(f, cst, xw, rw, zz, ny, nx, v, std::make_integer_sequence<int, Q19>{});
}

template <typename T, int N>
__global__ void __launch_bounds__(M3_THREADS, 512 / M3_THREADS)
k19_march(const T* __restrict__ fin, T* __restrict__ fout,
          const typename Storage<T>::C* __restrict__ rs,
          const __grid_constant__ StepParams<typename Storage<T>::C> p, int H)
{
    using C = typename Storage<T>::C;
    extern __shared__ __align__(16) unsigned char m3_raw[];
    C* rring = reinterpret_cast<C*>(m3_raw);
    C* nring = rring + 3 * N * M3_ROWS * 32;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const int x0 = blockIdx.x * M3_OUT_X, y0 = blockIdx.y * M3_OUT_Y, z0 = blockIdx.z * H;
    const int Hc = min(H, nz - z0);
    const unsigned cst = 19u * (unsigned)p.S;   // stored values of one component

    // the lane's column and its neighbours
    int xw[3];
    xw[1] = pmod(x0 - 2 + lane, nx);
    xw[0] = dec_wrap(xw[1], nx);
    xw[2] = inc_wrap(xw[1], nx);

    // rows of phase A and B: r = warp + M3_WARPS j while r < M3_ROWS; of phase C: r = warp +
    // 2 + M3_WARPS j, j < M3_RC (one row at a time: a site's 19 N pulled values fill the
    // registers)
    constexpr int NA = (M3_ROWS + M3_WARPS - 1) / M3_WARPS;
    const bool xout = lane >= 2 && lane < 30 && x0 + lane - 2 < nx;

    const int nk = Hc + 4;
    for (int k = 0; k < nk; ++k) {
        const int m = z0 - 2 + k;
        // ---- A: rho^s of the lead plane m on every row and lane of the tile
        {
            const int zm = pmod(m, nz);
            const int q = k % 3;
#pragma unroll
            for (int j = 0; j < NA; ++j) {
                const int r = warp + M3_WARPS * j;
                if (r < M3_ROWS) {
                    const int y = pmod(y0 - 2 + r, ny);
                    const size_t site = ((size_t)zm * ny + y) * nx + xw[1];
#pragma unroll
                    for (int s = 0; s < N; ++s)
                        rring[m3_at<N>(q, s, r, lane)] = rs[(size_t)s * p.S + site];
                }
            }
        }
        __syncthreads();
        // ---- B: nu^s of plane m - 1 on rows 1 .. M3_ROWS - 2 and lanes 1 .. 30
        if (k >= 2 && lane >= 1 && lane < 31) {
            const int qc = (k + 2) % 3;          // density slot of plane m - 1
            const int qz[3] = {(k + 1) % 3, qc, k % 3};   // planes m - 2, m - 1, m
#pragma unroll 1
            for (int j = 0; j < NA; ++j) {
                const int r = warp + M3_WARPS * j;
                if (r >= 1 && r < M3_ROWS - 1) {
                    C rr[N], acc[N], lap[N], out[N];
#pragma unroll
                    for (int s = 0; s < N; ++s) {
                        rr[s] = rring[m3_at<N>(qc, s, r, lane)];
                        acc[s] = C(0);
                    }
#pragma unroll
                    for (int i = 1; i < Q19; ++i) {
                        const int q = qz[1 + c19(i, 2)];
                        const int rn = r + c19(i, 1), ln = lane + c19(i, 0);
#pragma unroll
                        for (int s = 0; s < N; ++s)
                            acc[s] += w19<C>(i) * (rring[m3_at<N>(q, s, rn, ln)] - rr[s]);
                    }
#pragma unroll
                    for (int s = 0; s < N; ++s) lap[s] = C(6) * acc[s];
                    site_nu<C, N>(p, rr, lap, out);
#pragma unroll
                    for (int s = 0; s < N; ++s) nring[m3_at<N>(k % 3, s, r, lane)] = out[s];
                }
            }
        }
        __syncthreads();
        // ---- C: collision of plane m - 2
        if (k >= 4) {
            int zz[3];
            zz[1] = pmod(m - 2, nz);
            zz[0] = dec_wrap(zz[1], nz);
            zz[2] = inc_wrap(zz[1], nz);
            const int qn[3] = {(k + 1) % 3, (k + 2) % 3, k % 3};   // nu planes m - 3 .. m - 1
#pragma unroll 1
            for (int j = 0; j < M3_RC; ++j) {
                const int r = warp + 2 + M3_WARPS * j;
                if (!xout || y0 + r - 2 >= ny) continue;
                const M3Rows rw = m3_rows(y0 - 2 + r, ny);
                C v[N][Q19];
                m3_pull<T, N>(fin, cst, xw, rw, zz, ny, nx, v);
                C rs[N], js[N][3];
#pragma unroll
                for (int s = 0; s < N; ++s) rs[s] = js[s][0] = js[s][1] = js[s][2] = C(0);
#pragma unroll
                for (int i = 0; i < Q19; ++i)
#pragma unroll
                    for (int s = 0; s < N; ++s) {
                        rs[s] += v[s][i];
#pragma unroll
                        for (int d = 0; d < 3; ++d)
                            if (c19(i, d)) js[s][d] += C(c19(i, d)) * v[s][i];
                    }
                C rho = C(0), jt[3] = {C(0), C(0), C(0)};
#pragma unroll
                for (int s = 0; s < N; ++s) {
                    rho += rs[s];
#pragma unroll
                    for (int d = 0; d < 3; ++d) jt[d] += js[s][d];
                }
                const C inv = C(1) / rho;
                const C u[3] = {jt[0] * inv, jt[1] * inv, jt[2] * inv};
                const C base = C(-1.5) * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
                // a^s = -(1 - 1/2tau) grad nu^s + g, grad g = 3 sum_i w_i v_i g(r + v_i)
                C a[N][3];
#pragma unroll
                for (int s = 0; s < N; ++s) a[s][0] = a[s][1] = a[s][2] = C(0);
#pragma unroll
                for (int i = 1; i < Q19; ++i) {
                    const int q = qn[1 + c19(i, 2)];
                    const int rn = r + c19(i, 1), ln = lane + c19(i, 0);
#pragma unroll
                    for (int s = 0; s < N; ++s) {
                        const C g = w19<C>(i) * nring[m3_at<N>(q, s, rn, ln)];
#pragma unroll
                        for (int d = 0; d < 3; ++d)
                            if (c19(i, d)) a[s][d] += C(c19(i, d)) * g;
                    }
                }
                const C gb[3] = {p.gx, p.gy, p.gz};
#pragma unroll
                for (int s = 0; s < N; ++s)
#pragma unroll
                    for (int d = 0; d < 3; ++d) a[s][d] = -p.fcoef * (C(3) * a[s][d]) + gb[d];
                // f* = f (1 - 1/tau) + (rho^s/tau) e_i + w_i [3 rho^s (v.a) + 9 (v.a)(v.J)
                // - 3 a.J + rho^s/tau] (as in k19_collide)
                C r3[N], omr[N], m3aj[N];
#pragma unroll
                for (int s = 0; s < N; ++s) {
                    if (p.bary)
#pragma unroll
                        for (int d = 0; d < 3; ++d) js[s][d] = rs[s] * u[d];
                    r3[s] = C(3) * rs[s];
                    omr[s] = p.omega * rs[s];
                    m3aj[s] = fma(C(-3), a[s][0] * js[s][0] + a[s][1] * js[s][1] + a[s][2] * js[s][2],
                                  omr[s]);
                }
                const C keep = C(1) - p.omega;
                const unsigned here = m3_rowbase(zz[1], rw.y[1], ny, nx) + (unsigned)xw[1];
#pragma unroll
                for (int i = 0; i < Q19; ++i) {
                    C cu = C(0);
#pragma unroll
                    for (int d = 0; d < 3; ++d)
                        if (c19(i, d)) cu += C(c19(i, d)) * u[d];
                    const C e = (i == 0) ? w19<C>(0) * base
                                         : w19<C>(i) * fma(cu, fma(C(4.5), cu, C(3)), base);
#pragma unroll
                    for (int s = 0; s < N; ++s) {
                        C ca = C(0), cj = C(0);
#pragma unroll
                        for (int d = 0; d < 3; ++d)
                            if (c19(i, d)) {
                                ca += C(c19(i, d)) * a[s][d];
                                cj += C(c19(i, d)) * js[s][d];
                            }
                        const C F = (i == 0) ? w19<C>(0) * m3aj[s]
                                             : w19<C>(i) * fma(ca, fma(C(9), cj, r3[s]), m3aj[s]);
                        fout[(size_t)s * cst + here + (unsigned)(i * nx)] =
                            T(fma(keep, v[s][i], fma(omr[s], e, F)));
                    }
                }
                if (!(rho > C(0)) || !isfinite(rho)) atomicOr(p.status, STATUS_NONFINITE);
            }
        }
    }
}

}  // namespace mclb
