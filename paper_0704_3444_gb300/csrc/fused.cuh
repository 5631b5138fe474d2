// fused.cuh -- one launch per timestep: pull streaming, moments, Flory-Huggins
// potentials with the gradient term, the Eq. definef force, equilibria, forcing
// and BGK collision in a single pass over the distributions.
//
// Decomposition.  A CTA owns a strip of W columns and sweeps a segment of H rows.
// The force at a site needs nu^s on its 8 neighbours, and nu^s needs rho^s on its
// neighbours (the kappa Laplacian), and rho^s needs the pulled distributions, so
// a collision at row r depends on source rows r-3 .. r+3.  The sweep keeps
//   - a ring of NS shared-memory stages, each holding one source row of all 9N
//     distribution planes over columns [x0 - hx, x0 + W + hx), filled by one
//     3-D TMA box copy (cp.async.bulk.tensor) per row and tracked by an mbarrier;
//   - a 4-row ring of rho^s over columns [x0 - 2, x0 + W + 2);
//   - a 4-row ring of nu^s over columns [x0 - 1, x0 + W + 1).
// Iteration j computes rho for row j-2, nu for row j-3 and collides row j-4
// (rows relative to the segment start), so each distribution is read from HBM
// once per step (plus the halo columns/rows shared with neighbouring tiles, which
// mostly hit L2) and written once.  Ghost columns in the global layout make every
// TMA box an in-bounds, 16-byte aligned row segment; periodicity in y is the row
// index modulo ny.
//
// Threads: W compute threads (one per column) plus one helper warp whose lane 0
// issues the TMA copies and whose lanes 0..3 handle the halo columns of rho and nu.
// Every wait on an mbarrier is bounded; on expiry the CTA sets STATUS_TIMEOUT,
// drains the copies it issued (again bounded) and returns.
#pragma once

#include "physics.cuh"

namespace mclb {

constexpr int FUSED_MAX_W = 128;
constexpr int FUSED_MAX_NS = 16;
constexpr int FUSED_HDR = 256;                 // barrier + flag header bytes
constexpr long long WAIT_LIMIT_CYCLES = 4000000000LL;  // about 2 s at the boost clock

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase with the given parity; false if it did not complete.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > WAIT_LIMIT_CYCLES) return false;
    return true;
}

// One 3-D TMA box (columns, 1 row, all planes) into shared memory.
__device__ __forceinline__ void tma_load_row(void* dst, const CUtensorMap* map, uint64_t* bar,
                                             int col, int row)
{
    const uint64_t desc = reinterpret_cast<uint64_t>(map);
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
        "l"(desc), "r"(smem_u32(bar)), "r"(col), "r"(row), "r"(0)
        : "memory");
}

template <typename T>
__device__ __forceinline__ typename Storage<T>::C to_c(T v);
template <>
__device__ __forceinline__ double to_c<double>(double v) { return v; }
template <>
__device__ __forceinline__ float to_c<float>(float v) { return v; }
template <>
__device__ __forceinline__ float to_c<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <>
__device__ __forceinline__ float to_c<__half>(__half v) { return __half2float(v); }

__host__ __device__ constexpr size_t round_up_sz(size_t a, size_t b) { return (a + b - 1) / b * b; }

template <typename T, int N>
__host__ __device__ constexpr size_t fused_stage_bytes(int W, int hx)
{
    return round_up_sz((size_t)N * Q * (W + 2 * hx) * sizeof(T), 128);
}

template <typename T, int N>
__host__ __device__ constexpr size_t fused_smem_bytes(int W, int NS, int hx)
{
    using C = typename Storage<T>::C;
    return FUSED_HDR + (size_t)NS * fused_stage_bytes<T, N>(W, hx) +
           (size_t)4 * N * (W + 4) * sizeof(C) + (size_t)4 * N * (W + 2) * sizeof(C);
}

template <typename T, int N>
__global__ void __launch_bounds__(FUSED_MAX_W + 32, 1)
k_fused(const __grid_constant__ CUtensorMap tmap, T* __restrict__ fout,
        const __grid_constant__ StepParams<typename Storage<T>::C> p, const int W, const int NS,
        const int H)
{
    using C = typename Storage<T>::C;
    constexpr int NP = N * Q;
    const int hx = p.hx;
    const int WI = W + 2 * hx;   // staged columns per plane
    const int RW = W + 4;        // rho ring columns: x0-2 .. x0+W+1
    const int VW = W + 2;        // nu ring columns:  x0-1 .. x0+W
    const int x0 = blockIdx.x * W;
    const int y0 = blockIdx.y * H;
    const int Hc = min(H, p.ny - y0);
    const int nrows = Hc + 6;    // source rows k <-> global row y0 - 3 + k (mod ny)
    const int tid = threadIdx.x;
    const bool compute = tid < W;
    const int lane = tid - W;

    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + 8 * FUSED_MAX_NS);
    const size_t stage_elems = fused_stage_bytes<T, N>(W, hx) / sizeof(T);
    T* stages = reinterpret_cast<T*>(smem + FUSED_HDR);
    C* rho_ring = reinterpret_cast<C*>(smem + FUSED_HDR + NS * stage_elems * sizeof(T));
    C* nu_ring = rho_ring + 4 * N * RW;

    const uint32_t tx_bytes = (uint32_t)(NP * WI * sizeof(T));
    if (tid == W) {
        for (int s = 0; s < NS; ++s) mbar_init(&full[s], 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();

    auto issue = [&](int k) {
        const int st = k % NS;
        int row = (y0 - 3 + k) % p.ny;
        row += row < 0 ? p.ny : 0;
        mbar_arrive_expect_tx(&full[st], tx_bytes);
        tma_load_row(stages + st * stage_elems, &tmap, &full[st], x0, row);
    };
    int issued = 0;  // rows issued so far (meaningful in the producer thread)
    if (tid == W) {
        const int pre = min(NS, nrows);
        for (int k = 0; k < pre; ++k) issue(k);
        issued = pre;
    }
    auto wait_row = [&](int k) -> bool { return mbar_wait(&full[k % NS], (k / NS) & 1); };
    auto stage_of = [&](int k) -> const T* { return stages + (k % NS) * stage_elems; };

    bool ok = wait_row(0);
    ok = wait_row(1) && ok;
    if (!ok) *abort_flag = 1;

    int j = 0;
    for (; j < Hc + 4; ++j) {
        if (!wait_row(j + 2)) *abort_flag = 1;

        // ---- phase A: rho^s of row j-2 into ring slot j&3 (source rows j .. j+2)
        {
            const T* sr[3] = {stage_of(j + 2), stage_of(j + 1), stage_of(j)};  // dy = -1, 0, +1
            C* rr = rho_ring + (j & 3) * N * RW;
            auto rho_col = [&](int c) {
#pragma unroll
                for (int s = 0; s < N; ++s) {
                    C acc = C(0);
#pragma unroll
                    for (int i = 0; i < Q; ++i) {
                        const T* row = sr[vy(i) + 1];
                        C v = to_c<T>(row[(s * Q + i) * WI + c - 2 + hx - vx(i)]);
                        if constexpr (Storage<T>::shifted) v += p.shift[s * Q + i];
                        acc += v;
                    }
                    rr[s * RW + c] = acc;
                }
            };
            if (compute) rho_col(tid + 2);
            else if (lane < 4) rho_col(lane < 2 ? lane : W + lane);
        }
        __syncthreads();
        if (*abort_flag) break;
        if (tid == W && j >= 3) {
            const int k = j - 3 + NS;  // reuse the stage of row j-3, last read by phase C of j-1
            if (k < nrows) {
                issue(k);
                issued = k + 1;
            }
        }

        // ---- phase B: nu^s of row j-3 into ring slot j&3 (rho rows j-4 .. j-2)
        if (j >= 2) {
            const C* rrow[3] = {rho_ring + ((j - 2) & 3) * N * RW, rho_ring + ((j - 1) & 3) * N * RW,
                                rho_ring + (j & 3) * N * RW};  // dy = -1, 0, +1
            C* nn = nu_ring + (j & 3) * N * VW;
            auto nu_col = [&](int cc) {
                const int c = cc + 1;
                C r[N], lap[N], out[N];
#pragma unroll
                for (int s = 0; s < N; ++s) r[s] = rrow[1][s * RW + c];
#pragma unroll
                for (int s = 0; s < N; ++s) {
                    C acc = C(0);
#pragma unroll
                    for (int i = 0; i < Q; ++i)
                        acc += wq<C>(i) * (rrow[vy(i) + 1][s * RW + c + vx(i)] - r[s]);
                    lap[s] = C(6) * acc;
                }
                site_nu<C, N>(p, r, lap, out);
#pragma unroll
                for (int s = 0; s < N; ++s) nn[s * VW + cc] = out[s];
            };
            if (compute) nu_col(tid + 1);
            else if (lane < 2) nu_col(lane == 0 ? 0 : W + 1);
        }
        __syncthreads();

        // ---- phase C: collide row j-4 (source rows j-2 .. j, nu rows j-5 .. j-3)
        if (j >= 4 && compute) {
            const int x = x0 + tid;
            const int r = j - 4;
            if (x < p.nx) {
                const T* sr[3] = {stage_of(j), stage_of(j - 1), stage_of(j - 2)};  // dy = -1, 0, +1
                const C* vrow[3] = {nu_ring + ((j - 2) & 3) * N * VW,
                                    nu_ring + ((j - 1) & 3) * N * VW, nu_ring + (j & 3) * N * VW};
                C f[N][Q];
                C rs[N], jx[N], jy[N];
                C rho = C(0), jxt = C(0), jyt = C(0);
#pragma unroll
                for (int s = 0; s < N; ++s) {
#pragma unroll
                    for (int i = 0; i < Q; ++i) {
                        C v = to_c<T>(sr[vy(i) + 1][(s * Q + i) * WI + tid + hx - vx(i)]);
                        if constexpr (Storage<T>::shifted) v += p.shift[s * Q + i];
                        f[s][i] = v;
                    }
                    const C a = f[s][0] + f[s][1] + f[s][2] + f[s][3] + f[s][4] + f[s][5] +
                                f[s][6] + f[s][7] + f[s][8];
                    const C bx = (f[s][1] + f[s][5] + f[s][8]) - (f[s][3] + f[s][6] + f[s][7]);
                    const C by = (f[s][2] + f[s][5] + f[s][6]) - (f[s][4] + f[s][7] + f[s][8]);
                    rs[s] = a;
                    jx[s] = bx;
                    jy[s] = by;
                    rho += a;
                    jxt += bx;
                    jyt += by;
                }
                const C inv_rho = C(1) / rho;
                const C ux = jxt * inv_rho, uy = jyt * inv_rho;
                C e[Q];
                eq_weights(ux, uy, e);
                const long long rowoff = (long long)(y0 + r) * p.pitch;
#pragma unroll
                for (int s = 0; s < N; ++s) {
                    // grad nu = 3 sum_i w_i v_i nu(r + v_i)
                    C gx = C(0), gy = C(0);
#pragma unroll
                    for (int i = 1; i < Q; ++i) {
                        const C v = vrow[vy(i) + 1][s * VW + tid + 1 + vx(i)];
                        gx += wq<C>(i) * C(vx(i)) * v;
                        gy += wq<C>(i) * C(vy(i)) * v;
                    }
                    const C ax = -p.fcoef * (C(3) * gx) + p.gx;
                    const C ay = -p.fcoef * (C(3) * gy) + p.gy;
                    C out[Q];
                    collide(p, f[s], e, rs[s], jx[s], jy[s], ax, ay, out);
#pragma unroll
                    for (int i = 0; i < Q; ++i) {
                        C v = out[i];
                        if constexpr (Storage<T>::shifted) v -= p.shift[s * Q + i];
                        store_row(fout + (long long)(s * Q + i) * p.plane + rowoff, x, p.nx, hx, v);
                    }
                }
                if (!(rho > C(0)) || !isfinite(rho)) atomicOr(p.status, STATUS_NONFINITE);
            }
        }
    }

    if (*abort_flag) {
        if (tid == 0) atomicOr(p.status, STATUS_TIMEOUT);
        // drain the copies still in flight before the shared memory is released
        if (tid == W)
            for (int k = j + 3; k < issued; ++k) wait_row(k);
    }
}

}  // namespace mclb
