// fused.cuh -- one launch per timestep: pull streaming, moments, Flory-Huggins
// potentials with the gradient term, the Eq. definef force, equilibria, forcing
// and BGK collision in a single pass over the distributions.
//
// Decomposition.  A CTA owns a strip of W columns and sweeps a segment of H rows.
// The force at a site needs nu^s on its 8 neighbours, and nu^s needs rho^s on its
// neighbours (the kappa Laplacian), and rho^s needs the pulled distributions, so
// a collision at row r depends on source rows r-3 .. r+3.  The sweep keeps
//   - a ring of NS shared-memory stages, each holding one source row of all 9N
//     distribution lines over columns [x0 - hx, x0 + W + hx), filled by one
//     4-D TMA box copy (cp.async.bulk.tensor) per row and tracked by an mbarrier;
//   - a 4-row ring of the moments rho^s, j^s over columns [x0 - 2, x0 + W + 2);
//   - a 4-row ring of nu^s over columns [x0 - 1, x0 + W + 1).
// Iteration j computes the moments of row j-2, nu of row j-3 and collides row j-4
// (rows relative to the segment start), so each distribution is read from HBM
// once per step (plus the halo columns/rows shared with neighbouring tiles, which
// mostly hit L2) and written once.  Ghost columns in the global layout make every
// TMA box an in-bounds, 16-byte aligned row segment; periodicity in y is the row
// index modulo ny.
//
// Threads.  One warp group of W threads per component: thread (s, c) handles
// component s at column x0 + c in every phase, so a CTA runs N*W threads on the
// interior plus one helper warp, whose lanes compute the halo columns of the
// moment and nu rings and whose lane 0 issues the TMA copies.  Every wait on an
// mbarrier is bounded; on expiry the CTA sets STATUS_TIMEOUT, drains the copies it
// issued (again bounded) and returns.
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

// One 4-D TMA box (columns, 9 velocities, 1 row, all components) into shared memory.
__device__ __forceinline__ void tma_load_row(void* dst, const CUtensorMap* map, uint64_t* bar,
                                             int col, int row)
{
    const uint64_t desc = reinterpret_cast<uint64_t>(map);
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5, %6}], [%2];" ::"r"(smem_u32(dst)),
        "l"(desc), "r"(smem_u32(bar)), "r"(col), "r"(0), "r"(row), "r"(0)
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
           (size_t)4 * 3 * N * (W + 4) * sizeof(C) + (size_t)4 * N * (W + 2) * sizeof(C);
}

constexpr int FUSED_MAX_THREADS = 1024;

template <typename T, int N>
__global__ void __launch_bounds__(FUSED_MAX_THREADS, 1)
k_fused(const __grid_constant__ CUtensorMap tmap, T* __restrict__ fout,
        const __grid_constant__ StepParams<typename Storage<T>::C> p, const int W, const int NS,
        const int H)
{
    using C = typename Storage<T>::C;
    const int hx = p.hx;
    const int WI = W + 2 * hx;   // staged columns per line
    const int RW = W + 4;        // moment ring columns: x0-2 .. x0+W+1
    const int VW = W + 2;        // nu ring columns:     x0-1 .. x0+W
    const int x0 = blockIdx.x * W;
    const int y0 = blockIdx.y * H;
    const int Hc = min(H, p.ny - y0);
    const int nrows = Hc + 6;    // source rows k <-> global row y0 - 3 + k (mod ny)
    const int tid = threadIdx.x;
    const int nct = N * W;
    const bool helper = tid >= nct;
    const int g = helper ? 0 : tid / W;   // component of this thread
    const int c = helper ? 0 : tid - g * W;
    const int lane = tid - nct;           // helper lane

    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + 8 * FUSED_MAX_NS);
    const size_t stage_elems = fused_stage_bytes<T, N>(W, hx) / sizeof(T);
    T* stages = reinterpret_cast<T*>(smem + FUSED_HDR);
    C* mom = reinterpret_cast<C*>(smem + FUSED_HDR + NS * stage_elems * sizeof(T));
    C* nur = mom + 4 * 3 * N * RW;
    // moment ring: slot, quantity (rho, jx, jy), component, column
    auto mom_at = [&](int slot, int q, int s, int col) -> C& {
        return mom[((slot * 3 + q) * N + s) * RW + col];
    };

    const uint32_t tx_bytes = (uint32_t)(N * Q * WI * sizeof(T));
    if (tid == nct) {
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
    int issued = 0;
    if (tid == nct) {
        const int pre = min(NS, nrows);
        for (int k = 0; k < pre; ++k) issue(k);
        issued = pre;
    }
    auto wait_row = [&](int k) -> bool { return mbar_wait(&full[k % NS], (k / NS) & 1); };
    auto stage_of = [&](int k) -> const T* { return stages + (k % NS) * stage_elems; };

    // per-thread constants of its component
    C shift[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) shift[i] = Storage<T>::shifted ? p.shift[g * Q + i] : C(0);

    // moments rho, jx, jy of component s at ring column cc of the row whose source
    // rows are sr[0..2] (dy = -1, 0, +1)
    auto moments_at = [&](const T* const (&sr)[3], int s, int cc, int slot, const C* sh) {
        C v[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            v[i] = to_c<T>(sr[vy(i) + 1][(s * Q + i) * WI + cc - 2 + hx - vx(i)]);
            if constexpr (Storage<T>::shifted) v[i] += sh[i];
        }
        C r = C(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) r += v[i];
        mom_at(slot, 0, s, cc) = r;
        mom_at(slot, 1, s, cc) = (v[1] + v[5] + v[8]) - (v[3] + v[6] + v[7]);
        mom_at(slot, 2, s, cc) = (v[2] + v[5] + v[6]) - (v[4] + v[7] + v[8]);
    };

    // nu^s at nu-ring column vc of row r (moment slots rs[0..2] for rows r-1, r, r+1)
    auto nu_at = [&](const int (&rs)[3], int s, int vc) -> C {
        const int cc = vc + 1;
        C r[N];
        C rho = C(0);
#pragma unroll
        for (int t = 0; t < N; ++t) {
            r[t] = mom_at(rs[1], 0, t, cc);
            rho += r[t];
        }
        const C inv_rho = C(1) / rho;
        C phi[N];
#pragma unroll
        for (int t = 0; t < N; ++t) phi[t] = r[t] * inv_rho;
        C sum_phi_m = C(0);
#pragma unroll
        for (int t = 0; t < N; ++t) sum_phi_m += phi[t] * p.inv_m[t];
        C quad = C(0);
#pragma unroll
        for (int t = 0; t < N; ++t) {
            C acc = C(0);
#pragma unroll
            for (int u = 0; u < N; ++u) acc += p.chi[t * N + u] * phi[u];
            quad += C(0.5) * phi[t] * acc;
        }
        C chiphi = C(0);
#pragma unroll
        for (int u = 0; u < N; ++u) chiphi += p.chi[s * N + u] * phi[u];
        C rs_own = mom_at(rs[1], 0, s, cc);
        C acc = C(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) acc += wq<C>(i) * (mom_at(rs[vy(i) + 1], 0, s, cc + vx(i)) - rs_own);
        const C lap = C(6) * acc;
        C logs = -p.th_m[s] * dev_log(rho);
        if (p.log_mask & (1u << s)) {
            const C fl = p.log_floor * rho;
            logs += p.logc[s] * dev_log(rs_own > fl ? rs_own : fl);
        }
        const C bulk = p.theta * (p.m_inv_m1[s] - sum_phi_m + chiphi - quad);
        return logs + bulk - p.kappa * lap;
    };

    bool ok = wait_row(0);
    ok = wait_row(1) && ok;
    if (!ok) *abort_flag = 1;

    int j = 0;
    for (; j < Hc + 4; ++j) {
        if (!wait_row(j + 2)) *abort_flag = 1;

        // ---- phase A: moments of row j-2 into ring slot j&3 (source rows j .. j+2)
        {
            const T* const sr[3] = {stage_of(j + 2), stage_of(j + 1), stage_of(j)};
            if (!helper) {
                moments_at(sr, g, c + 2, j & 3, shift);
            } else if (lane < 4 * N) {
                const int hc = lane / N, s = lane - hc * N;
                C sh[Q];
#pragma unroll
                for (int i = 0; i < Q; ++i) sh[i] = Storage<T>::shifted ? p.shift[s * Q + i] : C(0);
                moments_at(sr, s, hc < 2 ? hc : W + hc, j & 3, sh);
            }
        }
        __syncthreads();
        if (*abort_flag) break;
        if (tid == nct && j >= 3) {
            const int k = j - 3 + NS;  // reuse the stage of row j-3, last read by phase C of j-1
            if (k < nrows) {
                issue(k);
                issued = k + 1;
            }
        }

        // ---- phase B: nu of row j-3 into ring slot j&3 (moment rows j-4 .. j-2)
        if (j >= 2) {
            const int rs[3] = {(j - 2) & 3, (j - 1) & 3, j & 3};
            C* nn = nur + (j & 3) * N * VW;
            if (!helper) {
                nn[g * VW + c + 1] = nu_at(rs, g, c + 1);
            } else if (lane < 2 * N) {
                const int hv = lane / N, s = lane - hv * N;
                const int vc = hv == 0 ? 0 : W + 1;
                nn[s * VW + vc] = nu_at(rs, s, vc);
            }
        }
        __syncthreads();

        // ---- phase C: collide row j-4 (source rows j-2 .. j, nu rows j-5 .. j-3)
        if (j >= 4 && !helper) {
            const int x = x0 + c;
            const int r = j - 4;
            if (x < p.nx) {
                const T* const sr[3] = {stage_of(j), stage_of(j - 1), stage_of(j - 2)};
                C f[Q];
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    f[i] = to_c<T>(sr[vy(i) + 1][(g * Q + i) * WI + c + hx - vx(i)]);
                    if constexpr (Storage<T>::shifted) f[i] += shift[i];
                }
                const int ms = (j - 2) & 3;  // moment slot of row j-4
                const int cc = c + 2;
                C rho = C(0), jxt = C(0), jyt = C(0);
#pragma unroll
                for (int t = 0; t < N; ++t) {
                    rho += mom_at(ms, 0, t, cc);
                    jxt += mom_at(ms, 1, t, cc);
                    jyt += mom_at(ms, 2, t, cc);
                }
                const C rg = mom_at(ms, 0, g, cc);
                const C jxg = mom_at(ms, 1, g, cc);
                const C jyg = mom_at(ms, 2, g, cc);
                const C inv_rho = C(1) / rho;
                C e[Q];
                eq_weights(jxt * inv_rho, jyt * inv_rho, e);
                // grad nu = 3 sum_i w_i v_i nu(r + v_i)
                const C* vrow[3] = {nur + ((j - 2) & 3) * N * VW + g * VW,
                                    nur + ((j - 1) & 3) * N * VW + g * VW,
                                    nur + (j & 3) * N * VW + g * VW};
                C gx = C(0), gy = C(0);
#pragma unroll
                for (int i = 1; i < Q; ++i) {
                    const C v = vrow[vy(i) + 1][c + 1 + vx(i)];
                    if (vx(i) != 0) gx += wq<C>(i) * C(vx(i)) * v;
                    if (vy(i) != 0) gy += wq<C>(i) * C(vy(i)) * v;
                }
                const C ax = -p.fcoef * (C(3) * gx) + p.gx;
                const C ay = -p.fcoef * (C(3) * gy) + p.gy;
                C out[Q];
                collide(p, f, e, rg, jxg, jyg, ax, ay, out);
                T* line = fout + line_off(p, g, y0 + r, 0);
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    C v = out[i];
                    if constexpr (Storage<T>::shifted) v -= shift[i];
                    store_row(line + i * p.pitch, x, p.nx, hx, v);
                }
                if (g == 0 && (!(rho > C(0)) || !isfinite(rho))) atomicOr(p.status, STATUS_NONFINITE);
            }
        }
    }

    if (*abort_flag) {
        if (tid == 0) atomicOr(p.status, STATUS_TIMEOUT);
        // drain the copies still in flight before the shared memory is released
        if (tid == nct)
            for (int k = j + 2; k < issued; ++k) wait_row(k);
    }
}

}  // namespace mclb
