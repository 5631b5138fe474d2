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
// Threads.  One warp per component: lane c handles that component at columns
// x0 + c and x0 + c + 32 of a 64-column strip in every phase, which halves the
// per-thread index and control work per site.  Two "site" warps (one column per
// thread) compute, once per site, what all components share: rho, 1/rho, ln rho,
// the common part of the Flory-Huggins potential and the nine equilibrium weights
// e_i.  One helper warp computes the halo columns of the rings; its last lane issues
// the TMA copies plus an L2 prefetch four rows beyond each copy.  Every wait on an
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

// try_wait with a suspend-time hint: a thread whose phase is not complete sleeps in
// hardware (up to the hint) instead of re-polling.
constexpr uint32_t WAIT_SUSPEND_NS = 200000;

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        "selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(WAIT_SUSPEND_NS)
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

// One 3-D TMA box (columns, 1 row, all components) of the FP32 density lines.
__device__ __forceinline__ void tma_load_rline(void* dst, const CUtensorMap* map, uint64_t* bar,
                                               int col, int row)
{
    const uint64_t desc = reinterpret_cast<uint64_t>(map);
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
        "l"(desc), "r"(smem_u32(bar)), "r"(col), "r"(row), "r"(0)
        : "memory");
}

// Prefetch the same 4-D box into L2 only (no shared memory, no barrier).
__device__ __forceinline__ void tma_prefetch_row(const CUtensorMap* map, int col, int row)
{
    const uint64_t desc = reinterpret_cast<uint64_t>(map);
    asm volatile("cp.async.bulk.prefetch.tensor.4d.L2.global [%0, {%1, %2, %3, %4}];" ::"l"(desc),
                 "r"(col), "r"(0), "r"(row), "r"(0)
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

// Compile-time geometry of one CTA: a strip of W = 32 COLS columns; each component
// thread handles the COLS columns c, c + 32, ... of its component; COLS site warps
// handle one column per thread; one helper warp does the halo columns and issues the
// copies.
template <typename T, int N, int COLS>
struct FusedGeom {
    using C = typename Storage<T>::C;
    static constexpr int W = 32 * COLS;
    static constexpr int NS = 6;                       // source-row stages
    static constexpr int PF = 4;                       // L2 prefetch distance (rows) of a copy
    static constexpr int HX = (16 / (int)sizeof(T)) < 4 ? 4 : 16 / (int)sizeof(T);
    static constexpr int WI = W + 2 * HX;              // staged columns per line
    static constexpr int RW = W + 4;                   // moment ring: x0-2 .. x0+W+1
    static constexpr int VW = W + 2;                   // nu ring:     x0-1 .. x0+W
    static constexpr int NCT = N * 32;                 // component threads (2 columns each)
    static constexpr int NST = W;                      // site threads (1 column each)
    static constexpr int THREADS = NCT + NST + 32;     // + helper warp
    static constexpr int PRODUCER = THREADS - 1;       // helper lane issuing the copies
    // one stage: the 9 N lines of a source row, then (16-bit formats) its N FP32
    // density lines at byte offset DEV_BYTES
    static constexpr bool SHIFTED = Storage<T>::shifted;
    static constexpr size_t DEV_BYTES = round_up_sz((size_t)N * Q * WI * sizeof(T), 128);
    static constexpr size_t R_BYTES = SHIFTED ? (size_t)N * WI * sizeof(float) : 0;
    static constexpr size_t STAGE_BYTES = round_up_sz(DEV_BYTES + R_BYTES, 128);
    static constexpr int STAGE_ELEMS = (int)(STAGE_BYTES / sizeof(T));
    static constexpr int STAGE_FLOATS = (int)(STAGE_BYTES / sizeof(float));
    static constexpr int R_FLOAT0 = (int)(DEV_BYTES / sizeof(float));
    static constexpr uint32_t TX = (uint32_t)((size_t)N * Q * WI * sizeof(T) + R_BYTES);
    // rings (elements of C).  Slot counts follow from who reads a row after the barrier
    // that follows its write: moments of row r are read until phase C two iterations
    // later and are overwritten by the next phase A without a barrier in between (4);
    // nu of row r is read by three collisions (3); site terms and equilibrium weights
    // of row r are written in phase A one iteration before the collision of row r, and
    // the next phase A may run before that collision ends (3 for the weights; the site
    // terms are read only by the phase B of the iteration that wrote them (1)).
    static constexpr int MOM_SLOT = 3 * N * RW;        // (rho, jx, jy), component, column
    static constexpr int MOM = 4 * MOM_SLOT;
    static constexpr int NU_SLOT = N * VW;             // component, column
    static constexpr int NU = 3 * NU_SLOT;
    static constexpr int SH = 4 * VW;                  // (rho, 1/rho, ln rho, G), nu column
    static constexpr int EQ_SLOT = Q * W;              // velocity, column
    static constexpr int EQ = 3 * EQ_SLOT;
    static constexpr size_t SMEM = FUSED_HDR + NS * STAGE_BYTES + (size_t)(MOM + NU + SH + EQ) * sizeof(C);
    static constexpr int MIN_CTAS = (2 * (SMEM + 1024) <= 228 * 1024) ? 2 : 1;
};

constexpr int FUSED_MAX_THREADS = 1024;

template <typename T, int N, int COLS>
__global__ void __launch_bounds__(FusedGeom<T, N, COLS>::THREADS, FusedGeom<T, N, COLS>::MIN_CTAS)
k_fused(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ CUtensorMap tmapr,
        T* __restrict__ fout, const __grid_constant__ StepParams<typename Storage<T>::C> p,
        const int H)
{
    using G = FusedGeom<T, N, COLS>;
    using C = typename Storage<T>::C;
    constexpr int W = G::W, NS = G::NS, HX = G::HX, WI = G::WI, RW = G::RW, VW = G::VW;
    constexpr int NCT = G::NCT, NST = G::NST;
    const int x0 = blockIdx.x * W;
    const int y0 = blockIdx.y * H;
    const int Hc = min(H, p.ny - y0);
    const int nrows = Hc + 6;    // source rows k <-> global row y0 - 3 + k (mod ny)
    const int tid = threadIdx.x;
    const bool comp = tid < NCT;
    const bool site = !comp && tid < NCT + NST;
    const int g = comp ? (tid >> 5) : 0;               // component of a component thread
    const int c = comp ? (tid & 31) : (site ? tid - NCT : 0);  // first column
    const int lane = tid - NCT - NST;                  // helper lane (>= 0 in the helper warp)

    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + 8 * FUSED_MAX_NS);
    T* stg = reinterpret_cast<T*>(smem + FUSED_HDR);
    const float* stgr = reinterpret_cast<const float*>(smem + FUSED_HDR) + G::R_FLOAT0;
    C* mom = reinterpret_cast<C*>(smem + FUSED_HDR + NS * G::STAGE_BYTES);
    C* nur = mom + G::MOM;
    C* shr = nur + G::NU;
    C* eqr = shr + G::SH;

    if (tid == G::PRODUCER) {
        for (int s = 0; s < NS; ++s) mbar_init(&full[s], 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();

    constexpr uint32_t TX = G::TX;
    auto grow = [&](int k) {
        int row = (y0 - 3 + k) % p.ny;
        return row + (row < 0 ? p.ny : 0);
    };
    auto issue = [&](int k) {
        const int st = k % NS;
        mbar_arrive_expect_tx(&full[st], TX);
        tma_load_row(stg + st * G::STAGE_ELEMS, &tmap, &full[st], x0, grow(k));
        if constexpr (G::SHIFTED)
            tma_load_rline(smem + FUSED_HDR + st * G::STAGE_BYTES + G::DEV_BYTES, &tmapr, &full[st],
                           x0, grow(k));
        if (k + G::PF < nrows) tma_prefetch_row(&tmap, x0, grow(k + G::PF));
    };
    int issued = 0;
    if (tid == G::PRODUCER) {
        const int pre = min(NS, nrows);
        for (int k = 0; k < pre; ++k) issue(k);
        issued = pre;
    }
    auto wait_row = [&](int k) -> bool { return mbar_wait(&full[k % NS], (k / NS) & 1); };

    // constants of this thread's component, kept in registers
    C chi_row[N];
#pragma unroll
    for (int u = 0; u < N; ++u) chi_row[u] = p.chi[g * N + u];
    const C th_m = p.th_m[g], logc = p.logc[g], minv1 = p.m_inv_m1[g];
    const bool has_log = (p.log_mask >> g) & 1u;

    // pulled value of velocity i: a = stage element offset of the velocity-0 line (column
    // applied) of the source row; in the 16-bit formats the deviation plus w_i times the
    // density line of the same source site (float offset ra)
    auto pulled = [&](int i, int a, int ra) -> C {
        C v = to_c<T>(stg[a + i * WI - vx(i)]);
        if constexpr (G::SHIFTED) v = fma(wq<C>(i), stgr[ra - vx(i)], v);
        return v;
    };
    // stage float offset of a density-line column, from the stage element offset of the
    // stage and the component/column part
    auto roff = [&](int st, int s, int colx) -> int {
        return st * (int)sizeof(T) / (int)sizeof(float) + s * WI + colx;
    };

    // moments of one component at one column: s0/s1/s2 are the stage element offsets of
    // the source rows for dy = -1, 0, +1, s the component, cx the staged column
    auto moments_to = [&](int s0, int s1, int s2, int s, int cx, int dst) {
        const int sr[3] = {s0, s1, s2};
        const int col = s * Q * WI + cx;
        C v[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int st = sr[vy(i) + 1];
            v[i] = pulled(i, st + col, G::SHIFTED ? roff(st, s, cx) : 0);
        }
        C r = C(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) r += v[i];
        mom[dst] = r;
        mom[dst + N * RW] = (v[1] + v[5] + v[8]) - (v[3] + v[6] + v[7]);
        mom[dst + 2 * N * RW] = (v[2] + v[5] + v[6]) - (v[4] + v[7] + v[8]);
    };

    // site terms from the densities of all components at one column (offset of
    // component 0, stride RW): returns rho and 1/rho, stores rho, 1/rho, ln rho and
    // G = -theta (sum phi/m + 1/2 sum chi phi phi) at nu column vc
    auto site_terms = [&](int m0, int vc, C& inv_out) -> C {
        C r[N];
        C rho = C(0);
#pragma unroll
        for (int t = 0; t < N; ++t) {
            r[t] = mom[m0 + t * RW];
            rho += r[t];
        }
        const C inv = C(1) / rho;
        C sm = C(0), quad = C(0);
#pragma unroll
        for (int t = 0; t < N; ++t) {
            sm += r[t] * p.inv_m[t];
            C acc = C(0);
#pragma unroll
            for (int u = 0; u < N; ++u) acc += p.chi[t * N + u] * r[u];
            quad += r[t] * acc;
        }
        shr[vc] = rho;
        shr[VW + vc] = inv;
        shr[2 * VW + vc] = dev_log(rho);
        shr[3 * VW + vc] = -p.theta * (sm * inv + C(0.5) * quad * inv * inv);
        inv_out = inv;
        return rho;
    };

    // nu^s at one column: m[dy+1] = moment offsets of component s at the column in rows
    // r-1, r, r+1; d0 = offset of component 0 in row r; site terms at nu column vc
    auto nu_of = [&](int mm, int m0, int mp, int d0, int vc, int s, const C (&chi_s)[N], C thm,
                     C lc, C mi1, bool lg) -> C {
        const int mr[3] = {mm, m0, mp};
        C acc = C(0);
#pragma unroll
        for (int u = 0; u < N; ++u) acc += chi_s[u] * mom[d0 + u * RW];
        const C own = mom[m0];
        C lap = C(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) lap += wq<C>(i) * (mom[mr[vy(i) + 1] + vx(i)] - own);
        C logs = -thm * shr[2 * VW + vc];
        if (lg) {
            const C fl = p.log_floor * shr[vc];
            logs += lc * dev_log(own > fl ? own : fl);
        }
        (void)s;
        return logs + p.theta * (mi1 + acc * shr[VW + vc]) + shr[3 * VW + vc] - p.kappa * (C(6) * lap);
    };

    // collision of component g at first-column offset cc (0 or 32) of the strip
    auto collide_col = [&](int cc, int s0, int s1, int s2, int momr, int eqo, int n0, int n1, int n2,
                           T* line, float* rline, bool ghost) {
        const int x = x0 + c + cc;
        if (x >= p.nx) return;
        const int cx = c + cc + HX;
        const int col = g * Q * WI + cx;
        const int sr[3] = {s0, s1, s2};
        C f[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int st = sr[vy(i) + 1];
            f[i] = pulled(i, st + col, G::SHIFTED ? roff(st, g, cx) : 0);
        }
        const int mg = momr + g * RW + c + cc + 2;
        const C rg = mom[mg], jxg = mom[mg + N * RW], jyg = mom[mg + 2 * N * RW];
        C e[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) e[i] = eqr[eqo + i * W + c + cc];
        const int vo = g * VW + c + cc + 1;
        const int nr[3] = {n0 + vo, n1 + vo, n2 + vo};
        C gx = C(0), gy = C(0);
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const C v = nur[nr[vy(i) + 1] + vx(i)];
            if (vx(i) != 0) gx += wq<C>(i) * C(vx(i)) * v;
            if (vy(i) != 0) gy += wq<C>(i) * C(vy(i)) * v;
        }
        const C ax = -p.fcoef * (C(3) * gx) + p.gx;
        const C ay = -p.fcoef * (C(3) * gy) + p.gy;
        C out[Q];
        collide(p, f, e, rg, jxg, jyg, ax, ay, out);
        C rref = C(0);
        if constexpr (G::SHIFTED) {
            // deviations from w_i M, rounded to storage, and the compensated reference
            // density R = M - sum_i d_i (the same rule as store_site)
            C M = C(0);
#pragma unroll
            for (int i = 0; i < Q; ++i) M += out[i];
            C dsum = C(0);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                out[i] = Storage<T>::round(out[i] - wq<C>(i) * M);
                dsum += out[i];
            }
            rref = M - dsum;
        }
        if (!ghost) {
            T* q = line + HX + x;
#pragma unroll
            for (int i = 0; i < Q; ++i) Storage<T>::store(q + i * p.pitch, out[i]);
            if constexpr (G::SHIFTED) rline[HX + x] = rref;
        } else {
#pragma unroll
            for (int i = 0; i < Q; ++i) store_row(line + i * p.pitch, x, p.nx, HX, out[i]);
            if constexpr (G::SHIFTED) store_row(rline, x, p.nx, HX, rref);
        }
    };

    // columns whose value is repeated in a ghost column
    auto has_ghost = [&](int x) { return p.nx < HX || x < HX || x >= p.nx - HX; };
    bool ghost[COLS];
#pragma unroll
    for (int k = 0; k < COLS; ++k) ghost[k] = has_ghost(x0 + c + 32 * k);

    bool ok = true;
    if (!site) {
        ok = wait_row(0);
        ok = wait_row(1) && ok;
    }
    if (!ok) *abort_flag = 1;

    int j = 0;
    int sj = 0;   // stage of source row j
    int j3 = 0;   // j mod 3
    for (; j < Hc + 4; ++j) {
        if (!site && !wait_row(j + 2)) *abort_flag = 1;
        auto stage_off = [&](int d) -> int {  // element offset of the stage of row j + d
            int s_ = sj + d;
            s_ += (s_ < 0) ? NS : 0;
            s_ -= (s_ >= NS) ? NS : 0;
            return s_ * G::STAGE_ELEMS;
        };
        const int st0 = stage_off(0), stp1 = stage_off(1), stp2 = stage_off(2);
        const int stm1 = stage_off(-1), stm2 = stage_off(-2);
        const int momA = (j & 3) * G::MOM_SLOT;        // row j-2
        const int momB = ((j - 1) & 3) * G::MOM_SLOT;  // row j-3
        const int momC = ((j - 2) & 3) * G::MOM_SLOT;  // row j-4
        const int j3p1 = (j3 == 2) ? 0 : j3 + 1, j3p2 = (j3 == 0) ? 2 : j3 - 1;
        const int nuw = j3 * G::NU_SLOT;               // nu row j-3
        const int nuA = j3p1 * G::NU_SLOT;             // nu row j-5
        const int nuB = j3p2 * G::NU_SLOT;             // nu row j-4
        const int eqw = j3 * G::EQ_SLOT;               // equilibrium row j-3
        const int eqc = j3p2 * G::EQ_SLOT;             // equilibrium row j-4

        // ---- phase A: moments of row j-2 (source rows j .. j+2); site terms and
        //      equilibrium weights of row j-3 (moments complete since the last phase A)
        if (comp) {
#pragma unroll
            for (int k = 0; k < COLS; ++k)
                moments_to(stp2, stp1, st0, g, c + 32 * k + HX, momA + g * RW + c + 32 * k + 2);
        } else if (site) {
            if (j >= 1) {
                C inv;
                const C rho = site_terms(momB + c + 2, c + 1, inv);
                const int mj = momB + N * RW + c + 2;
                C jx = C(0), jy = C(0);
#pragma unroll
                for (int t = 0; t < N; ++t) {
                    jx += mom[mj + t * RW];
                    jy += mom[mj + N * RW + t * RW];
                }
                C e[Q];
                eq_weights(jx * inv, jy * inv, e);
#pragma unroll
                for (int i = 0; i < Q; ++i) eqr[eqw + i * W + c] = e[i];
                const int r = j - 3;
                if (r >= 0 && r < Hc && x0 + c < p.nx && (!(rho > C(0)) || !isfinite(rho)))
                    atomicOr(p.status, STATUS_NONFINITE);
            }
        } else {
            if (lane < 4 * N) {
                const int hc = lane / N, s = lane - hc * N;
                const int cc = hc < 2 ? hc : W + hc;     // moment-ring column of the halo site
                moments_to(stp2, stp1, st0, s, cc - 2 + HX, momA + s * RW + cc);
            }
            // halo site terms of row j-3 on two lanes (the last two when they are free)
            const int hl = (4 * N + 2 <= 32) ? 4 * N : 0;
            if (j >= 1 && (lane == hl || lane == hl + 1)) {
                C inv;
                const int vc = lane == hl ? 0 : W + 1;
                site_terms(momB + vc + 1, vc, inv);
            }
        }
        __syncthreads();
        if (*abort_flag) break;
        if (tid == G::PRODUCER && j >= 3) {
            const int k = j - 3 + NS;  // reuse the stage of row j-3, last read by phase C of j-1
            if (k < nrows) {
                issue(k);
                issued = k + 1;
            }
        }

        // ---- phase B: nu of row j-3 (moment rows j-4 .. j-2)
        if (j >= 2) {
            if (comp) {
#pragma unroll
                for (int k = 0; k < COLS; ++k) {
                    const int o = g * RW + c + 32 * k + 2;
                    nur[nuw + g * VW + c + 32 * k + 1] =
                        nu_of(momC + o, momB + o, momA + o, momB + c + 32 * k + 2, c + 32 * k + 1, g,
                              chi_row, th_m, logc, minv1, has_log);
                }
            } else if (!site && lane < 2 * N) {
                const int hv = lane / N, s = lane - hv * N;
                const int vc = hv == 0 ? 0 : W + 1;
                const int o = s * RW + vc + 1;
                C chi_s[N];
#pragma unroll
                for (int u = 0; u < N; ++u) chi_s[u] = p.chi[s * N + u];
                nur[nuw + s * VW + vc] = nu_of(momC + o, momB + o, momA + o, momB + vc + 1, vc, s, chi_s,
                                               p.th_m[s], p.logc[s], p.m_inv_m1[s],
                                               (p.log_mask >> s) & 1u);
            }
        }
        __syncthreads();

        // ---- phase C: collide row j-4 (source rows j-2 .. j, nu rows j-5 .. j-3)
        if (comp && j >= 4) {
            T* line = fout + line_off(p, g, y0 + j - 4, 0);
            float* rline = nullptr;
            if constexpr (G::SHIFTED) rline = rho_line(fout, p, g, y0 + j - 4);
#pragma unroll
            for (int k = 0; k < COLS; ++k)
                collide_col(32 * k, st0, stm1, stm2, momC, eqc, nuA, nuB, nuw, line, rline, ghost[k]);
        }
        sj = (sj + 1 == NS) ? 0 : sj + 1;
        j3 = j3p1;
    }

    if (*abort_flag) {
        if (tid == 0) atomicOr(p.status, STATUS_TIMEOUT);
        // drain the copies still in flight before the shared memory is released
        if (tid == G::PRODUCER)
            for (int k = j + 2; k < issued; ++k) wait_row(k);
    }
}

}  // namespace mclb
