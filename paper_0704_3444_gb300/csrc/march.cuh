// march.cuh -- one launch per timestep by column marching: every lane owns one column
// of a strip and carries its components down a segment of rows in registers.
//
// The step at a site needs (Sec. 3, Eqs. ssLB, ff1-ff3, chemicalpotential, definef):
// the pulled populations f^s_i(x - v_i) for its moments, rho^s on the 8 neighbours
// for the kappa Laplacian in nu^s, and nu^s on the 8 neighbours for the force.  A
// lane at column x marching down rows keeps the vertical neighbours of those fields
// in registers and gets the horizontal ones from lanes x -+ 1 by warp shuffles.
// Iteration k of the march handles
//   - the moments and site terms of the lead row m = y0 - 2 + k,
//   - nu^s of row m - 1 (rho^s of rows m - 2 .. m now known),
//   - the collision of row m - 2 (nu^s of rows m - 3 .. m - 1 now known).
// A warp of 32 lanes covers 32 columns: nu is valid on lanes 1..30 and the collision
// on lanes 2..29, so a warp writes 28 columns and neighbouring warps overlap by 4.
//
// Shared memory holds the pulled distributions: a ring of NS stages, stage k holding
// everything that row m = y0 - 2 + k pulls, i.e. for each velocity i the line of source
// row m - v_i,y (all N components, columns [x0 - hx, x0 - hx + WI)).  A producer warp
// fills each stage with nine TMA box copies (one per velocity, cp.async.bulk.tensor) on
// one mbarrier, plus an L2 prefetch one row ahead; in the 16-bit formats it also brings
// the FP32 reference-density line of row m + 1 into a ring that holds those of the rows
// the live stages pull from.  A stage is read by the moments of row m and two iterations
// later by the collision of row m; each compute warp then arrives on the stage's "empty"
// mbarrier and the producer refills it.  So each stored value is loaded from HBM once per
// step (plus the strip and segment halos), and only the 16-bit box stores synchronise the
// compute warps once per row.  Every mbarrier wait is bounded; a timeout sets
// STATUS_TIMEOUT, the copies in flight are drained and the CTA returns.
//
// The kernel writes columns [0, nx) only; k_ghosts (ghosts.cuh) then refreshes the
// periodic ghost columns.  (Writing the few ghost copies from inside the march, with plain stores next
// to the bulk tensor stores of the same lines, halved the speed of the CTAs that did it,
// and the step waits for the slowest CTA.)
#pragma once

#include <type_traits>

#include "tma.cuh"

namespace mclb {

constexpr int MARCH_HDR = 256;   // full, empty and row mbarriers + abort flag
constexpr int MARCH_MAX_NS = 8;
constexpr int MARCH_OUT = 28;    // columns written per warp
constexpr int MARCH_PF = 1;      // L2 prefetch distance in rows (2 and more thrash L2)

// vy of velocity i from a runtime index (bits 2i..2i+1 hold vy + 1)
__device__ __forceinline__ int vy_rt(int i) { return (int)((0x2865u >> (2 * i)) & 3u) - 1; }

template <typename T, int N, int NW, int NS>
struct MarchGeomT {
    using C = typename Storage<T>::C;
    static constexpr bool SHIFTED = Storage<T>::shifted;
    static constexpr int NWC = NW;                                // column groups
    static constexpr int NCW = NW;                                // compute warps
    static constexpr int STAGES = NS;
    static constexpr int HX = (16 / (int)sizeof(T)) < 4 ? 4 : 16 / (int)sizeof(T);
    static constexpr int WOUT = MARCH_OUT * NW;                   // columns written per CTA
    static constexpr int AL = 16 / (int)sizeof(T);                // elements per 16 bytes
    static constexpr int WI = (WOUT + 3 + HX + AL - 1) / AL * AL; // staged columns
    static constexpr int THREADS = 32 * NCW + 32;                 // + producer warp
    static constexpr size_t VBYTES = round_up_sz((size_t)N * WI * sizeof(T), 128);
    static constexpr size_t STAGE_BYTES = Q * VBYTES;
    static constexpr uint32_t TXV = (uint32_t)(Q * (size_t)N * WI * sizeof(T));
    // 16-bit formats: the FP32 reference-density line of every source row is loaded once
    // into a ring of NS + 2 lines (a stage of row m reads rows m - 1 .. m + 1, and the
    // collision reads them again two iterations later)
    static constexpr int NR = SHIFTED ? NS + 2 : 0;
    static constexpr size_t RBYTES = SHIFTED ? round_up_sz((size_t)N * WI * sizeof(float), 128) : 0;
    static constexpr uint32_t TXR = SHIFTED ? (uint32_t)((size_t)N * WI * sizeof(float)) : 0u;
    // FP32/FP64: each compute warp stages its 28 output columns of the 9 N lines in shared
    // memory and writes them with one TMA box per row (28 columns are 16-byte multiples)
    static constexpr bool TMA_STORE = !SHIFTED && (MARCH_OUT * sizeof(T)) % 16 == 0;
    static constexpr size_t OBYTES = TMA_STORE ? round_up_sz((size_t)N * Q * MARCH_OUT * sizeof(T), 128) : 0;
    // 16-bit formats (28 columns are not a 16-byte multiple): the compute warps fill a CTA
    // staging area (deviations and FP32 reference densities of the WOUT columns, NB
    // buffers) and one thread writes it with two TMA boxes per row
    static constexpr bool CTA_STORE = SHIFTED && (WOUT * sizeof(T)) % 16 == 0;
    static constexpr size_t CDEV = CTA_STORE ? round_up_sz((size_t)N * Q * WOUT * sizeof(T), 128) : 0;
    static constexpr size_t CBUF = CTA_STORE ? CDEV + round_up_sz((size_t)N * WOUT * sizeof(float), 128) : 0;
    static constexpr size_t BASE = MARCH_HDR + NS * STAGE_BYTES + NR * RBYTES + NCW * OBYTES;
    // one staging buffer instead of two where that alone lets a third CTA share the SM
    // (the warps then wait, before refilling it, until the previous row's box has been
    // read out of it)
    static constexpr int NB = (CTA_STORE && 3 * (BASE + 2 * CBUF + 1024) > 228 * 1024 &&
                               3 * (BASE + CBUF + 1024) <= 228 * 1024) ? 1 : 2;
    static constexpr size_t SMEM = BASE + NB * CBUF;
    static constexpr bool FITS = SMEM <= 227 * 1024 && WI <= 256;
    static constexpr int MIN_CTAS = (3 * (SMEM + 1024) <= 228 * 1024) ? 3
                                    : (2 * (SMEM + 1024) <= 228 * 1024) ? 2 : 1;
    // registers per thread that let MIN_CTAS CTAs share the register file: each of the 4
    // SM sub-partitions holds 16K registers and its share of the warps (multiple of 8)
    static constexpr int WARPS_SP = (MIN_CTAS * (THREADS / 32) + 3) / 4;
    static constexpr int MAXREG_RAW = 16384 / (32 * WARPS_SP) / 8 * 8;
    static constexpr int MAXREG = MAXREG_RAW > 255 ? 255 : MAXREG_RAW;
};

// Strip width and ring depth per storage type and N: the first of (4 column groups,
// 5 stages), (4, 4) that lets three CTAs share an SM (three stages per CTA leave too few
// bytes in flight), else the first of (4, 5), (4, 4), (2, 5), (2, 4) that lets two CTAs
// share an SM, else the first that fits one CTA.  A third CTA hides more of the
// per-row latency: 2048^2 x 5 BF16 64.7k -> 72.1k and 8192 x 2048 x 3 FP32 73.6k ->
// 81.6k MLUPS x N.
template <typename T, int N>
struct MarchPick {
    using A = MarchGeomT<T, N, 4, 5>;
    using B = MarchGeomT<T, N, 4, 4>;
    using D = MarchGeomT<T, N, 2, 5>;
    using E = MarchGeomT<T, N, 2, 4>;
    static constexpr bool A3 = A::FITS && A::MIN_CTAS >= 3;
    static constexpr bool B3 = B::FITS && B::MIN_CTAS >= 3;
    static constexpr bool A2 = A::FITS && A::MIN_CTAS >= 2;
    static constexpr bool B2 = B::FITS && B::MIN_CTAS >= 2;
    static constexpr bool D2 = D::FITS && D::MIN_CTAS >= 2;
    static constexpr bool E2 = E::FITS && E::MIN_CTAS >= 2;
    static constexpr int NW = A3 ? 4 : B3 ? 4 : A2 ? 4 : B2 ? 4 : D2 ? 2 : E2 ? 2
                              : A::FITS ? 4 : B::FITS ? 4 : D::FITS ? 2 : 2;
    static constexpr int NS = A3 ? 5 : B3 ? 4 : A2 ? 5 : B2 ? 4 : D2 ? 5 : E2 ? 4
                              : A::FITS ? 5 : B::FITS ? 4 : D::FITS ? 5 : 4;
    using G = MarchGeomT<T, N, NW, NS>;
};

template <typename T, int N>
using MarchGeom = typename MarchPick<T, N>::G;

// The narrow alternative the batch's autotuner may pick: two compute warps (56-column
// strips) with the same ring depth, for groups of narrow instances whose last strip would
// leave many of a wide strip's lanes idle.  Only where the pick above has four warps.
template <typename T, int N>
using MarchNarrow = MarchGeomT<T, N, 2, MarchPick<T, N>::NS>;
template <typename T, int N>
constexpr bool has_narrow() { return MarchPick<T, N>::NW == 4 && MarchNarrow<T, N>::FITS; }


// The march of one CTA over the strip starting at column x0 and the segment of H rows
// starting at row y0 (tmap/tmapr: load views of the input buffer; tmapw/tmapwr: store
// views of fout; p may live in parameter or shared memory; G: the geometry).
template <typename T, int N, typename G = MarchGeom<T, N>, bool GD = false>
__device__ __forceinline__ void march_cta(const CUtensorMap* tmap, const CUtensorMap* tmapr,
                                          const CUtensorMap* tmapw, const CUtensorMap* tmapwr,
                                          T* __restrict__ fout,
                                          const StepParams<typename Storage<T>::C>& p,
                                          const int x0, const int y0, const int H,
                                          unsigned char* smem)
{
    using C = typename Storage<T>::C;
    constexpr int NS = G::STAGES, WI = G::WI, NCW = G::NCW;
    const int Hc = min(H, p.ny - y0);
    const int nk = Hc + 4;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // rows whose density the status word checks: with walls, the three rows next to each
    // wall are written here with periodic neighbours and then rewritten by the wall-aware
    // staged launches, so only those launches check them
    const int ychk0 = p.walls ? max(y0, 3) : y0;
    const int ychk1 = p.walls ? min(y0 + Hc, p.ny - 3) : y0 + Hc;

    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    uint64_t* empty = full + MARCH_MAX_NS;
    uint64_t* rowbar = empty + MARCH_MAX_NS;   // compute warps, once per collided row
    uint64_t* sfree = rowbar + 1;              // single staging buffer read out (NB = 1)
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + 24 * MARCH_MAX_NS);
    unsigned char* stages = smem + MARCH_HDR;
    unsigned char* rring = stages + NS * G::STAGE_BYTES;   // 16-bit formats: R lines
    unsigned char* obufs = rring + G::NR * G::RBYTES;
    constexpr int NR1 = G::NR > 0 ? G::NR : 1;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NCW);
        }
        mbar_init(rowbar, NCW);
        mbar_init(sfree, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();

    if (warp == NCW) {
        // ---- producer warp: stage k (lead row y0 - 2 + k) holds, for each velocity i, the
        // line of source row m - v_i,y; it reuses the slot of stage k - NS once all
        // compute warps have released that one
        auto grow = [&](int r) {
            r %= p.ny;
            return r + (r < 0 ? p.ny : 0);
        };
        int issued = 0;
        // (test hook: with p.withhold no copy is issued, so that every compute warp's first
        // bounded wait runs out and the CTA takes the timeout path)
        for (int k = 0; k < (p.withhold ? 0 : nk); ++k) {
            const int slot = k % NS;
            if (k >= NS) {
                bool ok = true;
                if (lane == 0) ok = mbar_wait(&empty[slot], ((k / NS) - 1) & 1);
                if (!__shfl_sync(0xffffffffu, ok, 0)) {
                    *abort_flag = 1;
                    break;
                }
            }
            if (*abort_flag) break;
            const int m = y0 - 2 + k;
            unsigned char* st = stages + (size_t)slot * G::STAGE_BYTES;
            // the first stage also brings the R lines of rows m - 1 and m; every stage brings
            // that of row m + 1, into ring slot (k + 2) mod NR (ring index k + j holds row
            // m - 1 + j)
            if (lane == 0)
                mbar_arrive_expect_tx(&full[slot], G::TXV + (k == 0 ? 3u : 1u) * G::TXR);
            __syncwarp();
            if (lane < Q) {
                tma_load_row(st + lane * G::VBYTES, tmap, &full[slot], x0, grow(m - vy_rt(lane)), lane);
            } else if (G::SHIFTED && lane < Q + 3 && (k == 0 || lane == Q + 2)) {
                const int j = lane - Q;
                tma_load_rline(rring + (size_t)((k + j) % NR1) * G::RBYTES, tmapr, &full[slot], x0,
                               grow(m - 1 + j));
            } else if (lane >= 16 && lane < 16 + Q && k + MARCH_PF < nk) {
                tma_prefetch_row(tmap, x0, grow(m + MARCH_PF - vy_rt(lane - 16)), lane - 16);
            }
            issued = k + 1;
        }
        __syncthreads();
        if (*abort_flag && lane == 0) {
            atomicOr(p.status, STATUS_TIMEOUT);
            // the copies still in flight land before the shared memory is released
            for (int k = max(0, issued - NS); k < issued; ++k) mbar_wait(&full[k % NS], (k / NS) & 1);
        }
        return;
    }

    // ---- compute warps: warp cg covers columns x0 - 2 + 28 cg .. x0 + 29 + 28 cg
    const int cg = warp;
    const int X = x0 - 2 + MARCH_OUT * cg + lane;         // this lane's column
    const int col = G::HX - 2 + MARCH_OUT * cg + lane;    // its staged column
    const bool out_lane = lane >= 2 && lane < 30 && X < p.nx;
    [[maybe_unused]] T* obuf = reinterpret_cast<T*>(obufs + warp * G::OBYTES);
    [[maybe_unused]] unsigned char* cbufs = obufs + G::NCW * G::OBYTES;
    [[maybe_unused]] const int ocol = MARCH_OUT * cg + lane - 2;   // column within the CTA's WOUT

    // R lines of rows m - 1, m, m + 1 for the stage of iteration kk (16-bit formats), as
    // offsets in floats from the ring
    const float* rbase = reinterpret_cast<const float*>(rring) + col;
    struct RLines { int o[3]; };
    auto rlines = [&](int kk) {
        RLines L;
#pragma unroll
        for (int j = 0; j < 3; ++j) L.o[j] = ((kk + j) % NR1) * (int)(G::RBYTES / sizeof(float));
        return L;
    };
    // pulled value of velocity i (compile-time) for component s from a stage
    auto pulled = [&](const unsigned char* st, const RLines& L, int i, int s) -> C {
        const T* line = reinterpret_cast<const T*>(st + i * G::VBYTES) + s * WI;
        C v = to_c<T>(line[col - vx(i)]);
        if constexpr (G::SHIFTED) v = fma(wq<C>(i), C(rbase[L.o[1 - vy(i)] + s * WI - vx(i)]), v);
        return v;
    };

    // FP32 storage collides two components at a time with the packed pair instructions
    constexpr bool PAIRS = std::is_same<T, float>::value && N >= 2;
    const C theta = p.theta, kappa6 = C(6) * p.kappa;
    const C c9 = C(1.0 / 9.0), c36 = C(1.0 / 36.0), c59 = C(5.0 / 9.0);

    // The march over rows.  State carried from row to row
    // (m = lead row of the iteration about to start), per component:
    //   Q1 = L(m-1) - 6 kappa (B(m-2) + Cc(m-1)),  Q0 = -6 kappa B(m-1)   (partial nu)
    //   GX = D(m-2)/9 + D(m-3)/36,  Dp = D(m-2),  T2 = T(m-3),  T1 = T(m-2)
    //   R/X/Y2, R/X/Y1 = rho^s, j^s of rows m-2, m-1;  and u of rows m-2, m-1
    // with B = rho/9 + A/36, Cc = A/9 - 5 rho/9 (A = rho(x-1) + rho(x+1)), so that
    // 6 sum_i w_i (rho_i - rho_0) at row r is 6 (B(r-1) + B(r+1) + Cc(r)); and with
    // D = nu(x+1) - nu(x-1), T = nu/9 + (nu(x+1) + nu(x-1))/36, so that the force gradient
    // 3 sum_i w_i v_i nu(x + v_i) at row r is 3 (D(r)/9 + (D(r-1) + D(r+1))/36,
    // T(r+1) - T(r-1)).
    auto march = [&]() {
        C Q1[N], Q0[N], GX[N], Dp[N], T2[N], T1[N];
        C R2[N], X2[N], Y2[N], R1[N], X1[N], Y1[N];
        C ux2 = C(0), uy2 = C(0), ux1 = C(0), uy1 = C(0);
        // GD (the Gibbs-Duhem total force): the same D and T sums of the total density for
        // rows m - 1, m - 2, m - 3, and the total density of rows m - 1, m - 2
        [[maybe_unused]] C Dr1 = C(0), Dr2 = C(0), Dr3 = C(0), Tr1 = C(0), Tr3 = C(0), Tr2 = C(0);
        [[maybe_unused]] C it1 = C(0), it2 = C(0);   // 1 / rho of rows m - 1, m - 2
#pragma unroll
        for (int c = 0; c < N; ++c) {
            Q1[c] = Q0[c] = GX[c] = Dp[c] = T2[c] = T1[c] = C(0);
            R2[c] = X2[c] = Y2[c] = R1[c] = X1[c] = Y1[c] = C(0);
        }

        for (int k = 0; k < nk; ++k) {
            const int m = y0 - 2 + k;
            const int slot = k % NS;
            const unsigned char* st = stages + (size_t)slot * G::STAGE_BYTES;
            const bool ok = mbar_wait(&full[slot], (k / NS) & 1);
            if (__any_sync(0xffffffffu, !ok)) {
                *abort_flag = 1;
                break;
            }

            // ---- moments of row m
            C R0[N], X0[N], Y0[N];
            C jxp = C(0), jyp = C(0);
            [[maybe_unused]] const RLines Lm = rlines(k);
#pragma unroll
            for (int c = 0; c < N; ++c) {
                C v[Q];
#pragma unroll
                for (int i = 0; i < Q; ++i) v[i] = pulled(st, Lm, i, c);
                const C a = v[5] - v[7], b = v[6] - v[8];
                R0[c] = ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7])) + v[8];
                X0[c] = (v[1] - v[3]) + (a - b);
                Y0[c] = (v[2] - v[4]) + (a + b);
                jxp += X0[c];
                jyp += Y0[c];
            }

            // ---- site terms of row m
            C rho = C(0);
#pragma unroll
            for (int t = 0; t < N; ++t) rho += R0[t];
            const C inv = C(1) / rho;
            const C ux0 = jxp * inv, uy0 = jyp * inv;
            if (out_lane && m >= ychk0 && m < ychk1 && (!(rho > C(0)) || !isfinite(rho)))
                atomicOr(p.status, STATUS_NONFINITE);
            const C lnr = dev_log(rho);
            C acc[N];
            C sm = C(0), quad = C(0);
#pragma unroll
            for (int t = 0; t < N; ++t) {
                C a = C(0);
#pragma unroll
                for (int u = 0; u < N; ++u) a += p.chi[t * N + u] * R0[u];
                acc[t] = a;
                sm += R0[t] * p.inv_m[t];
                quad += R0[t] * a;
            }
            const C Gs = -theta * (sm * inv + C(0.5) * quad * inv * inv);
            [[maybe_unused]] C Drn = C(0), Trn = C(0);
            if constexpr (GD) {
                const C rl = __shfl_up_sync(0xffffffffu, rho, 1);
                const C rr = __shfl_down_sync(0xffffffffu, rho, 1);
                Drn = rr - rl;
                Trn = rho * c9 + (rr + rl) * c36;
            }

            // ---- nu of row m - 1, partial nu of rows m and m + 1
            C Dn[N], Tn[N];
#pragma unroll
            for (int s = 0; s < N; ++s) {
                const int c = s;
                C logs = -p.th_m[s] * lnr;
                if ((p.log_mask >> s) & 1u) {
                    const C fl = p.log_floor * rho;
                    logs += p.logc[s] * dev_log(R0[c] > fl ? R0[c] : fl);
                }
                const C L0 = logs + theta * (p.m_inv_m1[s] + acc[s] * inv) + Gs;
                const C A = __shfl_up_sync(0xffffffffu, R0[c], 1) + __shfl_down_sync(0xffffffffu, R0[c], 1);
                const C B0 = R0[c] * c9 + A * c36;
                const C C0 = A * c9 - c59 * R0[c];
                const C nu = Q1[c] - kappa6 * B0;
                Q1[c] = Q0[c] + L0 - kappa6 * C0;
                Q0[c] = -kappa6 * B0;
                const C nl = __shfl_up_sync(0xffffffffu, nu, 1);
                const C nr = __shfl_down_sync(0xffffffffu, nu, 1);
                Dn[c] = nr - nl;
                Tn[c] = nu * c9 + (nr + nl) * c36;
            }

            // ---- collision of row r = m - 2 (stage of iteration k - 2)
            if (k >= 4) {
                const unsigned char* sc = stages + (size_t)((k - 2) % NS) * G::STAGE_BYTES;
                const int r = m - 2;
                if constexpr (G::TMA_STORE) {
                    // the previous row's box has been read out of the staging buffer
                    if (lane == 0) bulk_wait_read();
                    __syncwarp();
                }
                [[maybe_unused]] const RLines Lc = rlines(k - 2);
                if constexpr (G::CTA_STORE && G::NB == 1) {
                    // the box stored one row earlier has left the staging buffer
                    if (k >= 5) {
                        if (threadIdx.x == 0) {
                            bulk_wait_read();
                            mbar_arrive(sfree);
                        }
                        if (__any_sync(0xffffffffu, !mbar_wait(sfree, (k - 5) & 1))) {
                            *abort_flag = 1;
                            break;
                        }
                    }
                }
                // post-collision values of component s to the store path of this format
                auto store_out = [&](const int s, C (&out)[Q]) {
                    const int c = s;
                    if constexpr (G::TMA_STORE) {
                        if (lane >= 2 && lane < 30) {
#pragma unroll
                            for (int i = 0; i < Q; ++i) obuf[(s * Q + i) * MARCH_OUT + lane - 2] = T(out[i]);
                        }
                    } else if constexpr (G::CTA_STORE) {
                        if (lane >= 2 && lane < 30) {
                            // deviations from w_i M rounded to storage, and the compensated
                            // reference density R = M - sum_i d_i: the stored site mass is
                            // then rho^s to FP32 rounding
                            unsigned char* cb = cbufs + (G::NB == 2 ? ((k - 4) & 1) : 0) * G::CBUF;
                            T* dv = reinterpret_cast<T*>(cb);
                            float* rv = reinterpret_cast<float*>(cb + G::CDEV);
                            const C M = R2[c];
                            C dsum = C(0);
#pragma unroll
                            for (int i = 0; i < Q; ++i) {
                                const T d = Storage<T>::pack(out[i]);
                                dsum = add_wide<T>(dsum, d);
                                dv[(s * Q + i) * G::WOUT + ocol] = d;
                            }
                            rv[s * G::WOUT + ocol] = float(M - dsum);
                        }
                    } else if (out_lane) {
                        T* line = fout + line_off(p, s, r, 0) + G::HX;
                        if constexpr (G::SHIFTED) {
                            // out_i is the deviation f*_i - w_i M already (see below): rounded
                            // once, stored, and summed for the compensated reference density
                            const C M = R2[c];
                            C dsum = C(0);
#pragma unroll
                            for (int i = 0; i < Q; ++i) {
                                const T d = Storage<T>::pack(out[i]);
                                dsum = add_wide<T>(dsum, d);
                                line[i * p.pitch + X] = d;
                            }
                            rho_line(fout, p, s, r)[G::HX + X] = float(M - dsum);
                        } else {
#pragma unroll
                            for (int i = 0; i < Q; ++i) Storage<T>::store(line + i * p.pitch + X, out[i]);
                        }
                    }
                };
                // acceleration a^s of row r (Eq. definef plus the body force)
                auto accel0 = [&](const int c, C& ax, C& ay) {
                    const C gx = GX[c] + Dn[c] * c36;
                    const C gy = Tn[c] - T2[c];
                    ax = -p.fcoef * (C(3) * gx) + p.gx;
                    ay = -p.fcoef * (C(3) * gy) + p.gy;
                };
                // GD: every component's a^s first, then the shift (A_c - A)/rho with A_c =
                // (1 - 1/2tau) (1/3) grad rho from the total-density sums of rows r - 1 .. r + 1
                // (gibbs_duhem_shift's terms, with the row's 1/rho and (1 - 1/2tau)/3 * 3
                // folded: no division per site)
                [[maybe_unused]] C axg[N], ayg[N];
                if constexpr (GD) {
                    C Ax = C(0), Ay = C(0);
#pragma unroll
                    for (int c = 0; c < N; ++c) {
                        accel0(c, axg[c], ayg[c]);
                        Ax += R2[c] * (axg[c] - p.gx);
                        Ay += R2[c] * (ayg[c] - p.gy);
                    }
                    const C dx = (p.fcoef * (Dr2 * c9 + (Dr3 + Dr1) * c36) - Ax) * it2;
                    const C dy = (p.fcoef * (Tr1 - Tr3) - Ay) * it2;
#pragma unroll
                    for (int c = 0; c < N; ++c) {
                        axg[c] += dx;
                        ayg[c] += dy;
                    }
                }
                auto accel = [&](const int c, C& ax, C& ay) {
                    if constexpr (GD) {
                        ax = axg[c];
                        ay = ayg[c];
                    } else {
                        accel0(c, ax, ay);
                    }
                };
                // 16-bit formats: out_i is already the deviation f*_i - w_i M, with M the
                // site's pre-collision mass rho^s, which the collision conserves
                if constexpr (PAIRS) {
                    // FP32: components (c, c + 1) together with the packed pair instructions
                    float2 e2[Q];
                    eq_weights2(ux2, uy2, e2);
#pragma unroll
                    for (int c = 0; c + 1 < N; c += 2) {
                        float2 f2[Q], out2[Q];
#pragma unroll
                        for (int i = 0; i < Q; ++i)
                            f2[i] = make_float2(pulled(sc, Lc, i, c), pulled(sc, Lc, i, c + 1));
                        C ax0, ay0, ax1, ay1, jx0, jy0, jx1, jy1;
                        accel(c, ax0, ay0);
                        accel(c + 1, ax1, ay1);
                        forcing_momentum(p, R2[c], X2[c], Y2[c], ux2, uy2, jx0, jy0);
                        forcing_momentum(p, R2[c + 1], X2[c + 1], Y2[c + 1], ux2, uy2, jx1, jy1);
                        const float2 r2 = make_float2(R2[c], R2[c + 1]);
                        collide2(p, f2, e2, r2, make_float2(jx0, jx1), make_float2(jy0, jy1),
                                 make_float2(ax0, ax1), make_float2(ay0, ay1), out2,
                                 G::SHIFTED ? r2 : pdup(0.0f));
                        C o0[Q], o1[Q];
#pragma unroll
                        for (int i = 0; i < Q; ++i) {
                            o0[i] = out2[i].x;
                            o1[i] = out2[i].y;
                        }
                        store_out(c, o0);
                        store_out(c + 1, o1);
                    }
                    if constexpr (N % 2 == 1) {
                        constexpr int c = N - 1;
                        C f[Q], e[Q], out[Q], ax, ay, fjx, fjy;
#pragma unroll
                        for (int i = 0; i < Q; ++i) {
                            f[i] = pulled(sc, Lc, i, c);
                            e[i] = e2[i].x;
                        }
                        accel(c, ax, ay);
                        forcing_momentum(p, R2[c], X2[c], Y2[c], ux2, uy2, fjx, fjy);
                        collide(p, f, e, R2[c], fjx, fjy, ax, ay, out, G::SHIFTED ? R2[c] : C(0));
                        store_out(c, out);
                    }
                } else {
                    C e[Q];
                    eq_weights(ux2, uy2, e);
#pragma unroll
                    for (int c = 0; c < N; ++c) {
                        C f[Q], out[Q], ax, ay, fjx, fjy;
#pragma unroll
                        for (int i = 0; i < Q; ++i) f[i] = pulled(sc, Lc, i, c);
                        accel(c, ax, ay);
                        forcing_momentum(p, R2[c], X2[c], Y2[c], ux2, uy2, fjx, fjy);
                        collide(p, f, e, R2[c], fjx, fjy, ax, ay, out, G::SHIFTED ? R2[c] : C(0));
                        store_out(c, out);
                    }
                }
            }
            if constexpr (G::TMA_STORE) {
                if (k >= 4) {
                    fence_async_smem();
                    __syncwarp();
                    // boxes that start at or past column nx are not issued (the view
                    // clips the others at nx)
                    if (lane == 0 && x0 + MARCH_OUT * cg < p.nx) {
                        tma_store_box(tmapw, obuf, x0 + MARCH_OUT * cg + G::HX, 0, m - 2, 0);
                        bulk_commit();
                    }
                }
            }
            if constexpr (G::CTA_STORE) {
                if (k >= 4) {
                    fence_async_smem();
                    // two buffers: the box issued one row earlier has been read out of the
                    // other buffer before any warp passes this barrier and refills that one
                    if (G::NB == 2 && threadIdx.x == 0) bulk_wait_read();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(rowbar);
                    if (__any_sync(0xffffffffu, !mbar_wait(rowbar, (k - 4) & 1))) {
                        *abort_flag = 1;
                        break;
                    }
                    if (threadIdx.x == 0) {
                        const unsigned char* cb = cbufs + (G::NB == 2 ? ((k - 4) & 1) : 0) * G::CBUF;
                        tma_store_box(tmapw, cb, x0 + G::HX, 0, m - 2, 0);
                        tma_store_box3(tmapwr, cb + G::CDEV, x0 + G::HX, m - 2, 0);
                        bulk_commit();
                    }
                }
            }
            if (k >= 2) {
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[(k - 2) % NS]);   // stage of row m - 2 done
            }
            // ---- advance the carried state by one row
#pragma unroll
            for (int c = 0; c < N; ++c) {
                GX[c] = Dn[c] * c9 + Dp[c] * c36;
                Dp[c] = Dn[c];
                T2[c] = T1[c];
                T1[c] = Tn[c];
                R2[c] = R1[c];
                X2[c] = X1[c];
                Y2[c] = Y1[c];
                R1[c] = R0[c];
                X1[c] = X0[c];
                Y1[c] = Y0[c];
            }
            ux2 = ux1;
            uy2 = uy1;
            ux1 = ux0;
            uy1 = uy0;
            if constexpr (GD) {
                Dr3 = Dr2;
                Dr2 = Dr1;
                Dr1 = Drn;
                Tr3 = Tr2;
                Tr2 = Tr1;
                Tr1 = Trn;
                it2 = it1;
                it1 = inv;
            }
        }
    };

    march();
    if constexpr (G::TMA_STORE) {
        if (lane == 0) bulk_wait_all();
    }
    if constexpr (G::CTA_STORE) {
        if (threadIdx.x == 0) bulk_wait_all();
    }
    __syncthreads();
}

template <typename T, int N, bool GD = false>
__global__ void __launch_bounds__(MarchGeom<T, N>::THREADS) __maxnreg__((MarchGeom<T, N>::MAXREG))
k_march(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ CUtensorMap tmapr,
        const __grid_constant__ CUtensorMap tmapw, const __grid_constant__ CUtensorMap tmapwr,
        T* __restrict__ fout, const __grid_constant__ StepParams<typename Storage<T>::C> p,
        const int H)
{
    extern __shared__ __align__(128) unsigned char smem[];
    march_cta<T, N, MarchGeom<T, N>, GD>(&tmap, &tmapr, &tmapw, &tmapwr, fout, p,
                                         blockIdx.x * MarchGeom<T, N>::WOUT, blockIdx.y * H, H,
                                         smem);
}

}  // namespace mclb
