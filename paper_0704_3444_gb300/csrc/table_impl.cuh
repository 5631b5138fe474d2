// table_impl.cuh -- host launchers for one storage type, dispatched on N at run time.
#pragma once

#include <algorithm>

#include "batch.cuh"
#include "ghosts.cuh"
#include "march.cuh"
#include "staged.cuh"

namespace mclb {

#define MCLB_DISPATCH_N(n, ...)                      \
    switch (n) {                                      \
        case 1: { constexpr int NN = 1; __VA_ARGS__ }       \
        case 2: { constexpr int NN = 2; __VA_ARGS__ }       \
        case 3: { constexpr int NN = 3; __VA_ARGS__ }       \
        case 4: { constexpr int NN = 4; __VA_ARGS__ }       \
        case 5: { constexpr int NN = 5; __VA_ARGS__ }       \
        case 6: { constexpr int NN = 6; __VA_ARGS__ }       \
        case 7: { constexpr int NN = 7; __VA_ARGS__ }       \
        case 8: { constexpr int NN = 8; __VA_ARGS__ }       \
        default: return cudaErrorInvalidValue;        \
    }

inline unsigned site_blocks(long long S) { return (unsigned)((S + SITE_THREADS - 1) / SITE_THREADS); }

template <typename T>
struct Launch {
    using C = typename Storage<T>::C;

    static cudaError_t init(const Problem& P, const Scratch& sc, const double* rho, const double* u,
                            void* f, cudaStream_t st)
    {
        const auto p = make_params<C>(P, sc.status);
        MCLB_DISPATCH_N(P.N, {
            k_init<T, NN><<<site_blocks(P.S), SITE_THREADS, 0, st>>>(rho, u, (T*)f, p);
            return cudaGetLastError();
        });
    }

    template <int N>
    static cudaError_t fields_n(const StepParams<C>& p, const Scratch& sc, const T* f,
                                cudaStream_t st)
    {
        k_density<T, N><<<site_blocks(p.S), SITE_THREADS, 0, st>>>(f, (C*)sc.rho_s, p);
        k_potential<C, N><<<site_blocks(p.S), SITE_THREADS, 0, st>>>((const C*)sc.rho_s,
                                                                      (C*)sc.nu, p);
        return cudaGetLastError();
    }

    static cudaError_t step_staged(const Problem& P, const Scratch& sc, const void* fin, void* fout,
                                   cudaStream_t st)
    {
        const auto p = make_params<C>(P, sc.status);
        MCLB_DISPATCH_N(P.N, {
            cudaError_t e = fields_n<NN>(p, sc, (const T*)fin, st);
            if (e != cudaSuccess) return e;
            k_collide<T, NN><<<site_blocks(P.S), SITE_THREADS, 0, st>>>(
                (const T*)fin, (T*)fout, (const C*)sc.nu, p);
            return cudaGetLastError();
        });
    }

    // Strips of WOUT columns, segments of H rows: one wave of CTAs, each segment as
    // tall as the resident CTAs allow (every segment re-reads 4 halo rows and spends 4
    // warm-up iterations), at least 8 rows.
    template <int N>
    static FusedPlan plan_n(const Problem& P, int sm_count)
    {
        using G = MarchGeom<T, N>;
        FusedPlan pl{};
        pl.ok = false;
        if (!G::FITS) return pl;
        if (cudaFuncSetAttribute(k_march<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)G::SMEM) != cudaSuccess)
            return pl;
        // the largest shared-memory carveout, so that the resident CTAs the occupancy
        // query counts (it assumes the largest) are the ones the launch gets
        if (cudaFuncSetAttribute(k_march<T, N>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess)
            return pl;
        int ctas = 0;  // resident CTAs per SM as the runtime computes them (smem, registers)
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ctas, k_march<T, N>, G::THREADS,
                                                          G::SMEM) != cudaSuccess || ctas < 1)
            return pl;
        pl.W = G::WOUT;
        pl.box_w = G::WI;
        pl.out_w = G::TMA_STORE ? MARCH_OUT : (G::CTA_STORE ? G::WOUT : 0);
        pl.NS = G::STAGES;
        pl.smem = G::SMEM;
        pl.threads = G::THREADS;
        pl.nstrips = (P.nx + G::WOUT - 1) / G::WOUT;
        const int slots = ctas * std::max(1, sm_count);
        int nsegs = std::max(1, slots / pl.nstrips);
        nsegs = std::min(nsegs, std::max(1, P.ny / 8));
        pl.H = (P.ny + nsegs - 1) / nsegs;
        pl.nsegs = (P.ny + pl.H - 1) / pl.H;
        pl.ok = true;
        return pl;
    }

    static FusedPlan plan_fused(const Problem& P, int sm_count)
    {
        FusedPlan none{};
        none.ok = false;
        switch (P.N) {
            case 1: return plan_n<1>(P, sm_count);
            case 2: return plan_n<2>(P, sm_count);
            case 3: return plan_n<3>(P, sm_count);
            case 4: return plan_n<4>(P, sm_count);
            case 5: return plan_n<5>(P, sm_count);
            case 6: return plan_n<6>(P, sm_count);
            case 7: return plan_n<7>(P, sm_count);
            case 8: return plan_n<8>(P, sm_count);
            default: return none;
        }
    }

    static cudaError_t step_fused(const Problem& P, const Scratch& sc, const FusedPlan& pl,
                                  const CUtensorMap* tmap_in, const CUtensorMap* tmapr_in,
                                  const CUtensorMap* tmapw_out, const CUtensorMap* tmapwr_out,
                                  void* fout, cudaStream_t st)
    {
        const auto p = make_params<C>(P, sc.status);
        const dim3 grid(pl.nstrips, pl.nsegs);
        const CUtensorMap& tr = Storage<T>::shifted ? *tmapr_in : *tmap_in;
        const CUtensorMap& tw = pl.out_w > 0 ? *tmapw_out : *tmap_in;
        const CUtensorMap& twr = (pl.out_w > 0 && Storage<T>::shifted) ? *tmapwr_out : *tmap_in;
        MCLB_DISPATCH_N(P.N, {
            k_march<T, NN><<<grid, pl.threads, pl.smem, st>>>(*tmap_in, tr, tw, twr, (T*)fout, p, pl.H);
            const long long ghosts = (long long)NN * P.ny * (Q + (Storage<T>::shifted ? 1 : 0)) * 2 * P.hx;
            k_ghosts<T><<<(unsigned)((ghosts + 255) / 256), 256, 0, st>>>((T*)fout, p, NN);
            return cudaGetLastError();
        });
    }

    static cudaError_t moments(const Problem& P, const Scratch& sc, const void* f, double* rho,
                               double* U, double* mu, double* Pt, cudaStream_t st)
    {
        const auto p = make_params<C>(P, sc.status);
        MCLB_DISPATCH_N(P.N, {
            cudaError_t e = fields_n<NN>(p, sc, (const T*)f, st);
            if (e != cudaSuccess) return e;
            k_moments<T, NN><<<site_blocks(P.S), SITE_THREADS, 0, st>>>(
                (const T*)f, (const C*)sc.rho_s, (const C*)sc.nu, rho, U, mu, Pt, p);
            return cudaGetLastError();
        });
    }

    static cudaError_t conservation(const Problem& P, const Scratch& sc, const void* f, double* out,
                                    cudaStream_t st)
    {
        const auto p = make_params<C>(P, sc.status);
        MCLB_DISPATCH_N(P.N, {
            cudaError_t e = fields_n<NN>(p, sc, (const T*)f, st);
            if (e != cudaSuccess) return e;
            if (sc.partial_cap < (size_t)REDUCE_BLOCKS * (NN + 4)) return cudaErrorInvalidValue;
            k_conservation<T, NN><<<REDUCE_BLOCKS, SITE_THREADS, 0, st>>>(
                (const T*)f, (const C*)sc.rho_s, (const C*)sc.nu, sc.partial, p);
            k_reduce_partials<<<1, SITE_THREADS, 0, st>>>(sc.partial, REDUCE_BLOCKS, NN + 4, out);
            return cudaGetLastError();
        });
    }

    static cudaError_t compositions(const Problem& P, const Scratch& sc, const void* f, double* phi,
                                    double* bulk, double tol, cudaStream_t st)
    {
        const auto p = make_params<C>(P, sc.status);
        MCLB_DISPATCH_N(P.N, {
            k_density<T, NN><<<site_blocks(P.S), SITE_THREADS, 0, st>>>((const T*)f,
                                                                         (C*)sc.rho_s, p);
            k_compositions<T, NN><<<site_blocks(P.S), SITE_THREADS, 0, st>>>(
                (const C*)sc.rho_s, phi, bulk, tol, p);
            return cudaGetLastError();
        });
    }

    static cudaError_t get_state(const Problem& P, const Scratch& sc, const void* f, double* out,
                                 cudaStream_t st)
    {
        const auto p = make_params<C>(P, sc.status);
        MCLB_DISPATCH_N(P.N, {
            k_get_state<T, NN><<<site_blocks(P.S), SITE_THREADS, 0, st>>>((const T*)f, out, p);
            return cudaGetLastError();
        });
    }

    static cudaError_t set_state(const Problem& P, const Scratch& sc, const double* in, void* f,
                                 cudaStream_t st)
    {
        const auto p = make_params<C>(P, sc.status);
        MCLB_DISPATCH_N(P.N, {
            k_set_state<T, NN><<<site_blocks(P.S), SITE_THREADS, 0, st>>>(in, (T*)f, p);
            return cudaGetLastError();
        });
    }
};

template <typename T>
inline KernelTable make_table(CUtensorMapDataType tt)
{
    KernelTable t{};
    t.storage_bytes = sizeof(T);
    t.shifted = Storage<T>::shifted;
    t.tma_type = tt;
    t.hx = (int)std::max<size_t>(4, 16 / sizeof(T));
    t.plan_fused = &Launch<T>::plan_fused;
    t.init = &Launch<T>::init;
    t.step_fused = &Launch<T>::step_fused;
    t.step_staged = &Launch<T>::step_staged;
    t.moments = &Launch<T>::moments;
    t.conservation = &Launch<T>::conservation;
    t.compositions = &Launch<T>::compositions;
    t.get_state = &Launch<T>::get_state;
    t.set_state = &Launch<T>::set_state;
    t.batch_create = &batch_group_create<T>;
    t.batch_step = &batch_group_step<T>;
    t.batch_launches = &batch_group_launches<T>;
    t.batch_tune = &batch_group_tune<T>;
    t.batch_waves = &batch_group_waves<T>;
    t.batch_destroy = &batch_group_destroy<T>;
    return t;
}

}  // namespace mclb
