// table_impl.cuh -- host launchers for one storage type, dispatched on N at run time.
#pragma once

#include <algorithm>

#include "batch.cuh"
#include "cube.cuh"
#include "cube_march.cuh"
#include "ghosts.cuh"
#include "line3.cuh"
#include "march.cuh"
#include "mass.cuh"
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
                (const T*)fin, (T*)fout, (const C*)sc.rho_s, (const C*)sc.nu, p);
            return cudaGetLastError();
        });
    }

    // Strips of WOUT columns, segments of H rows: one wave of CTAs, each segment as
    // tall as the resident CTAs allow (every segment re-reads 4 halo rows and spends 4
    // warm-up iterations), at least 8 rows.
    template <int N, bool GD>
    static FusedPlan plan_k(const Problem& P, int sm_count)
    {
        using G = MarchGeom<T, N>;
        FusedPlan pl{};
        pl.ok = false;
        if (!G::FITS) return pl;
        if (cudaFuncSetAttribute(k_march<T, N, GD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)G::SMEM) != cudaSuccess)
            return pl;
        // the largest shared-memory carveout, so that the resident CTAs the occupancy
        // query counts (it assumes the largest) are the ones the launch gets
        if (cudaFuncSetAttribute(k_march<T, N, GD>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess)
            return pl;
        int ctas = 0;  // resident CTAs per SM as the runtime computes them (smem, registers)
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ctas, k_march<T, N, GD>, G::THREADS,
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

    // The Gibbs-Duhem force form has its own single-pass instance for FP64 and FP32 storage
    // and N <= 3 (the paper's polymer binary and ternary); elsewhere it runs staged.
    template <int N>
    static constexpr bool gd_single_pass()
    {
        return (std::is_same<T, float>::value || std::is_same<T, double>::value) && N <= 3;
    }
    template <int N>
    static FusedPlan plan_n(const Problem& P, int sm_count)
    {
        if (P.force_form == FORCE_GIBBS_DUHEM) {
            if constexpr (gd_single_pass<N>()) return plan_k<N, true>(P, sm_count);
            FusedPlan none{};
            none.ok = false;
            return none;
        }
        return plan_k<N, false>(P, sm_count);
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

    // Walls on the single pass.  A row's new state reaches three rows of the old one (the
    // pull of rho^s two rows away, which nu^s one row away needs), so rows 3 .. ny - 4 of
    // k_march, which treats y as periodic, are already those of the walled lattice.  The
    // wall-aware staged kernels then rewrite the three rows next to each wall, from the
    // bands of fields they need (rho^s on five rows, nu^s on four); ghosts included.
    template <int N>
    static cudaError_t wall_rows(StepParams<C> p, const Scratch& sc, const T* fin, T* fout,
                                 cudaStream_t st)
    {
        const auto band = [&](int rows) { return 2 * rows >= p.ny ? 0LL : (long long)rows * p.nx; };
        const auto blocks = [&]() { return site_blocks(p.band ? 2 * p.band : p.S); };
        p.band = band(5);
        k_density<T, N, true><<<blocks(), SITE_THREADS, 0, st>>>(fin, (C*)sc.rho_s, p);
        p.band = band(4);
        k_potential<C, N, true><<<blocks(), SITE_THREADS, 0, st>>>((const C*)sc.rho_s, (C*)sc.nu, p);
        p.band = band(3);
        k_collide<T, N, true><<<blocks(), SITE_THREADS, 0, st>>>(fin, fout, (const C*)sc.rho_s,
                                                            (const C*)sc.nu, p);
        return cudaGetLastError();
    }

    static cudaError_t step_fused(const Problem& P, const Scratch& sc, const FusedPlan& pl,
                                  const CUtensorMap* tmap_in, const CUtensorMap* tmapr_in,
                                  const CUtensorMap* tmapw_out, const CUtensorMap* tmapwr_out,
                                  const void* fin, void* fout, cudaStream_t st)
    {
        const auto p = make_params<C>(P, sc.status);
        const dim3 grid(pl.nstrips, pl.nsegs);
        const CUtensorMap& tr = Storage<T>::shifted ? *tmapr_in : *tmap_in;
        const CUtensorMap& tw = pl.out_w > 0 ? *tmapw_out : *tmap_in;
        const CUtensorMap& twr = (pl.out_w > 0 && Storage<T>::shifted) ? *tmapwr_out : *tmap_in;
        MCLB_DISPATCH_N(P.N, {
            bool launched = false;
            if constexpr (gd_single_pass<NN>()) {
                if (P.force_form == FORCE_GIBBS_DUHEM) {
                    k_march<T, NN, true><<<grid, pl.threads, pl.smem, st>>>(*tmap_in, tr, tw, twr,
                                                                          (T*)fout, p, pl.H);
                    launched = true;
                }
            }
            if (!launched)
                k_march<T, NN><<<grid, pl.threads, pl.smem, st>>>(*tmap_in, tr, tw, twr, (T*)fout, p, pl.H);
            const long long ghosts = (long long)NN * P.ny * (Q + (Storage<T>::shifted ? 1 : 0)) * 2 * P.hx;
            k_ghosts<T><<<(unsigned)((ghosts + 255) / 256), 256, 0, st>>>((T*)fout, p, NN);
            if (P.walls) return wall_rows<NN>(p, sc, (const T*)fin, (T*)fout, st);
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
        return conservation_rows(P, sc, f, 0, P.ny, out, st);
    }

    static cudaError_t conservation_rows(const Problem& P, const Scratch& sc, const void* f,
                                         int y0, int nrows, double* out, cudaStream_t st)
    {
        const auto p = make_params<C>(P, sc.status);
        const long long s0 = (long long)y0 * P.nx, s1 = (long long)(y0 + nrows) * P.nx;
        MCLB_DISPATCH_N(P.N, {
            cudaError_t e = fields_n<NN>(p, sc, (const T*)f, st);
            if (e != cudaSuccess) return e;
            if (sc.partial_cap < (size_t)REDUCE_BLOCKS * (NN + 4)) return cudaErrorInvalidValue;
            k_conservation<T, NN><<<REDUCE_BLOCKS, SITE_THREADS, 0, st>>>(
                (const T*)f, (const C*)sc.rho_s, (const C*)sc.nu, sc.partial, s0, s1, p);
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

    // Per-component mass compensation (mass.cuh), either lattice: record != 0 stores the
    // FP64 mass of every component of f in sc.mass_ref; record == 0 restores it.
    static cudaError_t mass(const Problem& P, const Scratch& sc, void* f, int record, cudaStream_t st)
    {
        MassView v{};
        v.q = P.lattice == LATTICE_D1Q3 ? 3 : (P.lattice == LATTICE_D3Q19 ? Q19 : Q);
        v.lines = (int)(P.S / P.nx) * v.q;   // (layers x) rows x velocities
        v.rlines = Storage<T>::shifted ? P.ny : 0;
        v.comp_stride = P.plane;
        v.pitch = P.pitch;
        v.rbytes = P.rbytes;
        v.S = P.S;
        v.first = P.hx;
        v.nx = P.nx;
        v.span = P.nx + 2 * P.hx;
        v.vec = (P.hx * sizeof(T)) % 16 == 0 && (P.pitch * sizeof(T)) % 16 == 0 &&
                P.rbytes % 16 == 0 && (P.hx * sizeof(float)) % 16 == 0 &&
                (P.pitch * sizeof(float)) % 16 == 0;
        k_mass_partials<T><<<dim3(MASS_BLOCKS, P.N), MASS_THREADS, 0, st>>>((const T*)f, v, sc.partial);
        const unsigned gx = record ? 1u : (unsigned)std::min(P.ny, 1024);
        k_mass_apply<T><<<dim3(gx, P.N), MASS_THREADS, 0, st>>>((T*)f, v, sc.partial, sc.mass_ref,
                                                                record);
        return cudaGetLastError();
    }
};

// Launchers of the D1Q3 kernels (line3.cuh) for one storage type.
template <typename T>
struct Line3Launch {
    using C = typename Storage<T>::C;
    static constexpr size_t SMEM_CAP = 227 * 1024 - sizeof(StepParams<C>) - 256;

    static int max_resident(int N)
    {
        const size_t per = (size_t)5 * N * sizeof(C);
        return (int)std::min<size_t>(SMEM_CAP / per, (size_t)L3_MAX_SITES);
    }

    static Line3Item<T> item(const Problem& P, const Scratch& sc, void* f0, void* f1)
    {
        Line3Item<T> it{};
        it.p = make_params<C>(P, sc.status);
        it.f[0] = (T*)f0;
        it.f[1] = (T*)f1;
        return it;
    }

    static cudaError_t prepare(const Problem& P, const Scratch& sc, void* const* f)
    {
        const Line3Item<T> it = item(P, sc, f[0], f[1]);
        return cudaMemcpy(sc.line_item, &it, sizeof(it), cudaMemcpyHostToDevice);
    }

    template <int N>
    static cudaError_t resident(const Line3Item<T>* items, int count, int nxmax, int parity,
                                int nsteps, cudaStream_t st)
    {
        static const cudaError_t attr = cudaFuncSetAttribute(
            k_line3_resident<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_CAP);
        if (attr != cudaSuccess) return attr;
        const size_t smem = Line3Smem<T, N>::bytes(nxmax);
        const int threads = (nxmax + 31) / 32 * 32;
        k_line3_resident<T, N><<<count, threads, smem, st>>>(items, parity, nsteps);
        return cudaGetLastError();
    }

    template <int N>
    static cudaError_t tile(const StepParams<C>& p, const void* fin, void* fout, cudaStream_t st)
    {
        const unsigned blocks = (unsigned)((p.nx + L3_TILE - 5) / (L3_TILE - 4));
        k_line3_tile<T, N><<<blocks, L3_TILE, 0, st>>>((const T*)fin, (T*)fout, p);
        return cudaGetLastError();
    }

    static unsigned line_blocks(int nx) { return (unsigned)((nx + SITE_THREADS - 1) / SITE_THREADS); }

    static cudaError_t init(const Problem& P, const Scratch& sc, const double* rho, const double* u,
                            void* f, cudaStream_t st)
    {
        const auto p = make_params<C>(P, sc.status);
        MCLB_DISPATCH_N(P.N, {
            k_line3_init<T, NN><<<line_blocks(P.nx), SITE_THREADS, 0, st>>>(rho, u, (T*)f, p);
            return cudaGetLastError();
        });
    }

    static cudaError_t step(const Problem& P, const Scratch& sc, void* const* f, int* cur,
                            long nsteps, cudaStream_t st)
    {
        const auto p = make_params<C>(P, sc.status);
        const bool res = P.nx <= max_resident(P.N);
        MCLB_DISPATCH_N(P.N, {
            while (nsteps > 0) {
                cudaError_t e;
                if (res) {
                    const int k = (int)std::min<long>(nsteps, L3_CHUNK);
                    e = resident<NN>((const Line3Item<T>*)sc.line_item, 1, P.nx, *cur, k, st);
                    nsteps -= k;
                } else {
                    e = tile<NN>(p, f[*cur], f[*cur ^ 1], st);
                    nsteps -= 1;
                }
                if (e != cudaSuccess) return e;
                *cur ^= 1;
            }
            return cudaSuccess;
        });
    }

    static cudaError_t moments(const Problem& P, const Scratch& sc, const void* f, double* rho,
                               double* U, double* mu, double* Pt, cudaStream_t st)
    {
        const auto p = make_params<C>(P, sc.status);
        MCLB_DISPATCH_N(P.N, {
            k_line3_moments<T, NN><<<line_blocks(P.nx), SITE_THREADS, 0, st>>>((const T*)f, rho, U,
                                                                               mu, Pt, p);
            return cudaGetLastError();
        });
    }

    static cudaError_t conservation(const Problem& P, const Scratch& sc, const void* f, double* out,
                                    cudaStream_t st)
    {
        const auto p = make_params<C>(P, sc.status);
        MCLB_DISPATCH_N(P.N, {
            if (sc.partial_cap < (size_t)REDUCE_BLOCKS * (NN + 4)) return cudaErrorInvalidValue;
            k_line3_conservation<T, NN><<<REDUCE_BLOCKS, SITE_THREADS, 0, st>>>((const T*)f,
                                                                                sc.partial, p);
            k_reduce_partials<<<1, SITE_THREADS, 0, st>>>(sc.partial, REDUCE_BLOCKS, NN + 4, out);
            return cudaGetLastError();
        });
    }

    static cudaError_t compositions(const Problem& P, const Scratch& sc, const void* f, double* phi,
                                    double* bulk, double tol, cudaStream_t st)
    {
        const auto p = make_params<C>(P, sc.status);
        MCLB_DISPATCH_N(P.N, {
            k_line3_compositions<T, NN><<<line_blocks(P.nx), SITE_THREADS, 0, st>>>(
                (const T*)f, phi, bulk, tol, p);
            return cudaGetLastError();
        });
    }

    static cudaError_t get_state(const Problem& P, const Scratch& sc, const void* f, double* out,
                                 cudaStream_t st)
    {
        const auto p = make_params<C>(P, sc.status);
        MCLB_DISPATCH_N(P.N, {
            k_line3_get_state<T, NN><<<line_blocks(P.nx), SITE_THREADS, 0, st>>>((const T*)f, out, p);
            return cudaGetLastError();
        });
    }

    static cudaError_t set_state(const Problem& P, const Scratch& sc, const double* in, void* f,
                                 cudaStream_t st)
    {
        const auto p = make_params<C>(P, sc.status);
        MCLB_DISPATCH_N(P.N, {
            k_line3_set_state<T, NN><<<line_blocks(P.nx), SITE_THREADS, 0, st>>>(in, (T*)f, p);
            return cudaGetLastError();
        });
    }

    // ---- batches of lines with one N
    struct Group {
        int N = 0;
        Line3Item<T>* d_items = nullptr;     // lines the resident kernel holds
        int nres = 0, nxmax = 1;
        std::vector<Line3Item<T>> longs;     // lines stepped with the tile kernel
        std::vector<size_t> long_bytes;
    };

    static void* batch_create(int N, int count, const Problem* probs, const Scratch* scs,
                              void* const* fa, void* const* fb, cudaStream_t st)
    {
        auto* g = new (std::nothrow) Group();
        if (!g) return nullptr;
        g->N = N;
        std::vector<Line3Item<T>> res;
        for (int k = 0; k < count; ++k) {
            const Line3Item<T> it = item(probs[k], scs[k], fa[k], fb[k]);
            if (probs[k].nx <= max_resident(N)) {
                res.push_back(it);
                g->nxmax = std::max(g->nxmax, probs[k].nx);
            } else {
                g->longs.push_back(it);
                g->long_bytes.push_back((size_t)N * 3 * probs[k].nx * sizeof(T));
            }
        }
        g->nres = (int)res.size();
        if (g->nres > 0) {
            if (cudaMalloc(&g->d_items, sizeof(Line3Item<T>) * res.size()) != cudaSuccess ||
                cudaMemcpyAsync(g->d_items, res.data(), sizeof(Line3Item<T>) * res.size(),
                                cudaMemcpyHostToDevice, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess) {
                cudaGetLastError();
                batch_destroy(g);
                return nullptr;
            }
        }
        return g;
    }

    static cudaError_t batch_step(void* gv, int parity, int nsteps, cudaStream_t st)
    {
        auto* g = static_cast<Group*>(gv);
        MCLB_DISPATCH_N(g->N, {
            if (g->nres > 0) {
                cudaError_t e = resident<NN>(g->d_items, g->nres, g->nxmax, parity, nsteps, st);
                if (e != cudaSuccess) return e;
            }
            for (size_t k = 0; k < g->longs.size(); ++k) {
                const Line3Item<T>& it = g->longs[k];
                int c = parity;
                for (int t = 0; t < nsteps; ++t, c ^= 1) {
                    cudaError_t e = tile<NN>(it.p, it.f[c], it.f[c ^ 1], st);
                    if (e != cudaSuccess) return e;
                }
                if (c == parity) {   // an even number of steps: the result goes to parity ^ 1
                    cudaError_t e = cudaMemcpyAsync(it.f[parity ^ 1], it.f[parity], g->long_bytes[k],
                                                    cudaMemcpyDeviceToDevice, st);
                    if (e != cudaSuccess) return e;
                }
            }
            return cudaSuccess;
        });
    }

    static int batch_launches(const void* gv)
    {
        auto* g = static_cast<const Group*>(gv);
        return (g->nres > 0 ? 1 : 0) + (int)g->longs.size();
    }

    static void batch_destroy(void* gv)
    {
        auto* g = static_cast<Group*>(gv);
        if (!g) return;
        if (g->d_items) cudaFree(g->d_items);
        delete g;
    }

    static const LatticeTable* table()
    {
        static const LatticeTable t = [] {
            LatticeTable x{};
            x.max_resident = &max_resident;
            x.item_bytes = sizeof(Line3Item<T>);
            x.prepare = &prepare;
            x.init = &init;
            x.step = &step;
            x.moments = &moments;
            x.conservation = &conservation;
            x.compositions = &compositions;
            x.get_state = &get_state;
            x.set_state = &set_state;
            x.batch_create = &batch_create;
            x.batch_step = &batch_step;
            x.batch_launches = &batch_launches;
            x.batch_destroy = &batch_destroy;
            return x;
        }();
        return &t;
    }
};

// Launchers of the D3Q19 kernels (cube.cuh) for one storage type: the staged step (three
// launches) and the diagnostics; no batches.
template <typename T>
struct Launch19 {
    using C = typename Storage<T>::C;

    static int max_resident(int) { return 0; }
    static cudaError_t prepare(const Problem&, const Scratch&, void* const*) { return cudaSuccess; }

    // The march (cube_march.cuh) after a density pass: tiles of M3_OUT_X x M3_OUT_Y, z
    // segments of H planes.  The CTAs are latency bound, so more of them than one wave
    // of resident slots helps; a segment of H planes costs about H + 4 plane iterations (four
    // warm-up planes) and the launch about waves x (H + 4) of them, so the segment count
    // that minimises that product is taken.  Not for N > M3_NMAX, the Gibbs-Duhem reading
    // (it needs grad rho on the density planes the next iteration overwrites) or
    // 19 S >= 2^31 (32-bit offsets).
    template <int N>
    static int plan_n(Problem& P, int sm_count)
    {
        if constexpr (N > M3_NMAX) {
            return 0;
        } else {
            if (P.force_form != 0 || 19.0 * (double)P.S >= 2147483647.0) return 0;
            const int smem = (int)m3_smem_bytes<C, N>();
            if (cudaFuncSetAttribute(k19_march<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     smem) != cudaSuccess)
                return -1;
            int ctas = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ctas, k19_march<T, N>, M3_THREADS,
                                                              smem) != cudaSuccess)
                return -1;
            if (ctas < 1) return 0;
            const long long tx = (P.nx + M3_OUT_X - 1) / M3_OUT_X, ty = (P.ny + M3_OUT_Y - 1) / M3_OUT_Y;
            const long long slots = (long long)ctas * std::max(1, sm_count);
            int best = 1;
            long long best_cost = -1;
            for (int nseg = 1; nseg <= std::max(1, P.nz / 4); ++nseg) {
                const long long H = (P.nz + nseg - 1) / nseg, segs = (P.nz + H - 1) / H;
                const long long waves = (tx * ty * segs + slots - 1) / slots;
                const long long cost = waves * (H + 4);
                if (best_cost < 0 || cost < best_cost) {
                    best_cost = cost;
                    best = nseg;
                }
            }
            const int H = (P.nz + best - 1) / best;
            P.grid3[0] = (int)tx;
            P.grid3[1] = (int)ty;
            P.grid3[2] = (P.nz + H - 1) / H;
            P.seg3 = H;
            return 1;
        }
    }
    static int plan(Problem& P, int sm_count)
    {
        switch (P.N) {
            case 1: return plan_n<1>(P, sm_count);
            case 2: return plan_n<2>(P, sm_count);
            case 3: return plan_n<3>(P, sm_count);
            case 4: return plan_n<4>(P, sm_count);
            default: return 0;
        }
    }

    static cudaError_t init(const Problem& P, const Scratch& sc, const double* rho, const double* u,
                            void* f, cudaStream_t st)
    {
        const auto p = make_params<C>(P, sc.status);
        MCLB_DISPATCH_N(P.N, {
            k19_init<T, NN><<<site_blocks(P.S), SITE_THREADS, 0, st>>>(rho, u, (T*)f, p);
            return cudaGetLastError();
        });
    }

    // density and potential fields of state f into the scratch
    template <int N>
    static cudaError_t fields_n(const StepParams<C>& p, const Scratch& sc, const T* f, cudaStream_t st)
    {
        k19_density<T, N><<<site_blocks(p.S), SITE_THREADS, 0, st>>>(f, (C*)sc.rho_s, (C*)sc.js, p);
        k19_potential<C, N><<<site_blocks(p.S), SITE_THREADS, 0, st>>>((const C*)sc.rho_s,
                                                                        (C*)sc.nu, p);
        return cudaGetLastError();
    }

    static cudaError_t step(const Problem& P, const Scratch& sc, void* const* f, int* cur,
                            long nsteps, cudaStream_t st)
    {
        const auto p = make_params<C>(P, sc.status);
        MCLB_DISPATCH_N(P.N, {
            if constexpr (NN <= M3_NMAX) {
                if (P.seg3 > 0) {
                    const dim3 grid(P.grid3[0], P.grid3[1], P.grid3[2]);
                    for (; nsteps > 0; --nsteps) {
                        const T* fi = (const T*)f[*cur];
                        k19_density<T, NN><<<site_blocks(P.S), SITE_THREADS, 0, st>>>(
                            fi, (C*)sc.rho_s, nullptr, p);
                        k19_march<T, NN><<<grid, M3_THREADS, m3_smem_bytes<C, NN>(), st>>>(
                            fi, (T*)f[*cur ^ 1], (const C*)sc.rho_s, p, P.seg3);
                        const cudaError_t e = cudaGetLastError();
                        if (e != cudaSuccess) return e;
                        *cur ^= 1;
                    }
                    return cudaSuccess;
                }
            }
            for (; nsteps > 0; --nsteps) {
                cudaError_t e = fields_n<NN>(p, sc, (const T*)f[*cur], st);
                if (e != cudaSuccess) return e;
                k19_collide<T, NN><<<site_blocks(P.S), SITE_THREADS, 0, st>>>(
                    (const T*)f[*cur], (T*)f[*cur ^ 1], (const C*)sc.rho_s, (const C*)sc.js,
                    (const C*)sc.nu, p);
                e = cudaGetLastError();
                if (e != cudaSuccess) return e;
                *cur ^= 1;
            }
            return cudaSuccess;
        });
    }

    static cudaError_t moments(const Problem& P, const Scratch& sc, const void* f, double* rho,
                               double* U, double* mu, double* Pt, cudaStream_t st)
    {
        const auto p = make_params<C>(P, sc.status);
        MCLB_DISPATCH_N(P.N, {
            cudaError_t e = fields_n<NN>(p, sc, (const T*)f, st);
            if (e != cudaSuccess) return e;
            k19_moments<T, NN><<<site_blocks(P.S), SITE_THREADS, 0, st>>>(
                (const T*)f, (const C*)sc.rho_s, (const C*)sc.nu, rho, U, mu, Pt, p);
            return cudaGetLastError();
        });
    }

    static cudaError_t conservation(const Problem& P, const Scratch& sc, const void* f, double* out,
                                    cudaStream_t st)
    {
        const auto p = make_params<C>(P, sc.status);
        MCLB_DISPATCH_N(P.N, {
            if (sc.partial_cap < (size_t)REDUCE_BLOCKS * (NN + 6)) return cudaErrorInvalidValue;
            cudaError_t e = fields_n<NN>(p, sc, (const T*)f, st);
            if (e != cudaSuccess) return e;
            k19_conservation<T, NN><<<REDUCE_BLOCKS, SITE_THREADS, 0, st>>>(
                (const T*)f, (const C*)sc.rho_s, (const C*)sc.nu, sc.partial, p);
            k_reduce_partials<<<1, SITE_THREADS, 0, st>>>(sc.partial, REDUCE_BLOCKS, NN + 6, out);
            return cudaGetLastError();
        });
    }

    static cudaError_t compositions(const Problem& P, const Scratch& sc, const void* f, double* phi,
                                    double* bulk, double tol, cudaStream_t st)
    {
        const auto p = make_params<C>(P, sc.status);
        MCLB_DISPATCH_N(P.N, {
            k19_density<T, NN><<<site_blocks(P.S), SITE_THREADS, 0, st>>>((const T*)f,
                                                                          (C*)sc.rho_s, nullptr, p);
            k19_compositions<T, NN><<<site_blocks(P.S), SITE_THREADS, 0, st>>>(
                (const C*)sc.rho_s, phi, bulk, tol, p);
            return cudaGetLastError();
        });
    }

    static cudaError_t get_state(const Problem& P, const Scratch& sc, const void* f, double* out,
                                 cudaStream_t st)
    {
        const auto p = make_params<C>(P, sc.status);
        MCLB_DISPATCH_N(P.N, {
            k19_get_state<T, NN><<<site_blocks(P.S), SITE_THREADS, 0, st>>>((const T*)f, out, p);
            return cudaGetLastError();
        });
    }

    static cudaError_t set_state(const Problem& P, const Scratch& sc, const double* in, void* f,
                                 cudaStream_t st)
    {
        const auto p = make_params<C>(P, sc.status);
        MCLB_DISPATCH_N(P.N, {
            k19_set_state<T, NN><<<site_blocks(P.S), SITE_THREADS, 0, st>>>(in, (T*)f, p);
            return cudaGetLastError();
        });
    }

    static const LatticeTable* table()
    {
        static const LatticeTable t = [] {
            LatticeTable x{};
            x.max_resident = &max_resident;
            x.plan = &plan;
            x.item_bytes = 0;
            x.prepare = &prepare;
            x.init = &init;
            x.step = &step;
            x.moments = &moments;
            x.conservation = &conservation;
            x.compositions = &compositions;
            x.get_state = &get_state;
            x.set_state = &set_state;
            return x;
        }();
        return &t;
    }
};

// The kernel table of one storage type is assembled from three parts, each instantiated
// in a translation unit of its own (prec_<type>_<part>.cu) so that
// the build compiles them in parallel; prec_<type>.cu puts the table together.
template <typename T>
inline void table_base(KernelTable& t, CUtensorMapDataType tt)
{
    t.storage_bytes = sizeof(T);
    t.shifted = Storage<T>::shifted;
    t.tma_type = tt;
    t.hx = (int)std::max<size_t>(4, 16 / sizeof(T));
    t.line3 = nullptr;
    t.d3q19 = nullptr;
}

// single handles on D2Q9: the single pass
template <typename T>
inline void fill_march(KernelTable& t)
{
    t.plan_fused = &Launch<T>::plan_fused;
    t.step_fused = &Launch<T>::step_fused;
}

// single handles on D2Q9: the staged schedule and the diagnostics
template <typename T>
inline void fill_staged(KernelTable& t)
{
    t.init = &Launch<T>::init;
    t.step_staged = &Launch<T>::step_staged;
    t.moments = &Launch<T>::moments;
    t.conservation = &Launch<T>::conservation;
    t.conservation_rows = &Launch<T>::conservation_rows;
    t.compositions = &Launch<T>::compositions;
    t.get_state = &Launch<T>::get_state;
    t.set_state = &Launch<T>::set_state;
    t.mass = &Launch<T>::mass;
}

// batches of D2Q9 instances
template <typename T>
inline void fill_batch(KernelTable& t)
{
    t.batch_create = &batch_group_create<T>;
    t.batch_step = &batch_group_step<T>;
    t.batch_launches = &batch_group_launches<T>;
    t.batch_tune = &batch_group_tune<T>;
    t.batch_waves = &batch_group_waves<T>;
    t.batch_destroy = &batch_group_destroy<T>;
    t.narrow_boxes = &batch_narrow_boxes<T>;
    t.batch_force = &batch_group_force<T>;
}

// the D1Q3 lattice (FP64 and FP32 storage)
template <typename T>
inline void fill_line3(KernelTable& t)
{
    static_assert(!Storage<T>::shifted, "D1Q3 stores FP64 or FP32");
    t.line3 = Line3Launch<T>::table();
}

// the D3Q19 lattice (FP64 and FP32 storage)
template <typename T>
inline void fill_cube(KernelTable& t)
{
    static_assert(!Storage<T>::shifted, "D3Q19 stores FP64 or FP32");
    t.d3q19 = Launch19<T>::table();
}

}  // namespace mclb
