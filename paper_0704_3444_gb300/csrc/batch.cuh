// batch.cuh -- many independent simulations advanced together.  All instances that share
// N are advanced by one launch of the single-pass march (kb_march: each CTA looks up its
// instance, strip and segment in a table and runs march_cta with that instance's
// parameters and tensor maps) followed by one ghost-column refresh (kb_ghosts).  When an
// instance cannot use the march (its tensor maps could not be built), the group falls
// back to the staged schedule over a block-to-instance table (kb_density, kb_potential,
// kb_collide), which runs the same per-site code as the single-simulation kernels.
#pragma once

#include <algorithm>
#include <vector>

#include "march.cuh"
#include "staged.cuh"

namespace mclb {

// Device-side description of one instance of a batch.
template <typename T>
struct BatchItem {
    StepParams<typename Storage<T>::C> p;
    T* f[2];                                 // ping-pong distribution buffers
    typename Storage<T>::C* rs;              // density scratch (N * S)
    typename Storage<T>::C* nu;              // potential scratch (N * S)
    long long block0;                        // first block of this instance
};

template <typename T, int N>
__global__ void __launch_bounds__(SITE_THREADS)
kb_density(const BatchItem<T>* __restrict__ items, const int* __restrict__ blk2inst, int parity)
{
    const BatchItem<T>& it = items[blk2inst[blockIdx.x]];
    const long long site = (long long)(blockIdx.x - it.block0) * SITE_THREADS + threadIdx.x;
    if (site >= it.p.S) return;
    density_site<T, N, false>(it.f[parity], it.rs, it.p, site);   // batches are periodic
}

template <typename T, int N>
__global__ void __launch_bounds__(SITE_THREADS)
kb_potential(const BatchItem<T>* __restrict__ items, const int* __restrict__ blk2inst)
{
    const BatchItem<T>& it = items[blk2inst[blockIdx.x]];
    const long long site = (long long)(blockIdx.x - it.block0) * SITE_THREADS + threadIdx.x;
    if (site >= it.p.S) return;
    potential_site<typename Storage<T>::C, N, false>(it.rs, it.nu, it.p, site);
}

template <typename T, int N>
__global__ void __launch_bounds__(SITE_THREADS)
kb_collide(const BatchItem<T>* __restrict__ items, const int* __restrict__ blk2inst, int parity)
{
    const BatchItem<T>& it = items[blk2inst[blockIdx.x]];
    const long long site = (long long)(blockIdx.x - it.block0) * SITE_THREADS + threadIdx.x;
    if (site >= it.p.S) return;
    collide_site<T, N, false>(it.f[parity], it.f[parity ^ 1], it.rs, it.nu, it.p, site);
}

// Device-side description of one instance for the batched march: its tensor maps
// ([buffer][load view, density-line load view, store view, density-line store view]) for
// the wide geometry (maps) and the narrow one (maps2: the same views with that geometry's
// box widths), parameters and buffers.  Tensor maps in global memory must be 64-byte
// aligned.
template <typename T>
struct alignas(64) MarchItem {
    CUtensorMap maps[2][4];
    CUtensorMap maps2[2][4];
    StepParams<typename Storage<T>::C> p;
    T* f[2];
};

// One CTA of the batched march: instance, first written column, first row, rows.
struct MarchCta {
    int inst, x0, y0, H;
};

// G: the march geometry of this launch (MarchGeom, or MarchNarrow with NARROW = true, which
// selects the instance's maps2)
template <typename T, int N, typename G, bool NARROW>
__global__ void __launch_bounds__(G::THREADS) __maxnreg__((G::MAXREG))
kb_march(const MarchItem<T>* __restrict__ items, const MarchCta* __restrict__ ctas, int parity)
{
    using C = typename Storage<T>::C;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ StepParams<C> ps;
    const MarchCta c = ctas[blockIdx.x];
    const MarchItem<T>& it = items[c.inst];
    const CUtensorMap (&maps)[2][4] = NARROW ? it.maps2 : it.maps;
    static_assert(sizeof(StepParams<C>) % sizeof(int) == 0, "parameter copy by words");
    const int* src = reinterpret_cast<const int*>(&it.p);
    int* dst = reinterpret_cast<int*>(&ps);
    for (int k = threadIdx.x; k < (int)(sizeof(StepParams<C>) / sizeof(int)); k += blockDim.x) dst[k] = src[k];
    if (threadIdx.x == 0) {
        // the tensor maps were written to global memory before the launch; make them
        // visible to the tensor-map proxy before the first copy uses them
        for (int b = 0; b < 2; ++b)
            for (int j = 0; j < 4; ++j)
                asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&maps[b][j])
                             : "memory");
    }
    __syncthreads();
    march_cta<T, N, G>(&maps[parity][0], &maps[parity][1], &maps[parity ^ 1][2], &maps[parity ^ 1][3],
                       it.f[parity ^ 1], ps, c.x0, c.y0, c.H, smem);
}

// Ghost columns of every instance's new buffer (parity ^ 1), laid out per instance as in
// k_ghosts: instance k owns ghost values [0, start[k + 1] - start[k]), handled by the
// blocks [first[k], first[k + 1]) of 256 threads; blk2inst gives each block's instance.
template <typename T>
__global__ void __launch_bounds__(256)
kb_ghosts(const MarchItem<T>* __restrict__ items, const long long* __restrict__ start,
          const int* __restrict__ first, const int* __restrict__ blk2inst, int parity, int ncomp)
{
    const int k = blk2inst[blockIdx.x];
    const long long u = (long long)(blockIdx.x - first[k]) * blockDim.x + threadIdx.x;
    if (u >= start[k + 1] - start[k]) return;
    const MarchItem<T>& it = items[k];
    const auto& p = it.p;
    const int hx = p.hx, nx = p.nx, per = 2 * hx;
    const long long nl = (long long)ncomp * p.ny * Q;
    const long long l = u / per;
    const int j = (int)(u - l * per);
    const int gcol = j < hx ? j - hx : nx + (j - hx);
    const int srcc = ((gcol % nx) + nx) % nx;
    T* f = it.f[parity ^ 1];
    if (l < nl) {
        T* row = f + l * p.pitch + hx;
        row[gcol] = row[srcc];
    } else {
        float* row = reinterpret_cast<float*>(reinterpret_cast<char*>(f) + p.rbytes) + (l - nl) * p.pitch + hx;
        row[gcol] = row[srcc];
    }
}

// One group of instances sharing N.
template <typename T>
struct BatchGroup {
    int N = 0;
    // staged schedule
    int nblocks = 0;
    BatchItem<T>* items = nullptr;
    int* blk2inst = nullptr;
    // batched march: candidate CTA tables (the wide and, where it exists, the narrow strip
    // geometry, each with segment heights for different wave counts), the one in use picked
    // by timing them at the first step
    bool march = false;
    bool tuned = false;
    int count = 0;
    MarchItem<T>* mitems = nullptr;
    std::vector<MarchCta*> cand;
    std::vector<int> cand_n;
    std::vector<int> cand_waves;
    std::vector<int> cand_geo;   // 0: MarchGeom (wide strips), 1: MarchNarrow
    int pick = 0;
    long long* gstart = nullptr;
    int* gfirst = nullptr;      // first ghost block of each instance
    int* gblk2inst = nullptr;   // instance of each ghost block
    int gblocks = 0;
};

constexpr int MARCH_WAVES[] = {2, 4, 8, 16};

// Table of the batched march's CTAs: strips of WOUT columns, segments of about the same
// height everywhere (chosen so that the launch is about `waves` waves deep), tallest first.
template <typename T, int N, typename G = MarchGeom<T, N>>
std::vector<MarchCta> march_ctas(int count, const Problem* probs, int slots, int waves)
{
    long long rows = 0;
    for (int k = 0; k < count; ++k) rows += (long long)((probs[k].nx + G::WOUT - 1) / G::WOUT) * probs[k].ny;
    const int target = (int)std::max<long long>(8, rows / std::max(1, waves * slots));
    std::vector<MarchCta> v;
    for (int k = 0; k < count; ++k) {
        const int nx = probs[k].nx, ny = probs[k].ny;
        const int nsegs = std::max(1, (ny + target / 2) / target);
        const int H = (ny + nsegs - 1) / nsegs;
        for (int x0 = 0; x0 < nx; x0 += G::WOUT)
            for (int y0 = 0; y0 < ny; y0 += H) v.push_back(MarchCta{k, x0, y0, std::min(H, ny - y0)});
    }
    std::stable_sort(v.begin(), v.end(), [](const MarchCta& a, const MarchCta& b) { return a.H > b.H; });
    return v;
}

// Kernel attributes of one geometry's batched march; *per_sm receives its resident CTAs.
template <typename T, int N, typename G, bool NARROW>
bool march_geometry_ready(int* per_sm)
{
    auto kern = kb_march<T, N, G, NARROW>;
    if (!G::FITS ||
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM) != cudaSuccess ||
        cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kern, G::THREADS, G::SMEM) != cudaSuccess ||
        *per_sm < 1) {
        cudaGetLastError();
        return false;
    }
    return true;
}

// The candidate CTA tables of one geometry (one per wave count) appended to the group.
template <typename T, int N, typename G>
bool march_add_candidates(BatchGroup<T>* g, int geo, int count, const Problem* probs, int slots,
                          cudaStream_t st)
{
    for (int waves : MARCH_WAVES) {
        const std::vector<MarchCta> ctas = march_ctas<T, N, G>(count, probs, slots, waves);
        if (ctas.empty() || ctas.size() > (size_t)INT32_MAX) return false;
        MarchCta* d = nullptr;
        if (cudaMalloc(&d, sizeof(MarchCta) * ctas.size()) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        g->cand.push_back(d);
        g->cand_n.push_back((int)ctas.size());
        g->cand_waves.push_back(waves);
        g->cand_geo.push_back(geo);
        if (cudaMemcpyAsync(d, ctas.data(), sizeof(MarchCta) * ctas.size(), cudaMemcpyHostToDevice, st) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
    }
    return true;
}

template <typename T, int N>
bool march_group_create(BatchGroup<T>* g, int count, const Problem* probs, const Scratch* scs,
                        void* const* fa, void* const* fb, const CUtensorMap* maps,
                        const CUtensorMap* maps2, int sm_count, cudaStream_t st)
{
    using C = typename Storage<T>::C;
    int per_sm = 0, per_sm2 = 0;
    if (!march_geometry_ready<T, N, MarchGeom<T, N>, false>(&per_sm)) return false;
    bool narrow = false;
    if constexpr (has_narrow<T, N>())
        narrow = maps2 && march_geometry_ready<T, N, MarchNarrow<T, N>, true>(&per_sm2);
    std::vector<MarchItem<T>> items(count);
    std::vector<long long> gstart(count + 1, 0);
    std::vector<int> gfirst(count + 1, 0), gmap;
    for (int k = 0; k < count; ++k) {
        for (int b = 0; b < 2; ++b)
            for (int j = 0; j < 4; ++j) {
                items[k].maps[b][j] = maps[(size_t)k * 8 + b * 4 + j];
                items[k].maps2[b][j] = narrow ? maps2[(size_t)k * 8 + b * 4 + j] : maps[(size_t)k * 8 + b * 4 + j];
            }
        items[k].p = make_params<C>(probs[k], scs[k].status);
        items[k].f[0] = static_cast<T*>(fa[k]);
        items[k].f[1] = static_cast<T*>(fb[k]);
        const long long lines = (long long)N * probs[k].ny * (Q + (Storage<T>::shifted ? 1 : 0));
        gstart[k + 1] = gstart[k] + lines * 2 * probs[k].hx;
        const long long nb = (gstart[k + 1] - gstart[k] + 255) / 256;
        if ((long long)gmap.size() + nb > INT32_MAX) return false;
        gfirst[k] = (int)gmap.size();
        gmap.insert(gmap.end(), (size_t)nb, k);
    }
    gfirst[count] = (int)gmap.size();
    if (cudaMalloc(&g->mitems, sizeof(MarchItem<T>) * count) != cudaSuccess ||
        cudaMalloc(&g->gstart, sizeof(long long) * (count + 1)) != cudaSuccess ||
        cudaMalloc(&g->gfirst, sizeof(int) * (count + 1)) != cudaSuccess ||
        cudaMalloc(&g->gblk2inst, sizeof(int) * gmap.size()) != cudaSuccess ||
        cudaMemcpyAsync(g->gfirst, gfirst.data(), sizeof(int) * (count + 1), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(g->gblk2inst, gmap.data(), sizeof(int) * gmap.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(g->mitems, items.data(), sizeof(MarchItem<T>) * count, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(g->gstart, gstart.data(), sizeof(long long) * (count + 1), cudaMemcpyHostToDevice, st) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const int slots = per_sm * std::max(1, sm_count);
    if (!march_add_candidates<T, N, MarchGeom<T, N>>(g, 0, count, probs, slots, st)) return false;
    if constexpr (has_narrow<T, N>())
        if (narrow && !march_add_candidates<T, N, MarchNarrow<T, N>>(g, 1, count, probs,
                                                                   per_sm2 * std::max(1, sm_count), st))
            return false;
    if (cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    g->march = true;
    g->count = count;
    g->pick = 1;   // wide strips, four waves, until tuned
    g->gblocks = (int)gmap.size();
    return true;
}

// One launch of the batched march with candidate table c.
template <typename T, int N>
cudaError_t march_launch(const BatchGroup<T>* g, int c, int parity, cudaStream_t st)
{
    if (g->cand_geo[c] == 0) {
        using G = MarchGeom<T, N>;
        kb_march<T, N, G, false><<<g->cand_n[c], G::THREADS, G::SMEM, st>>>(g->mitems, g->cand[c], parity);
    } else {
        if constexpr (has_narrow<T, N>()) {
            using G = MarchNarrow<T, N>;
            kb_march<T, N, G, true><<<g->cand_n[c], G::THREADS, G::SMEM, st>>>(g->mitems, g->cand[c], parity);
        } else {
            return cudaErrorInvalidValue;
        }
    }
    return cudaGetLastError();
}

// Time every candidate CTA table -- both strip geometries, every wave count -- on the
// current state (each run reads buffer `parity` and rewrites the other buffer with the
// same values, so the state is unchanged) and keep the fastest.  Synchronises the stream.
template <typename T, int N>
cudaError_t march_group_tune(BatchGroup<T>* g, int parity, cudaStream_t st)
{
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t err = cudaEventCreate(&e0);
    if (err == cudaSuccess) err = cudaEventCreate(&e1);
    float best = 1e30f;
    for (size_t c = 0; c < g->cand.size() && err == cudaSuccess; ++c) {
        err = march_launch<T, N>(g, (int)c, parity, st);
        if (err == cudaSuccess) err = cudaEventRecord(e0, st);
        for (int r = 0; r < 3 && err == cudaSuccess; ++r) err = march_launch<T, N>(g, (int)c, parity, st);
        if (err == cudaSuccess) err = cudaEventRecord(e1, st);
        if (err == cudaSuccess) err = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
        if (err == cudaSuccess && ms < best) {
            best = ms;
            g->pick = (int)c;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    g->tuned = true;
    return err;
}

template <typename T>
void batch_group_destroy(void* group);

template <typename T>
void* batch_group_create(int N, int count, const Problem* probs, const Scratch* scs,
                         void* const* fa, void* const* fb, const CUtensorMap* maps,
                         const CUtensorMap* maps2, int sm_count, cudaStream_t st)
{
    using C = typename Storage<T>::C;
    if (maps) {
        auto* g = new BatchGroup<T>();
        g->N = N;
        bool ok = false;
        switch (N) {
            case 1: ok = march_group_create<T, 1>(g, count, probs, scs, fa, fb, maps, maps2, sm_count, st); break;
            case 2: ok = march_group_create<T, 2>(g, count, probs, scs, fa, fb, maps, maps2, sm_count, st); break;
            case 3: ok = march_group_create<T, 3>(g, count, probs, scs, fa, fb, maps, maps2, sm_count, st); break;
            case 4: ok = march_group_create<T, 4>(g, count, probs, scs, fa, fb, maps, maps2, sm_count, st); break;
            case 5: ok = march_group_create<T, 5>(g, count, probs, scs, fa, fb, maps, maps2, sm_count, st); break;
            case 6: ok = march_group_create<T, 6>(g, count, probs, scs, fa, fb, maps, maps2, sm_count, st); break;
            case 7: ok = march_group_create<T, 7>(g, count, probs, scs, fa, fb, maps, maps2, sm_count, st); break;
            case 8: ok = march_group_create<T, 8>(g, count, probs, scs, fa, fb, maps, maps2, sm_count, st); break;
            default: break;
        }
        if (ok) return g;
        batch_group_destroy<T>(g);
    }
    std::vector<BatchItem<T>> items(count);
    std::vector<int> map;
    long long blocks = 0;
    for (int k = 0; k < count; ++k) {
        items[k].p = make_params<C>(probs[k], scs[k].status);
        items[k].f[0] = static_cast<T*>(fa[k]);
        items[k].f[1] = static_cast<T*>(fb[k]);
        items[k].rs = static_cast<C*>(scs[k].rho_s);
        items[k].nu = static_cast<C*>(scs[k].nu);
        items[k].block0 = blocks;
        const long long nb = (probs[k].S + SITE_THREADS - 1) / SITE_THREADS;
        for (long long b = 0; b < nb; ++b) map.push_back(k);
        blocks += nb;
    }
    if (blocks > (1LL << 31) - 1) return nullptr;
    auto* g = new BatchGroup<T>();
    g->N = N;
    g->nblocks = (int)blocks;
    if (cudaMalloc(&g->items, sizeof(BatchItem<T>) * count) != cudaSuccess ||
        cudaMalloc(&g->blk2inst, sizeof(int) * map.size()) != cudaSuccess ||
        cudaMemcpyAsync(g->items, items.data(), sizeof(BatchItem<T>) * count,
                        cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(g->blk2inst, map.data(), sizeof(int) * map.size(), cudaMemcpyHostToDevice,
                        st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        if (g->items) cudaFree(g->items);
        if (g->blk2inst) cudaFree(g->blk2inst);
        delete g;
        return nullptr;
    }
    return g;
}

// Part 0 of a group step: the batched march (or the whole staged step); part 1: the
// ghost-column refresh of the buffer part 0 wrote (nothing for the staged schedule).
template <typename T, int N>
cudaError_t batch_group_step_n(const BatchGroup<T>* g, int parity, cudaStream_t st, int part)
{
    if (g->march) {
        if (part == 0) return march_launch<T, N>(g, g->pick, parity, st);
        kb_ghosts<T><<<g->gblocks, 256, 0, st>>>(g->mitems, g->gstart, g->gfirst, g->gblk2inst, parity, N);
        return cudaGetLastError();
    }
    if (part != 0) return cudaSuccess;
    kb_density<T, N><<<g->nblocks, SITE_THREADS, 0, st>>>(g->items, g->blk2inst, parity);
    kb_potential<T, N><<<g->nblocks, SITE_THREADS, 0, st>>>(g->items, g->blk2inst);
    kb_collide<T, N><<<g->nblocks, SITE_THREADS, 0, st>>>(g->items, g->blk2inst, parity);
    return cudaGetLastError();
}

template <typename T>
cudaError_t batch_group_step(void* group, int parity, cudaStream_t st, int part)
{
    const auto* g = static_cast<const BatchGroup<T>*>(group);
    switch (g->N) {
        case 1: return batch_group_step_n<T, 1>(g, parity, st, part);
        case 2: return batch_group_step_n<T, 2>(g, parity, st, part);
        case 3: return batch_group_step_n<T, 3>(g, parity, st, part);
        case 4: return batch_group_step_n<T, 4>(g, parity, st, part);
        case 5: return batch_group_step_n<T, 5>(g, parity, st, part);
        case 6: return batch_group_step_n<T, 6>(g, parity, st, part);
        case 7: return batch_group_step_n<T, 7>(g, parity, st, part);
        case 8: return batch_group_step_n<T, 8>(g, parity, st, part);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T>
cudaError_t batch_group_tune(void* group, int parity, cudaStream_t st)
{
    auto* g = static_cast<BatchGroup<T>*>(group);
    if (!g->march || g->tuned) return cudaSuccess;
    switch (g->N) {
        case 1: return march_group_tune<T, 1>(g, parity, st);
        case 2: return march_group_tune<T, 2>(g, parity, st);
        case 3: return march_group_tune<T, 3>(g, parity, st);
        case 4: return march_group_tune<T, 4>(g, parity, st);
        case 5: return march_group_tune<T, 5>(g, parity, st);
        case 6: return march_group_tune<T, 6>(g, parity, st);
        case 7: return march_group_tune<T, 7>(g, parity, st);
        case 8: return march_group_tune<T, 8>(g, parity, st);
        default: return cudaErrorInvalidValue;
    }
}

// Test hook: use candidate (narrow, waves) from now on, untimed.
template <typename T>
bool batch_group_force(void* group, int narrow, int waves)
{
    auto* g = static_cast<BatchGroup<T>*>(group);
    if (!g->march) return false;
    for (size_t c = 0; c < g->cand.size(); ++c)
        if (g->cand_geo[c] == (narrow ? 1 : 0) && g->cand_waves[c] == waves) {
            g->pick = (int)c;
            g->tuned = true;
            return true;
        }
    return false;
}

// waves of the CTA table in use (0 for the staged schedule), plus 1000 when the narrow
// strip geometry was picked
template <typename T>
int batch_group_waves(const void* group)
{
    const auto* g = static_cast<const BatchGroup<T>*>(group);
    return g->march ? g->cand_waves[g->pick] + 1000 * g->cand_geo[g->pick] : 0;
}

// Box widths of the narrow geometry's views for N components (load boxes, store boxes);
// false where the group has no narrow candidate.
template <typename T, int N>
bool narrow_boxes_n(int* box_w, int* out_w)
{
    if constexpr (has_narrow<T, N>()) {
        using G = MarchNarrow<T, N>;
        *box_w = G::WI;
        *out_w = G::TMA_STORE ? MARCH_OUT : (G::CTA_STORE ? G::WOUT : 0);
        return true;
    }
    return false;
}
template <typename T>
bool batch_narrow_boxes(int N, int* box_w, int* out_w)
{
    switch (N) {
        case 1: return narrow_boxes_n<T, 1>(box_w, out_w);
        case 2: return narrow_boxes_n<T, 2>(box_w, out_w);
        case 3: return narrow_boxes_n<T, 3>(box_w, out_w);
        case 4: return narrow_boxes_n<T, 4>(box_w, out_w);
        case 5: return narrow_boxes_n<T, 5>(box_w, out_w);
        case 6: return narrow_boxes_n<T, 6>(box_w, out_w);
        case 7: return narrow_boxes_n<T, 7>(box_w, out_w);
        case 8: return narrow_boxes_n<T, 8>(box_w, out_w);
        default: return false;
    }
}

template <typename T>
int batch_group_launches(const void* group)
{
    return static_cast<const BatchGroup<T>*>(group)->march ? 2 : 3;
}

template <typename T>
void batch_group_destroy(void* group)
{
    auto* g = static_cast<BatchGroup<T>*>(group);
    if (!g) return;
    if (g->items) cudaFree(g->items);
    if (g->blk2inst) cudaFree(g->blk2inst);
    if (g->mitems) cudaFree(g->mitems);
    for (MarchCta* d : g->cand) cudaFree(d);
    if (g->gstart) cudaFree(g->gstart);
    if (g->gfirst) cudaFree(g->gfirst);
    if (g->gblk2inst) cudaFree(g->gblk2inst);
    delete g;
}

}  // namespace mclb
