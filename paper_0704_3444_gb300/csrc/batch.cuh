// batch.cuh -- many independent simulations advanced by the staged schedule in one set
// of launches: each block works on one instance, found through a block-to-instance
// table, and runs the same per-site code as the single-simulation kernels.
#pragma once

#include <vector>

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
    density_site<T, N>(it.f[parity], it.rs, it.p, site);
}

template <typename T, int N>
__global__ void __launch_bounds__(SITE_THREADS)
kb_potential(const BatchItem<T>* __restrict__ items, const int* __restrict__ blk2inst)
{
    const BatchItem<T>& it = items[blk2inst[blockIdx.x]];
    const long long site = (long long)(blockIdx.x - it.block0) * SITE_THREADS + threadIdx.x;
    if (site >= it.p.S) return;
    potential_site<typename Storage<T>::C, N>(it.rs, it.nu, it.p, site);
}

template <typename T, int N>
__global__ void __launch_bounds__(SITE_THREADS)
kb_collide(const BatchItem<T>* __restrict__ items, const int* __restrict__ blk2inst, int parity)
{
    const BatchItem<T>& it = items[blk2inst[blockIdx.x]];
    const long long site = (long long)(blockIdx.x - it.block0) * SITE_THREADS + threadIdx.x;
    if (site >= it.p.S) return;
    collide_site<T, N>(it.f[parity], it.f[parity ^ 1], it.nu, it.p, site);
}

// One group of instances sharing N.
template <typename T>
struct BatchGroup {
    int N = 0;
    int nblocks = 0;
    BatchItem<T>* items = nullptr;
    int* blk2inst = nullptr;
};

template <typename T>
void* batch_group_create(int N, int count, const Problem* probs, const Scratch* scs,
                         void* const* fa, void* const* fb, cudaStream_t st)
{
    using C = typename Storage<T>::C;
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

template <typename T, int N>
cudaError_t batch_group_step_n(const BatchGroup<T>* g, int parity, cudaStream_t st)
{
    kb_density<T, N><<<g->nblocks, SITE_THREADS, 0, st>>>(g->items, g->blk2inst, parity);
    kb_potential<T, N><<<g->nblocks, SITE_THREADS, 0, st>>>(g->items, g->blk2inst);
    kb_collide<T, N><<<g->nblocks, SITE_THREADS, 0, st>>>(g->items, g->blk2inst, parity);
    return cudaGetLastError();
}

template <typename T>
cudaError_t batch_group_step(void* group, int parity, cudaStream_t st)
{
    const auto* g = static_cast<const BatchGroup<T>*>(group);
    switch (g->N) {
        case 1: return batch_group_step_n<T, 1>(g, parity, st);
        case 2: return batch_group_step_n<T, 2>(g, parity, st);
        case 3: return batch_group_step_n<T, 3>(g, parity, st);
        case 4: return batch_group_step_n<T, 4>(g, parity, st);
        case 5: return batch_group_step_n<T, 5>(g, parity, st);
        case 6: return batch_group_step_n<T, 6>(g, parity, st);
        case 7: return batch_group_step_n<T, 7>(g, parity, st);
        case 8: return batch_group_step_n<T, 8>(g, parity, st);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T>
void batch_group_destroy(void* group)
{
    auto* g = static_cast<BatchGroup<T>*>(group);
    if (!g) return;
    if (g->items) cudaFree(g->items);
    if (g->blk2inst) cudaFree(g->blk2inst);
    delete g;
}

}  // namespace mclb
