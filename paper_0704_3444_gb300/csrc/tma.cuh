// tma.cuh -- mbarrier and TMA (cp.async.bulk.tensor) helpers for the single-pass
// kernel, with bounded waits.
#pragma once

#include "physics.cuh"

namespace mclb {

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

// Plain arrival (release semantics: the caller's earlier shared-memory reads are done).
__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
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

// One 4-D TMA box (columns, velocity lines from `line`, 1 row, all components) into
// shared memory; the box extents are those the tensor map was encoded with.
__device__ __forceinline__ void tma_load_row(void* dst, const CUtensorMap* map, uint64_t* bar,
                                             int col, int row, int line = 0)
{
    const uint64_t desc = reinterpret_cast<uint64_t>(map);
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5, %6}], [%2];" ::"r"(smem_u32(dst)),
        "l"(desc), "r"(smem_u32(bar)), "r"(col), "r"(line), "r"(row), "r"(0)
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
__device__ __forceinline__ void tma_prefetch_row(const CUtensorMap* map, int col, int row,
                                                 int line = 0)
{
    const uint64_t desc = reinterpret_cast<uint64_t>(map);
    asm volatile("cp.async.bulk.prefetch.tensor.4d.L2.global [%0, {%1, %2, %3, %4}];" ::"l"(desc),
                 "r"(col), "r"(line), "r"(row), "r"(0)
                 : "memory");
}

// One 4-D TMA box from shared memory to global (bulk async-group completion).
__device__ __forceinline__ void tma_store_box(const CUtensorMap* map, const void* src, int col,
                                              int line, int row, int comp)
{
    const uint64_t desc = reinterpret_cast<uint64_t>(map);
    asm volatile("cp.async.bulk.tensor.4d.global.shared::cta.bulk_group [%0, {%2, %3, %4, %5}], [%1];" ::"l"(desc),
                 "r"(smem_u32(src)), "r"(col), "r"(line), "r"(row), "r"(comp)
                 : "memory");
}
// One 3-D TMA box (columns, 1 row, all components) from shared memory to global.
__device__ __forceinline__ void tma_store_box3(const CUtensorMap* map, const void* src, int col,
                                               int row, int comp)
{
    const uint64_t desc = reinterpret_cast<uint64_t>(map);
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(desc),
                 "r"(smem_u32(src)), "r"(col), "r"(row), "r"(comp)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// wait until the bulk stores of this thread have finished reading shared memory
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// wait until the bulk stores of this thread are complete
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// order this thread's generic-proxy shared-memory writes before later async-proxy reads
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

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

// acc + v for a value in storage precision, the widening folded into the add (PTX mixed
// precision add, .f32 result from a .bf16/.f16 operand; exact widening, one rounding as
// to_c(v) + acc)
template <typename T>
__device__ __forceinline__ float add_wide(float acc, T v);
template <>
__device__ __forceinline__ float add_wide<__nv_bfloat16>(float acc, __nv_bfloat16 v)
{
    float r;
    asm("add.rn.f32.bf16 %0, %1, %2;" : "=f"(r) : "h"(__bfloat16_as_ushort(v)), "f"(acc));
    return r;
}
template <>
__device__ __forceinline__ float add_wide<__half>(float acc, __half v)
{
    float r;
    asm("add.rn.f32.f16 %0, %1, %2;" : "=f"(r) : "h"(__half_as_ushort(v)), "f"(acc));
    return r;
}

__host__ __device__ constexpr size_t round_up_sz(size_t a, size_t b) { return (a + b - 1) / b * b; }

}  // namespace mclb
