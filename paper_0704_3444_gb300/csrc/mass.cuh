// mass.cuh -- per-component mass compensation (optional, every mass_every steps).
//
// Eq. ff1 makes the forcing term carry no mass, and the BGK collision keeps each
// component's mass, so sum over sites of rho^s is constant in exact arithmetic.  Stored
// in FP32 or in the 16-bit formats, every site's post-collision values are rounded; at a
// stationary state the same roundings repeat step after step, and the total mass walks
// away linearly in time.  The compensation holds one FP64 reference mass per component
// (taken when the state is set) and, when called, measures the current mass (compensated
// per-thread sums, combined in FP64) and adds the deficit, spread evenly over the sites, to each site's rest population: a
// zero-velocity population, so the momentum is untouched.  In the 16-bit formats the
// deficit goes to the FP32 reference density R, which hands w_i times it to each
// population the site's neighbours pull (sum_i w_i = 1, sum_i w_i v_i = 0).
//
// Both kernels read the stored buffer generically: per component, `lines` lines of
// `pitch` elements with data columns [first, first + nx), plus, in the 16-bit formats,
// `rlines` FP32 lines of the reference density; the rest population is line 0 of each
// row's q velocity lines.  Sums run in a fixed order (fixed grid, fixed block tree,
// partials added in block order), so the result does not depend on scheduling.
#pragma once

#include <type_traits>

#include "lattice.cuh"

namespace mclb {

constexpr int MASS_BLOCKS = 256;
constexpr int MASS_THREADS = 256;

struct MassView {
    long long comp_stride;   // elements from one component's lines to the next
    long long pitch;         // elements per line
    long long rbytes;        // 16-bit formats: byte offset of the FP32 density lines
    long long S;             // sites
    int lines;               // velocity lines per component (rows * q)
    int rlines;              // FP32 density lines per component (16-bit formats: rows), else 0
    int q;                   // velocity lines per row; line 0 of a row is the rest population
    int first;               // first data column of a line (the ghost columns before it)
    int nx;                  // data columns
    int span;                // columns of a line the correction covers, ghosts included
    int vec;                 // lines (and density lines) start on 16-byte boundaries
};

// Running sum in the compute type: FP64 storage adds in FP64; the others keep a
// compensated FP32 sum (Kahan: c carries the low-order part each addition loses), whose
// error does not grow with the number of terms.  FP64 arithmetic runs at a small
// fraction of the FP32 rate on this GPU, so per-element FP64 additions would make the
// reduction, not the memory, its bound.
template <typename C>
struct MassAcc {
    C sum = C(0), c = C(0);
    __device__ __forceinline__ void add(C x)
    {
        if constexpr (std::is_same<C, double>::value) {
            sum += x;
        } else {
            const C y = x - c;
            const C t = sum + y;
            c = (t - sum) - y;
            sum = t;
        }
    }
    __device__ __forceinline__ double value() const { return (double)sum - (double)c; }
};

__device__ __forceinline__ float mass_val(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float mass_val(__half v) { return __half2float(v); }
__device__ __forceinline__ float mass_val(float v) { return v; }
__device__ __forceinline__ double mass_val(double v) { return v; }

// One line's values into a lane's running sum: lane l takes the 16-byte vectors l, l + 32,
// ... (when the line is 16-byte aligned), then the columns of the ragged tail.  Whole
// vectors, four in flight per lane, so that the read runs at memory speed.
template <typename U, typename C>
__device__ __forceinline__ void mass_line(const U* __restrict__ line, int nx, bool vec, int lane,
                                          MassAcc<C>& acc)
{
    constexpr int W = 16 / sizeof(U);
    int done = 0;
    if (vec) {
        const int nv = nx / W;
        const uint4* p = reinterpret_cast<const uint4*>(line);
#pragma unroll 4
        for (int k = lane; k < nv; k += 32) {
            const uint4 q = __ldg(p + k);
            const U* e = reinterpret_cast<const U*>(&q);
#pragma unroll
            for (int j = 0; j < W; ++j) acc.add(C(mass_val(e[j])));
        }
        done = nv * W;
    }
    for (int x = done + lane; x < nx; x += 32) acc.add(C(mass_val(line[x])));
}

// part[s * MASS_BLOCKS + b]: block b's sum of component s's stored values.  Each warp
// takes whole lines (warp w of the grid: lines w, w + all warps, ...); lanes keep
// compensated sums, combined in FP64 by a fixed tree over the lanes and the warps.
template <typename T>
__global__ void __launch_bounds__(MASS_THREADS)
k_mass_partials(const T* __restrict__ f, const MassView v, double* __restrict__ part)
{
    using C = typename Storage<T>::C;
    constexpr int WARPS = MASS_THREADS / 32;
    __shared__ double red[WARPS];
    const int s = blockIdx.y;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const T* base = f + (long long)s * v.comp_stride + v.first;
    const float* rbase = reinterpret_cast<const float*>(reinterpret_cast<const char*>(f) + v.rbytes) +
                         (long long)s * v.rlines * v.pitch + v.first;
    MassAcc<C> acc;
    for (int l = blockIdx.x * WARPS + warp; l < v.lines + v.rlines; l += gridDim.x * WARPS) {
        if (l < v.lines)
            mass_line<T, C>(base + (long long)l * v.pitch, v.nx, v.vec, lane, acc);
        else
            mass_line<float, C>(rbase + (long long)(l - v.lines) * v.pitch, v.nx, v.vec, lane, acc);
    }
    double m = acc.value();
    for (int o = 16; o > 0; o >>= 1) m += __shfl_down_sync(0xffffffffu, m, o);
    if (lane == 0) red[warp] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int w = 0; w < WARPS; ++w) b += red[w];
        part[s * MASS_BLOCKS + blockIdx.x] = b;
    }
}

// record != 0: ref[s] = the measured mass (launch with one block per component).
// record == 0: add (ref[s] - mass) / S to the rest population (or R) of every site.
template <typename T>
__global__ void __launch_bounds__(MASS_THREADS)
k_mass_apply(T* __restrict__ f, const MassView v, const double* __restrict__ part,
             double* __restrict__ ref, int record)
{
    using C = typename Storage<T>::C;
    static_assert(MASS_BLOCKS % 32 == 0, "partials are summed by one warp");
    __shared__ double delta;
    const int s = blockIdx.y;
    if (threadIdx.x < 32) {
        // the same fixed-shape sum in every block: lane l adds partials l, l + 32, ... in
        // order, then a fixed butterfly over the lanes
        double m = 0.0;
        for (int b = threadIdx.x; b < MASS_BLOCKS; b += 32) m += part[s * MASS_BLOCKS + b];
        for (int o = 16; o > 0; o >>= 1) m += __shfl_xor_sync(0xffffffffu, m, o);
        if (threadIdx.x == 0) {
            if (record) {
                if (blockIdx.x == 0) ref[s] = m;
            } else {
                delta = (ref[s] - m) / (double)v.S;
            }
        }
    }
    if (record) return;
    __syncthreads();
    const int rows = v.lines / v.q;
    for (int y = blockIdx.x; y < rows; y += gridDim.x) {
        if (v.rlines > 0) {
            float* line = reinterpret_cast<float*>(reinterpret_cast<char*>(f) + v.rbytes) +
                          ((long long)s * v.rlines + y) * v.pitch;
            const float d = (float)delta;
            for (int x = threadIdx.x; x < v.span; x += blockDim.x) line[x] = line[x] + d;
        } else {
            T* line = f + (long long)s * v.comp_stride + (long long)y * v.q * v.pitch;
            const C d = (C)delta;
            for (int x = threadIdx.x; x < v.span; x += blockDim.x) line[x] = T(C(line[x]) + d);
        }
    }
}

}  // namespace mclb
