// ghosts.cuh -- refresh of the periodic ghost columns after a single-pass step.
#pragma once

#include "lattice.cuh"

namespace mclb {

// Periodic ghost columns of every line of f (and of the FP32 density lines in the
// 16-bit formats): column g in [-hx, 0) and [nx, nx + hx) takes the value of column
// g mod nx.  One thread per ghost column of a line, consecutive threads on the same
// line, so that a warp touches a few contiguous runs.
template <typename T>
__global__ void __launch_bounds__(256)
k_ghosts(T* __restrict__ f, const __grid_constant__ StepParams<typename Storage<T>::C> p, int ncomp)
{
    const int hx = p.hx, nx = p.nx, per = 2 * hx;
    const long long nl = (long long)ncomp * p.ny * Q;
    const long long nr = Storage<T>::shifted ? (long long)ncomp * p.ny : 0;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (nl + nr) * per) return;
    const long long l = t / per;
    const int j = (int)(t - l * per);
    const int gcol = j < hx ? j - hx : nx + (j - hx);            // ghost column
    const int src = ((gcol % nx) + nx) % nx;                      // the column it repeats
    if (l < nl) {
        T* row = f + l * p.pitch + hx;
        row[gcol] = row[src];
    } else {
        float* row = reinterpret_cast<float*>(reinterpret_cast<char*>(f) + p.rbytes) + (l - nl) * p.pitch + hx;
        row[gcol] = row[src];
    }
}

}  // namespace mclb
