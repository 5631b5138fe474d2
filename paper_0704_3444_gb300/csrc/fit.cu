// fit.cu -- the bulk-phase fit of mclb_fit_equilibrium, on the device in FP64.
//
// Input: compositions phi^s = rho^s / rho ([s][site], N * S doubles) and bulk flags
// (S doubles, 1 where the site is away from interfaces), both written by a
// compositions kernel of the handle's lattice.  Output: the mean composition of each
// of nphase bulk phases -- the coexisting compositions that Sec. 4 compares with the
// Flory-Huggins binodals.  k-means over the bulk sites: phase c is seeded at the bulk
// site richest in component c (the lowest such site index on ties); each iteration
// assigns every bulk site to the nearest centroid (squared distance in composition
// space, the lower phase index on ties) and replaces each centroid by the mean of its
// sites; it stops when the centroids no longer change.  Every sum is taken in a fixed
// order (a fixed grid of blocks, fixed-shape block reductions, block partials summed in
// block order), so the result does not depend on scheduling.  Only the nphase * N
// centroid values and a flag cross to the host per iteration.
#include <cfloat>

#include "mclb_internal.h"

namespace mclb {

namespace {

constexpr int FIT_BLOCKS = 256;
constexpr int FIT_THREADS = 256;
constexpr int FIT_VALS = NMAX * (NMAX + 1);  // per phase: count + N sums

// Seed search: per block, for each phase c < nphase, the bulk site with the largest
// phi^c (smallest index on ties).  part[(b * nphase + c) * 2 + {0, 1}] = (value, index).
__global__ void __launch_bounds__(FIT_THREADS)
k_fit_seed_blocks(const double* __restrict__ phi, const double* __restrict__ bulk, long long S,
                  int nphase, double* __restrict__ part)
{
    __shared__ double sv[FIT_THREADS];
    __shared__ long long si[FIT_THREADS];
    for (int c = 0; c < nphase; ++c) {
        double best = -DBL_MAX;
        long long arg = -1;
        for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < S;
             t += (long long)gridDim.x * blockDim.x) {
            if (bulk[t] < 0.5) continue;
            const double v = phi[(long long)c * S + t];
            if (v > best) {   // strictly greater: the first (smallest) index wins ties
                best = v;
                arg = t;
            }
        }
        sv[threadIdx.x] = best;
        si[threadIdx.x] = arg;
        __syncthreads();
        for (int w = FIT_THREADS / 2; w > 0; w >>= 1) {
            if ((int)threadIdx.x < w) {
                const double vo = sv[threadIdx.x + w];
                const long long io = si[threadIdx.x + w];
                const bool take = io >= 0 && (si[threadIdx.x] < 0 || vo > sv[threadIdx.x] ||
                                              (vo == sv[threadIdx.x] && io < si[threadIdx.x]));
                if (take) {
                    sv[threadIdx.x] = vo;
                    si[threadIdx.x] = io;
                }
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            part[((long long)blockIdx.x * nphase + c) * 2] = sv[0];
            part[((long long)blockIdx.x * nphase + c) * 2 + 1] = (double)si[0];
        }
        __syncthreads();
    }
}

// Seed centroids from the block results (one thread per phase, blocks in order);
// out[nphase * N] receives -1 if some phase has no bulk site.
__global__ void k_fit_seed_finish(const double* __restrict__ phi, long long S, int N, int nphase,
                                  int nblocks, const double* __restrict__ part,
                                  double* __restrict__ cen, double* __restrict__ out)
{
    const int c = threadIdx.x;
    if (c >= nphase) return;
    double best = -DBL_MAX;
    long long arg = -1;
    for (int b = 0; b < nblocks; ++b) {
        const double v = part[((long long)b * nphase + c) * 2];
        const long long i = (long long)part[((long long)b * nphase + c) * 2 + 1];
        if (i >= 0 && (arg < 0 || v > best || (v == best && i < arg))) {
            best = v;
            arg = i;
        }
    }
    if (arg < 0) {
        out[nphase * N] = -1.0;
        return;
    }
    for (int s = 0; s < N; ++s) {
        cen[c * N + s] = phi[(long long)s * S + arg];
        out[c * N + s] = cen[c * N + s];
    }
    if (c == 0) out[nphase * N] = 0.0;
}

// One k-means pass: every bulk site joins its nearest centroid; per block, per phase,
// the site count and the N composition sums (part[b][c][0..N]).
__global__ void __launch_bounds__(FIT_THREADS)
k_fit_assign(const double* __restrict__ phi, const double* __restrict__ bulk, long long S, int N,
             int nphase, const double* __restrict__ cen, double* __restrict__ part)
{
    __shared__ double sc[NMAX * NMAX];
    __shared__ double red[FIT_THREADS];
    for (int k = threadIdx.x; k < nphase * N; k += blockDim.x) sc[k] = cen[k];
    __syncthreads();
    double acc[FIT_VALS];
    for (int k = 0; k < nphase * (N + 1); ++k) acc[k] = 0.0;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < S;
         t += (long long)gridDim.x * blockDim.x) {
        if (bulk[t] < 0.5) continue;
        double ph[NMAX];
        for (int s = 0; s < N; ++s) ph[s] = phi[(long long)s * S + t];
        int lab = 0;
        double bd = DBL_MAX;
        for (int c = 0; c < nphase; ++c) {
            double d = 0.0;
            for (int s = 0; s < N; ++s) {
                const double e = ph[s] - sc[c * N + s];
                d += e * e;
            }
            if (d < bd) {
                bd = d;
                lab = c;
            }
        }
        acc[lab * (N + 1)] += 1.0;
        for (int s = 0; s < N; ++s) acc[lab * (N + 1) + 1 + s] += ph[s];
    }
    for (int k = 0; k < nphase * (N + 1); ++k) {
        red[threadIdx.x] = acc[k];
        __syncthreads();
        for (int w = FIT_THREADS / 2; w > 0; w >>= 1) {
            if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) part[(long long)blockIdx.x * FIT_VALS + k] = red[0];
        __syncthreads();
    }
}

// New centroids from the block partials (phases with no site keep theirs); out receives
// them and, at [nphase * N], 1 if any centroid changed, else 0.
__global__ void k_fit_update(int N, int nphase, int nblocks, const double* __restrict__ part,
                             double* __restrict__ cen, double* __restrict__ out)
{
    __shared__ int changed;
    if (threadIdx.x == 0) changed = 0;
    __syncthreads();
    const int c = threadIdx.x;
    if (c < nphase) {
        double cnt = 0.0, sum[NMAX];
        for (int s = 0; s < N; ++s) sum[s] = 0.0;
        for (int b = 0; b < nblocks; ++b) {
            const double* pb = part + (long long)b * FIT_VALS + c * (N + 1);
            cnt += pb[0];
            for (int s = 0; s < N; ++s) sum[s] += pb[1 + s];
        }
        if (cnt > 0.0)
            for (int s = 0; s < N; ++s) {
                const double v = sum[s] / cnt;
                if (v != cen[c * N + s]) atomicOr(&changed, 1);
                cen[c * N + s] = v;
            }
        for (int s = 0; s < N; ++s) out[c * N + s] = cen[c * N + s];
    }
    __syncthreads();
    if (threadIdx.x == 0) out[nphase * N] = changed ? 1.0 : 0.0;
}

}  // namespace

size_t fit_work_doubles() { return (size_t)FIT_BLOCKS * FIT_VALS + 2 * NMAX * NMAX + 16; }

cudaError_t fit_phases(const double* phi, const double* bulk, int N, long long S, int nphase,
                       double* work, double* host_out, int* found, cudaStream_t st)
{
    double* part = work;
    double* cen = work + (size_t)FIT_BLOCKS * FIT_VALS;
    double* out = cen + NMAX * NMAX;
    const int nout = nphase * N + 1;
    k_fit_seed_blocks<<<FIT_BLOCKS, FIT_THREADS, 0, st>>>(phi, bulk, S, nphase, part);
    k_fit_seed_finish<<<1, 32, 0, st>>>(phi, S, N, nphase, FIT_BLOCKS, part, cen, out);
    cudaError_t e = cudaMemcpyAsync(host_out, out, sizeof(double) * nout, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    *found = host_out[nphase * N] >= 0.0;
    if (!*found) return cudaSuccess;
    for (int it = 0; it < 100; ++it) {
        k_fit_assign<<<FIT_BLOCKS, FIT_THREADS, 0, st>>>(phi, bulk, S, N, nphase, cen, part);
        k_fit_update<<<1, 32, 0, st>>>(N, nphase, FIT_BLOCKS, part, cen, out);
        e = cudaMemcpyAsync(host_out, out, sizeof(double) * nout, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return e;
        if (host_out[nphase * N] == 0.0) break;
    }
    return cudaGetLastError();
}

}  // namespace mclb
