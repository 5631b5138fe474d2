// checks.cu -- validation of FP64 boundary data on the device (the C ABI checks the
// fields and states a caller hands over here, after their upload, before they touch
// a handle's state).
#include <climits>

#include "mclb_internal.h"

namespace mclb {

namespace {

constexpr int CHECK_THREADS = 256;
constexpr int CHECK_BLOCKS = 1216;   // 8 per SM on a 152-SM part; grid-stride beyond

// smallest site whose N densities are not all finite, whose total is not positive, or
// whose velocity (ud components; u may be null) is not finite
__global__ void __launch_bounds__(CHECK_THREADS)
k_check_fields(const double* __restrict__ rho, const double* __restrict__ u, int N, int ud,
               long long S, unsigned long long* first_bad)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < S; c += stride) {
        double tot = 0.0;
        bool ok = true;
        for (int s = 0; s < N; ++s) {
            const double v = rho[s * S + c];
            ok = ok && isfinite(v);
            tot += v;
        }
        ok = ok && tot > 0.0;
        if (u)
            for (int d = 0; d < ud; ++d) ok = ok && isfinite(u[d * S + c]);
        if (!ok) atomicMin(first_bad, (unsigned long long)c);
    }
}

__global__ void __launch_bounds__(CHECK_THREADS)
k_check_finite(const double* __restrict__ a, long long n, unsigned long long* first_bad)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride)
        if (!isfinite(a[k])) atomicMin(first_bad, (unsigned long long)k);
}

}  // namespace

cudaError_t check_fields(const double* rho, const double* u, int N, int ud, long long S,
                         unsigned long long* first_bad, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(first_bad, 0xff, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    k_check_fields<<<CHECK_BLOCKS, CHECK_THREADS, 0, st>>>(rho, u, N, ud, S, first_bad);
    return cudaGetLastError();
}

cudaError_t check_finite(const double* a, long long n, unsigned long long* first_bad,
                         cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(first_bad, 0xff, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    k_check_finite<<<CHECK_BLOCKS, CHECK_THREADS, 0, st>>>(a, n, first_bad);
    return cudaGetLastError();
}

}  // namespace mclb
