// noalloc.cu -- mclb_step_noalloc: one FP64 timestep of the staged schedule for callers
// that cannot allocate device memory.
//
// The staged schedule needs two scratch fields (rho^s and nu^s, N values per site).
// The handle-based API allocates them per handle; here they live in one file-scope
// __device__ array of fixed size instead, so the call allocates nothing.  The
// distributions are caller-owned device arrays in the compact pre-collision layout
// of mclb_get_state ([s][i][y][x], FP64): f_in is read, f_out is written (streamed,
// i.e. the pre-collision state of the next time level).
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/mclb.h"
#include "staged.cuh"

namespace mclb {

int check_params(const mclb_params* p);     // capi.cu
int report(int code, const char* msg);      // capi.cu

namespace {

// Scratch of the allocation-free step: rho^s then nu^s, N * nx * ny doubles each.
constexpr long long NOALLOC_MAX = MCLB_NOALLOC_MAX_COMP_SITES;
static __device__ __align__(256) double g_noalloc_scratch[2 * NOALLOC_MAX];

// Device address of g_noalloc_scratch per device (host code must not pass the symbol
// itself to a kernel: on the host it only names a stand-in).  It is looked up again on
// every call made outside a stream capture, so that a device reset or a new context on
// the same device (which reloads the module at another address) is followed; inside a
// capture the address of the last call outside one is used.
constexpr int MAX_DEVICES = 64;
void* g_scratch_addr[MAX_DEVICES];
std::mutex g_scratch_mu;

int scratch_for_current_device(cudaStream_t st, double** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
        cudaGetLastError();
        return report(MCLB_ECUDA, "mclb_step_noalloc: no usable CUDA device");
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
        cudaGetLastError();
        return report(MCLB_ECUDA, "mclb_step_noalloc: cudaStreamIsCapturing failed");
    }
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (cap != cudaStreamCaptureStatusNone && !g_scratch_addr[dev])
        return report(MCLB_EINVAL, "mclb_step_noalloc: the first call on a device must come "
                                   "before any stream capture");
    if (cap == cudaStreamCaptureStatusNone) {
        void* ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) {
            char msg[256];
            snprintf(msg, sizeof(msg), "mclb_step_noalloc: cudaGetSymbolAddress failed: %s",
                     cudaGetErrorString(e));
            cudaGetLastError();
            return report(MCLB_ECUDA, msg);
        }
        g_scratch_addr[dev] = ptr;
    }
    *out = static_cast<double*>(g_scratch_addr[dev]);
    return MCLB_OK;
}

// rho^s from the local pre-collision populations (same summation order as k_density).
template <int N>
__global__ void __launch_bounds__(SITE_THREADS)
k_na_density(const double* __restrict__ f, double* __restrict__ rs, const __grid_constant__ StepParams<double> p)
{
    const long long site = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (site >= p.S) return;
#pragma unroll
    for (int s = 0; s < N; ++s) {
        double r = 0.0;
#pragma unroll
        for (int i = 0; i < Q; ++i) r += f[(long long)(s * Q + i) * p.S + site];
        rs[s * p.S + site] = r;
    }
}

// Collision at the site, then streaming by writing each population to x + v_i.
template <int N>
__global__ void __launch_bounds__(SITE_THREADS)
k_na_collide(const double* __restrict__ fin, double* __restrict__ fout, const double* __restrict__ nu,
             const __grid_constant__ StepParams<double> p)
{
    const long long site = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (site >= p.S) return;
    const int y = (int)(site / p.nx), x = (int)(site - (long long)y * p.nx);
    double f[N][Q], r[N], jx[N], jy[N];
    double rho = 0.0, jxt = 0.0, jyt = 0.0;
#pragma unroll
    for (int s = 0; s < N; ++s) {
        double a = 0.0, bx = 0.0, by = 0.0;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const double v = fin[(long long)(s * Q + i) * p.S + site];
            f[s][i] = v;
            a += v;
            bx += v * double(vx(i));
            by += v * double(vy(i));
        }
        r[s] = a;
        jx[s] = bx;
        jy[s] = by;
        rho += a;
        jxt += bx;
        jyt += by;
    }
    double e[Q];
    eq_weights(jxt / rho, jyt / rho, e);
#pragma unroll
    for (int s = 0; s < N; ++s) {
        double gx, gy;
        field_grad(nu + s * p.S, p, x, y, gx, gy);
        double out[Q], fjx, fjy;
        forcing_momentum(p, r[s], jx[s], jy[s], jxt / rho, jyt / rho, fjx, fjy);
        collide(p, f[s], e, r[s], fjx, fjy, -p.fcoef * gx + p.gx, -p.fcoef * gy + p.gy, out);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int xx = wrap_add(x, vx(i), p.nx), yy = wrap_add(y, vy(i), p.ny);
            fout[(long long)(s * Q + i) * p.S + (long long)yy * p.nx + xx] = out[i];
        }
    }
}

template <int N>
cudaError_t launch(const StepParams<double>& p, const double* fin, double* fout, double* scratch,
                   cudaStream_t st)
{
    double* rs = scratch;
    double* nu = scratch + N * p.S;
    const unsigned blocks = (unsigned)((p.S + SITE_THREADS - 1) / SITE_THREADS);
    k_na_density<N><<<blocks, SITE_THREADS, 0, st>>>(fin, rs, p);
    k_potential<double, N><<<blocks, SITE_THREADS, 0, st>>>(rs, nu, p);
    k_na_collide<N><<<blocks, SITE_THREADS, 0, st>>>(fin, fout, nu, p);
    return cudaGetLastError();
}

}  // namespace
}  // namespace mclb

using namespace mclb;

extern "C" int mclb_step_noalloc(const mclb_params* params, const double* f_in, double* f_out)
{
    int rc = check_params(params);
    if (rc) return rc;
    if (params->precision != MCLB_FP64)
        return report(MCLB_EINVAL, "mclb_step_noalloc: only precision MCLB_FP64 is supported");
    if (params->walls != 0)
        return report(MCLB_EINVAL, "mclb_step_noalloc: the lattice must be periodic (walls = 0)");
    if (params->mass_every != 0)
        return report(MCLB_EINVAL, "mclb_step_noalloc: mass_every must be 0 (one step, no handle)");
    if (params->lattice != MCLB_D2Q9)
        return report(MCLB_EINVAL, "mclb_step_noalloc: only the D2Q9 lattice is supported");
    if (params->force_form != MCLB_FORCE_COMPONENT)
        return report(MCLB_EINVAL, "mclb_step_noalloc: only the component forces of Eq. definef");
    const long long S = (long long)params->nx * params->ny;
    if (!f_in || !f_out)
        return report(MCLB_EINVAL, "mclb_step_noalloc: f_in and f_out must be device arrays");
    if ((long long)params->ncomp * S > NOALLOC_MAX) {
        char msg[256];
        snprintf(msg, sizeof(msg),
                 "mclb_step_noalloc: ncomp * nx * ny = %lld exceeds the fixed scratch of %lld",
                 (long long)params->ncomp * S, NOALLOC_MAX);
        return report(MCLB_EINVAL, msg);
    }
    {
        // the collision scatters into f_out while other threads still read f_in: the two
        // ranges of N * 9 * nx * ny doubles must not overlap at all
        const unsigned long long n = (unsigned long long)params->ncomp * Q * (unsigned long long)S;
        const uintptr_t a = reinterpret_cast<uintptr_t>(f_in), b = reinterpret_cast<uintptr_t>(f_out);
        if (a < b + n * sizeof(double) && b < a + n * sizeof(double))
            return report(MCLB_EINVAL, "mclb_step_noalloc: f_in and f_out overlap");
    }
    double* scratch = nullptr;
    rc = scratch_for_current_device((cudaStream_t)params->stream, &scratch);
    if (rc) return rc;

    Problem P;
    memset(&P, 0, sizeof(P));
    P.N = params->ncomp;
    P.nx = params->nx;
    P.ny = params->ny;
    P.S = S;
    P.pitch = params->nx;
    P.plane = S;
    P.tau = params->tau;
    P.theta = params->theta > 0.0 ? params->theta : 1.0 / 3.0;
    P.kappa = params->kappa;
    P.gx = params->force[0];
    P.gy = params->force[1];
    P.forcing_velocity = params->forcing_velocity;
    for (int a = 0; a < P.N; ++a) {
        for (int b = 0; b < P.N; ++b) P.chi[a * P.N + b] = params->chi[a * P.N + b];
        P.m[a] = params->m ? params->m[a] : 1.0;
    }
    const StepParams<double> p = make_params<double>(P, nullptr);
    const cudaStream_t st = (cudaStream_t)params->stream;
    cudaError_t e;
    switch (P.N) {
        case 1: e = launch<1>(p, f_in, f_out, scratch, st); break;
        case 2: e = launch<2>(p, f_in, f_out, scratch, st); break;
        case 3: e = launch<3>(p, f_in, f_out, scratch, st); break;
        case 4: e = launch<4>(p, f_in, f_out, scratch, st); break;
        case 5: e = launch<5>(p, f_in, f_out, scratch, st); break;
        case 6: e = launch<6>(p, f_in, f_out, scratch, st); break;
        case 7: e = launch<7>(p, f_in, f_out, scratch, st); break;
        default: e = launch<8>(p, f_in, f_out, scratch, st); break;
    }
    if (e != cudaSuccess) {
        char msg[256];
        snprintf(msg, sizeof(msg), "mclb_step_noalloc: launch failed: %s", cudaGetErrorString(e));
        return report(MCLB_ECUDA, msg);
    }
    return MCLB_OK;
}
