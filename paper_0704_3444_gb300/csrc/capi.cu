// capi.cu -- the C ABI declared in include/mclb.h: handle lifetime, validation,
// device buffers, TMA descriptors, CUDA-graph replay of timestep chunks and
// status reporting.  All arithmetic of the method runs in the kernels of the
// prec_*.cu units; this file only orchestrates.
#include <cudaTypedefs.h>

#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/mclb.h"
#include "mclb_internal.h"

using namespace mclb;

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CK(call)                                                                           \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail(MCLB_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                        __FILE__, __LINE__);                                               \
    } while (0)

constexpr uint32_t MAGIC = 0x4d434c42u;  // "MCLB"
constexpr uint32_t DEAD = 0xdeadbeefu;
constexpr int GRAPH_STEPS = 32;          // timesteps per captured graph (even)

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

const KernelTable& table_for(int precision)
{
    switch (precision) {
        case MCLB_FP64: return table_fp64();
        case MCLB_BF16_SHIFTED: return table_bf16();
        case MCLB_FP16_SHIFTED: return table_fp16();
        default: return table_fp32();
    }
}

// velocities per site and velocity components of a problem's lattice
int lattice_q(const Problem& P)
{
    return P.lattice == MCLB_D1Q3 ? 3 : (P.lattice == MCLB_D3Q19 ? 19 : Q);
}
int vel_dims(const Problem& P) { return P.lattice == MCLB_D3Q19 ? 3 : 2; }

int validate(const mclb_params* p)
{
    if (!p) return fail(MCLB_EINVAL, "params is NULL");
    if (p->ncomp < 1 || p->ncomp > MCLB_NMAX)
        return fail(MCLB_EINVAL, "ncomp=%d outside 1..%d", p->ncomp, MCLB_NMAX);
    if (p->nx < 1 || p->ny < 1) return fail(MCLB_EINVAL, "grid %dx%d invalid", p->nx, p->ny);
    if ((long long)p->nx * p->ny > (1LL << 31))
        return fail(MCLB_EINVAL, "grid %dx%d exceeds 2^31 sites", p->nx, p->ny);
    if (!(p->tau > 0.5) || !std::isfinite(p->tau))
        return fail(MCLB_EINVAL, "tau=%g must be finite and > 1/2", p->tau);
    if (!p->chi) return fail(MCLB_EINVAL, "chi is NULL");
    const int N = p->ncomp;
    for (int a = 0; a < N; ++a)
        for (int b = 0; b < N; ++b) {
            const double v = p->chi[a * N + b];
            if (!std::isfinite(v)) return fail(MCLB_EINVAL, "chi[%d][%d] not finite", a, b);
            if (v != p->chi[b * N + a])
                return fail(MCLB_EINVAL, "chi not symmetric at (%d,%d)", a, b);
        }
    if (p->m)
        for (int a = 0; a < N; ++a)
            if (!(p->m[a] > 0.0) || !std::isfinite(p->m[a]))
                return fail(MCLB_EINVAL, "m[%d]=%g must be finite and > 0", a, p->m[a]);
    if (!std::isfinite(p->theta)) return fail(MCLB_EINVAL, "theta not finite");
    if (!std::isfinite(p->kappa) || p->kappa < 0.0)
        return fail(MCLB_EINVAL, "kappa=%g must be finite and >= 0", p->kappa);
    if (!std::isfinite(p->force[0]) || !std::isfinite(p->force[1]))
        return fail(MCLB_EINVAL, "force not finite");
    if (p->precision < MCLB_FP64 || p->precision > MCLB_FP16_SHIFTED)
        return fail(MCLB_EINVAL, "precision=%d unknown", p->precision);
    if (p->kernel < MCLB_KERNEL_AUTO || p->kernel > MCLB_KERNEL_STAGED)
        return fail(MCLB_EINVAL, "kernel=%d unknown", p->kernel);
    if (p->forcing_velocity != MCLB_FORCING_COMPONENT && p->forcing_velocity != MCLB_FORCING_BARYCENTRIC)
        return fail(MCLB_EINVAL, "forcing_velocity=%d unknown", p->forcing_velocity);
    if (p->lattice != MCLB_D2Q9 && p->lattice != MCLB_D1Q3 && p->lattice != MCLB_D3Q19)
        return fail(MCLB_EINVAL, "lattice=%d unknown", p->lattice);
    if (p->nz < 0) return fail(MCLB_EINVAL, "nz=%d must be >= 0", p->nz);
    if (p->lattice != MCLB_D3Q19 && p->nz > 1)
        return fail(MCLB_EINVAL, "nz=%d > 1 needs the D3Q19 lattice", p->nz);
    if (!std::isfinite(p->force_z)) return fail(MCLB_EINVAL, "force_z not finite");
    if (p->lattice != MCLB_D3Q19 && p->force_z != 0.0)
        return fail(MCLB_EINVAL, "force_z != 0 needs the D3Q19 lattice");
    if ((long long)p->nx * p->ny * (p->nz > 1 ? p->nz : 1) > (1LL << 31))
        return fail(MCLB_EINVAL, "grid %dx%dx%d exceeds 2^31 sites", p->nx, p->ny, p->nz);
    if (p->force_form != MCLB_FORCE_COMPONENT && p->force_form != MCLB_FORCE_GIBBS_DUHEM)
        return fail(MCLB_EINVAL, "force_form=%d unknown", p->force_form);
    if (p->force_form == MCLB_FORCE_GIBBS_DUHEM) {
        if (p->kappa != 0.0)
            return fail(MCLB_EINVAL, "the Gibbs-Duhem force form is defined for kappa = 0");
    }
    if (p->mass_every < 0) return fail(MCLB_EINVAL, "mass_every=%d must be >= 0", p->mass_every);
    if (p->walls != 0 && p->walls != 1) return fail(MCLB_EINVAL, "walls=%d unknown", p->walls);
    if (p->walls && p->lattice != MCLB_D2Q9)
        return fail(MCLB_EINVAL, "walls are a D2Q9 option (lattice=%d)", p->lattice);
    if (p->lattice == MCLB_D3Q19 && p->precision != MCLB_FP64 && p->precision != MCLB_FP32)
        return fail(MCLB_EINVAL, "lattice D3Q19 stores FP64 or FP32 (precision=%d)", p->precision);
    if (p->lattice == MCLB_D1Q3) {
        if (p->ny != 1) return fail(MCLB_EINVAL, "lattice D1Q3 needs ny = 1 (ny=%d)", p->ny);
        if (p->precision != MCLB_FP64 && p->precision != MCLB_FP32)
            return fail(MCLB_EINVAL, "lattice D1Q3 stores FP64 or FP32 (precision=%d)", p->precision);
    }
    return MCLB_OK;
}

void fill_problem(const mclb_params* p, const KernelTable& tab, Problem& P)
{
    // ghost columns only in the D2Q9 layout (the D1Q3 and D3Q19 kernels wrap by index)
    const int hx = p->lattice == MCLB_D2Q9 ? tab.hx : 0;
    memset(&P, 0, sizeof(P));
    P.N = p->ncomp;
    P.nx = p->nx;
    P.ny = p->ny;
    P.nz = (p->lattice == MCLB_D3Q19 && p->nz > 1) ? p->nz : 1;
    P.S = (long long)p->nx * p->ny * P.nz;
    P.hx = hx;
    P.pitch = 2LL * hx + (long long)((p->nx + ROW_ALIGN - 1) / ROW_ALIGN) * ROW_ALIGN;
    P.plane = P.pitch * Q * p->ny;
    P.lattice = p->lattice;
    if (P.lattice == MCLB_D1Q3) {   // compact [s][3][nx], no ghost columns
        P.pitch = p->nx;
        P.plane = 3LL * p->nx;
    }
    if (P.lattice == MCLB_D3Q19) {  // compact [s][z][y][19][x], no ghost columns
        P.pitch = p->nx;
        P.plane = 19LL * P.S;
    }
    // 16-bit formats: the FP32 density lines follow the deviations, 256-byte aligned
    P.rbytes = tab.shifted ? (long long)((P.plane * P.N * (long long)tab.storage_bytes + 255) / 256 * 256) : 0;
    P.tau = p->tau;
    P.theta = p->theta > 0.0 ? p->theta : 1.0 / 3.0;
    P.kappa = p->kappa;
    P.gx = p->force[0];
    P.gy = p->force[1];
    P.gz = p->force_z;
    P.forcing_velocity = p->forcing_velocity;
    P.force_form = p->force_form;
    P.mass_every = p->mass_every;
    P.walls = p->walls;
    for (int a = 0; a < P.N; ++a) {
        for (int b = 0; b < P.N; ++b) P.chi[a * P.N + b] = p->chi[a * P.N + b];
        P.m[a] = p->m ? p->m[a] : 1.0;
    }
}

}  // namespace

namespace mclb {
// Parameter validation and error reporting shared with the allocation-free entry point.
int check_params(const mclb_params* p) { return validate(p); }
int report(int code, const char* msg) { return fail(code, "%s", msg); }
}  // namespace mclb

struct mclb_handle_s {
    uint32_t magic;
    int precision, kernel;
    const KernelTable* tab;
    Problem P;
    Scratch sc;
    FusedPlan plan;
    bool fused;
    const LatticeTable* alt;      // D1Q3 and D3Q19 handles: their kernels (null for D2Q9)
    cudaStream_t stream;
    bool own_stream;
    void* f[2];
    CUtensorMap tmap[2];
    CUtensorMap tmapr[2];         // density lines of the 16-bit formats
    CUtensorMap tmapw[2];         // columns [0, nx) of the lines, for the kernel's box stores
    CUtensorMap tmapwr[2];        // the same for the density lines of the 16-bit formats
    int cur;                      // buffer holding the current state
    long steps;
    long since_mass;              // steps since the last mass compensation
    size_t fbytes;                // bytes of one distribution buffer
    unsigned int* status_host;    // pinned mirror of the device status word
    cudaEvent_t status_event;     // the mirror's copy has landed
    bool status_pending;
    // the status word is copied on its own stream, after an event that marks the work
    // queued so far, so that the next step's kernels do not wait behind the copy
    cudaStream_t status_stream;
    cudaEvent_t queued;
    cudaGraphExec_t graph[2];     // GRAPH_STEPS steps starting from buffer 0 / 1
    bool graph_tried[2];
    double* dtmp;                 // device FP64 staging for host copies
    size_t dtmp_cap;
};

namespace {

int check_handle(mclb_handle h)
{
    if (!h) return fail(MCLB_EHANDLE, "handle is NULL");
    if (h->magic != MAGIC) return fail(MCLB_EHANDLE, "handle destroyed or not a handle");
    return MCLB_OK;
}

int status_code(unsigned int s)
{
    if (s & STATUS_TIMEOUT) return fail(MCLB_ETIMEOUT, "a bounded device wait gave up");
    if (s & STATUS_NONFINITE)
        return fail(MCLB_ENONFINITE, "non-finite value or non-positive total density");
    return MCLB_OK;
}

int ensure_dtmp(mclb_handle h, size_t doubles)
{
    if (h->dtmp_cap >= doubles) return MCLB_OK;
    if (h->dtmp) cudaFree(h->dtmp);
    h->dtmp = nullptr;
    h->dtmp_cap = 0;
    if (cudaMalloc(&h->dtmp, doubles * sizeof(double)) != cudaSuccess)
        return fail(MCLB_ENOMEM, "device staging of %zu bytes failed", doubles * sizeof(double));
    h->dtmp_cap = doubles;
    return MCLB_OK;
}

// The four views of buffer b with load boxes of box_w columns and store boxes of out_w
// columns (0: no store views): v[0] load, v[1] density-line load (16-bit formats), v[2]
// store, v[3] density-line store (16-bit formats).
int encode_views(mclb_handle h, int b, int box_w, int out_w, CUtensorMap* const* v)
{
    auto fn = encode_fn();
    if (!fn) return fail(MCLB_ECUDA, "cuTensorMapEncodeTiled unavailable");
    const Problem& P = h->P;
    const size_t sz = h->tab->storage_bytes;
    // 4-D view (x, velocity, row, component); one box = one velocity line of one row,
    // all components, box_w columns.  The view ends after the right ghost columns, so the
    // part of a box beyond them (line padding) is filled with zeros, not read from memory.
    cuuint64_t dims[4] = {(cuuint64_t)(P.nx + 2 * P.hx), (cuuint64_t)Q, (cuuint64_t)P.ny, (cuuint64_t)P.N};
    cuuint64_t strides[3] = {(cuuint64_t)(P.pitch * sz), (cuuint64_t)(Q * P.pitch * sz),
                             (cuuint64_t)(P.plane * sz)};
    cuuint32_t box[4] = {(cuuint32_t)box_w, 1u, 1u, (cuuint32_t)P.N};
    cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
    CUresult r = fn(v[0], h->tab->tma_type, 4, h->f[b], dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(MCLB_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    if (out_w > 0) {
        // the same 4-D view ending at column nx (boxes that reach past it are clipped):
        // one box = out_w columns of the 9 lines of one row, all components
        cuuint64_t wdims[4] = {(cuuint64_t)(P.nx + P.hx), (cuuint64_t)Q, (cuuint64_t)P.ny, (cuuint64_t)P.N};
        cuuint32_t wbox[4] = {(cuuint32_t)out_w, (cuuint32_t)Q, 1u, (cuuint32_t)P.N};
        r = fn(v[2], h->tab->tma_type, 4, h->f[b], wdims, strides, wbox, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS)
            return fail(MCLB_ECUDA, "cuTensorMapEncodeTiled (store view) failed (%d)", (int)r);
        if (h->tab->shifted) {
            cuuint64_t rdims[3] = {(cuuint64_t)(P.nx + P.hx), (cuuint64_t)P.ny, (cuuint64_t)P.N};
            cuuint64_t rstrides[2] = {(cuuint64_t)(P.pitch * sizeof(float)),
                                      (cuuint64_t)(P.ny * P.pitch * sizeof(float))};
            cuuint32_t rbox[3] = {(cuuint32_t)out_w, 1u, (cuuint32_t)P.N};
            r = fn(v[3], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                   static_cast<char*>(h->f[b]) + P.rbytes, rdims, rstrides, rbox, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS)
                return fail(MCLB_ECUDA, "cuTensorMapEncodeTiled (density store view) failed (%d)", (int)r);
        }
    }
    if (h->tab->shifted) {
        // 3-D view (x, row, component) of the FP32 density lines; same columns per box
        cuuint64_t rdims[3] = {(cuuint64_t)(P.nx + 2 * P.hx), (cuuint64_t)P.ny, (cuuint64_t)P.N};
        cuuint64_t rstrides[2] = {(cuuint64_t)(P.pitch * sizeof(float)),
                                  (cuuint64_t)(P.ny * P.pitch * sizeof(float))};
        cuuint32_t rbox[3] = {(cuuint32_t)box_w, 1u, (cuuint32_t)P.N};
        r = fn(v[1], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
               static_cast<char*>(h->f[b]) + P.rbytes, rdims, rstrides, rbox, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS)
            return fail(MCLB_ECUDA, "cuTensorMapEncodeTiled (density lines) failed (%d)", (int)r);
    }
    return MCLB_OK;
}

int make_tmap(mclb_handle h, int b)
{
    CUtensorMap* const v[4] = {&h->tmap[b], &h->tmapr[b], &h->tmapw[b], &h->tmapwr[b]};
    return encode_views(h, b, h->plan.box_w, h->plan.out_w, v);
}

cudaError_t launch_one_step(mclb_handle h, int from)
{
    const Problem& P = h->P;
    if (h->fused)
        return h->tab->step_fused(P, h->sc, h->plan, &h->tmap[from], &h->tmapr[from],
                                  &h->tmapw[from ^ 1], &h->tmapwr[from ^ 1], h->f[from],
                                  h->f[from ^ 1], h->stream);
    return h->tab->step_staged(P, h->sc, h->f[from], h->f[from ^ 1], h->stream);
}

void try_capture(mclb_handle h, int from)
{
    h->graph_tried[from] = true;
    h->graph[from] = nullptr;
    if (h->stream == nullptr) return;
    if (cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    int b = from;
    bool ok = true;
    for (int k = 0; k < GRAPH_STEPS && ok; ++k) {
        ok = launch_one_step(h, b) == cudaSuccess;
        b ^= 1;
    }
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(h->stream, &g);
    if (ok && e == cudaSuccess && g) {
        cudaGraphExec_t ex = nullptr;
        if (cudaGraphInstantiate(&ex, g, 0) == cudaSuccess) h->graph[from] = ex;
    }
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
}

int enqueue_status_copy(mclb_handle h)
{
    CK(cudaEventRecord(h->queued, h->stream));
    CK(cudaStreamWaitEvent(h->status_stream, h->queued, 0));
    CK(cudaMemcpyAsync(h->status_host, h->sc.status, sizeof(unsigned int),
                       cudaMemcpyDeviceToHost, h->status_stream));
    CK(cudaEventRecord(h->status_event, h->status_stream));
    h->status_pending = true;
    return MCLB_OK;
}

// A status copy still in flight lands before the status word is cleared.
int settle_status(mclb_handle h)
{
    if (h->status_pending) {
        CK(cudaEventSynchronize(h->status_event));
        h->status_pending = false;
    }
    return MCLB_OK;
}

// The mass compensation's reference: each component's mass of the state just set.
int record_mass(mclb_handle h)
{
    h->since_mass = 0;
    if (h->P.mass_every > 0) CK(h->tab->mass(h->P, h->sc, h->f[h->cur], 1, h->stream));
    return MCLB_OK;
}

// nsteps timesteps, graph-replayed in GRAPH_STEPS chunks where possible.
int advance(mclb_handle h, long nsteps)
{
    if (h->alt) {
        CK(h->alt->step(h->P, h->sc, h->f, &h->cur, nsteps, h->stream));
        return MCLB_OK;
    }
    long left = nsteps;
    while (left >= GRAPH_STEPS && !h->P.withhold) {
        if (!h->graph_tried[h->cur]) try_capture(h, h->cur);
        if (!h->graph[h->cur]) break;
        CK(cudaGraphLaunch(h->graph[h->cur], h->stream));
        left -= GRAPH_STEPS;
    }
    for (; left > 0; --left) {
        CK(launch_one_step(h, h->cur));
        h->cur ^= 1;
    }
    return MCLB_OK;
}

int sync_status(mclb_handle h)
{
    int rc = enqueue_status_copy(h);
    if (rc) return rc;
    CK(cudaEventSynchronize(h->status_event));
    h->status_pending = false;
    return status_code(*h->status_host);
}

}  // namespace

extern "C" {

const char* mclb_last_error(void) { return g_err.c_str(); }

int mclb_create(const mclb_params* params, mclb_handle* out)
{
    if (!out) return fail(MCLB_EINVAL, "out is NULL");
    *out = nullptr;
    int rc = validate(params);
    if (rc) return rc;
    mclb_handle h = new (std::nothrow) mclb_handle_s();
    if (!h) return fail(MCLB_ENOMEM, "host allocation failed");
    memset(h, 0, sizeof(*h));
    h->precision = params->precision;
    h->kernel = params->kernel;
    h->tab = &table_for(params->precision);
    fill_problem(params, *h->tab, h->P);
    const Problem& P = h->P;
    auto bail = [&](int code) {
        h->magic = MAGIC;
        mclb_destroy(h);
        return code;
    };
    int dev = 0, sms = 1;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(MCLB_ECUDA, "no usable CUDA device"));
    }
    if (params->stream) {
        h->stream = (cudaStream_t)params->stream;
    } else {
        if (cudaStreamCreate(&h->stream) != cudaSuccess)
            return bail(fail(MCLB_ECUDA, "cudaStreamCreate failed"));
        h->own_stream = true;
    }
    h->fbytes = (size_t)P.plane * P.N * h->tab->storage_bytes;
    if (h->tab->shifted) h->fbytes = (size_t)P.rbytes + (size_t)P.N * P.ny * P.pitch * sizeof(float);
    if (P.lattice == MCLB_D1Q3) {
        h->alt = h->tab->line3;
        if (!h->alt) return bail(fail(MCLB_EINVAL, "no D1Q3 kernels for this precision"));
    }
    if (P.lattice == MCLB_D3Q19) {
        h->alt = h->tab->d3q19;
        if (!h->alt) return bail(fail(MCLB_EINVAL, "no D3Q19 kernels for this precision"));
    }
    const size_t jbytes = (P.lattice == MCLB_D3Q19)
                              ? (size_t)3 * P.N * P.S * ((h->precision == MCLB_FP64) ? sizeof(double) : sizeof(float))
                              : 0;
    if (jbytes && cudaMalloc(&h->sc.js, jbytes) != cudaSuccess)
        return bail(fail(MCLB_ENOMEM, "D3Q19 momentum scratch"));
    const size_t cbytes = (h->precision == MCLB_FP64) ? sizeof(double) : sizeof(float);
    for (int b = 0; b < 2; ++b) {
        if (cudaMalloc(&h->f[b], h->fbytes) != cudaSuccess)
            return bail(fail(MCLB_ENOMEM, "distribution buffer of %zu bytes", h->fbytes));
        // on the handle's stream: a stream created non-blocking is not ordered with the
        // legacy default stream, so a plain cudaMemset could land after the first init
        if (cudaMemsetAsync(h->f[b], 0, h->fbytes, h->stream) != cudaSuccess)
            return bail(fail(MCLB_ECUDA, "cudaMemset failed"));
    }
    if (cudaMalloc(&h->sc.rho_s, (size_t)P.N * P.S * cbytes) != cudaSuccess ||
        cudaMalloc(&h->sc.nu, (size_t)P.N * P.S * cbytes) != cudaSuccess)
        return bail(fail(MCLB_ENOMEM, "scratch fields"));
    h->sc.partial_cap = (size_t)REDUCE_BLOCKS * (NMAX + 6) + 64;
    if (cudaMalloc(&h->sc.partial, h->sc.partial_cap * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&h->sc.status, sizeof(unsigned int)) != cudaSuccess ||
        cudaMalloc(&h->sc.mass_ref, NMAX * sizeof(double)) != cudaSuccess)
        return bail(fail(MCLB_ENOMEM, "reduction scratch"));
    if (cudaMemsetAsync(h->sc.status, 0, sizeof(unsigned int), h->stream) != cudaSuccess)
        return bail(fail(MCLB_ECUDA, "cudaMemset failed"));
    if (cudaMallocHost(&h->status_host, sizeof(unsigned int)) != cudaSuccess)
        return bail(fail(MCLB_ENOMEM, "pinned status word"));
    *h->status_host = 0;
    if (cudaEventCreateWithFlags(&h->status_event, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->queued, cudaEventDisableTiming) != cudaSuccess)
        return bail(fail(MCLB_ECUDA, "cudaEventCreate failed"));
    if (cudaStreamCreateWithFlags(&h->status_stream, cudaStreamNonBlocking) != cudaSuccess)
        return bail(fail(MCLB_ECUDA, "cudaStreamCreate failed"));
    h->fused = false;
    if (h->alt) {
        if (h->alt->item_bytes > 0 && cudaMalloc(&h->sc.line_item, h->alt->item_bytes) != cudaSuccess)
            return bail(fail(MCLB_ENOMEM, "D1Q3 line description"));
        // the upload is a plain cudaMemcpy (legacy default stream), which may return before
        // the copy lands: wait for it, since the handle's stream need not be ordered with it
        if (h->alt->prepare(P, h->sc, h->f) != cudaSuccess ||
            cudaStreamSynchronize(cudaStreamLegacy) != cudaSuccess)
            return bail(fail(MCLB_ECUDA, "D1Q3 line description upload failed"));
        if (h->alt->plan && h->kernel != MCLB_KERNEL_STAGED) {
            const int r = h->alt->plan(h->P, sms);
            if (r < 0) return bail(fail(MCLB_ECUDA, "single-pass kernel set-up failed"));
            h->fused = r == 1;
            if (!h->fused && h->kernel == MCLB_KERNEL_FUSED)
                return bail(fail(MCLB_EINVAL, "fused kernel unavailable for this problem"));
        }
    } else if (h->kernel != MCLB_KERNEL_STAGED) {
        h->plan = h->tab->plan_fused(P, sms);
        if (h->plan.ok && make_tmap(h, 0) == MCLB_OK && make_tmap(h, 1) == MCLB_OK) h->fused = true;
        if (!h->fused && h->kernel == MCLB_KERNEL_FUSED)
            return bail(fail(MCLB_EINVAL, "fused kernel unavailable for this problem"));
    }
    cudaGetLastError();
    if (cudaStreamSynchronize(h->stream) != cudaSuccess)   // the zeroed buffers and status
        return bail(fail(MCLB_ECUDA, "stream synchronisation after set-up failed"));
    h->magic = MAGIC;
    *out = h;
    return MCLB_OK;
}

int mclb_destroy(mclb_handle h)
{
    if (!h) return MCLB_OK;
    if (h->magic != MAGIC) return fail(MCLB_EHANDLE, "handle destroyed or not a handle");
    // queued steps and a status copy still in flight finish before anything is freed
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->status_stream) cudaStreamSynchronize(h->status_stream);
    for (int b = 0; b < 2; ++b) {
        if (h->graph[b]) cudaGraphExecDestroy(h->graph[b]);
        if (h->f[b]) cudaFree(h->f[b]);
    }
    if (h->sc.rho_s) cudaFree(h->sc.rho_s);
    if (h->sc.nu) cudaFree(h->sc.nu);
    if (h->sc.partial) cudaFree(h->sc.partial);
    if (h->sc.status) cudaFree(h->sc.status);
    if (h->sc.line_item) cudaFree(h->sc.line_item);
    if (h->sc.mass_ref) cudaFree(h->sc.mass_ref);
    if (h->sc.js) cudaFree(h->sc.js);
    if (h->dtmp) cudaFree(h->dtmp);
    if (h->status_host) cudaFreeHost(h->status_host);
    if (h->status_event) cudaEventDestroy(h->status_event);
    if (h->queued) cudaEventDestroy(h->queued);
    if (h->status_stream) cudaStreamDestroy(h->status_stream);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    h->magic = DEAD;
    delete h;
    return MCLB_OK;
}

static int init_common(mclb_handle h, const double* rho_d, const double* u_d)
{
    int rc = settle_status(h);
    if (rc) return rc;
    CK(cudaMemsetAsync(h->sc.status, 0, sizeof(unsigned int), h->stream));
    if (h->alt)
        CK(h->alt->init(h->P, h->sc, rho_d, u_d, h->f[0], h->stream));
    else
        CK(h->tab->init(h->P, h->sc, rho_d, u_d, h->f[0], h->stream));
    h->cur = 0;
    h->steps = 0;
    return record_mass(h);
}

int mclb_init_fields(mclb_handle h, const double* rho, const double* u)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (!rho) return fail(MCLB_EINVAL, "rho is NULL");
    const Problem& P = h->P;
    // upload, then check on the device; the state is touched only if every site passes
    const int ud = vel_dims(P);
    rc = ensure_dtmp(h, (size_t)(P.N + ud) * P.S + 1);
    if (rc) return rc;
    CK(cudaMemcpyAsync(h->dtmp, rho, sizeof(double) * P.N * P.S, cudaMemcpyHostToDevice,
                       h->stream));
    if (u)
        CK(cudaMemcpyAsync(h->dtmp + P.N * P.S, u, sizeof(double) * ud * P.S,
                           cudaMemcpyHostToDevice, h->stream));
    unsigned long long* d_bad = reinterpret_cast<unsigned long long*>(h->dtmp + (P.N + ud) * P.S);
    CK(check_fields(h->dtmp, u ? h->dtmp + P.N * P.S : nullptr, P.N, ud, P.S, d_bad, h->stream));
    unsigned long long bad = 0;
    CK(cudaMemcpyAsync(&bad, d_bad, sizeof(bad), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (bad != ULLONG_MAX) {   // name the first failing site and what failed there
        const long long c = (long long)bad;
        double tot = 0.0;
        for (int s = 0; s < P.N; ++s) {
            const double v = rho[s * P.S + c];
            if (!std::isfinite(v)) return fail(MCLB_EINVAL, "rho not finite at site %lld", c);
            tot += v;
        }
        if (!(tot > 0.0)) return fail(MCLB_EINVAL, "total density <= 0 at site %lld", c);
        return fail(MCLB_EINVAL, "u not finite at site %lld", c);
    }
    rc = init_common(h, h->dtmp, u ? h->dtmp + P.N * P.S : nullptr);
    if (rc) return rc;
    CK(cudaStreamSynchronize(h->stream));
    return MCLB_OK;
}

int mclb_init_fields_device(mclb_handle h, const double* rho, const double* u)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (!rho) return fail(MCLB_EINVAL, "rho is NULL");
    return init_common(h, rho, u);
}

int mclb_step(mclb_handle h, long nsteps)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (nsteps < 0) return fail(MCLB_EINVAL, "nsteps=%ld < 0", nsteps);
    // status of work that has already finished (non-blocking)
    int prev = MCLB_OK;
    if (h->status_pending && cudaEventQuery(h->status_event) == cudaSuccess) {
        h->status_pending = false;
        prev = status_code(*h->status_host);
    }
    cudaGetLastError();
    // with the mass compensation on, every mass_every-th step (counted since the state
    // was set) is followed by the compensation
    const long every = h->P.mass_every;
    long left = nsteps;
    while (left > 0) {
        const long chunk = every > 0 ? std::min(left, every - h->since_mass) : left;
        rc = advance(h, chunk);
        if (rc) return rc;
        left -= chunk;
        if (every > 0 && (h->since_mass += chunk) == every) {
            CK(h->tab->mass(h->P, h->sc, h->f[h->cur], 0, h->stream));
            h->since_mass = 0;
        }
    }
    h->steps += nsteps;
    if (nsteps > 0) {
        rc = enqueue_status_copy(h);
        if (rc) return rc;
    }
    return prev;
}

int mclb_status(mclb_handle h)
{
    int rc = check_handle(h);
    if (rc) return rc;
    return sync_status(h);
}

long mclb_step_count(mclb_handle h) { return check_handle(h) ? -1 : h->steps; }

int mclb_test_withhold_copies(mclb_handle h, int on)
{
    int rc = check_handle(h);
    if (rc) return rc;
    h->P.withhold = on ? 1 : 0;
    return MCLB_OK;
}

double mclb_bytes_per_step(mclb_handle h)
{
    if (check_handle(h)) return -1.0;
    const double q = (double)lattice_q(h->P);
    const double per = q * (double)h->tab->storage_bytes + (h->tab->shifted ? sizeof(float) : 0.0);
    return 2.0 * h->P.N * (double)h->P.S * per;
}

int mclb_launches_per_step(mclb_handle h)
{
    if (check_handle(h)) return -1;
    if (h->P.lattice == MCLB_D1Q3) return 1;
    if (h->P.lattice == MCLB_D3Q19) return h->fused ? 2 : 3;   // density + march, or staged
    if (h->fused) return h->P.walls ? 5 : 2;   // k_march, k_ghosts (+ three wall-row launches)
    return 3;
}

int mclb_moments_device(mclb_handle h, double* rho, double* U, double* mu, double* P)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (!rho && !U && !mu && !P) return MCLB_OK;
    if (h->alt)
        CK(h->alt->moments(h->P, h->sc, h->f[h->cur], rho, U, mu, P, h->stream));
    else
        CK(h->tab->moments(h->P, h->sc, h->f[h->cur], rho, U, mu, P, h->stream));
    return MCLB_OK;
}

int mclb_moments(mclb_handle h, double* rho, double* U, double* mu, double* P)
{
    int rc = check_handle(h);
    if (rc) return rc;
    const Problem& Pb = h->P;
    const long long S = Pb.S;
    const int ud = vel_dims(Pb), np = ud == 3 ? 6 : 3;
    rc = ensure_dtmp(h, (size_t)(2 * Pb.N + ud + np) * S);
    if (rc) return rc;
    double* d_rho = rho ? h->dtmp : nullptr;
    double* d_U = U ? h->dtmp + Pb.N * S : nullptr;
    double* d_mu = mu ? h->dtmp + (Pb.N + ud) * S : nullptr;
    double* d_P = P ? h->dtmp + (2 * Pb.N + ud) * S : nullptr;
    rc = mclb_moments_device(h, d_rho, d_U, d_mu, d_P);
    if (rc) return rc;
    if (rho) CK(cudaMemcpyAsync(rho, d_rho, sizeof(double) * Pb.N * S, cudaMemcpyDeviceToHost, h->stream));
    if (U) CK(cudaMemcpyAsync(U, d_U, sizeof(double) * ud * S, cudaMemcpyDeviceToHost, h->stream));
    if (mu) CK(cudaMemcpyAsync(mu, d_mu, sizeof(double) * Pb.N * S, cudaMemcpyDeviceToHost, h->stream));
    if (P) CK(cudaMemcpyAsync(P, d_P, sizeof(double) * np * S, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return MCLB_OK;
}

int mclb_conservation(mclb_handle h, double* mass, double* mom, double* force_sum)
{
    int rc = check_handle(h);
    if (rc) return rc;
    const int N = h->P.N, ud = vel_dims(h->P);
    rc = ensure_dtmp(h, NMAX + 6);
    if (rc) return rc;
    if (h->alt)
        CK(h->alt->conservation(h->P, h->sc, h->f[h->cur], h->dtmp, h->stream));
    else
        CK(h->tab->conservation(h->P, h->sc, h->f[h->cur], h->dtmp, h->stream));
    double out[NMAX + 6];
    CK(cudaMemcpyAsync(out, h->dtmp, sizeof(double) * (N + 2 * ud), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (mass) memcpy(mass, out, sizeof(double) * N);
    if (mom) memcpy(mom, out + N, sizeof(double) * ud);
    if (force_sum) memcpy(force_sum, out + N + ud, sizeof(double) * ud);
    return MCLB_OK;
}

namespace {

// Bytes of nrows stored rows of every component of a D2Q9 handle: per component the nine
// velocity lines of each row (ghost columns included) and, in the 16-bit formats, the
// row's FP32 density line.  Rows [y0, y0 + n) of one component are contiguous in both
// arrays, so a band is N (or 2N) contiguous pieces.
size_t band_bytes(const mclb_handle_s* h, int nrows)
{
    const Problem& P = h->P;
    size_t b = (size_t)P.N * nrows * Q * P.pitch * h->tab->storage_bytes;
    if (h->tab->shifted) b += (size_t)P.N * nrows * P.pitch * sizeof(float);
    return b;
}

int check_band(mclb_handle h, int y0, int nrows, const char* what)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (h->P.lattice != MCLB_D2Q9) return fail(MCLB_EINVAL, "%s: D2Q9 handles only", what);
    if (y0 < 0 || nrows < 0 || (long long)y0 + nrows > h->P.ny)
        return fail(MCLB_EINVAL, "%s: rows [%d, %d + %d) outside [0, %d)", what, y0, y0, nrows,
                    h->P.ny);
    return MCLB_OK;
}

// Copy N pieces of `width` bytes, one per component, between the state (component s at
// state + s * stride) and a packed buffer (at buf + s * width): one 2-D copy, or one copy
// per component where the stride is beyond a 2-D copy's pitch limit.
int copy_pieces(mclb_handle h, char* state, size_t stride, char* buf, size_t width, bool pack)
{
    const int N = h->P.N;
    int dev = 0, max_pitch = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&max_pitch, cudaDevAttrMaxPitch, dev));
    if (stride <= (size_t)max_pitch) {
        if (pack)
            CK(cudaMemcpy2DAsync(buf, width, state, stride, width, N, cudaMemcpyDefault, h->stream));
        else
            CK(cudaMemcpy2DAsync(state, stride, buf, width, width, N, cudaMemcpyDefault, h->stream));
        return MCLB_OK;
    }
    for (int s = 0; s < N; ++s) {
        char* a = state + (size_t)s * stride;
        char* b = buf + (size_t)s * width;
        CK(cudaMemcpyAsync(pack ? b : a, pack ? a : b, width, cudaMemcpyDefault, h->stream));
    }
    return MCLB_OK;
}

// Copy the band [y0, y0 + nrows) of the current state to (pack) or from (!pack) buf.
int copy_band(mclb_handle h, int y0, int nrows, char* buf, bool pack)
{
    const Problem& P = h->P;
    const size_t line = (size_t)Q * P.pitch * h->tab->storage_bytes;   // one row, one component
    char* base = static_cast<char*>(h->f[h->cur]);
    int rc = copy_pieces(h, base + (size_t)y0 * line, (size_t)P.ny * line, buf, nrows * line, pack);
    if (rc || !h->tab->shifted) return rc;
    const size_t rl = (size_t)P.pitch * sizeof(float);
    return copy_pieces(h, base + P.rbytes + (size_t)y0 * rl, (size_t)P.ny * rl,
                       buf + (size_t)P.N * nrows * line, nrows * rl, pack);
}

}  // namespace

size_t mclb_rows_bytes(mclb_handle h, int nrows)
{
    if (check_handle(h) || h->P.lattice != MCLB_D2Q9 || nrows < 0) return 0;
    return band_bytes(h, nrows);
}

int mclb_pack_rows_device(mclb_handle h, int y0, int nrows, void* buf)
{
    int rc = check_band(h, y0, nrows, "mclb_pack_rows_device");
    if (rc) return rc;
    if (nrows == 0) return MCLB_OK;
    if (!buf) return fail(MCLB_EINVAL, "mclb_pack_rows_device: buf is NULL");
    return copy_band(h, y0, nrows, static_cast<char*>(buf), true);
}

int mclb_unpack_rows_device(mclb_handle h, int y0, int nrows, const void* buf)
{
    int rc = check_band(h, y0, nrows, "mclb_unpack_rows_device");
    if (rc) return rc;
    if (nrows == 0) return MCLB_OK;
    if (!buf) return fail(MCLB_EINVAL, "mclb_unpack_rows_device: buf is NULL");
    return copy_band(h, y0, nrows, const_cast<char*>(static_cast<const char*>(buf)), false);
}

int mclb_conservation_rows(mclb_handle h, int y0, int nrows, double* mass, double* mom,
                           double* force_sum)
{
    int rc = check_band(h, y0, nrows, "mclb_conservation_rows");
    if (rc) return rc;
    const int N = h->P.N;
    rc = ensure_dtmp(h, NMAX + 6);
    if (rc) return rc;
    double out[NMAX + 6] = {0.0};
    if (nrows > 0) {
        CK(h->tab->conservation_rows(h->P, h->sc, h->f[h->cur], y0, nrows, h->dtmp, h->stream));
        CK(cudaMemcpyAsync(out, h->dtmp, sizeof(double) * (N + 4), cudaMemcpyDeviceToHost,
                           h->stream));
        CK(cudaStreamSynchronize(h->stream));
    }
    if (mass) memcpy(mass, out, sizeof(double) * N);
    if (mom) memcpy(mom, out + N, sizeof(double) * 2);
    if (force_sum) memcpy(force_sum, out + N + 2, sizeof(double) * 2);
    return MCLB_OK;
}

int mclb_get_state(mclb_handle h, double* f, size_t count)
{
    int rc = check_handle(h);
    if (rc) return rc;
    const size_t want = (size_t)h->P.N * lattice_q(h->P) * h->P.S;
    if (!f || count != want) return fail(MCLB_EINVAL, "count=%zu, expected %zu", count, want);
    rc = ensure_dtmp(h, want);
    if (rc) return rc;
    if (h->alt)
        CK(h->alt->get_state(h->P, h->sc, h->f[h->cur], h->dtmp, h->stream));
    else
        CK(h->tab->get_state(h->P, h->sc, h->f[h->cur], h->dtmp, h->stream));
    CK(cudaMemcpyAsync(f, h->dtmp, sizeof(double) * want, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return MCLB_OK;
}

int mclb_set_state(mclb_handle h, const double* f, size_t count)
{
    int rc = check_handle(h);
    if (rc) return rc;
    const Problem& P = h->P;
    const size_t want = (size_t)P.N * lattice_q(P) * P.S;
    if (!f || count != want) return fail(MCLB_EINVAL, "count=%zu, expected %zu", count, want);
    rc = ensure_dtmp(h, want + 1);
    if (rc) return rc;
    CK(cudaMemcpyAsync(h->dtmp, f, sizeof(double) * want, cudaMemcpyHostToDevice, h->stream));
    unsigned long long* d_bad = reinterpret_cast<unsigned long long*>(h->dtmp + want);
    CK(check_finite(h->dtmp, (long long)want, d_bad, h->stream));
    unsigned long long bad = 0;
    CK(cudaMemcpyAsync(&bad, d_bad, sizeof(bad), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (bad != ULLONG_MAX) return fail(MCLB_EINVAL, "state not finite at value %llu", bad);
    rc = settle_status(h);
    if (rc) return rc;
    CK(cudaMemsetAsync(h->sc.status, 0, sizeof(unsigned int), h->stream));
    if (h->alt)
        CK(h->alt->set_state(P, h->sc, h->dtmp, h->f[0], h->stream));
    else
        CK(h->tab->set_state(P, h->sc, h->dtmp, h->f[0], h->stream));
    h->cur = 0;
    h->steps = 0;
    rc = record_mass(h);
    if (rc) return rc;
    CK(cudaStreamSynchronize(h->stream));
    return MCLB_OK;
}

int mclb_fit_equilibrium(mclb_handle h, int nphase, double* phi)
{
    int rc = check_handle(h);
    if (rc) return rc;
    const Problem& P = h->P;
    if (nphase < 1 || nphase > P.N || !phi)
        return fail(MCLB_EINVAL, "nphase=%d must be in 1..N=%d (phi non-NULL)", nphase, P.N);
    const long long S = P.S;
    rc = ensure_dtmp(h, (size_t)(P.N + 1) * S + fit_work_doubles());
    if (rc) return rc;
    double* d_phi = h->dtmp;
    double* d_bulk = h->dtmp + P.N * S;
    double* d_work = d_bulk + S;
    if (h->alt)
        CK(h->alt->compositions(P, h->sc, h->f[h->cur], d_phi, d_bulk, 1e-3, h->stream));
    else
        CK(h->tab->compositions(P, h->sc, h->f[h->cur], d_phi, d_bulk, 1e-3, h->stream));
    // k-means of the bulk sites on the device; only the centroids come back
    std::vector<double> out((size_t)nphase * P.N + 1);
    int found = 0;
    CK(fit_phases(d_phi, d_bulk, P.N, S, nphase, d_work, out.data(), &found, h->stream));
    if (!found) return fail(MCLB_EINVAL, "no bulk sites (composition gradients all >= 1e-3)");
    memcpy(phi, out.data(), sizeof(double) * nphase * P.N);
    return MCLB_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ batches

struct mclb_batch_s {
    uint32_t magic;
    std::vector<mclb_handle> items;   // one handle per instance (buffers, scratch, status)
    cudaStream_t stream;
    bool own_stream;
    const KernelTable* tab;
    std::vector<void*> groups;        // batched launches, one group per distinct N
    std::vector<void*> lgroups;       // D1Q3 instances, one group per distinct N
    bool dirty;                       // groups must be rebuilt before the next step
    int parity;                       // buffer holding every D2Q9 instance's current state
    int lparity;                      // the same for the D1Q3 instances
    cudaGraphExec_t graph[2];
    bool graph_tried[2];
    // a group's ghost refresh runs on the side stream, overlapping the next group's march;
    // ev_main[g] = group g's march done, ev_side[g] = its ghost refresh done
    cudaStream_t side;
    std::vector<cudaEvent_t> ev_main, ev_side;
};

namespace {

void batch_drop(mclb_batch b)
{
    for (void* g : b->groups) b->tab->batch_destroy(g);
    b->groups.clear();
    for (void* g : b->lgroups) b->tab->line3->batch_destroy(g);
    b->lgroups.clear();
    for (cudaEvent_t e : b->ev_main) cudaEventDestroy(e);
    for (cudaEvent_t e : b->ev_side) cudaEventDestroy(e);
    b->ev_main.clear();
    b->ev_side.clear();
    for (int k = 0; k < 2; ++k) {
        if (b->graph[k]) cudaGraphExecDestroy(b->graph[k]);
        b->graph[k] = nullptr;
        b->graph_tried[k] = false;
    }
}

int batch_build(mclb_batch b)
{
    batch_drop(b);
    for (int n = 1; n <= NMAX; ++n) {
        std::vector<Problem> probs;
        std::vector<Scratch> scs;
        std::vector<void*> fa, fb;
        std::vector<CUtensorMap> maps, maps2;
        bool fused = true;
        // the narrow strip geometry's views, a second candidate for the autotuner
        int nbox = 0, nout = 0;
        bool narrow = b->tab->narrow_boxes(n, &nbox, &nout);
        std::vector<Problem> lprobs;
        std::vector<Scratch> lscs;
        std::vector<void*> la, lb;
        for (auto h : b->items)
            if (h->P.N == n && h->alt) {
                lprobs.push_back(h->P);
                lscs.push_back(h->sc);
                la.push_back(h->f[0]);
                lb.push_back(h->f[1]);
            }
        if (!lprobs.empty()) {
            void* g = b->tab->line3->batch_create(n, (int)lprobs.size(), lprobs.data(), lscs.data(),
                                                  la.data(), lb.data(), b->stream);
            if (!g) {
                batch_drop(b);
                return fail(MCLB_ENOMEM, "D1Q3 batch tables for N=%d could not be built", n);
            }
            b->lgroups.push_back(g);
        }
        for (auto h : b->items)
            if (h->P.N == n && !h->alt) {
                probs.push_back(h->P);
                scs.push_back(h->sc);
                fa.push_back(h->f[0]);
                fb.push_back(h->f[1]);
                // the batched march has no Gibbs-Duhem instance: such a group runs staged
                fused = fused && h->fused && h->P.force_form != FORCE_GIBBS_DUHEM;
                for (int k = 0; k < 2; ++k) {
                    maps.push_back(h->tmap[k]);
                    maps.push_back(h->tmapr[k]);
                    maps.push_back(h->tmapw[k]);
                    maps.push_back(h->tmapwr[k]);
                    if (narrow && h->fused) {
                        CUtensorMap m[4] = {};
                        CUtensorMap* const v[4] = {&m[0], &m[1], &m[2], &m[3]};
                        if (encode_views(h, k, nbox, nout, v) == MCLB_OK) {
                            maps2.insert(maps2.end(), m, m + 4);
                        } else {
                            narrow = false;
                            cudaGetLastError();
                        }
                    }
                }
            }
        if (probs.empty()) continue;
        int dev = 0, sms = 1;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            cudaGetLastError();
        narrow = narrow && fused && maps2.size() == maps.size();
        void* g = b->tab->batch_create(n, (int)probs.size(), probs.data(), scs.data(), fa.data(),
                                       fb.data(), fused ? maps.data() : nullptr,
                                       narrow ? maps2.data() : nullptr, sms, b->stream);
        if (!g) {
            batch_drop(b);
            return fail(MCLB_ENOMEM, "batched launch tables for N=%d could not be built", n);
        }
        b->groups.push_back(g);
        cudaEvent_t e1 = nullptr, e2 = nullptr;
        if (cudaEventCreateWithFlags(&e1, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&e2, cudaEventDisableTiming) != cudaSuccess) {
            if (e1) cudaEventDestroy(e1);
            batch_drop(b);
            return fail(MCLB_ECUDA, "cudaEventCreate failed");
        }
        b->ev_main.push_back(e1);
        b->ev_side.push_back(e2);
    }
    b->dirty = false;
    return MCLB_OK;
}

// One batched timestep.  Group g's march waits for g's previous ghost refresh (side
// stream); its own refresh then runs on the side stream while the next group marches.
// wait_side = false skips the first wait (the first step of a stream capture, whose
// stream has already joined the side stream: a captured stream may not wait on an event
// recorded outside the capture).
cudaError_t batch_launch(mclb_batch b, int parity, bool wait_side = true)
{
    for (size_t g = 0; g < b->groups.size(); ++g) {
        cudaError_t e = wait_side ? cudaStreamWaitEvent(b->stream, b->ev_side[g], 0) : cudaSuccess;
        if (e == cudaSuccess) e = b->tab->batch_step(b->groups[g], parity, b->stream, 0);
        if (e == cudaSuccess) e = cudaEventRecord(b->ev_main[g], b->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->side, b->ev_main[g], 0);
        if (e == cudaSuccess) e = b->tab->batch_step(b->groups[g], parity, b->side, 1);
        if (e == cudaSuccess) e = cudaEventRecord(b->ev_side[g], b->side);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// The main stream waits for every ghost refresh issued so far.
cudaError_t batch_join(mclb_batch b)
{
    for (cudaEvent_t e : b->ev_side) {
        const cudaError_t r = cudaStreamWaitEvent(b->stream, e, 0);
        if (r != cudaSuccess) return r;
    }
    return cudaSuccess;
}

void batch_capture(mclb_batch b, int from)
{
    b->graph_tried[from] = true;
    b->graph[from] = nullptr;
    if (batch_join(b) != cudaSuccess) {   // outside the capture
        cudaGetLastError();
        return;
    }
    if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    int par = from;
    bool ok = true;
    for (int k = 0; k < GRAPH_STEPS && ok; ++k) {
        ok = batch_launch(b, par, k > 0) == cudaSuccess;
        par ^= 1;
    }
    ok = ok && batch_join(b) == cudaSuccess;   // the side stream rejoins before the capture ends
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    // the events were last recorded inside the capture; record them again outside it so
    // that later waits outside a capture refer to an ordinary record
    for (cudaEvent_t ev : b->ev_main) cudaEventRecord(ev, b->stream);
    for (cudaEvent_t ev : b->ev_side) cudaEventRecord(ev, b->stream);
    if (ok && e == cudaSuccess && g) {
        cudaGraphExec_t ex = nullptr;
        if (cudaGraphInstantiate(&ex, g, 0) == cudaSuccess) b->graph[from] = ex;
    }
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
}

}  // namespace

extern "C" {

int mclb_batch_create(const mclb_params* params, int count, mclb_batch* out)
{
    if (!out) return fail(MCLB_EINVAL, "out is NULL");
    *out = nullptr;
    if (!params || count < 1) return fail(MCLB_EINVAL, "count=%d must be >= 1", count);
    for (int k = 0; k < count; ++k) {
        if (params[k].mass_every != 0)
            return fail(MCLB_EINVAL, "instance %d: mass_every must be 0 in a batch", k);
        if (params[k].lattice == MCLB_D3Q19)
            return fail(MCLB_EINVAL, "instance %d: batches hold D2Q9 and D1Q3 lattices", k);
        if (params[k].walls)
            return fail(MCLB_EINVAL, "instance %d: batches are periodic (walls must be 0)", k);
    }
    mclb_batch b = new (std::nothrow) mclb_batch_s();
    if (!b) return fail(MCLB_ENOMEM, "host allocation failed");
    b->magic = MAGIC;
    b->tab = &table_for(params[0].precision);
    b->stream = (cudaStream_t)params[0].stream;
    b->own_stream = false;
    b->dirty = true;
    b->parity = 0;
    b->lparity = 0;
    if (!b->stream) {
        if (cudaStreamCreate(&b->stream) != cudaSuccess) {
            delete b;
            return fail(MCLB_ECUDA, "cudaStreamCreate failed");
        }
        b->own_stream = true;
    }
    if (cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking) != cudaSuccess) {
        b->side = nullptr;
        mclb_batch_destroy(b);
        return fail(MCLB_ECUDA, "cudaStreamCreate failed");
    }
    for (int k = 0; k < count; ++k) {
        mclb_params p = params[k];
        p.precision = params[0].precision;
        p.kernel = MCLB_KERNEL_AUTO;   // builds the tensor maps the batched march uses
        p.stream = b->stream;
        mclb_handle h = nullptr;
        int rc = mclb_create(&p, &h);
        if (rc) {
            std::string msg = g_err;
            mclb_batch_destroy(b);
            return fail(rc, "instance %d: %s", k, msg.c_str());
        }
        b->items.push_back(h);
    }
    *out = b;
    return MCLB_OK;
}

static int batch_item(mclb_batch b, int index, mclb_handle* h)
{
    if (!b || b->magic != MAGIC) return fail(MCLB_EHANDLE, "batch destroyed or not a batch");
    if (index < 0 || index >= (int)b->items.size())
        return fail(MCLB_EINVAL, "index %d outside 0..%zu", index, b->items.size() - 1);
    *h = b->items[index];
    return MCLB_OK;
}

int mclb_batch_init_fields(mclb_batch b, int index, const double* rho, const double* u)
{
    mclb_handle h = nullptr;
    int rc = batch_item(b, index, &h);
    if (rc) return rc;
    rc = mclb_init_fields(h, rho, u);  // writes buffer 0
    if (rc) return rc;
    if ((h->alt ? b->lparity : b->parity) == 1) {   // the state lives in the batch's buffer
        CK(cudaMemcpyAsync(h->f[1], h->f[0], h->fbytes, cudaMemcpyDeviceToDevice, b->stream));
        CK(cudaStreamSynchronize(b->stream));
        h->cur = 1;
    }
    b->dirty = true;
    return MCLB_OK;
}

int mclb_batch_step(mclb_batch b, long nsteps)
{
    if (!b || b->magic != MAGIC) return fail(MCLB_EHANDLE, "batch destroyed or not a batch");
    if (nsteps < 0) return fail(MCLB_EINVAL, "nsteps=%ld < 0", nsteps);
    if (b->dirty) {
        int rc = batch_build(b);
        if (rc) return rc;
    }
    cudaGetLastError();
    if (nsteps > 0)
        for (void* g : b->groups) CK(b->tab->batch_tune(g, b->parity, b->stream));
    // D1Q3 lines: every group in chunks of resident steps (each chunk moves the lines to
    // the other buffer)
    for (long left = b->lgroups.empty() ? 0 : nsteps; left > 0;) {
        const int k = (int)(left < LINE3_CHUNK ? left : LINE3_CHUNK);
        for (void* g : b->lgroups) CK(b->tab->line3->batch_step(g, b->lparity, k, b->stream));
        b->lparity ^= 1;
        left -= k;
    }
    long left = b->groups.empty() ? 0 : nsteps;
    while (left >= GRAPH_STEPS) {
        if (!b->graph_tried[b->parity]) batch_capture(b, b->parity);
        if (!b->graph[b->parity]) break;
        CK(cudaGraphLaunch(b->graph[b->parity], b->stream));
        left -= GRAPH_STEPS;  // an even number of steps: the parity is unchanged
    }
    for (; left > 0; --left) {
        CK(batch_launch(b, b->parity));
        b->parity ^= 1;
    }
    CK(batch_join(b));   // later work on the batch's stream sees every ghost refresh
    for (auto h : b->items) {
        h->cur = h->alt ? b->lparity : b->parity;
        h->steps += nsteps;
    }
    return MCLB_OK;
}

int mclb_batch_launches_per_step(mclb_batch b)
{
    if (!b || b->magic != MAGIC) return -1;
    if (b->dirty && batch_build(b)) return -1;
    int n = 0;
    for (const void* g : b->groups) n += b->tab->batch_launches(g);
    for (const void* g : b->lgroups) n += b->tab->line3->batch_launches(g);
    return n;
}

int mclb_batch_tuning(mclb_batch b, int* narrow, int* waves, int cap)
{
    if (!b || b->magic != MAGIC || cap < 0) return -1;
    if (b->dirty && batch_build(b)) return -1;
    int n = 0;
    for (const void* g : b->groups) {
        const int w = b->tab->batch_waves(g);
        if (n < cap) {
            if (narrow) narrow[n] = w >= 1000 ? 1 : 0;
            if (waves) waves[n] = w % 1000;
        }
        ++n;
    }
    return n;
}

int mclb_test_batch_partition(mclb_batch b, int narrow, int waves)
{
    if (!b || b->magic != MAGIC) return -1;
    if (waves != 2 && waves != 4 && waves != 8 && waves != 16) return -1;
    if (b->dirty && batch_build(b)) return -1;
    int n = 0;
    for (void* g : b->groups) n += b->tab->batch_force(g, narrow, waves) ? 1 : 0;
    // graphs captured with the previous pick would replay it (let queued replays finish)
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    for (int k = 0; k < 2; ++k) {
        if (b->graph[k]) cudaGraphExecDestroy(b->graph[k]);
        b->graph[k] = nullptr;
        b->graph_tried[k] = false;
    }
    return n;
}

int mclb_batch_moments(mclb_batch b, int index, double* rho, double* U, double* mu, double* P)
{
    mclb_handle h = nullptr;
    int rc = batch_item(b, index, &h);
    return rc ? rc : mclb_moments(h, rho, U, mu, P);
}

int mclb_batch_fit_equilibrium(mclb_batch b, int index, int nphase, double* phi)
{
    mclb_handle h = nullptr;
    int rc = batch_item(b, index, &h);
    return rc ? rc : mclb_fit_equilibrium(h, nphase, phi);
}

int mclb_batch_get_state(mclb_batch b, int index, double* f, size_t count)
{
    mclb_handle h = nullptr;
    int rc = batch_item(b, index, &h);
    return rc ? rc : mclb_get_state(h, f, count);
}

int mclb_batch_status(mclb_batch b, int* per_instance)
{
    if (!b || b->magic != MAGIC) return fail(MCLB_EHANDLE, "batch destroyed or not a batch");
    int first = MCLB_OK;
    for (size_t k = 0; k < b->items.size(); ++k) {
        int rc = mclb_status(b->items[k]);
        if (per_instance) per_instance[k] = rc;
        if (rc && !first) first = rc;
    }
    return first;
}

double mclb_batch_bytes_per_step(mclb_batch b)
{
    if (!b || b->magic != MAGIC) return -1.0;
    double t = 0.0;
    for (auto h : b->items) t += mclb_bytes_per_step(h);
    return t;
}

int mclb_batch_destroy(mclb_batch b)
{
    if (!b) return MCLB_OK;
    if (b->magic != MAGIC) return fail(MCLB_EHANDLE, "batch destroyed or not a batch");
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->side) cudaStreamSynchronize(b->side);
    batch_drop(b);
    for (auto h : b->items) mclb_destroy(h);
    if (b->side) cudaStreamDestroy(b->side);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    b->magic = DEAD;
    delete b;
    return MCLB_OK;
}

}  // extern "C"
