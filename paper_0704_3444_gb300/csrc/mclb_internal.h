// mclb_internal.h -- interface between the C ABI runtime (capi.cu) and the
// per-precision kernel translation units.  Host-only types; no torch anywhere.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace mclb {

constexpr int NMAX = 8;
constexpr int Q = 9;
constexpr int ROW_ALIGN = 128;  // data columns per row are padded to a multiple of this
constexpr int LATTICE_D1Q3 = 1; // Problem::lattice of a D1Q3 lattice (MCLB_D1Q3)
constexpr int LATTICE_D3Q19 = 2; // Problem::lattice of a D3Q19 lattice (MCLB_D3Q19)
constexpr int FORCE_GIBBS_DUHEM = 1; // Problem::force_form of the Gibbs-Duhem total force

// Everything a launcher needs to know about one simulation, in FP64 as given at
// the boundary; each precision unit converts it to its own kernel parameters.
//
// Distribution layout (every schedule): component s, row y, velocity i, column x at
//   ((s * ny + y) * 9 + i) * pitch + hx + x,
// i.e. the nine velocity lines of one component row are adjacent, so that they
// sit at small constant offsets from one address and one source row of every
// component is a single 4-D TMA box.  hx ghost columns on each side of a line
// repeat the periodic neighbours (ghost column g in [-hx, 0) u [nx, nx + hx)
// holds column g mod nx) and a line is padded to pitch = 2 hx + roundup(nx,
// ROW_ALIGN) elements.  The ghosts are rewritten after every write of the
// distributions (by the staged kernels themselves, by k_ghosts after the single-pass
// kernel), so that the single-pass kernel moves whole aligned row segments with TMA.
struct Problem {
    int N, nx, ny;
    int nz;                 // layers (D3Q19), 1 otherwise
    long long S;            // nx * ny * nz sites
    int hx;                 // ghost columns per side
    long long pitch;        // elements per (row, velocity) line
    long long plane;        // elements per component = ny * 9 * pitch
    double tau, theta, kappa, gx, gy, gz;
    double chi[NMAX * NMAX];
    double m[NMAX];
    int forcing_velocity;   // MCLB_FORCING_COMPONENT (0) or MCLB_FORCING_BARYCENTRIC (1)
    int lattice;            // MCLB_D2Q9 (0), MCLB_D1Q3 (1: ny = 1, layout [s][i][x], no ghosts) or
                            // MCLB_D3Q19 (2: layout [s][z][y][i][x], no ghosts)
    int force_form;         // MCLB_FORCE_COMPONENT (0) or MCLB_FORCE_GIBBS_DUHEM (1)
    int walls;              // 1: solid walls in y (D2Q9), 0: periodic
    int mass_every;         // period of the per-component mass compensation, 0 = off
    int withhold;           // test hook: the single-pass kernel issues no copies
    long long rbytes;       // 16-bit formats: byte offset of the FP32 density lines
                            // ([s][y][pitch], same ghosts) after the deviations; else 0
    int seg3;               // D3Q19: > 0 = density pass + march, z segments of seg3 planes
    int grid3[3];           // over grid3 CTAs (x tiles, y tiles, segments); 0 = staged
};

// Device scratch owned by a handle: component densities and the potentials
// nu^s = mu^s - (1/3) ln rho^s in the compute type (used by the staged schedule and
// by the diagnostics), block partial sums for FP64 reductions, and the status word.
struct Scratch {
    void* rho_s;            // N * S compute-type values
    void* nu;               // N * S compute-type values
    double* partial;        // reduction partials
    size_t partial_cap;     // capacity in doubles
    unsigned int* status;   // device status bits (see STATUS_*)
    void* line_item;        // D1Q3 handles: the device description the resident kernel reads
    double* mass_ref;       // NMAX FP64 reference masses of the mass compensation
    void* js;               // D3Q19 handles: momenta j^s, 3 N S compute-type values ([s][d][site])
};

enum : unsigned int {
    STATUS_NONFINITE = 1u,  // NaN/Inf or non-positive total density seen
    STATUS_TIMEOUT = 2u     // a bounded device wait gave up
};

constexpr int REDUCE_BLOCKS = 256;    // fixed grid of the FP64 reductions (deterministic)

// Launch plan of the single-pass kernel: strips of W written columns (TMA boxes of
// box_w columns, one velocity line each), segments of H rows, NS stages.
struct FusedPlan {
    int W, box_w, out_w, NS, H;
    int nstrips, nsegs;
    int threads;
    size_t smem;
    bool ok;
};

// Kernels of a lattice other than the D2Q9 family -- D1Q3 (line3.cuh) or D3Q19 (cube.cuh)
// -- for one storage type (FP64 and FP32 only).  Distributions: post-collision values
// ([s][3][nx] for D1Q3, [s][z][y][19][x] for D3Q19); pre-collision f_i(r) = f*_i(r - v_i).
// The batch entries are D1Q3 only (null for D3Q19).
struct LatticeTable {
    int (*max_resident)(int N);   // longest line the resident (shared-memory) kernel holds
    // set up the single-pass step where it applies (P.seg3, P.grid3): 1 = set up, 0 = the
    // staged step, -1 = CUDA error; null for lattices with one step kernel
    int (*plan)(Problem& P, int sm_count);
    size_t item_bytes;            // size of the device description at Scratch::line_item
    // write the description of buffers f[0], f[1] to sc.line_item (synchronous)
    cudaError_t (*prepare)(const Problem&, const Scratch&, void* const* f);
    cudaError_t (*init)(const Problem&, const Scratch&, const double* rho, const double* u,
                        void* f, cudaStream_t st);
    // nsteps timesteps from f[*cur]; *cur receives the buffer holding the result
    cudaError_t (*step)(const Problem&, const Scratch&, void* const* f, int* cur, long nsteps,
                        cudaStream_t st);
    cudaError_t (*moments)(const Problem&, const Scratch&, const void* f, double* rho,
                           double* U, double* mu, double* P, cudaStream_t st);
    cudaError_t (*conservation)(const Problem&, const Scratch&, const void* f, double* out,
                                cudaStream_t st);
    cudaError_t (*compositions)(const Problem&, const Scratch&, const void* f, double* phi,
                                double* bulk, double tol, cudaStream_t st);
    cudaError_t (*get_state)(const Problem&, const Scratch&, const void* f, double* out,
                             cudaStream_t st);
    cudaError_t (*set_state)(const Problem&, const Scratch&, const double* in, void* f,
                             cudaStream_t st);
    // batches: every line of one N; a step of k <= L3_CHUNK timesteps reads buffer
    // `parity` of every line and leaves the result in buffer parity ^ 1 (lines that fit
    // share one resident launch, one CTA each; longer ones step with the tile kernel)
    void* (*batch_create)(int N, int count, const Problem* probs, const Scratch* scs,
                          void* const* fa, void* const* fb, cudaStream_t st);
    cudaError_t (*batch_step)(void* group, int parity, int nsteps, cudaStream_t st);
    int (*batch_launches)(const void* group);
    void (*batch_destroy)(void* group);
};

constexpr int LINE3_CHUNK = 4096;   // most timesteps one resident D1Q3 launch advances

struct KernelTable {
    size_t storage_bytes;   // bytes of one stored distribution value
    bool shifted;
    CUtensorMapDataType tma_type;
    int hx;                 // ghost columns per side for this storage type
    FusedPlan (*plan_fused)(const Problem&, int sm_count);
    // f^s_i(r) = equilibrium of (rho, u) (device FP64 inputs; u may be null)
    cudaError_t (*init)(const Problem&, const Scratch&, const double* rho, const double* u,
                        void* f, cudaStream_t st);
    // one fused timestep fin -> fout (tmap_in describes fin's lines, tmapr_in its density
    // lines in the 16-bit formats, tmapw_out / tmapwr_out the columns [0, nx) of fout's
    // lines / density lines; with walls the rows next to them are redone from fin)
    cudaError_t (*step_fused)(const Problem&, const Scratch&, const FusedPlan&,
                              const CUtensorMap* tmap_in, const CUtensorMap* tmapr_in,
                              const CUtensorMap* tmapw_out, const CUtensorMap* tmapwr_out,
                              const void* fin, void* fout, cudaStream_t st);
    // one staged timestep fin -> fout (three launches through scratch)
    cudaError_t (*step_staged)(const Problem&, const Scratch&, const void* fin, void* fout,
                               cudaStream_t st);
    // macroscopic output fields into device FP64 arrays (any may be null)
    cudaError_t (*moments)(const Problem&, const Scratch&, const void* f, double* rho,
                           double* U, double* mu, double* P, cudaStream_t st);
    // FP64 sums into out: [0, N) mass, [N, N+2) momentum, [N+2, N+4) force
    cudaError_t (*conservation)(const Problem&, const Scratch&, const void* f, double* out,
                                cudaStream_t st);
    // the same sums over the rows [y0, y0 + nrows) only
    cudaError_t (*conservation_rows)(const Problem&, const Scratch&, const void* f, int y0,
                                     int nrows, double* out, cudaStream_t st);
    // FP64 compositions phi (N * S) and bulk flags (S, 1.0 where max |grad phi| < tol)
    cudaError_t (*compositions)(const Problem&, const Scratch&, const void* f, double* phi,
                                double* bulk, double tol, cudaStream_t st);
    // pre-collision FP64 state out / in, layout [s][i][y][x]
    cudaError_t (*get_state)(const Problem&, const Scratch&, const void* f, double* out,
                             cudaStream_t st);
    cudaError_t (*set_state)(const Problem&, const Scratch&, const double* in, void* f,
                             cudaStream_t st);
    // per-component mass compensation of the stored state f, either lattice (mass.cuh):
    // record != 0 stores each component's FP64 mass in sc.mass_ref; record == 0 adds the
    // deficit against it, spread over the sites, to the rest populations (16-bit: to R)
    cudaError_t (*mass)(const Problem&, const Scratch&, void* f, int record, cudaStream_t st);
    // batches: a group of `count` instances with the same N (buffers fa/fb, scratch scs,
    // 8 tensor maps per instance [buffer][load, density load, store, density store] or
    // NULL); one step of the whole group reads buffer `parity` and writes the other, by
    // the batched march when the maps are given and it fits, else by the staged schedule
    // maps2 (or NULL): the same 8 maps per instance with the narrow geometry's box widths
    // (narrow_boxes), a second strip shape for the autotuner
    void* (*batch_create)(int N, int count, const Problem* probs, const Scratch* scs,
                          void* const* fa, void* const* fb, const CUtensorMap* maps,
                          const CUtensorMap* maps2, int sm_count, cudaStream_t st);
    bool (*narrow_boxes)(int N, int* box_w, int* out_w);
    // part 0: the batched march (or the whole staged step); part 1: the ghost refresh of
    // the buffer part 0 wrote (nothing for the staged schedule)
    cudaError_t (*batch_step)(void* group, int parity, cudaStream_t st, int part);
    int (*batch_launches)(const void* group);   // kernel launches of one group step
    // pick the group's work partition by timing the candidates on the current state
    // (reads buffer `parity`, rewrites the other with the same values; synchronises)
    cudaError_t (*batch_tune)(void* group, int parity, cudaStream_t st);
    // test hook: use the candidate (narrow, waves) instead of the timed pick; false if absent
    bool (*batch_force)(void* group, int narrow, int waves);
    int (*batch_waves)(const void* group);      // waves of the partition in use, 0 if staged
    void (*batch_destroy)(void* group);
    const LatticeTable* line3;  // D1Q3 kernels (null for the 16-bit formats)
    const LatticeTable* d3q19;  // D3Q19 kernels (null for the 16-bit formats)
};

// Device checks of FP64 boundary data (checks.cu).  *first_bad receives the smallest
// failing site (check_fields: a density not finite, total density not positive, or one
// of the ud velocity components, u may be null, not finite) or index (check_finite), and
// stays ULLONG_MAX when everything passes.  Stream ordered; the caller reads first_bad back.
cudaError_t check_fields(const double* rho, const double* u, int N, int ud, long long S,
                         unsigned long long* first_bad, cudaStream_t st);
cudaError_t check_finite(const double* a, long long n, unsigned long long* first_bad,
                         cudaStream_t st);

// Bulk-phase fit on the device (fit.cu): k-means of the bulk sites' compositions into
// nphase phases in FP64 with fixed-order sums.  phi: N * S, bulk: S (device).  work:
// fit_work_doubles() device doubles.  host_out: nphase * N + 1 host doubles; receives the
// centroids, phase c first.  *found = 0 if there is no bulk site.  Synchronises st.
size_t fit_work_doubles();
cudaError_t fit_phases(const double* phi, const double* bulk, int N, long long S, int nphase,
                       double* work, double* host_out, int* found, cudaStream_t st);

const KernelTable& table_fp64();
const KernelTable& table_fp32();
const KernelTable& table_bf16();
const KernelTable& table_fp16();

}  // namespace mclb
