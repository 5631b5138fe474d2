/*
 * mclb.h -- C ABI of the GB300 (sm_103a) multicomponent lattice Boltzmann library.
 *
 * The library advances the symmetric free-energy multicomponent lattice
 * Boltzmann method of Li & Wagner (arXiv:0704.3444) on a periodic D2Q9 lattice, or
 * on the D1Q3 lattice of the paper's own simulations (Sec. 4):
 * one lattice Boltzmann equation per component with BGK relaxation towards an
 * equilibrium built on the shared barycentric velocity, plus the forcing term
 *     rho^s a^s = -(1 - 1/(2 tau)) rho^s grad( mu^s - (1/3) ln rho^s )   (Eq. definef)
 * with mu^s the Flory-Huggins chemical potential of Eq. lgf (plus a gradient
 * term kappa), and streaming (Eq. ssLB).
 *
 * Conventions shared by every entry point
 *   - Return value: MCLB_OK (0) on success, a negative MCLB_E* code on failure;
 *     mclb_last_error() then returns a message (thread-local, valid until the
 *     next call on the same thread).
 *   - Host arrays are owned by the caller; the library copies in and out and keeps
 *     no pointer to them after the call returns.  Device memory of a handle is
 *     owned by the library and released by mclb_destroy / mclb_batch_destroy.
 *   - Field arrays are FP64, row-major [component][y][x] with x fastest;
 *     velocity-like arrays are [2][y][x] (x component first).  This holds in every
 *     storage precision.
 *   - D2Q9 velocity order: v_0 = (0,0); v_1..4 = (1,0), (0,1), (-1,0), (0,-1);
 *     v_5..8 = (1,1), (-1,1), (-1,-1), (1,-1).  Weights 4/9, 1/9, 1/36.
 *   - D1Q3 (params.lattice = MCLB_D1Q3, ny = 1): v_0 = 0, v_1 = +1, v_2 = -1, weights
 *     2/3, 1/6, 1/6; the discrete gradient and Laplacian are (g(x+1) - g(x-1))/2 and
 *     g(x+1) + g(x-1) - 2 g(x).  Field arrays keep the D2Q9 shapes with ny = 1
 *     (velocity-like [2][1][nx] with a zero y component).
 *   - In FP32 the weights are rounded so that they sum to exactly 1 (w_5..8 of D2Q9 and
 *     w_1,2 of D1Q3 sit one unit in the last place below the nearest float), so that
 *     the equilibria keep every site's mass to rounding.
 *   - All device work of a handle is ordered on the stream given at creation
 *     (NULL: a stream the handle creates with cudaStreamCreate and owns, which is
 *     ordered with the legacy default stream but not with other streams).  Calls that
 *     return host data synchronise that stream.  Handles are not thread-safe.
 */
#ifndef MCLB_H
#define MCLB_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MCLB_NMAX 8 /* largest number of components */

enum {
    MCLB_OK = 0,
    MCLB_EINVAL = -1,     /* invalid argument or parameter                          */
    MCLB_ENOMEM = -2,     /* device or host allocation failed                       */
    MCLB_ECUDA = -3,      /* a CUDA runtime call failed (message has the CUDA error) */
    MCLB_ENONFINITE = -4, /* a NaN/Inf or a non-positive total density appeared     */
    MCLB_ETIMEOUT = -5,   /* a bounded device wait ran out                          */
    MCLB_EHANDLE = -6     /* NULL, destroyed or foreign handle                      */
};

/* Storage precision of the distributions.  Arithmetic is FP64 in MCLB_FP64 and
 * FP32 otherwise.  The *_SHIFTED modes store, per site and component, a reference
 * density R in FP32 and the deviations d_i = f_i - w_i M (M = sum_i f_i after the
 * collision) in 16 bits, with R = M - sum_i d_i so that the stored site mass is M to
 * FP32 rounding: f_i is read back as d_i + w_i R.  This needs 9*2 + 4 = 22 bytes per
 * site and component instead of 36 (FP32) or 72 (FP64). */
typedef enum {
    MCLB_FP64 = 0,
    MCLB_FP32 = 1,
    MCLB_BF16_SHIFTED = 2,
    MCLB_FP16_SHIFTED = 3
} mclb_precision;

/* Which kernel schedule performs a timestep. */
typedef enum {
    MCLB_KERNEL_AUTO = 0,   /* the fused single-pass kernel                         */
    MCLB_KERNEL_FUSED = 1,  /* stream, moments, potentials, force, collision in one
                               pass over the distributions, then a small launch that
                               refreshes the periodic ghost columns                 */
    MCLB_KERNEL_STAGED = 2  /* three launches per step through density and
                               potential fields in device scratch memory            */
} mclb_kernel;

/* Velocity in the second moment of the forcing term (Eq. ff3). */
typedef enum {
    MCLB_FORCING_COMPONENT = 0,   /* rho^s (a^s u^s + u^s a^s), u^s = j^s / rho^s, as Eq. ff3
                                     prints it (the default)                             */
    MCLB_FORCING_BARYCENTRIC = 1  /* rho^s (a^s u + u a^s) with the barycentric u: a reading
                                     whose sum over the components is the one-fluid forcing
                                     moment rho (a u + u a) of Eq. olso; the paper's remark
                                     after Eq. olso calls the difference higher order     */
} mclb_forcing_velocity;

/* How the component forces of Eq. definef are summed. */
typedef enum {
    MCLB_FORCE_COMPONENT = 0,     /* each component's force as Eq. definef prints it (the
                                     default)                                              */
    MCLB_FORCE_GIBBS_DUHEM = 1    /* a reading for kappa = 0 (the paper's setting): every
                                     component's acceleration gets the same shift, so that
                                     their differences are kept and their density-weighted
                                     sum is the continuum total (1 - 1/(2 tau)) (1/3) grad rho
                                     that Gibbs-Duhem gives for the Flory-Huggins free energy
                                     (its pressure sum rho mu - psi vanishes); the total force
                                     is then a discrete gradient and total momentum is kept.
                                     D2Q9: the single pass for FP64/FP32 and N <= 3 (kernel
                                     AUTO or FUSED; FUSED fails with MCLB_EINVAL otherwise),
                                     else the staged schedule; D1Q3; D3Q19 staged only      */
} mclb_force_form;

/* Lattice. */
typedef enum {
    MCLB_D2Q9 = 0,   /* two-dimensional, nine velocities (see the conventions above)      */
    MCLB_D1Q3 = 1,   /* the one-dimensional lattice of the paper's simulations (Sec. 4):
                        v_0 = 0, v_1 = +1, v_2 = -1, weights 2/3, 1/6, 1/6; ny must be 1   */
    MCLB_D3Q19 = 2   /* three dimensions, nz layers: the rest velocity (weight 1/3), the six
                        axis directions (1/18) and the twelve face diagonals (1/36), in the
                        order 0; (+-1,0,0), (0,+-1,0), (0,0,+-1); (1,1,0), (-1,-1,0),
                        (1,-1,0), (-1,1,0), (1,0,1), (-1,0,-1), (1,0,-1), (-1,0,1),
                        (0,1,1), (0,-1,-1), (0,1,-1), (0,-1,1).  Not a lattice the paper
                        uses: its equations hold for any lattice whose weights give the
                        Sec. 3 moments, which these do.  FP64 or FP32 storage, single
                        handles only.  Kernel AUTO or FUSED: a density pass and a march
                        over z planes that forms the potentials on chip and collides (two
                        launches per step; N <= 4, Eq. definef as printed; FUSED fails
                        with MCLB_EINVAL otherwise, AUTO falls back); STAGED: three
                        launches.  The two schedules give the same values bit for bit.
                        Fields are [.][z][y][x]; U has 3 components, P 6 (xx, xy, xz, yy,
                        yz, zz), the momentum and force sums 3                             */
} mclb_lattice;

/* Problem statement (Sec. 3 and Sec. 4 of the paper).
 *   ncomp      N, number of components, 1..MCLB_NMAX
 *   nx, ny     periodic lattice size, >= 1 each
 *   tau        one relaxation time for every component (Eq. ssLB), > 1/2
 *   chi        N*N Flory-Huggins interaction matrix (Eq. lgf), row-major, must be
 *              symmetric and finite; the paper sets the diagonal to zero
 *   m          N polymerisations m^s (Eq. lgf), > 0; NULL means all 1
 *   theta      Flory-Huggins temperature of Eq. lgf; <= 0 selects 1/3
 *   kappa      gradient coefficient: the free energy gains sum_s (kappa/2)|grad rho^s|^2,
 *              so mu^s gains -kappa lap rho^s (the paper names kappa and sets it to 0)
 *   force      body acceleration g (Eq. NSEeq), added to every a^s
 *   precision  mclb_precision
 *   kernel     mclb_kernel
 *   stream     cudaStream_t to order all work on, or NULL (the handle creates its own)
 *   forcing_velocity  mclb_forcing_velocity (0: Eq. ff3 as printed)
 *   lattice    mclb_lattice (0: D2Q9)
 *   force_form mclb_force_form (0: Eq. definef as printed)
 *   nz         layers of a D3Q19 lattice (0 or 1 for the other lattices, which reject more)
 *   force_z    z component of the body acceleration (D3Q19 only; 0 otherwise)
 *   walls      0: periodic in y (the paper's setting); 1: stationary solid walls halfway
 *              between rows, below row 0 and above row ny - 1 (the paper has no walls:
 *              a reading for non-periodic set-ups such as a slab in contact with a solid).
 *              A population that would stream across a wall returns to its site with
 *              the opposite velocity (halfway bounce-back), which keeps every component's
 *              mass; the stencils of rho^s and nu^s see the rows beyond a wall as mirror
 *              images of the rows next to it (zero normal gradient: neutral wetting).
 *              x stays periodic.  D2Q9 only; both schedules: the single pass computes
 *              every row at least three rows from a wall (their update reaches no row
 *              beyond one) and three staged launches then redo the rows next to the
 *              walls.  Single handles only (batches and mclb_step_noalloc reject it)
 *   mass_every 0 (off, the default) or the period, in timesteps, of the per-component
 *              mass compensation.  Eq. ff1 and the collision keep every component's total
 *              mass exactly; stored in FP32 or 16 bits, the rounding of each site's
 *              post-collision values does not, and at a stationary state it repeats step
 *              after step (measured: 1e-5 relative over 40000 steps).  With mass_every =
 *              k, every k-th mclb_step timestep (counted from the last mclb_init_fields or
 *              mclb_set_state, which record the reference) is followed by an FP64 sum of
 *              each component's stored mass and the addition of its deficit against the
 *              reference, spread evenly over the sites, to every site's rest population
 *              (in the 16-bit formats to R, which gives w_i of it to each population):
 *              zero velocity, so momentum is unchanged.  What remains is the rounding of
 *              that addition, below one unit in the last place of the rest population per
 *              site.  Costs one read of the state and one read and write of the rest
 *              populations per k steps.  Single handles only: mclb_batch_create and
 *              mclb_step_noalloc reject a non-zero value; < 0 is EINVAL. */
typedef struct {
    int ncomp;
    int nx, ny;
    double tau;
    const double* chi;
    const double* m;
    double theta;
    double kappa;
    double force[2];
    int precision;
    int kernel;
    void* stream;
    int forcing_velocity;
    int lattice;
    int force_form;
    int mass_every;
    int nz;
    double force_z;
    int walls;
} mclb_params;

typedef struct mclb_handle_s* mclb_handle;

/* Validate params and allocate the device state of one simulation.  The
 * distributions start at zero: call mclb_init_fields or mclb_set_state next.
 * A D1Q3 lattice needs ny = 1 and FP64 or FP32 storage; params->kernel is ignored
 * there (lines of up to a few hundred to 1024 sites, depending on N and precision,
 * live in one CTA's shared memory and advance up to 4096 timesteps per launch; longer
 * lines advance one timestep per launch).
 * Errors: EINVAL (any parameter out of range, asymmetric or non-finite chi),
 * ENOMEM, ECUDA.  *out is set to NULL on failure. */
int mclb_create(const mclb_params* params, mclb_handle* out);

/* Set f^s_i(r, 0) to the equilibrium of the given fields (Sec. 3 equilibrium
 * moments with the barycentric u).  rho: N*ny*nx component densities rho^s, each
 * > 0 in total per site; u: 2*ny*nx barycentric velocity (D3Q19: N*nz*ny*nx densities,
 * 3*nz*ny*nx velocity) or NULL for rest.
 * Host pointers; the copy is synchronous.  The values are checked on the device after
 * the upload; on EINVAL the message names the first failing site and the state is
 * left as it was.  Resets the step counter.  Errors: EHANDLE, EINVAL (NULL rho,
 * non-finite value, non-positive total density), ECUDA. */
int mclb_init_fields(mclb_handle h, const double* rho, const double* u);

/* As mclb_init_fields, but rho and u are device pointers (same layouts) read in
 * stream order; the call does not synchronise and does not validate the values. */
int mclb_init_fields_device(mclb_handle h, const double* rho, const double* u);

/* Enqueue nsteps timesteps (Eq. ssLB with the Eq. definef force) on the handle's
 * stream and return without waiting for them.  nsteps >= 0.  The return value
 * reports the device status word of earlier work that has already completed
 * (ENONFINITE once a non-finite value or a non-positive total density was seen);
 * mclb_status synchronises and reports everything enqueued so far. */
int mclb_step(mclb_handle h, long nsteps);

/* Synchronise the stream and return the device status: OK, ENONFINITE or ETIMEOUT. */
int mclb_status(mclb_handle h);

/* Macroscopic fields of the current state (any pointer may be NULL).  Host
 * pointers, synchronises.
 *   rho (N*ny*nx)  component densities rho^s = sum_i f^s_i               (Sec. 3)
 *   U   (2*ny*nx)  fluid velocity U = u + a/2 with rho a = sum_s rho^s a^s (Eq. scon)
 *                  (D3Q19: every field over nz*ny*nx sites, U 3 and P 6 components)
 *   mu  (N*ny*nx)  chemical potential per unit mass mu^s/m^s, gradient term included
 *   P   (3*ny*nx)  pressure tensor P_xx, P_xy, P_yy:
 *                  (sum_s rho^s mu^s/m^s - psi) I + kappa sum_s grad rho^s grad rho^s,
 *                  psi the Eq. lgf density plus the gradient energy (Eq. ppp, diagnostic) */
int mclb_moments(mclb_handle h, double* rho, double* U, double* mu, double* P);

/* As mclb_moments into device pointers, in stream order, without synchronising. */
int mclb_moments_device(mclb_handle h, double* rho, double* U, double* mu, double* P);

/* FP64 global sums of the current state (any pointer may be NULL), synchronises:
 *   mass (N)       sum over sites of rho^s                (kept by Eq. ff1)
 *   mom (2)        sum over sites of rho u                (Sec. 3 moments)
 *   force_sum (2)  sum over sites of sum_s rho^s a^s      (the next step adds it to mom)
 * (D3Q19: mom and force_sum have 3 components.) */
int mclb_conservation(mclb_handle h, double* mass, double* mom, double* force_sum);

/* Mean compositions phi^s = rho^s / rho of the nphase bulk phases of the current
 * state, all computed on the device in FP64: the compositions, the bulk mask (sites
 * whose composition gradient is below 1e-3 in every component) and a k-means of the
 * bulk sites into nphase groups, group c started at the bulk site richest in component
 * c, with sums in a fixed order (the result is deterministic); only the nphase*N means
 * come back.  phi receives nphase*N values, group c first.  nphase in 1..N.  Synchronises.  Errors: EHANDLE, EINVAL (nphase out
 * of range, no bulk site), ENOMEM, ECUDA.  Sec. 4 compares these coexisting
 * compositions with the Flory-Huggins binodal. */
int mclb_fit_equilibrium(mclb_handle h, int nphase, double* phi);

/* Copy the distributions in or out as FP64 pre-collision values f^s_i(r, t), layout
 * [s][i][y][x] (count must equal N*9*ny*nx; on D1Q3 [s][i][x], count N*3*nx; on D3Q19
 * [s][i][z][y][x], count N*19*nz*ny*nx).  Host pointers, synchronous.  Getting
 * and setting a state is exact in FP64 and FP32; in the shifted modes setting
 * stores the state as R and 16-bit deviations (see mclb_precision), so a state
 * read back differs by the rounding of the deviations.  set_state checks the values
 * on the device after the upload and leaves the state as it was if one is not finite.
 * Errors: EHANDLE, EINVAL (count, NULL, a non-finite value), ECUDA. */
int mclb_get_state(mclb_handle h, double* f, size_t count);
int mclb_set_state(mclb_handle h, const double* f, size_t count);

/* Timesteps taken since the last init / set_state. */
long mclb_step_count(mclb_handle h);

/* ----------------------------------------------------------------------------
 * Bands of rows, for splitting one periodic D2Q9 lattice into y slabs (one handle per
 * slab, on one or several GPUs).  The paper has one periodic lattice; the split rests on
 * how far one timestep reaches.  A site's post-collision values depend on the stored
 * values at most 3 rows away: the pull of Eq. ssLB reaches 1 row, the force of Eq.
 * definef takes a centred gradient of mu^s (1 row more), and mu^s holds the Laplacian
 * -kappa lap rho^s (1 row more).  So a slab of h rows stored in a handle of h + 2G rows,
 * whose G rows on each side are copies of the neighbouring slabs' rows, advances its own
 * h rows exactly as the whole lattice would for G / 3 timesteps, whatever the handle does
 * beyond its edges (the paper_0704_3444_gb300 package gives it walls = 1); then the G
 * outer rows are refreshed from the neighbours' bands.  The package's SlabDecomposition
 * and LocalSlabs do this.
 *
 * A band is the stored (post-collision, pull-scheme) representation itself, copied
 * byte for byte: per component, the nine velocity lines of each row with their ghost
 * columns, then in the 16-bit formats each row's FP32 density line.  Packing a band of
 * one handle and unpacking it into another handle with the same N, nx and precision is
 * exact in every format.  Rows are [y0, y0 + nrows), 0 <= y0, y0 + nrows <= ny.
 *
 * mclb_rows_bytes: bytes of a band of nrows rows (0 on a bad handle, a lattice other than
 *   D2Q9, or nrows < 0).
 * mclb_pack_rows_device / mclb_unpack_rows_device: copy the band between the current
 *   state and buf, a buffer of mclb_rows_bytes(h, nrows) bytes in device memory (or host
 *   memory pinned for the device), in stream order, without synchronising.  The caller
 *   owns buf and keeps it alive until the stream has passed the copy.  Unpacking does not
 *   check the values, leaves the step counter alone and is not seen by the mass
 *   compensation (mass_every), whose reference is the whole handle.
 *   Errors: EHANDLE, EINVAL (lattice not D2Q9, rows out of range, NULL buffer with
 *   nrows > 0), ECUDA.
 * mclb_conservation_rows: the sums of mclb_conservation over the rows [y0, y0 + nrows)
 *   only (mass N, mom 2, force_sum 2; zeros for nrows = 0).  Host pointers, any may be
 *   NULL; synchronises.  Errors: EHANDLE, EINVAL, ECUDA. */
size_t mclb_rows_bytes(mclb_handle h, int nrows);
int mclb_pack_rows_device(mclb_handle h, int y0, int nrows, void* buf);
int mclb_unpack_rows_device(mclb_handle h, int y0, int nrows, const void* buf);
int mclb_conservation_rows(mclb_handle h, int y0, int nrows, double* mass, double* mom,
                           double* force_sum);

/* Test hook for the failure path of the single-pass kernel (no counterpart in the
 * paper): while on != 0, its steps issue no copies, so every CTA's first bounded wait
 * runs out (after about 2 s), the CTA returns, and mclb_status then reports
 * MCLB_ETIMEOUT.  The distributions are left unspecified: initialise again after
 * switching it off.  Steps are not replayed from CUDA graphs while it is on.  No effect
 * on the staged schedule.  Errors: EHANDLE. */
int mclb_test_withhold_copies(mclb_handle h, int on);

/* HBM bytes one timestep must move at least: every stored value read once and
 * written once, 2 * N * ny * nx * (9 * storage size) in FP64 and FP32 and
 * 2 * N * ny * nx * (9 * 2 + 4) in the shifted modes (3 in place of 9 on D1Q3). */
double mclb_bytes_per_step(mclb_handle h);

/* Kernel launches one timestep issues (2 for the fused schedule: the single pass and
 * the refresh of the periodic ghost columns; 3 for the staged; 1 on D1Q3, where one
 * launch advances a resident line by up to 4096 timesteps). */
int mclb_launches_per_step(mclb_handle h);

/* Release everything the handle owns.  NULL is accepted.  Synchronises. */
int mclb_destroy(mclb_handle h);

/* Message describing the most recent failure on this thread ("" if none). */
const char* mclb_last_error(void);

/* ----------------------------------------------------------------------------
 * Allocation-free timestep.  (The paper has no counterpart; this is a service for
 * callers that cannot allocate device memory: code that runs inside a host
 * application which owns a fixed, pre-reserved device memory budget, or code that must
 * not call cudaMalloc/cudaFree because those calls synchronise the device and would
 * break the caller's own overlap of work.)
 *
 * mclb_step_noalloc advances the distributions by one timestep with the staged
 * schedule in FP64 on the D2Q9 lattice (params->precision must be MCLB_FP64 and
 * params->lattice MCLB_D2Q9; params->kernel is ignored).
 * Its two scratch fields live in one fixed array inside the library (a static device
 * array of 2 * MCLB_NOALLOC_MAX_COMP_SITES doubles, 8 MiB, which every GPU that loads
 * the library holds until the process exits); the call allocates nothing.
 *   f_in   device array, N*9*ny*nx doubles, pre-collision f^s_i(r, t) in the layout of
 *          mclb_get_state ([s][i][y][x]); read only
 *   f_out  device array of the same size that shares no byte with f_in; receives
 *          f^s_i(r, t + 1)
 * Work is enqueued on params->stream (NULL: the legacy default stream) and the call
 * returns without waiting.  Errors: EINVAL for invalid params, a precision other than
 * FP64, another lattice, NULL or overlapping arrays, or N*nx*ny above
 * MCLB_NOALLOC_MAX_COMP_SITES; ECUDA if no device is usable or a launch fails.
 * Non-finite values are not reported.  Every call made outside a stream capture looks
 * up the array's device address on the current device (so a device reset is followed);
 * a call inside a capture reuses the address of the last call outside one, so make the
 * first call on a device before any stream capture (EINVAL otherwise).  All calls share
 * the one array, so calls that overlap on the GPU (on different streams, or from
 * several threads) race with each other; serialise them.
 * ------------------------------------------------------------------------- */
#define MCLB_NOALLOC_MAX_COMP_SITES 524288 /* largest N * nx * ny */
int mclb_step_noalloc(const mclb_params* params, const double* f_in, double* f_out);

/* ----------------------------------------------------------------------------
 * Batched simulations: count independent problems (each its own N, grid, chi, tau,
 * ...) advanced together.  Per timestep, for each distinct N in the batch, one launch
 * of the single-pass kernel covers every instance with that N (each CTA finds its
 * instance, column strip and row segment in a table built at the first step) and one
 * launch refreshes their ghost columns; where that kernel cannot be set up the group
 * falls back to the staged schedule (three launches).  The first step after the batch
 * is (re)built picks each group's work partition -- the strip shape (the single-lattice
 * kernel's, or a narrow one with two compute warps and 56 columns per CTA) and the segment
 * height (2, 4, 8 or 16 waves of resident CTAs) -- by timing every candidate on the current
 * state (the state is not changed; the call synchronises; mclb_batch_tuning reports it).
 * Steps are replayed from a CUDA graph in chunks of 32.  D1Q3 instances of one N
 * advance together in one launch per 4096 timesteps (one CTA per line, the line in
 * shared memory; lines too long for that step one launch per timestep).  precision
 * and stream are taken from params[0]; kernel is ignored.  D3Q19 instances are rejected.
 * Instances share no data.  Every instance must be initialised
 * (mclb_batch_init_fields) before the first mclb_batch_step.  Errors as for the
 * single-simulation calls, and EINVAL for an index outside 0..count-1.
 * ------------------------------------------------------------------------- */
typedef struct mclb_batch_s* mclb_batch;

int mclb_batch_create(const mclb_params* params, int count, mclb_batch* out);
int mclb_batch_init_fields(mclb_batch b, int index, const double* rho, const double* u);
/* Enqueue nsteps timesteps of every instance; returns without waiting. */
int mclb_batch_step(mclb_batch b, long nsteps);
/* Kernel launches one batched timestep issues (2 per distinct N, 3 for a group on the
 * staged schedule; D1Q3 lines: 1 per distinct N, plus 1 per line too long for shared
 * memory). */
int mclb_batch_launches_per_step(mclb_batch b);

/* The work partition the autotuner picked for each group of D2Q9 instances that share N
 * (groups in ascending N; D1Q3 lines are not included): narrow[g] = 1 where it picked the
 * narrow strip shape (two compute warps, 56 written columns per CTA) over the wide one (the
 * single-lattice kernel's, 112 columns where it has four compute warps), waves[g] = how many
 * waves of resident CTAs its segment height makes (2, 4, 8 or 16), or 0 where the group
 * runs the staged schedule.  The pick is made by timing every candidate on the first step
 * after the batch is (re)built; before that the defaults are reported.  Host arrays of cap
 * entries; returns the number of groups (entries beyond cap are not written), or -1 on an
 * invalid batch.  Synchronises only if the batch's tables have to be built. */
int mclb_batch_tuning(mclb_batch b, int* narrow, int* waves, int cap);

/* Test hook (no counterpart in the paper): make every group of D2Q9 instances use the
 * candidate partition (narrow strips or not, waves 2, 4, 8 or 16) instead of the timed
 * pick, so that each candidate's results can be checked.  Groups without that candidate
 * (no narrow shape for their N, the staged schedule) keep theirs.  Returns the number of
 * groups that switched, or -1 on an invalid batch or argument. */
int mclb_test_batch_partition(mclb_batch b, int narrow, int waves);
int mclb_batch_moments(mclb_batch b, int index, double* rho, double* U, double* mu, double* P);
/* mclb_fit_equilibrium of one instance (Sec. 4 coexisting compositions). */
int mclb_batch_fit_equilibrium(mclb_batch b, int index, int nphase, double* phi);
int mclb_batch_get_state(mclb_batch b, int index, double* f, size_t count);
/* per_instance (count ints, may be NULL) receives each instance's status; the
 * return value is the first non-OK status or OK.  Synchronises. */
int mclb_batch_status(mclb_batch b, int* per_instance);
double mclb_batch_bytes_per_step(mclb_batch b);
int mclb_batch_destroy(mclb_batch b);

#ifdef __cplusplus
}
#endif

#endif /* MCLB_H */
