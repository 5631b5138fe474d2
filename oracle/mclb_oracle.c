/*
 * mclb_oracle.c -- plain FP64 CPU oracle for one timestep of the symmetric
 * free-energy multicomponent lattice Boltzmann method (Li & Wagner,
 * arXiv:0704.3444, "A Symmetric Free Energy Based Multi-Component Lattice
 * Boltzmann Method").
 *
 * TEST INFRASTRUCTURE ONLY.  The test suite, the smoke check and the
 * benchmark's CPU-baseline leg are the only callers.  This file shares no code,
 * header, table or constant generator with the CUDA library; the two meet only
 * through the seeded input generators and through arrays compared in tests.
 *
 * The step follows the paper in its own order, one plain loop per stage, FP64
 * throughout, fixed summation orders (velocities i = 0..8, components
 * sigma = 0..N-1), two buffers and periodic wrap:
 *
 *   1. moments        rho^s = sum_i f^s_i, rho^s u^s = sum_i f^s_i v_i,
 *                     rho = sum_s rho^s, rho u = sum_s rho^s u^s       (Sec. 3)
 *   2. potentials     Flory-Huggins chemical potential (Eq. lgf, Eq.
 *                     chemicalpotential) plus the gradient term, and
 *                     nu^s = mu^s - (1/3) ln rho^s                     (Eq. definef)
 *   3. forces         rho^s a^s = -(1 - 1/(2 tau)) rho^s grad nu^s     (Eq. definef)
 *                     plus the body acceleration g of the momentum
 *                     equation (Eq. NSEeq)
 *   4. collision      f* = f + (f^e - f)/tau + F                       (Eq. ssLB)
 *                     with f^e and F the D2Q9 polynomials whose moments
 *                     are the ones listed in Sec. 3
 *   5. streaming      f(r + v_i, t + 1) = f*(r, t)                     (Eq. ssLB)
 *
 * Readings of points the paper leaves open:
 *   - mu is used per unit mass, mu^s / m^s = d psi / d rho^s, so that
 *     rho^s grad(mu^s/m^s) = n^s grad mu^s (identical for m = 1);
 *   - theta, the Flory-Huggins temperature, is a free parameter;
 *   - gradient term: psi += sum_s (kappa/2) |grad rho^s|^2, hence
 *     mu^s gains -kappa lap rho^s;
 *   - discrete operators: grad g = 3 sum_i w_i v_i g(r + v_i),
 *     lap g = 6 sum_i w_i (g(r + v_i) - g(r));
 *   - the logarithms of nu^s are combined as
 *     (theta/m^s - 1/3) ln rho^s - (theta/m^s) ln rho, the first term is
 *     dropped when its coefficient is exactly zero and otherwise uses
 *     max(rho^s, 1e-12 rho);
 *   - f^e is built with the bare barycentric u, F with rho^s u^s = j^s as
 *     Eq. ff3 prints it (or, when forcing_velocity = 1, with rho^s u);
 *   - the forces are those of Eq. definef for each component (or, when
 *     force_form = 1 and kappa = 0, shifted so that their sum is the Gibbs-Duhem
 *     total (1 - 1/(2 tau)) (1/3) grad rho);
 *     the output velocity is U = u + a/2 with rho a = sum_s rho^s a^s;
 *   - initial distributions are the equilibria of the given fields;
 *   - optional solid walls in y (walls = 1; the paper has none): halfway bounce-back
 *     of the populations, mirrored rows in the stencils (see oracle_params).
 *
 * Layout: f[((s * 9 + i) * ny + y) * nx + x], the pre-collision distribution
 * of component s, velocity i at site (x, y) at the current time.
 * D2Q9 velocities: v_0 = (0,0); v_1..4 = (1,0), (0,1), (-1,0), (0,-1);
 * v_5..8 = (1,1), (-1,1), (-1,-1), (1,-1).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_QMAX 9
#define OR_NMAX 8

/* forcing_velocity selects the velocity in the second moment of the forcing
 * (Eq. ff3): 0 = the component velocity u^s as printed, rho^s (a^s u^s + u^s a^s);
 * 1 = the barycentric u, rho^s (a^s u + u a^s), the form whose sum over the
 * components is the one-fluid forcing moment rho (a u + u a) (Eq. olso). */
/* force_form selects how the component forces of Eq. definef are summed: 0 = each
 * component's force as Eq. definef prints it; 1 = the Gibbs-Duhem reading (kappa = 0
 * only): the forces keep their differences but their sum over the components is
 * replaced by the continuum total that Gibbs-Duhem gives for the Flory-Huggins free
 * energy (whose pressure sum rho mu - psi vanishes), (1 - 1/(2 tau)) (1/3) grad rho. */
/* nz and gz are read by the D3Q19 path only (the other lattices ignore them).
 * walls (D2Q9 only): 0 = periodic in y; 1 = stationary solid walls halfway between
 * rows, below row 0 and above row ny - 1 (the paper has no walls: a reading for the
 * membrane-formation set-up its introduction motivates).  A population that would
 * stream across a wall returns to its site with the opposite velocity (halfway
 * bounce-back), and the stencils of rho^s, nu^s and rho see the wall rows as mirror
 * images of the rows next to them (zero normal gradient: neutral wetting). */
typedef struct {
    int ncomp, nx, ny;
    double tau, theta, kappa, gx, gy;
    double chi[OR_NMAX * OR_NMAX];
    double m[OR_NMAX];
    int forcing_velocity;
    int force_form;
    int nz;
    double gz;
    int walls;
} oracle_params;

static const int VX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int VY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double WT[9] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};   /* v_OPP[i] = -v_i */
static const double LOG_FLOOR = 1e-12;

int oracle_nthreads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static int check(const oracle_params* p)
{
    if (!p || p->ncomp < 1 || p->ncomp > OR_NMAX || p->nx < 1 || p->ny < 1) return -1;
    if (!(p->tau > 0.5)) return -1;
    if (p->forcing_velocity != 0 && p->forcing_velocity != 1) return -1;
    if (p->force_form != 0 && p->force_form != 1) return -1;
    if (p->force_form == 1 && p->kappa != 0.0) return -1;
    if (p->walls != 0 && p->walls != 1) return -1;
    return 0;
}

static inline long wrap(long a, long n) { a %= n; return a < 0 ? a + n : a; }

/* ---------------------------------------------------------------- per site */

/* f^e_i with sum f^e = rho^s, sum f^e v = rho^s u, sum f^e v v = rho^s/3 I + rho^s u u
 * (Sec. 3, equilibrium moments of one component; the D2Q9 second-order polynomial). */
void oracle_equilibrium(double rho_s, double ux, double uy, double* fe)
{
    double uu = ux * ux + uy * uy;
    for (int i = 0; i < 9; ++i) {
        double cu = VX[i] * ux + VY[i] * uy;
        fe[i] = WT[i] * rho_s * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
    }
}

/* F_i with sum F = 0, sum F v = rho^s a^s, sum F v v = rho^s (a^s u^s + u^s a^s)
 * (Eqs. ff1-ff3), rho^s u^s = j^s. */
void oracle_forcing(double rho_s, double jx, double jy, double ax, double ay, double* F)
{
    double aj = ax * jx + ay * jy;
    for (int i = 0; i < 9; ++i) {
        double ca = VX[i] * ax + VY[i] * ay;
        double cj = VX[i] * jx + VY[i] * jy;
        F[i] = WT[i] * (3.0 * rho_s * ca + 9.0 * ca * cj - 3.0 * aj);
    }
}

/* Flory-Huggins free energy density of Eq. lgf with n^s = rho^s / m^s and
 * phi^s = rho^s / rho:  psi = theta [ -sum n m + sum n ln phi + 1/2 sum chi m n phi' ]. */
double oracle_psi(const oracle_params* p, const double* rs)
{
    int N = p->ncomp;
    double rho = 0.0;
    for (int s = 0; s < N; ++s) rho += rs[s];
    double psi = 0.0;
    for (int s = 0; s < N; ++s) {
        double n = rs[s] / p->m[s];
        double phi = rs[s] / rho;
        psi += -p->theta * n * p->m[s];
        psi += n * p->theta * log(phi);
        for (int t = 0; t < N; ++t)
            psi += 0.5 * p->chi[s * N + t] * p->theta * p->m[s] * n * (rs[t] / rho);
    }
    return psi;
}

/* Mass-specific bulk chemical potential mu^s/m^s = d psi / d rho^s of Eq. lgf:
 * theta [ (ln phi^s + 1)/m^s - 1 - sum_t phi^t/m^t + sum_t chi^{st} phi^t
 *         - 1/2 sum_{t,t'} chi^{tt'} phi^t phi^t' ]. */
void oracle_mu_bulk(const oracle_params* p, const double* rs, double* mu)
{
    int N = p->ncomp;
    double rho = 0.0;
    for (int s = 0; s < N; ++s) rho += rs[s];
    double phi[OR_NMAX], chiphi[OR_NMAX];
    double sum_phi_m = 0.0, quad = 0.0;
    for (int s = 0; s < N; ++s) phi[s] = rs[s] / rho;
    for (int s = 0; s < N; ++s) sum_phi_m += phi[s] / p->m[s];
    for (int s = 0; s < N; ++s) {
        chiphi[s] = 0.0;
        for (int t = 0; t < N; ++t) chiphi[s] += p->chi[s * N + t] * phi[t];
    }
    for (int s = 0; s < N; ++s) quad += 0.5 * phi[s] * chiphi[s];
    for (int s = 0; s < N; ++s) {
        double ph = phi[s] > LOG_FLOOR ? phi[s] : LOG_FLOOR;
        mu[s] = p->theta * ((log(ph) + 1.0) / p->m[s] - 1.0 - sum_phi_m + chiphi[s] - quad);
    }
}

/* ------------------------------------------------------------- whole field */

typedef struct {
    long S;
    double *rs, *jx, *jy;      /* per component: rho^s, j^s = rho^s u^s   (N*S) */
    double *rho, *ux, *uy;     /* total density and barycentric velocity  (S)   */
    double *nu;                /* mu^s - 1/3 ln rho^s                     (N*S) */
    double *ax, *ay;           /* a^s                                     (N*S) */
} work_t;

static int work_alloc(const oracle_params* p, work_t* w)
{
    long S = (long)p->nx * p->ny, N = p->ncomp;
    w->S = S;
    w->rs = malloc(sizeof(double) * N * S);
    w->jx = malloc(sizeof(double) * N * S);
    w->jy = malloc(sizeof(double) * N * S);
    w->rho = malloc(sizeof(double) * S);
    w->ux = malloc(sizeof(double) * S);
    w->uy = malloc(sizeof(double) * S);
    w->nu = malloc(sizeof(double) * N * S);
    w->ax = malloc(sizeof(double) * N * S);
    w->ay = malloc(sizeof(double) * N * S);
    return (w->rs && w->jx && w->jy && w->rho && w->ux && w->uy && w->nu && w->ax && w->ay) ? 0 : -2;
}

static void work_free(work_t* w)
{
    free(w->rs); free(w->jx); free(w->jy); free(w->rho); free(w->ux); free(w->uy);
    free(w->nu); free(w->ax); free(w->ay);
}

/* Row of the neighbour y + dy seen by a stencil: periodic, or with walls the mirror
 * image of the row next to the wall (rows -1 and ny read rows 0 and ny - 1). */
static long stencil_row(long y, int dy, int ny, int walls)
{
    long yy = y + dy;
    if (!walls) return wrap(yy, ny);
    return yy < 0 ? 0 : (yy >= ny ? ny - 1 : yy);
}

/* Discrete lap g = 6 sum_i w_i (g(r + v_i) - g(r)) of one scalar field. */
static double lap_at(const double* g, int nx, int ny, int walls, int x, int y)
{
    double c = g[(long)y * nx + x], acc = 0.0;
    for (int i = 0; i < 9; ++i) {
        long xx = wrap(x + VX[i], nx), yy = stencil_row(y, VY[i], ny, walls);
        acc += WT[i] * (g[yy * nx + xx] - c);
    }
    return 6.0 * acc;
}

/* Discrete grad g = 3 sum_i w_i v_i g(r + v_i). */
static void grad_at(const double* g, int nx, int ny, int walls, int x, int y, double* gx,
                    double* gy)
{
    double ax = 0.0, ay = 0.0;
    for (int i = 0; i < 9; ++i) {
        long xx = wrap(x + VX[i], nx), yy = stencil_row(y, VY[i], ny, walls);
        double v = g[yy * nx + xx];
        ax += WT[i] * VX[i] * v;
        ay += WT[i] * VY[i] * v;
    }
    *gx = 3.0 * ax;
    *gy = 3.0 * ay;
}

/* Stage 1: moments of the pre-collision distributions (Sec. 3). */
static void stage_moments(const oracle_params* p, const double* f, work_t* w)
{
    int N = p->ncomp, nx = p->nx, ny = p->ny;
    long S = w->S;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            long c = (long)y * nx + x;
            double rho = 0.0, jxt = 0.0, jyt = 0.0;
            for (int s = 0; s < N; ++s) {
                double r = 0.0, jx = 0.0, jy = 0.0;
                for (int i = 0; i < 9; ++i) {
                    double v = f[(long)(s * 9 + i) * S + c];
                    r += v;
                    jx += v * VX[i];
                    jy += v * VY[i];
                }
                w->rs[s * S + c] = r;
                w->jx[s * S + c] = jx;
                w->jy[s * S + c] = jy;
                rho += r;
                jxt += jx;
                jyt += jy;
            }
            w->rho[c] = rho;
            w->ux[c] = jxt / rho;
            w->uy[c] = jyt / rho;
        }
    }
}

/* Stage 2: nu^s = mu^s/m^s - kappa lap rho^s - (1/3) ln rho^s (Eq. lgf, Eq.
 * chemicalpotential, Eq. definef), logarithms combined as described above. */
static void stage_potentials(const oracle_params* p, work_t* w)
{
    int N = p->ncomp, nx = p->nx, ny = p->ny;
    long S = w->S;
    double th = p->theta;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            long c = (long)y * nx + x;
            double rho = w->rho[c];
            double phi[OR_NMAX], chiphi[OR_NMAX];
            double sum_phi_m = 0.0, quad = 0.0;
            for (int s = 0; s < N; ++s) phi[s] = w->rs[s * S + c] / rho;
            for (int s = 0; s < N; ++s) sum_phi_m += phi[s] / p->m[s];
            for (int s = 0; s < N; ++s) {
                chiphi[s] = 0.0;
                for (int t = 0; t < N; ++t) chiphi[s] += p->chi[s * N + t] * phi[t];
            }
            for (int s = 0; s < N; ++s) quad += 0.5 * phi[s] * chiphi[s];
            double lnrho = log(rho);
            for (int s = 0; s < N; ++s) {
                double rs = w->rs[s * S + c];
                double coef = th / p->m[s] - 1.0 / 3.0;
                double logs = -(th / p->m[s]) * lnrho;
                if (coef != 0.0) {
                    double r = rs > LOG_FLOOR * rho ? rs : LOG_FLOOR * rho;
                    logs += coef * log(r);
                }
                double bulk = th * (1.0 / p->m[s] - 1.0 - sum_phi_m + chiphi[s] - quad);
                double grad_term = -p->kappa * lap_at(w->rs + s * S, nx, ny, p->walls, x, y);
                w->nu[s * S + c] = logs + bulk + grad_term;
            }
        }
    }
}

/* Stage 3: a^s = -(1 - 1/(2 tau)) grad nu^s + g (Eq. definef; g from Eq. NSEeq). */
static void stage_forces(const oracle_params* p, work_t* w)
{
    int N = p->ncomp, nx = p->nx, ny = p->ny;
    long S = w->S;
    double coef = 1.0 - 1.0 / (2.0 * p->tau);
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            long c = (long)y * nx + x;
            for (int s = 0; s < N; ++s) {
                double gx, gy;
                grad_at(w->nu + s * S, nx, ny, p->walls, x, y, &gx, &gy);
                w->ax[s * S + c] = -coef * gx + p->gx;
                w->ay[s * S + c] = -coef * gy + p->gy;
            }
        }
    }
    if (p->force_form == 1) {
        /* Gibbs-Duhem reading: every a^s shifted by the same (A_c - A)/rho, where
         * A = sum_s rho^s (a^s - g) and A_c = (1 - 1/(2 tau)) (1/3) grad rho, so that the
         * components' forces sum to A_c + rho g and their differences are kept */
#pragma omp parallel for schedule(static)
        for (int y = 0; y < ny; ++y) {
            for (int x = 0; x < nx; ++x) {
                long c = (long)y * nx + x;
                double Ax = 0.0, Ay = 0.0, gx, gy;
                for (int s = 0; s < N; ++s) {
                    Ax += w->rs[s * S + c] * (w->ax[s * S + c] - p->gx);
                    Ay += w->rs[s * S + c] * (w->ay[s * S + c] - p->gy);
                }
                grad_at(w->rho, nx, ny, p->walls, x, y, &gx, &gy);
                double dx = (coef * gx / 3.0 - Ax) / w->rho[c];
                double dy = (coef * gy / 3.0 - Ay) / w->rho[c];
                for (int s = 0; s < N; ++s) {
                    w->ax[s * S + c] += dx;
                    w->ay[s * S + c] += dy;
                }
            }
        }
    }
}

/* Stages 4 and 5: BGK collision with forcing, then streaming (Eq. ssLB). */
static void stage_collide_stream(const oracle_params* p, const double* f, const work_t* w,
                                 double* fnew)
{
    int N = p->ncomp, nx = p->nx, ny = p->ny;
    long S = w->S;
    double tau = p->tau;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            long c = (long)y * nx + x;
            for (int s = 0; s < N; ++s) {
                double fe[9], F[9];
                double rs = w->rs[s * S + c];
                double jx = w->jx[s * S + c], jy = w->jy[s * S + c];
                if (p->forcing_velocity) { jx = rs * w->ux[c]; jy = rs * w->uy[c]; }
                oracle_equilibrium(rs, w->ux[c], w->uy[c], fe);
                oracle_forcing(rs, jx, jy, w->ax[s * S + c], w->ay[s * S + c], F);
                for (int i = 0; i < 9; ++i) {
                    double fi = f[(long)(s * 9 + i) * S + c];
                    double post = fi + (fe[i] - fi) / tau + F[i];
                    long yy = y + VY[i];
                    if (p->walls && (yy < 0 || yy >= ny)) {
                        /* halfway bounce-back: back to this site, opposite velocity */
                        fnew[(long)(s * 9 + OPP[i]) * S + c] = post;
                    } else {
                        long xx = wrap(x + VX[i], nx);
                        fnew[(long)(s * 9 + i) * S + wrap(yy, ny) * nx + xx] = post;
                    }
                }
            }
        }
    }
}

static void compute_fields(const oracle_params* p, const double* f, work_t* w)
{
    stage_moments(p, f, w);
    stage_potentials(p, w);
    stage_forces(p, w);
}

/* f(r, 0) = f^e(rho^s(r), u(r)) for every component. */
int oracle_init(const oracle_params* p, const double* rho, const double* u, double* f)
{
    if (check(p)) return -1;
    int N = p->ncomp;
    long S = (long)p->nx * p->ny;
    for (int s = 0; s < N; ++s)
        for (long c = 0; c < S; ++c) {
            double fe[9];
            oracle_equilibrium(rho[s * S + c], u ? u[c] : 0.0, u ? u[S + c] : 0.0, fe);
            for (int i = 0; i < 9; ++i) f[(long)(s * 9 + i) * S + c] = fe[i];
        }
    return 0;
}

/* Advance f (in place) by nsteps timesteps.  Returns 0, -1 for invalid
 * parameters, -2 if memory ran out, 1 if a non-finite value appeared. */
int oracle_run(const oracle_params* p, double* f, long nsteps)
{
    if (check(p)) return -1;
    work_t w;
    if (work_alloc(p, &w)) { work_free(&w); return -2; }
    long total = (long)9 * p->ncomp * w.S;
    double* g = malloc(sizeof(double) * total);
    if (!g) { work_free(&w); return -2; }
    double *cur = f, *nxt = g;
    for (long t = 0; t < nsteps; ++t) {
        compute_fields(p, cur, &w);
        stage_collide_stream(p, cur, &w, nxt);
        double* tmp = cur; cur = nxt; nxt = tmp;
    }
    if (cur != f) memcpy(f, cur, sizeof(double) * total);
    free(g);
    work_free(&w);
    for (long k = 0; k < total; ++k)
        if (!isfinite(f[k])) return 1;
    return 0;
}

/* Macroscopic output fields of state f (any pointer may be NULL):
 *   rho (N*S)  rho^s
 *   U   (2*S)  U = u + a/2, rho a = sum_s rho^s a^s         (Eq. scon)
 *   mu  (N*S)  mu^s/m^s - kappa lap rho^s                    (Eq. lgf + gradient term)
 *   P   (3*S)  P_xx, P_xy, P_yy with
 *              P = (sum_s rho^s mu^s - psi) I + kappa sum_s grad rho^s grad rho^s,
 *              psi the Eq. lgf density plus sum_s (kappa/2)|grad rho^s|^2. */
int oracle_moments(const oracle_params* p, const double* f, double* rho_out, double* U,
                   double* mu, double* P)
{
    if (check(p)) return -1;
    work_t w;
    if (work_alloc(p, &w)) { work_free(&w); return -2; }
    compute_fields(p, f, &w);
    int N = p->ncomp, nx = p->nx, ny = p->ny;
    long S = w.S;
    if (rho_out) memcpy(rho_out, w.rs, sizeof(double) * N * S);
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            long c = (long)y * nx + x;
            if (U) {
                double fx = 0.0, fy = 0.0;
                for (int s = 0; s < N; ++s) {
                    fx += w.rs[s * S + c] * w.ax[s * S + c];
                    fy += w.rs[s * S + c] * w.ay[s * S + c];
                }
                U[c] = w.ux[c] + 0.5 * fx / w.rho[c];
                U[S + c] = w.uy[c] + 0.5 * fy / w.rho[c];
            }
            if (mu || P) {
                double rsl[OR_NMAX], mub[OR_NMAX], muf[OR_NMAX];
                for (int s = 0; s < N; ++s) rsl[s] = w.rs[s * S + c];
                oracle_mu_bulk(p, rsl, mub);
                for (int s = 0; s < N; ++s)
                    muf[s] = mub[s] - p->kappa * lap_at(w.rs + s * S, nx, ny, p->walls, x, y);
                if (mu)
                    for (int s = 0; s < N; ++s) mu[s * S + c] = muf[s];
                if (P) {
                    double psi = oracle_psi(p, rsl), rmu = 0.0, gg = 0.0;
                    double pxx = 0.0, pxy = 0.0, pyy = 0.0;
                    for (int s = 0; s < N; ++s) {
                        double gx, gy;
                        grad_at(w.rs + s * S, nx, ny, p->walls, x, y, &gx, &gy);
                        rmu += rsl[s] * muf[s];
                        gg += 0.5 * p->kappa * (gx * gx + gy * gy);
                        pxx += p->kappa * gx * gx;
                        pxy += p->kappa * gx * gy;
                        pyy += p->kappa * gy * gy;
                    }
                    double iso = rmu - (psi + gg);
                    P[c] = iso + pxx;
                    P[S + c] = pxy;
                    P[2 * S + c] = iso + pyy;
                }
            }
        }
    work_free(&w);
    return 0;
}

/* Global sums of state f: mass^s = sum_r rho^s (N), momentum sum_r rho u (2),
 * force sum_r sum_s rho^s a^s (2).  Plain sums in site order. */
int oracle_conservation(const oracle_params* p, const double* f, double* mass, double* mom,
                        double* force_sum)
{
    if (check(p)) return -1;
    work_t w;
    if (work_alloc(p, &w)) { work_free(&w); return -2; }
    compute_fields(p, f, &w);
    int N = p->ncomp;
    long S = w.S;
    for (int s = 0; s < N; ++s) {
        double acc = 0.0;
        for (long c = 0; c < S; ++c) acc += w.rs[s * S + c];
        if (mass) mass[s] = acc;
    }
    double mx = 0.0, my = 0.0, fx = 0.0, fy = 0.0;
    for (long c = 0; c < S; ++c)
        for (int s = 0; s < N; ++s) {
            mx += w.jx[s * S + c];
            my += w.jy[s * S + c];
            fx += w.rs[s * S + c] * w.ax[s * S + c];
            fy += w.rs[s * S + c] * w.ay[s * S + c];
        }
    if (mom) { mom[0] = mx; mom[1] = my; }
    if (force_sum) { force_sum[0] = fx; force_sum[1] = fy; }
    work_free(&w);
    return 0;
}

/* ------------------------------------------------------------------- D1Q3
 *
 * The lattice the paper's own simulations use (Sec. 4): velocities v = 0, +1, -1
 * with weights 2/3, 1/6, 1/6 (c_s^2 = 1/3), one line of nx sites, periodic.  The
 * same stages as above in the same order; the discrete operators keep their
 * definition through the lattice's weights, grad g = 3 sum_i w_i v_i g(x + v_i) and
 * lap g = 6 sum_i w_i (g(x + v_i) - g(x)), i.e. (g(x+1) - g(x-1))/2 and
 * g(x+1) + g(x-1) - 2 g(x).  The body force is p->gx; p->ny is ignored.
 *
 * Layout: f[(s * 3 + i) * nx + x], pre-collision, velocity order 0, +1, -1. */

static const int V1[3] = {0, 1, -1};
static const double W1[3] = {2.0 / 3.0, 1.0 / 6.0, 1.0 / 6.0};

static int check1(const oracle_params* p)
{
    if (!p || p->ncomp < 1 || p->ncomp > OR_NMAX || p->nx < 1 || p->walls != 0) return -1;
    if (!(p->tau > 0.5)) return -1;
    if (p->forcing_velocity != 0 && p->forcing_velocity != 1) return -1;
    if (p->force_form != 0 && p->force_form != 1) return -1;
    if (p->force_form == 1 && p->kappa != 0.0) return -1;
    return 0;
}

/* f^e_i = w_i rho^s (1 + 3 v u + 9/2 (v u)^2 - 3/2 u^2): moments rho^s, rho^s u,
 * rho^s/3 + rho^s u^2 (Sec. 3 in one dimension). */
static void d1_equilibrium(double rs, double u, double* fe)
{
    for (int i = 0; i < 3; ++i) {
        double cu = V1[i] * u;
        fe[i] = W1[i] * rs * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * u * u);
    }
}

/* F_i = w_i (3 rho^s v a + 9 (v a)(v j) - 3 a j): moments 0, rho^s a, 2 a j (Eqs.
 * ff1-ff3 in one dimension). */
static void d1_forcing(double rs, double j, double a, double* F)
{
    for (int i = 0; i < 3; ++i) {
        double ca = V1[i] * a, cj = V1[i] * j;
        F[i] = W1[i] * (3.0 * rs * ca + 9.0 * ca * cj - 3.0 * a * j);
    }
}

static double d1_grad(const double* g, int nx, int x)
{
    double acc = 0.0;
    for (int i = 0; i < 3; ++i) acc += W1[i] * V1[i] * g[wrap(x + V1[i], nx)];
    return 3.0 * acc;
}

static double d1_lap(const double* g, int nx, int x)
{
    double acc = 0.0;
    for (int i = 0; i < 3; ++i) acc += W1[i] * (g[wrap(x + V1[i], nx)] - g[x]);
    return 6.0 * acc;
}

typedef struct {
    double *rs, *j, *rho, *u, *nu, *a;
} work1_t;

static int work1_alloc(const oracle_params* p, work1_t* w)
{
    long nx = p->nx, N = p->ncomp;
    w->rs = malloc(sizeof(double) * N * nx);
    w->j = malloc(sizeof(double) * N * nx);
    w->rho = malloc(sizeof(double) * nx);
    w->u = malloc(sizeof(double) * nx);
    w->nu = malloc(sizeof(double) * N * nx);
    w->a = malloc(sizeof(double) * N * nx);
    return (w->rs && w->j && w->rho && w->u && w->nu && w->a) ? 0 : -2;
}

static void work1_free(work1_t* w)
{
    free(w->rs); free(w->j); free(w->rho); free(w->u); free(w->nu); free(w->a);
}

/* Stages 1-3 of one D1Q3 step: moments, potentials nu^s, accelerations a^s. */
static void d1_fields(const oracle_params* p, const double* f, work1_t* w)
{
    int N = p->ncomp, nx = p->nx;
    double th = p->theta;
    for (int x = 0; x < nx; ++x) {
        double rho = 0.0, jt = 0.0;
        for (int s = 0; s < N; ++s) {
            double r = 0.0, j = 0.0;
            for (int i = 0; i < 3; ++i) {
                double v = f[(long)(s * 3 + i) * nx + x];
                r += v;
                j += v * V1[i];
            }
            w->rs[s * nx + x] = r;
            w->j[s * nx + x] = j;
            rho += r;
            jt += j;
        }
        w->rho[x] = rho;
        w->u[x] = jt / rho;
    }
    for (int x = 0; x < nx; ++x) {
        double rho = w->rho[x];
        double phi[OR_NMAX], chiphi[OR_NMAX];
        double sum_phi_m = 0.0, quad = 0.0;
        for (int s = 0; s < N; ++s) phi[s] = w->rs[s * nx + x] / rho;
        for (int s = 0; s < N; ++s) sum_phi_m += phi[s] / p->m[s];
        for (int s = 0; s < N; ++s) {
            chiphi[s] = 0.0;
            for (int t = 0; t < N; ++t) chiphi[s] += p->chi[s * N + t] * phi[t];
        }
        for (int s = 0; s < N; ++s) quad += 0.5 * phi[s] * chiphi[s];
        double lnrho = log(rho);
        for (int s = 0; s < N; ++s) {
            double rs = w->rs[s * nx + x];
            double coef = th / p->m[s] - 1.0 / 3.0;
            double logs = -(th / p->m[s]) * lnrho;
            if (coef != 0.0) {
                double r = rs > LOG_FLOOR * rho ? rs : LOG_FLOOR * rho;
                logs += coef * log(r);
            }
            double bulk = th * (1.0 / p->m[s] - 1.0 - sum_phi_m + chiphi[s] - quad);
            w->nu[s * nx + x] = logs + bulk - p->kappa * d1_lap(w->rs + s * nx, nx, x);
        }
    }
    double coef = 1.0 - 1.0 / (2.0 * p->tau);
    for (int x = 0; x < nx; ++x)
        for (int s = 0; s < N; ++s)
            w->a[s * nx + x] = -coef * d1_grad(w->nu + s * nx, nx, x) + p->gx;
    if (p->force_form == 1) {   /* Gibbs-Duhem reading, as in stage_forces */
        for (int x = 0; x < nx; ++x) {
            double A = 0.0;
            for (int s = 0; s < N; ++s) A += w->rs[s * nx + x] * (w->a[s * nx + x] - p->gx);
            double d = (coef * d1_grad(w->rho, nx, x) / 3.0 - A) / w->rho[x];
            for (int s = 0; s < N; ++s) w->a[s * nx + x] += d;
        }
    }
}

/* f(x, 0) = f^e(rho^s(x), u(x)); u may be NULL (rest). */
int oracle_d1q3_init(const oracle_params* p, const double* rho, const double* u, double* f)
{
    if (check1(p)) return -1;
    int N = p->ncomp, nx = p->nx;
    for (int s = 0; s < N; ++s)
        for (int x = 0; x < nx; ++x) {
            double fe[3];
            d1_equilibrium(rho[s * nx + x], u ? u[x] : 0.0, fe);
            for (int i = 0; i < 3; ++i) f[(long)(s * 3 + i) * nx + x] = fe[i];
        }
    return 0;
}

/* Advance f (in place) by nsteps D1Q3 timesteps.  Returns 0, -1, -2, or 1 if a
 * non-finite value appeared. */
int oracle_d1q3_run(const oracle_params* p, double* f, long nsteps)
{
    if (check1(p)) return -1;
    int N = p->ncomp, nx = p->nx;
    work1_t w;
    if (work1_alloc(p, &w)) { work1_free(&w); return -2; }
    long total = (long)3 * N * nx;
    double* g = malloc(sizeof(double) * total);
    if (!g) { work1_free(&w); return -2; }
    double *cur = f, *nxt = g;
    double tau = p->tau;
    for (long t = 0; t < nsteps; ++t) {
        d1_fields(p, cur, &w);
        for (int x = 0; x < nx; ++x)
            for (int s = 0; s < N; ++s) {
                double fe[3], F[3];
                double rs = w.rs[s * nx + x];
                double j = p->forcing_velocity ? rs * w.u[x] : w.j[s * nx + x];
                d1_equilibrium(rs, w.u[x], fe);
                d1_forcing(rs, j, w.a[s * nx + x], F);
                for (int i = 0; i < 3; ++i) {
                    double fi = cur[(long)(s * 3 + i) * nx + x];
                    double post = fi + (fe[i] - fi) / tau + F[i];
                    nxt[(long)(s * 3 + i) * nx + wrap(x + V1[i], nx)] = post;
                }
            }
        double* tmp = cur; cur = nxt; nxt = tmp;
    }
    if (cur != f) memcpy(f, cur, sizeof(double) * total);
    free(g);
    work1_free(&w);
    for (long k = 0; k < total; ++k)
        if (!isfinite(f[k])) return 1;
    return 0;
}

/* Output fields of a D1Q3 state, in the shapes of a D2Q9 state with ny = 1 (any
 * pointer may be NULL): rho (N*nx); U (2*nx) = (u + a/2, 0); mu (N*nx); P (3*nx) =
 * (iso + kappa sum_s (d_x rho^s)^2, 0, iso) with iso = sum_s rho^s mu^s - psi -
 * sum_s (kappa/2) (d_x rho^s)^2. */
int oracle_d1q3_moments(const oracle_params* p, const double* f, double* rho_out, double* U,
                        double* mu, double* P)
{
    if (check1(p)) return -1;
    int N = p->ncomp, nx = p->nx;
    work1_t w;
    if (work1_alloc(p, &w)) { work1_free(&w); return -2; }
    d1_fields(p, f, &w);
    if (rho_out) memcpy(rho_out, w.rs, sizeof(double) * N * nx);
    for (int x = 0; x < nx; ++x) {
        if (U) {
            double fx = 0.0;
            for (int s = 0; s < N; ++s) fx += w.rs[s * nx + x] * w.a[s * nx + x];
            U[x] = w.u[x] + 0.5 * fx / w.rho[x];
            U[nx + x] = 0.0;
        }
        if (mu || P) {
            double rsl[OR_NMAX], mub[OR_NMAX], muf[OR_NMAX];
            for (int s = 0; s < N; ++s) rsl[s] = w.rs[s * nx + x];
            oracle_mu_bulk(p, rsl, mub);
            for (int s = 0; s < N; ++s) muf[s] = mub[s] - p->kappa * d1_lap(w.rs + s * nx, nx, x);
            if (mu)
                for (int s = 0; s < N; ++s) mu[s * nx + x] = muf[s];
            if (P) {
                double psi = oracle_psi(p, rsl), rmu = 0.0, gg = 0.0, pxx = 0.0;
                for (int s = 0; s < N; ++s) {
                    double gx = d1_grad(w.rs + s * nx, nx, x);
                    rmu += rsl[s] * muf[s];
                    gg += 0.5 * p->kappa * gx * gx;
                    pxx += p->kappa * gx * gx;
                }
                double iso = rmu - (psi + gg);
                P[x] = iso + pxx;
                P[nx + x] = 0.0;
                P[2 * nx + x] = iso;
            }
        }
    }
    work1_free(&w);
    return 0;
}

/* Global sums of a D1Q3 state: mass^s (N), momentum (2: x, 0), force (2: x, 0). */
int oracle_d1q3_conservation(const oracle_params* p, const double* f, double* mass,
                             double* mom, double* force_sum)
{
    if (check1(p)) return -1;
    int N = p->ncomp, nx = p->nx;
    work1_t w;
    if (work1_alloc(p, &w)) { work1_free(&w); return -2; }
    d1_fields(p, f, &w);
    for (int s = 0; s < N; ++s) {
        double acc = 0.0;
        for (int x = 0; x < nx; ++x) acc += w.rs[s * nx + x];
        if (mass) mass[s] = acc;
    }
    double mx = 0.0, fx = 0.0;
    for (int x = 0; x < nx; ++x)
        for (int s = 0; s < N; ++s) {
            mx += w.j[s * nx + x];
            fx += w.rs[s * nx + x] * w.a[s * nx + x];
        }
    if (mom) { mom[0] = mx; mom[1] = 0.0; }
    if (force_sum) { force_sum[0] = fx; force_sum[1] = 0.0; }
    work1_free(&w);
    return 0;
}

/* ------------------------------------------------------------------ D3Q19
 *
 * A three-dimensional lattice for the same method (not one the paper uses; its
 * equations are written for any lattice whose weights give the Sec. 3 moments).
 * Nineteen velocities: the rest velocity (weight 1/3), the six axis directions
 * (1/18) and the twelve face diagonals (1/36), c_s^2 = 1/3; the weights are
 * isotropic to fourth order, so the equilibrium and forcing polynomials of the
 * D2Q9 path, written with three-component dot products, have the Sec. 3 and
 * Eqs. ff1-ff3 moments.  The stages are those of the D2Q9 path in the same order,
 * with grad g = 3 sum_i w_i v_i g(r + v_i) and lap g = 6 sum_i w_i (g(r + v_i) - g(r))
 * over the nineteen velocities, periodic in x, y and z, body force (gx, gy, gz).
 *
 * Layout: f[(s * 19 + i) * S + (z * ny + y) * nx + x], S = nx ny nz, pre-collision.
 * Velocity order: 0; (+-1,0,0), (0,+-1,0), (0,0,+-1); (1,1,0), (-1,-1,0), (1,-1,0),
 * (-1,1,0), (1,0,1), (-1,0,-1), (1,0,-1), (-1,0,1), (0,1,1), (0,-1,-1), (0,1,-1),
 * (0,-1,1): velocity 2k has the opposite of velocity 2k - 1. */

static const int V3X[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
static const int V3Y[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
static const int V3Z[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
static const double W3[19] = {1.0 / 3.0,
                              1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0,
                              1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
                              1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

static int check3(const oracle_params* p)
{
    if (!p || p->ncomp < 1 || p->ncomp > OR_NMAX || p->nx < 1 || p->ny < 1 || p->nz < 1) return -1;
    if (p->walls != 0) return -1;
    if (!(p->tau > 0.5)) return -1;
    if (p->forcing_velocity != 0 && p->forcing_velocity != 1) return -1;
    if (p->force_form != 0 && p->force_form != 1) return -1;
    if (p->force_form == 1 && p->kappa != 0.0) return -1;
    return 0;
}

/* f^e_i = w_i rho^s (1 + 3 v.u + 9/2 (v.u)^2 - 3/2 u.u) (Sec. 3). */
void oracle_d3q19_equilibrium(double rho_s, double ux, double uy, double uz, double* fe)
{
    double uu = ux * ux + uy * uy + uz * uz;
    for (int i = 0; i < 19; ++i) {
        double cu = V3X[i] * ux + V3Y[i] * uy + V3Z[i] * uz;
        fe[i] = W3[i] * rho_s * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
    }
}

/* F_i = w_i (3 rho^s v.a + 9 (v.a)(v.j) - 3 a.j) (Eqs. ff1-ff3). */
void oracle_d3q19_forcing(double rho_s, double jx, double jy, double jz, double ax, double ay,
                          double az, double* F)
{
    double aj = ax * jx + ay * jy + az * jz;
    for (int i = 0; i < 19; ++i) {
        double ca = V3X[i] * ax + V3Y[i] * ay + V3Z[i] * az;
        double cj = V3X[i] * jx + V3Y[i] * jy + V3Z[i] * jz;
        F[i] = W3[i] * (3.0 * rho_s * ca + 9.0 * ca * cj - 3.0 * aj);
    }
}

static long site3(const oracle_params* p, long x, long y, long z)
{
    return (wrap(z, p->nz) * p->ny + wrap(y, p->ny)) * p->nx + wrap(x, p->nx);
}

static double lap3_at(const oracle_params* p, const double* g, int x, int y, int z)
{
    double c = g[site3(p, x, y, z)], acc = 0.0;
    for (int i = 0; i < 19; ++i) acc += W3[i] * (g[site3(p, x + V3X[i], y + V3Y[i], z + V3Z[i])] - c);
    return 6.0 * acc;
}

static void grad3_at(const oracle_params* p, const double* g, int x, int y, int z, double* gr)
{
    double a[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < 19; ++i) {
        double v = g[site3(p, x + V3X[i], y + V3Y[i], z + V3Z[i])];
        a[0] += W3[i] * V3X[i] * v;
        a[1] += W3[i] * V3Y[i] * v;
        a[2] += W3[i] * V3Z[i] * v;
    }
    for (int d = 0; d < 3; ++d) gr[d] = 3.0 * a[d];
}

typedef struct {
    long S;
    double *rs, *j[3];     /* per component: rho^s, j^s             (N*S) */
    double *rho, *u[3];    /* total density, barycentric velocity   (S)   */
    double *nu, *a[3];     /* nu^s, a^s                             (N*S) */
} work3_t;

static int work3_alloc(const oracle_params* p, work3_t* w)
{
    long S = (long)p->nx * p->ny * p->nz, N = p->ncomp;
    int ok = 1;
    w->S = S;
    w->rs = malloc(sizeof(double) * N * S);
    w->rho = malloc(sizeof(double) * S);
    w->nu = malloc(sizeof(double) * N * S);
    ok = w->rs && w->rho && w->nu;
    for (int d = 0; d < 3; ++d) {
        w->j[d] = malloc(sizeof(double) * N * S);
        w->u[d] = malloc(sizeof(double) * S);
        w->a[d] = malloc(sizeof(double) * N * S);
        ok = ok && w->j[d] && w->u[d] && w->a[d];
    }
    return ok ? 0 : -2;
}

static void work3_free(work3_t* w)
{
    free(w->rs); free(w->rho); free(w->nu);
    for (int d = 0; d < 3; ++d) { free(w->j[d]); free(w->u[d]); free(w->a[d]); }
}

/* Stages 1-3 of one D3Q19 step: moments, potentials nu^s, accelerations a^s. */
static void d3_fields(const oracle_params* p, const double* f, work3_t* w)
{
    int N = p->ncomp, nx = p->nx, ny = p->ny, nz = p->nz;
    long S = w->S;
    double th = p->theta;
    double g[3] = {p->gx, p->gy, p->gz};
#pragma omp parallel for schedule(static)
    for (long c = 0; c < S; ++c) {
        double rho = 0.0, jt[3] = {0.0, 0.0, 0.0};
        for (int s = 0; s < N; ++s) {
            double r = 0.0, j[3] = {0.0, 0.0, 0.0};
            for (int i = 0; i < 19; ++i) {
                double v = f[(long)(s * 19 + i) * S + c];
                r += v;
                j[0] += v * V3X[i];
                j[1] += v * V3Y[i];
                j[2] += v * V3Z[i];
            }
            w->rs[s * S + c] = r;
            for (int d = 0; d < 3; ++d) {
                w->j[d][s * S + c] = j[d];
                jt[d] += j[d];
            }
            rho += r;
        }
        w->rho[c] = rho;
        for (int d = 0; d < 3; ++d) w->u[d][c] = jt[d] / rho;
    }
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                long c = ((long)z * ny + y) * nx + x;
                double rho = w->rho[c];
                double phi[OR_NMAX], chiphi[OR_NMAX];
                double sum_phi_m = 0.0, quad = 0.0;
                for (int s = 0; s < N; ++s) phi[s] = w->rs[s * S + c] / rho;
                for (int s = 0; s < N; ++s) sum_phi_m += phi[s] / p->m[s];
                for (int s = 0; s < N; ++s) {
                    chiphi[s] = 0.0;
                    for (int t = 0; t < N; ++t) chiphi[s] += p->chi[s * N + t] * phi[t];
                }
                for (int s = 0; s < N; ++s) quad += 0.5 * phi[s] * chiphi[s];
                double lnrho = log(rho);
                for (int s = 0; s < N; ++s) {
                    double rs = w->rs[s * S + c];
                    double coef = th / p->m[s] - 1.0 / 3.0;
                    double logs = -(th / p->m[s]) * lnrho;
                    if (coef != 0.0) {
                        double r = rs > LOG_FLOOR * rho ? rs : LOG_FLOOR * rho;
                        logs += coef * log(r);
                    }
                    double bulk = th * (1.0 / p->m[s] - 1.0 - sum_phi_m + chiphi[s] - quad);
                    w->nu[s * S + c] = logs + bulk - p->kappa * lap3_at(p, w->rs + s * S, x, y, z);
                }
            }
    double coef = 1.0 - 1.0 / (2.0 * p->tau);
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                long c = ((long)z * ny + y) * nx + x;
                for (int s = 0; s < N; ++s) {
                    double gr[3];
                    grad3_at(p, w->nu + s * S, x, y, z, gr);
                    for (int d = 0; d < 3; ++d) w->a[d][s * S + c] = -coef * gr[d] + g[d];
                }
                if (p->force_form == 1) {   /* Gibbs-Duhem reading, as in stage_forces */
                    double A[3] = {0.0, 0.0, 0.0}, gr[3];
                    for (int s = 0; s < N; ++s)
                        for (int d = 0; d < 3; ++d)
                            A[d] += w->rs[s * S + c] * (w->a[d][s * S + c] - g[d]);
                    grad3_at(p, w->rho, x, y, z, gr);
                    for (int d = 0; d < 3; ++d) {
                        double sh = (coef * gr[d] / 3.0 - A[d]) / w->rho[c];
                        for (int s = 0; s < N; ++s) w->a[d][s * S + c] += sh;
                    }
                }
            }
}

/* f(r, 0) = f^e(rho^s(r), u(r)); u (3*S: x, y, z components) may be NULL. */
int oracle_d3q19_init(const oracle_params* p, const double* rho, const double* u, double* f)
{
    if (check3(p)) return -1;
    int N = p->ncomp;
    long S = (long)p->nx * p->ny * p->nz;
    for (int s = 0; s < N; ++s)
        for (long c = 0; c < S; ++c) {
            double fe[19];
            oracle_d3q19_equilibrium(rho[s * S + c], u ? u[c] : 0.0, u ? u[S + c] : 0.0,
                                     u ? u[2 * S + c] : 0.0, fe);
            for (int i = 0; i < 19; ++i) f[(long)(s * 19 + i) * S + c] = fe[i];
        }
    return 0;
}

/* Advance f (in place) by nsteps D3Q19 timesteps.  Returns 0, -1, -2, or 1 if a
 * non-finite value appeared. */
int oracle_d3q19_run(const oracle_params* p, double* f, long nsteps)
{
    if (check3(p)) return -1;
    int N = p->ncomp, nx = p->nx, ny = p->ny, nz = p->nz;
    work3_t w;
    if (work3_alloc(p, &w)) { work3_free(&w); return -2; }
    long S = w.S, total = 19L * N * S;
    double* gbuf = malloc(sizeof(double) * total);
    if (!gbuf) { work3_free(&w); return -2; }
    double *cur = f, *nxt = gbuf;
    double tau = p->tau;
    for (long t = 0; t < nsteps; ++t) {
        d3_fields(p, cur, &w);
#pragma omp parallel for schedule(static)
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    long c = ((long)z * ny + y) * nx + x;
                    for (int s = 0; s < N; ++s) {
                        double fe[19], F[19], j[3];
                        double rs = w.rs[s * S + c];
                        for (int d = 0; d < 3; ++d)
                            j[d] = p->forcing_velocity ? rs * w.u[d][c] : w.j[d][s * S + c];
                        oracle_d3q19_equilibrium(rs, w.u[0][c], w.u[1][c], w.u[2][c], fe);
                        oracle_d3q19_forcing(rs, j[0], j[1], j[2], w.a[0][s * S + c],
                                             w.a[1][s * S + c], w.a[2][s * S + c], F);
                        for (int i = 0; i < 19; ++i) {
                            double fi = cur[(long)(s * 19 + i) * S + c];
                            double post = fi + (fe[i] - fi) / tau + F[i];
                            nxt[(long)(s * 19 + i) * S + site3(p, x + V3X[i], y + V3Y[i], z + V3Z[i])] = post;
                        }
                    }
                }
        double* tmp = cur; cur = nxt; nxt = tmp;
    }
    if (cur != f) memcpy(f, cur, sizeof(double) * total);
    free(gbuf);
    work3_free(&w);
    for (long k = 0; k < total; ++k)
        if (!isfinite(f[k])) return 1;
    return 0;
}

/* Output fields of a D3Q19 state (any pointer may be NULL): rho (N*S); U (3*S) =
 * u + a/2 with rho a = sum_s rho^s a^s (Eq. scon); mu (N*S) = mu^s/m^s - kappa lap
 * rho^s; P (6*S) = P_xx, P_xy, P_xz, P_yy, P_yz, P_zz with P = (sum_s rho^s mu^s - psi) I
 * + kappa sum_s grad rho^s grad rho^s, psi the Eq. lgf density plus the gradient energy. */
int oracle_d3q19_moments(const oracle_params* p, const double* f, double* rho_out, double* U,
                         double* mu, double* P)
{
    if (check3(p)) return -1;
    int N = p->ncomp, nx = p->nx, ny = p->ny, nz = p->nz;
    work3_t w;
    if (work3_alloc(p, &w)) { work3_free(&w); return -2; }
    d3_fields(p, f, &w);
    long S = w.S;
    if (rho_out) memcpy(rho_out, w.rs, sizeof(double) * N * S);
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                long c = ((long)z * ny + y) * nx + x;
                if (U)
                    for (int d = 0; d < 3; ++d) {
                        double fd = 0.0;
                        for (int s = 0; s < N; ++s) fd += w.rs[s * S + c] * w.a[d][s * S + c];
                        U[d * S + c] = w.u[d][c] + 0.5 * fd / w.rho[c];
                    }
                if (mu || P) {
                    double rsl[OR_NMAX], mub[OR_NMAX], muf[OR_NMAX];
                    for (int s = 0; s < N; ++s) rsl[s] = w.rs[s * S + c];
                    oracle_mu_bulk(p, rsl, mub);
                    for (int s = 0; s < N; ++s)
                        muf[s] = mub[s] - p->kappa * lap3_at(p, w.rs + s * S, x, y, z);
                    if (mu)
                        for (int s = 0; s < N; ++s) mu[s * S + c] = muf[s];
                    if (P) {
                        double psi = oracle_psi(p, rsl), rmu = 0.0, gg = 0.0;
                        double t[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
                        for (int s = 0; s < N; ++s) {
                            double gr[3];
                            grad3_at(p, w.rs + s * S, x, y, z, gr);
                            rmu += rsl[s] * muf[s];
                            gg += 0.5 * p->kappa * (gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2]);
                            t[0] += p->kappa * gr[0] * gr[0];
                            t[1] += p->kappa * gr[0] * gr[1];
                            t[2] += p->kappa * gr[0] * gr[2];
                            t[3] += p->kappa * gr[1] * gr[1];
                            t[4] += p->kappa * gr[1] * gr[2];
                            t[5] += p->kappa * gr[2] * gr[2];
                        }
                        double iso = rmu - (psi + gg);
                        P[c] = iso + t[0];
                        P[S + c] = t[1];
                        P[2 * S + c] = t[2];
                        P[3 * S + c] = iso + t[3];
                        P[4 * S + c] = t[4];
                        P[5 * S + c] = iso + t[5];
                    }
                }
            }
    work3_free(&w);
    return 0;
}

/* Global sums of a D3Q19 state: mass^s (N), momentum (3), force sum_s rho^s a^s (3). */
int oracle_d3q19_conservation(const oracle_params* p, const double* f, double* mass,
                              double* mom, double* force_sum)
{
    if (check3(p)) return -1;
    int N = p->ncomp;
    work3_t w;
    if (work3_alloc(p, &w)) { work3_free(&w); return -2; }
    d3_fields(p, f, &w);
    long S = w.S;
    for (int s = 0; s < N; ++s) {
        double acc = 0.0;
        for (long c = 0; c < S; ++c) acc += w.rs[s * S + c];
        if (mass) mass[s] = acc;
    }
    double m3[3] = {0.0, 0.0, 0.0}, f3[3] = {0.0, 0.0, 0.0};
    for (long c = 0; c < S; ++c)
        for (int s = 0; s < N; ++s)
            for (int d = 0; d < 3; ++d) {
                m3[d] += w.j[d][s * S + c];
                f3[d] += w.rs[s * S + c] * w.a[d][s * S + c];
            }
    for (int d = 0; d < 3; ++d) {
        if (mom) mom[d] = m3[d];
        if (force_sum) force_sum[d] = f3[d];
    }
    work3_free(&w);
    return 0;
}
