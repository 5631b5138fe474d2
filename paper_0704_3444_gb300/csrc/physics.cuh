// physics.cuh -- per-site arithmetic of one timestep (Li & Wagner, arXiv:0704.3444),
// shared by the staged, fused and diagnostic kernels.
#pragma once

#include "lattice.cuh"

namespace mclb {

template <typename C>
__device__ __forceinline__ C dev_log(C x);
template <>
__device__ __forceinline__ double dev_log<double>(double x) { return log(x); }
template <>
__device__ __forceinline__ float dev_log<float>(float x) { return logf(x); }

// nu^s = mu^s/m^s - kappa lap rho^s - (1/3) ln rho^s for every component at one site
// (Eq. lgf, Eq. chemicalpotential, Eq. definef).  The Flory-Huggins potential per
// unit mass is
//   theta [ (ln phi^s + 1)/m^s - 1 - sum_t phi^t/m^t + sum_t chi^{st} phi^t
//           - 1/2 sum_{t,t'} chi^{tt'} phi^t phi^t' ],
// and its logarithms are combined with -(1/3) ln rho^s as
//   (theta/m^s - 1/3) ln rho^s - (theta/m^s) ln rho,
// the first term skipped when its coefficient is zero (theta = m^s/3) and otherwise
// evaluated at max(rho^s, 1e-12 rho).
template <typename C, int N>
__device__ __forceinline__ void site_nu(const StepParams<C>& p, const C (&r)[N],
                                        const C (&lap)[N], C (&nu)[N])
{
    C rho = C(0);
#pragma unroll
    for (int s = 0; s < N; ++s) rho += r[s];
    const C inv_rho = C(1) / rho;
    C phi[N];
#pragma unroll
    for (int s = 0; s < N; ++s) phi[s] = r[s] * inv_rho;
    C sum_phi_m = C(0);
#pragma unroll
    for (int s = 0; s < N; ++s) sum_phi_m += phi[s] * p.inv_m[s];
    C chiphi[N];
    C quad = C(0);
#pragma unroll
    for (int s = 0; s < N; ++s) {
        C acc = C(0);
#pragma unroll
        for (int t = 0; t < N; ++t) acc += p.chi[s * N + t] * phi[t];
        chiphi[s] = acc;
    }
#pragma unroll
    for (int s = 0; s < N; ++s) quad += C(0.5) * phi[s] * chiphi[s];
    const C lnrho = dev_log(rho);
#pragma unroll
    for (int s = 0; s < N; ++s) {
        C logs = -p.th_m[s] * lnrho;
        if (p.log_mask & (1u << s)) {
            const C fl = p.log_floor * rho;
            logs += p.logc[s] * dev_log(r[s] > fl ? r[s] : fl);
        }
        const C bulk = p.theta * (p.m_inv_m1[s] - sum_phi_m + chiphi[s] - quad);
        nu[s] = logs + bulk - p.kappa * lap[s];
    }
}

// Chemical potential per unit mass mu^s/m^s including the gradient term (output
// diagnostic; ln phi^s evaluated at max(phi^s, 1e-12)).
template <typename C, int N>
__device__ __forceinline__ void site_mu(const StepParams<C>& p, const C (&r)[N],
                                        const C (&lap)[N], C (&mu)[N])
{
    C rho = C(0);
#pragma unroll
    for (int s = 0; s < N; ++s) rho += r[s];
    C phi[N];
#pragma unroll
    for (int s = 0; s < N; ++s) phi[s] = r[s] / rho;
    C sum_phi_m = C(0), quad = C(0);
    C chiphi[N];
#pragma unroll
    for (int s = 0; s < N; ++s) sum_phi_m += phi[s] * p.inv_m[s];
#pragma unroll
    for (int s = 0; s < N; ++s) {
        C acc = C(0);
#pragma unroll
        for (int t = 0; t < N; ++t) acc += p.chi[s * N + t] * phi[t];
        chiphi[s] = acc;
    }
#pragma unroll
    for (int s = 0; s < N; ++s) quad += C(0.5) * phi[s] * chiphi[s];
#pragma unroll
    for (int s = 0; s < N; ++s) {
        const C ph = phi[s] > p.log_floor ? phi[s] : p.log_floor;
        mu[s] = p.theta * ((dev_log(ph) + C(1)) * p.inv_m[s] - C(1) - sum_phi_m + chiphi[s] - quad)
                - p.kappa * lap[s];
    }
}

// Flory-Huggins free energy density of Eq. lgf (n^s = rho^s/m^s), with the
// phi ln phi term taken as 0 at phi = 0.
template <typename C, int N>
__device__ __forceinline__ C site_psi(const StepParams<C>& p, const C (&r)[N])
{
    C rho = C(0);
#pragma unroll
    for (int s = 0; s < N; ++s) rho += r[s];
    C psi = C(0);
#pragma unroll
    for (int s = 0; s < N; ++s) {
        const C n = r[s] * p.inv_m[s];
        C phi = r[s] / rho;
        C ph = phi > p.log_floor ? phi : p.log_floor;
        psi += -p.theta * n * p.m[s];
        psi += n * p.theta * dev_log(ph);
        C acc = C(0);
#pragma unroll
        for (int t = 0; t < N; ++t) acc += p.chi[s * N + t] * (r[t] / rho);
        psi += C(0.5) * p.theta * p.m[s] * n * acc;
    }
    return psi;
}

// The nine products v_i . (x, y) of one vector, formed without multiplying by 0 or
// +-1 (i is a compile-time constant once the direction loops are unrolled).
template <typename C>
struct VDots {
    C x, y, sp, sm;  // x, y, x + y, x - y
    __device__ __forceinline__ VDots(C x_, C y_) : x(x_), y(y_), sp(x_ + y_), sm(x_ - y_) {}
    __device__ __forceinline__ C operator()(int i) const
    {
        switch (i) {
            case 1: return x;
            case 2: return y;
            case 3: return -x;
            case 4: return -y;
            case 5: return sp;
            case 6: return -sm;
            case 7: return -sp;
            case 8: return sm;
            default: return C(0);
        }
    }
};

// Velocity-dependent part of the equilibrium, shared by every component:
// e_i = w_i (3 v_i.u + 9/2 (v_i.u)^2 - 3/2 u.u), so that f^{s,e}_i = rho^s (w_i + e_i)
// (Sec. 3 equilibrium moments, all components built on the barycentric u).  The constant
// w_i is added by collide() through its forcing bracket, so that 1 - 3/2 u.u is never
// rounded: in FP32 that rounding has a sign set by u and changed the component masses
// systematically (by up to 3e-8 of the density per step).
template <typename C>
__device__ __forceinline__ void eq_weights(C ux, C uy, C (&e)[Q])
{
    const C base = C(-1.5) * (ux * ux + uy * uy);
    const VDots<C> du(ux, uy);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if (i == 0) {
            e[0] = wq<C>(0) * base;
        } else {
            const C cu = du(i);
            e[i] = wq<C>(i) * fma(cu, fma(C(4.5), cu, C(3)), base);
        }
    }
}

// Gibbs-Duhem reading of the sum of the component forces (kappa = 0): every a^s gets
// the same shift (A_c - A) / rho, with A = sum_s rho^s (a^s - g) the sum of the Eq. definef
// forces and A_c = (1 - 1/(2 tau)) (1/3) grad rho their continuum total for the
// Flory-Huggins free energy (Gibbs-Duhem with the pressure sum rho mu - psi = 0); the
// differences between the components' accelerations are kept.
template <typename C, int N>
__device__ __forceinline__ void gibbs_duhem_shift(const StepParams<C>& p, const C (&r)[N], C rho,
                                                  C grx, C gry, C (&ax)[N], C (&ay)[N])
{
    C Ax = C(0), Ay = C(0);
#pragma unroll
    for (int s = 0; s < N; ++s) {
        Ax += r[s] * (ax[s] - p.gx);
        Ay += r[s] * (ay[s] - p.gy);
    }
    const C k = p.fcoef * C(1.0 / 3.0), inv = C(1) / rho;
    const C dx = (k * grx - Ax) * inv;
    const C dy = (k * gry - Ay) * inv;
#pragma unroll
    for (int s = 0; s < N; ++s) {
        ax[s] += dx;
        ay[s] += dy;
    }
}

// Momentum of the forcing's second moment (Eq. ff3): j^s = rho^s u^s as printed, or
// rho^s u with the barycentric u when the barycentric reading is selected.
template <typename C>
__device__ __forceinline__ void forcing_momentum(const StepParams<C>& p, C r, C jx, C jy, C ux,
                                                 C uy, C& fx, C& fy)
{
    fx = p.bary ? r * ux : jx;
    fy = p.bary ? r * uy : jy;
}

// Post-collision populations of one component (Eq. ssLB):
//   f* = f + (f^e - f)/tau + F,  f^e_i = rho^s (w_i + e_i),
//   F_i = w_i [3 rho^s (v_i.a) + 9 (v_i.a)(v_i.j) - 3 a.j]   (Eqs. ff1-ff3, j from
//   forcing_momentum),
// evaluated as f (1 - 1/tau) + (rho^s/tau) e_i + w_i [(v_i.a)(9 v_i.j + 3 rho^s) - 3 a.j
// + rho^s/tau].  With a nonzero `shift` M it returns f*_i - w_i M instead (the deviations
// the 16-bit formats store), the subtraction folded into the same bracket.
template <typename C>
__device__ __forceinline__ void collide(const StepParams<C>& p, const C (&f)[Q], const C (&e)[Q],
                                        C r, C jx, C jy, C ax, C ay, C (&out)[Q], C shift = C(0))
{
    const VDots<C> da(ax, ay), dj(jx, jy);
    const C r3 = C(3) * r;
    const C omr = p.omega * r;
    const C m3aj = fma(C(-3), ax * jx + ay * jy, omr - shift);
    const C keep = C(1) - p.omega;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const C F = (i == 0) ? wq<C>(0) * m3aj
                             : wq<C>(i) * fma(da(i), fma(C(9), dj(i), r3), m3aj);
        out[i] = fma(keep, f[i], fma(omr, e[i], F));
    }
}

// ---------------------------------------------------------------- component pairs
//
// In FP32 two components of a site are collided together with the packed pair
// instructions of sm_100 and later (fma/add/mul .f32x2: one instruction for both), which
// halves the issue slots of the collision.  The pair layout is (component c, c + 1).

__device__ __forceinline__ float2 pdup(float x) { return make_float2(x, x); }
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }

// eq_weights for a pair of components: the same per-site values in both halves.
__device__ __forceinline__ void eq_weights2(float ux, float uy, float2 (&e)[Q])
{
    const float2 u = pdup(ux), v = pdup(uy);
    const float2 base = pmul(pdup(-1.5f), pfma(u, u, pmul(v, v)));
    const float2 sp = padd(u, v), sm = pfma(v, pdup(-1.0f), u);
    const float2 k45 = pdup(4.5f), k3 = pdup(3.0f), km3 = pdup(-3.0f);
    e[0] = pmul(pdup(wq<float>(0)), base);
    // v_i . u and its opposite -v_i . u share (v_i.u)^2: 4.5 x^2 + 3 x and 4.5 x^2 - 3 x
    auto two = [&](int i, int j, float2 x) {
        const float2 q = pfma(pmul(k45, x), x, base);
        e[i] = pmul(pdup(wq<float>(i)), pfma(k3, x, q));
        e[j] = pmul(pdup(wq<float>(j)), pfma(km3, x, q));
    };
    two(1, 3, u);
    two(2, 4, v);
    two(5, 7, sp);
    two(8, 6, sm);
}

// collide() for the pair of components (c, c + 1): every argument but e holds the two
// components' values.  The opposite velocity of i gets the same bracket with the sign of
// the 3 rho^s term flipped, (-v.a)(9 (-v.j) + 3 rho) = (v.a)(9 v.j - 3 rho), so no operand
// needs negating.
__device__ __forceinline__ void collide2(const StepParams<float>& p, const float2 (&f)[Q],
                                         const float2 (&e)[Q], float2 r, float2 jx, float2 jy,
                                         float2 ax, float2 ay, float2 (&out)[Q], float2 shift)
{
    const float2 mone = pdup(-1.0f);
    const float2 sa = padd(ax, ay), da = pfma(ay, mone, ax);
    const float2 sj = padd(jx, jy), dj = pfma(jy, mone, jx);
    const float2 omr = pmul(pdup(p.omega), r);
    const float2 r3 = pmul(pdup(3.0f), r), r3n = pmul(pdup(-3.0f), r);
    const float2 aj = pfma(ay, jy, pmul(ax, jx));
    const float2 m3aj = pfma(pdup(-3.0f), aj, pfma(shift, mone, omr));
    const float2 keep = pdup(1.0f - p.omega), nine = pdup(9.0f);
    out[0] = pfma(keep, f[0], pfma(omr, e[0], pmul(pdup(wq<float>(0)), m3aj)));
    auto term = [&](int i, float2 a, float2 j, float2 r3s) {
        const float2 F = pmul(pdup(wq<float>(i)), pfma(a, pfma(nine, j, r3s), m3aj));
        out[i] = pfma(keep, f[i], pfma(omr, e[i], F));
    };
    term(1, ax, jx, r3);
    term(3, ax, jx, r3n);
    term(2, ay, jy, r3);
    term(4, ay, jy, r3n);
    term(5, sa, sj, r3);
    term(7, sa, sj, r3n);
    term(8, da, dj, r3);
    term(6, da, dj, r3n);
}

}  // namespace mclb
