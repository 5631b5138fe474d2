"""Independent numpy transcriptions of the paper's update, used only to pin the oracle.

These are written differently from the C oracle on purpose, so that a
mistake in one (a dropped term, a wrong sign, a swapped index) shows up as
a disagreement:

* chemical potentials come from a complex-step derivative of the free
  energy density psi of Eq. lgf (mu^s/m^s = d psi / d rho^s), not from a
  hand-derived formula;
* D2Q9 equilibria and forcing terms come from the generic second-order
  Hermite expansion built with explicit tensors and the moments listed in
  Sec. 3 (equilibrium: rho^s, rho^s u, rho^s/3 I + rho^s u u; forcing: 0,
  rho^s a^s, rho^s (a^s u^s + u^s a^s));
* the D1Q3 update (the paper's own lattice, Sec. 4) solves the three moment
  conditions for the three populations directly;
* ``bary=True`` puts the barycentric u in place of the component velocity in the
  forcing's second moment (rho^s (a^s u + u a^s) instead of Eq. ff3's
  rho^s (a^s u^s + u^s a^s));
* ``gd=True`` (kappa = 0) keeps the differences of the component accelerations and
  makes their density-weighted sum the Gibbs-Duhem total (1 - 1/(2 tau)) (1/3) grad rho
  (plus rho g), by adding the same vector to every a^s;
* streaming uses numpy.roll, the stencils are the explicit 9-point forms.
"""
from __future__ import annotations

import numpy as np

CS2 = 1.0 / 3.0
C9 = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1], [1, 1], [-1, 1], [-1, -1], [1, -1]])
W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def psi_fh(rho_s, chi, m, theta):
    """Eq. lgf density with n = rho/m, phi = rho^s/rho.  rho_s: (N, ...), may be complex."""
    rho = rho_s.sum(0)
    N = rho_s.shape[0]
    out = 0.0
    for s in range(N):
        n = rho_s[s] / m[s]
        phi = rho_s[s] / rho
        out = out - theta * n * m[s] + n * theta * np.log(phi)
        for t in range(N):
            out = out + 0.5 * chi[s, t] * theta * m[s] * n * (rho_s[t] / rho)
    return out


def mu_complex_step(rho_s, chi, m, theta, h=1e-30):
    """d psi / d rho^s by the complex-step derivative (exact to rounding)."""
    N = rho_s.shape[0]
    mu = np.empty_like(rho_s, dtype=np.float64)
    for s in range(N):
        z = rho_s.astype(np.complex128)
        z[s] = z[s] + 1j * h
        mu[s] = np.imag(psi_fh(z, chi, m, theta)) / h
    return mu


# ------------------------------------------------------------ 2D stencils

def sh(g, dx, dy):
    """g(x + dx, y + dy) on a periodic (..., ny, nx) array."""
    return np.roll(np.roll(g, -dx, axis=-1), -dy, axis=-2)


def grad9(g):
    """Isotropic 9-point gradient: [4 (E - W) + (NE + SE - NW - SW)] / 12 and likewise in y."""
    gx = (4 * (sh(g, 1, 0) - sh(g, -1, 0)) + sh(g, 1, 1) + sh(g, 1, -1) - sh(g, -1, 1)
          - sh(g, -1, -1)) / 12.0
    gy = (4 * (sh(g, 0, 1) - sh(g, 0, -1)) + sh(g, 1, 1) + sh(g, -1, 1) - sh(g, 1, -1)
          - sh(g, -1, -1)) / 12.0
    return gx, gy


def lap9(g):
    """Isotropic 9-point Laplacian: [4 (E + W + N + S) + (NE + NW + SE + SW) - 20 g] / 6."""
    s4 = sh(g, 1, 0) + sh(g, -1, 0) + sh(g, 0, 1) + sh(g, 0, -1)
    d4 = sh(g, 1, 1) + sh(g, -1, 1) + sh(g, 1, -1) + sh(g, -1, -1)
    return (4 * s4 + d4 - 20 * g) / 6.0


def hermite2(zeroth, first, second):
    """Populations w_i [A + c.B/cs2 + (M - cs2 A I):(c c - cs2 I)/(2 cs2^2)] with the
    given zeroth (A), first (B_a) and full second (M_ab) moments; site arrays broadcast."""
    out = []
    I = np.eye(2)
    for i in range(9):
        c = C9[i].astype(np.float64)
        H2 = np.outer(c, c) - CS2 * I
        v = zeroth + (c[0] * first[0] + c[1] * first[1]) / CS2
        acc = 0.0
        for a in range(2):
            for b in range(2):
                acc = acc + (second[a][b] - CS2 * zeroth * I[a, b]) * H2[a, b]
        out.append(W9[i] * (v + acc / (2 * CS2 * CS2)))
    return np.stack(out)


def step_d2q9(f, chi, m, theta, kappa, tau, g=(0.0, 0.0), bary=False, gd=False):
    """One update of f (N, 9, ny, nx) by the alternative formulation above."""
    N = f.shape[0]
    rs = f.sum(1)
    jx = np.einsum("sixy,i->sxy", f, C9[:, 0].astype(float))
    jy = np.einsum("sixy,i->sxy", f, C9[:, 1].astype(float))
    rho = rs.sum(0)
    ux, uy = jx.sum(0) / rho, jy.sum(0) / rho
    mu = mu_complex_step(rs, chi, m, theta)
    fnew = np.empty_like(f)
    c = 1.0 - 1.0 / (2.0 * tau)
    acc = []
    for s in range(N):
        nu = mu[s] - kappa * lap9(rs[s]) - np.log(rs[s]) / 3.0
        gx, gy = grad9(nu)
        acc.append([-c * gx, -c * gy])
    if gd:
        Ax = sum(rs[s] * acc[s][0] for s in range(N))
        Ay = sum(rs[s] * acc[s][1] for s in range(N))
        rgx, rgy = grad9(rho)
        for s in range(N):
            acc[s][0] = acc[s][0] + (c * rgx / 3.0 - Ax) / rho
            acc[s][1] = acc[s][1] + (c * rgy / 3.0 - Ay) / rho
    for s in range(N):
        ax, ay = acc[s][0] + g[0], acc[s][1] + g[1]
        feq = hermite2(rs[s], (rs[s] * ux, rs[s] * uy),
                       [[rs[s] / 3 + rs[s] * ux * ux, rs[s] * ux * uy],
                        [rs[s] * uy * ux, rs[s] / 3 + rs[s] * uy * uy]])
        zero = np.zeros_like(rs[s])
        # second moment rho^s (a v + v a) with v = u^s (jx/rho^s) or the barycentric u
        vx_, vy_ = (ux, uy) if bary else (jx[s] / rs[s], jy[s] / rs[s])
        F = hermite2(zero, (rs[s] * ax, rs[s] * ay),
                     [[rs[s] * 2 * ax * vx_, rs[s] * (ax * vy_ + ay * vx_)],
                      [rs[s] * (ay * vx_ + ax * vy_), rs[s] * 2 * ay * vy_]])
        post = f[s] + (feq - f[s]) / tau + F
        for i in range(9):
            fnew[s, i] = sh(post[i], -C9[i, 0], -C9[i, 1])
    return fnew


# ------------------------------------------------------------------ D1Q3

def d1q3_equilibrium(rs, u):
    """Populations (v = -1, 0, +1) with moments rho, rho u, rho/3 + rho u^2."""
    p2 = rs / 3.0 + rs * u * u
    return np.stack([(p2 - rs * u) / 2.0, rs - p2, (p2 + rs * u) / 2.0])


def d1q3_forcing(rs, j, a):
    """Populations with moments 0, rho a, 2 a j (Eqs. ff1-ff3 in one dimension; j is
    rho^s times the velocity of the second moment)."""
    p2 = 2.0 * a * j
    return np.stack([(p2 - rs * a) / 2.0, -p2, (p2 + rs * a) / 2.0])


def d1q3_init(rho_s, u):
    return np.stack([d1q3_equilibrium(rho_s[s], u) for s in range(rho_s.shape[0])])


def d1q3_step(f, chi, m, theta, kappa, tau, g=0.0, bary=False, gd=False):
    """One update of f (N, 3, nx) on the D1Q3 lattice of Sec. 4 (velocities -1, 0, +1)."""
    N = f.shape[0]
    v = np.array([-1.0, 0.0, 1.0])
    rs = f.sum(1)
    j = np.einsum("sqx,q->sx", f, v)
    rho = rs.sum(0)
    u = j.sum(0) / rho
    mu = mu_complex_step(rs, chi, m, theta)
    out = np.empty_like(f)
    c = 1.0 - 1.0 / (2.0 * tau)
    d1 = lambda q: (np.roll(q, -1) - np.roll(q, 1)) / 2.0
    acc = []
    for s in range(N):
        lap = np.roll(rs[s], -1) + np.roll(rs[s], 1) - 2 * rs[s]
        nu = mu[s] - kappa * lap - np.log(rs[s]) / 3.0
        acc.append(-c * d1(nu))
    if gd:
        A = sum(rs[s] * acc[s] for s in range(N))
        acc = [a + (c * d1(rho) / 3.0 - A) / rho for a in acc]
    for s in range(N):
        a = acc[s] + g
        js = rs[s] * u if bary else j[s]
        post = f[s] + (d1q3_equilibrium(rs[s], u) - f[s]) / tau + d1q3_forcing(rs[s], js, a)
        out[s, 0] = np.roll(post[0], -1)
        out[s, 1] = post[1]
        out[s, 2] = np.roll(post[2], 1)
    return out
