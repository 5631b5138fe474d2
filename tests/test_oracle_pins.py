"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: each test checks it against a
moment condition stated in Sec. 3, a conservation law or balance that follows
from them, an independent transcription (complex-step chemical potentials,
generic Hermite populations, the paper's D1Q3 lattice), a closed-form rate
from Eq. woche, or a symmetry of the method.
"""

import numpy as np
import pytest

import oracle
from oracle import Oracle
from paper_0704_3444_gb300 import inputs
from tests import transcriptions as tr

C9 = tr.C9


def _chi(n, seed):
    r = inputs.uniform(seed, n * n, 3).reshape(n, n)
    c = 2.0 + (r + r.T)
    np.fill_diagonal(c, 0.0)
    return c


# ------------------------------------------------------------ moment conditions

@pytest.mark.parametrize("k", range(5))
def test_equilibrium_moments(k):
    """Sec. 3: sum f^e = rho^s, sum f^e v = rho^s u, sum f^e v v = rho^s/3 I + rho^s u u,
    third moment rho^s/3 (u_a d_bc + u_b d_ac + u_c d_ab)."""
    r = inputs.uniform(100 + k, 3)
    rs, ux, uy = 0.2 + r[0], 0.2 * (r[1] - 0.5), 0.2 * (r[2] - 0.5)
    fe = oracle.equilibrium(rs, ux, uy)
    u = np.array([ux, uy])
    c = C9.astype(float)
    assert abs(fe.sum() - rs) < 1e-15
    np.testing.assert_allclose(c.T @ fe, rs * u, atol=1e-15)
    M2 = np.einsum("i,ia,ib->ab", fe, c, c)
    np.testing.assert_allclose(M2, rs / 3 * np.eye(2) + rs * np.outer(u, u), atol=1e-15)
    M3 = np.einsum("i,ia,ib,ic->abc", fe, c, c, c)
    I = np.eye(2)
    want = rs / 3 * (np.einsum("a,bc->abc", u, I) + np.einsum("b,ac->abc", u, I)
                     + np.einsum("c,ab->abc", u, I))
    np.testing.assert_allclose(M3, want, atol=1e-15)


@pytest.mark.parametrize("k", range(5))
def test_forcing_moments(k):
    """Eqs. ff1-ff3: sum F = 0, sum F v = rho^s a^s, sum F v v = rho^s (a u^s + u^s a),
    and the third moment rho^s/3 (a_a d_bc + a_b d_ac + a_c d_ab)."""
    r = inputs.uniform(200 + k, 5)
    rs = 0.2 + r[0]
    j = 0.1 * (r[1:3] - 0.5)
    a = 0.01 * (r[3:5] - 0.5)
    F = oracle.forcing(rs, j[0], j[1], a[0], a[1])
    c = C9.astype(float)
    assert abs(F.sum()) < 1e-17
    np.testing.assert_allclose(c.T @ F, rs * a, atol=1e-17)
    us = j / rs
    M2 = np.einsum("i,ia,ib->ab", F, c, c)
    np.testing.assert_allclose(M2, rs * (np.outer(a, us) + np.outer(us, a)), atol=1e-17)
    M3 = np.einsum("i,ia,ib,ic->abc", F, c, c, c)
    I = np.eye(2)
    want = rs / 3 * (np.einsum("a,bc->abc", a, I) + np.einsum("b,ac->abc", a, I)
                     + np.einsum("c,ab->abc", a, I))
    np.testing.assert_allclose(M3, want, atol=1e-17)


@pytest.mark.parametrize("n", [2, 3, 5])
def test_mu_bulk_is_derivative_of_psi(n):
    """Eq. chemicalpotential with Eq. lgf: mu^s/m^s = d psi / d rho^s (complex step)."""
    chi = _chi(n, 7 + n)
    m = 1.0 + 9.0 * inputs.uniform(11 + n, n)
    o = Oracle(n, 1, 1, 1.0, chi, m, theta=0.45)
    for k in range(4):
        rs = 0.05 + inputs.uniform(300 + 10 * n + k, n)
        mu = o.mu_bulk(rs)
        want = tr.mu_complex_step(rs.reshape(n, 1), chi, m, 0.45)[:, 0]
        np.testing.assert_allclose(mu, want, rtol=1e-12, atol=1e-13)
        # psi itself against the independent numpy transcription of Eq. lgf
        assert abs(o.psi(rs) - tr.psi_fh(rs.reshape(n, 1), chi, m, 0.45)[0]) < 1e-13


@pytest.mark.parametrize("n", [2, 3, 4])
def test_flory_huggins_pressure_vanishes(n):
    """Eq. ppp: p = sum n mu - psi; the Flory-Huggins psi is homogeneous of degree one in
    the densities, so p = 0 (Euler) -- a check on every term of mu at once."""
    chi = _chi(n, 20 + n)
    m = 1.0 + 4.0 * inputs.uniform(21 + n, n)
    o = Oracle(n, 1, 1, 1.0, chi, m, theta=0.7)
    rs = 0.1 + inputs.uniform(22 + n, n)
    assert abs(np.dot(rs, o.mu_bulk(rs)) - o.psi(rs)) < 1e-13


# ------------------------------------------------------------------ invariants

def test_uniform_state_is_fixed_point():
    """Uniform fields: every gradient vanishes, F = 0, f = f^e, streaming moves equal values."""
    n, nx, ny = 3, 4, 4
    rho = np.stack([np.full((ny, nx), v) for v in (0.2, 0.5, 0.3)])
    u = np.stack([np.full((ny, nx), 0.03), np.full((ny, nx), -0.02)])
    o = Oracle(n, nx, ny, 0.8, _chi(3, 1), theta=0.4, kappa=0.02)
    o.init(rho, u)
    f0 = o.f.copy()
    o.run(25)
    np.testing.assert_allclose(o.f, f0, rtol=0, atol=1e-15)


def test_mass_conservation_binary_64():
    """sum_i F_i = 0 (Eq. ff1) and sum f^e = rho^s: per-component mass is kept to rounding."""
    p = inputs.binary_noise(steps=1000)
    o = Oracle.from_problem(p)
    m0 = o.conservation()["mass"]
    o.run(1000)
    m1 = o.conservation()["mass"]
    assert np.max(np.abs(m1 / m0 - 1.0)) < 1e-13


def test_momentum_balance():
    """Sum over sites and components of Eq. ssLB's first moment: the total momentum
    changes by exactly sum_r sum_s rho^s a^s per step (Eq. ff2 with sum f^e v = rho^s u)."""
    rho, u = inputs.random_state(3, 12, 9, seed=5, amp=0.3, umax=0.05)
    o = Oracle(3, 12, 9, 0.7, _chi(3, 2), m=[1.0, 2.0, 5.0], theta=0.4, kappa=0.03,
               force=(1e-4, -2e-4))
    o.init(rho, u)
    for _ in range(5):
        c0 = o.conservation()
        o.run(1)
        c1 = o.conservation()
        np.testing.assert_allclose(c1["mom"] - c0["mom"], c0["force"], rtol=1e-10, atol=1e-15)
        assert np.max(np.abs(c0["force"])) > 1e-6


# ------------------------------------------------ independent transcriptions

@pytest.mark.parametrize("fv", [0, 1], ids=["component_u", "barycentric_u"])
@pytest.mark.parametrize("shape", [(4, 4), (5, 3), (7, 6)])
def test_step_matches_hermite_transcription(shape, fv):
    """One to three steps on tiny grids against the generic-Hermite numpy transcription
    (every site, every population), with every term switched on, for both readings of
    the velocity in the forcing's second moment (Eq. ff3 as printed, and barycentric)."""
    nx, ny = shape
    n = 3
    chi = _chi(n, 40)
    m = np.array([1.0, 3.0, 10.0])
    rho, u = inputs.random_state(n, nx, ny, seed=41, amp=0.4, umax=0.05)
    o = Oracle(n, nx, ny, 0.9, chi, m, theta=0.42, kappa=0.05, force=(3e-4, -1e-4),
               forcing_velocity=fv)
    o.init(rho, u)
    f = o.f.copy()
    for _ in range(3):
        o.run(1)
        f = tr.step_d2q9(f, chi, m, 0.42, 0.05, 0.9, g=(3e-4, -1e-4), bary=bool(fv))
        np.testing.assert_allclose(o.f, f, rtol=1e-12, atol=1e-14)


def _one_fluid_forcing(A, rho, u):
    """D2Q9 populations with moments 0, A, A u + u A (the overall fluid's forcing with
    rho a = A, Eq. olso), written out per velocity for 2-vectors A, u."""
    c = C9.astype(float)
    out = []
    for i in range(9):
        cA = c[i, 0] * A[0] + c[i, 1] * A[1]
        cu = c[i, 0] * u[0] + c[i, 1] * u[1]
        Au = A[0] * u[0] + A[1] * u[1]
        out.append(tr.W9[i] * (3 * cA + 9 * cA * cu - 3 * Au))
    return np.stack(out)


def test_barycentric_forcing_sums_to_one_fluid():
    """With the barycentric u in the forcing's second moment, summing Eq. ssLB over the
    components gives exactly the one-fluid update with the overall forcing of Eq. olso
    (moments 0, rho a, rho (a u + u a), rho a = sum_s rho^s a^s).  The total force comes
    from the oracle's own output velocity U = u + a/2 (Eq. scon), the rest from the
    populations, so this pins the option at the level of the whole step.  With Eq. ff3 as
    printed (component velocities) the same sum differs by sum_s rho^s a^s (u^s - u)
    terms, which the test also checks is not zero."""
    n, nx, ny = 3, 9, 7
    chi = _chi(n, 43)
    rho, u = inputs.random_state(n, nx, ny, seed=44, amp=0.4, umax=0.05)
    diffs = []
    for fv in (1, 0):
        o = Oracle(n, nx, ny, 0.85, chi, [1.0, 2.0, 1.0], theta=0.4, kappa=0.03,
                   force=(2e-4, 1e-4), forcing_velocity=fv)
        o.init(rho, u)
        o.run(2)  # component velocities differ from u after the first steps
        f0 = o.f.copy()
        tot = f0.sum(0)
        r = tot.sum(0)
        c = C9.astype(float)
        uu = np.stack([np.einsum("ixy,i->xy", tot, c[:, 0]), np.einsum("ixy,i->xy", tot, c[:, 1])]) / r
        A = 2.0 * r * (o.moments()["U"] - uu)
        feq = np.stack([tr.W9[i] * r * (1 + 3 * (c[i, 0] * uu[0] + c[i, 1] * uu[1])
                                        + 4.5 * (c[i, 0] * uu[0] + c[i, 1] * uu[1]) ** 2
                                        - 1.5 * (uu[0] ** 2 + uu[1] ** 2)) for i in range(9)])
        post = tot + (feq - tot) / 0.85 + _one_fluid_forcing(A, r, uu)
        want = np.stack([tr.sh(post[i], -C9[i, 0], -C9[i, 1]) for i in range(9)])
        o.run(1)
        diffs.append(np.max(np.abs(o.f.sum(0) - want)))
    assert diffs[0] < 1e-15, diffs
    assert diffs[1] > 1e-9, diffs


def test_single_perturbed_site():
    """A 4x4 grid at rest with one perturbed site: after one step only the 5x5
    neighbourhood feels the force, and everything agrees with the transcription."""
    n, nx, ny = 2, 4, 4
    rho = np.stack([np.full((ny, nx), 0.5), np.full((ny, nx), 0.5)])
    rho[0, 1, 2] += 0.05
    rho[1, 1, 2] -= 0.05
    chi = np.array([[0.0, 2.5], [2.5, 0.0]])
    o = Oracle(n, nx, ny, 1.0, chi, kappa=0.0)
    o.init(rho, np.zeros((2, ny, nx)))
    f = o.f.copy()
    o.run(1)
    np.testing.assert_allclose(o.f, tr.step_d2q9(f, chi, np.ones(2), 1 / 3, 0.0, 1.0),
                               rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("axis", ["x", "y"])
def test_d1q3_reduction(axis):
    """Sec. 4 uses D1Q3, a projection of D2Q9: a y-invariant (or x-invariant) D2Q9 run
    equals an independent D1Q3 update that solves the moment conditions directly."""
    n, L = 3, 48
    chi = np.array([[0.0, 3.0, 0.5], [3.0, 0.0, 0.2], [0.5, 0.2, 0.0]])
    m = np.array([2.0, 1.0, 1.0])
    x = np.arange(L)
    phi0 = np.array([0.4, 0.35, 0.25])
    line = np.stack([phi0[0] + 0.05 * np.sin(2 * np.pi * x / L),
                     phi0[1] - 0.05 * np.sin(2 * np.pi * x / L), np.full(L, phi0[2])])
    theta, kappa, tau = 0.4, 0.02, 1 / 0.9
    if axis == "x":
        nx, ny = L, 2
        rho = np.repeat(line[:, None, :], ny, axis=1)
        g2 = (2e-5, 0.0)
    else:
        nx, ny = 3, L
        rho = np.repeat(line[:, :, None], nx, axis=2)
        g2 = (0.0, 2e-5)
    o = Oracle(n, nx, ny, tau, chi, m, theta=theta, kappa=kappa, force=g2)
    o.init(rho, np.zeros((2, ny, nx)))
    f1 = tr.d1q3_init(line, np.zeros(L))
    for _ in range(60):
        f1 = tr.d1q3_step(f1, chi, m, theta, kappa, tau, g=2e-5)
    o.run(60)
    mom = o.moments()
    r1 = f1.sum(1)
    U1 = (np.einsum("sqx,q->x", f1, np.array([-1.0, 0.0, 1.0])) / r1.sum(0))
    if axis == "x":
        np.testing.assert_allclose(mom["rho"][:, 0, :], r1, rtol=1e-12, atol=1e-14)
        assert np.max(np.abs(mom["U"][1])) < 1e-15
    else:
        np.testing.assert_allclose(mom["rho"][:, :, 0], r1, rtol=1e-12, atol=1e-14)
        assert np.max(np.abs(mom["U"][0])) < 1e-15
    assert np.max(np.abs(r1 - line)) > 1e-4  # the run did evolve


# ------------------------------------------------------------------ symmetries

def test_component_permutation():
    """The method is symmetric in the components: relabelling them (with chi, m)
    relabels the result."""
    n, nx, ny = 4, 16, 12
    chi = _chi(n, 50)
    m = np.array([1.0, 2.0, 1.0, 4.0])
    rho, u = inputs.random_state(n, nx, ny, seed=51, amp=0.3, umax=0.02)
    perm = np.array([2, 0, 3, 1])
    a = Oracle(n, nx, ny, 0.8, chi, m, theta=0.4, kappa=0.02)
    a.init(rho, u)
    b = Oracle(n, nx, ny, 0.8, chi[np.ix_(perm, perm)], m[perm], theta=0.4, kappa=0.02)
    b.init(rho[perm], u)
    a.run(40)
    b.run(40)
    np.testing.assert_allclose(b.f, a.f[perm], rtol=1e-12, atol=1e-15)


def test_identical_components_stay_identical():
    """Two components with the same chi row, m and field remain bitwise equal."""
    chi = np.array([[0.0, 3.0, 3.0], [3.0, 0.0, 1.0], [3.0, 1.0, 0.0]])
    rho, u = inputs.random_state(3, 16, 16, seed=52, amp=0.3)
    rho[2] = rho[1]
    o = Oracle(3, 16, 16, 0.8, chi, theta=1 / 3, kappa=0.01)
    o.init(rho, u)
    o.run(100)
    assert np.array_equal(o.f[1], o.f[2])


def test_component_splitting():
    """Splitting B into B1 + B2 (chi rows copied, chi_{B1 B2} = 0, halves of the field)
    reproduces the binary run: nu^{B1} - nu^B is constant, so the forces agree (kappa = 0)."""
    nx, ny = 20, 14
    rho2, u = inputs.random_state(2, nx, ny, seed=53, amp=0.4, umax=0.02)
    chi2 = np.array([[0.0, 2.4], [2.4, 0.0]])
    rho3 = np.stack([rho2[0], rho2[1] / 2, rho2[1] / 2])
    chi3 = np.array([[0.0, 2.4, 2.4], [2.4, 0.0, 0.0], [2.4, 0.0, 0.0]])
    a = Oracle(2, nx, ny, 0.9, chi2, theta=0.45)
    a.init(rho2, u)
    b = Oracle(3, nx, ny, 0.9, chi3, theta=0.45)
    b.init(rho3, u)
    a.run(60)
    b.run(60)
    np.testing.assert_allclose(b.f[0], a.f[0], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(b.f[1] + b.f[2], a.f[1], rtol=1e-12, atol=1e-15)


def test_scale_invariance_kappa0():
    """kappa = 0: rho -> lambda rho changes every potential by a constant (logs only),
    so f -> lambda f exactly (Sec. 4 uses rho = 100)."""
    rho, u = inputs.random_state(3, 12, 10, seed=54, amp=0.3, umax=0.02)
    chi = _chi(3, 55)
    a = Oracle(3, 12, 10, 0.8, chi, m=[1.0, 2.0, 1.0], theta=0.4)
    a.init(rho, u)
    b = Oracle(3, 12, 10, 0.8, chi, m=[1.0, 2.0, 1.0], theta=0.4)
    b.init(100.0 * rho, u)
    a.run(50)
    b.run(50)
    np.testing.assert_allclose(b.f, 100.0 * a.f, rtol=1e-11, atol=1e-13)


def test_rotation_symmetry():
    """A quarter turn of the lattice maps D2Q9 onto itself: rotating the initial fields
    (and the velocity) rotates the result."""
    n, L = 2, 10
    rho, u = inputs.random_state(n, L, L, seed=56, amp=0.3, umax=0.03)
    chi = np.array([[0.0, 2.6], [2.6, 0.0]])
    # np.rot90 over (y, x) sends the site (x, y) to (y, L-1-x): a quarter turn that maps
    # a vector (vx, vy) to (vy, -vx)
    rot = lambda a: np.rot90(a, k=1, axes=(-2, -1))
    rho_r = rot(rho)
    ux, uy = u
    u_r = np.stack([rot(uy), -rot(ux)])
    a = Oracle(n, L, L, 0.85, chi, theta=0.4, kappa=0.02)
    a.init(rho, u)
    b = Oracle(n, L, L, 0.85, chi, theta=0.4, kappa=0.02)
    b.init(rho_r, u_r)
    a.run(30)
    b.run(30)
    ma, mb = a.moments(), b.moments()
    np.testing.assert_allclose(mb["rho"], rot(ma["rho"]), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(mb["U"][0], rot(ma["U"][1]), rtol=1e-10, atol=1e-15)
    np.testing.assert_allclose(mb["U"][1], -rot(ma["U"][0]), rtol=1e-10, atol=1e-15)


# --------------------------------------------------- floor of the logarithm

def _floored_state(nx, ny, value):
    """Three components, the third at `value` (times the local total density) on a block
    of sites and at O(0.1) elsewhere, with a ring of sites at 1e-3 around the block."""
    rho, u = inputs.random_state(3, nx, ny, seed=61, amp=0.3, umax=0.02)
    tot = rho.sum(0)
    rho[2, 2:5, 3:7] = 1e-3 * tot[2:5, 3:7]
    rho[2, 3, 4:6] = value * tot[3, 4:6]
    return rho, u


@pytest.mark.parametrize("fv", [0, 1])
def test_log_floor_scale_invariance(fv):
    """Eq. definef's logarithm of a component that vanishes is taken at max(rho^s,
    1e-12 rho): the floor is relative to the local total density, so the rho -> lambda rho
    invariance of the kappa = 0 update (f -> lambda f; every potential shifts by a
    constant) still holds where the floor binds.  theta/m^s != 1/3 for every component,
    so the logarithm is evaluated; the third component is exactly 0 at some sites and
    1e-14 rho at others.  A floor without the factor rho would break this at lambda = 100
    (the paper's density)."""
    nx, ny = 10, 8
    chi = _chi(3, 62)
    for value in (0.0, 1e-14):
        rho, u = _floored_state(nx, ny, value)
        a = Oracle(3, nx, ny, 0.9, chi, [1.0, 2.0, 1.0], theta=0.45, forcing_velocity=fv)
        a.init(rho, u)
        b = Oracle(3, nx, ny, 0.9, chi, [1.0, 2.0, 1.0], theta=0.45, forcing_velocity=fv)
        b.init(100.0 * rho, u)
        a.run(3)
        b.run(3)
        assert np.all(np.isfinite(a.f))
        np.testing.assert_allclose(b.f, 100.0 * a.f, rtol=1e-11, atol=1e-12)


def test_log_floor_binds_below_1e_12():
    """Below the floor the update does not see the value of the vanishing density: the
    third component at 0, 1e-14 rho or 5e-13 rho on the same sites gives the same step up
    to those densities themselves (1e-12).  A missing floor (ln 0) or one lower than
    5e-13 would change the potentials there by O(1) and the forces on the neighbours."""
    nx, ny = 10, 8
    chi = _chi(3, 63)
    res = []
    for value in (0.0, 1e-14, 5e-13):
        rho, u = _floored_state(nx, ny, value)
        o = Oracle(3, nx, ny, 0.9, chi, [1.0, 2.0, 1.0], theta=0.45, kappa=0.02)
        o.init(rho, u)
        o.run(2)
        assert np.all(np.isfinite(o.f))
        res.append(o.f)
    assert np.max(np.abs(res[1] - res[0])) < 1e-12
    assert np.max(np.abs(res[2] - res[0])) < 1e-11


def test_log_floor_inactive_above_1e_12():
    """Just above the floor (2e-12 rho) the oracle equals the transcription, which takes
    bare logarithms: the floor does not bind there.  A floor placed higher (1e-11, say)
    would change the potential of those sites by O(1)."""
    nx, ny = 10, 8
    chi = _chi(3, 64)
    m = np.array([1.0, 2.0, 1.0])
    rho, u = _floored_state(nx, ny, 2e-12)
    o = Oracle(3, nx, ny, 0.9, chi, m, theta=0.45, kappa=0.02)
    o.init(rho, u)
    f = o.f.copy()
    o.run(1)
    want = tr.step_d2q9(f, chi, m, 0.45, 0.02, 0.9)
    np.testing.assert_allclose(o.f, want, rtol=1e-10, atol=1e-13)


def test_log_term_dropped_when_its_coefficient_vanishes():
    """theta = m^s/3 for every component: the logarithm of rho^s cancels from nu^s
    exactly (Eq. definef with Eq. lgf), so the oracle drops it and a component that is
    exactly 0 on some sites needs no floor.  The transcription keeps both logarithms (its
    complex-step derivative needs a density well above its step 1e-30) and is evaluated
    with that density at 1e-16 there: the two agree to that density."""
    nx, ny = 10, 8
    chi = _chi(3, 65)
    rho, u = _floored_state(nx, ny, 0.0)
    o = Oracle(3, nx, ny, 0.9, chi, None, theta=1 / 3, kappa=0.02)
    o.init(rho, u)
    f = o.f.copy()
    o.run(1)
    assert np.all(np.isfinite(o.f))
    f_tr = f.copy()
    zero = f_tr[2].sum(0) == 0.0
    assert zero.sum() == 2
    for i in range(9):
        f_tr[2, i][zero] = tr.W9[i] * 1e-16
    want = tr.step_d2q9(f_tr, chi, np.ones(3), 1 / 3, 0.02, 0.9)
    np.testing.assert_allclose(o.f, want, rtol=1e-10, atol=1e-13)


# ------------------------------------------------------------ the D1Q3 path

@pytest.mark.parametrize("fv", [0, 1])
def test_d1q3_path_matches_transcription(fv):
    """The oracle's own D1Q3 path (Sec. 4's lattice, weights 2/3, 1/6, 1/6) against the
    transcription that solves the three moment conditions directly, 60 steps with every
    term on (m != 1, theta != 1/3, kappa, body force), both forcing readings."""
    n, L = 3, 48
    chi = np.array([[0.0, 3.0, 0.5], [3.0, 0.0, 0.2], [0.5, 0.2, 0.0]])
    m = np.array([2.0, 1.0, 1.0])
    x = np.arange(L)
    line = np.stack([0.4 + 0.05 * np.sin(2 * np.pi * x / L),
                     0.35 - 0.05 * np.sin(2 * np.pi * x / L), np.full(L, 0.25)])
    u0 = 0.02 * np.cos(2 * np.pi * x / L)
    theta, kappa, tau, g = 0.4, 0.02, 1 / 0.9, 2e-5
    o = Oracle(n, L, 1, tau, chi, m, theta=theta, kappa=kappa, force=(g, 0.0),
               forcing_velocity=fv, lattice="d1q3")
    o.init(line[:, None, :], np.stack([u0, 0 * u0])[:, None, :])
    f1 = tr.d1q3_init(line, u0)
    # the transcription orders velocities (-1, 0, +1), the oracle (0, +1, -1)
    np.testing.assert_allclose(o.f, f1[:, [1, 2, 0]], rtol=1e-14, atol=1e-16)
    for _ in range(60):
        f1 = tr.d1q3_step(f1, chi, m, theta, kappa, tau, g=g, bary=bool(fv))
    o.run(60)
    np.testing.assert_allclose(o.f, f1[:, [1, 2, 0]], rtol=1e-12, atol=1e-14)
    assert np.max(np.abs(f1.sum(1) - line)) > 1e-4


@pytest.mark.parametrize("fv", [0, 1])
def test_d1q3_path_equals_one_row_d2q9(fv):
    """A D2Q9 lattice of one row is y-invariant, and D1Q3 is its projection (the rest,
    +x and -x populations summed over v_y): the oracle's two paths give the same
    densities, velocities, potentials and pressure tensor, and the projected populations,
    over 100 steps of a phase-separating polymer mixture."""
    n, L = 3, 40
    chi = np.array([[0.0, 2.6, 1.0], [2.6, 0.0, 0.4], [1.0, 0.4, 0.0]])
    m = np.array([3.0, 1.0, 1.0])
    rho, u = inputs.random_state(n, L, 1, seed=66, amp=0.4, umax=0.03)
    u[1] = 0.0
    kw = dict(m=m, theta=0.38, kappa=0.03, force=(1e-5, 0.0), forcing_velocity=fv)
    a = Oracle(n, L, 1, 0.8, chi, lattice="d1q3", **kw)
    b = Oracle(n, L, 1, 0.8, chi, **kw)
    a.init(rho, u)
    b.init(rho, u)
    a.run(100)
    b.run(100)
    proj = np.stack([b.f[:, [0, 2, 4]].sum(1), b.f[:, [1, 5, 8]].sum(1),
                     b.f[:, [3, 6, 7]].sum(1)], axis=1)[:, :, 0, :]
    np.testing.assert_allclose(a.f, proj, rtol=1e-12, atol=1e-15)
    ma, mb = a.moments(), b.moments()
    for k in ("rho", "U", "mu", "P"):
        np.testing.assert_allclose(ma[k], mb[k], rtol=1e-11, atol=1e-14, err_msg=k)
    ca, cb = a.conservation(), b.conservation()
    for k in ("mass", "mom", "force"):
        np.testing.assert_allclose(ca[k], cb[k], rtol=1e-11, atol=1e-15, err_msg=k)


def test_d1q3_conservation_and_momentum_balance():
    """D1Q3: per-component mass kept to rounding (Eq. ff1) and the momentum changed by
    exactly the summed force (Eq. ff2) each step."""
    n, L = 2, 64
    rho, u = inputs.random_state(n, L, 1, seed=67, amp=0.3, umax=0.03)
    o = Oracle(n, L, 1, 0.9, np.array([[0.0, 1.3], [1.3, 0.0]]), [4.0, 1.0], theta=0.5,
               kappa=0.01, force=(3e-5, 0.0), lattice="d1q3")
    o.init(rho, u)
    m0 = o.conservation()["mass"]
    for _ in range(5):
        c0 = o.conservation()
        o.run(1)
        c1 = o.conservation()
        np.testing.assert_allclose(c1["mom"] - c0["mom"], c0["force"], rtol=1e-10, atol=1e-16)
    o.run(500)
    np.testing.assert_allclose(o.conservation()["mass"], m0, rtol=1e-13)


# ------------------------------------------- Gibbs-Duhem reading of the force sum

@pytest.mark.parametrize("fv", [0, 1])
@pytest.mark.parametrize("shape", [(5, 3), (7, 6)])
def test_gibbs_duhem_matches_transcription(shape, fv):
    """force_form = 1 (kappa = 0): three steps against the transcription that adds the
    same vector to every component's acceleration so that their weighted sum is
    (1 - 1/(2 tau)) (1/3) grad rho + rho g."""
    nx, ny = shape
    n = 3
    chi = _chi(n, 70)
    m = np.array([1.0, 3.0, 10.0])
    rho, u = inputs.random_state(n, nx, ny, seed=71, amp=0.4, umax=0.05)
    o = Oracle(n, nx, ny, 0.9, chi, m, theta=0.42, force=(3e-4, -1e-4), forcing_velocity=fv,
               force_form=1)
    o.init(rho, u)
    f = o.f.copy()
    for _ in range(3):
        o.run(1)
        f = tr.step_d2q9(f, chi, m, 0.42, 0.0, 0.9, g=(3e-4, -1e-4), bary=bool(fv), gd=True)
        np.testing.assert_allclose(o.f, f, rtol=1e-12, atol=1e-14)


def test_gibbs_duhem_total_force_and_momentum():
    """The Gibbs-Duhem reading's defining identity, checked on the oracle's own output:
    the density-weighted sum of the accelerations (2 rho (U - u), Eq. scon) equals
    (1 - 1/(2 tau)) (1/3) grad rho + rho g at every site; with g = 0 that sum is a
    discrete gradient, so total momentum is conserved to rounding, which Eq. definef's
    component forces as printed do not give (their sum is not a discrete divergence)."""
    n, nx, ny = 3, 11, 9
    chi = _chi(n, 72)
    m = np.array([2.0, 1.0, 1.0])
    rho, u = inputs.random_state(n, nx, ny, seed=73, amp=0.4, umax=0.03)
    g = (2e-5, -1e-5)
    o = Oracle(n, nx, ny, 0.8, chi, m, theta=0.4, force=g, force_form=1)
    o.init(rho, u)
    o.run(3)
    tot = o.f.sum(0)
    r = tot.sum(0)
    c = C9.astype(float)
    ux = np.einsum("ixy,i->xy", tot, c[:, 0]) / r
    uy = np.einsum("ixy,i->xy", tot, c[:, 1]) / r
    U = o.moments()["U"]
    gx, gy = tr.grad9(r)
    coef = 1 - 1 / (2 * 0.8)
    np.testing.assert_allclose(2 * r * (U[0] - ux), coef * gx / 3 + r * g[0], rtol=0, atol=1e-13)
    np.testing.assert_allclose(2 * r * (U[1] - uy), coef * gy / 3 + r * g[1], rtol=0, atol=1e-13)
    drift = {}
    for ff in (1, 0):
        o = Oracle(n, nx, ny, 0.8, chi, m, theta=0.4, force_form=ff)
        o.init(rho, u)
        m0 = o.conservation()["mom"]
        o.run(200)
        drift[ff] = np.max(np.abs(o.conservation()["mom"] - m0))
    assert drift[1] < 1e-13, drift
    assert drift[0] > 1e-8, drift


@pytest.mark.parametrize("fv", [0, 1])
def test_gibbs_duhem_d1q3_matches_transcription(fv):
    n, L = 3, 40
    chi = np.array([[0.0, 3.0, 0.5], [3.0, 0.0, 0.2], [0.5, 0.2, 0.0]])
    m = np.array([10.0, 1.0, 1.0])
    x = np.arange(L)
    line = np.stack([0.3 + 0.1 * np.sin(2 * np.pi * x / L),
                     0.3 - 0.1 * np.sin(2 * np.pi * x / L), np.full(L, 0.4)])
    o = Oracle(n, L, 1, 1 / 0.9, chi, m, theta=1 / 3, force=(1e-5, 0.0), forcing_velocity=fv,
               lattice="d1q3", force_form=1)
    o.init(line[:, None, :])
    f1 = tr.d1q3_init(line, np.zeros(L))
    for _ in range(40):
        f1 = tr.d1q3_step(f1, chi, m, 1 / 3, 0.0, 1 / 0.9, g=1e-5, bary=bool(fv), gd=True)
    o.run(40)
    np.testing.assert_allclose(o.f, f1[:, [1, 2, 0]], rtol=1e-12, atol=1e-14)


def test_gibbs_duhem_rejects_kappa():
    """The reading is defined for kappa = 0 (the paper's setting): the oracle refuses it
    with a gradient term."""
    o = Oracle(2, 4, 4, 1.0, np.array([[0.0, 2.0], [2.0, 0.0]]), kappa=0.01, force_form=1)
    with pytest.raises(ValueError):
        o.init(np.full((2, 4, 4), 0.5))


def test_gibbs_duhem_polymer_density_level():
    """The paper's polymer binary (m = (10, 1), chi = 0.94, kappa = 0, 1/tau = 0.9, Sec. 4)
    on its D1Q3 lattice, two slabs started at the Flory-Huggins binodal: with the
    Gibbs-Duhem total force (and the barycentric forcing velocity) the total density is
    uniform to better than the paper's 1e-5 after 20000 steps, where Eq. definef's
    component forces as printed leave a step of about 1e-3 between the phases."""
    from oracle import thermo
    lo, hi = thermo.binodal_binary(0.94, 10.0, 1.0)
    nx = 128
    x = np.arange(nx)
    phi = np.where((x >= nx // 4) & (x < 3 * nx // 4), hi, lo)
    rho = np.stack([phi, 1 - phi])[:, None, :]
    chi = np.array([[0.0, 0.94], [0.94, 0.0]])
    step = {}
    for ff in (1, 0):
        o = Oracle(2, nx, 1, 1 / 0.9, chi, [10.0, 1.0], forcing_velocity=1, lattice="d1q3",
                   force_form=ff)
        o.init(rho)
        assert o.run(20000) == 0
        r = o.moments()["rho"].sum(0)
        step[ff] = (r.max() - r.min()) / r.mean()
    assert step[1] < 1e-5, step
    assert step[0] > 1e-4, step
