"""Pins of the oracle's D3Q19 path (the method's equations on a three-dimensional
lattice whose weights give the Sec. 3 moments).

* The velocity set is rebuilt here from its definition (every vector of {-1, 0, 1}^3
  with |v|^2 <= 2, weights 1/3, 1/18, 1/36 by |v|^2) and the oracle's per-site
  equilibrium and forcing are checked against the Sec. 3 and Eqs. ff1-ff3 moments to
  third order.
* Projection: summing the D3Q19 populations that share their in-plane velocity gives
  the D2Q9 weights; equilibria, forcing and the gradient and Laplacian stencils are
  linear in the weights, so a D3Q19 run whose fields do not depend on one axis equals,
  after that sum, the D2Q9 run of the plane -- for each of the three axes.
* Conservation: per-component mass to rounding, momentum changing by exactly the force
  sum; uniform states are fixed points; the Gibbs-Duhem reading keeps total momentum.
* A mode along the body diagonal (1, 1, 1), which no plane run contains, decays at the
  ideal-mixture rate D = (tau - 1/2) theta of Eq. woche, with O(k^2) convergence.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import Oracle, equilibrium3, forcing3
from paper_0704_3444_gb300 import inputs

# the oracle's velocity order, as documented in oracle/__init__.py
V3 = np.array([(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
               (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0), (1, 0, 1), (-1, 0, -1),
               (1, 0, -1), (-1, 0, 1), (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)])
V2 = np.array([(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)])


def _weights(v):
    return np.array([{0: 1 / 3, 1: 1 / 18, 2: 1 / 36}[int(np.dot(c, c))] for c in v])


def test_velocity_set_is_the_d3q19_set():
    full = [c for c in itertools.product((-1, 0, 1), repeat=3) if sum(x * x for x in c) <= 2]
    assert sorted(map(tuple, V3)) == sorted(full)
    w = _weights(V3)
    assert abs(w.sum() - 1.0) < 1e-15
    # isotropy to fourth order: sum w v_a v_b = delta / 3,
    # sum w v_a v_b v_c v_d = (d_ab d_cd + d_ac d_bd + d_ad d_bc) / 9
    I = np.eye(3)
    np.testing.assert_allclose(np.einsum("i,ia,ib->ab", w, V3, V3), I / 3, atol=1e-15)
    t4 = np.einsum("i,ia,ib,ic,id->abcd", w, V3, V3, V3, V3)
    want = (np.einsum("ab,cd->abcd", I, I) + np.einsum("ac,bd->abcd", I, I)
            + np.einsum("ad,bc->abcd", I, I)) / 9
    np.testing.assert_allclose(t4, want, atol=1e-15)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_equilibrium_and_forcing_moments(seed):
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.2, 2.0)
    u = rng.uniform(-0.1, 0.1, 3)
    j = rng.uniform(-0.1, 0.1, 3)
    a = rng.uniform(-0.01, 0.01, 3)
    fe = equilibrium3(rho, *u)
    assert abs(fe.sum() - rho) < 1e-14
    np.testing.assert_allclose(fe @ V3, rho * u, atol=1e-15)
    np.testing.assert_allclose(np.einsum("i,ia,ib->ab", fe, V3, V3),
                               rho / 3 * np.eye(3) + rho * np.outer(u, u), atol=1e-15)
    # third moment: (rho / 3) (u_a d_bc + u_b d_ac + u_c d_ab)
    I = np.eye(3)
    t3 = np.einsum("i,ia,ib,ic->abc", fe, V3, V3, V3)
    want = rho / 3 * (np.einsum("a,bc->abc", u, I) + np.einsum("b,ac->abc", u, I)
                      + np.einsum("c,ab->abc", u, I))
    np.testing.assert_allclose(t3, want, atol=1e-15)
    F = forcing3(rho, *j, *a)
    assert abs(F.sum()) < 1e-16
    np.testing.assert_allclose(F @ V3, rho * a, atol=1e-16)
    np.testing.assert_allclose(np.einsum("i,ia,ib->ab", F, V3, V3),
                               np.outer(a, j) + np.outer(j, a), atol=1e-16)


def _plane_map(axis):
    """For a run invariant along `axis`, the two remaining axes as D2Q9's (x, y) and, per
    D3Q19 velocity, the D2Q9 velocity its in-plane part is."""
    keep = [d for d in range(3) if d != axis]
    idx = []
    for c in V3:
        inplane = (int(c[keep[0]]), int(c[keep[1]]))
        idx.append([tuple(v) for v in V2].index(inplane))
    return keep, np.array(idx)


def _random_plane(n, nx, ny, seed):
    rho, u = inputs.random_state(n, nx, ny, seed=seed, amp=0.3, umax=0.03)
    return rho, u


@pytest.mark.parametrize("fv,ff", [(0, 0), (1, 0), (1, 1)])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_invariant_run_projects_onto_d2q9(axis, fv, ff):
    """Fields independent of `axis` (3 layers along it): after 4 steps the D3Q19
    populations summed over the velocities that share an in-plane velocity equal the
    D2Q9 run of the plane, and so do rho, U, mu and the in-plane P, to 1e-13 -- with
    m != 1, theta != 1/3, kappa > 0 (not with the Gibbs-Duhem reading, which needs
    kappa = 0) and an in-plane body force."""
    n, a, b = 3, 7, 6                       # plane size (D2Q9 nx = a, ny = b)
    rho2, u2 = _random_plane(n, a, b, seed=90 + axis)
    chi = inputs.uniform_chi(n, 1.7)
    kappa = 0.0 if ff else 0.02
    g2 = (2e-5, -1e-5)
    common = dict(m=[1.0, 3.0, 1.5], theta=0.42, kappa=kappa, forcing_velocity=fv, force_form=ff)
    o2 = Oracle(n, a, b, 0.85, chi, force=g2, **common)
    o2.init(rho2, u2)
    keep, idx = _plane_map(axis)
    # 3-D arrays with axes (z, y, x) = dims (2, 1, 0): the plane's x is keep[0], y keep[1]
    size = [0, 0, 0]
    size[keep[0]], size[keep[1]], size[axis] = a, b, 3
    nx, ny, nz = size
    g3 = [0.0, 0.0, 0.0]
    g3[keep[0]], g3[keep[1]] = g2

    def lift(field2):          # (c, b, a) plane field -> (c, nz, ny, nx)
        c = field2.shape[0]
        out = np.empty((c, nz, ny, nx))
        for z in range(nz):
            for y in range(ny):
                for x in range(nx):
                    pos = (x, y, z)
                    out[:, z, y, x] = field2[:, pos[keep[1]], pos[keep[0]]]
        return out

    u3 = np.zeros((3, nz, ny, nx))
    lifted_u = lift(u2)
    u3[keep[0]], u3[keep[1]] = lifted_u[0], lifted_u[1]
    o3 = Oracle(n, nx, ny, 0.85, chi, force=tuple(g3), lattice="d3q19", nz=nz, **common)
    o3.init(lift(rho2), u3)
    assert o2.run(4) == 0 and o3.run(4) == 0
    proj = np.zeros((n, 9, nz, ny, nx))
    for i in range(19):
        proj[:, idx[i]] += o3.f[:, i]
    want = lift(o2.f.reshape(n * 9, b, a)).reshape(n, 9, nz, ny, nx)
    assert np.max(np.abs(proj - want)) < 1e-13 * np.abs(want).max()
    m2, m3 = o2.moments(), o3.moments()
    np.testing.assert_allclose(m3["rho"], lift(m2["rho"]), rtol=0, atol=1e-13)
    np.testing.assert_allclose(m3["mu"], lift(m2["mu"]), rtol=0, atol=1e-12)
    U2 = lift(m2["U"])
    np.testing.assert_allclose(m3["U"][keep[0]], U2[0], rtol=0, atol=1e-14)
    np.testing.assert_allclose(m3["U"][keep[1]], U2[1], rtol=0, atol=1e-14)
    assert np.max(np.abs(m3["U"][axis])) < 1e-15
    # P components (xx, xy, xz, yy, yz, zz) of the plane's (xx, xy, yy)
    comp = {(0, 0): 0, (0, 1): 1, (0, 2): 2, (1, 1): 3, (1, 2): 4, (2, 2): 5}
    P2 = lift(m2["P"])
    for (r, c), k2 in (((0, 0), 0), ((0, 1), 1), ((1, 1), 2)):
        key = tuple(sorted((keep[r], keep[c])))
        np.testing.assert_allclose(m3["P"][comp[key]], P2[k2], rtol=0, atol=1e-13)


def _random3(n, nx, ny, nz, seed):
    rng = np.random.default_rng(seed)
    phi = 1.0 / n + 0.05 * rng.uniform(-1, 1, (n, nz, ny, nx))
    phi -= phi.mean(axis=0, keepdims=True) - 1.0 / n
    u = 0.02 * rng.uniform(-1, 1, (3, nz, ny, nx))
    return phi, u


def test_conservation_and_momentum_balance():
    """Random 3-D state, every term on: each component's mass is kept to 1e-13
    (relative) over 50 steps, and one step changes the momentum by the force sum."""
    n = 3
    rho, u = _random3(n, 6, 5, 4, seed=7)
    o = Oracle(n, 6, 5, 0.9, inputs.uniform_chi(n, 1.6), m=[1.0, 2.0, 1.0], theta=0.4,
               kappa=0.01, force=(1e-5, 2e-5, -3e-5), lattice="d3q19", nz=4)
    o.init(rho, u)
    c0 = o.conservation()
    assert o.run(1) == 0
    c1 = o.conservation()
    np.testing.assert_allclose(c1["mom"] - c0["mom"], c0["force"], rtol=1e-10, atol=1e-15)
    assert o.run(49) == 0
    c2 = o.conservation()
    assert np.all(np.abs(c2["mass"] / c0["mass"] - 1.0) < 1e-13)


def test_uniform_state_is_a_fixed_point():
    n = 2
    rho = np.empty((n, 3, 4, 5))
    rho[0], rho[1] = 0.3, 0.7
    u = np.zeros((3, 3, 4, 5))
    u[0], u[1], u[2] = 0.01, -0.02, 0.015
    o = Oracle(n, 5, 4, 0.8, inputs.uniform_chi(n, 2.5), kappa=0.05, lattice="d3q19", nz=3)
    o.init(rho, u)
    f0 = o.f.copy()
    o.run(3)
    assert np.max(np.abs(o.f - f0)) < 1e-15


def test_gibbs_duhem_keeps_total_momentum():
    """Gibbs-Duhem reading (kappa = 0, no body force): the total force is a discrete
    gradient, so total momentum stays at its start to rounding; the printed form changes
    it by the non-vanishing force sum."""
    n = 3
    rho, u = _random3(n, 6, 6, 5, seed=11)
    drift = {}
    for ff in (0, 1):
        o = Oracle(n, 6, 6, 0.9, inputs.uniform_chi(n, 1.6), m=[1.0, 2.0, 1.0], theta=0.4,
                   lattice="d3q19", nz=5, force_form=ff)
        o.init(rho, u)
        m0 = o.conservation()["mom"]
        assert o.run(20) == 0
        drift[ff] = np.max(np.abs(o.conservation()["mom"] - m0))
    assert drift[1] < 1e-13, drift
    assert drift[0] > 1e-8, drift


def _diagonal_rate(n, theta, tau, t_span, t0=60, amp=1e-5):
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    k = 2 * math.pi / n
    s = np.sin(k * (x + y + z))
    rho = np.stack([0.5 + amp * s, 0.5 - amp * s])
    o = Oracle(2, n, n, tau, np.zeros((2, 2)), theta=theta, lattice="d3q19", nz=n)
    o.init(rho)

    def amplitude():
        r = o.moments()["rho"][0]
        return 2.0 * np.mean((r - r.mean()) * s)

    o.run(t0)
    a0 = amplitude()
    o.run(t_span)
    return math.log(amplitude() / a0) / t_span, 3 * k * k


def test_body_diagonal_mode_decays_at_the_ideal_mixture_rate():
    """Eq. woche for an ideal mixture (chi = kappa = 0): a concentration mode along
    (1, 1, 1) decays at D |k|^2 with D = (tau - 1/2) theta; theta != 1/3 makes it depend
    on the force coefficient 1 - 1/(2 tau).  Relative error O(k^2): about 4x smaller
    from n = 16 to n = 32."""
    theta, tau = 0.5, 0.8
    D = (tau - 0.5) * theta
    errs = []
    for n in (16, 32):
        k2 = 3 * (2 * math.pi / n) ** 2
        rate, k2 = _diagonal_rate(n, theta, tau, int(2.0 / (D * k2)))
        errs.append(rate / (-D * k2) - 1.0)
    assert abs(errs[1]) < 5e-3, errs
    assert 3.0 < errs[0] / errs[1] < 5.0, errs
