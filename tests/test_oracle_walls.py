"""Pins of the oracle's solid walls in y (D2Q9, walls = 1; the paper has no walls).

The reading: stationary walls halfway between rows, below row 0 and above row ny - 1; a
population that would stream across a wall returns to its site with the opposite
velocity (halfway bounce-back); the stencils of rho^s, nu^s and rho see the rows beyond
a wall as mirror images of the rows next to it (zero normal gradient, neutral wetting).

* Bounce-back keeps every population inside the lattice, so each component's mass is
  conserved to rounding (Eq. ff1 and the collision keep it site by site).
* A uniform mixture at rest stays at rest: it is a fixed point.
* The set-up is symmetric under the reflection y -> ny - 1 - y, so a reflected start
  gives the reflected result.
* Plane Poiseuille flow: a body force g along x between the walls (channel width H = ny,
  walls at y = -1/2 and H - 1/2) drives the steady profile U(y) = g / (2 nu) (y + 1/2)
  (H - y - 1/2) with the shear viscosity nu = (tau - 1/2)/3 of the overall fluid (pinned
  separately by the shear-wave decay).  The lattice profile converges at O(1/H^2).
"""
import numpy as np
import pytest

from oracle import Oracle
from paper_0704_3444_gb300 import inputs

VY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
MIRROR = [0, 1, 4, 3, 2, 8, 7, 6, 5]     # velocity index with v_y flipped


def test_mass_is_conserved_with_walls():
    n, nx, ny = 3, 9, 8
    rho, u = inputs.random_state(n, nx, ny, seed=71, amp=0.3, umax=0.03)
    o = Oracle(n, nx, ny, 0.9, inputs.uniform_chi(n, 1.6), m=[1.0, 2.0, 1.0], theta=0.4,
               kappa=0.02, force=(1e-5, -2e-5), walls=1)
    o.init(rho, u)
    m0 = o.conservation()["mass"]
    assert o.run(300) == 0
    assert np.all(np.abs(o.conservation()["mass"] / m0 - 1.0) < 1e-13)


def test_uniform_rest_state_is_a_fixed_point():
    n, nx, ny = 2, 5, 6
    rho = np.empty((n, ny, nx))
    rho[0], rho[1] = 0.3, 0.7
    o = Oracle(n, nx, ny, 0.8, inputs.uniform_chi(n, 2.5), kappa=0.05, walls=1)
    o.init(rho)
    f0 = o.f.copy()
    o.run(5)
    assert np.max(np.abs(o.f - f0)) < 1e-15


@pytest.mark.parametrize("fv", [0, 1])
def test_reflection_symmetry(fv):
    """Reflect the start in y (fields, v_y and the body force's y component): after 20
    steps the state is the reflection of the unreflected run's, to 1e-13."""
    n, nx, ny = 3, 7, 9
    rho, u = inputs.random_state(n, nx, ny, seed=73, amp=0.3, umax=0.03)
    kw = dict(m=[1.0, 2.0, 1.0], theta=0.4, kappa=0.02, forcing_velocity=fv, walls=1)
    chi = inputs.uniform_chi(n, 1.6)
    a = Oracle(n, nx, ny, 0.9, chi, force=(1e-5, -2e-5), **kw)
    a.init(rho, u)
    ur = u[:, ::-1].copy()
    ur[1] *= -1.0
    b = Oracle(n, nx, ny, 0.9, chi, force=(1e-5, 2e-5), **kw)
    b.init(np.ascontiguousarray(rho[:, ::-1]), ur)
    assert a.run(20) == 0 and b.run(20) == 0
    want = a.f[:, MIRROR, ::-1, :]
    assert np.max(np.abs(b.f - want)) < 1e-13 * np.abs(want).max()


def _poiseuille_error(H, tau, g=1e-6, ncomp=1):
    chi = np.zeros((ncomp, ncomp))
    rho = np.full((ncomp, H, 1), 1.0 / ncomp)
    o = Oracle(ncomp, 1, H, tau, chi, force=(g, 0.0), walls=1)
    o.init(rho)
    nu = (tau - 0.5) / 3.0
    steps = int(12 * H * H / nu / np.pi ** 2) + 1000
    assert o.run(steps) == 0
    U = o.moments()["U"][0, :, 0]
    y = np.arange(H) + 0.5
    want = g / (2.0 * nu) * y * (H - y)
    return np.max(np.abs(U - want)) / want.max(), U


@pytest.mark.parametrize("tau", [0.8, 1.2])
def test_poiseuille_profile_converges(tau):
    """The steady profile between the walls approaches the parabola at O(1/H^2): its
    largest relative error falls 3-5x from H = 16 to H = 32 and is below 2e-2 at H = 32.
    The same flow of an ideal binary mixture (two identical components) gives the same
    profile to 1e-12 of its maximum."""
    e16, _ = _poiseuille_error(16, tau)
    e32, U1 = _poiseuille_error(32, tau)
    assert e32 < 2e-2, (e16, e32)
    assert 3.0 < e16 / e32 < 5.0, (e16, e32)
    _, U2 = _poiseuille_error(32, tau, ncomp=2)
    assert np.max(np.abs(U2 - U1)) < 1e-12 * np.abs(U1).max()


@pytest.mark.parametrize("fv", [0, 1])
def test_layered_state_equals_its_mirrored_periodic_double(fv):
    """A state that varies only in y, with no x-velocity and no x-force, keeps that
    symmetry; for it bounce-back returns exactly what a mirror image of the channel would
    send (the x-mirrored velocity carries the same population), and the mirrored stencil
    rows are the mirror image's rows.  So the walled channel of height H evolves as rows
    0..H-1 of the periodic channel of height 2H started with the state and its mirror
    image (y -> 2H - 1 - y, v_y -> -v_y).  Checked after 200 steps with a phase-separating
    binary layer profile, kappa > 0, m != 1 and a y-velocity, to 1e-13."""
    n, nx, H = 2, 3, 10
    y = np.arange(H)
    phi = 0.5 + 0.3 * np.tanh((y - 3.5) / 1.5)
    rho = np.empty((n, H, nx))
    rho[0] = phi[:, None]
    rho[1] = 1.0 - phi[:, None]
    u = np.zeros((2, H, nx))
    u[1] = 0.01 * np.sin(np.pi * (y + 0.5) / H)[:, None]
    kw = dict(m=[2.0, 1.0], theta=0.4, kappa=0.05, forcing_velocity=fv)
    chi = np.array([[0.0, 1.8], [1.8, 0.0]])
    a = Oracle(n, nx, H, 0.9, chi, walls=1, **kw)
    a.init(rho, u)
    rho2 = np.concatenate([rho, rho[:, ::-1]], axis=1)
    u2 = np.concatenate([u, u[:, ::-1]], axis=1)
    u2[1, H:] *= -1.0
    b = Oracle(n, nx, 2 * H, 0.9, chi, **kw)
    b.init(np.ascontiguousarray(rho2), np.ascontiguousarray(u2))
    assert a.run(200) == 0 and b.run(200) == 0
    assert np.max(np.abs(a.f - b.f[:, :, :H])) < 1e-13 * np.abs(a.f).max()
    ma, mb = a.moments(), b.moments()
    for k in ("rho", "mu", "P"):
        assert np.max(np.abs(ma[k] - mb[k][:, :H])) < 1e-12, k
