"""GPU: the D3Q19 lattice against the FP64 oracle's D3Q19 path, on both schedules: the
density pass + z-plane march (cube_march.cuh, N <= 4) and the staged one (cube.cuh).

Tolerances as on D2Q9: FP64 1e-12 of the field's max-norm (P absolute), FP32 1e-5 per
field after 100 steps.  Plus the projection property on the GPU (a z-invariant D3Q19 run
summed over v_z equals the D2Q9 handle's run), resume, the mass compensation and the
bulk-phase fit.
"""
import numpy as np
import pytest

import paper_0704_3444_gb300 as mclb
from oracle import Oracle
from paper_0704_3444_gb300 import inputs

pytestmark = pytest.mark.gpu

V3 = np.array([(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
               (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0), (1, 0, 1), (-1, 0, -1),
               (1, 0, -1), (-1, 0, 1), (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)])
V2 = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]


@pytest.fixture(scope="module", autouse=True)
def built():
    mclb.build()
    mclb.load()


def _rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def _state(n, nx, ny, nz, seed, amp=0.3, umax=0.03):
    rng = np.random.default_rng(seed)
    phi = 1.0 / n + (amp / n) * rng.uniform(-1, 1, (n, nz, ny, nx))
    phi -= phi.mean(axis=0, keepdims=True) - 1.0 / n
    u = umax * rng.uniform(-1, 1, (3, nz, ny, nx))
    return phi, u


# (nx, ny, nz, N): lattices smaller than the march's 28 x 8 tiles, several tiles in x and y
# with ragged last ones and several z segments (60 x 37 x 20), one and two layers (every
# z neighbour the layer itself or the other one), one component, and N = 5, which only the
# staged schedule takes
CASES = [(5, 4, 3, 2), (17, 6, 5, 3), (33, 9, 4, 4), (60, 37, 20, 3), (9, 7, 1, 2), (6, 5, 2, 3),
         (9, 5, 6, 1), (7, 3, 11, 5)]
KERNELS = [mclb.KERNEL_FUSED, mclb.KERNEL_STAGED]
MARCH_NMAX = 4


@pytest.mark.parametrize("fv", [0, 1])
@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}x{c[1]}x{c[2]}N{c[3]}")
def test_fp64_parity(case, kernel, fv):
    """10 FP64 steps with every term on (m != 1, theta != 1/3, kappa > 0, a 3-D body
    force): the state, rho, U, mu within 1e-12 of the oracle (relative to the field's
    max), P to 1e-12 absolute, and the conservation sums."""
    nx, ny, nz, n = case
    rho, u = _state(n, nx, ny, nz, seed=300 + nx + n)
    chi = inputs.uniform_chi(n, 1.6)
    kw = dict(m=[1.0 + (k % 3) for k in range(n)], theta=0.4, kappa=0.02,
              force=(1e-5, -2e-5, 3e-5), forcing_velocity=fv, lattice="d3q19", nz=nz)
    if kernel == mclb.KERNEL_FUSED and n > MARCH_NMAX:
        with pytest.raises(mclb.MclbError, match="fused kernel unavailable"):
            mclb.Simulation(n, nx, ny, 0.9, chi, precision="fp64", kernel=kernel, **kw)
        return
    sim = mclb.Simulation(n, nx, ny, 0.9, chi, precision="fp64", kernel=kernel, **kw)
    assert sim.launches_per_step == (2 if kernel == mclb.KERNEL_FUSED else 3)
    orc = Oracle(n, nx, ny, 0.9, chi, **kw)
    sim.init_fields(rho, u)
    orc.init(rho, u)
    sim.step(10)
    assert orc.run(10) == 0
    assert sim.status() == 0
    assert _rel(sim.get_state(), orc.f) < 1e-12
    gm, om = sim.moments(), orc.moments()
    for k in ("rho", "U", "mu"):
        assert _rel(gm[k], om[k]) < 1e-12, k
    assert np.max(np.abs(gm["P"] - om["P"])) < 1e-12
    gc, oc = sim.conservation(), orc.conservation()
    np.testing.assert_allclose(gc["mass"], oc["mass"], rtol=1e-13)
    np.testing.assert_allclose(gc["mom"], oc["mom"], rtol=1e-10, atol=1e-14)
    np.testing.assert_allclose(gc["force"], oc["force"], rtol=1e-9, atol=1e-15)
    sim.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("shape", [(60, 37, 20), (100, 17, 40)], ids=lambda s: "x".join(map(str, s)))
def test_march_equals_staged_bitwise(shape, precision):
    """The march forms the same sums in the same order as the three staged kernels, so
    after 25 steps of the 3-D ternary (every term on, a body force) the two schedules'
    states are identical bit for bit, on lattices of several tiles and z segments."""
    nx, ny, nz = shape
    chi = np.array([[0.0, 3.0, 0.5], [3.0, 0.0, 0.2], [0.5, 0.2, 0.0]])  # the paper's ternary set
    rho, u = _state(3, nx, ny, nz, seed=nx + nz)
    kw = dict(m=[1.0, 2.0, 1.0], theta=0.4, kappa=0.02, force=(1e-5, -2e-5, 3e-5),
              lattice="d3q19", nz=nz, precision=precision)
    sims = [mclb.Simulation(3, nx, ny, 0.9, chi, kernel=k, **kw) for k in KERNELS]
    for s in sims:
        s.init_fields(rho, u)
        s.step(25)
        assert s.status() == 0
    assert sims[0].launches_per_step == 2 and sims[1].launches_per_step == 3
    assert np.array_equal(sims[0].get_state(), sims[1].get_state())
    for s in sims:
        s.close()


def test_fp64_gibbs_duhem():
    """The Gibbs-Duhem force reading (kappa = 0) with the barycentric forcing velocity:
    20 FP64 steps within 1e-12 of the oracle, total momentum kept to 1e-13."""
    n, nx, ny, nz = 3, 12, 10, 8
    rho, u = _state(n, nx, ny, nz, seed=41)
    chi = inputs.uniform_chi(n, 1.6)
    kw = dict(m=[1.0, 2.0, 1.0], theta=0.4, forcing_velocity=1, force_form=1, lattice="d3q19",
              nz=nz)
    sim = mclb.Simulation(n, nx, ny, 0.9, chi, precision="fp64", **kw)
    orc = Oracle(n, nx, ny, 0.9, chi, **kw)
    sim.init_fields(rho, u)
    orc.init(rho, u)
    m0 = sim.conservation()["mom"]
    sim.step(20)
    assert orc.run(20) == 0
    assert sim.status() == 0
    assert _rel(sim.get_state(), orc.f) < 1e-12
    assert np.max(np.abs(sim.conservation()["mom"] - m0)) < 1e-13
    sim.close()


@pytest.mark.parametrize("kernel", KERNELS)
def test_fp32_four_fields(kernel):
    """The 3-D ternary recipe (paper's chi set at (0.4, 0.4, 0.2), inside the A-B
    spinodal) on 24^3: rho, U, mu and P within 1e-5 of the oracle after 100 FP32 steps."""
    p = inputs.ternary3d(24, steps=100)
    sim = mclb.Simulation.from_problem(p, precision="fp32", kernel=kernel)
    orc = Oracle.from_problem(p)
    sim.step(100)
    assert orc.run(100) == 0
    assert sim.status() == 0
    gm, om = sim.moments(), orc.moments()
    err = {k: float(np.max(np.abs(gm[k] - om[k]))) for k in ("rho", "U", "mu", "P")}
    assert all(e < 1e-5 for e in err.values()), err
    sim.close()


@pytest.mark.parametrize("kernel", KERNELS)
def test_z_invariant_run_equals_d2q9_handle(kernel):
    """A D3Q19 handle whose fields do not depend on z (4 layers), after 30 FP64 steps and
    a sum over v_z, equals the D2Q9 staged handle of the plane to 1e-12."""
    n, nx, ny, nz = 3, 19, 13, 4
    rho2, u2 = inputs.random_state(n, nx, ny, seed=57, amp=0.3, umax=0.03)
    chi = inputs.uniform_chi(n, 1.7)
    common = dict(m=[1.0, 3.0, 1.5], theta=0.42, kappa=0.02, precision="fp64")
    s2 = mclb.Simulation(n, nx, ny, 0.85, chi, force=(2e-5, -1e-5), kernel=mclb.KERNEL_STAGED,
                         **common)
    s2.init_fields(rho2, u2)
    rho3 = np.repeat(rho2[:, None], nz, axis=1)
    u3 = np.zeros((3, nz, ny, nx))
    u3[0], u3[1] = u2[0][None], u2[1][None]
    s3 = mclb.Simulation(n, nx, ny, 0.85, chi, force=(2e-5, -1e-5, 0.0), kernel=kernel,
                         lattice="d3q19", nz=nz, **common)
    s3.init_fields(rho3, u3)
    s2.step(30)
    s3.step(30)
    assert s2.status() == 0 and s3.status() == 0
    f3 = s3.get_state()
    proj = np.zeros((n, 9, nz, ny, nx))
    for i, c in enumerate(V3):
        proj[:, V2.index((int(c[0]), int(c[1])))] += f3[:, i]
    f2 = s2.get_state()
    for z in range(nz):
        assert _rel(proj[:, :, z], f2) < 1e-12
    s2.close()
    s3.close()


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_resume_equals_uninterrupted(precision, kernel):
    """get_state after 13 steps, set_state into a new handle, 17 more steps there equal
    17 more steps of the original, bitwise."""
    p = inputs.ternary3d(20)
    a = mclb.Simulation.from_problem(p, precision=precision, kernel=kernel)
    a.step(13)
    b = mclb.Simulation(p.ncomp, p.nx, p.ny, p.tau, p.chi, p.m, p.theta, p.kappa, p.force,
                        precision, kernel, lattice="d3q19", nz=p.nz)
    b.set_state(a.get_state())
    a.step(17)
    b.step(17)
    assert a.status() == 0 and b.status() == 0
    assert np.array_equal(a.get_state(), b.get_state())
    a.close()
    b.close()


def test_mass_compensation():
    """FP32 with the compensation every 50 steps: masses within 1e-6 of the start after
    1000 steps of the 3-D ternary on 32^3."""
    p = inputs.ternary3d(32, steps=1000)
    sim = mclb.Simulation.from_problem(p, precision="fp32", mass_every=50)
    m0 = sim.conservation()["mass"]
    sim.step(1000)
    assert sim.status() == 0
    drift = np.abs(sim.conservation()["mass"] / m0 - 1.0)
    assert np.all(drift < 1e-6), drift
    sim.close()


def test_fit_equilibrium_on_slabs():
    """The paper's ternary chi set started as two slabs (in x) at the ends of the
    Flory-Huggins tie line through (0.4, 0.4, 0.2), 24 x 8 x 8, 2000 FP64 steps: the
    device fit of the two phases equals the k-means definition on the handle's own
    compositions to 1e-12, and lies within 0.05 of the tie line."""
    from oracle import thermo
    from tests.test_gpu_batch_fit import _fit_by_definition
    chi = np.zeros((3, 3))
    chi[0, 1] = chi[1, 0] = 3.0
    chi[0, 2] = chi[2, 0] = 0.5
    chi[1, 2] = chi[2, 1] = 0.2
    q1, q2 = thermo.tie_line(chi, np.ones(3), [0.4, 0.4, 0.2])
    hi, lo = (np.asarray(q1), np.asarray(q2)) if q1[0] > q2[0] else (np.asarray(q2), np.asarray(q1))
    nx, ny, nz = 24, 8, 8
    x = np.arange(nx)
    inside = (x >= nx // 4) & (x < 3 * nx // 4)
    phi = np.where(inside[None, :], hi[:, None], lo[:, None])
    rho = np.ascontiguousarray(np.broadcast_to(phi[:, None, None, :], (3, nz, ny, nx)))
    sim = mclb.Simulation(3, nx, ny, 1 / 0.9, chi, precision="fp64", lattice="d3q19", nz=nz)
    sim.init_fields(rho)
    sim.step(2000)
    assert sim.status() == 0
    fit = sim.fit_equilibrium(2)
    want = _fit_by_definition(sim.moments(U=False, mu=False, P=False)["rho"], 2, lattice="d3q19")
    assert np.max(np.abs(fit - want)) < 1e-12
    assert np.max(np.abs(fit[0] - hi)) < 0.05 and np.max(np.abs(fit[1] - lo)) < 0.05
    sim.close()
