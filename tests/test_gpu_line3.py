"""GPU: the D1Q3 lattice (the paper's own, Sec. 4) through the C ABI, against the oracle's
D1Q3 path and against the library's own one-row D2Q9 lattice.

Tolerances: FP64 1e-12 of the field's max-norm (populations; rho, U, mu; P absolute);
FP32 1e-5 absolute on the densities after short runs.  Lines up to the resident limit
run in shared memory (one CTA advances a whole line by up to 4096 steps per launch);
longer ones step once per launch with the tile kernel: both are covered.
"""
import numpy as np
import pytest

import paper_0704_3444_gb300 as mclb
from oracle import Oracle, thermo
from paper_0704_3444_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    mclb.build()
    mclb.load()


def _chi(n, seed):
    r = inputs.uniform(seed, n * n, 3).reshape(n, n)
    c = 2.0 + (r + r.T)
    np.fill_diagonal(c, 0.0)
    return c


def _rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def _line_pair(n, nx, tau, chi, m, theta, kappa, g, precision, fv, seed):
    rho, u = inputs.random_state(n, nx, 1, seed=seed, amp=0.3, umax=0.03)
    u[1] = 0.0
    sim = mclb.Simulation(n, nx, 1, tau, chi, m, theta, kappa, (g, 0.0), precision,
                          forcing_velocity=fv, lattice="d1q3")
    orc = Oracle(n, nx, 1, tau, chi, m, theta, kappa, (g, 0.0), forcing_velocity=fv,
                 lattice="d1q3")
    sim.init_fields(rho, u)
    orc.init(rho, u)
    return sim, orc


LINES = [
    # (nx, N, steps, tau, theta, kappa, m, g)
    (1, 2, 30, 1.0, 1 / 3, 0.0, None, 0.0),
    (2, 3, 30, 0.8, 0.4, 0.05, [1.0, 3.0, 10.0], 3e-4),
    (5, 1, 30, 0.9, 1 / 3, 0.02, None, 1e-4),
    (64, 2, 50, 0.7, 0.45, 0.01, None, 0.0),
    (130, 4, 50, 1.0, 1 / 3, 0.01, None, 2e-5),
    (250, 5, 40, 1.2, 0.4, 0.01, None, 0.0),
    (300, 8, 20, 1.1, 1 / 3, 0.01, [1, 1, 2, 1, 1, 3, 1, 1], 0.0),
    (1000, 3, 25, 0.8, 0.5, 0.01, [2.0, 1.0, 1.0], 1e-5),
    # longer than the resident limit for N = 3 in FP64: the tile kernel, ragged last tile
    (3001, 3, 25, 0.9, 0.4, 0.02, None, 1e-5),
]


@pytest.mark.parametrize("fv", [0, 1], ids=["component_u", "barycentric_u"])
@pytest.mark.parametrize("case", LINES, ids=lambda c: f"{c[0]}N{c[1]}")
def test_line3_fp64_parity(case, fv):
    nx, n, steps, tau, theta, kappa, m, g = case
    sim, orc = _line_pair(n, nx, tau, _chi(n, n + nx), m, theta, kappa, g, "fp64", fv,
                          seed=2000 + nx + n)
    assert sim.launches_per_step == 1
    np.testing.assert_allclose(sim.get_state(), orc.f, rtol=0, atol=1e-15 * np.abs(orc.f).max())
    sim.step(steps)
    assert orc.run(steps) == 0
    assert sim.status() == 0
    assert _rel(sim.get_state(), orc.f) < 1e-12
    gm, om = sim.moments(), orc.moments()
    for k in ("rho", "U", "mu"):
        assert _rel(gm[k], om[k]) < 1e-11, k
    assert np.max(np.abs(gm["P"] - om["P"])) < 1e-12 * max(1.0, np.abs(om["P"]).max())
    gc, oc = sim.conservation(), orc.conservation()
    np.testing.assert_allclose(gc["mass"], oc["mass"], rtol=1e-13)
    np.testing.assert_allclose(gc["force"], oc["force"], rtol=1e-9, atol=1e-16)
    sim.close()


@pytest.mark.parametrize("nx", [200, 3001])
def test_line3_fp32(nx):
    """FP32 storage and arithmetic (exactly summing weights) on a resident and a tiled
    line: densities and velocity within 1e-5 of the oracle after 100 steps."""
    n = 3
    sim, orc = _line_pair(n, nx, 0.9, inputs.uniform_chi(n, 1.5), [1.0, 2.0, 1.0], 0.4, 0.02, 1e-5,
                          "fp32", 0, seed=77 + nx)
    sim.step(100)
    assert orc.run(100) == 0
    assert sim.status() == 0
    gm, om = sim.moments(), orc.moments()
    for k in ("rho", "U", "mu", "P"):
        assert np.max(np.abs(gm[k] - om[k])) < 1e-5, k
    sim.close()


def test_line3_equals_one_row_d2q9_on_the_gpu():
    """The library's D1Q3 line and its D2Q9 lattice of one row (y-invariant, whose
    projection D1Q3 is) give the same fields after 200 FP64 steps."""
    n, nx = 3, 96
    chi = np.array([[0.0, 2.6, 1.0], [2.6, 0.0, 0.4], [1.0, 0.4, 0.0]])
    rho, u = inputs.random_state(n, nx, 1, seed=88, amp=0.4, umax=0.03)
    u[1] = 0.0
    kw = dict(m=[3.0, 1.0, 1.0], theta=0.38, kappa=0.03, force=(1e-5, 0.0), precision="fp64")
    a = mclb.Simulation(n, nx, 1, 0.8, chi, lattice="d1q3", **kw)
    b = mclb.Simulation(n, nx, 1, 0.8, chi, kernel=mclb.KERNEL_FUSED, **kw)
    a.init_fields(rho, u)
    b.init_fields(rho, u)
    a.step(200)
    b.step(200)
    ma, mb = a.moments(), b.moments()
    for k in ("rho", "U", "mu", "P"):
        np.testing.assert_allclose(ma[k], mb[k], rtol=1e-11, atol=1e-14, err_msg=k)
    fa, fb = a.get_state(), b.get_state()
    proj = np.stack([fb[:, [0, 2, 4]].sum(1), fb[:, [1, 5, 8]].sum(1),
                     fb[:, [3, 6, 7]].sum(1)], axis=1)[:, :, 0, :]
    np.testing.assert_allclose(fa, proj, rtol=1e-11, atol=1e-15)


def test_line3_many_chunks_and_state_roundtrip():
    """10000 steps (three resident launches: two of 4096 steps and one of 1808) of the
    binary flat interface against the oracle, then get_state / set_state / 100 more steps
    equal to 100 uninterrupted steps, bitwise (FP64)."""
    chi = np.array([[0.0, 2.2], [2.2, 0.0]])
    p = inputs.flat_interface([0.5, 0.5], chi=chi, nx=128, ny=1, kappa=0.0, tau=1 / 0.9)
    p.lattice = "d1q3"
    sim = mclb.Simulation.from_problem(p, precision="fp64")
    orc = Oracle.from_problem(p)
    sim.step(10000)
    orc.run(10000)
    assert sim.status() == 0
    assert _rel(sim.get_state(), orc.f) < 1e-11
    f = sim.get_state()
    other = mclb.Simulation.from_problem(p, precision="fp64")
    other.set_state(f)
    other.step(100)
    sim.step(100)
    assert np.array_equal(other.get_state(), sim.get_state())


def test_line3_fit_equilibrium():
    """The fitted bulk compositions of a stationary D1Q3 flat interface equal the
    oracle's plateaus (Sec. 4, binary chi = 2.2, 1/tau = 0.9)."""
    chi = np.array([[0.0, 2.2], [2.2, 0.0]])
    p = inputs.flat_interface([0.5, 0.5], chi=chi, nx=64, ny=1, kappa=0.0, tau=1 / 0.9)
    p.lattice = "d1q3"
    sim = mclb.Simulation.from_problem(p, precision="fp64")
    sim.step(40000)
    assert sim.status() == 0
    fit = sim.fit_equilibrium(2)
    o = Oracle.from_problem(p)
    o.run(40000)
    m = o.moments()["rho"][:, 0, :]
    phi = m / m.sum(0)
    # the fit's definition on the oracle's fields: bulk sites have every |d_x phi| < 1e-3
    # (central difference), grouped by the richer component
    grad = 0.5 * np.abs(np.roll(phi, -1, axis=1) - np.roll(phi, 1, axis=1))
    bulk = np.all(grad < 1e-3, axis=0)
    rich = phi[0] > 0.5
    want = np.stack([phi[:, bulk & rich].mean(1), phi[:, bulk & ~rich].mean(1)])
    np.testing.assert_allclose(fit, want, rtol=0, atol=1e-9)
    lo, hi = thermo.binodal_binary(2.2)
    assert abs(fit[0, 0] - hi) < 0.015 and abs(fit[1, 0] - lo) < 0.015


def test_line3_batch_mixed_with_d2q9():
    """A batch holding D1Q3 lines of N = 2 and 3 (one longer than the resident limit) and
    D2Q9 lattices: after 5000 steps every line equals its own handle's run bitwise (the
    same kernels) and the oracle's to 1e-11, and the D2Q9 instances are unaffected."""
    probs = []
    for k, (nx, n) in enumerate([(64, 2), (100, 3), (37, 2), (3001, 3), (128, 3)]):
        rho, u = inputs.random_state(n, nx, 1, seed=600 + k, amp=0.2, umax=0.02)
        u[1] = 0.0
        probs.append(inputs.Problem(name=f"line{k}", ncomp=n, nx=nx, ny=1, tau=0.8 + 0.05 * k,
                                    chi=inputs.uniform_chi(n, 1.6 + 0.1 * k), m=np.ones(n),
                                    theta=1 / 3, kappa=0.01, force=(0.0, 0.0), rho=rho, u=u,
                                    lattice="d1q3"))
    for k, (nx, ny, n) in enumerate([(40, 33, 2), (67, 29, 3)]):
        rho, u = inputs.random_state(n, nx, ny, seed=700 + k, amp=0.3, umax=0.02)
        probs.append(inputs.Problem(name=f"grid{k}", ncomp=n, nx=nx, ny=ny, tau=0.9,
                                    chi=inputs.uniform_chi(n, 1.8), m=np.ones(n), theta=1 / 3,
                                    kappa=0.01, force=(0.0, 0.0), rho=rho, u=u))
    b = mclb.Batch(probs, precision="fp64")
    b.init_all()
    b.step(3)           # odd: the lines and the grids now live in their second buffers
    b.init_fields(1, probs[1].rho, probs[1].u)
    b.step(4997)
    rc, per = b.status()
    assert rc == 0 and all(v == 0 for v in per)
    for k, p in enumerate(probs):
        steps = 4997 if k == 1 else 5000
        if p.lattice == "d1q3":
            sim = mclb.Simulation.from_problem(p, precision="fp64")
            sim.step(steps)
            assert np.array_equal(b.get_state(k), sim.get_state()), p.name
            sim.close()
        else:
            o = Oracle.from_problem(p)
            o.run(steps)
            assert _rel(b.get_state(k), o.f) < 1e-11, p.name
    for k in (0, 3):
        o = Oracle.from_problem(probs[k])
        o.run(5000)
        assert _rel(b.get_state(k), o.f) < 1e-11, probs[k].name
    b.close()


def test_line3_batch_binodal_sweep():
    """The paper's binodal experiment on the paper's lattice (Sec. 4: D1Q3, m = (1, 1),
    kappa = 0, 1/tau = 0.7 and 0.9, chi = 2.1 ... 2.5), as one batch of ten 64-site lines
    started at their Flory-Huggins binodals, 40000 FP64 steps (one resident launch per
    4096 steps for all ten lines): both plateaus of every line equal the oracle's to
    1e-9, and their gap to the binodal grows with chi."""
    nx = 64
    x = np.arange(nx)
    inside = (x >= nx // 4) & (x < 3 * nx // 4)
    probs, binodals = [], []
    for itau in (0.7, 0.9):
        for chi_v in (2.1, 2.2, 2.3, 2.4, 2.5):
            lo, hi = thermo.binodal_binary(chi_v)
            phi_a = np.where(inside, hi, lo)
            probs.append(inputs.Problem(
                name=f"binodal_{itau}_{chi_v}", ncomp=2, nx=nx, ny=1, tau=1 / itau,
                chi=np.array([[0.0, chi_v], [chi_v, 0.0]]), m=np.ones(2), theta=1 / 3,
                kappa=0.0, force=(0.0, 0.0), rho=np.stack([phi_a, 1 - phi_a])[:, None, :],
                u=np.zeros((2, 1, nx)), lattice="d1q3"))
            binodals.append(hi)
    b = mclb.Batch(probs, precision="fp64")
    b.init_all()
    assert b.launches_per_step == 1
    b.step(40000)
    rc, per = b.status()
    assert rc == 0 and all(v == 0 for v in per)
    gaps = []
    for k, p in enumerate(probs):
        o = Oracle.from_problem(p)
        o.run(40000)
        mo = o.moments()["rho"]
        want = mo[0] / mo.sum(0)
        mg = b.moments(k)["rho"]
        got = mg[0] / mg.sum(0)
        assert np.max(np.abs(got - want)) < 1e-9, p.name
        gaps.append(got[0, nx // 2] - binodals[k])
    gaps = np.array(gaps).reshape(2, 5)
    assert np.all(np.diff(gaps, axis=1) > 0), gaps
    b.close()


def test_line3_batch_ternary_polymer_near_critical():
    """The paper's ternary polymer (Sec. 4: m = (10, 1, 1), chi_AB = 3, chi_AC = 0.5,
    chi_BC = 0.2, kappa = 0, 1/tau = 0.9) on D1Q3, mean compositions s = 0.02, 0.05, 0.08
    of the way from the printed critical point toward (0.5, 0.5, 0), with the barycentric
    forcing velocity (with and, at s = 0.05, without the Gibbs-Duhem total force): one
    FP64 batch of 128-site lines, 60000 steps.  Every line stays finite and equals the
    oracle's compositions to 1e-9; the separated plateaus lie within 0.04 of the
    Flory-Huggins tie line (the oracle's gap at 60000 steps: 0.010, 0.021, 0.032, growing
    toward depletion as the paper reports)."""
    nx, steps = 128, 60000
    chi = np.zeros((3, 3))
    chi[0, 1] = chi[1, 0] = 3.0
    chi[0, 2] = chi[2, 0] = 0.5
    chi[1, 2] = chi[2, 1] = 0.2
    m = np.array([10.0, 1.0, 1.0])
    cr, end = np.array([0.14, 0.11, 0.75]), np.array([0.5, 0.5, 0.0])
    probs, means = [], []
    for s, ff in ((0.02, 1), (0.05, 1), (0.08, 1), (0.05, 0)):
        pb = cr + s * (end - cr)
        p = inputs.flat_interface(pb, chi=chi, m=m, nx=nx, tau=1 / 0.9, kappa=0.0, amp=0.1,
                                  name=f"ternary_polymer_{s}_{ff}")
        p.lattice, p.forcing_velocity, p.force_form = "d1q3", 1, ff
        probs.append(p)
        means.append(pb)
    b = mclb.Batch(probs, precision="fp64")
    b.init_all()
    b.step(steps)
    rc, per = b.status()
    assert rc == 0 and all(v == 0 for v in per)
    for k, p in enumerate(probs):
        o = Oracle.from_problem(p)
        o.run(steps)
        mo = o.moments()["rho"]
        want = mo / mo.sum(0)
        mg = b.moments(k)["rho"]
        got = mg / mg.sum(0)
        assert np.max(np.abs(got - want)) < 1e-9, p.name
        phi = got[:, 0, :]
        tl = np.array(thermo.tie_line(chi, m, means[k]))
        rich, poor = phi[:, np.argmax(phi[0])], phi[:, np.argmin(phi[0])]
        assert np.abs(rich - tl[np.argmax(tl[:, 0])]).max() < 0.04, p.name
        assert np.abs(poor - tl[np.argmin(tl[:, 0])]).max() < 0.04, p.name
    b.close()
