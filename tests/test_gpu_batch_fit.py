"""GPU: batched simulations and the equilibrium fit, against the FP64 oracle."""
import itertools

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


def _instances():
    probs = []
    shapes = [(40, 33, 2), (67, 29, 3), (32, 32, 2), (91, 45, 3), (16, 70, 2), (50, 50, 3)]
    for k, (nx, ny, n) in enumerate(shapes):
        rho, u = inputs.random_state(n, nx, ny, seed=500 + k, amp=0.3, umax=0.02)
        chi = inputs.uniform_chi(n, 1.8 + 0.15 * k)
        p = inputs.Problem(name=f"b{k}", ncomp=n, nx=nx, ny=ny, tau=0.7 + 0.1 * k, chi=chi,
                           m=np.ones(n), theta=1 / 3, kappa=0.01, force=(0.0, 0.0), rho=rho, u=u)
        probs.append(p)
    return probs


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_batch_matches_oracle(precision, tol):
    """Mixed N and ragged grids; 45 steps = one 32-step graph chunk plus 13 single steps."""
    probs = _instances()
    b = mclb.Batch(probs, precision=precision)
    b.init_all()
    assert b.launches_per_step == 4  # march + ghost refresh per distinct N (2 and 3)
    b.step(45)
    rc, per = b.status()
    assert rc == 0 and all(v == 0 for v in per)
    for k, p in enumerate(probs):
        o = Oracle.from_problem(p)
        o.run(45)
        g = b.get_state(k)
        err = np.max(np.abs(g - o.f)) / np.abs(o.f).max()
        assert err < tol, (k, err)
    b.close()


def test_batch_reinit_at_odd_parity():
    probs = _instances()[:3]
    b = mclb.Batch(probs, precision="fp64")
    b.init_all()
    b.step(3)                      # every instance now lives in the second buffer
    b.init_fields(1, probs[1].rho, probs[1].u)
    b.step(4)
    o = Oracle.from_problem(probs[1])
    o.run(4)
    assert np.max(np.abs(b.get_state(1) - o.f)) < 1e-12 * np.abs(o.f).max()
    o0 = Oracle.from_problem(probs[0])
    o0.run(7)
    assert np.max(np.abs(b.get_state(0) - o0.f)) < 1e-12 * np.abs(o0.f).max()
    b.close()


def test_fit_equilibrium_flat_interface():
    """Binary flat interface (chi = 2.2, kappa = 0) run to stationarity in FP64 on the GPU:
    the fitted bulk compositions equal the oracle's plateau values and sit within 0.015 of
    the Flory-Huggins binodal (Sec. 4)."""
    chi = np.array([[0.0, 2.2], [2.2, 0.0]])
    p = inputs.flat_interface([0.5, 0.5], chi=chi, nx=64, ny=4, kappa=0.0, tau=1 / 0.9)
    sim = mclb.Simulation.from_problem(p, precision="fp64", kernel=mclb.KERNEL_FUSED)
    sim.step(40000)
    assert sim.status() == 0
    fit = sim.fit_equilibrium(2)        # phase 0 richest in component 0
    o = Oracle.from_problem(p)
    o.run(40000)
    m = o.moments()
    phi = m["rho"][0] / m["rho"].sum(0)
    assert abs(fit[0, 0] - phi.max()) < 1e-3 and abs(fit[1, 0] - phi.min()) < 1e-3
    lo, hi = thermo.binodal_binary(2.2)
    assert abs(fit[0, 0] - hi) < 0.015 and abs(fit[1, 0] - lo) < 0.015
    np.testing.assert_allclose(fit.sum(1), 1.0, atol=1e-12)


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-6), ("bf16", 2e-4)])
def test_batch_matches_single_handles(precision, tol):
    """The batched march runs the single-lattice kernel's per-site arithmetic on another
    tiling (one common segment height, instances packed into one launch, parameters read
    from shared memory); after the same steps every instance's densities agree with those
    of its own handle to the rounding of the storage format (the two kernels are compiled
    separately, so their FMA contractions may differ in the last bit)."""
    probs = _instances()
    b = mclb.Batch(probs, precision=precision)
    b.init_all()
    b.step(37)
    rc, per = b.status()
    assert rc == 0 and all(v == 0 for v in per)
    for k, p in enumerate(probs):
        sim = mclb.Simulation.from_problem(p, precision=precision, kernel=mclb.KERNEL_FUSED)
        sim.step(37)
        assert sim.status() == 0
        a, c = sim.moments(mu=False, P=False)["rho"], b.moments(k)["rho"]
        assert np.max(np.abs(a - c)) <= tol * np.abs(a).max(), k
        sim.close()
    b.close()


@pytest.fixture(scope="module")
def ternary_flat():
    """The paper's ternary chi set (chi_AB = 3, chi_AC = 0.5, chi_BC = 0.2, 1/tau = 0.9,
    Sec. 4) started as two slabs at the ends of the Flory-Huggins tie line through
    (0.4, 0.4, 0.2), run by the oracle to stationarity; returns the problem and the
    oracle's plateau compositions (means over 16 columns in the middle of each slab)."""
    chi = np.zeros((3, 3))
    chi[0, 1] = chi[1, 0] = 3.0
    chi[0, 2] = chi[2, 0] = 0.5
    chi[1, 2] = chi[2, 1] = 0.2
    q1, q2 = thermo.tie_line(chi, np.ones(3), [0.4, 0.4, 0.2])
    hi, lo = (q1, q2) if q1[0] > q2[0] else (q2, q1)
    nx, ny = 128, 4
    x = np.arange(nx)
    inside = (x >= nx // 4) & (x < 3 * nx // 4)
    phi = np.where(inside[None, :], np.asarray(hi)[:, None], np.asarray(lo)[:, None])
    rho = np.repeat(phi[:, None, :], ny, axis=1)
    p = inputs.Problem(name="ternary_slabs", ncomp=3, nx=nx, ny=ny, tau=1 / 0.9, chi=chi,
                       m=np.ones(3), theta=1 / 3, kappa=0.0, force=(0.0, 0.0), rho=rho,
                       u=np.zeros((2, ny, nx)))
    o = Oracle.from_problem(p)
    o.run(20000)
    m = o.moments()
    ph = m["rho"] / m["rho"].sum(0)
    a = ph[:, :, nx // 2 - 8:nx // 2 + 8].mean(axis=(1, 2))
    b = np.concatenate([ph[:, :, :8], ph[:, :, -8:]], axis=2).mean(axis=(1, 2))
    return p, a, b, hi, lo


@pytest.mark.parametrize("precision", ["fp32", "bf16", "fp16"])
def test_fit_equilibrium_ternary_slabs(precision, ternary_flat):
    """Two coexisting ternary phases (Sec. 4): after 20000 steps the fitted bulk
    compositions equal the oracle's plateaus to 1e-3 in every storage format, and lie
    within 0.05 of the Flory-Huggins tie line they started from."""
    p, a, b, hi, lo = ternary_flat
    sim = mclb.Simulation.from_problem(p, precision=precision, kernel=mclb.KERNEL_FUSED)
    sim.step(20000)
    assert sim.status() == 0
    fit = sim.fit_equilibrium(2)        # phase 0 seeded at the site richest in component 0
    assert np.max(np.abs(fit[0] - a)) < 1e-3, (fit, a)
    assert np.max(np.abs(fit[1] - b)) < 1e-3, (fit, b)
    assert np.max(np.abs(fit[0] - hi)) < 0.05 and np.max(np.abs(fit[1] - lo)) < 0.05


def test_polymer_binary_matches_oracle():
    """The paper's polymer binary (m = (10, 1), chi = 0.94, kappa = 0, 1/tau = 0.9,
    Sec. 4), started as two slabs at the Flory-Huggins binodal: the polymer's logarithmic
    terms (theta/m - 1/3 != 0) run through the floored-log path.  After 20000 steps the
    FP32 volume-fraction profile equals the oracle's to 1e-3 at every site, and the BF16
    fit of both phases equals the FP32 one to 1e-3."""
    chi = np.array([[0.0, 0.94], [0.94, 0.0]])
    m = np.array([10.0, 1.0])
    lo, hi = thermo.binodal_binary(0.94, 10.0, 1.0)
    nx, ny = 128, 4
    x = np.arange(nx)
    phi_a = np.where((x >= nx // 4) & (x < 3 * nx // 4), hi, lo)
    rho = np.stack([np.tile(phi_a, (ny, 1)), np.tile(1 - phi_a, (ny, 1))])
    p = inputs.Problem(name="polymer_slabs", ncomp=2, nx=nx, ny=ny, tau=1 / 0.9, chi=chi, m=m,
                       theta=1 / 3, kappa=0.0, force=(0.0, 0.0), rho=rho, u=np.zeros((2, ny, nx)))
    o = Oracle.from_problem(p)
    o.run(20000)
    mo = o.moments()
    phi_o = mo["rho"][0] / mo["rho"].sum(0)
    fits = {}
    for precision in ("fp32", "bf16"):
        sim = mclb.Simulation.from_problem(p, precision=precision, kernel=mclb.KERNEL_FUSED)
        sim.step(20000)
        assert sim.status() == 0
        if precision == "fp32":
            g = sim.moments(mu=False, P=False)
            assert np.max(np.abs(g["rho"][0] / g["rho"].sum(0) - phi_o)) < 1e-3
        fits[precision] = sim.fit_equilibrium(2)
        sim.close()
    assert np.max(np.abs(fits["bf16"] - fits["fp32"])) < 1e-3


def test_batch_binodal_sweep_matches_oracle():
    """The paper's monomer binodal experiment (Sec. 4: m = (1, 1), kappa = 0, 1/tau = 0.7
    and 0.9) as one batch of ten flat interfaces, chi = 2.1 ... 2.5, each started as two
    slabs at its Flory-Huggins binodal.  After 40000 FP32 steps both plateaus of every
    instance equal the oracle's to 1e-3; their distance from the binodal grows with chi
    (the sharp-interface lattice gap, which the oracle shows vanishing as kappa widens the
    interface)."""
    nx, ny = 64, 2
    x = np.arange(nx)
    inside = (x >= nx // 4) & (x < 3 * nx // 4)
    probs, binodals = [], []
    for itau in (0.7, 0.9):
        for chi_v in (2.1, 2.2, 2.3, 2.4, 2.5):
            lo, hi = thermo.binodal_binary(chi_v)
            phi_a = np.where(inside, hi, lo)
            rho = np.stack([np.tile(phi_a, (ny, 1)), np.tile(1 - phi_a, (ny, 1))])
            chi = np.array([[0.0, chi_v], [chi_v, 0.0]])
            probs.append(inputs.Problem(name=f"binodal_{itau}_{chi_v}", ncomp=2, nx=nx, ny=ny,
                                        tau=1 / itau, chi=chi, m=np.ones(2), theta=1 / 3,
                                        kappa=0.0, force=(0.0, 0.0), rho=rho,
                                        u=np.zeros((2, ny, nx))))
            binodals.append(hi)
    b = mclb.Batch(probs, precision="fp32")
    b.init_all()
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
        for c in (nx // 2, 0):
            assert abs(got[0, c] - want[0, c]) < 1e-3, (p.name, c, got[0, c], want[0, c])
        gaps.append(got[0, nx // 2] - binodals[k])
    gaps = np.array(gaps).reshape(2, 5)
    assert np.all(np.diff(gaps, axis=1) > 0), gaps
    b.close()


def test_batch_ternary_sweep_matches_oracle():
    """The paper's ternary monomer sweep (Sec. 4: chi_AB = 3, chi_AC = 0.5, chi_BC = 0.2,
    1/tau = 0.9): mean compositions on the line from the printed critical point
    (0.32, 0.32, 0.36) toward (0.5, 0.5, 0), at 0.1, 0.4 and 0.7 of the way, each started
    as two slabs at the ends of its Flory-Huggins tie line and run as one batch.  After
    20000 FP32 steps both plateaus of every instance equal the oracle's to 1e-3, and their
    distance from the tie line grows along the line (the sharp-interface gap)."""
    chi = np.zeros((3, 3))
    chi[0, 1] = chi[1, 0] = 3.0
    chi[0, 2] = chi[2, 0] = 0.5
    chi[1, 2] = chi[2, 1] = 0.2
    nx, ny = 128, 2
    x = np.arange(nx)
    inside = (x >= nx // 4) & (x < 3 * nx // 4)
    pc, end = np.array([0.32, 0.32, 0.36]), np.array([0.5, 0.5, 0.0])
    probs, ties = [], []
    for s in (0.1, 0.4, 0.7):
        q1, q2 = thermo.tie_line(chi, np.ones(3), pc + s * (end - pc))
        hi, lo = (q1, q2) if q1[0] > q2[0] else (q2, q1)
        phi = np.where(inside[None, :], np.asarray(hi)[:, None], np.asarray(lo)[:, None])
        probs.append(inputs.Problem(name=f"ternary_sweep_{s}", ncomp=3, nx=nx, ny=ny, tau=1 / 0.9,
                                    chi=chi, m=np.ones(3), theta=1 / 3, kappa=0.0,
                                    force=(0.0, 0.0), rho=np.repeat(phi[:, None, :], ny, axis=1),
                                    u=np.zeros((2, ny, nx))))
        ties.append((np.asarray(hi), np.asarray(lo)))
    b = mclb.Batch(probs, precision="fp32")
    b.init_all()
    b.step(20000)
    rc, per = b.status()
    assert rc == 0 and all(v == 0 for v in per)
    gaps = []
    for k, p in enumerate(probs):
        o = Oracle.from_problem(p)
        o.run(20000)
        mo = o.moments()["rho"]
        want = mo / mo.sum(0)
        mg = b.moments(k)["rho"]
        got = mg / mg.sum(0)
        for c in (nx // 2, 0):
            assert np.max(np.abs(got[:, 0, c] - want[:, 0, c])) < 1e-3, (p.name, c)
        gaps.append(np.max(np.abs(got[:, 0, nx // 2] - ties[k][0])))
    assert gaps[0] < gaps[1] < gaps[2], gaps
    b.close()


def _fit_by_definition(rho, nphase, lattice="d2q9"):
    """mclb_fit_equilibrium written out in numpy: compositions; bulk sites where every
    component's lattice gradient 3 sum_i w_i v_i phi(x + v_i) (D2Q9, or D3Q19 for fields
    (N, nz, ny, nx)) is below 1e-3 in magnitude; k-means seeded at the bulk site richest
    in component c (first on ties), nearest centroid by squared distance (lower phase on
    ties), until the centroids stop moving."""
    phi = rho / rho.sum(0)
    if lattice == "d3q19":
        vel = [c for c in itertools.product((-1, 0, 1), repeat=3) if 0 < sum(x * x for x in c) <= 2]
        g2 = 0.0
        for d in range(3):
            g = sum(3 * (1 / 18 if sum(x * x for x in c) == 1 else 1 / 36) * c[d]
                    * np.roll(phi, (-c[2], -c[1], -c[0]), axis=(1, 2, 3)) for c in vel)
            g2 = g2 + g * g
        bulk = np.all(g2 < 1e-6, axis=0).ravel()
    else:
        cx = [0, 1, 0, -1, 0, 1, -1, -1, 1]
        cy = [0, 0, 1, 0, -1, 1, 1, -1, -1]
        w = [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4
        gx = sum(3 * w[i] * cx[i] * np.roll(phi, (-cy[i], -cx[i]), axis=(1, 2)) for i in range(9))
        gy = sum(3 * w[i] * cy[i] * np.roll(phi, (-cy[i], -cx[i]), axis=(1, 2)) for i in range(9))
        bulk = np.all(gx * gx + gy * gy < 1e-6, axis=0).ravel()
    pts = phi.reshape(phi.shape[0], -1)[:, bulk].T
    cen = np.stack([pts[np.argmax(pts[:, c])] for c in range(nphase)])
    for _ in range(100):
        d = ((pts[:, None, :] - cen[None]) ** 2).sum(-1)
        lab = np.argmin(d, axis=1)
        new = np.stack([pts[lab == c].mean(0) if np.any(lab == c) else cen[c]
                        for c in range(nphase)])
        if np.array_equal(new, cen):
            break
        cen = new
    return cen


@pytest.mark.parametrize("nphase", [2, 3])
def test_fit_equilibrium_matches_its_definition(nphase):
    """The device k-means of mclb_fit_equilibrium against the same fit written out in
    numpy on the handle's own densities (FP64 state of the ternary droplet workload after
    1500 steps): equal to 1e-12 for two and three phases."""
    p = inputs.ternary_droplets(256, 192)
    sim = mclb.Simulation.from_problem(p, precision="fp64")
    sim.step(1500)
    assert sim.status() == 0
    got = sim.fit_equilibrium(nphase)
    want = _fit_by_definition(sim.moments(U=False, mu=False, P=False)["rho"], nphase)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)
    sim.close()


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_every_autotuner_candidate_matches_single_handles(precision):
    """The autotuner times every partition (wide and narrow strips, segment heights for 2,
    4, 8 and 16 waves) and keeps the fastest; each one must compute the same step.  With
    each candidate forced in turn, 23 steps of the mixed batch equal the instances' own
    handles to the storage format's rounding (FP32 2e-5, BF16 3e-3 of the density scale);
    the tuner's own pick is reported as a valid candidate."""
    probs = _instances()
    tol = {"fp32": 2e-5, "bf16": 3e-3}[precision]
    want = []
    for p in probs:
        sim = mclb.Simulation.from_problem(p, precision=precision, kernel=mclb.KERNEL_FUSED)
        sim.step(23)
        assert sim.status() == 0
        want.append(sim.moments(U=False, mu=False, P=False)["rho"])
        sim.close()
    b = mclb.Batch(probs, precision=precision)
    b.init_all()
    b.step(1)
    for nar, w in b.tuning():
        assert w in (2, 4, 8, 16)
    b.close()
    switched = 0
    for narrow in (False, True):
        for waves in (2, 4, 8, 16):
            b = mclb.Batch(probs, precision=precision)
            b.init_all()
            switched += b.test_force_partition(narrow, waves)
            b.step(23)
            rc, per = b.status()
            assert rc == 0 and all(v == 0 for v in per)
            for k in range(len(probs)):
                got = b.moments(k)["rho"]
                assert np.max(np.abs(got - want[k])) <= tol * np.abs(want[k]).max(), (narrow, waves, k)
            b.close()
    assert switched >= 2 * 4          # every candidate of at least one group, both shapes
