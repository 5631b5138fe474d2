"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances (stated per field, max-norm of the difference):
  * FP64 storage and arithmetic: 1e-12 relative to the field's max-norm, up to 50 steps
    on every case and for 1000 steps on the 64 x 64 binary (still in its linear regime);
  * FP32: 1e-5 absolute (lattice units; densities are O(1/N), velocities O(1e-3)) on each
    of rho, U, mu and P after 100 steps on the ternary 256 x 256 workload and on two
    phase-separated states at its parameters (droplets, and the polymer slab);
  * one step at the full 2048 x 2048 (N = 5) and 8192 x 2048 (N = 3) sizes from the same
    state: 2e-6 relative to the largest population (one FP32 step from identical input).
Every case runs both schedules (fused single pass and staged three launches).
"""
import numpy as np
import pytest

import paper_0704_3444_gb300 as mclb
from oracle import Oracle
from paper_0704_3444_gb300 import inputs

pytestmark = pytest.mark.gpu

KERNELS = [mclb.KERNEL_FUSED, mclb.KERNEL_STAGED]


@pytest.fixture(scope="module", autouse=True)
def built():
    mclb.build()
    mclb.load()


def _chi(n, seed):
    r = inputs.uniform(seed, n * n, 3).reshape(n, n)
    c = 2.0 + (r + r.T)
    np.fill_diagonal(c, 0.0)
    return c


def _pair(n, nx, ny, tau, chi, m=None, theta=1 / 3, kappa=0.0, force=(0.0, 0.0),
          precision="fp64", kernel=mclb.KERNEL_FUSED, rho=None, u=None, fv=0):
    sim = mclb.Simulation(n, nx, ny, tau, chi, m, theta, kappa, force, precision, kernel,
                          forcing_velocity=fv)
    orc = Oracle(n, nx, ny, tau, chi, m, theta, kappa, force, forcing_velocity=fv)
    sim.init_fields(rho, u)
    orc.init(rho, u)
    return sim, orc


def _rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


CASES = [
    # (nx, ny, N, steps, tau, theta, kappa, m, force)
    (4, 4, 2, 20, 1.0, 1 / 3, 0.0, None, (0.0, 0.0)),
    (5, 3, 3, 20, 0.8, 0.4, 0.05, [1.0, 3.0, 10.0], (3e-4, -1e-4)),
    (7, 6, 1, 20, 0.9, 1 / 3, 0.02, None, (1e-4, 0.0)),
    (1, 9, 2, 20, 0.7, 0.45, 0.01, None, (0.0, 2e-4)),
    (130, 37, 4, 30, 1.0, 1 / 3, 0.01, None, (0.0, 0.0)),
    (300, 170, 3, 25, 0.8, 0.5, 0.01, [2.0, 1.0, 1.0], (1e-5, 1e-5)),
    (40, 33, 5, 15, 1.2, 1 / 3, 0.01, None, (0.0, 0.0)),
    (40, 33, 6, 10, 0.9, 0.4, 0.01, None, (0.0, 0.0)),
    (33, 40, 7, 10, 1.0, 1 / 3, 0.02, None, (0.0, 0.0)),
    (64, 20, 8, 10, 1.1, 1 / 3, 0.01, [1, 1, 2, 1, 1, 3, 1, 1], (0.0, 0.0)),
    # degenerate and ragged shapes: one and two rows (every row its own vertical
    # neighbour), fewer columns than ghost columns, one column past a 112-column strip
    (9, 1, 2, 20, 0.9, 1 / 3, 0.01, None, (1e-4, 0.0)),
    (6, 2, 3, 20, 1.0, 0.4, 0.02, None, (0.0, 1e-4)),
    (2, 7, 2, 20, 0.8, 1 / 3, 0.01, None, (0.0, 0.0)),
    (113, 5, 2, 15, 1.0, 1 / 3, 0.01, None, (0.0, 0.0)),
]


@pytest.mark.parametrize("fv", [0, 1], ids=["component_u", "barycentric_u"])
@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}x{c[1]}N{c[2]}")
def test_fp64_state_parity(case, kernel, fv):
    nx, ny, n, steps, tau, theta, kappa, m, force = case
    rho, u = inputs.random_state(n, nx, ny, seed=1000 + nx * ny + n, amp=0.3, umax=0.03)
    sim, orc = _pair(n, nx, ny, tau, _chi(n, n + nx), m, theta, kappa, force, "fp64", kernel,
                     rho, u, fv=fv)
    np.testing.assert_allclose(sim.get_state(), orc.f, rtol=0, atol=1e-15 * np.abs(orc.f).max())
    sim.step(steps)
    orc.run(steps)
    assert sim.status() == 0
    assert _rel(sim.get_state(), orc.f) < 1e-12
    gm, om = sim.moments(), orc.moments()
    for k in ("rho", "U", "mu"):
        assert _rel(gm[k], om[k]) < 1e-11, k
    # P: compare against the scale of its gradient part (its isotropic bulk part is ~0)
    assert np.max(np.abs(gm["P"] - om["P"])) < 1e-12 * max(1.0, np.abs(om["P"]).max())
    sim.close()


@pytest.mark.parametrize("precision,tol,fv", [("fp32", 1e-5, 0), ("bf16", 2e-3, 0),
                                               ("fp16", 2e-3, 0), ("fp32", 1e-5, 1),
                                               ("bf16", 2e-3, 1)])
@pytest.mark.parametrize("n", range(1, 9))
def test_fused_every_n(n, precision, tol, fv):
    """The single-pass kernel for every component count in FP32 and the 16-bit formats:
    each N compiles its own geometry (4- or 2-warp strips, two or three CTAs per SM, one
    or two box-store staging buffers), so each runs 12 steps on a 130 x 37 grid (two
    112-column or three 56-column strips, ragged in both directions) with kappa, m != 1,
    theta != 1/3 and a body force on; densities within tol (relative to their max: FP32
    rounding, or one 16-bit rounding of the deviations) of the oracle's, and component
    masses kept to 1e-6."""
    nx, ny = 130, 37
    rho, u = inputs.random_state(n, nx, ny, seed=4000 + n, amp=0.3, umax=0.03)
    m = [1.0 + (k % 3) for k in range(n)]
    sim, orc = _pair(n, nx, ny, 0.9, _chi(n, 77 + n), m, 0.4, 0.02, (1e-5, -2e-5), precision,
                     mclb.KERNEL_FUSED, rho, u, fv=fv)
    m0 = sim.conservation()["mass"]
    sim.step(12)
    orc.run(12)
    assert sim.status() == 0
    got, want = sim.moments(mu=False, P=False)["rho"], orc.moments()["rho"]
    assert _rel(got, want) < tol
    np.testing.assert_allclose(sim.conservation()["mass"], m0, rtol=1e-6)
    sim.close()


@pytest.mark.parametrize("kernel", KERNELS)
def test_binary_64_full_horizon_fp64(kernel):
    """The 64 x 64 binary workload (chi = 2.2, kappa = 0.01, tau = 1), all 1000 steps in FP64."""
    p = inputs.binary_noise()
    sim = mclb.Simulation.from_problem(p, precision="fp64", kernel=kernel)
    orc = Oracle.from_problem(p)
    sim.step(1000)
    orc.run(1000)
    assert sim.status() == 0
    assert _rel(sim.get_state(), orc.f) < 1e-11
    c = sim.conservation()
    mass0 = p.rho.reshape(2, -1).sum(1)
    assert np.max(np.abs(c["mass"] / mass0 - 1)) < 1e-13


def _four_fields_fp32(p, kernel, steps, tol=1e-5, fv=0):
    """rho, U, mu and P of the FP32 path after `steps` steps, each within `tol` (absolute
    max-norm, lattice units) of the FP64 oracle's; returns the errors."""
    p.forcing_velocity = fv
    sim = mclb.Simulation.from_problem(p, precision="fp32", kernel=kernel)
    orc = Oracle.from_problem(p)
    sim.step(steps)
    orc.run(steps)
    assert sim.status() == 0
    gm, om = sim.moments(), orc.moments()
    sim.close()
    err = {k: float(np.max(np.abs(gm[k] - om[k]))) for k in ("rho", "U", "mu", "P")}
    for k, e in err.items():
        assert e < tol, (k, err)
    return err


@pytest.mark.parametrize("kernel", KERNELS)
def test_ternary_256_fp32(kernel):
    """Ternary 256 x 256 (chi = 2.4, tau = 0.8, kappa = 0.01) in FP32: rho, U, mu and P
    within 1e-5 of the oracle after 100 steps."""
    _four_fields_fp32(inputs.ternary_gauss(steps=100), kernel, 100)


@pytest.mark.parametrize("fv", [0, 1], ids=["component_u", "barycentric_u"])
@pytest.mark.parametrize("kernel", KERNELS)
def test_ternary_droplets_fp32(kernel, fv):
    """The ternary workload's parameters on a phase-separated state (A-rich discs in a
    B-rich matrix, interfaces everywhere): rho, U, mu and P within 1e-5 of the oracle
    after 100 FP32 steps, for both readings of the forcing velocity."""
    _four_fields_fp32(inputs.ternary_droplets(), kernel, 100, fv=fv)


@pytest.mark.parametrize("kernel", KERNELS)
def test_slab_phase_separating_fp32(kernel):
    """A phase-separating case in FP32: the polymer/solvent | non-solvent slab (paper's
    ternary chi set, sharp initial contacts) on 256 x 64; rho, U, mu and P within 1e-5 of
    the oracle after 100 steps (the FP32 tolerance's horizon) and rho after 300."""
    _four_fields_fp32(inputs.slab(256, 64, steps=100), kernel, 100)
    p = inputs.slab(256, 64, steps=300)
    sim = mclb.Simulation.from_problem(p, precision="fp32", kernel=kernel)
    orc = Oracle.from_problem(p)
    sim.step(300)
    orc.run(300)
    assert sim.status() == 0
    assert np.max(np.abs(sim.moments(U=False, mu=False, P=False)["rho"]
                         - orc.moments()["rho"])) < 1e-5
    sim.close()


def _floored_state(nx, ny, value):
    """Three components, the third at `value` times the local total density on two sites
    and at 1e-3 around them (the oracle's log-floor pins use the same layout)."""
    rho, u = inputs.random_state(3, nx, ny, seed=61, amp=0.3, umax=0.02)
    tot = rho.sum(0)
    rho[2, 2:5, 3:7] = 1e-3 * tot[2:5, 3:7]
    rho[2, 3, 4:6] = value * tot[3, 4:6]
    return rho, u


@pytest.mark.parametrize("fv", [0, 1])
@pytest.mark.parametrize("value", [0.0, 1e-14], ids=["zero", "1e-14"])
@pytest.mark.parametrize("kernel", KERNELS)
def test_log_floor_parity_fp64(kernel, value, fv):
    """Eq. definef's logarithm where the floor max(rho^s, 1e-12 rho) binds: theta/m^s !=
    1/3, one component exactly 0 (or 1e-14 rho) on two sites, kappa on; FP64 GPU within
    1e-12 of the oracle after 10 steps, for both schedules and both forcing readings."""
    nx, ny = 10, 8
    rho, u = _floored_state(nx, ny, value)
    chi = _chi(3, 62)
    sim, orc = _pair(3, nx, ny, 0.9, chi, [1.0, 2.0, 1.0], 0.45, 0.02, (0.0, 0.0), "fp64",
                     kernel, rho, u, fv=fv)
    sim.step(10)
    orc.run(10)
    assert sim.status() == 0
    assert np.all(np.isfinite(orc.f))
    assert _rel(sim.get_state(), orc.f) < 1e-12
    sim.close()


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-5), ("bf16", 2e-3)])
def test_log_floor_parity_reduced(precision, tol):
    """The same floored state on a multi-strip grid (130 x 37) through the single-pass
    kernel in FP32 and BF16: densities within the format's tolerance after 10 steps."""
    nx, ny = 130, 37
    rho, u = _floored_state(nx, ny, 0.0)
    chi = _chi(3, 62)
    sim, orc = _pair(3, nx, ny, 0.9, chi, [1.0, 2.0, 1.0], 0.45, 0.02, (0.0, 0.0), precision,
                     mclb.KERNEL_FUSED, rho, u)
    sim.step(10)
    orc.run(10)
    assert sim.status() == 0
    got, want = sim.moments(mu=False, P=False)["rho"], orc.moments()["rho"]
    assert _rel(got, want) < tol
    sim.close()


def test_fused_matches_staged_fp32():
    p = inputs.ternary_gauss(128, 96, steps=50)
    a = mclb.Simulation.from_problem(p, precision="fp32", kernel=mclb.KERNEL_FUSED)
    b = mclb.Simulation.from_problem(p, precision="fp32", kernel=mclb.KERNEL_STAGED)
    assert a.launches_per_step == 2 and b.launches_per_step == 3
    a.step(50)
    b.step(50)
    assert np.max(np.abs(a.get_state() - b.get_state())) < 1e-6


@pytest.mark.parametrize("kernel", KERNELS)
def test_momentum_balance_gpu(kernel):
    """Total momentum changes by exactly the summed force (Eq. ff2), FP64."""
    n, nx, ny = 3, 50, 30
    rho, u = inputs.random_state(n, nx, ny, seed=77, amp=0.3, umax=0.02)
    sim = mclb.Simulation(n, nx, ny, 0.7, _chi(n, 9), [1.0, 2.0, 5.0], 0.4, 0.03, (1e-4, -2e-4),
                          "fp64", kernel)
    sim.init_fields(rho, u)
    for _ in range(3):
        c0 = sim.conservation()
        sim.step(1)
        c1 = sim.conservation()
        np.testing.assert_allclose(c1["mom"] - c0["mom"], c0["force"], rtol=1e-9, atol=1e-14)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16", "fp16"])
def test_state_roundtrip(precision):
    n, nx, ny = 3, 37, 11
    rho, u = inputs.random_state(n, nx, ny, seed=5, amp=0.2, umax=0.02)
    orc = Oracle(n, nx, ny, 1.0, _chi(n, 1))
    orc.init(rho, u)
    sim = mclb.Simulation(n, nx, ny, 1.0, _chi(n, 1), precision=precision)
    sim.set_state(orc.f)
    g = sim.get_state()
    if precision == "fp64":
        assert np.array_equal(g, orc.f)
    elif precision == "fp32":
        assert np.array_equal(g, orc.f.astype(np.float32).astype(np.float64))
    else:
        tol = 2e-3 if precision == "bf16" else 2e-4
        assert np.max(np.abs(g - orc.f)) < tol * np.abs(orc.f).max()


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16"])
def test_invalid_host_input_rejected(precision):
    """init_fields and set_state check their host data on the device after the upload:
    a non-finite density, a non-positive total density, a non-finite velocity or a
    non-finite population is rejected with EINVAL naming the first failing site or value,
    and the handle's state is left as it was."""
    n, nx, ny = 3, 40, 30
    rho, u = inputs.random_state(n, nx, ny, seed=91, amp=0.2, umax=0.02)
    sim = mclb.Simulation(n, nx, ny, 0.9, inputs.uniform_chi(n, 1.5), precision=precision)
    sim.init_fields(rho, u)
    sim.step(3)
    before = sim.get_state()
    cases = []
    r = rho.copy(); r[1, 7, 11] = np.nan; r[0, 20, 5] = np.inf
    cases.append((r, u, "rho not finite at site %d" % (7 * nx + 11)))
    r = rho.copy(); r[:, 12, 30] = -0.1
    cases.append((r, u, "total density <= 0 at site %d" % (12 * nx + 30)))
    v = u.copy(); v[1, 25, 2] = np.nan
    cases.append((rho, v, "u not finite at site %d" % (25 * nx + 2)))
    for r, v, msg in cases:
        with pytest.raises(mclb.MclbError) as ei:
            sim.init_fields(r, v)
        assert mclb.STATUS[ei.value.code] == "EINVAL" and msg in str(ei.value)
        assert np.array_equal(sim.get_state(), before)
    f = before.copy()
    f[2, 4, 9, 13] = np.nan
    with pytest.raises(mclb.MclbError) as ei:
        sim.set_state(f)
    assert mclb.STATUS[ei.value.code] == "EINVAL"
    assert "value %d" % np.ravel_multi_index((2, 4, 9, 13), f.shape) in str(ei.value)
    assert np.array_equal(sim.get_state(), before)
    assert sim.status() == 0
    sim.close()


def test_nonpositive_density_sets_status():
    """A host-made bad input (negative total density at one site, passed through the
    unvalidated device entry point) is reported as ENONFINITE after the step."""
    torch = pytest.importorskip("torch")
    n, nx, ny = 2, 16, 16
    rho = np.full((n, ny, nx), 0.5)
    rho[:, 3, 4] = -0.5
    sim = mclb.Simulation(n, nx, ny, 1.0, np.array([[0.0, 2.0], [2.0, 0.0]]))
    t = torch.tensor(rho, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    sim.init_fields_device(t)
    sim.step(2)
    assert sim.status() == -4


@pytest.mark.parametrize("name,make", [
    ("n5_2048x2048", lambda: inputs.multi_uniform(steps=1)),
    ("slab_8192x2048", lambda: inputs.slab(steps=1)),
])
def test_full_size_single_step_fp32(name, make):
    """At the full benchmark sizes and in the fused launch configuration the benchmark
    times: advance 10 steps on the GPU, then one more step on both sides from the
    GPU's own state, compared at every population."""
    p = make()
    sim = mclb.Simulation.from_problem(p, precision="fp32", kernel=mclb.KERNEL_FUSED)
    sim.step(10)
    f0 = sim.get_state()
    orc = Oracle(p.ncomp, p.nx, p.ny, p.tau, p.chi, p.m, p.theta, p.kappa, p.force)
    orc.set_state(f0)
    del f0
    orc.run(1)
    sim.step(1)
    assert sim.status() == 0
    g = sim.get_state()
    err = np.max(np.abs(g - orc.f)) / np.abs(orc.f).max()
    assert err < 2e-6, err


@pytest.mark.parametrize("name,make", [
    ("n5_2048x2048", lambda: inputs.multi_uniform(steps=1)),
    ("slab_8192x2048", lambda: inputs.slab(steps=1)),
])
def test_full_size_single_step_bf16(name, make):
    """BF16-shifted storage at the full sizes, in the launch configuration the benchmark
    times: 10 steps on the GPU, then one more on both sides from the GPU's own state.
    The post-collision mass of every site and component (the stored populations taken
    back to the site that wrote them) is the oracle's to FP32 rounding, because the
    reference density makes each site's stored mass exact; every population is within
    two BF16 roundings of the largest deviation from w_i rho^s."""
    p = make()
    sim = mclb.Simulation.from_problem(p, precision="bf16", kernel=mclb.KERNEL_FUSED)
    sim.step(10)
    f0 = sim.get_state()
    orc = Oracle(p.ncomp, p.nx, p.ny, p.tau, p.chi, p.m, p.theta, p.kappa, p.force)
    orc.set_state(f0)
    del f0
    orc.run(1)
    sim.step(1)
    assert sim.status() == 0
    g = sim.get_state()
    o = orc.f
    vx = [0, 1, 0, -1, 0, 1, -1, -1, 1]
    vy = [0, 0, 1, 0, -1, 1, 1, -1, -1]
    mass_g = sum(np.roll(g[:, i], (-vy[i], -vx[i]), axis=(1, 2)) for i in range(9))
    mass_o = sum(np.roll(o[:, i], (-vy[i], -vx[i]), axis=(1, 2)) for i in range(9))
    assert np.max(np.abs(mass_g - mass_o)) < 2e-6 * np.abs(mass_o).max()
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)[None, :, None, None]
    dev = np.abs(o - w * o.sum(axis=1, keepdims=True)).max()
    assert np.max(np.abs(g - o)) < 2.0 ** -7 * dev + 2e-6 * np.abs(o).max()


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-5), ("bf16", 2e-3)])
def test_maximum_size_by_periodic_tiling(precision, tol):
    """A lattice whose buffers exceed 2^32 elements (12288 x 8192, N = 5: 4.5e9 values and
    line-plane strides above 4 GB per buffer) holding a field that repeats a 96 x 64 tile:
    the periodic lattice then evolves as the tile does, so after 5 steps every one of the
    16384 tiles equals the oracle's run on the tile alone (to the format's tolerance)."""
    n, tw, th, reps_x, reps_y = 5, 96, 64, 128, 128
    rho_t, u_t = inputs.random_state(n, tw, th, seed=4242, amp=0.3, umax=0.02)
    chi = _chi(n, 77)
    orc = Oracle(n, tw, th, 0.9, chi, None, 1 / 3, 0.01, (0.0, 0.0))
    orc.init(rho_t, u_t)
    orc.run(5)
    want = orc.moments()["rho"]
    nx, ny = tw * reps_x, th * reps_y
    sim = mclb.Simulation(n, nx, ny, 0.9, chi, None, 1 / 3, 0.01, (0.0, 0.0), precision,
                          mclb.KERNEL_FUSED)
    sim.init_fields(np.tile(rho_t, (1, reps_y, reps_x)), np.tile(u_t, (1, reps_y, reps_x)))
    sim.step(5)
    assert sim.status() == 0
    got = sim.moments(U=False, mu=False, P=False)["rho"]
    sim.close()
    tiles = got.reshape(n, reps_y, th, reps_x, tw)
    err = np.max(np.abs(tiles - want[:, None, :, None, :]))
    assert err < tol * np.abs(want).max(), err


def test_n5_recipe_long_horizon_per_field():
    """The N = 5 workload's recipe (random symmetric chi in [0.8, 1.5] x critical, tau = 1,
    kappa = 0.01, noise 0.01) on 256 x 256, against the FP64 oracle per field.  FP64 after
    500 steps: each of rho, U, mu, P within 10x the oracle's own sensitivity (its
    divergence from a start perturbed by 2^-52 relative, floored at 8 units of roundoff of
    the field's scale).  FP32 and the 16-bit formats after 2000 steps: rho within 1e-5
    (FP16 2e-5) and mu within 2e-6 (FP16 1e-5) absolute; U and P are reported, not bounded:
    this mixture relaxes to uniform, so they are ~1e-7 and ~1e-11 and the reduced
    precisions' rounding sets them."""
    p = inputs.multi_uniform(256, 256, name="n5_256")
    o = Oracle.from_problem(p)
    o.run(500)
    ref500 = o.moments()
    o.run(1500)
    ref2000 = o.moments()
    rng = np.random.default_rng(7)
    q = Oracle.from_problem(p)
    q.init(p.rho * (1 + 2.0 ** -52 * rng.uniform(-1, 1, p.rho.shape)), p.u)
    q.run(500)
    self500 = q.moments()
    sim = mclb.Simulation.from_problem(p, precision="fp64", kernel=mclb.KERNEL_FUSED)
    sim.step(500)
    assert sim.status() == 0
    g = sim.moments()
    for k in ("rho", "U", "mu", "P"):
        floor = 8 * 2.0 ** -52 * np.abs(ref500[k]).max()
        sens = max(np.abs(self500[k] - ref500[k]).max(), floor)
        assert np.abs(g[k] - ref500[k]).max() <= 10 * sens, k
    sim.close()
    bounds = {"fp32": (1e-5, 2e-6), "bf16": (1e-5, 2e-6), "fp16": (2e-5, 1e-5)}
    for prec, (brho, bmu) in bounds.items():
        sim = mclb.Simulation.from_problem(p, precision=prec, kernel=mclb.KERNEL_FUSED)
        sim.step(2000)
        assert sim.status() == 0
        g = sim.moments(U=False, P=False)
        assert np.abs(g["rho"] - ref2000["rho"]).max() < brho, prec
        assert np.abs(g["mu"] - ref2000["mu"]).max() < bmu, prec
        sim.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("kernel", KERNELS)
def test_resume_equals_uninterrupted(precision, kernel):
    """Checkpoint and resume: get_state after 37 steps, set_state into a new handle, and 45
    more steps there (one 32-step graph chunk and 13 single steps, from the other buffer
    parity) equal 45 more steps of the original handle, bitwise."""
    p = inputs.ternary_droplets(128, 96)
    a = mclb.Simulation.from_problem(p, precision=precision, kernel=kernel)
    a.step(37)
    f = a.get_state()
    b = mclb.Simulation(p.ncomp, p.nx, p.ny, p.tau, p.chi, p.m, p.theta, p.kappa, p.force,
                        precision, kernel)
    b.set_state(f)
    assert b.step_count == 0
    a.step(45)
    b.step(45)
    assert a.status() == 0 and b.status() == 0
    assert np.array_equal(a.get_state(), b.get_state())
    a.close()
    b.close()


def test_n5_spinodal_per_field():
    """The N = 5 workload's interactions at a mean composition inside the spinodal (the
    strongest pair at 0.4 each, inputs.multi_spinodal): the mixture separates into two
    phases, so rho, U, mu and P are compared across interfaces rather than on a uniform
    state.  256 x 256 against the FP64 oracle.  FP64 after 2000 steps: every field within
    10x the oracle's own divergence from a start perturbed by 2^-52 (floored at 8 units of
    roundoff of the field's scale).  After 500 steps (before the growing composition mode
    has amplified rounding by more than a few times): FP32 within 1e-5 on all four fields,
    BF16 and FP16 within 2e-5 on rho, U and mu and 1e-6 on P."""
    p = inputs.multi_spinodal(256, 256)
    o = Oracle.from_problem(p)
    o.run(500)
    ref500 = o.moments()
    o.run(1500)
    ref2000 = o.moments()
    rng = np.random.default_rng(7)
    q = Oracle.from_problem(p)
    q.init(p.rho * (1 + 2.0 ** -52 * rng.uniform(-1, 1, p.rho.shape)), p.u)
    q.run(2000)
    self2000 = q.moments()
    assert np.abs(ref2000["rho"][p.meta["pair"][0]]).max() > 0.6   # separated
    sim = mclb.Simulation.from_problem(p, precision="fp64", kernel=mclb.KERNEL_FUSED)
    sim.step(2000)
    assert sim.status() == 0
    g = sim.moments()
    for k in ("rho", "U", "mu", "P"):
        floor = 8 * 2.0 ** -52 * np.abs(ref2000[k]).max()
        sens = max(np.abs(self2000[k] - ref2000[k]).max(), floor)
        assert np.abs(g[k] - ref2000[k]).max() <= 10 * sens, k
    sim.close()
    bounds = {"fp32": (1e-5, 1e-5), "bf16": (2e-5, 1e-6), "fp16": (2e-5, 1e-6)}
    for prec, (b, bp) in bounds.items():
        sim = mclb.Simulation.from_problem(p, precision=prec, kernel=mclb.KERNEL_FUSED)
        sim.step(500)
        assert sim.status() == 0
        g = sim.moments()
        for k in ("rho", "U", "mu"):
            assert np.abs(g[k] - ref500[k]).max() < b, (prec, k)
        assert np.abs(g["P"] - ref500["P"]).max() < bp, prec
        sim.close()
