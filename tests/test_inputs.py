"""The seeded input generators (paper_0704_3444_gb300/inputs.py), without a GPU.

They feed both the CUDA path and the oracle, so they are pinned on their own: SplitMix64
against the first outputs of its published reference implementation (seed 0), the uniform
and Gaussian draws by their first two moments, and every workload recipe by the
invariants it states (compositions summing to 1 per site, chi symmetric with a zero
diagonal and inside its stated range, the batch's shapes and parameter ranges).
"""
import numpy as np

from paper_0704_3444_gb300 import inputs


def test_splitmix64_reference_outputs():
    # first three outputs of the SplitMix64 reference generator started from state 0
    want = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    assert [int(v) for v in inputs.splitmix64(0, 3)] == want


def test_streams_are_deterministic_and_distinct():
    a, b = inputs.uniform(7, 1000, 3), inputs.uniform(7, 1000, 3)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, inputs.uniform(7, 1000, 4))
    assert not np.array_equal(a, inputs.uniform(8, 1000, 3))


def test_uniform_and_gaussian_moments():
    n = 1_000_000
    u = inputs.uniform(3, n)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 5 * np.sqrt(1 / 12 / n)
    assert abs(u.var() - 1 / 12) < 5 * np.sqrt(1 / 180 / n)
    g = inputs.gaussian(3, n)
    assert abs(g.mean()) < 5 / np.sqrt(n)
    assert abs(g.var() - 1.0) < 5 * np.sqrt(2 / n)


def _check_chi(chi, lo, hi):
    assert np.array_equal(chi, chi.T) and np.all(np.diag(chi) == 0.0)
    off = chi[~np.eye(len(chi), dtype=bool)]
    assert np.all(off >= lo - 1e-12) and np.all(off <= hi + 1e-12)


def test_workload_recipes():
    for p, amp in ((inputs.binary_noise(16, 12), 0.01), (inputs.multi_uniform(16, 12), 0.01)):
        phi = p.rho / p.rho.sum(0)
        np.testing.assert_allclose(p.rho.sum(0), 1.0, atol=1e-15)
        # the mass-neutral step (subtracting the across-component mean) can stretch one
        # component's deviation to 2 (N - 1) / N times the drawn amplitude
        bound = amp * max(1.0, 2.0 * (p.ncomp - 1) / p.ncomp)
        assert np.max(np.abs(phi - 1.0 / p.ncomp)) <= bound * (1 + 1e-12)
        assert np.all(p.u == 0.0)
    _check_chi(inputs.multi_uniform(16, 12).chi, 2 * 0.8, 2 * 1.5)
    t = inputs.ternary_gauss(32, 32)
    np.testing.assert_allclose(t.rho.sum(0), 1.0, atol=1e-15)
    assert abs(t.rho.std() - 0.005) < 0.002 and np.all(t.rho > 0)
    s = inputs.slab(64, 16)
    np.testing.assert_allclose(s.rho.sum(0), 1.0, atol=1e-15)
    assert np.allclose(s.rho[:, :, 8], [[0.3], [0.7], [0.0]]) and np.allclose(s.rho[:, :, 40], [[0], [0], [1]])
    _check_chi(s.chi, 0.2, 3.0)


def test_batch_recipe():
    probs = inputs.batch(64)
    assert len(probs) == 64 and {p.ncomp for p in probs} == {2, 3}
    for p in probs:
        assert 32 <= p.nx <= 512 and 32 <= p.ny <= 512 and 0.6 <= p.tau <= 1.5 and p.kappa == 0.01
        off = p.chi[~np.eye(p.ncomp, dtype=bool)]
        assert np.all(off >= 2 * 0.9 - 1e-12) and np.all(off <= 2 * 1.6 + 1e-12)
        np.testing.assert_allclose(p.rho.sum(0), 1.0, atol=1e-14)
