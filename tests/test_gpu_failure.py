"""GPU failure detection without a GPU fault: the single-pass kernel's bounded waits.

Every mbarrier wait of the kernel gives up after about 2 s; the CTA then records
STATUS_TIMEOUT, waits (bounded) for its own copies and returns, so the context stays
usable.  The test makes the wait run out on purpose: with the test hook on, no copy is
issued, so nothing ever completes the barrier.  It checks that the host reads
MCLB_ETIMEOUT, and that the same handle then runs normally again."""
import time

import numpy as np
import pytest

import paper_0704_3444_gb300 as mclb
from oracle import Oracle
from paper_0704_3444_gb300 import inputs

pytestmark = pytest.mark.gpu

ETIMEOUT = -5


@pytest.fixture(scope="module", autouse=True)
def built():
    mclb.build()
    mclb.load()


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_bounded_wait_reports_timeout_and_recovers(precision):
    n, nx, ny = 3, 70, 40
    rho, u = inputs.random_state(n, nx, ny, seed=91, amp=0.2, umax=0.02)
    chi = inputs.uniform_chi(n, 2.0)
    sim = mclb.Simulation(n, nx, ny, 0.9, chi, precision=precision, kernel=mclb.KERNEL_FUSED)
    sim.init_fields(rho, u)
    sim.step(2)
    assert sim.status() == 0
    sim.test_withhold_copies(True)
    t0 = time.perf_counter()
    sim.step(1)
    assert sim.status() == ETIMEOUT
    waited = time.perf_counter() - t0
    assert 0.5 < waited < 30.0          # the wait ran out after its bound, not at once
    sim.test_withhold_copies(False)
    sim.init_fields(rho, u)             # state is unspecified after the failed step
    sim.step(5)
    assert sim.status() == 0
    orc = Oracle(n, nx, ny, 0.9, chi)
    orc.init(rho, u)
    orc.run(5)
    tol = 1e-5 if precision == "fp32" else 5e-3
    assert np.max(np.abs(sim.moments(mu=False, P=False)["rho"] - orc.moments()["rho"])) < tol
