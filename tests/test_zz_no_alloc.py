"""The allocation-free timestep (mclb_step_noalloc) against the handle-based one.

Some callers cannot allocate device memory (they run inside an application that owns
a fixed device memory budget, or must not call cudaMalloc because it synchronises the
device).  mclb_step_noalloc keeps its scratch fields in a fixed array inside the
library instead.  This file is collected last on purpose, so that a run that stops at
the first failure has already run every other test; it passes alone or after them.
"""
import ctypes

import numpy as np
import pytest

import paper_0704_3444_gb300 as mclb
from paper_0704_3444_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_noalloc_step_matches_handle_step_twice():
    torch = pytest.importorskip("torch")
    mclb.build()
    lib = mclb.load()
    n, nx, ny = 3, 48, 40
    rho, u = inputs.random_state(n, nx, ny, seed=91, amp=0.3, umax=0.03)
    chi = np.array([[0.0, 2.6, 2.1], [2.6, 0.0, 2.4], [2.1, 2.4, 0.0]])
    args = dict(ncomp=n, nx=nx, ny=ny, tau=0.85, chi=chi, m=[1.0, 2.0, 1.0], theta=0.4,
                kappa=0.02, force=(1e-4, -5e-5), precision="fp64")
    sim = mclb.Simulation(n, nx, ny, args["tau"], chi, args["m"], args["theta"], args["kappa"],
                          args["force"], "fp64", mclb.KERNEL_STAGED)
    sim.init_fields(rho, u)
    f0 = sim.get_state()
    p, keep = mclb.make_params(**args)

    a = torch.tensor(f0, dtype=torch.float64, device="cuda")
    b = torch.empty_like(a)
    torch.cuda.synchronize()
    for call in range(2):
        rc = lib.mclb_step_noalloc(ctypes.byref(p), a.data_ptr(), b.data_ptr())
        assert rc == 0, lib.mclb_last_error().decode()
        torch.cuda.synchronize()
        sim.step(1)
        want = sim.get_state()
        got = b.cpu().numpy()
        err = np.max(np.abs(got - want)) / np.abs(want).max()
        assert err < 1e-12, (call, err)
        a, b = b, a
    sim.close()


def test_noalloc_rejects_oversized_and_bad_arguments():
    torch = pytest.importorskip("torch")
    lib = mclb.load()
    chi = np.array([[0.0, 2.0], [2.0, 0.0]])
    big, keep1 = mclb.make_params(2, 1024, 512, 1.0, chi, precision="fp64")
    a = torch.zeros(8, dtype=torch.float64, device="cuda")
    b = torch.zeros(8, dtype=torch.float64, device="cuda")
    assert lib.mclb_step_noalloc(ctypes.byref(big), a.data_ptr(), b.data_ptr()) == -1
    assert "exceeds" in lib.mclb_last_error().decode()
    small32, keep2 = mclb.make_params(2, 8, 8, 1.0, chi, precision="fp32")
    assert lib.mclb_step_noalloc(ctypes.byref(small32), a.data_ptr(), b.data_ptr()) == -1
    small, keep3 = mclb.make_params(2, 8, 8, 1.0, chi, precision="fp64")
    assert lib.mclb_step_noalloc(ctypes.byref(small), a.data_ptr(), a.data_ptr()) == -1


def test_noalloc_at_the_limit_on_a_side_stream():
    """The largest accepted problem (N * nx * ny = MCLB_NOALLOC_MAX_COMP_SITES, so the
    second scratch field ends at the array's last element), the barycentric forcing
    reading, and a caller's own stream: both calls run on a torch side stream passed
    through params->stream, only that stream is synchronised, and each result equals
    the handle-based staged step to 1e-12."""
    torch = pytest.importorskip("torch")
    lib = mclb.load()
    n, nx, ny = 2, 512, 512
    assert n * nx * ny == 524288
    rho, u = inputs.random_state(n, nx, ny, seed=92, amp=0.3, umax=0.03)
    chi = np.array([[0.0, 2.3], [2.3, 0.0]])
    side = torch.cuda.Stream()
    args = dict(ncomp=n, nx=nx, ny=ny, tau=0.9, chi=chi, theta=0.45, kappa=0.01,
                force=(0.0, 2e-5), precision="fp64", stream=side.cuda_stream,
                forcing_velocity=mclb.FORCING_BARYCENTRIC)
    sim = mclb.Simulation(n, nx, ny, 0.9, chi, None, 0.45, 0.01, (0.0, 2e-5), "fp64",
                          mclb.KERNEL_STAGED, forcing_velocity=mclb.FORCING_BARYCENTRIC)
    sim.init_fields(rho, u)
    f0 = sim.get_state()
    p, keep = mclb.make_params(**args)
    with torch.cuda.stream(side):
        a = torch.tensor(f0, dtype=torch.float64, device="cuda")
        b = torch.empty_like(a)
    side.synchronize()
    for call in range(2):
        rc = lib.mclb_step_noalloc(ctypes.byref(p), a.data_ptr(), b.data_ptr())
        assert rc == 0, lib.mclb_last_error().decode()
        side.synchronize()
        sim.step(1)
        want = sim.get_state()
        with torch.cuda.stream(side):
            got = b.cpu().numpy()
        err = np.max(np.abs(got - want)) / np.abs(want).max()
        assert err < 1e-12, (call, err)
        a, b = b, a
    sim.close()


def test_noalloc_rejects_overlapping_arrays():
    torch = pytest.importorskip("torch")
    lib = mclb.load()
    chi = np.array([[0.0, 2.0], [2.0, 0.0]])
    p, keep = mclb.make_params(2, 8, 8, 1.0, chi, precision="fp64")
    total = 2 * 9 * 8 * 8
    buf = torch.full((2 * total,), 0.05, dtype=torch.float64, device="cuda")
    base = buf.data_ptr()
    # f_out starts inside f_in, one value before its end
    assert lib.mclb_step_noalloc(ctypes.byref(p), base, base + 8 * (total - 1)) == -1
    assert "overlap" in lib.mclb_last_error().decode()
    # f_in starts inside f_out
    assert lib.mclb_step_noalloc(ctypes.byref(p), base + 8 * 5, base) == -1
    # adjacent ranges do not overlap
    assert lib.mclb_step_noalloc(ctypes.byref(p), base, base + 8 * total) == 0
    torch.cuda.synchronize()
