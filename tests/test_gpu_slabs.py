"""Slabs of one periodic D2Q9 lattice on the GPU: the library's bands of rows
(mclb_rows_bytes, mclb_pack_rows_device, mclb_unpack_rows_device, mclb_conservation_rows)
and the slab decomposition over them, several slabs on one GPU in one process.

Tolerances: FP64 slabs against the FP64 oracle of the whole lattice, 1e-12 relative to
each field's max-norm and 1e-12 absolute on P (the FP64 parity bounds); FP32 slabs against the whole FP32 handle,
1e-5 absolute on rho, U, mu and P after 100 steps (the FP32 per-field bound); band copies
byte for byte in every storage format."""
import numpy as np
import pytest

import paper_0704_3444_gb300 as mclb
from oracle import Oracle
from paper_0704_3444_gb300 import inputs, slabs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

KW = dict(ncomp=3, tau=0.8, chi=inputs.random_chi(3, 0.9, 1.4, seed=42),
          m=np.array([1.0, 2.0, 1.0]), theta=0.3, kappa=0.02, force=(1e-4, -2e-4))


@pytest.fixture(scope="module", autouse=True)
def built():
    mclb.build()
    mclb.load()


def _rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def _buf(n):
    return torch.empty(n, dtype=torch.uint8, device="cuda")


def test_a_handle_on_a_non_blocking_stream_starts_from_its_init():
    """A handle's set-up (zeroed buffers and status word) is ordered on its own stream: one
    made on a non-blocking stream while another handle's steps are still queued starts from
    its own initial fields, not from set-up work that lands later.  (The slabs run on such
    a stream.)"""
    busy = mclb.Simulation(nx=1024, ny=1024, precision="fp32", **KW)
    busy.init_fields(*inputs.random_state(3, 1024, 1024, seed=3))
    busy.step(300)   # queued, not waited for
    ts = torch.cuda.Stream()
    sim = mclb.Simulation(nx=64, ny=48, precision="fp64", stream=ts.cuda_stream, **KW)
    rho, u = inputs.random_state(3, 64, 48, seed=4)
    sim.init_fields(rho, u)
    sim.step(2)
    assert sim.status() == 0
    orc = Oracle(KW["ncomp"], 64, 48, KW["tau"], KW["chi"], KW["m"], KW["theta"], KW["kappa"],
                 KW["force"])
    orc.init(rho, u)
    orc.run(2)
    assert _rel(sim.get_state(), orc.f) < 1e-12
    assert busy.status() == 0


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16", "fp16"])
def test_band_round_trip_is_byte_exact(precision):
    nx, ny = 150, 40
    # both handles and the buffers on one stream: the unpack into b follows the pack of a
    ts = torch.cuda.Stream()
    a = mclb.Simulation(nx=nx, ny=ny, precision=precision, stream=ts.cuda_stream, **KW)
    b = mclb.Simulation(nx=nx, ny=ny, precision=precision, stream=ts.cuda_stream, **KW)
    a.init_fields(*inputs.random_state(3, nx, ny, seed=7))
    b.init_fields(*inputs.random_state(3, nx, ny, seed=8))
    a.step(3)
    nb = a.rows_bytes(4)
    assert nb > 0 and nb == 4 * a.rows_bytes(1) == b.rows_bytes(4)
    with torch.cuda.stream(ts):
        one, two = _buf(nb), _buf(nb)
    a.pack_rows(5, 4, one)
    b.unpack_rows(20, 4, one)
    b.pack_rows(20, 4, two)
    torch.cuda.synchronize()
    assert torch.equal(one, two)
    # rows away from the band keep b's own values
    fa, fb = a.get_state(), b.get_state()
    b0 = mclb.Simulation(nx=nx, ny=ny, precision=precision, **KW)
    b0.init_fields(*inputs.random_state(3, nx, ny, seed=8))
    assert np.array_equal(fb[:, :, :19], b0.get_state()[:, :, :19])
    # the band's inner rows read back as a's rows (their pulls stay inside the band)
    assert np.array_equal(fb[:, :, 21:23], fa[:, :, 6:8])


def test_row_sums_partition_the_whole_sums():
    nx, ny = 130, 61
    sim = mclb.Simulation(nx=nx, ny=ny, precision="fp64", **KW)
    sim.init_fields(*inputs.random_state(3, nx, ny, seed=9))
    sim.step(5)
    whole = sim.conservation()
    all_rows = sim.conservation_rows(0, ny)
    for k in whole:
        assert np.array_equal(whole[k], all_rows[k]), k
    parts = [sim.conservation_rows(y0, h) for y0, h in slabs.split_rows(ny, 3)]
    for k in whole:
        tot = sum(p[k] for p in parts)
        np.testing.assert_allclose(tot, whole[k], rtol=1e-12, atol=1e-15)
    empty = sim.conservation_rows(10, 0)
    assert all(not np.any(v) for v in empty.values())


def test_band_arguments_are_checked():
    sim = mclb.Simulation(nx=20, ny=10, precision="fp32", **KW)
    buf = _buf(sim.rows_bytes(12))
    for y0, n in [(-1, 2), (9, 2), (0, 11)]:
        with pytest.raises(mclb.MclbError) as e:
            sim.pack_rows(y0, n, buf)
        assert e.value.code == -1
        with pytest.raises(mclb.MclbError):
            sim.conservation_rows(y0, n)
    with pytest.raises(ValueError):
        sim.unpack_rows(0, 10, _buf(16))   # buffer too small for the band
    line = mclb.Simulation(nx=64, ny=1, precision="fp32", lattice="d1q3",
                           **dict(KW, force=(1e-4, 0.0)))
    assert line.rows_bytes(1) == 0
    with pytest.raises(mclb.MclbError):
        line.conservation_rows(0, 1)


@pytest.mark.parametrize("kernel,parts,period,edges", [
    (mclb.KERNEL_FUSED, 2, 1, "walls"), (mclb.KERNEL_FUSED, 3, 2, "walls"),
    (mclb.KERNEL_FUSED, 1, 1, "walls"), (mclb.KERNEL_STAGED, 2, 1, "walls"),
    (mclb.KERNEL_STAGED, 3, 2, "walls"), (mclb.KERNEL_STAGED, 1, 1, "walls"),
    (mclb.KERNEL_FUSED, 3, 2, "periodic"), (mclb.KERNEL_STAGED, 2, 1, "periodic")])
def test_fp64_slabs_match_the_oracle(parts, period, kernel, edges):
    nx, ny, steps = 130, 61, 30
    rho, u = inputs.random_state(3, nx, ny, seed=11, amp=0.2, umax=0.03)
    orc = Oracle(KW["ncomp"], nx, ny, KW["tau"], KW["chi"], KW["m"], KW["theta"], KW["kappa"],
                 KW["force"])
    orc.init(rho, u)
    orc.run(steps)
    ls = slabs.LocalSlabs(nx, ny, parts, period, precision="fp64", kernel=kernel, edges=edges,
                          **KW)
    ls.init_fields(rho, u)
    ls.step(11)
    ls.step(steps - 11)
    assert all(s == 0 for s in ls.status())
    assert _rel(ls.get_state(), orc.f) < 1e-12
    m, mo = ls.moments(), orc.moments()
    for k in ("rho", "U", "mu"):
        assert _rel(m[k], mo[k]) < 1e-12, k
    # P is a difference of O(1) terms (sum rho mu - psi): bounded in absolute terms, as the
    # whole-lattice FP64 parity bounds it
    assert np.max(np.abs(m["P"] - mo["P"])) < 1e-12 * max(1.0, np.abs(mo["P"]).max())
    c, co = ls.conservation(), orc.conservation()
    np.testing.assert_allclose(c["mass"], co["mass"], rtol=1e-12)
    for k in ("mom", "force"):
        assert np.max(np.abs(c[k] - co[k])) < 1e-12 * nx * ny, k
    ls.close()


@pytest.mark.parametrize("edges", ["walls", "periodic"])
def test_fp32_slabs_match_the_whole_handle(edges):
    nx, ny, steps = 256, 256, 100
    prob = inputs.ternary_droplets(nx, ny, precision="fp32")
    kw = dict(ncomp=prob.ncomp, tau=prob.tau, chi=prob.chi, m=prob.m, theta=prob.theta,
              kappa=prob.kappa, force=prob.force)
    whole = mclb.Simulation(nx=nx, ny=ny, precision="fp32", **kw)
    whole.init_fields(prob.rho, prob.u)
    whole.step(steps)
    ls = slabs.LocalSlabs(nx, ny, 2, 1, precision="fp32", edges=edges, **kw)
    ls.init_fields(prob.rho, prob.u)
    ls.step(steps)
    assert all(s == 0 for s in ls.status()) and whole.status() == 0
    m, mw = ls.moments(), whole.moments()
    for k in ("rho", "U", "mu", "P"):
        assert np.max(np.abs(m[k] - mw[k])) < 1e-5, k
    ls.close()


def test_slab_decomposition_on_one_nccl_rank():
    """SlabDecomposition over a one-rank NCCL group: the slab is its own neighbour (the bands
    are copied in place) and the FP64 sums go through an NCCL all-reduce on the slab's
    stream; the result is the whole lattice's."""
    import socket

    import torch.distributed as dist

    if dist.is_initialized():
        pytest.skip("a process group is already initialised")
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1,
                            device_id=torch.device("cuda", torch.cuda.current_device()))
    try:
        nx, ny, steps = 96, 40, 20
        rho, u = inputs.random_state(3, nx, ny, seed=13, amp=0.2, umax=0.03)
        orc = Oracle(KW["ncomp"], nx, ny, KW["tau"], KW["chi"], KW["m"], KW["theta"],
                     KW["kappa"], KW["force"])
        orc.init(rho, u)
        orc.run(steps)
        sd = slabs.SlabDecomposition(nx, ny, 2, precision="fp64", **KW)
        assert sd.rows == (0, ny)
        sd.init_fields(rho, u)
        sd.step(steps)
        assert sd.status() == 0
        assert _rel(sd.get_state(), orc.f) < 1e-12
        c, co = sd.conservation(), orc.conservation()
        np.testing.assert_allclose(c["mass"], co["mass"], rtol=1e-12)
        assert np.max(np.abs(c["mom"] - co["mom"])) < 1e-12 * nx * ny
        sd.close()
    finally:
        dist.destroy_process_group()
