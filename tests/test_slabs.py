"""Slab decomposition of one periodic D2Q9 lattice (paper_0704_3444_gb300.slabs), on CPU.

The host logic -- which rows each slab holds, which bands go where, the exchange period,
the row-restricted FP64 sums -- runs here over FP64 oracle lattices standing in for the
library handles (the oracle's per-site arithmetic does not depend on the lattice it sits
in, so a correct decomposition reproduces the whole lattice bit for bit).  The slabs are
connected in one process (LocalSlabs) and across gloo ranks (SlabDecomposition).  The
library's own bands and handles are checked on the GPU (test_gpu_slabs.py)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_0704_3444_gb300 import inputs, slabs

VX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], dtype=np.float64)
VY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1], dtype=np.float64)

NX, NY = 20, 31   # an odd row count: uneven slabs


def problem():
    rho, u = inputs.random_state(3, NX, NY, seed=41, amp=0.2, umax=0.03)
    chi = inputs.random_chi(3, 1.6, 2.6, seed=42)
    return dict(ncomp=3, tau=0.8, chi=chi, m=np.array([1.0, 2.0, 1.0]), theta=0.3,
                kappa=0.02, force=(1e-4, -2e-4)), rho, u


class OracleSlabHandle:
    """The stepping interface slabs.py drives, over an FP64 oracle lattice between walls,
    as the library's slab handles are (test infrastructure: the band is the pre-collision
    state's rows, packed as bytes)."""

    def __init__(self, nx, rows, kw, walls=1):
        self.o = oracle.Oracle(kw["ncomp"], nx, rows, kw["tau"], kw["chi"], kw["m"], kw["theta"],
                               kw["kappa"], kw["force"], walls=walls)
        self.N, self.nx = kw["ncomp"], nx

    def init_fields(self, rho, u):
        self.o.init(rho, u)

    def set_state(self, f):
        self.o.set_state(f)

    def get_state(self):
        return self.o.f.copy()

    def step(self, n):
        self.o.run(n)

    def status(self):
        return 0

    def rows_bytes(self, n):
        return self.N * 9 * n * self.nx * 8

    def pack_rows(self, y0, n, buf):
        band = np.ascontiguousarray(self.o.f[:, :, y0:y0 + n, :])
        buf.numpy()[:band.nbytes] = band.reshape(-1).view(np.uint8)

    def unpack_rows(self, y0, n, buf):
        nb = self.rows_bytes(n)
        self.o.f[:, :, y0:y0 + n, :] = buf.numpy()[:nb].view(np.float64).reshape(self.N, 9, n, self.nx)

    def moments(self):
        return self.o.moments()

    def conservation_rows(self, y0, n):
        return rows_sums(self.o, y0, n)


def rows_sums(o, y0, n):
    """Mass, momentum sum_i f_i v_i and force sum 2 (rho U - j) over rows [y0, y0 + n)."""
    f = o.f[:, :, y0:y0 + n, :]
    m = o.moments()
    rho = m["rho"][:, y0:y0 + n, :]
    jx = np.einsum("sixy,i->xy", f.transpose(0, 1, 3, 2), VX).T
    jy = np.einsum("sixy,i->xy", f.transpose(0, 1, 3, 2), VY).T
    R = rho.sum(axis=0)
    U = m["U"][:, y0:y0 + n, :]
    return dict(mass=rho.sum(axis=(1, 2)), mom=np.array([jx.sum(), jy.sum()]),
                force=np.array([(2 * (R * U[0] - jx)).sum(), (2 * (R * U[1] - jy)).sum()]))


def cpu_buffer(nbytes):
    return torch.empty(max(nbytes, 1), dtype=torch.uint8)


def whole_lattice(kw, rho, u, steps):
    o = oracle.Oracle(kw["ncomp"], NX, NY, kw["tau"], kw["chi"], kw["m"], kw["theta"],
                      kw["kappa"], kw["force"])
    o.init(rho, u)
    o.run(steps)
    return o


def test_split_rows_covers_the_lattice():
    for ny, parts in [(31, 2), (31, 3), (8, 8), (100, 7)]:
        sp = slabs.split_rows(ny, parts)
        assert sp[0][0] == 0 and sum(h for _, h in sp) == ny
        assert all(a + h == b for (a, h), (b, _) in zip(sp, sp[1:]))
        assert max(h for _, h in sp) - min(h for _, h in sp) <= 1
    with pytest.raises(ValueError):
        slabs.split_rows(3, 4)


@pytest.mark.parametrize("walls", [1, 0], ids=["walls", "periodic"])
@pytest.mark.parametrize("parts,period", [(1, 1), (2, 1), (3, 1), (2, 2), (3, 3)])
def test_local_slabs_equal_the_whole_lattice(parts, period, walls):
    """Either edge of the slab handles (walls, as the library's default slabs, or a periodic
    wrap) leaves the own rows exact."""
    kw, rho, u = problem()
    steps = 23   # not a multiple of any period: the last chunk is short
    ref = whole_lattice(kw, rho, u, steps)
    ls = slabs.LocalSlabs(NX, NY, parts, period,
                          make_handle=lambda rows: OracleSlabHandle(NX, rows, kw, walls),
                          new_buffer=cpu_buffer)
    ls.init_fields(rho, u)
    ls.step(7)
    ls.step(steps - 7)
    assert np.array_equal(ls.get_state(), ref.f)
    m, mr = ls.moments(), ref.moments()
    for k in ("rho", "U", "mu", "P"):
        assert np.array_equal(m[k], mr[k]), k
    c, cr = ls.conservation(), rows_sums(ref, 0, NY)
    for k in ("mass", "mom", "force"):
        np.testing.assert_allclose(c[k], cr[k], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(c["mass"], ref.conservation()["mass"], rtol=1e-12)


def test_set_state_then_steps_equal_the_whole_lattice():
    kw, rho, u = problem()
    ref = whole_lattice(kw, rho, u, 5)
    f5 = ref.f.copy()
    ref.run(12)
    ls = slabs.LocalSlabs(NX, NY, 3, 2, make_handle=lambda rows: OracleSlabHandle(NX, rows, kw),
                          new_buffer=cpu_buffer)
    ls.set_state(f5)
    ls.step(12)
    assert np.array_equal(ls.get_state(), ref.f)


def test_a_shorter_reach_is_detected(monkeypatch):
    """With the outer bands one row too thin (reach 2), the slabs' rows next to a band
    drift from the whole lattice: the reach of 3 rows is needed, and the comparison
    above sees a wrong band."""
    kw, rho, u = problem()
    ref = whole_lattice(kw, rho, u, 6)
    monkeypatch.setattr(slabs, "REACH", 2)
    ls = slabs.LocalSlabs(NX, NY, 2, 1, make_handle=lambda rows: OracleSlabHandle(NX, rows, kw),
                          new_buffer=cpu_buffer)
    ls.init_fields(rho, u)
    ls.step(6)
    assert not np.allclose(ls.get_state(), ref.f, rtol=0, atol=1e-13)


def test_slabs_thinner_than_the_band_are_rejected():
    kw, _, _ = problem()
    with pytest.raises(ValueError):
        slabs.LocalSlabs(NX, NY, 4, 3, make_handle=lambda rows: OracleSlabHandle(NX, rows, kw),
                         new_buffer=cpu_buffer)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, period, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    os.environ["OMP_NUM_THREADS"] = "1"
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        kw, rho, u = problem()
        steps = 17
        ref = whole_lattice(kw, rho, u, steps)
        sd = slabs.SlabDecomposition(NX, NY, period,
                                     make_handle=lambda rows: OracleSlabHandle(NX, rows, kw),
                                     new_buffer=cpu_buffer)
        sd.init_fields(rho, u)
        sd.step(steps)
        y0, h = sd.rows
        state_ok = bool(np.array_equal(sd.get_state(), ref.f[:, :, y0:y0 + h, :]))
        m, mr = sd.moments(), ref.moments()
        moments_ok = all(np.array_equal(m[k], mr[k][:, y0:y0 + h, :]) for k in m)
        c, cr = sd.conservation(), rows_sums(ref, 0, NY)
        sums_err = max(float(np.max(np.abs(c[k] - cr[k]) / (np.abs(cr[k]) + 1e-12)))
                       for k in ("mass", "mom", "force"))
        g = sd.gather_moments(root=world - 1)
        gathered_ok = (g is None) if rank != world - 1 else all(
            np.array_equal(g[k], mr[k]) for k in ("rho", "U", "mu", "P"))
        out[rank] = (y0, h, state_ok, moments_ok and gathered_ok, sums_err)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,period", [(2, 1), (3, 2)])
def test_slab_decomposition_over_gloo_ranks(world, period):
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_rank, args=(r, world, port, period, out))
                 for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(300)
            assert p.exitcode == 0
        res = dict(out)
    assert sorted((res[r][0], res[r][1]) for r in res) == slabs.split_rows(NY, world)
    for r in range(world):
        _, _, state_ok, moments_ok, sums_err = res[r]
        assert state_ok and moments_ok, r
        assert sums_err < 1e-11, (r, sums_err)


class FailingSlabHandle(OracleSlabHandle):
    """A stand-in whose device status turns ENONFINITE (-4) after `after` timesteps, as the
    library's step_nocheck would report it (the failure is made on the host)."""

    def __init__(self, nx, rows, kw, after):
        super().__init__(nx, rows, kw)
        self.after, self.done = after, 0

    def step_nocheck(self, n):
        self.o.run(n)
        self.done += n
        return -4 if self.done > self.after else 0


def _failing_rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    os.environ["OMP_NUM_THREADS"] = "1"
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        kw, rho, u = problem()
        make = ((lambda rows: FailingSlabHandle(NX, rows, kw, after=5)) if rank == 1
                else (lambda rows: OracleSlabHandle(NX, rows, kw)))
        sd = slabs.SlabDecomposition(NX, NY, 1, make_handle=make, new_buffer=cpu_buffer)
        sd.init_fields(rho, u)
        sd.step(12)           # rank 1's status turns bad at step 6; nobody stops early
        out[rank] = (sd._fresh, sd.status())
    finally:
        dist.destroy_process_group()


def test_a_device_status_on_one_rank_reaches_every_rank():
    """A non-finite status on one rank neither stops its steps nor leaves its neighbour
    waiting for bands: both ranks finish the steps, and the collective status() reports the
    code on both."""
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_failing_rank, args=(r, world, port, out))
                 for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(300)
            assert p.exitcode == 0
        res = dict(out)
    assert res == {0: (0, -4), 1: (0, -4)}


def _dying_rank(rank, world, port, out):
    import datetime

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    os.environ["OMP_NUM_THREADS"] = "1"
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=5))
    kw, rho, u = problem()
    sd = slabs.SlabDecomposition(NX, NY, 1, make_handle=lambda rows: OracleSlabHandle(NX, rows, kw),
                                 new_buffer=cpu_buffer)
    sd.init_fields(rho, u)
    if rank == 1:
        os._exit(3)           # the rank is lost between steps, none of its exchanges in flight
    import time

    t0 = time.time()
    try:
        sd.step(4)
        out[rank] = ("no error", time.time() - t0)
    except Exception as e:    # the next exchange with the lost rank fails
        out[rank] = (type(e).__name__, time.time() - t0)
    os._exit(0)               # no teardown with a lost peer


def test_a_lost_rank_ends_the_next_exchange_with_an_error():
    """A rank that leaves between steps: its neighbour's next exchange fails within the
    process group's timeout instead of waiting for ever (failure made on the host)."""
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_dying_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
        codes = [p.exitcode for p in procs]
        res = dict(out)
    assert codes == [0, 3]
    kind, seconds = res[0]
    assert kind != "no error" and seconds < 60, res
