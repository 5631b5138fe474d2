"""One periodic D2Q9 lattice split into slabs of rows (y), one simulation handle per slab.

The paper advances one periodic lattice (Sec. 3, Eq. ssLB).  A lattice can also be cut
into y slabs held by separate handles -- one per GPU of a process group, or several in
one process -- without changing a single value, because one timestep reaches a bounded
number of rows.  The stored post-collision value at a site depends on the stored values
at most R = 3 rows away: the pull of Eq. ssLB reaches one row, the force of Eq. definef
takes a centred gradient of mu^s (one row more), and mu^s holds -kappa lap rho^s (one
row more).  A slab of h rows therefore lives in a handle of h + 2G rows, G = R * period,
whose G outer rows on each side are copies of the neighbouring slabs' rows.  Beyond its
edges the handle is either closed by solid walls (``edges="walls"``, the default: walls =
1, mirrored rows and bounce-back) or periodic (``edges="periodic"``: its last row meets its
first, two rows that are far apart in the lattice).  Either way every timestep makes R
more outer rows differ from the lattice's, so after ``period`` timesteps the slab's own h
rows are still what the whole lattice would hold, and the outer rows are then refreshed
from the neighbours (G rows each way).  The walls keep the outer rows physical where a
periodic seam would join two different phases; the periodic edges save the three
wall-row launches per step.  The bands are the handles' stored
representation copied byte for byte (mclb_pack_rows_device / mclb_unpack_rows_device),
exact in every storage format.

Two ways to connect the slabs:

* ``SlabDecomposition`` -- one slab per rank of a ``torch.distributed`` process group
  (NCCL between GPUs, gloo on CPU): the bands move by point-to-point sends and receives,
  the FP64 conservation sums by an all-reduce.  Every method that exchanges or reduces
  (``step``, ``moments``, ``conservation``, ``init_fields``, ``set_state``, ``status``) is
  collective.  A device status (a non-finite density) does not stop ``step`` on one rank
  and leave the others waiting: every rank keeps stepping and exchanging, and ``status``
  reports the worst code on all of them.  A rank that dies (an exception, a lost process)
  is seen by the others only when their next exchange fails, so give the process group a
  short ``timeout``.
* ``LocalSlabs`` -- every slab in this process (for instance several slabs on one GPU):
  the bands move by copies on the handles' common stream.

The lattice is periodic D2Q9 (walls = 0 in its statement; walls, if any, are the slab
handles' edges), without the mass compensation (whose reference would span the copies).
Every slab needs h >= G rows, so that the G rows it sends are its own.
"""
from __future__ import annotations

import contextlib
from typing import Callable, List, Optional, Tuple

import numpy as np

REACH = 3   # rows one timestep reaches: pull (1) + gradient of mu (1) + Laplacian in mu (1)

__all__ = ["REACH", "split_rows", "Slab", "LocalSlabs", "SlabDecomposition"]


def split_rows(ny: int, parts: int) -> List[Tuple[int, int]]:
    """(first row, rows) of each of ``parts`` slabs of an ny-row lattice: ny // parts rows
    each, the first ny % parts slabs one more."""
    if parts < 1 or ny < parts:
        raise ValueError(f"cannot split {ny} rows into {parts} slabs")
    base, extra = divmod(ny, parts)
    out, y0 = [], 0
    for r in range(parts):
        h = base + (1 if r < extra else 0)
        out.append((y0, h))
        y0 += h
    return out


EDGES = {"periodic": 0, "walls": 1}


def _simulation_factory(nx: int, kw: dict, stream, edges: str) -> Callable[[int], object]:
    """Handles of the library for a slab of ``rows`` stored rows (the default)."""
    from . import Simulation, D2Q9, LATTICES

    kw = dict(kw)
    lattice = kw.pop("lattice", "d2q9")
    if (LATTICES[lattice] if isinstance(lattice, str) else int(lattice)) != D2Q9:
        raise ValueError("slabs are D2Q9 lattices")
    if kw.pop("walls", 0):
        raise ValueError("the lattice split into slabs is periodic in y (walls = 0)")
    if kw.pop("mass_every", 0):
        raise ValueError("the mass compensation is per handle; slabs run without it")
    kw.pop("nz", None)
    if edges not in EDGES:
        raise ValueError(f"edges {edges!r}: 'periodic' or 'walls'")
    kw["walls"] = EDGES[edges]   # the slab handle's own edges (see the module docstring)
    if stream is not None:
        kw["stream"] = stream

    def make(rows: int):
        return Simulation(nx=nx, ny=rows, **kw)

    return make


def _common_stream(stream):
    """The torch stream every slab handle and band buffer uses: the caller's (a cudaStream_t
    as an integer) or a new one.  Handles created without a stream would each create their
    own, and a band packed on one of them and unpacked on another would race."""
    import torch

    return torch.cuda.ExternalStream(stream) if stream else torch.cuda.Stream()


def _device_buffers(ts):
    import torch

    def make(nbytes: int):
        with torch.cuda.stream(ts):   # the allocator ties the block to the slabs' stream
            return torch.empty(max(nbytes, 1), dtype=torch.uint8,
                               device=torch.device("cuda", torch.cuda.current_device()))
    return make


def _on(ts):
    """Context that makes ts torch's current stream (nothing for CPU stand-ins)."""
    if ts is None:
        return contextlib.nullcontext()
    import torch

    return torch.cuda.stream(ts)


class Slab:
    """Rows [y0, y0 + h) of an ny-row periodic lattice, stored in a handle of h + 2G rows
    (G = REACH * period): stored row e holds lattice row (y0 - G + e) mod ny."""

    def __init__(self, handle, nx: int, ny: int, y0: int, h: int, period: int, new_buffer,
                 receive: bool = False):
        self.nx, self.ny, self.y0, self.h = int(nx), int(ny), int(y0), int(h)
        self.period = int(period)
        self.G = REACH * self.period
        if self.h < self.G:
            raise ValueError(f"a slab of {self.h} rows cannot send {self.G} own rows "
                             f"(period {self.period}): use fewer slabs or a shorter period")
        self.rows = self.h + 2 * self.G
        self.handle = handle
        nb = handle.rows_bytes(self.G)
        # outgoing bands: the top G own rows (to the slab above) and the bottom G (below);
        # incoming ones only where the bands arrive by messages (slabs in one process read
        # their neighbours' outgoing buffers directly)
        self.send_up, self.send_down = new_buffer(nb), new_buffer(nb)
        self.recv_below = self.recv_above = None
        if receive:
            self.recv_below, self.recv_above = new_buffer(nb), new_buffer(nb)

    @property
    def lattice_rows(self) -> np.ndarray:
        return (self.y0 - self.G + np.arange(self.rows)) % self.ny

    def own(self, a: np.ndarray) -> np.ndarray:
        """The slab's own rows of a stored-row field (axis -2 is y)."""
        return a[..., self.G:self.G + self.h, :]

    def init_fields(self, rho: np.ndarray, u: Optional[np.ndarray]):
        idx = self.lattice_rows
        rho = np.ascontiguousarray(np.asarray(rho, dtype=np.float64)[:, idx, :])
        u = None if u is None else np.ascontiguousarray(np.asarray(u, dtype=np.float64)[:, idx, :])
        self.handle.init_fields(rho, u)

    def set_state(self, f: np.ndarray):
        self.handle.set_state(np.ascontiguousarray(np.asarray(f, dtype=np.float64)[:, :, self.lattice_rows, :]))

    def pack(self):
        self.handle.pack_rows(self.h, self.G, self.send_up)        # own rows [h - G, h)
        self.handle.pack_rows(self.G, self.G, self.send_down)      # own rows [0, G)

    def unpack(self, below, above):
        """Outer rows from the band the slab below sent up and the one above sent down."""
        self.handle.unpack_rows(0, self.G, below)
        self.handle.unpack_rows(self.G + self.h, self.G, above)


class _Stepper:
    """Timesteps in chunks of at most ``period``, with an exchange after each full chunk;
    ``_fresh`` counts the timesteps since the outer rows were last refreshed.  Subclasses
    provide ``_handles()`` (the handles stepped here) and ``_exchange()``."""

    period: int
    _fresh: int = 0

    def _advance(self, hd, c: int):
        hd.step(c)   # the library binding raises on a non-zero status

    def step(self, n: int = 1):
        n = int(n)
        if n < 0:
            raise ValueError("n < 0")
        while n > 0:
            c = min(n, self.period - self._fresh)
            for hd in self._handles():
                self._advance(hd, c)
            self._fresh += c
            n -= c
            if self._fresh == self.period:
                self._exchange()

    def refresh(self):
        """Bring the outer rows up to date (before diagnostics that read neighbours)."""
        if self._fresh:
            self._exchange()


class LocalSlabs(_Stepper):
    """An ny-row periodic D2Q9 lattice held as ``parts`` slabs in this process.

    ``sim_kwargs`` are those of ``Simulation`` (ncomp, tau, chi, m, theta, kappa, force,
    precision, kernel, forcing_velocity, force_form); ``edges`` is "walls" or "periodic"
    (the slab handles' edges, see the module docstring).  Every slab handle and band buffer
    lives on one stream: ``stream`` (a cudaStream_t as an integer) or, if it is None or 0,
    a stream made here (``self.stream``, a torch stream); the caller orders other work
    with it.  ``make_handle(rows)`` and ``new_buffer(nbytes)`` replace the library handles
    and the device band buffers (tests run the same logic over other stepping objects)."""

    def __init__(self, nx: int, ny: int, parts: int, period: int = 1, stream=None,
                 make_handle: Optional[Callable[[int], object]] = None,
                 new_buffer: Optional[Callable[[int], object]] = None, edges: str = "walls",
                 **sim_kwargs):
        self.nx, self.ny, self.parts, self.period = int(nx), int(ny), int(parts), int(period)
        if self.period < 1:
            raise ValueError("period >= 1")
        self.stream = None
        if make_handle is None:
            self.stream = _common_stream(stream)
            make_handle = _simulation_factory(nx, sim_kwargs, self.stream.cuda_stream, edges)
            new_buffer = new_buffer or _device_buffers(self.stream)
        if new_buffer is None:
            raise ValueError("new_buffer is needed with make_handle")
        G = REACH * self.period
        self.slabs = []
        for y0, h in split_rows(self.ny, self.parts):
            if h < G:
                raise ValueError(f"a slab of {h} rows cannot send {G} own rows (period "
                                 f"{self.period}): use fewer slabs or a shorter period")
            self.slabs.append(Slab(make_handle(h + 2 * G), nx, ny, y0, h, period, new_buffer))
        self._fresh = 0

    def _handles(self):
        return [s.handle for s in self.slabs]

    def _exchange(self):
        # every handle and buffer is on one stream, so the unpacks follow the packs
        for s in self.slabs:
            s.pack()
        P = len(self.slabs)
        for r, s in enumerate(self.slabs):
            s.unpack(self.slabs[(r - 1) % P].send_up, self.slabs[(r + 1) % P].send_down)
        self._fresh = 0

    def init_fields(self, rho, u=None):
        for s in self.slabs:
            s.init_fields(rho, u)
        self._exchange()   # the extended handles' own wrap-around touched their outer rows

    def set_state(self, f):
        for s in self.slabs:
            s.set_state(f)
        self._exchange()

    def get_state(self) -> np.ndarray:
        return np.concatenate([s.own(s.handle.get_state()) for s in self.slabs], axis=-2)

    def moments(self) -> dict:
        self.refresh()
        parts = [s.handle.moments() for s in self.slabs]
        return {k: np.concatenate([s.own(p[k]) for s, p in zip(self.slabs, parts)], axis=-2)
                for k in parts[0]}

    def conservation(self) -> dict:
        """FP64 sums over the lattice: each slab's own rows, added slab by slab."""
        self.refresh()
        out = None
        for s in self.slabs:
            c = s.handle.conservation_rows(s.G, s.h)
            out = c if out is None else {k: out[k] + c[k] for k in out}
        return out

    def status(self) -> List[int]:
        return [s.handle.status() for s in self.slabs]

    def close(self):
        for s in self.slabs:
            close = getattr(s.handle, "close", None)
            if close:
                close()


class SlabDecomposition(_Stepper):
    """This rank's slab of an ny-row periodic D2Q9 lattice split over a process group.

    Rank r of the group holds rows split_rows(ny, world)[r]; its neighbours are ranks r - 1
    (below) and r + 1 (above), periodically.  Bands move by point-to-point sends and
    receives on the group (NCCL: device buffers, issued with the handle's stream as torch's
    current stream, so that the sends follow the packs and the unpacks follow the
    receives; gloo: the buffers ``new_buffer`` makes).  With one rank the slab is its own
    neighbour and the bands are copied in place.
    ``reduce_device`` holds the all-reduced FP64 sums ("cuda" for NCCL, "cpu" for gloo by
    default).  Other arguments as ``LocalSlabs``."""

    def __init__(self, nx: int, ny: int, period: int = 1, group=None, stream=None,
                 make_handle: Optional[Callable[[int], object]] = None,
                 new_buffer: Optional[Callable[[int], object]] = None,
                 reduce_device: Optional[str] = None, edges: str = "walls", **sim_kwargs):
        import torch
        import torch.distributed as dist

        self.dist, self.torch, self.group = dist, torch, group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.nx, self.ny, self.period = int(nx), int(ny), int(period)
        if self.period < 1:
            raise ValueError("period >= 1")
        backend = dist.get_backend(group)
        self.stream = None
        if make_handle is None:
            self.stream = _common_stream(stream)
            make_handle = _simulation_factory(nx, sim_kwargs, self.stream.cuda_stream, edges)
            new_buffer = new_buffer or _device_buffers(self.stream)
        if new_buffer is None:
            raise ValueError("new_buffer is needed with make_handle")
        self.reduce_device = reduce_device or ("cuda" if backend == "nccl" else "cpu")
        G = REACH * self.period
        split = split_rows(self.ny, self.world)
        short = [r for r, (_, h) in enumerate(split) if h < G]
        if short:   # every rank raises, so that none waits on a peer that gave up
            raise ValueError(f"slabs of ranks {short} have fewer than {G} rows (period "
                             f"{self.period}): use fewer ranks or a shorter period")
        y0, h = split[self.rank]
        self.slab = Slab(make_handle(h + 2 * G), nx, ny, y0, h, period, new_buffer,
                         receive=self.world > 1)
        self._fresh = 0
        self._error = 0

    def _advance(self, hd, c: int):
        """Steps do not raise between exchanges: a rank that stopped here would leave its
        neighbours waiting for its bands.  The first non-zero status (the binding's
        step_nocheck returns it) is kept, and status() reports it on every rank."""
        nocheck = getattr(hd, "step_nocheck", None)
        rc = nocheck(c) if nocheck else hd.step(c)
        if rc and not self._error:
            self._error = int(rc)

    def _peer(self, r: int) -> int:
        r %= self.world
        return r if self.group is None else self.dist.get_global_rank(self.group, r)

    def _handles(self):
        return [self.slab.handle]

    def _exchange(self):
        s = self.slab
        with _on(self.stream):
            s.pack()
            if self.world == 1:
                s.unpack(s.send_up, s.send_down)
            else:
                d = self.dist
                up, down = self._peer(self.rank + 1), self._peer(self.rank - 1)
                # per peer, sends and receives are matched in issue order: the band going
                # up (tag 0) before the band going down (tag 1) on both sides
                ops = [d.P2POp(d.isend, s.send_up, up, self.group, 0),
                       d.P2POp(d.isend, s.send_down, down, self.group, 1),
                       d.P2POp(d.irecv, s.recv_below, down, self.group, 0),
                       d.P2POp(d.irecv, s.recv_above, up, self.group, 1)]
                for req in d.batch_isend_irecv(ops):
                    req.wait()
                s.unpack(s.recv_below, s.recv_above)
        self._fresh = 0

    @property
    def rows(self) -> Tuple[int, int]:
        """(first lattice row, rows) of this rank's slab."""
        return self.slab.y0, self.slab.h

    def init_fields(self, rho, u=None):
        """rho (N, ny, nx), u (2, ny, nx) or None: the whole lattice's fields (every rank
        passes the same arrays; each takes its rows)."""
        self.slab.init_fields(rho, u)
        self._exchange()

    def set_state(self, f):
        """f (N, 9, ny, nx): the whole lattice's pre-collision populations."""
        self.slab.set_state(f)
        self._exchange()

    def get_state(self) -> np.ndarray:
        """Pre-collision populations of this rank's rows, (N, 9, h, nx)."""
        return self.slab.own(self.slab.handle.get_state())

    def moments(self) -> dict:
        """Macroscopic fields of this rank's rows (collective)."""
        self.refresh()
        m = self.slab.handle.moments()
        return {k: np.ascontiguousarray(self.slab.own(v)) for k, v in m.items()}

    def gather_moments(self, root: int = 0) -> Optional[dict]:
        """The whole lattice's macroscopic fields on rank ``root`` of the group, None on the
        other ranks (collective; the slabs' rows are sent as pickled host arrays, for output;
        with NCCL the current CUDA device must be this rank's)."""
        mine = (self.slab.y0, self.moments())
        parts = [None] * self.world if self.rank == root else None
        dst = root if self.group is None else self.dist.get_global_rank(self.group, root)
        self.dist.gather_object(mine, parts, dst=dst, group=self.group)
        if self.rank != root:
            return None
        parts.sort(key=lambda p: p[0])
        return {k: np.concatenate([p[1][k] for p in parts], axis=-2) for k in parts[0][1]}

    def conservation(self) -> dict:
        """FP64 sums over the whole lattice (collective): each rank's own rows, all-reduced."""
        self.refresh()
        s = self.slab
        c = s.handle.conservation_rows(s.G, s.h)
        n = len(c["mass"])
        with _on(self.stream):
            t = self.torch.tensor(np.concatenate([c["mass"], c["mom"], c["force"]]),
                                  dtype=self.torch.float64, device=self.reduce_device)
            self.dist.all_reduce(t, group=self.group)
            v = t.cpu().numpy()
        return dict(mass=v[:n], mom=v[n:n + 2], force=v[n + 2:n + 4])

    def status(self) -> int:
        """Device status over the whole group (collective): 0, or the smallest (negative)
        MCLB_E* code any rank's handle has reported since it was created."""
        local = min(int(self.slab.handle.status() or 0), self._error)
        with _on(self.stream):
            t = self.torch.tensor([local], dtype=self.torch.int64, device=self.reduce_device)
            self.dist.all_reduce(t, op=self.dist.ReduceOp.MIN, group=self.group)
            return int(t.item())

    def close(self):
        close = getattr(self.slab.handle, "close", None)
        if close:
            close()
