"""GB300 (sm_103a) symmetric free-energy multicomponent lattice Boltzmann.

A thin ctypes binding of ``libmclb.so`` (C ABI in ``include/mclb.h``).  Every
step of the method runs in the library's CUDA kernels; this module only
marshals arguments.  The library is built in-tree by ``build()`` and loaded on
first use; if it is missing the call raises -- there is no fallback.

Functions carry the C names (``mclb_create``, ``mclb_step`` ...).  The classes
``Simulation`` and ``Batch`` wrap a handle for convenience.  Host arrays are
numpy float64; device arrays may be torch tensors (float64, contiguous, on the
handle's device) passed to the ``*_device`` calls.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional, Sequence

import numpy as np

from ._build import LIB as _LIB_PATH
from ._build import build as _build

__all__ = ["build", "load", "Simulation", "Batch", "MclbError", "FP64", "FP32", "BF16_SHIFTED",
           "FP16_SHIFTED", "KERNEL_AUTO", "KERNEL_FUSED", "KERNEL_STAGED", "FORCING_COMPONENT",
           "FORCING_BARYCENTRIC", "FORCE_COMPONENT", "FORCE_GIBBS_DUHEM", "D2Q9", "D1Q3"]

FP64, FP32, BF16_SHIFTED, FP16_SHIFTED = 0, 1, 2, 3
KERNEL_AUTO, KERNEL_FUSED, KERNEL_STAGED = 0, 1, 2
FORCING_COMPONENT, FORCING_BARYCENTRIC = 0, 1
FORCE_COMPONENT, FORCE_GIBBS_DUHEM = 0, 1
D2Q9, D1Q3, D3Q19 = 0, 1, 2
LATTICES = {"d2q9": D2Q9, "d1q3": D1Q3, "d3q19": D3Q19}
PRECISIONS = {"fp64": FP64, "fp32": FP32, "bf16": BF16_SHIFTED, "fp16": FP16_SHIFTED}
NMAX = 8
STATUS = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ENONFINITE", -5: "ETIMEOUT",
          -6: "EHANDLE"}

_lock = threading.Lock()
_lib = None


class MclbError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class mclb_params(ctypes.Structure):
    _fields_ = [("ncomp", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("tau", ctypes.c_double), ("chi", ctypes.POINTER(ctypes.c_double)),
                ("m", ctypes.POINTER(ctypes.c_double)), ("theta", ctypes.c_double),
                ("kappa", ctypes.c_double), ("force", ctypes.c_double * 2),
                ("precision", ctypes.c_int), ("kernel", ctypes.c_int),
                ("stream", ctypes.c_void_p), ("forcing_velocity", ctypes.c_int),
                ("lattice", ctypes.c_int), ("force_form", ctypes.c_int),
                ("mass_every", ctypes.c_int), ("nz", ctypes.c_int), ("force_z", ctypes.c_double),
                ("walls", ctypes.c_int)]


def build(force: bool = False) -> str:
    return _build(force=force)


def load():
    """Load libmclb.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(f"{_LIB_PATH} is missing: build it with "
                               "paper_0704_3444_gb300.build() (needs nvcc)")
        lib = ctypes.CDLL(_LIB_PATH)
        H = ctypes.c_void_p
        dp = ctypes.POINTER(ctypes.c_double)
        sig = {
            "mclb_create": ([ctypes.POINTER(mclb_params), ctypes.POINTER(H)], ctypes.c_int),
            "mclb_init_fields": ([H, dp, dp], ctypes.c_int),
            "mclb_init_fields_device": ([H, ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
            "mclb_step": ([H, ctypes.c_long], ctypes.c_int),
            "mclb_test_withhold_copies": ([H, ctypes.c_int], ctypes.c_int),
            "mclb_status": ([H], ctypes.c_int),
            "mclb_moments": ([H, dp, dp, dp, dp], ctypes.c_int),
            "mclb_moments_device": ([H] + [ctypes.c_void_p] * 4, ctypes.c_int),
            "mclb_conservation": ([H, dp, dp, dp], ctypes.c_int),
            "mclb_fit_equilibrium": ([H, ctypes.c_int, dp], ctypes.c_int),
            "mclb_get_state": ([H, dp, ctypes.c_size_t], ctypes.c_int),
            "mclb_set_state": ([H, dp, ctypes.c_size_t], ctypes.c_int),
            "mclb_step_count": ([H], ctypes.c_long),
            "mclb_bytes_per_step": ([H], ctypes.c_double),
            "mclb_launches_per_step": ([H], ctypes.c_int),
            "mclb_destroy": ([H], ctypes.c_int),
            "mclb_last_error": ([], ctypes.c_char_p),
            "mclb_batch_create": ([ctypes.POINTER(mclb_params), ctypes.c_int, ctypes.POINTER(H)],
                                  ctypes.c_int),
            "mclb_batch_init_fields": ([H, ctypes.c_int, dp, dp], ctypes.c_int),
            "mclb_batch_step": ([H, ctypes.c_long], ctypes.c_int),
            "mclb_batch_moments": ([H, ctypes.c_int, dp, dp, dp, dp], ctypes.c_int),
            "mclb_batch_get_state": ([H, ctypes.c_int, dp, ctypes.c_size_t], ctypes.c_int),
            "mclb_batch_fit_equilibrium": ([H, ctypes.c_int, ctypes.c_int, dp], ctypes.c_int),
            "mclb_batch_status": ([H, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
            "mclb_batch_bytes_per_step": ([H], ctypes.c_double),
            "mclb_batch_launches_per_step": ([H], ctypes.c_int),
            "mclb_batch_tuning": ([H, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                   ctypes.c_int], ctypes.c_int),
            "mclb_test_batch_partition": ([H, ctypes.c_int, ctypes.c_int], ctypes.c_int),
            "mclb_batch_destroy": ([H], ctypes.c_int),
            "mclb_step_noalloc": ([ctypes.POINTER(mclb_params), ctypes.c_void_p, ctypes.c_void_p],
                                  ctypes.c_int),
            "mclb_rows_bytes": ([H, ctypes.c_int], ctypes.c_size_t),
            "mclb_pack_rows_device": ([H, ctypes.c_int, ctypes.c_int, ctypes.c_void_p], ctypes.c_int),
            "mclb_unpack_rows_device": ([H, ctypes.c_int, ctypes.c_int, ctypes.c_void_p],
                                        ctypes.c_int),
            "mclb_conservation_rows": ([H, ctypes.c_int, ctypes.c_int, dp, dp, dp], ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def _check(rc: int, what: str = ""):
    if rc != 0:
        msg = load().mclb_last_error().decode(errors="replace")
        raise MclbError(rc, f"{what}: {msg}" if what else msg)
    return rc


def _dp(a: Optional[np.ndarray]):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"], "float64 C-contiguous array needed"
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _tensor_ptr(t) -> Optional[int]:
    if t is None:
        return None
    return int(t.data_ptr())


def _check_buf(buf, nbytes: int):
    if not buf.is_contiguous() or buf.numel() * buf.element_size() < nbytes:
        raise ValueError(f"band buffer must be contiguous with at least {nbytes} bytes")


def _fields(rho, u, ncomp, ny, nx, device=False, nz=1, ud=2):
    """Check the sizes of initial fields (the C call reads N*nz*ny*nx and ud*nz*ny*nx
    doubles; nz = 1 and ud = 2 except on D3Q19)."""
    if not device:
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        u = None if u is None else np.ascontiguousarray(u, dtype=np.float64)
    for name, a, want in (("rho", rho, ncomp * nz * ny * nx), ("u", u, ud * nz * ny * nx)):
        if a is None:
            continue
        n = a.numel() if device else a.size
        if n != want:
            raise ValueError(f"{name} has {n} values, expected {want} ({name} layout [k][y][x])")
        if device and (str(a.dtype) != "torch.float64" or not a.is_contiguous() or not a.is_cuda):
            raise ValueError(f"{name} must be a contiguous float64 CUDA tensor")
    return rho, u


def make_params(ncomp, nx, ny, tau, chi, m=None, theta=1.0 / 3.0, kappa=0.0, force=(0.0, 0.0),
                precision="fp32", kernel=KERNEL_AUTO, stream=None, forcing_velocity=0,
                lattice="d2q9", force_form=0, mass_every=0, nz=1, walls=0):
    """Build an mclb_params struct; returns (struct, keep-alive arrays).  ``force`` has
    two components, or three on D3Q19 (the third is force_z)."""
    chi = np.ascontiguousarray(np.asarray(chi, dtype=np.float64).reshape(ncomp, ncomp))
    marr = None if m is None else np.ascontiguousarray(np.asarray(m, dtype=np.float64))
    p = mclb_params()
    p.ncomp, p.nx, p.ny = int(ncomp), int(nx), int(ny)
    p.tau, p.theta, p.kappa = float(tau), float(theta), float(kappa)
    p.chi = _dp(chi)
    p.m = _dp(marr)
    p.force[0], p.force[1] = float(force[0]), float(force[1])
    p.force_z = float(force[2]) if len(force) > 2 else 0.0
    p.nz = int(nz)
    p.walls = int(walls)
    p.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    p.kernel = int(kernel)
    p.stream = ctypes.c_void_p(stream) if stream else None
    p.forcing_velocity = int(forcing_velocity)
    p.lattice = LATTICES[lattice] if isinstance(lattice, str) else int(lattice)
    p.force_form = int(force_form)
    p.mass_every = int(mass_every)
    return p, (chi, marr)


class Simulation:
    """One simulation handle (mclb_create ... mclb_destroy).  Fields are (., ny, nx), or
    (., nz, ny, nx) with three velocity and six pressure components on D3Q19."""

    def __init__(self, ncomp, nx, ny, tau, chi, m=None, theta=1.0 / 3.0, kappa=0.0,
                 force=(0.0, 0.0), precision="fp32", kernel=KERNEL_AUTO, stream=None,
                 forcing_velocity=0, lattice="d2q9", force_form=0, mass_every=0, nz=1, walls=0):
        self.lib = load()
        self.ncomp, self.nx, self.ny = int(ncomp), int(nx), int(ny)
        p, keep = make_params(ncomp, nx, ny, tau, chi, m, theta, kappa, force, precision, kernel,
                              stream, forcing_velocity, lattice, force_form, mass_every, nz, walls)
        self.q = {D1Q3: 3, D3Q19: 19}.get(p.lattice, 9)
        self.nz = max(int(nz), 1) if p.lattice == D3Q19 else 1
        self.ud = 3 if p.lattice == D3Q19 else 2
        h = ctypes.c_void_p()
        _check(self.lib.mclb_create(ctypes.byref(p), ctypes.byref(h)), "mclb_create")
        self.h = h

    @classmethod
    def from_problem(cls, prob, precision=None, kernel=KERNEL_AUTO, stream=None, mass_every=0):
        s = cls(prob.ncomp, prob.nx, prob.ny, prob.tau, prob.chi, prob.m, prob.theta, prob.kappa,
                prob.force, precision or prob.precision, kernel, stream,
                getattr(prob, "forcing_velocity", 0), getattr(prob, "lattice", "d2q9"),
                getattr(prob, "force_form", 0), mass_every, getattr(prob, "nz", 1),
                getattr(prob, "walls", 0))
        s.init_fields(prob.rho, prob.u)
        return s

    def close(self):
        if getattr(self, "h", None):
            self.lib.mclb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx) if self.q == 19 else (self.ny, self.nx)

    def init_fields(self, rho, u=None):
        rho, uu = _fields(rho, u, self.ncomp, self.ny, self.nx, nz=self.nz, ud=self.ud)
        _check(self.lib.mclb_init_fields(self.h, _dp(rho), _dp(uu)), "mclb_init_fields")

    def init_fields_device(self, rho_t, u_t=None):
        _fields(rho_t, u_t, self.ncomp, self.ny, self.nx, device=True, nz=self.nz, ud=self.ud)
        _check(self.lib.mclb_init_fields_device(self.h, _tensor_ptr(rho_t), _tensor_ptr(u_t)),
               "mclb_init_fields_device")

    def step(self, n: int = 1) -> int:
        return _check(self.lib.mclb_step(self.h, int(n)), "mclb_step")

    def step_nocheck(self, n: int = 1) -> int:
        return self.lib.mclb_step(self.h, int(n))

    def status(self) -> int:
        return self.lib.mclb_status(self.h)

    def moments(self, rho=True, U=True, mu=True, P=True):
        N, S = self.ncomp, self.shape
        npc = 6 if self.ud == 3 else 3
        out = dict(rho=np.empty((N,) + S) if rho else None,
                   U=np.empty((self.ud,) + S) if U else None,
                   mu=np.empty((N,) + S) if mu else None, P=np.empty((npc,) + S) if P else None)
        _check(self.lib.mclb_moments(self.h, _dp(out["rho"]), _dp(out["U"]), _dp(out["mu"]),
                                     _dp(out["P"])), "mclb_moments")
        return out

    def moments_device(self, rho=None, U=None, mu=None, P=None):
        _check(self.lib.mclb_moments_device(self.h, _tensor_ptr(rho), _tensor_ptr(U),
                                            _tensor_ptr(mu), _tensor_ptr(P)), "mclb_moments_device")

    def conservation(self):
        mass, mom, fs = np.empty(self.ncomp), np.empty(self.ud), np.empty(self.ud)
        _check(self.lib.mclb_conservation(self.h, _dp(mass), _dp(mom), _dp(fs)),
               "mclb_conservation")
        return dict(mass=mass, mom=mom, force=fs)

    def fit_equilibrium(self, nphase: int):
        out = np.empty((nphase, self.ncomp))
        _check(self.lib.mclb_fit_equilibrium(self.h, int(nphase), _dp(out)), "mclb_fit_equilibrium")
        return out

    # bands of rows (mclb_rows_bytes, mclb_pack_rows_device, ...): D2Q9 only
    def rows_bytes(self, nrows: int) -> int:
        return int(self.lib.mclb_rows_bytes(self.h, int(nrows)))

    def pack_rows(self, y0: int, nrows: int, buf):
        """Copy the stored rows [y0, y0 + nrows) into ``buf`` (a contiguous torch tensor of
        at least rows_bytes(nrows) bytes on the handle's device), in stream order."""
        _check_buf(buf, self.rows_bytes(nrows))
        _check(self.lib.mclb_pack_rows_device(self.h, int(y0), int(nrows), _tensor_ptr(buf)),
               "mclb_pack_rows_device")

    def unpack_rows(self, y0: int, nrows: int, buf):
        """Overwrite the stored rows [y0, y0 + nrows) from ``buf`` (as pack_rows)."""
        _check_buf(buf, self.rows_bytes(nrows))
        _check(self.lib.mclb_unpack_rows_device(self.h, int(y0), int(nrows), _tensor_ptr(buf)),
               "mclb_unpack_rows_device")

    def conservation_rows(self, y0: int, nrows: int):
        mass, mom, fs = np.empty(self.ncomp), np.empty(2), np.empty(2)
        _check(self.lib.mclb_conservation_rows(self.h, int(y0), int(nrows), _dp(mass), _dp(mom),
                                               _dp(fs)), "mclb_conservation_rows")
        return dict(mass=mass, mom=mom, force=fs)

    def get_state(self):
        """Pre-collision populations: (N, 9, ny, nx) on D2Q9, (N, 3, nx) on D1Q3,
        (N, 19, nz, ny, nx) on D3Q19."""
        if self.q == 3:
            f = np.empty((self.ncomp, 3, self.nx))
        else:
            f = np.empty((self.ncomp, self.q) + self.shape)
        _check(self.lib.mclb_get_state(self.h, _dp(f), f.size), "mclb_get_state")
        return f

    def set_state(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        _check(self.lib.mclb_set_state(self.h, _dp(f), f.size), "mclb_set_state")

    @property
    def step_count(self) -> int:
        return self.lib.mclb_step_count(self.h)

    def test_withhold_copies(self, on: bool):
        """Test hook (mclb_test_withhold_copies): single-pass steps issue no copies."""
        _check(self.lib.mclb_test_withhold_copies(self.h, int(bool(on))), "mclb_test_withhold_copies")

    @property
    def bytes_per_step(self) -> float:
        return self.lib.mclb_bytes_per_step(self.h)

    @property
    def launches_per_step(self) -> int:
        return self.lib.mclb_launches_per_step(self.h)


class Batch:
    """Independent simulations advanced together (mclb_batch_*)."""

    def __init__(self, problems: Sequence, precision="fp32", stream=None):
        self.lib = load()
        self.problems = list(problems)
        arr = (mclb_params * len(self.problems))()
        self._keep = []
        for k, pr in enumerate(self.problems):
            p, keep = make_params(pr.ncomp, pr.nx, pr.ny, pr.tau, pr.chi, pr.m, pr.theta, pr.kappa,
                                  pr.force, precision, KERNEL_AUTO, stream,
                                  getattr(pr, "forcing_velocity", 0), getattr(pr, "lattice", "d2q9"),
                                  getattr(pr, "force_form", 0))
            arr[k] = p
            self._keep.append(keep)
        h = ctypes.c_void_p()
        _check(self.lib.mclb_batch_create(arr, len(self.problems), ctypes.byref(h)),
               "mclb_batch_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.mclb_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_fields(self, index, rho, u=None):
        pr = self.problems[int(index)]
        rho, uu = _fields(rho, u, pr.ncomp, pr.ny, pr.nx)
        _check(self.lib.mclb_batch_init_fields(self.h, int(index), _dp(rho), _dp(uu)),
               "mclb_batch_init_fields")

    def init_all(self):
        for k, pr in enumerate(self.problems):
            self.init_fields(k, pr.rho, pr.u)

    def step(self, n=1):
        return _check(self.lib.mclb_batch_step(self.h, int(n)), "mclb_batch_step")

    def moments(self, index):
        pr = self.problems[index]
        S = (pr.ny, pr.nx)
        rho, U = np.empty((pr.ncomp,) + S), np.empty((2,) + S)
        _check(self.lib.mclb_batch_moments(self.h, int(index), _dp(rho), _dp(U), None, None),
               "mclb_batch_moments")
        return dict(rho=rho, U=U)

    def fit_equilibrium(self, index, nphase: int):
        out = np.empty((nphase, self.problems[index].ncomp))
        _check(self.lib.mclb_batch_fit_equilibrium(self.h, int(index), int(nphase), _dp(out)),
               "mclb_batch_fit_equilibrium")
        return out

    def get_state(self, index):
        pr = self.problems[index]
        q = 3 if getattr(pr, "lattice", "d2q9") == "d1q3" else 9
        f = np.empty((pr.ncomp, q, pr.nx) if q == 3 else (pr.ncomp, 9, pr.ny, pr.nx))
        _check(self.lib.mclb_batch_get_state(self.h, int(index), _dp(f), f.size),
               "mclb_batch_get_state")
        return f

    def status(self):
        per = (ctypes.c_int * len(self.problems))()
        rc = self.lib.mclb_batch_status(self.h, per)
        return rc, list(per)

    @property
    def bytes_per_step(self):
        return self.lib.mclb_batch_bytes_per_step(self.h)

    @property
    def launches_per_step(self):
        return self.lib.mclb_batch_launches_per_step(self.h)

    def tuning(self):
        """Per group of D2Q9 instances (ascending N): (narrow strips picked, waves)."""
        cap = 16
        nar, wav = (ctypes.c_int * cap)(), (ctypes.c_int * cap)()
        n = self.lib.mclb_batch_tuning(self.h, nar, wav, cap)
        if n < 0:
            raise MclbError(n, "mclb_batch_tuning")
        return [(bool(nar[k]), int(wav[k])) for k in range(min(n, cap))]

    def test_force_partition(self, narrow: bool, waves: int) -> int:
        """Test hook (mclb_test_batch_partition): groups that switched to the candidate."""
        n = self.lib.mclb_test_batch_partition(self.h, int(bool(narrow)), int(waves))
        if n < 0:
            raise MclbError(n, "mclb_test_batch_partition")
        return n
