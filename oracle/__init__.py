"""FP64 CPU oracle of the symmetric free-energy multicomponent LB update.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only code allowed to import this
package.  The CUDA library never imports it and shares no code with it.

The lattice update itself is plain C (``mclb_oracle.c``), built with gcc on
first use into ``oracle/_build``; this module marshals numpy arrays to it.
``oracle.thermo`` holds the Flory-Huggins thermodynamics (binodals, critical
points) the paper compares its simulations against.

Three lattices, each a plain path of its own in the C file: D2Q9 (the
two-dimensional workloads), D1Q3 (the lattice of the paper's own simulations,
Sec. 4) and D3Q19 (three dimensions; the same equations on a lattice whose
weights give the same moments).
Optional solid walls in y on D2Q9 (``walls=1``; the paper has none): halfway
bounce-back of the populations and mirrored rows in the stencils.
Two readings of the velocity in the forcing's second moment (Eq. ff3):
``forcing_velocity=0`` is the component velocity u^s as printed (the default),
``forcing_velocity=1`` the barycentric u.  Two readings of the sum of the component
forces of Eq. definef: ``force_form=0`` as printed (the default), ``force_form=1`` the
Gibbs-Duhem total (kappa = 0 only).

Parity unpinned: none of the lattice-update functions; every stage is pinned
by tests against moment conditions, closed forms and independent numpy
transcriptions.  The floor of the logarithm in Eq. definef is pinned by the
rho -> lambda rho invariance with the floor binding and by bracketing where it
binds; the barycentric forcing reading by its transcription and by the one-fluid
sum of Eq. olso; the D1Q3 path by its moment-solving transcription and by the
one-row D2Q9 lattice it is the projection of; the D3Q19 path by its own moment
conditions, by the D2Q9 run that a z-, y- or x-invariant D3Q19 run projects onto
(summing the populations that share their in-plane velocity gives the D2Q9 weights,
equilibria, forcing and stencils exactly), by conservation, and by the ideal-mixture
diffusion rate of a mode along a body diagonal, which no two-dimensional run
reaches.  The paper's printed ternary critical points are not reproduced by the
symmetric-chi reading and are reported, not asserted.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mclb_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

NMAX = 8


class OracleParams(ctypes.Structure):
    _fields_ = [("ncomp", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("tau", ctypes.c_double), ("theta", ctypes.c_double),
                ("kappa", ctypes.c_double), ("gx", ctypes.c_double), ("gy", ctypes.c_double),
                ("chi", ctypes.c_double * (NMAX * NMAX)), ("m", ctypes.c_double * NMAX),
                ("forcing_velocity", ctypes.c_int), ("force_form", ctypes.c_int),
                ("nz", ctypes.c_int), ("gz", ctypes.c_double), ("walls", ctypes.c_int)]


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (OpenMP, no FP contraction so that x86 and
    Arm hosts round identically).  Returns the shared-library path."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            pp = ctypes.POINTER(OracleParams)
            lib.oracle_nthreads.restype = ctypes.c_int
            lib.oracle_equilibrium.argtypes = [ctypes.c_double] * 3 + [dp]
            lib.oracle_forcing.argtypes = [ctypes.c_double] * 5 + [dp]
            lib.oracle_psi.argtypes = [pp, dp]
            lib.oracle_psi.restype = ctypes.c_double
            lib.oracle_mu_bulk.argtypes = [pp, dp, dp]
            lib.oracle_init.argtypes = [pp, dp, dp, dp]
            lib.oracle_run.argtypes = [pp, dp, ctypes.c_long]
            lib.oracle_moments.argtypes = [pp, dp] + [dp] * 4
            lib.oracle_conservation.argtypes = [pp, dp, dp, dp, dp]
            lib.oracle_d1q3_init.argtypes = [pp, dp, dp, dp]
            lib.oracle_d1q3_run.argtypes = [pp, dp, ctypes.c_long]
            lib.oracle_d1q3_moments.argtypes = [pp, dp] + [dp] * 4
            lib.oracle_d1q3_conservation.argtypes = [pp, dp, dp, dp, dp]
            lib.oracle_d3q19_equilibrium.argtypes = [ctypes.c_double] * 4 + [dp]
            lib.oracle_d3q19_forcing.argtypes = [ctypes.c_double] * 7 + [dp]
            lib.oracle_d3q19_init.argtypes = [pp, dp, dp, dp]
            lib.oracle_d3q19_run.argtypes = [pp, dp, ctypes.c_long]
            lib.oracle_d3q19_moments.argtypes = [pp, dp] + [dp] * 4
            lib.oracle_d3q19_conservation.argtypes = [pp, dp, dp, dp, dp]
            _lib = lib
    return _lib


def _ptr(a: Optional[np.ndarray]):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def nthreads() -> int:
    return _load().oracle_nthreads()


class Oracle:
    """One oracle simulation: parameters plus the FP64 distribution array.

    D2Q9: ``f`` has shape (N, 9, ny, nx), pre-collision distributions at the
    current time, velocity order (0,0), (1,0), (0,1), (-1,0), (0,-1), (1,1),
    (-1,1), (-1,-1), (1,-1).  D1Q3 (``lattice="d1q3"``, ny must be 1): ``f`` has
    shape (N, 3, nx), velocity order 0, +1, -1; output fields keep the D2Q9
    shapes with ny = 1.  D3Q19 (``lattice="d3q19"``, ``nz`` layers): ``f`` has shape
    (N, 19, nz, ny, nx), velocity order 0; (+-1,0,0), (0,+-1,0), (0,0,+-1); (1,1,0),
    (-1,-1,0), (1,-1,0), (-1,1,0), (1,0,1), (-1,0,-1), (1,0,-1), (-1,0,1), (0,1,1),
    (0,-1,-1), (0,1,-1), (0,-1,1); fields have shape (., nz, ny, nx), U three
    components, P six (xx, xy, xz, yy, yz, zz), momentum and force sums three.
    """

    def __init__(self, ncomp, nx, ny, tau, chi, m=None, theta=1.0 / 3.0, kappa=0.0,
                 force=(0.0, 0.0), forcing_velocity=0, lattice="d2q9", force_form=0, nz=1,
                 walls=0):
        if lattice not in ("d2q9", "d1q3", "d3q19"):
            raise ValueError(f"lattice {lattice!r}")
        if lattice == "d1q3" and int(ny) != 1:
            raise ValueError("a D1Q3 lattice has ny = 1")
        if lattice != "d3q19" and int(nz) != 1:
            raise ValueError("nz > 1 needs the D3Q19 lattice")
        if walls and lattice != "d2q9":
            raise ValueError("walls are a D2Q9 option")
        self.lattice = lattice
        self.lib = _load()
        p = OracleParams()
        p.ncomp, p.nx, p.ny = int(ncomp), int(nx), int(ny)
        p.tau, p.theta, p.kappa = float(tau), float(theta), float(kappa)
        p.gx, p.gy = float(force[0]), float(force[1])
        p.gz = float(force[2]) if len(force) > 2 else 0.0
        p.nz = int(nz)
        p.walls = int(walls)
        chi = np.asarray(chi, dtype=np.float64).reshape(ncomp, ncomp)
        for a in range(ncomp):
            for b in range(ncomp):
                p.chi[a * ncomp + b] = chi[a, b]
        m = np.ones(ncomp) if m is None else np.asarray(m, dtype=np.float64)
        for a in range(ncomp):
            p.m[a] = m[a]
        p.forcing_velocity = int(forcing_velocity)
        p.force_form = int(force_form)
        self.p = p
        self.ncomp, self.nx, self.ny, self.nz = int(ncomp), int(nx), int(ny), int(nz)
        self.f = np.zeros(self._fshape)

    @classmethod
    def from_problem(cls, prob):
        o = cls(prob.ncomp, prob.nx, prob.ny, prob.tau, prob.chi, prob.m, prob.theta,
                prob.kappa, prob.force, getattr(prob, "forcing_velocity", 0),
                getattr(prob, "lattice", "d2q9"), getattr(prob, "force_form", 0),
                getattr(prob, "nz", 1), getattr(prob, "walls", 0))
        o.init(prob.rho, prob.u)
        return o

    @property
    def _d1(self):
        return self.lattice == "d1q3"

    @property
    def _d3(self):
        return self.lattice == "d3q19"

    @property
    def _fshape(self):
        if self._d1:
            return (self.ncomp, 3, self.nx)
        if self._d3:
            return (self.ncomp, 19, self.nz, self.ny, self.nx)
        return (self.ncomp, 9, self.ny, self.nx)

    def _fn(self, name):
        prefix = "oracle_d1q3_" if self._d1 else ("oracle_d3q19_" if self._d3 else "oracle_")
        return getattr(self.lib, prefix + name)

    @property
    def _pp(self):
        return ctypes.byref(self.p)

    def init(self, rho, u=None):
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        uu = None if u is None else np.ascontiguousarray(u, dtype=np.float64)
        if self._d1 and uu is not None:
            uu = np.ascontiguousarray(uu.reshape(-1)[:self.nx])   # x component only
        rc = self._fn("init")(self._pp, _ptr(rho), _ptr(uu), _ptr(self.f))
        if rc:
            raise ValueError(f"oracle_init failed ({rc})")

    def set_state(self, f):
        self.f = np.ascontiguousarray(np.asarray(f, dtype=np.float64).reshape(self._fshape)).copy()

    def run(self, nsteps: int) -> int:
        rc = self._fn("run")(self._pp, _ptr(self.f), int(nsteps))
        if rc < 0:
            raise ValueError(f"oracle_run failed ({rc})")
        return rc

    def moments(self):
        N = self.ncomp
        S = (self.nz, self.ny, self.nx) if self._d3 else (self.ny, self.nx)
        nu, npp = (3, 6) if self._d3 else (2, 3)
        rho, U, mu, P = np.zeros((N,) + S), np.zeros((nu,) + S), np.zeros((N,) + S), np.zeros((npp,) + S)
        self._fn("moments")(self._pp, _ptr(self.f), _ptr(rho), _ptr(U), _ptr(mu), _ptr(P))
        return dict(rho=rho, U=U, mu=mu, P=P)

    def conservation(self):
        nd = 3 if self._d3 else 2
        mass, mom, fs = np.zeros(self.ncomp), np.zeros(nd), np.zeros(nd)
        self._fn("conservation")(self._pp, _ptr(self.f), _ptr(mass), _ptr(mom), _ptr(fs))
        return dict(mass=mass, mom=mom, force=fs)

    # per-site helpers used by the pins
    def psi(self, rs) -> float:
        rs = np.ascontiguousarray(rs, dtype=np.float64)
        return self.lib.oracle_psi(self._pp, _ptr(rs))

    def mu_bulk(self, rs):
        rs = np.ascontiguousarray(rs, dtype=np.float64)
        out = np.zeros(self.ncomp)
        self.lib.oracle_mu_bulk(self._pp, _ptr(rs), _ptr(out))
        return out


def equilibrium(rho_s, ux, uy):
    out = np.zeros(9)
    _load().oracle_equilibrium(float(rho_s), float(ux), float(uy), _ptr(out))
    return out


def forcing(rho_s, jx, jy, ax, ay):
    out = np.zeros(9)
    _load().oracle_forcing(float(rho_s), float(jx), float(jy), float(ax), float(ay), _ptr(out))
    return out


def equilibrium3(rho_s, ux, uy, uz):
    out = np.zeros(19)
    _load().oracle_d3q19_equilibrium(float(rho_s), float(ux), float(uy), float(uz), _ptr(out))
    return out


def forcing3(rho_s, jx, jy, jz, ax, ay, az):
    out = np.zeros(19)
    _load().oracle_d3q19_forcing(float(rho_s), float(jx), float(jy), float(jz), float(ax),
                                 float(ay), float(az), _ptr(out))
    return out
