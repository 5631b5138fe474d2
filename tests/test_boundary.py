"""The C ABI boundary without a GPU: the library loads, exports every entry point that
include/mclb.h declares, and rejects bad arguments before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_0704_3444_gb300 as mclb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mclb.h")


@pytest.fixture(scope="module")
def lib():
    mclb.build()
    return mclb.load()


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mclb_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared()
    for n in ("mclb_create", "mclb_init_fields", "mclb_step", "mclb_moments", "mclb_destroy",
              "mclb_conservation", "mclb_get_state", "mclb_set_state", "mclb_batch_create",
              "mclb_batch_step", "mclb_last_error"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def _params(**kw):
    base = dict(ncomp=2, nx=8, ny=8, tau=1.0, chi=np.array([[0.0, 2.2], [2.2, 0.0]]))
    base.update(kw)
    return mclb.make_params(**base)


@pytest.mark.parametrize("kw,frag", [
    (dict(ncomp=0, chi=np.zeros((0, 0))), "ncomp"),
    (dict(ncomp=9, chi=np.zeros((9, 9))), "ncomp"),
    (dict(nx=0), "grid"),
    (dict(tau=0.5), "tau"),
    (dict(tau=float("nan")), "tau"),
    (dict(chi=np.array([[0.0, 2.2], [2.1, 0.0]])), "symmetric"),
    (dict(chi=np.array([[0.0, np.inf], [np.inf, 0.0]])), "finite"),
    (dict(m=np.array([1.0, 0.0])), "m[1]"),
    (dict(kappa=-1.0), "kappa"),
    (dict(precision=7), "precision"),
    (dict(kernel=5), "kernel"),
    (dict(forcing_velocity=2), "forcing_velocity"),
    (dict(lattice="d1q3", ny=2), "ny = 1"),
    (dict(lattice="d1q3", ny=1, precision="bf16"), "FP64 or FP32"),
    (dict(force_form=2), "force_form"),
    (dict(force_form=1, kappa=0.01), "kappa = 0"),
    (dict(mass_every=-1), "mass_every"),
    (dict(lattice=3), "lattice"),
    (dict(walls=2), "walls"),
    (dict(walls=1, lattice="d1q3", ny=1), "D2Q9 option"),
    (dict(lattice="d3q19", nz=2, precision="bf16"), "FP64 or FP32"),
    (dict(nz=2), "D3Q19"),
    (dict(nz=-1), "nz"),
    (dict(force=(0.0, 0.0, 1e-5)), "force_z"),
    (dict(lattice="d3q19", nz=4, force=(0.0, 0.0, float("inf"))), "force_z"),
])
def test_invalid_parameters_are_rejected(lib, kw, frag):
    p, keep = _params(**kw)
    h = ctypes.c_void_p()
    rc = lib.mclb_create(ctypes.byref(p), ctypes.byref(h))
    assert rc == -1 and not h.value
    assert frag in lib.mclb_last_error().decode()


def test_batches_and_noalloc_reject_walls(lib):
    p, keep = _params(walls=1)
    b = ctypes.c_void_p()
    assert lib.mclb_batch_create(ctypes.byref(p), 1, ctypes.byref(b)) == -1 and not b.value
    assert "periodic" in lib.mclb_last_error().decode()
    p, keep = _params(walls=1, precision="fp64")
    assert lib.mclb_step_noalloc(ctypes.byref(p), None, None) == -1
    assert "periodic" in lib.mclb_last_error().decode()


def test_batches_reject_d3q19(lib):
    p, keep = _params(lattice="d3q19", nz=3)
    b = ctypes.c_void_p()
    assert lib.mclb_batch_create(ctypes.byref(p), 1, ctypes.byref(b)) == -1 and not b.value
    assert "D2Q9 and D1Q3" in lib.mclb_last_error().decode()


def test_mass_compensation_is_for_single_handles(lib):
    """A non-zero mass_every is refused where there is no handle step to follow: in a
    batch and in the allocation-free single step (checked before any device call)."""
    p, keep = _params(mass_every=8)
    b = ctypes.c_void_p()
    assert lib.mclb_batch_create(ctypes.byref(p), 1, ctypes.byref(b)) == -1 and not b.value
    assert "mass_every" in lib.mclb_last_error().decode()
    p, keep = _params(mass_every=8, precision="fp64")
    assert lib.mclb_step_noalloc(ctypes.byref(p), None, None) == -1
    assert "mass_every" in lib.mclb_last_error().decode()


def test_null_and_foreign_handles(lib):
    assert lib.mclb_step(None, 1) == -6
    assert lib.mclb_status(None) == -6
    assert lib.mclb_destroy(None) == 0
    assert lib.mclb_batch_step(None, 1) == -6
    assert lib.mclb_step_count(None) == -1
    h = ctypes.c_void_p()
    assert lib.mclb_create(None, ctypes.byref(h)) == -1
    assert lib.mclb_create(ctypes.byref(_params()[0]), None) == -1
    # the band calls check the handle before anything else
    assert lib.mclb_rows_bytes(None, 3) == 0
    assert lib.mclb_pack_rows_device(None, 0, 3, None) == -6
    assert lib.mclb_unpack_rows_device(None, 0, 3, None) == -6
    assert lib.mclb_conservation_rows(None, 0, 3, None, None, None) == -6


def test_binding_checks_field_sizes():
    """The binding refuses initial fields whose sizes do not match the handle (the C call
    would read N*ny*nx and 2*ny*nx doubles from the host pointers)."""
    rho, u = np.full((3, 4, 5), 1 / 3), np.zeros((2, 4, 5))
    r, v = mclb._fields(rho, u, 3, 4, 5)
    assert r.flags["C_CONTIGUOUS"] and r.dtype == np.float64 and v.shape == (2, 4, 5)
    assert mclb._fields(rho, None, 3, 4, 5)[1] is None
    with pytest.raises(ValueError, match="rho has 60 values, expected 80"):
        mclb._fields(rho, u, 4, 4, 5)
    with pytest.raises(ValueError, match="u has 20 values, expected 40"):
        mclb._fields(rho, np.zeros((1, 4, 5)), 3, 4, 5)
