"""CPU-side checks of the C ABI: the library builds, loads, exports every symbol declared in
include/*.h, and validates arguments (these paths return before any CUDA call)."""
import ctypes
import glob
import os
import re

import pytest

from paper_1909_05423_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        with open(h) as fh:
            txt = fh.read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names.update(re.findall(r"\b(pp_[a-z_0-9]+)\s*\(", txt))
    return sorted(names)


def test_exports_every_declared_symbol(lib):
    declared = _declared()
    assert "pp_solve" in declared and "pp_plan_create" in declared
    for name in declared:
        assert hasattr(lib, name), name
    assert set(_lib.EXPORTS) <= set(declared)


def test_version(lib):
    assert b"sm_103a" in lib.pp_version()


def _create(lib, nx, ny, nz, bc, dx=1.0, dtype=0):
    h = ctypes.c_void_p()
    st = lib.pp_plan_create(ctypes.byref(h), nx, ny, nz, _lib.bc_array(bc), dx, 1.0, 1.0, dtype, None)
    return st, h


@pytest.mark.parametrize("nx,ny,nz,bc,code", [
    (22, 8, 8, "PPPPDD", 2),     # 22 has the prime factor 11 (radices 2, 3, 5, 7 only)
    (9, 8, 8, "PPPPDD", 2),      # odd
    (8, 8, 1, "PPPPDD", 2),      # nz < 2
    (8, 8, 2, "NNNNPP", 2),      # periodic z needs nz >= 3
    (8192, 8, 8, "PPPPDD", 2),   # too long
    (2, 4096, 1 << 20, "NNNNDD", 2),  # 2^32 x lines in one launch
    (8, 8, 8, "PNPPDD", 3),      # periodic paired with Neumann
    (8, 8, 8, "PPNNDP", 3),
])
def test_validation(lib, nx, ny, nz, bc, code):
    st, h = _create(lib, nx, ny, nz, bc)
    assert st == code
    assert h.value is None
    assert len(lib.pp_last_error_string()) > 0


def test_invalid_spacing_and_dtype(lib):
    st, _ = _create(lib, 8, 8, 8, "PPPPDD", dx=0.0)
    assert st == 1
    st, _ = _create(lib, 8, 8, 8, "PPPPDD", dtype=7)
    assert st == 1
    bad = (ctypes.c_int * 6)(0, 0, 0, 0, 2, 5)
    h = ctypes.c_void_p()
    assert lib.pp_plan_create(ctypes.byref(h), 8, 8, 8, bad, 1.0, 1.0, 1.0, 0, None) == 1


def test_null_arguments(lib):
    assert lib.pp_solve(None, None, None, None) == 1
    assert lib.pp_solve_adjoint(None, None, None, None) == 1
    assert lib.pp_plan_destroy(None) == 0
    assert lib.pp_solve_batched(None, None, None, 0, None) == 0
    assert lib.pp_solve_batched(None, None, None, -1, None) == 1


def test_fold_bc_rejects_null_arguments(lib):
    vp = ctypes.c_void_p
    faces = (vp * 6)()
    assert lib.pp_fold_bc(None, None, None, faces, None) == 1  # PP_ERR_INVALID_ARG, no device work
    assert lib.pp_fold_bc(None, vp(16), vp(16), None, None) == 1


def test_fault_injection_alloc_fails_cleanly(lib, monkeypatch):
    """An injected allocation failure is reported as PP_ERR_OUT_OF_MEMORY with a message and no
    plan; the failure is made on the host before any device work (runs without a GPU)."""
    monkeypatch.setenv("PP_FAULT_INJECT", "alloc")
    st, h = _create(lib, 8, 8, 8, "PPPPDD")
    assert st == 4
    assert h.value is None
    assert b"injected" in lib.pp_last_error_string()


def test_z_method_validation(lib):
    """options.z_method: 2 (z transform) needs periodic z and a 7-smooth nz <= 4096; values outside
    0..2 are rejected.  Both checks return before any device work."""
    def create(nz, bc, zm):
        o = _lib.PlanOptions()
        o.z_method = zm
        h = ctypes.c_void_p()
        return lib.pp_plan_create(ctypes.byref(h), 8, 8, nz, _lib.bc_array(bc), 1.0, 1.0, 1.0, 0, ctypes.byref(o)), h
    for nz, bc, zm, code in ((37, "PPPPPP", 2, 2), (8, "PPPPDD", 2, 2), (8192, "PPPPPP", 2, 2),
                             (8, "PPPPPP", 3, 1), (8, "PPPPPP", -1, 1)):
        st, h = create(nz, bc, zm)
        assert st == code, (nz, bc, zm, st)
        assert h.value is None


def test_z_split_validation(lib):
    """options.z_split: 0, 1, 8, 16 or 32 (else PP_ERR_INVALID_ARG); a partitioned solve takes at
    most 512 chunks per line (else PP_ERR_UNSUPPORTED_SIZE); reserved must stay zero.  All three
    checks return before any device work."""
    def create(nz, zs, reserved=0):
        o = _lib.PlanOptions()
        o.z_split = zs
        o.reserved[0] = reserved
        h = ctypes.c_void_p()
        return lib.pp_plan_create(ctypes.byref(h), 8, 8, nz, _lib.bc_array("NNDDNN"), 1.0, 1.0, 1.0, 0,
                                  ctypes.byref(o)), h
    for nz, zs, res, code in ((64, 2, 0, 1), (64, 64, 0, 1), (64, -1, 0, 1), (64, 0, 1, 1),
                              (8 * 512 + 1, 8, 0, 2), (16 * 512 + 1, 16, 0, 2), (32 * 512 + 1, 32, 0, 2)):
        st, h = create(nz, zs, res)
        assert st == code, (nz, zs, res, st)
        assert h.value is None
