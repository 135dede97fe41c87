"""CPU oracle for the FFT/tridiagonal Poisson solve (arXiv 1909.05423, PittPack).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The GPU
library never imports it, and it imports nothing from the GPU library.

The arithmetic lives in ``pp_oracle.c`` (plain C, FP64, naive O(N^2) line
transforms, textbook Thomas / Sherman-Morrison); this module only builds it
with gcc and marshals numpy arrays through ctypes.

Boundary conditions are given as a 6-letter string, one letter per face in
the order x-, x+, y-, y+, z-, z+: ``P`` periodic (both faces of an axis),
``N`` Neumann, ``D`` Dirichlet (homogeneous unless face data are given to the
``*_g`` / ``fold_bc`` functions).  Grids are real arrays of shape (nz, ny, nx), x
fastest.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pp_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libpp_oracle.so")
_lock = threading.Lock()
_lib = None

BC_CODE = {"P": 0, "N": 1, "D": 2}
# axis kinds, same numbering as pp_oracle.c
AX_P, AX_NN, AX_DD, AX_DN, AX_ND = 0, 1, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile pp_oracle.c into a shared library (gcc, OpenMP).  Returns its path."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O3", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-Wall", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            i64p = ctypes.POINTER(ctypes.c_int64)
            lib.oracle_solve.argtypes = [ctypes.c_int] * 3 + [ip] + [ctypes.c_double] * 3 + [dp, dp]
            lib.oracle_laplacian.argtypes = [ctypes.c_int] * 3 + [ip] + [ctypes.c_double] * 3 + [dp, dp]
            lib.oracle_laplacian_at.argtypes = ([ctypes.c_int] * 3 + [ip] + [ctypes.c_double] * 3 +
                                                [dp, i64p, ctypes.c_int64, dp])
            lib.oracle_line_forward.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp, dp]
            lib.oracle_line_inverse.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp, dp]
            lib.oracle_thomas.argtypes = [ctypes.c_int, dp, dp, dp, dp, dp]
            lib.oracle_cyclic.argtypes = [ctypes.c_int, dp, dp, dp, ctypes.c_double, ctypes.c_double, dp, dp]
            lib.oracle_eigenvalue.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
            lib.oracle_eigenvalue.restype = ctypes.c_double
            lib.oracle_axis_kind.argtypes = [ctypes.c_int, ctypes.c_int]
            lib.oracle_num_threads.argtypes = []
            dpp = ctypes.POINTER(dp)
            lib.oracle_laplacian_g.argtypes = [ctypes.c_int] * 3 + [ip] + [ctypes.c_double] * 3 + [dpp, dp, dp]
            lib.oracle_fold_bc.argtypes = [ctypes.c_int] * 3 + [ip] + [ctypes.c_double] * 3 + [dpp, dp, dp]
            _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _bc(bc: str):
    if len(bc) != 6 or any(c not in BC_CODE for c in bc):
        raise ValueError("bc must be 6 letters from P/N/D (faces x-,x+,y-,y+,z-,z+): %r" % (bc,))
    return (ctypes.c_int * 6)(*[BC_CODE[c] for c in bc])


def axis_kind(lo: str, hi: str) -> int:
    return _load().oracle_axis_kind(BC_CODE[lo], BC_CODE[hi])


def num_threads() -> int:
    return _load().oracle_num_threads()


def solve(f: np.ndarray, bc: str, spacing=(1.0, 1.0, 1.0)) -> np.ndarray:
    """u with A_h u = f (or, with no Dirichlet face, the zero-mean u with A_h u = f - mean f)."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    nz, ny, nx = f.shape
    u = np.empty_like(f)
    rc = _load().oracle_solve(nx, ny, nz, _bc(bc), *map(float, spacing), _dp(f), _dp(u))
    if rc != 0:
        raise ValueError("oracle_solve failed with code %d" % rc)
    return u


def laplacian(u: np.ndarray, bc: str, spacing=(1.0, 1.0, 1.0)) -> np.ndarray:
    """A_h u: the cell-centred 7-point Laplacian with the face ghost rules."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    nz, ny, nx = u.shape
    out = np.empty_like(u)
    rc = _load().oracle_laplacian(nx, ny, nz, _bc(bc), *map(float, spacing), _dp(u), _dp(out))
    if rc != 0:
        raise ValueError("oracle_laplacian failed with code %d" % rc)
    return out


def laplacian_at(u: np.ndarray, bc: str, spacing, idx: np.ndarray) -> np.ndarray:
    """A_h u at the given flat cell indices only."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    nz, ny, nx = u.shape
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    out = np.empty(idx.shape, dtype=np.float64)
    rc = _load().oracle_laplacian_at(nx, ny, nz, _bc(bc), *map(float, spacing), _dp(u),
                                     idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), idx.size, _dp(out))
    if rc != 0:
        raise ValueError("oracle_laplacian_at failed with code %d" % rc)
    return out


def _faces(faces, shape, bc):
    """Face data as a ctypes double** (None entries: homogeneous faces) plus the arrays kept alive."""
    nz, ny, nx = shape
    fshape = [(nz, ny), (nz, ny), (nz, nx), (nz, nx), (ny, nx), (ny, nx)]
    keep = []
    arr = (ctypes.POINTER(ctypes.c_double) * 6)()
    for i in range(6):
        v = None if faces is None else faces[i]
        if v is None:
            arr[i] = ctypes.POINTER(ctypes.c_double)()
            continue
        v = np.ascontiguousarray(v, dtype=np.float64)
        if v.shape != fshape[i]:
            raise ValueError("face %d data must have shape %s" % (i, fshape[i]))
        keep.append(v)
        arr[i] = _dp(v)
    return arr, keep


def laplacian_g(u: np.ndarray, bc: str, spacing, faces) -> np.ndarray:
    """L_g u: the 7-point Laplacian whose ghosts carry face data (Dirichlet values, Neumann
    outward normal derivatives); faces = 6 entries (x-,x+,y-,y+,z-,z+), None = homogeneous."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    nz, ny, nx = u.shape
    arr, keep = _faces(faces, u.shape, bc)
    out = np.empty_like(u)
    rc = _load().oracle_laplacian_g(nx, ny, nz, _bc(bc), *map(float, spacing), arr, _dp(u), _dp(out))
    if rc != 0:
        raise ValueError("oracle_laplacian_g failed with code %d" % rc)
    return out


def fold_bc(f: np.ndarray, bc: str, spacing, faces) -> np.ndarray:
    """f - L_g(0): the source of the homogeneous problem equivalent to L_g u = f."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    nz, ny, nx = f.shape
    arr, keep = _faces(faces, f.shape, bc)
    out = np.empty_like(f)
    rc = _load().oracle_fold_bc(nx, ny, nz, _bc(bc), *map(float, spacing), arr, _dp(f), _dp(out))
    if rc != 0:
        raise ValueError("oracle_fold_bc failed with code %d" % rc)
    return out


def solve_g(f: np.ndarray, bc: str, spacing, faces) -> np.ndarray:
    """u with L_g u = f (zero-mean u of the projected problem when no face is Dirichlet)."""
    return solve(fold_bc(f, bc, spacing, faces), bc, spacing)


def line_forward(kind: int, x: np.ndarray) -> np.ndarray:
    """Y_k = sum_n x_n b_k(n) for the axis kind's basis (complex in/out)."""
    x = np.asarray(x, dtype=np.complex128)
    n = x.size
    ir, ii = np.ascontiguousarray(x.real), np.ascontiguousarray(x.imag)
    orr, oi = np.empty(n), np.empty(n)
    if _load().oracle_line_forward(kind, n, _dp(ir), _dp(ii), _dp(orr), _dp(oi)) != 0:
        raise ValueError("bad line transform")
    return orr + 1j * oi


def line_inverse(kind: int, y: np.ndarray) -> np.ndarray:
    """x_n = sum_k c_k Y_k conj(b_k(n)) with c_k = 1/||b_k||^2."""
    y = np.asarray(y, dtype=np.complex128)
    n = y.size
    ir, ii = np.ascontiguousarray(y.real), np.ascontiguousarray(y.imag)
    orr, oi = np.empty(n), np.empty(n)
    if _load().oracle_line_inverse(kind, n, _dp(ir), _dp(ii), _dp(orr), _dp(oi)) != 0:
        raise ValueError("bad line transform")
    return orr + 1j * oi


def eigenvalue(kind: int, n: int, k: int) -> float:
    return _load().oracle_eigenvalue(kind, n, k)


def thomas(a, b, c, d) -> np.ndarray:
    a, b, c, d = (np.ascontiguousarray(v, dtype=np.float64) for v in (a, b, c, d))
    x = np.empty_like(d)
    _load().oracle_thomas(d.size, _dp(a), _dp(b), _dp(c), _dp(d), _dp(x))
    return x


def cyclic(a, b, c, alpha, beta, d) -> np.ndarray:
    a, b, c, d = (np.ascontiguousarray(v, dtype=np.float64) for v in (a, b, c, d))
    x = np.empty_like(d)
    _load().oracle_cyclic(d.size, _dp(a), _dp(b), _dp(c), float(alpha), float(beta), _dp(d), _dp(x))
    return x
