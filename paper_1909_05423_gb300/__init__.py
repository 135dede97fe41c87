"""GB300-native FFT / tridiagonal Poisson solver: the hot path of PittPack (arXiv 1909.05423).

Solves the cell-centred 7-point discretisation of Laplacian(u) = f on an nx x ny x nz grid
(Sec. "Mathematical Formulation") by x/y line transforms chosen per boundary condition, one
tridiagonal solve along z per (kx,ky) pair, and inverse transforms -- all in hand-written
sm_103a kernels behind the C ABI of ``include/pittpack_gb.h``.  This module only marshals
torch tensors (device memory, streams) into that ABI.

Boundary conditions are a 6-letter string over faces x-, x+, y-, y+, z-, z+ with ``P``
(periodic, both faces of an axis), ``N`` (Neumann) or ``D`` (Dirichlet); faces are
homogeneous unless face data are folded in (``Plan.fold_bc``).  Grids are tensors of shape
(nz, ny, nx).
"""
from __future__ import annotations

import ctypes

from . import _lib

__all__ = ["Plan", "solve", "solve_batched", "PoissonSolve", "PPError", "version"]

PPError = _lib.PPError


def version() -> str:
    return _lib.load().pp_version().decode()


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Plan:
    """A solver plan for one grid shape, boundary set, spacing and arithmetic mode.

    dtype: "f64" (FP64 I/O, double-float arithmetic), "mixed_f64io" (FP64 I/O, FP32
    transforms) or "mixed_f32io" (FP32 I/O, FP32 transforms).
    """

    def __init__(self, shape, bc: str, spacing=(1.0, 1.0, 1.0), dtype: str = "f64", options=None):
        lib = _lib.load()
        nz, ny, nx = (int(v) for v in shape)
        if dtype not in _lib.DTYPES:
            raise ValueError("dtype must be one of %s" % list(_lib.DTYPES))
        self.shape = (nz, ny, nx)
        self.bc = bc
        self.spacing = tuple(float(s) for s in spacing)
        self.dtype = dtype
        opt = None
        if options:
            o = _lib.PlanOptions()
            for k, v in options.items():
                setattr(o, k, int(v))
            opt = ctypes.byref(o)
        h = ctypes.c_void_p()
        _lib.check(lib.pp_plan_create(ctypes.byref(h), nx, ny, nz, _lib.bc_array(bc), *self.spacing,
                                      _lib.DTYPES[dtype], opt))
        self._h = h

    @property
    def handle(self):
        return self._h

    @property
    def io_dtype(self):
        import torch
        return torch.float32 if self.dtype == "mixed_f32io" else torch.float64

    def _check_tensor(self, t, name):
        import torch
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise TypeError("%s must be a CUDA tensor" % name)
        if tuple(t.shape) != self.shape or t.dtype != self.io_dtype or not t.is_contiguous():
            raise ValueError("%s must be a contiguous %s tensor of shape %s" % (name, self.io_dtype, self.shape))

    def _call(self, fn, f, out, stream):
        import torch
        self._check_tensor(f, "f")
        if out is None:
            out = torch.empty_like(f)
        self._check_tensor(out, "out")
        _lib.check(fn(self._h, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                      _stream_handle(stream)))
        return out

    def solve(self, f, out=None, stream=None):
        """u with A_h u = f (zero-mean u for f - mean f when no face is Dirichlet)."""
        return self._call(_lib.load().pp_solve, f, out, stream)

    def solve_refined(self, f, out=None, stream=None):
        """Mixed precision plus one FP64 residual-refinement step (mixed_f64io plans)."""
        return self._call(_lib.load().pp_solve_refined, f, out, stream)

    def solve_adjoint(self, g, out=None, stream=None):
        """S^T g through the transposed pipeline."""
        return self._call(_lib.load().pp_solve_adjoint, g, out, stream)

    def solve_host(self, f_host, out_host=None, stream=None):
        """Solve on host (CPU, ideally pinned) tensors; copies in and out inside the call."""
        import torch
        if f_host.is_cuda or tuple(f_host.shape) != self.shape or f_host.dtype != self.io_dtype:
            raise ValueError("f_host must be a host tensor of shape %s and dtype %s" % (self.shape, self.io_dtype))
        f_host = f_host.contiguous()
        if out_host is None:
            out_host = torch.empty_like(f_host)
        _lib.check(_lib.load().pp_solve_host(self._h, ctypes.c_void_p(f_host.data_ptr()),
                                             ctypes.c_void_p(out_host.data_ptr()), _stream_handle(stream)))
        return out_host

    def face_shapes(self):
        """Shapes of the face-data arrays, faces x-, x+, y-, y+, z-, z+."""
        nz, ny, nx = self.shape
        return [(nz, ny), (nz, ny), (nz, nx), (nz, nx), (ny, nx), (ny, nx)]

    def fold_bc(self, f, faces, out=None, stream=None):
        """Source of the homogeneous problem equivalent to faces with data: faces = 6 entries
        (x-, x+, y-, y+, z-, z+), None for a homogeneous face, else a CUDA tensor of the face's
        shape (``face_shapes``) holding the Dirichlet face values or the Neumann outward normal
        derivatives.  out may be f (in place)."""
        import torch
        self._check_tensor(f, "f")
        if out is None:
            out = torch.empty_like(f)
        self._check_tensor(out, "out")
        if len(faces) != 6:
            raise ValueError("faces must have 6 entries (x-, x+, y-, y+, z-, z+)")
        ptrs = (ctypes.c_void_p * 6)()
        for i, (g, shp) in enumerate(zip(faces, self.face_shapes())):
            if g is None:
                continue
            if (not isinstance(g, torch.Tensor) or not g.is_cuda or tuple(g.shape) != shp or g.dtype != self.io_dtype
                    or not g.is_contiguous()):
                raise ValueError("face %d data must be a contiguous CUDA %s tensor of shape %s" % (i, self.io_dtype, shp))
            ptrs[i] = g.data_ptr()
        _lib.check(_lib.load().pp_fold_bc(self._h, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                          ptrs, _stream_handle(stream)))
        return out

    def solve_bc(self, f, faces, out=None, stream=None):
        """Solve with faces with data: fold them into a copy of f, then solve."""
        return self.solve(self.fold_bc(f, faces, stream=stream), out=out, stream=stream)

    def status(self):
        _lib.check(_lib.load().pp_plan_status(self._h))

    def device_bytes(self) -> int:
        return int(_lib.load().pp_plan_device_bytes(self._h))

    def launch_shapes(self) -> dict:
        """(threads per CTA, lines per CTA) of the four line kernels."""
        v = (ctypes.c_int * 8)()
        _lib.check(_lib.load().pp_plan_launch_shapes(self._h, v))
        names = ["x-forward", "y-forward", "y-inverse", "x-inverse"]
        return {k: (v[2 * i], v[2 * i + 1]) for i, k in enumerate(names)}

    def z_method(self) -> str:
        """How z is solved: "thomas" (non-periodic z), "sherman-morrison" or "transform" (periodic z)."""
        v = ctypes.c_int()
        _lib.check(_lib.load().pp_plan_z_method(self._h, ctypes.byref(v)))
        return {0: "thomas", 1: "sherman-morrison", 2: "transform"}[v.value]

    def z_split(self) -> int:
        """Rows per chunk of the partitioned z solve (8, 16 or 32), or 1 for the Thomas sweeps."""
        v = ctypes.c_int()
        _lib.check(_lib.load().pp_plan_z_split(self._h, ctypes.byref(v)))
        return v.value

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.load().pp_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve(f, bc: str, spacing=(1.0, 1.0, 1.0), dtype: str = "f64", refined: bool = False, faces=None):
    """One-shot solve of Laplacian_h(u) = f on a CUDA tensor f of shape (nz, ny, nx); faces:
    optional face data (see Plan.fold_bc)."""
    plan = Plan(tuple(f.shape), bc, spacing, dtype)
    try:
        if faces is not None:
            f = plan.fold_bc(f, faces)
        return plan.solve_refined(f) if refined else plan.solve(f)
    finally:
        import torch
        torch.cuda.current_stream().synchronize()
        plan.close()


def solve_batched(plans, fs, outs=None, stream=None):
    """Enqueue len(plans) independent solves with one C call."""
    import torch
    n = len(plans)
    if outs is None:
        outs = [torch.empty_like(f) for f in fs]
    for p, f, o in zip(plans, fs, outs):
        p._check_tensor(f, "f")
        p._check_tensor(o, "out")
    arr = ctypes.c_void_p * max(n, 1)
    hp = arr(*[p.handle.value for p in plans])
    fp = arr(*[f.data_ptr() for f in fs])
    op = arr(*[o.data_ptr() for o in outs])
    _lib.check(_lib.load().pp_solve_batched(hp, fp, op, n, _stream_handle(stream)))
    return outs


def _poisson_solve_cls():
    import torch

    class PoissonSolve(torch.autograd.Function):
        """u = S f with dL/df = S^T dL/du, both through the CUDA pipeline."""

        @staticmethod
        def forward(ctx, f, plan):
            ctx.plan = plan
            return plan.solve(f.contiguous())

        @staticmethod
        def backward(ctx, grad_u):
            return ctx.plan.solve_adjoint(grad_u.contiguous()), None

    return PoissonSolve


class _Lazy:
    def __init__(self):
        self._cls = None

    def apply(self, f, plan):
        if self._cls is None:
            self._cls = _poisson_solve_cls()
        return self._cls.apply(f, plan)


PoissonSolve = _Lazy()
