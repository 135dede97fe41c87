"""The plan's device status word: the z solve's range report (pp_plan_status -> PP_ERR_RANGE).

The double-float and FP32 arithmetic have FP32's exponent range.  A source far below it (1e-32
on a unit-cube 32^3 grid: the scaled right-hand sides of the tridiagonal solves fall below
2^-100) or far above it (1e37: the transforms overflow) must be reported; sources inside the
range of full accuracy (1e-20, 1e25), Gaussian sources whose tails underflow FP64 itself, and the
zero source must not.  Reading the status clears it."""
import math

import numpy as np
import pytest

from paper_1909_05423_gb300 import _lib, workloads
from tests.gpu_common import need_gpu, rel_l2, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup(oracle):
    need_gpu()


def _solve_status(plan, f):
    """Solve, synchronise, read the status: None for PP_OK, else the PPError."""
    io = torch.float32 if plan.dtype == "mixed_f32io" else torch.float64
    ft = torch.from_numpy(np.ascontiguousarray(f)).to(device="cuda", dtype=io)
    u = plan.solve(ft)
    torch.cuda.synchronize()
    try:
        plan.status()
    except _lib.PPError as e:
        return u, e
    return u, None


@pytest.mark.parametrize("dtype", ["f64", "mixed_f64io"])
@pytest.mark.parametrize("bc", ["NNDDNN", "PPPPDD", "NNNNNN"])
def test_range_flag(oracle, dtype, bc):
    import paper_1909_05423_gb300 as pp
    n = 32
    shape = (n, n, n)
    sp = (1.0 / n,) * 3
    f = workloads.uniform_source(shape, seed=51)
    ref = oracle.solve(f, bc, sp)
    plan = pp.Plan(shape, bc, sp, dtype)
    tol = 1e-12 if dtype == "f64" else 1e-6
    for scale in (1e-20, 1e25, 1.0):
        u, err = _solve_status(plan, f * scale)
        assert err is None, (scale, err)
        assert rel_l2(u.cpu().numpy(), ref * scale) <= tol, scale
    for scale in (1e-32, 1e37):
        _, err = _solve_status(plan, f * scale)
        assert err is not None and err.status == _lib.PP_ERR_RANGE, (scale, err)
        # reading cleared it: a source in range reports nothing again
        _, err = _solve_status(plan, f)
        assert err is None, (scale, err)
    plan.close()


def test_range_flag_non_finite():
    import paper_1909_05423_gb300 as pp
    shape = (16, 16, 16)
    plan = pp.Plan(shape, "NNDDNN", (1.0 / 16,) * 3, "f64")
    f = workloads.uniform_source(shape, seed=52)
    for bad in (math.inf, math.nan):
        g = f.copy()
        g[3, 4, 5] = bad
        _, err = _solve_status(plan, g)
        assert err is not None and err.status == _lib.PP_ERR_RANGE, bad
    plan.close()


def test_range_flag_quiet_cases():
    """Gaussian blobs (tails far below FP32's range, to 1e-140) and the zero source."""
    import paper_1909_05423_gb300 as pp
    n = 64
    shape = (n, n, n)
    sp = (1.0 / n,) * 3
    amp, centre, width = workloads.gaussian_blobs(shape, sp, seed=5, count=4)
    f = workloads.blob_field(shape, sp, amp, centre, np.asarray(width) * 0.5)
    assert np.abs(f[f != 0]).min() < 1e-100  # far below FP32's range
    for dtype in ("f64", "mixed_f64io", "mixed_f32io"):
        plan = pp.Plan(shape, "PPPPDD", sp, dtype)
        for src in (f, np.zeros(shape)):
            _, err = _solve_status(plan, src)
            assert err is None, (dtype, err)
        plan.close()


def test_range_flag_z_transform():
    """The diagonal solve of periodic z by transform reports the same way."""
    import paper_1909_05423_gb300 as pp
    n = 32
    shape = (n, n, n)
    sp = (1.0 / n,) * 3
    f = workloads.uniform_source(shape, seed=53)
    plan = pp.Plan(shape, "PPPPPP", sp, "f64", options={"z_method": 2})
    assert plan.z_method() == "transform"
    for scale, flagged in ((1.0, False), (1e-20, False), (1e-32, True), (1e37, True), (1.0, False)):
        _, err = _solve_status(plan, f * scale)
        assert (err is not None) == flagged, (scale, err)
        if flagged:
            assert err.status == _lib.PP_ERR_RANGE
    plan.close()


def test_range_flag_ignores_stale_padding():
    """A plan's spectral rows end in padding slots that no transform writes; memory a closed plan
    left behind (here: NaN from a non-finite source) must reach neither the solution nor the range
    report of a new plan whose buffers reuse it."""
    import paper_1909_05423_gb300 as pp
    n = 32
    shape = (n, n, n)
    sp = (1.0 / n,) * 3
    f = workloads.uniform_source(shape, seed=54)
    for zm in (2, 1):
        for _ in range(3):
            old = pp.Plan(shape, "PPPPPP", sp, "f64", options={"z_method": zm})
            g = f.copy()
            g[:] = math.nan
            _solve_status(old, g)
            old.close()
            plan = pp.Plan(shape, "PPPPPP", sp, "f64", options={"z_method": zm})
            u, err = _solve_status(plan, f)
            assert err is None, (zm, err)
            assert np.isfinite(u.cpu().numpy()).all()
            _, err = _solve_status(plan, f * 1e-32)
            assert err is not None and err.status == _lib.PP_ERR_RANGE, zm
            plan.close()
