"""The partitioned z solve (options.z_split = 8 / 16 / 32 rows per chunk) against the CPU oracle,
element by element.  Shapes put the chunk boundaries everywhere a recurrence can go wrong: a line
shorter than one chunk (one chunk, no carries), lengths that are and are not multiples of the chunk,
chunk counts that are not powers of two (ragged recursive-doubling levels) and that round the CTA
up to whole warps, few modes on long lines (the setting of the paper's solver comparison: the
weakly dominant low modes carry their multiplier prefix over many chunks), every pair of
non-periodic z faces, singular problems (the pinned column is left to the Thomas sweep) and the
three precisions."""
import numpy as np
import pytest

from paper_1909_05423_gb300 import _lib, workloads
from tests.gpu_common import gpu_solve, need_gpu, rel_l2, torch

pytestmark = pytest.mark.gpu
TOL_F64 = 1e-12
TOL_MIXED = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _setup(oracle):
    need_gpu()


def _plan(shape, bc, sp, dtype="f64", **opt):
    import paper_1909_05423_gb300 as pp
    return pp.Plan(shape, bc, sp, dtype, options=opt or None)


@pytest.mark.parametrize("rows", [8, 16, 32])
@pytest.mark.parametrize("shape", [(5, 6, 8), (8, 10, 12), (37, 12, 10), (100, 8, 6), (256, 6, 4),
                                   (1023, 8, 8), (2047, 4, 6)])
@pytest.mark.parametrize("bc", ["NNDDNN", "DDNNDD", "PPDDND", "NDPPDN", "NNNNNN"])
def test_partitioned_matches_oracle(oracle, rows, shape, bc):
    nz, ny, nx = shape
    sp = (1.0 / nx, 1.0 / ny, 1.0 / nz)
    f = workloads.uniform_source(shape, seed=nz + rows, remove_mean=False)
    ref = oracle.solve(f, bc, sp)
    opt = dict(z_split=rows)
    u = gpu_solve(f, bc, sp, options=opt)
    assert rel_l2(u, ref) <= TOL_F64, rel_l2(u, ref)
    for dtype in ("mixed_f64io", "mixed_f32io"):
        um = gpu_solve(f, bc, sp, dtype, options=opt)
        assert rel_l2(um, ref) <= TOL_MIXED, (dtype, rel_l2(um, ref))


@pytest.mark.parametrize("bc", ["NNDDNN", "NNNNDD", "DNDNND", "NNNNNN"])
def test_partitioned_long_lines_low_modes(oracle, bc):
    """4095 rows (the paper's longest PCR line) on 8 x 8 modes: the low modes' multipliers converge
    over hundreds of rows, so the table prefix spans many chunks; a z-only source puts the energy
    into the (0,0)-neighbourhood, the weakest modes."""
    shape = (4095, 8, 8)
    nz, ny, nx = shape
    sp = (1.0 / nx, 1.0 / ny, 1.0 / nz)
    f = workloads.uniform_source(shape, seed=23, remove_mean=False)
    fz = np.broadcast_to(np.random.default_rng(24).uniform(-1, 1, size=(nz, 1, 1)), shape).copy()
    for src in (f, fz):
        ref = oracle.solve(src, bc, sp)
        for rows in (8, 32):
            u = gpu_solve(src, bc, sp, options=dict(z_split=rows))
            assert rel_l2(u, ref) <= TOL_F64, (rows, rel_l2(u, ref))


def test_partitioned_singular_zero_mean(oracle):
    """No Dirichlet face: the partitioned kernel skips the pinned (0,0) column and the plan solves it
    with the Thomas sweep; the result has zero mean and matches the oracle."""
    shape = (300, 12, 16)
    f = np.random.default_rng(25).uniform(0, 1, size=shape)
    for bc in ("NNNNNN", "PPNNNN", "NNPPNN", "PPPPNN"):
        sp = (0.1, 0.2, 0.3)
        u = gpu_solve(f, bc, sp, options=dict(z_split=16))
        assert abs(u.mean()) <= 1e-13 * np.abs(u).max(), bc
        assert rel_l2(u, oracle.solve(f, bc, sp)) <= TOL_F64, bc


def test_partitioned_refined_and_adjoint(oracle):
    """The refined mixed solve runs the partitioned z twice (FP64-class result); the adjoint of a
    partitioned plan runs the transposed Thomas factorisation (S is symmetric: S^T g = S g)."""
    shape = (513, 16, 12)
    nz, ny, nx = shape
    sp = (1.0 / nx, 1.0 / ny, 1.0 / nz)
    f = workloads.uniform_source(shape, seed=26, remove_mean=False)
    ref = oracle.solve(f, "NNDDND", sp)
    u = gpu_solve(f, "NNDDND", sp, "mixed_f64io", how="solve_refined", options=dict(z_split=8))
    assert rel_l2(u, ref) <= 1e-10
    ua = gpu_solve(f, "NNDDND", sp, how="solve_adjoint", options=dict(z_split=8))
    assert rel_l2(ua, ref) <= TOL_F64


def test_partitioned_range_status():
    """The partitioned kernel reports the z solve's range like the sweeps."""
    import paper_1909_05423_gb300 as pp
    shape = (200, 16, 16)
    sp = (1.0 / 16, 1.0 / 16, 1.0 / 200)
    f = workloads.uniform_source(shape, seed=27)
    plan = pp.Plan(shape, "NNDDNN", sp, "f64", options=dict(z_split=16))
    assert plan.z_split() == 16
    for scale, flagged in ((1.0, False), (1e-20, False), (1e-32, True), (1e37, True), (1.0, False)):
        ft = torch.from_numpy(f * scale).cuda()
        plan.solve(ft)
        torch.cuda.synchronize()
        try:
            plan.status()
            err = None
        except _lib.PPError as e:
            err = e
        assert (err is not None) == flagged, (scale, err)
        if flagged:
            assert err.status == _lib.PP_ERR_RANGE
    plan.close()


def test_periodic_z_ignores_split(oracle):
    """Periodic z keeps the Sherman-Morrison sweeps (the split is a non-periodic solver)."""
    shape = (64, 8, 12)
    sp = (1.0 / 12, 1.0 / 8, 1.0 / 64)
    plan = _plan(shape, "NNDDPP", sp, z_split=8)
    assert plan.z_split() == 1 and plan.z_method() == "sherman-morrison"
    plan.close()
    f = workloads.uniform_source(shape, seed=28, remove_mean=False)
    assert rel_l2(gpu_solve(f, "NNDDPP", sp, options=dict(z_split=8)), oracle.solve(f, "NNDDPP", sp)) <= TOL_F64


def test_autotuned_split(oracle):
    """With autotune = 1 the plan times the sweeps and the three chunk sizes and keeps one; few modes
    on long lines (64 x 64 x 2047) is the case the partitioned solve exists for.  Whatever it keeps
    matches the oracle; a fixed z_split is kept as given."""
    shape = (2047, 16, 16)
    nz, ny, nx = shape
    sp = (1.0 / nx, 1.0 / ny, 1.0 / nz)
    f = workloads.uniform_source(shape, seed=29, remove_mean=False)
    ref = oracle.solve(f, "NNDDNN", sp)
    plan = _plan(shape, "NNDDNN", sp, autotune=1)
    assert plan.z_split() in (1, 8, 16, 32)
    ft = torch.from_numpy(f).cuda()
    u = plan.solve(ft).cpu().numpy()
    plan.status()
    plan.close()
    assert rel_l2(u, ref) <= TOL_F64
    plan = _plan(shape, "NNDDNN", sp, autotune=1, z_split=1)
    assert plan.z_split() == 1
    plan.close()
    plan = _plan(shape, "NNDDNN", sp, autotune=1, z_split=32)
    assert plan.z_split() == 32
    plan.close()


def test_partitioned_batched(oracle):
    """Plans with partitioned z inside one batched graph, beside a Thomas plan."""
    import paper_1909_05423_gb300 as pp
    cases = [((130, 12, 8), "NNDDNN", 8), ((77, 8, 16), "DDNNND", 16), ((64, 10, 6), "NNNNNN", 32),
             ((90, 6, 6), "NDNDDN", 1)]
    plans, fs, refs = [], [], []
    for shape, bc, rows in cases:
        sp = (1.0 / shape[2], 1.0 / shape[1], 1.0 / shape[0])
        f = workloads.uniform_source(shape, seed=shape[0], remove_mean=False)
        plans.append(pp.Plan(shape, bc, sp, "f64", options=dict(z_split=rows)))
        fs.append(torch.from_numpy(f).cuda())
        refs.append(oracle.solve(f, bc, sp))
    us = [torch.empty_like(x) for x in fs]
    for _ in range(2):  # capture, then replay
        pp.solve_batched(plans, fs, us)
        torch.cuda.synchronize()
        for p, u, r in zip(plans, us, refs):
            p.status()
            assert rel_l2(u.cpu().numpy(), r) <= TOL_F64
    for p in plans:
        p.close()


def test_partitioned_residual_256(oracle):
    """256^3, Neumann x / Dirichlet y / Neumann z, each chunk size: ||A u - f|| / ||f|| < 1e-12 and
    agreement with the Thomas sweeps."""
    n = 256
    shape = (n, n, n)
    sp = (1.0 / n,) * 3
    f = workloads.uniform_source(shape, seed=2, remove_mean=True)
    ut = gpu_solve(f, "NNDDNN", sp, options=dict(z_split=1))
    for rows in (8, 16, 32):
        u = gpu_solve(f, "NNDDNN", sp, options=dict(z_split=rows))
        r = oracle.laplacian(u, "NNDDNN", sp) - f
        assert np.linalg.norm(r) / np.linalg.norm(f) < 1e-12, rows
        assert rel_l2(u, ut) <= 1e-13, (rows, rel_l2(u, ut))
