"""Mixed precision (FP32 transforms, double-float z solve), refinement, adjoint and autograd."""
import math

import numpy as np
import pytest

from paper_1909_05423_gb300 import workloads
from tests.gpu_common import gpu_solve, need_gpu, rel_l2, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup(oracle):
    need_gpu()


@pytest.mark.parametrize("bc", ["PPPPPP", "NNNNNN", "NNDDNN", "DNPPDD"])
@pytest.mark.parametrize("dtype", ["mixed_f64io", "mixed_f32io"])
def test_mixed_error_bound(oracle, bc, dtype):
    shape = (24, 48, 96)
    sp = (1.0 / 96, 1.0 / 48, 1.0 / 24)
    f = workloads.uniform_source(shape, seed=3)
    ref = oracle.solve(f, bc, sp)
    u = gpu_solve(f, bc, sp, dtype)
    assert rel_l2(u, ref) <= 1e-6, rel_l2(u, ref)


@pytest.mark.parametrize("bc", ["PPPPPP", "NNNNNN", "NNDDNN"])
@pytest.mark.parametrize("sp", [(1.0 / 96, 1.0 / 48, 1.0 / 24), (0.01, 0.01, 0.01)])
def test_refined_recovers_fp64(oracle, bc, sp):
    """Unequal spacings scale each axis's second difference; equal ones scale their sum once."""
    shape = (24, 48, 96)
    f = workloads.uniform_source(shape, seed=3)
    ref = oracle.solve(f, bc, sp)
    u = gpu_solve(f, bc, sp, "mixed_f64io", how="solve_refined")
    assert rel_l2(u, ref) <= 1e-10, rel_l2(u, ref)


@pytest.mark.parametrize("bc", ["NNDDNN", "NNNNNN", "PPPPPP", "DNNDPP"])
@pytest.mark.parametrize("spacing", [(1.0 / 20, 1.0 / 12, 1.0 / 10), (0.1, 0.1, 0.1)])
def test_refined_alignment_paths(bc, spacing):
    """The residual r = f - A u0 runs four cells a thread when nx is a multiple of 4 and f is 16-byte
    aligned, the update u = u0 + delta four values a thread when u is; otherwise one a thread.  Both
    forms do the same operations on the same operands, so a source or an output that starts 8 bytes
    past a 16-byte boundary (and a row length that is not a multiple of 4) gives the same bits."""
    import paper_1909_05423_gb300 as pp
    for shape in ((10, 12, 20), (6, 10, 14)):
        plan = pp.Plan(shape, bc, spacing, "mixed_f64io")
        h = workloads.uniform_source(shape, seed=31)
        f = torch.from_numpy(h).cuda()
        u_al = plan.solve_refined(f)
        fbuf = torch.empty((f.numel() + 1,), dtype=torch.float64, device="cuda")
        f_off = fbuf[1:].view(shape)
        f_off.copy_(f)
        ubuf = torch.full((f.numel() + 1,), float("nan"), dtype=torch.float64, device="cuda")
        u_off = ubuf[1:].view(shape)
        assert f_off.data_ptr() % 16 == 8 and u_off.data_ptr() % 16 == 8
        plan.solve_refined(f_off, u_off)
        torch.cuda.synchronize()
        assert torch.equal(u_al, u_off), shape
        plan.close()


@pytest.mark.parametrize("bc", ["PPPPDD", "NNDDNN", "DNPPNN", "PPPPPP", "NNNNNN"])
def test_adjoint_dot_product(oracle, bc):
    import paper_1909_05423_gb300 as pp
    shape = (12, 24, 36)
    rng = np.random.default_rng(1)
    f = rng.standard_normal(shape)
    g = rng.standard_normal(shape)
    plan = pp.Plan(shape, bc, (0.3, 0.2, 0.5), "f64")
    ft, gt = torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda()
    sf = plan.solve(ft)
    stg = plan.solve_adjoint(gt)
    torch.cuda.synchronize()
    a = torch.dot(sf.flatten(), gt.flatten()).item()
    b = torch.dot(ft.flatten(), stg.flatten()).item()
    assert abs(a - b) <= 1e-12 * max(abs(a), 1e-30) + 1e-13 * (np.linalg.norm(f) * np.linalg.norm(g))
    # S is symmetric: the adjoint equals the oracle's S g
    assert rel_l2(stg.cpu().numpy(), oracle.solve(g, bc, (0.3, 0.2, 0.5))) <= 1e-12
    plan.close()


def test_autograd_blob_amplitudes():
    """Config-5 shaped check at 32^3: L = 0.5||S f(A) - u_t||^2 with f a sum of Gaussian blobs;
    dL/dA from autograd through PoissonSolve vs central finite differences (exact up to rounding,
    L is quadratic in A)."""
    import paper_1909_05423_gb300 as pp
    n = 32
    shape = (n, n, n)
    sp = (1.0 / n,) * 3
    amp, centre, width = workloads.gaussian_blobs(shape, sp, seed=5, count=4)
    ut = torch.from_numpy(np.random.default_rng(6).uniform(-1, 1, size=shape)).cuda()
    basis = torch.stack([torch.from_numpy(workloads.blob_field(shape, sp, [1.0], [c], [w])).cuda()
                         for c, w in zip(centre, width)])
    plan = pp.Plan(shape, "PPPPDD", sp, "f64")
    A = torch.tensor(amp, dtype=torch.float64, device="cuda", requires_grad=True)

    def loss(a):
        f = (a[:, None, None, None] * basis).sum(0)
        u = pp.PoissonSolve.apply(f, plan)
        return 0.5 * ((u - ut) ** 2).sum()

    L = loss(A)
    L.backward()
    g = A.grad.clone()
    eps = 1e-3
    for i in range(len(amp)):
        e = torch.zeros_like(A)
        e[i] = eps
        with torch.no_grad():
            fd = (loss(A + e) - loss(A - e)) / (2 * eps)
        assert abs(fd.item() - g[i].item()) <= 1e-7 * max(1.0, abs(fd.item()))
    plan.close()
