"""Gradients of L = 0.5 ||S f(theta) - u_t||^2 through the autograd Function, where f(theta) is
a sum of Gaussian blobs A_i exp(-|x - c_i|^2 / (2 w_i^2)) sampled at cell centres and S is the
solution operator (forward solve; its transpose through the adjoint pipeline).

* amplitudes: L is quadratic in A, so central differences equal the derivative up to rounding;
* centres and widths: central differences carry an O(eps^2) truncation term, checked at
  eps = 1e-4 and 1e-5 (relative agreement 1e-6; the difference of the two losses is evaluated
  through the linearity of S, see central_difference);
* the GPU's dL/df against the oracle's S^T (S f - u_t) = S (S f - u_t) (A_h is symmetric).
"""
import numpy as np
import pytest

from paper_1909_05423_gb300 import workloads
from tests.gpu_common import need_gpu, rel_l2, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup(oracle):
    need_gpu()


def _grid(shape, sp):
    nz, ny, nx = shape
    x = (torch.arange(nx, dtype=torch.float64, device="cuda") + 0.5) * sp[0]
    y = (torch.arange(ny, dtype=torch.float64, device="cuda") + 0.5) * sp[1]
    z = (torch.arange(nz, dtype=torch.float64, device="cuda") + 0.5) * sp[2]
    return x[None, None, :], y[None, :, None], z[:, None, None]


def _blobs(xyz, amp, centre, width):
    """Differentiable blob field (torch, FP64) -- the parametrised source."""
    x, y, z = xyz
    f = 0.0
    for i in range(amp.shape[0]):
        r2 = (x - centre[i, 0]) ** 2 + (y - centre[i, 1]) ** 2 + (z - centre[i, 2]) ** 2
        f = f + amp[i] * torch.exp(-r2 / (2.0 * width[i] ** 2))
    return f


def _setup_problem(n, count, bc, seed=5):
    import paper_1909_05423_gb300 as pp
    shape = (n, n, n)
    sp = (1.0 / n,) * 3
    amp, centre, width = workloads.gaussian_blobs(shape, sp, seed=seed, count=count)
    ut = torch.from_numpy(np.random.default_rng(6).uniform(-1, 1, size=shape)).cuda()
    plan = pp.Plan(shape, bc, sp, "f64")
    xyz = _grid(shape, sp)

    def loss(a, c, w):
        u = pp.PoissonSolve.apply(_blobs(xyz, a, c, w).contiguous(), plan)
        return 0.5 * ((u - ut) ** 2).sum()

    def central_difference(fp, fm, eps):
        """(L(theta+eps) - L(theta-eps)) / (2 eps) for the sources fp = f(theta+eps), fm = f(theta-eps).
        L itself is ~1e4 while the difference is ~1e-6, so forming L twice and subtracting keeps only
        ~1e-6 of the difference in FP64.  By the linearity of S the difference is instead evaluated
        as 0.5 <S(fp - fm), S fp + S fm - 2 u_t>: the same central difference, without the
        cancellation."""
        up, um = plan.solve(fp.contiguous()), plan.solve(fm.contiguous())
        du = plan.solve((fp - fm).contiguous())
        return 0.5 * torch.dot(du.flatten(), (up + um - 2.0 * ut).flatten()).item() / (2.0 * eps)

    t = lambda v: torch.tensor(v, dtype=torch.float64, device="cuda")
    return plan, loss, central_difference, t(amp), t(centre), t(width), ut, shape, sp, xyz


@pytest.mark.parametrize("bc", ["PPPPDD", "NNDDNN"])
def test_fd_centres_and_widths(bc):
    n = 48
    plan, loss, cdiff, A, C, W, _, _, _, xyz = _setup_problem(n, 4, bc)
    C.requires_grad_(True)
    W.requires_grad_(True)
    L = loss(A, C, W)
    L.backward()
    gc, gw = C.grad.clone(), W.grad.clone()
    with torch.no_grad():
        for name, param, grad in (("centre", C, gc), ("width", W, gw)):
            flat = param.view(-1)
            for idx in range(flat.numel()):
                g = grad.view(-1)[idx].item()
                fds = {}
                for eps in (1e-4, 1e-5):
                    old = flat[idx].item()
                    flat[idx] = old + eps
                    fp = _blobs(xyz, A, C, W)
                    flat[idx] = old - eps
                    fm = _blobs(xyz, A, C, W)
                    flat[idx] = old
                    fds[eps] = cdiff(fp, fm, eps)
                rel = {e: abs(v - g) / abs(g) for e, v in fds.items()}
                # eps = 1e-5: within 1e-6
                assert rel[1e-5] <= 1e-6, (name, idx, rel)
                # eps = 1e-4: within 1e-6, or else the O(eps^2) truncation term shows (the width
                # derivatives of the narrow blobs: ~3e-5 with the CPU oracle as well) -- then the
                # error must fall 100-fold with eps, and Richardson's combination of the two steps,
                # which cancels the eps^2 term, must agree to 1e-6
                if rel[1e-4] > 1e-6:
                    assert 50.0 <= rel[1e-4] / rel[1e-5] <= 200.0, (name, idx, rel)
                rich = fds[1e-5] + (fds[1e-5] - fds[1e-4]) / 99.0
                assert abs(rich - g) <= 1e-6 * abs(g), (name, idx, rel, rich, g)
    plan.close()


def test_fd_amplitudes_256():
    """Config-5 size (256^3, periodic x/y, Dirichlet z) with three blobs: dL/dA vs central
    differences, exact up to rounding because L is quadratic in A."""
    plan, loss, _, A, C, W, _, _, _, _ = _setup_problem(256, 3, "PPPPDD")
    A.requires_grad_(True)
    L = loss(A, C, W)
    L.backward()
    g = A.grad.clone()
    eps = 0.1  # L is exactly quadratic in A: a large step only shrinks the rounding part
    with torch.no_grad():
        for i in range(A.numel()):
            e = torch.zeros_like(A)
            e[i] = eps
            fd = (loss(A + e, C, W) - loss(A - e, C, W)).item() / (2 * eps)
            assert abs(fd - g[i].item()) <= 1e-8 * max(1.0, abs(fd)), (i, fd, g[i].item())
    plan.close()


def test_grad_f_matches_oracle(oracle):
    """dL/df = S^T (S f - u_t) from the adjoint pipeline equals the oracle's S (S f - u_t)."""
    n = 32
    plan, loss, _, A, C, W, ut, shape, sp, xyz = _setup_problem(n, 4, "PPPPDD")
    import paper_1909_05423_gb300 as pp
    f = _blobs(xyz, A, C, W).contiguous().detach().requires_grad_(True)
    u = pp.PoissonSolve.apply(f, plan)
    (0.5 * ((u - ut) ** 2).sum()).backward()
    fn = f.detach().cpu().numpy()
    r = oracle.solve(fn, "PPPPDD", sp) - ut.cpu().numpy()
    ref = oracle.solve(r, "PPPPDD", sp)
    assert rel_l2(f.grad.cpu().numpy(), ref) <= 1e-12
    plan.close()
