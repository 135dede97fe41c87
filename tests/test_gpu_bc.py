"""Faces with data on the GPU (pp_fold_bc + pp_solve) against the oracle's L_g solve.

The fold is FP64 arithmetic on the face cells; the solve is the homogeneous path, so the
tolerances are those of the plain solve (1e-12 FP64 path, 1e-6 mixed)."""
import numpy as np
import pytest

import oracle
from tests.gpu_common import need_gpu, rel_l2, torch
from tests.test_oracle_bc import cell_centres, face_data

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup():
    need_gpu()


def _problem(bc, shape, sp, seed):
    """A smooth field with non-zero data on every non-periodic face, plus a random source."""
    per = [bc[2 * a] == "P" for a in range(3)]
    nz, ny, nx = shape
    L = (nx * sp[0], ny * sp[1], nz * sp[2])

    def u(X, Y, Z):
        fx = np.cos(2 * np.pi * X / L[0]) if per[0] else np.cos(1.3 * X + 0.2)
        fy = np.cos(2 * np.pi * Y / L[1]) if per[1] else np.sin(0.8 * Y + 0.4)
        fz = np.cos(2 * np.pi * Z / L[2]) if per[2] else np.cosh(0.6 * Z) + 0.5
        return fx * fy * fz

    def grad(X, Y, Z):
        fx = np.cos(2 * np.pi * X / L[0]) if per[0] else np.cos(1.3 * X + 0.2)
        dfx = -2 * np.pi / L[0] * np.sin(2 * np.pi * X / L[0]) if per[0] else -1.3 * np.sin(1.3 * X + 0.2)
        fy = np.cos(2 * np.pi * Y / L[1]) if per[1] else np.sin(0.8 * Y + 0.4)
        dfy = -2 * np.pi / L[1] * np.sin(2 * np.pi * Y / L[1]) if per[1] else 0.8 * np.cos(0.8 * Y + 0.4)
        fz = np.cos(2 * np.pi * Z / L[2]) if per[2] else np.cosh(0.6 * Z) + 0.5
        dfz = -2 * np.pi / L[2] * np.sin(2 * np.pi * Z / L[2]) if per[2] else 0.6 * np.sinh(0.6 * Z)
        return dfx * fy * fz, fx * dfy * fz, fx * fy * dfz

    faces = face_data(bc, shape, sp, u, grad)
    f = np.random.default_rng(seed).uniform(-1.0, 1.0, shape)
    return f, faces


CASES = [((12, 12, 16), "DNNDND"), ((9, 8, 12), "PPDNND"), ((10, 12, 8), "NDDNPP"), ((8, 6, 12), "DDDDDD"),
         ((7, 12, 6), "NNNNNN"), ((16, 18, 24), "NNDDNN"), ((6, 8, 6), "DNPPND")]


@pytest.mark.parametrize("shape,bc", CASES)
@pytest.mark.parametrize("dtype,tol", [("f64", 1e-12), ("mixed_f64io", 1e-6), ("mixed_f32io", 1e-5)])
def test_fold_and_solve_match_oracle(shape, bc, dtype, tol):
    import paper_1909_05423_gb300 as pp
    sp = (0.7 / shape[2], 1.1 / shape[1], 0.9 / shape[0])
    f, faces = _problem(bc, shape, sp, seed=len(bc) + shape[0])
    ref_fold = oracle.fold_bc(f, bc, sp, faces)
    ref = oracle.solve(ref_fold, bc, sp)
    plan = pp.Plan(shape, bc, sp, dtype)
    io = plan.io_dtype
    ft = torch.from_numpy(f).to(device="cuda", dtype=io)
    gt = [None if g is None else torch.from_numpy(np.ascontiguousarray(g)).to(device="cuda", dtype=io) for g in faces]
    folded = plan.fold_bc(ft, gt)
    u = plan.solve(folded)
    torch.cuda.synchronize()
    plan.status()
    if dtype == "f64":
        assert np.abs(folded.cpu().numpy() - ref_fold).max() <= 1e-14 * np.abs(ref_fold).max()
    assert rel_l2(u.double().cpu().numpy(), ref) <= tol
    plan.close()


def test_fold_in_place_and_one_shot():
    import paper_1909_05423_gb300 as pp
    shape, bc = (8, 12, 16), "DNDNDN"
    sp = (1 / 16, 1 / 12, 1 / 8)
    f, faces = _problem(bc, shape, sp, seed=3)
    ref = oracle.solve_g(f, bc, sp, faces)
    gt = [torch.from_numpy(np.ascontiguousarray(g)).cuda() for g in faces]
    ft = torch.from_numpy(f).cuda()
    u1 = pp.solve(ft.clone(), bc, sp, faces=gt)
    plan = pp.Plan(shape, bc, sp)
    fi = ft.clone()
    plan.fold_bc(fi, gt, out=fi)
    u2 = plan.solve(fi)
    torch.cuda.synchronize()
    for u in (u1, u2):
        assert rel_l2(u.cpu().numpy(), ref) <= 1e-12
    plan.close()


def test_manufactured_solution_converges():
    """Source = Laplacian of a smooth u*, faces = its values / outward derivatives: second order."""
    import paper_1909_05423_gb300 as pp
    bc = "DNNDND"

    def u(X, Y, Z):
        return np.cos(1.1 * X + 0.3) * np.sin(0.9 * Y + 0.5) * np.cosh(0.7 * Z)

    def grad(X, Y, Z):
        return (-1.1 * np.sin(1.1 * X + 0.3) * np.sin(0.9 * Y + 0.5) * np.cosh(0.7 * Z),
                0.9 * np.cos(1.1 * X + 0.3) * np.cos(0.9 * Y + 0.5) * np.cosh(0.7 * Z),
                0.7 * np.cos(1.1 * X + 0.3) * np.sin(0.9 * Y + 0.5) * np.sinh(0.7 * Z))

    errs = []
    for n in (16, 32, 64):
        shape, sp = (n, n, n), (1.0 / n,) * 3
        Z, Y, X = cell_centres(shape, sp)
        f = (-1.21 - 0.81 + 0.49) * u(X, Y, Z)
        gt = [torch.from_numpy(np.ascontiguousarray(g)).cuda() for g in face_data(bc, shape, sp, u, grad)]
        got = pp.solve(torch.from_numpy(f).cuda(), bc, sp, faces=gt).cpu().numpy()
        errs.append(np.sqrt(np.mean((got - u(X, Y, Z)) ** 2)))
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5, errs


def test_periodic_face_with_data_is_rejected():
    import paper_1909_05423_gb300 as pp
    plan = pp.Plan((4, 6, 8), "PPNNDD", (1, 1, 1))
    f = torch.zeros((4, 6, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(pp.PPError) as ei:
        plan.fold_bc(f, [torch.zeros((4, 6), dtype=torch.float64, device="cuda"), None, None, None, None, None])
    assert ei.value.status == 1
    plan.close()
