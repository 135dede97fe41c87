"""Periodic z by transform (a DFT along z, a diagonal solve per (kx, ky, kz), the inverse DFT) against
the CPU oracle, which solves periodic z by Sherman-Morrison: the two methods solve the same
circulant systems, so they must agree to the FP64 bound.  Covers complex spectra (x or y periodic)
and all-real spectra (two real modes per complex z line), odd and 7-smooth nz, the singular mode,
the adjoint, and the autotuner's choice between the methods."""
import numpy as np
import pytest

from paper_1909_05423_gb300 import workloads
from tests.gpu_common import gpu_solve, need_gpu, rel_l2, torch

pytestmark = pytest.mark.gpu
TOL = {"f64": 1e-12, "mixed_f64io": 1e-6, "mixed_f32io": 1e-6}
FFT_Z = {"z_method": 2}


@pytest.fixture(scope="module", autouse=True)
def _setup(oracle):
    need_gpu()


@pytest.mark.parametrize("bc", ["PPPPPP", "NNNNPP", "DDDDPP", "PPNNPP", "DNNDPP", "NDPPPP", "DNDDPP"])
@pytest.mark.parametrize("shape", [(45, 48, 96), (12, 72, 54), (3, 8, 16), (7, 18, 20), (64, 10, 12)])
def test_zfft_parity(oracle, bc, shape):
    nz, ny, nx = shape
    sp = (1.0 / nx, 1.3 / ny, 0.9 / nz)
    f = workloads.uniform_source(shape, seed=61, remove_mean=False)
    ref = oracle.solve(f, bc, sp)
    for dtype, tol in TOL.items():
        u = gpu_solve(f, bc, sp, dtype, options=FFT_Z)
        assert rel_l2(u, ref) <= tol, (dtype, rel_l2(u, ref))


def _axis_eigs(kind, n, h):
    """Per-axis eigenvalues of the 1-D second difference, -4 sin^2(theta/2) / h^2 (no cancellation)."""
    k = np.arange(n, dtype=np.float64)
    theta = {"PP": 2 * np.pi * k / n, "NN": np.pi * k / n, "DD": np.pi * (k + 1) / n}.get(kind, np.pi * (k + 0.5) / n)
    return -4.0 * np.sin(theta / 2) ** 2 / (h * h)


def _oracle_rounding_bound(shape, bc, sp):
    """The oracle (and the Sherman-Morrison sweeps) form the z diagonal b = -2/dz^2 + lambda_xy in
    FP64: the rounding moves a mode's shift lambda_xy by up to ulp(2/dz^2)/2, a relative change of
    2^-53 (2/dz^2) / |sigma| in a mode of eigenvalue sigma.  The transform method divides by sigma
    itself, so it may differ from the oracle by about that much in the smallest nonzero |sigma|."""
    nz, ny, nx = shape
    ex = _axis_eigs(bc[0:2], nx, sp[0])
    ey = _axis_eigs(bc[2:4], ny, sp[1])
    ez = _axis_eigs(bc[4:6], nz, sp[2])
    sig = np.abs(ex[:, None, None] + ey[None, :, None] + ez[None, None, :])
    smin = sig[sig > 1e-9 * sig.max()].min()
    return 2.0 ** -53 * (2.0 / sp[2] ** 2) / smin


@pytest.mark.parametrize("shape,bc", [((1024, 4, 6), "DDNNPP"), ((700, 8, 16), "PPPPPP"), ((512, 6, 4), "NNNNPP")])
def test_zfft_long_lines(oracle, shape, bc):
    """Long periodic z lines.  Against the oracle the transform method keeps the FP64 bound plus the
    oracle's own rounding of its z diagonal (see _oracle_rounding_bound: 2.4e-11 for the first
    case, 2.9e-12 and 6.2e-12 for the others)."""
    nz, ny, nx = shape
    sp = (1.0 / nx, 1.0 / ny, 1.0 / nz)
    f = workloads.uniform_source(shape, seed=62, remove_mean=False)
    ref = oracle.solve(f, bc, sp)
    tol = TOL["f64"] + _oracle_rounding_bound(shape, bc, sp)
    assert rel_l2(gpu_solve(f, bc, sp, options=FFT_Z), ref) <= tol
    assert rel_l2(gpu_solve(f, bc, sp, "mixed_f64io", options=FFT_Z), ref) <= TOL["mixed_f64io"]
    # the two methods of the library differ by the same rounding only
    assert rel_l2(gpu_solve(f, bc, sp, options=FFT_Z), gpu_solve(f, bc, sp, options={"z_method": 1})) <= tol


def test_zfft_singular_zero_mean(oracle):
    shape = (16, 24, 36)
    f = np.random.default_rng(63).uniform(0, 1, size=shape)  # non-zero mean: solved as f - mean(f)
    for bc in ("PPPPPP", "NNNNPP", "PPNNPP"):
        u = gpu_solve(f, bc, (0.1, 0.2, 0.3), options=FFT_Z)
        assert abs(u.mean()) <= 1e-13 * np.abs(u).max()
        assert rel_l2(u, oracle.solve(f, bc, (0.1, 0.2, 0.3))) <= TOL["f64"]


@pytest.mark.parametrize("bc", ["PPPPPP", "NNDDPP"])
def test_zfft_adjoint(oracle, bc):
    import paper_1909_05423_gb300 as pp
    shape = (12, 24, 36)
    rng = np.random.default_rng(64)
    f, g = rng.standard_normal(shape), rng.standard_normal(shape)
    sp = (0.3, 0.2, 0.5)
    plan = pp.Plan(shape, bc, sp, "f64", options=FFT_Z)
    assert plan.z_method() == "transform"
    ft, gt = torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda()
    sf, stg = plan.solve(ft), plan.solve_adjoint(gt)
    torch.cuda.synchronize()
    a = torch.dot(sf.flatten(), gt.flatten()).item()
    b = torch.dot(ft.flatten(), stg.flatten()).item()
    assert abs(a - b) <= 1e-12 * max(abs(a), 1e-30) + 1e-13 * (np.linalg.norm(f) * np.linalg.norm(g))
    assert rel_l2(stg.cpu().numpy(), oracle.solve(g, bc, sp)) <= 1e-12
    plan.close()


def test_z_method_choice(oracle):
    """Default: Sherman-Morrison; z_method 1 / 2 force a method; autotune times both and keeps the
    faster, and the plan reports which.  Every choice matches the oracle."""
    import paper_1909_05423_gb300 as pp
    shape = (48, 32, 64)
    sp = (1.0 / 64, 1.0 / 32, 1.0 / 48)
    f = workloads.uniform_source(shape, seed=65)
    ref = oracle.solve(f, "PPPPPP", sp)
    for opts, want in (({}, "sherman-morrison"), ({"z_method": 1}, "sherman-morrison"), (FFT_Z, "transform"),
                       ({"autotune": 1}, None)):
        plan = pp.Plan(shape, "PPPPPP", sp, "f64", options=opts)
        got = plan.z_method()
        assert got in ("sherman-morrison", "transform") and (want is None or got == want), (opts, got)
        u = plan.solve(torch.from_numpy(f).cuda())
        torch.cuda.synchronize()
        plan.status()
        assert rel_l2(u.cpu().numpy(), ref) <= TOL["f64"], opts
        plan.close()
    assert pp.Plan((8, 8, 8), "PPPPDD", (1.0, 1.0, 1.0)).z_method() == "thomas"


def test_zfft_batched_and_host(oracle):
    """The transform method inside a batched graph and through host buffers."""
    import paper_1909_05423_gb300 as pp
    shapes = [(24, 16, 32), (9, 20, 12)]
    plans, fs, refs = [], [], []
    for i, shape in enumerate(shapes):
        nz, ny, nx = shape
        sp = (1.0 / nx, 1.0 / ny, 1.0 / nz)
        bc = ["PPPPPP", "NDDNPP"][i]
        f = workloads.uniform_source(shape, seed=66 + i)
        plans.append(pp.Plan(shape, bc, sp, "f64", options=FFT_Z))
        fs.append(torch.from_numpy(f).cuda())
        refs.append(oracle.solve(f, bc, sp))
    us = pp.solve_batched(plans, fs)
    torch.cuda.synchronize()
    for u, r in zip(us, refs):
        assert rel_l2(u.cpu().numpy(), r) <= TOL["f64"]
    uh = plans[0].solve_host(fs[0].cpu().pin_memory())
    assert rel_l2(uh.numpy(), refs[0]) <= TOL["f64"]
    for p in plans:
        p.close()
