"""Pins for the CPU oracle: each test ties it to something other than itself
(the paper's printed tables, dense Gaussian elimination of the assembled
7-point matrix, library transforms, closed-form discrete solutions,
invariants).  CPU only."""
import itertools
import math
import os

import numpy as np
import pytest
import scipy.fft

from paper_1909_05423_gb300 import workloads
from tests import helpers

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "mms_tables.txt")


def _golden_rows():
    rows = []
    with open(GOLDEN) as fh:
        lines = fh.read().splitlines()
    for line in lines:
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        t, bc, kx, ky, kz, la, n, e = line.split()
        rows.append((t, bc, float(kx), float(ky), float(kz), float(la), int(n), float(e)))
    return rows


def test_closed_form_reproduces_paper_tables():
    """Tables tb3-tb7: the exact discrete error |u*|_rms * |sum k^2 / sum lambda_d - 1|
    reproduces every printed value to the 6 printed digits."""
    rows = _golden_rows()
    assert len(rows) == 20
    for t, bc, kx, ky, kz, la, n, printed in rows:
        h = 1.0 / n
        err = 2.0 ** la * abs(helpers.discrete_solution_ratio([kx * math.pi, ky * math.pi, kz * math.pi],
                                                               [h, h, h]) - 1.0)
        assert abs(err - printed) <= 5e-6 * printed, (t, n, err, printed)


def _mms_solve_and_check(oracle, bc, kappas, n, tol=1e-12):
    """Oracle on f = Laplacian(u*) for every real product of the manufactured mode: the result
    must be the exact discrete solution u* * ratio (element by element); returns the RMS error
    of the complex-valued (periodic) / real field against u*."""
    shape = (n, n, n)
    sp = (1.0 / n,) * 3
    ratio = helpers.discrete_solution_ratio(kappas, [1.0 / n] * 3)
    sq = 0.0
    per_axis = helpers.mms_terms(bc, *kappas)
    # periodic axes carry cos+i sin: the complex product is a sum of real products with
    # coefficients i^m; its squared modulus error adds up over the real and imaginary parts.
    combos = list(itertools.product(*per_axis))
    parts = {0: np.zeros(shape), 1: np.zeros(shape)}
    parts_star = {0: np.zeros(shape), 1: np.zeros(shape)}
    for comps in combos:
        m = sum(1 for c, pair in zip(comps, (bc[0:2], bc[2:4], bc[4:6])) if pair == "PP" and c[0] == "sin")
        coef = (1j) ** m
        u_star, f = helpers.mms_field(shape, sp, list(comps))
        u = oracle.solve(f, bc, sp)
        np.testing.assert_allclose(u, u_star * ratio, rtol=0, atol=tol * np.abs(u_star).max())
        re, im = coef.real, coef.imag
        parts[0] += re * u; parts[1] += im * u
        parts_star[0] += re * u_star; parts_star[1] += im * u_star
    e2 = (parts[0] - parts_star[0]) ** 2 + (parts[1] - parts_star[1]) ** 2
    return math.sqrt(e2.mean())


@pytest.mark.parametrize("row", [r for r in _golden_rows() if r[6] == 128 and r[0] in ("tb4", "tb6")],
                         ids=lambda r: r[0])
def test_oracle_matches_paper_table_at_128(oracle, row):
    """The oracle itself reproduces a printed table entry at N = 128."""
    t, bc, kx, ky, kz, la, n, printed = row
    err = _mms_solve_and_check(oracle, bc, [kx * math.pi, ky * math.pi, kz * math.pi], n)
    assert abs(err - printed) <= 5e-6 * printed, (t, err, printed)


@pytest.mark.parametrize("row", [r for r in _golden_rows() if r[6] == 128], ids=lambda r: r[0])
def test_oracle_exact_discrete_solution_all_tables(oracle, row):
    """Same manufactured modes at N = 32: oracle = exact discrete solution elementwise, and the RMS
    error equals the closed form."""
    t, bc, kx, ky, kz, la, _, _ = row
    n = 32
    kap = [kx * math.pi, ky * math.pi, kz * math.pi]
    err = _mms_solve_and_check(oracle, bc, kap, n)
    closed = 2.0 ** la * abs(helpers.discrete_solution_ratio(kap, [1.0 / n] * 3) - 1.0)
    assert abs(err - closed) <= 1e-9 * closed


def test_config1_error_and_order(oracle):
    """32^3, periodic x/y, Dirichlet z, u* = sin 2pi x sin 2pi y sin pi z: RMS error 1.042987e-03
    (closed form), second order between 32 and 64."""
    errs = []
    for n in (32, 64):
        sp = (1.0 / n,) * 3
        u_star, f = workloads.manufactured((n, n, n), sp,
                                           [(1.0, ("sin", 2 * math.pi), ("sin", 2 * math.pi), ("sin", math.pi))])
        u = oracle.solve(f, "PPPPDD", sp)
        errs.append(math.sqrt(((u - u_star) ** 2).mean()))
    assert abs(errs[0] - 1.042987e-03) <= 1e-6 * 1.042987e-03
    assert abs(errs[1] - 2.604164e-4) <= 1e-5 * 2.604164e-4
    order = math.log(errs[0] / errs[1]) / math.log(2.0)
    assert abs(order - 2.0) < 0.01


def test_sign_convention(oracle):
    """The solver solves Laplacian(u) = f (paper sign): a sign slip would give relative error 2."""
    n = 16
    sp = (1.0 / n,) * 3
    u_star, f = workloads.manufactured((n, n, n), sp, [(1.0, ("sin", math.pi), ("sin", math.pi), ("sin", math.pi))])
    u = oracle.solve(f, "DDDDDD", sp)
    rel = np.linalg.norm(u - u_star) / np.linalg.norm(u_star)
    rel_wrong = np.linalg.norm(-u - u_star) / np.linalg.norm(u_star)
    assert rel < 0.02 and abs(rel_wrong - 2.0) < 0.02


@pytest.mark.parametrize("shape", [(5, 6, 4), (3, 4, 6), (4, 3, 5)])
def test_dense_gauss_all_axis_kinds(oracle, shape):
    """All 5x5x5 per-axis boundary kinds on tiny uneven grids: oracle = dense Gaussian elimination
    of the assembled 7-point matrix (bordered system when no face is Dirichlet)."""
    rng = np.random.default_rng(11)
    sp = (0.7, 1.3, 0.9)
    for kinds in itertools.product(helpers.AXIS_KINDS, repeat=3):
        bc = "".join(kinds)
        f = rng.uniform(-1, 1, size=shape)
        u = oracle.solve(f, bc, sp)
        ref = helpers.dense_solve(f, bc, sp)
        np.testing.assert_allclose(u, ref, rtol=0, atol=1e-12 * np.abs(ref).max(), err_msg=bc)


def test_laplacian_matches_assembly(oracle):
    rng = np.random.default_rng(3)
    sp = (0.5, 0.25, 2.0)
    for kinds in itertools.product(helpers.AXIS_KINDS, repeat=3):
        bc = "".join(kinds)
        u = rng.standard_normal((3, 5, 4))
        A = helpers.assemble(4, 5, 3, bc, sp)
        np.testing.assert_allclose(oracle.laplacian(u, bc, sp).ravel(), A @ u.ravel(), rtol=1e-13, atol=1e-12)
        idx = np.array([0, 7, 59, 13])
        np.testing.assert_allclose(oracle.laplacian_at(u, bc, sp, idx), (A @ u.ravel())[idx], rtol=1e-13, atol=1e-12)


@pytest.mark.parametrize("bc", ["PPPPDD", "NNDDNN", "PPPPPP", "NNNNNN", "DNNDPP", "NDPPDN"])
def test_residual_invariant(oracle, bc):
    """||A_h u - f|| / ||f|| < 1e-12 on a larger uneven grid (f mean-free when singular)."""
    shape = (20, 18, 24)
    sp = (1.0 / 24, 1.0 / 18, 1.0 / 20)
    f = workloads.uniform_source(shape, seed=5, remove_mean=True)
    u = oracle.solve(f, bc, sp)
    r = oracle.laplacian(u, bc, sp) - f
    assert np.linalg.norm(r) / np.linalg.norm(f) < 1e-12
    if "D" not in bc:
        assert abs(u.mean()) < 1e-14 * np.abs(u).max()


def test_singular_source_mean_removed(oracle):
    """All-Neumann: a source with non-zero mean is solved as f - mean(f); zero-mean result."""
    rng = np.random.default_rng(8)
    f = rng.uniform(0, 1, size=(6, 8, 10))
    u = oracle.solve(f, "NNNNNN")
    r = oracle.laplacian(u, "NNNNNN") - (f - f.mean())
    assert np.linalg.norm(r) / np.linalg.norm(f) < 1e-12
    assert abs(u.mean()) < 1e-13


def test_operator_symmetric(oracle):
    """Dot-product test <S f, g> = <f, S g> (A_h symmetric for P/N/D faces)."""
    rng = np.random.default_rng(2)
    for bc in ("PPPPDD", "NNDDNN", "DNNDPP", "NNNNNN"):
        f = rng.standard_normal((6, 8, 10)); g = rng.standard_normal((6, 8, 10))
        a = np.vdot(oracle.solve(f, bc), g); b = np.vdot(f, oracle.solve(g, bc))
        assert abs(a - b) <= 1e-12 * abs(a) + 1e-13


def test_line_transforms_vs_library(oracle):
    """Forward bases against numpy's FFT and scipy's DCT/DST (scipy's unnormalised type II/IV
    carry a factor 2); inverse = exact inverse."""
    rng = np.random.default_rng(4)
    for n in (2, 5, 6, 12, 17):
        x = rng.standard_normal(n)
        z = x + 1j * rng.standard_normal(n)
        np.testing.assert_allclose(oracle.line_forward(0, z), np.fft.fft(z), atol=1e-12)
        np.testing.assert_allclose(oracle.line_forward(1, x).real, scipy.fft.dct(x, 2) / 2, atol=1e-12)
        np.testing.assert_allclose(oracle.line_forward(2, x).real, scipy.fft.dst(x, 2) / 2, atol=1e-12)
        np.testing.assert_allclose(oracle.line_forward(3, x).real, scipy.fft.dst(x, 4) / 2, atol=1e-12)
        np.testing.assert_allclose(oracle.line_forward(4, x).real, scipy.fft.dct(x, 4) / 2, atol=1e-12)
        for kind in range(5):
            np.testing.assert_allclose(oracle.line_inverse(kind, oracle.line_forward(kind, z)), z, atol=1e-12)


def test_eigenvalues_vs_assembled_1d(oracle):
    """Per-axis eigenvalues (Table 'Eigenvalues', plus the mixed D/N axis) equal the spectrum of
    the assembled 1-D matrix, and each basis vector is an eigenvector."""
    for kind_idx, pair in enumerate(helpers.AXIS_KINDS):
        for n in (3, 6, 9):
            A = helpers.assemble(n, 1, 1, pair + "PPPP")  # y, z periodic with one cell: zero contribution
            lam = np.array([oracle.eigenvalue(kind_idx, n, k) for k in range(n)])
            np.testing.assert_allclose(np.sort(lam), np.sort(np.linalg.eigvalsh(A)), atol=1e-12)
            for k in range(n):
                e = np.zeros(n, complex); e[k] = 1.0
                v = np.conj(oracle.line_inverse(kind_idx, e))  # conj(b_k) up to weight
                np.testing.assert_allclose(A @ v, lam[k] * v, atol=1e-12)


def test_thomas_and_cyclic_vs_dense(oracle):
    rng = np.random.default_rng(9)
    for n in (2, 3, 7, 40):
        a = rng.uniform(0.5, 1.0, n); c = rng.uniform(0.5, 1.0, n)
        b = -(a + c + rng.uniform(0.1, 1.0, n)); d = rng.standard_normal(n)
        T = np.diag(b) + np.diag(a[1:], -1) + np.diag(c[:-1], 1)
        np.testing.assert_allclose(oracle.thomas(a, b, c, d), np.linalg.solve(T, d), atol=1e-12)
        C = T.copy(); C[0, n - 1] += 0.6; C[n - 1, 0] += 0.8
        np.testing.assert_allclose(oracle.cyclic(a, b, c, 0.8, 0.6, d), np.linalg.solve(C, d), atol=1e-12)


def _pinned_exact(g, dz, periodic):
    """Zero-mean solution of the 1-D cell-centred singular problem (u_{k-1} - 2 u_k + u_{k+1}) / dz^2
    = g_k - mean(g), Neumann ends (u_{-1} = u_0, u_n = u_{n-1}) or periodic, in exact rational
    arithmetic: u_0 pinned to 0, rows 1..n-1 by elimination, then the mean subtracted."""
    from fractions import Fraction as Fr
    n = len(g)
    h2 = 1 / (Fr(dz) * Fr(dz))
    gf = [Fr(float(x)) for x in g]
    mean = sum(gf) / n
    d = [x - mean for x in gf]
    m = n - 1
    b = [-2 * h2] * m
    if not periodic:
        b[-1] = -h2  # Neumann top: the ghost equals the last cell
    cp, dp = [Fr(0)] * m, [Fr(0)] * m
    cp[0], dp[0] = h2 / b[0], d[1] / b[0]
    for i in range(1, m):
        mm = b[i] - h2 * cp[i - 1]
        cp[i] = h2 / mm
        dp[i] = (d[i + 1] - h2 * dp[i - 1]) / mm
    x = [Fr(0)] * m
    x[-1] = dp[-1]
    for i in range(m - 2, -1, -1):
        x[i] = dp[i] - cp[i] * x[i + 1]
    u = [Fr(0)] + x
    mu = sum(u) / n
    return np.array([float(v - mu) for v in u])


@pytest.mark.parametrize("n,tol", [(64, 1e-13), (256, 1e-12)])
@pytest.mark.parametrize("bcz", ["NN", "PP"])
def test_singular_mode_exact_rational(oracle, n, tol, bcz):
    """The pinned singular mode (Sec. "Well-posedness") against exact rational arithmetic: a source
    constant in x and y with a non-zero mean has only the (0,0) mode, so the oracle's solution is
    the 1-D zero-mean solution in every column."""
    rng = np.random.default_rng(n)
    g = rng.uniform(0, 1, size=n)
    f = np.broadcast_to(g[:, None, None], (n, 2, 2)).copy()
    sp = (0.5, 0.5, 1.0 / n)
    u = oracle.solve(f, "NNNN" + bcz, sp)
    ue = _pinned_exact(g, sp[2], bcz == "PP")
    assert np.abs(u - u[:, :1, :1]).max() <= 1e-13 * np.abs(u).max()
    assert np.linalg.norm(u[:, 0, 0] - ue) / np.linalg.norm(ue) <= tol
