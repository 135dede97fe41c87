"""Pins of the oracle's faces with data (Dirichlet face values, Neumann outward normal
derivatives), CPU only.

The ghost rules u_ghost = 2 g - u_inside (Dirichlet, linear extrapolation to the face value) and
u_ghost = u_inside + h q (Neumann) are exact for functions that are linear across the face, and
the Neumann rule is exact for quadratics too, while the cell-centred second difference is exact
for quadratics.  So for such manufactured solutions the discrete problem has the sampled
function itself as its solution; a wrong factor, sign or normal direction in the fold breaks
that.  A smooth non-polynomial solution checks second-order convergence for every face pair.
"""
import numpy as np
import pytest

import oracle

# face order x-, x+, y-, y+, z-, z+ ; axis of each face and whether it is the high face
FACE_AXIS = [0, 0, 1, 1, 2, 2]


def cell_centres(shape, spacing):
    nz, ny, nx = shape
    hx, hy, hz = spacing
    x = (np.arange(nx) + 0.5) * hx
    y = (np.arange(ny) + 0.5) * hy
    z = (np.arange(nz) + 0.5) * hz
    return np.meshgrid(z, y, x, indexing="ij")  # Z, Y, X arrays of shape (nz, ny, nx)


def face_data(bc, shape, spacing, u, grad):
    """Face values (D) or outward normal derivatives (N) of the function u(x, y, z) with
    gradient grad(x, y, z) -> (ux, uy, uz), at the face centres; None on periodic faces."""
    nz, ny, nx = shape
    hx, hy, hz = spacing
    L = (nx * hx, ny * hy, nz * hz)
    x = (np.arange(nx) + 0.5) * hx
    y = (np.arange(ny) + 0.5) * hy
    z = (np.arange(nz) + 0.5) * hz
    out = []
    for face, c in enumerate(bc):
        if c == "P":
            out.append(None)
            continue
        ax, hi = FACE_AXIS[face], face % 2
        pos = L[ax] if hi else 0.0
        if ax == 0:
            Zg, Yg = np.meshgrid(z, y, indexing="ij")
            X, Y, Z = np.full_like(Zg, pos), Yg, Zg
        elif ax == 1:
            Zg, Xg = np.meshgrid(z, x, indexing="ij")
            X, Y, Z = Xg, np.full_like(Zg, pos), Zg
        else:
            Yg, Xg = np.meshgrid(y, x, indexing="ij")
            X, Y, Z = Xg, Yg, np.full_like(Yg, pos)
        if c == "D":
            out.append(u(X, Y, Z))
        else:
            d = grad(X, Y, Z)[ax]
            out.append(d if hi else -d)
    return out


BCS = ["DDDDDD", "NNNNNN", "DNNDND", "NDDNDN", "NNDDNN", "DDNNDD", "PPDNND", "NDPPDD", "DNNDPP"]


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("bc", BCS)
def test_linear_solution_is_exact(bc):
    """u* linear in the non-periodic coordinates (times a discrete Fourier mode along each
    periodic axis): the ghosts are exact, so solving with the exact discrete source returns u*."""
    shape, sp = (6, 5, 7), (0.3, 0.45, 0.25)
    nz, ny, nx = shape
    L = (nx * sp[0], ny * sp[1], nz * sp[2])
    coef = (0.7, -1.3, 0.4)
    per = [bc[2 * a] == "P" for a in range(3)]

    def parts(X, Y, Z):
        # per axis: linear factor a + b t on non-periodic axes, cos(2 pi t / L) on periodic ones
        out = []
        for a, t in enumerate((X, Y, Z)):
            if per[a]:
                out.append((np.cos(2 * np.pi * t / L[a]), -2 * np.pi / L[a] * np.sin(2 * np.pi * t / L[a])))
            else:
                out.append((1.0 + coef[a] * t, coef[a] * np.ones_like(t)))
        return out

    def u(X, Y, Z):
        (fx, _), (fy, _), (fz, _) = parts(X, Y, Z)
        return fx * fy * fz

    def grad(X, Y, Z):
        (fx, dx), (fy, dy), (fz, dz) = parts(X, Y, Z)
        return dx * fy * fz, fx * dy * fz, fx * fy * dz

    Z, Y, X = cell_centres(shape, sp)
    us = u(X, Y, Z)
    # exact discrete source: the second difference of a linear factor is 0; a periodic cosine
    # factor is an eigenvector with eigenvalue (2 cos(2 pi h / L) - 2) / h^2
    lam = sum((2 * np.cos(2 * np.pi * sp[a] / L[a]) - 2) / sp[a] ** 2 for a in range(3) if per[a])
    f = lam * us
    faces = face_data(bc, shape, sp, u, grad)
    got = oracle.solve_g(f, bc, sp, faces)
    if "D" not in bc:
        got, us = got - got.mean(), us - us.mean()
    assert _rel(got, us) < 1e-12, _rel(got, us)
    # and the operator itself reproduces the exact source
    assert np.abs(oracle.laplacian_g(u(X, Y, Z), bc, sp, faces) - f).max() < 1e-10


@pytest.mark.parametrize("bc", ["NNNNNN", "NNNNPP", "PPNNNN"])
def test_quadratic_neumann_is_exact(bc):
    """Neumann ghosts are exact for quadratics and so is the second difference: with f = the
    (constant) Laplacian and the outward derivatives as data, the zero-mean solution is u*."""
    shape, sp = (5, 6, 4), (0.2, 0.3, 0.25)
    nz, ny, nx = shape
    L = (nx * sp[0], ny * sp[1], nz * sp[2])
    per = [bc[2 * a] == "P" for a in range(3)]
    q = [(0.0 if per[0] else 1.0), (0.0 if per[1] else -0.5), (0.0 if per[2] else 0.75)]
    cxy = 0.0 if (per[0] or per[1]) else 0.6

    def u(X, Y, Z):
        return q[0] * X ** 2 + q[1] * Y ** 2 + q[2] * Z ** 2 + cxy * X * Y + 0.3

    def grad(X, Y, Z):
        return 2 * q[0] * X + cxy * Y, 2 * q[1] * Y + cxy * X, 2 * q[2] * Z

    Z, Y, X = cell_centres(shape, sp)
    f = np.full(shape, 2 * (q[0] + q[1] + q[2]))
    faces = face_data(bc, shape, sp, u, grad)
    got = oracle.solve_g(f, bc, sp, faces)
    us = u(X, Y, Z)
    assert _rel(got - got.mean(), us - us.mean()) < 1e-12


@pytest.mark.parametrize("bc", ["DDDDDD", "NNDDNN", "DNNDND", "NDDNDN", "PPDNND"])
def test_second_order_convergence(bc):
    """Smooth manufactured solution with non-zero face data: the error falls by ~4 per halving."""
    per = [bc[2 * a] == "P" for a in range(3)]

    def u(X, Y, Z):
        fx = np.cos(2 * np.pi * X) if per[0] else np.cos(1.1 * X + 0.3)
        return fx * np.sin(0.9 * Y + 0.5) * np.cosh(0.7 * Z)

    def grad(X, Y, Z):
        fx = np.cos(2 * np.pi * X) if per[0] else np.cos(1.1 * X + 0.3)
        dfx = -2 * np.pi * np.sin(2 * np.pi * X) if per[0] else -1.1 * np.sin(1.1 * X + 0.3)
        return (dfx * np.sin(0.9 * Y + 0.5) * np.cosh(0.7 * Z), fx * 0.9 * np.cos(0.9 * Y + 0.5) * np.cosh(0.7 * Z),
                fx * np.sin(0.9 * Y + 0.5) * 0.7 * np.sinh(0.7 * Z))

    def lap(X, Y, Z):
        kx2 = (2 * np.pi) ** 2 if per[0] else 1.1 ** 2
        return (-kx2 - 0.81 + 0.49) * u(X, Y, Z)

    errs = []
    for n in (8, 16, 32):
        shape, sp = (n, n, n), (1.0 / n,) * 3
        Z, Y, X = cell_centres(shape, sp)
        got = oracle.solve_g(lap(X, Y, Z), bc, sp, face_data(bc, shape, sp, u, grad))
        us = u(X, Y, Z)
        if "D" not in bc:
            got, us = got - got.mean(), us - us.mean()
        errs.append(np.sqrt(np.mean((got - us) ** 2)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.5 < r2 < 4.5 and 3.0 < r1 < 5.0, errs


def test_periodic_face_data_rejected():
    with pytest.raises(ValueError):
        oracle.fold_bc(np.zeros((3, 4, 4)), "PPNNDD", (1, 1, 1), [np.zeros((3, 4)), None, None, None, None, None])
