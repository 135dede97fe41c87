"""Test helpers that come from the problem's definition, not from either solver.

* ``assemble``: the dense cell-centred 7-point matrix A_h, written from the stencil
  and the face ghost rules (periodic wrap, Neumann u[-1]=u[0], homogeneous
  Dirichlet u[-1]=-u[0]).
* ``mms``: manufactured eigenfunction products and the exact discrete solution
  u = u* . (-sum(k^2) / sum(lambda_d(k))), lambda_d(k) = (2 cos(k h) - 2)/h^2.
"""
import numpy as np

from paper_1909_05423_gb300 import workloads

AXIS_KINDS = ["PP", "NN", "DD", "DN", "ND"]


def assemble(nx, ny, nz, bc, spacing=(1.0, 1.0, 1.0)):
    n = nx * ny * nz
    A = np.zeros((n, n))
    hs = spacing
    dims = (nx, ny, nz)

    def flat(i, j, k):
        return (k * ny + j) * nx + i

    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                p = flat(i, j, k)
                idx = [i, j, k]
                for ax in range(3):
                    w = 1.0 / hs[ax] ** 2
                    A[p, p] -= 2.0 * w
                    for side, step in ((0, -1), (1, 1)):
                        q = list(idx)
                        q[ax] += step
                        face = bc[2 * ax + side]
                        if 0 <= q[ax] < dims[ax]:
                            A[p, flat(*q)] += w
                        elif face == "P":
                            q[ax] %= dims[ax]
                            A[p, flat(*q)] += w
                        elif face == "N":
                            A[p, p] += w
                        else:  # D
                            A[p, p] -= w
    return A


def dense_solve(f, bc, spacing=(1.0, 1.0, 1.0)):
    """Dense Gaussian elimination; with no Dirichlet face the bordered system
    [A 1; 1^T 0] [u; mu] = [f - mean f; 0] gives the zero-mean solution."""
    nz, ny, nx = f.shape
    A = assemble(nx, ny, nz, bc, spacing)
    b = f.reshape(-1)
    if "D" not in bc:
        n = b.size
        B = np.zeros((n + 1, n + 1))
        B[:n, :n] = A
        B[:n, n] = 1.0
        B[n, :n] = 1.0
        rhs = np.concatenate([b - b.mean(), [0.0]])
        return np.linalg.solve(B, rhs)[:n].reshape(f.shape)
    return np.linalg.solve(A, b).reshape(f.shape)


def lambda_d(kappa, h):
    return (2.0 * np.cos(kappa * h) - 2.0) / (h * h)


def mms_terms(bc, kx, ky, kz):
    """Real manufactured products for the face conditions: sin for D-D, cos for N-N,
    and for periodic axes both cos and sin (the real and imaginary parts of e^{ikx})."""
    per_axis = []
    for ax, k in enumerate((kx, ky, kz)):
        pair = bc[2 * ax: 2 * ax + 2]
        if pair == "DD":
            per_axis.append([("sin", k)])
        elif pair == "NN":
            per_axis.append([("cos", k)])
        elif pair == "PP":
            per_axis.append([("cos", k), ("sin", k)])
        else:
            raise ValueError(pair)
    return per_axis


def discrete_solution_ratio(kappas, hs):
    """Laplacian(u*) = -sum(k^2) u*, and A_h u* = sum(lambda_d) u* for a sampled eigenfunction,
    so the discrete solution of A_h u = Laplacian(u*) is u* * (-sum k^2 / sum lambda_d)."""
    return -sum(k * k for k in kappas) / sum(lambda_d(k, h) for k, h in zip(kappas, hs))


def mms_field(shape, spacing, comps):
    """One real product (amp 1) of per-axis components [(fx,kx),(fy,ky),(fz,kz)]."""
    return workloads.manufactured(shape, spacing, [(1.0, comps[0], comps[1], comps[2])])
