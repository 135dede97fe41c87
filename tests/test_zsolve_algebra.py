"""The algebra the z kernel uses, checked in FP64 on the CPU against dense solves: the Thomas
sweeps with the multipliers w_k = 1/(b_k - w_{k-1}) (rows scaled so the off-diagonals are 1),
and the cyclic (periodic z) solve by Sherman-Morrison where the back substitution runs directly
on v = y - c p (p = A'^{-1} e_{n-1}), so that x_k = v_k - c gamma q_k with q = A'^{-1} e_0."""
import numpy as np
import pytest


def _thomas_mult(b):
    w = np.empty(len(b))
    w[0] = 1.0 / b[0]
    for k in range(1, len(b)):
        w[k] = 1.0 / (b[k] - w[k - 1])
    return w


def _sweeps(w, d, v_last=None):
    n = len(d)
    g = np.empty(n)
    g[0] = d[0] * w[0]
    for k in range(1, n):
        g[k] = (d[k] - g[k - 1]) * w[k]
    u = np.empty(n)
    u[n - 1] = g[n - 1] if v_last is None else v_last(g[n - 1])
    for k in range(n - 2, -1, -1):
        u[k] = g[k] - w[k] * u[k + 1]
    return g, u


@pytest.mark.parametrize("n,shift", [(7, 0.3), (64, 1e-3), (200, 2.5)])
def test_thomas_multipliers_match_dense(n, shift):
    rng = np.random.default_rng(n)
    beta = -2.0 - shift
    b = np.full(n, beta)
    b[0] += 1.0   # Neumann bottom face
    b[-1] -= 1.0  # Dirichlet top face
    A = np.diag(b) + np.diag(np.ones(n - 1), 1) + np.diag(np.ones(n - 1), -1)
    d = rng.uniform(-1, 1, n)
    _, u = _sweeps(_thomas_mult(b), d)
    assert np.allclose(u, np.linalg.solve(A, d), rtol=0, atol=1e-12 * np.abs(u).max())


@pytest.mark.parametrize("n,shift", [(5, 0.7), (64, 1e-3), (300, 0.05)])
def test_cyclic_back_substitution_on_v(n, shift):
    rng = np.random.default_rng(100 + n)
    beta = -2.0 - shift
    A = np.diag(np.full(n, beta)) + np.diag(np.ones(n - 1), 1) + np.diag(np.ones(n - 1), -1)
    A[0, -1] = A[-1, 0] = 1.0
    d = rng.uniform(-1, 1, n)
    # A = A' + u v^T with u = (gamma, 0.., 1), v = (1, 0.., 1/gamma), gamma = -b_0
    gamma = -beta
    b = np.full(n, beta)
    b[0] -= gamma
    b[-1] -= 1.0 / gamma
    Ap = np.diag(b) + np.diag(np.ones(n - 1), 1) + np.diag(np.ones(n - 1), -1)
    w = _thomas_mult(b)
    q = np.linalg.solve(Ap, np.eye(n)[0])
    g, y = _sweeps(w, d)
    y0 = q @ d                     # first entry of y = A'^{-1} d (A' symmetric)
    p_last = w[-1]                 # (A'^{-1})_{n-1,n-1} = w_{n-1}
    z0 = gamma * q[0] + q[-1]
    zn = gamma * q[-1] + p_last
    c = (y0 + y[-1] / gamma) / (1.0 + z0 + zn / gamma)
    # back substitution on v = y - c p, started from v_{n-1} = g_{n-1} - c w_{n-1}
    _, v = _sweeps(w, d, v_last=lambda gl: gl - c * p_last)
    x = v - c * gamma * q
    ref = np.linalg.solve(A, d)
    assert np.allclose(x, ref, rtol=0, atol=1e-11 * np.abs(ref).max())
    # the same through p explicitly
    p = np.linalg.solve(Ap, np.eye(n)[-1])
    assert np.allclose(v, y - c * p, rtol=0, atol=1e-11 * np.abs(ref).max())
