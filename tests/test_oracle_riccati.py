"""Pins of the oracle's step-2 Riccati solve: it must equal the dense KKT
solution of the same equality-constrained LQ problem, and reduce to
discrete-time LQR on a long time-invariant horizon."""
import numpy as np
import pytest
import scipy.linalg


def _rand_lq(rng, N, ns, nu):
    A = np.eye(ns)[None] + 0.1 * rng.normal(size=(N, ns, ns))
    B = 0.2 * rng.normal(size=(N, ns, nu))
    c = 0.1 * rng.normal(size=(N, ns))
    Q = np.zeros((N + 1, ns, ns))
    for t in range(N + 1):
        L = rng.normal(size=(ns, ns))
        Q[t] = L @ L.T / ns + 0.1 * np.eye(ns)
    R = np.zeros((N, nu, nu))
    for t in range(N):
        L = rng.normal(size=(nu, nu))
        R[t] = L @ L.T / nu + 0.1 * np.eye(nu)
    q = rng.normal(size=(N + 1, ns))
    r = rng.normal(size=(N, nu))
    s0 = rng.normal(size=ns)
    return A, B, c, Q, q, R, r, s0


def _dense_kkt(A, B, c, Q, q, R, r, s0):
    N, ns, nu = B.shape
    nz = (N + 1) * ns + N * nu
    H = np.zeros((nz, nz))
    g = np.zeros(nz)
    si = lambda t: slice(t * ns, (t + 1) * ns)
    ui = lambda t: slice((N + 1) * ns + t * nu, (N + 1) * ns + (t + 1) * nu)
    for t in range(N + 1):
        H[si(t), si(t)] = Q[t]
        g[si(t)] = q[t]
    for t in range(N):
        H[ui(t), ui(t)] = R[t]
        g[ui(t)] = r[t]
    ne = (N + 1) * ns
    E = np.zeros((ne, nz))
    e = np.zeros(ne)
    E[0:ns, si(0)] = np.eye(ns)
    e[0:ns] = s0
    for t in range(N):
        row = slice((t + 1) * ns, (t + 2) * ns)
        E[row, si(t + 1)] = np.eye(ns)
        E[row, si(t)] = -A[t]
        E[row, ui(t)] = -B[t]
        e[row] = c[t]
    KKT = np.block([[H, E.T], [E, np.zeros((ne, ne))]])
    sol = np.linalg.solve(KKT, np.concatenate([-g, e]))
    z = sol[:nz]
    return z[:(N + 1) * ns].reshape(N + 1, ns), z[(N + 1) * ns:].reshape(N, nu)


@pytest.mark.parametrize("ns,nu,N", [(4, 2, 20), (5, 2, 50), (12, 4, 40)])
def test_riccati_equals_dense_kkt(ora, ns, nu, N):
    rng = np.random.default_rng(ns * 100 + N)
    prob = _rand_lq(rng, N, ns, nu)
    s, u, st = ora.riccati(*prob)
    assert st == 0
    s_ref, u_ref = _dense_kkt(*prob)
    assert np.abs(s - s_ref).max() < 1e-8 * (1 + np.abs(s_ref).max())
    assert np.abs(u - u_ref).max() < 1e-8 * (1 + np.abs(u_ref).max())


def test_riccati_long_horizon_is_lqr(ora):
    """Time-invariant, no affine terms: the first control of a long horizon
    is -K_inf s0 with K_inf from the discrete algebraic Riccati equation
    (costs 0.5 s'Qs + 0.5 u'Ru)."""
    rng = np.random.default_rng(3)
    ns, nu, N = 4, 2, 400
    A1 = np.eye(ns) + 0.05 * rng.normal(size=(ns, ns))
    B1 = 0.3 * rng.normal(size=(ns, nu))
    Q1 = np.diag(rng.uniform(0.5, 2, ns))
    R1 = np.diag(rng.uniform(0.5, 2, nu))
    A = np.repeat(A1[None], N, 0)
    B = np.repeat(B1[None], N, 0)
    Q = np.repeat(Q1[None], N + 1, 0)
    R = np.repeat(R1[None], N, 0)
    s0 = rng.normal(size=ns)
    s, u, st = ora.riccati(A, B, np.zeros((N, ns)), Q, np.zeros((N + 1, ns)), R, np.zeros((N, nu)), s0)
    P = scipy.linalg.solve_discrete_are(A1, B1, Q1, R1)
    K = np.linalg.solve(R1 + B1.T @ P @ B1, B1.T @ P @ A1)
    assert np.abs(u[0] + K @ s0).max() < 1e-8
