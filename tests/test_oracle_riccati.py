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


# ---- parallel-in-time form (ora_riccati_scan) ---------------------------------

@pytest.mark.parametrize("ns,nu,N", [(4, 2, 20), (5, 2, 50), (12, 4, 16), (12, 4, 40), (3, 1, 1), (5, 2, 63)])
def test_riccati_scan_equals_dense_kkt(ora, ns, nu, N):
    """The associative composition of the stage relations solves the same LQ
    problem: the dense KKT solution, in both composition orders."""
    rng = np.random.default_rng(ns * 1000 + N)
    prob = _rand_lq(rng, N, ns, nu)
    s_ref, u_ref = _dense_kkt(*prob)
    for tree in (True, False):
        s, u, P, p, st = ora.riccati_scan(*prob, tree=tree)
        assert st == 0
        assert np.abs(s - s_ref).max() < 1e-8 * (1 + np.abs(s_ref).max())
        assert np.abs(u - u_ref).max() < 1e-8 * (1 + np.abs(u_ref).max())


def test_riccati_scan_orders_agree_and_value_function_is_valid(ora):
    """Associativity: pairwise rounds and the right-to-left fold give the same
    value functions; each P_t is symmetric positive semidefinite and equals
    Q_N at the terminal stage."""
    rng = np.random.default_rng(17)
    prob = _rand_lq(rng, 37, 6, 3)
    _, _, P1, p1, _ = ora.riccati_scan(*prob, tree=True)
    _, _, P2, p2, _ = ora.riccati_scan(*prob, tree=False)
    assert np.abs(P1 - P2).max() < 1e-10 * (1 + np.abs(P2).max())
    assert np.abs(p1 - p2).max() < 1e-10 * (1 + np.abs(p2).max())
    Q = prob[3]
    assert np.array_equal(P1[-1], Q[-1]) and np.array_equal(p1[-1], prob[4][-1])
    for t in range(P1.shape[0]):
        assert np.abs(P1[t] - P1[t].T).max() < 1e-10 * (1 + np.abs(P1[t]).max())
        assert np.linalg.eigvalsh(0.5 * (P1[t] + P1[t].T)).min() > -1e-10


def test_riccati_scan_costate_is_cost_gradient(ora):
    """lam_0 = P_0 s_0 + p_0 is the gradient of the optimal cost in s_0: central
    differences of the dense KKT optimum (a quadratic in s_0, so exact up to
    rounding)."""
    rng = np.random.default_rng(23)
    A, B, c, Q, q, R, r, s0 = _rand_lq(rng, 12, 4, 2)

    def cost(x0):
        s, u = _dense_kkt(A, B, c, Q, q, R, r, x0)
        return (sum(0.5 * s[t] @ Q[t] @ s[t] + q[t] @ s[t] for t in range(len(s)))
                + sum(0.5 * u[t] @ R[t] @ u[t] + r[t] @ u[t] for t in range(len(u))))

    _, _, P, p, st = ora.riccati_scan(A, B, c, Q, q, R, r, s0)
    assert st == 0
    h = 1e-4
    g = np.array([(cost(s0 + h * e) - cost(s0 - h * e)) / (2 * h) for e in np.eye(len(s0))])
    lam = P[0] @ s0 + p[0]
    assert np.abs(g - lam).max() < 1e-6 * (1 + np.abs(lam).max())
