"""Independent reference computations used to pin the oracle.

Nothing here calls the oracle: each function computes a quantity the paper
fixes (the scale LP's optimum, the pair QP's optimum, ...) by brute force or
a closed form, so that the oracle can be checked against it.
"""
import itertools
import math

import numpy as np

from paper_2406_07048_gb300 import synth


# ----------------------------------------------------------------------------
# random single problems (body frame of the robot part)
# ----------------------------------------------------------------------------

def random_pair(rng, dim, nf_obs=None, dist=None, rot=True):
    """Robot box (A, b) and an obstacle (Cb, db) placed at a random offset."""
    if dim == 2:
        half = rng.uniform(0.5, 2.5, 2)
        A, b = synth.box_halfspaces(half)
        nf = nf_obs or int(rng.integers(3, 9))
        C, off = synth.random_polygon(rng, nf, 0.5, 2.0)
    else:
        half = rng.uniform(0.05, 0.5, 3)
        A, b = synth.box_halfspaces(half)
        nf = nf_obs or int(rng.integers(6, 11))
        C, off = synth.random_polyhedron(rng, nf, 0.3, 1.5)
    if rot:
        # rotate the robot box so faces are not axis aligned
        if dim == 2:
            a = rng.uniform(0, 2 * math.pi)
            Rr = np.array([[math.cos(a), -math.sin(a)], [math.sin(a), math.cos(a)]])
        else:
            Rr, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        A = A @ Rr.T
    r = dist if dist is not None else rng.uniform(0.0, 6.0 if dim == 2 else 2.0)
    u = rng.normal(size=dim)
    ctr = r * u / np.linalg.norm(u)
    db = off + C @ ctr
    return A, b, C, db


# ----------------------------------------------------------------------------
# scale LP pins
# ----------------------------------------------------------------------------

def alpha_dual_enum(A, b, C, d):
    """alpha* = max -d^T mu over all basic feasible solutions of the dual
    (eqn:scale_opt_dual): enumerate every (dim+1)-subset of columns."""
    dim = A.shape[1]
    nr, no = len(b), len(d)
    E = np.zeros((dim + 1, nr + no))
    E[0, :nr] = b
    E[1:, :nr] = A.T
    E[1:, nr:] = C.T
    rhs = np.zeros(dim + 1)
    rhs[0] = 1.0
    cost = np.concatenate([np.zeros(nr), -d])
    best = -np.inf
    for S in itertools.combinations(range(nr + no), dim + 1):
        B = E[:, S]
        if abs(np.linalg.det(B)) < 1e-12:
            continue
        yB = np.linalg.solve(B, rhs)
        if np.all(yB >= -1e-10):
            best = max(best, float(cost[list(S)] @ yB))
    return best


def polygon_vertices(C, d):
    """Vertices of {x: C x <= d} in 2D by pairwise intersection."""
    V = []
    for i, j in itertools.combinations(range(len(d)), 2):
        M = C[[i, j]]
        if abs(np.linalg.det(M)) < 1e-12:
            continue
        x = np.linalg.solve(M, d[[i, j]])
        if np.all(C @ x <= d + 1e-9):
            V.append(x)
    return np.array(V)


def alpha_geom_2d(A, b, C, d):
    """alpha* = min over the obstacle of the robot's gauge max_k a_k.x / b_k.
    The gauge is linear on each cone of the fan through the robot's
    vertices, so the minimum over the obstacle polygon is attained at an
    obstacle vertex, at an obstacle-edge crossing of a fan ray, or at the
    origin when the origin lies in the obstacle."""
    if np.all(d >= 0):
        return 0.0
    gauge = lambda x: float(np.max(A @ x / b))
    cands = list(polygon_vertices(C, d))
    for rv in polygon_vertices(A, b):
        for m in range(len(d)):
            den = C[m] @ rv
            if abs(den) < 1e-14:
                continue
            t = d[m] / den
            if t < 0:
                continue
            x = t * rv
            if np.all(C @ x <= d + 1e-9):
                cands.append(x)
    return min(gauge(x) for x in cands)


def sat_overlap_2d(A, b, C, d):
    """Separating-axis test of the two polygons (interior overlap)."""
    P, Q = polygon_vertices(A, b), polygon_vertices(C, d)
    for n in np.vstack([A, C]):
        n = n / np.linalg.norm(n)
        a, bq = P @ n, Q @ n
        if a.max() <= bq.min() + 1e-12 or bq.max() <= a.min() + 1e-12:
            return False
    return True


# ----------------------------------------------------------------------------
# pair QP pins
# ----------------------------------------------------------------------------

def build_K(A, b, C, d):
    """Rows of K (eqn:const_least_square) and kappa in the body frame."""
    dim = A.shape[1]
    nr, no = len(b), len(d)
    K = np.zeros((nr + no + 1, dim + 1))
    K[:nr, 1:] = A
    K[nr:nr + no, 0] = d
    K[nr:nr + no, 1:] = C
    K[-1, 0] = 1.0
    kappa = np.zeros(nr + no + 1)
    kappa[:nr] = b
    return K, kappa


def qp_brute_prox0(K, kappa, bq):
    """min 0.5|K^T y + bq|^2 s.t. kappa^T y = 1, y >= 0 by enumerating every
    support S of at most dim+2 generators with a robot face: the optimum is
    the affine minimiser of some such support."""
    n, V = K.shape
    lam = [i for i in range(n) if kappa[i] > 0]
    best = np.inf
    best_v = None
    for k in range(1, V + 2):
        for S in itertools.combinations(range(n), k):
            if not any(i in lam for i in S):
                continue
            G = K[list(S)]          # k x V
            ks = kappa[list(S)]
            # KKT of min 0.5|G^T y + bq|^2 s.t. ks^T y = 1
            M = np.zeros((k + 1, k + 1))
            M[:k, :k] = G @ G.T
            M[:k, k] = ks
            M[k, :k] = ks
            rhs = np.concatenate([-G @ bq, [1.0]])
            sol = np.linalg.lstsq(M, rhs, rcond=None)[0]
            y = sol[:k]
            if abs(ks @ y - 1) > 1e-8 or np.any(y < -1e-10):
                continue
            v = G.T @ y + bq
            if np.linalg.norm(M @ sol - rhs) > 1e-7:
                continue
            o = 0.5 * float(v @ v)
            if o < best:
                best, best_v = o, v
    return best, best_v


def qp_brute_prox(K, kappa, bq, prox, ybar):
    """min 0.5|K^T y + bq|^2 + 0.5 prox sum_i |K_i|^2 (y_i - ybar_i)^2
    s.t. kappa^T y = 1, y >= 0 (strictly convex): the minimum over every
    face {y_i = 0, i not in F} of the face's equality-constrained
    minimiser, when feasible."""
    n, V = K.shape
    Dg = (K ** 2).sum(axis=1)
    best, best_y = np.inf, None
    for k in range(1, n + 1):
        for F in itertools.combinations(range(n), k):
            F = list(F)
            if not np.any(kappa[F] > 0):
                continue
            G = K[F]
            M = np.zeros((k + 1, k + 1))
            M[:k, :k] = G @ G.T + prox * np.diag(Dg[F])
            M[:k, k] = kappa[F]
            M[k, :k] = kappa[F]
            rhs = np.concatenate([-G @ bq + prox * Dg[F] * ybar[F], [1.0]])
            sol = np.linalg.solve(M, rhs)
            yF = sol[:k]
            if np.any(yF < -1e-12):
                continue
            y = np.zeros(n)
            y[F] = yF
            v = K.T @ y + bq
            o = 0.5 * float(v @ v) + 0.5 * prox * float(Dg @ (y - ybar) ** 2)
            if o < best:
                best, best_y = o, y
    return best, best_y


def qp_kkt_residual(K, kappa, bq, y, prox=0.0, ybar=None):
    """Largest violation of the KKT conditions of the pair QP at y:
    primal feasibility, and g + nu kappa >= 0 with complementarity, where
    g = K (K^T y + bq) + prox Dg (y - ybar), Dg = |K_i|^2, and nu is fitted
    on the support."""
    g = K @ (K.T @ y + bq)
    if prox > 0:
        g = g + prox * (K ** 2).sum(axis=1) * (y - ybar)
    sup = [i for i in range(len(y)) if y[i] > 1e-9 and kappa[i] > 0]
    nu = -np.mean([g[i] / kappa[i] for i in sup]) if sup else -np.min(g[kappa > 0] / kappa[kappa > 0])
    s = g + nu * kappa
    viol = [abs(kappa @ y - 1.0), max(0.0, -y.min()), max(0.0, -s.min())]
    viol.append(np.max(np.abs(s * y)))
    return max(viol)


# ----------------------------------------------------------------------------
# certificate-margin pins (Sec. III-B weak duality)
# ----------------------------------------------------------------------------

def polytope_vertices(A, b):
    """Vertices of the bounded polytope {x: A x <= b} in 2-D or 3-D: every
    choice of dim faces whose normals are independent meets in one point;
    the feasible such points are the vertices."""
    dim = A.shape[1]
    out = []
    for S in itertools.combinations(range(len(b)), dim):
        M = A[list(S)]
        if abs(np.linalg.det(M)) < 1e-12:
            continue
        x = np.linalg.solve(M, b[list(S)])
        if np.all(A @ x <= b + 1e-9 * (1.0 + np.abs(b))):
            out.append(x)
    return np.array(out)


def random_certificate(rng, nr, no, kind):
    """Nonnegative (lambda, mu) that are in general NOT optimal: independent
    exponential draws, a sparse draw, or large multipliers."""
    if kind == 0:
        return rng.exponential(1.0, nr), rng.exponential(1.0, no)
    if kind == 1:
        lam = rng.exponential(1.0, nr) * (rng.uniform(size=nr) < 0.5)
        lam[rng.integers(nr)] += 0.5
        return lam, rng.exponential(2.0, no) * (rng.uniform(size=no) < 0.4)
    return rng.exponential(0.1, nr), rng.exponential(10.0, no)
