"""Pins of the oracle's scale LP (Sec. III-A eqn:scale_opt, Sec. III-B duality)."""
import numpy as np
import pytest

from tests import _pins
from paper_2406_07048_gb300 import synth


@pytest.mark.parametrize("dim", [2, 3])
def test_alpha_matches_dual_basis_enumeration(ora, dim):
    rng = np.random.default_rng(11 + dim)
    for _ in range(60):
        A, b, C, d = _pins.random_pair(rng, dim)
        al, lam, mu, x, st = ora.scale_lp(A, b, C, d)
        assert st == 0
        ref = _pins.alpha_dual_enum(A, b, C, d)
        assert al == pytest.approx(ref, rel=1e-10, abs=1e-10)


def test_alpha_matches_2d_geometric_brute_force(ora):
    rng = np.random.default_rng(5)
    for _ in range(150):
        A, b, C, d = _pins.random_pair(rng, 2)
        al = ora.scale_lp(A, b, C, d)[0]
        assert al == pytest.approx(_pins.alpha_geom_2d(A, b, C, d), rel=1e-9, abs=1e-9)


@pytest.mark.parametrize("dim", [2, 3])
def test_alpha_box_box_closed_form(ora, dim):
    """Axis-aligned box robot |x_i| <= h_i against box obstacle lo <= x <= hi:
    the gauge is separable, so alpha* = max_i dist(0, [lo_i, hi_i]) / h_i."""
    rng = np.random.default_rng(7)
    for _ in range(40):
        h = rng.uniform(0.2, 2.0, dim)
        A, b = synth.box_halfspaces(h)
        lo = rng.uniform(-6, 6, dim)
        hi = lo + rng.uniform(0.1, 3.0, dim)
        C, d = synth.box_halfspaces(np.ones(dim))
        d = np.where(np.arange(2 * dim) % 2 == 0, np.repeat(hi, 2), -np.repeat(lo, 2))
        dist = np.maximum(0, np.maximum(lo, -hi))
        al = ora.scale_lp(A, b, C, d)[0]
        assert al == pytest.approx(float(np.max(dist / h)), rel=1e-12, abs=1e-12)


def test_alpha_scaling_invariance(ora):
    """Scaling the robot by c divides alpha* by c."""
    rng = np.random.default_rng(3)
    for _ in range(40):
        A, b, C, d = _pins.random_pair(rng, 2)
        a1 = ora.scale_lp(A, b, C, d)[0]
        a2 = ora.scale_lp(A, 2.5 * b, C, d)[0]
        assert a2 == pytest.approx(a1 / 2.5, rel=1e-10, abs=1e-12)


@pytest.mark.parametrize("dim", [2, 3])
def test_strong_duality_and_feasibility(ora, dim):
    """The returned (lambda, mu) is dual feasible with -d^T mu = alpha*, and
    the returned x is primal feasible at alpha* (zero primal-dual gap)."""
    rng = np.random.default_rng(21)
    for _ in range(60):
        A, b, C, d = _pins.random_pair(rng, dim)
        al, lam, mu, x, st = ora.scale_lp(A, b, C, d)
        assert lam.min() >= -1e-12 and mu.min() >= -1e-12
        assert b @ lam == pytest.approx(1.0, abs=1e-10)
        assert np.abs(A.T @ lam + C.T @ mu).max() < 1e-9
        assert -d @ mu == pytest.approx(al, abs=1e-10)
        assert np.all(A @ x <= al * b + 1e-9)
        assert np.all(C @ x <= d + 1e-9)


def test_sat_verdict(ora):
    """alpha* < 1 iff the polygons overlap (separating-axis theorem)."""
    rng = np.random.default_rng(9)
    n_checked = 0
    for _ in range(200):
        A, b, C, d = _pins.random_pair(rng, 2)
        al = ora.scale_lp(A, b, C, d)[0]
        if abs(al - 1.0) < 1e-6:
            continue
        assert (al < 1.0) == _pins.sat_overlap_2d(A, b, C, d)
        n_checked += 1
    assert n_checked > 150


def test_origin_inside_gives_zero(ora):
    rng = np.random.default_rng(1)
    A, b, C, d = _pins.random_pair(rng, 2, dist=0.0)
    assert ora.scale_lp(A, b, C, d)[0] == pytest.approx(0.0, abs=1e-12)


def test_batch_matches_single_on_config_poses(ora):
    """The scene-level driver poses each part (Sec. IV-A y = R x + rho) and
    transforms the obstacle into the part frame; the result must equal the
    single-pair LP on C' = C R, d' = d - C rho computed here."""
    sc = synth.config2()
    rng = np.random.default_rng(0)
    st = synth.random_states(sc, rng)
    pairs = rng.choice(sc.n_pairs, 200, replace=False)
    r = ora.scale_batch(sc, st, pairs)
    N = int(sc.horizon[0])
    for l, p in enumerate(pairs):
        t = p % N + 1
        pt = (p // N) % 2
        j = p // (2 * N)
        s = st[t]
        if pt == 0:
            a = s[2]
            rho = s[:2] + np.array([[np.cos(a), -np.sin(a)], [np.sin(a), np.cos(a)]]) @ sc.part_off[0]
        else:
            a = s[4]
            th = s[2]
            hitch = s[:2] - sc.model.param[1] * np.array([np.cos(th), np.sin(th)])
            rho = hitch + np.array([[np.cos(a), -np.sin(a)], [np.sin(a), np.cos(a)]]) @ sc.part_off[1]
        R = np.array([[np.cos(a), -np.sin(a)], [np.sin(a), np.cos(a)]])
        nf = sc.obs_nf[j]
        C = sc.obs_C[j, :nf]
        d = sc.obs_d[j, :nf]
        al = ora.scale_lp(sc.part_A[pt], sc.part_b[pt], C @ R, d - C @ rho)[0]
        assert r["alpha"][l] == pytest.approx(al, rel=1e-12, abs=1e-12)
        assert r["margin"][l] == pytest.approx(al, rel=1e-8, abs=1e-8)


@pytest.mark.parametrize("dim", [2, 3])
def test_envelope_derivatives_match_central_differences(ora, dim):
    """Sensitivity of alpha* (Sec. III-B, the dual Lagrangian at fixed
    multipliers): dalpha/dd'_m = -mu_m and dalpha/dC'_mi = mu_m x_i, with
    (mu, x) the oracle's certificate and primal point, against central
    differences of the oracle's own alpha*.  Random pairs have a unique
    optimal basis with probability one; the few whose basis changes within
    the step are recognised by a one-sided disagreement and skipped."""
    rng = np.random.default_rng(40 + dim)
    h = 1e-7
    checked = 0
    for _ in range(60):
        A, b, C, d = _pins.random_pair(rng, dim)
        al, lam, mu, x, st = ora.scale_lp(A, b, C, d)
        assert st == 0
        f = lambda C2, d2: ora.scale_lp(A, b, C2, d2)[0]
        gd_fd, gc_fd = np.zeros(len(d)), np.zeros(C.shape)
        smooth = True
        for m in range(len(d)):
            e = np.zeros(len(d))
            e[m] = h
            fp, fm = f(C, d + e), f(C, d - e)
            smooth &= abs((fp - al) - (al - fm)) < 1e-6 * h * (1 + abs(al))
            gd_fd[m] = (fp - fm) / (2 * h)
            for i in range(dim):
                E = np.zeros(C.shape)
                E[m, i] = h
                gc_fd[m, i] = (f(C + E, d) - f(C - E, d)) / (2 * h)
        if not smooth:
            continue
        checked += 1
        assert np.allclose(gd_fd, -mu, atol=1e-6 * (1 + np.abs(mu).max()))
        assert np.allclose(gc_fd, np.outer(mu, x), atol=1e-6 * (1 + np.abs(np.outer(mu, x)).max()))
    assert checked >= 40


# ----------------------------------------------------------------------------
# The FP64 certificate margin (Sec. III-B weak duality) away from the LP
# optimum, where r = A^T lambda + C'^T mu != 0 and the part radius D matters.
# ----------------------------------------------------------------------------

def test_cert_margin_hand_derived_2d(ora):
    """Robot |x| <= 1, |y| <= 2 (vertices (+-1, +-2), so D = sqrt(5));
    obstacle 3 <= x <= 5, |y| <= 1 (alpha* = 3).  With lambda = 1 on the
    face x <= 1 and mu = t on the face -x <= -3 (and s on y <= 1):
      b^T lambda = 1,  -d^T mu = 3t - s,  r = (1 - t, s),
      margin = (3t - s) / (1 + sqrt((1 - t)^2 + s^2) sqrt(5)).
    t = 1, s = 0 is the LP certificate (margin = alpha* = 3)."""
    A, b = synth.box_halfspaces(np.array([1.0, 2.0]))
    C = np.array([[1.0, 0.0], [-1.0, 0.0], [0.0, 1.0], [0.0, -1.0]])
    d = np.array([5.0, -3.0, 1.0, 1.0])
    # face order of box_halfspaces: +x, -x, +y, -y
    assert np.allclose(A, C) and np.allclose(b, [1, 1, 2, 2])
    assert ora.scale_lp(A, b, C, d)[0] == pytest.approx(3.0, abs=1e-12)
    r5 = np.sqrt(5.0)
    for t, s, want in [(1.0, 0.0, 3.0), (0.5, 0.0, 1.5 / (1 + 0.5 * r5)), (2.0, 0.0, 6.0 / (1 + r5)),
                       (1.0, 0.25, 2.75 / (1 + 0.25 * r5)), (0.0, 0.0, 0.0 / (1 + r5))]:
        lam = np.array([1.0, 0.0, 0.0, 0.0])
        mu = np.array([0.0, t, s, 0.0])
        got = ora.cert_margin(A, b, C, d, lam, mu)
        assert got == pytest.approx(want, rel=1e-13, abs=1e-13), (t, s)
        assert got <= 3.0 + 1e-12


def test_cert_margin_hand_derived_3d(ora):
    """Robot box |x|, |y| <= 0.3, |z| <= 0.1 (D = sqrt(0.3^2 + 0.3^2 + 0.1^2));
    obstacle 1 <= z <= 2, |x|, |y| <= 1 (alpha* = 10).  lambda = 10 on z <= 0.1
    (b^T lambda = 1), mu = t on -z <= -1, s on x <= 1:
      -d^T mu = t - s,  r = (s, 0, 10 - t),
      margin = (t - s) / (1 + sqrt(s^2 + (10 - t)^2) D)."""
    A, b = synth.box_halfspaces(np.array([0.3, 0.3, 0.1]))
    C, _ = synth.box_halfspaces(np.ones(3))
    d = np.array([1.0, 1.0, 1.0, 1.0, 2.0, -1.0])
    assert ora.scale_lp(A, b, C, d)[0] == pytest.approx(10.0, abs=1e-11)
    D = np.sqrt(0.19)
    for t, s in [(10.0, 0.0), (5.0, 0.0), (12.0, 0.0), (9.0, 0.5), (10.0, 2.0)]:
        lam = np.zeros(6)
        lam[4] = 10.0
        mu = np.zeros(6)
        mu[5], mu[0] = t, s
        want = (t - s) / (1 + np.hypot(s, 10 - t) * D)
        assert ora.cert_margin(A, b, C, d, lam, mu) == pytest.approx(want, rel=1e-13, abs=1e-13), (t, s)


@pytest.mark.parametrize("dim", [2, 3])
def test_cert_margin_is_a_lower_bound(ora, dim):
    """Weak duality: for every lambda, mu >= 0 the margin is at most alpha*
    (brute-force dual-basis enumeration).  Random certificates have r far
    from 0, so a dropped |r| D term or a part radius that is too small shows
    up as a margin above alpha*."""
    rng = np.random.default_rng(70 + dim)
    above_naive = 0
    for _ in range(40):
        A, b, C, d = _pins.random_pair(rng, dim)
        al = _pins.alpha_dual_enum(A, b, C, d)
        mu_opt = ora.scale_lp(A, b, C, d)[2]
        cands = [_pins.random_certificate(rng, len(b), len(d), kind) for kind in range(3)]
        # the optimal mu scaled up next to a random lambda: -d^T mu / b^T lambda
        # alone would overstate alpha*; only the |r| D term keeps the bound valid
        lam = rng.exponential(1.0, len(b))
        cands.append((lam / (b @ lam), rng.uniform(1.5, 3.0) * mu_opt))
        for lam, mu in cands:
            m = ora.cert_margin(A, b, C, d, lam, mu)
            assert m <= al + 1e-10 * max(1.0, al)
            if -d @ mu / (b @ lam) > al + 1e-6:
                above_naive += 1
    assert above_naive >= 15


@pytest.mark.parametrize("dim", [2, 3])
def test_cert_margin_part_radius_and_rotation(ora, dim):
    """The radius entering the bound is the part's largest vertex norm:
    with lambda on one face and mu chosen so that r points from the centre
    to the farthest vertex, the bound must move exactly by that radius
    (vertices found by enumeration here); rotating the whole body frame
    leaves the margin unchanged."""
    rng = np.random.default_rng(90 + dim)
    for _ in range(20):
        A, b, C, d = _pins.random_pair(rng, dim)
        V = _pins.polytope_vertices(A, b)
        D = np.linalg.norm(V, axis=1).max()
        lam, mu = _pins.random_certificate(rng, len(b), len(d), 0)
        r = A.T @ lam + C.T @ mu
        m = ora.cert_margin(A, b, C, d, lam, mu)
        # solve the margin's definition for D: -d^T mu / m = b^T lambda + |r| D
        if abs(m) > 1e-6:
            D_implied = (-d @ mu / m - b @ lam) / np.linalg.norm(r)
            assert D_implied == pytest.approx(D, rel=1e-9)
        if dim == 2:
            a = rng.uniform(0, 2 * np.pi)
            Q = np.array([[np.cos(a), -np.sin(a)], [np.sin(a), np.cos(a)]])
        else:
            Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        m2 = ora.cert_margin(A @ Q.T, b, C @ Q.T, d, lam, mu)
        assert m2 == pytest.approx(m, rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("dim", [2, 3])
def test_cert_margin_tends_to_alpha_near_the_optimum(ora, dim):
    """Perturbing the LP's optimal certificate by eps moves the bound by
    O(eps): it approaches alpha* from below as eps -> 0."""
    rng = np.random.default_rng(110 + dim)
    for _ in range(20):
        A, b, C, d = _pins.random_pair(rng, dim)
        al, lam, mu, x, st = ora.scale_lp(A, b, C, d)
        gaps = []
        for eps in (1e-2, 1e-4, 1e-6):
            lp = lam + eps * rng.uniform(0, 1, len(lam))
            mp = mu + eps * rng.uniform(0, 1, len(mu))
            m = ora.cert_margin(A, b, C, d, lp, mp)
            assert m <= al + 1e-10 * max(1.0, al)
            gaps.append(al - m)
        assert gaps[2] < 1e-4 * max(1.0, al)
        assert gaps[2] <= gaps[0] + 1e-12
