"""Pins of the oracle's ADMM loop (Sec. IV-B) and its per-pair terms."""
import numpy as np
import pytest

from paper_2406_07048_gb300 import synth
from tests.test_oracle_riccati import _dense_kkt


def _pair_data(sc, p):
    """(scenario 0) obstacle j, part, t of pair p and its arrays."""
    N = int(sc.horizon[0])
    NP = sc.n_parts(0)
    t = p % N + 1
    pt = (p // N) % NP
    j = p // (N * NP)
    nf = int(sc.obs_nf[j])
    return j, pt, t, sc.obs_C[j, :nf], sc.obs_d[j, :nf]


@pytest.mark.parametrize("cfg", ["config1", "config2", "config4"])
def test_gn_jacobian_central_differences(ora, cfg):
    """J returned with r0 is the derivative of r0 = [T + zeta; R + xi] in s_t."""
    sc = synth.config4(n_scen=1, n_obs=8) if cfg == "config4" else getattr(synth, cfg)()
    rng = np.random.default_rng(1)
    st = synth.random_states(sc, rng, 0.3, 0.2)
    for p in rng.choice(sc.n_pairs, 12, replace=False):
        j, pt, t, C, d = _pair_data(sc, p)
        y = np.abs(rng.normal(0, 0.5, sc.ny_max))
        s = st[t]
        args = (sc.part_A[pt], C, d, sc.part_link[pt], sc.part_off[pt])
        xi = rng.normal(0, 0.1, sc.dim)
        r0, J = ora.pair_gn(sc.model, *args, s, y, sc.fr_max, sc.fo_max, 0.3, xi)
        h = 1e-6
        for a in range(sc.model.ns):
            e = np.zeros(sc.model.ns)
            e[a] = h
            rp = ora.pair_gn(sc.model, *args, s + e, y, sc.fr_max, sc.fo_max, 0.3, xi)[0]
            rm = ora.pair_gn(sc.model, *args, s - e, y, sc.fr_max, sc.fo_max, 0.3, xi)[0]
            assert np.abs((rp - rm) / (2 * h) - J[:, a]).max() < 1e-6 * (1 + np.abs(J).max())


def test_residual_zero_at_lp_certificate(ora):
    """At a collision-free pose, the LP certificate (lambda*, mu*) with
    gamma = alpha* - 1 makes T = R = 0 (Sec. IV-A with eqn:poly_colli_free_conts)."""
    sc = synth.config2()
    rng = np.random.default_rng(2)
    st = synth.random_states(sc, rng)
    pairs = rng.choice(sc.n_pairs, 80, replace=False)
    lp = ora.scale_batch(sc, st, pairs)
    n = 0
    for l, p in enumerate(pairs):
        if lp["alpha"][l] < 1.0:
            continue
        j, pt, t, C, d = _pair_data(sc, p)
        y = np.zeros(sc.ny_max)
        y[:sc.fr_max] = lp["lam"][l]
        y[sc.fr_max:sc.fr_max + sc.fo_max] = lp["mu"][l]
        y[-1] = lp["alpha"][l] - 1.0
        r0, _ = ora.pair_gn(sc.model, sc.part_A[pt], C, d, sc.part_link[pt], sc.part_off[pt], st[t], y,
                            sc.fr_max, sc.fo_max, 0.0, np.zeros(2))
        assert np.abs(r0).max() < 1e-9
        n += 1
    assert n > 40


@pytest.mark.parametrize("damp,rho_box", [(0.0, 0.0), (100.0, 100.0), (7.0, 30.0)])
def test_one_iteration_step2_matches_dense_assembly(ora, damp, rho_box):
    """After one iteration, s^1 and u^1 equal the dense-KKT solution of the
    step-2 problem built here independently: linearised Euler dynamics at
    (s^0, u^0), tracking cost of eqn:navigation_cost, the Gauss-Newton
    penalty sigma/2 |r0 + J (s_t - s_t^0)|^2 of every pair with y^1, the
    proximal damping damp/2 |(s,u) - (s,u)^0|^2 and the box block's term
    rho_box/2 |(s,u) - z + w|^2 on bounded components (z = clip((s,u)^0), w = 0)."""
    sc = synth.config1()
    m = sc.model
    sigma = 300.0
    rng = np.random.default_rng(4)
    s0 = synth.random_states(sc, rng, 0.5, 0.1)
    s0[0] = sc.s_ref[0]
    s0[:, 3] = np.clip(s0[:, 3] + rng.normal(0, 20, len(s0)), -5, 40)   # some speeds out of the box
    u0 = rng.normal(0, 0.3, sc.u_init.shape)
    out = ora.admm_batch(sc, sigma=sigma, prox=1e-3, max_iter=1, s=s0, u=u0, damp=damp, rho_box=rho_box)
    N, ns, nu = int(sc.horizon[0]), m.ns, m.nu
    A = np.zeros((N, ns, ns))
    B = np.zeros((N, ns, nu))
    c = np.zeros((N, ns))
    for t in range(N):
        f, fs, fu = ora.dynamics(m, s0[t], u0[t])
        A[t] = np.eye(ns) + m.dt * fs
        B[t] = m.dt * fu
        c[t] = s0[t] + m.dt * f - A[t] @ s0[t] - B[t] @ u0[t]
    Q = np.repeat(np.diag(2 * m.Qs)[None], N + 1, 0)
    q = -2 * m.Qs[None, :] * sc.s_ref
    R = np.repeat(np.diag(2 * m.Qu)[None], N, 0)
    r = np.zeros((N, nu))
    sb = np.isfinite(m.s_lo) | np.isfinite(m.s_hi)
    ub = np.isfinite(m.u_lo) | np.isfinite(m.u_hi)
    for t in range(1, N + 1):
        Q[t] += np.diag(damp + rho_box * sb)
        q[t] -= damp * s0[t] + rho_box * sb * np.clip(s0[t], m.s_lo, m.s_hi)
    for t in range(N):
        R[t] += np.diag(damp + rho_box * ub)
        r[t] -= damp * u0[t] + rho_box * ub * np.clip(u0[t], m.u_lo, m.u_hi)
    for p in range(sc.n_pairs):
        j, pt, t, C, d = _pair_data(sc, p)
        r0, J = ora.pair_gn(m, sc.part_A[pt], C, d, sc.part_link[pt], sc.part_off[pt], s0[t],
                            out["y"][p], sc.fr_max, sc.fo_max, 0.0, np.zeros(2))
        Q[t] += sigma * J.T @ J
        q[t] += sigma * J.T @ (r0 - J @ s0[t])
    s_ref, u_ref = _dense_kkt(A, B, c, Q, q, R, r, s0[0])
    assert np.abs(out["s"] - s_ref).max() < 1e-7
    assert np.abs(out["u"] - u_ref).max() < 1e-7


def test_zeta_increment_identity(ora):
    """eqn:ADMM_residue_updates: zeta^{k+1} - zeta^k = T(s^{k+1}, y^{k+1}),
    xi^{k+1} - xi^k = R(s^{k+1}, y^{k+1}), and r_pri is their squared sum."""
    sc = synth.config2()
    a = ora.admm_batch(sc, prox=1e-3, max_iter=3, rho_box=0.0)
    b = ora.admm_batch(sc, prox=1e-3, max_iter=4, rho_box=0.0)
    sk, yk = b["s"], b["y"]
    dz = b["zeta"] - a["zeta"]
    dx = b["xi"] - a["xi"]
    rng = np.random.default_rng(0)
    for p in rng.choice(sc.n_pairs, 100, replace=False):
        j, pt, t, C, d = _pair_data(sc, p)
        r0, _ = ora.pair_gn(sc.model, sc.part_A[pt], C, d, sc.part_link[pt], sc.part_off[pt], sk[t],
                            yk[p], sc.fr_max, sc.fo_max, 0.0, np.zeros(2))
        assert dz[p] == pytest.approx(r0[0], abs=1e-9)
        assert np.abs(dx[p] - r0[1:]).max() < 1e-9
    assert b["r_pri"][0] == pytest.approx(float((dz ** 2).sum() + (dx ** 2).sum()), rel=1e-9)


def test_converged_fixed_point_is_collision_free(ora):
    """At a point meeting the stopping rule, every pair's certificate is
    (nearly) feasible, so alpha* of the final trajectory is >= 1 - O(sqrt(eps)),
    and the box block holds the controls within their bounds."""
    sc = synth.config1()
    out = ora.admm_batch(sc, max_iter=300)
    assert out["status"][0] == 0
    assert out["r_pri"][0] <= 1e-4 and out["r_dual"][0] <= 1e-4
    al = ora.scale_batch(sc, out["s"])["alpha"]
    assert al.min() >= 1.0 - 2e-2
    # the reference runs through an obstacle: the plan deviates from it
    al_ref = ora.scale_batch(sc, sc.s_ref)["alpha"]
    assert al_ref.min() < 0.9
    m = sc.model
    assert (out["u"] >= m.u_lo - 1e-2).all() and (out["u"] <= m.u_hi + 1e-2).all()


def test_far_obstacles_reduce_to_tracking(ora):
    """With every obstacle far away the collision terms vanish at the fixed
    point and the plan is the obstacle-free optimum: the reference itself
    (dynamically feasible with u = 0, zero tracking cost).  The certificates
    add stiffness, so the plan drifts to it slowly: a tight tolerance is used."""
    sc = synth.config1()
    sc.obs_d = sc.obs_d + sc.obs_C @ np.array([0.0, 500.0]) * (np.arange(sc.fo_max) < sc.obs_nf[:, None])
    rng = np.random.default_rng(0)
    s0 = synth.random_states(sc, rng, 0.3, 0.05)
    s0[0] = sc.s_ref[0]
    out = ora.admm_batch(sc, prox=1e-3, max_iter=1000, s=s0, eps_pri=1e-14, eps_dual=1e-14, damp=0.0)
    assert np.abs(out["s"] - sc.s_ref).max() < 1e-4
    assert out["cost"][0] < 1e-8
