"""Pins of the oracle's closed loop (Sec. V-B receding horizon): the window,
shift and sensing bookkeeping around the pinned ADMM, dynamics and LP."""
import dataclasses

import numpy as np

from paper_2406_07048_gb300 import synth


def test_no_iterations_applies_the_shifted_warm_start(ora):
    """With max_iter = 0 nothing is solved: the control applied at step c is
    row c of the initial plan (the plan moves up one row per step), clipped
    to the box, and the true state follows the Euler rollout of them."""
    sc, ref = synth.closed_loop(2, N=16)
    rng = np.random.default_rng(0)
    sc = dataclasses.replace(sc, u_init=rng.uniform(-1.0, 1.0, sc.u_init.shape))
    x0 = ref[:, 0].copy()
    C = 6
    r = ora.mpc_run(sc, ref, x0, C, max_iter=0)
    m = sc.model
    for s in range(sc.n_scen):
        b = int(sc.ctrl_begin[s])
        x = x0[s].copy()
        for c in range(C):
            u0 = np.clip(sc.u_init[b + c], m.u_lo, m.u_hi)
            assert np.array_equal(r["u_hist"][s, c], u0)
            x = x + m.dt * ora.dynamics(m, x, u0)[0]
            assert np.allclose(r["x_hist"][s, c + 1], x, rtol=0, atol=1e-12)


def test_window_covering_everything_is_one_full_solve(ora):
    sc, ref = synth.closed_loop(2, N=16)
    x0 = ref[:, 0].copy()
    r = ora.mpc_run(sc, ref, x0, 1, window=(1e9, 1e9, 1e9), max_iter=20)
    full = ora.admm_batch(sc, max_iter=20)
    assert np.array_equal(r["iters"][:, 0], full["iters"])
    assert np.allclose(r["s"], full["s"], rtol=0, atol=1e-12)
    assert np.allclose(r["y"], full["y"], rtol=0, atol=1e-12)
    assert np.allclose(r["zeta"], full["zeta"], rtol=0, atol=1e-12)


def test_empty_window_leaves_every_pair_untouched(ora):
    sc, ref = synth.closed_loop(2, N=16)
    x0 = ref[:, 0].copy()
    r = ora.mpc_run(sc, ref, x0, 3, window=(1e-9, 1e-9, 1e-9), max_iter=10)
    assert np.array_equal(r["y"], sc.cold_y())
    assert np.all(r["zeta"] == 0) and np.all(r["xi"] == 0)
    assert (r["collided"] == -1).all()


def test_closed_loop_sensing_changes_during_the_run(ora):
    """The default window really culls: some obstacles are sensed only at
    later steps (re-entry keeps their shifted warm start)."""
    sc, ref = synth.closed_loop(1, N=16)
    x0 = ref[:, 0].copy()
    r = ora.mpc_run(sc, ref, x0, 60, max_iter=1)
    pos = r["x_hist"][0, :, :3]
    inside = np.abs(sc.obs_center[None, :, :] - pos[:, None, :]) <= np.array([10.0, 10.0, 3.0])
    sensed = inside.all(axis=2)
    assert sensed[0].sum() < sensed.any(axis=0).sum()
