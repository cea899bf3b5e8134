"""GPU parity: the CUDA path (through the C-ABI) against the FP64 oracle on the
same seeded inputs.  Tolerances: FP32 alpha* and the pair-QP objective within
1e-4 relative, identical collision verdicts where |alpha* - 1| > 1e-3; FP64
runs within 1e-9.  Where several results are correct (y* of the pair QP with
prox = 0) the unique quantities (v*, objective) are compared and the GPU's y
is checked for feasibility and optimality.

"Relative" errors here are floored at 1: |x_gpu - x_oracle| / max(1, |x_oracle|),
so for quantities below 1 in magnitude (most pair objectives, alpha* of
overlapping pairs) the bound is absolute.  The tests print the measured
errors (pytest -s)."""
import numpy as np
import pytest
import torch

from paper_2406_07048_gb300 import synth
from tests import _pins

pytestmark = pytest.mark.gpu

F32, F64 = torch.float32, torch.float64


@pytest.fixture(scope="module")
def B():
    from paper_2406_07048_gb300 import _build, binding
    _build.build()
    return binding


@pytest.fixture(scope="module")
def ctx(B):
    return B.Context(0)


def _scene(name):
    if name == "c1":
        return synth.config1()
    if name == "c2":
        return synth.config2()
    if name == "c3":
        return synth.config3(n_scen=12)
    if name == "c4":
        return synth.config4(n_scen=2, n_obs=24)
    if name == "c5":
        return synth.config5(n_scen=3)
    raise KeyError(name)


def _pose(ora, sc, states, p):
    s = int(np.searchsorted(sc.pair_begin, p, side="right") - 1)
    r = p - int(sc.pair_begin[s])
    N, NP = int(sc.horizon[s]), sc.n_parts(s)
    t, part, j = r % N + 1, (r // N) % NP, r // (N * NP)
    gp = int(sc.part_begin[s]) + part
    gm = int(sc.obs_begin[s]) + j
    rho, R, _, _ = ora.part_pose(sc.model, int(sc.part_link[gp]), sc.part_off[gp], states[int(sc.state_begin[s]) + t])
    nf, nr = int(sc.obs_nf[gm]), int(sc.part_nf[gp])
    C, d = sc.obs_C[gm, :nf], sc.obs_d[gm, :nf]
    return C @ R, d - C @ rho, sc.part_A[gp, :nr], sc.part_b[gp, :nr], nr, nf


@pytest.mark.parametrize("name,dtype", [("c1", F64), ("c1", F32), ("c2", F32), ("c3", F32), ("c4", F32),
                                        ("c4", F64)])
def test_scale_detect_parity(B, ctx, ora, name, dtype):
    sc = _scene(name)
    rng = np.random.default_rng(1)
    states = synth.random_states(sc, rng, 2.0, 0.5)
    ds = B.DeviceScene(ctx, sc, dtype)
    out = B.scale_detect(ds, ds.tensor(states))
    torch.cuda.synchronize()
    ref = ora.scale_batch(sc, states)
    a_g = out["alpha"].double().cpu().numpy()
    a_o = ref["alpha"]
    tol = 1e-9 if dtype == F64 else 1e-4
    err = np.abs(a_g - a_o) / np.maximum(1.0, np.abs(a_o))
    assert err.max() <= tol, (err.max(), int(err.argmax()), a_g[err.argmax()], a_o[err.argmax()])
    assert (out["status"].cpu().numpy() == 0).all()
    far = np.abs(a_o - 1.0) > 1e-3
    v_g = out["verdict"].cpu().numpy().astype(bool)
    assert (v_g[far] == (a_o[far] >= 1.0)).all()
    # FP64 certificate margin: a valid, tight lower bound of alpha*
    m_g = out["margin"].cpu().numpy()
    # a valid bound for the geometry as stored (FP32 rounding moves alpha* by ~1e-6 |d'|)
    assert (m_g <= a_o + (1e-9 if dtype == F64 else 1e-4) * np.maximum(1, a_o)).all()
    assert (m_g >= a_o - (1e-8 if dtype == F64 else 2e-3) * np.maximum(1, a_o)).all()
    # the returned certificate is dual feasible (checked here in FP64)
    lam = ds.to_host_pairs(out["lam"])
    mu = ds.to_host_pairs(out["mu"])
    for p in rng.choice(sc.n_pairs, min(300, sc.n_pairs), replace=False):
        Cb, db, A, b, nr, nf = _pose(ora, sc, states, p)
        l, m = lam[p, :nr], mu[p, :nf]
        ftol = 1e-9 if dtype == F64 else 2e-4
        assert l.min() >= 0 and m.min() >= 0
        assert abs(b @ l - 1) < ftol
        assert np.abs(A.T @ l + Cb.T @ m).max() < ftol * (1 + np.abs(m).sum())
        assert abs(-db @ m - a_o[p]) < (1e-8 if dtype == F64 else 1e-4) * max(1.0, a_o[p])


def _qp_inputs(sc, rng, warm):
    states = synth.random_states(sc, rng, 1.0, 0.3)
    zeta = rng.normal(0, 0.3, sc.n_pairs)
    xi = rng.normal(0, 0.3, (sc.n_pairs, sc.dim))
    y = sc.cold_y()
    if warm:
        # a random feasible point as warm start / proximal centre
        y = np.abs(rng.normal(0, 0.2, y.shape)) * (rng.uniform(size=y.shape) < 0.4)
        nrs = np.zeros(sc.n_pairs, int)
        nfs = np.zeros(sc.n_pairs, int)
        bvec = np.zeros((sc.n_pairs, sc.fr_max))
        for s in range(sc.n_scen):
            N, NP = int(sc.horizon[s]), sc.n_parts(s)
            for j in range(sc.n_obs(s)):
                for pt in range(NP):
                    gp, gm = int(sc.part_begin[s]) + pt, int(sc.obs_begin[s]) + j
                    p0 = sc.pair_index(s, j, pt, 1)
                    nrs[p0:p0 + N] = sc.part_nf[gp]
                    nfs[p0:p0 + N] = sc.obs_nf[gm]
                    bvec[p0:p0 + N] = sc.part_b[gp]
        for p in range(sc.n_pairs):
            y[p, nrs[p]:sc.fr_max] = 0
            y[p, sc.fr_max + nfs[p]:sc.fr_max + sc.fo_max] = 0
            lam = y[p, :nrs[p]]
            if lam.sum() == 0:
                lam[0] = 1.0
            y[p, :nrs[p]] = lam / (bvec[p, :nrs[p]] @ lam)
    return states, zeta, xi, y


@pytest.mark.parametrize("name,dtype,warm", [("c1", F64, False), ("c1", F32, True), ("c2", F32, False),
                                             ("c2", F32, True), ("c3", F32, True), ("c4", F32, False),
                                             ("c4", F64, True)])
def test_pair_qp_prox0_parity(B, ctx, ora, name, dtype, warm):
    """prox = 0: unique v* and objective agree; the GPU's y is feasible and optimal."""
    sc = _scene(name)
    rng = np.random.default_rng(2)
    states, zeta, xi, y = _qp_inputs(sc, rng, warm)
    ds = B.DeviceScene(ctx, sc, dtype)
    out = B.pair_qp(ds, ds.tensor(states), ds.tensor(zeta), ds.to_device_pairs(xi), ds.to_device_pairs(y), prox=0.0)
    torch.cuda.synchronize()
    ref = ora.pair_qp_batch(sc, states, zeta, xi, y, prox=0.0)
    o_g = out["obj"].double().cpu().numpy()
    o_o = ref["obj"]
    st = out["status"].cpu().numpy()
    tol = 1e-9 if dtype == F64 else 1e-4
    err = np.abs(o_g - o_o) / np.maximum(1.0, o_o)
    assert err.max() <= tol, (err.max(), int(err.argmax()), o_g[err.argmax()], o_o[err.argmax()], st[err.argmax()])
    v_g = ds.to_host_pairs(out["v"])
    verr = np.abs(v_g - ref["v"]).max(axis=1) / np.maximum(1.0, np.abs(ref["v"]).max(axis=1))
    print(f"[prox0 {name} {dtype} warm={warm}] obj rel err max {err.max():.3g}, v rel err max {verr.max():.3g} "
          f"median {np.median(verr):.3g}")
    # prox = 0 is the paper's QP as printed: v* is unique but, where nearly
    # parallel generators of distant obstacles meet, FP32 rounding moves it by
    # up to ~4e-3 (measured) while the objective stays within 1e-4
    assert verr.max() <= (1e-7 if dtype == F64 else 5e-3), (verr.max(), int(verr.argmax()))
    assert (st != 3).all() and (st == 0).mean() > 0.99
    yg = ds.to_host_pairs(out["y"])
    for p in rng.choice(sc.n_pairs, min(300, sc.n_pairs), replace=False):
        Cb, db, A, b, nr, nf = _pose(ora, sc, states, p)
        K, kappa = _pins.build_K(A, b, Cb, db)
        yy = np.concatenate([yg[p, :nr], yg[p, sc.fr_max:sc.fr_max + nf], [yg[p, -1]]])
        bq = np.concatenate([[1 + zeta[p]], xi[p]])
        assert np.abs(K.T @ yy + bq - v_g[p]).max() < (1e-9 if dtype == F64 else 1e-4) * (1 + np.abs(yy).sum())
        kk = _pins.qp_kkt_residual(K, kappa, bq, yy)
        assert kk < (1e-8 if dtype == F64 else 2e-3) * (1 + np.abs(yy).sum() * (1 + np.abs(db).max())), (p, kk)


@pytest.mark.parametrize("name,dtype,prox", [("c1", F64, 0.1), ("c1", F32, 0.1), ("c2", F32, 1e-2),
                                             ("c2", F32, 0.1), ("c3", F32, 0.1), ("c3", F32, 1e-2),
                                             ("c1", F64, 1.0), ("c3", F32, 1.0), ("c4", F32, 1.0),
                                             ("c4", F32, 0.1), ("c4", F64, 0.1)])
def test_pair_qp_prox_parity(B, ctx, ora, name, dtype, prox):
    """prox > 0: the solution is unique; y, v and objective agree.  Pairs the
    semismooth Newton solver reports as iteration-capped (a zig-zag at a
    degenerate kink, <= 0.1%) are counted and left out of the comparison."""
    sc = _scene(name)
    rng = np.random.default_rng(3)
    states, zeta, xi, y = _qp_inputs(sc, rng, True)
    ds = B.DeviceScene(ctx, sc, dtype)
    out = B.pair_qp(ds, ds.tensor(states), ds.tensor(zeta), ds.to_device_pairs(xi), ds.to_device_pairs(y), prox=prox)
    torch.cuda.synchronize()
    ref = ora.pair_qp_batch(sc, states, zeta, xi, y, prox=prox)
    assert (ref["status"] == 0).all()
    st = out["status"].cpu().numpy()
    assert (st == 3).sum() == 0 and (st != 0).mean() <= 1e-3, np.bincount(st)
    ok = st == 0
    o_g = out["obj"].double().cpu().numpy()
    err = np.abs(o_g - ref["obj"]) / np.maximum(1.0, ref["obj"])
    assert err[ok].max() <= (1e-9 if dtype == F64 else 1e-4), (err[ok].max(), int(np.argmax(err * ok)))
    yg = ds.to_host_pairs(out["y"])
    yerr = np.abs(yg - ref["y"]).max(axis=1) / np.maximum(1.0, np.abs(ref["y"]).max(axis=1))
    print(f"[prox {name} {dtype} {prox}] obj rel err max {err[ok].max():.3g}, y rel err max {yerr[ok].max():.3g} "
          f"median {np.median(yerr[ok]):.3g}, capped {(~ok).sum()}")
    # measured FP32 maxima 1e-6 .. 3e-5 on these scenes
    assert yerr[ok].max() <= (1e-7 if dtype == F64 else 2e-4), (yerr[ok].max(), int(np.argmax(yerr * ok)))


def test_pair_qp_in_place(B, ctx, ora):
    """y_out may alias y_in."""
    sc = _scene("c2")
    rng = np.random.default_rng(4)
    states, zeta, xi, y = _qp_inputs(sc, rng, True)
    ds = B.DeviceScene(ctx, sc, F32)
    yin = ds.to_device_pairs(y)
    a = B.pair_qp(ds, ds.tensor(states), ds.tensor(zeta), ds.to_device_pairs(xi), yin.clone(), prox=0.0)
    b = B.pair_qp(ds, ds.tensor(states), ds.tensor(zeta), ds.to_device_pairs(xi), yin, prox=0.0, y_out=yin)
    torch.cuda.synchronize()
    assert torch.equal(a["y"], yin) and torch.equal(a["obj"], b["obj"])


def _admm_both(B, ctx, ora, sc, dtype, **kw):
    ds = B.DeviceScene(ctx, sc, dtype)
    pb = B.Problem(ds)
    rep = pb.solve(**kw)
    torch.cuda.synchronize()
    ref = ora.admm_batch(sc, **kw)
    return ds, pb, rep, ref


def test_admm_plain_fp64_matches_oracle(B, ctx, ora):
    """Plain method, FP64 on the GPU: the whole ADMM solve agrees with the
    oracle iterate for iterate (same iteration count, same trajectory)."""
    sc = _scene("c1")
    ds, pb, rep, ref = _admm_both(B, ctx, ora, sc, F64, max_iter=300)
    assert int(rep["status"][0]) == 0 and ref["status"][0] == 0
    assert int(rep["iters"][0]) == ref["iters"][0]
    assert np.abs(pb.s.cpu().numpy() - ref["s"]).max() < 1e-7
    assert np.abs(pb.u.cpu().numpy() - ref["u"]).max() < 1e-7
    assert np.abs(pb.zeta.cpu().numpy() - ref["zeta"]).max() < 1e-6
    # y along directions that barely move the residual is fixed only by the
    # small proximal weight: its sensitivity accumulates over the iterations
    assert np.abs(ds.to_host_pairs(pb.y) - ref["y"]).max() < 1e-4
    assert float(rep["cost"][0]) == pytest.approx(ref["cost"][0], rel=1e-8)
    assert float(rep["r_pri"][0]) == pytest.approx(ref["r_pri"][0], rel=1e-5, abs=1e-12)


@pytest.mark.parametrize("kw", [dict(), dict(prox=0.05, damp=0.0, rho_box=0.0), dict(rho_box=10.0, damp=3.0)])
def test_admm_fixed_iterations_fp64(B, ctx, ora, kw):
    """Fixed iteration budget (no stop): every state array agrees."""
    sc = _scene("c1")
    ds, pb, rep, ref = _admm_both(B, ctx, ora, sc, F64, max_iter=7, eps_pri=0.0, eps_dual=0.0, **kw)
    assert int(rep["status"][0]) == 1 and int(rep["iters"][0]) == 7 and ref["iters"][0] == 7
    assert np.abs(pb.s.cpu().numpy() - ref["s"]).max() < 1e-8
    assert np.abs(pb.xi.cpu().numpy().T - ref["xi"]).max() < 1e-8


@pytest.mark.parametrize("name", ["c2", "c4"])
def test_admm_fixed_iterations_fp64_models(B, ctx, ora, name):
    """Trailer (two parts, hinge state) and quadrotor (3-D, three boxes):
    10 iterations without the stopping test agree iterate for iterate."""
    sc = _scene(name)
    ds, pb, rep, ref = _admm_both(B, ctx, ora, sc, F64, max_iter=10, eps_pri=0.0, eps_dual=0.0)
    assert (rep["iters"].cpu().numpy() == 10).all() and (ref["iters"] == 10).all()
    assert np.abs(pb.s.cpu().numpy() - ref["s"]).max() < 1e-7 * (1 + np.abs(ref["s"]).max())
    assert np.abs(pb.u.cpu().numpy() - ref["u"]).max() < 1e-7 * (1 + np.abs(ref["u"]).max())
    assert np.abs(pb.zeta.cpu().numpy() - ref["zeta"]).max() < 1e-7 * (1 + np.abs(ref["zeta"]).max())


@pytest.mark.parametrize("name", ["c2", "c3", "c5"])
def test_admm_fp32_matches_oracle(B, ctx, ora, name):
    """Precision/batching forms, FP32 pair QPs with an FP64 Riccati: every
    scenario the oracle solves converges on the GPU to residuals <= 1e-4 with
    the same trajectory (to FP32 accuracy) and identical collision verdicts."""
    sc = _scene(name)
    ds, pb, rep, ref = _admm_both(B, ctx, ora, sc, F32, max_iter=300)
    st = rep["status"].cpu().numpy()
    its = rep["iters"].cpu().numpy()
    for s in range(sc.n_scen):
        if ref["status"][s] != 0:
            continue
        assert st[s] == 0, (s, st[s], its[s], ref["iters"][s])
        assert float(rep["r_pri"][s]) <= 1e-4 and float(rep["r_dual"][s]) <= 1e-4
        assert abs(int(its[s]) - int(ref["iters"][s])) <= max(3, 0.1 * ref["iters"][s])
        a, b = int(sc.state_begin[s]), int(sc.state_begin[s + 1])
        ds_ = np.abs(pb.s.cpu().numpy()[a:b] - ref["s"][a:b]).max()
        print(f"[admm fp32 {name} scen {s}] iters gpu {int(its[s])} oracle {int(ref['iters'][s])}, "
              f"max |s_gpu - s_oracle| {ds_:.3g}, cost rel {abs(float(rep['cost'][s]) / ref['cost'][s] - 1):.3g}")
        # measured: trajectories within 2.4e-5, costs within 6e-6 relative
        assert ds_ < 1e-3, (s, ds_)
        assert float(rep["cost"][s]) == pytest.approx(ref["cost"][s], rel=1e-4)
    # collision verdicts of the final plans (GPU scale detection on the GPU plan,
    # oracle LP on the oracle plan)
    sd = B.scale_detect(ds, pb.s)
    a_g = sd["alpha"].double().cpu().numpy()
    a_o = ora.scale_batch(sc, ref["s"])["alpha"]
    ok = np.repeat(ref["status"] == 0, sc.pair_counts)
    sep = ok & (np.abs(a_o - 1) > 1e-3) & (np.abs(a_g - 1) > 1e-3)
    assert ((a_g[sep] >= 1) == (a_o[sep] >= 1)).all()


def test_edge_cases(B, ctx, ora):
    """Horizon 1, a triangle obstacle, an obstacle containing the part's
    centre (alpha* = 0), 3 faces with padding to fo_max, a single scenario."""
    sc = synth.config1()
    sc.horizon[:] = 1
    sc.s_ref = sc.s_ref[:2].copy()
    sc.s_init = sc.s_ref.copy()
    sc.u_init = sc.u_init[:1].copy()
    # obstacle 0 becomes a triangle around the robot's start position
    ang = np.array([0.3, 2.4, 4.3])
    C = np.stack([np.cos(ang), np.sin(ang)], 1)
    sc.obs_C[0] = 0
    sc.obs_C[0, :3] = C
    sc.obs_d[0] = 1
    sc.obs_d[0, :3] = 1.0 + C @ np.array([sc.s_ref[1, 0] + 1.25, sc.s_ref[1, 1]])
    sc.obs_nf[0] = 3
    states = sc.s_ref.copy()
    for dtype in (F64, F32):
        ds = B.DeviceScene(ctx, sc, dtype)
        out = B.scale_detect(ds, ds.tensor(states))
        ref = ora.scale_batch(sc, states)
        a = out["alpha"].double().cpu().numpy()
        assert np.abs(a - ref["alpha"]).max() < 1e-5
        assert ref["alpha"][0] == pytest.approx(0.0, abs=1e-12) and abs(a[0]) < 1e-6
        q = B.pair_qp(ds, ds.tensor(states), ds.tensor(np.zeros(sc.n_pairs)), ds.tensor(np.zeros((2, sc.n_pairs))),
                      ds.to_device_pairs(sc.cold_y()))
        rq = ora.pair_qp_batch(sc, states, np.zeros(sc.n_pairs), np.zeros((sc.n_pairs, 2)), sc.cold_y())
        assert np.abs(q["obj"].double().cpu().numpy() - rq["obj"]).max() < 1e-5
        pb = B.Problem(ds)
        rep = pb.solve(max_iter=50)
        rr = ora.admm_batch(sc, max_iter=50)
        it_g, it_o = int(rep["iters"][0]), int(rr["iters"][0])
        print(f"[edge {dtype}] iters gpu {it_g} oracle {it_o}")
        if dtype == F64:
            assert it_g == it_o
        else:
            # FP32 pair QPs: the stopping test may trigger a few iterations apart
            assert abs(it_g - it_o) <= max(3, it_o // 10), (it_g, it_o)


def _padding_mask(sc):
    """[P, ny_max] True where a component lies beyond the pair's own face counts."""
    pad = np.ones((sc.n_pairs, sc.ny_max), dtype=bool)
    for s in range(sc.n_scen):
        n = int(sc.horizon[s])
        for j in range(sc.n_obs(s)):
            no = int(sc.obs_nf[int(sc.obs_begin[s]) + j])
            for pt in range(sc.n_parts(s)):
                nr = int(sc.part_nf[int(sc.part_begin[s]) + pt])
                p0 = sc.pair_index(s, j, pt, 1)
                pad[p0:p0 + n, :nr] = False
                pad[p0:p0 + n, sc.fr_max:sc.fr_max + no] = False
                pad[p0:p0 + n, sc.fr_max + sc.fo_max] = False
    return pad


@pytest.mark.parametrize("iters", [3, 4])
def test_admm_y_padding_untouched(B, ctx, iters):
    """Components of y beyond a pair's face counts are neither read nor
    written (odd budgets end in the second y buffer and go through the
    final gather)."""
    sc = _scene("c3")
    pad = _padding_mask(sc)
    assert pad.any()
    y0 = sc.cold_y()
    y0[pad] = 7.0
    ds = B.DeviceScene(ctx, sc, F64)
    pb = B.Problem(ds, y_init=y0)
    pb.solve(max_iter=iters, eps_pri=0.0, eps_dual=0.0)
    y = ds.to_host_pairs(pb.y)
    assert (y[pad] == 7.0).all()
    ref = B.Problem(ds)
    ref.solve(max_iter=iters, eps_pri=0.0, eps_dual=0.0)
    assert np.array_equal(y[~pad], ds.to_host_pairs(ref.y)[~pad])
    ds.close()


def test_maximum_sizes(B, ctx, ora):
    """The compiled-in maxima (24 obstacle faces, 8 part faces, horizon 256)
    next to a horizon-3 scenario: scale LPs, pair QPs (prox 1: y unique;
    prox 0: objective) and five FP64 ADMM iterations against the oracle."""
    sc = synth.config_max()
    assert sc.fo_max == 24 and sc.fr_max == 8 and int(sc.horizon.max()) == 256
    rng = np.random.default_rng(5)
    states = synth.random_states(sc, rng, 2.0, 0.5)
    for dtype in (F64, F32):
        ds = B.DeviceScene(ctx, sc, dtype)
        out = B.scale_detect(ds, ds.tensor(states))
        ref = ora.scale_batch(sc, states)
        a_g = out["alpha"].double().cpu().numpy()
        err = np.abs(a_g - ref["alpha"]) / np.maximum(1.0, np.abs(ref["alpha"]))
        assert err.max() <= (1e-9 if dtype == F64 else 1e-4), err.max()
        far = np.abs(ref["alpha"] - 1.0) > 1e-3
        assert (out["verdict"].cpu().numpy().astype(bool)[far] == (ref["alpha"][far] >= 1.0)).all()
        st, zeta, xi, y = _qp_inputs(sc, rng, True)
        for prox in (1.0, 0.0):
            q = B.pair_qp(ds, ds.tensor(st), ds.tensor(zeta), ds.to_device_pairs(xi), ds.to_device_pairs(y),
                          prox=prox)
            rq = ora.pair_qp_batch(sc, st, zeta, xi, y, prox=prox)
            ok = (q["status"].cpu().numpy() == 0) & (rq["status"] == 0)
            assert ok.mean() >= 0.999
            o_g = q["obj"].double().cpu().numpy()
            e = np.abs(o_g - rq["obj"]) / np.maximum(1.0, rq["obj"])
            assert e[ok].max() <= (1e-9 if dtype == F64 else 1e-4), (prox, e[ok].max())
            if prox > 0:
                yg = ds.to_host_pairs(q["y"])
                ye = np.abs(yg - rq["y"]).max(axis=1) / np.maximum(1.0, np.abs(rq["y"]).max(axis=1))
                assert ye[ok].max() <= (1e-7 if dtype == F64 else 5e-3), ye[ok].max()
        ds.close()
    ds, pb, rep, ref = _admm_both(B, ctx, ora, sc, F64, max_iter=5, eps_pri=0.0, eps_dual=0.0)
    assert (rep["iters"].cpu().numpy() == 5).all() and (ref["iters"] == 5).all()
    assert np.abs(pb.s.cpu().numpy() - ref["s"]).max() < 1e-7 * (1 + np.abs(ref["s"]).max())
    assert np.abs(pb.zeta.cpu().numpy() - ref["zeta"]).max() < 1e-7 * (1 + np.abs(ref["zeta"]).max())


def test_scene_validation_errors(B, ctx):
    """oca_scene_create refuses what the header rules out, with its codes:
    OCA_ERR_INVALID_ARGUMENT (1) for an empty batch, a scenario without
    obstacles, a zero horizon, face counts outside 1..fo_max or below dim+1
    for a part, a bad link; OCA_ERR_CAPACITY (5) beyond the compiled-in
    maxima (horizon 256, 24 obstacle faces)."""
    import ctypes as C
    import dataclasses
    base = synth.config1()

    def code_of(sc):
        with pytest.raises(B.OcaError) as e:
            B.DeviceScene(ctx, sc, F64)
        return e.value.code

    def with_(field, idx, value):
        arr = getattr(base, field).copy()
        arr[idx] = value
        return dataclasses.replace(base, **{field: arr})

    assert code_of(with_("horizon", 0, 0)) == 1
    assert code_of(with_("horizon", 0, 257)) == 5
    assert code_of(with_("obs_nf", 0, 0)) == 1
    assert code_of(with_("obs_nf", 0, base.fo_max + 1)) == 1
    assert code_of(with_("part_nf", 0, 2)) == 1
    assert code_of(with_("part_link", 0, 2)) == 1
    assert code_of(with_("obs_begin", 1, 0)) == 1  # a scenario with no obstacle
    wide = dataclasses.replace(base, obs_C=np.pad(base.obs_C, ((0, 0), (0, 25 - base.fo_max), (0, 0))),
                               obs_d=np.pad(base.obs_d, ((0, 0), (0, 25 - base.fo_max)), constant_values=1.0))
    assert code_of(wide) == 5
    # an empty batch, through the raw descriptor of a valid scene
    ds = B.DeviceScene(ctx, base, F64)
    d = B.SceneDesc.from_buffer_copy(ds.desc)
    d.n_scen = 0
    h = C.c_void_p()
    assert B.lib().oca_scene_create(ctx.h, C.byref(d), C.byref(h)) == 1
    ds.close()


def _as_stored(sc, dtype):
    """The scene with its geometry rounded to the device precision, so that
    the oracle sees the numbers the GPU holds."""
    import dataclasses
    if dtype == F64:
        return sc
    r = lambda a: np.asarray(a, np.float32).astype(np.float64)
    return dataclasses.replace(sc, obs_C=r(sc.obs_C), obs_d=r(sc.obs_d), part_A=r(sc.part_A), part_b=r(sc.part_b),
                               part_off=r(sc.part_off))


def _oracle_margins(ora, sc, states, lam, mu, pairs):
    out = np.empty(len(pairs))
    for i, p in enumerate(pairs):
        Cb, db, A, b, nr, nf = _pose(ora, sc, states, int(p))
        out[i] = ora.cert_margin(A, b, Cb, db, lam[p, :nr], mu[p, :nf])
    return out


@pytest.mark.parametrize("name,dtype", [("c1", F64), ("c2", F32), ("c3", F32), ("c4", F32), ("c4", F64)])
def test_cert_margin_of_given_duals(B, ctx, ora, name, dtype):
    """oca_cert_margin_batch (Sec. III-B weak duality) on certificates that
    are NOT optimal, so that r = A^T lambda + C'^T mu != 0 and the part radius
    matters: random nonnegative (lambda, mu), and the LP's optimal certificate
    perturbed.  Element-wise against the oracle's FP64 margin on the same
    stored inputs (relative 1e-12, floored at 1), and a valid lower bound of
    the oracle's alpha* for every pair."""
    sc = _as_stored(_scene(name), dtype)
    rng = np.random.default_rng(17)
    states = synth.random_states(sc, rng, 2.0, 0.5)
    if dtype == F32:
        states = states.astype(np.float32).astype(np.float64)
    ds = B.DeviceScene(ctx, sc, dtype)
    st_d = ds.tensor(states)
    ref = ora.scale_batch(sc, states)
    P = sc.n_pairs
    lam_r = rng.exponential(1.0, (P, sc.fr_max)) * (rng.uniform(size=(P, sc.fr_max)) < 0.6)
    mu_r = rng.exponential(1.0, (P, sc.fo_max)) * (rng.uniform(size=(P, sc.fo_max)) < 0.5)
    lam_p = ref["lam"] + 1e-3 * rng.uniform(size=ref["lam"].shape)
    mu_p = ref["mu"] + 1e-3 * rng.uniform(size=ref["mu"].shape)
    for lam, mu in ((lam_r, mu_r), (lam_p, mu_p)):
        if dtype == F32:
            lam, mu = lam.astype(np.float32).astype(np.float64), mu.astype(np.float32).astype(np.float64)
        m_g = B.cert_margin(ds, st_d, ds.to_device_pairs(lam), ds.to_device_pairs(mu)).cpu().numpy()
        torch.cuda.synchronize()
        sample = rng.choice(P, min(400, P), replace=False)
        m_o = _oracle_margins(ora, sc, states, lam, mu, sample)
        g = m_g[sample]
        none = ~np.isfinite(m_o)                 # no bound (denominator 0): the GPU says -DBL_MAX
        assert (g[none] < -1e300).all()
        err = np.abs(g[~none] - m_o[~none]) / np.maximum(1.0, np.abs(m_o[~none]))
        assert err.max() <= 1e-12, (err.max(), sample[~none][err.argmax()])
        ok = m_g > -1e300
        assert (m_g[ok] <= ref["alpha"][ok] + 1e-9 * np.maximum(1.0, ref["alpha"][ok])).all()


def test_cert_margin_of_admm_duals(B, ctx, ora):
    """The final check of an ADMM solve: the margin of its returned y at the
    returned trajectory equals the oracle's on the same (FP64) numbers and
    never exceeds the oracle's alpha* there."""
    sc = synth.config2()
    ds = B.DeviceScene(ctx, sc, F64)
    pb = B.Problem(ds)
    pb.solve(max_iter=40)
    torch.cuda.synchronize()
    FR, FO = sc.fr_max, sc.fo_max
    m_g = B.cert_margin(ds, pb.s, pb.y[:FR], pb.y[FR:FR + FO]).cpu().numpy()
    y = ds.to_host_pairs(pb.y)
    s = pb.s.double().cpu().numpy()
    rng = np.random.default_rng(3)
    sample = rng.choice(sc.n_pairs, 500, replace=False)
    m_o = _oracle_margins(ora, sc, s, y[:, :FR], y[:, FR:FR + FO], sample)
    err = np.abs(m_g[sample] - m_o) / np.maximum(1.0, np.abs(m_o))
    assert err.max() <= 1e-12
    al = ora.scale_batch(sc, s)["alpha"]
    assert (m_g <= al + 1e-9 * np.maximum(1.0, al)).all()
    # the ADMM's multipliers are not the LP's optimum: r != 0 for most pairs
    assert np.mean(m_g < al - 1e-6) > 0.5
