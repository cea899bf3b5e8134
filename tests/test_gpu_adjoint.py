"""Adjoint of the unrolled ADMM (oca_admm_backward) against central finite
differences of the FP64 oracle's ADMM with the same fixed iteration count.

The gradient is that of the map the taped solve executed; with eps = 0 the
iteration count is max_iter on both sides, so the oracle's
(F(theta + h e) - F(theta - h e)) / 2h is the reference for every component
(theta: obstacle offsets, obstacle translations, the initial state).
"""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2406_07048_gb300 import synth

pytestmark = pytest.mark.gpu

H = 1e-6
KW = dict(sigma=300.0, eps_pri=0.0, eps_dual=0.0, prox=0.1, rho_box=100.0, damp=100.0)


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2406_07048_gb300 import binding
    return binding


@pytest.fixture(scope="module")
def ctx(B):
    return B.Context(0)


def _gpu_grads(B, ctx, sc, K, dtype):
    ds = B.DeviceScene(ctx, sc, dtype)
    pb = B.Problem(ds)
    tape = B.new_tape(ds, K)
    rep = B.admm_solve(ds, pb.s_ref, pb.s, pb.u, pb.y, pb.zeta, pb.xi, tape=tape, max_iter=K, **KW)
    gc = torch.ones(sc.n_scen, dtype=dtype, device=ds.device)
    g = B.admm_backward(ds, pb.s_ref, tape, rep["iters"], gc, max_iter=K,
                        **{k: KW[k] for k in ("sigma", "prox", "rho_box", "damp")})
    out = {k: v.double().cpu().numpy() for k, v in g.items()}
    out["cost"] = rep["cost"].double().cpu().numpy()
    out["iters"] = rep["iters"].cpu().numpy()
    return out


def _fd(ora, sc, K, perturb):
    """Central difference of the oracle's total cost along `perturb(scene, +-h)`."""
    f = lambda eps: ora.admm_batch(perturb(sc, eps), max_iter=K, **KW)["cost"].sum()
    return (f(H) - f(-H)) / (2 * H)


def _offset(j, m):
    def p(sc, eps):
        d = sc.obs_d.copy()
        d[j, m] += eps
        return dataclasses.replace(sc, obs_d=d)
    return p


def _centre(j, i):
    def p(sc, eps):
        d = sc.obs_d.copy()
        d[j] += eps * sc.obs_C[j, :, i]
        return dataclasses.replace(sc, obs_d=d)
    return p


def _state0(s0_row, i):
    def p(sc, eps):
        s = sc.s_init.copy()
        s[s0_row, i] += eps
        return dataclasses.replace(sc, s_init=s)
    return p


def _check(pairs, rtol):
    fd = np.array([a for a, _ in pairs])
    ad = np.array([b for _, b in pairs])
    scale = np.abs(fd).max()
    err = np.abs(fd - ad)
    # relative to each component, with a floor of 1e-3 of the largest
    assert np.all(err <= rtol * (np.abs(fd) + 1e-3 * scale)), (err / (np.abs(fd) + 1e-3 * scale)).max()


@pytest.mark.parametrize("K", [1, 10, 50])
def test_adjoint_fp64_matches_oracle_fd_bicycle(B, ctx, ora, K):
    """Bicycle scene (one part, four obstacles, N = 20): every offset,
    every obstacle translation and the initial state."""
    sc = synth.config1()
    g = _gpu_grads(B, ctx, sc, K, torch.float64)
    assert int(g["iters"][0]) == K
    ref = ora.admm_batch(sc, max_iter=K, **KW)["cost"]
    assert np.allclose(g["cost"], ref, rtol=1e-10)
    offs = [(j, m) for j in range(sc.obs_d.shape[0]) for m in range(int(sc.obs_nf[j]))]
    _check([(_fd(ora, sc, K, _offset(j, m)), g["obs_offset"][j, m]) for j, m in offs], 1e-4)
    _check([(_fd(ora, sc, K, _centre(j, i)), g["obs_center"][j, i])
            for j in range(sc.obs_d.shape[0]) for i in range(sc.dim)], 1e-4)
    _check([(_fd(ora, sc, K, _state0(0, i)), g["state0"][0, i]) for i in range(sc.model.ns)], 1e-5)
    # pad faces carry no gradient
    for j in range(sc.obs_d.shape[0]):
        assert np.all(g["obs_offset"][j, int(sc.obs_nf[j]):] == 0.0)


def test_adjoint_fp64_matches_oracle_fd_trailer(B, ctx, ora):
    """Tractor-trailer scene (two parts, 32 obstacles, N = 50), 20
    iterations: sampled offsets and translations, every initial-state
    component (the trailer's hinge angle included)."""
    sc = synth.config2(0)
    K = 20
    g = _gpu_grads(B, ctx, sc, K, torch.float64)
    rng = np.random.default_rng(3)
    offs = [(j, m) for j in range(sc.obs_d.shape[0]) for m in range(int(sc.obs_nf[j]))]
    pick = [offs[i] for i in rng.choice(len(offs), 24, replace=False)]
    _check([(_fd(ora, sc, K, _offset(j, m)), g["obs_offset"][j, m]) for j, m in pick], 1e-3)
    _check([(_fd(ora, sc, K, _centre(j, i)), g["obs_center"][j, i])
            for j in rng.choice(sc.obs_d.shape[0], 6, replace=False) for i in range(sc.dim)], 1e-3)
    _check([(_fd(ora, sc, K, _state0(0, i)), g["state0"][0, i]) for i in range(sc.model.ns)], 1e-5)


def test_adjoint_batched_scenarios_are_independent(B, ctx):
    """A batch's gradient equals the gradients of its scenarios solved one
    by one (no cross-talk between scenarios in the accumulators)."""
    sc = synth.config3(n_scen=4, first=5)
    K = 8
    full = _gpu_grads(B, ctx, sc, K, torch.float64)
    for s in range(sc.n_scen):
        one = _gpu_grads(B, ctx, synth.subset(sc, [s]), K, torch.float64)
        j0, j1 = int(sc.obs_begin[s]), int(sc.obs_begin[s + 1])
        assert np.allclose(one["obs_offset"], full["obs_offset"][j0:j1], rtol=1e-9, atol=1e-12)
        assert np.allclose(one["state0"][0], full["state0"][s], rtol=1e-9, atol=1e-12)


def test_taped_solve_equals_plain_solve(B, ctx):
    sc = synth.config2(1)
    out = []
    for taped in (False, True):
        ds = B.DeviceScene(ctx, sc, torch.float32)
        pb = B.Problem(ds)
        tape = B.new_tape(ds, 30) if taped else None
        rep = B.admm_solve(ds, pb.s_ref, pb.s, pb.u, pb.y, pb.zeta, pb.xi, max_iter=30, tape=tape)
        out.append((pb.s.cpu(), pb.y.cpu(), rep["iters"].cpu()))
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])
    assert torch.equal(out[0][2], out[1][2])


def test_autograd_function_matches_backward(B, ctx):
    """torch.autograd through AdmmCost gives oca_admm_backward's offset and
    translation gradients."""
    sc = synth.config1()
    K = 10
    ds = B.DeviceScene(ctx, sc, torch.float64)
    pb = B.Problem(ds)
    d = ds.obs_d.clone().requires_grad_(True)
    shift = torch.zeros(sc.obs_d.shape[0], sc.dim, dtype=torch.float64, device=ds.device, requires_grad=True)
    cost = B.admm_cost(pb, d, shift, max_iter=K, **KW)
    # another forward on the same problem (other offsets) and a plain solve of
    # its scene between this forward and its backward change nothing: each
    # forward solves on a scene of its own
    other = B.admm_cost(pb, d.detach() + 0.05, shift.detach(), max_iter=K, **KW)
    B.Problem(ds).solve(max_iter=3, **KW)
    gd, gs = torch.autograd.grad(cost.sum(), (d, shift))
    assert torch.isfinite(other).all()
    g = _gpu_grads(B, ctx, sc, K, torch.float64)
    assert np.allclose(gd.cpu().numpy(), g["obs_offset"], rtol=1e-12, atol=1e-14)
    assert np.allclose(gs.cpu().numpy(), g["obs_center"], rtol=1e-12, atol=1e-14)
    # the scene's own offsets are left as they were
    assert torch.equal(ds.obs_d, torch.as_tensor(sc.obs_d, device=ds.device))


def test_backward_argument_errors(B, ctx):
    sc = synth.config1()
    ds = B.DeviceScene(ctx, sc, torch.float64)
    pb = B.Problem(ds)
    tape = B.new_tape(ds, 4)
    rep = B.admm_solve(ds, pb.s_ref, pb.s, pb.u, pb.y, pb.zeta, pb.xi, tape=tape, max_iter=4, **KW)
    gc = torch.ones(1, dtype=torch.float64, device=ds.device)
    with pytest.raises(B.OcaError) as e:
        B.admm_backward(ds, pb.s_ref, tape, rep["iters"], gc, max_iter=4, prox=0.0)
    assert e.value.code == 4  # OCA_ERR_UNSUPPORTED: the prox = 0 QP has no unique solution
    small = tape[: tape.numel() // 2]
    with pytest.raises(B.OcaError) as e:
        B.admm_backward(ds, pb.s_ref, small, rep["iters"], gc, max_iter=4)
    assert e.value.code == 5  # OCA_ERR_CAPACITY
    with pytest.raises(B.OcaError) as e:
        B.admm_solve(ds, pb.s_ref, pb.s, pb.u, pb.y, pb.zeta, pb.xi, tape=small, max_iter=4)
    assert e.value.code == 5


def test_alpha_gradient_matches_oracle_fd(B, ctx, ora):
    """L = sum_p g_p alpha*_p at the returned trajectory (plus the cost):
    oca_admm_backward against central differences of the oracle's ADMM
    followed by its scale LP at the returned states."""
    sc = synth.config1()
    K = 10
    rng = np.random.default_rng(7)
    ga = rng.uniform(-1.0, 1.0, sc.n_pairs)
    ds = B.DeviceScene(ctx, sc, torch.float64)
    pb = B.Problem(ds)
    tape = B.new_tape(ds, K)
    rep = B.admm_solve(ds, pb.s_ref, pb.s, pb.u, pb.y, pb.zeta, pb.xi, tape=tape, max_iter=K, **KW)
    gc = torch.full((1,), 0.5, dtype=torch.float64, device=ds.device)
    g = B.admm_backward(ds, pb.s_ref, tape, rep["iters"], gc, grad_alpha=torch.as_tensor(ga, device=ds.device),
                        max_iter=K, **{k: KW[k] for k in ("sigma", "prox", "rho_box", "damp")})
    g = {k: v.cpu().numpy() for k, v in g.items()}

    def fd(perturb):
        def L(eps):
            s2 = perturb(sc, eps)
            r = ora.admm_batch(s2, max_iter=K, **KW)
            return 0.5 * r["cost"].sum() + ga @ ora.scale_batch(s2, r["s"])["alpha"]
        return (L(H) - L(-H)) / (2 * H)

    offs = [(j, m) for j in range(sc.obs_d.shape[0]) for m in range(int(sc.obs_nf[j]))]
    _check([(fd(_offset(j, m)), g["obs_offset"][j, m]) for j, m in offs], 1e-4)
    _check([(fd(_centre(j, i)), g["obs_center"][j, i]) for j in range(sc.obs_d.shape[0]) for i in range(sc.dim)],
           1e-4)
    _check([(fd(_state0(0, i)), g["state0"][0, i]) for i in range(sc.model.ns)], 1e-5)


KFP = 8000  # the bicycle scene's ADMM contracts by ~0.998 per iteration: 0.998^8000 ~ 1e-7


def _fp_grads(B, ctx, sc, K, dtype, n_rev=None):
    """Fixed-point form: a solve of K iterations taping its returned iterate,
    then n_rev (default K) reverse steps at it."""
    ds = B.DeviceScene(ctx, sc, dtype)
    pb = B.Problem(ds)
    tape = B.new_tape(ds, K, fixed_point=True)
    rep = B.admm_solve(ds, pb.s_ref, pb.s, pb.u, pb.y, pb.zeta, pb.xi, tape=tape, max_iter=K,
                       flags=B.OCA_ADMM_FIXED_POINT, **KW)
    gc = torch.ones(sc.n_scen, dtype=dtype, device=ds.device)
    g = B.admm_backward(ds, pb.s_ref, tape, rep["iters"], gc, max_iter=K if n_rev is None else n_rev,
                        flags=B.OCA_ADMM_FIXED_POINT, **{k: KW[k] for k in ("sigma", "prox", "rho_box", "damp")})
    out = {k: v.double().cpu().numpy() for k, v in g.items()}
    out["cost"] = rep["cost"].double().cpu().numpy()
    out["tape_bytes"] = tape.numel()
    return out


def test_fixed_point_adjoint_matches_oracle_fd(B, ctx, ora):
    """The implicit-function gradient of the converged solution (one taped
    iterate, 8,000 reverse steps) against central differences of the oracle's
    ADMM run 8,000 iterations from the same start, where the iteration has
    converged to rounding level and the executed map's derivative equals the
    fixed point's."""
    sc = synth.config1()
    g = _fp_grads(B, ctx, sc, KFP, torch.float64)
    ref = ora.admm_batch(sc, max_iter=KFP, **KW)
    assert np.allclose(g["cost"], ref["cost"], rtol=1e-9)
    rng = np.random.default_rng(11)
    offs = [(j, m) for j in range(sc.obs_d.shape[0]) for m in range(int(sc.obs_nf[j]))]
    pick = [offs[i] for i in rng.choice(len(offs), 3, replace=False)]
    _check([(_fd(ora, sc, KFP, _offset(j, m)), g["obs_offset"][j, m]) for j, m in pick], 1e-4)
    _check([(_fd(ora, sc, KFP, _centre(j, i)), g["obs_center"][j, i]) for j in (0, 2) for i in range(sc.dim)], 1e-4)
    _check([(_fd(ora, sc, KFP, _state0(0, i)), g["state0"][0, i]) for i in (0, 2)], 1e-4)


def test_fixed_point_adjoint_equals_long_unroll(B, ctx):
    """At convergence the Neumann series and the unrolled adjoint of the
    same 8,000 iterations agree; the fixed-point tape holds one iterate
    (its size does not depend on the iteration count)."""
    sc = synth.config1()
    fp = _fp_grads(B, ctx, sc, KFP, torch.float64)
    un = _gpu_grads(B, ctx, sc, KFP, torch.float64)
    for k in ("obs_offset", "obs_center", "state0"):
        scale = np.abs(un[k]).max()
        assert np.abs(fp[k] - un[k]).max() <= 1e-6 * scale, k
    ds = B.DeviceScene(ctx, sc, torch.float64)
    assert B.tape_bytes(ds, 10, fixed_point=True) == B.tape_bytes(ds, KFP, fixed_point=True)
    assert B.tape_bytes(ds, KFP, fixed_point=True) * 1000 < B.tape_bytes(ds, KFP)


def test_fixed_point_series_truncation(B, ctx):
    """Fewer reverse steps truncate the Neumann series: the gradient moves
    toward the full one as the step count grows."""
    sc = synth.config1()
    full = _fp_grads(B, ctx, sc, KFP, torch.float64)["obs_offset"]
    errs = [np.abs(_fp_grads(B, ctx, sc, KFP, torch.float64, n_rev=n)["obs_offset"] - full).max()
            for n in (500, 2000, 5000)]
    assert errs[0] > errs[1] > errs[2]
