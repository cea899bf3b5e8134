"""Differentiation form at its stated shape: 256 tractor-trailer scenarios
(N = 50, 2 parts, 32 obstacles of 3-12 faces), batched FP32 forward with the
library's default ADMM parameters and stopping rule, then the adjoint
(oca_admm_backward) against FP64 central differences (h = 1e-6) of the
oracle's ADMM on 16 sampled scenarios among those the forward converged.

The gradient is that of the executed map: scenario s ran K_s iterations, so
the oracle runs exactly K_s iterations of the same ADMM (stopping rule off)
on the perturbed scene.  The objective of scenario s is its trajectory cost
(eqn:navigation_cost) plus, through grad_alpha, a weighted sum of alpha*
(eqn:scale_opt) of its 8 closest pairs at the returned trajectory (the LP
envelope terms of Sec. III-B).  Each scenario is checked along one random
direction of its obstacle offsets and one of its obstacle translations:
|fd - g.v| <= 1e-3 (|fd| + 1e-3 |g| |v|).  The measured errors are printed
(pytest -s).

A central difference is a reference only where the map is smooth at the
scale h: over hundreds of iterations some pair QP can change its active set
within +-h, a kink of the executed map where its derivative is not defined.
The oracle's one-sided differences expose it, (f(+h) - f(0)) - (f(0) - f(-h))
= f'' h^2 for a smooth map but ~ h |jump| at a kink; scenarios whose
asymmetry exceeds 1e-4 h (|fd| + 1) in either direction are replaced by the
next sampled converged scenario, and the number replaced is printed.
"""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2406_07048_gb300 import synth

pytestmark = pytest.mark.gpu

H = 1e-6
N_SAMPLE = 16
N_ALPHA = 8


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2406_07048_gb300 import _build, binding
    _build.build()
    return binding


def test_diffform_fp32_adjoint_matches_fp64_fd(B, ora):
    sc = synth.config5(256)
    ctx = B.Context(0)
    ds = B.DeviceScene(ctx, sc, torch.float32)
    pb = B.Problem(ds)
    kw = dict(B.DEFAULTS)
    tape = B.new_tape(ds, kw["max_iter"])
    rep = B.admm_solve(ds, pb.s_ref, pb.s, pb.u, pb.y, pb.zeta, pb.xi, tape=tape, **kw)
    iters = rep["iters"].cpu().numpy()
    status = rep["status"].cpu().numpy()
    conv = np.where(status == 0)[0]
    print(f"[diffform] {len(conv)} of {sc.n_scen} scenarios converged (iterations "
          f"{iters[conv].min()}..{iters[conv].max()})")
    assert len(conv) >= N_SAMPLE
    rng = np.random.default_rng(11)
    picks = conv   # every converged scenario carries its objective; the check samples among them
    # objective: cost of the sampled scenarios + weighted alpha* of their closest pairs
    sd = B.scale_detect(ds, pb.s, want_certificate=False, want_margin=False)
    alpha = sd["alpha"].double().cpu().numpy()
    P = sc.n_pairs
    gcost = np.zeros(sc.n_scen)
    galpha = np.zeros(P)
    alpha_pairs = {}
    for s in picks:
        gcost[s] = 1.0
        p0, p1 = int(sc.pair_begin[s]), int(sc.pair_begin[s + 1])
        loc = np.argsort(alpha[p0:p1])[:N_ALPHA]
        w = rng.uniform(0.5, 2.0, N_ALPHA) * rng.choice([-1.0, 1.0], N_ALPHA)
        galpha[p0 + loc] = w
        alpha_pairs[int(s)] = (loc, w)
    g = B.admm_backward(ds, pb.s_ref, tape, rep["iters"], torch.as_tensor(gcost, device=ds.device),
                        grad_alpha=torch.as_tensor(galpha, device=ds.device),
                        **{k: kw[k] for k in ("sigma", "prox", "max_iter", "rho_box", "damp", "eps_pri", "eps_dual")})
    g_d = g["obs_offset"].double().cpu().numpy()
    g_c = g["obs_center"].double().cpu().numpy()

    oracle_kw = {k: kw[k] for k in ("sigma", "prox", "rho_box", "damp")}
    worst, checked, skipped = 0.0, 0, 0
    order = rng.permutation(conv)
    for s in order:
        if checked == N_SAMPLE:
            break
        s = int(s)
        if s not in alpha_pairs:
            continue
        sub = synth.subset(sc, [s])
        K = int(iters[s])
        loc, w = alpha_pairs[s]
        j0, j1 = int(sc.obs_begin[s]), int(sc.obs_begin[s + 1])
        M = j1 - j0
        nf = sc.obs_nf[j0:j1]
        mask = np.arange(sc.fo_max)[None, :] < nf[:, None]
        v_d = rng.normal(size=(M, sc.fo_max)) * mask
        v_c = rng.normal(size=(M, sc.dim))
        dirs = [("offsets", v_d, float((g_d[j0:j1] * v_d).sum())),
                ("translations", np.einsum("jmi,ji->jm", sub.obs_C, v_c) * mask, float((g_c[j0:j1] * v_c).sum()))]
        # the scenario at 0, +h, -h along both directions: five copies solved side by side
        cp = synth.subset(sc, [s] * 5)
        d = cp.obs_d.copy()
        for k, (eps, dd) in enumerate([(H, dirs[0][1]), (-H, dirs[0][1]), (H, dirs[1][1]), (-H, dirs[1][1])]):
            d[(k + 1) * M:(k + 2) * M] += eps * dd
        cp = dataclasses.replace(cp, obs_d=d)
        r = ora.admm_batch(cp, max_iter=K, eps_pri=0.0, eps_dual=0.0, **oracle_kw)
        Ps = int(sub.n_pairs)
        a_o = ora.scale_batch(cp, r["s"], pairs=np.concatenate([k * Ps + loc for k in range(5)]))["alpha"]
        f = [float(r["cost"][k]) + float(w @ a_o[k * N_ALPHA:(k + 1) * N_ALPHA]) for k in range(5)]
        fds = [((f[1] - f[2]) / (2 * H), f[1] - f[0] - (f[0] - f[2])), ((f[3] - f[4]) / (2 * H), f[3] - f[0] - (f[0] - f[4]))]
        if any(abs(asym) > 1e-4 * H * (abs(fd) + 1.0) for fd, asym in fds):
            skipped += 1
            print(f"[diffform scen {s} K={K}] not smooth at h: one-sided asymmetry "
                  f"{[float(a) for _, a in fds]}, replaced")
            continue
        scale_g = np.sqrt((g_d[j0:j1] ** 2).sum() + (g_c[j0:j1] ** 2).sum())
        a, b = int(sc.state_begin[s]), int(sc.state_begin[s + 1])
        s_o = r["s"][: b - a]
        dev = np.abs(pb.s[a:b].double().cpu().numpy() - s_o).max() / (1.0 + np.abs(s_o).max())
        print(f"[diffform scen {s} K={K}] FP32 forward vs FP64 oracle after K iterations: "
              f"max state deviation {dev:.3g} (relative)")
        for (name, dd, ad), (fd, _) in zip(dirs, fds):
            err = abs(fd - ad) / (abs(fd) + 1e-3 * scale_g * np.linalg.norm(dd))
            worst = max(worst, err)
            print(f"[diffform scen {s} K={K} {name}] fd {fd:.6g} adjoint {ad:.6g} rel err {err:.3g}")
            assert err <= 1e-3, (s, name, fd, ad)
        checked += 1
    print(f"[diffform] {checked} scenarios checked, {skipped} replaced (not smooth at h); "
          f"worst relative error {worst:.3g}")
    assert checked == N_SAMPLE
