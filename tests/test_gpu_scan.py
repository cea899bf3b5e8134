"""The step-2 LQ problem (Sec. IV-B, one QP per iteration) solved on the GPU
in parallel-in-time form (oca_lq_solve, OCA_LQ_SCAN: associative composition
of the stage relations of its optimality conditions) and by the sequential
Riccati recursion (OCA_LQ_SEQUENTIAL), against the oracle's scan
(ora_riccati_scan, the same composition order) and its textbook recursion
(ora_riccati), on random problems with dense stage matrices.  FP64 on both
sides: states, controls and value functions within 1e-9 relative (floored
at 1)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from tests.test_oracle_riccati import _rand_lq

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2406_07048_gb300 import _build, binding
    _build.build()
    return binding


@pytest.fixture(scope="module")
def ctx(B):
    return B.Context(0)


def _batch(rng, S, N, ns, nu):
    probs = [_rand_lq(rng, N, ns, nu) for _ in range(S)]
    return [np.stack([pr[i] for pr in probs]) for i in range(8)], probs


def _dev(arrs):
    return [torch.as_tensor(a, dtype=torch.float64, device="cuda") for a in arrs]


def _rel(a, b):
    return np.abs(a - b).max() / max(1.0, np.abs(b).max()) if a.size else 0.0


@pytest.mark.parametrize("ns,nu,N,S", [(4, 2, 0, 2), (4, 2, 1, 1), (5, 2, 2, 3), (3, 1, 7, 2), (5, 2, 50, 3),
                                       (12, 4, 40, 2), (12, 4, 256, 1), (8, 3, 100, 4)])
@pytest.mark.parametrize("method", [0, 1])
def test_lq_solve_matches_oracle(B, ctx, ora, ns, nu, N, S, method):
    rng = np.random.default_rng(1000 * ns + N + S)
    arrs, probs = _batch(rng, S, N, ns, nu)
    A, Bm, c, Q, q, R, r, s0 = _dev(arrs)
    out = B.lq_solve(ctx, A, Bm, c, Q, q, R, r, s0, method=method)
    torch.cuda.synchronize()
    assert (out["status"].cpu().numpy() == 0).all()
    s_g, u_g = out["s"].cpu().numpy(), out["u"].cpu().numpy()
    P_g, p_g = out["P"].cpu().numpy(), out["p"].cpu().numpy()
    errs = []
    for k, pr in enumerate(probs):
        s_o, u_o, P_o, p_o, st = ora.riccati_scan(*pr, tree=True)
        assert st == 0
        s_r, u_r, st2 = ora.riccati(*pr)
        assert st2 == 0
        errs += [_rel(s_g[k], s_o), _rel(u_g[k], u_o), _rel(P_g[k], P_o), _rel(p_g[k], p_o),
                 _rel(s_g[k], s_r), _rel(u_g[k], u_r)]
    print(f"[lq {'scan' if method else 'sequential'} ns={ns} nu={nu} N={N} S={S}] max rel err {max(errs):.3g}")
    assert max(errs) <= 1e-9, errs


def test_lq_methods_agree_on_a_long_horizon(B, ctx):
    """N = 1,000: the scan's 10 rounds and the 1,000-step recursion agree."""
    rng = np.random.default_rng(7)
    arrs, _ = _batch(rng, 2, 1000, 6, 2)
    dev = _dev(arrs)
    a = B.lq_solve(ctx, *dev, method=0)
    b = B.lq_solve(ctx, *dev, method=1)
    torch.cuda.synchronize()
    for k in ("s", "u", "P", "p"):
        x, y = a[k].cpu().numpy(), b[k].cpu().numpy()
        assert _rel(y, x) <= 1e-9, k


def test_lq_status_and_argument_errors(B, ctx):
    rng = np.random.default_rng(3)
    arrs, _ = _batch(rng, 2, 6, 4, 2)
    # problem 1: R = 0 and B = 0: no input can be eliminated (singular R_t and R_t + B^T P B)
    arrs[5][1] = 0.0
    arrs[1][1] = 0.0
    dev = _dev(arrs)
    for method in (0, 1):
        out = B.lq_solve(ctx, *dev, method=method)
        torch.cuda.synchronize()
        assert out["status"].cpu().numpy().tolist() == [0, 1]
    with pytest.raises(B.OcaError) as e:
        B.lq_workspace_bytes(13, 2, 4, 1)
    assert e.value.code == 5
    with pytest.raises(B.OcaError) as e:
        B.lq_solve(ctx, *dev, method=1, work=torch.empty(64, dtype=torch.uint8, device="cuda"))
    assert e.value.code == 5
    with pytest.raises(B.OcaError) as e:
        B.lq_solve(ctx, *dev, method=7)
    assert e.value.code == 1
