"""Closed loop (oca_mpc_run) against the oracle's closed loop."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2406_07048_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2406_07048_gb300 import binding
    return binding


@pytest.fixture(scope="module")
def ctx(B):
    return B.Context(0)


@pytest.mark.parametrize("window", [(10.0, 10.0, 3.0), (4.0, 4.0, 0.0)])
def test_closed_loop_fp64_matches_oracle(B, ctx, ora, window):
    """FP64: every control step agrees with the oracle (true states, applied
    controls, iteration counts, collision steps, final pair arrays); the
    sensing window changes which obstacles take part as the vehicle moves."""
    sc, ref = synth.closed_loop(3, N=16)
    x0 = ref[:, 0].copy()
    C = 10
    kw = dict(max_iter=40)
    ds = B.DeviceScene(ctx, sc, torch.float64)
    g = B.mpc_run(ds, ref, sc.obs_center, x0, C, window=window, **kw)
    r = ora.mpc_run(sc, ref, x0, C, window=window, **kw)
    assert np.array_equal(g["iters"].cpu().numpy(), r["iters"])
    assert np.array_equal(g["collided"].cpu().numpy(), r["collided"])
    assert np.abs(g["x_hist"].cpu().numpy() - r["x_hist"]).max() < 1e-9
    assert np.abs(g["u_hist"].cpu().numpy() - r["u_hist"]).max() < 1e-8
    assert np.abs(g["s"].cpu().numpy() - r["s"]).max() < 1e-8
    assert np.abs(g["zeta"].cpu().numpy() - r["zeta"]).max() < 1e-6
    assert np.abs(ds.to_host_pairs(g["y"]) - r["y"]).max() < 1e-4


def test_closed_loop_fp32_batch(B, ctx):
    """FP32, 64 scenarios, 40 control steps: finite histories, every solve
    within its iteration cap, and the vehicles advance along the reference
    (the damped, warm-started controller lags it by a few metres)."""
    sc, ref = synth.closed_loop(64, N=16)
    x0 = ref[:, 0].copy()
    ds = B.DeviceScene(ctx, sc, torch.float32)
    g = B.mpc_run(ds, ref, sc.obs_center, x0, 40, max_iter=50)
    xh = g["x_hist"].double().cpu().numpy()
    assert np.isfinite(xh).all()
    assert (g["iters"].cpu().numpy() <= 50).all()
    progress = (xh[:, -1, 1] - xh[:, 0, 1]) / (ref[:, 40, 1] - ref[:, 0, 1])
    assert np.median(progress) > 0.5
