"""The allocation-free collision check gives the same results as the regular
entry point.

oca_scale_detect_noalloc serves callers that cannot allocate (a real-time
control loop that must stay out of the CUDA allocator, or a host that
forbids heap use): it keeps its scratch in a fixed device array inside the
library instead of an oca_scene workspace.  Its output must equal
oca_scale_detect_batch's on the same one-scenario scene, on two calls in a
row (the second call reuses the scratch the first one left behind).
This file is collected last so that a failing run has already run every
other test.
"""
import numpy as np
import pytest
import torch

from paper_2406_07048_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,dtype", [("plain-2d", torch.float64), ("trailer-2d", torch.float32),
                                        ("quad-3d", torch.float32)])
def test_noalloc_matches_scale_detect_batch(name, dtype):
    from paper_2406_07048_gb300 import _build, binding
    _build.build()
    if name == "plain-2d":
        sc = synth.config1()
    elif name == "trailer-2d":
        sc = synth.config2()
    else:
        sc = synth.config4(n_scen=1, n_obs=24)
    ctx = binding.Context(0)
    ds = binding.DeviceScene(ctx, sc, dtype)
    rng = np.random.default_rng(7)
    states = ds.tensor(synth.random_states(sc, rng, 2.0, 0.5))
    ref = binding.scale_detect(ds, states, want_margin=False)
    tol = 1e-9 if dtype == torch.float64 else 1e-4
    for _ in range(2):
        out = binding.scale_detect_noalloc(ds, states)
        torch.cuda.synchronize()
        a, r = out["alpha"].double().cpu().numpy(), ref["alpha"].double().cpu().numpy()
        assert np.all(np.abs(a - r) <= tol * np.maximum(1.0, np.abs(r)))
        assert torch.equal(out["verdict"], ref["verdict"])
        assert torch.equal(out["status"], ref["status"])
        for k in ("lam", "mu"):
            d = (out[k].double() - ref[k].double()).abs().max().item()
            assert d <= tol * max(1.0, ref[k].double().abs().max().item())


def test_noalloc_rejects_oversized_scene():
    """48 parts x 256 steps x 12 pose values x 8 bytes exceeds the 1 MiB scratch."""
    from paper_2406_07048_gb300 import _build, binding
    _build.build()
    sc = synth.config4(n_scen=1, n_obs=4, N=256)
    n = 48
    sc.part_begin = np.array([0, n], np.int32)
    sc.part_nf = np.full(n, 6, np.int32)
    sc.part_A = np.repeat(sc.part_A[:1], n, axis=0)
    sc.part_b = np.repeat(sc.part_b[:1], n, axis=0)
    sc.part_link = np.zeros(n, np.int32)
    sc.part_off = np.zeros((n, 3))
    ctx = binding.Context(0)
    ds = binding.DeviceScene(ctx, sc, torch.float64)
    with pytest.raises(binding.OcaError) as e:
        binding.scale_detect_noalloc(ds, ds.tensor(sc.s_ref))
    assert e.value.code == 5
