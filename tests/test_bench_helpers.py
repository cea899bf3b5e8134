"""Host-side arithmetic of bench.py's roofline figures, checked against a
direct enumeration of what they count."""
import numpy as np

import bench
from paper_2406_07048_gb300 import synth


def _ric_fmas_enumerated(ns, nu):
    """FMAs of one stage, counted loop by loop as the trajectory kernel runs
    them: Y = P [A|B|c] (+ p on the last column), the upper triangle and the
    gradient column of the stage matrix, [K|k], the upper triangle of P and p,
    then the sweep's u = K s + k and s' = A s + B u + c."""
    nx, nz = ns + nu + 1, ns + nu
    n = 0
    for k in range(ns):
        for j in range(nx):
            n += ns                      # Y[k][j] = sum_l P[k][l] G[l][j]
    for i in range(nz):
        for j in range(i, nz + 1):       # upper triangle and the gradient column
            if j == nz and i > nz:
                continue
            n += ns
    for a in range(nu):
        for j in range(ns + 1):
            n += nu                      # [K|k] = -Quu^-1 [Qus|qu]
    for i in range(ns):
        for j in range(i, ns):
            n += nu                      # P upper triangle
        n += nu                          # p
    n += nu * ns                         # u = K s + k
    n += ns * (ns + nu)                  # s' = A s + B u + c
    return n


def test_ric_flops_per_stage_matches_enumeration():
    for ns, nu in ((4, 2), (5, 2), (12, 4)):
        assert bench.ric_flops_per_stage(ns, nu) == 2 * _ric_fmas_enumerated(ns, nu)
    assert bench.ric_flops_per_stage(5, 2) == 968


def test_pair_bytes_is_the_per_pair_definition():
    """4 [2 (d+1) + 2 n_y] bytes per pair, n_y = faces of the part + faces of
    the obstacle + 1, summed over a scenario's pairs."""
    sc = synth.config3(n_scen=3)
    got = bench.pair_bytes(sc)
    for s in range(sc.n_scen):
        want = 0
        for j in range(sc.n_obs(s)):
            no = int(sc.obs_nf[int(sc.obs_begin[s]) + j])
            for pt in range(sc.n_parts(s)):
                nr = int(sc.part_nf[int(sc.part_begin[s]) + pt])
                want += int(sc.horizon[s]) * 4 * (2 * (sc.dim + 1) + 2 * (nr + no + 1))
        assert got[s] == want


def test_reference_arm_prints_the_contract_line():
    """bench.py --impl reference (the oracle on the host cores) prints one JSON
    line with the keys the benchmark contract names, on a tiny sample."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--scen", "4", "--max-iter", "5"],
                         capture_output=True, text=True, timeout=300, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    d = json.loads(out.stdout.strip().splitlines()[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
