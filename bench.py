#!/usr/bin/env python
"""Benchmark of the batched ADMM collision-avoidance solver on one GB300.

A step is one whole ADMM solve (Sec. IV-B) of a batch of independent 2-D
tractor-trailer scenarios shaped like the batching form (N ~ U[20,80],
obstacles ~ U[8,64], 3-16 faces, 1-2 parts), from the same cold start, plus
the scale-based collision check (Sec. III-A) of the returned plans.
Metrics: pair-QP solves/s (value) and ADMM solves/s at residual <= 1e-4.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1: one process per GPU (torchrun, NCCL), each rank solving its own batch
of scenarios (weak scaling, no data-path collective); timing is the max over
ranks.  --impl reference times the FP64 CPU oracle on a bounded sample of the
same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pair-QP solves/s and ADMM solves/s at residual<=1e-4, batched FP32 vs plain GPU form"
UNIT = "pair-QP solves/s"


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of the SM clock and throttle reasons (read only)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def pair_bytes(scene, itemsize=4):
    """Algorithmic bytes of one fused pair-kernel launch per scenario:
    read and write zeta (1), xi (d) and y (n_y of each pair)."""
    d = scene.dim
    out = np.zeros(scene.n_scen)
    for s in range(scene.n_scen):
        N, NP = int(scene.horizon[s]), scene.n_parts(s)
        m0, m1 = int(scene.obs_begin[s]), int(scene.obs_begin[s + 1])
        p0 = int(scene.part_begin[s])
        nr = scene.part_nf[p0:p0 + NP].sum()
        ny = (scene.obs_nf[m0:m1].sum() + (m1 - m0)) * NP * N + nr * (m1 - m0) * N   # sum over pairs of n_y
        P = (m1 - m0) * NP * N
        out[s] = itemsize * (2 * (d + 1) * P + 2 * ny)
    return out


def shard_first(rank: int, per_rank: int) -> int:
    """Weak scaling: rank r solves its own scenarios r*S .. (r+1)*S - 1 (their
    seeds), so no data crosses ranks."""
    return rank * per_rank


def reduce_over_ranks(tot, dist, device):
    """Whole-job totals of the per-rank vector `tot` (solves, converged
    scenarios, timed ms, algorithmic bytes, kernel ms, launches, pair units):
    sums over ranks, except the timed region (index 2), which is the slowest
    rank's."""
    import torch
    t = torch.tensor(np.asarray(tot, dtype=np.float64), device=device)
    tmax = t.clone()
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    out = t.cpu().numpy()
    out[2] = float(tmax[2].item())
    return out


class Workload:
    """One FP32 workload resident on the GPU: the scene, its ADMM state at
    the cold start, and the benchmark step (solve + checks)."""

    def __init__(self, ctx, scene, params, warps=0):
        import torch

        from paper_2406_07048_gb300 import binding
        self.torch, self.binding = torch, binding
        self.scene, self.params = scene, params
        self.ds = binding.DeviceScene(ctx, scene, torch.float32)
        self.pb = binding.Problem(self.ds)
        self.s0, self.u0, self.y0 = self.pb.s.clone(), self.pb.u.clone(), self.pb.y.clone()
        # tile shape: the library's tuner times the fused pair kernel of short
        # solves from the cold start for each candidate
        self.tune = self.ds.autotune_warps(self.pb, params) if warps <= 0 else {}
        if warps > 0:
            self.ds.warps = warps

    def reset(self):
        pb = self.pb
        pb.s.copy_(self.s0)
        pb.u.copy_(self.u0)
        pb.y.copy_(self.y0)
        pb.zeta.zero_()
        pb.xi.zero_()

    def step(self, **over):
        """One step: the whole ADMM solve from the cold start, then the scale-LP
        collision check of the returned plan (Sec. III-A) and the FP64
        certificate margin of the returned duals (Sec. III-B)."""
        B, pb, FR, FO = self.binding, self.pb, self.scene.fr_max, self.scene.fo_max
        self.reset()
        rep = pb.solve(**dict(self.params, **over))
        sd = B.scale_detect(self.ds, pb.s, want_certificate=False, want_margin=False)
        margin = B.cert_margin(self.ds, pb.s, pb.y[:FR], pb.y[FR:FR + FO])
        return rep, sd, margin


def time_workload(wl, steps, warmup, device, dist=None, clocks=None):
    """Warm-up, then `steps` timed steps with kernel timing on; returns the
    per-rank totals and per-step reports."""
    torch = wl.torch
    for _ in range(warmup):
        wl.step()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
    ctx = wl.ds.ctx
    ctx.profile(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    reps = []
    for _ in range(steps):
        rep, sd, margin = wl.step()
        reps.append({k: v.clone() for k, v in rep.items()})
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    prof = ctx.profile_read()
    ctx.profile(False)
    if dist:
        dist.barrier()
    clk = clocks.stop() if clocks else None
    return ms, prof, reps, clk, margin


def solve_totals(scene, reps, itemsize=4):
    """Pair-QP solves (all, and of converged scenarios only), converged
    scenarios, algorithmic bytes of every pair-kernel launch, pair units and
    Riccati stages of a list of per-step reports."""
    bpp = pair_bytes(scene, itemsize)
    pc = scene.pair_counts.astype(np.float64)
    hz = scene.horizon.astype(np.float64)
    d1 = scene.dim + 1
    ny_sum = (bpp / itemsize - 2 * d1 * pc) / 2          # sum over a scenario's pairs of n_y
    b_first = itemsize * (d1 * pc + 2 * ny_sum)          # j = 0: zeta, xi read; y read and written
    b_full = itemsize * (2 * d1 * pc + 2 * ny_sum)       # dual update + QP: zeta, xi, y read and written
    b_head = itemsize * (2 * d1 * pc + ny_sum)           # dual update only (j = max_iter)
    t = dict(qp=0.0, qp_conv=0.0, conv=0, bytes=0.0, units=0.0, stages=0.0, iters=[])
    for rep in reps:
        it = rep["iters"].cpu().numpy().astype(np.float64)
        st = rep["status"].cpu().numpy()
        t["qp"] += float((pc * it).sum())
        t["qp_conv"] += float((pc * it)[st == 0].sum())
        t["conv"] += int((st == 0).sum())
        t["iters"].append(it)
        # a scenario retired at check j ran launches 0..j; one that reached
        # max_iter ran 0..max_iter-1 in full and a dual-update-only launch
        capped = st == 1
        n_full = np.where(capped, np.maximum(it - 1, 0), it)
        t["bytes"] += float((b_first + n_full * b_full + capped * b_head).sum())
        t["units"] += float((pc * (it + 1)).sum())
        t["stages"] += float((hz * it).sum())
    return t


def iteration_histogram(iters, max_iter):
    edges = [0, 25, 50, 100, 150, 200, 250, max_iter, max_iter + 1]
    edges = sorted(set(e for e in edges if e <= max_iter + 1))
    h = np.histogram(np.concatenate(iters), bins=edges)[0]
    return {"edges": edges, "counts": h.tolist()}


def issue_fraction(prof_pair_ms, pair_units, n_sm, sm_mhz):
    """FP32-issue side of the pair kernel's roofline: warp instructions per
    pair-iteration from the committed ncu counters of the current kernel
    sources, times the pair-iterations of the timed launches, over their
    event time, against 4 warp-instruction issue slots per SM per clock."""
    kv = _read_kv(os.path.join(ROOT, "profiles", "k_pair_traffic.txt"))
    if kv.get("kernel_sha") != _kernel_sha() or "warp_inst_per_pair" not in kv or prof_pair_ms <= 0:
        return None
    achieved = float(kv["warp_inst_per_pair"]) * pair_units / (prof_pair_ms / 1e3)
    peak = n_sm * 4 * sm_mhz * 1e6
    return {"achieved_warp_inst_per_s": achieved, "peak_warp_inst_per_s": peak, "frac": achieved / peak,
            "warp_inst_per_pair": float(kv["warp_inst_per_pair"]),
            "lanes_per_inst": float(kv["lanes_per_inst"]) if "lanes_per_inst" in kv else None,
            "source": "ncu smsp__inst_executed.sum of the current kernel (profiles/k_pair_traffic.txt); "
                      f"peak = {n_sm} SMs x 4 issue slots x {sm_mhz:.0f} MHz (median SM clock of the timed region)"}


def _read_kv(path):
    kv = {}
    if os.path.exists(path):
        with open(path) as f:
            for line in f:
                if "=" in line and not line.startswith("#"):
                    k, v = line.strip().split("=", 1)
                    kv[k] = v
    return kv


def gpu_arm(args):
    import torch

    from paper_2406_07048_gb300 import binding, synth

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    S = args.scen
    scene = synth.config3(n_scen=S, first=shard_first(rank, S))
    ctx = binding.Context(local)
    params = dict(binding.DEFAULTS)
    params["max_iter"] = args.max_iter
    for k in ("prox", "damp"):
        if getattr(args, k) is not None:
            params[k] = getattr(args, k)
    if args.riccati_f32:
        params["flags"] = binding.OCA_ADMM_RICCATI_F32
    wl = Workload(ctx, scene, params, args.warps)
    pb, ds = wl.pb, wl.ds

    clocks = ClockSampler(local)
    ms, prof, reps, clk, margin = time_workload(wl, args.steps, args.warmup, dev, dist, clocks)
    t = solve_totals(scene, reps)
    pc = scene.pair_counts.astype(np.float64)
    tot = np.array([t["qp"], t["conv"], ms, t["bytes"], prof["pair_ms"], prof["traj_ms"], prof["pair_launches"],
                    t["units"], t["qp_conv"]], dtype=np.float64)
    if dist:
        tot = reduce_over_ranks(tot, dist, dev)
        ms = float(tot[2])
    value = tot[0] / (ms / 1e3)
    admm_rate = tot[1] / (ms / 1e3)
    m_last = margin.cpu().numpy()

    # --- the same scenarios at a higher iteration cap (untimed): how many
    # more meet the stopping rule
    cap2 = max(1000, args.max_iter)
    rep2, _, _ = wl.step(max_iter=cap2)
    st2 = rep2["status"].cpu().numpy()

    # --- end to end through the public API with host buffers (pinned)
    h_in = {k: v.cpu().pin_memory() for k, v in dict(s_ref=pb.s_ref, s=wl.s0, u=wl.u0, y=wl.y0,
                                                      zeta=torch.zeros_like(pb.zeta),
                                                      xi=torch.zeros_like(pb.xi)).items()}
    h_out = {k: torch.empty_like(v, device="cpu").pin_memory() for k, v in dict(s=pb.s, u=pb.u).items()}
    h2d = sum(v.numel() * v.element_size() for v in h_in.values())
    d2h = sum(v.numel() * v.element_size() for v in h_out.values()) + S * 4 * 2     # + iters and status
    e_qp = 0.0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        pb.s_ref.copy_(h_in["s_ref"], non_blocking=True)
        pb.s.copy_(h_in["s"], non_blocking=True)
        pb.u.copy_(h_in["u"], non_blocking=True)
        pb.y.copy_(h_in["y"], non_blocking=True)
        pb.zeta.copy_(h_in["zeta"], non_blocking=True)
        pb.xi.copy_(h_in["xi"], non_blocking=True)
        rep = pb.solve(**params)
        h_out["s"].copy_(pb.s, non_blocking=True)
        h_out["u"].copy_(pb.u, non_blocking=True)
        it = rep["iters"].cpu().numpy()
        rep["status"].cpu()
        e_qp += float((pc * it).sum())
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0

    # --- plain per-scenario GPU form (one scenario per call, legacy stream, no graphs)
    plain = None
    if rank == 0 and args.plain > 0:
        idx = list(range(min(args.plain, S)))
        sub_ms, sub_solves = 0.0, 0.0
        for s in idx:
            sc1 = synth.subset(scene, [s])
            d1s = binding.DeviceScene(ctx, sc1, torch.float32)
            p1 = binding.Problem(d1s)
            p1.solve(**params)  # warm the path
            p1 = binding.Problem(d1s)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r1 = binding.admm_solve(d1s, p1.s_ref, p1.s, p1.u, p1.y, p1.zeta, p1.xi, stream=torch.cuda.default_stream(),
                                    **params)
            torch.cuda.synchronize()
            sub_ms += (time.perf_counter() - t0) * 1e3
            sub_solves += float(sc1.pair_counts[0] * int(r1["iters"][0]))
            d1s.close()
        plain = {"scenarios_timed": len(idx), "ms_per_scenario": sub_ms / len(idx),
                 "pair_qp_solves_per_s": sub_solves / (sub_ms / 1e3),
                 "batched_speedup": (sub_ms / len(idx)) / (ms / args.steps / S)}

    peak, peak_kind = _peaks()
    achieved = tot[3] / (tot[4] / 1e3) / 1e9 if tot[4] > 0 else 0.0
    traffic = None
    kv = _read_kv(os.path.join(ROOT, "profiles", "k_pair_traffic.txt"))
    if kv.get("kernel_sha") == _kernel_sha() and tot[6] > 0:
        # measured DRAM bytes per pair, scaled to the pairs an average launch processed
        traffic = float(kv["dram_bytes_per_pair"]) * tot[7] / tot[6]
    # per step: reset, 2 box inits, poses, gather, scale-detect poses + LP,
    # certificate margin = 8, and per iteration launch: pair kernel,
    # trajectory kernel, counter advance
    launches = int(8 * args.steps * world + 3 * tot[6])
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    sm_mhz = clk["sm_mhz"] if clk else 2070.0

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"batching form, 2-D tractor-trailer, {S} scenarios per GPU (N~U[20,80], "
                               f"obstacles~U[8,64], 3-16 faces, 1-2 parts), cold start, max_iter {args.max_iter}",
                   "scenarios_per_gpu": S, "pairs_per_gpu": int(scene.n_pairs),
                   "admm": {k: params[k] for k in ("sigma", "eps_pri", "eps_dual", "prox", "rho_box", "damp")},
                   "precision": "pair QPs / residuals / duals FP32, Riccati factorisation "
                                + ("FP32" if args.riccati_f32 else "FP64") + ", certificate margin FP64",
                   "step": "whole ADMM solve + scale-LP check + FP64 certificate margin of the returned duals",
                   "warps_per_tile": ds.warps, "tuner_ms": {str(k): round(v, 4) for k, v in wl.tune.items()},
                   "l2": "inputs larger than L2 (y alone %.0f MB)" % (pb.y.numel() * 4 / 1e6),
                   "parallelism": f"scenario shards x{world}"},
        "value_counts": "pair-QP solves of every scenario, converged or not (pairs x iterations)",
        "pair_qp_solves_per_s_converged": tot[8] / (ms / 1e3),
        "admm_solves_per_s": admm_rate,
        "converged_fraction": tot[1] / (S * world * args.steps),
        f"converged_fraction_at_{cap2}": float((st2 == 0).mean()),
        "failed_fraction": float((reps[-1]["status"].cpu().numpy() == 2).mean()),
        "mean_iterations": float(np.mean(np.concatenate(t["iters"]))),
        "iteration_histogram": iteration_histogram(t["iters"], args.max_iter),
        "certified_free_fraction": float((m_last >= 1.0).mean()),
        "kernel_ms": {"pair": tot[4], "trajectory": tot[5], "pair_launches": int(tot[6])},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "kernel": "k_pair (fused dual update + pair QP)",
                     "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else peak_kind,
                     "issue": issue_fraction(tot[4], tot[7], n_sm, sm_mhz)},
        "e2e": {"value": e_qp / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": launches,
        "plain_form": plain,
    }
    if clk:
        out["clocks"] = clk
    fp64 = binding.fp64_peak(local) if rank == 0 else 0.0
    if rank == 0 and prof["traj_ms"] > 0:
        out["roofline_trajectory"] = traj_roofline(scene, t["stages"], prof["traj_ms"], fp64)
    if rank == 0 and args.quad > 0:
        out["quad"] = quad_workload(ctx, args, params, fp64, world == 1 and not args.no_cpu_baseline, n_sm, sm_mhz)
    if rank == 0 and args.precision:
        out["precision_form"] = precision_form(ctx)
    if rank == 0 and not args.no_lemke:
        out["pair_solver_comparison"] = solver_comparison(ds, wl.s0, wl.y0, params)
    if rank == 0 and args.lq:
        out["lq_scan_vs_sequential"] = lq_crossover(ctx)
    if rank == 0 and args.closed_loop > 0:
        out["closed_loop"] = closed_loop(ctx, args, params, world == 1 and not args.no_cpu_baseline)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(scene, params, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


def traj_roofline(scene, stages, traj_ms, fp64):
    """Trajectory kernel against the measured FP64 rate: algorithmic FP64
    flops of its backward recursion and forward sweep per stage."""
    f_stage = ric_flops_per_stage(scene.model.ns, scene.model.nu)
    ach = f_stage * stages / (traj_ms / 1e3) / 1e9
    return {"bound": "fp64", "achieved": ach, "peak": fp64, "unit": "GFLOP/s", "frac": ach / fp64 if fp64 > 0 else None,
            "kernel": "k_riccati (FP64 backward Riccati recursion + forward sweep; the FP32 stage assembly not counted)",
            "flops_per_stage": f_stage, "stages": stages,
            "peak_source": "measured on this GPU (oca_fp64_peak: FP64 FMA microbenchmark)"}


def quad_workload(ctx, args, params, fp64, with_oracle, n_sm, sm_mhz):
    """The 3-D quadrotor workload (Sec. V-A's vehicle): 64 scenes x 128
    polyhedra (6-20 faces, half in narrow-gap pairs) x 3 boxes x N = 40,
    FP32 pair QPs, FP64 Riccati; the same step and metrics as the headline."""
    from paper_2406_07048_gb300 import synth
    sc = synth.config4(n_scen=args.quad)
    wl = Workload(ctx, sc, params, 0)
    ms, prof, reps, _, margin = time_workload(wl, args.quad_steps, 2, None)
    t = solve_totals(sc, reps)
    peak, peak_kind = _peaks()
    achieved = t["bytes"] / (prof["pair_ms"] / 1e3) / 1e9 if prof["pair_ms"] > 0 else 0.0
    pb = pair_bytes(sc)
    out = {"workload": f"3-D quadrotor, {args.quad} scenes x 128 polyhedra (6-20 faces) x 3 boxes x N=40, "
                       f"cold start, max_iter {params['max_iter']}, FP32 pair QPs, FP64 Riccati",
           "pairs": int(sc.n_pairs), "steps": args.quad_steps, "ms_per_step": ms / args.quad_steps,
           "pair_qp_solves_per_s": t["qp"] / (ms / 1e3),
           "pair_qp_solves_per_s_converged": t["qp_conv"] / (ms / 1e3),
           "admm_solves_per_s": t["conv"] / (ms / 1e3),
           "converged_fraction": t["conv"] / (args.quad * args.quad_steps),
           "mean_iterations": float(np.mean(np.concatenate(t["iters"]))),
           "certified_free_fraction": float((margin.cpu().numpy() >= 1.0).mean()),
           "warps_per_tile": wl.ds.warps,
           "algorithmic_bytes_per_pair_iteration": float(pb.sum() / sc.n_pairs),
           "kernel_ms": {"pair": prof["pair_ms"], "trajectory": prof["traj_ms"],
                         "pair_launches": int(prof["pair_launches"])},
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                        "kernel": "k_pair (fused dual update + pair QP)", "traffic": None,
                        "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"},
           "roofline_trajectory": traj_roofline(sc, t["stages"], prof["traj_ms"], fp64) if prof["traj_ms"] > 0 else None}
    if with_oracle:
        import oracle
        n = min(16, args.quad)
        sub = synth.subset(sc, list(range(n)))
        kw = {k: params[k] for k in ("sigma", "eps_pri", "eps_dual", "prox", "rho_box", "damp")}
        t0 = time.perf_counter()
        r = oracle.admm_batch(sub, max_iter=20, **kw)
        el = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": float((sub.pair_counts * r["iters"]).sum()) / el, "unit": UNIT,
                               "cores": oracle.num_threads(), "kind": "oracle",
                               "sample": f"scenes 0..{n - 1}, the first 20 ADMM iterations, {el:.1f} s"}
    wl.ds.close()
    return out


def precision_form(ctx):
    """Precision form (config 2: tractor-trailer, N = 50, 32 obstacles, 3,200
    pairs, 300 iterations): the FP32 GPU path against the FP64 oracle, error
    per result.  alpha* and the pair-QP objective are compared on identical
    inputs (the GPU's final plan and duals, as stored); the trajectory and its
    cost compare the two whole solves."""
    import torch

    import oracle
    from paper_2406_07048_gb300 import binding, synth
    sc = synth.config2()
    P = sc.n_pairs
    ds = binding.DeviceScene(ctx, sc, torch.float32)
    out = {"workload": f"config 2: 2-D tractor-trailer, N=50, 32 obstacles of 3-12 faces, {P} pairs, 300 iterations"}
    for K in (10, 300):
        pb = binding.Problem(ds)
        rep = pb.solve(max_iter=K)
        ref = oracle.admm_batch(sc, max_iter=K)
        s_g = pb.s.double().cpu().numpy()
        e = np.abs(s_g - ref["s"])
        c_g, c_o = float(rep["cost"][0]), float(ref["cost"][0])
        out[f"after_{K}_iterations"] = {
            "trajectory_max_abs": float(e.max()), "trajectory_median_abs": float(np.median(e)),
            "cost_rel": abs(c_g - c_o) / abs(c_o), "iters_gpu": int(rep["iters"][0]), "iters_oracle": int(ref["iters"][0]),
            "r_pri_gpu": float(rep["r_pri"][0]), "r_pri_oracle": float(ref["r_pri"][0]),
            "r_dual_gpu": float(rep["r_dual"][0]), "r_dual_oracle": float(ref["r_dual"][0])}
    # per pair on identical inputs: the GPU's final plan (FP32) and duals
    s32 = pb.s.double().cpu().numpy()
    sd = binding.scale_detect(ds, pb.s)
    a_g = sd["alpha"].double().cpu().numpy()
    a_o = oracle.scale_batch(sc, s32)["alpha"]
    ea = np.abs(a_g - a_o) / np.maximum(1.0, np.abs(a_o))
    far = np.abs(a_o - 1.0) > 1e-3
    v_g = sd["verdict"].cpu().numpy().astype(bool)
    y = ds.to_host_pairs(pb.y)
    z = pb.zeta.double().cpu().numpy()
    x = ds.to_host_pairs(pb.xi)
    q = binding.pair_qp(ds, pb.s, pb.zeta, pb.xi, pb.y, prox=binding.DEFAULTS["prox"], want_v=True)
    qo = oracle.pair_qp_batch(sc, s32, z, x, y, prox=binding.DEFAULTS["prox"])
    o_g = q["obj"].double().cpu().numpy()
    eo = np.abs(o_g - qo["obj"]) / np.maximum(1.0, np.abs(qo["obj"]))
    FR, FO = sc.fr_max, sc.fo_max
    m_g = binding.cert_margin(ds, pb.s, pb.y[:FR], pb.y[FR:FR + FO]).cpu().numpy()
    out["per_pair"] = {
        "alpha_rel_max": float(ea.max()), "alpha_rel_median": float(np.median(ea)),
        "verdicts_identical_where_far_from_1": bool((v_g[far] == (a_o[far] >= 1.0)).all()),
        "qp_objective_rel_max": float(eo.max()), "qp_objective_rel_median": float(np.median(eo)),
        "certificate_margin_min": float(m_g.min()),
        "note": "relative errors floored at 1: |gpu - oracle| / max(1, |oracle|); the pair QP is the step-1 "
                "QP at the final iterate (prox as the solve)"}
    ds.close()
    return out


def lq_crossover(ctx, grid=((12, 4, (16, 64, 256, 1024), (1, 4, 16, 64, 256)),
                               (5, 2, (16, 64, 256, 1024), (1, 16, 256)))):
    """The step-2 LQ problem solved by the sequential Riccati recursion and in
    parallel-in-time form (oca_lq_solve), on random problems of the models'
    sizes (12 states / 4 inputs: quadrotor; 5 / 2: tractor-trailer): device
    time of one batched solve (CUDA events, mean of 10 after 2 warm-ups)."""
    import torch

    from paper_2406_07048_gb300 import binding
    rows = []
    rng = np.random.default_rng(0)
    for ns, nu, Ns, Ss in grid:
        for N in Ns:
            for S in Ss:
                A = torch.eye(ns, dtype=torch.float64, device="cuda").expand(S, N, ns, ns) + \
                    0.05 * torch.randn(S, N, ns, ns, dtype=torch.float64, device="cuda")
                Bm = 0.2 * torch.randn(S, N, ns, nu, dtype=torch.float64, device="cuda")
                c = 0.1 * torch.randn(S, N, ns, dtype=torch.float64, device="cuda")
                L = torch.randn(S, N + 1, ns, ns, dtype=torch.float64, device="cuda")
                Q = L @ L.transpose(-1, -2) / ns + 0.1 * torch.eye(ns, dtype=torch.float64, device="cuda")
                q = torch.randn(S, N + 1, ns, dtype=torch.float64, device="cuda")
                Lr = torch.randn(S, N, nu, nu, dtype=torch.float64, device="cuda")
                R = Lr @ Lr.transpose(-1, -2) / nu + 0.1 * torch.eye(nu, dtype=torch.float64, device="cuda")
                r = torch.randn(S, N, nu, dtype=torch.float64, device="cuda")
                s0 = torch.randn(S, ns, dtype=torch.float64, device="cuda")
                work = torch.empty(binding.lq_workspace_bytes(ns, nu, N, S), dtype=torch.uint8, device="cuda")
                row = {"ns": ns, "nu": nu, "N": N, "S": S}
                outs = {}
                for name, method in (("sequential_ms", binding.OCA_LQ_SEQUENTIAL), ("scan_ms", binding.OCA_LQ_SCAN)):
                    for _ in range(2):
                        o = binding.lq_solve(ctx, A, Bm, c, Q, q, R, r, s0, method=method, want_value=False, work=work)
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    for _ in range(10):
                        o = binding.lq_solve(ctx, A, Bm, c, Q, q, R, r, s0, method=method, want_value=False, work=work)
                    e1.record()
                    torch.cuda.synchronize()
                    row[name] = e0.elapsed_time(e1) / 10
                    outs[name] = o
                d = (outs["scan_ms"]["s"] - outs["sequential_ms"]["s"]).abs().max().item()
                row["max_state_diff"] = d
                row["scan_speedup"] = row["sequential_ms"] / row["scan_ms"]
                rows.append(row)
    return {"what": "step-2 LQ problem, FP64, random dense stage matrices: sequential Riccati recursion "
                    "(one CTA per problem) vs parallel-in-time composition (log2(N+1) rounds), "
                    "device time per batched solve incl. gains and rollout",
            "rows": rows}


def solver_comparison(ds, s0, y_cold, params):
    """Step 1 of one ADMM iteration on the benchmark's scenes (cold start) by
    the hot path's solver and by the paper's Lemke route (one thread per LCP
    row), each timed with CUDA events over 3 launches after a warm-up."""
    import torch

    from paper_2406_07048_gb300 import binding
    zeta = torch.zeros(ds.n_pairs, dtype=ds.dtype, device=ds.device)
    xi = torch.zeros(ds.scene.dim, ds.n_pairs, dtype=ds.dtype, device=ds.device)
    prox = params["prox"]
    res = {}
    for name, fn in (("semismooth_newton", lambda: binding.pair_qp(ds, s0, zeta, xi, y_cold, prox=prox, want_v=True)),
                     ("lemke", lambda: binding.pair_qp_lemke(ds, s0, zeta, xi, y_cold, prox=prox))):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(3):
            out = fn()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 3
        st = out["status"].cpu().numpy()
        res[name] = {"ms_per_launch": ms, "pair_qp_solves_per_s": ds.n_pairs / (ms / 1e3),
                     "ok_fraction": float((st == 0).mean())}
    res["workload"] = f"step 1 of the first ADMM iteration, {ds.n_pairs} pairs, prox {prox}, FP32 (launch includes poses)"
    res["speedup"] = res["lemke"]["ms_per_launch"] / res["semismooth_newton"]["ms_per_launch"]
    return res


def ric_flops_per_stage(ns: int, nu: int) -> int:
    """FP64 flops (2 per FMA) of one stage of the trajectory kernel's backward
    recursion and forward sweep: Y = P [A | B | c] (ns x (ns+nu+1), ns terms
    each), the upper triangle and gradient column of the stage matrix (ns
    terms each), [K | k] = -Quu^-1 [Qus | qu], the upper triangle of P and p,
    then u = K s + k and s' = A s + B u + c."""
    nx, nz = ns + nu + 1, ns + nu
    fma = (ns * nx * ns + (nz * (nz + 1) // 2 + nz) * ns + nu * (ns + 1) * nu
           + (ns * (ns + 1) // 2 + ns) * nu + nu * ns + ns * nz)
    return 2 * fma


def closed_loop(ctx, args, params, with_oracle):
    """Receding-horizon runs shaped like the paper's simulation (Sec. V-B):
    quadrotor, 32 polyhedra, N = 16, 25 s reference, 20 x 20 x 6 m sensing;
    every scenario advanced by args.closed_loop control steps in one
    oca_mpc_run call.  The oracle's loop is timed beside it on 2 scenarios."""
    import torch

    from paper_2406_07048_gb300 import binding, synth
    S, C, mi = 256, args.closed_loop, 50
    sc, ref = synth.closed_loop(S)
    x0 = ref[:, 0].copy()
    ds = binding.DeviceScene(ctx, sc, torch.float32)
    kw = dict(params)
    kw["max_iter"] = mi
    kw.pop("flags", None)
    binding.mpc_run(ds, ref, sc.obs_center, x0, 2, **kw)  # warm the path
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g = binding.mpc_run(ds, ref, sc.obs_center, x0, C, **kw)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    xh = g["x_hist"].double().cpu().numpy()
    uh = g["u_hist"].double().cpu().numpy()
    col = g["collided"].cpu().numpy()
    m = sc.model
    e = xh[:, :C + 1] - ref[:, :C + 1]
    cost = (e * e * m.Qs).sum(axis=(1, 2)) + (uh * uh * m.Qu).sum(axis=(1, 2))
    out = {"workload": f"closed loop, 3-D quadrotor, {S} scenarios x {C} control steps (dt 0.1 s), 32 polyhedra in "
                       f"70x20x6 m, N=16, sensing 20x20x6 m, warm-started ADMM max_iter {mi}, FP32",
           "control_steps_per_s": S * C / dt, "wall_s": dt,
           "mean_admm_iterations_per_step": float(g["iters"].float().mean()),
           "success_rate": float(np.mean(col < 0)), "navigation_cost_mean": float(cost.mean())}
    if with_oracle:
        import oracle
        sub = synth.subset(sc, [0, 1])
        cs = min(C, 10)
        t0 = time.perf_counter()
        oracle.mpc_run(sub, ref[:2], x0[:2], cs, max_iter=mi, **{k: kw[k] for k in
                                                                  ("sigma", "eps_pri", "eps_dual", "prox", "rho_box",
                                                                   "damp")})
        od = time.perf_counter() - t0
        out["oracle"] = {"control_steps_per_s": 2 * cs / od, "sample": f"2 scenarios x {cs} control steps",
                         "cores": oracle.num_threads()}
    ds.close()
    return out


def _kernel_sha():
    import hashlib
    h = hashlib.sha1()
    for f in ("oca_pair.cu", "oca_solvers.cuh", "oca_common.cuh"):
        with open(os.path.join(ROOT, "paper_2406_07048_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def cpu_baseline(scene, params, seconds):
    """The FP64 oracle as it stands on a bounded sample of the workload."""
    import oracle
    from paper_2406_07048_gb300 import synth
    oracle.build()
    cores = oracle.num_threads()
    done, solves, conv = 0, 0.0, 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < seconds and done < scene.n_scen:
        idx = list(range(done, min(done + cores, scene.n_scen)))
        sub = synth.subset(scene, idx)
        r = oracle.admm_batch(sub, nthreads=cores, **{k: params[k] for k in
                                                       ("sigma", "eps_pri", "eps_dual", "prox", "max_iter",
                                                        "rho_box", "damp")})
        solves += float((sub.pair_counts * r["iters"]).sum())
        conv += int((r["status"] == 0).sum())
        done += len(idx)
    el = time.perf_counter() - t0
    # the same oracle on one thread: whole solves of the first scenarios, for
    # about a quarter of the all-core budget
    one_solves, n1 = 0.0, 0
    t1 = time.perf_counter()
    while time.perf_counter() - t1 < seconds / 4 and n1 < scene.n_scen:
        sub = synth.subset(scene, [n1])
        r = oracle.admm_batch(sub, nthreads=1, **{k: params[k] for k in
                                                  ("sigma", "eps_pri", "eps_dual", "prox", "max_iter", "rho_box",
                                                   "damp")})
        one_solves += float((sub.pair_counts * r["iters"]).sum())
        n1 += 1
    el1 = time.perf_counter() - t1
    one = one_solves / el1
    oracle.admm_batch(synth.subset(scene, [0]), nthreads=cores, max_iter=0)  # restore the thread count
    return {"value": solves / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{done} of the {scene.n_scen} scenarios, whole ADMM solves, {el:.1f} s",
            "admm_solves_per_s": conv / el,
            "single_thread": {"value": one, "unit": UNIT, "cores": 1,
                              "sample": f"scenarios 0..{n1 - 1}, whole ADMM solves, {el1:.1f} s"}}


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_2406_07048_gb300 import binding, synth
    oracle.build()
    cores = oracle.num_threads()
    S = args.scen
    scene = synth.config3(n_scen=S)
    params = dict(binding.DEFAULTS)
    params["max_iter"] = args.max_iter
    for k in ("prox", "damp"):
        if getattr(args, k) is not None:
            params[k] = getattr(args, k)
    kw = {k: params[k] for k in ("sigma", "eps_pri", "eps_dual", "prox", "max_iter", "rho_box", "damp")}
    per_step = max(1, cores)

    def one(step_i):
        idx = [(step_i * per_step + k) % S for k in range(per_step)]
        sub = synth.subset(scene, idx)
        r = oracle.admm_batch(sub, nthreads=cores, **kw)
        return float((sub.pair_counts * r["iters"]).sum()), int((r["status"] == 0).sum())

    for w in range(args.warmup):
        one(w)
    t0 = time.perf_counter()
    solves, conv = 0.0, 0
    for k in range(args.steps):
        a, b = one(args.warmup + k)
        solves += a
        conv += b
    el = time.perf_counter() - t0
    v = solves / el
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"batching form, 2-D tractor-trailer, {S} scenarios (bounded sample of "
                                  f"{per_step} scenarios per step on the host cores)", "max_iter": args.max_iter},
           "admm_solves_per_s": conv / el,
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": f"{per_step} scenarios per step, {args.steps} steps"},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--scen", type=int, default=2048)
    ap.add_argument("--max-iter", type=int, default=300)
    ap.add_argument("--plain", type=int, default=16, help="scenarios timed in the plain per-scenario form")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--warps", type=int, default=0, help="warps per tile (0: autotune)")
    ap.add_argument("--riccati-f32", action="store_true", help="factorise the trajectory QP in FP32")
    ap.add_argument("--no-lemke", action="store_true", help="skip the pair-solver comparison line")
    ap.add_argument("--closed-loop", type=int, default=250, help="control steps of the closed-loop line (0: off)")
    ap.add_argument("--prox", type=float, default=None, help="proximal weight of the pair QP (default: library default)")
    ap.add_argument("--damp", type=float, default=None, help="proximal damping of the trajectory step")
    ap.add_argument("--quad", type=int, default=64, help="scenes of the quadrotor line (0: off)")
    ap.add_argument("--quad-steps", type=int, default=3, help="timed steps of the quadrotor line")
    ap.add_argument("--precision", type=int, default=1, help="precision-form line (config 2 vs the oracle; 0: off)")
    ap.add_argument("--lq", type=int, default=1, help="sequential vs parallel-in-time LQ solve line (0: off)")
    args = ap.parse_args()
    if args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
