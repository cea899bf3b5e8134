"""Python binding of the C-ABI in include/oca.h (argument marshalling only).

Device memory and streams come from PyTorch; every computation runs in
``liboca.so``.  There is no CPU fallback: if the library is missing this
module raises.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np
import torch

from . import synth

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liboca.so")
_lib = None

OCA_OK = 0
STATUS_NAMES = {0: "OCA_OK", 1: "OCA_ERR_INVALID_ARGUMENT", 2: "OCA_ERR_CUDA", 3: "OCA_ERR_NO_MEMORY",
                4: "OCA_ERR_UNSUPPORTED", 5: "OCA_ERR_CAPACITY"}
OCA_ADMM_RICCATI_F32 = 1
OCA_ADMM_FIXED_POINT = 2
MAX_OBS_FACES, MAX_PART_FACES, MAX_HORIZON = 24, 8, 256


class OcaError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(code, code)}")
        self.code = code


class SceneDesc(C.Structure):
    _fields_ = [("dim", C.c_int32), ("dtype", C.c_int32), ("n_scen", C.c_int32), ("fo_max", C.c_int32),
                ("fr_max", C.c_int32), ("obs_begin", C.c_void_p), ("obs_nf", C.c_void_p),
                ("part_begin", C.c_void_p), ("part_nf", C.c_void_p), ("part_link", C.c_void_p),
                ("horizon", C.c_void_p), ("obs_C", C.c_void_p), ("obs_d", C.c_void_p), ("part_A", C.c_void_p),
                ("part_b", C.c_void_p), ("part_off", C.c_void_p)]


class SceneInfo(C.Structure):
    _fields_ = [("n_pairs", C.c_int64), ("n_states", C.c_int64), ("n_ctrls", C.c_int64), ("ny_max", C.c_int32),
                ("n_tiles", C.c_int32), ("pair_begin", C.POINTER(C.c_int64)),
                ("state_begin", C.POINTER(C.c_int64)), ("ctrl_begin", C.POINTER(C.c_int64))]


class ModelC(C.Structure):
    _fields_ = [("kind", C.c_int32), ("dt", C.c_double), ("param", C.c_double * 8), ("Qs", C.c_double * 12),
                ("Qu", C.c_double * 4), ("s_lo", C.c_double * 12), ("s_hi", C.c_double * 12),
                ("u_lo", C.c_double * 4), ("u_hi", C.c_double * 4)]


class AdmmParams(C.Structure):
    _fields_ = [("sigma", C.c_double), ("eps_pri", C.c_double), ("eps_dual", C.c_double), ("prox", C.c_double),
                ("max_iter", C.c_int32), ("flags", C.c_int32), ("rho_box", C.c_double), ("damp", C.c_double)]


class ProfileStats(C.Structure):
    _fields_ = [("pair_ms", C.c_double), ("traj_ms", C.c_double), ("pair_launches", C.c_int64),
                ("traj_launches", C.c_int64)]


class MpcParams(C.Structure):
    _fields_ = [("n_steps", C.c_int32), ("reserved", C.c_int32), ("window", C.c_double * 3)]


class Report(C.Structure):
    _fields_ = [("iters", C.c_void_p), ("status", C.c_void_p), ("r_pri", C.c_void_p), ("r_dual", C.c_void_p),
                ("cost", C.c_void_p)]


EXPORTED = ["oca_create", "oca_destroy", "oca_status_string", "oca_scene_create", "oca_scene_destroy",
            "oca_scene_info_get", "oca_scene_set_warps", "oca_scene_get_warps", "oca_scale_detect_batch",
            "oca_pair_qp_batch", "oca_admm_solve", "oca_profile_enable", "oca_profile_read",
            "oca_scale_detect_noalloc", "oca_admm_tape_bytes", "oca_admm_solve_taped", "oca_admm_backward",
            "oca_mpc_run", "oca_pair_qp_lemke_batch", "oca_admm_fixed_point_tape_bytes", "oca_fp64_peak",
            "oca_cert_margin_batch", "oca_lq_workspace_bytes", "oca_lq_solve"]


def lib():
    """Load liboca.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        P, I, D = C.c_void_p, C.c_int, C.c_double
        L.oca_create.argtypes = [C.POINTER(P), I]
        L.oca_create.restype = I
        L.oca_destroy.argtypes = [P]
        L.oca_destroy.restype = None
        L.oca_status_string.argtypes = [I]
        L.oca_status_string.restype = C.c_char_p
        L.oca_scene_create.argtypes = [P, C.POINTER(SceneDesc), C.POINTER(P)]
        L.oca_scene_create.restype = I
        L.oca_scene_destroy.argtypes = [P]
        L.oca_scene_destroy.restype = None
        L.oca_scene_info_get.argtypes = [P, C.POINTER(SceneInfo)]
        L.oca_scene_info_get.restype = I
        L.oca_scene_set_warps.argtypes = [P, I]
        L.oca_scene_set_warps.restype = I
        L.oca_scene_get_warps.argtypes = [P]
        L.oca_scene_get_warps.restype = I
        L.oca_scale_detect_batch.argtypes = [P, P, C.POINTER(ModelC), P, P, P, P, P, P, P, P]
        L.oca_scale_detect_batch.restype = I
        L.oca_cert_margin_batch.argtypes = [P, P, C.POINTER(ModelC), P, P, P, P, P]
        L.oca_cert_margin_batch.restype = I
        L.oca_lq_workspace_bytes.argtypes = [I, I, I, I, C.POINTER(C.c_int64)]
        L.oca_lq_workspace_bytes.restype = I
        L.oca_lq_solve.argtypes = [P, I, I, I, I, I, P, P, P, P, P, P, P, P, P, P, P, P, P, P, C.c_int64, P]
        L.oca_lq_solve.restype = I
        L.oca_pair_qp_batch.argtypes = [P, P, C.POINTER(ModelC), P, P, P, D, P, P, P, P, P, P]
        L.oca_pair_qp_batch.restype = I
        L.oca_admm_solve.argtypes = [P, P, C.POINTER(ModelC), C.POINTER(AdmmParams), P, P, P, P, P, P,
                                     C.POINTER(Report), P]
        L.oca_admm_solve.restype = I
        L.oca_profile_enable.argtypes = [P, I]
        L.oca_profile_enable.restype = I
        L.oca_profile_read.argtypes = [P, C.POINTER(ProfileStats)]
        L.oca_profile_read.restype = I
        L.oca_scale_detect_noalloc.argtypes = [C.POINTER(SceneDesc), C.POINTER(ModelC), P, P, P, P, P, P, P]
        L.oca_scale_detect_noalloc.restype = I
        L.oca_admm_tape_bytes.argtypes = [P, C.POINTER(ModelC), I, C.POINTER(C.c_int64)]
        L.oca_admm_tape_bytes.restype = I
        L.oca_admm_fixed_point_tape_bytes.argtypes = [P, C.POINTER(ModelC), C.POINTER(C.c_int64)]
        L.oca_admm_fixed_point_tape_bytes.restype = I
        L.oca_fp64_peak.argtypes = [I, C.POINTER(C.c_double)]
        L.oca_fp64_peak.restype = I
        L.oca_admm_solve_taped.argtypes = [P, P, C.POINTER(ModelC), C.POINTER(AdmmParams), P, P, P, P, P, P,
                                           C.POINTER(Report), P, C.c_int64, P]
        L.oca_admm_solve_taped.restype = I
        L.oca_admm_backward.argtypes = [P, P, C.POINTER(ModelC), C.POINTER(AdmmParams), P, P, C.c_int64, P, P, P,
                                        P, P, P, P]
        L.oca_admm_backward.restype = I
        L.oca_mpc_run.argtypes = [P, P, C.POINTER(ModelC), C.POINTER(AdmmParams), C.POINTER(MpcParams), P, I, P, P,
                                  P, P, P, P, P, P, P, P, P, P, P]
        L.oca_mpc_run.restype = I
        L.oca_pair_qp_lemke_batch.argtypes = [P, P, C.POINTER(ModelC), P, P, P, D, P, P, P, P, P, P]
        L.oca_pair_qp_lemke_batch.restype = I
        _lib = L
    return _lib


def _check(code: int, where: str):
    if code != OCA_OK:
        raise OcaError(code, where)


def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous(), "device tensors must be contiguous CUDA tensors"
    return C.c_void_p(t.data_ptr())


def _stream(stream) -> C.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def model_c(m: synth.Model) -> ModelC:
    mc = ModelC()
    mc.kind = int(m.kind)
    mc.dt = float(m.dt)
    for i, v in enumerate(m.param):
        mc.param[i] = float(v)
    for i, v in enumerate(m.Qs):
        mc.Qs[i] = float(v)
    for i, v in enumerate(m.Qu):
        mc.Qu[i] = float(v)
    for i in range(12):
        mc.s_lo[i], mc.s_hi[i] = -float("inf"), float("inf")
    for i in range(4):
        mc.u_lo[i], mc.u_hi[i] = -float("inf"), float("inf")
    for name in ("s_lo", "s_hi", "u_lo", "u_hi"):
        arr = getattr(m, name, None)
        if arr is not None:
            for i, v in enumerate(arr):
                getattr(mc, name)[i] = float(v)
    return mc


class Context:
    """oca_create / oca_destroy."""

    def __init__(self, device: int = 0):
        self.device = device
        h = C.c_void_p()
        _check(lib().oca_create(C.byref(h), int(device)), "oca_create")
        self.h = h

    def profile(self, enable: bool = True):
        _check(lib().oca_profile_enable(self.h, int(bool(enable))), "oca_profile_enable")

    def profile_read(self) -> dict:
        ps = ProfileStats()
        _check(lib().oca_profile_read(self.h, C.byref(ps)), "oca_profile_read")
        return dict(pair_ms=ps.pair_ms, traj_ms=ps.traj_ms, pair_launches=ps.pair_launches,
                    traj_launches=ps.traj_launches)

    def close(self):
        if self.h:
            lib().oca_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class DeviceScene:
    """A synthetic scene uploaded to the GPU and prepared by oca_scene_create."""

    def __init__(self, ctx: Context, scene: synth.Scene, dtype=torch.float32):
        self.ctx, self.scene, self.dtype = ctx, scene, dtype
        dev = torch.device("cuda", ctx.device)
        f = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device=dev).contiguous()
        self.obs_C, self.obs_d = f(scene.obs_C), f(scene.obs_d)
        self.part_A, self.part_b, self.part_off = f(scene.part_A), f(scene.part_b), f(scene.part_off)
        i32 = lambda a: np.ascontiguousarray(a, dtype=np.int32)
        self._host = [i32(scene.obs_begin), i32(scene.obs_nf), i32(scene.part_begin), i32(scene.part_nf),
                      i32(scene.part_link), i32(scene.horizon)]
        d = SceneDesc()
        d.dim, d.dtype, d.n_scen = scene.dim, 1 if dtype == torch.float64 else 0, scene.n_scen
        d.fo_max, d.fr_max = scene.fo_max, scene.fr_max
        d.obs_begin, d.obs_nf, d.part_begin, d.part_nf, d.part_link, d.horizon = [a.ctypes.data for a in self._host]
        d.obs_C, d.obs_d = self.obs_C.data_ptr(), self.obs_d.data_ptr()
        d.part_A, d.part_b, d.part_off = self.part_A.data_ptr(), self.part_b.data_ptr(), self.part_off.data_ptr()
        self._create(d, dev)

    def _create(self, d: "SceneDesc", dev):
        self.desc = d
        h = C.c_void_p()
        _check(lib().oca_scene_create(self.ctx.h, C.byref(d), C.byref(h)), "oca_scene_create")
        self.h = h
        info = SceneInfo()
        _check(lib().oca_scene_info_get(h, C.byref(info)), "oca_scene_info_get")
        self.n_pairs, self.n_states, self.n_ctrls = info.n_pairs, info.n_states, info.n_ctrls
        self.ny_max, self.n_tiles = info.ny_max, info.n_tiles
        assert self.n_pairs == self.scene.n_pairs and self.ny_max == self.scene.ny_max
        self.model = model_c(self.scene.model)
        self.device = dev

    def with_offsets(self, obs_d: torch.Tensor) -> "DeviceScene":
        """A second scene over the same device geometry except the obstacle
        offsets, which are `obs_d` [M_tot, fo_max] (kept alive by the new
        scene).  It has its own workspace, so solves on it leave this scene
        and its offsets untouched."""
        new = DeviceScene.__new__(DeviceScene)
        new.ctx, new.scene, new.dtype = self.ctx, self.scene, self.dtype
        new.obs_C, new.part_A, new.part_b, new.part_off = self.obs_C, self.part_A, self.part_b, self.part_off
        new.obs_d = obs_d.detach().to(self.dtype).contiguous()
        assert new.obs_d.shape == self.obs_d.shape and new.obs_d.device == self.obs_d.device
        new._host = self._host
        d = SceneDesc()
        for name, _ in SceneDesc._fields_:
            setattr(d, name, getattr(self.desc, name))
        d.obs_d = new.obs_d.data_ptr()
        new._create(d, self.device)
        new.warps = self.warps
        return new

    def autotune_warps(self, problem: "Problem", params: Optional[dict] = None,
                       candidates=(1, 2, 3, 4, 6, 8, 16), iters: int = 8) -> dict:
        """Choose the warps per tile of the pair kernels by timing the fused
        pair kernel as the ADMM runs it: for each candidate, a short solve of
        `iters` iterations from the problem's current state (restored after
        every trial) with kernel timing on; the candidate with the least mean
        pair-kernel time per launch is set.  Returns {warps: ms per launch}."""
        kw = dict(DEFAULTS)
        kw.update(params or {})
        kw["max_iter"] = iters
        saved = [t.clone() for t in (problem.s, problem.u, problem.y, problem.zeta, problem.xi)]

        def restore():
            for dst, src in zip((problem.s, problem.u, problem.y, problem.zeta, problem.xi), saved):
                dst.copy_(src)

        times = {}
        for w in candidates:
            try:
                self.warps = w
            except OcaError as e:
                if e.code == 5:      # too many warps for the shared memory of this scene's face counts
                    continue
                raise
            restore()
            problem.solve(**kw)          # first use of this tile shape
            restore()
            torch.cuda.synchronize(self.device)
            self.ctx.profile(True)
            problem.solve(**kw)
            pr = self.ctx.profile_read()
            self.ctx.profile(False)
            times[w] = pr["pair_ms"] / max(pr["pair_launches"], 1)
        restore()
        self.warps = min(times, key=times.get)
        return times

    @property
    def warps(self) -> int:
        return int(lib().oca_scene_get_warps(self.h))

    @warps.setter
    def warps(self, w: int):
        _check(lib().oca_scene_set_warps(self.h, int(w)), "oca_scene_set_warps")

    def close(self):
        if getattr(self, "h", None):
            lib().oca_scene_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- helpers for pair-indexed arrays ----------------------------------
    def tensor(self, a, dtype=None) -> torch.Tensor:
        return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype or self.dtype, device=self.device).contiguous()

    def to_device_pairs(self, pair_major: np.ndarray) -> torch.Tensor:
        """[P, k] pair-major host array -> [k, P] component-major device tensor."""
        return self.tensor(np.ascontiguousarray(np.asarray(pair_major).reshape(self.n_pairs, -1).T))

    @staticmethod
    def to_host_pairs(comp_major: torch.Tensor) -> np.ndarray:
        """[k, P] component-major device tensor -> [P, k] pair-major float64 array."""
        return comp_major.double().cpu().numpy().T.copy()


def scale_detect(ds: DeviceScene, states: torch.Tensor, want_certificate: bool = True, want_margin: bool = True,
                 stream=None):
    """oca_scale_detect_batch: alpha*, lambda*, mu*, FP64 margin, verdict, status."""
    P = ds.n_pairs
    alpha = torch.empty(P, dtype=ds.dtype, device=ds.device)
    lam = torch.zeros(ds.scene.fr_max, P, dtype=ds.dtype, device=ds.device) if want_certificate else None
    mu = torch.zeros(ds.scene.fo_max, P, dtype=ds.dtype, device=ds.device) if want_certificate else None
    margin = torch.empty(P, dtype=torch.float64, device=ds.device) if want_margin else None
    verdict = torch.empty(P, dtype=torch.int32, device=ds.device)
    status = torch.empty(P, dtype=torch.int32, device=ds.device)
    _check(lib().oca_scale_detect_batch(ds.ctx.h, ds.h, C.byref(ds.model), _ptr(states), _ptr(alpha), _ptr(lam),
                                        _ptr(mu), _ptr(margin), _ptr(verdict), _ptr(status), _stream(stream)),
           "oca_scale_detect_batch")
    return dict(alpha=alpha, lam=lam, mu=mu, margin=margin, verdict=verdict, status=status)


def cert_margin(ds: DeviceScene, states: torch.Tensor, lam: torch.Tensor, mu: torch.Tensor, stream=None):
    """oca_cert_margin_batch: FP64 weak-duality margin [P] of the given
    lambda [fr_max, P] and mu [fo_max, P] (e.g. an ADMM solve's y[:fr_max]
    and y[fr_max:fr_max + fo_max]) at the given states."""
    margin = torch.empty(ds.n_pairs, dtype=torch.float64, device=ds.device)
    _check(lib().oca_cert_margin_batch(ds.ctx.h, ds.h, C.byref(ds.model), _ptr(states), _ptr(lam.contiguous()),
                                       _ptr(mu.contiguous()), _ptr(margin), _stream(stream)), "oca_cert_margin_batch")
    return margin


OCA_LQ_SEQUENTIAL, OCA_LQ_SCAN = 0, 1


def lq_workspace_bytes(ns: int, nu: int, N: int, n_problems: int) -> int:
    """oca_lq_workspace_bytes."""
    n = C.c_int64(0)
    _check(lib().oca_lq_workspace_bytes(int(ns), int(nu), int(N), int(n_problems), C.byref(n)),
           "oca_lq_workspace_bytes")
    return int(n.value)


def lq_solve(ctx: Context, A, B, c, Q, q, R, r, s0, method: int = OCA_LQ_SCAN, want_value=True, work=None,
             stream=None):
    """oca_lq_solve on FP64 device tensors shaped [S][N][..] (A, B, c, R, r),
    [S][N+1][..] (Q, q), [S][ns] (s0): returns s, u, P, p and status."""
    S, N1, ns = Q.shape[0], Q.shape[1], Q.shape[2]
    N = N1 - 1
    nu = R.shape[-1] if R is not None and R.dim() == 4 else 1
    dev = Q.device
    f64 = lambda t: None if t is None else t.to(torch.float64).contiguous()
    A, B, c, Q, q, R, r, s0 = map(f64, (A, B, c, Q, q, R, r, s0))
    s = torch.empty(S, N + 1, ns, dtype=torch.float64, device=dev)
    u = torch.empty(S, max(N, 0), nu, dtype=torch.float64, device=dev)
    P = torch.empty(S, N + 1, ns, ns, dtype=torch.float64, device=dev) if want_value else None
    p = torch.empty(S, N + 1, ns, dtype=torch.float64, device=dev) if want_value else None
    status = torch.empty(S, dtype=torch.int32, device=dev)
    wb = lq_workspace_bytes(ns, nu, N, S)
    if work is None:
        work = torch.empty(wb, dtype=torch.uint8, device=dev)
    _check(lib().oca_lq_solve(ctx.h, int(method), int(ns), int(nu), int(N), int(S), _ptr(A) if N > 0 else None,
                              _ptr(B) if N > 0 else None, _ptr(c) if N > 0 else None, _ptr(Q), _ptr(q),
                              _ptr(R) if N > 0 else None, _ptr(r) if N > 0 else None, _ptr(s0), _ptr(s),
                              _ptr(u) if N > 0 else None, _ptr(P), _ptr(p), _ptr(status), _ptr(work),
                              C.c_int64(work.numel()), _stream(stream)), "oca_lq_solve")
    return dict(s=s, u=u, P=P, p=p, status=status)


def scale_detect_noalloc(ds: DeviceScene, states: torch.Tensor, want_certificate: bool = True, stream=None):
    """oca_scale_detect_noalloc on a one-scenario scene (the library allocates
    nothing; the output tensors are allocated here by PyTorch)."""
    P = ds.n_pairs
    alpha = torch.empty(P, dtype=ds.dtype, device=ds.device)
    lam = torch.zeros(ds.scene.fr_max, P, dtype=ds.dtype, device=ds.device) if want_certificate else None
    mu = torch.zeros(ds.scene.fo_max, P, dtype=ds.dtype, device=ds.device) if want_certificate else None
    verdict = torch.empty(P, dtype=torch.int32, device=ds.device)
    status = torch.empty(P, dtype=torch.int32, device=ds.device)
    _check(lib().oca_scale_detect_noalloc(C.byref(ds.desc), C.byref(ds.model), _ptr(states), _ptr(alpha), _ptr(lam),
                                          _ptr(mu), _ptr(verdict), _ptr(status), _stream(stream)),
           "oca_scale_detect_noalloc")
    return dict(alpha=alpha, lam=lam, mu=mu, verdict=verdict, status=status)


def pair_qp(ds: DeviceScene, states, zeta, xi, y_in, prox: float = 0.0, y_out=None, want_v=True, stream=None):
    """oca_pair_qp_batch: y_out, v = K^T y + bq, obj, status."""
    P = ds.n_pairs
    if y_out is None:
        y_out = torch.zeros_like(y_in)
    v = torch.empty(ds.scene.dim + 1, P, dtype=ds.dtype, device=ds.device) if want_v else None
    obj = torch.empty(P, dtype=ds.dtype, device=ds.device) if want_v else None
    status = torch.empty(P, dtype=torch.int32, device=ds.device)
    _check(lib().oca_pair_qp_batch(ds.ctx.h, ds.h, C.byref(ds.model), _ptr(states), _ptr(zeta), _ptr(xi),
                                   float(prox), _ptr(y_in), _ptr(y_out), _ptr(v), _ptr(obj), _ptr(status),
                                   _stream(stream)), "oca_pair_qp_batch")
    return dict(y=y_out, v=v, obj=obj, status=status)


def pair_qp_lemke(ds: DeviceScene, states, zeta, xi, y_in, prox: float = 0.0, stream=None):
    """oca_pair_qp_lemke_batch (the paper's Lemke route): y_out, v, obj, status."""
    P = ds.n_pairs
    y_out = torch.zeros_like(y_in)
    v = torch.empty(ds.scene.dim + 1, P, dtype=ds.dtype, device=ds.device)
    obj = torch.empty(P, dtype=ds.dtype, device=ds.device)
    status = torch.empty(P, dtype=torch.int32, device=ds.device)
    _check(lib().oca_pair_qp_lemke_batch(ds.ctx.h, ds.h, C.byref(ds.model), _ptr(states), _ptr(zeta), _ptr(xi),
                                         float(prox), _ptr(y_in), _ptr(y_out), _ptr(v), _ptr(obj), _ptr(status),
                                         _stream(stream)), "oca_pair_qp_lemke_batch")
    return dict(y=y_out, v=v, obj=obj, status=status)


DEFAULTS = dict(sigma=300.0, eps_pri=1e-4, eps_dual=1e-4, prox=1.0, max_iter=300, rho_box=100.0, damp=100.0)


def admm_solve(ds: DeviceScene, s_ref, s, u, y, zeta, xi, sigma=300.0, eps_pri=1e-4, eps_dual=1e-4, prox=1.0,
               max_iter=300, flags=0, rho_box=100.0, damp=100.0, stream=None, tape=None):
    """oca_admm_solve (oca_admm_solve_taped when `tape` is given): updates s,
    u, y, zeta, xi in place; returns the report."""
    S = ds.scene.n_scen
    rep_t = dict(iters=torch.zeros(S, dtype=torch.int32, device=ds.device),
                 status=torch.full((S,), -1, dtype=torch.int32, device=ds.device),
                 r_pri=torch.zeros(S, dtype=ds.dtype, device=ds.device),
                 r_dual=torch.zeros(S, dtype=ds.dtype, device=ds.device),
                 cost=torch.zeros(S, dtype=ds.dtype, device=ds.device))
    rep = Report(rep_t["iters"].data_ptr(), rep_t["status"].data_ptr(), rep_t["r_pri"].data_ptr(),
                 rep_t["r_dual"].data_ptr(), rep_t["cost"].data_ptr())
    pr = AdmmParams(float(sigma), float(eps_pri), float(eps_dual), float(prox), int(max_iter), int(flags),
                    float(rho_box), float(damp))
    if tape is None:
        _check(lib().oca_admm_solve(ds.ctx.h, ds.h, C.byref(ds.model), C.byref(pr), _ptr(s_ref), _ptr(s), _ptr(u),
                                    _ptr(y), _ptr(zeta), _ptr(xi), C.byref(rep), _stream(stream)), "oca_admm_solve")
    else:
        _check(lib().oca_admm_solve_taped(ds.ctx.h, ds.h, C.byref(ds.model), C.byref(pr), _ptr(s_ref), _ptr(s),
                                          _ptr(u), _ptr(y), _ptr(zeta), _ptr(xi), C.byref(rep), _ptr(tape),
                                          C.c_int64(tape.numel()), _stream(stream)), "oca_admm_solve_taped")
    return rep_t


def fp64_peak(device: int = 0) -> float:
    """oca_fp64_peak: measured FP64 FMA throughput (GFLOP/s)."""
    g = C.c_double(0.0)
    _check(lib().oca_fp64_peak(int(device), C.byref(g)), "oca_fp64_peak")
    return float(g.value)


def tape_bytes(ds: DeviceScene, max_iter: int, fixed_point: bool = False) -> int:
    """oca_admm_tape_bytes (oca_admm_fixed_point_tape_bytes with fixed_point)."""
    n = C.c_int64(0)
    if fixed_point:
        _check(lib().oca_admm_fixed_point_tape_bytes(ds.h, C.byref(ds.model), C.byref(n)),
               "oca_admm_fixed_point_tape_bytes")
    else:
        _check(lib().oca_admm_tape_bytes(ds.h, C.byref(ds.model), int(max_iter), C.byref(n)), "oca_admm_tape_bytes")
    return int(n.value)


def new_tape(ds: DeviceScene, max_iter: int, fixed_point: bool = False) -> torch.Tensor:
    """A device byte tensor large enough for a taped solve of max_iter
    iterations (one iterate, any count, with fixed_point)."""
    return torch.empty(tape_bytes(ds, max_iter, fixed_point), dtype=torch.uint8, device=ds.device)


def admm_backward(ds: DeviceScene, s_ref, tape, iters, grad_cost, grad_alpha=None, sigma=300.0, prox=1.0,
                  max_iter=300, rho_box=100.0, damp=100.0, eps_pri=1e-4, eps_dual=1e-4, flags=0, stream=None):
    """oca_admm_backward: gradients of sum_s grad_cost[s] * cost_s (+ sum_p
    grad_alpha[p] * alpha*_p at the returned trajectory) of a taped solve
    w.r.t. obstacle offsets [M_tot, fo_max], obstacle translations
    [M_tot, dim] and initial states [S, ns]."""
    sc = ds.scene
    m_tot = int(sc.obs_begin[-1])
    g_d = torch.zeros(m_tot, sc.fo_max, dtype=ds.dtype, device=ds.device)
    g_c = torch.zeros(m_tot, sc.dim, dtype=ds.dtype, device=ds.device)
    g_s0 = torch.zeros(sc.n_scen, sc.model.ns, dtype=ds.dtype, device=ds.device)
    pr = AdmmParams(float(sigma), float(eps_pri), float(eps_dual), float(prox), int(max_iter), int(flags),
                    float(rho_box), float(damp))
    gc = grad_cost.to(ds.dtype).contiguous()
    ga = None if grad_alpha is None else grad_alpha.to(ds.dtype).contiguous()
    _check(lib().oca_admm_backward(ds.ctx.h, ds.h, C.byref(ds.model), C.byref(pr), _ptr(s_ref), _ptr(tape),
                                   C.c_int64(tape.numel()), _ptr(iters), _ptr(gc), _ptr(ga), _ptr(g_d), _ptr(g_c),
                                   _ptr(g_s0), _stream(stream)), "oca_admm_backward")
    return dict(obs_offset=g_d, obs_center=g_c, state0=g_s0)


class AdmmCost(torch.autograd.Function):
    """Trajectory cost per scenario (eqn:navigation_cost) after an ADMM solve,
    as a differentiable function of the obstacle offsets d [M_tot, fo_max]
    and translations delta [M_tot, dim] (the solved obstacle j has offsets
    d_jm + c_jm . delta_j).  Forward: a taped oca_admm_solve from the
    problem's current state (left unchanged) on a scene of its own that holds
    the moved offsets (the problem's scene is not touched); backward:
    oca_admm_backward on that scene."""

    @staticmethod
    def forward(ctx, obs_d, obs_shift, problem, kw):
        ds = problem.ds
        with torch.no_grad():
            d_eff = obs_d + torch.einsum("jmi,ji->jm", ds.obs_C.view(obs_d.shape[0], obs_d.shape[1], -1), obs_shift)
            dsx = ds.with_offsets(d_eff)
            st = [t.clone() for t in (problem.s, problem.u, problem.y, problem.zeta, problem.xi)]
            tape = new_tape(dsx, kw.get("max_iter", 300))
            rep = admm_solve(dsx, problem.s_ref, *st, tape=tape, **kw)
        ctx.problem, ctx.kw, ctx.tape, ctx.iters, ctx.scene = problem, kw, tape, rep["iters"], dsx
        return rep["cost"].clone()

    @staticmethod
    def backward(ctx, grad_cost):
        problem, kw = ctx.problem, ctx.kw
        with torch.no_grad():
            keys = ("sigma", "prox", "max_iter", "rho_box", "damp", "eps_pri", "eps_dual", "flags")
            g = admm_backward(ctx.scene, problem.s_ref, ctx.tape, ctx.iters, grad_cost,
                              **{k: kw[k] for k in keys if k in kw})
        return g["obs_offset"], g["obs_center"], None, None


def admm_cost(problem, obs_d, obs_shift, **kw):
    """Differentiable trajectory cost of every scenario (AdmmCost)."""
    return AdmmCost.apply(obs_d, obs_shift, problem, kw)


class Problem:
    """Device-resident ADMM state of a synthetic scene (initial guess, cold y)."""

    def __init__(self, ds: DeviceScene, s_init=None, u_init=None, y_init=None):
        sc = ds.scene
        self.ds = ds
        self.s_ref = ds.tensor(sc.s_ref)
        self.s = ds.tensor(sc.s_init if s_init is None else s_init)
        self.u = ds.tensor(sc.u_init if u_init is None else u_init)
        self.y = ds.to_device_pairs(sc.cold_y() if y_init is None else y_init)
        self.zeta = torch.zeros(ds.n_pairs, dtype=ds.dtype, device=ds.device)
        self.xi = torch.zeros(sc.dim, ds.n_pairs, dtype=ds.dtype, device=ds.device)

    def solve(self, **kw):
        return admm_solve(self.ds, self.s_ref, self.s, self.u, self.y, self.zeta, self.xi, **kw)


def mpc_run(ds: DeviceScene, ref, obs_center, x0, n_steps: int, window=(10.0, 10.0, 3.0), s_init=None, stream=None,
            **admm):
    """oca_mpc_run: the closed loop of every scenario for n_steps control
    steps from the true states x0 [S, ns], with the scene's first window as
    the first warm start.  Returns the histories, iteration counts, the
    first colliding step per scenario (-1: none) and the final arrays."""
    sc = ds.scene
    S, ns, nu = sc.n_scen, sc.model.ns, sc.model.nu
    kw = dict(DEFAULTS)
    kw.update(admm)
    pr = AdmmParams(float(kw["sigma"]), float(kw["eps_pri"]), float(kw["eps_dual"]), float(kw["prox"]),
                    int(kw["max_iter"]), int(kw.get("flags", 0)), float(kw["rho_box"]), float(kw["damp"]))
    mp = MpcParams(int(n_steps), 0, (C.c_double * 3)(*[float(w) for w in window]))
    ref_t = ds.tensor(ref)
    ctr = ds.tensor(obs_center)
    x = ds.tensor(x0)
    s_ref = ds.tensor(sc.s_ref)
    s = ds.tensor(sc.s_init if s_init is None else s_init)
    u = ds.tensor(sc.u_init)
    y = ds.to_device_pairs(sc.cold_y())
    zeta = torch.zeros(ds.n_pairs, dtype=ds.dtype, device=ds.device)
    xi = torch.zeros(sc.dim, ds.n_pairs, dtype=ds.dtype, device=ds.device)
    x_hist = torch.zeros(S, n_steps + 1, ns, dtype=ds.dtype, device=ds.device)
    u_hist = torch.zeros(S, n_steps, nu, dtype=ds.dtype, device=ds.device)
    it_hist = torch.zeros(S, n_steps, dtype=torch.int32, device=ds.device)
    coll = torch.zeros(S, dtype=torch.int32, device=ds.device)
    _check(lib().oca_mpc_run(ds.ctx.h, ds.h, C.byref(ds.model), C.byref(pr), C.byref(mp), _ptr(ref_t),
                             int(ref_t.shape[1]), _ptr(ctr), _ptr(x), _ptr(s_ref), _ptr(s), _ptr(u), _ptr(y),
                             _ptr(zeta), _ptr(xi), _ptr(x_hist), _ptr(u_hist), _ptr(it_hist), _ptr(coll),
                             _stream(stream)), "oca_mpc_run")
    return dict(x=x, x_hist=x_hist, u_hist=u_hist, iters=it_hist, collided=coll, s=s, u=u, y=y, zeta=zeta, xi=xi,
                s_ref=s_ref)
