"""FP64 CPU oracle of the scale-based collision-avoidance ADMM (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The arithmetic lives in
``oca_oracle.c`` (plain C, FP64); this file compiles it with gcc, marshals
numpy arrays, and composes the closed loop (``mpc_run``) from those routines.
It shares nothing with the CUDA path.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oca_oracle.c")
_LIB = os.path.join(_HERE, "liboca_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", "-o", _LIB + ".tmp",
               _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class OraModel(C.Structure):
    _fields_ = [("kind", C.c_int), ("dt", C.c_double), ("param", C.c_double * 8),
                ("Qs", C.c_double * 12), ("Qu", C.c_double * 4), ("s_lo", C.c_double * 12),
                ("s_hi", C.c_double * 12), ("u_lo", C.c_double * 4), ("u_hi", C.c_double * 4)]


class OraScene(C.Structure):
    _fields_ = [("dim", C.c_int), ("n_scen", C.c_int), ("fo_max", C.c_int), ("fr_max", C.c_int),
                ("obs_begin", C.c_void_p), ("obs_nf", C.c_void_p), ("obs_C", C.c_void_p),
                ("obs_d", C.c_void_p), ("part_begin", C.c_void_p), ("part_nf", C.c_void_p),
                ("part_link", C.c_void_p), ("part_A", C.c_void_p), ("part_b", C.c_void_p),
                ("part_off", C.c_void_p), ("horizon", C.c_void_p)]


class OraParams(C.Structure):
    _fields_ = [("sigma", C.c_double), ("eps_pri", C.c_double), ("eps_dual", C.c_double),
                ("prox", C.c_double), ("max_iter", C.c_int), ("jacobi", C.c_int),
                ("rho_box", C.c_double), ("damp", C.c_double)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            P, I, D = C.c_void_p, C.c_int, C.c_double
            _lib.ora_scale_lp.argtypes = [I, I, P, P, I, P, P, P, P, P, P]
            _lib.ora_pair_qp.argtypes = [I, I, P, P, I, P, P, P, D, P, P, P, P, P]
            _lib.ora_dynamics.argtypes = [P, P, P, P, P, P]
            _lib.ora_part_pose.argtypes = [P, I, P, P, P, P, P, P]
            _lib.ora_riccati.argtypes = [I, I, I, P, P, P, P, P, P, P, P, P, P]
            _lib.ora_riccati_scan.argtypes = [I, I, I, P, P, P, P, P, P, P, P, P, P, P, P, I]
            _lib.ora_cert_margin.argtypes = [I, I, P, P, I, P, P, P, P]
            _lib.ora_cert_margin.restype = D
            _lib.ora_scale_batch.argtypes = [P, P, P, P, P, C.c_longlong, P, P, P, P, P, P, P, I]
            _lib.ora_pair_qp_batch.argtypes = [P, P, P, P, P, P, P, D, C.c_longlong, P, P, P, P, P,
                                               P, I]
            _lib.ora_admm_batch.argtypes = [P, P, P, P, P, P, P, P, P, P, P, P, I, P, P, P, I]
            _lib.ora_admm_scenario.argtypes = [P, P, I, P, P, P, P, P, P, P, P]
            _lib.ora_pair_gn.argtypes = [P, I, I, P, I, P, P, P, P, P, P, P, I, I, D, P, P, P]
            _lib.ora_num_threads.restype = I
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _i64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


def make_model(m) -> OraModel:
    om = OraModel()
    om.kind = int(m.kind)
    om.dt = float(m.dt)
    for i, v in enumerate(m.param):
        om.param[i] = float(v)
    for i, v in enumerate(m.Qs):
        om.Qs[i] = float(v)
    for i, v in enumerate(m.Qu):
        om.Qu[i] = float(v)
    for i in range(12):
        om.s_lo[i], om.s_hi[i] = -1e30, 1e30
    for i in range(4):
        om.u_lo[i], om.u_hi[i] = -1e30, 1e30
    clip = lambda v: float(min(max(v, -1e30), 1e30))
    for name in ("s_lo", "s_hi", "u_lo", "u_hi"):
        arr = getattr(m, name, None)
        if arr is not None:
            for i, v in enumerate(arr):
                getattr(om, name)[i] = clip(v)
    return om


class _SceneRef:
    """Keeps the numpy buffers of an OraScene alive."""

    def __init__(self, scene):
        self.keep = dict(obs_begin=_i32(scene.obs_begin), obs_nf=_i32(scene.obs_nf),
                         obs_C=_f64(scene.obs_C), obs_d=_f64(scene.obs_d),
                         part_begin=_i32(scene.part_begin), part_nf=_i32(scene.part_nf),
                         part_link=_i32(scene.part_link), part_A=_f64(scene.part_A),
                         part_b=_f64(scene.part_b), part_off=_f64(scene.part_off),
                         horizon=_i32(scene.horizon))
        s = OraScene()
        s.dim, s.n_scen, s.fo_max, s.fr_max = scene.dim, scene.n_scen, scene.fo_max, scene.fr_max
        for k, v in self.keep.items():
            setattr(s, k, v.ctypes.data)
        self.c = s
        self.model = make_model(scene.model)
        self.pair_begin = _i64(scene.pair_begin)
        self.state_begin = _i64(scene.state_begin)
        self.ctrl_begin = _i64(scene.ctrl_begin)


# ---------------------------------------------------------------------------
# single-problem entry points
# ---------------------------------------------------------------------------

def scale_lp(A, b, Cb, db):
    """alpha*, lambda*, mu*, x* of eqn:scale_opt in the body frame of the part."""
    A, b, Cb, db = _f64(A), _f64(b), _f64(Cb), _f64(db)
    d = A.shape[1]
    lam = np.zeros(len(b))
    mu = np.zeros(len(db))
    x = np.zeros(d)
    al = np.zeros(1)
    st = lib().ora_scale_lp(d, len(b), _p(A), _p(b), len(db), _p(Cb), _p(db), _p(al), _p(lam),
                            _p(mu), _p(x))
    return float(al[0]), lam, mu, x, st


def pair_qp(A, b, Cb, db, bq, prox: float = 0.0, ybar=None):
    """y*, v* = K^T y* + bq, obj = 0.5|v*|^2 of eqn:const_least_square (compact y)."""
    A, b, Cb, db, bq = _f64(A), _f64(b), _f64(Cb), _f64(db), _f64(bq)
    d = A.shape[1]
    ny = len(b) + len(db) + 1
    yb = _f64(np.zeros(ny) if ybar is None else ybar)
    y = np.zeros(ny)
    v = np.zeros(d + 1)
    obj = np.zeros(1)
    npiv = np.zeros(1, np.int32)
    st = lib().ora_pair_qp(d, len(b), _p(A), _p(b), len(db), _p(Cb), _p(db), _p(bq), float(prox),
                           _p(yb), _p(y), _p(v), _p(obj), _p(npiv))
    return y, v, float(obj[0]), st


def dynamics(model, s, u):
    """f_c(s,u), df/ds, df/du (continuous time; s_{t+1} = s_t + dt f_c)."""
    m = make_model(model)
    s, u = _f64(s), _f64(u)
    ns, nu = len(s), len(u)
    f = np.zeros(ns)
    fs = np.zeros((ns, ns))
    fu = np.zeros((ns, nu))
    lib().ora_dynamics(C.byref(m), _p(s), _p(u), _p(f), _p(fs), _p(fu))
    return f, fs, fu


def part_pose(model, link: int, off, s):
    """rho, R, drho/ds, dR/ds of a robot part."""
    m = make_model(model)
    s, off = _f64(s), _f64(off)
    d = model.dim
    ns = len(s)
    rho = np.zeros(d)
    R = np.zeros((d, d))
    drho = np.zeros((d, ns))
    dR = np.zeros((ns, d, d))
    lib().ora_part_pose(C.byref(m), int(link), _p(off), _p(s), _p(rho), _p(R), _p(drho), _p(dR))
    return rho, R, drho, dR


def riccati(A, B, c, Q, q, R, r, s0):
    A, B, c, Q, q, R, r, s0 = map(_f64, (A, B, c, Q, q, R, r, s0))
    N, ns, nu = B.shape[0], B.shape[1], B.shape[2]
    s = np.zeros((N + 1, ns))
    u = np.zeros((N, nu))
    st = lib().ora_riccati(ns, nu, N, _p(A), _p(B), _p(c), _p(Q), _p(q), _p(R), _p(r), _p(s0),
                           _p(s), _p(u))
    return s, u, st


def riccati_scan(A, B, c, Q, q, R, r, s0, tree: bool = True):
    """The same LQ problem as riccati(), by associative composition of its
    stage relations (tree: log N rounds of pairwise compositions; else right
    to left).  Returns s, u, the value functions P [N+1][ns][ns], p [N+1][ns]
    and the status."""
    A, B, c, Q, q, R, r, s0 = map(_f64, (A, B, c, Q, q, R, r, s0))
    N, ns, nu = B.shape[0], B.shape[1], B.shape[2]
    s = np.zeros((N + 1, ns))
    u = np.zeros((N, nu))
    P = np.zeros((N + 1, ns, ns))
    p = np.zeros((N + 1, ns))
    st = lib().ora_riccati_scan(ns, nu, N, _p(A), _p(B), _p(c), _p(Q), _p(q), _p(R), _p(r), _p(s0),
                                _p(s), _p(u), _p(P), _p(p), int(bool(tree)))
    return s, u, P, p, st


def pair_gn(model, A, Cw, dd, link, off, s, y_pad, fr_max, fo_max, zeta, xi):
    """r0 = [T + zeta; R + xi] of one pair at state s and its Jacobian dr/ds
    (Cw, dd: the obstacle's world-frame halfspaces)."""
    m = make_model(model)
    A, Cw, dd, off, s, y_pad, xi = map(_f64, (A, Cw, dd, off, s, y_pad, xi))
    d = A.shape[1]
    ns = len(s)
    rho = np.zeros(d)
    R = np.zeros((d, d))
    drho = np.zeros((d, ns))
    dR = np.zeros((ns, d, d))
    lib().ora_part_pose(C.byref(m), int(link), _p(off), _p(s), _p(rho), _p(R), _p(drho), _p(dR))
    r0 = np.zeros(d + 1)
    J = np.zeros((d + 1, ns))
    lib().ora_pair_gn(C.byref(m), d, A.shape[0], _p(A), len(dd), _p(Cw), _p(dd), _p(rho), _p(R),
                      _p(drho), _p(dR), _p(y_pad), int(fr_max), int(fo_max), float(zeta), _p(xi),
                      _p(r0), _p(J))
    return r0, J


def cert_margin(A, b, Cb, db, lam, mu):
    A, b, Cb, db, lam, mu = map(_f64, (A, b, Cb, db, lam, mu))
    return float(lib().ora_cert_margin(A.shape[1], len(b), _p(A), _p(b), len(db), _p(Cb), _p(db),
                                       _p(lam), _p(mu)))


# ---------------------------------------------------------------------------
# batch entry points over a synthetic scene
# ---------------------------------------------------------------------------

def scale_batch(scene, states, pairs=None, nthreads: int = 0):
    """alpha*, lambda*, mu*, x*, certificate margin and status for listed pairs."""
    sr = _SceneRef(scene)
    pl = _i64(np.arange(scene.n_pairs) if pairs is None else pairs)
    n = len(pl)
    st_arr = _f64(states)
    alpha = np.zeros(n)
    lam = np.zeros((n, scene.fr_max))
    mu = np.zeros((n, scene.fo_max))
    x = np.zeros((n, scene.dim))
    margin = np.zeros(n)
    status = np.zeros(n, np.int32)
    lib().ora_scale_batch(C.byref(sr.model), C.byref(sr.c), _p(sr.pair_begin), _p(sr.state_begin),
                          _p(st_arr), n, _p(pl), _p(alpha), _p(lam), _p(mu), _p(x), _p(margin),
                          _p(status), int(nthreads))
    return dict(alpha=alpha, lam=lam, mu=mu, x=x, margin=margin, status=status)


def pair_qp_batch(scene, states, zeta, xi, y_in, prox: float = 0.0, pairs=None, nthreads: int = 0):
    """Pair QPs for listed pairs; y_in is pair-major [len(pairs), ny_max]."""
    sr = _SceneRef(scene)
    pl = _i64(np.arange(scene.n_pairs) if pairs is None else pairs)
    n = len(pl)
    st_arr, z, x, yi = _f64(states), _f64(zeta), _f64(xi), _f64(y_in)
    y_out = np.zeros((n, scene.ny_max))
    v = np.zeros((n, scene.dim + 1))
    obj = np.zeros(n)
    status = np.zeros(n, np.int32)
    lib().ora_pair_qp_batch(C.byref(sr.model), C.byref(sr.c), _p(sr.pair_begin), _p(sr.state_begin),
                            _p(st_arr), _p(z), _p(x), float(prox), n, _p(pl), _p(yi), _p(y_out), _p(v),
                            _p(obj), _p(status), int(nthreads))
    return dict(y=y_out, v=v, obj=obj, status=status)


def admm_batch(scene, sigma=300.0, eps_pri=1e-4, eps_dual=1e-4, prox=1.0, max_iter=300,
               jacobi=False, scenarios=None, s=None, u=None, y=None, zeta=None, xi=None,
               nthreads: int = 0, rho_box=100.0, damp=100.0):
    """Whole ADMM solves; returns the updated state arrays and the report."""
    sr = _SceneRef(scene)
    pr = OraParams(float(sigma), float(eps_pri), float(eps_dual), float(prox), int(max_iter),
                   int(bool(jacobi)), float(rho_box), float(damp))
    sl = _i32(np.arange(scene.n_scen) if scenarios is None else scenarios)
    s = _f64(scene.s_init if s is None else s).copy()
    u = _f64(scene.u_init if u is None else u).copy()
    y = _f64(scene.cold_y() if y is None else y).copy()
    zeta = _f64(np.zeros(scene.n_pairs) if zeta is None else zeta).copy()
    xi = _f64(np.zeros((scene.n_pairs, scene.dim)) if xi is None else xi).copy()
    report = np.zeros((scene.n_scen, 4))
    status = np.full(scene.n_scen, -1, np.int32)
    s_ref = _f64(scene.s_ref)
    lib().ora_admm_batch(C.byref(sr.model), C.byref(sr.c), C.byref(pr), _p(sr.pair_begin),
                         _p(sr.state_begin), _p(sr.ctrl_begin), _p(s_ref), _p(s), _p(u), _p(y),
                         _p(zeta), _p(xi), len(sl), _p(sl), _p(report), _p(status), int(nthreads))
    return dict(s=s, u=u, y=y, zeta=zeta, xi=xi, iters=report[:, 0].astype(int),
                r_pri=report[:, 1], r_dual=report[:, 2], cost=report[:, 3], status=status)


def num_threads() -> int:
    return int(lib().ora_num_threads())


# ---------------------------------------------------------------------------
# closed-loop receding-horizon control (Sec. V-B), composed from the routines
# above; kept in Python because it is bookkeeping around them
# ---------------------------------------------------------------------------

def _sensed_subscene(scene, keep):
    """The scene restricted to the obstacles with keep[j] (scenario structure,
    parts and states unchanged) and, for every scenario, the indices of its
    kept pairs in the full scene (obstacle-major blocks, kept in order)."""
    import dataclasses
    keep = np.asarray(keep, bool)
    ob = np.asarray(scene.obs_begin)
    counts = [int(keep[ob[s]:ob[s + 1]].sum()) for s in range(scene.n_scen)]
    sub = dataclasses.replace(scene, obs_C=scene.obs_C[keep], obs_d=scene.obs_d[keep], obs_nf=scene.obs_nf[keep],
                              obs_center=scene.obs_center[keep], obs_off=scene.obs_off[keep],
                              obs_begin=np.concatenate([[0], np.cumsum(counts)]).astype(np.int32))
    idx = []
    for s in range(scene.n_scen):
        N, NP = int(scene.horizon[s]), scene.n_parts(s)
        for j in range(scene.n_obs(s)):
            if keep[ob[s] + j]:
                p0 = int(scene.pair_begin[s]) + j * NP * N
                idx.append(np.arange(p0, p0 + NP * N))
    idx = np.concatenate(idx) if idx else np.zeros(0, np.int64)
    return sub, idx


def mpc_run(scene, ref, x0, n_steps, window=(10.0, 10.0, 3.0), s_init=None, nthreads: int = 0, **admm):
    """The closed loop of every scenario (same steps as the GPU's
    oca_mpc_run): per control step the horizon window of the reference, the
    warm start shifted one step, s_0 = the true state, the ADMM over the
    sensed obstacles only (admm_batch on the sub-scene; the other pairs keep
    y, zeta, xi), the plant x += dt f_c(x, u_0) with u_0 clipped to the
    control box, and the collision test alpha* < 1 against every obstacle."""
    sc = scene
    S, ns, nu, d = sc.n_scen, sc.model.ns, sc.model.nu, sc.dim
    ref = np.asarray(ref, np.float64)
    T_ref = ref.shape[1]
    s = np.array(sc.s_init if s_init is None else s_init, np.float64)
    u = np.array(sc.u_init, np.float64)
    s_ref = np.array(sc.s_ref, np.float64)
    y = sc.cold_y().astype(np.float64)
    zeta = np.zeros(sc.n_pairs)
    xi = np.zeros((sc.n_pairs, d))
    x = np.array(x0, np.float64)
    x_hist = np.zeros((S, n_steps + 1, ns))
    u_hist = np.zeros((S, n_steps, nu))
    it_hist = np.zeros((S, n_steps), np.int32)
    collided = np.full(S, -1, np.int32)
    x_hist[:, 0] = x
    win = np.asarray(window, np.float64)
    for c in range(n_steps):
        keep = np.zeros(len(sc.obs_nf), bool)
        for si in range(S):
            N, a, b = int(sc.horizon[si]), int(sc.state_begin[si]), int(sc.ctrl_begin[si])
            for t in range(N + 1):
                s_ref[a + t] = ref[si, min(c + t, T_ref - 1)]
            if c > 0:
                s[a + 1:a + N] = s[a + 2:a + N + 1].copy()
                u[b:b + N - 1] = u[b + 1:b + N].copy()
                NP = sc.n_parts(si)
                for blk in range(sc.n_obs(si) * NP):
                    p0 = int(sc.pair_begin[si]) + blk * N
                    y[p0:p0 + N - 1] = y[p0 + 1:p0 + N].copy()
                    zeta[p0:p0 + N - 1] = zeta[p0 + 1:p0 + N].copy()
                    xi[p0:p0 + N - 1] = xi[p0 + 1:p0 + N].copy()
            s[a] = x[si]
            for j in range(sc.n_obs(si)):
                gm = int(sc.obs_begin[si]) + j
                inside = True
                for i in range(d):
                    if win[i] > 0:
                        inside &= abs(sc.obs_center[gm, i] - x[si, i]) <= win[i]
                keep[gm] = inside
        sub, idx = _sensed_subscene(sc, keep)
        import dataclasses
        sub = dataclasses.replace(sub, s_ref=s_ref.copy())
        r = admm_batch(sub, s=s, u=u, y=y[idx], zeta=zeta[idx], xi=xi[idx], nthreads=nthreads, **admm)
        y[idx], zeta[idx], xi[idx] = r["y"], r["zeta"], r["xi"]
        s, u = r["s"], r["u"]
        it_hist[:, c] = r["iters"]
        m = sc.model
        for si in range(S):
            b = int(sc.ctrl_begin[si])
            u0 = np.where(np.isfinite(u[b]), u[b], 0.0)
            u0 = np.minimum(np.maximum(u0, m.u_lo), m.u_hi)
            f = dynamics(m, x[si], u0)[0]
            x[si] = x[si] + m.dt * f
            u_hist[si, c] = u0
            x_hist[si, c + 1] = x[si]
            for part in range(sc.n_parts(si)):
                gp = int(sc.part_begin[si]) + part
                rho, R, _, _ = part_pose(m, int(sc.part_link[gp]), sc.part_off[gp], x[si])
                nr = int(sc.part_nf[gp])
                for j in range(sc.n_obs(si)):
                    gm = int(sc.obs_begin[si]) + j
                    nf = int(sc.obs_nf[gm])
                    Cw, dw = sc.obs_C[gm, :nf], sc.obs_d[gm, :nf]
                    al = scale_lp(sc.part_A[gp, :nr], sc.part_b[gp, :nr], Cw @ R, dw - Cw @ rho)[0]
                    if al < 1.0 and collided[si] < 0:
                        collided[si] = c + 1
    return dict(x=x, x_hist=x_hist, u_hist=u_hist, iters=it_hist, collided=collided, s=s, u=u, y=y, zeta=zeta,
                xi=xi, s_ref=s_ref)
