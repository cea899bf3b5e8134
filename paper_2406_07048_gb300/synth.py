"""Seeded synthetic scenes for the scale-based collision-avoidance ADMM.

This module only *draws inputs*: obstacle and robot H-polyhedra, reference
trajectories, initial guesses and model constants.  It holds none of the
method's arithmetic (no poses, no LP/QP, no dynamics), so both the CUDA path
and the CPU oracle may consume its output.

Geometry follows Sec. III-A / IV-A of the paper: a robot part is
``A x <= b`` in its own body frame (``b > 0``: the part's centre is interior,
which is what the centre-scaling of the scale LP needs), an obstacle is
``C y <= d`` in the world frame.  The paper's AirSim scene, its reference
trajectories and the quadrotor constants are not available; the distributions
below stand in for them (sizes, face counts, obstacle counts and horizons of
the vehicle and quadrotor workloads).

Array conventions (shared by the C-ABI and the oracle):
  obs_C   [M_tot, FO, dim]  outward unit normals c_m, world frame (pad: 0)
  obs_d   [M_tot, FO]       offsets d_m (pad: 1 -> inert 0 <= 1)
  obs_nf  [M_tot]           face counts
  obs_begin [S+1]           CSR over scenarios
  part_A  [P_tot, FR, dim]  body-frame normals a_k
  part_b  [P_tot, FR]       offsets b_k > 0
  part_nf [P_tot], part_begin [S+1]
  part_link [P_tot]         0 = vehicle body, 1 = trailer (tractor model)
  part_off  [P_tot, dim]    part centre in its link frame
  horizon [S]               N_s (constraint steps t = 1..N_s)
  s_ref  [sum(N_s+1), n_s]  reference states (t = 0..N_s)
Pairs of scenario s are enumerated p = (j * n_parts_s + part) * N_s + (t - 1)
(obstacle slowest, time fastest).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

MODEL_BICYCLE = 0
MODEL_TRAILER = 1
MODEL_QUAD = 2

MODEL_DIMS = {MODEL_BICYCLE: (4, 2, 2), MODEL_TRAILER: (5, 2, 2), MODEL_QUAD: (12, 4, 3)}


@dataclasses.dataclass
class Model:
    """Dynamics model and cost weights (constants are not given by the paper)."""
    kind: int
    dt: float
    param: np.ndarray   # bicycle: [L]; trailer: [L, M, L2]; quad: [m, g, Jx, Jy, Jz, ell, km]
    Qs: np.ndarray      # diagonal state weights (n_s)
    Qu: np.ndarray      # diagonal control weights (n_u)
    s_lo: np.ndarray = None   # state box of the MPC problem (-inf/inf: none)
    s_hi: np.ndarray = None
    u_lo: np.ndarray = None   # control box
    u_hi: np.ndarray = None

    @property
    def ns(self) -> int:
        return MODEL_DIMS[self.kind][0]

    @property
    def nu(self) -> int:
        return MODEL_DIMS[self.kind][1]

    @property
    def dim(self) -> int:
        return MODEL_DIMS[self.kind][2]


@dataclasses.dataclass
class Scene:
    dim: int
    model: Model
    obs_begin: np.ndarray
    obs_nf: np.ndarray
    obs_C: np.ndarray
    obs_d: np.ndarray
    obs_center: np.ndarray   # [M_tot, dim] the centre each obstacle was drawn around
    obs_off: np.ndarray      # [M_tot, FO] the drawn offsets (d = off + C @ centre)
    part_begin: np.ndarray
    part_nf: np.ndarray
    part_A: np.ndarray
    part_b: np.ndarray
    part_link: np.ndarray
    part_off: np.ndarray
    horizon: np.ndarray
    s_ref: np.ndarray
    s_init: np.ndarray       # initial guess, s_init[t=0] is the fixed initial state
    u_init: np.ndarray       # [sum N_s, n_u]
    name: str = ""

    # ---- sizes -------------------------------------------------------------
    @property
    def n_scen(self) -> int:
        return len(self.horizon)

    @property
    def fo_max(self) -> int:
        return self.obs_C.shape[1]

    @property
    def fr_max(self) -> int:
        return self.part_A.shape[1]

    @property
    def ny_max(self) -> int:
        return self.fr_max + self.fo_max + 1

    def n_obs(self, s: int) -> int:
        return int(self.obs_begin[s + 1] - self.obs_begin[s])

    def n_parts(self, s: int) -> int:
        return int(self.part_begin[s + 1] - self.part_begin[s])

    @property
    def state_begin(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum(self.horizon + 1)]).astype(np.int64)

    @property
    def ctrl_begin(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum(self.horizon)]).astype(np.int64)

    @property
    def pair_counts(self) -> np.ndarray:
        m = np.diff(self.obs_begin)
        p = np.diff(self.part_begin)
        return (m * p * self.horizon).astype(np.int64)

    @property
    def pair_begin(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum(self.pair_counts)]).astype(np.int64)

    @property
    def n_pairs(self) -> int:
        return int(self.pair_counts.sum())

    def pair_index(self, s: int, j: int, part: int, t: int) -> int:
        """Global pair index of (scenario s, obstacle j, part, step t in 1..N_s)."""
        n = int(self.horizon[s])
        return int(self.pair_begin[s]) + (j * self.n_parts(s) + part) * n + (t - 1)

    def cold_y(self) -> np.ndarray:
        """Cold-start y, pair-major [P, ny_max]: lambda = e_e / b_e with e the
        largest robot offset (lowest index on ties), mu = 0, gamma = 0."""
        y = np.zeros((self.n_pairs, self.ny_max))
        for s in range(self.n_scen):
            n, npt = int(self.horizon[s]), self.n_parts(s)
            for j in range(self.n_obs(s)):
                for pt in range(npt):
                    gp = int(self.part_begin[s]) + pt
                    nr = int(self.part_nf[gp])
                    bb = self.part_b[gp, :nr]
                    e = int(np.argmax(bb))
                    p0 = self.pair_index(s, j, pt, 1)
                    y[p0:p0 + n, e] = 1.0 / bb[e]
        return y


# ---------------------------------------------------------------------------
# model constants (documented readings: the paper gives none except dt, sigma)
# ---------------------------------------------------------------------------

INF = float("inf")


KAPPA_MAX = math.tan(0.6) / 2.7   # curvature of a 0.6 rad steering angle, wheelbase 2.7 m


def bicycle_model(dt: float = 0.1) -> Model:
    # controls: acceleration and path curvature kappa = tan(steer) / L;
    # speed in [0, 30] m/s, acceleration in [-6, 6] m/s^2, |steer| <= 0.6 rad
    return Model(MODEL_BICYCLE, dt, np.array([2.7]), np.array([1.0, 1.0, 0.1, 0.1]),
                 np.array([0.1, 10.0]), np.array([-INF, -INF, -INF, 0.0]), np.array([INF, INF, INF, 30.0]),
                 np.array([-6.0, -KAPPA_MAX]), np.array([6.0, KAPPA_MAX]))


def trailer_model(dt: float = 0.1) -> Model:
    # wheelbase 2.7 m, hitch 1 m behind the rear axle, hitch->trailer axle 5 m
    return Model(MODEL_TRAILER, dt, np.array([2.7, 1.0, 5.0]),
                 np.array([1.0, 1.0, 0.1, 0.1, 0.1]), np.array([0.1, 10.0]),
                 np.array([-INF, -INF, -INF, 0.0, -INF]), np.array([INF, INF, INF, 30.0, INF]),
                 np.array([-6.0, -KAPPA_MAX]), np.array([6.0, KAPPA_MAX]))


def quad_model(dt: float = 0.1) -> Model:
    # m = 1 kg, J = diag(0.01, 0.01, 0.02), arm 0.25 m, yaw-torque coeff 0.016;
    # controls are rotor thrusts relative to hover (m g / 4 each), each rotor
    # thrust within [0, 3 m g / 4]; roll and pitch within +-0.8 rad
    hover = 9.81 / 4
    return Model(MODEL_QUAD, dt, np.array([1.0, 9.81, 0.01, 0.01, 0.02, 0.25, 0.016]),
                 np.array([1.0, 1.0, 1.0, 0.1, 0.1, 0.1, 0.1, 0.1, 0.1, 0.01, 0.01, 0.01]),
                 np.array([0.05, 0.05, 0.05, 0.05]),
                 np.array([-INF] * 6 + [-0.8, -0.8] + [-INF] * 4), np.array([INF] * 6 + [0.8, 0.8] + [INF] * 4),
                 np.full(4, -hover), np.full(4, 2 * hover))


# ---------------------------------------------------------------------------
# polytopes
# ---------------------------------------------------------------------------

def box_halfspaces(half: np.ndarray):
    """Axis-aligned box |x_i| <= h_i as (A, b)."""
    dim = len(half)
    A = np.zeros((2 * dim, dim))
    b = np.zeros(2 * dim)
    for i in range(dim):
        A[2 * i, i] = 1.0
        A[2 * i + 1, i] = -1.0
        b[2 * i] = b[2 * i + 1] = half[i]
    return A, b


def random_polygon(rng: np.random.Generator, nf: int, off_lo: float, off_hi: float):
    """Convex polygon: sorted uniform normal angles, resampled until every
    angular gap is below pi (bounded); offsets uniform."""
    while True:
        ang = np.sort(rng.uniform(0.0, 2.0 * math.pi, nf))
        gaps = np.diff(np.concatenate([ang, [ang[0] + 2.0 * math.pi]]))
        if gaps.max() < math.pi - 0.05:
            break
    C = np.stack([np.cos(ang), np.sin(ang)], axis=1)
    off = rng.uniform(off_lo, off_hi, nf)
    return C, off


def random_polyhedron(rng: np.random.Generator, nf: int, off_lo: float, off_hi: float):
    """Convex polyhedron: normals uniform on the sphere, resampled until the
    origin is strictly inside their convex hull (bounded); offsets uniform."""
    from scipy.spatial import ConvexHull
    while True:
        g = rng.normal(size=(nf, 3))
        C = g / np.linalg.norm(g, axis=1, keepdims=True)
        try:
            hull = ConvexHull(C)
        except Exception:
            continue
        if np.all(hull.equations[:, -1] < -0.05):
            break
    off = rng.uniform(off_lo, off_hi, nf)
    return C, off


# ---------------------------------------------------------------------------
# scenario assembly
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class _Scen:
    obs: list            # list of (C, off, centre)
    parts: list          # list of (A, b, link, off)
    N: int
    s_ref: np.ndarray
    u_init: np.ndarray


def _assemble(model: Model, scens: List[_Scen], name: str) -> Scene:
    dim = model.dim
    fo = max(len(o[1]) for sc in scens for o in sc.obs)
    fr = max(len(p[1]) for sc in scens for p in sc.parts)
    m_tot = sum(len(sc.obs) for sc in scens)
    p_tot = sum(len(sc.parts) for sc in scens)
    obs_C = np.zeros((m_tot, fo, dim))
    obs_d = np.ones((m_tot, fo))
    obs_off = np.zeros((m_tot, fo))
    obs_nf = np.zeros(m_tot, np.int32)
    obs_center = np.zeros((m_tot, dim))
    part_A = np.zeros((p_tot, fr, dim))
    part_b = np.ones((p_tot, fr))
    part_nf = np.zeros(p_tot, np.int32)
    part_link = np.zeros(p_tot, np.int32)
    part_off = np.zeros((p_tot, dim))
    obs_begin = [0]
    part_begin = [0]
    mi = pi = 0
    for sc in scens:
        for (C, off, ctr) in sc.obs:
            k = len(off)
            obs_C[mi, :k] = C
            obs_off[mi, :k] = off
            obs_d[mi, :k] = off + C @ ctr
            obs_nf[mi] = k
            obs_center[mi] = ctr
            mi += 1
        obs_begin.append(mi)
        for (A, b, link, off) in sc.parts:
            k = len(b)
            part_A[pi, :k] = A
            part_b[pi, :k] = b
            part_nf[pi] = k
            part_link[pi] = link
            part_off[pi] = off
            pi += 1
        part_begin.append(pi)
    s_ref = np.concatenate([sc.s_ref for sc in scens], axis=0)
    u_init = np.concatenate([sc.u_init for sc in scens], axis=0)
    return Scene(dim=dim, model=model, obs_begin=np.array(obs_begin, np.int32), obs_nf=obs_nf,
                 obs_C=obs_C, obs_d=obs_d, obs_center=obs_center, obs_off=obs_off,
                 part_begin=np.array(part_begin, np.int32), part_nf=part_nf, part_A=part_A,
                 part_b=part_b, part_link=part_link, part_off=part_off,
                 horizon=np.array([sc.N for sc in scens], np.int32), s_ref=s_ref,
                 s_init=s_ref.copy(), u_init=u_init, name=name)


def _ref_2d(model: Model, N: int, x0: float, x1: float, yc: float) -> np.ndarray:
    """Straight reference at constant speed covering [x0, x1] over the horizon."""
    v = (x1 - x0) / (N * model.dt)
    ref = np.zeros((N + 1, model.ns))
    ref[:, 0] = x0 + v * model.dt * np.arange(N + 1)
    ref[:, 1] = yc
    ref[:, 3] = v
    return ref


def _place_2d(rng, n_obs, fmin, fmax, xlo, xhi, ylo, yhi, keep_out, keep_r):
    obs = []
    while len(obs) < n_obs:
        ctr = np.array([rng.uniform(xlo, xhi), rng.uniform(ylo, yhi)])
        if any(np.linalg.norm(ctr - k) < keep_r for k in keep_out):
            continue
        nf = int(rng.integers(fmin, fmax + 1))
        C, off = random_polygon(rng, nf, 0.5, 2.0)
        obs.append((C, off, ctr))
    return obs


# part geometry (documented readings)
def _bicycle_body():
    A, b = box_halfspaces(np.array([2.25, 1.0]))       # 4.5 x 2.0 m
    return (A, b, 0, np.array([1.25, 0.0]))             # centre 1.25 m ahead of rear axle


def _tractor():
    A, b = box_halfspaces(np.array([2.0, 1.0]))        # 4 x 2 m
    return (A, b, 0, np.array([1.5, 0.0]))


def _trailer():
    A, b = box_halfspaces(np.array([3.0, 1.1]))        # 6 x 2.2 m
    return (A, b, 1, np.array([-3.5, 0.0]))             # centre 3.5 m behind the hitch


def config1() -> Scene:
    """Plain method, 2D: bicycle, N=20, one 4.5x2 m rectangle, 4 obstacles of
    4-8 faces in a 40x10 m corridor, seed 0 (80 pairs per iteration)."""
    model = bicycle_model()
    rng = np.random.default_rng(0)
    N = 20
    keep = [np.array([0.0, 5.0]), np.array([40.0, 5.0])]
    obs = _place_2d(rng, 4, 4, 8, 0.0, 40.0, 0.0, 10.0, keep, 5.0)
    ref = _ref_2d(model, N, 0.0, 40.0, 5.0)
    sc = _Scen(obs, [_bicycle_body()], N, ref, np.zeros((N, model.nu)))
    return _assemble(model, [sc], "plain-2d-bicycle-N20-M4")


def config_max() -> Scene:
    """Sizes at the library's compiled-in maxima next to a minimal scenario
    (a ragged batch of two): bicycle; scenario 0 has horizon 256, a regular
    octagonal body (8 faces, inradius 1 m) and 6 obstacles of 24 faces in a
    120 x 12 m corridor; scenario 1 has horizon 3, the 4.5 x 2 m rectangle
    and 2 triangles."""
    model = bicycle_model()
    rng = np.random.default_rng(11)
    ang = 2.0 * math.pi * np.arange(8) / 8.0
    octagon = (np.stack([np.cos(ang), np.sin(ang)], 1), np.ones(8), 0, np.array([1.25, 0.0]))
    N = 256
    keep = [np.array([0.0, 6.0]), np.array([120.0, 6.0])]
    big = _Scen(_place_2d(rng, 6, 24, 24, 0.0, 120.0, 0.0, 12.0, keep, 6.0), [octagon], N,
                _ref_2d(model, N, 0.0, 120.0, 6.0), np.zeros((N, model.nu)))
    keep = [np.array([0.0, 5.0]), np.array([3.0, 5.0])]
    small = _Scen(_place_2d(rng, 2, 3, 3, 0.0, 20.0, 0.0, 10.0, keep, 5.0), [_bicycle_body()], 3,
                  _ref_2d(model, 3, 0.0, 3.0, 5.0), np.zeros((3, model.nu)))
    return _assemble(model, [big, small], "max-sizes-2d-bicycle-N256-F24-R8")


def _trailer_scen(rng, model, N, n_obs, fmin, fmax, length, width, n_parts, v_ref=10.0):
    """Obstacles over length x width; the reference runs along the centre line
    at v_ref (the horizon covers min(length, v_ref N dt) of it)."""
    reach = min(length, v_ref * N * model.dt)
    keep = [np.array([0.0, width / 2]), np.array([reach, width / 2])]
    obs = _place_2d(rng, n_obs, fmin, fmax, 0.0, length, 0.0, width, keep, 8.0)
    ref = _ref_2d(model, N, 0.0, reach, width / 2)
    parts = [_tractor(), _trailer()][:n_parts]
    return _Scen(obs, parts, N, ref, np.zeros((N, model.nu)))


def config2(seed: int = 0) -> Scene:
    """Precision form: tractor-trailer (hinge angle as 5th state), N=50,
    2 parts, 32 obstacles of 3-12 faces in 100x20 m (3,200 pairs/iter)."""
    model = trailer_model()
    rng = np.random.default_rng([2, seed])
    sc = _trailer_scen(rng, model, 50, 32, 3, 12, 100.0, 20.0, 2)
    return _assemble(model, [sc], "precision-2d-trailer-N50-M32")


def config3(n_scen: int = 2048, first: int = 0) -> Scene:
    """Batching form: independent scenarios with N ~ U[20,80], obstacle count
    ~ U[8,64], face counts ~ U[3,16], robot 1-2 rectangles (tractor[-trailer]).
    Region length 2 m per step along x (20 m/s reference), width 20 m."""
    model = trailer_model()
    scens = []
    for s in range(first, first + n_scen):
        rng = np.random.default_rng([3, s])
        N = int(rng.integers(20, 81))
        M = int(rng.integers(8, 65))
        npart = int(rng.integers(1, 3))
        scens.append(_trailer_scen(rng, model, N, M, 3, 16, 2.0 * N, 20.0, npart))
    return _assemble(model, scens, f"batch-2d-trailer-S{n_scen}")


def config5(n_scen: int = 256, first: int = 0) -> Scene:
    """Differentiation form: scenarios shaped like the precision form
    (N=50, 2 parts, 32 obstacles of 3-12 faces, 100x20 m)."""
    model = trailer_model()
    scens = []
    for s in range(first, first + n_scen):
        rng = np.random.default_rng([5, s])
        scens.append(_trailer_scen(rng, model, 50, 32, 3, 12, 100.0, 20.0, 2))
    return _assemble(model, scens, f"diff-2d-trailer-S{n_scen}")


def _quad_parts():
    body = box_halfspaces(np.array([0.15, 0.15, 0.05]))     # 0.3 x 0.3 x 0.1
    armx = box_halfspaces(np.array([0.25, 0.025, 0.025]))   # 0.5 x 0.05 x 0.05
    army = box_halfspaces(np.array([0.025, 0.25, 0.025]))
    z = np.zeros(3)
    return [(body[0], body[1], 0, z), (armx[0], armx[1], 0, z), (army[0], army[1], 0, z)]


def config4(n_scen: int = 64, first: int = 0, n_obs: int = 128, N: int = 40) -> Scene:
    """3D quadrotor: N=40, 3 boxes, 128 polyhedra of 6-20 faces in a
    20x20x5 m volume; half of them placed in pairs leaving a 0.6-1.0 m gap
    across the reference path (narrow-gap placement, a documented guess)."""
    model = quad_model()
    scens = []
    for s in range(first, first + n_scen):
        rng = np.random.default_rng([4, s])
        start = np.array([0.0, 10.0, 2.5])
        goal = np.array([20.0, 10.0, 2.5])
        obs = []
        n_pairs = n_obs // 4
        for _ in range(n_pairs):
            # a gap pair straddling a random point of the straight path
            a = rng.uniform(0.15, 0.85)
            pt = start + a * (goal - start)
            C1, o1 = random_polyhedron(rng, int(rng.integers(6, 21)), 0.3, 1.5)
            C2, o2 = random_polyhedron(rng, int(rng.integers(6, 21)), 0.3, 1.5)
            gap = rng.uniform(0.6, 1.0)
            axis = np.array([0.0, 1.0, 0.0]) if rng.uniform() < 0.5 else np.array([0.0, 0.0, 1.0])
            r1, r2 = o1.max(), o2.max()
            obs.append((C1, o1, pt + axis * (gap / 2 + r1)))
            obs.append((C2, o2, pt - axis * (gap / 2 + r2)))
        while len(obs) < n_obs:
            ctr = np.array([rng.uniform(0, 20), rng.uniform(0, 20), rng.uniform(0, 5)])
            if min(np.linalg.norm(ctr - start), np.linalg.norm(ctr - goal)) < 2.0:
                continue
            C, off = random_polyhedron(rng, int(rng.integers(6, 21)), 0.3, 1.5)
            obs.append((C, off, ctr))
        ref = np.zeros((N + 1, model.ns))
        tt = np.arange(N + 1) / N
        ref[:, 0:3] = start[None, :] + tt[:, None] * (goal - start)[None, :]
        ref[:, 3:6] = (goal - start)[None, :] / (N * model.dt)
        scens.append(_Scen(obs, _quad_parts(), N, ref, np.zeros((N, model.nu))))
    return _assemble(model, scens, f"quad-3d-S{n_scen}-M{n_obs}-N{N}")


def closed_loop(n_scen: int = 256, first: int = 0, N: int = 16, duration: float = 25.0):
    """Receding-horizon quadrotor runs shaped like the paper's simulation
    (Sec. V-B): a 70 x 20 x 6 m volume (flight along +y from (0, 0, 1) to
    (0, 70, 1)), 32 polyhedra of 6-20 faces (8 in a sparse first half, 24 in
    a dense second half), horizon N = 16, dt = 0.1 s, and a reference of
    `duration` seconds interpolated through the start, 5 random waypoints and
    the goal.  Returns (scene, ref): the scene holds the first horizon window
    (s_ref, s_init = s_ref, u_init = 0); ref[s] is scenario s's reference for
    every control step, [round(duration / dt) + N + 1][ns] (the goal, at rest,
    after the end)."""
    model = quad_model()
    T = int(round(duration / model.dt))
    scens, refs = [], []
    for s in range(first, first + n_scen):
        rng = np.random.default_rng([6, s])
        start = np.array([0.0, 0.0, 1.0])
        goal = np.array([0.0, 70.0, 1.0])
        wy = np.sort(rng.uniform(5.0, 65.0, 5))
        pts = np.vstack([start, np.stack([rng.uniform(-5, 5, 5), wy, rng.uniform(1.0, 3.0, 5)], 1), goal])
        seg = np.linalg.norm(np.diff(pts, axis=0), axis=1)
        tk = np.concatenate([[0.0], np.cumsum(seg)]) / seg.sum() * duration
        tt = np.arange(T + N + 1) * model.dt
        ref = np.zeros((T + N + 1, model.ns))
        for i in range(3):
            ref[:, i] = np.interp(tt, tk, pts[:, i])
        ref[:-1, 3:6] = np.diff(ref[:, 0:3], axis=0) / model.dt
        ref[tt >= duration, 3:6] = 0.0
        obs = []
        while len(obs) < 32:
            dense = len(obs) >= 8
            ctr = np.array([rng.uniform(-10, 10), rng.uniform(35, 68) if dense else rng.uniform(3, 35), rng.uniform(0, 6)])
            if min(np.linalg.norm(ctr - start), np.linalg.norm(ctr - goal)) < 2.5:
                continue
            C, off = random_polyhedron(rng, int(rng.integers(6, 21)), 0.3, 1.5)
            obs.append((C, off, ctr))
        scens.append(_Scen(obs, _quad_parts(), N, ref[:N + 1].copy(), np.zeros((N, model.nu))))
        refs.append(ref)
    return _assemble(model, scens, f"closed-loop-quad-S{n_scen}-N{N}"), np.stack(refs)


def subset(scene: Scene, idx) -> Scene:
    """The scenarios ``idx`` of ``scene`` as a scene of their own."""
    idx = list(idx)
    sb, cb = scene.state_begin, scene.ctrl_begin
    mb = [int(scene.obs_begin[s]) for s in idx]
    me = [int(scene.obs_begin[s + 1]) for s in idx]
    pb = [int(scene.part_begin[s]) for s in idx]
    pe = [int(scene.part_begin[s + 1]) for s in idx]
    om = np.concatenate([np.arange(a, b) for a, b in zip(mb, me)])
    pm = np.concatenate([np.arange(a, b) for a, b in zip(pb, pe)])
    sm = np.concatenate([np.arange(sb[s], sb[s + 1]) for s in idx])
    cm = np.concatenate([np.arange(cb[s], cb[s + 1]) for s in idx])
    return Scene(dim=scene.dim, model=scene.model,
                 obs_begin=np.concatenate([[0], np.cumsum([b - a for a, b in zip(mb, me)])]).astype(np.int32),
                 obs_nf=scene.obs_nf[om], obs_C=scene.obs_C[om], obs_d=scene.obs_d[om],
                 obs_center=scene.obs_center[om], obs_off=scene.obs_off[om],
                 part_begin=np.concatenate([[0], np.cumsum([b - a for a, b in zip(pb, pe)])]).astype(np.int32),
                 part_nf=scene.part_nf[pm], part_A=scene.part_A[pm], part_b=scene.part_b[pm],
                 part_link=scene.part_link[pm], part_off=scene.part_off[pm],
                 horizon=scene.horizon[idx], s_ref=scene.s_ref[sm], s_init=scene.s_init[sm],
                 u_init=scene.u_init[cm], name=scene.name + "-subset")


def random_states(scene: Scene, rng: np.random.Generator, pos_sigma: float = 1.0,
                  ang_sigma: float = 0.3) -> np.ndarray:
    """Reference states perturbed by Gaussian noise (positions and angles),
    for step-level tests that need poses away from the reference."""
    s = scene.s_ref.copy()
    m = scene.model
    if m.kind in (MODEL_BICYCLE, MODEL_TRAILER):
        s[:, 0:2] += rng.normal(0, pos_sigma, (len(s), 2))
        s[:, 2] += rng.normal(0, ang_sigma, len(s))
        if m.kind == MODEL_TRAILER:
            s[:, 4] = s[:, 2] + rng.normal(0, ang_sigma, len(s))
    else:
        s[:, 0:3] += rng.normal(0, pos_sigma, (len(s), 3))
        s[:, 6:9] += rng.normal(0, ang_sigma, (len(s), 3))
    return s
