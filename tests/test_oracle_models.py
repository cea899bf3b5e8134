"""Pins of the oracle's dynamics (Sec. IV-A eqn:system_eqn) and part poses."""
import math

import numpy as np
import pytest

from paper_2406_07048_gb300 import synth

MODELS = [synth.bicycle_model(), synth.trailer_model(), synth.quad_model()]


def _rand_su(rng, m):
    s = rng.normal(0, 0.5, m.ns)
    s[3] = rng.uniform(1, 10) if m.kind != 2 else s[3]
    u = rng.normal(0, 0.3, m.nu)
    return s, u


@pytest.mark.parametrize("m", MODELS, ids=["bicycle", "trailer", "quad"])
def test_dynamics_jacobians_central_differences(ora, m):
    rng = np.random.default_rng(m.kind)
    h = 1e-6
    for _ in range(20):
        s, u = _rand_su(rng, m)
        f, fs, fu = ora.dynamics(m, s, u)
        for a in range(m.ns):
            e = np.zeros(m.ns)
            e[a] = h
            fd = (ora.dynamics(m, s + e, u)[0] - ora.dynamics(m, s - e, u)[0]) / (2 * h)
            assert np.abs(fd - fs[:, a]).max() < 1e-6 * (1 + np.abs(fd).max())
        for a in range(m.nu):
            e = np.zeros(m.nu)
            e[a] = h
            fd = (ora.dynamics(m, s, u + e)[0] - ora.dynamics(m, s, u - e)[0]) / (2 * h)
            assert np.abs(fd - fu[:, a]).max() < 1e-6 * (1 + np.abs(fd).max())


def test_bicycle_closed_forms(ora):
    m = synth.bicycle_model()
    f = ora.dynamics(m, [1.0, 2.0, 0.0, 5.0], [0.7, 0.0])[0]
    assert np.allclose(f, [5.0, 0.0, 0.0, 0.7])
    # yaw rate of a kinematic bicycle: v * kappa with kappa = tan(steer) / L
    kap = math.tan(0.2) / 2.7
    f = ora.dynamics(m, [0, 0, math.pi / 2, 4.0], [0, kap])[0]
    assert np.allclose(f, [0.0, 4.0, 4.0 * kap, 0.0], atol=1e-12)
    # constant curvature and speed: the Euler steps stay on a circle of radius 1/kappa to O(dt^2)
    s = np.array([0.0, 0.0, 0.0, 5.0])
    for _ in range(200):
        s = s + 1e-3 * ora.dynamics(m, s, [0.0, 0.25])[0]
    assert np.hypot(s[0], s[1] - 4.0) == pytest.approx(4.0, abs=2e-3)


def test_trailer_closed_forms(ora):
    m = synth.trailer_model()
    # aligned, no steering: the trailer heading is steady
    assert ora.dynamics(m, [0, 0, 0.3, 5.0, 0.3], [0, 0])[0][4] == pytest.approx(0.0, abs=1e-14)
    # tractor turned left of the trailer: trailer swings left at v sin(th-psi)/L2
    f = ora.dynamics(m, [0, 0, 0.2, 5.0, 0.0], [0, 0])[0]
    assert f[4] == pytest.approx(5.0 * math.sin(0.2) / 5.0)


def test_quad_closed_forms(ora):
    m = synth.quad_model()
    s = np.zeros(12)
    f = ora.dynamics(m, s, np.zeros(4))[0]
    assert np.abs(f).max() < 1e-14                       # hover is an equilibrium
    s[6:9] = [0.1, 0.0, 0.0]                             # roll right: thrust tilts to -y
    f = ora.dynamics(m, s, np.zeros(4))[0]
    assert f[4] == pytest.approx(-9.81 * math.sin(0.1)) and f[3] == pytest.approx(0.0, abs=1e-14)
    s = np.zeros(12)
    s[9:12] = [0.3, -0.2, 0.5]                           # Euler rates equal body rates at 0
    f = ora.dynamics(m, s, np.zeros(4))[0]
    assert np.allclose(f[6:9], [0.3, -0.2, 0.5])
    f = ora.dynamics(m, np.zeros(12), [0, 1.0, 0, 0])[0]  # +y rotor: +x torque, -z yaw torque
    assert f[9] == pytest.approx(0.25 / 0.01) and f[11] == pytest.approx(-0.016 / 0.02)


@pytest.mark.parametrize("m,link,off", [
    (synth.bicycle_model(), 0, [1.25, 0.0]),
    (synth.trailer_model(), 0, [1.5, 0.0]),
    (synth.trailer_model(), 1, [-3.5, 0.0]),
    (synth.quad_model(), 0, [0.1, -0.05, 0.02]),
], ids=["bicycle", "tractor", "trailer", "quad"])
def test_pose_derivatives_and_rotation(ora, m, link, off):
    rng = np.random.default_rng(4)
    h = 1e-6
    for _ in range(10):
        s, _ = _rand_su(rng, m)
        rho, R, drho, dR = ora.part_pose(m, link, off, s)
        assert np.allclose(R @ R.T, np.eye(m.dim), atol=1e-13)
        assert np.linalg.det(R) == pytest.approx(1.0)
        for a in range(m.ns):
            e = np.zeros(m.ns)
            e[a] = h
            p1, R1, _, _ = ora.part_pose(m, link, off, s + e)
            p0, R0, _, _ = ora.part_pose(m, link, off, s - e)
            assert np.abs((p1 - p0) / (2 * h) - drho[:, a]).max() < 1e-7
            assert np.abs((R1 - R0) / (2 * h) - dR[a]).max() < 1e-7


def test_pose_closed_forms(ora):
    m = synth.trailer_model()
    s = np.array([10.0, 5.0, math.pi / 2, 3.0, math.pi / 2])
    rho, R, _, _ = ora.part_pose(m, 0, [1.5, 0.0], s)
    assert np.allclose(rho, [10.0, 6.5])
    # straight-aligned trailer: hitch 1 m behind the axle, centre 3.5 m further
    rho, R, _, _ = ora.part_pose(m, 1, [-3.5, 0.0], s)
    assert np.allclose(rho, [10.0, 0.5])
    s[4] = 0.0                                           # trailer at right angle, pointing +x
    rho, R, _, _ = ora.part_pose(m, 1, [-3.5, 0.0], s)
    assert np.allclose(rho, [10.0 - 3.5, 4.0])
    q = synth.quad_model()
    s = np.zeros(12)
    s[0:3] = [1, 2, 3]
    s[8] = math.pi / 2                                   # yaw 90 deg
    rho, R, _, _ = ora.part_pose(q, 0, [1.0, 0, 0], s)
    assert np.allclose(rho, [1, 3, 3])
