"""Pins of the oracle's pair QP (Sec. IV-C eqn:const_least_square) solved by
the paper's route (elimination, KKT -> LCP, Lemke)."""
import numpy as np
import pytest

from tests import _pins


@pytest.mark.parametrize("dim", [2, 3])
def test_qp_matches_support_enumeration(ora, dim):
    """prox = 0: the optimum equals the best affine minimiser over all
    supports of at most dim+2 generators (brute force, n_y <= 11)."""
    rng = np.random.default_rng(100 + dim)
    for _ in range(40):
        if dim == 2:
            A, b, C, d = _pins.random_pair(rng, 2, nf_obs=int(rng.integers(3, 6)))
        else:
            A, b, C, d = _pins.random_pair(rng, 3, nf_obs=4)
        bq = np.concatenate([[1.0 + rng.normal(0, 0.5)], rng.normal(0, 0.5, dim)])
        y, v, obj, st = ora.pair_qp(A, b, C, d, bq)
        assert st == 0
        K, kappa = _pins.build_K(A, b, C, d)
        ref, vref = _pins.qp_brute_prox0(K, kappa, bq)
        assert obj == pytest.approx(ref, rel=1e-9, abs=1e-11)
        # v* is unique (strictly convex in v)
        assert np.abs(v - vref).max() < 1e-6
        assert np.abs(K.T @ y + bq - v).max() < 1e-10


@pytest.mark.parametrize("dim", [2, 3])
def test_qp_kkt(ora, dim):
    rng = np.random.default_rng(7 + dim)
    for _ in range(100):
        A, b, C, d = _pins.random_pair(rng, dim)
        bq = np.concatenate([[1.0 + rng.normal(0, 1.0)], rng.normal(0, 1.0, dim)])
        y, v, obj, st = ora.pair_qp(A, b, C, d, bq)
        assert st == 0
        K, kappa = _pins.build_K(A, b, C, d)
        assert _pins.qp_kkt_residual(K, kappa, bq, y) < 1e-8


@pytest.mark.parametrize("dim", [2, 3])
def test_qp_prox_matches_face_enumeration(ora, dim):
    """prox > 0 (strictly convex, unique y*): equals the best face minimiser."""
    rng = np.random.default_rng(300 + dim)
    for _ in range(30):
        A, b, C, d = _pins.random_pair(rng, dim, nf_obs=4 if dim == 2 else 4)
        K, kappa = _pins.build_K(A, b, C, d)
        bq = np.concatenate([[1.0 + rng.normal(0, 0.5)], rng.normal(0, 0.5, dim)])
        ybar = np.abs(rng.normal(0, 0.3, len(kappa)))
        ybar[: len(b)] /= b @ ybar[: len(b)]
        prox = float(rng.choice([1e-3, 1e-2, 1e-1]))
        y, v, obj, st = ora.pair_qp(A, b, C, d, bq, prox=prox, ybar=ybar)
        assert st == 0
        ref, yref = _pins.qp_brute_prox(K, kappa, bq, prox, ybar)
        assert np.abs(y - yref).max() < 1e-8
        assert _pins.qp_kkt_residual(K, kappa, bq, y, prox, ybar) < 1e-8


@pytest.mark.parametrize("dim", [2, 3])
def test_zero_residual_iff_collision_free(ora, dim):
    """zeta = xi = 0: the pair QP reaches 0 exactly when a dual certificate
    with -d^T mu >= 1 exists, i.e. alpha* >= 1 (eqn:poly_colli_free_conts)."""
    rng = np.random.default_rng(55 + dim)
    n = 0
    for _ in range(200):
        A, b, C, d = _pins.random_pair(rng, dim)
        al = ora.scale_lp(A, b, C, d)[0]
        if abs(al - 1.0) < 1e-6:
            continue
        y, v, obj, st = ora.pair_qp(A, b, C, d, np.eye(dim + 1)[0])
        assert (obj < 1e-16) == (al >= 1.0), (al, obj)
        n += 1
    assert n > 150


def test_lp_certificate_is_qp_zero(ora):
    """(lambda*, mu*) of the LP with gamma = alpha* - 1 zeroes T and R
    (Sec. IV-A) when alpha* >= 1: the two oracle routines agree."""
    rng = np.random.default_rng(77)
    for _ in range(60):
        A, b, C, d = _pins.random_pair(rng, 2)
        al, lam, mu, x, st = ora.scale_lp(A, b, C, d)
        if al < 1:
            continue
        K, kappa = _pins.build_K(A, b, C, d)
        y = np.concatenate([lam, mu, [al - 1.0]])
        assert np.abs(K.T @ y + np.eye(3)[0]).max() < 1e-9
