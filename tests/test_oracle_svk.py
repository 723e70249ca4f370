"""Pins of the oracle's Saint Venant-Kirchhoff law, by facts independent of its formulas:
P is the derivative of the stored energy (central differences of psi), the tangent is the
derivative of P (central differences), P is frame-indifferent (P(QF) = Q P(F) for rotations
Q), and at small strain P reduces to the linear Cauchy stress lam tr(eps) I + 2 mu eps."""
import numpy as np
import pytest

from oracle import svk


def _F(d, seed, scale=0.3):
    return np.eye(d) + scale * np.random.default_rng(seed).standard_normal((d, d))


@pytest.mark.parametrize("d", [2, 3])
def test_first_pk_is_the_energy_derivative(d):
    lam, mu = 1.5, 1.0
    F = _F(d, 1)
    h = 1e-6
    P = svk.first_pk(F, lam, mu)
    for i in range(d):
        for J in range(d):
            dF = np.zeros((d, d))
            dF[i, J] = h
            fd = (svk.energy(F + dF, lam, mu) - svk.energy(F - dF, lam, mu)) / (2 * h)
            assert abs(fd - P[i, J]) < 1e-7 * max(1.0, abs(P[i, J]))


@pytest.mark.parametrize("d", [2, 3])
def test_tangent_is_the_derivative_of_P(d):
    lam, mu = 1.5, 1.0
    F = _F(d, 2)
    A = svk.tangent(F, lam, mu)
    h = 1e-6
    for k in range(d):
        for L in range(d):
            dF = np.zeros((d, d))
            dF[k, L] = h
            fd = (svk.first_pk(F + dF, lam, mu) - svk.first_pk(F - dF, lam, mu)).ravel() / (2 * h)
            assert np.abs(fd - A[:, k * d + L]).max() < 1e-7 * max(1.0, np.abs(A).max())


def test_frame_indifference():
    lam, mu = 1.5, 1.0
    F = _F(3, 3)
    Q, _ = np.linalg.qr(np.random.default_rng(4).standard_normal((3, 3)))
    if np.linalg.det(Q) < 0:
        Q[:, 0] = -Q[:, 0]
    assert np.abs(svk.first_pk(Q @ F, lam, mu) - Q @ svk.first_pk(F, lam, mu)).max() < 1e-13
    assert np.abs(svk.second_pk(Q @ F, lam, mu) - svk.second_pk(F, lam, mu)).max() < 1e-13


def test_small_strain_limit_is_linear_elasticity():
    lam, mu = 1.5, 1.0
    H = np.random.default_rng(5).standard_normal((3, 3))
    eps = 0.5 * (H + H.T)
    lin = lam * np.trace(eps) * np.eye(3) + 2.0 * mu * eps
    for t in (1e-3, 1e-4):
        P = svk.first_pk(np.eye(3) + t * H, lam, mu)
        assert np.abs(P / t - lin).max() < 20 * t * np.abs(lin).max()
