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


def test_plate_solution_satisfies_the_equations():
    """Central differences (not the symbolic derivatives) of the plate data: dF/dt = grad v,
    rho dv/dt - div P = f, P = P_SVK(F), and v = 0 on the clamped sides."""
    pytest.importorskip("sympy")
    lam, mu, rho = 1.5, 1.0, 1.0
    sol = svk.plate_solution(lam, mu, rho)
    rng = np.random.default_rng(6)
    x = np.column_stack([rng.uniform(0.1, 0.9, 5), rng.uniform(0.1, 0.9, 5), rng.uniform(0.0, 0.01, 5)])
    t, h = 0.37, 1e-5
    F = sol["F"](x, t).reshape(-1, 3, 3)
    dFdt = (sol["F"](x, t + h) - sol["F"](x, t - h)).reshape(-1, 3, 3) / (2 * h)
    dvdt = (sol["v"](x, t + h) - sol["v"](x, t - h)) / (2 * h)
    gradv = np.zeros_like(dFdt)
    divP = np.zeros((x.shape[0], 3))
    for J in range(3):
        e = np.zeros(3)
        e[J] = h
        gradv[:, :, J] = (sol["v"](x + e, t) - sol["v"](x - e, t)) / (2 * h)
        dP = (sol["P"](x + e, t) - sol["P"](x - e, t)).reshape(-1, 3, 3) / (2 * h)
        divP += dP[:, :, J]
    assert np.abs(dFdt - gradv).max() < 1e-6
    assert np.abs(rho * dvdt - divP - sol["f"](x, t)).max() < 1e-5
    for q in range(x.shape[0]):
        assert np.abs(sol["P"](x[q:q + 1], t).reshape(3, 3) - svk.first_pk(F[q], lam, mu)).max() < 1e-13
    sides = np.array([[0.0, 0.3, 0.005], [1.0, 0.6, 0.0], [0.4, 0.0, 0.01], [0.2, 1.0, 0.003]])
    assert np.abs(sol["v"](sides, t)).max() < 1e-15
