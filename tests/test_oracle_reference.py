"""Pins for the oracle's quadrature and bases (Sec. 2.2 spaces) against closed forms."""
import math

import numpy as np
import pytest

from oracle import reference as ref


def _monomial_integral(exps):
    # int over the unit d-simplex of prod x_i^a_i = prod a_i! / (sum a_i + d)!
    d = len(exps)
    return math.prod(math.factorial(a) for a in exps) / math.factorial(sum(exps) + d)


@pytest.mark.parametrize("dim", [1, 2, 3])
@pytest.mark.parametrize("n", [1, 2, 3, 4, 6])
def test_quadrature_exact_to_degree_2n_minus_1(dim, n):
    pts, w = ref.simplex_rule(dim, n)
    deg = 2 * n - 1
    for exps in np.ndindex(*([deg + 1] * dim)):
        if sum(exps) > deg:
            continue
        approx = np.sum(w * np.prod(pts ** np.array(exps), axis=1))
        assert abs(approx - _monomial_integral(exps)) < 1e-14


@pytest.mark.parametrize("dim", [1, 2, 3])
@pytest.mark.parametrize("k", [0, 1, 2, 3, 4])
def test_basis_orthonormal(dim, k):
    pts, w = ref.simplex_rule(dim, k + 2)
    V, _ = ref.basis(dim, k, pts)
    assert V.shape[1] == ref.n_modes(dim, k)
    M = V.T @ (w[:, None] * V)
    assert np.abs(M - np.eye(V.shape[1])).max() < 1e-13


@pytest.mark.parametrize("dim", [1, 2, 3])
@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_basis_gradient_matches_finite_differences(dim, k):
    rng = np.random.default_rng(k + 10 * dim)
    p = rng.dirichlet(np.ones(dim + 1), size=7)[:, :dim]
    _, G = ref.basis(dim, k, p)
    h = 1e-6
    for r in range(dim):
        e = np.zeros(dim)
        e[r] = h
        Vp, _ = ref.basis(dim, k, p + e)
        Vm, _ = ref.basis(dim, k, p - e)
        assert np.abs((Vp - Vm) / (2 * h) - G[:, :, r]).max() < 1e-6


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_basis_spans_Pk(dim, k):
    """Every monomial of degree <= k is reproduced exactly by its projection."""
    pts, w = ref.simplex_rule(dim, k + 2)
    V, _ = ref.basis(dim, k, pts)
    rng = np.random.default_rng(3)
    test_pts = rng.dirichlet(np.ones(dim + 1), size=11)[:, :dim]
    Vt, _ = ref.basis(dim, k, test_pts)
    for exps in np.ndindex(*([k + 1] * dim)):
        if sum(exps) > k:
            continue
        f = np.prod(pts ** np.array(exps), axis=1)
        coef = V.T @ (w * f)
        ft = np.prod(test_pts ** np.array(exps), axis=1)
        assert np.abs(Vt @ coef - ft).max() < 1e-12
    # and the space has exactly dim P_k modes
    assert V.shape[1] == math.comb(k + dim, dim)
