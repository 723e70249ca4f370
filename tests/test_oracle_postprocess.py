"""Pins of the oracle's element-local post-processing p* in P_{k+1} (acoustic).

The post-processing is the local Neumann problem (grad p*, grad w)_K = (q_h, grad w)_K,
(p*, 1)_K = (p_h, 1)_K, with q_h the discrete gradient of the local momentum equation.
It is pinned by facts that do not restate it:
  * exactness: for a polynomial P of degree k + 1, projected data (p_h = volume L2
    projection onto P_k, p_hat_h = face L2 projection) give back p* = P exactly. A dropped
    face term, a wrong normal sign, a transposed derivative table or a lost mean condition
    each break it;
  * the element means of p* and p_h agree for arbitrary data;
  * superconvergence on the exact standing mode: p* converges one order faster than p_h.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import acoustic as ac
from oracle import reference as ref
from paper_1807_00086_gb300 import inputs


def _mesh(dim, N):
    return inputs.unit_square_tri(N) if dim == 2 else inputs.unit_cube_tet(N)


def _poly(dim, deg, seed):
    rng = np.random.default_rng(seed)
    exps = [m for m in itertools.product(range(deg + 1), repeat=dim) if sum(m) <= deg]
    cf = rng.standard_normal(len(exps))

    def P(x):
        return sum(c * np.prod(x ** np.array(m), axis=1) for c, m in zip(cf, exps))
    return P


@pytest.mark.parametrize("dim,k,N", [(2, 1, 2), (2, 2, 2), (2, 3, 1), (3, 1, 1), (3, 2, 1)])
def test_projected_polynomial_of_degree_k_plus_1_is_reproduced(dim, k, N):
    vert, elem = _mesh(dim, N)
    prob = ac.build_problem(vert, elem, k, 1.0, 1.0, 1.0)
    P = _poly(dim, k + 1, 10 * dim + k)
    u = ac.project_volume(prob, lambda x: np.column_stack([P(x)] + [np.zeros(len(x))] * dim))
    lam = np.array([ac.project_face(prob, f, lambda x, t: P(x), 0.0) for f in range(prob.sk.faces.shape[0])])
    ps = ac.postprocess_pressure(prob, u, lam)
    assert ps.shape == (elem.shape[0], ref.n_modes(dim, k + 1))
    scale = ac.l2_error_post(prob, np.zeros_like(ps), lambda x: np.column_stack([P(x)]))
    assert ac.l2_error_post(prob, ps, lambda x: np.column_stack([P(x)])) < 1e-12 * scale
    # p_h itself is not exact at this degree: the test data exercise the k + 1 modes
    assert ac.l2_error(prob, u, lambda x: np.column_stack([P(x)] * (dim + 1))) > 1e-6 * scale


def test_element_means_are_preserved_for_arbitrary_data():
    dim, k = 3, 2
    vert, elem = _mesh(dim, 1)
    prob = ac.build_problem(vert, elem, k, 1.0, 1.0, 1.0)
    rng = np.random.default_rng(4)
    u = rng.standard_normal((elem.shape[0], (dim + 1) * prob.Np))
    lam = rng.standard_normal((prob.sk.faces.shape[0], prob.Nf))
    ps = ac.postprocess_pressure(prob, u, lam)
    xi, wq = ref.simplex_rule(dim, k + 3)
    V, _ = ref.basis(dim, k, xi)
    V1, _ = ref.basis(dim, k + 1, xi)
    for e in range(elem.shape[0]):
        assert abs(wq @ (V1 @ ps[e]) - wq @ (V @ u[e, :prob.Np])) < 1e-13


@pytest.mark.parametrize("k,min_rate", [(1, 2.5), (2, 3.6)])
def test_post_processed_pressure_superconverges_on_the_standing_mode(k, min_rate):
    ex = ac.standing_mode(2)
    T = 0.2
    eh, es = [], []
    for N in (2, 4, 8):
        vert, elem = inputs.unit_square_tri(N)
        prob = ac.build_problem(vert, elem, k, 1.0, 1.0, 1.0)
        prob.dirichlet = lambda x, t: ex(x, t)[:, 0]
        u0 = ac.project_volume(prob, lambda x: ex(x, 0.0))
        nst = 4 * N if k < 2 else 8 * N
        u, lam, t = ac.run_dirk3(prob, u0, T / nst, nst)
        eh.append(ac.l2_error(prob, u, lambda x: ex(x, T)))
        es.append(ac.l2_error_post(prob, ac.postprocess_pressure(prob, u, lam), lambda x: ex(x, T)))
    rate_h = math.log2(eh[-2] / eh[-1])
    rate_s = math.log2(es[-2] / es[-1])
    assert abs(rate_h - (k + 1)) < 0.25, (eh, rate_h)
    assert rate_s > min_rate and es[-1] < 0.5 * eh[-1], (es, rate_s)
