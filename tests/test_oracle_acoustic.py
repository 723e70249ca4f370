"""Pins for the oracle's acoustic HDG scheme: brute force, invariants, closed forms.

* static condensation (Sec. 2.4, Eq. LS) reproduces the uncondensed [A B; C D] solve;
* S_K symmetric negative definite, A_K's symmetric part positive definite;
* constant state reproduced exactly by BE, BDF2 and DIRK3;
* the backward-Euler discrete energy identity (the acoustic analogue of the energy
  identity of Sec. 4.2) holds step by step;
* the exact standing mode converges at order k + 1 in L2;
* BDF/DIRK coefficients satisfy the textbook order conditions (Sec. 2.3).
"""
import math

import numpy as np
import pytest

from oracle import acoustic as ac
from oracle import reference as ref
from paper_1807_00086_gb300 import inputs


def _problem(dim, N, k, seed=1, dirichlet=True, source=True):
    vert, elem = inputs.unit_square_tri(N) if dim == 2 else inputs.unit_cube_tet(N)
    ne = elem.shape[0]
    prob = ac.build_problem(vert, elem, k, 1.0, inputs.loguniform(ne, 0.5, 2.0, seed + 7),
                            inputs.loguniform(ne, 1.0, 3.0, seed))
    if dirichlet:
        prob.dirichlet = lambda x, t: np.cos(np.pi * x[:, 0]) * np.sin(np.pi * x[:, 1] + t) + 0.3 * x[:, -1]
    if source:
        ac.add_point_source(prob, [0.41, 0.37, 0.33][:dim], 10.0, 0.05, amp=2.0)
    return prob


def test_skeleton_counts():
    for N in (1, 2, 3):
        vert, elem = inputs.unit_cube_tet(N)
        sk = ac.skeleton(elem)
        assert sk.boundary.sum() == 12 * N * N
        assert (~sk.boundary).sum() == 12 * N ** 3 - 6 * N * N
        vert, elem = inputs.unit_square_tri(N)
        sk = ac.skeleton(elem)
        assert sk.boundary.sum() == 4 * N
        assert (~sk.boundary).sum() == 3 * N * N - 2 * N
    # every interior face is shared by exactly two elements, boundary faces by one
    vert, elem = inputs.unit_cube_tet(2)
    sk = ac.skeleton(elem)
    for f, inc in enumerate(sk.face_elems):
        assert len(inc) == (1 if sk.boundary[f] else 2)
        for (e, j) in inc:
            assert sk.elem_face[e, j] == f


def test_mass_matrix_is_detJ_identity():
    rng = np.random.default_rng(0)
    for dim in (2, 3):
        X = rng.standard_normal((dim + 1, dim))
        bl = ac.element_blocks(X, 3, 1.0, 1.0, 1.0)
        Np = ref.n_modes(dim, 3)
        M = bl.Mw[:Np, :Np]
        assert np.abs(M - bl.detJ * np.eye(Np)).max() < 1e-12 * bl.detJ
        # detJ is the simplex volume times d!
        assert abs(bl.detJ - abs(np.linalg.det((X[1:] - X[0]).T))) < 1e-12


def test_face_geometry_consistent_between_neighbours():
    vert, elem = inputs.unit_cube_tet(2)
    prob = ac.build_problem(vert, elem, 1, 1.0, 1.0, 1.0)
    for f, inc in enumerate(prob.sk.face_elems):
        if len(inc) == 2:
            (e0, j0), (e1, j1) = inc
            n0 = prob.blocks[e0].normal[j0]
            n1 = prob.blocks[e1].normal[j1]
            assert np.allclose(n0, -n1, atol=1e-14)
            # the trace-trace face mass is the same seen from both sides
            assert np.allclose(prob.blocks[e0].G[j0], prob.blocks[e1].G[j1], atol=1e-14)


@pytest.mark.parametrize("dim,N,k", [(2, 2, 1), (2, 2, 2), (2, 2, 3), (2, 1, 4), (3, 1, 1), (3, 1, 2), (3, 1, 3)])
def test_condensed_equals_monolithic(dim, N, k):
    prob = _problem(dim, N, k)
    rng = np.random.default_rng(5)
    h = rng.standard_normal((prob.sk.elem.shape[0], (dim + 1) * prob.Np))
    for alpha in (0.5, 40.0):
        cond = ac.condense(prob, alpha)
        u, lam = ac.solve_stage(prob, cond, h, 0.07)
        um, lm = ac.solve_monolithic(prob, alpha, h, 0.07)
        assert np.abs(u - um).max() <= 1e-12 * np.abs(um).max()
        assert np.abs(lam - lm).max() <= 1e-12 * np.abs(lm).max()


@pytest.mark.parametrize("dim,k", [(2, 1), (2, 3), (3, 2), (3, 4)])
def test_schur_symmetric_negative_definite(dim, k):
    prob = _problem(dim, 1, k)
    for alpha in (0.1, 100.0):
        cond = ac.condense(prob, alpha)
        for e, S in enumerate(cond.S):
            assert np.abs(S - S.T).max() <= 1e-12 * np.abs(S).max()
            assert np.linalg.eigvalsh(0.5 * (S + S.T)).max() < 0
            A = alpha * prob.blocks[e].Mw + prob.blocks[e].A0
            assert np.linalg.eigvalsh(0.5 * (A + A.T)).min() > 0


def test_trace_apply_matches_assembled_operator():
    prob = _problem(3, 2, 2)
    cond = ac.condense(prob, 3.0)
    x = np.random.default_rng(2).standard_normal(cond.K.shape[0])
    assert np.abs(ac.trace_apply(prob, cond, x) - cond.K @ x).max() < 1e-12 * np.abs(cond.K @ x).max()


@pytest.mark.parametrize("dim", [2, 3])
def test_constant_state_is_exact(dim):
    prob = _problem(dim, 2 if dim == 2 else 1, 2, dirichlet=False, source=False)
    prob.dirichlet = lambda x, t: np.ones(x.shape[0])
    u0 = ac.project_volume(prob, lambda x: np.concatenate([np.ones((x.shape[0], 1)), np.zeros((x.shape[0], dim))], axis=1))
    for run in (lambda: ac.run_bdf(prob, u0, 0.05, 3, 1), lambda: ac.run_bdf(prob, u0, 0.05, 3, 2),
                lambda: ac.run_dirk3(prob, u0, 0.05, 2)):
        u, lam, _ = run()
        assert np.abs(u - u0).max() < 1e-12
        assert np.abs(lam - 1.0 * (np.arange(prob.Nf) == 0) * lam[:, :1]).max() < 1e-12


@pytest.mark.parametrize("dim,N", [(2, 3), (3, 1)])
def test_backward_euler_energy_identity(dim, N):
    """E^{n+1} - E^n + 1/2|u^{n+1}-u^n|_M^2 + dt sum_dK <tau (p - p_hat)^2, 1>
       = dt [(s, p^{n+1}) - <p_hat, v_hat.n>_{Gamma_D}]."""
    prob = _problem(dim, N, 2)
    ex = ac.standing_mode(dim)
    u0 = ac.project_volume(prob, lambda x: ex(x, 0.1))
    dt = 0.01
    prev = [u0]

    def check(n, t, u, lam):
        diss, bwork, src = ac.energy_terms(prob, u, lam, t)
        du = u - prev[-1]
        lhs = (ac.energy(prob, u) - ac.energy(prob, prev[-1])
               + 0.5 * sum(du[e] @ bl.Mw @ du[e] for e, bl in enumerate(prob.blocks)) + dt * diss)
        rhs = dt * (src - bwork)
        assert abs(lhs - rhs) <= 1e-11 * (abs(lhs) + dt * abs(diss) + 1e-300)
        prev.append(u)

    ac.run_bdf(prob, u0, dt, 3, 1, on_step=check)


def test_standing_mode_solves_the_pde():
    for dim in (2, 3):
        f = ac.standing_mode(dim)
        x = np.random.default_rng(0).uniform(0, 1, size=(5, dim))
        t, h = 0.37, 1e-5
        dp_dt = (f(x, t + h)[:, 0] - f(x, t - h)[:, 0]) / (2 * h)
        div_v = sum((f(x + h * np.eye(dim)[j], t)[:, j + 1] - f(x - h * np.eye(dim)[j], t)[:, j + 1]) / (2 * h)
                    for j in range(dim))
        assert np.abs(dp_dt + div_v).max() < 1e-7
        for j in range(dim):
            dv = (f(x, t + h)[:, j + 1] - f(x, t - h)[:, j + 1]) / (2 * h)
            dp = (f(x + h * np.eye(dim)[j], t)[:, 0] - f(x - h * np.eye(dim)[j], t)[:, 0]) / (2 * h)
            assert np.abs(dv + dp).max() < 1e-7


@pytest.mark.parametrize("k", [1, 2, 3])
def test_standing_mode_converges_at_order_k_plus_1_2d(k):
    ex = ac.standing_mode(2)
    T = 0.2
    errs = []
    for N in (2, 4, 8):
        vert, elem = inputs.unit_square_tri(N)
        prob = ac.build_problem(vert, elem, k, 1.0, 1.0, 1.0)
        prob.dirichlet = lambda x, t: ex(x, t)[:, 0]
        u0 = ac.project_volume(prob, lambda x: ex(x, 0.0))
        nst = 4 * N if k < 3 else 8 * N
        u, lam, t = ac.run_dirk3(prob, u0, T / nst, nst)
        errs.append(ac.l2_error(prob, u, lambda x: ex(x, T)))
    rate = math.log2(errs[-2] / errs[-1])
    assert rate > k + 1 - 0.25, (errs, rate)


def test_standing_mode_converges_3d():
    ex = ac.standing_mode(3)
    T = 0.1
    errs = []
    for N in (1, 2, 4):
        vert, elem = inputs.unit_cube_tet(N)
        prob = ac.build_problem(vert, elem, 1, 1.0, 1.0, 1.0)
        prob.dirichlet = lambda x, t: ex(x, t)[:, 0]
        u0 = ac.project_volume(prob, lambda x: ex(x, 0.0))
        nst = 2 * N
        u, lam, t = ac.run_dirk3(prob, u0, T / nst, nst)
        errs.append(ac.l2_error(prob, u, lambda x: ex(x, T)))
    rate = math.log2(errs[-2] / errs[-1])
    assert rate > 1.7, (errs, rate)


def test_dirk3_order_conditions_and_L_stability():
    a, b, c = ac.dirk3_tableau()
    assert abs(b.sum() - 1) < 1e-14
    assert np.abs(a.sum(axis=1) - c).max() < 1e-14
    assert abs(b @ c - 0.5) < 1e-14
    assert abs(b @ c ** 2 - 1 / 3) < 1e-14
    assert abs(b @ a @ c - 1 / 6) < 1e-14
    assert np.allclose(np.diag(a), a[0, 0]) and np.all(np.triu(a, 1) == 0)
    z = -1e8
    R = 1 + z * b @ np.linalg.solve(np.eye(3) - z * a, np.ones(3))
    assert abs(R) < 1e-6
    # eq10_2 weights: stiffly accurate, so u^{n+1} = u^{n,3}
    d = np.linalg.inv(a)
    e = b @ d
    assert np.abs(e - [0, 0, 1]).max() < 1e-13 and abs(1 - b @ d.sum(axis=1)) < 1e-13


def test_bdf_order_conditions():
    for s, (a, bs) in ac.BDF.items():
        i = np.arange(s + 1)
        assert abs(np.sum(a)) < 1e-15
        for q in range(1, s + 1):            # sum a_i i^q = q s^{q-1} b_s
            assert abs(np.sum(np.array(a) * i ** q) - q * s ** (q - 1) * bs) < 1e-14


def test_ricker_wavelet_closed_form_points():
    f0, t0 = 10.0, 0.12
    assert ac.ricker(t0, f0, t0) == 1.0
    tz = t0 + 1.0 / (math.sqrt(2) * math.pi * f0)
    assert abs(ac.ricker(tz, f0, t0)) < 1e-15


def test_ricker_wavelet_is_the_normalised_second_derivative_of_a_gaussian():
    """r(t) = -g''(t) / g''(t0) with g(t) = exp(-pi^2 f0^2 (t - t0)^2): the Ricker wavelet as the
    scaled negative curvature of a Gaussian pulse, checked by central differences of g."""
    f0, t0, h = 10.0, 0.12, 1e-5
    g = lambda t: math.exp(-(math.pi * f0 * (t - t0)) ** 2)
    d2 = lambda t: (g(t + h) - 2.0 * g(t) + g(t - h)) / (h * h)
    scale = -d2(t0)
    for t in np.linspace(0.0, 0.3, 31):
        assert abs(ac.ricker(t, f0, t0) - (-d2(t) / scale)) < 1e-5


def test_point_location_takes_the_lowest_id_element_containing_the_point():
    """The source element is the lowest id whose closed simplex holds x_s (brute force over
    barycentric coordinates computed from the vertices, not from the blocks' inverse maps):
    interior points, points on shared faces and edges, and a vertex shared by many tets."""
    vert, elem = inputs.unit_cube_tet(2)
    prob = ac.build_problem(vert, elem, 1, 1.0, np.ones(elem.shape[0]), np.ones(elem.shape[0]))

    def holders(x):
        out = []
        for e, tet in enumerate(elem):
            X = vert[np.sort(tet)]
            lam = np.linalg.solve(np.vstack([X.T, np.ones(4)]), np.append(x, 1.0))
            if lam.min() >= -1e-12:
                out.append(e)
        return out

    for x in ([0.3, 0.2, 0.1], [0.5, 0.5, 0.5], [0.25, 0.25, 0.5], [0.5, 0.25, 0.25], [0.7, 0.6, 0.2]):
        h = holders(np.array(x))
        e, xi = ac.locate(prob, x)
        assert h and e == min(h)
        assert len(h) > 1 or x == [0.3, 0.2, 0.1] or x == [0.7, 0.6, 0.2]
    assert len(holders(np.array([0.5, 0.5, 0.5]))) >= 6


def test_point_source_evaluates_polynomials():
    """(delta_xs, w) for w = projection of a P_k polynomial equals the polynomial at xs."""
    prob = _problem(3, 1, 3, dirichlet=False, source=False)
    xs = np.array([0.3, 0.6, 0.45])
    ac.add_point_source(prob, xs, 10.0, 0.0)
    q = lambda x: np.stack([1 + x[:, 0] ** 2 * x[:, 1] - 2 * x[:, 2] ** 3] + [np.zeros(x.shape[0])] * 3, axis=1)
    u = ac.project_volume(prob, q)
    e, phi = prob.sources[0][0], prob.sources[0][1]
    assert abs(phi @ u[e, :prob.Np] - q(xs[None])[0, 0]) < 1e-12
