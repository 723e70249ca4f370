"""Pins for the oracle's time-marching loops against the exact semi-discrete solution.

The HDG semi-discretisation of Sec. 2.3 (Eq. ch5appendx1:eq8) is the index-1 DAE
  Mw u' = -A0 u - B lam + s(t),   0 = C u + D lam   (interior faces),
with D block diagonal and invertible (-tau times the face mass on each face, summed over
the face's two elements). Eliminating lam = -D^{-1} C u leaves the linear ODE
  u' = L u + Mw^{-1} s(t),   L = -Mw^{-1} (A0 - B D^{-1} C),
whose exact solution is expm(t L) u0 without a source. These tests assemble Mw, A0, B, C
and D from the element blocks (a plain global assembly written here, independent of the
oracle's condensation and of its marching code) and check that

  * BE, BDF2 (Eq. ch5appendx1:eq9b) and DIRK(3,3) (Eqs. ch5appendx1:eq10_1-2) converge to
    expm(T L) u0 at orders 1, 2 and 3 when dt is halved: a swapped history level, a wrong
    BDF coefficient or a wrong DIRK weight lowers the observed order;
  * with a Ricker source and a start from rest (the benchmark's situation, where the
    reading u^{-1} = u^0 = 0 is exact), BDF2 and DIRK3 converge at orders 2 and 3 to a
    high-accuracy reference integration of the forced ODE (scipy's DOP853): this also
    pins the times at which the source is evaluated (t^{n+1} for BDF, t_n + c_i dt for
    the DIRK stages).
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla
from scipy.integrate import solve_ivp

from oracle import acoustic as ac
from paper_1807_00086_gb300 import inputs


def _semidiscrete(prob):
    """Global Mw, A0, B, C, D over elements and interior faces (homogeneous Dirichlet)."""
    sk, Nf = prob.sk, prob.Nf
    ne = sk.elem.shape[0]
    n = (sk.dim + 1) * prob.Np
    interior = np.nonzero(~sk.boundary)[0]
    pos = -np.ones(sk.faces.shape[0], dtype=np.int64)
    pos[interior] = np.arange(interior.size)
    nu, nl = ne * n, interior.size * Nf
    Mw, A0 = np.zeros((nu, nu)), np.zeros((nu, nu))
    B, C, D = np.zeros((nu, nl)), np.zeros((nl, nu)), np.zeros((nl, nl))
    for e, bl in enumerate(prob.blocks):
        ue = slice(e * n, (e + 1) * n)
        Mw[ue, ue] = bl.Mw
        A0[ue, ue] = bl.A0
        for a in range(sk.dim + 1):
            p = pos[sk.elem_face[e, a]]
            if p < 0:
                continue
            fa = slice(p * Nf, (p + 1) * Nf)
            la = slice(a * Nf, (a + 1) * Nf)
            B[ue, fa] += bl.B[:, la]
            C[fa, ue] += bl.C[la, :]
            D[fa, fa] += bl.D[la, la]
    return Mw, A0, B, C, D


def _generator(prob):
    Mw, A0, B, C, D = _semidiscrete(prob)
    L = -np.linalg.solve(Mw, A0 - B @ np.linalg.solve(D, C))
    return L, Mw


def _problem(seed=3):
    vert, elem = inputs.unit_square_tri(2)
    ne = elem.shape[0]
    return ac.build_problem(vert, elem, 2, 1.0, inputs.loguniform(ne, 0.5, 2.0, seed + 7),
                            inputs.loguniform(ne, 1.0, 3.0, seed))


def _smooth_start(prob):
    """A smooth state compatible with homogeneous Dirichlet data."""
    def f(x):
        p = np.sin(np.pi * x[:, 0]) * np.sin(np.pi * x[:, 1])
        return np.stack([p, 0.3 * np.cos(np.pi * x[:, 1]), -0.2 * x[:, 0] * (1 - x[:, 0])], axis=1)
    return ac.project_volume(prob, f)


def _rate(errs):
    return [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]


def test_semidiscrete_generator_is_dissipative():
    """Energy decays along the exact flow: L is Mw-dissipative (the semi-discrete analogue of
    the energy identity); also the elimination reproduces the oracle's stage solve at one step."""
    prob = _problem()
    L, Mw = _generator(prob)
    sym = Mw @ L + L.T @ Mw
    assert np.linalg.eigvalsh(0.5 * (sym + sym.T)).max() < 1e-10 * np.abs(sym).max()
    # one backward-Euler step through the oracle equals (I - dt L)^{-1} u0
    u0 = _smooth_start(prob)
    dt = 0.05
    u1, _, _ = ac.run_bdf(prob, u0, dt, 1, 1)
    ue = np.linalg.solve(np.eye(L.shape[0]) - dt * L, u0.ravel())
    assert np.abs(u1.ravel() - ue).max() < 1e-12 * np.abs(ue).max()


@pytest.mark.parametrize("scheme,order,n0", [("be", 1, 8), ("bdf2", 2, 8), ("dirk3", 3, 4)])
def test_marching_converges_to_the_exact_semidiscrete_solution(scheme, order, n0):
    prob = _problem()
    L, _ = _generator(prob)
    u0 = _smooth_start(prob)
    T = 0.4
    exact = (sla.expm(T * L) @ u0.ravel()).reshape(u0.shape)
    errs = []
    for nst in (n0, 2 * n0, 4 * n0):
        dt = T / nst
        if scheme == "be":
            u, _, t = ac.run_bdf(prob, u0, dt, nst, 1)
        elif scheme == "bdf2":
            # exact history level u(-dt): the start-up then carries no first-order error
            um1 = (sla.expm(-dt * L) @ u0.ravel()).reshape(u0.shape)
            u, _, t = ac.run_bdf(prob, u0, dt, nst, 2, u_prev=um1)
        else:
            u, _, t = ac.run_dirk3(prob, u0, dt, nst)
        assert abs(t - T) < 1e-13
        errs.append(np.abs(u - exact).max() / np.abs(exact).max())
    rates = _rate(errs)
    assert abs(rates[-1] - order) < 0.2, (errs, rates)


def test_bdf2_planted_history_swap_loses_its_order():
    """The order test above detects a BDF2 loop that combines its history levels in the wrong
    order: the same formula with the two levels exchanged is not a consistent method."""
    prob = _problem()
    L, _ = _generator(prob)
    u0 = _smooth_start(prob)
    T = 0.4
    exact = (sla.expm(T * L) @ u0.ravel()).reshape(u0.shape)
    a, bs = ac.BDF[2]
    errs = []
    for nst in (8, 16, 32):
        dt = T / nst
        cond = ac.condense(prob, a[-1] / (bs * dt))
        hist = [(sla.expm(-dt * L) @ u0.ravel()).reshape(u0.shape), u0.copy()]
        for n in range(nst):
            h = -(a[0] * hist[1] + a[1] * hist[0]) / a[-1]          # planted: levels swapped
            u, _ = ac.solve_stage(prob, cond, h, (n + 1) * dt)
            hist = [hist[1], u]
        errs.append(np.abs(hist[-1] - exact).max() / np.abs(exact).max())
    rates = _rate(errs)
    assert not abs(rates[-1] - 2) < 0.2 or errs[-1] > 1e-2, (errs, rates)


@pytest.mark.parametrize("scheme,order", [("bdf2", 2), ("dirk3", 3)])
def test_forced_start_from_rest_converges(scheme, order):
    """Ricker point source, zero initial state; the source is ~1e-10 of its peak at t <= 0, so
    the BDF2 start-up u^{-1} = u^0 = 0 is exact to that level. DIRK3 is measured where
    dt |eig L| < 1: at larger steps the stiff modes reduce its observed order (2.7 at
    dt |eig L| between 2 and 7)."""
    prob = _problem()
    f0, t0 = 4.0, 0.4
    ac.add_point_source(prob, [0.41, 0.37], f0, t0, amp=2.0)
    assert abs(ac.ricker(0.0, f0, t0)) < 1e-9
    L, Mw = _generator(prob)
    ne, n = prob.sk.elem.shape[0], (prob.sk.dim + 1) * prob.Np
    e_src, phi = prob.sources[0][0], prob.sources[0][1]
    s_vec = np.zeros(ne * n)
    s_vec[e_src * n:e_src * n + prob.Np] = 2.0 * phi
    g = np.linalg.solve(Mw, s_vec)
    T = 0.6
    ref = solve_ivp(lambda t, u: L @ u + ac.ricker(t, f0, t0) * g, (0.0, T), np.zeros(ne * n), method="DOP853",
                    rtol=1e-12, atol=1e-15).y[:, -1].reshape(ne, n)
    u0 = np.zeros((ne, n))
    errs = []
    for nst in ((60, 120, 240) if scheme == "bdf2" else (120, 240, 480)):
        dt = T / nst
        if scheme == "bdf2":
            u, _, _ = ac.run_bdf(prob, u0, dt, nst, 2)
        else:
            u, _, _ = ac.run_dirk3(prob, u0, dt, nst)
        errs.append(np.abs(u - ref).max() / np.abs(ref).max())
    rates = _rate(errs)
    assert abs(rates[-1] - order) < 0.2, (errs, rates)
