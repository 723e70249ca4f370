"""Nonlinear (Saint Venant-Kirchhoff) elastodynamics on the GPU (Sec. 4.4, Eqs. UNEL,
eq:HDG_nelas1-5): the Newton stages of hdg_step (condensation of every Newton iteration, trace
solve, recovery) through the C ABI against oracle/elastic_svk.py.

* per DIRK(3,3) step, fields and traces within 1e-11 relative of the oracle (FP64 path), and
  the same Newton iteration count in every stage, k = 1, 2, 3, in the nonlinear regime
  (|H| ~ 0.3, so F S(F) is far from its linearisation);
* the clamped vibrating plate with body force and traction faces (the forcing callback): the
  same per-step agreement, and the velocity error converging at order k + 1 under refinement;
* the Newton loop ends by itself at newton_maxit (HDG_ENOCONV); a state at rest stays at rest;
  unsupported configurations are rejected.
"""
import math

import numpy as np
import pytest

from gpu_helpers import relerr
from oracle import elastic_svk as nl
from paper_1807_00086_gb300 import inputs

pytestmark = pytest.mark.gpu

RHO, LAM, MU = 1.0, 1.5, 1.0


def _gpu(vert, elem, k, **kw):
    from paper_1807_00086_gb300 import hdg
    ne = elem.shape[0]
    return hdg.Solver(vert, elem, k, 1.0, np.full(ne, RHO), lam=np.full(ne, LAM), mu=np.full(ne, MU), svk=True,
                      rtol=1e-12, **kw)


def _state(ne, Np, seed, amp_v=0.5, amp_h=0.3, amp_p=0.2):
    rng = np.random.default_rng(seed)
    u = np.zeros((ne, 21 * Np))
    u[:, :3 * Np] = amp_v * rng.standard_normal((ne, 3 * Np))
    u[:, 3 * Np:12 * Np] = amp_h * rng.standard_normal((ne, 9 * Np)) / Np
    u[:, 12 * Np:] = amp_p * rng.standard_normal((ne, 9 * Np))
    return u


@pytest.mark.parametrize("k,N", [(1, 2), (2, 1), (3, 1)])
def test_svk_dirk3_steps_match_oracle(k, N):
    import torch
    vert, elem = inputs.unit_cube_tet(N)
    prob = nl.build_problem(vert, elem, k, RHO, LAM, MU)
    ne, Np = elem.shape[0], prob.Np
    u0 = _state(ne, Np, 10 + k)
    dt, nsteps = 0.02, 3
    ref = []
    _, _, its = nl.run_dirk3(prob, u0, dt, nsteps, on_step=lambda n, t, u, lam: ref.append((u.copy(), lam.copy())))
    assert max(its) >= 3          # genuinely nonlinear stages
    s = _gpu(vert, elem, k)
    s.hdg_set_state(torch.tensor(u0, device="cuda"), 0.0)
    for n in range(nsteps):
        info = s.hdg_step(dt, "dirk3", 1)
        u, lam, t = s.hdg_get_state()
        assert relerr(u.cpu().numpy(), ref[n][0]) < 1e-11, n
        assert relerr(lam.cpu().numpy(), ref[n][1]) < 1e-11, n
        assert s.hdg_svk_newton_counts() == list(its[3 * n:3 * n + 3]), n
        assert info["sweeps"] == sum(its[3 * n:3 * n + 3]) and info["iterations"] > 0


@pytest.mark.parametrize("k,N", [(1, 2), (2, 1), (3, 1)])
def test_svk_fp32_jacobian_converges_to_the_same_stage_solutions(k, N):
    """prec="mixed": tangent, condensation and factor in FP32 around the FP64 residual. Newton
    with the approximate Jacobian converges to the same stage solutions (parity bar 1e-9; the
    stopping test is the same 1e-11), at most a few Newton iterations more per stage."""
    import torch
    vert, elem = inputs.unit_cube_tet(N)
    prob = nl.build_problem(vert, elem, k, RHO, LAM, MU)
    ne, Np = elem.shape[0], prob.Np
    u0 = _state(ne, Np, 20 + k)
    dt, nsteps = 0.02, 3
    ref = []
    _, _, its = nl.run_dirk3(prob, u0, dt, nsteps, on_step=lambda n, t, u, lam: ref.append((u.copy(), lam.copy())))
    s = _gpu(vert, elem, k, prec="mixed")
    s.hdg_set_state(torch.tensor(u0, device="cuda"), 0.0)
    for n in range(nsteps):
        s.hdg_step(dt, "dirk3", 1)
        u, lam, t = s.hdg_get_state()
        assert relerr(u.cpu().numpy(), ref[n][0]) < 1e-9, n
        assert relerr(lam.cpu().numpy(), ref[n][1]) < 1e-9, n
        got = s.hdg_svk_newton_counts()
        for g_, o_ in zip(got, its[3 * n:3 * n + 3]):
            assert o_ <= g_ <= o_ + 3, (got, its[3 * n:3 * n + 3])


def _plate(n, k):
    """The clamped plate of Sec. 4.5 with the deformation phi = X + A sin(pi t) sin(pi X) sin(pi Y) e_z
    (A = 0.4): exact v, F, P = F S(F); the body force f = rho v_t - div P with div P by
    4th-order central differences (the same callable drives the oracle and the GPU)."""
    A = 0.4

    def F_of(x, t):
        X, Y = x[:, 0], x[:, 1]
        wx = A * math.sin(math.pi * t) * math.pi * np.cos(math.pi * X) * np.sin(math.pi * Y)
        wy = A * math.sin(math.pi * t) * math.pi * np.sin(math.pi * X) * np.cos(math.pi * Y)
        F = np.zeros((x.shape[0], 3, 3))
        F[:, 0, 0] = F[:, 1, 1] = F[:, 2, 2] = 1.0
        F[:, 2, 0], F[:, 2, 1] = wx, wy
        return F

    def P_of(x, t):
        return nl.pk_batch(F_of(x, t), LAM, MU)

    def v_of(x, t):
        v = np.zeros((x.shape[0], 3))
        v[:, 2] = A * math.pi * math.cos(math.pi * t) * np.sin(math.pi * x[:, 0]) * np.sin(math.pi * x[:, 1])
        return v

    def f_of(x, t):
        h = 1e-3
        divP = np.zeros((x.shape[0], 3))
        for J in range(3):
            e = np.zeros(3)
            e[J] = h
            d = (-P_of(x + 2 * e, t) + 8 * P_of(x + e, t) - 8 * P_of(x - e, t) + P_of(x - 2 * e, t)) / (12 * h)
            divP += d[:, :, J]
        vt = np.zeros((x.shape[0], 3))
        vt[:, 2] = -A * math.pi ** 2 * math.sin(math.pi * t) * np.sin(math.pi * x[:, 0]) * np.sin(math.pi * x[:, 1])
        return RHO * vt - divP

    vert, elem = inputs.plate_tet(n)
    return vert, elem, F_of, P_of, v_of, f_of


def _plate_gpu(n, k):
    import torch
    vert, elem, F_of, P_of, v_of, f_of = _plate(n, k)
    s = _gpu(vert, elem, k)
    xb = s.hdg_quadrature_points(1)                     # [n_bnd, nq_face, 3]
    zb = xb[:, :, 2]
    top = np.all(np.abs(zb - 0.01) < 1e-13, axis=1)
    bot = np.all(np.abs(zb) < 1e-13, axis=1)
    s.hdg_svk_set_traction_faces(top | bot)
    xv = s.hdg_quadrature_points(0)                     # [n_elem, nq_vol, 3]
    nq = xv.shape[1]
    nrm = np.where(top[:, None], 1.0, -1.0)             # outward normals +-e_z on the traction faces

    def forcing(t, f, g):
        f[:] = f_of(xv.reshape(-1, 3), t).reshape(f.shape)
        P = P_of(xb.reshape(-1, 3), t).reshape(xb.shape[0], xb.shape[1], 3, 3)
        g[:] = P[:, :, :, 2] * nrm[:, :, None]
    s.hdg_svk_set_forcing(forcing)
    I9 = np.eye(3).ravel()
    vals = np.concatenate([v_of(xv.reshape(-1, 3), 0.0), F_of(xv.reshape(-1, 3), 0.0).reshape(-1, 9) - I9,
                           P_of(xv.reshape(-1, 3), 0.0).reshape(-1, 9)], axis=1).reshape(s.n_elem, nq, 21)
    u0 = s.hdg_project_volume(vals)
    s.hdg_set_state(u0, 0.0)
    return s, (vert, elem, F_of, P_of, v_of, f_of), u0


def test_svk_plate_with_traction_and_body_force_matches_oracle():
    k, n = 1, 2
    s, (vert, elem, F_of, P_of, v_of, f_of), u0 = _plate_gpu(n, k)

    def top_or_bottom(Y):
        z = Y[:, 2]
        return bool(np.all(np.abs(z - z[0]) < 1e-14) and (abs(z[0]) < 1e-14 or abs(z[0] - 0.01) < 1e-14))
    prob = nl.build_problem(vert, elem, k, RHO, LAM, MU, neumann_face=top_or_bottom)
    prob.body_force = f_of
    prob.traction = lambda x, nrm, t: np.einsum("qij,j->qi", P_of(x, t), nrm)
    uo0 = nl.project(prob, v_of, lambda x, t: F_of(x, t).reshape(-1, 9) - np.eye(3).ravel(),
                     lambda x, t: P_of(x, t).reshape(-1, 9), 0.0)
    assert relerr(u0.cpu().numpy(), uo0) < 1e-12       # the projections agree
    dt, nsteps = 0.125 / 4, 4
    ref = []
    _, _, its = nl.run_dirk3(prob, uo0, dt, nsteps, on_step=lambda n_, t, u, lam: ref.append((u.copy(), lam.copy())))
    for m in range(nsteps):
        s.hdg_step(dt, "dirk3", 1)
        u, lam, t = s.hdg_get_state()
        assert relerr(u.cpu().numpy(), ref[m][0]) < 1e-11, m
        assert relerr(lam.cpu().numpy(), ref[m][1]) < 1e-11, m
        assert s.hdg_svk_newton_counts() == list(its[3 * m:3 * m + 3]), m


def test_svk_plate_velocity_converges_at_order_k_plus_1():
    """Sec. 4.5, Table tab:eoc_nonlinear_elastodyn: k = 1, the velocity error at T = 0.125 on
    n x n x 1 plates, dt = T / (2 n) (DIRK3 is third order). The paper prints 1.97 on its finest
    mesh; here 2 -> 4 gives 1.98 and 4 -> 8 2.36 (the oracle's own values at these meshes), so
    the first rate is held to 2 +- 0.3 and the second to at least 1.7."""
    errs = []
    for n in (2, 4, 8):
        s, (vert, elem, F_of, P_of, v_of, f_of), _ = _plate_gpu(n, 1)
        T = 0.125
        s.hdg_step(T / (2 * n), "dirk3", 2 * n)
        u, lam, t = s.hdg_get_state()
        u = u.cpu().numpy()
        xv = s.hdg_quadrature_points(0)
        prob = nl.build_problem(vert, elem, 1, RHO, LAM, MU)
        err = 0.0
        for e, g in enumerate(prob.geo):
            vh = np.stack([g.V @ u[e, i * prob.Np:(i + 1) * prob.Np] for i in range(3)], axis=1)
            err += np.sum(g.w[:, None] * (vh - v_of(g.xq, T)) ** 2)
        errs.append(math.sqrt(err))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert abs(rates[0] - 2.0) < 0.3 and rates[1] > 1.7, (errs, rates)


def test_svk_newton_stops_at_newton_maxit_and_rest_stays_at_rest():
    import torch
    from paper_1807_00086_gb300 import hdg
    vert, elem = inputs.unit_cube_tet(1)
    s = _gpu(vert, elem, 2, newton_maxit=1)
    Np = s.Np
    s.hdg_set_state(torch.tensor(_state(s.n_elem, Np, 3), device="cuda"), 0.0)
    with pytest.raises(hdg.HDGError) as ei:
        s.hdg_step(0.02, "dirk3", 1)
    assert ei.value.status == -4
    r = _gpu(vert, elem, 2)
    r.hdg_set_state(torch.zeros((r.n_elem, r.n), dtype=torch.float64, device="cuda"), 0.0)
    info = r.hdg_step(0.02, "dirk3", 2)
    u, lam, t = r.hdg_get_state()
    assert torch.count_nonzero(u) == 0 and torch.count_nonzero(lam) == 0
    assert r.hdg_svk_newton_counts() == [1] * 6 and info["sweeps"] == 6


def test_svk_rejects_unsupported_configurations():
    from paper_1807_00086_gb300 import hdg
    vert, elem = inputs.unit_cube_tet(1)
    ne = elem.shape[0]
    for kw in ({"prec": "mixed16"}, {"nrhs": 2}, {"solver": "gmres"}):
        with pytest.raises(hdg.HDGError):
            hdg.Solver(vert, elem, 2, 1.0, 1.0, lam=np.full(ne, LAM), mu=np.full(ne, MU), svk=True, **kw)
    with pytest.raises(hdg.HDGError):
        hdg.Solver(vert, elem, 4, 1.0, 1.0, lam=np.full(ne, LAM), mu=np.full(ne, MU), svk=True)
    s = _gpu(vert, elem, 1)
    with pytest.raises(hdg.HDGError):
        s.hdg_condense(10.0)
    with pytest.raises(hdg.HDGError):
        s.hdg_step(0.01, "bdf2", 1)
