"""Per-element degrees (3D elastodynamics, k_K in {1..4}, face degree k_F = max of the
neighbours): CUDA path through the C ABI against the variable-degree FP64 oracle.

Fields and traces are flat on this path (element by element, face by face). Clamped
boundary, element-wise lognormal Lame parameters. FP64 path <= 1e-11 per step (operators
<= 1e-12), mixed precision <= 1e-9."""
import numpy as np
import pytest

from gpu_helpers import relerr
from oracle import elastic as el
from oracle import elastic_vardeg as vd
from paper_1807_00086_gb300 import inputs

pytestmark = pytest.mark.gpu


def pair(N, ks, prec="fp64", seed=2):
    from paper_1807_00086_gb300 import hdg
    vert, elem = inputs.unit_cube_tet(N)
    ne = elem.shape[0]
    rho = inputs.loguniform(ne, 0.5, 2.0, seed + 5)
    lam = inputs.lognormal(ne, 1.5, 0.5, seed)
    mu = inputs.lognormal(ne, 1.0, 0.5, seed + 1)
    s = hdg.Solver(vert, elem, int(max(ks)), 1.0, rho, lam=lam, mu=mu, prec=prec,
                   rtol=1e-13 if prec == "fp64" else 1e-12, elem_k=ks)
    prob = vd.build_problem(vert, elem, ks, rho, lam, mu)
    return s, prob


def interior_mask(prob):
    m = np.zeros(int(prob.t_off[-1]), dtype=bool)
    for f in np.nonzero(~prob.sk.boundary)[0]:
        m[prob.t_off[f]:prob.t_off[f + 1]] = True
    return m


@pytest.mark.parametrize("N,seed", [(1, 3), (2, 4)])
def test_vardeg_trace_operators_match_oracle(N, seed):
    import torch
    ks = inputs.element_degrees(6 * N ** 3, 1, 4, seed)
    s, prob = pair(N, ks)
    assert s.vardeg and s._tshape == (int(prob.t_off[-1]),)
    alpha = 17.0
    s.hdg_condense(alpha)
    cond = vd.condense(prob, alpha)
    mask = interior_mask(prob)
    rng = np.random.default_rng(seed)
    lam = rng.standard_normal(mask.size) * mask
    y = s.hdg_trace_apply(torch.tensor(lam, device="cuda")).cpu().numpy()
    yo = np.zeros_like(lam)
    yo[mask] = cond.K @ lam[mask]
    assert relerr(y, yo) < 1e-12
    # condensed right-hand side and recovery of random element data
    F = rng.standard_normal(int(prob.u_off[-1]))
    r = s.hdg_condensed_rhs(torch.tensor(F, device="cuda")).cpu().numpy()
    import scipy.linalg as sla
    ro = np.zeros_like(lam)
    for e, bl in enumerate(prob.blocks):
        g = -bl.C @ sla.lu_solve(cond.lu[e], vd.field(prob, F, e))
        for a in range(4):
            f = prob.sk.elem_face[e, a]
            if not prob.sk.boundary[f]:
                ro[prob.t_off[f]:prob.t_off[f + 1]] += g[bl.loc_off[a]:bl.loc_off[a + 1]]
    assert relerr(r, ro) < 1e-12
    u = s.hdg_recover(torch.tensor(F, device="cuda"), torch.tensor(lam, device="cuda")).cpu().numpy()
    uo = np.concatenate([sla.lu_solve(cond.lu[e], vd.field(prob, F, e) - bl.B @ vd.local_traces(prob, e, lam))
                         for e, bl in enumerate(prob.blocks)])
    assert relerr(u, uo) < 1e-12


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("mixed", 1e-9), ("mixed16", 1e-9)])
def test_vardeg_dirk3_steps_match_oracle(prec, tol):
    import torch
    N, seed = 2, 5
    ks = inputs.element_degrees(6 * N ** 3, 1, 4, seed)
    assert set(ks.tolist()) == {1, 2, 3, 4}
    s, prob = pair(N, ks, prec)
    rng = np.random.default_rng(seed)
    u0 = rng.standard_normal(int(prob.u_off[-1]))
    dt, nst = 0.01, 2
    uo_steps = []
    vd.run_dirk3(prob, u0, dt, nst, on_step=lambda n, t, u, lam: uo_steps.append((u.copy(), lam.copy())))
    s.hdg_set_state(torch.tensor(u0, device="cuda"), 0.0)
    for n in range(nst):
        s.hdg_step(dt, "dirk3", 1)
        u, lam, t = s.hdg_get_state()
        assert relerr(u.cpu().numpy(), uo_steps[n][0]) < tol
        assert relerr(lam.cpu().numpy(), uo_steps[n][1]) < tol
    tun = s.hdg_get_tuning()
    assert tun["tuned"] == 1 and all(nth in (64, 128, 256) for nth in tun["local_threads"])
    assert tun["apply64_tile"][0] in (4, 8) and tun["apply64_tile"][1] in (4, 8, 16)


def test_uniform_degree_4_elastic_matches_uniform_oracle():
    """3D elastic k = 4 everywhere runs through the per-element-degree path."""
    import torch
    from paper_1807_00086_gb300 import hdg
    vert, elem = inputs.unit_cube_tet(1)
    ne = elem.shape[0]
    rho = inputs.loguniform(ne, 0.5, 2.0, 7)
    lam = inputs.lognormal(ne, 1.5, 0.5, 8)
    mu = inputs.lognormal(ne, 1.0, 0.5, 9)
    s = hdg.Solver(vert, elem, 4, 1.0, rho, lam=lam, mu=mu, rtol=1e-13)
    prob = el.build_problem(vert, elem, 4, rho, lam, mu)
    rng = np.random.default_rng(9)
    u0 = rng.standard_normal((ne, (3 + prob.nt) * prob.Np))
    uo, lo, _ = el.run_dirk3(prob, u0, 0.01, 2)
    s.hdg_set_state(torch.tensor(u0.ravel(), device="cuda"), 0.0)
    s.hdg_step(0.01, "dirk3", 2)
    u, lamg, t = s.hdg_get_state()
    assert relerr(u.cpu().numpy(), uo.ravel()) < 1e-11
    assert relerr(lamg.cpu().numpy(), lo.ravel()) < 1e-11
