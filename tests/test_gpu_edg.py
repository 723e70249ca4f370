"""Continuous trace spaces on the GPU (Sec. 2.2, Eq. e:spaces2): IEDG (continuous on interior
faces) and EDG (continuous on all faces, boundary nodes fixed), CUDA path through the C ABI
against oracle/edg.py (the Galerkin restriction R^T K R mu = R^T r of the HDG trace system).

Bars: FP64 path <= 1e-11 relative on traces and fields, mixed precision <= 1e-9."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from gpu_helpers import dirichlet_profile, mesh, relerr
from oracle import acoustic as ac
from oracle import edg
from paper_1807_00086_gb300 import inputs

pytestmark = pytest.mark.gpu

PRECS = [("fp64", 1e-11, None), ("mixed", 1e-9, None), ("mixed16", 1e-9, 1e-3)]


def _pair(dim, N, k, variant, prec, inner=None, seed=3, dirichlet=False, source=None):
    from paper_1807_00086_gb300 import hdg
    vert, elem = mesh(dim, N)
    ne = elem.shape[0]
    rho = inputs.loguniform(ne, 0.5, 2.0, seed + 7)
    c = inputs.loguniform(ne, 1.0, 3.0, seed)
    s = hdg.Solver(vert, elem, k, 1.0, rho, c, prec=prec, rtol=1e-13 if prec == "fp64" else 1e-12,
                   inner_rtol=inner, trace_space=variant)
    prob = ac.build_problem(vert, elem, k, 1.0, rho, c)
    if dirichlet:
        xb = s.hdg_quadrature_points(1)
        s.hdg_set_dirichlet(np.stack([dirichlet_profile(x) for x in xb]), 3.0, 0.2)
        prob.dirichlet = lambda x, t: dirichlet_profile(x) * np.cos(3.0 * t + 0.2)
    if source is not None:
        s.hdg_set_sources([source], [1.0], 10.0, 0.02)
        ac.add_point_source(prob, source, 10.0, 0.02)
    return s, prob


@pytest.mark.parametrize("prec,tol,inner", PRECS)
@pytest.mark.parametrize("variant", ["iedg", "edg"])
@pytest.mark.parametrize("dim,N,k", [(2, 4, 2), (3, 2, 3), (3, 2, 1), (3, 1, 4)])
def test_restricted_trace_solve_matches_oracle(dim, N, k, variant, prec, tol, inner):
    import torch
    s, prob = _pair(dim, N, k, variant, prec, inner)
    tm = edg.trace_map(prob, variant)
    assert s.sizes.trace_unknowns == tm.n_free
    alpha = 40.0
    s.hdg_condense(alpha)
    cond = ac.condense(prob, alpha)
    r = inputs.random_traces(s.n_faces, s.Nf, 12)
    r[prob.sk.boundary] = 0.0
    lam = torch.zeros((s.n_faces, s.Nf), dtype=torch.float64, device="cuda")
    info = s.hdg_trace_solve(torch.tensor(r, device="cuda"), lam)
    Kr = (tm.R.T @ cond.K @ tm.R).tocsc()
    mu = spla.spsolve(Kr, tm.R.T @ r[cond.interior].ravel())
    lo = np.zeros_like(r)
    lo[cond.interior] = (tm.R @ mu).reshape(-1, s.Nf)
    assert info["rel_residual"] <= (1e-13 if prec == "fp64" else 1e-12)
    assert relerr(lam.cpu().numpy(), lo) < tol


@pytest.mark.parametrize("prec,tol,inner", PRECS)
@pytest.mark.parametrize("scheme", ["bdf2", "dirk3"])
def test_iedg_steps_with_dirichlet_data_and_source(scheme, prec, tol, inner):
    import torch
    dim, N, k = 3, 2, 3
    s, prob = _pair(dim, N, k, "iedg", prec, inner, seed=4, dirichlet=True, source=[0.65, 0.65, 0.65])
    tm = edg.trace_map(prob, "iedg")
    solve = edg.make_stage_solver(tm)
    u0 = inputs.random_state(s.n_elem, s.n, 21)
    dt, nsteps = 2e-3, 5
    ref = []
    cb = lambda n, t, u, lam: ref.append((u.copy(), lam.copy()))
    if scheme == "bdf2":
        ac.run_bdf(prob, u0, dt, nsteps, 2, on_step=cb, solve=solve)
    else:
        ac.run_dirk3(prob, u0, dt, nsteps, on_step=cb, solve=solve)
    s.hdg_set_state(torch.tensor(u0, device="cuda"), 0.0)
    for n in range(nsteps):
        s.hdg_step(dt, scheme, 1)
        u, lam, t = s.hdg_get_state()
        assert relerr(u.cpu().numpy(), ref[n][0]) < tol, n
        assert relerr(lam.cpu().numpy(), ref[n][1]) < tol, n


@pytest.mark.parametrize("prec,tol,inner", PRECS)
@pytest.mark.parametrize("dim,N,k", [(2, 4, 2), (3, 2, 3)])
def test_edg_bdf2_steps_match_oracle(dim, N, k, prec, tol, inner):
    import torch
    src = [0.41, 0.37, 0.33][:dim]
    s, prob = _pair(dim, N, k, "edg", prec, inner, seed=5, source=src)
    tm = edg.trace_map(prob, "edg")
    u0 = inputs.random_state(s.n_elem, s.n, 22)
    dt, nsteps = 2e-3, 5
    ref = []
    ac.run_bdf(prob, u0, dt, nsteps, 2, on_step=lambda n, t, u, lam: ref.append((u.copy(), lam.copy())),
               solve=edg.make_stage_solver(tm))
    s.hdg_set_state(torch.tensor(u0, device="cuda"), 0.0)
    for n in range(nsteps):
        s.hdg_step(dt, "bdf2", 1)
        u, lam, t = s.hdg_get_state()
        assert relerr(u.cpu().numpy(), ref[n][0]) < tol, n
        assert relerr(lam.cpu().numpy(), ref[n][1]) < tol, n


def test_continuous_traces_need_fewer_krylov_iterations_than_hdg():
    """The restricted systems converge in fewer Jacobi-CG iterations at the benchmark's
    c dt / h (dt scaled with h from the 32^3 x 6 mesh), the same finding as the CPU study of
    the oracle's operators; at much smaller c dt / h HDG's face Jacobi is the better one."""
    import torch
    N = 6
    w = inputs.acoustic_3d_workload(N=N)
    its = {}
    for variant in ("hdg", "iedg", "edg"):
        from paper_1807_00086_gb300 import hdg
        s = hdg.Solver(w["vert"], w["elem"], w["k"], w["tau"], w["rho"], w["c"], rtol=1e-12, trace_space=variant,
                       guess_history=0)
        s.hdg_condense(1.5 / (2e-3 * 32.0 / N))
        r = inputs.random_traces(s.n_faces, s.Nf, 3)
        r[np.asarray(ac.skeleton(w["elem"]).boundary)] = 0.0
        lam = torch.zeros((s.n_faces, s.Nf), dtype=torch.float64, device="cuda")
        its[variant] = s.hdg_trace_solve(torch.tensor(r, device="cuda"), lam)["iterations"]
    assert its["iedg"] < its["hdg"] and its["edg"] < its["hdg"], its


def test_edg_rejects_nonzero_dirichlet_data_and_unsupported_configurations():
    from paper_1807_00086_gb300 import hdg
    vert, elem = mesh(2, 2)
    s = hdg.Solver(vert, elem, 2, 1.0, 1.0, 1.0, trace_space="edg")
    xb = s.hdg_quadrature_points(1)
    with pytest.raises(hdg.HDGError):
        s.hdg_set_dirichlet(np.ones(xb.shape[:2]), 1.0, 0.0)
    with pytest.raises(hdg.HDGError):
        hdg.Solver(vert, elem, 2, 1.0, 1.0, 1.0, trace_space="iedg", nrhs=4)
    with pytest.raises(hdg.HDGError):
        hdg.Solver(vert, elem, 2, 1.0, 1.0, 1.0, trace_space="iedg", device_loops=False)
