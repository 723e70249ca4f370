"""Mixed precision (FP32 S_K inside FP64 iterative refinement) against the FP64 oracle.

Bar: <= 1e-9 relative (max norm) on fields and traces per step; the refinement stops at
an FP64 relative trace residual of rtol = 1e-12.
"""
import math

import numpy as np
import pytest

from gpu_helpers import make_pair, mesh, relerr
from oracle import acoustic as ac
from paper_1807_00086_gb300 import inputs

pytestmark = pytest.mark.gpu


def mixed_pair(dim, N, k, prec="mixed", inner_rtol=None, max_sweeps=None, **kw):
    import torch
    from paper_1807_00086_gb300 import hdg
    s, prob, _ = make_pair(dim, N, k, **kw)
    vert, elem = mesh(dim, N)
    ne = elem.shape[0]
    sm = hdg.Solver(vert, elem, k, 1.0, inputs.loguniform(ne, 0.5, 2.0, kw.get("seed", 1) + 7),
                    inputs.loguniform(ne, 1.0, 3.0, kw.get("seed", 1)), prec=prec, rtol=1e-12,
                    inner_rtol=inner_rtol, max_sweeps=max_sweeps)
    return s, sm, prob, torch


# the FP16 operator (HDG_MIXED16) runs with the benchmark's inner tolerance 1e-3
PRECS = [("mixed", None), ("mixed16", 1e-3)]


@pytest.mark.parametrize("prec,inner", PRECS)
@pytest.mark.parametrize("dim,N,k", [(2, 4, 2), (3, 2, 3), (3, 2, 1), (3, 1, 4)])
def test_mixed_trace_solve_matches_direct_solve(dim, N, k, prec, inner):
    import scipy.sparse.linalg as spla
    s, sm, prob, torch = mixed_pair(dim, N, k, prec=prec, inner_rtol=inner)
    sm.hdg_condense(40.0)
    cond = ac.condense(prob, 40.0)
    r = inputs.random_traces(sm.n_faces, sm.Nf, 12)
    r[prob.sk.boundary] = 0.0
    lam = torch.zeros((sm.n_faces, sm.Nf), dtype=torch.float64, device="cuda")
    info = sm.hdg_trace_solve(torch.tensor(r, device="cuda"), lam)
    lo = np.zeros_like(r)
    lo[cond.interior] = spla.spsolve(cond.K.tocsc(), r[cond.interior].ravel()).reshape(-1, sm.Nf)
    assert info["rel_residual"] <= 1e-12 and info["sweeps"] >= 1
    assert relerr(lam.cpu().numpy(), lo) < 1e-10


@pytest.mark.parametrize("prec,inner", PRECS)
@pytest.mark.parametrize("scheme", ["bdf2", "dirk3"])
def test_mixed_3d_point_source_steps(scheme, prec, inner):
    dim, N, k = 3, 2, 3
    h = 1.0 / N
    src = [[0.5 + 0.3 * h, 0.5 + 0.3 * h, 0.5 + 0.3 * h]]
    s, sm, prob, torch = mixed_pair(dim, N, k, prec=prec, inner_rtol=inner, seed=4, sources=src, f0=10.0, t0=0.02)
    from gpu_helpers import dirichlet_profile
    xb = sm.hdg_quadrature_points(1)
    sm.hdg_set_dirichlet(np.stack([dirichlet_profile(x) for x in xb]), 3.0, 0.2)
    sm.hdg_set_sources(src, [1.0], 10.0, 0.02)
    u0 = inputs.random_state(sm.n_elem, sm.n, 21)
    sm.hdg_set_state(torch.tensor(u0, device="cuda"), 0.0)
    dt, nsteps = 2e-3, 6
    ref = []
    cb = lambda n, t, u, lam: ref.append((u.copy(), lam.copy()))
    if scheme == "bdf2":
        ac.run_bdf(prob, u0, dt, nsteps, 2, on_step=cb)
    else:
        ac.run_dirk3(prob, u0, dt, nsteps, on_step=cb)
    for n in range(nsteps):
        info = sm.hdg_step(dt, scheme, 1)
        u, lam, t = sm.hdg_get_state()
        assert relerr(u.cpu().numpy(), ref[n][0]) < 1e-9, n
        assert relerr(lam.cpu().numpy(), ref[n][1]) < 1e-9, n
        assert info["rel_residual"] <= 1e-12


@pytest.mark.parametrize("prec,inner", PRECS)
def test_mixed_2d_standing_mode_backward_euler(prec, inner):
    import torch
    from paper_1807_00086_gb300 import hdg
    vert, elem = mesh(2, 16)
    ex = ac.standing_mode(2)
    k, dt, nsteps = 2, 0.01, 20
    s = hdg.Solver(vert, elem, k, 1.0, 1.0, 1.0, prec=prec, rtol=1e-12, inner_rtol=inner)
    xb = s.hdg_quadrature_points(1)
    s.hdg_set_dirichlet(np.stack([np.cos(np.pi * x[:, 0]) * np.cos(np.pi * x[:, 1]) for x in xb]),
                        math.sqrt(2) * math.pi, 0.0)
    xv = s.hdg_quadrature_points(0)
    s.hdg_set_state(s.hdg_project_volume(np.stack([ex(x, 0.0) for x in xv])), 0.0)
    prob = ac.build_problem(vert, elem, k, 1.0, 1.0, 1.0)
    prob.dirichlet = lambda x, t: ex(x, t)[:, 0]
    ref = []
    ac.run_bdf(prob, ac.project_volume(prob, lambda x: ex(x, 0.0)), dt, nsteps, 1,
               on_step=lambda n, t, u, lam: ref.append((u.copy(), lam.copy())))
    for n in range(nsteps):
        s.hdg_step(dt, "be", 1)
        u, lam, t = s.hdg_get_state()
        assert relerr(u.cpu().numpy(), ref[n][0]) < 1e-9, n
        assert relerr(lam.cpu().numpy(), ref[n][1]) < 1e-9, n


def test_mixed_full_size_step_matches_fp64_path():
    """Benchmark workload (196,608 tets, the launch configuration bench.py times): two BDF2
    steps from a random state with the FP32 and with the FP16 inner operator, each against the
    FP64 path."""
    import torch
    from paper_1807_00086_gb300 import hdg
    w = inputs.acoustic_3d_workload()
    u0 = torch.tensor(inputs.random_state(w["elem"].shape[0], 80, 33), device="cuda")
    out = {}
    for prec in ("fp64", "mixed", "mixed16"):
        s = hdg.Solver(w["vert"], w["elem"], w["k"], w["tau"], w["rho"], w["c"], prec=prec, rtol=1e-12,
                       inner_rtol=1e-3 if prec == "mixed16" else None)
        s.hdg_set_sources(w["sources"], [1.0], w["f0"], w["t0"])
        s.hdg_set_state(u0, 0.0)
        info = s.hdg_step(2e-3, "bdf2", 2)
        u, lam, t = s.hdg_get_state()
        out[prec] = (u.cpu().numpy(), lam.cpu().numpy(), info)
        s.close()
        del s
        torch.cuda.empty_cache()
    for prec in ("mixed", "mixed16"):
        assert relerr(out[prec][0], out["fp64"][0]) < 1e-9, prec
        assert relerr(out[prec][1], out["fp64"][1]) < 1e-9, prec
        assert out[prec][2]["rel_residual"] <= 1e-12


def test_mixed16_switches_to_fp32_operator_and_still_converges():
    """A refinement sweep of HDG_MIXED16 that gains less than a factor 10 switches the rest of
    the solve to the FP32 copy of S_K. An inner tolerance of 0.5 makes every sweep gain about
    2x, so the first check switches; the solve must still reach the FP64 solution."""
    import scipy.sparse.linalg as spla
    s, sm, prob, torch = mixed_pair(3, 2, 3, prec="mixed16", inner_rtol=0.5, max_sweeps=80)
    sm.hdg_condense(40.0)
    cond = ac.condense(prob, 40.0)
    r = inputs.random_traces(sm.n_faces, sm.Nf, 13)
    r[prob.sk.boundary] = 0.0
    lam = torch.zeros((sm.n_faces, sm.Nf), dtype=torch.float64, device="cuda")
    sm.hdg_enable_stats(True)
    sm.hdg_get_stats(reset=True)
    info = sm.hdg_trace_solve(torch.tensor(r, device="cuda"), lam)
    st = sm.hdg_get_stats(reset=True)
    lo = np.zeros_like(r)
    lo[cond.interior] = spla.spsolve(cond.K.tocsc(), r[cond.interior].ravel()).reshape(-1, sm.Nf)
    assert info["rel_residual"] <= 1e-12 and info["sweeps"] > 10
    assert st["apply16_launches"] > 0 and st["apply32_launches"] > 0
    assert relerr(lam.cpu().numpy(), lo) < 1e-10
