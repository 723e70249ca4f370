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


def mixed_pair(dim, N, k, **kw):
    import torch
    from paper_1807_00086_gb300 import hdg
    s, prob, _ = make_pair(dim, N, k, **kw)
    vert, elem = mesh(dim, N)
    ne = elem.shape[0]
    sm = hdg.Solver(vert, elem, k, 1.0, inputs.loguniform(ne, 0.5, 2.0, kw.get("seed", 1) + 7),
                    inputs.loguniform(ne, 1.0, 3.0, kw.get("seed", 1)), prec="mixed", rtol=1e-12)
    return s, sm, prob, torch


@pytest.mark.parametrize("dim,N,k", [(2, 4, 2), (3, 2, 3), (3, 2, 1), (3, 1, 4)])
def test_mixed_trace_solve_matches_direct_solve(dim, N, k):
    import scipy.sparse.linalg as spla
    s, sm, prob, torch = mixed_pair(dim, N, k)
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


@pytest.mark.parametrize("scheme", ["bdf2", "dirk3"])
def test_mixed_3d_point_source_steps(scheme):
    dim, N, k = 3, 2, 3
    h = 1.0 / N
    src = [[0.5 + 0.3 * h, 0.5 + 0.3 * h, 0.5 + 0.3 * h]]
    s, sm, prob, torch = mixed_pair(dim, N, k, seed=4, sources=src, f0=10.0, t0=0.02)
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


def test_mixed_2d_standing_mode_backward_euler():
    import torch
    from paper_1807_00086_gb300 import hdg
    vert, elem = mesh(2, 16)
    ex = ac.standing_mode(2)
    k, dt, nsteps = 2, 0.01, 20
    s = hdg.Solver(vert, elem, k, 1.0, 1.0, 1.0, prec="mixed", rtol=1e-12)
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
    """Benchmark workload (196,608 tets): one BDF2 step from a random state, mixed vs FP64 path."""
    import torch
    from paper_1807_00086_gb300 import hdg
    w = inputs.acoustic_3d_workload()
    u0 = torch.tensor(inputs.random_state(w["elem"].shape[0], 80, 33), device="cuda")
    out = {}
    for prec in ("fp64", "mixed"):
        s = hdg.Solver(w["vert"], w["elem"], w["k"], w["tau"], w["rho"], w["c"], prec=prec, rtol=1e-12)
        s.hdg_set_sources(w["sources"], [1.0], w["f0"], w["t0"])
        s.hdg_set_state(u0, 0.0)
        info = s.hdg_step(2e-3, "bdf2", 2)
        u, lam, t = s.hdg_get_state()
        out[prec] = (u.cpu().numpy(), lam.cpu().numpy(), info)
        s.close()
        del s
        torch.cuda.empty_cache()
    assert relerr(out["mixed"][0], out["fp64"][0]) < 1e-9
    assert relerr(out["mixed"][1], out["fp64"][1]) < 1e-9
