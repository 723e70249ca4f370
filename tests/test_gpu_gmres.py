"""Restarted GMRES with iterated classical Gram-Schmidt (the paper's Krylov method, Sec. 2.4) on
the GPU, through the C ABI, against the oracle's direct solve and per-step fields.

Bar: FP64, <= 1e-11 relative on traces and fields (rtol 1e-13)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from gpu_helpers import make_pair, mesh, relerr
from oracle import acoustic as ac
from paper_1807_00086_gb300 import inputs

pytestmark = pytest.mark.gpu


def _solver(dim, N, k, seed=1, **kw):
    from paper_1807_00086_gb300 import hdg
    vert, elem = mesh(dim, N)
    ne = elem.shape[0]
    return hdg.Solver(vert, elem, k, 1.0, inputs.loguniform(ne, 0.5, 2.0, seed + 7), inputs.loguniform(ne, 1.0, 3.0, seed),
                      solver="gmres", **kw)


@pytest.mark.parametrize("restart", [40, 5])
@pytest.mark.parametrize("dim,N,k", [(2, 4, 2), (3, 2, 3), (3, 1, 4)])
def test_gmres_trace_solve_matches_direct_solve(dim, N, k, restart):
    import torch
    _, prob, _ = make_pair(dim, N, k, dirichlet=False)
    s = _solver(dim, N, k, gmres_restart=restart)
    for alpha in (40.0, 2.0):
        s.hdg_condense(alpha)
        cond = ac.condense(prob, alpha)
        r = inputs.random_traces(s.n_faces, s.Nf, 12)
        r[prob.sk.boundary] = 0.0
        lam = torch.zeros((s.n_faces, s.Nf), dtype=torch.float64, device="cuda")
        info = s.hdg_trace_solve(torch.tensor(r, device="cuda"), lam)
        lo = np.zeros_like(r)
        lo[cond.interior] = spla.spsolve(cond.K.tocsc(), r[cond.interior].ravel()).reshape(-1, s.Nf)
        assert info["rel_residual"] <= 1e-13 and info["iterations"] > 0
        if restart == 5:
            assert info["sweeps"] > 1          # restarted
        assert relerr(lam.cpu().numpy(), lo) < 1e-11


@pytest.mark.parametrize("scheme", ["bdf2", "dirk3"])
def test_gmres_steps_match_oracle(scheme):
    import torch
    dim, N, k = 3, 2, 3
    s0, prob, _ = make_pair(dim, N, k, seed=4, sources=[[0.65, 0.65, 0.65]], f0=10.0, t0=0.02)
    s = _solver(dim, N, k, seed=4)
    from gpu_helpers import dirichlet_profile
    xb = s.hdg_quadrature_points(1)
    s.hdg_set_dirichlet(np.stack([dirichlet_profile(x) for x in xb]), 3.0, 0.2)
    s.hdg_set_sources([[0.65, 0.65, 0.65]], [1.0], 10.0, 0.02)
    u0 = inputs.random_state(s.n_elem, s.n, 21)
    s.hdg_set_state(torch.tensor(u0, device="cuda"), 0.0)
    dt, nsteps = 2e-3, 4
    ref = []
    cb = lambda n, t, u, lam: ref.append((u.copy(), lam.copy()))
    if scheme == "bdf2":
        ac.run_bdf(prob, u0, dt, nsteps, 2, on_step=cb)
    else:
        ac.run_dirk3(prob, u0, dt, nsteps, on_step=cb)
    for n in range(nsteps):
        info = s.hdg_step(dt, scheme, 1)
        assert info["rel_residual"] <= 1e-13
        u, lam, t = s.hdg_get_state()
        assert relerr(u.cpu().numpy(), ref[n][0]) < 1e-11, n
        assert relerr(lam.cpu().numpy(), ref[n][1]) < 1e-11, n


def test_gmres_rejects_unsupported_configurations():
    from paper_1807_00086_gb300 import hdg
    vert, elem = mesh(2, 2)
    for kw in ({"prec": "mixed"}, {"nrhs": 4}, {"trace_space": "iedg"}, {"gmres_restart": 1}, {"gmres_restart": 65}):
        with pytest.raises(hdg.HDGError):
            hdg.Solver(vert, elem, 2, 1.0, 1.0, 1.0, solver="gmres", **kw)
