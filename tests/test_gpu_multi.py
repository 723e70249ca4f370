"""Multiple right-hand sides (nrhs = R columns sharing every S_K) against the oracle.

Each column is an independent wave problem with its own point source and initial state;
column j of the batched GPU solve must match the oracle's single-column run for that
source and state (FP64 path <= 1e-11, mixed precision <= 1e-9, per step).
"""
import numpy as np
import pytest

from gpu_helpers import dirichlet_profile, mesh, relerr
from oracle import acoustic as ac
from paper_1807_00086_gb300 import inputs

pytestmark = pytest.mark.gpu


def _setup(prec, R, dim=3, N=2, k=2, seed=3):
    import torch
    from paper_1807_00086_gb300 import hdg
    vert, elem = mesh(dim, N)
    ne = elem.shape[0]
    rho = inputs.loguniform(ne, 0.5, 2.0, seed + 7)
    c = inputs.loguniform(ne, 1.0, 3.0, seed)
    s = hdg.Solver(vert, elem, k, 1.0, rho, c, prec=prec, rtol=1e-12, nrhs=R)
    xb = s.hdg_quadrature_points(1)
    s.hdg_set_dirichlet(np.stack([dirichlet_profile(x) for x in xb]), 3.0, 0.2)
    pos = inputs.uniform_points(R, dim, 0.1, 0.9, seed + 1)
    s.hdg_set_sources(pos, np.linspace(1.0, 2.0, R), 10.0, 0.02, col=np.arange(R))
    u0 = inputs.random_state(ne, s.n * R, seed + 2).reshape(ne, s.n, R)
    s.hdg_set_state(torch.tensor(u0, device="cuda"), 0.0)
    prob = ac.build_problem(vert, elem, k, 1.0, rho, c)
    prob.dirichlet = lambda x, t: dirichlet_profile(x) * np.cos(3.0 * t + 0.2)
    return s, prob, pos, u0


@pytest.mark.parametrize("R", [2, 4, 8, 32, 64])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("mixed", 1e-9)])
def test_multi_source_batch_matches_single_column_oracle(prec, tol, R):
    """R < 32 runs the narrow kernels (several elements per warp), R = 32 the wide ones with
    one column group, R = 64 (the multi-source workload's width) two column groups. In the
    mixed path R = 2 keeps the one-column-per-thread Krylov vector kernels and R = 4, 8, 32, 64
    take the four-columns-per-thread ones (R = 4: one column group per thread)."""
    dt, nsteps = 2e-3, 3
    s, prob, pos, u0 = _setup(prec, R)
    amps = np.linspace(1.0, 2.0, R)
    for n in range(nsteps):
        info = s.hdg_step(dt, "bdf2", 1)
    u, lam, t = s.hdg_get_state()
    u, lam = u.cpu().numpy(), lam.cpu().numpy()
    for j in range(R):
        prob.sources = []
        ac.add_point_source(prob, pos[j], 10.0, 0.02, amp=amps[j])
        uo, lo, to = ac.run_bdf(prob, u0[:, :, j], dt, nsteps, 2)
        assert relerr(u[:, :, j], uo) < tol, j
        assert relerr(lam[:, :, j], lo) < tol, j


def test_multi_operators_match_oracle_per_column():
    import torch
    R = 4
    s, prob, pos, u0 = _setup("fp64", R)
    alpha = 11.0
    s.hdg_condense(alpha)
    cond = ac.condense(prob, alpha)
    lam = inputs.random_traces(s.n_faces, s.Nf * R, 5).reshape(s.n_faces, s.Nf, R)
    y = s.hdg_trace_apply(torch.tensor(lam, device="cuda")).cpu().numpy()
    F = inputs.random_state(s.n_elem, s.n * R, 6).reshape(s.n_elem, s.n, R)
    Ft = torch.tensor(F, device="cuda")
    r = s.hdg_condensed_rhs(Ft).cpu().numpy()
    u = s.hdg_recover(Ft, torch.tensor(lam, device="cuda")).cpu().numpy()
    for j in range(R):
        yo = np.zeros((s.n_faces, s.Nf))
        yo[cond.interior] = ac.trace_apply(prob, cond, lam[cond.interior, :, j].ravel()).reshape(-1, s.Nf)
        assert relerr(y[:, :, j], yo) < 1e-12
        ro = np.zeros((s.n_faces, s.Nf))
        ro[cond.interior] = ac.condensed_rhs(prob, cond, F[:, :, j]).reshape(-1, s.Nf)
        assert relerr(r[:, :, j], ro) < 1e-12
        assert relerr(u[:, :, j], ac.recover(prob, cond, F[:, :, j], lam[:, :, j])) < 1e-12
