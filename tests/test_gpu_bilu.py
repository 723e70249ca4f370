"""Block ILU(0) preconditioner of the GMRES trace solve (Sec. 2.4) on the GPU, through the C
ABI, against oracle/bilu.py on the oracle's own trace operator.

* the preconditioner itself: z = (L U)^{-1} r element by element against the oracle's ILU(0)
  of -K (FP64, <= 1e-11 relative);
* GMRES + block ILU(0) trace solves against the direct solve (<= 1e-11), in fewer iterations
  than GMRES + Jacobi at the benchmark's c dt / h;
* BDF2 steps with it against the oracle's per-step fields (<= 1e-11).
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from gpu_helpers import make_pair, mesh, relerr
from oracle import acoustic as ac
from oracle import bilu
from paper_1807_00086_gb300 import inputs

pytestmark = pytest.mark.gpu


def _solver(dim, N, k, precond="bilu0", seed=1, **kw):
    from paper_1807_00086_gb300 import hdg
    vert, elem = mesh(dim, N)
    ne = elem.shape[0]
    return hdg.Solver(vert, elem, k, 1.0, inputs.loguniform(ne, 0.5, 2.0, seed + 7), inputs.loguniform(ne, 1.0, 3.0, seed),
                      solver="gmres", precond=precond, **kw)


@pytest.mark.parametrize("dim,N,k", [(2, 4, 2), (3, 2, 3), (3, 2, 1)])
def test_bilu0_preconditioner_matches_oracle(dim, N, k):
    import torch
    _, prob, _ = make_pair(dim, N, k, dirichlet=False)
    s = _solver(dim, N, k)
    alpha = 1.5 / (2e-3 * 32.0 / N)
    s.hdg_condense(alpha)
    cond = ac.condense(prob, alpha)
    A = (-cond.K).toarray()
    interior = ~np.asarray(prob.sk.boundary)
    ids = np.asarray(cond.interior)
    where = {int(f): t for t, f in enumerate(ids)}
    Nf = s.Nf
    rows, cols = bilu.pattern_from_skeleton(prob.sk.elem_face, interior)
    blocks = bilu.assemble_blocks(rows, cols, lambda i, j: A[where[i] * Nf:(where[i] + 1) * Nf,
                                                             where[j] * Nf:(where[j] + 1) * Nf])
    F, Dinv = bilu.factor(rows, cols, blocks)
    r = inputs.random_traces(s.n_faces, Nf, 5)
    zo = bilu.solve(rows, cols, F, Dinv, {f: r[f] for f in rows})
    z = s.hdg_precond_apply(torch.tensor(r, device="cuda")).cpu().numpy()
    ref = np.zeros_like(r)
    for f in rows:
        ref[f] = zo[f]
    assert relerr(z, ref) < 1e-11
    assert np.all(z[~interior] == 0.0)


@pytest.mark.parametrize("dim,N,k", [(2, 4, 2), (3, 2, 3)])
def test_gmres_bilu0_trace_solve_matches_direct_solve_in_fewer_iterations(dim, N, k):
    import torch
    _, prob, _ = make_pair(dim, N, k, dirichlet=False)
    alpha = 1.5 / (2e-3 * 32.0 / N)
    cond = ac.condense(prob, alpha)
    its = {}
    for pc in ("jacobi", "bilu0"):
        s = _solver(dim, N, k, precond=pc)
        s.hdg_condense(alpha)
        r = inputs.random_traces(s.n_faces, s.Nf, 12)
        r[prob.sk.boundary] = 0.0
        lam = torch.zeros((s.n_faces, s.Nf), dtype=torch.float64, device="cuda")
        info = s.hdg_trace_solve(torch.tensor(r, device="cuda"), lam)
        lo = np.zeros_like(r)
        lo[cond.interior] = spla.spsolve(cond.K.tocsc(), r[cond.interior].ravel()).reshape(-1, s.Nf)
        assert info["rel_residual"] <= 1e-13
        assert relerr(lam.cpu().numpy(), lo) < 1e-11
        its[pc] = info["iterations"]
    assert its["bilu0"] < 0.7 * its["jacobi"], its


def test_gmres_bilu0_bdf2_steps_match_oracle():
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
    ac.run_bdf(prob, u0, dt, nsteps, 2, on_step=lambda n, t, u, lam: ref.append((u.copy(), lam.copy())))
    for n in range(nsteps):
        info = s.hdg_step(dt, "bdf2", 1)
        assert info["rel_residual"] <= 1e-13
        u, lam, t = s.hdg_get_state()
        assert relerr(u.cpu().numpy(), ref[n][0]) < 1e-11, n
        assert relerr(lam.cpu().numpy(), ref[n][1]) < 1e-11, n


def test_bilu0_needs_the_gmres_solver():
    from paper_1807_00086_gb300 import hdg
    vert, elem = mesh(2, 2)
    with pytest.raises(hdg.HDGError):
        hdg.Solver(vert, elem, 2, 1.0, 1.0, 1.0, precond="bilu0")
