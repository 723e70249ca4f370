"""Element-local post-processing of the pressure into P_{k+1}: CUDA path through the C ABI
against the oracle's postprocess_pressure, element by element (FP64 both sides, <= 1e-12).

Inputs are seeded random fields and traces (boundary entries included: they stand for the
Dirichlet trace), so every term of the local problem is exercised; at the benchmark size
(196,608 tets, k = 3) sampled elements are compared through an oracle problem built on
those elements alone (the step is element-local)."""
import numpy as np
import pytest

from gpu_helpers import mesh, relerr
from oracle import acoustic as ac
from paper_1807_00086_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dim,N,k", [(2, 3, 1), (2, 2, 2), (2, 2, 3), (2, 1, 4), (3, 1, 1), (3, 2, 2), (3, 1, 3),
                                     (3, 1, 4)])
def test_postprocess_matches_oracle(dim, N, k):
    import torch
    from paper_1807_00086_gb300 import hdg
    vert, elem = mesh(dim, N)
    ne = elem.shape[0]
    rho = inputs.loguniform(ne, 0.5, 2.0, 3)
    c = inputs.loguniform(ne, 1.0, 3.0, 4)
    s = hdg.Solver(vert, elem, k, 1.0, rho, c)
    prob = ac.build_problem(vert, elem, k, 1.0, rho, c)
    u = inputs.random_state(ne, s.n, 10 * dim + k)
    lam = inputs.random_traces(s.n_faces, s.Nf, 20 * dim + k)
    ps = s.hdg_postprocess(torch.tensor(u, device="cuda"), torch.tensor(lam, device="cuda")).cpu().numpy()
    po = ac.postprocess_pressure(prob, u, lam)
    assert ps.shape == po.shape
    assert relerr(ps, po) < 1e-12


def test_postprocess_of_solver_state_matches_oracle_and_superconverges():
    """After DIRK3 steps of the 2D standing mode the GPU's p* equals the oracle's p* of the
    oracle's own solution, and is closer to the exact pressure than p_h."""
    import torch
    from paper_1807_00086_gb300 import hdg
    k, N, T, nst = 2, 8, 0.2, 64
    ex = ac.standing_mode(2)
    vert, elem = mesh(2, N)
    s = hdg.Solver(vert, elem, k, 1.0, 1.0, 1.0)
    prob = ac.build_problem(vert, elem, k, 1.0, 1.0, 1.0)
    prob.dirichlet = lambda x, t: ex(x, t)[:, 0]
    u0 = ac.project_volume(prob, lambda x: ex(x, 0.0))
    xb = s.hdg_quadrature_points(1)
    # p_D(x, t) = cos(pi x) cos(pi y) cos(sqrt(2) pi t): profile times cos(omega t + 0)
    s.hdg_set_dirichlet(np.stack([ex(xb[b], 0.0)[:, 0] for b in range(xb.shape[0])]), np.sqrt(2.0) * np.pi, 0.0)
    s.hdg_set_state(torch.tensor(u0, device="cuda"), 0.0)
    s.hdg_step(T / nst, "dirk3", nst)
    u, lam, t = s.hdg_get_state()
    ps = s.hdg_postprocess(u, lam).cpu().numpy()
    uo, lo, _ = ac.run_dirk3(prob, u0, T / nst, nst)
    po = ac.postprocess_pressure(prob, uo, lo)
    assert relerr(ps, po) < 1e-9
    e_post = ac.l2_error_post(prob, ps, lambda x: ex(x, T))
    e_h = ac.l2_error(prob, u.cpu().numpy(), lambda x: ex(x, T))
    assert e_post < 0.2 * e_h, (e_post, e_h)


def test_postprocess_full_size_sampled():
    import torch
    from paper_1807_00086_gb300 import hdg
    w = inputs.acoustic_3d_workload()
    vert, elem, k = w["vert"], w["elem"], w["k"]
    ne = elem.shape[0]
    s = hdg.Solver(vert, elem, k, w["tau"], w["rho"], w["c"])
    u = inputs.random_state(ne, s.n, 41)
    lam = inputs.random_traces(s.n_faces, s.Nf, 42)
    ps = s.hdg_postprocess(torch.tensor(u, device="cuda"), torch.tensor(lam, device="cuda")).cpu().numpy()
    assert np.isfinite(ps).all() and np.array_equal(ps[:, 0], u[:, 0])
    rng = np.random.default_rng(43)
    sample = np.unique(np.concatenate([[0, ne - 1], rng.integers(0, ne, 14)]))
    sk = ac.skeleton(elem)
    fid = {tuple(f): i for i, f in enumerate(sk.faces.tolist())}
    sub = ac.build_problem(vert, elem[sample], k, w["tau"], w["rho"][sample], w["c"][sample])
    lam_sub = np.stack([lam[fid[tuple(f)]] for f in sub.sk.faces.tolist()])
    po = ac.postprocess_pressure(sub, u[sample], lam_sub)
    assert relerr(ps[sample], po) < 1e-12
