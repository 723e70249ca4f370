"""Linear elastodynamics (Sec. 4.1, velocity / symmetric-stress form): CUDA path through
the C ABI against the FP64 elastic oracle. Clamped boundaries (v_hat = 0), element-wise
lognormal Lame parameters, s = 2 rho c_s. FP64 path <= 1e-11 (operators <= 1e-12),
mixed precision <= 1e-9, per step."""
import numpy as np
import pytest

from gpu_helpers import relerr
from oracle import elastic as el
from paper_1807_00086_gb300 import inputs

pytestmark = pytest.mark.gpu


def pair(dim, N, k, prec="fp64", seed=2):
    from paper_1807_00086_gb300 import hdg
    vert, elem = inputs.unit_square_tri(N) if dim == 2 else inputs.unit_cube_tet(N)
    ne = elem.shape[0]
    rho = inputs.loguniform(ne, 0.5, 2.0, seed + 5)
    lam = inputs.lognormal(ne, 1.5, 0.5, seed)
    mu = inputs.lognormal(ne, 1.0, 0.5, seed + 1)
    s = hdg.Solver(vert, elem, k, 1.0, rho, lam=lam, mu=mu, prec=prec, rtol=1e-13 if prec == "fp64" else 1e-12)
    prob = el.build_problem(vert, elem, k, rho, lam, mu)
    return s, prob


CASES = [(2, 3, 1), (2, 2, 2), (2, 2, 3), (2, 1, 4), (3, 2, 1), (3, 1, 2), (3, 1, 3)]


@pytest.mark.parametrize("dim,N,k", CASES)
def test_elastic_schur_blocks_match_oracle(dim, N, k):
    s, prob = pair(dim, N, k)
    for alpha in (0.9, 300.0):
        s.hdg_condense(alpha)
        S = s.hdg_get_schur().cpu().numpy()
        assert relerr(S, np.stack(el.condense(prob, alpha).S)) < 1e-12


@pytest.mark.parametrize("dim,N,k", CASES)
def test_elastic_operators_match_oracle(dim, N, k):
    import torch
    s, prob = pair(dim, N, k)
    alpha = 13.0
    s.hdg_condense(alpha)
    cond = el.condense(prob, alpha)
    mf = s.Nf
    interior = cond.interior
    lam = inputs.random_traces(s.n_faces, mf, 4)
    lam[prob.sk.boundary] = 0.0
    y = s.hdg_trace_apply(torch.tensor(lam, device="cuda")).cpu().numpy()
    yo = np.zeros_like(lam)
    yo[interior] = (cond.K @ lam[interior].ravel()).reshape(-1, mf)
    assert relerr(y, yo) < 1e-12
    F = inputs.random_state(s.n_elem, s.n, 5)
    Ft = torch.tensor(F, device="cuda")
    r = s.hdg_condensed_rhs(Ft).cpu().numpy()
    import scipy.linalg as sla
    ro = np.zeros_like(lam)
    for e, bl in enumerate(prob.blocks):
        g = -bl.C @ sla.lu_solve(cond.lu[e], F[e])
        for a in range(dim + 1):
            f = prob.sk.elem_face[e, a]
            if not prob.sk.boundary[f]:
                ro[f] += g[a * mf:(a + 1) * mf]
    assert relerr(r, ro) < 1e-12
    u = s.hdg_recover(Ft, torch.tensor(lam, device="cuda")).cpu().numpy()
    uo = np.stack([sla.lu_solve(cond.lu[e], F[e] - bl.B @ el.local_traces(prob, e, lam)) for e, bl in enumerate(prob.blocks)])
    assert relerr(u, uo) < 1e-12


@pytest.mark.parametrize("dim,N,k,scheme,prec", [(3, 2, 2, "bdf2", "fp64"), (2, 3, 3, "dirk3", "fp64"),
                                                  (3, 1, 3, "dirk3", "fp64"), (3, 2, 2, "dirk3", "mixed"),
                                                  (2, 3, 2, "bdf2", "mixed")])
def test_elastic_steps_match_oracle(dim, N, k, scheme, prec):
    import torch
    s, prob = pair(dim, N, k, prec)
    u0 = inputs.random_state(s.n_elem, s.n, 7)
    s.hdg_set_state(torch.tensor(u0, device="cuda"), 0.0)
    dt, nsteps = 1e-3, 4
    ref = []
    cb = lambda n, t, u, lam: ref.append((u.copy(), lam.copy()))
    if scheme == "bdf2":
        el.run_bdf(prob, u0, dt, nsteps, 2, on_step=cb)
    else:
        el.run_dirk3(prob, u0, dt, nsteps, on_step=cb)
    tol = 1e-11 if prec == "fp64" else 1e-9
    for n in range(nsteps):
        s.hdg_step(dt, scheme, 1)
        u, lam, t = s.hdg_get_state()
        assert relerr(u.cpu().numpy(), ref[n][0]) < tol, n
        assert relerr(lam.cpu().numpy(), ref[n][1]) < tol, n
