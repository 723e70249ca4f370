"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bar (FP64 path): <= 1e-11 relative (max-norm) on traces and fields per step; the
element-level operators (S_K, apply, condensed rhs, recovery) at <= 1e-12.
"""
import math

import numpy as np
import pytest

from gpu_helpers import make_pair, mesh, relerr
from oracle import acoustic as ac
from paper_1807_00086_gb300 import inputs

pytestmark = pytest.mark.gpu

CASES = [(2, 3, 1), (2, 3, 2), (2, 2, 3), (2, 2, 4), (3, 2, 1), (3, 2, 2), (3, 2, 3), (3, 1, 4)]


@pytest.mark.parametrize("dim,N,k", CASES)
def test_schur_blocks_match_oracle(dim, N, k):
    s, prob, torch = make_pair(dim, N, k)
    for alpha in (0.7, 250.0):
        s.hdg_condense(alpha)
        S = s.hdg_get_schur().cpu().numpy()
        cond = ac.condense(prob, alpha)
        So = np.stack(cond.S)
        assert relerr(S, So) < 1e-12


@pytest.mark.parametrize("dim,N,k", CASES)
def test_trace_apply_matches_oracle(dim, N, k):
    s, prob, torch = make_pair(dim, N, k)
    s.hdg_condense(3.0)
    cond = ac.condense(prob, 3.0)
    lam = inputs.random_traces(s.n_faces, s.Nf, 5)
    y = s.hdg_trace_apply(torch.tensor(lam, device="cuda")).cpu().numpy()
    yo = np.zeros_like(lam)
    yo[cond.interior] = ac.trace_apply(prob, cond, lam[cond.interior].ravel()).reshape(-1, s.Nf)
    assert relerr(y, yo) < 1e-12
    assert np.all(y[prob.sk.boundary] == 0)


@pytest.mark.parametrize("dim,N,k", CASES)
def test_condensed_rhs_and_recovery_match_oracle(dim, N, k):
    s, prob, torch = make_pair(dim, N, k)
    alpha = 11.0
    s.hdg_condense(alpha)
    cond = ac.condense(prob, alpha)
    F = inputs.random_state(s.n_elem, s.n, 6)
    lamD = inputs.random_traces(s.n_faces, s.Nf, 8)
    lamD[~prob.sk.boundary] = 0.0
    Ft = torch.tensor(F, device="cuda")
    r = s.hdg_condensed_rhs(Ft, torch.tensor(lamD, device="cuda")).cpu().numpy()
    Fo = np.stack([F[e] - bl.B @ ac.local_traces(prob, e, lamD) for e, bl in enumerate(prob.blocks)])
    ro = np.zeros_like(lamD)
    ro[cond.interior] = ac.condensed_rhs(prob, cond, Fo).reshape(-1, s.Nf)
    assert relerr(r, ro) < 1e-12
    lam = inputs.random_traces(s.n_faces, s.Nf, 9)
    u = s.hdg_recover(Ft, torch.tensor(lam, device="cuda")).cpu().numpy()
    uo = ac.recover(prob, cond, F, lam)
    assert relerr(u, uo) < 1e-12


@pytest.mark.parametrize("dim,N,k", [(2, 4, 2), (3, 2, 3)])
def test_trace_solve_matches_direct_solve(dim, N, k):
    import scipy.sparse.linalg as spla
    s, prob, torch = make_pair(dim, N, k)
    s.hdg_condense(40.0)
    cond = ac.condense(prob, 40.0)
    r = inputs.random_traces(s.n_faces, s.Nf, 12)
    r[prob.sk.boundary] = 0.0
    lam = torch.zeros((s.n_faces, s.Nf), dtype=torch.float64, device="cuda")
    info = s.hdg_trace_solve(torch.tensor(r, device="cuda"), lam)
    lo = np.zeros_like(r)
    lo[cond.interior] = spla.spsolve(cond.K.tocsc(), r[cond.interior].ravel()).reshape(-1, s.Nf)
    assert info["rel_residual"] <= 1e-13
    assert relerr(lam.cpu().numpy(), lo) < 1e-11


def test_acoustic_2d_standing_mode_backward_euler_50_steps():
    """2D acoustic, k = 2, tau = 1, rho = c = 1, 16x16 squares -> 512 triangles, BE dt = 0.01,
    50 steps, exact standing mode as initial and Dirichlet data: traces and fields per step."""
    import torch
    from paper_1807_00086_gb300 import hdg
    vert, elem = mesh(2, 16)
    ex = ac.standing_mode(2)
    k, dt, nsteps = 2, 0.01, 50
    s = hdg.Solver(vert, elem, k, 1.0, 1.0, 1.0)
    xb = s.hdg_quadrature_points(1)
    s.hdg_set_dirichlet(np.stack([np.cos(np.pi * x[:, 0]) * np.cos(np.pi * x[:, 1]) for x in xb]),
                        math.sqrt(2) * math.pi, 0.0)
    xv = s.hdg_quadrature_points(0)
    u0 = s.hdg_project_volume(np.stack([ex(x, 0.0) for x in xv]))
    s.hdg_set_state(u0, 0.0)
    prob = ac.build_problem(vert, elem, k, 1.0, 1.0, 1.0)
    prob.dirichlet = lambda x, t: ex(x, t)[:, 0]
    uo0 = ac.project_volume(prob, lambda x: ex(x, 0.0))
    assert relerr(u0.cpu().numpy(), uo0) < 1e-13
    ref = []
    ac.run_bdf(prob, uo0, dt, nsteps, 1, on_step=lambda n, t, u, lam: ref.append((u.copy(), lam.copy())))
    worst = 0.0
    for n in range(nsteps):
        s.hdg_step(dt, "be", 1)
        u, lam, t = s.hdg_get_state()
        eu = relerr(u.cpu().numpy(), ref[n][0])
        el = relerr(lam.cpu().numpy(), ref[n][1])
        worst = max(worst, eu, el)
        assert eu < 1e-11 and el < 1e-11, (n, eu, el)
    assert abs(t - nsteps * dt) < 1e-12
    # the discrete solution also tracks the exact mode (time-error dominated at dt = 0.01)
    assert ac.l2_error(prob, u.cpu().numpy(), lambda x: ex(x, t)) < 0.05


@pytest.mark.parametrize("scheme", ["bdf2", "dirk3"])
def test_acoustic_3d_point_source_steps(scheme):
    """3D acoustic, k = 3, c ~ logU[1,3], Ricker point source, Dirichlet data, random start."""
    dim, N, k = 3, 2, 3
    h = 1.0 / N
    src = [[0.5 + 0.3 * h, 0.5 + 0.3 * h, 0.5 + 0.3 * h]]
    s, prob, torch = make_pair(dim, N, k, seed=4, sources=src, f0=10.0, t0=0.02)
    u0 = inputs.random_state(s.n_elem, s.n, 21)
    s.hdg_set_state(torch.tensor(u0, device="cuda"), 0.0)
    dt, nsteps = 2e-3, 6
    ref = []
    cb = lambda n, t, u, lam: ref.append((u.copy(), lam.copy()))
    if scheme == "bdf2":
        ac.run_bdf(prob, u0, dt, nsteps, 2, on_step=cb)
    else:
        ac.run_dirk3(prob, u0, dt, nsteps, on_step=cb)
    for n in range(nsteps):
        s.hdg_step(dt, scheme, 1)
        u, lam, t = s.hdg_get_state()
        assert relerr(u.cpu().numpy(), ref[n][0]) < 1e-11, n
        assert relerr(lam.cpu().numpy(), ref[n][1]) < 1e-11, n


def test_steps_are_deterministic():
    dim, N, k = 3, 2, 2
    outs = []
    for rep in range(2):
        s, prob, torch = make_pair(dim, N, k, seed=2, sources=[[0.31, 0.42, 0.53]])
        s.hdg_set_state(torch.tensor(inputs.random_state(s.n_elem, s.n, 3), device="cuda"), 0.0)
        s.hdg_step(2e-3, "bdf2", 3)
        u, lam, t = s.hdg_get_state()
        outs.append((u.cpu().numpy(), lam.cpu().numpy()))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


def test_full_size_3d_workload_sampled():
    """196,608 tets, k = 3 (the benchmark workload): S_K, apply, condensed rhs and recovery
    checked on sampled elements/faces against the oracle's element-level computation;
    the full BDF2 step checked by its own true trace residual and bitwise determinism."""
    import torch
    from paper_1807_00086_gb300 import hdg
    w = inputs.acoustic_3d_workload()
    vert, elem, k = w["vert"], w["elem"], w["k"]
    ne = elem.shape[0]
    s = hdg.Solver(vert, elem, k, w["tau"], w["rho"], w["c"])
    assert s.n_elem == 196608 and s.n_faces == 399360 and s.n_bnd == 12288
    alpha = 1.5 / 2e-3
    s.hdg_condense(alpha)
    sk = ac.skeleton(elem)
    rng = np.random.default_rng(77)
    sample = np.unique(np.concatenate([[0, ne - 1], rng.integers(0, ne, 10)]))
    S = s.hdg_get_schur()
    blocks = {}

    def blk(e):
        if e not in blocks:
            b = ac.element_blocks(vert[sk.elem[e]], k, w["rho"][e], w["c"][e], w["tau"])
            A = alpha * b.Mw + b.A0
            blocks[e] = (b, A, b.D - b.C @ np.linalg.solve(A, b.B))
        return blocks[e]

    for e in sample:
        assert relerr(S[e].cpu().numpy(), blk(e)[2]) < 1e-12
    del S
    lam = inputs.random_traces(s.n_faces, s.Nf, 31)
    lam[sk.boundary] = 0.0
    lam_t = torch.tensor(lam, device="cuda")
    y = s.hdg_trace_apply(lam_t).cpu().numpy()
    Nf = s.Nf
    faces = rng.choice(np.nonzero(~sk.boundary)[0], 8, replace=False)
    for f in faces:
        yo = np.zeros(Nf)
        for (e, j) in sk.face_elems[f]:
            lk = np.concatenate([lam[sk.elem_face[e, a]] for a in range(4)])
            yo += (blk(e)[2] @ lk)[j * Nf:(j + 1) * Nf]
        assert relerr(y[f], yo) < 1e-12
    F = inputs.random_state(ne, s.n, 32)
    u = s.hdg_recover(torch.tensor(F, device="cuda"), lam_t).cpu().numpy()
    for e in sample:
        b, A, _ = blk(e)
        lk = np.concatenate([lam[sk.elem_face[e, a]] for a in range(4)])
        assert relerr(u[e], np.linalg.solve(A, F[e] - b.B @ lk)) < 1e-12
    # one full BDF2 step from a random state with the Ricker source
    s.hdg_set_sources(w["sources"], [1.0], w["f0"], w["t0"])
    u0 = torch.tensor(inputs.random_state(ne, s.n, 33), device="cuda")
    res = []
    for rep in range(2):
        # a condensation drops the least-squares guess's stored pairs (hdg_set_state keeps
        # them), so both repetitions start from the same solver state
        s.hdg_condense(alpha)
        s.hdg_set_state(u0, 0.0)
        info = s.hdg_step(2e-3, "bdf2", 1)
        assert info["rel_residual"] <= 1e-13
        u1, lam1, t1 = s.hdg_get_state()
        res.append((u1.cpu().numpy(), lam1.cpu().numpy()))
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])
