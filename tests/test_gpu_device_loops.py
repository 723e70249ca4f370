"""Device-driven trace solves (one CUDA-graph launch per solve, loop conditions set on the
device) against the oracle and against the host-driven loops.

* per-step parity with the oracle on both paths (FP64 <= 1e-11, mixed <= 1e-9), acoustic and
  per-element-degree elastic;
* the two paths agree with each other to the solver tolerance;
* the device loops end on their own at maxit / max_sweeps and report HDG_ENOCONV.
"""
import numpy as np
import pytest

from gpu_helpers import make_pair, mesh, relerr
from oracle import acoustic as ac
from oracle import elastic_vardeg as vd
from paper_1807_00086_gb300 import inputs

pytestmark = pytest.mark.gpu


def _acoustic(prec, device_loops, N=2, k=3, seed=4, **kw):
    from paper_1807_00086_gb300 import hdg
    from gpu_helpers import dirichlet_profile
    vert, elem = mesh(3, N)
    ne = elem.shape[0]
    s = hdg.Solver(vert, elem, k, 1.0, inputs.loguniform(ne, 0.5, 2.0, seed + 7), inputs.loguniform(ne, 1.0, 3.0, seed),
                   prec=prec, rtol=1e-13 if prec == "fp64" else 1e-12, device_loops=device_loops,
                   inner_rtol=1e-3 if prec == "mixed16" else None, **kw)
    xb = s.hdg_quadrature_points(1)
    s.hdg_set_dirichlet(np.stack([dirichlet_profile(x) for x in xb]), 3.0, 0.2)
    h = 1.0 / N
    src = [[0.5 + 0.3 * h] * 3]
    s.hdg_set_sources(src, [1.0], 10.0, 0.02)
    return s, src


@pytest.mark.parametrize("scheme", ["bdf2", "dirk3"])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("mixed", 1e-9), ("mixed16", 1e-9)])
def test_device_loops_match_oracle_and_host_loops(prec, tol, scheme):
    import torch
    dim, N, k = 3, 2, 3
    _, prob, _ = make_pair(dim, N, k, seed=4, sources=[[0.5 + 0.15] * 3], f0=10.0, t0=0.02)
    u0 = inputs.random_state(6 * N ** 3, 4 * 20, 21)
    dt, nsteps = 2e-3, 6
    ref = []
    cb = lambda n, t, u, lam: ref.append((u.copy(), lam.copy()))
    if scheme == "bdf2":
        ac.run_bdf(prob, u0, dt, nsteps, 2, on_step=cb)
    else:
        ac.run_dirk3(prob, u0, dt, nsteps, on_step=cb)
    out = {}
    for dl in (True, False):
        s, _ = _acoustic(prec, dl)
        s.hdg_set_state(torch.tensor(u0, device="cuda"), 0.0)
        traj = []
        for n in range(nsteps):
            info = s.hdg_step(dt, scheme, 1)
            assert info["rel_residual"] <= (1e-13 if prec == "fp64" else 1e-12)
            assert info["iterations"] > 0 and info["sweeps"] >= 1
            u, lam, t = s.hdg_get_state()
            traj.append((u.cpu().numpy(), lam.cpu().numpy()))
            assert relerr(traj[-1][0], ref[n][0]) < tol, (dl, n)
            assert relerr(traj[-1][1], ref[n][1]) < tol, (dl, n)
        out[dl] = traj
    for n in range(nsteps):
        assert relerr(out[True][n][0], out[False][n][0]) < tol


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("mixed16", 1e-9)])
def test_device_loops_per_element_degree_elastic(prec, tol):
    import torch
    from paper_1807_00086_gb300 import hdg
    N, seed = 2, 5
    ks = inputs.element_degrees(6 * N ** 3, 1, 4, seed)
    vert, elem = inputs.unit_cube_tet(N)
    ne = elem.shape[0]
    rho = inputs.loguniform(ne, 0.5, 2.0, 7)
    lam = inputs.lognormal(ne, 1.5, 0.5, 2)
    mu = inputs.lognormal(ne, 1.0, 0.5, 3)
    prob = vd.build_problem(vert, elem, ks, rho, lam, mu)
    u0 = np.random.default_rng(seed).standard_normal(int(prob.u_off[-1]))
    ref = []
    vd.run_dirk3(prob, u0, 0.01, 2, on_step=lambda n, t, u, l: ref.append((u.copy(), l.copy())))
    for dl in (True, False):
        s = hdg.Solver(vert, elem, 4, 1.0, rho, lam=lam, mu=mu, prec=prec, rtol=1e-13 if prec == "fp64" else 1e-12,
                       elem_k=ks, device_loops=dl)
        s.hdg_set_state(torch.tensor(u0, device="cuda"), 0.0)
        for n in range(2):
            s.hdg_step(0.01, "dirk3", 1)
            u, lg, t = s.hdg_get_state()
            assert relerr(u.cpu().numpy(), ref[n][0]) < tol, (dl, n)
            assert relerr(lg.cpu().numpy(), ref[n][1]) < tol, (dl, n)


def test_device_krylov_loop_stops_at_maxit():
    """FP64: maxit = 3 cannot reach rtol 1e-13; the WHILE loop ends by itself and the call
    reports HDG_ENOCONV with the three iterations it ran."""
    import torch
    from paper_1807_00086_gb300 import hdg
    s, _ = _acoustic("fp64", True, maxit=3)
    s.hdg_condense(40.0)
    r = torch.tensor(inputs.random_traces(s.n_faces, s.Nf, 3), device="cuda")
    lam = torch.zeros_like(r)
    with pytest.raises(hdg.HDGError) as ei:
        s.hdg_trace_solve(r, lam)
    assert ei.value.status == -4
    # the context stays usable: a solve with a reachable target succeeds afterwards
    s2, _ = _acoustic("fp64", True)
    s2.hdg_condense(40.0)
    info = s2.hdg_trace_solve(r, torch.zeros_like(r))
    assert info["rel_residual"] <= 1e-13


def test_device_sweep_loop_stops_at_max_sweeps():
    import torch
    from paper_1807_00086_gb300 import hdg
    s, _ = _acoustic("mixed16", True, max_sweeps=1)
    s.hdg_condense(40.0)
    r = torch.tensor(inputs.random_traces(s.n_faces, s.Nf, 3), device="cuda")
    with pytest.raises(hdg.HDGError) as ei:
        s.hdg_trace_solve(r, torch.zeros_like(r))
    assert ei.value.status == -4


def test_device_loops_zero_right_hand_side():
    """A zero right-hand side gives the zero solution on interior faces (boundary entries of
    the initial guess untouched), on both paths."""
    import torch
    for prec in ("fp64", "mixed16"):
        s, _ = _acoustic(prec, True)
        s.hdg_condense(40.0)
        r = torch.zeros((s.n_faces, s.Nf), dtype=torch.float64, device="cuda")
        lam = torch.tensor(inputs.random_traces(s.n_faces, s.Nf, 8), device="cuda")
        bnd = torch.tensor(np.asarray(ac.skeleton(mesh(3, 2)[1]).boundary), device="cuda")
        lam0 = lam.clone()
        info = s.hdg_trace_solve(r, lam)
        assert info["rel_residual"] == 0.0
        assert torch.all(lam[~bnd] == 0) and torch.equal(lam[bnd], lam0[bnd])


@pytest.mark.parametrize("R", [4, 64])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("mixed", 1e-9)])
def test_device_loops_multi_column_match_host_loops_and_oracle(prec, tol, R):
    """R columns: one graph launch per trace solve (per-column Krylov loop inside the sweep
    loop) against the host-driven loops and, for two columns, against the oracle."""
    import torch
    from paper_1807_00086_gb300 import hdg
    from gpu_helpers import dirichlet_profile
    vert, elem = mesh(3, 2)
    ne = elem.shape[0]
    k, seed = 2, 3
    rho = inputs.loguniform(ne, 0.5, 2.0, seed + 7)
    c = inputs.loguniform(ne, 1.0, 3.0, seed)
    pos = inputs.uniform_points(R, 3, 0.1, 0.9, seed + 1)
    amps = np.linspace(1.0, 2.0, R)
    dt, nsteps = 2e-3, 3
    out = {}
    for dl in (True, False):
        s = hdg.Solver(vert, elem, k, 1.0, rho, c, prec=prec, rtol=1e-12, nrhs=R, device_loops=dl)
        xb = s.hdg_quadrature_points(1)
        s.hdg_set_dirichlet(np.stack([dirichlet_profile(x) for x in xb]), 3.0, 0.2)
        s.hdg_set_sources(pos, amps, 10.0, 0.02, col=np.arange(R))
        u0 = inputs.random_state(ne, s.n * R, seed + 2).reshape(ne, s.n, R)
        s.hdg_set_state(torch.tensor(u0, device="cuda"), 0.0)
        for _ in range(nsteps):
            info = s.hdg_step(dt, "bdf2", 1)
            assert info["rel_residual"] <= 1e-12 and info["iterations"] > 0
        u, lam, t = s.hdg_get_state()
        out[dl] = (u.cpu().numpy(), lam.cpu().numpy())
    assert relerr(out[True][0], out[False][0]) < tol and relerr(out[True][1], out[False][1]) < tol
    prob = ac.build_problem(vert, elem, k, 1.0, rho, c)
    prob.dirichlet = lambda x, t: dirichlet_profile(x) * np.cos(3.0 * t + 0.2)
    for j in (0, R - 1):
        prob.sources = []
        ac.add_point_source(prob, pos[j], 10.0, 0.02, amp=amps[j])
        uo, lo, to = ac.run_bdf(prob, u0[:, :, j], dt, nsteps, 2)
        assert relerr(out[True][0][:, :, j], uo) < tol, j
        assert relerr(out[True][1][:, :, j], lo) < tol, j

