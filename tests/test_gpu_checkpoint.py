"""Checkpoint / resume: n steps, save, load into a fresh context, n more steps gives bitwise the
same fields and traces as 2n uninterrupted steps (the checkpoint holds the whole solver state:
fields, previous level, trace history, the least-squares guess's stored solutions)."""
import numpy as np
import pytest

from gpu_helpers import dirichlet_profile, mesh
from paper_1807_00086_gb300 import inputs

pytestmark = pytest.mark.gpu


def _acoustic(dim, N, k, prec, nrhs=1, trace_space="hdg"):
    import torch
    from paper_1807_00086_gb300 import hdg
    vert, elem = mesh(dim, N)
    ne = elem.shape[0]
    s = hdg.Solver(vert, elem, k, 1.0, inputs.loguniform(ne, 0.5, 2.0, 9), inputs.loguniform(ne, 1.0, 3.0, 2),
                   prec=prec, rtol=1e-13 if prec == "fp64" else 1e-12, nrhs=nrhs, trace_space=trace_space,
                   inner_rtol=1e-3 if prec == "mixed16" else None)
    if trace_space != "edg":
        xb = s.hdg_quadrature_points(1)
        s.hdg_set_dirichlet(np.stack([dirichlet_profile(x) for x in xb]), 3.0, 0.2)
    pos = inputs.uniform_points(nrhs, dim, 0.2, 0.8, 5)
    s.hdg_set_sources(pos, np.ones(nrhs), 10.0, 0.02, col=np.arange(nrhs))
    shape = (ne, s.n) if nrhs == 1 else (ne, s.n, nrhs)
    s.hdg_set_state(torch.tensor(inputs.random_state(ne, s.n * nrhs, 3).reshape(shape), device="cuda"), 0.0)
    return s


def _elastic_vardeg(prec):
    import torch
    from paper_1807_00086_gb300 import hdg
    vert, elem = inputs.unit_cube_tet(2)
    ne = elem.shape[0]
    ks = inputs.element_degrees(ne, 1, 4, 5)
    s = hdg.Solver(vert, elem, 4, 1.0, 1.0, lam=inputs.lognormal(ne, 1.5, 0.5, 2), mu=inputs.lognormal(ne, 1.0, 0.5, 3),
                   prec=prec, rtol=1e-12, elem_k=ks, inner_rtol=1e-3 if prec == "mixed16" else None)
    s.hdg_set_state(torch.tensor(np.random.default_rng(4).standard_normal(s._fshape), device="cuda"), 0.0)
    return s


def _svk(prec):
    import torch
    from paper_1807_00086_gb300 import hdg
    vert, elem = inputs.unit_cube_tet(1)
    ne = elem.shape[0]
    s = hdg.Solver(vert, elem, 2, 1.0, np.ones(ne), lam=np.full(ne, 1.5), mu=np.ones(ne), svk=True, rtol=1e-12,
                   prec=prec)
    rng = np.random.default_rng(6)
    u = np.zeros((ne, s.n))
    u[:, :3 * s.Np] = 0.5 * rng.standard_normal((ne, 3 * s.Np))
    u[:, 3 * s.Np:12 * s.Np] = 0.03 * rng.standard_normal((ne, 9 * s.Np))
    s.hdg_set_state(torch.tensor(u, device="cuda"), 0.0)
    return s


CASES = [
    ("acoustic 3D k=3 mixed16 BDF2", lambda: _acoustic(3, 2, 3, "mixed16"), "bdf2", 2e-3),
    ("acoustic 2D k=2 FP64 DIRK3", lambda: _acoustic(2, 4, 2, "fp64"), "dirk3", 1e-2),
    ("acoustic 3D k=2 mixed, 4 columns, BDF2", lambda: _acoustic(3, 2, 2, "mixed", nrhs=4), "bdf2", 2e-3),
    ("acoustic 3D k=3 IEDG mixed16 BDF2", lambda: _acoustic(3, 2, 3, "mixed16", trace_space="iedg"), "bdf2", 2e-3),
    ("elastic per-element degree mixed16 DIRK3", lambda: _elastic_vardeg("mixed16"), "dirk3", 1e-2),
    ("SVK k=2 FP32 Jacobian DIRK3", lambda: _svk("mixed"), "dirk3", 2e-2),
]


@pytest.mark.parametrize("name,make,scheme,dt", CASES, ids=[c[0] for c in CASES])
def test_resume_from_checkpoint_is_bitwise(name, make, scheme, dt):
    n = 4
    a = make()
    a.hdg_step(dt, scheme, 2 * n)
    ua, la, ta = a.hdg_get_state()
    b = make()
    b.hdg_step(dt, scheme, n)
    ck = b.hdg_save_checkpoint()
    c = make()
    c.hdg_load_checkpoint(ck)
    c.hdg_step(dt, scheme, n)
    uc, lc, tc = c.hdg_get_state()
    assert tc == ta
    assert np.array_equal(ua.cpu().numpy(), uc.cpu().numpy()), name
    assert np.array_equal(la.cpu().numpy(), lc.cpu().numpy()), name
    # a checkpoint of other sizes is refused
    from paper_1807_00086_gb300 import hdg
    other = _acoustic(2, 2, 1, "fp64")
    with pytest.raises(hdg.HDGError):
        other.hdg_load_checkpoint(ck)


@pytest.mark.parametrize("prec,nrhs", [("mixed16", 1), ("fp64", 1), ("mixed", 4)])
def test_rebinding_the_stream_mid_run_is_bitwise_neutral(prec, nrhs):
    """hdg_set_stream: 2 steps on the creation stream, rebind to a library-created stream,
    2 more steps (device-loop graphs captured before the switch are launched on the new
    stream) gives bitwise the fields and traces of 4 steps on one stream."""
    import torch
    from paper_1807_00086_gb300 import hdg
    a = _acoustic(3, 2, 3, prec, nrhs)
    b = _acoustic(3, 2, 3, prec, nrhs)
    a.hdg_step(2e-3, "bdf2", 4)
    b.hdg_step(2e-3, "bdf2", 2)
    st = hdg.own_stream()
    try:
        b.hdg_set_stream(st)
        b.hdg_step(2e-3, "bdf2", 2)
        ua, la, ta = a.hdg_get_state()
        ub, lb, tb = b.hdg_get_state()
        torch.cuda.synchronize()
        assert ta == tb
        assert torch.equal(ua, ub) and torch.equal(la, lb)
    finally:
        b.close()
        hdg.release_stream(st)
