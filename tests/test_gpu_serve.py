"""Continuous batching on the GPU: each request's result is the same alone and in the mix
(mixed precision, within 1e-9), and one request matches the oracle."""
import numpy as np
import pytest

from gpu_helpers import relerr
from oracle import acoustic as ac
from paper_1807_00086_gb300.serve import F0, T0, Request, Server, mesh_for

pytestmark = pytest.mark.gpu


def _requests():
    rng = np.random.default_rng(9)
    reqs = []
    for i in range(7):
        dim = 2 if i % 2 == 0 else 3
        N, k = (8, 2) if dim == 2 else (2, 2)
        reqs.append(Request(i, 0.01 * i, dim, N, k, 6 + 2 * i, rng.uniform(0.2, 0.8, size=dim)))
    return reqs


def test_results_are_the_same_alone_and_in_the_mix():
    mix = _requests()
    srv = Server(budget_bytes=8 << 30, R=4)
    stats = srv.run(mix)
    srv.close()
    assert stats["requests"] == len(mix)
    for r in mix:
        alone = Request(r.rid, 0.0, r.dim, r.N, r.k, r.nsteps, r.source)
        s1 = Server(budget_bytes=8 << 30, R=4)
        s1.run([alone])
        s1.close()
        assert relerr(r.result, alone.result) < 1e-9, r.rid


def test_served_request_matches_oracle():
    r = Request(0, 0.0, 2, 8, 2, 8, np.array([0.37, 0.61]))
    srv = Server(budget_bytes=8 << 30, R=4)
    srv.run([r])
    srv.close()
    vert, elem = mesh_for(2, 8)
    prob = ac.build_problem(vert, elem, 2, 1.0, 1.0, 1.0)
    ac.add_point_source(prob, r.source, F0, T0)
    u0 = np.zeros((elem.shape[0], 3 * prob.Np))
    uo, lo, to = ac.run_bdf(prob, u0, 2e-3, r.nsteps, 2)
    assert relerr(r.result, uo) < 1e-9
