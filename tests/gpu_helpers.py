"""Shared helpers for the GPU parity tests (CUDA path through the C ABI vs the oracle)."""
import numpy as np

from oracle import acoustic as ac
from paper_1807_00086_gb300 import inputs


def mesh(dim, N):
    return inputs.unit_square_tri(N) if dim == 2 else inputs.unit_cube_tet(N)


def relerr(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def dirichlet_profile(x):
    return np.cos(np.pi * x[:, 0]) * np.sin(np.pi * x[:, 1] + 0.3) + 0.3 * x[:, -1]


def make_pair(dim, N, k, seed=1, tau=1.0, dirichlet=True, omega=3.0, phase=0.2, sources=None, f0=10.0, t0=0.05):
    """Builds the same problem on the GPU (hdg.Solver) and in the oracle."""
    import torch
    from paper_1807_00086_gb300 import hdg
    vert, elem = mesh(dim, N)
    ne = elem.shape[0]
    rho = inputs.loguniform(ne, 0.5, 2.0, seed + 7)
    c = inputs.loguniform(ne, 1.0, 3.0, seed)
    s = hdg.Solver(vert, elem, k, tau, rho, c)
    prob = ac.build_problem(vert, elem, k, tau, rho, c)
    if dirichlet:
        xb = s.hdg_quadrature_points(1)
        vals = np.stack([dirichlet_profile(xb[b]) for b in range(xb.shape[0])]) if xb.shape[0] else None
        s.hdg_set_dirichlet(vals, omega, phase)
        prob.dirichlet = lambda x, t: dirichlet_profile(x) * np.cos(omega * t + phase)
    if sources is not None:
        s.hdg_set_sources(sources, np.ones(len(sources)), f0, t0)
        for xs in sources:
            ac.add_point_source(prob, xs, f0, t0)
    return s, prob, torch
