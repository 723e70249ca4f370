"""Pins for the oracle's variable-degree elastodynamics HDG scheme (per-element k_K, face
degree k_F = max over the neighbours; Sec. 4.1 with the spaces of Sec. 2.2 taken per element).

* with one degree everywhere it reproduces the uniform-degree oracle (itself pinned by brute
  force, an energy identity and the paper's convergence orders);
* static condensation (Eq. LS) reproduces the uncondensed [A B; C D] solve on meshes whose
  degrees jump between neighbours;
* a linear velocity field with a stress growing linearly in time is an exact solution of
  the continuous problem (uniform material); the scheme reproduces it to rounding across
  degree jumps, which fails if a face coupling between different degrees is wrong;
* the backward-Euler discrete energy identity holds step by step.
"""
import numpy as np
import pytest

from oracle import elastic as el
from oracle import elastic_vardeg as vd
from paper_1807_00086_gb300 import inputs


def _mesh(dim, N):
    return inputs.unit_square_tri(N) if dim == 2 else inputs.unit_cube_tet(N)


def _materials(ne):
    return inputs.loguniform(ne, 0.5, 2.0, 4), 1.5 * inputs.lognormal(ne, 1.0, 0.5, 2), inputs.lognormal(ne, 1.0, 0.5, 3)


def _dirichlet(dim):
    return lambda x, t: np.stack([np.sin(x[:, 0] + t), np.cos(x[:, 1]), x[:, 0] * x[:, -1]][:dim], axis=1)


@pytest.mark.parametrize("dim,N,k", [(2, 2, 2), (3, 1, 2)])
def test_uniform_degree_reproduces_uniform_oracle(dim, N, k):
    vert, elem = _mesh(dim, N)
    ne = elem.shape[0]
    rho, lam, mu = _materials(ne)
    pu = el.build_problem(vert, elem, k, rho, lam, mu)
    pv = vd.build_problem(vert, elem, np.full(ne, k), rho, lam, mu)
    pu.dirichlet = pv.dirichlet = _dirichlet(dim)
    rng = np.random.default_rng(5)
    u0 = rng.standard_normal((ne, (dim + pu.nt) * pu.Np))
    uu, lu, _ = el.run_dirk3(pu, u0, 0.01, 2)
    uv, lv, _ = vd.run_dirk3(pv, u0.ravel(), 0.01, 2)
    assert np.abs(uv - uu.ravel()).max() <= 1e-12 * np.abs(uu).max()
    assert np.abs(lv - lu.ravel()).max() <= 1e-12 * np.abs(lu).max()


@pytest.mark.parametrize("dim,N,seed", [(2, 2, 11), (2, 3, 12), (3, 1, 13)])
def test_condensed_equals_monolithic_across_degree_jumps(dim, N, seed):
    vert, elem = _mesh(dim, N)
    ne = elem.shape[0]
    ks = inputs.element_degrees(ne, 1, 3, seed)
    assert len(set(ks.tolist())) > 1
    prob = vd.build_problem(vert, elem, ks, *_materials(ne))
    prob.dirichlet = _dirichlet(dim)
    rng = np.random.default_rng(seed)
    h = rng.standard_normal(int(prob.u_off[-1]))
    for alpha in (0.3, 60.0):
        cond = vd.condense(prob, alpha)
        u, lam = vd.solve_stage(prob, cond, h, 0.3)
        um, lm = vd.solve_monolithic(prob, alpha, h, 0.3)
        assert np.abs(u - um).max() <= 1e-11 * np.abs(um).max()
        assert np.abs(lam - lm).max() <= 1e-11 * np.abs(lm).max()


@pytest.mark.parametrize("dim,N", [(2, 3), (3, 1)])
def test_linear_patch_solution_is_reproduced_across_degree_jumps(dim, N):
    """v = A x, sigma = sigma0 + t C eps(A): rho v_t - div sigma = 0 and C^-1 sigma_t = eps(v)."""
    vert, elem = _mesh(dim, N)
    ne = elem.shape[0]
    ks = inputs.element_degrees(ne, 1, 3, 21 + dim)
    lam0, mu0, rho0 = 1.3, 0.7, 1.1
    prob = vd.build_problem(vert, elem, ks, rho0, lam0, mu0)
    rng = np.random.default_rng(7)
    A = rng.standard_normal((dim, dim))
    comps = el.sym_components(dim)
    eps = 0.5 * (A + A.T)
    rate = lam0 * np.trace(eps) * np.eye(dim) + 2 * mu0 * eps
    s0 = rng.standard_normal((dim, dim))
    s0 = s0 + s0.T
    sig = lambda t: s0 + t * rate
    v_ex = lambda x: x @ A.T
    t_ex = lambda x, t: np.tile([sig(t)[i, j] for (i, j) in comps], (x.shape[0], 1))
    prob.dirichlet = lambda x, t: v_ex(x)
    u0 = vd.project(prob, v_ex, lambda x: t_ex(x, 0.0))
    u, lamh, T = vd.run_dirk3(prob, u0, 0.02, 3)
    want = vd.project(prob, v_ex, lambda x: t_ex(x, T))
    assert np.abs(u - want).max() <= 1e-11 * np.abs(want).max()


@pytest.mark.parametrize("dim,N", [(2, 2), (3, 1)])
def test_backward_euler_energy_identity_mixed_degree(dim, N):
    """E^{n+1} - E^n + 1/2 |u^{n+1} - u^n|_M^2 + dt sum_dK <s (v - v_hat)^2, 1> = 0 (clamped)."""
    vert, elem = _mesh(dim, N)
    ne = elem.shape[0]
    prob = vd.build_problem(vert, elem, inputs.element_degrees(ne, 1, 3, 31), *_materials(ne))
    rng = np.random.default_rng(3)
    u0 = rng.standard_normal(int(prob.u_off[-1]))
    dt = 0.01
    prev = [u0]

    def check(n, t, u, lam):
        diss, bwork = vd.energy_terms(prob, u, lam)
        du = u - prev[-1]
        lhs = (vd.energy(prob, u) - vd.energy(prob, prev[-1])
               + 0.5 * sum(vd.field(prob, du, e) @ bl.Mw @ vd.field(prob, du, e) for e, bl in enumerate(prob.blocks))
               + dt * diss)
        assert abs(lhs - dt * bwork) <= 1e-11 * (abs(lhs) + dt * abs(diss))
        prev.append(u)

    vd.run_bdf(prob, u0, dt, 3, 1, on_step=check)
