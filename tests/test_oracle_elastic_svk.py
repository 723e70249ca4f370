"""Pins of the oracle's nonlinear (SVK) elastodynamics HDG scheme, by facts independent of it:
  * the batched stress and tangent equal the pinned pointwise SVK law;
  * the element Jacobian equals central differences of the element residual (Newton's
    matrix is the derivative of the equations it solves);
  * at small amplitude the scheme reduces to the pinned linear v-F oracle: the difference
    of the solutions shrinks linearly with the amplitude (the nonlinearity is quadratic);
  * on the clamped vibrating plate (Sec. 4.5, SVK material, one element through the
    thickness, traction data on the faces) the velocity converges at order k + 1, as the
    paper reports for the nonlinear case. tests/golden/eoc_nonlinear_elastodyn.txt holds the
    paper's printed finest-mesh rates; its meshes are finer and of unstated type, so the rate
    is compared, not the error.
"""
import math
import os

import numpy as np
import pytest

from oracle import elastic as el
from oracle import elastic_svk as nl
from oracle import svk
from paper_1807_00086_gb300 import inputs


def test_batched_law_matches_the_pointwise_law():
    F = np.eye(3) + 0.3 * np.random.default_rng(1).standard_normal((5, 3, 3))
    P = nl.pk_batch(F, 1.5, 1.0)
    A = nl.tangent_batch(F, 1.5, 1.0)
    for q in range(5):
        assert np.abs(P[q] - svk.first_pk(F[q], 1.5, 1.0)).max() < 1e-14
        assert np.abs(A[q] - svk.tangent(F[q], 1.5, 1.0)).max() < 1e-13


def test_element_jacobian_is_the_derivative_of_the_residual():
    vert, elem = inputs.unit_cube_tet(1)
    prob = nl.build_problem(vert, elem, 1, 1.0, 1.5, 1.0)
    prob.body_force = lambda x, t: np.sin(x) * t
    rng = np.random.default_rng(2)
    Np, Nf = prob.Np, prob.Nf
    u = 0.2 * rng.standard_normal(21 * Np)
    lamK = rng.standard_normal(12 * Nf)
    h = rng.standard_normal(21 * Np)
    R, Rh, A, B, C, D = nl.element_system(prob, 3, u, lamK, h, 7.0, 0.1)
    J = np.block([[A, B], [C, D]])
    z = np.concatenate([u, lamK])
    eps = 1e-6
    for j in range(z.size):
        zp, zm = z.copy(), z.copy()
        zp[j] += eps
        zm[j] -= eps
        rp = np.concatenate(nl.element_system(prob, 3, zp[:21 * Np], zp[21 * Np:], h, 7.0, 0.1)[:2])
        rm = np.concatenate(nl.element_system(prob, 3, zm[:21 * Np], zm[21 * Np:], h, 7.0, 0.1)[:2])
        assert np.abs((rp - rm) / (2 * eps) - J[:, j]).max() < 1e-7 * np.abs(J).max()


def test_small_amplitude_limit_is_the_linear_scheme():
    vert, elem = inputs.unit_cube_tet(1)
    ne = elem.shape[0]
    diffs = []
    for amp in (1e-3, 1e-4):
        lin = el.build_problem(vert, elem, 1, 1.0, 1.5, 1.0, form="F")
        non = nl.build_problem(vert, elem, 1, 1.0, 1.5, 1.0)
        Np = non.Np
        v0 = amp * np.random.default_rng(3).standard_normal((ne, 3 * Np))
        ul0 = np.zeros((ne, 12 * Np))
        ul0[:, :3 * Np] = v0
        un0 = np.zeros((ne, 21 * Np))
        un0[:, :3 * Np] = v0
        ul, _, _ = el.run_dirk3(lin, ul0, 0.01, 2)
        un, _, its = nl.run_dirk3(non, un0, 0.01, 2)
        diffs.append(np.abs(un[:, :12 * Np] - ul).max() / np.abs(ul).max())
        assert max(its) <= 5
    assert diffs[0] < 1e-4
    assert abs(diffs[0] / diffs[1] - 10.0) < 0.5


def test_plate_velocity_converges_at_order_k_plus_1():
    pytest.importorskip("sympy")
    lam, mu, rho, k = 1.5, 1.0, 1.0, 1
    sol = svk.plate_solution(lam, mu, rho)
    I9 = np.eye(3).ravel()

    def top_or_bottom(Y):
        z = Y[:, 2]
        return bool(np.all(np.abs(z - z[0]) < 1e-14) and (abs(z[0]) < 1e-14 or abs(z[0] - 0.01) < 1e-14))
    errs = []
    for n in (2, 4):
        vert, elem = inputs.plate_tet(n)
        prob = nl.build_problem(vert, elem, k, rho, lam, mu, neumann_face=top_or_bottom)
        assert prob.neumann.sum() == 4 * n * n
        prob.body_force = sol["f"]
        prob.traction = lambda x, nrm, t: np.einsum("qij,j->qi", sol["P"](x, t).reshape(-1, 3, 3), nrm)
        u0 = nl.project(prob, sol["v"], lambda x, t: sol["F"](x, t) - I9, sol["P"], 0.0)
        T = 0.125
        u, _, _ = nl.run_dirk3(prob, u0, T / (2 * n), 2 * n)
        errs.append(nl.l2_error_velocity(prob, u, sol["v"], T))
    rate = math.log2(errs[0] / errs[1])
    golden = os.path.join(os.path.dirname(__file__), "golden", "eoc_nonlinear_elastodyn.txt")
    rows = [ln.split() for ln in open(golden) if ln.strip() and not ln.startswith("#")]
    paper_rate = float([r for r in rows if int(r[0]) == k][0][3])
    assert rate > k + 1 - 0.3 and abs(rate - paper_rate) < 0.3, (errs, rate, paper_rate)
