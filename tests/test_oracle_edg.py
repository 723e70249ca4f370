"""Pins of the oracle's EDG / IEDG trace spaces (continuous traces on all faces / on the
interior faces), against facts that do not restate the construction:
  * the number of global unknowns equals the mesh-combinatorial count of skeleton nodes
    (vertices, k - 1 per edge, (k-1)(k-2)/2 per triangular face);
  * the nodal values of a global polynomial of degree k map, face by face, to that
    polynomial's L2 projection (exact in P_k), so R is the identity on continuous P_k;
  * traces in the range of R are continuous where faces meet;
  * on the exact standing mode the pressure converges at order k + 1.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import acoustic as ac
from oracle import edg
from oracle import reference as ref
from paper_1807_00086_gb300 import inputs


def _mesh(dim, N):
    return inputs.unit_square_tri(N) if dim == 2 else inputs.unit_cube_tet(N)


def _expected_unknowns(sk, k, variant):
    dim = sk.dim
    faces = sk.faces[~sk.boundary] if variant == "iedg" else sk.faces
    bverts = set(sk.faces[sk.boundary].ravel().tolist())
    bedges = {e for f in sk.faces[sk.boundary] for e in itertools.combinations(f.tolist(), 2)}
    verts = set(faces.ravel().tolist())
    if variant == "edg":
        verts -= bverts
    count = len(verts)
    if dim == 2:            # faces are edges: k - 1 nodes inside each
        fs = [tuple(f) for f in faces.tolist()]
        if variant == "edg":
            fs = [f for f in fs if f not in bedges]
        return count + (k - 1) * len(fs)
    edges = {e for f in faces for e in itertools.combinations(f.tolist(), 2)}
    if variant == "edg":
        edges -= bedges
    nface_int = int((~sk.boundary).sum())   # EDG: boundary faces' inner nodes are fixed
    return count + (k - 1) * len(edges) + (k - 1) * (k - 2) // 2 * nface_int


@pytest.mark.parametrize("dim,N,k", [(2, 3, 1), (2, 3, 3), (3, 2, 2), (3, 1, 4)])
@pytest.mark.parametrize("variant", ["edg", "iedg"])
def test_unknown_count_is_the_skeleton_node_count(dim, N, k, variant):
    vert, elem = _mesh(dim, N)
    prob = ac.build_problem(vert, elem, k, 1.0, 1.0, 1.0)
    tm = edg.trace_map(prob, variant)
    assert tm.n_free == _expected_unknowns(prob.sk, k, variant)
    hdg_unknowns = int((~prob.sk.boundary).sum()) * prob.Nf
    assert tm.n_free < hdg_unknowns


@pytest.mark.parametrize("dim,N,k", [(2, 2, 2), (3, 1, 3)])
def test_nodal_values_of_a_global_polynomial_give_its_face_projections(dim, N, k):
    vert, elem = _mesh(dim, N)
    prob = ac.build_problem(vert, elem, k, 1.0, 1.0, 1.0)
    rng = np.random.default_rng(7)
    exps = [m for m in itertools.product(range(k + 1), repeat=dim) if sum(m) <= k]
    cf = rng.standard_normal(len(exps))

    def P(x):
        return sum(c * np.prod(x ** np.array(m), axis=1) for c, m in zip(cf, exps))
    tm = edg.trace_map(prob, "iedg")
    # nodal values at the free nodes: evaluate P at each node through its faces' nodes
    bs, _ = edg.face_nodes(dim, k)
    mu = np.zeros(tm.n_free)
    interior = np.nonzero(~prob.sk.boundary)[0]
    free_index = {}
    for f in interior:
        ids, _ = tm.face_modal[f]
        fv = prob.sk.faces[f]
        for a, b in enumerate(bs):
            x = sum(b[i] * vert[fv[i]] for i in range(dim)) / k
            free_index[ids[a]] = P(x[None, :])[0]
    # the free numbering of IEDG follows first appearance over the interior faces
    for node, val in free_index.items():
        mu[node] = val
    lam = tm.R @ mu
    for r, f in enumerate(interior):
        want = ac.project_face(prob, f, lambda x, t: P(x), 0.0)
        assert np.abs(lam[r * prob.Nf:(r + 1) * prob.Nf] - want).max() < 1e-12 * max(1.0, np.abs(want).max())


@pytest.mark.parametrize("dim,N,k", [(2, 2, 3), (3, 1, 2)])
@pytest.mark.parametrize("variant", ["edg", "iedg"])
def test_traces_in_the_range_of_R_are_continuous(dim, N, k, variant):
    vert, elem = _mesh(dim, N)
    prob = ac.build_problem(vert, elem, k, 1.0, 1.0, 1.0)
    tm = edg.trace_map(prob, variant)
    lam = tm.R @ np.random.default_rng(3).standard_normal(tm.n_free)
    interior = np.nonzero(~prob.sk.boundary)[0]
    faces = {f: lam[r * prob.Nf:(r + 1) * prob.Nf] for r, f in enumerate(interior)}

    def value(f, x):
        Y = vert[prob.sk.faces[f]]
        eta = np.linalg.lstsq((Y[1:] - Y[0]).T, x - Y[0], rcond=None)[0]
        U, _ = ref.basis(dim - 1, k, eta[None, :])
        return float(U[0] @ faces[f])

    checked = 0
    fl = list(faces)
    for a, b in itertools.combinations(fl, 2):
        shared = sorted(set(prob.sk.faces[a].tolist()) & set(prob.sk.faces[b].tolist()))
        if len(shared) != dim - 1:
            continue
        P = vert[shared]
        # 2D: the shared vertex; 3D: k + 1 points inside the shared edge (a degree-k polynomial
        # of the edge coordinate is fixed by them; the face basis is singular at one vertex)
        pts = [P[0]] if dim == 2 else [P[0] + (i + 0.5) / (k + 1) * (P[1] - P[0]) for i in range(k + 1)]
        for x in pts:
            assert abs(value(a, x) - value(b, x)) < 1e-11
            checked += 1
    assert checked > 0


@pytest.mark.parametrize("variant", ["edg", "iedg"])
def test_pressure_converges_at_order_k_plus_1_on_the_standing_mode(variant):
    k = 2
    ex = ac.standing_mode(2)
    T = 0.2
    errs = []
    for N in (2, 4, 8):
        vert, elem = inputs.unit_square_tri(N)
        prob = ac.build_problem(vert, elem, k, 1.0, 1.0, 1.0)
        prob.dirichlet = lambda x, t: ex(x, t)[:, 0]
        u0 = ac.project_volume(prob, lambda x: ex(x, 0.0))
        solve = edg.make_stage_solver(edg.trace_map(prob, variant))
        u, lam, t = ac.run_dirk3(prob, u0, T / (8 * N), 8 * N, solve=solve)
        errs.append(ac.l2_error(prob, u, lambda x: ex(x, T)))
    rate = math.log2(errs[-2] / errs[-1])
    assert rate > k + 1 - 0.25, (errs, rate)


def test_continuous_traces_need_no_more_jacobi_cg_iterations_than_hdg():
    """At the benchmark's c dt / h (acoustic recipe, k = 3, 384 tets) the restricted systems
    R^T (-K) R of EDG and IEDG converge in fewer Jacobi-CG iterations than HDG's -K (run with
    -s to print the counts): fewer unknowns, and no more passes over the same S_K."""
    import scipy.sparse.linalg as spla
    N = 4
    w = inputs.acoustic_3d_workload(N=N, k=3)
    prob = ac.build_problem(w["vert"], w["elem"], 3, w["tau"], w["rho"], w["c"])
    cond = ac.condense(prob, 1.5 / (2e-3 * 32.0 / N))
    b0 = np.random.default_rng(1807).standard_normal(cond.K.shape[0])
    counts = {}
    for name in ("hdg", "iedg", "edg"):
        if name == "hdg":
            A, b = (-cond.K).tocsr(), b0
        else:
            tm = edg.trace_map(prob, name)
            A, b = (tm.R.T @ (-cond.K) @ tm.R).tocsr(), tm.R.T @ b0
        d, n = A.diagonal(), A.shape[0]
        it = [0]

        def cb(_):
            it[0] += 1
        x, info = spla.cg(A, b, rtol=1e-12, atol=0.0, maxiter=2000,
                          M=spla.LinearOperator((n, n), matvec=lambda r: r / d), callback=cb)
        assert info == 0
        counts[name] = (n, it[0])
    print("\nJacobi CG (unknowns, iterations):", counts)
    assert counts["edg"][0] < counts["iedg"][0] < counts["hdg"][0]
    assert counts["edg"][1] <= counts["hdg"][1] and counts["iedg"][1] <= counts["hdg"][1]
