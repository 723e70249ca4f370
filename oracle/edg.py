"""EDG and IEDG trace spaces for the acoustic scheme, plain FP64 oracle (test infrastructure only).

Sec. 2.2 defines the trace space M_h as the piecewise-P_k functions on the skeleton that are
continuous on a subset E^E of the faces: E^E empty gives HDG, E^E = all faces gives EDG, and
E^E = the interior faces gives IEDG (continuous inside, discontinuous across the boundary
faces). The local problems and the element blocks do not change; only the global unknowns do.

A continuous trace on E^E is fixed by its values at the degree-k equispaced nodes of the
faces in E^E, shared between faces that meet at a vertex or edge. On a face F the modal
coefficients (orthonormal face basis mu) are lam_F = V_F^{-1} (nodal values), with
V_F[a][m] = mu_m(eta_a) at the face's reference nodes eta_a. A node is identified globally by
the vertices of the smallest sub-simplex containing it and its integer barycentric weights
on them.

Readings (the paper defines the spaces but writes no EDG/IEDG scheme out):
  * IEDG keeps the HDG treatment of Dirichlet faces: a boundary face carries the L2
    projection of p_D and is not tied to its neighbours. Every node of an interior face is
    an unknown, including the nodes on the boundary.
  * EDG imposes p_D by nodal interpolation. A boundary face's trace is the interpolant of
    p_D at its nodes, and nodes on the boundary are fixed to p_D there.
  * The discrete equations are the HDG jump conditions tested with the continuous test
    functions, that is R^T (K lam - r) = 0, with R the map from free nodal values to modal
    face coefficients (Galerkin restriction of the HDG trace system).
"""
import itertools
from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import acoustic as ac
from . import reference as ref


def face_nodes(dim, k):
    """Integer barycentric weights (b_0..b_{dim-1}, sum k) of the degree-k equispaced nodes of a
    face with dim vertices, and the reference coordinates eta = (b_1, .., b_{dim-1}) / k."""
    nv = dim
    bs = [b for b in itertools.product(range(k + 1), repeat=nv) if sum(b) == k]
    eta = np.array([[b[i] / k for i in range(1, nv)] for b in bs])
    return bs, eta


def nodal_to_modal(fdim, k, eta):
    """Matrix taking values at the nodes eta (unisolvent for P_k on the reference face) to
    coefficients in the orthonormal face basis: the L2 projection of each Lagrange function,
    with the Lagrange functions built from monomials (no evaluation of the collapsed-coordinate
    basis at the nodes, where it is singular at the top vertex)."""
    exps = [m for m in itertools.product(range(k + 1), repeat=fdim) if sum(m) <= k]
    W = np.array([[np.prod(x ** np.array(m)) for m in exps] for x in eta])
    xq, wq = ref.simplex_rule(fdim, k + 2)
    Wq = np.array([[np.prod(x ** np.array(m)) for m in exps] for x in xq])
    L = Wq @ np.linalg.inv(W)              # L[q][a] = ell_a(x_q)
    Uq, _ = ref.basis(fdim, k, xq)
    return np.einsum("q,qm,qa->ma", wq, Uq, L)


@dataclass
class TraceMap:
    variant: str
    R: object              # sparse [n_int * Nf, n_free]: free nodal values -> interior-face modal coefficients
    R_fix: object          # sparse [n_int * Nf, n_fixed] (EDG: nodes on the boundary)
    fixed_xyz: np.ndarray  # [n_fixed, d] positions of the fixed nodes
    n_free: int
    face_modal: list       # per face: (node ids, is_free mask) in the face's node order
    Vinv: np.ndarray       # V_F^{-1}, the same for every face (reference nodes, reference basis)


def trace_map(prob, variant):
    """R for variant "edg" or "iedg" (interior trace unknowns in the order of ac.condense)."""
    assert variant in ("edg", "iedg")
    sk, k, Nf = prob.sk, prob.k, prob.Nf
    dim = sk.dim
    bs, eta = face_nodes(dim, k)
    Vinv = nodal_to_modal(dim - 1, k, eta)
    faces = range(sk.faces.shape[0]) if variant == "edg" else np.nonzero(~sk.boundary)[0]
    bnd_subsimplices = set()
    for f in np.nonzero(sk.boundary)[0]:
        fv = sk.faces[f]
        for r in range(1, dim + 1):
            for sub in itertools.combinations(fv.tolist(), r):
                bnd_subsimplices.add(sub)
    key_id, keys, on_bnd, xyz = {}, [], [], []
    face_modal = {}
    for f in faces:
        fv = sk.faces[f]                     # ascending global ids = the face parametrisation
        ids = []
        for b in bs:
            key = tuple((int(fv[i]), b[i]) for i in range(dim) if b[i] > 0)
            if key not in key_id:
                key_id[key] = len(keys)
                keys.append(key)
                support = tuple(v for v, _ in key)
                on_bnd.append(support in bnd_subsimplices)
                xyz.append(sum(w * prob.vert[v] for v, w in key) / k)
            ids.append(key_id[key])
        face_modal[f] = ids
    on_bnd = np.array(on_bnd, dtype=bool)
    fixed = on_bnd if variant == "edg" else np.zeros(len(keys), dtype=bool)
    free_pos = -np.ones(len(keys), dtype=np.int64)
    free_pos[~fixed] = np.arange(int((~fixed).sum()))
    fix_pos = -np.ones(len(keys), dtype=np.int64)
    fix_pos[fixed] = np.arange(int(fixed.sum()))
    interior = np.nonzero(~sk.boundary)[0]
    rows, cols, vals, frows, fcols, fvals = [], [], [], [], [], []
    for r_f, f in enumerate(interior):
        ids = face_modal[f]
        for m in range(Nf):
            for a, node in enumerate(ids):
                if fixed[node]:
                    frows.append(r_f * Nf + m); fcols.append(fix_pos[node]); fvals.append(Vinv[m, a])
                else:
                    rows.append(r_f * Nf + m); cols.append(free_pos[node]); vals.append(Vinv[m, a])
    n_free, n_fixed = int((~fixed).sum()), int(fixed.sum())
    R = sp.csr_matrix((vals, (rows, cols)), shape=(interior.size * Nf, n_free))
    R_fix = sp.csr_matrix((fvals, (frows, fcols)), shape=(interior.size * Nf, n_fixed))
    fixed_xyz = np.array(xyz)[fixed] if n_fixed else np.zeros((0, dim))
    fm = [None] * sk.faces.shape[0]
    for f, ids in face_modal.items():
        fm[f] = (np.array(ids), ~fixed[np.array(ids)])
    return TraceMap(variant, R, R_fix, fixed_xyz, n_free, fm, Vinv)


def boundary_traces(prob, tm, t):
    """Traces of the boundary faces at time t ([Nfaces, Nf], zero on interior faces): the L2
    projection of p_D (IEDG, as in HDG) or its interpolant at the face nodes (EDG)."""
    if tm.variant == "iedg":
        return ac.dirichlet_values(prob, t)
    sk = prob.sk
    lam = np.zeros((sk.faces.shape[0], prob.Nf))
    if prob.dirichlet is None:
        return lam
    dim, k = sk.dim, prob.k
    bs, _ = face_nodes(dim, k)
    for f in np.nonzero(sk.boundary)[0]:
        fv = sk.faces[f]
        x = np.array([sum(b[i] * prob.vert[fv[i]] for i in range(dim)) / k for b in bs])
        lam[f] = tm.Vinv @ prob.dirichlet(x, t)
    return lam


def make_stage_solver(tm):
    """Stage solve of the restricted trace system, same signature as ac.solve_stage."""

    def solve(prob, cond, hist, t):
        lamB = boundary_traces(prob, tm, t)
        F = ac.element_rhs(prob, cond, hist, t, lamB)
        r = ac.condensed_rhs(prob, cond, F)
        lam_int = np.zeros(r.size)
        if tm.R_fix.shape[1]:
            mu_fix = prob.dirichlet(tm.fixed_xyz, t) if prob.dirichlet is not None else np.zeros(tm.R_fix.shape[1])
            lam_int += tm.R_fix @ mu_fix
        rhs = tm.R.T @ (r - cond.K @ lam_int)
        Kr = (tm.R.T @ cond.K @ tm.R).tocsc()
        mu = spla.spsolve(Kr, rhs) if rhs.size else rhs
        lam_int = lam_int + tm.R @ mu
        lam_I = np.zeros_like(lamB)
        lam_I[cond.interior] = lam_int.reshape(-1, prob.Nf)
        u = ac.recover(prob, cond, F, lam_I)
        return u, lam_I + lamB

    return solve
