"""Acoustic HDG scheme, plain FP64 oracle (test infrastructure only).

Physics. First-order acoustics (1/(rho c^2)) dp/dt + div v = s, rho dv/dt + grad p = 0.
The paper does not write this scheme out; it is the scalar (m = 1) specialisation of
the paper's HDG template: spaces of Eqs. e:spaces1/e:spaces2 (Sec. 2.2), the numerical
flux pattern of Eq. eq:HDG_linelas5 (v_hat.n = v.n + tau (p - p_hat)) and the global
jump condition of Eq. eq:HDG_linelas4, with the trace p_hat prescribed on Dirichlet faces.

Local equations on each element K, for all test functions (w, r) in P_k x [P_k]^d:
  (dp/dt/(rho c^2), w) + (div v, w) + <tau (p - p_hat), w>_dK - (s, w) = 0
  (rho dv/dt, r) - (p, div r) + <p_hat, r.n>_dK = 0
and on every interior face F, for all mu in P_k(F):
  sum_{K ∋ F} <v.n + tau (p - p_hat), mu>_F = 0.

This is the DAE M du/dt + f(u, v_hat, t) = 0, g(u, v_hat, t) = 0 of Sec. 2.3
(Eq. ch5appendx1:eq8). Each implicit BDF step (Eq. ch5appendx1:eq9b) or DIRK stage
(Eq. ch5appendx1:eq10_1) is the linear system
  A u + B lam = F,   C u + D lam = 0   (interior faces)
with A = alpha M + df/du, alpha = a_s / (b_s dt) (BDF) or d_ii / dt (DIRK), which is
eliminated element by element (Sec. 2.4, Eq. LS): K = D - C A^{-1} B,
r = -C A^{-1} F, local recovery u = A^{-1} (F - B lam).

Conventions (readings of a paper that fixes none of them; the CUDA library follows
the same ones, written independently):
  * element vertices are taken in ascending global id; x = X0 + sum_r xi_r (X_r - X0);
  * local face j is the face opposite local vertex j; a face is parametrised from its
    vertices in ascending global id (so both neighbours see the same face basis);
  * faces are numbered in lexicographic order of their sorted vertex tuples;
  * element unknowns are ordered [p, v_1, ..., v_d], each a block of N_p coefficients
    in the orthonormal reference basis of oracle/reference.py (unscaled, so the
    physical mass matrix is |det J| I);
  * element trace unknowns are ordered [face 0, ..., face d], N_f coefficients each;
  * quadrature uses n = k + 2 collapsed Gauss points per direction (degree 2k + 3).
The Ricker wavelet (pinned as the normalised second derivative of a Gaussian) and the
point-source element (the lowest id among elements containing the point, pinned by a brute-force
barycentric search) are conventions of the workload, not results of the method; both are
pinned by tests in tests/test_oracle_acoustic.py.
"""
import math
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import reference as ref


# ----------------------------------------------------------------------------- mesh (Sec. 2.1)

@dataclass
class Skeleton:
    """Faces of the mesh (E_h = E_h^I u E_h^B, Sec. 2.1) and element-face incidence."""
    dim: int
    elem: np.ndarray        # [Ne, d+1] vertex ids, ascending per element
    faces: np.ndarray       # [Nf, d] sorted vertex ids, lexicographic order
    elem_face: np.ndarray   # [Ne, d+1] face id of local face j (opposite local vertex j)
    face_elems: list        # per face: list of (element, local face), element ascending
    boundary: np.ndarray    # [Nf] bool, True for faces on the domain boundary


def skeleton(elem_vert):
    elem = np.sort(np.asarray(elem_vert, dtype=np.int64), axis=1)
    ne, nv = elem.shape
    dim = nv - 1
    keys = {}
    for e in range(ne):
        for j in range(nv):
            f = tuple(int(v) for i, v in enumerate(elem[e]) if i != j)
            keys.setdefault(f, []).append((e, j))
    faces_sorted = sorted(keys)
    fid = {f: i for i, f in enumerate(faces_sorted)}
    elem_face = np.zeros((ne, nv), dtype=np.int64)
    face_elems = []
    for f in faces_sorted:
        inc = sorted(keys[f])
        if len(inc) > 2:
            raise ValueError("non-manifold face %r" % (f,))
        face_elems.append(inc)
        for (e, j) in inc:
            elem_face[e, j] = fid[f]
    boundary = np.array([len(x) == 1 for x in face_elems])
    return Skeleton(dim, elem, np.array(faces_sorted, dtype=np.int64), elem_face, face_elems, boundary)


# ----------------------------------------------------------------------------- element blocks

@dataclass
class ElementBlocks:
    """Per-element matrices of the local Galerkin projection (ingredient (i) of the abstract)."""
    Mw: np.ndarray    # weighted mass blockdiag(M/(rho c^2), rho M, ..)  (n x n)
    A0: np.ndarray    # df/du (spatial part of A)                         (n x n)
    B: np.ndarray     # df/dlam                                            (n x m)
    C: np.ndarray     # dg/du                                              (m x n)
    D: np.ndarray     # dg/dlam                                            (m x m)
    E: list           # per local face, <phi_i, phi_l>_F                  (Np x Np)
    Fm: list          # per local face, <phi_i, mu_m>_F                   (Np x Nf)
    G: list           # per local face, <mu_m, mu_m'>_F                   (Nf x Nf)
    normal: np.ndarray
    detJ: float
    Jinv: np.ndarray
    X: np.ndarray


def face_local_vertices(dim, j):
    return [i for i in range(dim + 1) if i != j]


def face_frame(Y):
    """Face map Jacobian (length or area scaling) for a face with vertex rows Y."""
    if Y.shape[0] == 2:
        return np.linalg.norm(Y[1] - Y[0])
    return np.linalg.norm(np.cross(Y[1] - Y[0], Y[2] - Y[0]))


def outward_normal(X, j):
    dim = X.shape[1]
    Y = X[face_local_vertices(dim, j)]
    if dim == 2:
        t = Y[1] - Y[0]
        n = np.array([t[1], -t[0]])
    else:
        n = np.cross(Y[1] - Y[0], Y[2] - Y[0])
    n = n / np.linalg.norm(n)
    if np.dot(n, X[j] - Y[0]) > 0:
        n = -n
    return n


def element_blocks(X, k, rho, c, tau):
    """Local blocks of one element with vertex coordinates X (rows in ascending global id)."""
    X = np.asarray(X, dtype=np.float64)
    dim = X.shape[1]
    Np = ref.n_modes(dim, k)
    Nf = ref.n_modes(dim - 1, k)
    J = (X[1:] - X[0]).T
    detJ = abs(np.linalg.det(J))
    Jinv = np.linalg.inv(J)
    xi, wq = ref.simplex_rule(dim, k + 2)
    V, G = ref.basis(dim, k, xi)
    Gx = np.einsum("qir,rj->qij", G, Jinv)          # physical gradients
    M = np.einsum("q,qi,ql->il", wq * detJ, V, V)
    Dx = [np.einsum("q,qi,ql->il", wq * detJ, V, Gx[:, :, j]) for j in range(dim)]  # (d_j phi_l, phi_i)

    eta, wf = ref.simplex_rule(dim - 1, k + 2)
    U, _ = ref.basis(dim - 1, k, eta)
    E, Fm, Gm, normals = [], [], [], []
    for j in range(dim + 1):
        Y = X[face_local_vertices(dim, j)]
        xq = Y[0] + eta @ (Y[1:] - Y[0])
        JF = face_frame(Y)
        xiq = (xq - X[0]) @ Jinv.T
        Vf, _ = ref.basis(dim, k, xiq)
        E.append(np.einsum("q,qi,ql->il", wf * JF, Vf, Vf))
        Fm.append(np.einsum("q,qi,qm->im", wf * JF, Vf, U))
        Gm.append(np.einsum("q,qm,qn->mn", wf * JF, U, U))
        normals.append(outward_normal(X, j))
    normals = np.array(normals)

    n = (dim + 1) * Np
    m = (dim + 1) * Nf
    P = slice(0, Np)
    Vs = [slice((j + 1) * Np, (j + 2) * Np) for j in range(dim)]
    Fs = [slice(f * Nf, (f + 1) * Nf) for f in range(dim + 1)]
    Mw = np.zeros((n, n))
    Mw[P, P] = M / (rho * c * c)
    for j in range(dim):
        Mw[Vs[j], Vs[j]] = rho * M
    A0 = np.zeros((n, n))
    A0[P, P] = tau * sum(E)
    for j in range(dim):
        A0[P, Vs[j]] = Dx[j]
        A0[Vs[j], P] = -Dx[j].T
    B = np.zeros((n, m))
    C = np.zeros((m, n))
    D = np.zeros((m, m))
    for f in range(dim + 1):
        B[P, Fs[f]] = -tau * Fm[f]
        C[Fs[f], P] = tau * Fm[f].T
        for j in range(dim):
            B[Vs[j], Fs[f]] = normals[f, j] * Fm[f]
            C[Fs[f], Vs[j]] = normals[f, j] * Fm[f].T
        D[Fs[f], Fs[f]] = -tau * Gm[f]
    return ElementBlocks(Mw, A0, B, C, D, E, Fm, Gm, normals, detJ, Jinv, X)


# ----------------------------------------------------------------------------- problem

def ricker(t, f0, t0):
    """Ricker wavelet (1 - 2 pi^2 f0^2 (t-t0)^2) exp(-pi^2 f0^2 (t-t0)^2)."""
    a = (math.pi * f0 * (t - t0)) ** 2
    return (1.0 - 2.0 * a) * math.exp(-a)


@dataclass
class Problem:
    """Mesh + degree + material + data; element blocks formed once (alpha-independent)."""
    vert: np.ndarray
    sk: Skeleton
    k: int
    tau: float
    rho: np.ndarray
    c: np.ndarray
    blocks: list
    Np: int
    Nf: int
    sources: list = field(default_factory=list)     # (elem, phi values at x_s, f0, t0, amp)
    dirichlet: object = None                         # callable (x[nq, d], t) -> values, or None (zero)


def build_problem(vert, elem_vert, k, tau, rho, c):
    vert = np.asarray(vert, dtype=np.float64)
    sk = skeleton(elem_vert)
    ne = sk.elem.shape[0]
    rho = np.broadcast_to(np.asarray(rho, dtype=np.float64), (ne,)).copy()
    c = np.broadcast_to(np.asarray(c, dtype=np.float64), (ne,)).copy()
    blocks = [element_blocks(vert[sk.elem[e]], k, rho[e], c[e], tau) for e in range(ne)]
    return Problem(vert, sk, k, tau, rho, c, blocks,
                   ref.n_modes(sk.dim, k), ref.n_modes(sk.dim - 1, k))


def locate(prob, x):
    """Lowest-id element whose closure contains x (barycentric test)."""
    x = np.asarray(x, dtype=np.float64)
    for e in range(prob.sk.elem.shape[0]):
        bl = prob.blocks[e]
        xi = bl.Jinv @ (x - bl.X[0])
        if xi.min() >= -1e-12 and xi.sum() <= 1.0 + 1e-12:
            return e, xi
    raise ValueError("point outside mesh")


def add_point_source(prob, x, f0, t0, amp=1.0):
    """Point source s = amp r(t) delta(x - x_s) in the pressure equation: (s, w)_K = amp r(t) w(x_s)."""
    e, xi = locate(prob, x)
    V, _ = ref.basis(prob.sk.dim, prob.k, xi[None, :])
    prob.sources.append((e, V[0].copy(), f0, t0, amp))


def project_volume(prob, func):
    """Element-wise L2 projection of func(x[nq, d]) -> [nq, d+1] values of (p, v_1..v_d)."""
    dim, k, Np = prob.sk.dim, prob.k, prob.Np
    xi, wq = ref.simplex_rule(dim, k + 2)
    V, _ = ref.basis(dim, k, xi)
    u = np.zeros((prob.sk.elem.shape[0], (dim + 1) * Np))
    for e, bl in enumerate(prob.blocks):
        J = (bl.X[1:] - bl.X[0]).T
        x = bl.X[0] + xi @ J.T
        vals = func(x)
        M = np.einsum("q,qi,ql->il", wq * bl.detJ, V, V)
        for comp in range(dim + 1):
            rhs = np.einsum("q,qi,q->i", wq * bl.detJ, V, vals[:, comp])
            u[e, comp * Np:(comp + 1) * Np] = np.linalg.solve(M, rhs)
    return u


def project_face(prob, f, func, t):
    """L2 projection of a scalar func(x, t) on face f onto its trace basis."""
    dim, k = prob.sk.dim, prob.k
    Y = prob.vert[prob.sk.faces[f]]
    eta, wf = ref.simplex_rule(dim - 1, k + 2)
    U, _ = ref.basis(dim - 1, k, eta)
    xq = Y[0] + eta @ (Y[1:] - Y[0])
    JF = face_frame(Y)
    G = np.einsum("q,qm,qn->mn", wf * JF, U, U)
    return np.linalg.solve(G, np.einsum("q,qm,q->m", wf * JF, U, func(xq, t)))


def dirichlet_values(prob, t):
    """Trace values on boundary faces at time t ([Nfaces, Nf], zero on interior faces)."""
    nf = prob.sk.faces.shape[0]
    lam = np.zeros((nf, prob.Nf))
    if prob.dirichlet is None:
        return lam
    for f in np.nonzero(prob.sk.boundary)[0]:
        lam[f] = project_face(prob, f, prob.dirichlet, t)
    return lam


def source_vector(prob, e, t):
    s = np.zeros((prob.sk.dim + 1) * prob.Np)
    for (es, phi, f0, t0, amp) in prob.sources:
        if es == e:
            s[:prob.Np] += amp * ricker(t, f0, t0) * phi
    return s


def local_traces(prob, e, lam):
    """Gather lam_K = [lam_{face 0}, ..., lam_{face d}] from a face-major array."""
    return np.concatenate([lam[prob.sk.elem_face[e, j]] for j in range(prob.sk.dim + 1)])


# ----------------------------------------------------------------------------- condensation (Eq. LS)

@dataclass
class Condensed:
    alpha: float
    lu: list          # per element LU of A_K = alpha Mw + A0 (partial pivoting)
    S: list           # per element S_K = D_K - C_K A_K^{-1} B_K
    K: object         # assembled interior trace operator (sparse)
    interior: np.ndarray   # interior face ids in trace-unknown order


def condense(prob, alpha):
    """Static condensation at mass shift alpha: K = sum_K P_K^T S_K P_K over interior faces."""
    sk, Nf = prob.sk, prob.Nf
    interior = np.nonzero(~sk.boundary)[0]
    pos = -np.ones(sk.faces.shape[0], dtype=np.int64)
    pos[interior] = np.arange(interior.size)
    lus, Ss = [], []
    rows, cols, vals = [], [], []
    for e, bl in enumerate(prob.blocks):
        A = alpha * bl.Mw + bl.A0
        lu = sla.lu_factor(A)
        S = bl.D - bl.C @ sla.lu_solve(lu, bl.B)
        lus.append(lu)
        Ss.append(S)
        for a in range(sk.dim + 1):
            pa = pos[sk.elem_face[e, a]]
            if pa < 0:
                continue
            for b in range(sk.dim + 1):
                pb = pos[sk.elem_face[e, b]]
                if pb < 0:
                    continue
                blk = S[a * Nf:(a + 1) * Nf, b * Nf:(b + 1) * Nf]
                ii, jj = np.meshgrid(np.arange(Nf) + pa * Nf, np.arange(Nf) + pb * Nf, indexing="ij")
                rows.append(ii.ravel())
                cols.append(jj.ravel())
                vals.append(blk.ravel())
    nI = interior.size * Nf
    if rows:
        K = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(nI, nI))
    else:
        K = sp.csr_matrix((nI, nI))
    return Condensed(alpha, lus, Ss, K, interior)


def element_rhs(prob, cond, hist, t, lamD):
    """F~_K = alpha Mw h_K + s_K(t) - B_K lam_D,K (Dirichlet traces moved to the right)."""
    ne = prob.sk.elem.shape[0]
    F = np.zeros_like(hist)
    for e, bl in enumerate(prob.blocks):
        F[e] = cond.alpha * bl.Mw @ hist[e] + source_vector(prob, e, t) - bl.B @ local_traces(prob, e, lamD)
    return F


def condensed_rhs(prob, cond, F):
    """r = -sum_K P_K^T C_K A_K^{-1} F~_K restricted to interior faces (Eq. LS)."""
    sk, Nf = prob.sk, prob.Nf
    pos = -np.ones(sk.faces.shape[0], dtype=np.int64)
    pos[cond.interior] = np.arange(cond.interior.size)
    r = np.zeros(cond.interior.size * Nf)
    for e, bl in enumerate(prob.blocks):
        g = -bl.C @ sla.lu_solve(cond.lu[e], F[e])
        for a in range(sk.dim + 1):
            pa = pos[sk.elem_face[e, a]]
            if pa >= 0:
                r[pa * Nf:(pa + 1) * Nf] += g[a * Nf:(a + 1) * Nf]
    return r


def trace_apply(prob, cond, lam_int):
    """y = K lam for interior trace values lam_int[(n_int*Nf)] (element by element)."""
    sk, Nf = prob.sk, prob.Nf
    lam = np.zeros((sk.faces.shape[0], Nf))
    lam[cond.interior] = lam_int.reshape(-1, Nf)
    y = np.zeros_like(lam)
    for e in range(sk.elem.shape[0]):
        z = cond.S[e] @ local_traces(prob, e, lam)
        for a in range(sk.dim + 1):
            y[sk.elem_face[e, a]] += z[a * Nf:(a + 1) * Nf]
    return y[cond.interior].ravel()


def recover(prob, cond, F, lam):
    """Local recovery u_K = A_K^{-1} (F~_K - B_K lam_K), lam zero on Dirichlet faces."""
    u = np.zeros_like(F)
    for e, bl in enumerate(prob.blocks):
        u[e] = sla.lu_solve(cond.lu[e], F[e] - bl.B @ local_traces(prob, e, lam))
    return u


def solve_stage(prob, cond, hist, t):
    """One implicit solve: alpha Mw u + f(u, lam, t) = alpha Mw hist, g = 0; returns (u, lam)."""
    lamD = dirichlet_values(prob, t)
    F = element_rhs(prob, cond, hist, t, lamD)
    r = condensed_rhs(prob, cond, F)
    lam_int = spla.spsolve(cond.K.tocsc(), r) if r.size else r
    lam_I = np.zeros_like(lamD)
    lam_I[cond.interior] = lam_int.reshape(-1, prob.Nf)
    u = recover(prob, cond, F, lam_I)
    return u, lam_I + lamD


# ----------------------------------------------------------------------------- time marching (Sec. 2.3)

BDF = {1: ([-1.0, 1.0], 1.0), 2: ([0.5, -2.0, 1.5], 1.0)}   # (a_0..a_s, b_s), Eq. ch5appendx1:eq9b


def dirk3_tableau():
    """Alexander's 3-stage L-stable SDIRK (the DIRK(3,3) the paper cites; tableau not printed).

    gamma is the root in (1/3, 1/2) of gamma^3 - 3 gamma^2 + 3/2 gamma - 1/6 = 0.
    """
    roots = np.roots([1.0, -3.0, 1.5, -1.0 / 6.0])
    g = float([r.real for r in roots if abs(r.imag) < 1e-12 and 1 / 3 < r.real < 0.5][0])
    b1 = -(6 * g * g - 16 * g + 1) / 4
    b2 = (6 * g * g - 20 * g + 5) / 4
    a = np.array([[g, 0, 0], [(1 - g) / 2, g, 0], [b1, b2, g]])
    b = np.array([b1, b2, g])
    c = np.array([g, (1 + g) / 2, 1.0])
    return a, b, c


def run_bdf(prob, u0, dt, nsteps, order, t0=0.0, u_prev=None, on_step=None, solve=None):
    """BDF(order) marching (Eq. ch5appendx1:eq9b); order 2 starts from u^{-1} = u_prev (default u0).
    solve(prob, cond, hist, t) -> (u, lam) is the stage solve (default: solve_stage, HDG traces)."""
    solve = solve or solve_stage
    a, bs = BDF[order]
    alpha = a[-1] / (bs * dt)
    cond = condense(prob, alpha)
    hist_u = [u0.copy()] if order == 1 else [(u0 if u_prev is None else u_prev).copy(), u0.copy()]
    lam = None
    t = t0
    for n in range(nsteps):
        t = t0 + (n + 1) * dt
        h = -sum(a[i] * hist_u[i] for i in range(order)) / a[-1]
        u, lam = solve(prob, cond, h, t)
        hist_u = hist_u[1:] + [u]
        if on_step is not None:
            on_step(n, t, u, lam)
    return hist_u[-1], lam, t


def run_dirk3(prob, u0, dt, nsteps, t0=0.0, on_step=None, solve=None):
    """DIRK(3,3) marching in the stage form of Eq. ch5appendx1:eq10_1 with update Eq. 10_2.
    solve(prob, cond, hist, t) -> (u, lam) is the stage solve (default: solve_stage, HDG traces)."""
    solve = solve or solve_stage
    a, b, c = dirk3_tableau()
    d = np.linalg.inv(a)
    e = b @ d
    s = len(b)
    cond = condense(prob, d[0, 0] / dt)
    u = u0.copy()
    lam = None
    for n in range(nsteps):
        tn = t0 + n * dt
        stages = []
        for i in range(s):
            if abs(d[i, i] / dt - cond.alpha) > 1e-12 * cond.alpha:
                cond = condense(prob, d[i, i] / dt)
            # sum_j d_ij (u^{n,j} - u^n) + dt f(u^{n,i}) = 0, j <= i (d lower triangular)
            h = (sum(d[i, j] for j in range(i + 1)) * u - sum(d[i, j] * stages[j] for j in range(i))) / d[i, i]
            ui, lam = solve(prob, cond, h, tn + c[i] * dt)
            stages.append(ui)
        u = (1.0 - b @ d.sum(axis=1)) * u + sum(e[j] * stages[j] for j in range(s))
        if on_step is not None:
            on_step(n, tn + dt, u, lam)
    return u, lam, t0 + nsteps * dt


# ----------------------------------------------------------------------------- brute force and diagnostics

def solve_monolithic(prob, alpha, hist, t):
    """Uncondensed [A B; C D] system over all element and face unknowns, dense LU.

    Element rows: A_K u_K + B_K lam_K = alpha Mw h_K + s_K; interior face rows: the jump
    condition; Dirichlet face rows: <lam - p_D, mu>_F = 0.
    """
    sk, Np, Nf = prob.sk, prob.Np, prob.Nf
    ne, nf = sk.elem.shape[0], sk.faces.shape[0]
    n = (sk.dim + 1) * Np
    N = ne * n + nf * Nf
    Mat = np.zeros((N, N))
    rhs = np.zeros(N)
    lamD = dirichlet_values(prob, t)
    for e, bl in enumerate(prob.blocks):
        r0 = e * n
        Mat[r0:r0 + n, r0:r0 + n] = alpha * bl.Mw + bl.A0
        rhs[r0:r0 + n] = alpha * bl.Mw @ hist[e] + source_vector(prob, e, t)
        for a in range(sk.dim + 1):
            fa = sk.elem_face[e, a]
            c0 = ne * n + fa * Nf
            Mat[r0:r0 + n, c0:c0 + Nf] = bl.B[:, a * Nf:(a + 1) * Nf]
            if not sk.boundary[fa]:
                Mat[c0:c0 + Nf, r0:r0 + n] += bl.C[a * Nf:(a + 1) * Nf]
                Mat[c0:c0 + Nf, c0:c0 + Nf] += bl.D[a * Nf:(a + 1) * Nf, a * Nf:(a + 1) * Nf]
    for f in np.nonzero(sk.boundary)[0]:
        c0 = ne * n + f * Nf
        e, a = sk.face_elems[f][0]
        G = prob.blocks[e].G[a]
        Mat[c0:c0 + Nf, c0:c0 + Nf] = G
        rhs[c0:c0 + Nf] = G @ lamD[f]
    x = np.linalg.solve(Mat, rhs)
    return x[:ne * n].reshape(ne, n), x[ne * n:].reshape(nf, Nf)


def energy(prob, u):
    """Discrete energy E = 1/2 sum_K u_K^T Mw_K u_K = 1/2 (p/(rho c^2), p) + 1/2 (rho v, v)."""
    return 0.5 * sum(u[e] @ bl.Mw @ u[e] for e, bl in enumerate(prob.blocks))


def energy_terms(prob, u, lam, t):
    """Dissipation sum_dK <tau (p - p_hat)^2, 1>, boundary work <p_hat, v_hat.n>_{Gamma_D}, (s, p)."""
    sk, Np, Nf, tau = prob.sk, prob.Np, prob.Nf, prob.tau
    diss, bwork, src = 0.0, 0.0, 0.0
    for e, bl in enumerate(prob.blocks):
        p = u[e, :Np]
        lk = local_traces(prob, e, lam)
        flux = bl.C @ u[e] + bl.D @ lk            # <v.n + tau (p - lam), mu>_F per local face
        for a in range(sk.dim + 1):
            la = lk[a * Nf:(a + 1) * Nf]
            diss += tau * (p @ bl.E[a] @ p - 2 * p @ bl.Fm[a] @ la + la @ bl.G[a] @ la)
            if sk.boundary[sk.elem_face[e, a]]:
                bwork += la @ flux[a * Nf:(a + 1) * Nf]
        src += source_vector(prob, e, t) @ u[e]
    return diss, bwork, src


def l2_error(prob, u, exact, comp=0, nq=None):
    """|| u_h[comp] - exact(x)[comp] ||_{L2(Omega)} with a high-order rule."""
    dim, k, Np = prob.sk.dim, prob.k, prob.Np
    xi, wq = ref.simplex_rule(dim, nq or k + 4)
    V, _ = ref.basis(dim, k, xi)
    err = 0.0
    for e, bl in enumerate(prob.blocks):
        J = (bl.X[1:] - bl.X[0]).T
        x = bl.X[0] + xi @ J.T
        uh = V @ u[e, comp * Np:(comp + 1) * Np]
        err += np.sum(wq * bl.detJ * (uh - exact(x)[:, comp]) ** 2)
    return math.sqrt(err)


def standing_mode(dim):
    """Exact standing mode of the unit-square/cube acoustic problem, rho = c = 1.

    p = prod cos(pi x_i) cos(sqrt(d) pi t), v_j = sin(sqrt(d) pi t)/sqrt(d) sin(pi x_j) prod_{i!=j} cos(pi x_i).
    """
    w = math.sqrt(dim) * math.pi

    def fields(x, t):
        cs = np.cos(math.pi * x)
        sn = np.sin(math.pi * x)
        out = np.zeros((x.shape[0], dim + 1))
        out[:, 0] = np.prod(cs, axis=1) * math.cos(w * t)
        for j in range(dim):
            prod = sn[:, j].copy()
            for i in range(dim):
                if i != j:
                    prod *= cs[:, i]
            out[:, j + 1] = math.sin(w * t) / math.sqrt(dim) * prod
        return out

    return fields


# ----------------------------------------------------------------------------- local post-processing

def postprocess_pressure(prob, u, lam):
    """Element-local post-processed pressure p* in P_{k+1}(K) (Sec. 1: the HDG local
    post-processing step that gives a superconvergent scalar; the paper names the step but
    writes no formula for this scheme).

    Reading (the standard HDG post-processing with the method's own discrete gradient):
      1. q_h in [P_k(K)]^d is the gradient of (p_h, p_hat_h) that the local momentum
         equation defines: (q_h, r)_K = -(p_h, div r)_K + <p_hat_h, r.n>_dK for every
         r in [P_k(K)]^d, so that rho dv_h/dt = -q_h;
      2. p* solves (grad p*, grad w)_K = (q_h, grad w)_K for every w in P_{k+1}(K) and
         (p*, 1)_K = (p_h, 1)_K (the constant mode of the Neumann problem).
    u: [Ne, (d+1) Np] fields (pressure block first); lam: [Nfaces, Nf] traces including the
    Dirichlet values on boundary faces. Returns [Ne, Np(k+1)] coefficients of p* in the
    orthonormal degree-(k+1) basis of oracle/reference.py.
    """
    dim, k, Np, Nf = prob.sk.dim, prob.k, prob.Np, prob.Nf
    Np1 = ref.n_modes(dim, k + 1)
    xi, wq = ref.simplex_rule(dim, k + 3)
    V, G = ref.basis(dim, k, xi)
    V1, G1 = ref.basis(dim, k + 1, xi)
    eta, wf = ref.simplex_rule(dim - 1, k + 3)
    U, _ = ref.basis(dim - 1, k, eta)
    out = np.zeros((prob.sk.elem.shape[0], Np1))
    for e, bl in enumerate(prob.blocks):
        Gx = np.einsum("qir,rj->qij", G, bl.Jinv)       # grad phi_i at the points, [nq, Np, d]
        G1x = np.einsum("qir,rj->qij", G1, bl.Jinv)
        w = wq * bl.detJ
        ph = V @ u[e, :Np]                              # p_h at the points
        # step 1: the discrete gradient q_h, one component at a time
        M = np.einsum("q,qi,ql->il", w, V, V)
        q = np.zeros((dim, Np))
        for j in range(dim):
            rhs = -np.einsum("q,q,qi->i", w, ph, Gx[:, :, j])
            for f in range(dim + 1):
                Y = bl.X[face_local_vertices(dim, f)]
                xq = Y[0] + eta @ (Y[1:] - Y[0])
                Vf, _ = ref.basis(dim, k, (xq - bl.X[0]) @ bl.Jinv.T)
                phat = U @ lam[prob.sk.elem_face[e, f]]
                rhs += bl.normal[f, j] * np.einsum("q,q,qi->i", wf * face_frame(Y), phat, Vf)
            q[j] = np.linalg.solve(M, rhs)
        qx = V @ q.T                                    # q_h at the points, [nq, d]
        # step 2: Neumann problem in P_{k+1}; the constant mode's row (all zero in the
        # stiffness) carries the mean condition instead
        A = np.einsum("q,qid,qld->il", w, G1x, G1x)
        b = np.einsum("q,qd,qid->i", w, qx, G1x)
        A[0] = np.einsum("q,ql->l", w, V1)
        b[0] = np.sum(w * ph)
        out[e] = np.linalg.solve(A, b)
    return out


def l2_error_post(prob, pstar, exact, nq=None):
    """|| p* - exact(x)[0] ||_{L2(Omega)} for degree-(k+1) coefficients p*."""
    dim, k = prob.sk.dim, prob.k
    xi, wq = ref.simplex_rule(dim, nq or k + 5)
    V1, _ = ref.basis(dim, k + 1, xi)
    err = 0.0
    for e, bl in enumerate(prob.blocks):
        x = bl.X[0] + xi @ (bl.X[1:] - bl.X[0])
        err += np.sum(wq * bl.detJ * (V1 @ pstar[e] - exact(x)[:, 0]) ** 2)
    return math.sqrt(err)
