"""Variable-degree linear elastodynamics HDG, plain FP64 oracle (test infrastructure only).

The velocity / symmetric-stress scheme of oracle/elastic.py (Sec. 4.1, Eqs. LE, LEM,
eq:HDG_linelas1-5, eq:stab_matrix_lin) with a polynomial degree k_K chosen per element:
v_h and sigma_h are P_{k_K} on K (the spaces of Sec. 2.2, Eqs. e:spaces1, e:spaces2, taken
element by element), and the trace v_hat on a face F is P_{k_F}(F) with
k_F = max(k_K over the elements sharing F). The paper fixes one k for the whole mesh; the
max rule is the reading that keeps every face space at least as rich as the traces of its
neighbours' fields, so the face terms <sigma n, mu> and <v, mu> are integrated exactly.

Layouts (flat arrays with offsets):
  fields: element e holds u[u_off[e]:u_off[e+1]] = [v_1..v_d, sigma_1..sigma_nt] x N_p(k_e)
          (component-major, the ordering of oracle/elastic.py);
  traces: face f holds lam[t_off[f]:t_off[f+1]] = d components x N_f(k_F), component-major,
          face modes in the lexicographic order of oracle/reference.py.
The local trace vector of an element concatenates its faces in local order.

Every step follows oracle/elastic.py: per-element LU of alpha Mw + A0, S_K = D - C A^-1 B,
assembly over interior faces, a sparse direct trace solve, local recovery. Dirichlet data
are v_hat = v_D on boundary faces (L2 projection onto the face space), zero when absent.
"""
from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import acoustic as ac
from . import elastic as el
from . import reference as ref


def face_degrees(sk, elem_k):
    """k_F = max over the elements that share face F."""
    kf = np.zeros(sk.faces.shape[0], dtype=np.int64)
    for f, lst in enumerate(sk.face_elems):
        kf[f] = max(int(elem_k[e]) for (e, _) in lst)
    return kf


@dataclass
class Blocks:
    Mw: np.ndarray
    A0: np.ndarray
    B: np.ndarray
    C: np.ndarray
    D: np.ndarray
    Fm: list           # per face: (phi_l, mu_m)_f, N_p x N_f(k_F)
    E: list            # per face: (phi_l, phi_i)_f
    G: list            # per face: (mu_a, mu_b)_f
    loc_off: np.ndarray  # local trace offsets per face (d * N_f(k_F) each)
    normals: np.ndarray
    detJ: float
    X: np.ndarray
    V: np.ndarray
    xq: np.ndarray
    wq: np.ndarray


def element_blocks(X, k, kfaces, rho, lam, mu, s):
    """Local blocks of one element of degree k whose faces have degrees kfaces (>= k)."""
    X = np.asarray(X, dtype=np.float64)
    dim = X.shape[1]
    Np = ref.n_modes(dim, k)
    J = (X[1:] - X[0]).T
    detJ = abs(np.linalg.det(J))
    Jinv = np.linalg.inv(J)
    xi, wq = ref.simplex_rule(dim, k + 2)
    V, Gr = ref.basis(dim, k, xi)
    Gx = np.einsum("qir,rj->qij", Gr, Jinv)
    M = np.einsum("q,qi,ql->il", wq * detJ, V, V)
    Dx = [np.einsum("q,qi,ql->il", wq * detJ, V, Gx[:, :, j]) for j in range(dim)]
    Fm, E, Gm, normals, nfs = [], [], [], [], []
    for f in range(dim + 1):
        kf = int(kfaces[f])
        eta, wf = ref.simplex_rule(dim - 1, max(k, kf) + 2)
        U, _ = ref.basis(dim - 1, kf, eta)
        Y = X[ac.face_local_vertices(dim, f)]
        xqf = Y[0] + eta @ (Y[1:] - Y[0])
        JF = ac.face_frame(Y)
        Vf, _ = ref.basis(dim, k, (xqf - X[0]) @ Jinv.T)
        E.append(np.einsum("q,qi,ql->il", wf * JF, Vf, Vf))
        Fm.append(np.einsum("q,qi,qm->im", wf * JF, Vf, U))
        Gm.append(np.einsum("q,qm,qn->mn", wf * JF, U, U))
        normals.append(ac.outward_normal(X, f))
        nfs.append(U.shape[1])
    normals = np.array(normals)
    comps = el.sym_components(dim)
    nt = len(comps)
    n = (dim + nt) * Np
    loc_off = np.concatenate([[0], np.cumsum([dim * q for q in nfs])])
    m = int(loc_off[-1])
    Vb = lambda i: slice(i * Np, (i + 1) * Np)
    Tb = lambda a: slice((dim + a) * Np, (dim + a + 1) * Np)
    Fb = lambda f, i: slice(loc_off[f] + i * nfs[f], loc_off[f] + (i + 1) * nfs[f])
    Mw = np.zeros((n, n))
    A0 = np.zeros((n, n))
    B = np.zeros((n, m))
    C = np.zeros((m, n))
    D = np.zeros((m, m))
    Q = el.compliance(dim, lam, mu)
    for i in range(dim):
        Mw[Vb(i), Vb(i)] = rho * M
        A0[Vb(i), Vb(i)] = s * sum(E)                              # s <v, w>_dK
    for a in range(nt):
        for b in range(nt):
            Mw[Tb(a), Tb(b)] = Q[a, b] * M
    # tensor rows (test G_a): (v, div G) - <v_hat, G n>
    for a, (i, j) in enumerate(comps):
        pairs = [(i, j)] if i == j else [(i, j), (j, i)]
        for (p, q) in pairs:
            A0[Tb(a), Vb(p)] += Dx[q].T
            for f in range(dim + 1):
                B[Tb(a), Fb(f, p)] += -normals[f, q] * Fm[f]
    # velocity rows (test w_i): (sigma, grad w) - <sigma n, w> + s <v - v_hat, w>
    for i in range(dim):
        for j in range(dim):
            b = comps.index((i, j)) if (i, j) in comps else comps.index((j, i))
            A0[Vb(i), Tb(b)] += Dx[j].T - sum(normals[f, j] * E[f] for f in range(dim + 1))
            for f in range(dim + 1):
                C[Fb(f, i), Tb(b)] += normals[f, j] * Fm[f].T          # <sigma n, mu>
    for i in range(dim):
        for f in range(dim + 1):
            B[Vb(i), Fb(f, i)] += -s * Fm[f]                           # -s <v_hat, w>
            C[Fb(f, i), Vb(i)] += -s * Fm[f].T                         # -s <v, mu>
            D[Fb(f, i), Fb(f, i)] += s * Gm[f]                         # +s <v_hat, mu>
    xq = X[0] + xi @ J.T
    return Blocks(Mw, A0, B, C, D, Fm, E, Gm, loc_off, normals, detJ, X, V, xq, wq)


@dataclass
class Problem:
    vert: np.ndarray
    sk: ac.Skeleton
    elem_k: np.ndarray
    face_k: np.ndarray
    rho: np.ndarray
    lam: np.ndarray
    mu: np.ndarray
    s: np.ndarray
    blocks: list
    u_off: np.ndarray       # [Ne + 1]
    t_off: np.ndarray       # [Nfaces + 1]
    nt: int
    dirichlet: object = None   # callable (x[nq, d], t) -> [nq, d] (v_hat), or None (clamped)


def build_problem(vert, elem_vert, elem_k, rho, lam, mu, s=None):
    vert = np.asarray(vert, dtype=np.float64)
    sk = ac.skeleton(elem_vert)
    ne = sk.elem.shape[0]
    dim = sk.dim
    elem_k = np.broadcast_to(np.asarray(elem_k, dtype=np.int64), (ne,)).copy()
    bc = lambda a: np.broadcast_to(np.asarray(a, dtype=np.float64), (ne,)).copy()
    rho, lam, mu = bc(rho), bc(lam), bc(mu)
    s = 2.0 * rho * el.shear_speed(rho, mu) if s is None else bc(s)
    kf = face_degrees(sk, elem_k)
    blocks = [element_blocks(vert[sk.elem[e]], elem_k[e], kf[sk.elem_face[e]], rho[e], lam[e], mu[e], s[e])
              for e in range(ne)]
    nt = len(el.sym_components(dim))
    u_off = np.concatenate([[0], np.cumsum([(dim + nt) * ref.n_modes(dim, int(k)) for k in elem_k])])
    t_off = np.concatenate([[0], np.cumsum([dim * ref.n_modes(dim - 1, int(k)) for k in kf])])
    return Problem(vert, sk, elem_k, kf, rho, lam, mu, s, blocks, u_off, t_off, nt)


def n_local(prob, e):
    return int(prob.u_off[e + 1] - prob.u_off[e])


def field(prob, u, e):
    return u[prob.u_off[e]:prob.u_off[e + 1]]


def local_traces(prob, e, lam):
    return np.concatenate([lam[prob.t_off[f]:prob.t_off[f + 1]] for f in prob.sk.elem_face[e]])


def project_face(prob, f, func, t):
    """L2 projection of a vector func(x, t) -> [nq, d] on face f (component-major)."""
    dim, kf = prob.sk.dim, int(prob.face_k[f])
    Y = prob.vert[prob.sk.faces[f]]
    eta, wf = ref.simplex_rule(dim - 1, kf + 2)
    U, _ = ref.basis(dim - 1, kf, eta)
    xq = Y[0] + eta @ (Y[1:] - Y[0])
    JF = ac.face_frame(Y)
    G = np.einsum("q,qm,qn->mn", wf * JF, U, U)
    vals = func(xq, t)
    return np.concatenate([np.linalg.solve(G, np.einsum("q,qm,q->m", wf * JF, U, vals[:, i])) for i in range(dim)])


def dirichlet_values(prob, t):
    lam = np.zeros(int(prob.t_off[-1]))
    if prob.dirichlet is None:
        return lam
    for f in np.nonzero(prob.sk.boundary)[0]:
        lam[prob.t_off[f]:prob.t_off[f + 1]] = project_face(prob, f, prob.dirichlet, t)
    return lam


@dataclass
class Condensed:
    alpha: float
    lu: list
    S: list
    K: object
    interior: np.ndarray    # interior face ids
    i_off: np.ndarray       # offsets of the interior faces' unknowns in the trace system


def condense(prob, alpha):
    """Static condensation (Sec. 2.4, Eq. LS) of every element, assembled over interior faces."""
    sk = prob.sk
    interior = np.nonzero(~sk.boundary)[0]
    sizes = np.diff(prob.t_off)
    i_off = np.concatenate([[0], np.cumsum(sizes[interior])])
    pos = -np.ones(sk.faces.shape[0], dtype=np.int64)
    pos[interior] = i_off[:-1]
    lus, Ss, rows, cols, vals = [], [], [], [], []
    for e, bl in enumerate(prob.blocks):
        lu = sla.lu_factor(alpha * bl.Mw + bl.A0)
        S = bl.D - bl.C @ sla.lu_solve(lu, bl.B)
        lus.append(lu)
        Ss.append(S)
        for a in range(sk.dim + 1):
            pa = pos[sk.elem_face[e, a]]
            if pa < 0:
                continue
            ra = slice(bl.loc_off[a], bl.loc_off[a + 1])
            for b in range(sk.dim + 1):
                pb = pos[sk.elem_face[e, b]]
                if pb < 0:
                    continue
                rb = slice(bl.loc_off[b], bl.loc_off[b + 1])
                ii, jj = np.meshgrid(pa + np.arange(ra.stop - ra.start), pb + np.arange(rb.stop - rb.start),
                                     indexing="ij")
                rows.append(ii.ravel())
                cols.append(jj.ravel())
                vals.append(S[ra, rb].ravel())
    nI = int(i_off[-1])
    K = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(nI, nI)) if rows \
        else sp.csr_matrix((nI, nI))
    return Condensed(alpha, lus, Ss, K, interior, i_off)


def _interior_to_faces(prob, cond, x):
    lam = np.zeros(int(prob.t_off[-1]))
    for q, f in enumerate(cond.interior):
        lam[prob.t_off[f]:prob.t_off[f + 1]] = x[cond.i_off[q]:cond.i_off[q + 1]]
    return lam


def solve_stage(prob, cond, hist, t):
    """alpha Mw u + f(u, v_hat, t) = alpha Mw hist, jump condition = 0: returns (u, v_hat)."""
    sk = prob.sk
    lamD = dirichlet_values(prob, t)
    F = [cond.alpha * bl.Mw @ field(prob, hist, e) - bl.B @ local_traces(prob, e, lamD)
         for e, bl in enumerate(prob.blocks)]
    pos = -np.ones(sk.faces.shape[0], dtype=np.int64)
    pos[cond.interior] = cond.i_off[:-1]
    r = np.zeros(int(cond.i_off[-1]))
    for e, bl in enumerate(prob.blocks):
        g = -bl.C @ sla.lu_solve(cond.lu[e], F[e])
        for a in range(sk.dim + 1):
            pa = pos[sk.elem_face[e, a]]
            if pa >= 0:
                r[pa:pa + bl.loc_off[a + 1] - bl.loc_off[a]] += g[bl.loc_off[a]:bl.loc_off[a + 1]]
    x = spla.spsolve(cond.K.tocsc(), r) if r.size else r
    lamI = _interior_to_faces(prob, cond, x)
    u = np.concatenate([sla.lu_solve(cond.lu[e], F[e] - bl.B @ local_traces(prob, e, lamI))
                        for e, bl in enumerate(prob.blocks)])
    return u, lamI + lamD


def run_bdf(prob, u0, dt, nsteps, order, t0=0.0, on_step=None):
    a, bs = ac.BDF[order]
    cond = condense(prob, a[-1] / (bs * dt))
    hist_u = [u0.copy()] if order == 1 else [u0.copy(), u0.copy()]
    lam = None
    for n in range(nsteps):
        t = t0 + (n + 1) * dt
        h = -sum(a[i] * hist_u[i] for i in range(order)) / a[-1]
        u, lam = solve_stage(prob, cond, h, t)
        hist_u = hist_u[1:] + [u]
        if on_step is not None:
            on_step(n, t, u, lam)
    return hist_u[-1], lam, t0 + nsteps * dt


def run_dirk3(prob, u0, dt, nsteps, t0=0.0, on_step=None):
    """DIRK(3,3) in the stage form of Eq. ch5appendx1:eq10_1 with the update of Eq. 10_2."""
    a, b, c = ac.dirk3_tableau()
    d = np.linalg.inv(a)
    e = b @ d
    cond = condense(prob, d[0, 0] / dt)
    u = u0.copy()
    lam = None
    for n in range(nsteps):
        tn = t0 + n * dt
        stages = []
        for i in range(3):
            h = (sum(d[i, j] for j in range(i + 1)) * u - sum(d[i, j] * stages[j] for j in range(i))) / d[i, i]
            ui, lam = solve_stage(prob, cond, h, tn + c[i] * dt)
            stages.append(ui)
        u = (1.0 - b @ d.sum(axis=1)) * u + sum(e[j] * stages[j] for j in range(3))
        if on_step is not None:
            on_step(n, tn + dt, u, lam)
    return u, lam, t0 + nsteps * dt


def solve_monolithic(prob, alpha, hist, t):
    """Uncondensed [A B; C D] over all element and face unknowns (dense LU); Dirichlet faces
    carry <v_hat - v_D, mu> = 0."""
    sk = prob.sk
    dim = sk.dim
    ne = sk.elem.shape[0]
    nU = int(prob.u_off[-1])
    N = nU + int(prob.t_off[-1])
    Mat = np.zeros((N, N))
    rhs = np.zeros(N)
    lamD = dirichlet_values(prob, t)
    for e, bl in enumerate(prob.blocks):
        r0, n = int(prob.u_off[e]), n_local(prob, e)
        Mat[r0:r0 + n, r0:r0 + n] = alpha * bl.Mw + bl.A0
        rhs[r0:r0 + n] = alpha * bl.Mw @ field(prob, hist, e)
        for a in range(dim + 1):
            fa = sk.elem_face[e, a]
            c0, mf = nU + int(prob.t_off[fa]), int(prob.t_off[fa + 1] - prob.t_off[fa])
            la = slice(bl.loc_off[a], bl.loc_off[a + 1])
            Mat[r0:r0 + n, c0:c0 + mf] = bl.B[:, la]
            if not sk.boundary[fa]:
                Mat[c0:c0 + mf, r0:r0 + n] += bl.C[la]
                Mat[c0:c0 + mf, c0:c0 + mf] += bl.D[la, la]
    for f in np.nonzero(sk.boundary)[0]:
        c0, mf = nU + int(prob.t_off[f]), int(prob.t_off[f + 1] - prob.t_off[f])
        e, a = sk.face_elems[f][0]
        G = np.kron(np.eye(dim), prob.blocks[e].G[a])
        Mat[c0:c0 + mf, c0:c0 + mf] = G
        rhs[c0:c0 + mf] = G @ lamD[prob.t_off[f]:prob.t_off[f + 1]]
    x = np.linalg.solve(Mat, rhs)
    return x[:nU], x[nU:]


def energy(prob, u):
    """E = 1/2 (rho v, v) + 1/2 (C^{-1} sigma, sigma)."""
    return sum(0.5 * field(prob, u, e) @ bl.Mw @ field(prob, u, e) for e, bl in enumerate(prob.blocks))


def energy_terms(prob, u, lam):
    """Dissipation sum_dK <s (v - v_hat)^2, 1> and boundary work <v_hat, sigma_hat n>_{Gamma_D}."""
    sk = prob.sk
    dim = sk.dim
    diss = bwork = 0.0
    for e, bl in enumerate(prob.blocks):
        ue = field(prob, u, e)
        Np = ref.n_modes(dim, int(prob.elem_k[e]))
        lk = local_traces(prob, e, lam)
        flux = bl.C @ ue + bl.D @ lk
        for a in range(dim + 1):
            nf = bl.Fm[a].shape[1]
            for i in range(dim):
                v = ue[i * Np:(i + 1) * Np]
                la = lk[bl.loc_off[a] + i * nf:bl.loc_off[a] + (i + 1) * nf]
                diss += prob.s[e] * (v @ bl.E[a] @ v - 2 * v @ bl.Fm[a] @ la + la @ bl.G[a] @ la)
            if sk.boundary[sk.elem_face[e, a]]:
                sl = slice(bl.loc_off[a], bl.loc_off[a + 1])
                bwork += lk[sl] @ flux[sl]
    return diss, bwork


def project(prob, func_v, func_t):
    """L2 projection of velocity func_v(x) -> [nq, d] and tensor func_t(x) -> [nq, nt]."""
    dim = prob.sk.dim
    out = []
    for e, bl in enumerate(prob.blocks):
        Np = bl.V.shape[1]
        Mi = np.linalg.inv(np.einsum("q,qi,ql->il", bl.wq * bl.detJ, bl.V, bl.V))
        vals = np.concatenate([func_v(bl.xq), func_t(bl.xq)], axis=1)
        for c in range(dim + prob.nt):
            out.append(Mi @ np.einsum("q,qi,q->i", bl.wq * bl.detJ, bl.V, vals[:, c]))
    return np.concatenate(out)


def point_values(prob, u, e, xi):
    """Fields of element e at reference points xi [np, d] -> [np, d + nt]."""
    dim = prob.sk.dim
    V, _ = ref.basis(dim, int(prob.elem_k[e]), np.asarray(xi, dtype=np.float64))
    Np = V.shape[1]
    ue = field(prob, u, e)
    return np.stack([V @ ue[c * Np:(c + 1) * Np] for c in range(dim + prob.nt)], axis=1)
