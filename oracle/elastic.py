"""Linear elastodynamics HDG scheme, plain FP64 oracle (test infrastructure only).

Follows Sec. 4.1 (Eqs. LE, eq:sigma_cauchy, LEM, eq:HDG_linelas1-5, eq:stab_matrix_lin).

Reading of the sign (the paper writes rho v_t + div sigma = f in Eq. LE but
rho v_t - div P = f in Eq. UNEL): we take rho v_t - div sigma = f, the only choice under
which the energy identity of Sec. 4.2 (Eq. eq:energy_identity_nelas) holds with the
dissipative term <S (v - v_hat), v - v_hat>. The local equations are then
    (d_t F, G) + (v, div G) - <v_hat, G n> = 0
    (rho d_t v, w) + (sigma, grad w) - <sigma_hat n, w> = (f, w)
    sigma_hat n = sigma n - S (v - v_hat),   S = s I (Eq. eq:stab_matrix_lin)
with the global jump condition sum_K <sigma_hat n, mu> = 0 on interior faces and
v_hat = v_D on Dirichlet (clamped) faces (Eq. eq:HDG_linelas4).

Two forms are implemented, and they agree for element-wise constant Lame parameters:
  form "F":     unknowns (H, v), H = F - I the displacement gradient (9 components), with
                sigma(F) = mu (F + F^T) + (lam (tr F - d) - 2 mu) I = mu (H + H^T) + lam tr(H) I
                (Eq. eq:sigma_cauchy), the paper's own velocity / deformation-gradient form;
  form "sigma": unknowns (sigma, v) with sigma symmetric (6 components) and the compliance
                mass (C^{-1} d_t sigma, G), the velocity / symmetric-stress form.
Unknown ordering per element: [v_1..v_d, then the tensor components], N_p each. Tensor
components: form "F" row-major (i, j); form "sigma" (11, 22, 33, 23, 13, 12) in 3D and
(11, 22, 12) in 2D. Trace: v_hat per face, d components x N_f, component-major.

All other conventions (basis, faces, quadrature, time marching) are those of
oracle/acoustic.py. The Gaussian-bump initial data of the benchmark workload is input data
(the seeded generator module), a convention of the workload and no function of this oracle.
"""
import math
from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import acoustic as ac
from . import reference as ref


def sym_components(dim):
    return [(0, 0), (1, 1), (0, 1)] if dim == 2 else [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]


def full_components(dim):
    return [(i, j) for i in range(dim) for j in range(dim)]


def compliance(dim, lam, mu):
    """Matrix Q with (C^{-1} sigma, G) = sum_ab Q[a, b] sigma_b G_a for the symmetric components.

    C^{-1} sigma = (sigma - lam / (d lam + 2 mu) tr(sigma) I) / (2 mu); the tensor inner product
    counts each off-diagonal component twice.
    """
    comps = sym_components(dim)
    nc = len(comps)
    Q = np.zeros((nc, nc))
    for a, (i, j) in enumerate(comps):
        wa = 1.0 if i == j else 2.0
        for b, (k, l) in enumerate(comps):
            v = 0.0
            if a == b:
                v += wa / (2 * mu)
            if i == j and k == l:
                v -= lam / ((dim * lam + 2 * mu) * 2 * mu)
            Q[a, b] = v
    return Q


def stiffness_F(dim, lam, mu):
    """Matrix P with sigma(H)_{ij} = sum_kl P[(i,j),(k,l)] H_kl (Eq. eq:sigma_cauchy, F = I + H)."""
    comps = full_components(dim)
    P = np.zeros((dim * dim, dim * dim))
    for a, (i, j) in enumerate(comps):
        for b, (k, l) in enumerate(comps):
            v = 0.0
            if (k, l) == (i, j):
                v += mu
            if (k, l) == (j, i):
                v += mu
            if i == j and k == l:
                v += lam
            P[a, b] = v
    return P


@dataclass
class ElasticBlocks:
    Mw: np.ndarray
    A0: np.ndarray
    B: np.ndarray
    C: np.ndarray
    D: np.ndarray
    Fm: list
    E: list
    G: list
    normal: np.ndarray
    detJ: float
    Jinv: np.ndarray
    X: np.ndarray
    V: np.ndarray      # volume basis at quadrature points (for sources / errors)
    xq: np.ndarray
    wq: np.ndarray


def element_blocks(X, k, rho, lam, mu, s, form="sigma"):
    """Local blocks of one element (vertex rows X in ascending global id)."""
    X = np.asarray(X, dtype=np.float64)
    dim = X.shape[1]
    Np = ref.n_modes(dim, k)
    Nf = ref.n_modes(dim - 1, k)
    J = (X[1:] - X[0]).T
    detJ = abs(np.linalg.det(J))
    Jinv = np.linalg.inv(J)
    xi, wq = ref.simplex_rule(dim, k + 2)
    V, Gr = ref.basis(dim, k, xi)
    Gx = np.einsum("qir,rj->qij", Gr, Jinv)
    M = np.einsum("q,qi,ql->il", wq * detJ, V, V)
    Dx = [np.einsum("q,qi,ql->il", wq * detJ, V, Gx[:, :, j]) for j in range(dim)]   # (d_j phi_l, phi_i)
    eta, wf = ref.simplex_rule(dim - 1, k + 2)
    U, _ = ref.basis(dim - 1, k, eta)
    Fm, E, Gm, normals = [], [], [], []
    for f in range(dim + 1):
        Y = X[ac.face_local_vertices(dim, f)]
        xqf = Y[0] + eta @ (Y[1:] - Y[0])
        JF = ac.face_frame(Y)
        Vf, _ = ref.basis(dim, k, (xqf - X[0]) @ Jinv.T)
        E.append(np.einsum("q,qi,ql->il", wf * JF, Vf, Vf))
        Fm.append(np.einsum("q,qi,qm->im", wf * JF, Vf, U))
        Gm.append(np.einsum("q,qm,qn->mn", wf * JF, U, U))
        normals.append(ac.outward_normal(X, f))
    normals = np.array(normals)
    comps = sym_components(dim) if form == "sigma" else full_components(dim)
    nt = len(comps)
    n = (dim + nt) * Np
    m = (dim + 1) * dim * Nf
    Vb = lambda i: slice(i * Np, (i + 1) * Np)                    # velocity component i
    Tb = lambda a: slice((dim + a) * Np, (dim + a + 1) * Np)      # tensor component a
    Fb = lambda f, i: slice((f * dim + i) * Nf, (f * dim + i + 1) * Nf)
    Mw = np.zeros((n, n))
    A0 = np.zeros((n, n))
    B = np.zeros((n, m))
    C = np.zeros((m, n))
    D = np.zeros((m, m))
    for i in range(dim):
        Mw[Vb(i), Vb(i)] = rho * M
        A0[Vb(i), Vb(i)] = s * sum(E)                              # s <v, w>_dK
    if form == "sigma":
        Q = compliance(dim, lam, mu)
        for a in range(nt):
            for b in range(nt):
                Mw[Tb(a), Tb(b)] = Q[a, b] * M
    else:
        for a in range(nt):
            Mw[Tb(a), Tb(a)] = M
    P = None if form == "sigma" else stiffness_F(dim, lam, mu)
    # tensor rows (test G_a):  (v, div G) - <v_hat, G n>
    # velocity rows (test w_i): (sigma, grad w) - <sigma n, w> + s <v - v_hat, w>
    for a, (i, j) in enumerate(comps):
        # G = phi e_i e_j^T (+ e_j e_i^T for off-diagonal symmetric components)
        pairs = [(i, j)] if (form == "F" or i == j) else [(i, j), (j, i)]
        for (p, q) in pairs:
            # (v, div G): (div G)_p = d_q phi  ->  (v_p, d_q phi_a) = Dx[q]^T[a, l] v_p  i.e. Dx[q].T
            A0[Tb(a), Vb(p)] += Dx[q].T
            for f in range(dim + 1):
                B[Tb(a), Fb(f, p)] += -normals[f, q] * Fm[f]
    # sigma as a function of the tensor unknowns: sigma_pq = sum_b Sig[(p,q), b] T_b
    def sigma_coeffs(p, q):
        if form == "sigma":
            for b, (k2, l2) in enumerate(comps):
                if (k2, l2) == (p, q) or (k2, l2) == (q, p):
                    return {b: 1.0}
        cf = {}
        for b in range(nt):
            if P[full_components(dim).index((p, q)), b] != 0.0:
                cf[b] = P[full_components(dim).index((p, q)), b]
        return cf
    for i in range(dim):
        for j in range(dim):
            for b, cval in sigma_coeffs(i, j).items():
                # (sigma_ij, d_j w_i) - <sigma_ij n_j, w_i>
                A0[Vb(i), Tb(b)] += cval * (Dx[j].T - sum(normals[f, j] * E[f] for f in range(dim + 1)))
                for f in range(dim + 1):
                    C[Fb(f, i), Tb(b)] += cval * normals[f, j] * Fm[f].T        # <sigma n, mu>
    for i in range(dim):
        for f in range(dim + 1):
            B[Vb(i), Fb(f, i)] += -s * Fm[f]                               # -s <v_hat, w>
            C[Fb(f, i), Vb(i)] += -s * Fm[f].T                             # -s <v, mu>
            D[Fb(f, i), Fb(f, i)] += s * Gm[f]                             # +s <v_hat, mu>
    xq = X[0] + xi @ J.T
    return ElasticBlocks(Mw, A0, B, C, D, Fm, E, Gm, normals, detJ, Jinv, X, V, xq, wq)


@dataclass
class Problem:
    vert: np.ndarray
    sk: ac.Skeleton
    k: int
    form: str
    rho: np.ndarray
    lam: np.ndarray
    mu: np.ndarray
    s: np.ndarray
    blocks: list
    Np: int
    Nf: int
    nt: int
    body_force: object = None       # callable (x[nq, d], t) -> [nq, d], or None
    dirichlet: object = None        # callable (x[nq, d], t) -> [nq, d] (v_hat), or None (clamped)


def shear_speed(rho, mu):
    return np.sqrt(mu / rho)


def build_problem(vert, elem_vert, k, rho, lam, mu, form="sigma", s=None):
    """s: stabilisation per element; default 2 rho c_s (the paper's experiment, Sec. 4.3)."""
    vert = np.asarray(vert, dtype=np.float64)
    sk = ac.skeleton(elem_vert)
    ne = sk.elem.shape[0]
    rho = np.broadcast_to(np.asarray(rho, dtype=np.float64), (ne,)).copy()
    lam = np.broadcast_to(np.asarray(lam, dtype=np.float64), (ne,)).copy()
    mu = np.broadcast_to(np.asarray(mu, dtype=np.float64), (ne,)).copy()
    s = 2.0 * rho * shear_speed(rho, mu) if s is None else np.broadcast_to(np.asarray(s, dtype=np.float64), (ne,)).copy()
    blocks = [element_blocks(vert[sk.elem[e]], k, rho[e], lam[e], mu[e], s[e], form) for e in range(ne)]
    dim = sk.dim
    nt = len(sym_components(dim)) if form == "sigma" else dim * dim
    return Problem(vert, sk, k, form, rho, lam, mu, s, blocks, ref.n_modes(dim, k), ref.n_modes(dim - 1, k), nt)


def local_traces(prob, e, lam):
    return np.concatenate([lam[prob.sk.elem_face[e, j]] for j in range(prob.sk.dim + 1)])


def dirichlet_values(prob, t):
    """v_hat on boundary faces ([Nfaces, d*Nf], component-major per face); zero if clamped."""
    dim, Nf = prob.sk.dim, prob.Nf
    lam = np.zeros((prob.sk.faces.shape[0], dim * Nf))
    if prob.dirichlet is None:
        return lam
    for f in np.nonzero(prob.sk.boundary)[0]:
        for i in range(dim):
            lam[f, i * Nf:(i + 1) * Nf] = ac.project_face(prob, f, lambda x, tt: prob.dirichlet(x, tt)[:, i], t)
    return lam


def body_force_vector(prob, e, t):
    out = np.zeros((prob.sk.dim + prob.nt) * prob.Np)
    if prob.body_force is None:
        return out
    bl = prob.blocks[e]
    fvals = prob.body_force(bl.xq, t)
    for i in range(prob.sk.dim):
        out[i * prob.Np:(i + 1) * prob.Np] = np.einsum("q,qi,q->i", bl.wq * bl.detJ, bl.V, fvals[:, i])
    return out


@dataclass
class Condensed:
    alpha: float
    lu: list
    S: list
    K: object
    interior: np.ndarray


def condense(prob, alpha):
    """Static condensation (Sec. 2.4, Eq. LS) of every element, assembled over interior faces."""
    sk = prob.sk
    mf = prob.sk.dim * prob.Nf
    interior = np.nonzero(~sk.boundary)[0]
    pos = -np.ones(sk.faces.shape[0], dtype=np.int64)
    pos[interior] = np.arange(interior.size)
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
            for b in range(sk.dim + 1):
                pb = pos[sk.elem_face[e, b]]
                if pb < 0:
                    continue
                ii, jj = np.meshgrid(np.arange(mf) + pa * mf, np.arange(mf) + pb * mf, indexing="ij")
                rows.append(ii.ravel())
                cols.append(jj.ravel())
                vals.append(S[a * mf:(a + 1) * mf, b * mf:(b + 1) * mf].ravel())
    nI = interior.size * mf
    K = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(nI, nI)) if rows \
        else sp.csr_matrix((nI, nI))
    return Condensed(alpha, lus, Ss, K, interior)


def solve_stage(prob, cond, hist, t):
    """alpha Mw u + f(u, v_hat, t) = alpha Mw hist, jump condition = 0: returns (u, v_hat)."""
    sk = prob.sk
    mf = sk.dim * prob.Nf
    lamD = dirichlet_values(prob, t)
    F = np.stack([cond.alpha * bl.Mw @ hist[e] + body_force_vector(prob, e, t) - bl.B @ local_traces(prob, e, lamD)
                  for e, bl in enumerate(prob.blocks)])
    pos = -np.ones(sk.faces.shape[0], dtype=np.int64)
    pos[cond.interior] = np.arange(cond.interior.size)
    r = np.zeros(cond.interior.size * mf)
    for e, bl in enumerate(prob.blocks):
        g = -bl.C @ sla.lu_solve(cond.lu[e], F[e])
        for a in range(sk.dim + 1):
            pa = pos[sk.elem_face[e, a]]
            if pa >= 0:
                r[pa * mf:(pa + 1) * mf] += g[a * mf:(a + 1) * mf]
    lam_int = spla.spsolve(cond.K.tocsc(), r) if r.size else r
    lamI = np.zeros_like(lamD)
    lamI[cond.interior] = lam_int.reshape(-1, mf)
    u = np.stack([sla.lu_solve(cond.lu[e], F[e] - bl.B @ local_traces(prob, e, lamI)) for e, bl in enumerate(prob.blocks)])
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
    sk, Np, Nf = prob.sk, prob.Np, prob.Nf
    dim = sk.dim
    mf = dim * Nf
    ne, nf = sk.elem.shape[0], sk.faces.shape[0]
    n = (dim + prob.nt) * Np
    N = ne * n + nf * mf
    Mat = np.zeros((N, N))
    rhs = np.zeros(N)
    lamD = dirichlet_values(prob, t)
    for e, bl in enumerate(prob.blocks):
        r0 = e * n
        Mat[r0:r0 + n, r0:r0 + n] = alpha * bl.Mw + bl.A0
        rhs[r0:r0 + n] = alpha * bl.Mw @ hist[e] + body_force_vector(prob, e, t)
        for a in range(dim + 1):
            fa = sk.elem_face[e, a]
            c0 = ne * n + fa * mf
            Mat[r0:r0 + n, c0:c0 + mf] = bl.B[:, a * mf:(a + 1) * mf]
            if not sk.boundary[fa]:
                Mat[c0:c0 + mf, r0:r0 + n] += bl.C[a * mf:(a + 1) * mf]
                Mat[c0:c0 + mf, c0:c0 + mf] += bl.D[a * mf:(a + 1) * mf, a * mf:(a + 1) * mf]
    for f in np.nonzero(sk.boundary)[0]:
        c0 = ne * n + f * mf
        e, a = sk.face_elems[f][0]
        G = np.kron(np.eye(dim), prob.blocks[e].G[a])
        Mat[c0:c0 + mf, c0:c0 + mf] = G
        rhs[c0:c0 + mf] = G @ lamD[f]
    x = np.linalg.solve(Mat, rhs)
    return x[:ne * n].reshape(ne, n), x[ne * n:].reshape(nf, mf)


def energy(prob, u):
    """E = 1/2 (rho v, v) + 1/2 (C^{-1} sigma, sigma) (form sigma) or 1/2 (sigma(H), H) (form F)."""
    tot = 0.0
    dim, Np = prob.sk.dim, prob.Np
    for e, bl in enumerate(prob.blocks):
        if prob.form == "sigma":
            tot += 0.5 * u[e] @ bl.Mw @ u[e]
        else:
            v = u[e, :dim * Np]
            tot += 0.5 * v @ bl.Mw[:dim * Np, :dim * Np] @ v
            P = stiffness_F(dim, prob.lam[e], prob.mu[e])
            H = u[e, dim * Np:].reshape(dim * dim, Np)
            tot += 0.5 * bl.detJ * np.einsum("ai,ab,bi->", H, P, H)
    return tot


def energy_terms(prob, u, lam, t):
    """Dissipation sum_dK <s (v - v_hat)^2, 1>, boundary work <v_hat, sigma_hat n>_{Gamma_D}, (f, v)."""
    sk, Np, Nf = prob.sk, prob.Np, prob.Nf
    dim = sk.dim
    mf = dim * Nf
    diss = bwork = fv = 0.0
    for e, bl in enumerate(prob.blocks):
        lk = local_traces(prob, e, lam)
        flux = bl.C @ u[e] + bl.D @ lk           # -<sigma_hat n, mu> per local face
        for a in range(dim + 1):
            for i in range(dim):
                v = u[e, i * Np:(i + 1) * Np]
                la = lk[a * mf + i * Nf:a * mf + (i + 1) * Nf]
                diss += prob.s[e] * (v @ bl.E[a] @ v - 2 * v @ bl.Fm[a] @ la + la @ bl.G[a] @ la)
            if sk.boundary[sk.elem_face[e, a]]:
                bwork += lk[a * mf:(a + 1) * mf] @ flux[a * mf:(a + 1) * mf]
        fv += body_force_vector(prob, e, t) @ u[e]
    return diss, bwork, fv


def project(prob, func_v, func_t):
    """L2 projection of velocity func_v(x) -> [nq, d] and tensor func_t(x) -> [nq, nt] components."""
    dim, Np = prob.sk.dim, prob.Np
    u = np.zeros((prob.sk.elem.shape[0], (dim + prob.nt) * Np))
    for e, bl in enumerate(prob.blocks):
        Mi = np.linalg.inv(np.einsum("q,qi,ql->il", bl.wq * bl.detJ, bl.V, bl.V))
        vals = np.concatenate([func_v(bl.xq), func_t(bl.xq)], axis=1)
        for c in range(dim + prob.nt):
            u[e, c * Np:(c + 1) * Np] = Mi @ np.einsum("q,qi,q->i", bl.wq * bl.detJ, bl.V, vals[:, c])
    return u


def l2_error_velocity(prob, u, exact_v):
    dim, Np = prob.sk.dim, prob.Np
    xi, wq = ref.simplex_rule(dim, prob.k + 4)
    V, _ = ref.basis(dim, prob.k, xi)
    err = 0.0
    for e, bl in enumerate(prob.blocks):
        x = bl.X[0] + xi @ (bl.X[1:] - bl.X[0])
        ex = exact_v(x)
        for i in range(dim):
            err += np.sum(wq * bl.detJ * (V @ u[e, i * Np:(i + 1) * Np] - ex[:, i]) ** 2)
    return math.sqrt(err)
