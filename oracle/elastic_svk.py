"""Nonlinear (Saint Venant-Kirchhoff) elastodynamics HDG scheme, plain FP64 oracle (test
infrastructure only). Follows Sec. 4.4 (Eqs. UNEL, eq:HDG_nelas1-5) in 3D.

Unknowns per element: v (3 N_p), H = F - I (9 N_p, row-major (i, J)) and P (9 N_p), in that
order, each component a block of N_p orthonormal-basis coefficients; the trace v_hat has 3 N_f
coefficients per face, component-major. Local equations, with the sign reading of the linear
oracle (rho v_t - div P = f, P_hat n = P n - s (v - v_hat)):
    (d_t H, G) + (v, div G) - <v_hat, G n> = 0
    (rho d_t v, w) + (P, grad w) - <P_hat n, w> = (f, w)
    (P, Q) - (F S(F), Q) = 0                      (Eq. eq:HDG_nelas3, F = I + H)
and on faces sum_K <P_hat n, mu> = <g_N, mu> on Neumann faces (0 on interior faces), with
v_hat = v_D on Dirichlet faces. P carries no time derivative (an algebraic unknown of the DAE).

Each DIRK(3,3) stage solves alpha Mw (u - h) + f(u, v_hat, t) = 0 (alpha = d_ii / dt, Sec. 2.3)
by Newton's method; every Newton system [A B; C D] (delta u; delta v_hat) = -(R_u; R_hat) is
condensed element by element (Eq. LS) and its trace system solved directly. S = s I with
s = 2 rho c_s (Eq. eq:stab_matrix_lin; the plate experiment's choice).
Quadrature: 2k + 2 points per direction in the volume (the term F S(F) phi has degree 4k)
and k + 2 on faces; faces, bases and orientations are those of oracle/acoustic.py.
"""
import math
from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import acoustic as ac
from . import reference as ref


def pk_batch(F, lam, mu):
    """F S(F) at a batch of points, F[q, 3, 3] -> [q, 3, 3]."""
    I = np.eye(3)
    E = 0.5 * (np.einsum("qki,qkj->qij", F, F) - I)
    S = lam * np.einsum("qii->q", E)[:, None, None] * I + 2.0 * mu * E
    return np.einsum("qia,qaj->qij", F, S)


def tangent_batch(F, lam, mu):
    """dP_iJ / dF_kL at a batch of points, [q, 9, 9] in row-major (i, J), (k, L):
    delta_ik S_LJ + lam F_iJ F_kL + mu F_iL F_kJ + mu (F F^T)_ik delta_JL."""
    I = np.eye(3)
    E = 0.5 * (np.einsum("qki,qkj->qij", F, F) - I)
    S = lam * np.einsum("qii->q", E)[:, None, None] * I + 2.0 * mu * E
    FFt = np.einsum("qia,qka->qik", F, F)
    A = (np.einsum("ik,qLJ->qiJkL", I, S) + lam * np.einsum("qiJ,qkL->qiJkL", F, F)
         + mu * np.einsum("qiL,qkJ->qiJkL", F, F) + mu * np.einsum("qik,JL->qiJkL", FFt, I))
    return A.reshape(F.shape[0], 9, 9)


@dataclass
class Geo:
    detJ: float
    xq: np.ndarray       # physical volume points
    w: np.ndarray        # physical weights
    V: np.ndarray        # [nq, Np]
    M: np.ndarray
    Dx: list             # Dx[J][a, b] = int phi_a d_J phi_b
    E: list              # per face int_f phi_a phi_b
    Fm: list             # per face int_f phi_a mu_m
    Gm: list             # per face int_f mu_m mu_n
    normals: np.ndarray
    xqf: list            # per face physical points
    wf: list             # per face physical weights
    U: np.ndarray        # face basis at the face points [nqf, Nf]


@dataclass
class Problem:
    vert: np.ndarray
    sk: ac.Skeleton
    k: int
    rho: float
    lam: float
    mu: float
    s: float
    geo: list
    Np: int
    Nf: int
    neumann: np.ndarray                 # [Nfaces] bool: boundary faces with traction data
    body_force: object = None           # (x[n, 3], t) -> [n, 3]
    traction: object = None             # (x[n, 3], n[3], t) -> [n, 3] (P n on Neumann faces)
    dirichlet: object = None            # (x[n, 3], t) -> [n, 3] (v_hat on Dirichlet faces), None: clamped


def element_geo(X, k):
    X = np.asarray(X, dtype=np.float64)
    J = (X[1:] - X[0]).T
    detJ = abs(np.linalg.det(J))
    Jinv = np.linalg.inv(J)
    xi, wq = ref.simplex_rule(3, 2 * k + 2)
    V, Gr = ref.basis(3, k, xi)
    Gx = np.einsum("qir,rj->qij", Gr, Jinv)
    w = wq * detJ
    M = np.einsum("q,qa,qb->ab", w, V, V)
    Dx = [np.einsum("q,qa,qb->ab", w, V, Gx[:, :, j]) for j in range(3)]
    eta, wfr = ref.simplex_rule(2, k + 2)
    U, _ = ref.basis(2, k, eta)
    E, Fm, Gm, normals, xqf, wf = [], [], [], [], [], []
    for f in range(4):
        Y = X[ac.face_local_vertices(3, f)]
        xq = Y[0] + eta @ (Y[1:] - Y[0])
        JF = ac.face_frame(Y)
        Vf, _ = ref.basis(3, k, (xq - X[0]) @ Jinv.T)
        E.append(np.einsum("q,qa,qb->ab", wfr * JF, Vf, Vf))
        Fm.append(np.einsum("q,qa,qm->am", wfr * JF, Vf, U))
        Gm.append(np.einsum("q,qm,qn->mn", wfr * JF, U, U))
        normals.append(ac.outward_normal(X, f))
        xqf.append(xq)
        wf.append(wfr * JF)
    return Geo(detJ, X[0] + xi @ J.T, w, V, M, Dx, E, Fm, Gm, np.array(normals), xqf, wf, U)


def build_problem(vert, elem_vert, k, rho, lam, mu, neumann_face=None, s=None):
    """neumann_face(face vertex coordinates [3, 3]) -> bool marks traction boundary faces."""
    vert = np.asarray(vert, dtype=np.float64)
    sk = ac.skeleton(elem_vert)
    geo = [element_geo(vert[sk.elem[e]], k) for e in range(sk.elem.shape[0])]
    neu = np.zeros(sk.faces.shape[0], dtype=bool)
    if neumann_face is not None:
        for f in np.nonzero(sk.boundary)[0]:
            neu[f] = bool(neumann_face(vert[sk.faces[f]]))
    s = 2.0 * rho * math.sqrt(mu / rho) if s is None else s
    return Problem(vert, sk, k, rho, lam, mu, s, geo, ref.n_modes(3, k), ref.n_modes(2, k), neu)


def element_system(prob, e, u, lamK, h, alpha, t):
    """Residual and Jacobian of one element's stage equations at state u (21 N_p) and traces
    lamK (4 faces x 3 x N_f): (R_u, R_hat_K, A, B, C, D)."""
    g, Np, Nf, s = prob.geo[e], prob.Np, prob.Nf, prob.s
    vb = lambda i: slice(i * Np, (i + 1) * Np)
    Hb = lambda i, J: slice((3 + 3 * i + J) * Np, (4 + 3 * i + J) * Np)
    Pb = lambda i, J: slice((12 + 3 * i + J) * Np, (13 + 3 * i + J) * Np)
    fb = lambda f, i: slice((3 * f + i) * Nf, (3 * f + i + 1) * Nf)
    n, m = 21 * Np, 12 * Nf
    R = np.zeros(n)
    Rh = np.zeros(m)
    A = np.zeros((n, n))
    B = np.zeros((n, m))
    C = np.zeros((m, n))
    D = np.zeros((m, m))
    Esum = sum(g.E)
    H = np.stack([u[Hb(i, J)] for i in range(3) for J in range(3)])       # [9, Np]
    Fq = np.eye(3) + (g.V @ H.T).reshape(-1, 3, 3)
    PS = pk_batch(Fq, prob.lam, prob.mu).reshape(-1, 9)
    Aq = tangent_batch(Fq, prob.lam, prob.mu)
    fq = prob.body_force(g.xq, t) if prob.body_force is not None else np.zeros((g.xq.shape[0], 3))
    for i in range(3):
        v_i = u[vb(i)]
        R[vb(i)] += alpha * prob.rho * g.M @ (v_i - h[vb(i)]) + s * Esum @ v_i - g.V.T @ (g.w * fq[:, i])
        A[vb(i), vb(i)] += alpha * prob.rho * g.M + s * Esum
        for f in range(4):
            R[vb(i)] -= s * g.Fm[f] @ lamK[fb(f, i)]
            B[vb(i), fb(f, i)] -= s * g.Fm[f]
            Rh[fb(f, i)] += -s * g.Fm[f].T @ v_i + s * g.Gm[f] @ lamK[fb(f, i)]
            C[fb(f, i), vb(i)] -= s * g.Fm[f].T
            D[fb(f, i), fb(f, i)] += s * g.Gm[f]
        for J in range(3):
            a = 3 * i + J
            P_iJ, H_iJ = u[Pb(i, J)], u[Hb(i, J)]
            # (P, grad w) - <P n, w>
            blk = g.Dx[J].T - sum(g.normals[f, J] * g.E[f] for f in range(4))
            R[vb(i)] += blk @ P_iJ
            A[vb(i), Pb(i, J)] += blk
            # (d_t H, G) + (v, div G) - <v_hat, G n>
            R[Hb(i, J)] += alpha * g.M @ (H_iJ - h[Hb(i, J)]) + g.Dx[J].T @ v_i
            A[Hb(i, J), Hb(i, J)] += alpha * g.M
            A[Hb(i, J), vb(i)] += g.Dx[J].T
            for f in range(4):
                R[Hb(i, J)] -= g.normals[f, J] * g.Fm[f] @ lamK[fb(f, i)]
                B[Hb(i, J), fb(f, i)] -= g.normals[f, J] * g.Fm[f]
                Rh[fb(f, i)] += g.normals[f, J] * g.Fm[f].T @ P_iJ
                C[fb(f, i), Pb(i, J)] += g.normals[f, J] * g.Fm[f].T
            # (P, Q) - (F S(F), Q)
            R[Pb(i, J)] += g.M @ P_iJ - g.V.T @ (g.w * PS[:, a])
            A[Pb(i, J), Pb(i, J)] += g.M
    # d/dH of -(F S(F), Q): -(A(F) dH, Q), all 9 x 9 component pairs in one contraction
    dPH = np.einsum("q,qab,qx,qy->axby", g.w, Aq, g.V, g.V).reshape(9 * Np, 9 * Np)
    A[12 * Np:21 * Np, 3 * Np:12 * Np] -= dPH
    return R, Rh, A, B, C, D


def project(prob, func_v, func_H, func_P, t):
    """L2 projection of v, H = F - I and P given as callables of (x, t) -> [n, 3] / [n, 9]."""
    Np = prob.Np
    u = np.zeros((prob.sk.elem.shape[0], 21 * Np))
    for e, g in enumerate(prob.geo):
        vals = np.hstack([func_v(g.xq, t), func_H(g.xq, t), func_P(g.xq, t)])
        coef = np.linalg.solve(g.M, g.V.T @ (g.w[:, None] * vals))
        u[e] = coef.T.ravel()
    return u


def _dirichlet_traces(prob, t):
    sk, Nf = prob.sk, prob.Nf
    lam = np.zeros((sk.faces.shape[0], 3 * Nf))
    if prob.dirichlet is None:
        return lam
    for f in np.nonzero(sk.boundary & ~prob.neumann)[0]:
        e, j = sk.face_elems[f][0]
        g = prob.geo[e]
        vals = prob.dirichlet(g.xqf[j], t)
        G = np.einsum("q,qm,qn->mn", g.wf[j], g.U, g.U)
        lam[f] = np.concatenate([np.linalg.solve(G, g.U.T @ (g.wf[j] * vals[:, i])) for i in range(3)])
    return lam


def newton_stage(prob, u, lam, h, alpha, t, tol=1e-11, maxit=25):
    """Solves the stage equations from the guess (u [Ne, 21 Np], lam [Nfaces, 3 Nf]); returns
    (u, lam, Newton iterations)."""
    sk, Nf = prob.sk, prob.Nf
    nfc = sk.faces.shape[0]
    active = ~sk.boundary | prob.neumann
    pos = -np.ones(nfc, dtype=np.int64)
    pos[active] = np.arange(int(active.sum()))
    lamD = _dirichlet_traces(prob, t)
    lam = lam.copy()
    lam[~active] = lamD[~active]
    u = u.copy()
    m3 = 3 * Nf
    for it in range(1, maxit + 1):
        rows, cols, vals = [], [], []
        rhs = np.zeros(int(active.sum()) * m3)
        res = 0.0
        facts = []
        for e in range(sk.elem.shape[0]):
            lamK = np.concatenate([lam[sk.elem_face[e, j]] for j in range(4)])
            R, Rh, A, B, C, D = element_system(prob, e, u[e], lamK, h[e], alpha, t)
            res = max(res, np.abs(R).max())
            lu = sla.lu_factor(A)
            AiB = sla.lu_solve(lu, B)
            AiR = sla.lu_solve(lu, R)
            Sk = D - C @ AiB
            gk = -Rh + C @ AiR
            facts.append((lu, AiB, AiR))
            for a in range(4):
                pa = pos[sk.elem_face[e, a]]
                if pa < 0:
                    continue
                rhs[pa * m3:(pa + 1) * m3] += gk[a * m3:(a + 1) * m3]
                for b in range(4):
                    pb = pos[sk.elem_face[e, b]]
                    if pb < 0:
                        continue
                    ii, jj = np.meshgrid(np.arange(m3) + pa * m3, np.arange(m3) + pb * m3, indexing="ij")
                    rows.append(ii.ravel())
                    cols.append(jj.ravel())
                    vals.append(Sk[a * m3:(a + 1) * m3, b * m3:(b + 1) * m3].ravel())
        # Neumann data: -<g_N, mu> on traction faces (the residual of the face rows)
        if prob.traction is not None:
            for f in np.nonzero(prob.neumann)[0]:
                e, j = sk.face_elems[f][0]
                g = prob.geo[e]
                gN = prob.traction(g.xqf[j], g.normals[j], t)
                rhs[pos[f] * m3:(pos[f] + 1) * m3] += np.concatenate([g.U.T @ (g.wf[j] * gN[:, i]) for i in range(3)])
        # residual of the face rows at the current state (assembled), for the stopping test
        Kmat = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                             shape=(rhs.size, rhs.size))
        dlam = spla.spsolve(Kmat.tocsc(), rhs)
        dl_all = np.zeros((nfc, m3))
        dl_all[active] = dlam.reshape(-1, m3)
        step = np.abs(dlam).max() if dlam.size else 0.0
        for e in range(sk.elem.shape[0]):
            lu, AiB, AiR = facts[e]
            dlK = np.concatenate([dl_all[sk.elem_face[e, j]] for j in range(4)])
            du = -AiR - AiB @ dlK
            u[e] += du
            step = max(step, np.abs(du).max())
        lam += dl_all
        scale = max(1.0, np.abs(u).max())
        if step <= tol * scale:
            return u, lam, it
    raise RuntimeError("Newton did not converge (step %g)" % step)


def run_dirk3(prob, u0, dt, nsteps, t0=0.0, on_step=None):
    """DIRK(3,3) (stiffly accurate, so u^{n+1} = u^{n,3}) with a Newton solve per stage."""
    a, b, c = ac.dirk3_tableau()
    d = np.linalg.inv(a)
    u = u0.copy()
    lam = np.zeros((prob.sk.faces.shape[0], 3 * prob.Nf))
    newton = []
    for n in range(nsteps):
        tn = t0 + n * dt
        stages = []
        ui = u.copy()
        for i in range(3):
            h = (sum(d[i, j] for j in range(i + 1)) * u - sum(d[i, j] * stages[j] for j in range(i))) / d[i, i]
            ui, lam, its = newton_stage(prob, ui, lam, h, d[i, i] / dt, tn + c[i] * dt)
            newton.append(its)
            stages.append(ui)
        u = stages[-1]
        if on_step is not None:
            on_step(n, tn + dt, u, lam)
    return u, lam, newton


def l2_error_velocity(prob, u, exact_v, t):
    err = 0.0
    Np = prob.Np
    for e, g in enumerate(prob.geo):
        vh = np.stack([g.V @ u[e, i * Np:(i + 1) * Np] for i in range(3)], axis=1)
        err += np.sum(g.w[:, None] * (vh - exact_v(g.xq, t)) ** 2)
    return math.sqrt(err)
