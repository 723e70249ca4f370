"""Saint Venant-Kirchhoff hyperelasticity (Sec. 4.4, Eqs. eq:rel_P_S_Psi and eq:psi_SVK_NeoHook),
plain FP64 oracle (test infrastructure only).

With C = F^T F and the Lagrangian strain E = (C - I) / 2, the second Piola-Kirchhoff stress is
S = lam tr(E) I + 2 mu E and the first is P = F S. Both derive from the stored energy
psi(F) = lam / 2 tr(E)^2 + mu E : E (P = d psi / dF). The tangent A = dP/dF is the
derivative of F S(F): dP = dF S + F dS with dS = lam tr(dE) I + 2 mu dE and
dE = (dF^T F + F^T dF) / 2.
All tensors are d x d arrays, the tangent a (d*d) x (d*d) matrix in row-major (i, J) order.
"""
import numpy as np


def green_strain(F):
    return 0.5 * (F.T @ F - np.eye(F.shape[0]))


def energy(F, lam, mu):
    E = green_strain(F)
    return 0.5 * lam * np.trace(E) ** 2 + mu * np.sum(E * E)


def second_pk(F, lam, mu):
    E = green_strain(F)
    return lam * np.trace(E) * np.eye(F.shape[0]) + 2.0 * mu * E


def first_pk(F, lam, mu):
    return F @ second_pk(F, lam, mu)


def tangent(F, lam, mu):
    """A[(i, J), (k, L)] = d P_iJ / d F_kL."""
    d = F.shape[0]
    S = second_pk(F, lam, mu)
    A = np.zeros((d * d, d * d))
    for k in range(d):
        for L in range(d):
            dF = np.zeros((d, d))
            dF[k, L] = 1.0
            dE = 0.5 * (dF.T @ F + F.T @ dF)
            dS = lam * np.trace(dE) * np.eye(d) + 2.0 * mu * dE
            A[:, k * d + L] = (dF @ S + F @ dS).ravel()
    return A


def plate_solution(lam, mu, rho, amp=0.4):
    """The clamped vibrating plate of Sec. 4.5 with its data, as numpy callables of
    (x[n, 3], t). Reading of a garbled formula: the deformation map is
    phi = (X, Y, Z + amp sin(pi t) sin(pi X) sin(pi Y)) (the printed map has zeros in its
    first two components, which would not be the identity at t = 0). Returns a dict with
    v (velocity), F (deformation gradient, row-major 9 components), P (first Piola-Kirchhoff,
    SVK) and f = rho dv/dt - div P (body force); the traction on a face of normal n is P n."""
    import sympy as s
    X, Y, Z, t = s.symbols("X Y Z t", real=True)
    w = amp * s.sin(s.pi * t) * s.sin(s.pi * X) * s.sin(s.pi * Y)
    phi = s.Matrix([X, Y, Z + w])
    xs = [X, Y, Z]
    F = phi.jacobian(xs)
    v = phi.diff(t)
    E = (F.T * F - s.eye(3)) / 2
    S = lam * E.trace() * s.eye(3) + 2 * mu * E
    P = F * S
    divP = s.Matrix([sum(s.diff(P[i, J], xs[J]) for J in range(3)) for i in range(3)])
    f = rho * v.diff(t) - divP

    def vec(expr, n):
        fn = s.lambdify((X, Y, Z, t), list(expr), "numpy")

        def call(x, tt):
            x = np.atleast_2d(x)
            vals = fn(x[:, 0], x[:, 1], x[:, 2], tt)
            return np.stack([np.broadcast_to(np.asarray(c, dtype=float), (x.shape[0],)) for c in vals], axis=1)
        return call

    return {"v": vec(v, 3), "F": vec(F.reshape(9, 1), 9), "P": vec(P.reshape(9, 1), 9), "f": vec(f, 3)}
