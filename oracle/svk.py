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
