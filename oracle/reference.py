"""Reference-element quadrature and orthonormal polynomial bases (oracle copy).

The discrete spaces of Sec. 2.2 (Eqs. e:spaces1, e:spaces2) are discontinuous P_k per
element and P_k per face. This module fixes a concrete basis for them:

* volume: the orthonormal Dubiner (PKDO) basis on the unit reference simplex
  {xi_r >= 0, sum xi_r <= 1}, orthonormal for d(xi) on that simplex; modes ordered
  lexicographically in (i, j) (triangle) or (i, j, l) (tetrahedron), i + j (+ l) <= k;
* face: the same construction one dimension lower (Legendre on [0, 1] for edges,
  Dubiner on the unit triangle for triangular faces).

Quadrature is the collapsed Gauss-Jacobi (Stroud) product rule with n points per
direction, exact for polynomials of degree 2n - 1.

Test infrastructure only (see oracle/__init__.py).
"""
import math

import numpy as np
from scipy.special import eval_jacobi, roots_jacobi


# ----------------------------------------------------------------------------- quadrature

def gauss_segment(n):
    """n-point Gauss-Legendre rule on [0, 1] (points (n,1), weights sum to 1)."""
    x, w = roots_jacobi(n, 0.0, 0.0)
    return ((x + 1.0) / 2.0)[:, None], w / 2.0


def gauss_triangle(n):
    """Collapsed n x n rule on the unit triangle (weights sum to 1/2).

    x = (1+a)/2 (1-y), y = (1+b)/2, dx dy = (1-b)/8 da db; the (1-b) factor is the
    Gauss-Jacobi(1,0) weight.
    """
    a, wa = roots_jacobi(n, 0.0, 0.0)
    b, wb = roots_jacobi(n, 1.0, 0.0)
    A, B = np.meshgrid(a, b, indexing="ij")
    WA, WB = np.meshgrid(wa, wb, indexing="ij")
    y = (1.0 + B) / 2.0
    x = (1.0 + A) / 2.0 * (1.0 - y)
    pts = np.stack([x.ravel(), y.ravel()], axis=1)
    return pts, (WA * WB).ravel() / 8.0


def gauss_tetrahedron(n):
    """Collapsed n^3 rule on the unit tetrahedron (weights sum to 1/6).

    dx dy dz = (1-b)(1-c)^2/64 da db dc with Gauss-Jacobi(1,0) in b and (2,0) in c.
    """
    a, wa = roots_jacobi(n, 0.0, 0.0)
    b, wb = roots_jacobi(n, 1.0, 0.0)
    c, wc = roots_jacobi(n, 2.0, 0.0)
    A, B, C = np.meshgrid(a, b, c, indexing="ij")
    WA, WB, WC = np.meshgrid(wa, wb, wc, indexing="ij")
    z = (1.0 + C) / 2.0
    y = (1.0 + B) / 2.0 * (1.0 - z)
    x = (1.0 + A) / 2.0 * (1.0 - y - z)
    pts = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)
    return pts, (WA * WB * WC).ravel() / 64.0


def simplex_rule(dim, n):
    """Quadrature on the unit simplex of dimension dim (0 < dim <= 3)."""
    return {1: gauss_segment, 2: gauss_triangle, 3: gauss_tetrahedron}[dim](n)


# ----------------------------------------------------------------------------- bases

def n_modes(dim, k):
    """dim P_k on a dim-simplex: (k+1)...(k+dim)/dim!."""
    return math.comb(k + dim, dim)


def mode_indices(dim, k):
    """Lexicographic multi-indices of the Dubiner modes of total degree <= k."""
    if dim == 1:
        return [(i,) for i in range(k + 1)]
    if dim == 2:
        return [(i, j) for i in range(k + 1) for j in range(k + 1 - i)]
    return [(i, j, l) for i in range(k + 1) for j in range(k + 1 - i) for l in range(k + 1 - i - j)]


def _jac(n, a, b, x):
    if n < 0:
        return np.zeros_like(x)
    return eval_jacobi(n, a, b, x)


def _djac(n, a, b, x):
    """d/dx P_n^(a,b)(x) = (n+a+b+1)/2 P_{n-1}^(a+1,b+1)(x)."""
    if n <= 0:
        return np.zeros_like(x)
    return 0.5 * (n + a + b + 1) * eval_jacobi(n - 1, a + 1, b + 1, x)


def basis(dim, k, pts):
    """Orthonormal basis values and reference gradients at points of the unit simplex.

    Returns (V, G): V[q, i] = phi_i(pts[q]), G[q, i, r] = d phi_i / d xi_r.
    Points must be interior (collapsed coordinates are singular on some edges).
    """
    pts = np.asarray(pts, dtype=np.float64)
    nq = pts.shape[0]
    idx = mode_indices(dim, k)
    V = np.zeros((nq, len(idx)))
    G = np.zeros((nq, len(idx), dim))
    if dim == 1:
        s = pts[:, 0]
        for m, (i,) in enumerate(idx):
            c = math.sqrt(2 * i + 1)
            V[:, m] = c * _jac(i, 0, 0, 2 * s - 1)
            G[:, m, 0] = c * 2 * _djac(i, 0, 0, 2 * s - 1)
        return V, G
    if dim == 2:
        x, y = pts[:, 0], pts[:, 1]
        w = 1.0 - y
        a = 2.0 * x / w - 1.0
        b = 2.0 * y - 1.0
        for m, (i, j) in enumerate(idx):
            c = math.sqrt(2.0 * (2 * i + 1) * (i + j + 1))
            # phi = A(x,y) Bj(y),  A = P_i(a) w^i,  Bj = P_j^(2i+1,0)(2y-1)
            A = _jac(i, 0, 0, a) * w ** i
            dA_dx = 2.0 * _djac(i, 0, 0, a) * w ** (i - 1) if i > 0 else np.zeros(nq)
            dA_dy = (w ** (i - 1) * (_djac(i, 0, 0, a) * (a + 1.0) - i * _jac(i, 0, 0, a))
                     if i > 0 else np.zeros(nq))
            Bj = _jac(j, 2 * i + 1, 0, b)
            dBj = 2.0 * _djac(j, 2 * i + 1, 0, b)
            V[:, m] = c * A * Bj
            G[:, m, 0] = c * dA_dx * Bj
            G[:, m, 1] = c * (dA_dy * Bj + A * dBj)
        return V, G
    x, y, z = pts[:, 0], pts[:, 1], pts[:, 2]
    w = 1.0 - y - z
    q = 1.0 - z
    a = 2.0 * x / w - 1.0
    b = 2.0 * y / q - 1.0
    cc = 2.0 * z - 1.0
    for m, (i, j, l) in enumerate(idx):
        c = math.sqrt((2 * i + 1) * (2 * i + 2 * j + 2) * (2 * i + 2 * j + 2 * l + 3))
        # phi = A B C with A = P_i(a) w^i, B = P_j^(2i+1,0)(b) q^j, C = P_l^(2i+2j+2,0)(2z-1)
        A = _jac(i, 0, 0, a) * w ** i
        if i > 0:
            dA_dx = 2.0 * _djac(i, 0, 0, a) * w ** (i - 1)
            dA_dyz = w ** (i - 1) * (_djac(i, 0, 0, a) * (a + 1.0) - i * _jac(i, 0, 0, a))
        else:
            dA_dx = np.zeros(nq)
            dA_dyz = np.zeros(nq)
        B = _jac(j, 2 * i + 1, 0, b) * q ** j
        if j > 0:
            dB_dy = 2.0 * _djac(j, 2 * i + 1, 0, b) * q ** (j - 1)
            dB_dz = q ** (j - 1) * (_djac(j, 2 * i + 1, 0, b) * (b + 1.0) - j * _jac(j, 2 * i + 1, 0, b))
        else:
            dB_dy = np.zeros(nq)
            dB_dz = np.zeros(nq)
        C = _jac(l, 2 * i + 2 * j + 2, 0, cc)
        dC_dz = 2.0 * _djac(l, 2 * i + 2 * j + 2, 0, cc)
        V[:, m] = c * A * B * C
        G[:, m, 0] = c * dA_dx * B * C
        G[:, m, 1] = c * (dA_dyz * B * C + A * dB_dy * C)
        G[:, m, 2] = c * (dA_dyz * B * C + A * dB_dz * C + A * B * dC_dz)
    return V, G
