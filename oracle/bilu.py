"""Block ILU(0) of the assembled trace system (Sec. 2.4: the paper preconditions its GMRES
trace solves with block-ILU(0)), plain FP64 oracle. Test infrastructure only (see
oracle/__init__.py).

The matrix is taken in block sparse row form with one block row per face (N_f x N_f
blocks; the pattern is the face adjacency: two faces are coupled when they share an element).
ILU(0) keeps exactly that pattern: it computes block factors L (unit block diagonal) and U with
(L U)_ij = A_ij for every block (i, j) of the pattern, row by row in the given order (the IKJ
form of Gaussian elimination with every fill block outside the pattern dropped). The
preconditioner solves L U z = r by a forward and a backward block substitution.
"""
import numpy as np


def pattern_from_skeleton(elem_face, interior):
    """Block pattern of the assembled trace operator on the interior faces: rows = interior
    faces in increasing face id, columns = the interior faces sharing an element with the row
    face (itself included), ascending. Returns (rows, cols) as a list of face ids and a list of
    sorted column lists."""
    nbr = {}
    for e in range(elem_face.shape[0]):
        fs = [int(f) for f in elem_face[e] if interior[f]]
        for f in fs:
            nbr.setdefault(f, set()).update(fs)
    rows = sorted(nbr)
    return rows, [sorted(nbr[f]) for f in rows]


def assemble_blocks(rows, cols, block):
    """Dense block entries A[(i, j)] = block(i, j) on the pattern."""
    return {(i, j): np.array(block(i, j), dtype=np.float64) for i, cs in zip(rows, cols) for j in cs}


def factor(rows, cols, A):
    """ILU(0): returns (F, Dinv) with F[(i, j)] = L_ij for j < i and U_ij for j >= i, and
    Dinv[i] = U_ii^{-1}. Row i, for every k < i of its pattern in increasing order:
    L_ik = A_ik U_kk^{-1}; then A_ij -= L_ik U_kj for every j > k in both patterns."""
    F = {key: val.copy() for key, val in A.items()}
    Dinv = {}
    pos = {i: set(cs) for i, cs in zip(rows, cols)}
    for i, cs in zip(rows, cols):
        for k in cs:
            if k >= i:
                break
            F[(i, k)] = F[(i, k)] @ Dinv[k]
            for j in pos[k]:
                if j > k and j in pos[i]:
                    F[(i, j)] = F[(i, j)] - F[(i, k)] @ F[(k, j)]
        Dinv[i] = np.linalg.inv(F[(i, i)])
    return F, Dinv


def solve(rows, cols, F, Dinv, r):
    """z = (L U)^{-1} r for r given per row face (dict face -> vector)."""
    y = {}
    for i, cs in zip(rows, cols):
        s = np.array(r[i], dtype=np.float64)
        for k in cs:
            if k >= i:
                break
            s = s - F[(i, k)] @ y[k]
        y[i] = s
    z = {}
    for i, cs in reversed(list(zip(rows, cols))):
        s = y[i].copy()
        for j in cs:
            if j > i:
                s = s - F[(i, j)] @ z[j]
        z[i] = Dinv[i] @ s
    return z
