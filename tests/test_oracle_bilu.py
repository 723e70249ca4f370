"""Pins of the oracle's block ILU(0) (oracle/bilu.py), by facts independent of it:
  * on a full block pattern ILU(0) drops nothing, so it is the exact block LU and the
    preconditioner solves A z = r (checked against a dense solve);
  * on a block-diagonal pattern it is block Jacobi, z_i = A_ii^{-1} r_i;
  * on the face pattern of the acoustic trace operator -K (Eq. LS): the defining property of
    ILU(0), (L U)_ij = A_ij on every block of the pattern, and L U z = r for the solve;
  * a factorisation in the wrong row order breaks that property (the check can fail).
"""
import numpy as np

from oracle import acoustic as ac
from oracle import bilu
from paper_1807_00086_gb300 import inputs


def _lu_blocks(rows, cols, F, i, j, nb):
    """(L U)_ij with L unit block lower and U block upper, both on the pattern."""
    pos = {r: set(c) for r, c in zip(rows, cols)}
    s = np.zeros((nb, nb))
    for k in rows:
        if k > min(i, j):
            break
        lik = np.eye(nb) if k == i else (F[(i, k)] if k in pos[i] and k < i else None)
        ukj = F[(k, j)] if j in pos[k] and j >= k else None
        if lik is not None and ukj is not None:
            s += lik @ ukj
    return s


def test_full_pattern_is_exact_block_lu():
    rng = np.random.default_rng(1)
    n, nb = 5, 3
    A = rng.standard_normal((n * nb, n * nb)) + 4 * n * nb * np.eye(n * nb)
    rows = list(range(n))
    cols = [list(range(n)) for _ in rows]
    blocks = bilu.assemble_blocks(rows, cols, lambda i, j: A[i * nb:(i + 1) * nb, j * nb:(j + 1) * nb])
    F, Dinv = bilu.factor(rows, cols, blocks)
    r = rng.standard_normal(n * nb)
    z = bilu.solve(rows, cols, F, Dinv, {i: r[i * nb:(i + 1) * nb] for i in rows})
    zz = np.concatenate([z[i] for i in rows])
    assert np.abs(zz - np.linalg.solve(A, r)).max() < 1e-13 * np.abs(zz).max()


def test_block_diagonal_pattern_is_block_jacobi():
    rng = np.random.default_rng(2)
    n, nb = 4, 3
    rows = list(range(n))
    cols = [[i] for i in rows]
    D = {i: rng.standard_normal((nb, nb)) + 5 * np.eye(nb) for i in rows}
    F, Dinv = bilu.factor(rows, cols, bilu.assemble_blocks(rows, cols, lambda i, j: D[i]))
    r = {i: rng.standard_normal(nb) for i in rows}
    z = bilu.solve(rows, cols, F, Dinv, r)
    for i in rows:
        assert np.abs(z[i] - np.linalg.solve(D[i], r[i])).max() < 1e-14


def _trace_operator(N=2, k=2):
    w = inputs.acoustic_3d_workload(N=N, k=k)
    prob = ac.build_problem(w["vert"], w["elem"], k, w["tau"], w["rho"], w["c"])
    cond = ac.condense(prob, 1.5 / (2e-3 * 32.0 / N))
    A = (-cond.K).toarray()
    interior = ~np.asarray(prob.sk.boundary)
    ids = np.nonzero(interior)[0]
    where = {int(f): t for t, f in enumerate(ids)}
    Nf = prob.Nf
    rows, cols = bilu.pattern_from_skeleton(prob.sk.elem_face, interior)

    def block(i, j):
        a, b = where[i], where[j]
        return A[a * Nf:(a + 1) * Nf, b * Nf:(b + 1) * Nf]
    return A, rows, cols, bilu.assemble_blocks(rows, cols, block), Nf, where


def test_ilu0_reproduces_the_trace_operator_on_its_pattern():
    A, rows, cols, blocks, Nf, where = _trace_operator()
    # the pattern holds every nonzero block of -K (and -K has no block outside it)
    nz = {(i, j) for i in rows for j in rows
          if np.abs(A[where[i] * Nf:(where[i] + 1) * Nf, where[j] * Nf:(where[j] + 1) * Nf]).max() > 0}
    assert nz <= set(blocks)
    F, Dinv = bilu.factor(rows, cols, blocks)
    scale = max(np.abs(b).max() for b in blocks.values())
    for i, cs in zip(rows, cols):
        for j in cs:
            assert np.abs(_lu_blocks(rows, cols, F, i, j, Nf) - blocks[(i, j)]).max() < 1e-12 * scale, (i, j)
    rng = np.random.default_rng(3)
    r = {i: rng.standard_normal(Nf) for i in rows}
    z = bilu.solve(rows, cols, F, Dinv, r)
    # L U z = r
    y = {}
    for i, cs in zip(rows, cols):
        y[i] = sum((F[(i, j)] @ z[j] for j in cs if j >= i), np.zeros(Nf))       # U z
    for i, cs in zip(rows, cols):
        lu = y[i] + sum((F[(i, k)] @ y[k] for k in cs if k < i), np.zeros(Nf))    # L (U z)
        assert np.abs(lu - r[i]).max() < 1e-10 * max(np.abs(r[i]).max(), 1.0)


def test_factoring_rows_out_of_order_breaks_the_ilu0_property():
    A, rows, cols, blocks, Nf, where = _trace_operator()
    rev_rows = rows[::-1]
    rev_cols = [cs for cs in cols[::-1]]
    # process the rows in reverse with the same (ascending) column lists: rows then miss the
    # updates from their lower neighbours, and L U no longer matches A on the pattern
    F, _ = _factor_in_order(rev_rows, rev_cols, blocks)
    bad = 0.0
    for i, cs in zip(rows, cols):
        for j in cs:
            bad = max(bad, np.abs(_lu_blocks(rows, cols, F, i, j, Nf) - blocks[(i, j)]).max())
    assert bad > 1e-6


def _factor_in_order(rows, cols, A):
    """bilu.factor's steps with the rows visited in the given order (planted mistake)."""
    F = {key: val.copy() for key, val in A.items()}
    Dinv = {}
    pos = {i: set(cs) for i, cs in zip(rows, cols)}
    for i, cs in zip(rows, cols):
        for k in cs:
            if k >= i:
                break
            if k not in Dinv:
                Dinv[k] = np.linalg.inv(F[(k, k)])
            F[(i, k)] = F[(i, k)] @ Dinv[k]
            for j in pos[k]:
                if j > k and j in pos[i]:
                    F[(i, j)] = F[(i, j)] - F[(i, k)] @ F[(k, j)]
        Dinv[i] = np.linalg.inv(F[(i, i)])
    return F, Dinv
