"""Host code of the library, without a GPU: the C++ skeleton/geometry builder and the C++
reference tables, through the host-only entry points of the C ABI, against the oracle's
independent numpy construction of the same objects (skeleton, element geometry, orthonormal
bases and quadrature)."""
import ctypes

import numpy as np
import pytest

from oracle import acoustic as ac
from oracle import reference as ref
from paper_1807_00086_gb300 import inputs

GEO = 32


@pytest.fixture(scope="module")
def lib():
    import os
    from paper_1807_00086_gb300 import build, hdg
    if not os.path.exists(hdg.LIB_PATH):
        build.build()
    return hdg.load()


def _ptr(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def host_skeleton(lib, vert, elem):
    dim = vert.shape[1]
    ne, nc = elem.shape
    vert = np.ascontiguousarray(vert, dtype=np.float64)
    elem = np.ascontiguousarray(elem, dtype=np.int32)
    nf = ctypes.c_int64()
    ef = np.zeros((ne, nc), dtype=np.int32)
    fs = np.zeros((nc * ne, 2), dtype=np.int32)
    fb = np.zeros(nc * ne, dtype=np.int32)
    geo = np.zeros((ne, GEO))
    st = lib.hdg_host_skeleton(dim, vert.shape[0], ne, _ptr(vert, ctypes.c_double), _ptr(elem, ctypes.c_int32),
                               ctypes.byref(nf), _ptr(ef, ctypes.c_int32), _ptr(fs, ctypes.c_int32),
                               _ptr(fb, ctypes.c_int32), _ptr(geo, ctypes.c_double))
    assert st == 0
    n = nf.value
    return n, ef, fs[:n], fb[:n], geo


@pytest.mark.parametrize("dim,N", [(2, 3), (3, 2)])
def test_skeleton_and_geometry_match_the_oracle(lib, dim, N):
    vert, elem = inputs.unit_square_tri(N) if dim == 2 else inputs.unit_cube_tet(N)
    # shuffle each element's vertex order: the library sorts by global id like the oracle
    rng = np.random.default_rng(5)
    elem = np.array([rng.permutation(row) for row in elem])
    n, ef, fs, fb, geo = host_skeleton(lib, vert, elem)
    sk = ac.skeleton(elem)
    nc = dim + 1
    assert n == sk.faces.shape[0]
    assert np.array_equal(ef, sk.elem_face)
    for f, inc in enumerate(sk.face_elems):
        slots = [e * nc + j for (e, j) in inc] + [-1] * (2 - len(inc))
        assert list(fs[f]) == slots
        assert (fb[f] >= 0) == sk.boundary[f]
    assert sorted(fb[fb >= 0].tolist()) == list(range(int(sk.boundary.sum())))
    for e in range(elem.shape[0]):
        X = vert[sk.elem[e]]
        J = (X[1:] - X[0]).T
        assert abs(geo[e, 0] - abs(np.linalg.det(J))) < 1e-14
        assert np.allclose(geo[e, 1:1 + dim * dim].reshape(dim, dim), np.linalg.inv(J), atol=1e-13)
        for f in range(nc):
            Y = X[ac.face_local_vertices(dim, f)]
            assert abs(geo[e, 1 + dim * dim + f] - ac.face_frame(Y)) < 1e-14
            n_f = geo[e, 1 + dim * dim + nc + f * dim:1 + dim * dim + nc + (f + 1) * dim]
            assert np.allclose(n_f, ac.outward_normal(X, f), atol=1e-14)


def test_skeleton_rejects_invalid_meshes(lib):
    vert, elem = inputs.unit_square_tri(2)
    bad = elem.copy()
    bad[0, 1] = bad[0, 0]
    with pytest.raises(AssertionError):
        host_skeleton(lib, vert, bad)
    bad = elem.copy()
    bad[1, 2] = vert.shape[0]
    with pytest.raises(AssertionError):
        host_skeleton(lib, vert, bad)


def _oracle_tables(dim, k):
    Np, Nf, Np1 = ref.n_modes(dim, k), ref.n_modes(dim - 1, k), ref.n_modes(dim, k + 1)
    xi, w = ref.simplex_rule(dim, k + 3)
    V, G = ref.basis(dim, k, xi)
    V1, G1 = ref.basis(dim, k + 1, xi)
    Dr = np.einsum("q,qlr,qi->ril", w, G, V)
    K1 = np.einsum("q,qir,qls->rsil", w, G1, G1)
    E1 = np.einsum("q,qir,ql->ril", w, G1, V)
    eta, wf = ref.simplex_rule(dim - 1, k + 3)
    U, _ = ref.basis(dim - 1, k, eta)
    verts = np.vstack([np.zeros(dim), np.eye(dim)])
    Ff = np.zeros((dim + 1, Np, Nf))
    for f in range(dim + 1):
        Y = verts[[v for v in range(dim + 1) if v != f]]
        Vf, _ = ref.basis(dim, k, Y[0] + eta @ (Y[1:] - Y[0]))
        Ff[f] = np.einsum("q,qi,qm->im", wf, Vf, U)
    return Dr, Ff, K1, E1


@pytest.mark.parametrize("dim,k", [(2, 1), (2, 4), (3, 1), (3, 3), (3, 4)])
def test_reference_tables_match_the_oracle_bases(lib, dim, k):
    Np, Nf, Np1 = ref.n_modes(dim, k), ref.n_modes(dim - 1, k), ref.n_modes(dim, k + 1)
    Dr = np.zeros((dim, Np, Np))
    Ff = np.zeros((dim + 1, Np, Nf))
    K1 = np.zeros((dim, dim, Np1, Np1))
    E1 = np.zeros((dim, Np1, Np))
    assert lib.hdg_host_tables(dim, k, _ptr(Dr, ctypes.c_double), _ptr(Ff, ctypes.c_double),
                               _ptr(K1, ctypes.c_double), _ptr(E1, ctypes.c_double)) == 0
    for got, want in zip((Dr, Ff, K1, E1), _oracle_tables(dim, k)):
        assert np.abs(got - want).max() < 1e-13 * max(1.0, np.abs(want).max())


def test_reference_tables_reject_unsupported_degrees(lib):
    assert lib.hdg_host_tables(3, 5, None, None, None, None) == -1
    assert lib.hdg_host_tables(1, 2, None, None, None, None) == -1


@pytest.mark.parametrize("dim,N,k", [(2, 3, 2), (2, 2, 4), (3, 2, 2), (3, 1, 3)])
@pytest.mark.parametrize("variant", ["edg", "iedg"])
def test_trace_node_map_matches_the_oracle(lib, dim, N, k, variant):
    """The C++ continuous-trace node map and nodal-to-modal table give the oracle's
    restriction R (same node numbering convention, independent construction)."""
    from oracle import edg
    vert, elem = inputs.unit_square_tri(N) if dim == 2 else inputs.unit_cube_tet(N)
    vert = np.ascontiguousarray(vert, dtype=np.float64)
    elem = np.ascontiguousarray(elem, dtype=np.int32)
    ne, nc = elem.shape
    Nf = ref.n_modes(dim - 1, k)
    nfree = ctypes.c_int64()
    fn = np.zeros((nc * ne, Nf), dtype=np.int32)
    Vinv = np.zeros((Nf, Nf))
    st = lib.hdg_host_trace_nodes(dim, vert.shape[0], ne, _ptr(vert, ctypes.c_double), _ptr(elem, ctypes.c_int32), k,
                                  1 if variant == "edg" else 0, ctypes.byref(nfree), _ptr(fn, ctypes.c_int32),
                                  _ptr(Vinv, ctypes.c_double))
    assert st == 0
    prob = ac.build_problem(vert, elem, k, 1.0, 1.0, 1.0)
    tm = edg.trace_map(prob, variant)
    assert nfree.value == tm.n_free
    assert np.abs(Vinv - tm.Vinv).max() < 1e-12
    interior = np.nonzero(~prob.sk.boundary)[0]
    R = np.zeros((interior.size * Nf, tm.n_free))
    for r, f in enumerate(interior):
        for a in range(Nf):
            if fn[f, a] >= 0:
                R[r * Nf:(r + 1) * Nf, fn[f, a]] += Vinv[:, a]
    assert np.abs(R - tm.R.toarray()).max() < 1e-12
