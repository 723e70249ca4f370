"""Seeded synthetic inputs shared by the CUDA path, the tests and the benchmark.

This module holds none of the method's arithmetic: it only lays out structured simplex
meshes, draws per-element material fields, source positions and random states from a
seed. Both the CUDA library (through ``bench.py`` and the tests) and the CPU oracle
receive the same arrays from here.

Mesh recipes (the shapes of the paper's workloads, Sec. 2.1 meshes of simplices):
  * unit square, N x N squares, each cut by the (i, j) -> (i+1, j+1) diagonal: 2 N^2
    triangles;
  * unit cube, N^3 cubes, each cut into the 6 Kuhn tetrahedra that share the cube's main
    diagonal (conforming across cubes): 6 N^3 tetrahedra.
"""
import itertools

import numpy as np

DEFAULT_SEED = 1807


def unit_square_tri(N):
    """Returns (vert[(N+1)^2, 2], elem[2 N^2, 3]); vertex id = i + (N+1) j."""
    g = np.linspace(0.0, 1.0, N + 1)
    X, Y = np.meshgrid(g, g, indexing="xy")
    vert = np.stack([X.ravel(), Y.ravel()], axis=1)
    vid = lambda i, j: i + (N + 1) * j
    elem = []
    for j in range(N):
        for i in range(N):
            v00, v10, v01, v11 = vid(i, j), vid(i + 1, j), vid(i, j + 1), vid(i + 1, j + 1)
            elem.append((v00, v10, v11))
            elem.append((v00, v11, v01))
    return vert, np.array(elem, dtype=np.int32)


def unit_cube_tet(N):
    """Returns (vert[(N+1)^3, 3], elem[6 N^3, 4]); vertex id = i + (N+1)(j + (N+1) l)."""
    g = np.linspace(0.0, 1.0, N + 1)
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    vert = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    n1 = N + 1
    I, J, L = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    base = np.stack([I.ravel(), J.ravel(), L.ravel()], axis=1)   # cube corner (i, j, l)
    # order cubes by l, then j, then i (i fastest)
    order = np.lexsort((base[:, 0], base[:, 1], base[:, 2]))
    base = base[order]
    elems = []
    for perm in itertools.permutations(range(3)):
        c = base.copy()
        path = [c.copy()]
        for ax in perm:
            c = c.copy()
            c[:, ax] += 1
            path.append(c)
        ids = [p[:, 0] + n1 * (p[:, 1] + n1 * p[:, 2]) for p in path]
        elems.append(np.stack(ids, axis=1))
    elem = np.stack(elems, axis=1).reshape(-1, 4)   # 6 consecutive tets per cube
    return vert, elem.astype(np.int32)


def loguniform(n, lo, hi, seed=DEFAULT_SEED):
    rng = np.random.default_rng(seed)
    return np.exp(rng.uniform(np.log(lo), np.log(hi), size=n))


def lognormal(n, median, sigma, seed=DEFAULT_SEED):
    rng = np.random.default_rng(seed)
    return median * np.exp(sigma * rng.standard_normal(n))


def uniform_points(n, dim, lo=0.1, hi=0.9, seed=DEFAULT_SEED):
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=(n, dim))


def random_state(n_elem, n_local, seed=DEFAULT_SEED):
    """Seeded random element coefficients [n_elem, n_local] (for parity tests)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n_elem, n_local))


def random_traces(n_faces, n_face_dofs, seed=DEFAULT_SEED):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n_faces, n_face_dofs))


def plate_tet(n, thickness=0.01):
    """The unit square plate [0, 1]^2 x [0, thickness] with n x n x 1 cubes of 6 Kuhn tets each
    (one element layer through the thickness): (vert[(n+1)^2 2, 3], elem[6 n^2, 4])."""
    gx = np.linspace(0.0, 1.0, n + 1)
    vert, elem = [], []
    Z, Y, X = np.meshgrid(np.array([0.0, thickness]), gx, gx, indexing="ij")
    vert = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    n1 = n + 1
    for j in range(n):
        for i in range(n):
            for perm in itertools.permutations(range(3)):
                c = [i, j, 0]
                path = [tuple(c)]
                for ax in perm:
                    c = list(c)
                    c[ax] += 1
                    path.append(tuple(c))
                elem.append([p[0] + n1 * (p[1] + n1 * p[2]) for p in path])
    return vert, np.array(elem, dtype=np.int32)


def acoustic_3d_workload(N=32, k=3, seed=DEFAULT_SEED):
    """3D acoustic wave workload: unit cube, 6 N^3 tets, c ~ logU[1, 3] per element, rho = 1,
    one Ricker point source at the cube centre shifted by 0.3 h (1, 1, 1). The point lies on the
    main diagonal of its cell, the edge shared by the cell's 6 tets (no mesh vertex); the source
    goes to the lowest-id tet containing it."""
    vert, elem = unit_cube_tet(N)
    ne = elem.shape[0]
    c = loguniform(ne, 1.0, 3.0, seed)
    rho = np.ones(ne)
    h = 1.0 / N
    src = np.array([[0.5 + 0.3 * h, 0.5 + 0.3 * h, 0.5 + 0.3 * h]])
    return dict(vert=vert, elem=elem, k=k, rho=rho, c=c, tau=1.0, sources=src, f0=10.0, t0=1.2 / 10.0)


def acoustic_3d_multisource_workload(N=32, k=3, nsrc=64, seed=DEFAULT_SEED):
    """The 3D acoustic workload with `nsrc` Ricker point sources at seeded uniform interior
    points of [0.1, 0.9]^3, source i driving right-hand-side column i."""
    w = acoustic_3d_workload(N=N, k=k, seed=seed)
    w["sources"] = uniform_points(nsrc, 3, 0.1, 0.9, seed + 64)
    w["source_cols"] = np.arange(nsrc, dtype=np.int32)
    return w


def element_degrees(ne, kmin=1, kmax=4, seed=DEFAULT_SEED):
    """Per-element polynomial degree drawn uniformly from {kmin..kmax} (int32)."""
    return np.random.default_rng(seed).integers(kmin, kmax + 1, size=ne).astype(np.int32)


def elastic_3d_mixed_workload(N=24, seed=DEFAULT_SEED):
    """The elastic workload with a per-element degree drawn uniformly from {1, 2, 3, 4}."""
    w = elastic_3d_workload(N=N, k=4, seed=seed)
    w["elem_k"] = element_degrees(w["elem"].shape[0], 1, 4, seed + 7)
    return w


def elastic_3d_workload(N=24, k=3, seed=DEFAULT_SEED):
    """3D linear elastodynamics workload: unit cube, 6 N^3 tets, rho = 1, Lame parameters
    lognormal per element (sigma 0.5; medians lam = 1.5, mu = 1), clamped boundary, initial
    velocity e_z exp(-|x - x_c|^2 / (2 * 0.05^2)) with x_c the cube centre, zero stress."""
    vert, elem = unit_cube_tet(N)
    ne = elem.shape[0]
    return dict(vert=vert, elem=elem, k=k, rho=np.ones(ne), lam=lognormal(ne, 1.5, 0.5, seed),
                mu=lognormal(ne, 1.0, 0.5, seed + 1), center=np.array([0.5, 0.5, 0.5]), width=0.05)


def gaussian_velocity_values(xq, center, width, ncomp):
    """Point values [.., ncomp] of the elastic initial data at points xq [.., 3]: v_z bump."""
    r2 = np.sum((xq - center) ** 2, axis=-1)
    vals = np.zeros(xq.shape[:-1] + (ncomp,))
    vals[..., 2] = np.exp(-r2 / (2.0 * width * width))
    return vals
