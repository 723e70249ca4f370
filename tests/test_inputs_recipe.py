"""The seeded synthetic workloads against the recipes they stand for (CPU).

Sizes, value ranges and distributions of the generated inputs: the 196,608-tet acoustic mesh
with c ~ logU[1, 3], the 64 interior sources of the multi-source batch, the per-element
degrees and lognormal Lame parameters of the elastic workload, and the Poisson arrivals and
request mix of the serving workload. Statistical checks use bounds several standard errors
wide, on fixed seeds.
"""
import math

import numpy as np

from paper_1807_00086_gb300 import inputs
from paper_1807_00086_gb300.serve import serving_workload


def _holders(vert, elem, x):
    """Elements whose closed simplex holds x, by barycentric coordinates from the vertices."""
    X = vert[np.sort(elem, axis=1)]                                   # [ne][4][3]
    A = np.concatenate([np.transpose(X, (0, 2, 1)), np.ones((len(elem), 1, 4))], axis=1)
    lam = np.linalg.solve(A, np.broadcast_to(np.append(x, 1.0), (len(elem), 4))[..., None])[..., 0]
    return np.nonzero(lam.min(axis=1) >= -1e-12)[0]


def test_acoustic_workload_sizes_and_wave_speeds():
    w = inputs.acoustic_3d_workload(N=32, k=3)
    ne = w["elem"].shape[0]
    assert ne == 6 * 32 ** 3 == 196608 and w["vert"].shape == (33 ** 3, 3)
    c = w["c"]
    assert c.min() >= 1.0 and c.max() <= 3.0
    # log c uniform on [0, log 3]: mean log 3 / 2, variance (log 3)^2 / 12
    lc = np.log(c)
    se = math.log(3.0) / math.sqrt(12.0 * ne)
    assert abs(lc.mean() - 0.5 * math.log(3.0)) < 6 * se
    assert abs(np.mean(c < math.sqrt(3.0)) - 0.5) < 6 * 0.5 / math.sqrt(ne)
    assert np.all(w["rho"] == 1.0) and w["tau"] == 1.0 and w["f0"] == 10.0 and abs(w["t0"] - 0.12) < 1e-15


def test_acoustic_source_lies_on_a_cell_diagonal_shared_by_six_tets():
    """The source point at the centre + 0.3 h (1, 1, 1) is on the main diagonal of its cell:
    six tets hold it and the lowest id among them takes the source (same rule in the oracle
    and the library); it is no mesh vertex."""
    N = 8
    w = inputs.acoustic_3d_workload(N=N, k=3)
    x = w["sources"][0]
    h = _holders(w["vert"], w["elem"], x)
    assert len(h) == 6
    assert np.min(np.abs(w["vert"] - x).sum(axis=1)) > 0.1 / N


def test_multisource_positions_are_interior_and_distinct():
    w = inputs.acoustic_3d_multisource_workload(N=4, k=3, nsrc=64)
    p = w["sources"]
    assert p.shape == (64, 3) and p.min() >= 0.1 and p.max() <= 0.9
    d = np.linalg.norm(p[:, None, :] - p[None, :, :], axis=2) + np.eye(64)
    assert d.min() > 1e-3
    assert np.array_equal(w["source_cols"], np.arange(64))


def test_elastic_workload_degrees_and_lame_parameters():
    w = inputs.elastic_3d_mixed_workload(N=24)
    ne = w["elem"].shape[0]
    assert ne == 6 * 24 ** 3 == 82944
    k = w["elem_k"]
    assert set(np.unique(k)) == {1, 2, 3, 4}
    for j in range(1, 5):   # uniform over {1..4}
        assert abs(np.mean(k == j) - 0.25) < 6 * math.sqrt(0.25 * 0.75 / ne)
    for name, median in (("lam", 1.5), ("mu", 1.0)):
        lv = np.log(w[name])
        assert abs(np.median(lv) - math.log(median)) < 0.02
        assert abs(lv.std() - 0.5) < 0.01
    assert not np.allclose(w["lam"] / 1.5, w["mu"])   # independent draws
    assert np.all(w["rho"] == 1.0)


def test_serving_arrivals_are_poisson_at_the_stated_rate():
    reqs = serving_workload(n_req=1000, rate=20.0)
    t = np.array([r.arrival for r in reqs])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    # exponential gaps: mean 1/20 s, coefficient of variation 1
    assert abs(gaps.mean() - 0.05) < 6 * 0.05 / math.sqrt(1000)
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.15
    ks = np.array([r.k for r in reqs])
    steps = np.array([r.nsteps for r in reqs])
    dims = np.array([r.dim for r in reqs])
    assert set(np.unique(ks)) == {1, 2, 3, 4} and steps.min() >= 20 and steps.max() <= 200
    assert abs(np.mean(dims == 3) - 0.5) < 6 * 0.5 / math.sqrt(1000)
    ne = np.array([2 * r.N ** 2 if r.dim == 2 else 6 * r.N ** 3 for r in reqs])
    # the element counts snap to structured meshes around the log-uniform 1e3..1e5 draw
    assert ne.min() >= 500 and ne.max() <= 2e5
    assert 0.2 < np.mean(ne < 1e4) < 0.8
    for r in reqs:
        assert r.source.shape == (r.dim,) and r.source.min() >= 0.1 and r.source.max() <= 0.9
