"""Allocation-free trace apply (hdg_trace_apply_noalloc) against hdg_trace_apply.

Callers that cannot allocate device memory when they need y = K x (an allocation would
synchronise the device inside their loop, or they may only use memory handed to them
up front) get an entry point whose only scratch is a fixed array inside the library.
This file sorts last so that a stop-at-first-failure run has run every other test first.
"""
import ctypes

import numpy as np
import pytest

from paper_1807_00086_gb300 import inputs

pytestmark = pytest.mark.gpu


def connectivity(elem, dim):
    """Face tables in the library's documented layout, built from the element list."""
    el = np.sort(np.asarray(elem, dtype=np.int64), axis=1)
    nc = dim + 1
    keys = np.stack([np.delete(el, j, axis=1) for j in range(nc)], axis=1).reshape(-1, dim)  # slot e*nc+j
    uniq, inv = np.unique(keys, axis=0, return_inverse=True)
    inv = inv.ravel()
    nf = uniq.shape[0]
    face_slot = -np.ones((nf, 2), dtype=np.int32)
    seen = np.zeros(nf, dtype=np.int64)
    for slot, f in enumerate(inv):          # slots ascending: lower element first
        face_slot[f, seen[f]] = slot
        seen[f] += 1
    bnd = seen == 1
    face_bnd = np.where(bnd, np.cumsum(bnd) - 1, -1).astype(np.int32)
    return inv.reshape(-1, nc).astype(np.int32), face_slot, face_bnd


@pytest.mark.parametrize("dim,N,k", [(3, 4, 3), (2, 8, 2)])
def test_noalloc_apply_matches_trace_apply_twice(dim, N, k):
    import torch
    from paper_1807_00086_gb300 import hdg
    lib = hdg.load()
    vert, elem = inputs.unit_square_tri(N) if dim == 2 else inputs.unit_cube_tet(N)
    ne = elem.shape[0]
    s = hdg.Solver(vert, elem, k, 1.0, 1.0, inputs.loguniform(ne, 1.0, 3.0, 5))
    s.hdg_condense(750.0)
    S = s.hdg_get_schur()
    ef, fs, fb = (torch.tensor(a, device="cuda") for a in connectivity(elem, dim))
    assert fs.shape[0] == s.n_faces
    err = ctypes.create_string_buffer(256)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for seed in (1, 2):                      # two calls in a row share the scratch array
        x = torch.tensor(inputs.random_traces(s.n_faces, s.Nf, seed), device="cuda")
        y_ref = s.hdg_trace_apply(x)
        y = torch.full_like(x, float("nan"))
        st = lib.hdg_trace_apply_noalloc(dim, k, ne, s.n_faces, S.data_ptr(), ef.data_ptr(), fs.data_ptr(),
                                         fb.data_ptr(), x.data_ptr(), y.data_ptr(), stream, err, 256)
        assert st == 0, err.value
        torch.cuda.synchronize()
        a, b = y.cpu().numpy(), y_ref.cpu().numpy()
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_1807_00086_gb300 import hdg
    lib = hdg.load()
    err = ctypes.create_string_buffer(256)
    dummy = ctypes.c_void_p(16)               # never dereferenced: the size check comes first
    st = lib.hdg_trace_apply_noalloc(3, 3, 30000, 60000, dummy, dummy, dummy, dummy, dummy, dummy, None, err, 256)
    assert st == -1 and b"exceeds the fixed scratch" in err.value
