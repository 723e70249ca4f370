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


def _call(lib, dim, k, ne, nf, S, ef, fs, fb, x, y, stream, err):
    return lib.hdg_trace_apply_noalloc(dim, k, ne, nf, S.data_ptr(), ef.data_ptr(), fs.data_ptr(), fb.data_ptr(),
                                       x.data_ptr(), y.data_ptr(), stream, err, 256)


CASES = [(2, 4, 1), (2, 4, 2), (2, 3, 3), (2, 3, 4), (3, 2, 1), (3, 2, 2), (3, 4, 3), (3, 1, 4)]


@pytest.mark.parametrize("dim,N,k", CASES)
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
        st = _call(lib, dim, k, ne, s.n_faces, S, ef, fs, fb, x, y, stream, err)
        assert st == 0, err.value
        torch.cuda.synchronize()
        a, b = y.cpu().numpy(), y_ref.cpu().numpy()
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()


def test_noalloc_apply_of_a_nonsymmetric_block_and_no_device_allocation():
    """y = sum_K P_K^T S_K P_K x for arbitrary (non-symmetric) blocks, against a plain torch
    gather / batched mat-vec / scatter; device memory is the same before and after calls."""
    import torch
    from paper_1807_00086_gb300 import hdg
    lib = hdg.load()
    dim, N, k = 3, 3, 3
    vert, elem = inputs.unit_cube_tet(N)
    ne = elem.shape[0]
    ef_np, fs_np, fb_np = connectivity(elem, dim)
    nf = fs_np.shape[0]
    Nf = (k + 1) * (k + 2) // 2
    m = (dim + 1) * Nf
    S = torch.tensor(np.random.default_rng(3).standard_normal((ne, m, m)), device="cuda")
    ef, fs, fb = (torch.tensor(a, device="cuda") for a in (ef_np, fs_np, fb_np))
    err = ctypes.create_string_buffer(256)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    x = torch.tensor(inputs.random_traces(nf, Nf, 4), device="cuda")
    y = torch.empty_like(x)
    assert _call(lib, dim, k, ne, nf, S, ef, fs, fb, x, y, stream, err) == 0, err.value
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(3):
        assert _call(lib, dim, k, ne, nf, S, ef, fs, fb, x, y, stream, err) == 0, err.value
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0 and torch.cuda.memory_allocated() == alloc0
    # plain torch reference: boundary entries of x read as zero, y zero on boundary faces
    interior = torch.tensor(fb_np < 0, device="cuda")
    xi = torch.where(interior[:, None], x, torch.zeros_like(x))
    xl = xi[ef.long()].reshape(ne, m)
    z = torch.bmm(S, xl[:, :, None])[:, :, 0].reshape(ne * (dim + 1), Nf)
    y_ref = torch.zeros_like(x).index_add_(0, ef.long().reshape(-1), z)
    y_ref[~interior] = 0.0
    assert (y - y_ref).abs().max().item() <= 1e-12 * y_ref.abs().max().item()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_1807_00086_gb300 import hdg
    lib = hdg.load()
    err = ctypes.create_string_buffer(256)
    dummy = ctypes.c_void_p(16)               # never dereferenced: the size check comes first
    st = lib.hdg_trace_apply_noalloc(3, 3, 30000, 60000, dummy, dummy, dummy, dummy, dummy, dummy, None, err, 256)
    assert st == -1 and b"exceeds the fixed scratch" in err.value
