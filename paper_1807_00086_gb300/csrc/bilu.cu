// Block ILU(0) preconditioner of the GMRES trace solve (Sec. 2.4): the block pattern, the
// contributions of the element blocks S_K to each assembled block, the update lists of the
// factorisation and the level sets of the two block substitutions (host, once per mesh); the
// assembly and factorisation after every condensation, and the substitutions as one captured
// CUDA graph (one kernel node per level) applied to fixed buffers.
#include <algorithm>
#include <cstring>

#include "ctx.cuh"
#include "bilu.cuh"

using namespace hdg;

struct Bilu {
  int nr = 0;
  int64_t nnzb = 0;
  int32_t *d_rowface = nullptr, *d_rptr = nullptr, *d_col = nullptr, *d_dpos = nullptr, *d_uptr = nullptr;
  int32_t* d_ce = nullptr;
  int8_t *d_ca = nullptr, *d_cb = nullptr;
  int2* d_upd = nullptr;
  double *d_val = nullptr, *d_dinv = nullptr;
  int32_t *d_frows = nullptr, *d_brows = nullptr;
  std::vector<int> flev, blev;              // level pointers into the row lists
  double *d_pin = nullptr, *d_pmid = nullptr, *d_pout = nullptr;
  cudaGraphExec_t solve = nullptr;
  int* d_err = nullptr;
  int* h_err = nullptr;
  BiluDev dev{};
  bool factored = false;
};

namespace {

size_t factor_smem(int Nf) { return sizeof(double) * 4 * 3 * (size_t)Nf * Nf; }

// rows grouped by level (level-major, increasing row within a level)
void group_levels(const std::vector<int>& lev, std::vector<int32_t>& rows, std::vector<int>& ptr) {
  const int nl = lev.empty() ? 0 : *std::max_element(lev.begin(), lev.end()) + 1;
  ptr.assign((size_t)nl + 1, 0);
  for (int l : lev) ptr[(size_t)l + 1] += 1;
  for (int i = 0; i < nl; ++i) ptr[i + 1] += ptr[i];
  rows.assign(lev.size(), 0);
  std::vector<int> fill(ptr.begin(), ptr.end() - 1);
  for (size_t r = 0; r < lev.size(); ++r) rows[fill[lev[r]]++] = (int32_t)r;
}

}  // namespace

hdg_status bilu_setup(hdg_ctx* c) {
  Bilu* b = new (std::nothrow) Bilu();
  if (!b) return fail(c, HDG_ENOMEM, "out of host memory");
  c->bilu = b;
  const int64_t ne = c->sk.ne, nf = c->sk.nf;
  const int nc = c->nfc, Nf = c->Nf;
  if (Nf > 32) return fail(c, HDG_EINVAL, "block ILU(0): at most 32 trace entries per face");
  std::vector<int32_t> rowof((size_t)nf, -1), rowface;
  for (int64_t f = 0; f < nf; ++f)
    if (c->sk.face_bnd[f] < 0) { rowof[f] = (int32_t)rowface.size(); rowface.push_back((int32_t)f); }
  const int nr = (int)rowface.size();
  b->nr = nr;
  // per row: (column row, element, local face of the row, local face of the column)
  struct Ent { int32_t col, e; int8_t a, bb; };
  std::vector<std::vector<Ent>> nbr((size_t)nr);
  for (int64_t e = 0; e < ne; ++e)
    for (int a = 0; a < nc; ++a) {
      const int32_t ra = rowof[c->sk.elem_face[e * nc + a]];
      if (ra < 0) continue;
      for (int bb = 0; bb < nc; ++bb) {
        const int32_t rb = rowof[c->sk.elem_face[e * nc + bb]];
        if (rb >= 0) nbr[ra].push_back(Ent{rb, (int32_t)e, (int8_t)a, (int8_t)bb});
      }
    }
  std::vector<int32_t> rptr((size_t)nr + 1, 0), col, dpos((size_t)nr), ce;
  std::vector<int8_t> ca, cb;
  for (int r = 0; r < nr; ++r) {
    auto& v = nbr[r];
    std::sort(v.begin(), v.end(), [](const Ent& x, const Ent& y) { return x.col != y.col ? x.col < y.col : x.e < y.e; });
    for (size_t i = 0; i < v.size();) {
      size_t j = i;
      const int32_t cl = v[i].col;
      if (cl == r) dpos[r] = (int32_t)col.size();
      col.push_back(cl);
      for (int s = 0; s < 2; ++s) {
        if (j < v.size() && v[j].col == cl) {
          ce.push_back(v[j].e); ca.push_back(v[j].a); cb.push_back(v[j].bb);
          ++j;
        } else {
          ce.push_back(-1); ca.push_back(0); cb.push_back(0);
        }
      }
      if (j < v.size() && v[j].col == cl) return fail(c, HDG_EINVAL, "block ILU(0): a face block with three elements");
      i = j;
    }
    rptr[r + 1] = (int32_t)col.size();
  }
  const int64_t nnzb = (int64_t)col.size();
  b->nnzb = nnzb;
  // updates of the factorisation: for lower block p = (r, k), every block q = (k, j), j > k,
  // whose column j is also in row r, at position t
  std::vector<int32_t> uptr((size_t)nnzb + 1, 0);
  std::vector<int2> upd;
  for (int r = 0; r < nr; ++r)
    for (int p = rptr[r]; p < rptr[r + 1]; ++p) {
      const int k = col[p];
      if (k < r)
        for (int q = dpos[k] + 1; q < rptr[k + 1]; ++q) {
          const int j = col[q];
          const auto it = std::lower_bound(col.begin() + rptr[r], col.begin() + rptr[r + 1], j);
          if (it != col.begin() + rptr[r + 1] && *it == j) upd.push_back(make_int2(q, (int)(it - col.begin())));
        }
      uptr[(size_t)p + 1] = (int32_t)upd.size();
    }
  // level sets: forward (lower neighbours first), backward (upper neighbours first)
  std::vector<int> lf((size_t)nr, 0), lb((size_t)nr, 0);
  for (int r = 0; r < nr; ++r)
    for (int p = rptr[r]; p < dpos[r]; ++p) lf[r] = std::max(lf[r], lf[col[p]] + 1);
  for (int r = nr - 1; r >= 0; --r)
    for (int p = dpos[r] + 1; p < rptr[r + 1]; ++p) lb[r] = std::max(lb[r], lb[col[p]] + 1);
  std::vector<int32_t> frows, brows;
  group_levels(lf, frows, b->flev);
  group_levels(lb, brows, b->blev);
  hdg_status s;
  const size_t nfe = (size_t)nf * Nf, nb2 = (size_t)Nf * Nf;
  if ((s = dalloc(c, &b->d_rowface, std::max(nr, 1)))) return s;
  if ((s = dalloc(c, &b->d_rptr, rptr.size()))) return s;
  if ((s = dalloc(c, &b->d_col, col.size()))) return s;
  if ((s = dalloc(c, &b->d_dpos, std::max(nr, 1)))) return s;
  if ((s = dalloc(c, &b->d_uptr, uptr.size()))) return s;
  if ((s = dalloc(c, &b->d_upd, std::max<size_t>(upd.size(), 1)))) return s;
  if ((s = dalloc(c, &b->d_ce, ce.size()))) return s;
  if ((s = dalloc(c, &b->d_ca, ca.size()))) return s;
  if ((s = dalloc(c, &b->d_cb, cb.size()))) return s;
  if ((s = dalloc(c, &b->d_val, (size_t)nnzb * nb2))) return s;
  if ((s = dalloc(c, &b->d_dinv, (size_t)std::max(nr, 1) * nb2))) return s;
  if ((s = dalloc(c, &b->d_frows, std::max(nr, 1)))) return s;
  if ((s = dalloc(c, &b->d_brows, std::max(nr, 1)))) return s;
  for (double** p : {&b->d_pin, &b->d_pmid, &b->d_pout}) {
    if ((s = dalloc(c, p, nfe))) return s;
    CUDA_TRY(c, cudaMemsetAsync(*p, 0, nfe * 8, c->stream));
  }
  if ((s = dalloc(c, &b->d_err, 1))) return s;
  CUDA_TRY(c, cudaMallocHost((void**)&b->h_err, sizeof(int)));
  CUDA_TRY(c, cudaMemsetAsync(b->d_err, 0, sizeof(int), c->stream));
  auto up = [&](void* d, const void* h, size_t bytes) -> hdg_status {
    if (bytes) CUDA_TRY(c, cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, c->stream));
    return HDG_OK;
  };
  if ((s = up(b->d_rowface, rowface.data(), rowface.size() * 4))) return s;
  if ((s = up(b->d_rptr, rptr.data(), rptr.size() * 4))) return s;
  if ((s = up(b->d_col, col.data(), col.size() * 4))) return s;
  if ((s = up(b->d_dpos, dpos.data(), dpos.size() * 4))) return s;
  if ((s = up(b->d_uptr, uptr.data(), uptr.size() * 4))) return s;
  if ((s = up(b->d_upd, upd.data(), upd.size() * sizeof(int2)))) return s;
  if ((s = up(b->d_ce, ce.data(), ce.size() * 4))) return s;
  if ((s = up(b->d_ca, ca.data(), ca.size()))) return s;
  if ((s = up(b->d_cb, cb.data(), cb.size()))) return s;
  if ((s = up(b->d_frows, frows.data(), frows.size() * 4))) return s;
  if ((s = up(b->d_brows, brows.data(), brows.size() * 4))) return s;
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));   // the host vectors are released at return
  b->dev = BiluDev{Nf, b->d_rowface, b->d_rptr, b->d_col, b->d_dpos, b->d_uptr, b->d_upd, b->d_val, b->d_dinv};
  if (factor_smem(Nf) > 48 * 1024)
    CUDA_TRY(c, cudaFuncSetAttribute(bilu_factor_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)factor_smem(Nf)));
  return HDG_OK;
}

// assembled sgn K on the block pattern, then ILU(0) level by level
hdg_status bilu_factor(hdg_ctx* c) {
  Bilu* b = c->bilu;
  const int Nf = c->Nf;
  c->n_launch += 1;
  bilu_assemble_kernel<<<grid_for(c, b->nnzb * Nf * Nf), 256, 0, c->stream>>>(b->nnzb, Nf, c->m, b->d_ce, b->d_ca,
                                                                               b->d_cb, c->d_S, c->sgn, b->d_val);
  CUDA_TRY(c, cudaMemsetAsync(b->d_err, 0, sizeof(int), c->stream));
  for (size_t l = 0; l + 1 < b->flev.size(); ++l) {
    const int n = b->flev[l + 1] - b->flev[l];
    c->n_launch += 1;
    bilu_factor_kernel<<<(n + 3) / 4, 128, factor_smem(Nf), c->stream>>>(b->dev, b->d_frows + b->flev[l], n, b->d_err);
  }
  hdg_status s = check_launch(c, "bilu_factor");
  if (s) return s;
  CUDA_TRY(c, cudaMemcpyAsync(b->h_err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (*b->h_err) return fail(c, HDG_EINVAL, "block ILU(0): a zero pivot in a diagonal block");
  b->factored = true;
  return HDG_OK;
}

// out = M^{-1} in through the fixed buffers and the captured substitutions
hdg_status bilu_apply(hdg_ctx* c, const double* in, double* out) {
  Bilu* b = c->bilu;
  if (!b->factored) return fail(c, HDG_ESTATE, "block ILU(0): not factored (hdg_condense has not run)");
  const size_t nfe = (size_t)c->sk.nf * c->Nf;
  if (!b->solve) {
    if (!c->cap_stream) CUDA_TRY(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    cudaGraph_t G = nullptr;
    CUDA_TRY(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    for (size_t l = 0; l + 1 < b->flev.size(); ++l) {
      const int n = b->flev[l + 1] - b->flev[l];
      bilu_fwd_kernel<<<(n + 3) / 4, 128, 0, c->cap_stream>>>(b->dev, b->d_frows + b->flev[l], n, b->d_pin, b->d_pmid);
    }
    for (size_t l = 0; l + 1 < b->blev.size(); ++l) {
      const int n = b->blev[l + 1] - b->blev[l];
      bilu_bwd_kernel<<<(n + 3) / 4, 128, 0, c->cap_stream>>>(b->dev, b->d_brows + b->blev[l], n, b->d_pmid, b->d_pout);
    }
    cudaError_t e = cudaStreamEndCapture(c->cap_stream, &G);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->solve, G, 0);
    if (G) cudaGraphDestroy(G);
    if (e != cudaSuccess) return fail(c, HDG_ECUDA, std::string("block ILU(0) solve graph: ") + cudaGetErrorString(e));
  }
  if (in != b->d_pin) CUDA_TRY(c, cudaMemcpyAsync(b->d_pin, in, nfe * 8, cudaMemcpyDeviceToDevice, c->stream));
  CUDA_TRY(c, cudaGraphLaunch(b->solve, c->stream));
  c->n_launch += (int64_t)(b->flev.size() + b->blev.size() - 2);
  if (out != b->d_pout) CUDA_TRY(c, cudaMemcpyAsync(out, b->d_pout, nfe * 8, cudaMemcpyDeviceToDevice, c->stream));
  return HDG_OK;
}

void bilu_destroy(hdg_ctx* c) {
  Bilu* b = c->bilu;
  if (!b) return;
  if (b->solve) cudaGraphExecDestroy(b->solve);
  if (b->h_err) cudaFreeHost(b->h_err);
  delete b;
  c->bilu = nullptr;
}
