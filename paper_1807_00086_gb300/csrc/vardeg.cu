// Variable-degree elastodynamics (per-element k_K in 1..4, face degree k_F = max over the
// face's elements; 3D): setup of the compact index maps, condensation by classes
// (K, KT), the element-local solves, the generic matrix-free apply and the Krylov solves
// (FP64 CG, or FP32 inner PCG inside FP64 iterative refinement). The steps are those of
// Sec. 2.3-2.4 with the spaces of Sec. 2.2 chosen per element.
#include <cmath>
#include <cstring>
#include <map>

#include "ctx.cuh"
#include "vardeg.cuh"

using namespace hdg;

struct VarDeg {
  struct Cls {
    int K = 0, KT = 0;
    int64_t first = 0, count = 0;   // range in the grouped element list
    Tabs tabs{};
  };
  std::vector<Cls> cls;
  int32_t* d_elist = nullptr;
  int64_t *d_u_off = nullptr, *d_h_off = nullptr, *d_s_off = nullptr, *d_sdiag = nullptr;
  int32_t *d_m_off = nullptr, *d_gidx = nullptr, *d_gint = nullptr, *d_dslot = nullptr;
  int16_t* d_pidx = nullptr;
  double* d_tab = nullptr;
  double* d_scr = nullptr;
  int64_t scr_blocks = 0;
  int64_t m_tot = 0, s_tot = 0, h_tot = 0;
  float* d_S32 = nullptr;
  float* d_S32lo = nullptr;       // remainder of S_K beyond its FP32 copy (double-float residual apply)
  __half* d_S16 = nullptr;        // FP16 copy (HDG_MIXED16 inner operator) and its per-element scales
  float* d_sc16 = nullptr;
  // per-degree volume rules (initial-data projection) and per-element degree / point offsets
  std::vector<RefTables> rule;        // index k = 1..4
  std::vector<int32_t> ek;
  std::vector<int64_t> q_off;
  int32_t* d_ek = nullptr;
  int64_t* d_q_off = nullptr;
  double* d_qtab = nullptr;
  VdQuad quad{};
  // one-launch local solves and the autotuned tiles
  VdClassTable table{};
  size_t local_smem = 0;
  int tile32 = -1, tile64 = -1, tiledf = -1, tile16 = -1;   // index into kApplyTiles (-1: not tuned yet)
  int local_nth[2] = {0, 0};      // threads per element of the MODE 0 / MODE 1 launch (0: not tuned)
};

namespace {

constexpr int VD_MMAX = 180;      // 4 faces x 3 components x 15 modes (degree 4)
constexpr int64_t VD_CHUNK = 2048; // elements per condensation launch of a large class

int n_modes_h(int dim, int k) {
  int r = 1;
  for (int i = 1; i <= dim; ++i) r = r * (k + i) / i;
  return r;
}

VdIndex vd_index(const hdg_ctx* c, const VarDeg::Cls& k) {
  const VarDeg* v = c->vd;
  return VdIndex{v->d_elist + k.first, v->d_u_off, v->d_h_off, v->d_s_off, v->d_m_off, v->d_gidx, v->d_pidx};
}

#define VD_DISPATCH(KK, KKT, FN, ...)                  \
  switch ((KK) * 10 + (KKT)) {                         \
    case 11: FN<1, 1>(__VA_ARGS__); break;             \
    case 12: FN<1, 2>(__VA_ARGS__); break;             \
    case 13: FN<1, 3>(__VA_ARGS__); break;             \
    case 14: FN<1, 4>(__VA_ARGS__); break;             \
    case 22: FN<2, 2>(__VA_ARGS__); break;             \
    case 23: FN<2, 3>(__VA_ARGS__); break;             \
    case 24: FN<2, 4>(__VA_ARGS__); break;             \
    case 33: FN<3, 3>(__VA_ARGS__); break;             \
    case 34: FN<3, 4>(__VA_ARGS__); break;             \
    case 44: FN<4, 4>(__VA_ARGS__); break;             \
    default: break;                                    \
  }

template <int K, int KT>
void vd_local_smem(size_t& s) {
  s = std::max(s, sizeof(double) * (size_t)LocalVdSmem<3, K, KT>::TOTAL);
}

template <int K, int KT>
void vd_launch_condense(hdg_ctx* c, const VarDeg::Cls& k) {
  using C = CondVdCfg<3, K, KT>;
  cudaFuncSetAttribute(condense_vd_kernel<3, K, KT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
  VdIndex X = vd_index(c, k);
  const int64_t step = C::GH ? VD_CHUNK : k.count;
  for (int64_t s = 0; s < k.count; s += step) {
    const int64_t n = std::min(step, k.count - s);
    VdIndex Xs = X;
    Xs.elist = X.elist + s;
    c->n_launch += 1;
    condense_vd_kernel<3, K, KT><<<(unsigned)n, 256, C::SMEM, c->stream>>>(devmesh(c), k.tabs, c->d_lame, c->d_mue,
                                                                           c->alpha, Xs, c->d_S, c->d_Hinv,
                                                                           c->vd->d_scr, c->d_err);
  }
}

constexpr int kApplyTiles[6][2] = {{4, 4}, {4, 8}, {4, 16}, {8, 4}, {8, 8}, {8, 16}};   // (warps, unroll)
constexpr int kLocalThreads[3] = {64, 128, 256};

template <typename TV, typename ST, int WPB, int UNR>
void vd_apply_tile(hdg_ctx* c, const ST* S, const float* sc, const TV* x, TV* slot, const int* done) {
  apply_vd_kernel<TV, ST, VD_MMAX, WPB, UNR><<<(unsigned)((c->sk.ne + WPB - 1) / WPB), 32 * WPB, 0, c->stream>>>(
      c->sk.ne, c->vd->d_s_off, c->vd->d_m_off, c->vd->d_gint, S, sc, x, slot, done);
}

template <typename TV, typename ST = TV>
void vd_apply_variant(hdg_ctx* c, int tile, const ST* S, const TV* x, TV* slot, const int* done,
                      const float* sc = nullptr) {
  switch (tile) {
    case 0: vd_apply_tile<TV, ST, 4, 4>(c, S, sc, x, slot, done); break;
    case 1: vd_apply_tile<TV, ST, 4, 8>(c, S, sc, x, slot, done); break;
    case 2: vd_apply_tile<TV, ST, 4, 16>(c, S, sc, x, slot, done); break;
    case 3: vd_apply_tile<TV, ST, 8, 4>(c, S, sc, x, slot, done); break;
    case 4: vd_apply_tile<TV, ST, 8, 8>(c, S, sc, x, slot, done); break;
    default: vd_apply_tile<TV, ST, 8, 16>(c, S, sc, x, slot, done); break;
  }
}

template <int WPB, int UNR>
void vd_apply_df_tile(hdg_ctx* c, const double* x, double* slot) {
  apply_vd_df_kernel<VD_MMAX, WPB, UNR><<<(unsigned)((c->sk.ne + WPB - 1) / WPB), 32 * WPB, 0, c->stream>>>(
      c->sk.ne, c->vd->d_s_off, c->vd->d_m_off, c->vd->d_gint, c->vd->d_S32, c->vd->d_S32lo, x, slot);
}

void vd_apply_df_variant(hdg_ctx* c, int tile, const double* x, double* slot) {
  switch (tile) {
    case 0: vd_apply_df_tile<4, 4>(c, x, slot); break;
    case 1: vd_apply_df_tile<4, 8>(c, x, slot); break;
    case 2: vd_apply_df_tile<4, 16>(c, x, slot); break;
    case 3: vd_apply_df_tile<8, 4>(c, x, slot); break;
    case 4: vd_apply_df_tile<8, 8>(c, x, slot); break;
    default: vd_apply_df_tile<8, 16>(c, x, slot); break;
  }
}

// Autotuner: times every candidate tile (run(t) launches candidate t) on the context's own
// operator (the slot output is a workspace that the next use overwrites) and keeps the
// fastest: 3 timed launches per candidate, two interleaved passes, best of the two.
template <typename RUN>
int vd_tune(hdg_ctx* c, RUN run) {
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess) return 1;
  if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return 1; }
  // two interleaved passes, best time per candidate: a single pass right after the
  // condensation is skewed by the clock and cache state of the first candidates
  float tmin[6];
  for (int t = 0; t < 6; ++t) tmin[t] = 1e30f;
  run(0);
  for (int pass = 0; pass < 2; ++pass)
    for (int t = 0; t < 6; ++t) {
      cudaEventRecord(a, c->stream);
      for (int r = 0; r < 3; ++r) run(t);
      cudaEventRecord(b, c->stream);
      float ms = 0.f;
      if (cudaEventSynchronize(b) == cudaSuccess && cudaEventElapsedTime(&ms, a, b) == cudaSuccess)
        tmin[t] = std::min(tmin[t], ms);
    }
  int best = 1;
  for (int t = 0; t < 6; ++t)
    if (tmin[t] < tmin[best]) best = t;
  c->n_launch += 37;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return best;
}

template <int MODE>
void vd_local_launch(hdg_ctx* c, int nth, const double* F, const double* hist, const double* lam, double* out) {
  const VarDeg* v = c->vd;
  const VdIndex X{v->d_elist, v->d_u_off, v->d_h_off, v->d_s_off, v->d_m_off, v->d_gidx, v->d_pidx};
  const unsigned grid = (unsigned)c->sk.ne;
  c->n_launch += 1;
  if (nth == 64)
    local_vd_all_kernel<MODE, 64><<<grid, 64, v->local_smem, c->stream>>>(devmesh(c), v->table, c->d_lame, c->d_mue,
                                                                          c->d_Hinv, c->alpha, X, F, hist, lam, out);
  else if (nth == 128)
    local_vd_all_kernel<MODE, 128><<<grid, 128, v->local_smem, c->stream>>>(devmesh(c), v->table, c->d_lame, c->d_mue,
                                                                            c->d_Hinv, c->alpha, X, F, hist, lam, out);
  else
    local_vd_all_kernel<MODE, 256><<<grid, 256, v->local_smem, c->stream>>>(devmesh(c), v->table, c->d_lame, c->d_mue,
                                                                            c->d_Hinv, c->alpha, X, F, hist, lam, out);
}

// The element-local solves of every class in one launch. The first call of each mode times
// the block sizes on the live inputs (each candidate writes the same output) and keeps the
// fastest.
void vd_local(hdg_ctx* c, int mode, const double* F, const double* hist, const double* lam, double* out) {
  VarDeg* v = c->vd;
  auto run = [&](int nth) {
    if (mode == 0) vd_local_launch<0>(c, nth, F, hist, lam, out);
    else vd_local_launch<1>(c, nth, F, hist, lam, out);
  };
  if (v->local_nth[mode] == 0) {
    cudaEvent_t a, b;
    int best = 128;
    float best_ms = 1e30f;
    if (cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess) {
      run(kLocalThreads[0]);   // untimed first launch
      for (int pass = 0; pass < 2; ++pass)
        for (int nth : kLocalThreads) {
          cudaEventRecord(a, c->stream);
          run(nth);
          cudaEventRecord(b, c->stream);
          float ms = 0.f;
          if (cudaEventSynchronize(b) == cudaSuccess && cudaEventElapsedTime(&ms, a, b) == cudaSuccess && ms < best_ms) {
            best_ms = ms;
            best = nth;
          }
        }
      cudaEventDestroy(a);
      cudaEventDestroy(b);
    }
    v->local_nth[mode] = best;
  }
  run(v->local_nth[mode]);
}

void vd_apply64(hdg_ctx* c, const double* x, double* slot, const int* done, int iter) {
  c->n_launch += 1;
  cudaEvent_t stop = apply_begin(c, 0, iter);
  vd_apply_variant<double>(c, c->vd->tile64 < 0 ? 1 : c->vd->tile64, c->d_S, x, slot, done);
  apply_end(c, stop);
}

// FP64-accurate residual apply of the mixed path (double-float on the FP32 pipe)
void vd_apply_df(hdg_ctx* c, const double* x, double* slot) {
  c->n_launch += 1;
  cudaEvent_t stop = apply_begin(c, 2, -1);
  vd_apply_df_variant(c, c->vd->tiledf < 0 ? 1 : c->vd->tiledf, x, slot);
  apply_end(c, stop);
}

void vd_apply32(hdg_ctx* c, const float* x, float* slot, const int* done, int iter) {
  c->n_launch += 1;
  cudaEvent_t stop = apply_begin(c, 1, iter);
  vd_apply_variant<float>(c, c->vd->tile32 < 0 ? 1 : c->vd->tile32, c->vd->d_S32, x, slot, done);
  apply_end(c, stop);
}

void vd_apply16(hdg_ctx* c, const float* x, float* slot, const int* done, int iter) {
  c->n_launch += 1;
  cudaEvent_t stop = apply_begin(c, 3, iter);
  vd_apply_variant<float, __half>(c, c->vd->tile16 < 0 ? 1 : c->vd->tile16, c->vd->d_S16, x, slot, done,
                                  c->vd->d_sc16);
  apply_end(c, stop);
}

hdg_status vd_gather(hdg_ctx* c, const double* slot, double scale, double* out) {
  c->n_launch += 1;
  vd_face_gather_kernel<<<grid_for(c, c->ntr), 256, 0, c->stream>>>(c->ntr, c->vd->d_dslot, slot, scale, out);
  return check_launch(c, "vd_face_gather");
}

// PCG on (sgn K) x = bvec over interior trace entries (FP64).
hdg_status vd_cg(hdg_ctx* c, const double* bvec, double* x, hdg_solve_info* info) {
  const int64_t n = c->ntr;
  const int nb = c->nb_red;
  vd_apply64(c, x, c->d_slot, nullptr, -1);
  c->n_launch += 2;
  vd_cg_init_kernel<<<nb, 256, 0, c->stream>>>(n, c->sgn, c->vd->d_dslot, c->d_slot, bvec, c->d_dinv, c->d_r, c->d_z,
                                               c->d_p, c->d_part);
  cg_init_scalars<<<1, 256, 0, c->stream>>>(nb, c->d_part, c->opt.rtol, c->d_sc);
  hdg_status s = check_launch(c, "vd_cg_init");
  if (s) return s;
  CUDA_TRY(c, cudaMemcpyAsync(c->h_sc, c->d_sc, sizeof(CgScal), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (c->h_sc->bb == 0.0) {
    c->n_launch += 1;
    vd_zero_interior_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(n, c->vd->d_dslot, x);
    if (info) { info->rel_residual = 0.0; info->sweeps += 1; }
    return check_launch(c, "vd_zero_interior");
  }
  int it = 0;
  const int maxit = c->opt.maxit;
  const int chk = std::max(1, c->opt.check_every);
  while (!c->h_sc->done && it < maxit) {
    const int upto = std::min(maxit, it + chk);
    for (; it < upto; ++it) {
      const int par = it & 1;
      vd_apply64(c, c->d_p, c->d_slot, &c->d_sc->done, it);
      c->n_launch += 3;
      vd_face_q_kernel<double><<<nb, 256, 0, c->stream>>>(n, c->sgn, c->vd->d_dslot, c->d_slot, c->d_p, c->d_q,
                                                          c->d_part, c->d_sc);
      cg_update_kernel<<<nb, 256, 0, c->stream>>>(n, nb, par, c->d_part, c->d_p, c->d_q, c->d_dinv, x, c->d_r, c->d_z,
                                                  c->d_part + nb, c->d_sc);
      cg_direction_kernel<<<nb, 256, 0, c->stream>>>(n, nb, par, it, c->d_part + nb, c->d_z, c->d_p, c->d_sc, maxit, 0);
    }
    if ((s = check_launch(c, "vd_cg_iter"))) return s;
    CUDA_TRY(c, cudaMemcpyAsync(c->h_sc, c->d_sc, sizeof(CgScal), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    harvest(c, c->h_sc->done ? c->h_sc->iters : (1 << 30));
  }
  const CgScal sc = *c->h_sc;
  const double rel = sc.bb > 0 ? std::sqrt(sc.rr / sc.bb) : 0.0;
  if (info) { info->iterations += sc.iters; info->sweeps += 1; info->rel_residual = rel; }
  if (sc.done != 1) return fail(c, HDG_ENOCONV, "Krylov solve reached maxit with relative residual " + std::to_string(rel));
  return HDG_OK;
}

// FP32 PCG on (sgn K32) x32 = b32 from x32 = 0 (inner solve of the refinement).
hdg_status vd_cg32(hdg_ctx* c, double tol, int* iters, bool use16) {
  const int64_t n = c->ntr;
  const int nb = c->nb_red;
  const int64_t n4 = c->nfe4 / 4;
  c->n_launch += 2;
  cg32_init_kernel<<<nb, 256, 0, c->stream>>>(n4, (const float4*)c->d_b32, (const float4*)c->d_dinv32, (float4*)c->d_x32,
                                              (float4*)c->d_r32, (float4*)c->d_z32, (float4*)c->d_p32, c->d_part);
  cg32_init_scalars<<<1, 256, 0, c->stream>>>(nb, c->d_part, tol, c->d_sc, nullptr);
  hdg_status s = check_launch(c, "vd_cg32_init");
  if (s) return s;
  int it = 0;
  const int maxit = c->opt.maxit;
  const int chk = std::max(1, c->opt.check_every);
  c->h_sc->done = 0;
  while (!c->h_sc->done && it < maxit) {
    const int upto = std::min(maxit, it + chk);
    for (; it < upto; ++it) {
      const int par = it & 1;
      if (use16) vd_apply16(c, c->d_p32, c->d_slot32, &c->d_sc->done, it);
      else vd_apply32(c, c->d_p32, c->d_slot32, &c->d_sc->done, it);
      c->n_launch += 3;
      vd_face_q_kernel<float><<<nb, 256, 0, c->stream>>>(n, (float)c->sgn, c->vd->d_dslot, c->d_slot32, c->d_p32,
                                                         c->d_q32, c->d_part, c->d_sc);
      cg32_update_kernel<<<nb, 256, 0, c->stream>>>(n4, nb, par, c->d_part, (const float4*)c->d_p32,
                                                    (const float4*)c->d_q32, (const float4*)c->d_dinv32,
                                                    (float4*)c->d_x32, (float4*)c->d_r32, (float4*)c->d_z32,
                                                    c->d_part + nb, c->d_sc);
      cg32_direction_kernel<<<nb, 256, 0, c->stream>>>(n4, nb, par, it, c->d_part + nb, (const float4*)c->d_z32,
                                                       (float4*)c->d_p32, c->d_sc, maxit, 0);
    }
    if ((s = check_launch(c, "vd_cg32_iter"))) return s;
    CUDA_TRY(c, cudaMemcpyAsync(c->h_sc, c->d_sc, sizeof(CgScal), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    harvest(c, c->h_sc->done ? c->h_sc->iters : (1 << 30));
  }
  *iters = c->h_sc->iters;
  return HDG_OK;
}

// FP64 iterative refinement: FP64 residual with the FP64 S_K, FP32 correction solves.
hdg_status vd_refine(hdg_ctx* c, const double* bvec, double* x, hdg_solve_info* info) {
  const int64_t n = c->ntr;
  const int nb = c->nb_red;
  int total_it = 0;
  double rel = 0.0, rel_prev = 0.0;
  hdg_status s;
  bool use16 = c->vd->d_S16 != nullptr;   // FP16 inner operator until a sweep contracts poorly
  for (int sweep = 0;; ++sweep) {
    vd_apply_df(c, x, c->d_slot);
    c->n_launch += 2;
    vd_refine_residual_kernel<<<nb, 256, 0, c->stream>>>(n, c->sgn, c->vd->d_dslot, c->d_slot, bvec, c->d_res,
                                                         c->d_part);
    refine_scalars<<<1, 256, 0, c->stream>>>(nb, c->d_part, c->d_rs);
    if ((s = check_launch(c, "vd_refine_residual"))) return s;
    CUDA_TRY(c, cudaMemcpyAsync(c->h_rs, c->d_rs, sizeof(RefScal), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    harvest(c);
    const RefScal r = *c->h_rs;
    if (r.bb == 0.0) {
      c->n_launch += 1;
      vd_zero_interior_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(n, c->vd->d_dslot, x);
      if (info) { info->rel_residual = 0.0; info->sweeps += sweep; }
      return check_launch(c, "vd_zero_interior");
    }
    rel_prev = rel;
    rel = std::sqrt(r.rr / r.bb);
    // a sweep that gained less than 10x with the FP16 operator hands the rest to the FP32 copy
    if (use16 && sweep > 0 && rel > 0.1 * rel_prev) use16 = false;
    if (rel <= c->opt.rtol) {
      if (info) { info->iterations += total_it; info->sweeps += sweep; info->rel_residual = rel; }
      return HDG_OK;
    }
    if (sweep >= c->opt.max_sweeps) break;
    c->n_launch += 1;
    to32_scaled_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(n, c->d_res, c->d_rs, c->d_b32);
    const double tol = std::min(0.5, std::max(c->opt.inner_rtol, 0.25 * c->opt.rtol / rel));
    int it = 0;
    if ((s = vd_cg32(c, tol, &it, use16))) return s;
    total_it += it;
    c->n_launch += 1;
    vd_refine_update_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(n, c->vd->d_dslot, c->d_x32, c->d_rs, x);
    if ((s = check_launch(c, "vd_refine_update"))) return s;
  }
  if (info) { info->iterations += total_it; info->sweeps += c->opt.max_sweeps; info->rel_residual = rel; }
  return fail(c, HDG_ENOCONV, "mixed-precision refinement reached max_sweeps=" + std::to_string(c->opt.max_sweeps) +
                                  " with relative residual " + std::to_string(rel));
}

// ---- device-driven solves (one graph launch per trace solve; see devloop.cuh)
// Appends the solve of (sgn K) x = bvec to G after deps (deps: the solve's last nodes on return);
// dg, if given, receives the launch counts (outside the loops, per sweep body, per inner trip).
void vd_build_solve(hdg_ctx* c, GraphBuild& gb, cudaGraph_t G, std::vector<cudaGraphNode_t>& deps, const double* bvec,
                    double* x, hdg_ctx::DevGraph* dg) {
  const int64_t n = c->ntr;
  const int nb = c->nb_red, maxit = c->opt.maxit;
  std::vector<cudaGraphNode_t> bd, d16, d32;
  if (c->opt.prec == HDG_FP64) {
    const int64_t n0 = c->n_launch;
    gb.seq(G, deps, [&] {
      vd_apply64(c, x, c->d_slot, nullptr, -1);
      c->n_launch += 2;
      vd_cg_init_kernel<<<nb, 256, 0, c->stream>>>(n, c->sgn, c->vd->d_dslot, c->d_slot, bvec, c->d_dinv, c->d_r, c->d_z,
                                                   c->d_p, c->d_part);
      cg_init_scalars<<<1, 256, 0, c->stream>>>(nb, c->d_part, c->opt.rtol, c->d_sc);
    });
    const cudaGraphConditionalHandle h = gb.handle(G, 1, true);
    cudaGraph_t B = gb.loop(G, deps, h);
    const int64_t n1 = c->n_launch;
    gb.seq(B, bd, [&] {
      for (int par = 0; par < 2; ++par) {
        vd_apply64(c, c->d_p, c->d_slot, &c->d_sc->done, -1);
        c->n_launch += 3;
        vd_face_q_kernel<double><<<nb, 256, 0, c->stream>>>(n, c->sgn, c->vd->d_dslot, c->d_slot, c->d_p, c->d_q,
                                                            c->d_part, c->d_sc);
        cg_update_kernel<<<nb, 256, 0, c->stream>>>(n, nb, par, c->d_part, c->d_p, c->d_q, c->d_dinv, x, c->d_r, c->d_z,
                                                    c->d_part + nb, c->d_sc);
        cg_direction_kernel<<<nb, 256, 0, c->stream>>>(n, nb, par, -1, c->d_part + nb, c->d_z, c->d_p, c->d_sc, maxit, h);
      }
    });
    const int64_t n2 = c->n_launch;
    gb.seq(G, deps, [&] {
      c->n_launch += 2;
      cg_ctl_finish_kernel<<<1, 32, 0, c->stream>>>(c->d_sc, c->d_lc);
      zero_masked_if_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(n, c->d_intmask, c->d_lc, x);
    });
    if (dg) {
      dg->n_static = (n1 - n0) + (c->n_launch - n2);
      dg->n_body = 0;
      dg->n_trip = n2 - n1;
    }
    return;
  }
  const int64_t n4 = c->nfe4 / 4;
  const bool has16 = c->vd->d_S16 != nullptr;
  auto inner = [&](bool use16, cudaGraphConditionalHandle h) {
    for (int par = 0; par < 2; ++par) {
      if (use16) vd_apply16(c, c->d_p32, c->d_slot32, &c->d_sc->done, -1);
      else vd_apply32(c, c->d_p32, c->d_slot32, &c->d_sc->done, -1);
      c->n_launch += 3;
      vd_face_q_kernel<float><<<nb, 256, 0, c->stream>>>(n, (float)c->sgn, c->vd->d_dslot, c->d_slot32, c->d_p32,
                                                         c->d_q32, c->d_part, c->d_sc);
      cg32_update_kernel<<<nb, 256, 0, c->stream>>>(n4, nb, par, c->d_part, (const float4*)c->d_p32,
                                                    (const float4*)c->d_q32, (const float4*)c->d_dinv32,
                                                    (float4*)c->d_x32, (float4*)c->d_r32, (float4*)c->d_z32,
                                                    c->d_part + nb, c->d_sc);
      cg32_direction_kernel<<<nb, 256, 0, c->stream>>>(n4, nb, par, -1, c->d_part + nb, (const float4*)c->d_z32,
                                                       (float4*)c->d_p32, c->d_sc, maxit, h);
    }
  };
  const int64_t n0 = c->n_launch;
  gb.seq(G, deps, [&] {
    c->n_launch += 1;
    loopctl_init_kernel<<<1, 32, 0, c->stream>>>(c->d_lc, has16 ? 1 : 0);
  });
  const cudaGraphConditionalHandle h_sweep = gb.handle(G, 1, true);
  cudaGraph_t B = gb.loop(G, deps, h_sweep);
  const cudaGraphConditionalHandle h16 = has16 ? gb.handle(B, 0, false) : 0;
  const cudaGraphConditionalHandle h32 = gb.handle(B, 0, false);
  const int64_t n1 = c->n_launch;
  gb.seq(B, bd, [&] {
    vd_apply_df(c, x, c->d_slot);
    c->n_launch += 6;
    vd_refine_residual_kernel<<<nb, 256, 0, c->stream>>>(n, c->sgn, c->vd->d_dslot, c->d_slot, bvec, c->d_res,
                                                         c->d_part);
    refine_scalars<<<1, 256, 0, c->stream>>>(nb, c->d_part, c->d_rs);
    sweep_ctl_kernel<<<1, 32, 0, c->stream>>>(c->d_rs, c->d_sc, c->d_lc, c->opt.rtol, c->opt.inner_rtol,
                                              c->opt.max_sweeps, h_sweep, has16 ? 1 : 0, h16, h32);
    to32_scaled_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(n, c->d_res, c->d_rs, c->d_b32);
    cg32_init_kernel<<<nb, 256, 0, c->stream>>>(n4, (const float4*)c->d_b32, (const float4*)c->d_dinv32,
                                                (float4*)c->d_x32, (float4*)c->d_r32, (float4*)c->d_z32,
                                                (float4*)c->d_p32, c->d_part);
    cg32_init_scalars<<<1, 256, 0, c->stream>>>(nb, c->d_part, 0.5, c->d_sc, &c->d_lc->tol);
  });
  const int64_t n2 = c->n_launch;
  if (has16) {
    cudaGraph_t B16 = gb.loop(B, bd, h16);
    gb.seq(B16, d16, [&] { inner(true, h16); });
  }
  const int64_t n3 = c->n_launch;
  cudaGraph_t B32 = gb.loop(B, bd, h32);
  gb.seq(B32, d32, [&] { inner(false, h32); });
  const int64_t n4_ = c->n_launch;
  gb.seq(B, bd, [&] {
    c->n_launch += 1;
    vd_refine_update_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(n, c->vd->d_dslot, c->d_x32, c->d_rs, x);
  });
  const int64_t n5 = c->n_launch;
  gb.seq(G, deps, [&] {
    c->n_launch += 1;
    zero_masked_if_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(n, c->d_intmask, c->d_lc, x);
  });
  if (dg) {
    dg->n_static = (n1 - n0) + (c->n_launch - n5);
    dg->n_body = (n2 - n1) + (n5 - n4_);
    dg->n_trip = n4_ - n3;
  }
}

hdg_status vd_solve_graph(hdg_ctx* c, const double* bvec, double* x, hdg_solve_info* info) {
  auto build = [&](GraphBuild& gb, cudaGraph_t G, hdg_ctx::DevGraph& dg) {
    std::vector<cudaGraphNode_t> deps;
    vd_build_solve(c, gb, G, deps, bvec, x, &dg);
  };
  return devgraph_solve(c, c->opt.prec == HDG_FP64 ? 2 : 3, bvec, x, build, info);
}

hdg_status vd_solve(hdg_ctx* c, const double* bvec, double* x, hdg_solve_info* info) {
  if (use_devgraph(c)) return vd_solve_graph(c, bvec, x, info);
  return c->opt.prec == HDG_FP64 ? vd_cg(c, bvec, x, info) : vd_refine(c, bvec, x, info);
}

}  // namespace

hdg_status vd_setup(hdg_ctx* c, const int32_t* elem_k) {
  const int dim = c->dim, nfc = dim + 1, nt = dim * (dim + 1) / 2;
  if (c->phys != HDG_ELASTIC || dim != 3) return fail(c, HDG_EINVAL, "per-element degrees: 3D elastic meshes only");
  if (c->R != 1) return fail(c, HDG_EINVAL, "per-element degrees: nrhs = 1 only");
  const int64_t ne = c->sk.ne, nf = c->sk.nf;
  for (int64_t e = 0; e < ne; ++e)
    if (elem_k[e] < 1 || elem_k[e] > 4) return fail(c, HDG_EINVAL, "per-element degree must be in 1..4");
  VarDeg* v = new (std::nothrow) VarDeg();
  if (!v) return fail(c, HDG_ENOMEM, "host allocation");
  c->vd = v;
  // face degrees and per-element padded degree KT
  std::vector<int> fk(nf, 0), kt(ne, 0);
  for (int64_t f = 0; f < nf; ++f)
    for (int s = 0; s < 2; ++s) {
      const int32_t sl = c->sk.face_slot[2 * f + s];
      if (sl >= 0) fk[f] = std::max(fk[f], (int)elem_k[sl / nfc]);
    }
  for (int64_t e = 0; e < ne; ++e)
    for (int j = 0; j < nfc; ++j) kt[e] = std::max(kt[e], fk[c->sk.elem_face[e * nfc + j]]);
  // trace numbering: face f holds dim x Nf(k_F) entries, component-major
  std::vector<int64_t> t_off(nf + 1, 0);
  for (int64_t f = 0; f < nf; ++f) t_off[f + 1] = t_off[f] + dim * n_modes_h(dim - 1, fk[f]);
  c->ntr = t_off[nf];
  std::vector<int64_t> u_off(ne + 1, 0), h_off(ne + 1, 0), s_off(ne + 1, 0);
  std::vector<int32_t> m_off(ne + 1, 0);
  for (int64_t e = 0; e < ne; ++e) {
    const int np = n_modes_h(dim, elem_k[e]);
    int me = 0;
    for (int j = 0; j < nfc; ++j) me += dim * n_modes_h(dim - 1, fk[c->sk.elem_face[e * nfc + j]]);
    u_off[e + 1] = u_off[e] + (dim + nt) * np;
    h_off[e + 1] = h_off[e] + (int64_t)(dim * np) * (dim * np);
    m_off[e + 1] = m_off[e] + me;
    s_off[e + 1] = s_off[e] + (int64_t)me * me;
  }
  c->nfld = u_off[ne];
  v->m_tot = m_off[ne]; v->s_tot = s_off[ne]; v->h_tot = h_off[ne];
  c->nschur = v->s_tot;
  c->nslot = v->m_tot;
  // compact local entries: faces in local order, components, active modes in the padded order
  std::vector<std::vector<int>> mdeg(5);
  for (int k = 1; k <= 4; ++k) mdeg[k] = face_mode_degrees(dim, k);
  std::vector<int32_t> gidx(v->m_tot), gint(v->m_tot), dslot(2 * (size_t)c->ntr, -1);
  std::vector<int16_t> pidx(v->m_tot);
  std::vector<int64_t> sdiag(v->m_tot);
  for (int64_t e = 0; e < ne; ++e) {
    const int KT = kt[e], NFPT = n_modes_h(dim - 1, KT);
    const int me = m_off[e + 1] - m_off[e];
    int a = 0;
    for (int j = 0; j < nfc; ++j) {
      const int f = c->sk.elem_face[e * nfc + j];
      const int kf = fk[f], nfm = n_modes_h(dim - 1, kf);
      const bool bnd = c->sk.face_bnd[f] >= 0;
      const int s = c->sk.face_slot[2 * f] == (int32_t)(e * nfc + j) ? 0 : 1;
      for (int p = 0; p < dim; ++p) {
        int rank = 0;
        for (int mm = 0; mm < NFPT; ++mm) {
          if (mdeg[KT][mm] > kf) continue;
          const int64_t pos = m_off[e] + a;
          const int64_t d = t_off[f] + p * nfm + rank;
          pidx[pos] = (int16_t)((j * dim + p) * NFPT + mm);
          gidx[pos] = (int32_t)d;
          gint[pos] = bnd ? -1 : (int32_t)d;
          sdiag[pos] = s_off[e] + (int64_t)a * (me + 1);
          if (!bnd) dslot[2 * d + s] = (int32_t)pos;
          ++rank;
          ++a;
        }
      }
    }
  }
  // classes (K, KT) and their tables
  std::map<int, std::vector<int32_t>> groups;
  for (int64_t e = 0; e < ne; ++e) groups[elem_k[e] * 10 + kt[e]].push_back((int32_t)e);
  std::vector<int32_t> elist;
  std::vector<double> tab;
  std::vector<std::array<size_t, 6>> toff;
  // heaviest classes first (descending 10 K + KT): the one-launch local solves start them first
  for (auto it = groups.rbegin(); it != groups.rend(); ++it) {
    auto& g = *it;
    VarDeg::Cls k;
    k.K = g.first / 10; k.KT = g.first % 10;
    k.first = (int64_t)elist.size(); k.count = (int64_t)g.second.size();
    elist.insert(elist.end(), g.second.begin(), g.second.end());
    RefTables T;
    try {
      T = build_tables_pair(dim, k.K, k.KT);
    } catch (const std::exception& ex) {
      return fail(c, HDG_EINVAL, ex.what());
    }
    std::array<size_t, 6> o;
    const std::vector<double>* parts[6] = {&T.Dr, &T.Ff, &T.Ef, &T.Trs, &T.DFrf, &T.Pfg};
    for (int i = 0; i < 6; ++i) { o[i] = tab.size(); tab.insert(tab.end(), parts[i]->begin(), parts[i]->end()); }
    toff.push_back(o);
    v->cls.push_back(k);
  }
  hdg_status s;
  if ((s = dalloc(c, &v->d_tab, tab.size()))) return s;
  for (size_t i = 0; i < v->cls.size(); ++i) {
    Tabs& T = v->cls[i].tabs;
    T.Dr = v->d_tab + toff[i][0]; T.Ff = v->d_tab + toff[i][1]; T.Ef = v->d_tab + toff[i][2];
    T.Trs = v->d_tab + toff[i][3]; T.DFrf = v->d_tab + toff[i][4]; T.Pfg = v->d_tab + toff[i][5];
  }
  v->table.n = (int)v->cls.size();
  for (size_t i = 0; i < v->cls.size(); ++i) {
    v->table.start[i] = v->cls[i].first;
    v->table.key[i] = v->cls[i].K * 10 + v->cls[i].KT;
    v->table.tabs[i] = v->cls[i].tabs;
    VD_DISPATCH(v->cls[i].K, v->cls[i].KT, vd_local_smem, v->local_smem);
  }
  v->table.start[v->cls.size()] = ne;
  // scratch of the classes whose H does not fit shared memory
  v->scr_blocks = 0;
  size_t scr = 0;
  for (const auto& k : v->cls)
    if (k.K == 4) scr = std::max(scr, (size_t)std::min<int64_t>(k.count, VD_CHUNK) * CondVdCfg<3, 4, 4>::SCR);
  if (scr && (s = dalloc(c, &v->d_scr, scr))) return s;
  if ((s = dalloc(c, &v->d_elist, elist.size()))) return s;
  if ((s = dalloc(c, &v->d_u_off, (size_t)ne + 1))) return s;
  if ((s = dalloc(c, &v->d_h_off, (size_t)ne + 1))) return s;
  if ((s = dalloc(c, &v->d_s_off, (size_t)ne + 1))) return s;
  if ((s = dalloc(c, &v->d_m_off, (size_t)ne + 1))) return s;
  if ((s = dalloc(c, &v->d_gidx, (size_t)v->m_tot))) return s;
  if ((s = dalloc(c, &v->d_gint, (size_t)v->m_tot))) return s;
  if ((s = dalloc(c, &v->d_pidx, (size_t)v->m_tot))) return s;
  if ((s = dalloc(c, &v->d_sdiag, (size_t)v->m_tot))) return s;
  if ((s = dalloc(c, &v->d_dslot, 2 * (size_t)c->ntr))) return s;
  auto up = [&](void* dst, const void* src, size_t bytes) {
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c->stream);
  };
  CUDA_TRY(c, up(v->d_tab, tab.data(), tab.size() * 8));
  CUDA_TRY(c, up(v->d_elist, elist.data(), elist.size() * 4));
  CUDA_TRY(c, up(v->d_u_off, u_off.data(), u_off.size() * 8));
  CUDA_TRY(c, up(v->d_h_off, h_off.data(), h_off.size() * 8));
  CUDA_TRY(c, up(v->d_s_off, s_off.data(), s_off.size() * 8));
  CUDA_TRY(c, up(v->d_m_off, m_off.data(), m_off.size() * 4));
  CUDA_TRY(c, up(v->d_gidx, gidx.data(), gidx.size() * 4));
  CUDA_TRY(c, up(v->d_gint, gint.data(), gint.size() * 4));
  CUDA_TRY(c, up(v->d_pidx, pidx.data(), pidx.size() * 2));
  CUDA_TRY(c, up(v->d_sdiag, sdiag.data(), sdiag.size() * 8));
  CUDA_TRY(c, up(v->d_dslot, dslot.data(), dslot.size() * 4));
  // volume rules of each degree and per-element point offsets (initial-data projection)
  v->rule.resize(5);
  std::vector<double> qtab;
  size_t qw_off[5] = {0}, qp_off[5] = {0};
  for (int k = 1; k <= 4; ++k) {
    v->rule[k] = build_tables(dim, k);
    qw_off[k] = qtab.size();
    qtab.insert(qtab.end(), v->rule[k].qv_w.begin(), v->rule[k].qv_w.end());
    qp_off[k] = qtab.size();
    qtab.insert(qtab.end(), v->rule[k].qv_phi.begin(), v->rule[k].qv_phi.end());
    v->quad.nq[k] = v->rule[k].nqv;
    v->quad.np[k] = v->rule[k].Np;
  }
  v->ek.assign(elem_k, elem_k + ne);
  v->q_off.assign(ne + 1, 0);
  for (int64_t e = 0; e < ne; ++e) v->q_off[e + 1] = v->q_off[e] + v->rule[elem_k[e]].nqv;
  if ((s = dalloc(c, &v->d_qtab, qtab.size()))) return s;
  if ((s = dalloc(c, &v->d_ek, (size_t)ne))) return s;
  if ((s = dalloc(c, &v->d_q_off, (size_t)ne + 1))) return s;
  for (int k = 1; k <= 4; ++k) {
    v->quad.qw[k] = v->d_qtab + qw_off[k];
    v->quad.qphi[k] = v->d_qtab + qp_off[k];
  }
  CUDA_TRY(c, up(v->d_qtab, qtab.data(), qtab.size() * 8));
  CUDA_TRY(c, up(v->d_ek, v->ek.data(), v->ek.size() * 4));
  CUDA_TRY(c, up(v->d_q_off, v->q_off.data(), v->q_off.size() * 8));
  // operators and workspaces
  const size_t ntr = (size_t)c->ntr, nfld = (size_t)c->nfld;
  {
    int per_sm = 4;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cg32_update_kernel, 256, 0) != cudaSuccess || per_sm < 1)
      per_sm = 4;
    c->nb_red = std::max(1, std::min(per_sm * c->sms, (int)((ntr + 255) / 256)));
  }
  if ((s = dalloc(c, &c->d_S, (size_t)v->s_tot))) return s;
  if ((s = dalloc(c, &c->d_Hinv, (size_t)v->h_tot))) return s;
  if ((s = dalloc(c, &c->d_dinv, ntr))) return s;
  if ((s = dalloc(c, &c->d_err, 1))) return s;
  for (double** p : {&c->d_r, &c->d_z, &c->d_p, &c->d_q, &c->d_b, &c->d_lam, &c->d_lam_prev, &c->d_lam_prev2, &c->d_lam_x})
    if ((s = dalloc(c, p, ntr))) return s;
  if ((s = dalloc(c, &c->d_slot, (size_t)v->m_tot))) return s;
  if ((s = dalloc(c, &c->d_part, (size_t)c->nb_red * 3))) return s;
  if ((s = dalloc(c, &c->d_sc, 1))) return s;
  CUDA_TRY(c, cudaMallocHost((void**)&c->h_sc, sizeof(CgScal)));
  std::memset(c->h_sc, 0, sizeof(CgScal));
  for (double** p : {&c->d_u, &c->d_uprev, &c->d_h, &c->d_unew, &c->d_stage[0], &c->d_stage[1], &c->d_stage[2]})
    if ((s = dalloc(c, p, nfld))) return s;
  if (c->opt.prec != HDG_FP64) {
    if ((s = dalloc(c, &v->d_S32, (size_t)v->s_tot))) return s;
    if ((s = dalloc(c, &v->d_S32lo, (size_t)v->s_tot))) return s;
    if (c->opt.prec == HDG_MIXED16) {
      if ((s = dalloc(c, &v->d_S16, (size_t)v->s_tot))) return s;
      if ((s = dalloc(c, &v->d_sc16, (size_t)ne))) return s;
    }
    if ((s = dalloc(c, &c->d_slot32, (size_t)v->m_tot))) return s;
    c->nfe4 = (int64_t)((ntr + 3) / 4) * 4;
    for (float** p : {&c->d_dinv32, &c->d_r32, &c->d_z32, &c->d_p32, &c->d_q32, &c->d_x32, &c->d_b32}) {
      if ((s = dalloc(c, p, (size_t)c->nfe4))) return s;
      CUDA_TRY(c, cudaMemsetAsync(*p, 0, (size_t)c->nfe4 * 4, c->stream));
    }
    if ((s = dalloc(c, &c->d_res, ntr))) return s;
    if ((s = dalloc(c, &c->d_rs, 1))) return s;
    CUDA_TRY(c, cudaMallocHost((void**)&c->h_rs, sizeof(RefScal)));
  }
  CUDA_TRY(c, cudaMemsetAsync(c->d_lam, 0, ntr * 8, c->stream));
  CUDA_TRY(c, cudaMemsetAsync(c->d_u, 0, nfld * 8, c->stream));
  CUDA_TRY(c, cudaMemsetAsync(c->d_uprev, 0, nfld * 8, c->stream));
  // the host index arrays above are released at return: wait for their uploads
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  {
    std::vector<uint8_t> mask((size_t)c->ntr);
    for (int64_t d = 0; d < c->ntr; ++d) mask[d] = dslot[2 * d] >= 0 ? 1 : 0;
    if ((s = guess_setup(c, mask.data()))) return s;
  }
  c->have_state = true;
  return HDG_OK;
}

hdg_status vd_condense(hdg_ctx* c, double alpha) {
  if (!(alpha > 0.0) || !std::isfinite(alpha)) return fail(c, HDG_EINVAL, "alpha must be positive and finite");
  c->alpha = alpha;
  CUDA_TRY(c, cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
  for (const auto& k : c->vd->cls) VD_DISPATCH(k.K, k.KT, vd_launch_condense, c, k);
  hdg_status s = check_launch(c, "vd_condense");
  if (s) return s;
  c->n_launch += 1;
  vd_diag_kernel<<<grid_for(c, c->ntr), 256, 0, c->stream>>>(c->ntr, c->sgn, c->vd->d_dslot, c->vd->d_sdiag, c->d_S,
                                                             c->d_dinv);
  if (c->opt.prec != HDG_FP64) {
    c->n_launch += 2;
    to32_copy_kernel<<<grid_for(c, c->vd->s_tot), 256, 0, c->stream>>>(c->vd->s_tot, c->d_S, c->vd->d_S32);
    c->n_launch += 1;
    lo32_kernel<<<grid_for(c, c->vd->s_tot), 256, 0, c->stream>>>(c->vd->s_tot, c->d_S, c->vd->d_S32, c->vd->d_S32lo);
    if (c->vd->d_S16) {
      c->n_launch += 1;
      pack16_vd_kernel<<<grid_for(c, c->sk.ne * 32), 256, 0, c->stream>>>(c->sk.ne, c->vd->d_s_off, c->d_S,
                                                                          c->vd->d_sc16, c->vd->d_S16);
    }
    to32_kernel<<<grid_for(c, c->ntr), 256, 0, c->stream>>>(c->ntr, c->d_dinv, c->d_dinv32);
  }
  if ((s = check_launch(c, "vd_diag"))) return s;
  // tiles of the applies, tuned once per context on its own operator
  VarDeg* v = c->vd;
  if (c->opt.prec == HDG_FP64) {
    if (v->tile64 < 0)
      v->tile64 = vd_tune(c, [&](int t) { vd_apply_variant<double>(c, t, c->d_S, c->d_lam, c->d_slot, nullptr); });
  } else {
    if (v->tile32 < 0)
      v->tile32 = vd_tune(c, [&](int t) { vd_apply_variant<float>(c, t, v->d_S32, c->d_p32, c->d_slot32, nullptr); });
    if (v->tiledf < 0) v->tiledf = vd_tune(c, [&](int t) { vd_apply_df_variant(c, t, c->d_lam, c->d_slot); });
    if (v->d_S16 && v->tile16 < 0)
      v->tile16 = vd_tune(c, [&](int t) {
        vd_apply_variant<float, __half>(c, t, v->d_S16, c->d_p32, c->d_slot32, nullptr, v->d_sc16);
      });
  }
  if ((s = check_launch(c, "vd_tune"))) return s;
  int herr = 0;
  CUDA_TRY(c, cudaMemcpyAsync(&herr, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (herr) { c->condensed = false; return fail(c, HDG_EINVAL, "local velocity block not positive definite"); }
  c->condensed = true;
  return HDG_OK;
}

hdg_status vd_stage_solve(hdg_ctx* c, const double* hist, double tt, double* uout, hdg_solve_info* info) {
  (void)tt;   // no sources or time-dependent boundary data on this path
  vd_local(c, 0, nullptr, hist, c->d_lam, c->d_slot);
  hdg_status s = check_launch(c, "vd_rhs");
  if (s) return s;
  if ((s = vd_gather(c, c->d_slot, -c->sgn, c->d_b))) return s;
  if ((s = guess_before(c))) return s;
  if ((s = vd_solve(c, c->d_b, c->d_lam, info))) return s;
  if ((s = guess_after(c))) return s;
  vd_local(c, 1, nullptr, hist, c->d_lam, uout);
  return check_launch(c, "vd_recover");
}

// One DIRK(3,3) step (Eqs. 10_1-2) of the per-element-degree path as ONE graph launch: for each
// stage the history combination, the element right-hand sides of every degree class, the face
// gather, the least-squares guess, the device-driven trace solve and the recovery, then the
// update. Built once per (u, u_new) buffer pair and mass shift; the local-solve block sizes must
// have been tuned (the first step runs through individual launches).
hdg_status vd_dirk3_step_graph(hdg_ctx* c, const double hc[3][3], const double uc[4], hdg_solve_info* info, bool* done) {
  *done = false;
  VarDeg* v = c->vd;
  if (!use_devgraph(c) || v->local_nth[0] == 0 || v->local_nth[1] == 0 || !c->condensed) return HDG_OK;
  hdg_status s;
  if (!c->d_sacc) {
    if ((s = dalloc(c, &c->d_sacc, 1))) return s;
    CUDA_TRY(c, cudaMallocHost((void**)&c->h_sacc, sizeof(StepAcc)));
  }
  hdg_ctx::DevGraph* dg = nullptr;
  for (auto& g : c->dgraphs)
    if (g.kind == 10 && g.b == c->d_u && g.x == c->d_unew && g.alpha == c->alpha) dg = &g;
  if (!dg) {
    if (!c->cap_stream) CUDA_TRY(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    if (c->dgraphs.size() >= kMaxDevGraphs) {
      cudaGraphExecDestroy(c->dgraphs.front().exec);
      c->dgraphs.erase(c->dgraphs.begin());
    }
    cudaGraph_t G = nullptr;
    CUDA_TRY(c, cudaGraphCreate(&G, 0));
    GraphBuild gb;
    gb.st = c->cap_stream;
    const cudaStream_t keep = c->stream;
    const int64_t keep_launch = c->n_launch;
    c->stream = c->cap_stream;
    const int64_t n = c->nfld;
    std::vector<cudaGraphNode_t> deps;
    gb.seq(G, deps, [&] { step_acc_reset_kernel<<<1, 32, 0, c->stream>>>(c->d_sacc); });
    for (int i = 0; i < 3; ++i) {
      gb.seq(G, deps, [&] {
        combine_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(n, hc[i][0], c->d_u, hc[i][1],
                                                              i > 0 ? c->d_stage[0] : nullptr, hc[i][2],
                                                              i > 1 ? c->d_stage[1] : nullptr, 0, nullptr, c->d_h);
        vd_local(c, 0, nullptr, c->d_h, c->d_lam, c->d_slot);
        vd_gather(c, c->d_slot, -c->sgn, c->d_b);
        guess_before(c);
      });
      vd_build_solve(c, gb, G, deps, c->d_b, c->d_lam, nullptr);
      gb.seq(G, deps, [&] {
        step_acc_kernel<<<1, 32, 0, c->stream>>>(c->d_lc, c->d_sacc);
        guess_after(c);
        vd_local(c, 1, nullptr, c->d_h, c->d_lam, c->d_stage[i]);
      });
    }
    gb.seq(G, deps, [&] {
      combine_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(n, uc[0], c->d_u, uc[1], c->d_stage[0], uc[2], c->d_stage[1],
                                                            uc[3], c->d_stage[2], c->d_unew);
    });
    hdg_ctx::DevGraph ng{10, c->d_u, c->d_unew, nullptr, c->n_launch - keep_launch, 0, 0, c->alpha};
    c->stream = keep;
    c->n_launch = keep_launch;
    cudaGraphExec_t ex = nullptr;
    cudaError_t e = gb.err;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, G, 0);
    cudaGraphDestroy(G);
    if (e != cudaSuccess) return fail(c, HDG_ECUDA, std::string("step graph: ") + cudaGetErrorString(e));
    ng.exec = ex;
    c->dgraphs.push_back(ng);
    dg = &c->dgraphs.back();
  }
  CUDA_TRY(c, cudaGraphLaunch(dg->exec, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(c->h_sacc, c->d_sacc, sizeof(StepAcc), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  const StepAcc A = *c->h_sacc;
  c->n_launch += dg->n_static + (int64_t)A.iters * 3;
  if (info) {
    info->iterations += A.iters;
    info->sweeps += A.sweeps;
    info->rel_residual = A.rel;
  }
  *done = true;
  if (A.bad == 3)
    return fail(c, HDG_ENOCONV, "mixed-precision refinement reached max_sweeps=" + std::to_string(c->opt.max_sweeps));
  if (A.bad) return fail(c, HDG_ENOCONV, "trace solve reached maxit=" + std::to_string(c->opt.maxit));
  return HDG_OK;
}

hdg_status vd_trace_apply(hdg_ctx* c, const double* x, double* y) {
  vd_apply64(c, x, c->d_slot, nullptr, -1);
  return vd_gather(c, c->d_slot, 1.0, y);
}

hdg_status vd_condensed_rhs(hdg_ctx* c, const double* F, const double* lamD, double* r) {
  vd_local(c, 0, F, nullptr, lamD, c->d_slot);
  hdg_status s = check_launch(c, "vd_rhs");
  if (s) return s;
  return vd_gather(c, c->d_slot, -1.0, r);
}

hdg_status vd_trace_solve(hdg_ctx* c, const double* r, double* lam, hdg_solve_info* info) {
  c->n_launch += 1;
  combine_kernel<<<grid_for(c, c->ntr), 256, 0, c->stream>>>(c->ntr, c->sgn, r, 0, nullptr, 0, nullptr, 0, nullptr,
                                                             c->d_b);
  hdg_status s = vd_solve(c, c->d_b, lam, info);
  if (s == HDG_OK) CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return s;
}

hdg_status vd_recover(hdg_ctx* c, const double* F, const double* lam, double* u) {
  vd_local(c, 1, F, nullptr, lam, u);
  return check_launch(c, "vd_recover");
}

hdg_status vd_quadrature_points(hdg_ctx* c, int32_t which, double* xyz) {
  if (which != 0) return fail(c, HDG_EINVAL, "per-element degrees: clamped boundary, no face points");
  const int d = c->dim, nc = c->nfc;
  const VarDeg* v = c->vd;
  for (int64_t e = 0; e < c->sk.ne; ++e) {
    const RefTables& T = v->rule[v->ek[e]];
    const double* X = &c->h_vert_elem[(size_t)e * nc * d];
    for (int q = 0; q < T.nqv; ++q)
      for (int j = 0; j < d; ++j) {
        double val = X[j];
        for (int r = 0; r < d; ++r) val += T.qv_pts[(size_t)q * d + r] * (X[(r + 1) * d + j] - X[j]);
        xyz[((size_t)v->q_off[e] + q) * d + j] = val;
      }
  }
  return HDG_OK;
}

hdg_status vd_project_volume(hdg_ctx* c, const double* vals, double* u) {
  VarDeg* v = c->vd;
  const size_t cnt = (size_t)v->q_off[c->sk.ne] * c->ncomp;
  double* dv = nullptr;
  hdg_status s;
  if ((s = dalloc(c, &dv, cnt))) return s;
  cudaError_t e1 = cudaMemcpyAsync(dv, vals, cnt * 8, cudaMemcpyHostToDevice, c->stream);
  if (e1 == cudaSuccess) {
    c->n_launch += 1;
    project_vd_kernel<<<grid_for(c, c->sk.ne * 128, 128), 128, 0, c->stream>>>(c->sk.ne, c->ncomp, v->d_ek, v->d_q_off,
                                                                               v->d_u_off, v->quad, dv, u);
    e1 = cudaGetLastError();
  }
  if (e1 == cudaSuccess) e1 = cudaStreamSynchronize(c->stream);
  dfree(c, dv);
  c->bytes -= (int64_t)(cnt * 8);
  if (e1 != cudaSuccess) return fail(c, HDG_ECUDA, std::string("project_volume: ") + cudaGetErrorString(e1));
  return HDG_OK;
}

hdg_status vd_get_tuning(const hdg_ctx* c, hdg_tuning* o) {
  const VarDeg* v = c->vd;
  // the FP64-accurate apply is the FP64 kernel on the plain path and the double-float kernel
  // (residual of the refinement) on the mixed path
  const int tr = c->opt.prec == HDG_FP64 ? v->tile64 : v->tiledf;
  o->tuned = tr >= 0 ? 1 : 0;
  const int t32 = v->tile32 < 0 ? 1 : v->tile32, t64 = tr < 0 ? 1 : tr;
  o->apply32_warps = kApplyTiles[t32][0];
  o->apply32_unroll = kApplyTiles[t32][1];
  o->apply64_warps = kApplyTiles[t64][0];
  o->apply64_unroll = kApplyTiles[t64][1];
  o->local_threads[0] = v->local_nth[0];
  o->local_threads[1] = v->local_nth[1];
  return HDG_OK;
}

void vd_destroy(hdg_ctx* c) {
  delete c->vd;
  c->vd = nullptr;
}
