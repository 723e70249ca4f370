// The library context (hdg_ctx) and the host helpers shared by the translation units of
// the library: errors, device allocation, launch sizing, instrumentation, (dim, k) dispatch.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cstdint>
#include <string>
#include <utility>
#include <vector>

#include "../../include/hdg.h"
#include "kernels.cuh"
#include "devloop.cuh"
#include "dflocal.cuh"
#include "mesh.h"
#include "reftab.h"

using namespace hdg;

struct VarDeg;   // variable-degree (per-element k) data of an elastic context
struct Svk;      // nonlinear (Saint Venant-Kirchhoff) elastodynamics data
struct Bilu;     // block ILU(0) preconditioner of the GMRES trace solve

struct hdg_ctx {
  std::string err;
  cudaStream_t stream = nullptr;
  hdg_options opt{};
  int dim = 0, k = 0, Np = 0, Nf = 0, n = 0, m = 0, nfc = 0;
  int phys = 0;             // HDG_ACOUSTIC or HDG_ELASTIC
  int ncomp = 0;            // field components per element
  int nv = 0;               // size of the factored local block (H^{-1} is nv x nv)
  double sgn = -1.0;        // the Krylov operator is sgn * K (SPD)
  double *d_lame = nullptr, *d_mue = nullptr;
  int sms = 148;
  double tau = 1.0;
  Skeleton sk;
  RefTables T;
  std::vector<double> h_vert_elem;   // [ne][d+1][d] element vertex coordinates (sorted order)
  // device: mesh and tables
  double *d_geo = nullptr, *d_rho = nullptr, *d_c = nullptr, *d_tab = nullptr;
  int32_t *d_elem_face = nullptr, *d_face_slot = nullptr, *d_face_bnd = nullptr;
  int64_t* d_bnd_faces = nullptr;
  Tabs tabs{};
  double *d_qv_w = nullptr, *d_qv_phi = nullptr;
  // condensed operators
  double *d_S = nullptr, *d_Hinv = nullptr, *d_dinv = nullptr;
  double alpha = 0.0;
  bool condensed = false;
  int* d_err = nullptr;
  // Krylov workspace
  double *d_r = nullptr, *d_z = nullptr, *d_p = nullptr, *d_q = nullptr, *d_b = nullptr, *d_slot = nullptr;
  double* d_part = nullptr;
  CgScal* d_sc = nullptr;
  CgScal* h_sc = nullptr;   // pinned
  int nb_red = 0;
  int df_per_sm = 1;            // resident CTAs per SM of the persistent double-float apply
  int tcp_per_sm = 1;           // resident CTAs per SM of the persistent tensor-core column-block apply
  // mixed precision
  float *d_S32 = nullptr, *d_dinv32 = nullptr, *d_slot32 = nullptr;
  float* d_Sdf = nullptr;       // double-float diagonal-major copy of S_K (refinement apply)
  df2 *d_Hinvdf = nullptr, *d_geodf = nullptr, *d_tabdf = nullptr;   // double-float local solves
  double* d_post = nullptr;       // post-processing tables K1 | E1 (built at the first hdg_postprocess)
  int64_t post_k1 = 0;            // entries of K1
  TabsDf tabsdf{};
  __half* d_S16 = nullptr;      // FP16 packed S_K (inner Krylov operator of HDG_MIXED16)
  float* d_sc16 = nullptr;      // its per-element scales
  int32_t* d_gface16 = nullptr; // its trace gather table [whole groups][nfc] (face id, -1: none)
  int a16_per_sm = 1;           // resident CTAs per SM of the persistent FP16 apply
  double *d_pqpart = nullptr, *d_pq = nullptr;   // p.q block partials and result of the FP32/FP16 apply
  unsigned* d_ticket = nullptr;                   // last-block counter of that reduction
  DevTiming* d_dtime = nullptr;   // device-side launch timing: [0] FP32 apply, [1] FP16 apply
  float *d_r32 = nullptr, *d_z32 = nullptr, *d_p32 = nullptr, *d_q32 = nullptr, *d_x32 = nullptr, *d_b32 = nullptr;
  double* d_res = nullptr;   // FP64 refinement residual
  int64_t nfe4 = 0;          // FP32 face vectors padded to a multiple of 4 entries
  int last_it32 = 16, last_it64 = 16;   // iteration counts of the previous solves (poll schedule)
  int last_sweep_it[8] = {16, 16, 16, 16, 16, 16, 16, 16};   // the same per refinement sweep
  double *d_lam_prev = nullptr, *d_lam_prev2 = nullptr, *d_lam_x = nullptr;  // trace history (initial guess)
  int n_lam_hist = 0;           // valid entries of that history (lam^{n-1}, lam^{n-2})
  // multiple right-hand sides (R columns, innermost index)
  int R = 1;
  double *d_mslot = nullptr;            // FP64 slots [ne][m][R]
  float *d_mslot32 = nullptr;           // FP32 slots [ne][m][R]
  float *d_mShi = nullptr, *d_mSlo = nullptr;   // S_K as FP32 pairs [ne][m][m] (double-float residual apply)
  double *d_mrho0 = nullptr, *d_mrho1 = nullptr, *d_malpha = nullptr, *d_mbeta = nullptr, *d_mrr = nullptr,
         *d_mbb = nullptr, *d_mtol2 = nullptr, *d_mscale = nullptr, *d_mrr2 = nullptr, *d_mbb2 = nullptr;
  int *d_mconv = nullptr, *d_mdone = nullptr, *d_mnconv = nullptr, *d_miters = nullptr;
  int* h_mint = nullptr;                // pinned: [0] done flag, [1] nconv, [2] iterations
  // CUDA graphs of per-column Krylov iteration chunks, keyed by (vector type, x pointer)
  std::vector<std::pair<std::pair<int, const void*>, cudaGraphExec_t>> graphs;
  int32_t* d_src_col = nullptr;
  double* d_src_delay = nullptr;
  int src_cap = 0;                      // capacity of the per-source buffers (grow-only)
  RefScal* d_rs = nullptr;
  RefScal* h_rs = nullptr;   // pinned
  // time state
  double *d_u = nullptr, *d_uprev = nullptr, *d_lam = nullptr, *d_h = nullptr, *d_unew = nullptr;
  double* d_stage[3] = {nullptr, nullptr, nullptr};
  double t = 0.0;
  bool have_state = false;
  // data
  int nsrc = 0;
  int32_t* d_src_ptr = nullptr;
  double* d_src_phi = nullptr;
  double f0 = 0.0, t0 = 0.0;
  double* d_bnd_coef = nullptr;
  double omega = 0.0, phase = 0.0;
  int64_t bytes = 0;
  std::vector<void*> allocs;
  // instrumentation
  bool stats_on = false;
  int64_t n_launch = 0, n_apply = 0, n_apply32 = 0, n_applydf = 0, n_apply16 = 0, n_svkc = 0, n_svkr = 0;
  double apply_ms = 0.0, apply32_ms = 0.0, applydf_ms = 0.0, apply16_ms = 0.0, svkc_ms = 0.0, svkr_ms = 0.0;
  std::vector<cudaEvent_t> ev_pool;   // pairs (start, stop)
  std::vector<char> ev_kind;          // per pair: 0 FP64, 1 FP32, 2 double-float, 3 FP16 apply,
                                      // 4 SVK condensation, 5 SVK recovery
  std::vector<int> ev_iter;           // per pair: Krylov iteration index (-1: always live)
  size_t ev_used = 0;
  // entries of one field / trace column (n N_e and N_f N_faces for one degree; sums of the
  // per-element / per-face sizes on a variable-degree mesh)
  int64_t nfld = 0, ntr = 0;
  int64_t nschur = 0, nslot = 0;   // S_K entries and element trace entries summed over the elements
  // least-squares initial guess: ring of the last q stage right-hand sides b_i and solutions
  // lam_i (same alpha), their Gram matrix on the host, the interior-entry mask
  double *d_gb = nullptr, *d_gl = nullptr, *d_gdots = nullptr, *d_gpart = nullptr;
  uint8_t* d_intmask = nullptr;
  int g_q = 0, g_n = 0, g_next = 0;   // capacity, stored pairs, next slot
  double g_gram[8][8] = {};
  double g_dots[9] = {};   // dots of the current b with the stored b_i, then (b, b)
  // the same per column (nrhs > 1): Gram matrices [R][8][8], dots [9][R], coefficients [8][R]
  std::vector<double> gm_gram, gm_dots, gm_coef;
  double* d_gcoef = nullptr;
  GuessDev* d_gd = nullptr;   // the same on the device (one column): Gram matrix, ring counters
  // device-driven trace solves: control block, capture stream and the cached graphs (one per
  // solver kind and right-hand-side / solution buffers), with the kernel launches they hold
  LoopCtl* d_lc = nullptr;
  LoopCtl* h_lc = nullptr;   // pinned
  cudaStream_t cap_stream = nullptr;
  struct DevGraph {
    int kind;
    const void* b;
    const void* x;
    cudaGraphExec_t exec;
    int64_t n_static, n_body, n_trip;   // launches outside the loops, per sweep body, per inner trip
    double alpha;                       // mass shift baked into a whole-step graph (0 for a solve)
  };
  std::vector<DevGraph> dgraphs;
  bool guess_x = false;   // the solve being issued starts from the least-squares guess of its b
  StepAcc* d_sacc = nullptr;   // totals of a graph-launched step, and their pinned host copy
  StepAcc* h_sacc = nullptr;
  // continuous traces (IEDG / EDG): free face nodes, the node map and its incidence lists, the
  // nodal-to-modal table, the nodal unknowns and right-hand side, face work arrays
  int tspace = 0;                 // HDG_TRACE_HDG / IEDG / EDG
  int64_t n_mu = 0, n_mu4 = 0;    // free nodes; FP32 node vectors padded to a multiple of 4
  int32_t *d_face_node = nullptr, *d_node_ptr = nullptr, *d_node_inc = nullptr;
  double *d_vinv = nullptr, *d_mu = nullptr, *d_bmu = nullptr, *d_ew64 = nullptr, *d_w64 = nullptr;
  float *d_ew32 = nullptr, *d_w32 = nullptr;
  // restarted GMRES (allocated at the first GMRES solve): basis [m + 1][n], dot partials, the
  // dots of the last pass and the coefficients of the update
  double *d_gmV = nullptr, *d_gmpart = nullptr, *d_gmh = nullptr, *d_gmy = nullptr;
  VarDeg* vd = nullptr;
  Svk* svk = nullptr;   // set for HDG_SVK contexts (elastic trace layout, 21 N_p fields)
  bool svk_mixed = false; // HDG_SVK with HDG_MIXED: FP32 Jacobian, FP64 residual
  Bilu* bilu = nullptr;   // set when opt.precond == HDG_PRECOND_BILU0
};

namespace {

hdg_status fail(hdg_ctx* c, hdg_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

#define CUDA_TRY(ctx, call)                                                                       \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess) return fail(ctx, HDG_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <typename T>
hdg_status dalloc(hdg_ctx* c, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    return fail(c, HDG_ENOMEM, std::string("cudaMalloc(") + std::to_string(count * sizeof(T)) + "): " + cudaGetErrorString(e));
  }
  c->allocs.push_back(*p);
  c->bytes += (int64_t)(count * sizeof(T));
  return HDG_OK;
}

void dfree(hdg_ctx* c, void* p) {
  if (!p) return;
  cudaFree(p);
  auto it = std::find(c->allocs.begin(), c->allocs.end(), p);
  if (it != c->allocs.end()) c->allocs.erase(it);
}

hdg_status check_launch(hdg_ctx* c, const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(c, HDG_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return HDG_OK;
}

// a caller's device pointer may be read as 16-byte vectors only when it is 16-byte aligned
inline bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

int grid_for(const hdg_ctx* c, int64_t n, int block = 256) {
  int64_t g = (n + block - 1) / block;
  int64_t cap = (int64_t)c->sms * 8;
  return (int)std::max<int64_t>(1, std::min(g, cap));
}

SrcArgs srcargs(const hdg_ctx* c, double t) {
  SrcArgs a;
  a.ptr = c->nsrc > 0 ? c->d_src_ptr : nullptr;
  a.phi = c->d_src_phi; a.col = c->d_src_col; a.delay = c->d_src_delay;
  a.f0 = c->f0; a.t0 = c->t0; a.t = t;
  return a;
}

DevMesh devmesh(const hdg_ctx* c) {
  DevMesh m;
  m.ne = c->sk.ne; m.nf = c->sk.nf;
  m.geo = c->d_geo; m.rho = c->d_rho; m.c = c->d_c;
  m.elem_face = c->d_elem_face; m.face_slot = c->d_face_slot; m.face_bnd = c->d_face_bnd;
  return m;
}

// Event pair around one apply launch (instrumentation); returns the stop event or null.
cudaEvent_t apply_begin(hdg_ctx* c, int kind = 0, int iter = -1) {
  if (!c->stats_on) return nullptr;
  if (c->ev_used + 2 > c->ev_pool.size()) {
    for (int i = 0; i < 64; ++i) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
      c->ev_pool.push_back(e);
    }
    c->ev_kind.resize(c->ev_pool.size() / 2 + 1);
    c->ev_iter.resize(c->ev_pool.size() / 2 + 1);
  }
  cudaEvent_t a = c->ev_pool[c->ev_used];
  c->ev_kind[c->ev_used / 2] = (char)kind;
  c->ev_iter[c->ev_used / 2] = iter;
  cudaEventRecord(a, c->stream);
  return c->ev_pool[c->ev_used + 1];
}
void apply_end(hdg_ctx* c, cudaEvent_t stop) {
  if (!stop) return;
  cudaEventRecord(stop, c->stream);
  c->ev_used += 2;
}
// Harvests the recorded pairs (call after a stream synchronisation). Launches of Krylov
// iterations at or beyond live_iters returned early (the solve had converged) and are
// dropped, so the statistics time only launches that did the work.
void harvest(hdg_ctx* c, int live_iters = 1 << 30) {
  for (size_t i = 0; i + 1 < c->ev_used; i += 2) {
    float ms = 0.f;
    if (c->ev_iter[i / 2] >= live_iters) continue;
    if (cudaEventElapsedTime(&ms, c->ev_pool[i], c->ev_pool[i + 1]) == cudaSuccess) {
      if (c->ev_kind[i / 2] == 1) { c->apply32_ms += ms; c->n_apply32 += 1; }
      else if (c->ev_kind[i / 2] == 2) { c->applydf_ms += ms; c->n_applydf += 1; }
      else if (c->ev_kind[i / 2] == 3) { c->apply16_ms += ms; c->n_apply16 += 1; }
      else if (c->ev_kind[i / 2] == 4) { c->svkc_ms += ms; c->n_svkc += 1; }
      else if (c->ev_kind[i / 2] == 5) { c->svkr_ms += ms; c->n_svkr += 1; }
      else { c->apply_ms += ms; c->n_apply += 1; }
    }
  }
  c->ev_used = 0;
}

// ---- device-driven trace solves
// Runs the solve graph of this kind for the buffers (b, x), building it at the first use:
// build(gb, G, dg) adds the solve to G (while it runs, c->stream is the capture stream) and
// records in dg the kernel launches outside the loops, per sweep body and per inner trip of two
// Krylov iterations. The graph ends with the control block written; the call waits for it and
// maps the stop code to a status. At most kMaxDevGraphs graphs are kept (oldest dropped).
constexpr size_t kMaxDevGraphs = 12;

template <class BUILD>
hdg_status devgraph_solve(hdg_ctx* c, int kind, const void* b, const void* x, BUILD build, hdg_solve_info* info) {
  hdg_ctx::DevGraph* dg = nullptr;
  for (auto& g : c->dgraphs)
    if (g.kind == kind && g.b == b && g.x == x) dg = &g;
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
    hdg_ctx::DevGraph ng{kind, b, x, nullptr, 0, 0, 0, 0.0};
    const cudaStream_t keep = c->stream;
    const int64_t keep_launch = c->n_launch;
    c->stream = c->cap_stream;
    build(gb, G, ng);
    c->stream = keep;
    c->n_launch = keep_launch;
    cudaGraphExec_t ex = nullptr;
    cudaError_t e = gb.err;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, G, 0);
    cudaGraphDestroy(G);
    if (e != cudaSuccess) return fail(c, HDG_ECUDA, std::string("device-driven solve graph: ") + cudaGetErrorString(e));
    ng.exec = ex;
    c->dgraphs.push_back(ng);
    dg = &c->dgraphs.back();
  }
  CUDA_TRY(c, cudaGraphLaunch(dg->exec, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(c->h_lc, c->d_lc, sizeof(LoopCtl), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  const LoopCtl L = *c->h_lc;
  c->n_launch += dg->n_static + (int64_t)(L.sweep + 1) * dg->n_body + (int64_t)((L.total_it + 1) / 2 + L.sweep) * dg->n_trip;
  if (info) {
    info->iterations += L.total_it;
    info->sweeps += L.sweep;
    info->rel_residual = L.rel;
  }
  if (L.stop == 1 || L.stop == 2) return HDG_OK;
  if (L.stop == 3)
    return fail(c, HDG_ENOCONV, "mixed-precision refinement reached max_sweeps=" + std::to_string(c->opt.max_sweeps) +
                                    " with relative residual " + std::to_string(L.rel));
  return fail(c, HDG_ENOCONV, "trace solve reached maxit=" + std::to_string(c->opt.maxit) + " with relative residual " +
                                  std::to_string(L.rel));
}

inline bool use_devgraph(const hdg_ctx* c) { return c->opt.device_loops && !c->stats_on && c->R == 1 && c->d_lc; }

// ---- dispatch on (dim, k)
#define HDG_DISPATCH(c, FN, ...)                     \
  switch ((c)->dim * 10 + (c)->k) {                  \
    case 21: FN<2, 1>(__VA_ARGS__); break;           \
    case 22: FN<2, 2>(__VA_ARGS__); break;           \
    case 23: FN<2, 3>(__VA_ARGS__); break;           \
    case 24: FN<2, 4>(__VA_ARGS__); break;           \
    case 31: FN<3, 1>(__VA_ARGS__); break;           \
    case 32: FN<3, 2>(__VA_ARGS__); break;           \
    case 33: FN<3, 3>(__VA_ARGS__); break;           \
    case 34: FN<3, 4>(__VA_ARGS__); break;           \
    default: break;                                  \
  }

}  // namespace

// variable-degree elastic path (vardeg.cu)
hdg_status vd_setup(hdg_ctx* c, const int32_t* elem_k);
// least-squares initial guess around a stage solve (api.cu); both are no-ops when disabled
hdg_status guess_setup(hdg_ctx* c, const uint8_t* host_mask);
void guess_clear(hdg_ctx* c);
hdg_status guess_before(hdg_ctx* c);
hdg_status guess_after(hdg_ctx* c);
hdg_status guess_before_v(hdg_ctx* c, int64_t n, const double* b, double* x, const uint8_t* mask);
hdg_status guess_after_v(hdg_ctx* c, int64_t n, const double* b, const double* x);
void guess_reset_column(hdg_ctx* c, int j);
hdg_status vd_condense(hdg_ctx* c, double alpha);
hdg_status vd_stage_solve(hdg_ctx* c, const double* hist, double tt, double* uout, hdg_solve_info* info);
// one DIRK(3,3) step of a per-element-degree context as one graph launch (nullptr: not possible
// yet, the caller steps through the launches); hc[i] = history weights of stage i on (u, U_0,
// U_1), uc = update weights on (u, U_0, U_1, U_2)
hdg_status vd_dirk3_step_graph(hdg_ctx* c, const double hc[3][3], const double uc[4], hdg_solve_info* info,
                               bool* done);
hdg_status vd_trace_apply(hdg_ctx* c, const double* x, double* y);
hdg_status vd_condensed_rhs(hdg_ctx* c, const double* F, const double* lamD, double* r);
hdg_status vd_trace_solve(hdg_ctx* c, const double* r, double* lam, hdg_solve_info* info);
hdg_status vd_recover(hdg_ctx* c, const double* F, const double* lam, double* u);
hdg_status vd_quadrature_points(hdg_ctx* c, int32_t which, double* xyz);
hdg_status vd_project_volume(hdg_ctx* c, const double* vals, double* u);
hdg_status vd_get_tuning(const hdg_ctx* c, hdg_tuning* out);
void vd_destroy(hdg_ctx* c);
// nonlinear elastodynamics (svk.cu)
hdg_status svk_setup(hdg_ctx* c);
hdg_status svk_step(hdg_ctx* c, double dt, hdg_scheme scheme, int32_t nsteps, hdg_solve_info* info);
void svk_destroy(hdg_ctx* c);
// block ILU(0) (bilu.cu)
hdg_status bilu_setup(hdg_ctx* c);
hdg_status bilu_factor(hdg_ctx* c);
hdg_status bilu_apply(hdg_ctx* c, const double* in, double* out);
void bilu_destroy(hdg_ctx* c);
// api.cu: the context's trace solve (CG on the assembled S_K, device- or host-driven) and the
// DIRK(3,3) tableau
hdg_status trace_cg_solve(hdg_ctx* c, const double* b, double* x, hdg_solve_info* info);
void dirk3_tableau(double a[3][3], double b[3], double cc[3]);
