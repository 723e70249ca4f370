// Nonlinear (Saint Venant-Kirchhoff) elastodynamics, Sec. 4.4: set-up of the reference tables,
// the Newton loop of one implicit stage (condense -> trace solve -> recover, every iteration)
// and the DIRK(3,3) step of Sec. 2.3 around it. The element kernels are in svk.cuh; the trace
// system of each Newton iteration is the uniform elastic one (3 N_f unknowns per face, S_K
// symmetric positive definite) and goes through the context's CG.
#include <cmath>
#include <cstring>

#include "ctx.cuh"
#include "elastic.cuh"
#include "svk.cuh"

using namespace hdg;

struct Svk {
  double* d_tab = nullptr;
  float* d_tabf = nullptr;
  SvkTabs tabs{};
  SvkJT<double> tjd{};     // Jacobian-rule tables, FP64 and FP32 copies
  SvkJT<float> tjf{};
  bool fp32_jacobian = false;
  int nqr = 0, nqj = 0;
  double *d_L = nullptr, *d_zR = nullptr, *d_dl = nullptr, *d_b = nullptr;
  unsigned long long* d_umax = nullptr;   // [0] max |du|, [1] max |u|, [2] max |dlam|
  unsigned long long* h_umax = nullptr;   // pinned copy, followed by the error flag
  int* d_err = nullptr;
  // traction faces: per boundary face 1 = traction data (its traces are unknowns)
  std::vector<uint8_t> neu;
  uint8_t* d_neu = nullptr;
  int32_t* d_face_slot0 = nullptr;        // skeleton face slots (the owning element of each face)
  bool any_neu = false;
  // forcing: host buffers filled by the callback before each stage, and their device copies
  hdg_svk_forcing fn = nullptr;
  void* user = nullptr;
  double *h_f = nullptr, *h_g = nullptr, *d_f = nullptr, *d_g = nullptr;
  std::vector<int32_t> newton;            // Newton iterations per stage of the last hdg_step
};

namespace {

template <int K>
hdg_status svk_tables(hdg_ctx* c, Svk* v) {
  using D = SvkDims<K>;
  constexpr int NP = D::NP, NFP = D::NFP;
  const RefTables& T = c->T;
  std::vector<double> pr, wr, pj, wj;
  simplex_rule(3, D::QR, pr, wr);
  simplex_rule(3, D::QJ, pj, wj);
  std::vector<double> phiR((size_t)D::NQR * NP), phiJ((size_t)D::NQJ * NP);
  dubiner(3, K, pr.data(), D::NQR, phiR.data(), nullptr);
  dubiner(3, K, pj.data(), D::NQJ, phiJ.data(), nullptr);
  std::vector<double> GJ((size_t)D::NQJ * 3 * NP), PSJ((size_t)D::NQJ * 4 * NFP);
  for (int q = 0; q < D::NQJ; ++q) {
    for (int r = 0; r < 3; ++r)
      for (int a = 0; a < NP; ++a) {
        double s = 0.0;
        for (int b = 0; b < NP; ++b) s += T.Dr[((size_t)r * NP + a) * NP + b] * phiJ[(size_t)q * NP + b];
        GJ[((size_t)q * 3 + r) * NP + a] = s;
      }
    for (int f = 0; f < 4; ++f)
      for (int m = 0; m < NFP; ++m) {
        double s = 0.0;
        for (int a = 0; a < NP; ++a) s += T.Ff[((size_t)f * NP + a) * NFP + m] * phiJ[(size_t)q * NP + a];
        PSJ[((size_t)q * 4 + f) * NFP + m] = s;
      }
  }
  std::vector<double> tab;
  size_t off[11];
  const std::vector<double>* parts[11] = {&T.Dr, &T.Ff, &T.Ef, &phiR, &wr, &T.qf_mu, &T.qf_w, &phiJ, &wj, &GJ, &PSJ};
  for (int i = 0; i < 11; ++i) { off[i] = tab.size(); tab.insert(tab.end(), parts[i]->begin(), parts[i]->end()); }
  std::vector<float> tabf(tab.begin() + off[7], tab.end());
  hdg_status s;
  if ((s = dalloc(c, &v->d_tab, tab.size()))) return s;
  if ((s = dalloc(c, &v->d_tabf, tabf.size()))) return s;
  CUDA_TRY(c, cudaMemcpyAsync(v->d_tab, tab.data(), tab.size() * 8, cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(v->d_tabf, tabf.data(), tabf.size() * 4, cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  const double* b = v->d_tab;
  const float* bf = v->d_tabf - off[7];   // same offsets as the FP64 buffer
  v->tabs = SvkTabs{b + off[0], b + off[1], b + off[2], b + off[3], b + off[4], b + off[5], b + off[6], T.nqf};
  v->tjd = SvkJT<double>{b + off[7], b + off[8], b + off[9], b + off[10]};
  v->tjf = SvkJT<float>{bf + off[7], bf + off[8], bf + off[9], bf + off[10]};
  v->nqr = D::NQR;
  v->nqj = D::NQJ;
  CUDA_TRY(c, cudaFuncSetAttribute(svk_condense_kernel<K, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)D::template cond_bytes<double>()));
  CUDA_TRY(c, cudaFuncSetAttribute(svk_recover_kernel<K, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)D::template rec_bytes<double>()));
  CUDA_TRY(c, cudaFuncSetAttribute(svk_condense_kernel<K, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)D::template cond_bytes<float>()));
  CUDA_TRY(c, cudaFuncSetAttribute(svk_recover_kernel<K, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)D::template rec_bytes<float>()));
  return HDG_OK;
}

template <int K>
void svk_launch_condense(hdg_ctx* c, const SvkArgs& a) {
  using D = SvkDims<K>;
  c->n_launch += 1;
  cudaEvent_t stop = apply_begin(c, 4);
  const Svk* v = c->svk;
  if (v->fp32_jacobian)
    svk_condense_kernel<K, float><<<(unsigned)c->sk.ne, D::NT, D::template cond_bytes<float>(), c->stream>>>(
        a, v->tabs, v->tjf);
  else
    svk_condense_kernel<K, double><<<(unsigned)c->sk.ne, D::NT, D::template cond_bytes<double>(), c->stream>>>(
        a, v->tabs, v->tjd);
  apply_end(c, stop);
}

template <int K>
void svk_launch_recover(hdg_ctx* c, const SvkRecArgs& a) {
  using D = SvkDims<K>;
  c->n_launch += 1;
  cudaEvent_t stop = apply_begin(c, 5);
  const Svk* v = c->svk;
  if (v->fp32_jacobian)
    svk_recover_kernel<K, float><<<(unsigned)c->sk.ne, D::NT, D::template rec_bytes<float>(), c->stream>>>(
        a, v->tabs, v->tjf);
  else
    svk_recover_kernel<K, double><<<(unsigned)c->sk.ne, D::NT, D::template rec_bytes<double>(), c->stream>>>(
        a, v->tabs, v->tjd);
  apply_end(c, stop);
}

#define SVK_DISPATCH(c, FN, ...)          \
  switch ((c)->k) {                       \
    case 1: FN<1>(__VA_ARGS__); break;    \
    case 2: FN<2>(__VA_ARGS__); break;    \
    case 3: FN<3>(__VA_ARGS__); break;    \
    default: break;                       \
  }

// device face arrays of the trace solve: traction faces carry unknowns (face_bnd -1) and
// their missing second slot is the zero sentinel past the last element slot
hdg_status svk_upload_faces(hdg_ctx* c) {
  Svk* v = c->svk;
  const int64_t nf = c->sk.nf, ne = c->sk.ne;
  std::vector<int32_t> slot(c->sk.face_slot), bnd(c->sk.face_bnd);
  std::vector<uint8_t> mask((size_t)c->ntr);
  for (int64_t b = 0; b < c->sk.nb; ++b)
    if (v->neu[b]) {
      const int64_t f = c->sk.bnd_faces[b];
      bnd[f] = -1;
      slot[2 * f + 1] = (int32_t)(ne * 4);
    }
  for (int64_t f = 0; f < nf; ++f)
    for (int mm = 0; mm < c->Nf; ++mm) mask[(size_t)f * c->Nf + mm] = bnd[f] < 0 ? 1 : 0;
  CUDA_TRY(c, cudaMemcpyAsync(c->d_face_slot, slot.data(), slot.size() * 4, cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(c->d_face_bnd, bnd.data(), bnd.size() * 4, cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(c->d_intmask, mask.data(), mask.size(), cudaMemcpyHostToDevice, c->stream));
  if (c->sk.nb) CUDA_TRY(c, cudaMemcpyAsync(v->d_neu, v->neu.data(), v->neu.size(), cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return HDG_OK;
}

// Newton's method for one stage (Sec. 4.4): from the iterate (u, c->d_lam) until the largest
// increment is at most newton_tol * max(1, max |u|)
hdg_status svk_newton(hdg_ctx* c, double* u, const double* h, double alpha, double t, hdg_solve_info* si) {
  Svk* v = c->svk;
  const int64_t ne = c->sk.ne, nf = c->sk.nf, nfe = nf * c->Nf;
  // forcing of this stage time
  if (v->fn) {
    const size_t nfv = (size_t)ne * v->nqr * 3, ngv = (size_t)c->sk.nb * c->T.nqf * 3;
    std::memset(v->h_f, 0, nfv * 8);
    if (ngv) std::memset(v->h_g, 0, ngv * 8);
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));   // the previous stage's uploads are done
    if (v->fn(v->user, t, v->h_f, v->h_g) != 0) return fail(c, HDG_EINVAL, "SVK forcing callback reported an error");
    CUDA_TRY(c, cudaMemcpyAsync(v->d_f, v->h_f, nfv * 8, cudaMemcpyHostToDevice, c->stream));
    if (ngv) CUDA_TRY(c, cudaMemcpyAsync(v->d_g, v->h_g, ngv * 8, cudaMemcpyHostToDevice, c->stream));
  }
  c->alpha = alpha;
  c->condensed = true;
  CUDA_TRY(c, cudaMemsetAsync(v->d_err, 0, sizeof(int), c->stream));
  SvkArgs ca{ne, c->d_geo, c->d_rho, c->d_lame, c->d_mue, c->d_elem_face, c->d_face_bnd, alpha, u, c->d_lam, h,
             v->fn ? v->d_f : nullptr, c->d_S, v->d_L, v->d_zR, c->d_slot, v->d_err};
  SvkRecArgs ra{ne, c->d_geo, c->d_rho, c->d_lame, c->d_mue, c->d_elem_face, c->d_face_bnd, alpha, u, v->d_dl,
                v->d_L, v->d_zR, v->d_umax};
  const int maxit = c->opt.newton_maxit;
  for (int it = 1; it <= maxit; ++it) {
    CUDA_TRY(c, cudaMemsetAsync(v->d_umax, 0, 3 * sizeof(unsigned long long), c->stream));
    SVK_DISPATCH(c, svk_launch_condense, c, ca);
    c->n_launch += 2;
    face_gather_kernel<<<grid_for(c, nfe), 256, 0, c->stream>>>(nf, c->Nf, c->d_face_slot, c->d_face_bnd, c->d_slot, 1.0,
                                                                v->d_b);
    if (v->fn && v->any_neu) {
      c->n_launch += 1;
      svk_traction_kernel<<<grid_for(c, c->sk.nb * c->Nf), 256, 0, c->stream>>>(
          c->sk.nb, c->T.Nf, c->d_bnd_faces, v->d_face_slot0, v->d_neu, c->d_geo, v->d_g, v->tabs.muF, v->tabs.wF,
          c->T.nqf, v->d_b);
    }
    svk_diag_kernel<<<grid_for(c, nfe), 256, 0, c->stream>>>(nf, c->Nf, c->m, ne * 4, c->d_face_slot, c->d_face_bnd,
                                                            c->d_S, c->d_dinv);
    if (c->opt.prec != HDG_FP64) {
      // FP32 copies of S_K and of the Jacobi diagonal for the inner CG of the refined solve
      const int64_t nS = ne * (int64_t)c->m * c->m;
      c->n_launch += 2;
      to32_copy_kernel<<<grid_for(c, nS), 256, 0, c->stream>>>(nS, c->d_S, c->d_S32);
      to32_kernel<<<grid_for(c, nfe), 256, 0, c->stream>>>(nfe, c->d_dinv, c->d_dinv32);
    }
    CUDA_TRY(c, cudaMemsetAsync(v->d_dl, 0, nfe * 8, c->stream));
    hdg_status s = check_launch(c, "svk_condense");
    if (s) return s;
    hdg_solve_info li{};
    if ((s = trace_cg_solve(c, v->d_b, v->d_dl, &li))) return s;
    si->iterations += li.iterations;
    si->rel_residual = std::max(si->rel_residual, li.rel_residual);
    SVK_DISPATCH(c, svk_launch_recover, c, ra);
    c->n_launch += 1;
    svk_trace_update_kernel<<<grid_for(c, nfe), 256, 0, c->stream>>>(nf, c->Nf, c->d_face_bnd, v->d_dl, c->d_lam,
                                                                     v->d_umax + 2);
    if ((s = check_launch(c, "svk_recover"))) return s;
    CUDA_TRY(c, cudaMemcpyAsync(v->h_umax, v->d_umax, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(v->h_umax + 3, v->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (*reinterpret_cast<const int*>(v->h_umax + 3))
      return fail(c, HDG_EINVAL, "SVK: the velocity block S_v of an element is not positive definite "
                                 "(the tangent lost ellipticity)");
    double du, um, dl;
    std::memcpy(&du, v->h_umax, 8);
    std::memcpy(&um, v->h_umax + 1, 8);
    std::memcpy(&dl, v->h_umax + 2, 8);
    const double step = std::max(du, dl), scale = std::max(1.0, um);
    si->sweeps += 1;
    if (step <= c->opt.newton_tol * scale) {
      v->newton.push_back(it);
      return HDG_OK;
    }
  }
  return fail(c, HDG_ENOCONV, "SVK Newton iteration reached newton_maxit=" + std::to_string(maxit));
}

}  // namespace

hdg_status svk_setup(hdg_ctx* c) {
  Svk* v = new (std::nothrow) Svk();
  if (!v) return fail(c, HDG_ENOMEM, "out of host memory");
  c->svk = v;
  v->fp32_jacobian = c->svk_mixed;
  hdg_status s;
  switch (c->k) {
    case 1: s = svk_tables<1>(c, v); break;
    case 2: s = svk_tables<2>(c, v); break;
    case 3: s = svk_tables<3>(c, v); break;
    default: return fail(c, HDG_EINVAL, "SVK: degree k must be in 1..3");
  }
  if (s) return s;
  const int64_t ne = c->sk.ne, nfe = c->sk.nf * c->Nf;
  const int NV = 3 * c->Np;
  if ((s = dalloc(c, &v->d_L, (size_t)ne * NV * NV))) return s;
  if ((s = dalloc(c, &v->d_zR, (size_t)ne * c->n))) return s;
  if ((s = dalloc(c, &v->d_dl, (size_t)nfe))) return s;
  if ((s = dalloc(c, &v->d_b, (size_t)nfe))) return s;
  if ((s = dalloc(c, &v->d_umax, 3))) return s;
  if ((s = dalloc(c, &v->d_err, 1))) return s;
  if ((s = dalloc(c, &v->d_neu, (size_t)std::max<int64_t>(c->sk.nb, 1)))) return s;
  if ((s = dalloc(c, &v->d_face_slot0, c->sk.face_slot.size()))) return s;
  CUDA_TRY(c, cudaMallocHost((void**)&v->h_umax, 4 * sizeof(unsigned long long)));
  CUDA_TRY(c, cudaMemsetAsync(v->d_err, 0, sizeof(int), c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(v->d_face_slot0, c->sk.face_slot.data(), c->sk.face_slot.size() * 4, cudaMemcpyHostToDevice,
                              c->stream));
  v->neu.assign((size_t)c->sk.nb, 0);
  return svk_upload_faces(c);
}

void svk_destroy(hdg_ctx* c) {
  Svk* v = c->svk;
  if (!v) return;
  if (v->h_umax) cudaFreeHost(v->h_umax);
  if (v->h_f) cudaFreeHost(v->h_f);
  if (v->h_g) cudaFreeHost(v->h_g);
  delete v;
  c->svk = nullptr;
}

hdg_status svk_step(hdg_ctx* c, double dt, hdg_scheme scheme, int32_t nsteps, hdg_solve_info* info) {
  if (scheme != HDG_DIRK3) return fail(c, HDG_EINVAL, "SVK: hdg_step supports HDG_DIRK3 only");
  Svk* v = c->svk;
  double a[3][3], b[3], cc[3];
  dirk3_tableau(a, b, cc);
  double d[3][3] = {};
  for (int i = 0; i < 3; ++i) {
    d[i][i] = 1.0 / a[i][i];
    for (int j = 0; j < i; ++j) {
      double sum = 0.0;
      for (int q = j; q < i; ++q) sum += a[i][q] * d[q][j];
      d[i][j] = -sum / a[i][i];
    }
  }
  v->newton.clear();
  hdg_solve_info si{};
  const int64_t n = c->nfld;
  for (int32_t step = 0; step < nsteps; ++step) {
    const double tn = c->t;
    for (int i = 0; i < 3; ++i) {
      // stage i: alpha = d_ii / dt, h = [(sum_{j<=i} d_ij) u^n - sum_{j<i} d_ij U_j] / d_ii (Eq. 10_1);
      // Newton starts from the previous stage (u^n for the first) and the current traces
      double cu = 0.0;
      for (int j = 0; j <= i; ++j) cu += d[i][j];
      const double* in[2] = {nullptr, nullptr};
      double co[2] = {0, 0};
      for (int j = 0; j < i; ++j) { in[j] = c->d_stage[j]; co[j] = -d[i][j] / d[i][i]; }
      c->n_launch += 1;
      combine_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(n, cu / d[i][i], c->d_u, co[0], in[0], co[1], in[1], 0.0,
                                                            nullptr, c->d_h);
      CUDA_TRY(c, cudaMemcpyAsync(c->d_stage[i], i == 0 ? c->d_u : c->d_stage[i - 1], (size_t)n * 8,
                                  cudaMemcpyDeviceToDevice, c->stream));
      hdg_status s = svk_newton(c, c->d_stage[i], c->d_h, d[i][i] / dt, tn + cc[i] * dt, &si);
      if (s) return s;
    }
    // stiffly accurate: u^{n+1} is the last stage
    std::swap(c->d_uprev, c->d_u);
    std::swap(c->d_u, c->d_stage[2]);
    c->t = tn + dt;
  }
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (info) *info = si;
  return HDG_OK;
}

extern "C" {

hdg_status hdg_svk_set_traction_faces(hdg_ctx* c, const uint8_t* mask) {
  if (!c) return HDG_EINVAL;
  if (!c->svk) return fail(c, HDG_EINVAL, "not an SVK context");
  Svk* v = c->svk;
  v->any_neu = false;
  for (int64_t b = 0; b < c->sk.nb; ++b) {
    v->neu[b] = mask && mask[b] ? 1 : 0;
    v->any_neu = v->any_neu || v->neu[b];
  }
  return svk_upload_faces(c);
}

hdg_status hdg_svk_set_forcing(hdg_ctx* c, hdg_svk_forcing fn, void* user) {
  if (!c) return HDG_EINVAL;
  if (!c->svk) return fail(c, HDG_EINVAL, "not an SVK context");
  Svk* v = c->svk;
  v->fn = fn;
  v->user = user;
  if (fn && !v->h_f) {
    const size_t nfv = (size_t)c->sk.ne * v->nqr * 3, ngv = (size_t)std::max<int64_t>(c->sk.nb, 1) * c->T.nqf * 3;
    CUDA_TRY(c, cudaMallocHost((void**)&v->h_f, nfv * 8));
    CUDA_TRY(c, cudaMallocHost((void**)&v->h_g, ngv * 8));
    hdg_status s;
    if ((s = dalloc(c, &v->d_f, nfv))) return s;
    if ((s = dalloc(c, &v->d_g, ngv))) return s;
  }
  return HDG_OK;
}

hdg_status hdg_svk_newton_counts(const hdg_ctx* c, int32_t* out, int32_t cap, int32_t* count) {
  if (!c || !c->svk || !count) return HDG_EINVAL;
  const int32_t n = (int32_t)c->svk->newton.size();
  *count = n;
  for (int32_t i = 0; out && i < std::min(n, cap); ++i) out[i] = c->svk->newton[i];
  return HDG_OK;
}

}  // extern "C"
