// C ABI of the HDG library: context, memory, dispatch and the time-step driver.
// The steps follow Sec. 2.3 (BDF, Eq. ch5appendx1:eq9b; DIRK, Eqs. ch5appendx1:eq10_1-2)
// and Sec. 2.4 (static condensation, Eq. LS) of arXiv 1807.00086.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/hdg.h"
#include "kernels.cuh"
#include "post.cuh"
#include "dflocal.cuh"
#include "multi.cuh"
#include "elastic.cuh"
#include "edg.cuh"
#include "gmres.cuh"
#include "bilu.cuh"
#include "mesh.h"
#include "reftab.h"

using namespace hdg;

#include "ctx.cuh"

namespace {

template <int DIM, int K>
void launch_condense(hdg_ctx* c) {
  constexpr int NT = 128;
  c->n_launch += 2;
  if (c->phys == HDG_ELASTIC) {
    const size_t smem = CondElCfg<DIM, K>::SMEM;
    cudaFuncSetAttribute(condense_el_kernel<DIM, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    condense_el_kernel<DIM, K><<<(unsigned)c->sk.ne, 256, smem, c->stream>>>(devmesh(c), c->tabs, c->d_lame, c->d_mue,
                                                                            c->alpha, c->d_S, c->d_Hinv, c->d_err);
    diag_kernel<ElDims<DIM, K>><<<grid_for(c, c->sk.nf * c->Nf), 256, 0, c->stream>>>(devmesh(c), c->d_S, c->sgn, c->d_dinv);
    return;
  }
  condense_kernel<DIM, K, NT><<<(unsigned)c->sk.ne, NT, 0, c->stream>>>(devmesh(c), c->tabs, c->alpha, c->tau, c->d_S,
                                                                       c->d_Hinv, c->d_err);
  diag_kernel<Dims<DIM, K>><<<grid_for(c, c->sk.nf * c->Nf), 256, 0, c->stream>>>(devmesh(c), c->d_S, c->sgn, c->d_dinv);
}

template <int DIM, int K>
void launch_local(hdg_ctx* c, int mode, const double* F, const double* hist, double t, const double* lam, double* out) {
  if (c->phys == HDG_ELASTIC) {
    c->n_launch += 1;
    if (mode == 0)
      local_el_kernel<DIM, K, 0><<<(unsigned)c->sk.ne, 128, 0, c->stream>>>(devmesh(c), c->tabs, c->d_lame, c->d_mue,
                                                                            c->d_Hinv, c->alpha, F, hist, lam, out);
    else
      local_el_kernel<DIM, K, 1><<<(unsigned)c->sk.ne, 128, 0, c->stream>>>(devmesh(c), c->tabs, c->d_lame, c->d_mue,
                                                                            c->d_Hinv, c->alpha, F, hist, lam, out);
    return;
  }
  const SrcArgs sa = srcargs(c, t);
  c->n_launch += 1;
  if (c->d_Hinvdf) {
    using LD = LocalDfCfg<DIM, K>;
    const unsigned gd = (unsigned)((c->sk.ne + LD::EPB - 1) / LD::EPB);
    const float th = (float)c->tau;
    const df2 tau{th, (float)(c->tau - (double)th)};
    if (mode == 0)
      local_df_kernel<DIM, K, 0><<<gd, LD::NT, 0, c->stream>>>(devmesh(c), c->tabsdf, c->d_geodf, c->d_Hinvdf, c->alpha,
                                                               tau, F, hist, sa, lam, out);
    else
      local_df_kernel<DIM, K, 1><<<gd, LD::NT, 0, c->stream>>>(devmesh(c), c->tabsdf, c->d_geodf, c->d_Hinvdf, c->alpha,
                                                               tau, F, hist, sa, lam, out);
    return;
  }
  using L = LocalCfg<DIM, K>;
  const unsigned grid = (unsigned)((c->sk.ne + L::EPB - 1) / L::EPB);
  if (mode == 0)
    local_kernel<DIM, K, 0><<<grid, L::NT, 0, c->stream>>>(devmesh(c), c->tabs, c->d_Hinv, c->alpha, c->tau, F, hist, sa, lam,
                                                            out);
  else
    local_kernel<DIM, K, 1><<<grid, L::NT, 0, c->stream>>>(devmesh(c), c->tabs, c->d_Hinv, c->alpha, c->tau, F, hist, sa, lam,
                                                            out);
}

template <class L>
void launch_apply_l(hdg_ctx* c, const double* x, double* zslot, const int* done, int iter) {
  using C = ApplyCfg<L>;
  const unsigned grid = (unsigned)((c->sk.ne + C::EPB - 1) / C::EPB);
  c->n_launch += 1;
  cudaEvent_t stop = apply_begin(c, 0, iter);
  apply_kernel<L><<<grid, C::NT, 0, c->stream>>>(devmesh(c), c->d_S, x, zslot, done);
  apply_end(c, stop);
}

template <int DIM, int K>
void launch_apply(hdg_ctx* c, const double* x, double* zslot, const int* done, int iter = -1) {
  if (c->phys == HDG_ELASTIC) launch_apply_l<ElDims<DIM, K>>(c, x, zslot, done, iter);
  else launch_apply_l<Dims<DIM, K>>(c, x, zslot, done, iter);
}

template <int DIM, int K>
void launch_pack32(hdg_ctx* c) {
  using PK = Packed<DIM, K>;
  const int64_t n = ((c->sk.ne + 31) / 32) * PK::P4 * 128;
  c->n_launch += 1;
  pack32_kernel<DIM, K><<<grid_for(c, n), 256, 0, c->stream>>>(c->sk.ne, c->d_S, c->d_S32);
}

template <int DIM, int K>
void launch_face_q64(hdg_ctx* c) {
  if (c->phys == HDG_ELASTIC)
    cg_face_q_kernel<ElDims<DIM, K>><<<c->nb_red, 256, 0, c->stream>>>((int)c->sk.nf, c->sgn, c->d_face_slot, c->d_face_bnd,
                                                                       c->d_slot, c->d_p, c->d_q, c->d_part, c->d_sc);
  else
    cg_face_q_kernel<Dims<DIM, K>><<<c->nb_red, 256, 0, c->stream>>>((int)c->sk.nf, c->sgn, c->d_face_slot, c->d_face_bnd,
                                                                     c->d_slot, c->d_p, c->d_q, c->d_part, c->d_sc);
}

// zero the device-side launch timers (start stamps to the maximum, so the first CTA lowers them)
hdg_status reset_dev_timing(hdg_ctx* c) {
  const DevTiming z[2] = {{~0ull, 0, 0.0}, {~0ull, 0, 0.0}};
  CUDA_TRY(c, cudaMemcpyAsync(c->d_dtime, z, sizeof(z), cudaMemcpyHostToDevice, c->stream));
  return cudaStreamSynchronize(c->stream) == cudaSuccess ? HDG_OK : HDG_ECUDA;
}

// p.q reduction target of the single-column FP32/FP16 applies, with the launch-timing slot
PqOut pq_out(hdg_ctx* c, DevTiming* timing) { return PqOut{c->d_pqpart, c->d_ticket, c->d_pq, (float)c->sgn, timing}; }

template <int DIM, int K>
void launch_update_f32(hdg_ctx* c, int par) {
  cg32_update_f_kernel<Dims<DIM, K>><<<c->nb_red, 256, 0, c->stream>>>(
      c->nfe4 / 4, c->sk.nf * c->Nf, (float)c->sgn, par, c->d_face_slot, c->d_face_bnd, c->d_slot32,
      (const float4*)c->d_p32, (const float4*)c->d_dinv32, (float4*)c->d_x32, (float4*)c->d_r32, (float4*)c->d_z32,
      c->d_pq, c->d_part + c->nb_red, c->d_sc);
}

template <int DIM, int K>
void launch_face_q32(hdg_ctx* c) {
  if (c->phys == HDG_ELASTIC)
    cg32_face_q_kernel<ElDims<DIM, K>><<<c->nb_red, 256, 0, c->stream>>>((int)c->sk.nf, (float)c->sgn, c->d_face_slot,
                                                                         c->d_face_bnd, c->d_slot32, c->d_p32, c->d_q32,
                                                                         c->d_part, c->d_sc);
  else
    cg32_face_q_kernel<Dims<DIM, K>><<<c->nb_red, 256, 0, c->stream>>>((int)c->sk.nf, (float)c->sgn, c->d_face_slot,
                                                                       c->d_face_bnd, c->d_slot32, c->d_p32, c->d_q32,
                                                                       c->d_part, c->d_sc);
}

template <int DIM, int K>
void launch_packdf(hdg_ctx* c) {
  using PK = Packed<DIM, K>;
  const int64_t n = c->sk.ne * PK::P4 * 4;
  c->n_launch += 1;
  packdf_kernel<DIM, K><<<grid_for(c, n), 256, 0, c->stream>>>(c->sk.ne, c->d_S, c->d_Sdf);
}

template <int DIM, int K>
void launch_pack16(hdg_ctx* c) {
  using PK = Packed16<DIM, K>;
  const int64_t ne = c->sk.ne;
  c->n_launch += 2;
  scale16_kernel<DIM, K><<<grid_for(c, ne * 32), 256, 0, c->stream>>>(ne, c->d_S, c->d_sc16);
  pack16_kernel<DIM, K><<<grid_for(c, ((ne + 31) / 32) * PK::P8 * 256), 256, 0, c->stream>>>(ne, c->d_S, c->d_sc16,
                                                                                               c->d_S16);
  using C = Apply16Cfg<DIM, K>;
  const int64_t ng = ((ne + 31) / 32) * 32 * Dims<DIM, K>::NFC;
  c->n_launch += 1;
  gface_kernel<<<grid_for(c, ng), 256, 0, c->stream>>>(ng, ne * Dims<DIM, K>::NFC, c->d_elem_face, c->d_face_bnd,
                                                       c->d_gface16);
  cudaFuncSetAttribute(apply16_kernel<DIM, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
  int per_sm = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, apply16_kernel<DIM, K>, 32 * C::WARPS, C::SMEM) !=
          cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  c->a16_per_sm = per_sm;
}

template <int DIM, int K>
void launch_apply16(hdg_ctx* c, const float* x, float* slot, const int* done, int iter) {
  const int64_t ngroups = (c->sk.ne + 31) / 32;
  c->n_launch += 1;
  cudaEvent_t stop = apply_begin(c, 3, iter);
  using C = Apply16Cfg<DIM, K>;
  const unsigned grid = (unsigned)std::max<int64_t>(
      1, std::min<int64_t>((ngroups + C::WARPS - 1) / C::WARPS, (int64_t)c->sms * std::max(1, c->a16_per_sm)));
  apply16_kernel<DIM, K><<<grid, 32 * C::WARPS, C::SMEM, c->stream>>>(c->sk.ne, c->d_gface16, c->d_S16, c->d_sc16, x,
                                                                      slot, done, pq_out(c, c->d_dtime + 1));
  apply_end(c, stop);
}

template <int DIM, int K>
void launch_apply_df(hdg_ctx* c, const double* x, double* zslot, const int* skip = nullptr) {
  using C = ApplyDfCfg<DIM, K>;
  const int64_t ngroups = (c->sk.ne + C::EPB - 1) / C::EPB;
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ngroups, (int64_t)c->sms * std::max(1, c->df_per_sm)));
  c->n_launch += 1;
  cudaEvent_t stop = apply_begin(c, 2, -1);
  apply_df_kernel<DIM, K><<<grid, C::NT, C::SMEM, c->stream>>>(devmesh(c), c->d_Sdf, x, zslot, ngroups, skip);
  apply_end(c, stop);
}

// dynamic shared memory and resident CTAs per SM of the double-float apply (set outside any
// stream capture; the persistent grid is one resident wave)
template <int DIM, int K>
void attr_apply_df(hdg_ctx* c) {
  using C = ApplyDfCfg<DIM, K>;
  cudaFuncSetAttribute(apply_df_kernel<DIM, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
  int per_sm = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, apply_df_kernel<DIM, K>, C::NT, C::SMEM) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  c->df_per_sm = per_sm;
}

// dynamic shared memory of the tensor-core column-block apply (set outside any stream capture)
template <int DIM, int K>
void attr_apply_tc(hdg_ctx* c) {
  using CP = ApplyTcPCfg<DIM, K>;
  cudaFuncSetAttribute(apply_tc_kernel<DIM, K, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ApplyTcCfg<DIM, K>::SMEM);
  cudaFuncSetAttribute(apply_tc_kernel<DIM, K, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ApplyTcCfg<DIM, K>::SMEM);
  cudaFuncSetAttribute(apply_tc_pq_kernel<DIM, K, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CP::SMEM);
  cudaFuncSetAttribute(apply_tc_pq_kernel<DIM, K, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CP::SMEM);
  int per_sm = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, apply_tc_pq_kernel<DIM, K, 64>, 32 * CP::WPB, CP::SMEM) !=
          cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  c->tcp_per_sm = per_sm;
}

template <int DIM, int K>
void launch_pack32m(hdg_ctx* c) {
  using PK = Packed<DIM, K>;
  const int64_t n = c->sk.ne * PK::P4 * 4;
  c->n_launch += 1;
  pack32m_kernel<DIM, K><<<grid_for(c, n), 256, 0, c->stream>>>(c->sk.ne, c->d_S, c->d_S32);
}

template <int DIM, int K>
void launch_apply32(hdg_ctx* c, const float* x, float* slot, const int* done, int iter) {
  const int64_t ngroups = (c->sk.ne + 31) / 32;
  c->n_launch += 1;
  cudaEvent_t stop = apply_begin(c, 1, iter);
  if (c->phys == HDG_ELASTIC) {
    apply32f_kernel<ElDims<DIM, K>><<<(unsigned)((c->sk.ne + 3) / 4), 128, 0, c->stream>>>(
        c->sk.ne, c->d_elem_face, c->d_face_bnd, c->d_S32, x, slot, done);
    apply_end(c, stop);
    return;
  }
  apply32_kernel<DIM, K><<<(unsigned)((ngroups + 3) / 4), 128, 0, c->stream>>>(c->sk.ne, c->d_elem_face, c->d_face_bnd,
                                                                              c->d_S32, x, slot, done,
                                                                              pq_out(c, c->d_dtime));
  apply_end(c, stop);
}

// ---- continuous traces (IEDG / EDG): expansion lam = R mu and restriction R^T (face weights)
template <int DIM, int K>
void edg_expand64(hdg_ctx* c, const double* mu, double* lam, int zero_bnd) {
  constexpr int NF = Dims<DIM, K>::NF;
  c->n_launch += 1;
  edg_expand_kernel<double, NF><<<grid_for(c, c->sk.nf), 256, 0, c->stream>>>(c->sk.nf, c->d_face_bnd, c->d_face_node,
                                                                              c->d_vinv, mu, lam, zero_bnd);
}

template <int DIM, int K>
void edg_expand32(hdg_ctx* c, const float* mu, float* lam) {
  constexpr int NF = Dims<DIM, K>::NF;
  c->n_launch += 1;
  edg_expand_kernel<float, NF><<<grid_for(c, c->sk.nf), 256, 0, c->stream>>>(c->sk.nf, c->d_face_bnd, c->d_face_node,
                                                                             c->d_vinv, mu, lam, 1);
}

// face nodal weights from element slots (slot) or from a face array (yface)
template <int DIM, int K>
void edg_face_w64(hdg_ctx* c, const double* slot, const double* yface, double* w) {
  constexpr int NF = Dims<DIM, K>::NF;
  c->n_launch += 1;
  edg_face_w_kernel<double, NF><<<grid_for(c, c->sk.nf), 256, 0, c->stream>>>(c->sk.nf, c->d_face_slot, c->d_face_bnd,
                                                                              c->d_vinv, slot, yface, w);
}

template <int DIM, int K>
void edg_face_w32(hdg_ctx* c, const float* slot, float* w) {
  constexpr int NF = Dims<DIM, K>::NF;
  c->n_launch += 1;
  edg_face_w_kernel<float, NF><<<grid_for(c, c->sk.nf), 256, 0, c->stream>>>(c->sk.nf, c->d_face_slot, c->d_face_bnd,
                                                                             c->d_vinv, slot, nullptr, w);
}

// Jacobi diagonal of R^T K R (sgn convention of the Krylov operator), FP64 and FP32 copies
template <int DIM, int K>
void edg_diag(hdg_ctx* c) {
  using D = Dims<DIM, K>;
  c->n_launch += 2;
  edg_diag_elem_kernel<DIM, D::NF><<<grid_for(c, c->sk.ne * D::M), 256, 0, c->stream>>>(
      c->sk.ne, c->d_elem_face, c->d_face_node, c->d_vinv, c->d_S, c->d_slot);
  edg_diag_node_kernel<<<grid_for(c, c->n_mu), 256, 0, c->stream>>>(c->n_mu, D::NF, c->d_node_ptr, c->d_node_inc,
                                                                    c->d_face_slot, c->d_slot, c->sgn, c->d_dinv,
                                                                    c->d_dinv32);
}

hdg_status do_condense(hdg_ctx* c, double alpha) {
  if (c->svk) return fail(c, HDG_EINVAL, "SVK: the Newton iterations of hdg_step condense; there is no linear condensation");
  guess_clear(c);   // the stored stage solutions belong to the previous operator
  if (c->vd) return vd_condense(c, alpha);
  if (!(alpha > 0.0) || !std::isfinite(alpha)) return fail(c, HDG_EINVAL, "alpha must be positive and finite");
  c->alpha = alpha;
  CUDA_TRY(c, cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
  HDG_DISPATCH(c, launch_condense, c);
  hdg_status s = check_launch(c, "condense");
  if (s) return s;
  if (c->opt.prec != HDG_FP64) {
    if (c->phys == HDG_ELASTIC) {
      const int64_t nS = c->sk.ne * (int64_t)c->m * c->m;
      c->n_launch += 1;
      to32_copy_kernel<<<grid_for(c, nS), 256, 0, c->stream>>>(nS, c->d_S, c->d_S32);
    } else if (c->R > 1) {
      if (c->R >= 32) {
        HDG_DISPATCH(c, launch_pack32m, c);
        HDG_DISPATCH(c, attr_apply_tc, c);
      } else {
        HDG_DISPATCH(c, launch_pack32, c);   // group layout, read by the narrow multi-column apply
      }
      const int64_t nS = c->sk.ne * (int64_t)c->m * c->m;
      c->n_launch += 1;
      split_df_kernel<<<grid_for(c, nS), 256, 0, c->stream>>>(nS, c->d_S, c->d_mShi, c->d_mSlo);
      const int64_t nH = c->sk.ne * (int64_t)c->nv * c->nv;
      c->n_launch += 1;
      to_df_kernel<<<grid_for(c, nH), 256, 0, c->stream>>>(nH, c->d_Hinv, c->d_Hinvdf);
    } else {
      HDG_DISPATCH(c, launch_pack32, c);
      HDG_DISPATCH(c, launch_packdf, c);
      HDG_DISPATCH(c, attr_apply_df, c);
      if (c->d_S16) HDG_DISPATCH(c, launch_pack16, c);
      const int64_t nH = c->sk.ne * (int64_t)c->nv * c->nv;
      c->n_launch += 1;
      to_df_kernel<<<grid_for(c, nH), 256, 0, c->stream>>>(nH, c->d_Hinv, c->d_Hinvdf);
    }
    const int64_t nfe = c->sk.nf * c->Nf;
    c->n_launch += 1;
    to32_kernel<<<grid_for(c, nfe), 256, 0, c->stream>>>(nfe, c->d_dinv, c->d_dinv32);
    if ((s = check_launch(c, "pack32"))) return s;
  }
  if (c->tspace) {
    // the nodal Jacobi diagonal replaces the face one; FP32 padding entries stay zero
    HDG_DISPATCH(c, edg_diag, c);
    if (c->d_dinv32 && c->n_mu4 > c->n_mu)
      CUDA_TRY(c, cudaMemsetAsync(c->d_dinv32 + c->n_mu, 0, (size_t)(c->n_mu4 - c->n_mu) * 4, c->stream));
    if ((s = check_launch(c, "edg_diag"))) return s;
  }
  int herr = 0;
  CUDA_TRY(c, cudaMemcpyAsync(&herr, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (herr) { c->condensed = false; return fail(c, HDG_EINVAL, "local pressure block not positive definite"); }
  c->condensed = true;
  if (c->bilu && (s = bilu_factor(c))) return s;
  return HDG_OK;
}

// b (face array) = sum of gslot over each interior face's two slots
hdg_status faces_from_slots(hdg_ctx* c, double scale, double* out) {
  c->n_launch += 1;
  face_gather_kernel<<<grid_for(c, c->sk.nf * c->Nf), 256, 0, c->stream>>>(c->sk.nf, c->Nf, c->d_face_slot, c->d_face_bnd,
                                                                           c->d_slot, scale, out);
  return check_launch(c, "face_gather");
}

// FP32 PCG on (-K32) x32 = b32 from x32 = 0 (inner solve of the mixed path).
hdg_status cg32_inner(hdg_ctx* c, int* iters, double tol, int* last, bool use16) {
  const int64_t nfe = c->sk.nf * c->Nf;
  const int nb = c->nb_red;
  const int64_t n4 = c->nfe4 / 4;
  c->n_launch += 2;
  cg32_init_kernel<<<nb, 256, 0, c->stream>>>(n4, (const float4*)c->d_b32, (const float4*)c->d_dinv32, (float4*)c->d_x32,
                                              (float4*)c->d_r32, (float4*)c->d_z32, (float4*)c->d_p32, c->d_part);
  cg32_init_scalars<<<1, 256, 0, c->stream>>>(nb, c->d_part, tol, c->d_sc, nullptr);
  hdg_status s = check_launch(c, "cg32_init");
  if (s) return s;
  int it = 0;
  const int maxit = c->opt.maxit;
  const int chk = std::max(1, c->opt.check_every);
  c->h_sc->done = 0;
  const int first = std::max(2, std::min(chk, *last - 1));   // first poll near the last solve's count
  while (!c->h_sc->done && it < maxit) {
    // with statistics on, poll at check_every: a poll idles the GPU until the host enqueues the
    // next apply, and that gap would land inside the apply's event pair
    const int upto = std::min(maxit, it + (it == 0 ? first : (c->stats_on ? chk : std::min(chk, 3))));
    for (; it < upto; ++it) {
      const int par = it & 1;
      if (use16) {
        HDG_DISPATCH(c, launch_apply16, c, c->d_p32, c->d_slot32, &c->d_sc->done, it);
      } else {
        HDG_DISPATCH(c, launch_apply32, c, c->d_p32, c->d_slot32, &c->d_sc->done, it);
      }
      if (c->phys == HDG_ELASTIC) {
        c->n_launch += 3;
        HDG_DISPATCH(c, launch_face_q32, c);
        cg32_update_kernel<<<nb, 256, 0, c->stream>>>(n4, nb, par, c->d_part, (const float4*)c->d_p32,
                                                      (const float4*)c->d_q32, (const float4*)c->d_dinv32,
                                                      (float4*)c->d_x32, (float4*)c->d_r32, (float4*)c->d_z32,
                                                      c->d_part + nb, c->d_sc);
      } else {
        // p.q comes from the apply; the update forms q from the slots
        c->n_launch += 2;
        HDG_DISPATCH(c, launch_update_f32, c, par);
      }
      cg32_direction_kernel<<<nb, 256, 0, c->stream>>>(n4, nb, par, it, c->d_part + nb, (const float4*)c->d_z32,
                                                       (float4*)c->d_p32, c->d_sc, maxit, 0);
    }
    if ((s = check_launch(c, "cg32_iter"))) return s;
    CUDA_TRY(c, cudaMemcpyAsync(c->h_sc, c->d_sc, sizeof(CgScal), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    harvest(c, c->h_sc->done ? c->h_sc->iters : (1 << 30));
  }
  *iters = c->h_sc->iters;
  *last = std::max(1, c->h_sc->iters);
  return HDG_OK;
}

// Mixed precision: FP64 iterative refinement of (-K) x = bvec. Each sweep forms the FP64
// residual with the FP64 S_K, solves for the correction with FP32 S_K (inner PCG with FP64
// inner products) and adds it to x in FP64.
hdg_status solve_mixed(hdg_ctx* c, const double* bvec, double* x, hdg_solve_info* info) {
  const int64_t nfe = c->sk.nf * c->Nf;
  const int nb = c->nb_red;
  int total_it = 0;
  hdg_status s;
  double rel = 0.0, rel_prev = 0.0;
  bool use16 = c->d_S16 != nullptr;   // FP16 inner operator until a sweep contracts poorly
  for (int sweep = 0;; ++sweep) {
    if (c->d_Sdf) {
      HDG_DISPATCH(c, launch_apply_df, c, x, c->d_slot);
    } else {
      HDG_DISPATCH(c, launch_apply, c, x, c->d_slot, (const int*)nullptr);
    }
    c->n_launch += 2;
    refine_residual_kernel<<<nb, 256, 0, c->stream>>>(c->sk.nf, c->Nf, c->sgn, c->d_face_slot, c->d_face_bnd, c->d_slot, bvec,
                                                      c->d_res, c->d_part, nullptr);
    refine_scalars<<<1, 256, 0, c->stream>>>(nb, c->d_part, c->d_rs);
    if ((s = check_launch(c, "refine_residual"))) return s;
    CUDA_TRY(c, cudaMemcpyAsync(c->h_rs, c->d_rs, sizeof(RefScal), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    harvest(c);
    const RefScal r = *c->h_rs;
    if (r.bb == 0.0) {
      c->n_launch += 1;
      zero_interior_kernel<<<grid_for(c, nfe), 256, 0, c->stream>>>(c->sk.nf, c->Nf, c->d_face_bnd, x);
      if (info) { info->rel_residual = 0.0; info->sweeps += sweep; }
      return check_launch(c, "zero_interior");
    }
    rel_prev = rel;
    rel = std::sqrt(r.rr / r.bb);
    // the FP16 operator's rounding bounds the contraction of a sweep; if it gained less than
    // a factor 10, the remaining sweeps use the FP32 copy
    if (use16 && sweep > 0 && rel > 0.1 * rel_prev) use16 = false;
    if (rel <= c->opt.rtol) {
      if (info) { info->iterations += total_it; info->sweeps += sweep; info->rel_residual = rel; }
      return HDG_OK;
    }
    if (sweep >= c->opt.max_sweeps) break;
    c->n_launch += 1;
    to32_scaled_kernel<<<grid_for(c, nfe), 256, 0, c->stream>>>(nfe, c->d_res, c->d_rs, c->d_b32);
    // the inner solve needs to gain only what is left to rtol (with a margin): the last sweep
    // stops early instead of over-solving to inner_rtol
    const double tol = std::min(0.5, std::max(c->opt.inner_rtol, 0.25 * c->opt.rtol / rel));
    int it = 0;
    if ((s = cg32_inner(c, &it, tol, &c->last_sweep_it[std::min(sweep, 7)], use16))) return s;
    total_it += it;
    c->n_launch += 1;
    refine_update_kernel<<<grid_for(c, nfe), 256, 0, c->stream>>>(c->sk.nf, c->Nf, c->d_face_bnd, c->d_x32, c->d_rs, x);
    if ((s = check_launch(c, "refine_update"))) return s;
  }
  if (info) { info->iterations += total_it; info->sweeps += c->opt.max_sweeps; info->rel_residual = rel; }
  return fail(c, HDG_ENOCONV, "mixed-precision refinement reached max_sweeps=" + std::to_string(c->opt.max_sweeps) +
                                  " with relative residual " + std::to_string(rel));
}

// ---- device-driven solves (one graph launch per trace solve; loop conditions set on the device)
// FP64 PCG on (sgn K) x = bvec: the initial residual, then a WHILE loop of two iterations per trip.
hdg_status cg_solve_graph(hdg_ctx* c, const double* bvec, double* x, hdg_solve_info* info) {
  const int64_t nfe = c->sk.nf * c->Nf;
  const int nb = c->nb_red, maxit = c->opt.maxit;
  auto build = [&](GraphBuild& gb, cudaGraph_t G, hdg_ctx::DevGraph& dg) {
    std::vector<cudaGraphNode_t> deps, bd;
    const int64_t n0 = c->n_launch;
    gb.seq(G, deps, [&] {
      HDG_DISPATCH(c, launch_apply, c, x, c->d_slot, (const int*)nullptr, -1);
      c->n_launch += 2;
      cg_init_kernel<<<nb, 256, 0, c->stream>>>(c->sk.nf, c->Nf, c->sgn, c->d_face_slot, c->d_face_bnd, c->d_slot, bvec,
                                                c->d_dinv, c->d_r, c->d_z, c->d_p, c->d_part);
      cg_init_scalars<<<1, 256, 0, c->stream>>>(nb, c->d_part, c->opt.rtol, c->d_sc);
    });
    const cudaGraphConditionalHandle h = gb.handle(G, 1, true);
    cudaGraph_t B = gb.loop(G, deps, h);
    const int64_t n1 = c->n_launch;
    gb.seq(B, bd, [&] {
      for (int par = 0; par < 2; ++par) {
        HDG_DISPATCH(c, launch_apply, c, c->d_p, c->d_slot, &c->d_sc->done, -1);
        c->n_launch += 3;
        HDG_DISPATCH(c, launch_face_q64, c);
        cg_update_kernel<<<nb, 256, 0, c->stream>>>(nfe, nb, par, c->d_part, c->d_p, c->d_q, c->d_dinv, x, c->d_r, c->d_z,
                                                    c->d_part + nb, c->d_sc);
        cg_direction_kernel<<<nb, 256, 0, c->stream>>>(nfe, nb, par, -1, c->d_part + nb, c->d_z, c->d_p, c->d_sc, maxit, h);
      }
    });
    const int64_t n2 = c->n_launch;
    gb.seq(G, deps, [&] {
      c->n_launch += 2;
      cg_ctl_finish_kernel<<<1, 32, 0, c->stream>>>(c->d_sc, c->d_lc);
      zero_masked_if_kernel<<<grid_for(c, nfe), 256, 0, c->stream>>>(nfe, c->d_intmask, c->d_lc, x);
    });
    dg.n_static = (n1 - n0) + (c->n_launch - n2);
    dg.n_body = 0;
    dg.n_trip = n2 - n1;
  };
  return devgraph_solve(c, 0, bvec, x, build, info);
}

// Mixed precision: FP64 iterative refinement as a WHILE loop over sweeps; each sweep forms the
// FP64-accurate residual, lets the control kernel decide (stop, operator, inner tolerance), and
// runs the inner FP32 PCG with the FP16 or the FP32 copy of S_K as a nested WHILE loop.
hdg_status solve_mixed_graph(hdg_ctx* c, const double* bvec, double* x, hdg_solve_info* info) {
  const int64_t nfe = c->sk.nf * c->Nf;
  const int nb = c->nb_red, maxit = c->opt.maxit;
  const int64_t n4 = c->nfe4 / 4;
  const bool has16 = c->d_S16 != nullptr;
  // x = sum c_i lam_i from the least-squares guess just before this solve: the first residual
  // comes from the stored pairs instead of an apply (acoustic double-float path)
  const bool from_guess = c->guess_x && c->g_q && c->d_Sdf && c->phys == HDG_ACOUSTIC && c->R == 1;
  const int* skip = from_guess ? &c->d_lc->skip_res : nullptr;
  auto inner = [&](bool use16, cudaGraphConditionalHandle h) {
    for (int par = 0; par < 2; ++par) {
      if (use16) {
        HDG_DISPATCH(c, launch_apply16, c, c->d_p32, c->d_slot32, &c->d_sc->done, -1);
      } else {
        HDG_DISPATCH(c, launch_apply32, c, c->d_p32, c->d_slot32, &c->d_sc->done, -1);
      }
      if (c->phys == HDG_ELASTIC) {
        c->n_launch += 3;
        HDG_DISPATCH(c, launch_face_q32, c);
        cg32_update_kernel<<<nb, 256, 0, c->stream>>>(n4, nb, par, c->d_part, (const float4*)c->d_p32,
                                                      (const float4*)c->d_q32, (const float4*)c->d_dinv32,
                                                      (float4*)c->d_x32, (float4*)c->d_r32, (float4*)c->d_z32,
                                                      c->d_part + nb, c->d_sc);
      } else {
        c->n_launch += 2;
        HDG_DISPATCH(c, launch_update_f32, c, par);
      }
      cg32_direction_kernel<<<nb, 256, 0, c->stream>>>(n4, nb, par, -1, c->d_part + nb, (const float4*)c->d_z32,
                                                       (float4*)c->d_p32, c->d_sc, maxit, h);
    }
  };
  auto build = [&](GraphBuild& gb, cudaGraph_t G, hdg_ctx::DevGraph& dg) {
    std::vector<cudaGraphNode_t> deps, bd, d16, d32;
    const int64_t n0 = c->n_launch;
    gb.seq(G, deps, [&] {
      c->n_launch += 1;
      loopctl_init_kernel<<<1, 32, 0, c->stream>>>(c->d_lc, has16 ? 1 : 0);
      if (from_guess) {
        c->n_launch += 1;
        gresidual_kernel<<<nb, 256, 0, c->stream>>>(c->sk.nf, c->Nf, c->d_face_bnd, c->d_gd, c->d_gb, bvec, c->d_res,
                                                    c->d_part, c->d_lc);
      }
    });
    const cudaGraphConditionalHandle h_sweep = gb.handle(G, 1, true);
    cudaGraph_t B = gb.loop(G, deps, h_sweep);
    const cudaGraphConditionalHandle h16 = has16 ? gb.handle(B, 0, false) : 0;
    const cudaGraphConditionalHandle h32 = gb.handle(B, 0, false);
    const int64_t n1 = c->n_launch;
    gb.seq(B, bd, [&] {
      if (c->d_Sdf) {
        HDG_DISPATCH(c, launch_apply_df, c, x, c->d_slot, skip);
      } else {
        HDG_DISPATCH(c, launch_apply, c, x, c->d_slot, (const int*)nullptr, -1);
      }
      c->n_launch += 6;
      refine_residual_kernel<<<nb, 256, 0, c->stream>>>(c->sk.nf, c->Nf, c->sgn, c->d_face_slot, c->d_face_bnd, c->d_slot,
                                                        bvec, c->d_res, c->d_part, skip);
      refine_scalars<<<1, 256, 0, c->stream>>>(nb, c->d_part, c->d_rs);
      sweep_ctl_kernel<<<1, 32, 0, c->stream>>>(c->d_rs, c->d_sc, c->d_lc, c->opt.rtol, c->opt.inner_rtol,
                                                c->opt.max_sweeps, h_sweep, has16 ? 1 : 0, h16, h32);
      to32_scaled_kernel<<<grid_for(c, nfe), 256, 0, c->stream>>>(nfe, c->d_res, c->d_rs, c->d_b32);
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
      refine_update_kernel<<<grid_for(c, nfe), 256, 0, c->stream>>>(c->sk.nf, c->Nf, c->d_face_bnd, c->d_x32, c->d_rs, x);
    });
    const int64_t n5 = c->n_launch;
    gb.seq(G, deps, [&] {
      c->n_launch += 1;
      zero_masked_if_kernel<<<grid_for(c, nfe), 256, 0, c->stream>>>(nfe, c->d_intmask, c->d_lc, x);
    });
    dg.n_static = (n1 - n0) + (c->n_launch - n5);
    dg.n_body = (n2 - n1) + (n5 - n4_);
    dg.n_trip = n4_ - n3;
  };
  return devgraph_solve(c, from_guess ? 8 : 1, bvec, x, build, info);
}

// ---- continuous traces: device-driven solves of (sgn R^T K R) mu = b_mu on the free nodes
// FP64 PCG: every apply expands the nodal vector to face traces, applies the element blocks and
// gathers the face nodal weights back to the nodes in a fixed order.
hdg_status edg_cg_graph(hdg_ctx* c, const double* bvec, double* x, hdg_solve_info* info) {
  const int64_t n = c->n_mu;
  const int nb = c->nb_red, maxit = c->opt.maxit;
  auto build = [&](GraphBuild& gb, cudaGraph_t G, hdg_ctx::DevGraph& dg) {
    std::vector<cudaGraphNode_t> deps, bd;
    const int64_t n0 = c->n_launch;
    gb.seq(G, deps, [&] {
      HDG_DISPATCH(c, edg_expand64, c, x, c->d_ew64, 1);
      HDG_DISPATCH(c, launch_apply, c, c->d_ew64, c->d_slot, (const int*)nullptr, -1);
      HDG_DISPATCH(c, edg_face_w64, c, c->d_slot, (const double*)nullptr, c->d_w64);
      c->n_launch += 2;
      edg_cg_init_kernel<<<nb, 256, 0, c->stream>>>(n, c->sgn, c->d_node_ptr, c->d_node_inc, c->d_w64, bvec, c->d_dinv,
                                                    c->d_r, c->d_z, c->d_p, c->d_part);
      cg_init_scalars<<<1, 256, 0, c->stream>>>(nb, c->d_part, c->opt.rtol, c->d_sc);
    });
    const cudaGraphConditionalHandle h = gb.handle(G, 1, true);
    cudaGraph_t B = gb.loop(G, deps, h);
    const int64_t n1 = c->n_launch;
    gb.seq(B, bd, [&] {
      for (int par = 0; par < 2; ++par) {
        HDG_DISPATCH(c, edg_expand64, c, c->d_p, c->d_ew64, 1);
        HDG_DISPATCH(c, launch_apply, c, c->d_ew64, c->d_slot, &c->d_sc->done, -1);
        HDG_DISPATCH(c, edg_face_w64, c, c->d_slot, (const double*)nullptr, c->d_w64);
        c->n_launch += 3;
        edg_q64_kernel<<<nb, 256, 0, c->stream>>>(n, c->sgn, c->d_node_ptr, c->d_node_inc, c->d_w64, c->d_p, c->d_q,
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
      zero_masked_if_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(n, nullptr, c->d_lc, x);
    });
    dg.n_static = (n1 - n0) + (c->n_launch - n2);
    dg.n_body = 0;
    dg.n_trip = n2 - n1;
  };
  return devgraph_solve(c, 4, bvec, x, build, info);
}

// Mixed precision: FP64-accurate residual through the double-float apply of the expanded face
// traces, inner FP32 PCG on the nodes with the FP16 or FP32 element blocks.
hdg_status edg_mixed_graph(hdg_ctx* c, const double* bvec, double* x, hdg_solve_info* info) {
  const int64_t n = c->n_mu;
  const int nb = c->nb_red, maxit = c->opt.maxit;
  const int64_t n4 = c->n_mu4 / 4;
  const bool has16 = c->d_S16 != nullptr;
  auto inner = [&](bool use16, cudaGraphConditionalHandle h) {
    for (int par = 0; par < 2; ++par) {
      HDG_DISPATCH(c, edg_expand32, c, c->d_p32, c->d_ew32);
      if (use16) {
        HDG_DISPATCH(c, launch_apply16, c, c->d_ew32, c->d_slot32, &c->d_sc->done, -1);
      } else {
        HDG_DISPATCH(c, launch_apply32, c, c->d_ew32, c->d_slot32, &c->d_sc->done, -1);
      }
      HDG_DISPATCH(c, edg_face_w32, c, c->d_slot32, c->d_w32);
      c->n_launch += 2;
      edg_update32_kernel<<<nb, 256, 0, c->stream>>>(n, (float)c->sgn, c->d_node_ptr, c->d_node_inc, c->d_w32, c->d_p32,
                                                     c->d_dinv32, c->d_x32, c->d_r32, c->d_z32, par, c->d_pq, c->d_part,
                                                     c->d_sc);
      cg32_direction_kernel<<<nb, 256, 0, c->stream>>>(n4, nb, par, -1, c->d_part, (const float4*)c->d_z32,
                                                       (float4*)c->d_p32, c->d_sc, maxit, h);
    }
  };
  auto build = [&](GraphBuild& gb, cudaGraph_t G, hdg_ctx::DevGraph& dg) {
    std::vector<cudaGraphNode_t> deps, bd, d16, d32;
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
      HDG_DISPATCH(c, edg_expand64, c, x, c->d_ew64, 1);
      if (c->d_Sdf) {
        HDG_DISPATCH(c, launch_apply_df, c, c->d_ew64, c->d_slot);
      } else {
        HDG_DISPATCH(c, launch_apply, c, c->d_ew64, c->d_slot, (const int*)nullptr, -1);
      }
      HDG_DISPATCH(c, edg_face_w64, c, c->d_slot, (const double*)nullptr, c->d_w64);
      c->n_launch += 6;
      edg_residual_kernel<<<nb, 256, 0, c->stream>>>(n, c->sgn, c->d_node_ptr, c->d_node_inc, c->d_w64, bvec, c->d_res,
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
      flat_refine_update_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(n, c->d_x32, c->d_rs, x);
    });
    const int64_t n5 = c->n_launch;
    gb.seq(G, deps, [&] {
      c->n_launch += 1;
      zero_masked_if_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(n, nullptr, c->d_lc, x);
    });
    dg.n_static = (n1 - n0) + (c->n_launch - n5);
    dg.n_body = (n2 - n1) + (n5 - n4_);
    dg.n_trip = n4_ - n3;
  };
  return devgraph_solve(c, 5, bvec, x, build, info);
}

// b_mu = R^T b for a face array b (interior faces)
hdg_status edg_restrict(hdg_ctx* c, const double* b, double* bmu) {
  HDG_DISPATCH(c, edg_face_w64, c, (const double*)nullptr, b, c->d_w64);
  c->n_launch += 1;
  edg_node_gather_kernel<<<grid_for(c, c->n_mu), 256, 0, c->stream>>>(c->n_mu, c->d_node_ptr, c->d_node_inc, c->d_w64, 1.0,
                                                                      bmu);
  return check_launch(c, "edg_restrict");
}

// solve (sgn R^T K R) mu = bmu from the initial guess in mu
hdg_status edg_solve(hdg_ctx* c, const double* bmu, double* mu, hdg_solve_info* info) {
  return c->opt.prec != HDG_FP64 ? edg_mixed_graph(c, bmu, mu, info) : edg_cg_graph(c, bmu, mu, info);
}

// Restarted GMRES(m) on (sgn K) x = bvec with right Jacobi preconditioning and iterated
// classical Gram-Schmidt (two passes per Arnoldi step), FP64 (Sec. 2.4's Krylov method). The
// vector work runs in the kernels of gmres.cuh; the small Hessenberg least-squares problem
// (Givens rotations) and the restart / convergence decisions are on the host.
hdg_status gmres_solve(hdg_ctx* c, const double* bvec, double* x, hdg_solve_info* info) {
  const int m = c->opt.gmres_restart, nb = c->nb_red;
  const int64_t n = c->sk.nf * c->Nf;
  hdg_status s;
  if (!c->d_gmV) {
    // the FP64 residual vector and its scalars exist only in mixed-precision contexts
    if (!c->d_res && (s = dalloc(c, &c->d_res, (size_t)n))) return s;
    if (!c->d_rs && (s = dalloc(c, &c->d_rs, 1))) return s;
    if (!c->h_rs) CUDA_TRY(c, cudaMallocHost((void**)&c->h_rs, sizeof(RefScal)));
    if ((s = dalloc(c, &c->d_gmV, (size_t)(m + 1) * n))) return s;
    if ((s = dalloc(c, &c->d_gmpart, (size_t)(m + 2) * nb))) return s;
    if ((s = dalloc(c, &c->d_gmh, (size_t)m + 2))) return s;
    if ((s = dalloc(c, &c->d_gmy, (size_t)m + 1))) return s;
    CUDA_TRY(c, cudaMemsetAsync(c->d_gmV, 0, (size_t)(m + 1) * n * 8, c->stream));
  }
  double* V = c->d_gmV;
  std::vector<double> hv((size_t)m + 2);
  // dots of the first q basis vectors with w, then (w, w), into d_gmh and hv
  auto dots = [&](int q, const double* w) -> hdg_status {
    c->n_launch += 2;
    gm_dots_kernel<<<dim3((unsigned)nb, (unsigned)(q + 1)), 256, 0, c->stream>>>(n, q, V, w, c->d_gmpart);
    gm_dots_final_kernel<<<q + 1, 256, 0, c->stream>>>(nb, c->d_gmpart, c->d_gmh);
    CUDA_TRY(c, cudaMemcpyAsync(hv.data(), c->d_gmh, (size_t)(q + 1) * 8, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return check_launch(c, "gmres_dots");
  };
  // w = sgn K M^{-1} v (interior entries; zero on boundary faces); M^{-1} = Jacobi or block ILU(0)
  auto opK = [&](const double* v, double* w) -> hdg_status {
    c->n_launch += 1;
    if (c->bilu) {
      hdg_status s2 = bilu_apply(c, v, c->d_z);
      if (s2) return s2;
    } else {
      c->n_launch += 1;
      vmul_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(n, c->d_dinv, v, c->d_z);
    }
    HDG_DISPATCH(c, launch_apply, c, (const double*)c->d_z, c->d_slot, (const int*)nullptr, -1);
    face_gather_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(c->sk.nf, c->Nf, c->d_face_slot, c->d_face_bnd, c->d_slot,
                                                              c->sgn, w);
    return check_launch(c, "gmres_op");
  };
  if ((s = dots(0, bvec))) return s;
  const double bb = hv[0];
  if (bb == 0.0) {
    c->n_launch += 1;
    zero_interior_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(c->sk.nf, c->Nf, c->d_face_bnd, x);
    if (info) { info->rel_residual = 0.0; info->sweeps += 1; }
    return check_launch(c, "zero_interior");
  }
  const double bn = std::sqrt(bb);
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g((size_t)m + 1), y(m);
  int total = 0, cycles = 0;
  double rel = 0.0;
  for (;;) {
    // true residual r = b - sgn K x
    HDG_DISPATCH(c, launch_apply, c, (const double*)x, c->d_slot, (const int*)nullptr, -1);
    c->n_launch += 2;
    refine_residual_kernel<<<nb, 256, 0, c->stream>>>(c->sk.nf, c->Nf, c->sgn, c->d_face_slot, c->d_face_bnd, c->d_slot, bvec,
                                                      c->d_res, c->d_part, nullptr);
    refine_scalars<<<1, 256, 0, c->stream>>>(nb, c->d_part, c->d_rs);
    CUDA_TRY(c, cudaMemcpyAsync(c->h_rs, c->d_rs, sizeof(RefScal), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    const RefScal rs = *c->h_rs;
    const double beta = std::sqrt(rs.rr);
    rel = beta / bn;
    if (rel <= c->opt.rtol) break;
    if (total >= c->opt.maxit) {
      if (info) { info->iterations += total; info->sweeps += cycles; info->rel_residual = rel; }
      return fail(c, HDG_ENOCONV, "GMRES reached maxit=" + std::to_string(c->opt.maxit) + " with relative residual " +
                                      std::to_string(rel));
    }
    ++cycles;
    c->n_launch += 1;
    combine_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(n, 1.0 / beta, c->d_res, 0, nullptr, 0, nullptr, 0, nullptr, V);
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int k = 0;
    for (int j = 0; j < m && total < c->opt.maxit; ++j) {
      double* w = V + (int64_t)(j + 1) * n;
      if ((s = opK(V + (int64_t)j * n, w))) return s;
      // two classical Gram-Schmidt passes against V_0..V_j
      double hcol[66];
      if ((s = dots(j + 1, w))) return s;
      for (int i = 0; i <= j; ++i) hcol[i] = hv[i];
      c->n_launch += 1;
      gm_orth_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(n, j + 1, V, c->d_gmh, w);
      if ((s = dots(j + 1, w))) return s;
      for (int i = 0; i <= j; ++i) hcol[i] += hv[i];
      c->n_launch += 1;
      gm_orth_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(n, j + 1, V, c->d_gmh, w);
      if ((s = dots(0, w))) return s;
      const double hn = std::sqrt(std::max(0.0, hv[0]));
      hcol[j + 1] = hn;
      // previous rotations, then the one that zeroes the subdiagonal entry
      for (int i = 0; i < j; ++i) {
        const double a = hcol[i], b2 = hcol[i + 1];
        hcol[i] = cs[i] * a + sn[i] * b2;
        hcol[i + 1] = -sn[i] * a + cs[i] * b2;
      }
      const double r = std::hypot(hcol[j], hcol[j + 1]);
      cs[j] = r > 0.0 ? hcol[j] / r : 1.0;
      sn[j] = r > 0.0 ? hcol[j + 1] / r : 0.0;
      hcol[j] = r;
      hcol[j + 1] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = hcol[i];
      ++total;
      k = j + 1;
      if (std::fabs(g[j + 1]) <= c->opt.rtol * bn || hn == 0.0) break;
      c->n_launch += 1;
      combine_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(n, 1.0 / hn, w, 0, nullptr, 0, nullptr, 0, nullptr, w);
    }
    // y = H^{-1} g (upper triangular k x k), x += Dinv V y
    for (int i = k - 1; i >= 0; --i) {
      double v = g[i];
      for (int jj = i + 1; jj < k; ++jj) v -= H[(size_t)i * m + jj] * y[jj];
      y[i] = v / H[(size_t)i * m + i];
    }
    CUDA_TRY(c, cudaMemcpyAsync(c->d_gmy, y.data(), (size_t)k * 8, cudaMemcpyHostToDevice, c->stream));
    if (c->bilu) {
      // x += M^{-1} (V y)
      c->n_launch += 2;
      bilu_vcombine_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(n, k, V, c->d_gmy, c->d_p);
      if ((s = bilu_apply(c, c->d_p, c->d_z))) return s;
      bilu_add_masked_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(n, c->d_intmask, c->d_z, x);
    } else {
      c->n_launch += 1;
      gm_update_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(n, k, V, c->d_gmy, c->d_dinv, c->d_intmask, x);
    }
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));   // y is released by the next cycle
    if ((s = check_launch(c, "gmres_update"))) return s;
  }
  if (info) { info->iterations += total; info->sweeps += std::max(1, cycles); info->rel_residual = rel; }
  return HDG_OK;
}

// PCG on (-K) x = bvec over interior faces; x holds the initial guess (interior entries).
hdg_status cg_solve(hdg_ctx* c, const double* bvec, double* x, hdg_solve_info* info) {
  if (c->opt.solver == HDG_SOLVER_GMRES) return gmres_solve(c, bvec, x, info);
  if (use_devgraph(c)) return c->opt.prec != HDG_FP64 ? solve_mixed_graph(c, bvec, x, info) : cg_solve_graph(c, bvec, x, info);
  if (c->opt.prec != HDG_FP64) return solve_mixed(c, bvec, x, info);
  const int64_t nfe = c->sk.nf * c->Nf;
  const int nb = c->nb_red;
  HDG_DISPATCH(c, launch_apply, c, x, c->d_slot, (const int*)nullptr);
  c->n_launch += 2;
  cg_init_kernel<<<nb, 256, 0, c->stream>>>(c->sk.nf, c->Nf, c->sgn, c->d_face_slot, c->d_face_bnd, c->d_slot, bvec, c->d_dinv, c->d_r,
                                            c->d_z, c->d_p, c->d_part);
  cg_init_scalars<<<1, 256, 0, c->stream>>>(nb, c->d_part, c->opt.rtol, c->d_sc);
  hdg_status s = check_launch(c, "cg_init");
  if (s) return s;
  CUDA_TRY(c, cudaMemcpyAsync(c->h_sc, c->d_sc, sizeof(CgScal), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (c->h_sc->bb == 0.0) {
    c->n_launch += 1;
    zero_interior_kernel<<<grid_for(c, nfe), 256, 0, c->stream>>>(c->sk.nf, c->Nf, c->d_face_bnd, x);
    if (info) { info->rel_residual = 0.0; info->sweeps += 1; }
    return check_launch(c, "zero_interior");
  }
  int it = 0;
  const int maxit = c->opt.maxit;
  const int chk = std::max(1, c->opt.check_every);
  int first = std::max(2, std::min(chk, c->last_it64 - 1));   // first poll near the last solve's count
  while (!c->h_sc->done && it < maxit) {
    const int upto = std::min(maxit, it + (it == 0 ? first : (c->stats_on ? chk : std::min(chk, 4))));
    for (; it < upto; ++it) {
      const int par = it & 1;
      HDG_DISPATCH(c, launch_apply, c, c->d_p, c->d_slot, &c->d_sc->done, it);
      c->n_launch += 3;
      HDG_DISPATCH(c, launch_face_q64, c);
      cg_update_kernel<<<nb, 256, 0, c->stream>>>(nfe, nb, par, c->d_part, c->d_p, c->d_q, c->d_dinv, x, c->d_r, c->d_z,
                                                  c->d_part + nb, c->d_sc);
      cg_direction_kernel<<<nb, 256, 0, c->stream>>>(nfe, nb, par, it, c->d_part + nb, c->d_z, c->d_p, c->d_sc, maxit, 0);
    }
    s = check_launch(c, "cg_iter");
    if (s) return s;
    CUDA_TRY(c, cudaMemcpyAsync(c->h_sc, c->d_sc, sizeof(CgScal), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    harvest(c, c->h_sc->done ? c->h_sc->iters : (1 << 30));
  }
  const CgScal& h = *c->h_sc;
  c->last_it64 = std::max(1, h.iters);
  if (info) {
    info->iterations += h.iters;
    info->sweeps += 1;
    info->rel_residual = std::sqrt(std::max(0.0, h.rr) / h.bb);
  }
  if (h.done != 1)
    return fail(c, HDG_ENOCONV, "trace solve reached maxit=" + std::to_string(maxit) + " with relative residual " +
                                    std::to_string(std::sqrt(std::max(0.0, h.rr) / h.bb)));
  return HDG_OK;
}


// ======================================================================= multiple right-hand sides
MScal mscal(hdg_ctx* c) {
  MScal m;
  m.rho0 = c->d_mrho0; m.rho1 = c->d_mrho1; m.alpha = c->d_malpha; m.rr = c->d_mrr; m.bb = c->d_mbb;
  m.tol2 = c->d_mtol2; m.conv = c->d_mconv; m.done = c->d_mdone; m.iters = c->d_miters;
  return m;
}

template <int DIM, int K, int CWW>
void mlaunch_local_cw(hdg_ctx* c, int mode, const double* F, const double* hist, const SrcArgs& sa, const double* lam,
                      double* out) {
  using L = LocalMultiCfg<DIM, K, CWW>;
  dim3 grid((unsigned)c->sk.ne, (unsigned)((c->R + L::CW - 1) / L::CW));
  if (c->d_Hinvdf) {   // mixed precision: double-float on the FP32 pipe
    const float th = (float)c->tau;
    const df2 tau{th, (float)(c->tau - (double)th)};
    if (mode == 0)
      local_df_multi_kernel<DIM, K, 0, CWW><<<grid, L::NT, 0, c->stream>>>(devmesh(c), c->tabsdf, c->d_geodf, c->d_Hinvdf,
                                                                           c->alpha, tau, c->R, F, hist, sa, lam, out);
    else
      local_df_multi_kernel<DIM, K, 1, CWW><<<grid, L::NT, 0, c->stream>>>(devmesh(c), c->tabsdf, c->d_geodf, c->d_Hinvdf,
                                                                           c->alpha, tau, c->R, F, hist, sa, lam, out);
    return;
  }
  if (mode == 0)
    local_multi_kernel<DIM, K, 0, CWW><<<grid, L::NT, 0, c->stream>>>(devmesh(c), c->tabs, c->d_Hinv, c->alpha, c->tau,
                                                                       c->R, F, hist, sa, lam, out);
  else
    local_multi_kernel<DIM, K, 1, CWW><<<grid, L::NT, 0, c->stream>>>(devmesh(c), c->tabs, c->d_Hinv, c->alpha, c->tau,
                                                                       c->R, F, hist, sa, lam, out);
}

template <int DIM, int K>
void mlaunch_local(hdg_ctx* c, int mode, const double* F, const double* hist, double t, const double* lam, double* out) {
  const SrcArgs sa = srcargs(c, t);
  c->n_launch += 1;
  // as many columns per CTA as the batch has (up to the kernel's width)
  // (the double-float kernels of the mixed path take at most 16, for three CTAs per SM)
  if (c->R <= 2) mlaunch_local_cw<DIM, K, 2>(c, mode, F, hist, sa, lam, out);
  else if (c->R <= 4) mlaunch_local_cw<DIM, K, 4>(c, mode, F, hist, sa, lam, out);
  else if (c->R <= 8) mlaunch_local_cw<DIM, K, 8>(c, mode, F, hist, sa, lam, out);
  else if (c->R <= 16 || c->d_Hinvdf) mlaunch_local_cw<DIM, K, 16>(c, mode, F, hist, sa, lam, out);
  else mlaunch_local_cw<DIM, K, 32>(c, mode, F, hist, sa, lam, out);
}

template <int DIM, int K, typename TV, int CWN>
void mlaunch_apply_cw(hdg_ctx* c, const TV* x, TV* slot, const int* done) {
  constexpr int EPB = 4 * (32 / CWN);   // elements per 4-warp block
  dim3 grid((unsigned)((c->sk.ne + EPB - 1) / EPB), (unsigned)((c->R + CWN - 1) / CWN));
  apply_multi_kernel<DIM, K, TV, CWN><<<grid, 128, 0, c->stream>>>(c->sk.ne, c->R, c->d_elem_face, c->d_face_bnd,
                                                                   c->d_S32, c->d_S, x, slot, done);
}

template <int DIM, int K, typename TV>
void mlaunch_apply(hdg_ctx* c, const TV* x, TV* slot, const int* done, int iter) {
  c->n_launch += 1;
  cudaEvent_t stop = apply_begin(c, sizeof(TV) == 4 ? 1 : 0, iter);
  if (c->R <= 2) mlaunch_apply_cw<DIM, K, TV, 2>(c, x, slot, done);
  else if (c->R <= 4) mlaunch_apply_cw<DIM, K, TV, 4>(c, x, slot, done);
  else if (c->R <= 8) mlaunch_apply_cw<DIM, K, TV, 8>(c, x, slot, done);
  else if (c->R <= 16) mlaunch_apply_cw<DIM, K, TV, 16>(c, x, slot, done);
  else mlaunch_apply_cw<DIM, K, TV, 32>(c, x, slot, done);
  apply_end(c, stop);
}
template <int DIM, int K, int CWN>
void mlaunch_apply_df_cw(hdg_ctx* c, const double* x, double* slot) {
  constexpr int EPB = ApplyDfMCfg<DIM, K>::WPB * (32 / CWN);
  dim3 grid((unsigned)((c->sk.ne + EPB - 1) / EPB), (unsigned)((c->R + CWN - 1) / CWN));
  apply_df_multi_kernel<DIM, K, CWN><<<grid, 32 * ApplyDfMCfg<DIM, K>::WPB, 0, c->stream>>>(
      c->sk.ne, c->R, c->d_elem_face, c->d_face_bnd, c->d_mShi, c->d_mSlo, x, slot);
}

// FP64-accurate R-column apply of the mixed refinement (double-float on the FP32 pipe)
template <int DIM, int K>
void mlaunch_apply_df(hdg_ctx* c, const double* x, double* slot) {
  c->n_launch += 1;
  cudaEvent_t stop = apply_begin(c, 2, -1);
  if (c->R <= 2) mlaunch_apply_df_cw<DIM, K, 2>(c, x, slot);
  else if (c->R <= 4) mlaunch_apply_df_cw<DIM, K, 4>(c, x, slot);
  else if (c->R <= 8) mlaunch_apply_df_cw<DIM, K, 8>(c, x, slot);
  else if (c->R <= 16) mlaunch_apply_df_cw<DIM, K, 16>(c, x, slot);
  else mlaunch_apply_df_cw<DIM, K, 32>(c, x, slot);
  apply_end(c, stop);
}

template <int DIM, int K>
void mlaunch_apply64(hdg_ctx* c, const double* x, double* slot, const int* done, int iter) {
  mlaunch_apply<DIM, K, double>(c, x, slot, done, iter);
}
template <int DIM, int K>
void mlaunch_apply32(hdg_ctx* c, const float* x, float* slot, const int* done, int iter) {
  // fewer than 32 columns: several elements per warp over the group-layout FP32 S_K
  if (c->R < 32) {
    mlaunch_apply<DIM, K, float>(c, x, slot, done, iter);
    return;
  }
  // 32 columns or more: S_K times the column block on the tensor cores
  using AC = ApplyTcCfg<DIM, K>;
  const unsigned grid = (unsigned)((c->sk.ne + AC::WPB - 1) / AC::WPB);
  c->n_launch += 1;
  cudaEvent_t stop = apply_begin(c, 1, iter);
  if (c->R == 32)
    apply_tc_kernel<DIM, K, 32><<<grid, 32 * AC::WPB, AC::SMEM, c->stream>>>(c->sk.ne, c->R, c->d_elem_face, c->d_face_bnd,
                                                                             (const float4*)c->d_S32, x, slot, done);
  else
    apply_tc_kernel<DIM, K, 64><<<grid, 32 * AC::WPB, AC::SMEM, c->stream>>>(c->sk.ne, c->R, c->d_elem_face, c->d_face_bnd,
                                                                             (const float4*)c->d_S32, x, slot, done);
  apply_end(c, stop);
}


template <int DIM, int K, typename TV>
void mlaunch_face_q(hdg_ctx* c, const TV* slot, const TV* p, TV* q) {
  mface_q_kernel<DIM, K, TV><<<c->nb_red, 256, 0, c->stream>>>((int)c->sk.nf, c->R, c->d_face_slot, c->d_face_bnd, slot, p, q,
                                                                c->d_part, c->d_mdone);
}
template <int DIM, int K>
void mlaunch_face_q64(hdg_ctx* c, const double* slot, const double* p, double* q) { mlaunch_face_q<DIM, K, double>(c, slot, p, q); }
template <int DIM, int K>
void mlaunch_face_q32(hdg_ctx* c, const float* slot, const float* p, float* q) {
  if (c->R % 4 == 0)
    mface_q4_kernel<DIM, K><<<c->nb_red, 256, 0, c->stream>>>((int)c->sk.nf, c->R, (const int2*)c->d_face_slot,
                                                               c->d_face_bnd, (const float4*)slot, (const float4*)p,
                                                               (float4*)q, c->d_part, c->d_mdone);
  else
    mlaunch_face_q<DIM, K, float>(c, slot, p, q);
}

template <int DIM, int K, typename TV>
void mlaunch_init(hdg_ctx* c, const TV* slot, const TV* b, const TV* dinv, TV* r, TV* z, TV* p) {
  minit_kernel<DIM, K, TV><<<c->nb_red, 256, 0, c->stream>>>((int)c->sk.nf, c->R, c->d_face_slot, c->d_face_bnd, slot, b, dinv,
                                                              r, z, p, c->d_part);
}
template <int DIM, int K>
void mlaunch_init64(hdg_ctx* c, const double* slot, const double* b, const double* dinv, double* r, double* z, double* p) {
  mlaunch_init<DIM, K, double>(c, slot, b, dinv, r, z, p);
}
template <int DIM, int K>
void mlaunch_init32(hdg_ctx* c, const float* slot, const float* b, const float* dinv, float* r, float* z, float* p) {
  mlaunch_init<DIM, K, float>(c, slot, b, dinv, r, z, p);
}

template <int DIM, int K>
void mlaunch_gather(hdg_ctx* c, const double* slot, double scale, double* out) {
  const int64_t n = c->sk.nf * c->Nf * (int64_t)c->R;
  c->n_launch += 1;
  mface_gather_kernel<DIM, K><<<grid_for(c, n), 256, 0, c->stream>>>((int)c->sk.nf, c->R, c->d_face_slot, c->d_face_bnd, slot,
                                                                     scale, out);
}

template <int DIM, int K>
void mlaunch_refres(hdg_ctx* c, const double* b) {
  c->n_launch += 2;
  if (c->R % 2 == 0 && aligned16(b))
    mrefine_residual2_kernel<DIM, K><<<c->nb_red, 256, 0, c->stream>>>((int)c->sk.nf, c->R, (const int2*)c->d_face_slot,
                                                                        c->d_face_bnd, (const double2*)c->d_mslot,
                                                                        (const double2*)b, (double2*)c->d_res, c->d_part);
  else
    mrefine_residual_kernel<DIM, K><<<c->nb_red, 256, 0, c->stream>>>((int)c->sk.nf, c->R, c->d_face_slot, c->d_face_bnd,
                                                                       c->d_mslot, b, c->d_res, c->d_part);
  mrefine_scalars<<<1, 256, 0, c->stream>>>(c->nb_red, c->R, c->opt.rtol, c->d_part, c->d_mrr2, c->d_mbb2, c->d_mscale,
                                            c->d_mnconv);
}

// Column-block update and direction of the per-column PCG. FP32 with R a multiple of 4: four
// columns per thread (z is not stored, the direction forms it again); otherwise one column per
// thread. The overloads keep mcg generic in the vector type.
void mupdate_cols(hdg_ctx* c, int64_t n, const float* p, const float* q, const float* dinv, float* x, float* r, float* z) {
  if (c->R % 4 == 0)
    mupdate4_kernel<<<c->nb_red, 256, 0, c->stream>>>(n / 4, c->R, (const float4*)p, (const float4*)q, dinv, (float4*)x,
                                                      (float4*)r, c->d_part, mscal(c));
  else
    mupdate_kernel<float><<<c->nb_red, 256, 0, c->stream>>>(n, c->R, p, q, dinv, x, r, z, c->d_part, mscal(c));
}
void mupdate_cols(hdg_ctx* c, int64_t n, const double* p, const double* q, const double* dinv, double* x, double* r,
                  double* z) {
  mupdate_kernel<double><<<c->nb_red, 256, 0, c->stream>>>(n, c->R, p, q, dinv, x, r, z, c->d_part, mscal(c));
}
void mdirection_cols(hdg_ctx* c, int64_t n, const float* r, const float* z, const float* dinv, float* p) {
  if (c->R % 4 == 0)
    mdirection4_kernel<<<c->nb_red, 256, 0, c->stream>>>(n / 4, c->R, (const float4*)r, dinv, (float4*)p, c->d_mbeta,
                                                         c->d_mdone);
  else
    mdirection_kernel<float><<<c->nb_red, 256, 0, c->stream>>>(n, c->R, z, p, c->d_mbeta, c->d_mdone);
}
void mdirection_cols(hdg_ctx* c, int64_t n, const double* r, const double* z, const double* dinv, double* p) {
  mdirection_kernel<double><<<c->nb_red, 256, 0, c->stream>>>(n, c->R, z, p, c->d_mbeta, c->d_mdone);
}

// Ends of a refinement sweep: the inner right-hand side b32 = fl32(rho / |rho|_j), and
// lam += x32 |rho|_j; four columns per thread when R is a multiple of 4 (and lam 16-byte aligned)
void mto32_cols(hdg_ctx* c, int64_t n) {
  if (c->R % 4 == 0)
    mto32_scaled4_kernel<<<grid_for(c, n / 4), 256, 0, c->stream>>>(n / 4, c->R, (const double2*)c->d_res, c->d_mscale,
                                                                    (float4*)c->d_b32);
  else
    mto32_scaled_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(n, c->R, c->d_res, c->d_mscale, c->d_b32);
}
void mrefine_update_cols(hdg_ctx* c, int64_t n, double* lam) {
  if (c->R % 4 == 0 && aligned16(lam))
    mrefine_update4_kernel<<<grid_for(c, n / 4), 256, 0, c->stream>>>(n / 4, c->R, c->Nf, c->d_face_bnd,
                                                                      (const float4*)c->d_x32, c->d_mscale, (double2*)lam);
  else
    mrefine_update_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(n, c->R, c->Nf, c->d_face_bnd, c->d_x32, c->d_mscale, lam);
}

// One FP32 iteration of the inner column-block PCG on the context's FP32 vectors (p32, x32,
// r32, slots32), iteration parity par. R = 32 or 64: the persistent tensor-core apply forms
// (p, q) and alpha in its epilogue and the update reads q from the slots (4 launches). Other R:
// apply, face pass with (p, q), alpha, update (6 launches). dev != 0: the beta kernel also sets
// the device-driven loop's condition h.
template <int DIM, int K>
void m_iter32(hdg_ctx* c, int par, int maxit, int dev, cudaGraphConditionalHandle h, int iter) {
  const int64_t n = c->sk.nf * c->Nf * (int64_t)c->R;
  const int nb = c->nb_red, R = c->R;
  if (R == 32 || R == 64) {
    using CP = ApplyTcPCfg<DIM, K>;
    const int64_t nq = (c->sk.ne + CP::WPB - 1) / CP::WPB;
    // CTA partials [grid][R] fit the partials buffer ([3 nb_red][R])
    const int64_t g = std::min<int64_t>(std::min<int64_t>(nq, (int64_t)c->tcp_per_sm * c->sms), 3 * (int64_t)nb);
    const unsigned grid = (unsigned)std::max<int64_t>(1, g);
    const MPqOut o{c->d_part, c->d_ticket, mscal(c), par};
    c->n_launch += 4;
    cudaEvent_t stop = apply_begin(c, 1, iter);
    if (R == 32)
      apply_tc_pq_kernel<DIM, K, 32><<<grid, 32 * CP::WPB, CP::SMEM, c->stream>>>(
          c->sk.ne, c->d_elem_face, c->d_face_bnd, (const float4*)c->d_S32, c->d_p32, c->d_mslot32, o);
    else
      apply_tc_pq_kernel<DIM, K, 64><<<grid, 32 * CP::WPB, CP::SMEM, c->stream>>>(
          c->sk.ne, c->d_elem_face, c->d_face_bnd, (const float4*)c->d_S32, c->d_p32, c->d_mslot32, o);
    apply_end(c, stop);
    mupdate4s_kernel<DIM, K><<<nb, 256, 0, c->stream>>>((int)c->sk.nf, R, (const int2*)c->d_face_slot, c->d_face_bnd,
                                                         (const float4*)c->d_mslot32, (const float4*)c->d_p32,
                                                         c->d_dinv32, (float4*)c->d_x32, (float4*)c->d_r32, c->d_part,
                                                         mscal(c));
    mcols_beta<<<1, 256, 0, c->stream>>>(nb, R, par, maxit, c->d_part, mscal(c), c->d_mbeta, dev, h);
    mdirection_cols(c, n, c->d_r32, c->d_z32, c->d_dinv32, c->d_p32);
    return;
  }
  c->n_launch += 5;
  mlaunch_apply32<DIM, K>(c, (const float*)c->d_p32, c->d_mslot32, c->d_mdone, iter);
  mlaunch_face_q32<DIM, K>(c, (const float*)c->d_mslot32, (const float*)c->d_p32, c->d_q32);
  mcols_alpha<<<1, 256, 0, c->stream>>>(nb, R, par, c->d_part, mscal(c));
  mupdate_cols(c, n, c->d_p32, c->d_q32, c->d_dinv32, c->d_x32, c->d_r32, c->d_z32);
  mcols_beta<<<1, 256, 0, c->stream>>>(nb, R, par, maxit, c->d_part, mscal(c), c->d_mbeta, dev, h);
  mdirection_cols(c, n, c->d_r32, c->d_z32, c->d_dinv32, c->d_p32);
}

// Per-column PCG on (-K) x = b. FP64 (outer, x holds the initial guess) or FP32 (inner, x0 = 0).
template <typename TV>
hdg_status mcg(hdg_ctx* c, const TV* b, TV* x, TV* r, TV* z, TV* p, TV* q, TV* slot, const TV* dinv, double rtol,
               bool x0_zero, int* iters_out) {
  const int64_t n = c->sk.nf * c->Nf * (int64_t)c->R;
  const int nb = c->nb_red;
  hdg_status s;
  if (x0_zero) {
    CUDA_TRY(c, cudaMemsetAsync(x, 0, (size_t)n * sizeof(TV), c->stream));
  } else {
    if (sizeof(TV) == 8) {
      HDG_DISPATCH(c, mlaunch_apply64, c, (const double*)x, (double*)slot, (const int*)nullptr, -1);
    }
  }
  c->n_launch += 2;
  if (sizeof(TV) == 8) {
    HDG_DISPATCH(c, mlaunch_init64, c, x0_zero ? nullptr : (const double*)slot, (const double*)b, (const double*)dinv,
                 (double*)r, (double*)z, (double*)p);
  } else {
    HDG_DISPATCH(c, mlaunch_init32, c, nullptr, (const float*)b, (const float*)dinv, (float*)r, (float*)z, (float*)p);
  }
  if (sizeof(TV) == 4)   // inner solve of a refinement sweep: per-column relaxed tolerance
    mcols_init<<<1, 256, 0, c->stream>>>(nb, c->R, rtol, x0_zero ? 1 : 0, c->d_part, mscal(c), c->d_mrr2, c->d_mbb2,
                                         c->opt.rtol);
  else
    mcols_init<<<1, 256, 0, c->stream>>>(nb, c->R, rtol, x0_zero ? 1 : 0, c->d_part, mscal(c));
  if ((s = check_launch(c, "mcg_init"))) return s;
  const int maxit = c->opt.maxit;
  const int chk = std::max(1, c->opt.check_every);
  int& last = sizeof(TV) == 4 ? c->last_it32 : c->last_it64;
  const int first = std::max(2, std::min(chk, last - 1));
  int it = 0;
  c->h_mint[0] = 0;
  CUDA_TRY(c, cudaMemcpyAsync(c->h_mint, c->d_mdone, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  auto issue = [&](int it0, int count) {
    for (int i = it0; i < it0 + count; ++i) {
      const int par = i & 1;
      if (sizeof(TV) == 4) {   // the inner solve runs on the context's FP32 vectors
        HDG_DISPATCH(c, m_iter32, c, par, maxit, 0, cudaGraphConditionalHandle{}, i);
        continue;
      }
      c->n_launch += 5;
      HDG_DISPATCH(c, mlaunch_apply64, c, (const double*)p, (double*)slot, c->d_mdone, i);
      HDG_DISPATCH(c, mlaunch_face_q64, c, (const double*)slot, (const double*)p, (double*)q);
      mcols_alpha<<<1, 256, 0, c->stream>>>(nb, c->R, par, c->d_part, mscal(c));
      mupdate_cols(c, n, p, q, dinv, x, r, z);
      mcols_beta<<<1, 256, 0, c->stream>>>(nb, c->R, par, maxit, c->d_part, mscal(c), c->d_mbeta, 0, 0);
      mdirection_cols(c, n, r, z, dinv, p);
    }
  };
  // graph mode: chunks of GCH iterations (even, so the parity pattern repeats) captured once
  const int GCH = 4;
  cudaGraphExec_t gexec = nullptr;
  if (c->opt.use_graphs && !c->stats_on) {
    const std::pair<int, const void*> key((int)sizeof(TV), (const void*)x);
    for (auto& g : c->graphs)
      if (g.first == key) gexec = g.second;
    if (!gexec) {
      // the context's stream must be its own (a stream shared with another context would
      // capture that context's launches too); the capture is always ended, even on error
      cudaGraph_t graph = nullptr;
      CUDA_TRY(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
      issue(0, GCH);
      const cudaError_t le = cudaGetLastError();
      cudaError_t ce = cudaStreamEndCapture(c->stream, &graph);
      if (le != cudaSuccess || ce != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return fail(c, HDG_ECUDA, std::string("graph capture: ") + cudaGetErrorString(le != cudaSuccess ? le : ce));
      }
      ce = cudaGraphInstantiate(&gexec, graph, 0);
      cudaGraphDestroy(graph);
      if (ce != cudaSuccess) return fail(c, HDG_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(ce));
      c->graphs.push_back({key, gexec});
    }
  }
  while (!c->h_mint[0] && it < maxit) {
    if (gexec) {
      const int reps = it == 0 ? std::max(1, (first + GCH - 1) / GCH) : 1;
      for (int rr = 0; rr < reps; ++rr) CUDA_TRY(c, cudaGraphLaunch(gexec, c->stream));
      it += reps * GCH;
    } else {
      const int upto = std::min(maxit, it + (it == 0 ? first : std::min(chk, 3)));
      issue(it, upto - it);
      it = upto;
    }
    if ((s = check_launch(c, "mcg_iter"))) return s;
    CUDA_TRY(c, cudaMemcpyAsync(c->h_mint, c->d_mdone, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(c->h_mint + 2, c->d_miters, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    harvest(c, c->h_mint[0] ? c->h_mint[2] : (1 << 30));
  }
  *iters_out = c->h_mint[2];
  last = std::max(1, c->h_mint[2]);
  if (c->h_mint[0] == 0 || c->h_mint[0] == 2) return fail(c, HDG_ENOCONV, "multi-column Krylov solve reached maxit");
  return HDG_OK;
}

// Device-driven multi-column solve (one graph launch): the per-column Krylov iterations run as
// a WHILE loop whose condition the single-block beta kernel sets, and the mixed-precision sweeps
// as an outer WHILE loop with a one-thread control kernel (all columns converged / max_sweeps).
hdg_status msolve_graph(hdg_ctx* c, const double* b, double* x, hdg_solve_info* info) {
  const int64_t n = c->sk.nf * c->Nf * (int64_t)c->R;
  const int nb = c->nb_red, maxit = c->opt.maxit, R = c->R;
  const bool mixed = c->opt.prec != HDG_FP64;
  auto iters = [&](bool f32, cudaGraphConditionalHandle h) {
    for (int par = 0; par < 2; ++par) {
      if (f32) {
        HDG_DISPATCH(c, m_iter32, c, par, maxit, 1, h, -1);
      } else {
        c->n_launch += 5;
        HDG_DISPATCH(c, mlaunch_apply64, c, (const double*)c->d_p, c->d_mslot, c->d_mdone, -1);
        HDG_DISPATCH(c, mlaunch_face_q64, c, (const double*)c->d_mslot, (const double*)c->d_p, c->d_q);
        mcols_alpha<<<1, 256, 0, c->stream>>>(nb, R, par, c->d_part, mscal(c));
        mupdate_kernel<double><<<nb, 256, 0, c->stream>>>(n, R, c->d_p, c->d_q, c->d_dinv, x, c->d_r, c->d_z, c->d_part,
                                                          mscal(c));
        mcols_beta<<<1, 256, 0, c->stream>>>(nb, R, par, maxit, c->d_part, mscal(c), c->d_mbeta, 1, h);
        mdirection_kernel<double><<<nb, 256, 0, c->stream>>>(n, R, c->d_z, c->d_p, c->d_mbeta, c->d_mdone);
      }
    }
  };
  auto build = [&](GraphBuild& gb, cudaGraph_t G, hdg_ctx::DevGraph& dg) {
    std::vector<cudaGraphNode_t> deps, bd, di;
    const int64_t n0 = c->n_launch;
    if (!mixed) {
      gb.seq(G, deps, [&] {
        HDG_DISPATCH(c, mlaunch_apply64, c, (const double*)x, c->d_mslot, (const int*)nullptr, -1);
        c->n_launch += 2;
        HDG_DISPATCH(c, mlaunch_init64, c, (const double*)c->d_mslot, b, (const double*)c->d_dinv, c->d_r, c->d_z, c->d_p);
        mcols_init<<<1, 256, 0, c->stream>>>(nb, R, c->opt.rtol, 0, c->d_part, mscal(c));
      });
      const cudaGraphConditionalHandle h = gb.handle(G, 1, true);
      cudaGraph_t B = gb.loop(G, deps, h);
      const int64_t n1 = c->n_launch;
      gb.seq(B, bd, [&] { iters(false, h); });
      const int64_t n2 = c->n_launch;
      gb.seq(G, deps, [&] {
        c->n_launch += 1;
        mcg_finish_kernel<<<1, 32, 0, c->stream>>>(c->d_mdone, c->d_miters, c->d_lc);
      });
      dg.n_static = (n1 - n0) + (c->n_launch - n2);
      dg.n_body = 0;
      dg.n_trip = n2 - n1;
      return;
    }
    gb.seq(G, deps, [&] {
      c->n_launch += 1;
      loopctl_init_kernel<<<1, 32, 0, c->stream>>>(c->d_lc, 0);
    });
    const cudaGraphConditionalHandle h_sweep = gb.handle(G, 1, true);
    cudaGraph_t B = gb.loop(G, deps, h_sweep);
    const cudaGraphConditionalHandle h_in = gb.handle(B, 0, false);
    const int64_t n1 = c->n_launch;
    gb.seq(B, bd, [&] {
      HDG_DISPATCH(c, mlaunch_apply_df, c, (const double*)x, c->d_mslot);
      HDG_DISPATCH(c, mlaunch_refres, c, b);
      c->n_launch += 4;
      msweep_ctl_kernel<<<1, 32, 0, c->stream>>>(c->d_mnconv, c->d_miters, c->d_lc, c->opt.max_sweeps, h_sweep, h_in);
      mto32_cols(c, n);
      cudaMemsetAsync(c->d_x32, 0, (size_t)n * sizeof(float), c->stream);
      HDG_DISPATCH(c, mlaunch_init32, c, (const float*)nullptr, (const float*)c->d_b32, (const float*)c->d_dinv32,
                   c->d_r32, c->d_z32, c->d_p32);
      mcols_init<<<1, 256, 0, c->stream>>>(nb, R, c->opt.inner_rtol, 1, c->d_part, mscal(c), c->d_mrr2, c->d_mbb2,
                                           c->opt.rtol);
    });
    const int64_t n2 = c->n_launch;
    cudaGraph_t BI = gb.loop(B, bd, h_in);
    gb.seq(BI, di, [&] { iters(true, h_in); });
    const int64_t n3 = c->n_launch;
    gb.seq(B, bd, [&] {
      c->n_launch += 1;
      mrefine_update_cols(c, n, x);
    });
    const int64_t n4 = c->n_launch;
    dg.n_static = n1 - n0;
    dg.n_body = (n2 - n1) + (n4 - n3);
    dg.n_trip = n3 - n2;
  };
  hdg_status s = devgraph_solve(c, 6, b, x, build, info);
  if (s != HDG_OK) return s;
  // the worst column's relative residual (FP64 path: the CG recurrence's; mixed: the last sweep's)
  std::vector<double> rr(R), bb(R);
  CUDA_TRY(c, cudaMemcpyAsync(rr.data(), mixed ? c->d_mrr2 : c->d_mrr, R * 8, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(bb.data(), mixed ? c->d_mbb2 : c->d_mbb, R * 8, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  double worst = 0.0;
  for (int j = 0; j < R; ++j) worst = std::max(worst, bb[j] > 0 ? std::sqrt(rr[j] / bb[j]) : 0.0);
  if (info) info->rel_residual = std::max(info->rel_residual, worst);
  return HDG_OK;
}

hdg_status msolve(hdg_ctx* c, const double* b, double* x, hdg_solve_info* info) {
  if (c->opt.device_loops && !c->stats_on && c->d_lc) return msolve_graph(c, b, x, info);
  const int64_t n = c->sk.nf * c->Nf * (int64_t)c->R;
  hdg_status s;
  if (c->opt.prec == HDG_FP64) {
    int it = 0;
    if ((s = mcg<double>(c, b, x, c->d_r, c->d_z, c->d_p, c->d_q, c->d_mslot, c->d_dinv, c->opt.rtol, false, &it))) return s;
    std::vector<double> rr(c->R), bb(c->R);
    CUDA_TRY(c, cudaMemcpyAsync(rr.data(), c->d_mrr, c->R * 8, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(bb.data(), c->d_mbb, c->R * 8, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    double worst = 0.0;
    for (int j = 0; j < c->R; ++j) worst = std::max(worst, bb[j] > 0 ? std::sqrt(rr[j] / bb[j]) : 0.0);
    if (info) { info->iterations += it; info->sweeps += 1; info->rel_residual = std::max(info->rel_residual, worst); }
    return HDG_OK;
  }
  int total = 0;
  for (int sweep = 0;; ++sweep) {
    HDG_DISPATCH(c, mlaunch_apply_df, c, (const double*)x, c->d_mslot);
    HDG_DISPATCH(c, mlaunch_refres, c, b);
    if ((s = check_launch(c, "mrefine_residual"))) return s;
    CUDA_TRY(c, cudaMemcpyAsync(c->h_mint + 1, c->d_mnconv, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    harvest(c);
    if (c->h_mint[1] == 0 || sweep >= c->opt.max_sweeps) {
      std::vector<double> rr(c->R), bb(c->R);
      CUDA_TRY(c, cudaMemcpyAsync(rr.data(), c->d_mrr2, c->R * 8, cudaMemcpyDeviceToHost, c->stream));
      CUDA_TRY(c, cudaMemcpyAsync(bb.data(), c->d_mbb2, c->R * 8, cudaMemcpyDeviceToHost, c->stream));
      CUDA_TRY(c, cudaStreamSynchronize(c->stream));
      double worst = 0.0;
      for (int j = 0; j < c->R; ++j) worst = std::max(worst, bb[j] > 0 ? std::sqrt(rr[j] / bb[j]) : 0.0);
      if (info) { info->iterations += total; info->sweeps += sweep; info->rel_residual = std::max(info->rel_residual, worst); }
      if (c->h_mint[1] != 0) return fail(c, HDG_ENOCONV, "multi-column refinement reached max_sweeps");
      return HDG_OK;
    }
    c->n_launch += 1;
    mto32_cols(c, n);
    int it = 0;
    if ((s = mcg<float>(c, c->d_b32, c->d_x32, c->d_r32, c->d_z32, c->d_p32, c->d_q32, c->d_mslot32, c->d_dinv32,
                        c->opt.inner_rtol, true, &it)))
      if (s != HDG_ENOCONV) return s;
    total += it;
    c->n_launch += 1;
    mrefine_update_cols(c, n, x);
    if ((s = check_launch(c, "mrefine_update"))) return s;
  }
}


// one implicit solve at mass shift alpha: alpha Mw u + f(u, lam, t) = alpha Mw hist
hdg_status stage_solve(hdg_ctx* c, const double* hist, double tt, double* uout, hdg_solve_info* info) {
  if (c->vd) return vd_stage_solve(c, hist, tt, uout, info);
  const double fac = std::cos(c->omega * tt + c->phase);
  if (c->R > 1) {
    const int64_t nbe = c->sk.nb * c->Nf * (int64_t)c->R;
    c->n_launch += 1;
    mdirichlet_kernel<<<grid_for(c, nbe), 256, 0, c->stream>>>(c->sk.nb, c->Nf, c->R, c->d_bnd_faces, c->d_bnd_coef, fac,
                                                              c->d_lam);
    HDG_DISPATCH(c, mlaunch_local, c, 0, (const double*)nullptr, hist, tt, c->d_lam, c->d_mslot);
    HDG_DISPATCH(c, mlaunch_gather, c, (const double*)c->d_mslot, 1.0, c->d_b);
    hdg_status s = check_launch(c, "rhs_multi");
    if (s) return s;
    if ((s = guess_before(c))) return s;
    if ((s = msolve(c, c->d_b, c->d_lam, info))) return s;
    if ((s = guess_after(c))) return s;
    HDG_DISPATCH(c, mlaunch_local, c, 1, (const double*)nullptr, hist, tt, c->d_lam, uout);
    return check_launch(c, "recover_multi");
  }
  c->n_launch += 1;
  dirichlet_kernel<<<grid_for(c, c->sk.nb * c->Nf), 256, 0, c->stream>>>(c->sk.nb, c->Nf, c->d_bnd_faces, c->d_bnd_coef, fac,
                                                                         c->d_lam);
  HDG_DISPATCH(c, launch_local, c, 0, (const double*)nullptr, hist, tt, c->d_lam, c->d_slot);
  hdg_status s = check_launch(c, "rhs");
  if (s) return s;
  // Krylov right-hand side b = sgn r = -sgn sum_K C_K A_K^{-1} F~_K
  if ((s = faces_from_slots(c, -c->sgn, c->d_b))) return s;
  if (c->tspace) {
    // continuous traces: b_mu = R^T b, solve on the free nodes, lam = R mu on interior faces
    if ((s = edg_restrict(c, c->d_b, c->d_bmu))) return s;
    if ((s = guess_before_v(c, c->n_mu, c->d_bmu, c->d_mu, nullptr))) return s;
    if ((s = edg_solve(c, c->d_bmu, c->d_mu, info))) return s;
    if ((s = guess_after_v(c, c->n_mu, c->d_bmu, c->d_mu))) return s;
    HDG_DISPATCH(c, edg_expand64, c, c->d_mu, c->d_lam, 0);
    HDG_DISPATCH(c, launch_local, c, 1, (const double*)nullptr, hist, tt, c->d_lam, uout);
    return check_launch(c, "recover");
  }
  if ((s = guess_before(c))) return s;
  c->guess_x = true;
  s = cg_solve(c, c->d_b, c->d_lam, info);
  c->guess_x = false;
  if (s) return s;
  if ((s = guess_after(c))) return s;
  HDG_DISPATCH(c, launch_local, c, 1, (const double*)nullptr, hist, tt, c->d_lam, uout);
  return check_launch(c, "recover");
}

hdg_status ensure_alpha(hdg_ctx* c, double alpha) {
  if (c->condensed && std::fabs(alpha - c->alpha) <= 1e-14 * alpha) return HDG_OK;
  return do_condense(c, alpha);
}

void combine(hdg_ctx* c, double* out, double c0, const double* i0, double c1 = 0, const double* i1 = nullptr,
             double c2 = 0, const double* i2 = nullptr, double c3 = 0, const double* i3 = nullptr) {
  const int64_t n = c->nfld * (int64_t)c->R;
  c->n_launch += 1;
  combine_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(n, c0, i0, c1, i1, c2, i2, c3, i3, out);
}

// Alexander's L-stable DIRK(3,3): gamma is the root in (1/3, 1/2) of
// gamma^3 - 3 gamma^2 + 3/2 gamma - 1/6 = 0.
void dirk3(double a[3][3], double b[3], double cc[3]) {
  double g = 0.4358;
  for (int i = 0; i < 60; ++i) {
    const double f = ((g - 3.0) * g + 1.5) * g - 1.0 / 6.0, df = (3.0 * g - 6.0) * g + 1.5;
    g -= f / df;
  }
  const double b1 = -(6 * g * g - 16 * g + 1) / 4, b2 = (6 * g * g - 20 * g + 5) / 4;
  double A[3][3] = {{g, 0, 0}, {(1 - g) / 2, g, 0}, {b1, b2, g}};
  std::memcpy(a, A, sizeof(A));
  b[0] = b1; b[1] = b2; b[2] = g;
  cc[0] = g; cc[1] = (1 + g) / 2; cc[2] = 1.0;
}

}  // namespace

// entry points of this unit used by the other translation units
hdg_status trace_cg_solve(hdg_ctx* c, const double* b, double* x, hdg_solve_info* info) { return cg_solve(c, b, x, info); }
void dirk3_tableau(double a[3][3], double b[3], double cc[3]) { dirk3(a, b, cc); }

// ---- least-squares initial guess over earlier stage solutions (same alpha)
// The stored pairs satisfy K lam_i = b_i to the solver tolerance, so minimising
// |b - K sum c_i lam_i| over the span needs only the Gram matrix of the stored b_i and their
// dot products with the new b: damped normal equations (G + mu I) c = g, solved on the host,
// per column when there are several right-hand sides.
hdg_status guess_setup(hdg_ctx* c, const uint8_t* host_mask) {
  c->g_q = 0;
  hdg_status s;
  // the interior-entry mask and the control block of the device-driven solves exist always
  if ((s = dalloc(c, &c->d_intmask, (size_t)c->ntr))) return s;
  CUDA_TRY(c, cudaMemcpyAsync(c->d_intmask, host_mask, (size_t)c->ntr, cudaMemcpyHostToDevice, c->stream));
  if ((s = dalloc(c, &c->d_lc, 1))) return s;
  CUDA_TRY(c, cudaMallocHost((void**)&c->h_lc, sizeof(LoopCtl)));
  if (c->opt.guess_history <= 0) {
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));   // host_mask is released at return
    return HDG_OK;
  }
  const int q = std::min(c->opt.guess_history, 8), R = c->R;
  const size_t n = (size_t)c->ntr * R;
  if ((s = dalloc(c, &c->d_gb, q * n))) return s;
  if ((s = dalloc(c, &c->d_gl, q * n))) return s;
  if ((s = dalloc(c, &c->d_gdots, (size_t)9 * R))) return s;
  if ((s = dalloc(c, &c->d_gpart, (size_t)c->nb_red * 9 * R))) return s;
  if (R > 1) {
    if ((s = dalloc(c, &c->d_gcoef, (size_t)8 * R))) return s;
    c->gm_gram.assign((size_t)R * 64, 0.0);
    c->gm_dots.assign((size_t)9 * R, 0.0);
    c->gm_coef.assign((size_t)8 * R, 0.0);
  } else {
    if ((s = dalloc(c, &c->d_gd, 1))) return s;
  }
  CUDA_TRY(c, cudaMemsetAsync(c->d_gb, 0, q * n * 8, c->stream));
  CUDA_TRY(c, cudaMemsetAsync(c->d_gl, 0, q * n * 8, c->stream));
  c->g_q = q;
  guess_clear(c);
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return check_launch(c, "guess_setup");
}

// forget the stored pairs (new operator or new state)
void guess_clear(hdg_ctx* c) {
  c->g_n = c->g_next = 0;
  if (c->d_gd) {
    c->n_launch += 1;
    guess_reset_kernel<<<1, 32, 0, c->stream>>>(c->d_gd, c->g_q);
  }
}

namespace {
// (G + mu I) x = g for an m x m Gram matrix G (row stride 8), mu = 1e-13 max diag; false when
// G is zero or the factorisation breaks down (the caller keeps its current guess)
bool ls_solve(int m, const double* G, const double* g, double* x) {
  double L[8][8] = {}, y[8], dmax = 0.0;
  for (int i = 0; i < m; ++i) dmax = std::max(dmax, G[i * 8 + i]);
  if (!(dmax > 0.0)) return false;
  for (int j = 0; j < m; ++j) {
    double d = G[j * 8 + j] + 1e-13 * dmax;
    for (int k = 0; k < j; ++k) d -= L[j][k] * L[j][k];
    if (!(d > 0.0)) return false;
    L[j][j] = std::sqrt(d);
    for (int i = j + 1; i < m; ++i) {
      double v = G[i * 8 + j];
      for (int k = 0; k < j; ++k) v -= L[i][k] * L[j][k];
      L[i][j] = v / L[j][j];
    }
  }
  for (int i = 0; i < m; ++i) {
    double v = g[i];
    for (int k = 0; k < i; ++k) v -= L[i][k] * y[k];
    y[i] = v / L[i][i];
  }
  for (int i = m - 1; i >= 0; --i) {
    double v = y[i];
    for (int k = i + 1; k < m; ++k) v -= L[k][i] * x[k];
    x[i] = v / L[i][i];
  }
  return true;
}
}  // namespace

// one column, on the device: dots of the new right-hand side b (n entries) with the stored
// b_i, the damped normal equations, and the combination written into x (entries with mask != 0;
// null mask: every entry)
hdg_status guess_before_v(hdg_ctx* c, int64_t n, const double* b, double* x, const uint8_t* mask) {
  if (!c->g_q) return HDG_OK;
  const int nb = c->nb_red;
  c->n_launch += 3;
  gdots_kernel<<<nb, 256, 0, c->stream>>>(n, c->d_gd, c->d_gb, b, c->d_gpart);
  gsolve_kernel<<<1, 256, 0, c->stream>>>(nb, c->d_gpart, c->d_gd);
  glincomb_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(n, c->d_gd, c->d_gl, mask, x);
  return check_launch(c, "guess");
}

// one column: store (b, x) of the solve just finished and update the Gram matrix
hdg_status guess_after_v(hdg_ctx* c, int64_t n, const double* b, const double* x) {
  if (!c->g_q) return HDG_OK;
  c->n_launch += 2;
  gstore_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(n, c->d_gd, b, x, c->d_gb, c->d_gl);
  gupdate_kernel<<<1, 32, 0, c->stream>>>(c->d_gd);
  c->g_next = (c->g_next + 1) % c->g_q;
  c->g_n = std::min(c->g_n + 1, c->g_q);
  return check_launch(c, "guess_store");
}

hdg_status guess_before(hdg_ctx* c) {
  if (!c->g_q) return HDG_OK;
  const int R = c->R, m = c->g_n, nb = c->nb_red;
  const int64_t n = c->ntr * (int64_t)R;
  if (R == 1) return guess_before_v(c, n, c->d_b, c->d_lam, c->d_intmask);
  c->n_launch += 2;
  mdots_ring_kernel<<<nb, 256, 0, c->stream>>>(n, R, m, n, c->d_gb, c->d_b, c->d_gpart);
  mdots_final_kernel<<<1, 256, 0, c->stream>>>(nb, R, m, c->d_gpart, c->d_gdots);
  CUDA_TRY(c, cudaMemcpyAsync(c->gm_dots.data(), c->d_gdots, (size_t)(m + 1) * R * sizeof(double),
                              cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (m == 0) return HDG_OK;
  bool any = false;
  for (int j = 0; j < R; ++j) {
    double g[8], x[8];
    for (int i = 0; i < m; ++i) g[i] = c->gm_dots[(size_t)i * R + j];
    const bool ok = ls_solve(m, &c->gm_gram[(size_t)j * 64], g, x);
    any = any || ok;
    // a column without a usable history (all its pairs reset) keeps its current guess: NaN
    // in its first coefficient tells the combination kernel to skip it
    for (int i = 0; i < 8; ++i) c->gm_coef[(size_t)i * R + j] = ok && i < m ? x[i] : 0.0;
    if (!ok) c->gm_coef[(size_t)0 * R + j] = std::nan("");
  }
  if (!any) return HDG_OK;
  CUDA_TRY(c, cudaMemcpyAsync(c->d_gcoef, c->gm_coef.data(), (size_t)8 * R * sizeof(double), cudaMemcpyHostToDevice,
                              c->stream));
  c->n_launch += 1;
  mlincomb_ring_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(n, R, m, n, c->d_gl, c->d_gcoef, c->d_intmask, c->d_lam);
  return check_launch(c, "guess_multi");
}

hdg_status guess_after(hdg_ctx* c) {
  if (!c->g_q) return HDG_OK;
  const int R = c->R;
  const int64_t n = c->ntr * (int64_t)R;
  const int s = c->g_next;
  if (R == 1) return guess_after_v(c, n, c->d_b, c->d_lam);
  CUDA_TRY(c, cudaMemcpyAsync(c->d_gb + (int64_t)s * n, c->d_b, n * 8, cudaMemcpyDeviceToDevice, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(c->d_gl + (int64_t)s * n, c->d_lam, n * 8, cudaMemcpyDeviceToDevice, c->stream));
  for (int j = 0; j < R; ++j) {
    double* G = &c->gm_gram[(size_t)j * 64];
    for (int i = 0; i < c->g_n; ++i)
      if (i != s) G[s * 8 + i] = G[i * 8 + s] = c->gm_dots[(size_t)i * R + j];
    G[s * 8 + s] = c->gm_dots[(size_t)c->g_n * R + j];
  }
  c->g_next = (s + 1) % c->g_q;
  c->g_n = std::min(c->g_n + 1, c->g_q);
  return HDG_OK;
}

// a column that restarts (serving: a new request in a slot) drops its stored pairs
void guess_reset_column(hdg_ctx* c, int j) {
  if (!c->g_q || c->R == 1) return;
  // zero_column_kernel takes the entries of one column (ntr); a slot holds ntr x R values
  const int64_t per_col = c->ntr, slot = c->ntr * (int64_t)c->R;
  for (int i = 0; i < c->g_q; ++i) {
    c->n_launch += 2;
    zero_column_kernel<<<grid_for(c, per_col), 256, 0, c->stream>>>(per_col, c->R, j, c->d_gb + (int64_t)i * slot);
    zero_column_kernel<<<grid_for(c, per_col), 256, 0, c->stream>>>(per_col, c->R, j, c->d_gl + (int64_t)i * slot);
  }
  std::fill(c->gm_gram.begin() + (size_t)j * 64, c->gm_gram.begin() + (size_t)(j + 1) * 64, 0.0);
}

namespace {
template <int DIM, int K>
void launch_post(hdg_ctx* c, const double* u, const double* lam, double* pstar) {
  const PostTabs P{c->d_post, c->d_post + c->post_k1};
  c->n_launch += 1;
  post_kernel<DIM, K><<<grid_for(c, c->sk.ne * PostCfg<DIM, K>::NT, PostCfg<DIM, K>::NT), PostCfg<DIM, K>::NT, 0,
                        c->stream>>>(devmesh(c), c->tabs, P, u, lam, pstar);
}
}  // namespace

extern "C" {

void hdg_default_options(hdg_options* o) {
  if (!o) return;
  o->prec = HDG_FP64;
  o->rtol = 1e-13;
  o->maxit = 2000;
  o->check_every = 16;
  o->inner_rtol = 1e-4;
  o->max_sweeps = 20;
  o->nrhs = 1;
  o->use_graphs = 0;
  o->guess_history = 8;
  o->device_loops = 1;
  o->trace_space = HDG_TRACE_HDG;
  o->solver = HDG_SOLVER_CG;
  o->gmres_restart = 40;
  o->newton_tol = 1e-11;
  o->newton_maxit = 25;
  o->precond = HDG_PRECOND_JACOBI;
}

const char* hdg_last_error(const hdg_ctx* c) { return c ? c->err.c_str() : "null context"; }

hdg_status hdg_host_skeleton(int32_t dim, int64_t n_vert, int64_t n_elem, const double* vert, const int32_t* elem,
                             int64_t* n_faces, int32_t* elem_face, int32_t* face_slot, int32_t* face_bnd,
                             double* geo) {
  if (!vert || !elem || !n_faces || !elem_face || !face_slot || !face_bnd || !geo) return HDG_EINVAL;
  Skeleton sk;
  std::string err;
  if (!build_skeleton(dim, n_vert, n_elem, vert, elem, sk, err)) return HDG_EINVAL;
  *n_faces = sk.nf;
  std::copy(sk.elem_face.begin(), sk.elem_face.end(), elem_face);
  std::copy(sk.face_slot.begin(), sk.face_slot.end(), face_slot);
  std::copy(sk.face_bnd.begin(), sk.face_bnd.end(), face_bnd);
  std::copy(sk.geo.begin(), sk.geo.end(), geo);
  return HDG_OK;
}

hdg_status hdg_host_trace_nodes(int32_t dim, int64_t n_vert, int64_t n_elem, const double* vert, const int32_t* elem,
                                int32_t k, int32_t all_faces, int64_t* n_free, int32_t* face_node, double* Vinv) {
  if (!vert || !elem || !n_free || !face_node || !Vinv) return HDG_EINVAL;
  Skeleton sk;
  std::string err;
  if (!build_skeleton(dim, n_vert, n_elem, vert, elem, sk, err)) return HDG_EINVAL;
  std::vector<int32_t> fn;
  int64_t nfree = 0;
  if (!build_trace_nodes(sk, k, all_faces != 0, nfree, fn, err)) return HDG_EINVAL;
  std::vector<double> T;
  try {
    T = face_nodal_to_modal(dim, k);
  } catch (const std::exception&) {
    return HDG_EINVAL;
  }
  *n_free = nfree;
  std::copy(fn.begin(), fn.end(), face_node);
  std::copy(T.begin(), T.end(), Vinv);
  return HDG_OK;
}

hdg_status hdg_host_tables(int32_t dim, int32_t k, double* Dr, double* Ff, double* K1, double* E1) {
  if (dim < 2 || dim > 3 || k < 1 || k > 4) return HDG_EINVAL;
  try {
    const RefTables T = build_tables(dim, k);
    if (Dr) std::copy(T.Dr.begin(), T.Dr.end(), Dr);
    if (Ff) std::copy(T.Ff.begin(), T.Ff.end(), Ff);
    if (K1 || E1) {
      const PostTables P = build_post_tables(dim, k);
      if (K1) std::copy(P.K1.begin(), P.K1.end(), K1);
      if (E1) std::copy(P.E1.begin(), P.E1.end(), E1);
    }
  } catch (const std::exception&) {
    return HDG_EINVAL;
  }
  return HDG_OK;
}

void hdg_destroy(hdg_ctx* c) {
  if (!c) return;
  for (auto& g : c->graphs) cudaGraphExecDestroy(g.second);
  for (auto& g : c->dgraphs) cudaGraphExecDestroy(g.exec);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->h_lc) cudaFreeHost(c->h_lc);
  if (c->h_sacc) cudaFreeHost(c->h_sacc);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  for (void* p : c->allocs) cudaFree(p);
  if (c->h_sc) cudaFreeHost(c->h_sc);
  if (c->h_rs) cudaFreeHost(c->h_rs);
  if (c->h_mint) cudaFreeHost(c->h_mint);
  vd_destroy(c);
  svk_destroy(c);
  bilu_destroy(c);
  delete c;
}

hdg_status hdg_setup(const hdg_mesh* mesh, int32_t k, double tau, const hdg_material* mat, const hdg_options* opt,
                     void* cuda_stream, hdg_ctx** out) {
  if (!out) return HDG_EINVAL;
  *out = nullptr;
  hdg_ctx* c = new (std::nothrow) hdg_ctx();
  if (!c) return HDG_ENOMEM;
  *out = c;
  if (!mesh || !mat || !mesh->vert || !mesh->elem_vert || !mat->rho || (mat->phys == HDG_ACOUSTIC && !mat->c))
    return fail(c, HDG_EINVAL, "null mesh or material pointer");
  if (k < 1 || k > 4) return fail(c, HDG_EINVAL, "degree k must be in 1..4");
  if (!(tau > 0.0)) return fail(c, HDG_EINVAL, "tau must be positive");
  if (opt) c->opt = *opt; else hdg_default_options(&c->opt);
  if (c->opt.prec != HDG_FP64 && c->opt.prec != HDG_MIXED && c->opt.prec != HDG_MIXED16)
    return fail(c, HDG_EINVAL, "unknown precision mode");
  if (!(c->opt.rtol > 0.0) || c->opt.maxit < 1) return fail(c, HDG_EINVAL, "rtol must be > 0 and maxit >= 1");
  if (c->opt.prec != HDG_FP64 && (!(c->opt.inner_rtol > 0.0) || !(c->opt.inner_rtol < 1.0) || c->opt.max_sweeps < 1))
    return fail(c, HDG_EINVAL, "mixed precision needs 0 < inner_rtol < 1 and max_sweeps >= 1");
  if (c->opt.nrhs < 1 || c->opt.nrhs > 256 || (c->opt.nrhs & (c->opt.nrhs - 1)))
    return fail(c, HDG_EINVAL, "nrhs must be a power of two in 1..256");
  c->R = c->opt.nrhs;
  c->tspace = c->opt.trace_space;
  if (c->tspace < HDG_TRACE_HDG || c->tspace > HDG_TRACE_EDG) return fail(c, HDG_EINVAL, "unknown trace space");
  if (c->tspace != HDG_TRACE_HDG &&
      (mat->phys != HDG_ACOUSTIC || c->R != 1 || mesh->elem_k || !c->opt.device_loops))
    return fail(c, HDG_EINVAL, "IEDG / EDG traces: acoustic, uniform degree, nrhs = 1 and device_loops = 1 only");
  if (c->opt.solver != HDG_SOLVER_CG && c->opt.solver != HDG_SOLVER_GMRES) return fail(c, HDG_EINVAL, "unknown solver");
  if (c->opt.solver == HDG_SOLVER_GMRES &&
      (c->opt.prec != HDG_FP64 || c->R != 1 || mesh->elem_k || c->tspace != HDG_TRACE_HDG ||
       c->opt.gmres_restart < 2 || c->opt.gmres_restart > 64))
    return fail(c, HDG_EINVAL, "GMRES: FP64, HDG traces, uniform degree, nrhs = 1 and 2 <= gmres_restart <= 64 only");
  if (c->opt.precond != HDG_PRECOND_JACOBI && c->opt.precond != HDG_PRECOND_BILU0)
    return fail(c, HDG_EINVAL, "unknown preconditioner");
  if (c->opt.precond == HDG_PRECOND_BILU0 && c->opt.solver != HDG_SOLVER_GMRES)
    return fail(c, HDG_EINVAL, "block ILU(0) preconditions the GMRES solver only");
  std::string err;
  const bool svk = mat->phys == HDG_SVK;
  if (mat->phys != HDG_ACOUSTIC && mat->phys != HDG_ELASTIC && !svk) return fail(c, HDG_EINVAL, "unknown physics");
  if (svk && (mesh->dim != 3 || k > 3 || mesh->elem_k || c->R != 1 || c->tspace != HDG_TRACE_HDG ||
              c->opt.solver != HDG_SOLVER_CG || c->opt.prec == HDG_MIXED16))
    return fail(c, HDG_EINVAL, "SVK: 3D, uniform k in 1..3, nrhs = 1, HDG traces, CG, FP64 or MIXED only");
  // HDG_MIXED: FP32 Jacobian (tangent, condensation, factor) around the FP64 residual, and
  // the trace system of each Newton iteration solved by FP32 CG inside FP64 refinement
  if (svk) c->svk_mixed = c->opt.prec == HDG_MIXED;
  if (svk && (!(c->opt.newton_tol > 0.0) || c->opt.newton_maxit < 1))
    return fail(c, HDG_EINVAL, "SVK: newton_tol must be > 0 and newton_maxit >= 1");
  // SVK contexts share the elastic trace layout (3 N_f velocity traces per face)
  c->phys = svk ? HDG_ELASTIC : mat->phys;
  if (svk) c->opt.guess_history = 0;
  if (c->phys == HDG_ELASTIC && (!mat->lam || !mat->mu)) return fail(c, HDG_EINVAL, "elastic material needs lam and mu");
  if (c->phys == HDG_ELASTIC && c->opt.nrhs != 1) return fail(c, HDG_EINVAL, "elastic path supports nrhs = 1 only");
  // uniform degree 4 in 3D elastic runs through the per-element-degree path (its local
  // velocity block does not fit shared memory in the uniform condensation kernel)
  std::vector<int32_t> k4;
  const int32_t* elem_k = mesh->elem_k;
  if (!elem_k && mat->phys == HDG_ELASTIC && mesh->dim == 3 && k == 4) {
    k4.assign((size_t)std::max<int64_t>(mesh->n_elem, 0), 4);
    elem_k = k4.data();
  }
  if (elem_k && (mat->phys != HDG_ELASTIC || mesh->dim != 3))
    return fail(c, HDG_EINVAL, "per-element degrees: 3D elastic meshes only");
  if (elem_k && c->opt.nrhs != 1) return fail(c, HDG_EINVAL, "per-element degrees: nrhs = 1 only");
  for (int64_t e = 0; elem_k && e < mesh->n_elem; ++e)
    if (elem_k[e] < 1 || elem_k[e] > 4) return fail(c, HDG_EINVAL, "per-element degree must be in 1..4");
  if (!build_skeleton(mesh->dim, mesh->n_vert, mesh->n_elem, mesh->vert, mesh->elem_vert, c->sk, err))
    return fail(c, HDG_EINVAL, err);
  for (int64_t e = 0; e < mesh->n_elem; ++e) {
    if (!(mat->rho[e] > 0.0)) return fail(c, HDG_EINVAL, "rho must be positive");
    if (c->phys == HDG_ACOUSTIC && !(mat->c[e] > 0.0)) return fail(c, HDG_EINVAL, "c must be positive");
    if (c->phys == HDG_ELASTIC && (!(mat->mu[e] > 0.0) || !(mesh->dim * mat->lam[e] + 2.0 * mat->mu[e] > 0.0)))
      return fail(c, HDG_EINVAL, "Lame parameters must satisfy mu > 0 and d lam + 2 mu > 0");
  }
  c->dim = mesh->dim; c->k = k; c->tau = tau;
  try {
    c->T = build_tables(c->dim, k);
  } catch (const std::exception& ex) {
    return fail(c, HDG_EINVAL, ex.what());
  }
  if (svk) {
    // the SVK stress term F S(F) phi has degree 4k: volume rule of 2k + 2 points per direction
    simplex_rule(3, 2 * k + 2, c->T.qv_pts, c->T.qv_w);
    c->T.nqv = (int)c->T.qv_w.size();
    c->T.qv_phi.assign((size_t)c->T.nqv * c->T.Np, 0.0);
    dubiner(3, k, c->T.qv_pts.data(), c->T.nqv, c->T.qv_phi.data(), nullptr);
  }
  c->Np = c->T.Np; c->nfc = c->dim + 1;
  if (c->phys == HDG_ELASTIC) {
    const int nt = c->dim * (c->dim + 1) / 2;
    c->ncomp = svk ? 21 : c->dim + nt;
    c->Nf = c->dim * c->T.Nf;          // trace DOFs per face: d velocity components
    c->nv = c->dim * c->Np;
    c->sgn = 1.0;
  } else {
    c->ncomp = c->dim + 1;
    c->Nf = c->T.Nf;
    c->nv = c->Np;
    c->sgn = -1.0;
  }
  c->n = c->ncomp * c->Np; c->m = c->nfc * c->Nf;
  c->stream = (cudaStream_t)cuda_stream;
  int dev = 0;
  CUDA_TRY(c, cudaGetDevice(&dev));
  CUDA_TRY(c, cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev));
  {
    // reduction grid = one resident wave of the heaviest vector kernel (no partial second wave)
    int per_sm = 4;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cg32_update_kernel, 256, 0) != cudaSuccess || per_sm < 1)
      per_sm = 4;
    c->nb_red = std::max(1, std::min(per_sm * c->sms, (int)((c->sk.nf * c->Nf + 255) / 256)));
  }
  const int64_t ne = c->sk.ne, nf = c->sk.nf, nb = c->sk.nb, nc = c->nfc;
  // element vertex coordinates in sorted order (host, for quadrature points and point location)
  c->h_vert_elem.resize((size_t)ne * nc * c->dim);
  for (int64_t e = 0; e < ne; ++e)
    for (int a = 0; a < nc; ++a)
      for (int r = 0; r < c->dim; ++r)
        c->h_vert_elem[((size_t)e * nc + a) * c->dim + r] = mesh->vert[(int64_t)c->sk.elem[e * nc + a] * c->dim + r];
  hdg_status s;
  if ((s = dalloc(c, &c->d_geo, (size_t)ne * GEO_STRIDE))) return s;
  if ((s = dalloc(c, &c->d_rho, (size_t)ne))) return s;
  if ((s = dalloc(c, &c->d_c, (size_t)ne))) return s;
  if ((s = dalloc(c, &c->d_elem_face, (size_t)ne * nc))) return s;
  if ((s = dalloc(c, &c->d_face_slot, (size_t)nf * 2))) return s;
  if ((s = dalloc(c, &c->d_face_bnd, (size_t)nf))) return s;
  if ((s = dalloc(c, &c->d_bnd_faces, (size_t)nb))) return s;
  CUDA_TRY(c, cudaMemcpyAsync(c->d_geo, c->sk.geo.data(), c->sk.geo.size() * 8, cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(c->d_rho, mat->rho, ne * 8, cudaMemcpyHostToDevice, c->stream));
  if (c->phys == HDG_ACOUSTIC) {
    CUDA_TRY(c, cudaMemcpyAsync(c->d_c, mat->c, ne * 8, cudaMemcpyHostToDevice, c->stream));
  } else {
    if ((s = dalloc(c, &c->d_lame, (size_t)ne))) return s;
    if ((s = dalloc(c, &c->d_mue, (size_t)ne))) return s;
    CUDA_TRY(c, cudaMemcpyAsync(c->d_lame, mat->lam, ne * 8, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(c->d_mue, mat->mu, ne * 8, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(c->d_c, mat->rho, ne * 8, cudaMemcpyHostToDevice, c->stream));   // sound-speed slot unused
  }
  CUDA_TRY(c, cudaMemcpyAsync(c->d_elem_face, c->sk.elem_face.data(), c->sk.elem_face.size() * 4, cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(c->d_face_slot, c->sk.face_slot.data(), c->sk.face_slot.size() * 4, cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(c->d_face_bnd, c->sk.face_bnd.data(), c->sk.face_bnd.size() * 4, cudaMemcpyHostToDevice, c->stream));
  if (nb) CUDA_TRY(c, cudaMemcpyAsync(c->d_bnd_faces, c->sk.bnd_faces.data(), nb * 8, cudaMemcpyHostToDevice, c->stream));
  if (elem_k) {
    if ((s = vd_setup(c, elem_k))) return s;
    c->k = 0;
    for (int64_t e = 0; e < ne; ++e) c->k = std::max(c->k, (int)elem_k[e]);
    c->n = 0; c->m = 0;   // no common local size: fields and traces are flat (nfld, ntr entries)
    return HDG_OK;
  }
  c->nfld = ne * (int64_t)c->n;
  c->ntr = nf * (int64_t)c->Nf;
  c->nschur = ne * (int64_t)c->m * c->m;
  c->nslot = ne * (int64_t)c->m;
  // reference tables packed in one buffer
  std::vector<double> tab;
  size_t off[6];
  const std::vector<double>* parts[6] = {&c->T.Dr, &c->T.Ff, &c->T.Ef, &c->T.Trs, &c->T.DFrf, &c->T.Pfg};
  for (int i = 0; i < 6; ++i) { off[i] = tab.size(); tab.insert(tab.end(), parts[i]->begin(), parts[i]->end()); }
  if ((s = dalloc(c, &c->d_tab, tab.size()))) return s;
  CUDA_TRY(c, cudaMemcpyAsync(c->d_tab, tab.data(), tab.size() * 8, cudaMemcpyHostToDevice, c->stream));
  c->tabs.Dr = c->d_tab + off[0]; c->tabs.Ff = c->d_tab + off[1]; c->tabs.Ef = c->d_tab + off[2];
  c->tabs.Trs = c->d_tab + off[3]; c->tabs.DFrf = c->d_tab + off[4]; c->tabs.Pfg = c->d_tab + off[5];
  if ((s = dalloc(c, &c->d_qv_w, c->T.qv_w.size()))) return s;
  if ((s = dalloc(c, &c->d_qv_phi, c->T.qv_phi.size()))) return s;
  CUDA_TRY(c, cudaMemcpyAsync(c->d_qv_w, c->T.qv_w.data(), c->T.qv_w.size() * 8, cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(c->d_qv_phi, c->T.qv_phi.data(), c->T.qv_phi.size() * 8, cudaMemcpyHostToDevice, c->stream));
  // condensed operators and workspaces
  const size_t nfe = (size_t)nf * c->Nf;
  const size_t R = (size_t)c->R;
  if ((s = dalloc(c, &c->d_S, (size_t)ne * c->m * c->m))) return s;
  if ((s = dalloc(c, &c->d_Hinv, svk ? (size_t)1 : (size_t)ne * c->nv * c->nv))) return s;
  if ((s = dalloc(c, &c->d_dinv, nfe))) return s;
  if ((s = dalloc(c, &c->d_err, 1))) return s;
  for (double** p : {&c->d_r, &c->d_z, &c->d_p, &c->d_q, &c->d_b, &c->d_lam, &c->d_lam_prev, &c->d_lam_prev2, &c->d_lam_x})
    if ((s = dalloc(c, p, nfe * R))) return s;
  // element slots plus one zero slot past the last (the missing neighbour of an SVK traction face)
  if ((s = dalloc(c, &c->d_slot, (size_t)ne * std::max(c->m, 1) + c->Nf))) return s;
  CUDA_TRY(c, cudaMemsetAsync(c->d_slot, 0, ((size_t)ne * std::max(c->m, 1) + c->Nf) * 8, c->stream));
  if ((s = dalloc(c, &c->d_part, (size_t)c->nb_red * 3 * R))) return s;
  if (c->R > 1) {
    if ((s = dalloc(c, &c->d_mslot, (size_t)ne * c->m * R))) return s;
    for (double** p : {&c->d_mrho0, &c->d_mrho1, &c->d_malpha, &c->d_mbeta, &c->d_mrr, &c->d_mbb, &c->d_mtol2, &c->d_mscale,
                       &c->d_mrr2, &c->d_mbb2})
      if ((s = dalloc(c, p, R))) return s;
    if ((s = dalloc(c, &c->d_mconv, R))) return s;
    if ((s = dalloc(c, &c->d_mdone, 1))) return s;
    if ((s = dalloc(c, &c->d_mnconv, 1))) return s;
    if ((s = dalloc(c, &c->d_miters, 1))) return s;
    CUDA_TRY(c, cudaMemsetAsync(c->d_mdone, 0, sizeof(int), c->stream));
    CUDA_TRY(c, cudaMallocHost((void**)&c->h_mint, 4 * sizeof(int)));
  }
  if ((s = dalloc(c, &c->d_sc, 1))) return s;
  CUDA_TRY(c, cudaMallocHost((void**)&c->h_sc, sizeof(CgScal)));
  std::memset(c->h_sc, 0, sizeof(CgScal));
  for (double** p : {&c->d_u, &c->d_uprev, &c->d_h, &c->d_unew, &c->d_stage[0], &c->d_stage[1], &c->d_stage[2]})
    if ((s = dalloc(c, p, (size_t)ne * c->n * R))) return s;
  if (c->opt.prec != HDG_FP64) {
    const int64_t ngroups = (ne + 31) / 32;
    const int P4 = (c->m * (c->m + 1) / 2 + 3) / 4;
    const size_t nS32 = c->phys == HDG_ELASTIC ? (size_t)ne * c->m * c->m : (size_t)ngroups * P4 * 128;
    if ((s = dalloc(c, &c->d_S32, nS32))) return s;
    // element slots (whole 32-element groups) plus one zero slot past the last element (the
    // missing neighbour of an SVK traction face)
    if ((s = dalloc(c, &c->d_slot32, (size_t)ngroups * c->m * 32 + c->Nf))) return s;
    CUDA_TRY(c, cudaMemsetAsync(c->d_slot32, 0, ((size_t)ngroups * c->m * 32 + c->Nf) * 4, c->stream));
    c->nfe4 = (int64_t)((nfe + 3) / 4) * 4;
    const size_t n32 = c->R > 1 ? nfe * R : (size_t)c->nfe4;
    for (float** p : {&c->d_dinv32, &c->d_r32, &c->d_z32, &c->d_p32, &c->d_q32, &c->d_x32, &c->d_b32}) {
      const size_t cnt = p == &c->d_dinv32 ? (size_t)c->nfe4 : n32;
      if ((s = dalloc(c, p, cnt))) return s;
      CUDA_TRY(c, cudaMemsetAsync(*p, 0, cnt * 4, c->stream));
    }
    if (c->R > 1 && (s = dalloc(c, &c->d_mslot32, (size_t)ne * c->m * R))) return s;
    if (c->R > 1 && (s = dalloc(c, &c->d_mShi, (size_t)ne * c->m * c->m))) return s;
    if (c->R > 1 && (s = dalloc(c, &c->d_mSlo, (size_t)ne * c->m * c->m))) return s;
    if ((s = dalloc(c, &c->d_pqpart, (size_t)(ngroups + 3) / 4))) return s;
    if ((s = dalloc(c, &c->d_pq, 1))) return s;
    if ((s = dalloc(c, &c->d_ticket, 1))) return s;
    CUDA_TRY(c, cudaMemsetAsync(c->d_ticket, 0, sizeof(unsigned), c->stream));
    if ((s = dalloc(c, &c->d_dtime, 2))) return s;
    if ((s = reset_dev_timing(c))) return s;
    if (c->R == 1 && c->phys == HDG_ACOUSTIC) {
      // whole 32-element groups, so the per-CTA staging copy never runs past the end
      const size_t nSdf = (size_t)ngroups * 32 * 2 * P4 * 4;
      if ((s = dalloc(c, &c->d_Sdf, nSdf))) return s;
      if (c->opt.prec == HDG_MIXED16) {
        const int P8 = (c->m * (c->m + 1) / 2 + 7) / 8;
        const size_t n16 = (size_t)ngroups * P8 * 256;
        if ((s = dalloc(c, &c->d_S16, n16))) return s;
        if ((s = dalloc(c, &c->d_sc16, (size_t)ngroups * 32))) return s;
        if ((s = dalloc(c, &c->d_gface16, (size_t)ngroups * 32 * c->nfc))) return s;
        CUDA_TRY(c, cudaMemsetAsync(c->d_sc16, 0, (size_t)ngroups * 32 * 4, c->stream));
      }
      CUDA_TRY(c, cudaMemsetAsync(c->d_Sdf, 0, nSdf * 4, c->stream));
    }
    if (c->phys == HDG_ACOUSTIC) {
      // double-float local solves: H^{-1} (filled at each condensation), geometry, tables
      if ((s = dalloc(c, &c->d_Hinvdf, (size_t)ne * c->nv * c->nv))) return s;
      if ((s = dalloc(c, &c->d_geodf, (size_t)ne * GEO_STRIDE))) return s;
      c->n_launch += 1;
      to_df_kernel<<<grid_for(c, ne * GEO_STRIDE), 256, 0, c->stream>>>(ne * GEO_STRIDE, c->d_geo, c->d_geodf);
      const int NP = c->nv, NF = c->Nf, D = c->dim, NFC = c->dim + 1;
      std::vector<df2> td((size_t)2 * D * NP * NP + 2 * NFC * NP * NF);
      auto split = [](double v) { const float h = (float)v; return df2{h, (float)(v - (double)h)}; };
      df2* DrT = td.data();
      df2* Drd = DrT + D * NP * NP;
      df2* FfT = Drd + D * NP * NP;
      df2* Ffd = FfT + NFC * NP * NF;
      for (int r = 0; r < D; ++r)
        for (int l = 0; l < NP; ++l)
          for (int i = 0; i < NP; ++i) {
            DrT[(r * NP + l) * NP + i] = split(c->T.Dr[(r * NP + i) * NP + l]);
            Drd[(r * NP + l) * NP + i] = split(c->T.Dr[(r * NP + l) * NP + i]);
          }
      for (int f = 0; f < NFC; ++f)
        for (int i = 0; i < NP; ++i)
          for (int mm = 0; mm < NF; ++mm) {
            FfT[(f * NF + mm) * NP + i] = split(c->T.Ff[(f * NP + i) * NF + mm]);
            Ffd[(f * NP + i) * NF + mm] = split(c->T.Ff[(f * NP + i) * NF + mm]);
          }
      if ((s = dalloc(c, &c->d_tabdf, td.size()))) return s;
      CUDA_TRY(c, cudaMemcpyAsync(c->d_tabdf, td.data(), td.size() * sizeof(df2), cudaMemcpyHostToDevice, c->stream));
      // the host copy is released below only after the stream has consumed it
      CUDA_TRY(c, cudaStreamSynchronize(c->stream));
      c->tabsdf = TabsDf{c->d_tabdf, c->d_tabdf + (Drd - DrT), c->d_tabdf + (FfT - DrT), c->d_tabdf + (Ffd - DrT)};
    }
    if ((s = dalloc(c, &c->d_res, nfe * R))) return s;
    if ((s = dalloc(c, &c->d_rs, 1))) return s;
    CUDA_TRY(c, cudaMallocHost((void**)&c->h_rs, sizeof(RefScal)));
  }
  std::vector<int32_t> fnode, node_ptr, node_inc;
  std::vector<double> vinv;
  if (c->tspace) {
    // continuous traces: free face nodes, their incidence lists (face entries in increasing
    // order, so node sums run in a fixed order) and the nodal-to-modal table
    int64_t nfree = 0;
    if (!build_trace_nodes(c->sk, k, c->tspace == HDG_TRACE_EDG, nfree, fnode, err)) return fail(c, HDG_EINVAL, err);
    try {
      vinv = face_nodal_to_modal(c->dim, k);
    } catch (const std::exception& ex) {
      return fail(c, HDG_EINVAL, ex.what());
    }
    node_ptr.assign((size_t)nfree + 1, 0);
    for (int32_t v : fnode)
      if (v >= 0) node_ptr[(size_t)v + 1] += 1;
    for (int64_t i = 0; i < nfree; ++i) node_ptr[i + 1] += node_ptr[i];
    node_inc.assign((size_t)node_ptr[nfree], 0);
    std::vector<int32_t> fill(node_ptr.begin(), node_ptr.end() - 1);
    for (size_t t = 0; t < fnode.size(); ++t)
      if (fnode[t] >= 0) node_inc[fill[fnode[t]]++] = (int32_t)t;
    c->n_mu = nfree;
    c->n_mu4 = (nfree + 3) / 4 * 4;
    if ((s = dalloc(c, &c->d_face_node, fnode.size()))) return s;
    if ((s = dalloc(c, &c->d_node_ptr, node_ptr.size()))) return s;
    if ((s = dalloc(c, &c->d_node_inc, node_inc.size()))) return s;
    if ((s = dalloc(c, &c->d_vinv, vinv.size()))) return s;
    if ((s = dalloc(c, &c->d_mu, (size_t)nfree))) return s;
    if ((s = dalloc(c, &c->d_bmu, (size_t)nfree))) return s;
    if ((s = dalloc(c, &c->d_ew64, nfe))) return s;
    if ((s = dalloc(c, &c->d_w64, nfe))) return s;
    CUDA_TRY(c, cudaMemcpyAsync(c->d_face_node, fnode.data(), fnode.size() * 4, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(c->d_node_ptr, node_ptr.data(), node_ptr.size() * 4, cudaMemcpyHostToDevice, c->stream));
    if (!node_inc.empty())
      CUDA_TRY(c, cudaMemcpyAsync(c->d_node_inc, node_inc.data(), node_inc.size() * 4, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(c->d_vinv, vinv.data(), vinv.size() * 8, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemsetAsync(c->d_mu, 0, (size_t)nfree * 8, c->stream));
    if (c->opt.prec != HDG_FP64) {
      if ((s = dalloc(c, &c->d_ew32, (size_t)c->nfe4))) return s;
      if ((s = dalloc(c, &c->d_w32, nfe))) return s;
      CUDA_TRY(c, cudaMemsetAsync(c->d_ew32, 0, (size_t)c->nfe4 * 4, c->stream));
    }
  }
  CUDA_TRY(c, cudaMemsetAsync(c->d_lam, 0, nfe * R * 8, c->stream));
  CUDA_TRY(c, cudaMemsetAsync(c->d_u, 0, (size_t)ne * c->n * R * 8, c->stream));
  CUDA_TRY(c, cudaMemsetAsync(c->d_uprev, 0, (size_t)ne * c->n * R * 8, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  {
    std::vector<uint8_t> mask((size_t)c->ntr);
    for (int64_t f = 0; f < nf; ++f)
      for (int mm = 0; mm < c->Nf; ++mm) mask[(size_t)f * c->Nf + mm] = c->sk.face_bnd[f] < 0 ? 1 : 0;
    if ((s = guess_setup(c, mask.data()))) return s;
  }
  if (svk && (s = svk_setup(c))) return s;
  if (c->opt.precond == HDG_PRECOND_BILU0 && (s = bilu_setup(c))) return s;
  c->have_state = true;
  return HDG_OK;
}

hdg_status hdg_get_sizes(const hdg_ctx* c, hdg_sizes* o) {
  if (!c || !o) return HDG_EINVAL;
  o->dim = c->dim; o->k = c->k; o->Np = c->Np; o->Nf = c->Nf; o->n_local = c->n; o->n_trace_local = c->m;
  o->n_elem = c->sk.ne; o->n_faces = c->sk.nf; o->n_bnd_faces = c->sk.nb;
  o->nq_vol = c->T.nqv; o->nq_face = c->T.nqf;
  o->device_bytes = c->bytes;
  o->field_entries = c->nfld;
  o->trace_entries = c->ntr;
  o->schur_entries = c->nschur;
  o->slot_entries = c->nslot;
  int64_t nint = 0;
  if (!c->vd)
    for (int64_t f = 0; f < c->sk.nf; ++f) nint += c->sk.face_bnd[f] < 0 ? c->Nf : 0;
  else
    nint = c->ntr;
  o->trace_unknowns = c->tspace ? c->n_mu : nint;
  return HDG_OK;
}

hdg_status hdg_condense(hdg_ctx* c, double alpha) {
  if (!c) return HDG_EINVAL;
  if (c->svk) return fail(c, HDG_EINVAL, "SVK: every Newton iteration of hdg_step condenses; no hdg_condense");
  return do_condense(c, alpha);
}

hdg_status hdg_get_schur(hdg_ctx* c, double* S_dev) {
  if (c && c->vd) return fail(c, HDG_EINVAL, "not available with per-element degrees");
  if (!c || !S_dev) return fail(c, HDG_EINVAL, "null argument");
  if (!c->condensed) return fail(c, HDG_ESTATE, "hdg_condense has not run");
  CUDA_TRY(c, cudaMemcpyAsync(S_dev, c->d_S, (size_t)c->sk.ne * c->m * c->m * 8, cudaMemcpyDeviceToDevice, c->stream));
  return HDG_OK;
}

hdg_status hdg_trace_apply(hdg_ctx* c, const double* x, double* y) {
  if (!c || !x || !y) return fail(c, HDG_EINVAL, "null argument");
  if (!c->condensed) return fail(c, HDG_ESTATE, "hdg_condense has not run");
  if (c->vd) return vd_trace_apply(c, x, y);
  if (c->R > 1) {
    HDG_DISPATCH(c, mlaunch_apply64, c, x, c->d_mslot, (const int*)nullptr, -1);
    HDG_DISPATCH(c, mlaunch_gather, c, (const double*)c->d_mslot, 1.0, y);
    return check_launch(c, "apply_multi");
  }
  HDG_DISPATCH(c, launch_apply, c, x, c->d_slot, (const int*)nullptr);
  hdg_status s = check_launch(c, "apply");
  if (s) return s;
  return faces_from_slots(c, 1.0, y);
}

hdg_status hdg_condensed_rhs(hdg_ctx* c, const double* F, const double* lamD, double* r) {
  if (!c || !F || !r) return fail(c, HDG_EINVAL, "null argument");
  if (c->svk) return fail(c, HDG_EINVAL, "SVK: the Newton stages of hdg_step condense and recover");
  if (!c->condensed) return fail(c, HDG_ESTATE, "hdg_condense has not run");
  if (c->vd) return vd_condensed_rhs(c, F, lamD, r);
  if (c->R > 1) {
    HDG_DISPATCH(c, mlaunch_local, c, 0, F, (const double*)nullptr, 0.0, lamD, c->d_mslot);
    HDG_DISPATCH(c, mlaunch_gather, c, (const double*)c->d_mslot, -1.0, r);
    return check_launch(c, "condensed_rhs_multi");
  }
  HDG_DISPATCH(c, launch_local, c, 0, F, (const double*)nullptr, 0.0, lamD, c->d_slot);
  hdg_status s = check_launch(c, "condensed_rhs");
  if (s) return s;
  return faces_from_slots(c, -1.0, r);
}

hdg_status hdg_trace_solve(hdg_ctx* c, const double* r, double* lam, hdg_solve_info* info) {
  if (!c || !r || !lam) return fail(c, HDG_EINVAL, "null argument");
  if (!c->condensed) return fail(c, HDG_ESTATE, "hdg_condense has not run");
  if (info) { info->iterations = 0; info->sweeps = 0; info->rel_residual = 0; }
  if (c->vd) return vd_trace_solve(c, r, lam, info);
  // K lam = r  <=>  (sgn K) lam = sgn r
  const int64_t nfe = c->sk.nf * c->Nf * (int64_t)c->R;
  combine_kernel<<<grid_for(c, nfe), 256, 0, c->stream>>>(nfe, c->sgn, r, 0, nullptr, 0, nullptr, 0, nullptr, c->d_b);
  hdg_status s = check_launch(c, "negate");
  if (s) return s;
  if (c->R > 1) {
    if ((s = msolve(c, c->d_b, lam, info))) return s;
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return HDG_OK;
  }
  if (c->tspace) {
    // continuous traces: R^T K R mu = R^T r from mu = 0, lam = R mu on interior faces
    if ((s = edg_restrict(c, c->d_b, c->d_bmu))) return s;
    CUDA_TRY(c, cudaMemsetAsync(c->d_mu, 0, (size_t)c->n_mu * 8, c->stream));
    if ((s = edg_solve(c, c->d_bmu, c->d_mu, info))) return s;
    HDG_DISPATCH(c, edg_expand64, c, c->d_mu, lam, 0);
    if ((s = check_launch(c, "edg_expand"))) return s;
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return HDG_OK;
  }
  return cg_solve(c, c->d_b, lam, info);
}

hdg_status hdg_recover(hdg_ctx* c, const double* F, const double* lam, double* u) {
  if (!c || !F || !lam || !u) return fail(c, HDG_EINVAL, "null argument");
  if (c->svk) return fail(c, HDG_EINVAL, "SVK: the Newton stages of hdg_step condense and recover");
  if (!c->condensed) return fail(c, HDG_ESTATE, "hdg_condense has not run");
  if (c->vd) return vd_recover(c, F, lam, u);
  if (c->R > 1) {
    HDG_DISPATCH(c, mlaunch_local, c, 1, F, (const double*)nullptr, 0.0, lam, u);
    return check_launch(c, "recover_multi");
  }
  HDG_DISPATCH(c, launch_local, c, 1, F, (const double*)nullptr, 0.0, lam, u);
  return check_launch(c, "recover");
}

hdg_status hdg_postprocess(hdg_ctx* c, const double* u, const double* lam, double* pstar) {
  if (!c || !u || !lam || !pstar) return fail(c, HDG_EINVAL, "null argument");
  if (c->phys != HDG_ACOUSTIC || c->vd || c->R != 1)
    return fail(c, HDG_EINVAL, "post-processing is defined for acoustic contexts with nrhs = 1");
  if (!c->d_post) {
    PostTables P;
    try {
      P = build_post_tables(c->dim, c->k);
    } catch (const std::exception& ex) {
      return fail(c, HDG_EINVAL, std::string("post-processing tables: ") + ex.what());
    }
    std::vector<double> tab(P.K1);
    tab.insert(tab.end(), P.E1.begin(), P.E1.end());
    hdg_status s;
    if ((s = dalloc(c, &c->d_post, tab.size()))) return s;
    c->post_k1 = (int64_t)P.K1.size();
    CUDA_TRY(c, cudaMemcpyAsync(c->d_post, tab.data(), tab.size() * 8, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));   // tab is released at return
  }
  HDG_DISPATCH(c, launch_post, c, u, lam, pstar);
  return check_launch(c, "postprocess");
}

hdg_status hdg_set_sources(hdg_ctx* c, int32_t nsrc, const double* pos, const double* amp, const int32_t* col,
                           const double* delay, double f0, double t0) {
  if (!c || nsrc < 0 || (nsrc > 0 && (!pos || !amp))) return fail(c, HDG_EINVAL, "bad source arguments");
  for (int s2 = 0; col && s2 < nsrc; ++s2)
    if (col[s2] < 0 || col[s2] >= c->R) return fail(c, HDG_EINVAL, "source column out of range");
  if (c->phys == HDG_ELASTIC && nsrc > 0) return fail(c, HDG_EINVAL, "point sources are acoustic only");
  // buffers only grow, so re-setting sources (e.g. a serving loop recycling slots) never
  // frees device memory (cudaFree would synchronise the whole device)
  c->nsrc = 0;
  if (nsrc == 0) return HDG_OK;
  const int d = c->dim, nc = c->nfc, Np = c->Np;
  const int64_t ne = c->sk.ne;
  std::vector<std::pair<int64_t, int>> owner;   // (element, source)
  std::vector<double> xi_all((size_t)nsrc * d);
  for (int s = 0; s < nsrc; ++s) {
    int64_t found = -1;
    for (int64_t e = 0; e < ne && found < 0; ++e) {
      const double* g = &c->sk.geo[e * GEO_STRIDE];
      const double* X0 = &c->h_vert_elem[(size_t)e * nc * d];
      double xi[3], sum = 0.0, mn = 1e300;
      for (int r = 0; r < d; ++r) {
        double v = 0.0;
        for (int j = 0; j < d; ++j) v += g[1 + r * d + j] * (pos[s * d + j] - X0[j]);
        xi[r] = v; sum += v; mn = std::min(mn, v);
      }
      if (mn >= -1e-12 && sum <= 1.0 + 1e-12) {
        found = e;
        for (int r = 0; r < d; ++r) xi_all[(size_t)s * d + r] = xi[r];
      }
    }
    if (found < 0) return fail(c, HDG_EINVAL, "source " + std::to_string(s) + " lies outside the mesh");
    owner.push_back({found, s});
  }
  std::stable_sort(owner.begin(), owner.end());
  std::vector<int32_t> ptr(ne + 1, 0);
  std::vector<double> phi((size_t)nsrc * Np);
  std::vector<int32_t> cols(nsrc, 0);
  std::vector<double> delays(nsrc, 0.0);
  for (size_t i = 0; i < owner.size(); ++i) {
    ptr[owner[i].first + 1]++;
    const int s = owner[i].second;
    cols[i] = col ? col[s] : 0;
    delays[i] = delay ? delay[s] : 0.0;
    dubiner(d, c->k, &xi_all[(size_t)s * d], 1, &phi[i * Np], nullptr);
    for (int q = 0; q < Np; ++q) phi[i * Np + q] *= amp[s];
  }
  for (int64_t e = 0; e < ne; ++e) ptr[e + 1] += ptr[e];
  hdg_status st;
  if (!c->d_src_ptr && (st = dalloc(c, &c->d_src_ptr, (size_t)ne + 1))) return st;
  if (nsrc > c->src_cap) {
    const int cap = std::max(nsrc, 2 * c->src_cap);
    dfree(c, c->d_src_phi); dfree(c, c->d_src_col); dfree(c, c->d_src_delay);
    c->d_src_phi = nullptr; c->d_src_col = nullptr; c->d_src_delay = nullptr; c->src_cap = 0;
    if ((st = dalloc(c, &c->d_src_phi, (size_t)cap * Np))) return st;
    if ((st = dalloc(c, &c->d_src_col, (size_t)cap))) return st;
    if ((st = dalloc(c, &c->d_src_delay, (size_t)cap))) return st;
    c->src_cap = cap;
  }
  CUDA_TRY(c, cudaMemcpyAsync(c->d_src_delay, delays.data(), delays.size() * 8, cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(c->d_src_col, cols.data(), cols.size() * 4, cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(c->d_src_ptr, ptr.data(), ptr.size() * 4, cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(c->d_src_phi, phi.data(), phi.size() * 8, cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  c->nsrc = nsrc; c->f0 = f0; c->t0 = t0;
  return HDG_OK;
}

hdg_status hdg_quadrature_points(hdg_ctx* c, int32_t which, double* xyz) {
  if (!c || !xyz || (which != 0 && which != 1)) return fail(c, HDG_EINVAL, "bad arguments");
  if (c->vd) return vd_quadrature_points(c, which, xyz);
  const int d = c->dim, nc = c->nfc;
  if (which == 0) {
    const int nq = c->T.nqv;
    for (int64_t e = 0; e < c->sk.ne; ++e) {
      const double* X = &c->h_vert_elem[(size_t)e * nc * d];
      for (int q = 0; q < nq; ++q)
        for (int j = 0; j < d; ++j) {
          double v = X[j];
          for (int r = 0; r < d; ++r) v += c->T.qv_pts[(size_t)q * d + r] * (X[(r + 1) * d + j] - X[j]);
          xyz[((size_t)e * nq + q) * d + j] = v;
        }
    }
  } else {
    const int nq = c->T.nqf;
    for (int64_t b = 0; b < c->sk.nb; ++b) {
      const int64_t f = c->sk.bnd_faces[b];
      const int64_t slot = c->sk.face_slot[2 * f];
      const int64_t e = slot / nc;
      const int j = (int)(slot % nc);
      const double* X = &c->h_vert_elem[(size_t)e * nc * d];
      int fv[3], cnt = 0;
      for (int a = 0; a < nc; ++a) if (a != j) fv[cnt++] = a;
      for (int q = 0; q < nq; ++q)
        for (int jj = 0; jj < d; ++jj) {
          double v = X[fv[0] * d + jj];
          for (int r = 1; r < d; ++r) v += c->T.qf_pts[(size_t)q * (d - 1) + r - 1] * (X[fv[r] * d + jj] - X[fv[0] * d + jj]);
          xyz[((size_t)b * nq + q) * d + jj] = v;
        }
    }
  }
  return HDG_OK;
}

hdg_status hdg_project_volume(hdg_ctx* c, const double* vals, double* u) {
  if (!c || !vals || !u) return fail(c, HDG_EINVAL, "null argument");
  if (c->vd) return vd_project_volume(c, vals, u);
  const size_t cnt = (size_t)c->sk.ne * c->T.nqv * c->ncomp;
  double* dv = nullptr;
  hdg_status s;
  if ((s = dalloc(c, &dv, cnt))) return s;
  cudaError_t e1 = cudaMemcpyAsync(dv, vals, cnt * 8, cudaMemcpyHostToDevice, c->stream);
  if (e1 == cudaSuccess) {
    const int64_t n = c->nfld * (int64_t)c->R;
    if (c->R > 1)
      mproject_volume_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(c->sk.ne, c->Np, c->T.nqv, c->ncomp, c->R, c->d_qv_w,
                                                                   c->d_qv_phi, dv, u);
    else
      project_volume_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(c->sk.ne, c->Np, c->T.nqv, c->ncomp, c->d_qv_w, c->d_qv_phi,
                                                                  dv, u);
    e1 = cudaGetLastError();
  }
  if (e1 == cudaSuccess) e1 = cudaStreamSynchronize(c->stream);
  dfree(c, dv);
  c->bytes -= (int64_t)(cnt * 8);
  if (e1 != cudaSuccess) return fail(c, HDG_ECUDA, std::string("project_volume: ") + cudaGetErrorString(e1));
  return HDG_OK;
}

hdg_status hdg_set_dirichlet(hdg_ctx* c, const double* vals, double omega, double phase) {
  if (c && c->vd && vals) return fail(c, HDG_EINVAL, "per-element degrees: homogeneous (clamped) boundary only");
  if (!c) return HDG_EINVAL;
  dfree(c, c->d_bnd_coef);
  c->d_bnd_coef = nullptr;
  c->omega = omega; c->phase = phase;
  if (!vals || c->sk.nb == 0) return HDG_OK;
  if (c->phys == HDG_ELASTIC) return fail(c, HDG_EINVAL, "elastic path supports clamped boundaries (NULL data) only");
  if (c->tspace == HDG_TRACE_EDG) return fail(c, HDG_EINVAL, "EDG traces: homogeneous Dirichlet data (NULL) only");
  // lam_f[m] = sum_q w_q g(x_q) mu_m(eta_q)   (face mass J_F I cancels J_F)
  const int nq = c->T.nqf, Nf = c->Nf;
  std::vector<double> coef((size_t)c->sk.nb * Nf, 0.0);
  for (int64_t b = 0; b < c->sk.nb; ++b)
    for (int mm = 0; mm < Nf; ++mm) {
      double s = 0.0;
      for (int q = 0; q < nq; ++q) s += c->T.qf_w[q] * vals[(size_t)b * nq + q] * c->T.qf_mu[(size_t)q * Nf + mm];
      coef[(size_t)b * Nf + mm] = s;
    }
  hdg_status s;
  if ((s = dalloc(c, &c->d_bnd_coef, coef.size()))) return s;
  CUDA_TRY(c, cudaMemcpyAsync(c->d_bnd_coef, coef.data(), coef.size() * 8, cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return HDG_OK;
}

hdg_status hdg_set_state(hdg_ctx* c, const double* u, const double* uprev, const double* lam, double t) {
  if (!c || !u) return fail(c, HDG_EINVAL, "null argument");
  const size_t bytes = (size_t)c->nfld * c->R * 8;
  const size_t tbytes = (size_t)c->ntr * c->R * 8;
  // device or page-locked host buffers (unified addressing decides the direction)
  CUDA_TRY(c, cudaMemcpyAsync(c->d_u, u, bytes, cudaMemcpyDefault, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(c->d_uprev, uprev ? uprev : c->d_u, bytes, cudaMemcpyDefault, c->stream));
  if (lam)
    CUDA_TRY(c, cudaMemcpyAsync(c->d_lam, lam, tbytes, cudaMemcpyDefault, c->stream));
  else
    CUDA_TRY(c, cudaMemsetAsync(c->d_lam, 0, tbytes, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  c->t = t;
  c->have_state = true;
  c->n_lam_hist = 0;
  if (c->d_mu) CUDA_TRY(c, cudaMemsetAsync(c->d_mu, 0, (size_t)c->n_mu * 8, c->stream));
  // the least-squares guess keeps its pairs: K lam_i = b_i holds for any state
  return check_launch(c, "set_state");
}

hdg_status hdg_get_state(hdg_ctx* c, double* u, double* uprev, double* lam, double* t) {
  if (!c) return HDG_EINVAL;
  const size_t bytes = (size_t)c->nfld * c->R * 8;
  if (u) CUDA_TRY(c, cudaMemcpyAsync(u, c->d_u, bytes, cudaMemcpyDefault, c->stream));
  if (uprev) CUDA_TRY(c, cudaMemcpyAsync(uprev, c->d_uprev, bytes, cudaMemcpyDefault, c->stream));
  if (lam) CUDA_TRY(c, cudaMemcpyAsync(lam, c->d_lam, (size_t)c->ntr * c->R * 8, cudaMemcpyDefault, c->stream));
  if (t) *t = c->t;
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return HDG_OK;
}

// ---- checkpoint: a header, then the device arrays in a fixed order
namespace {
struct CkptHeader {
  char magic[8];
  int32_t version, dim, k, R, phys, prec, tspace, n_lam_hist, g_q, g_n, g_next, condensed;
  int64_t nfld, ntr, n_mu;
  double t, alpha;
};

// (device pointer, bytes) of every array the checkpoint holds, in order
std::vector<std::pair<void*, size_t>> ckpt_arrays(hdg_ctx* c) {
  std::vector<std::pair<void*, size_t>> a;
  const size_t fb = (size_t)c->nfld * c->R * 8, tb = (size_t)c->ntr * c->R * 8;
  a.push_back({c->d_u, fb});
  a.push_back({c->d_uprev, fb});
  for (double* p : {c->d_lam, c->d_lam_prev, c->d_lam_prev2})
    if (p) a.push_back({p, tb});
  if (c->g_q) {
    a.push_back({c->d_gb, (size_t)c->g_q * tb});
    a.push_back({c->d_gl, (size_t)c->g_q * tb});
  }
  if (c->d_gd) a.push_back({c->d_gd, sizeof(GuessDev)});
  if (c->d_mu) a.push_back({c->d_mu, (size_t)c->n_mu * 8});
  return a;
}

size_t ckpt_bytes(hdg_ctx* c) {
  size_t n = sizeof(CkptHeader) + c->gm_gram.size() * 8;
  for (auto& p : ckpt_arrays(c)) n += p.second;
  return n;
}
}  // namespace

hdg_status hdg_checkpoint_size(const hdg_ctx* c, int64_t* bytes) {
  if (!c || !bytes) return HDG_EINVAL;
  *bytes = (int64_t)ckpt_bytes(const_cast<hdg_ctx*>(c));
  return HDG_OK;
}

hdg_status hdg_save_checkpoint(hdg_ctx* c, void* buf) {
  if (!c || !buf) return fail(c, HDG_EINVAL, "null argument");
  CkptHeader h{};
  std::memcpy(h.magic, "HDGCKPT", 8);
  h.version = 1; h.dim = c->dim; h.k = c->k; h.R = c->R; h.phys = c->phys; h.prec = c->opt.prec; h.tspace = c->tspace;
  h.n_lam_hist = c->n_lam_hist; h.g_q = c->g_q; h.g_n = c->g_n; h.g_next = c->g_next; h.condensed = c->condensed ? 1 : 0;
  h.nfld = c->nfld; h.ntr = c->ntr; h.n_mu = c->n_mu; h.t = c->t; h.alpha = c->alpha;
  char* out = static_cast<char*>(buf);
  std::memcpy(out, &h, sizeof h);
  size_t off = sizeof h;
  if (!c->gm_gram.empty()) {
    std::memcpy(out + off, c->gm_gram.data(), c->gm_gram.size() * 8);
    off += c->gm_gram.size() * 8;
  }
  for (auto& p : ckpt_arrays(c)) {
    CUDA_TRY(c, cudaMemcpyAsync(out + off, p.first, p.second, cudaMemcpyDeviceToHost, c->stream));
    off += p.second;
  }
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return HDG_OK;
}

hdg_status hdg_load_checkpoint(hdg_ctx* c, const void* buf) {
  if (!c || !buf) return fail(c, HDG_EINVAL, "null argument");
  CkptHeader h;
  const char* in = static_cast<const char*>(buf);
  std::memcpy(&h, in, sizeof h);
  if (std::memcmp(h.magic, "HDGCKPT", 8) != 0 || h.version != 1)
    return fail(c, HDG_EINVAL, "not a checkpoint of this library version");
  if (h.dim != c->dim || h.k != c->k || h.R != c->R || h.phys != c->phys || h.prec != c->opt.prec ||
      h.tspace != c->tspace || h.g_q != c->g_q || h.nfld != c->nfld || h.ntr != c->ntr || h.n_mu != c->n_mu)
    return fail(c, HDG_EINVAL, "checkpoint of a context with other sizes or options");
  hdg_status s;
  // operators for the saved alpha first: a condensation clears the stored stage solutions
  if (h.condensed && !c->svk && (s = ensure_alpha(c, h.alpha))) return s;
  size_t off = sizeof h;
  if (!c->gm_gram.empty()) {
    std::memcpy(c->gm_gram.data(), in + off, c->gm_gram.size() * 8);
    off += c->gm_gram.size() * 8;
  }
  for (auto& p : ckpt_arrays(c)) {
    CUDA_TRY(c, cudaMemcpyAsync(p.first, in + off, p.second, cudaMemcpyHostToDevice, c->stream));
    off += p.second;
  }
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  c->t = h.t;
  c->n_lam_hist = h.n_lam_hist;
  c->g_n = h.g_n;
  c->g_next = h.g_next;
  c->have_state = true;
  return HDG_OK;
}

hdg_status hdg_step(hdg_ctx* c, double dt, hdg_scheme scheme, int32_t nsteps, hdg_solve_info* info) {
  if (!c) return HDG_EINVAL;
  if (!(dt > 0.0) || nsteps < 0) return fail(c, HDG_EINVAL, "dt must be positive and nsteps >= 0");
  if (scheme != HDG_BE && scheme != HDG_BDF2 && scheme != HDG_DIRK3) return fail(c, HDG_EINVAL, "unknown scheme");
  if (c->svk) return svk_step(c, dt, scheme, nsteps, info);
  if (info) { info->iterations = 0; info->sweeps = 0; info->rel_residual = 0; }
  hdg_solve_info si{};
  hdg_status s;
  for (int32_t step = 0; step < nsteps; ++step) {
    const double tn = c->t;
    if (scheme == HDG_BE || scheme == HDG_BDF2) {
      // Eq. ch5appendx1:eq9b with b_s = 1: alpha = a_s/dt, hist = -(sum_{i<s} a_i u^{n+i}) / a_s
      double alpha;
      if (scheme == HDG_BE) {
        alpha = 1.0 / dt;
        combine(c, c->d_h, 1.0, c->d_u);
      } else {
        alpha = 1.5 / dt;
        combine(c, c->d_h, 4.0 / 3.0, c->d_u, -1.0 / 3.0, c->d_uprev);
      }
      if ((s = ensure_alpha(c, alpha))) return s;
      // initial guess of the trace solve: polynomial extrapolation of the last traces,
      // 3 lam^n - 3 lam^{n-1} + lam^{n-2} (quadratic; linear / constant while the history fills)
      const int64_t nfe = c->ntr * (int64_t)c->R;
      if (c->n_lam_hist >= 1) {
        c->n_launch += 1;
        if (c->n_lam_hist >= 2)
          combine_kernel<<<grid_for(c, nfe), 256, 0, c->stream>>>(nfe, 3.0, c->d_lam, -3.0, c->d_lam_prev, 1.0,
                                                                  c->d_lam_prev2, 0, nullptr, c->d_lam_x);
        else
          combine_kernel<<<grid_for(c, nfe), 256, 0, c->stream>>>(nfe, 2.0, c->d_lam, -1.0, c->d_lam_prev, 0, nullptr, 0,
                                                                  nullptr, c->d_lam_x);
        // rotate: lam^{n-2} <- lam^{n-1} <- lam^n, lam <- guess
        double* t = c->d_lam_prev2;
        c->d_lam_prev2 = c->d_lam_prev;
        c->d_lam_prev = c->d_lam;
        c->d_lam = c->d_lam_x;
        c->d_lam_x = t;
        c->n_lam_hist = 2;
      } else {
        CUDA_TRY(c, cudaMemcpyAsync(c->d_lam_prev, c->d_lam, nfe * 8, cudaMemcpyDeviceToDevice, c->stream));
        c->n_lam_hist = 1;
      }
      if ((s = stage_solve(c, c->d_h, tn + dt, c->d_unew, &si))) return s;
      std::swap(c->d_uprev, c->d_u);   // u^{n-1} <- u^n
      std::swap(c->d_u, c->d_unew);    // u^n <- u^{n+1}
    } else {
      c->n_lam_hist = 0;
      double a[3][3], b[3], cc[3];
      dirk3(a, b, cc);
      // d = a^{-1} (lower triangular)
      double d[3][3] = {};
      for (int i = 0; i < 3; ++i) {
        d[i][i] = 1.0 / a[i][i];
        for (int j = 0; j < i; ++j) {
          double sum = 0.0;
          for (int q = j; q < i; ++q) sum += a[i][q] * d[q][j];
          d[i][j] = -sum / a[i][i];
        }
      }
      const double alpha = d[0][0] / dt;
      if ((s = ensure_alpha(c, alpha))) return s;
      // Eq. 10_2 weights: u^{n+1} = (1 - sum_i b_i sum_j d_ij) u^n + sum_j e_j U_j, e_j = sum_i b_i d_ij
      double e[3] = {0, 0, 0}, w0 = 1.0;
      for (int j = 0; j < 3; ++j)
        for (int i = 0; i < 3; ++i) e[j] += b[i] * d[i][j];
      for (int j = 0; j < 3; ++j) w0 -= e[j];
      if (c->vd) {
        // the whole step as one graph launch once the per-element-degree path is tuned
        double hc[3][3] = {}, uc[4] = {w0, e[0], e[1], e[2]};
        for (int i = 0; i < 3; ++i) {
          double cu = 0.0;
          for (int j = 0; j <= i; ++j) cu += d[i][j];
          hc[i][0] = cu / d[i][i];
          for (int j = 0; j < i; ++j) hc[i][1 + j] = -d[i][j] / d[i][i];
        }
        bool done = false;
        if ((s = vd_dirk3_step_graph(c, hc, uc, &si, &done))) return s;
        if (done) {
          std::swap(c->d_uprev, c->d_u);
          std::swap(c->d_u, c->d_unew);
          c->t = tn + dt;
          continue;
        }
      }
      for (int i = 0; i < 3; ++i) {
        // Eq. 10_1, stage i: d_ii Mw U_i + dt f(U_i) = Mw [ (sum_{j<=i} d_ij) u^n - sum_{j<i} d_ij U_j ]
        double cu = 0.0;
        for (int j = 0; j <= i; ++j) cu += d[i][j];
        const double* in[3] = {nullptr, nullptr, nullptr};
        double co[3] = {0, 0, 0};
        for (int j = 0; j < i; ++j) { in[j] = c->d_stage[j]; co[j] = -d[i][j] / d[i][i]; }
        combine(c, c->d_h, cu / d[i][i], c->d_u, co[0], in[0], co[1], in[1], co[2], in[2]);
        if ((s = stage_solve(c, c->d_h, tn + cc[i] * dt, c->d_stage[i], &si))) return s;
      }
      // Eq. 10_2 update
      combine(c, c->d_unew, w0, c->d_u, e[0], c->d_stage[0], e[1], c->d_stage[1], e[2], c->d_stage[2]);
      std::swap(c->d_uprev, c->d_u);
      std::swap(c->d_u, c->d_unew);
    }
    c->t = tn + dt;
  }
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (info) { info->iterations = si.iterations; info->sweeps = si.sweeps; info->rel_residual = si.rel_residual; }
  return HDG_OK;
}

hdg_status hdg_stream_create(void** out) {
  if (!out) return HDG_EINVAL;
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return HDG_ECUDA;
  *out = (void*)st;
  return HDG_OK;
}

hdg_status hdg_precond_apply(hdg_ctx* c, const double* r, double* z) {
  if (!c || !r || !z) return fail(c, HDG_EINVAL, "null argument");
  if (c->opt.solver != HDG_SOLVER_GMRES) return fail(c, HDG_EINVAL, "the preconditioner of the GMRES solver only");
  if (!c->condensed) return fail(c, HDG_ESTATE, "hdg_condense has not run");
  const int64_t n = c->sk.nf * c->Nf;
  hdg_status s;
  if (c->bilu) {
    if ((s = bilu_apply(c, r, z))) return s;
  } else {
    c->n_launch += 1;
    vmul_kernel<<<grid_for(c, n), 256, 0, c->stream>>>(n, c->d_dinv, r, z);
  }
  if ((s = check_launch(c, "precond_apply"))) return s;
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return HDG_OK;
}

hdg_status hdg_set_stream(hdg_ctx* c, void* cuda_stream) {
  if (!c) return HDG_EINVAL;
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  c->stream = (cudaStream_t)cuda_stream;
  return HDG_OK;
}

hdg_status hdg_stream_destroy(void* stream) {
  if (!stream) return HDG_EINVAL;
  return cudaStreamDestroy((cudaStream_t)stream) == cudaSuccess ? HDG_OK : HDG_ECUDA;
}

hdg_status hdg_reset_column(hdg_ctx* c, int32_t j) {
  if (!c) return HDG_EINVAL;
  if (j < 0 || j >= c->R) return fail(c, HDG_EINVAL, "column out of range");
  const int64_t nf = c->nfld, nt = c->ntr;
  for (double* a : {c->d_u, c->d_uprev}) {
    c->n_launch += 1;
    zero_column_kernel<<<grid_for(c, nf), 256, 0, c->stream>>>(nf, c->R, j, a);
  }
  for (double* a : {c->d_lam, c->d_lam_prev, c->d_lam_prev2}) {
    c->n_launch += 1;
    zero_column_kernel<<<grid_for(c, nt), 256, 0, c->stream>>>(nt, c->R, j, a);
  }
  guess_reset_column(c, j);
  return check_launch(c, "reset_column");
}

hdg_status hdg_get_tuning(const hdg_ctx* c, hdg_tuning* out) {
  if (!c || !out) return HDG_EINVAL;
  if (!c->vd) return HDG_EINVAL;
  return vd_get_tuning(c, out);
}

hdg_status hdg_enable_stats(hdg_ctx* c, int32_t enable) {
  if (!c) return HDG_EINVAL;
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  harvest(c);
  c->stats_on = enable != 0;
  return HDG_OK;
}

hdg_status hdg_get_stats(hdg_ctx* c, hdg_stats* o, int32_t reset) {
  if (!c || !o) return HDG_EINVAL;
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  harvest(c);
  DevTiming dt[2] = {{~0ull, 0, 0.0}, {~0ull, 0, 0.0}};
  if (c->d_dtime) {
    CUDA_TRY(c, cudaMemcpy(dt, c->d_dtime, sizeof(dt), cudaMemcpyDeviceToHost));
    if (reset) {
      hdg_status s = reset_dev_timing(c);
      if (s) return s;
      CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    }
  }
  o->dev_apply32_launches = (int64_t)dt[0].count;
  o->dev_apply32_ms = dt[0].ms;
  o->dev_apply16_launches = (int64_t)dt[1].count;
  o->dev_apply16_ms = dt[1].ms;
  o->kernel_launches = c->n_launch;
  o->apply_launches = c->n_apply;
  o->apply_ms = c->apply_ms;
  o->apply32_launches = c->n_apply32;
  o->apply32_ms = c->apply32_ms;
  o->applydf_launches = c->n_applydf;
  o->applydf_ms = c->applydf_ms;
  o->apply16_launches = c->n_apply16;
  o->apply16_ms = c->apply16_ms;
  o->svk_condense_launches = c->n_svkc;
  o->svk_condense_ms = c->svkc_ms;
  o->svk_recover_launches = c->n_svkr;
  o->svk_recover_ms = c->svkr_ms;
  if (reset) {
    c->n_launch = 0; c->n_apply = 0; c->apply_ms = 0.0; c->n_apply32 = 0; c->apply32_ms = 0.0;
    c->n_applydf = 0; c->applydf_ms = 0.0; c->n_apply16 = 0; c->apply16_ms = 0.0;
    c->n_svkc = 0; c->svkc_ms = 0.0; c->n_svkr = 0; c->svkr_ms = 0.0;
  }
  return HDG_OK;
}

}  // extern "C"
