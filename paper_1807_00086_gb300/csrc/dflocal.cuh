// Element-local solves of the acoustic scheme in double-float arithmetic on the FP32 pipe.
//
// The same two maps as local_kernel (Sec. 2.4, Eq. LS, the element blocks of the condensed
// system): MODE 0 forms gslot = C_K A_K^{-1} (F_K - B_K lamD_K), MODE 1 recovers
// u_K = A_K^{-1} (F_K - B_K lam_K). Every product and sum is carried as an unevaluated pair
// hi + lo of floats (about 48 significant bits): products by fmaf-based exact splitting
// (Dekker's two-product), sums by Knuth's two-sum, so the results agree with the FP64 kernel
// to a few units of 1e-14 relative while the work runs on the FP32 units (FP64 issues at a
// small fraction of the FP32 rate on this GPU). Only the conversions from and to FP64 and
// the per-element coefficients use FP64 instructions.
#pragma once

#include "kernels.cuh"
#include "multi.cuh"

namespace hdg {

__device__ __forceinline__ df2 df_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ df2 df_mul(df2 a, df2 b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, fmaf(a.l, b.h, e));
  const float s = p + e;
  return {s, e - (s - p)};
}
__device__ __forceinline__ df2 df_add(df2 a, df2 b) {
  df2 s = df_two_sum(a.h, b.h);
  const float err = s.l + (a.l + b.l);
  const float h = s.h + err;
  return {h, err - (h - s.h)};
}
__device__ __forceinline__ df2 df_neg(df2 a) { return {-a.h, -a.l}; }
// normalised value of a compensated accumulator
__device__ __forceinline__ df2 df_of(const DfAcc& a) { return df_two_sum(a.s, a.c); }

// Reference tables as double-floats, each laid out so that the NP rows of an element
// (consecutive threads) read consecutive entries:
//   DrT[r][l][i] = Dr[r][i][l]   (derivative matrices, row-wise sums)
//   Dr [r][l][i] = Dr[r][l][i]   (transposed products)
//   FfT[f][m][i] = Ff[f][i][m]   (face mass, volume-row sums)
//   Ff [f][q][m] = Ff[f][q][m]   (face mass, face-row sums)
struct TabsDf {
  const df2 *DrT, *Dr, *FfT, *Ff;
};

template <int DIM, int K>
struct LocalDfCfg {
  static constexpr int NP = Dims<DIM, K>::NP;
  static constexpr int EPB = NP <= 10 ? 16 : (NP <= 20 ? 8 : 4);
  static constexpr int NT = EPB * NP;
};

// Double-float copy of an FP64 array (H^{-1} after each condensation, the element geometry).
static __global__ void to_df_kernel(int64_t n, const double* __restrict__ a, df2* __restrict__ out) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    out[t] = df_from(a[t]);
}

// EPB elements per CTA, one thread per (element, row i < NP). geo: double-float copy of the
// element geometry; Hinv: double-float H^{-1} [ne][NP][NP] (symmetric, read as columns).
template <int DIM, int K, int MODE>
__global__ void __launch_bounds__(LocalDfCfg<DIM, K>::NT)
    local_df_kernel(DevMesh mesh, TabsDf T, const df2* __restrict__ geo, const df2* __restrict__ Hinv, double alpha,
                    df2 tau, const double* __restrict__ F, const double* __restrict__ hist, SrcArgs src,
                    const double* __restrict__ lam, double* __restrict__ out) {
  using D = Dims<DIM, K>;
  using L = LocalDfCfg<DIM, K>;
  constexpr int NP = D::NP, NF = D::NF, M = D::M, NFC = D::NFC, N = D::N, EPB = L::EPB, NT = L::NT;
  __shared__ df2 g[EPB][GEO_STRIDE];
  __shared__ df2 ll[EPB][M];
  __shared__ df2 Tr[EPB][DIM * NP];   // the face weights w_f (f < DIM) in MODE 0
  __shared__ df2 rp[EPB][NP];         // the last face's weights in MODE 0
  __shared__ df2 pp[EPB][NP];
  __shared__ df2 co[EPB][4];          // 1/b, a' dJ, b dJ, 1/(b dJ) with b = alpha rho, a' = alpha/(rho c^2)
  __shared__ int fuse[EPB][NFC];      // face contributes a trace (nonzero lam) to this element
  __shared__ int anyf[EPB];
  const int tid = threadIdx.x;
  const int64_t e0 = (int64_t)blockIdx.x * EPB;
  for (int t = tid; t < EPB * GEO_STRIDE; t += NT) {
    const int64_t e = e0 + t / GEO_STRIDE;
    g[t / GEO_STRIDE][t % GEO_STRIDE] =
        e < mesh.ne ? geo[e * GEO_STRIDE + t % GEO_STRIDE] : df2{t % GEO_STRIDE == 0 ? 1.f : 0.f, 0.f};
  }
  for (int t = tid; t < EPB * NFC; t += NT) {
    const int64_t e = e0 + t / NFC;
    int use = 0;
    if (e < mesh.ne && lam) {
      const int f = mesh.elem_face[e * NFC + t % NFC];
      use = (MODE == 1) || (mesh.face_bnd[f] >= 0);
    }
    fuse[t / NFC][t % NFC] = use;
  }
  for (int t = tid; t < EPB * M; t += NT) {
    const int64_t e = e0 + t / M;
    const int r = t % M;
    double v = 0.0;
    if (e < mesh.ne && lam) {
      const int f = mesh.elem_face[e * NFC + r / NF];
      if ((MODE == 1) || (mesh.face_bnd[f] >= 0)) v = lam[(int64_t)f * NF + r % NF];
    }
    ll[t / M][r] = df_from(v);
  }
  if (tid < EPB) {
    const int64_t e = e0 + tid;
    const bool ok = e < mesh.ne;
    const double rho = ok ? mesh.rho[e] : 1.0, cc = ok ? mesh.c[e] : 1.0;
    const double dJ = ok ? mesh.geo[e * GEO_STRIDE] : 1.0;
    const double b = alpha * rho, ap = alpha / (rho * cc * cc);
    co[tid][0] = df_from(1.0 / b);
    co[tid][1] = df_from(ap * dJ);
    co[tid][2] = df_from(b * dJ);
    co[tid][3] = df_from(1.0 / (b * dJ));
  }
  __syncthreads();
  if (tid < EPB) {
    int a = 0;
    for (int f = 0; f < NFC; ++f) a |= fuse[tid][f];
    anyf[tid] = a;
  }
  const int el = tid / NP, i = tid % NP;
  const int64_t e = e0 + el;
  const bool live = e < mesh.ne;
  const df2* ge = g[el];
  const df2 ib = co[el][0];
  __syncthreads();
  // row i of F~ for all components (+ the F^ lam face products it needs)
  df2 Fu[DIM + 1];
  {
    df2 Fl[NFC];
    const bool any = anyf[el] != 0;
#pragma unroll
    for (int f = 0; f < NFC; ++f) {
      DfAcc s;
      if (fuse[el][f])
        for (int mm = 0; mm < NF; ++mm) s.fma(T.FfT[(f * NF + mm) * NP + i], ll[el][f * NF + mm]);
      Fl[f] = df_of(s);
    }
#pragma unroll
    for (int comp = 0; comp <= DIM; ++comp) {
      df2 v{0.f, 0.f};
      if (live) {
        if (hist) {
          v = df_mul(co[el][comp == 0 ? 1 : 2], df_from(hist[e * N + comp * NP + i]));
          if (comp == 0 && src.ptr && src.ptr[e] < src.ptr[e + 1]) {
            double sv = 0.0;
            for (int q = src.ptr[e]; q < src.ptr[e + 1]; ++q) sv += ricker_at(src, q) * src.phi[(int64_t)q * NP + i];
            v = df_add(v, df_from(sv));
          }
        } else {
          v = df_from(F[e * N + comp * NP + i]);
        }
      }
      if (any) {
        DfAcc bl;
        if (comp == 0) {
#pragma unroll
          for (int f = 0; f < NFC; ++f) bl.fma(ge[D::OJF + f], Fl[f]);
          v = df_add(v, df_mul(tau, df_of(bl)));
        } else {
#pragma unroll
          for (int f = 0; f < NFC; ++f) bl.fma(df_mul(ge[D::ON + f * DIM + comp - 1], ge[D::OJF + f]), Fl[f]);
          v = df_add(v, df_neg(df_of(bl)));
        }
      }
      Fu[comp] = v;
    }
  }
  // Tr[r][i] = sum_j Jinv[r][j] F~v_j[i]
#pragma unroll
  for (int r = 0; r < DIM; ++r) {
    DfAcc s;
#pragma unroll
    for (int j = 0; j < DIM; ++j) s.fma(ge[1 + r * DIM + j], Fu[j + 1]);
    Tr[el][r * NP + i] = df_of(s);
  }
  __syncthreads();
  {
    DfAcc s;
#pragma unroll
    for (int r = 0; r < DIM; ++r)
#pragma unroll 4
      for (int l = 0; l < NP; ++l) s.fma(T.DrT[(r * NP + l) * NP + i], Tr[el][r * NP + l]);
    rp[el][i] = df_add(Fu[0], df_neg(df_mul(df_of(s), ib)));
  }
  __syncthreads();
  {
    // p = H^{-1} rp; H^{-1} is symmetric, so row i is read as column i (coalesced)
    const df2* He = Hinv + (live ? e : 0) * (int64_t)(NP * NP);
    DfAcc s;
#pragma unroll 4
    for (int l = 0; l < NP; ++l) s.fma(He[l * NP + i], rp[el][l]);
    pp[el][i] = df_of(s);
  }
  __syncthreads();
  df2 vv[DIM];
  {
    df2 qd[DIM];
#pragma unroll
    for (int r = 0; r < DIM; ++r) {
      DfAcc s;
#pragma unroll 4
      for (int l = 0; l < NP; ++l) s.fma(T.Dr[(r * NP + l) * NP + i], pp[el][l]);
      qd[r] = df_of(s);
    }
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      DfAcc s;
#pragma unroll
      for (int r = 0; r < DIM; ++r) s.fma(ge[1 + r * DIM + j], qd[r]);
      vv[j] = df_add(df_mul(Fu[j + 1], co[el][3]), df_mul(df_of(s), ib));
    }
  }
  if (MODE == 1) {
    if (live) {
      out[e * N + i] = df_to(pp[el][i]);
#pragma unroll
      for (int j = 0; j < DIM; ++j) out[e * N + (j + 1) * NP + i] = df_to(vv[j]);
    }
    return;
  }
  // MODE 0: w_f[i] = tau p[i] + sum_j n_fj v_j[i]
  df2* w = &Tr[el][0];
  __syncthreads();   // every thread is done reading Tr
  {
    const df2 tp = df_mul(tau, pp[el][i]);
#pragma unroll
    for (int f = 0; f < NFC; ++f) {
      DfAcc s;
#pragma unroll
      for (int j = 0; j < DIM; ++j) s.fma(ge[D::ON + f * DIM + j], vv[j]);
      const df2 wv = df_add(tp, df_of(s));
      if (f < DIM) w[f * NP + i] = wv;
      else rp[el][i] = wv;
    }
  }
  __syncthreads();
  for (int t = tid; t < EPB * M; t += NT) {
    const int el2 = t / M, r = t % M, f = r / NF, mm = r % NF;
    const int64_t e2 = e0 + el2;
    if (e2 >= mesh.ne) continue;
    const df2* wf = f < DIM ? &Tr[el2][f * NP] : &rp[el2][0];
    DfAcc s;
#pragma unroll 4
    for (int q = 0; q < NP; ++q) s.fma(T.Ff[(f * NP + q) * NF + mm], wf[q]);
    out[e2 * M + r] = df_to(df_mul(g[el2][D::OJF + f], df_of(s)));
  }
}


// R-column version (the multi-source and serving batches): CTA = one element x CW columns x
// NP rows, the layouts and work split of local_multi_kernel, every operation as in
// local_df_kernel (double-float products and sums on the FP32 pipe).
// Up to 320 threads per CTA the kernel is bounded to three resident CTAs per SM (64 registers):
// at its natural 96 registers a 640-thread CTA (32 columns of a 20-row element) held an SM alone.
template <int DIM, int K, int MODE, int CWW>
__global__ void __launch_bounds__(LocalMultiCfg<DIM, K, CWW>::NT, LocalMultiCfg<DIM, K, CWW>::NT <= 320 ? 3 : 1)
    local_df_multi_kernel(DevMesh mesh, TabsDf T, const df2* __restrict__ geo, const df2* __restrict__ Hinv,
                          double alpha, df2 tau, int R, const double* __restrict__ F, const double* __restrict__ hist,
                          SrcArgs src, const double* __restrict__ lam, double* __restrict__ out) {
  using D = Dims<DIM, K>;
  using L = LocalMultiCfg<DIM, K, CWW>;
  constexpr int NP = D::NP, NF = D::NF, M = D::M, NFC = D::NFC, N = D::N, CW = L::CW;
  __shared__ df2 g[GEO_STRIDE];
  __shared__ df2 Tr[DIM * NP][CW];
  __shared__ df2 rp[NP][CW];
  __shared__ df2 pp[NP][CW];
  __shared__ df2 ll[M][CW];
  __shared__ df2 co[4];   // 1/b, a' dJ, b dJ, 1/(b dJ) with b = alpha rho, a' = alpha/(rho c^2)
  __shared__ int fuse[NFC];
  const int64_t e = blockIdx.x;
  const int jl = threadIdx.x % CW, i = threadIdx.x / CW;
  const int j = blockIdx.y * CW + jl;
  const bool col = j < R;
  for (int t = threadIdx.x; t < GEO_STRIDE; t += L::NT) g[t] = geo[e * GEO_STRIDE + t];
  if (threadIdx.x < NFC) {
    int use = 0;
    if (lam) {
      const int f = mesh.elem_face[e * NFC + threadIdx.x];
      use = (MODE == 1) || (mesh.face_bnd[f] >= 0);
    }
    fuse[threadIdx.x] = use;
  }
  if (threadIdx.x == 0) {
    const double rho = mesh.rho[e], cc = mesh.c[e], dJ = mesh.geo[e * GEO_STRIDE];
    const double b = alpha * rho, ap = alpha / (rho * cc * cc);
    co[0] = df_from(1.0 / b);
    co[1] = df_from(ap * dJ);
    co[2] = df_from(b * dJ);
    co[3] = df_from(1.0 / (b * dJ));
  }
  for (int t = threadIdx.x; t < M * CW; t += L::NT) {
    const int r = t / CW, jj = blockIdx.y * CW + t % CW;
    double v = 0.0;
    if (lam && jj < R) {
      const int f = mesh.elem_face[e * NFC + r / NF];
      if ((MODE == 1) || (mesh.face_bnd[f] >= 0)) v = lam[((int64_t)f * NF + r % NF) * R + jj];
    }
    ll[r][t % CW] = df_from(v);
  }
  __syncthreads();
  const df2 ib = co[0];
  df2 Fu[DIM + 1];
  {
    df2 Fl[NFC];
#pragma unroll
    for (int f = 0; f < NFC; ++f) {
      DfAcc s;
      if (fuse[f])
        for (int mm = 0; mm < NF; ++mm) s.fma(T.FfT[(f * NF + mm) * NP + i], ll[f * NF + mm][jl]);
      Fl[f] = df_of(s);
    }
#pragma unroll
    for (int comp = 0; comp <= DIM; ++comp) {
      df2 v{0.f, 0.f};
      if (col) {
        const int64_t idx = (e * N + comp * NP + i) * R + j;
        if (hist) {
          v = df_mul(co[comp == 0 ? 1 : 2], df_from(hist[idx]));
          if (comp == 0 && src.ptr && src.ptr[e] < src.ptr[e + 1]) {
            double sv = 0.0;
            for (int q = src.ptr[e]; q < src.ptr[e + 1]; ++q)
              if (src.col[q] == j) sv += ricker_at(src, q) * src.phi[(int64_t)q * NP + i];
            v = df_add(v, df_from(sv));
          }
        } else {
          v = df_from(F[idx]);
        }
      }
      DfAcc bl;
      if (comp == 0) {
#pragma unroll
        for (int f = 0; f < NFC; ++f) bl.fma(g[D::OJF + f], Fl[f]);
        v = df_add(v, df_mul(tau, df_of(bl)));
      } else {
#pragma unroll
        for (int f = 0; f < NFC; ++f) bl.fma(df_mul(g[D::ON + f * DIM + comp - 1], g[D::OJF + f]), Fl[f]);
        v = df_add(v, df_neg(df_of(bl)));
      }
      Fu[comp] = v;
    }
  }
#pragma unroll
  for (int r = 0; r < DIM; ++r) {
    DfAcc s;
#pragma unroll
    for (int jj = 0; jj < DIM; ++jj) s.fma(g[1 + r * DIM + jj], Fu[jj + 1]);
    Tr[r * NP + i][jl] = df_of(s);
  }
  __syncthreads();
  {
    DfAcc s;
#pragma unroll
    for (int r = 0; r < DIM; ++r)
      for (int l = 0; l < NP; ++l) s.fma(T.DrT[(r * NP + l) * NP + i], Tr[r * NP + l][jl]);
    rp[i][jl] = df_add(Fu[0], df_neg(df_mul(df_of(s), ib)));
  }
  __syncthreads();
  {
    const df2* He = Hinv + e * (int64_t)(NP * NP);
    DfAcc s;
    for (int l = 0; l < NP; ++l) s.fma(He[l * NP + i], rp[l][jl]);
    pp[i][jl] = df_of(s);
  }
  __syncthreads();
  df2 vv[DIM];
  {
    df2 qd[DIM];
#pragma unroll
    for (int r = 0; r < DIM; ++r) {
      DfAcc s;
      for (int l = 0; l < NP; ++l) s.fma(T.Dr[(r * NP + l) * NP + i], pp[l][jl]);
      qd[r] = df_of(s);
    }
#pragma unroll
    for (int jj = 0; jj < DIM; ++jj) {
      DfAcc s;
#pragma unroll
      for (int r = 0; r < DIM; ++r) s.fma(g[1 + r * DIM + jj], qd[r]);
      vv[jj] = df_add(df_mul(Fu[jj + 1], co[3]), df_mul(df_of(s), ib));
    }
  }
  if (MODE == 1) {
    if (col) {
      out[(e * N + i) * R + j] = df_to(pp[i][jl]);
#pragma unroll
      for (int jj = 0; jj < DIM; ++jj) out[(e * N + (jj + 1) * NP + i) * R + j] = df_to(vv[jj]);
    }
    return;
  }
  __syncthreads();   // all reads of Tr done: reuse it (and rp) for the face weights
  {
    const df2 tp = df_mul(tau, pp[i][jl]);
#pragma unroll
    for (int f = 0; f < NFC; ++f) {
      DfAcc s;
#pragma unroll
      for (int jj = 0; jj < DIM; ++jj) s.fma(g[D::ON + f * DIM + jj], vv[jj]);
      const df2 wv = df_add(tp, df_of(s));
      if (f < DIM) Tr[f * NP + i][jl] = wv;
      else rp[i][jl] = wv;
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < M * CW; t += L::NT) {
    const int r = t / CW, jj2 = t % CW, f = r / NF, mm = r % NF;
    const int jc = blockIdx.y * CW + jj2;
    if (jc >= R) continue;
    DfAcc s;
    for (int q = 0; q < NP; ++q) s.fma(T.Ff[(f * NP + q) * NF + mm], f < DIM ? Tr[f * NP + q][jj2] : rp[q][jj2]);
    out[(e * M + r) * R + jc] = df_to(df_mul(g[D::OJF + f], df_of(s)));
  }
}

}  // namespace hdg
