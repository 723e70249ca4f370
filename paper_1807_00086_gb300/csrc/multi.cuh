// Multi-right-hand-side kernels: R columns (R a power of two, 2..256) share every S_K,
// H^{-1} and table read. Layouts put the column index innermost:
//   fields [n_elem][n][R], traces and Krylov vectors [n_faces][Nf][R], slots [n_elem][m][R].
// Each column is an independent problem (its own sources and Krylov recurrence); the
// operators are the same as in the single-column kernels of kernels.cuh.
#pragma once
#include "kernels.cuh"
#include "devloop.cuh"

namespace hdg {

// ------------------------------------------------------------------ element-local solves, R columns
// CTA = one element x CW columns x NP rows; with CW = 32 a warp is one row over 32 columns, so
// table, geometry and H^{-1} reads are warp-uniform and field reads are coalesced along columns.
// CW = columns per CTA: min(R, 32) (16 when N_p > 32), so a narrow batch (a few serving slots)
// keeps every thread busy.
template <int DIM, int K, int CWW = 32>
struct LocalMultiCfg {
  static constexpr int NP = Dims<DIM, K>::NP;
  static constexpr int CW = (NP <= 32 ? 32 : 16) < CWW ? (NP <= 32 ? 32 : 16) : CWW;
  static constexpr int NT = NP * CW;
};

template <int DIM, int K, int MODE, int CWW = 32>
__global__ void __launch_bounds__(LocalMultiCfg<DIM, K, CWW>::NT)
    local_multi_kernel(DevMesh mesh, Tabs T, const double* __restrict__ Hinv, double alpha, double tau, int R,
                       const double* __restrict__ F, const double* __restrict__ hist, SrcArgs src,
                       const double* __restrict__ lam, double* __restrict__ out) {
  using D = Dims<DIM, K>;
  using L = LocalMultiCfg<DIM, K, CWW>;
  constexpr int NP = D::NP, NF = D::NF, M = D::M, NFC = D::NFC, N = D::N, CW = L::CW;
  __shared__ double g[GEO_STRIDE];
  __shared__ double Tr[DIM * NP][CW];
  __shared__ double rp[NP][CW];
  __shared__ double pp[NP][CW];
  __shared__ double ll[M][CW];
  __shared__ int fuse[NFC];
  const int64_t e = blockIdx.x;
  const int jl = threadIdx.x % CW, i = threadIdx.x / CW;
  const int j = blockIdx.y * CW + jl;
  const bool col = j < R;
  for (int t = threadIdx.x; t < GEO_STRIDE; t += L::NT) g[t] = mesh.geo[e * GEO_STRIDE + t];   // NT may be < 32
  if (threadIdx.x < NFC) {
    int use = 0;
    if (lam) {
      const int f = mesh.elem_face[e * NFC + threadIdx.x];
      use = (MODE == 1) || (mesh.face_bnd[f] >= 0);
    }
    fuse[threadIdx.x] = use;
  }
  for (int t = threadIdx.x; t < M * CW; t += L::NT) {
    const int r = t / CW, jj = blockIdx.y * CW + t % CW;
    double v = 0.0;
    if (lam && jj < R) {
      const int f = mesh.elem_face[e * NFC + r / NF];
      if ((MODE == 1) || (mesh.face_bnd[f] >= 0)) v = lam[((int64_t)f * NF + r % NF) * R + jj];
    }
    ll[r][t % CW] = v;
  }
  __syncthreads();
  const double dJ = g[0];
  const double rho = mesh.rho[e], cc = mesh.c[e];
  const double b = alpha * rho;
  double Fu[DIM + 1];
  {
    double Fl[NFC];
#pragma unroll
    for (int f = 0; f < NFC; ++f) {
      double s = 0.0;
      if (fuse[f])
        for (int mm = 0; mm < NF; ++mm) s += T.Ff[(f * NP + i) * NF + mm] * ll[f * NF + mm][jl];
      Fl[f] = s;
    }
#pragma unroll
    for (int comp = 0; comp <= DIM; ++comp) {
      double v = 0.0;
      if (col) {
        const int64_t idx = (e * N + comp * NP + i) * R + j;
        if (hist) {
          v = (comp == 0 ? alpha * dJ / (rho * cc * cc) : b * dJ) * hist[idx];
          if (comp == 0 && src.ptr)
            for (int q = src.ptr[e]; q < src.ptr[e + 1]; ++q)
              if (src.col[q] == j) v += ricker_at(src, q) * src.phi[(int64_t)q * NP + i];
        } else {
          v = F[idx];
        }
      }
      double bl = 0.0;
      if (comp == 0) {
#pragma unroll
        for (int f = 0; f < NFC; ++f) bl += g[D::OJF + f] * Fl[f];
        v += tau * bl;
      } else {
#pragma unroll
        for (int f = 0; f < NFC; ++f) bl += g[D::ON + f * DIM + comp - 1] * g[D::OJF + f] * Fl[f];
        v -= bl;
      }
      Fu[comp] = v;
    }
  }
#pragma unroll
  for (int r = 0; r < DIM; ++r) {
    double s = 0.0;
#pragma unroll
    for (int jj = 0; jj < DIM; ++jj) s += g[1 + r * DIM + jj] * Fu[jj + 1];
    Tr[r * NP + i][jl] = s;
  }
  __syncthreads();
  {
    double s = 0.0;
#pragma unroll
    for (int r = 0; r < DIM; ++r)
      for (int l = 0; l < NP; ++l) s += T.Dr[(r * NP + i) * NP + l] * Tr[r * NP + l][jl];
    rp[i][jl] = Fu[0] - s / b;
  }
  __syncthreads();
  {
    const double* He = Hinv + e * (int64_t)(NP * NP);
    double s = 0.0;
    for (int l = 0; l < NP; ++l) s += He[i * NP + l] * rp[l][jl];
    pp[i][jl] = s;
  }
  __syncthreads();
  double vv[DIM];
  {
    double qd[DIM];
#pragma unroll
    for (int r = 0; r < DIM; ++r) {
      double s = 0.0;
      for (int l = 0; l < NP; ++l) s += T.Dr[(r * NP + l) * NP + i] * pp[l][jl];
      qd[r] = s;
    }
#pragma unroll
    for (int jj = 0; jj < DIM; ++jj) {
      double s = 0.0;
#pragma unroll
      for (int r = 0; r < DIM; ++r) s += g[1 + r * DIM + jj] * qd[r];
      vv[jj] = Fu[jj + 1] / (b * dJ) + s / b;
    }
  }
  if (MODE == 1) {
    if (col) {
      out[(e * N + i) * R + j] = pp[i][jl];
#pragma unroll
      for (int jj = 0; jj < DIM; ++jj) out[(e * N + (jj + 1) * NP + i) * R + j] = vv[jj];
    }
    return;
  }
  __syncthreads();   // all reads of Tr done: reuse it (and rp) for the face weights
#pragma unroll
  for (int f = 0; f < NFC; ++f) {
    double s = tau * pp[i][jl];
#pragma unroll
    for (int jj = 0; jj < DIM; ++jj) s += g[D::ON + f * DIM + jj] * vv[jj];
    if (f < DIM) Tr[f * NP + i][jl] = s;
    else rp[i][jl] = s;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < M * CW; t += L::NT) {
    const int r = t / CW, jj2 = t % CW, f = r / NF, mm = r % NF;
    const int jc = blockIdx.y * CW + jj2;
    if (jc >= R) continue;
    double s = 0.0;
    for (int q = 0; q < NP; ++q) s += T.Ff[(f * NP + q) * NF + mm] * (f < DIM ? Tr[f * NP + q][jj2] : rp[q][jj2]);
    out[(e * M + r) * R + jc] = g[D::OJF + f] * s;
  }
}

// ------------------------------------------------------------------ trace apply, R columns
// warp = (element, 32-column group); lane = column. S_K entries are warp-uniform loads.
// FP32: S from the packed group layout of pack32_kernel. FP64: S from [e][M][M].
// Warp = 32 / CWN elements x CWN columns (CWN = min(R, 32)); the FP32 S_K is read from the
// 32-element group layout of the single-column path (consecutive elements of a warp read
// consecutive float4s), the FP64 S_K from [e][m][m].
template <int DIM, int K, typename TV, int CWN = 32>
__global__ void __launch_bounds__(128) apply_multi_kernel(int64_t ne, int R, const int32_t* __restrict__ elem_face,
                                                          const int32_t* __restrict__ face_bnd,
                                                          const float* __restrict__ S32, const double* __restrict__ S64,
                                                          const TV* __restrict__ x, TV* __restrict__ slot,
                                                          const int* __restrict__ done) {
  using Dm = Dims<DIM, K>;
  using PK = Packed<DIM, K>;
  constexpr int NF = Dm::NF, M = Dm::M, NFC = Dm::NFC, P4 = PK::P4, EPW = 32 / CWN;
  if (done && *done) return;
  const int lane = threadIdx.x & 31;
  const int64_t e = ((int64_t)blockIdx.x * 4 + (threadIdx.x >> 5)) * EPW + lane / CWN;
  const int j = blockIdx.y * CWN + lane % CWN;
  if (e >= ne) return;
  const bool col = j < R;
  TV xl[M], y[M];
#pragma unroll
  for (int f = 0; f < NFC; ++f) {
    const int fid = elem_face[e * NFC + f];
    const bool use = face_bnd[fid] < 0 && col;
#pragma unroll
    for (int mm = 0; mm < NF; ++mm) xl[f * NF + mm] = use ? x[((int64_t)fid * NF + mm) * R + j] : TV(0);
  }
#pragma unroll
  for (int r = 0; r < M; ++r) y[r] = TV(0);
  if constexpr (sizeof(TV) == 4) {
    const float4* Sg = reinterpret_cast<const float4*>(S32) + (e >> 5) * (int64_t)P4 * 32 + (e & 31);
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int r = 0; r < M; ++r) {
#pragma unroll
      for (int c = r; c < M; ++c) {
        const int p = packed_index(M, r, c);
        if ((p & 3) == 0) v = Sg[(p >> 2) * 32];
        const float s = (p & 3) == 0 ? v.x : (p & 3) == 1 ? v.y : (p & 3) == 2 ? v.z : v.w;
        y[r] = fmaf(s, xl[c], y[r]);
        if (c != r) y[c] = fmaf(s, xl[r], y[c]);
      }
    }
  } else {
    const double* Se = S64 + e * (int64_t)(M * M);
#pragma unroll
    for (int r = 0; r < M; ++r) {
#pragma unroll
      for (int c = r; c < M; ++c) {
        const double s = Se[r * M + c];
        y[r] += s * xl[c];
        if (c != r) y[c] += s * xl[r];
      }
    }
  }
  if (col) {
#pragma unroll
    for (int r = 0; r < M; ++r) slot[(e * M + r) * R + j] = y[r];
  }
}

// FP64-accurate R-column apply on the FP32 pipe (the refinement residual of the mixed
// multi-column path): S_K = hi + lo as full row-major FP32 pairs [e][m][m], x split into
// double-floats and staged lane-contiguous in shared memory, one compensated accumulator per
// (row, lane). Warp = 32 / CWN elements x CWN columns.
template <int DIM, int K>
struct ApplyDfMCfg {   // warps per block: the staged x (M x 32 double-floats per warp) stays under 48 KB
  static constexpr int WPB = Dims<DIM, K>::M * 32 * 8 * 4 <= 48 * 1024 ? 4 : 2;
};

template <int DIM, int K, int CWN>
__global__ void __launch_bounds__(32 * ApplyDfMCfg<DIM, K>::WPB) apply_df_multi_kernel(int64_t ne, int R, const int32_t* __restrict__ elem_face,
                                                             const int32_t* __restrict__ face_bnd,
                                                             const float* __restrict__ Shi,
                                                             const float* __restrict__ Slo,
                                                             const double* __restrict__ x, double* __restrict__ slot) {
  using Dm = Dims<DIM, K>;
  constexpr int NF = Dm::NF, M = Dm::M, NFC = Dm::NFC, EPW = 32 / CWN, WPB = ApplyDfMCfg<DIM, K>::WPB;
  __shared__ df2 xs[WPB][M][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t e = ((int64_t)blockIdx.x * WPB + w) * EPW + lane / CWN;
  const int j = blockIdx.y * CWN + lane % CWN;
  const bool live = e < ne && j < R;
#pragma unroll
  for (int f = 0; f < NFC; ++f) {
    const int fid = live ? elem_face[e * NFC + f] : 0;
    const bool use = live && face_bnd[fid] < 0;
#pragma unroll
    for (int mm = 0; mm < NF; ++mm) xs[w][f * NF + mm][lane] = df_from(use ? x[((int64_t)fid * NF + mm) * R + j] : 0.0);
  }
  __syncwarp();
  if (!live) return;
  const float* Sh = Shi + e * (int64_t)(M * M);
  const float* Sl = Slo + e * (int64_t)(M * M);
  for (int r = 0; r < M; ++r) {
    DfAcc acc;
#pragma unroll 8
    for (int c = 0; c < M; ++c) acc.fma(df2{__ldg(Sh + r * M + c), __ldg(Sl + r * M + c)}, xs[w][c][lane]);
    slot[(e * M + r) * R + j] = acc.value();
  }
}

// hi = fl32(S), lo = fl32(S - hi), full [e][m][m]
static __global__ void split_df_kernel(int64_t n, const double* __restrict__ S, float* __restrict__ hi,
                                       float* __restrict__ lo) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const float h = __double2float_rn(S[t]);
    hi[t] = h;
    lo[t] = __double2float_rn(S[t] - (double)h);
  }
}

// FP32 S for the multi-column path: element-major packed upper triangles [e][P4] float4, so a
// CTA streams its elements' blocks contiguously into shared memory.
template <int DIM, int K>
__global__ void pack32m_kernel(int64_t ne, const double* __restrict__ S, float* __restrict__ S32m) {
  using PK = Packed<DIM, K>;
  constexpr int M = PK::M, P4 = PK::P4;
  const int64_t n = ne * P4 * 4;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = t / (P4 * 4);
    const int p = (int)(t % (P4 * 4));
    float v = 0.f;
    if (p < PK::P) {
      int r = 0;
      while (packed_index(M, r, M - 1) < p) ++r;
      const int c = r + (p - packed_index(M, r, r));
      v = (float)S[e * (int64_t)(M * M) + r * M + c];
    }
    S32m[t] = v;
  }
}

// CTA = EPB elements x all column groups (CG = R/32 warps per element); the elements' packed
// S_K are staged once in shared memory and read by every warp as broadcasts.
template <int DIM, int K>
struct Apply32mCfg {
  static constexpr int P4 = Packed<DIM, K>::P4;
  static constexpr int EPB = 4;
};

template <int DIM, int K>
__global__ void __launch_bounds__(256) apply32m_kernel(int64_t ne, int R, const int32_t* __restrict__ elem_face,
                                                       const int32_t* __restrict__ face_bnd, const float4* __restrict__ S32m,
                                                       const float* __restrict__ x, float* __restrict__ slot,
                                                       const int* __restrict__ done) {
  using Dm = Dims<DIM, K>;
  using PK = Packed<DIM, K>;
  constexpr int NF = Dm::NF, M = Dm::M, NFC = Dm::NFC, P4 = PK::P4, EPB = Apply32mCfg<DIM, K>::EPB;
  __shared__ float4 Ss[EPB * P4];
  if (done && *done) return;
  const int64_t e0 = (int64_t)blockIdx.x * EPB;
  const int nel = (int)((ne - e0) < EPB ? (ne - e0) : EPB);
  for (int t = threadIdx.x; t < nel * P4; t += blockDim.x) Ss[t] = __ldcs(S32m + e0 * P4 + t);
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int cgs = (R + 31) / 32;                 // column groups
  for (int task = w; task < nel * cgs; task += blockDim.x >> 5) {
    const int el = task / cgs, cg = task % cgs;
    const int64_t e = e0 + el;
    const int j = cg * 32 + lane;
    const bool col = j < R;
    float xl[M], y[M];
#pragma unroll
    for (int f = 0; f < NFC; ++f) {
      const int fid = elem_face[e * NFC + f];
      const bool use = face_bnd[fid] < 0 && col;
#pragma unroll
      for (int mm = 0; mm < NF; ++mm) xl[f * NF + mm] = use ? x[((int64_t)fid * NF + mm) * R + j] : 0.f;
    }
#pragma unroll
    for (int r = 0; r < M; ++r) y[r] = 0.f;
    const float4* Se = Ss + el * P4;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int r = 0; r < M; ++r) {
#pragma unroll
      for (int c = r; c < M; ++c) {
        const int p = packed_index(M, r, c);
        if ((p & 3) == 0) v = Se[p >> 2];
        const float s = (p & 3) == 0 ? v.x : (p & 3) == 1 ? v.y : (p & 3) == 2 ? v.z : v.w;
        y[r] = fmaf(s, xl[c], y[r]);
        if (c != r) y[c] = fmaf(s, xl[r], y[c]);
      }
    }
    if (col) {
#pragma unroll
      for (int r = 0; r < M; ++r) slot[(e * M + r) * R + j] = y[r];
    }
  }
}

// Tensor-core apply of S_K to the R-column trace block of every element, Y_K = S_K X_K (m x R),
// R a multiple of 8: the GEMM-shaped contraction of the multi-source batch, as warp-level
// mma.sync m16n8k8 with TF32 operands and FP32 accumulation. Each CTA stages WPB elements'
// packed S_K and gathered X_K (boundary faces read as 0) in shared memory; warp w multiplies
// element w: the A fragments (S_K rounded to TF32, rows and columns padded to the tile sizes with
// zeros) are loaded once per element, X is split into X_hi + X_lo (both TF32), so the product
// carries only the TF32 rounding of S_K (relative 2^-11, the accuracy class of the FP16 inner
// operator) and not that of the Krylov vector. Output slots [e][m][R] as apply32m_kernel.
template <int DIM, int K>
struct ApplyTcCfg {
  static constexpr int M = Dims<DIM, K>::M;
  static constexpr int P4 = Packed<DIM, K>::P4;
  static constexpr int MT = (M + 15) / 16;   // 16-row tiles of S_K
  static constexpr int KS = (M + 7) / 8;     // 8-wide k steps
  static constexpr int WPB = 4;              // warps (= elements in flight) per CTA
  static constexpr int XS = 64 + 8;          // padded row of the staged X (64 columns per pass; conflict-free B reads)
  static constexpr size_t SMEM = (size_t)WPB * (P4 * 16 + (size_t)KS * 8 * XS * 4);
};

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// NC columns per pass (32 for R = 32, else 64; R a multiple of NC)
template <int DIM, int K, int NC>
__global__ void __launch_bounds__(32 * ApplyTcCfg<DIM, K>::WPB) apply_tc_kernel(
    int64_t ne, int R, const int32_t* __restrict__ elem_face, const int32_t* __restrict__ face_bnd,
    const float4* __restrict__ S32m, const float* __restrict__ x, float* __restrict__ slot, const int* __restrict__ done) {
  using C = ApplyTcCfg<DIM, K>;
  using Dm = Dims<DIM, K>;
  constexpr int M = C::M, NF = Dm::NF, NFC = Dm::NFC, P4 = C::P4, MT = C::MT, KS = C::KS, WPB = C::WPB, XS = C::XS;
  constexpr int Q = NC / 4, NLD = KS * 8 * Q, LPL = (NLD + 31) / 32;   // float4 loads of X: total, per lane
  if (done && *done) return;
  extern __shared__ float4 smem4[];
  float* sS = reinterpret_cast<float*>(smem4);                 // [WPB][P4 * 4] packed S_K
  float* sX = sS + WPB * P4 * 4;                               // [WPB][KS * 8][XS] X_K, NC columns per pass
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int g = lane >> 2, tq = lane & 3;
  const int64_t e0 = (int64_t)blockIdx.x * WPB;
  const int nel = (int)((ne - e0) < WPB ? (ne - e0) : WPB);
  // packed S_K of the CTA's elements (contiguous in the element-major packed layout)
  for (int t = threadIdx.x; t < nel * P4; t += blockDim.x) smem4[t] = __ldcs(S32m + e0 * P4 + t);
  const int el = w;
  const bool act = el < nel;
  const int64_t e = e0 + (act ? el : 0);
  const float* Se = sS + el * P4 * 4;
  float* Xe = sX + (size_t)el * KS * 8 * XS;
  // the element's faces: lane f < NFC holds face f's trace offset (-1: boundary, read as zero)
  int64_t fo = -1;
  if (act && lane < NFC) {
    const int f = elem_face[e * NFC + lane];
    fo = face_bnd[f] < 0 ? (int64_t)f * NF * R : -1;
  }
  // A fragments of this warp's element, once: rows mt*16 + g (+8), columns ks*8 + tq (+4)
  uint32_t a[MT][KS][4];
  for (int c0 = 0; c0 < R; c0 += NC) {
    __syncthreads();   // S staged (first pass) / previous pass done with X
    // stage X_K (rows k < M from the element's faces, rows M..KS*8 and boundary faces zero) with
    // 16-byte asynchronous copies: every copy of the pass is in flight before the first is used;
    // a zero-filled chunk reads no global memory (source size 0, a valid address is passed)
    const unsigned xs = (unsigned)__cvta_generic_to_shared(Xe);
#pragma unroll 4
    for (int i = 0; i < LPL; ++i) {
      const int t = lane + 32 * i;
      const int r = (t < NLD ? t : 0) / Q, q = t % Q;
      const int64_t off = __shfl_sync(0xffffffffu, fo, (r < M ? r : 0) / NF);
      if (t < NLD) {
        const bool rd = act && r < M && off >= 0;
        const float* src = rd ? x + off + (int64_t)(r % NF) * R + c0 + 4 * q : x;
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(xs + 4u * (unsigned)(r * XS + 4 * q)),
                     "l"(src), "r"(rd ? 16 : 0)
                     : "memory");
      }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncwarp();
    if (!act) continue;
    if (c0 == 0) {
#pragma unroll
      for (int mt = 0; mt < MT; ++mt)
#pragma unroll
        for (int ks = 0; ks < KS; ++ks)
#pragma unroll
          for (int h = 0; h < 4; ++h) {
            const int r = mt * 16 + g + (h & 1) * 8, cc = ks * 8 + tq + (h >> 1) * 4;
            float sv = 0.f;
            if (r < M && cc < M) sv = Se[r <= cc ? packed_index(M, r, cc) : packed_index(M, cc, r)];
            a[mt][ks][h] = to_tf32(sv);
          }
    }
#pragma unroll 2
    for (int nt = 0; nt < NC / 8; ++nt) {
      float acc[MT][4];
#pragma unroll
      for (int mt = 0; mt < MT; ++mt) acc[mt][0] = acc[mt][1] = acc[mt][2] = acc[mt][3] = 0.f;
#pragma unroll
      for (int ks = 0; ks < KS; ++ks) {
        const float x0 = Xe[(ks * 8 + tq) * XS + nt * 8 + g];
        const float x1 = Xe[(ks * 8 + tq + 4) * XS + nt * 8 + g];
        const uint32_t h0 = to_tf32(x0), h1 = to_tf32(x1);
        const uint32_t l0 = to_tf32(x0 - __uint_as_float(h0)), l1 = to_tf32(x1 - __uint_as_float(h1));
#pragma unroll
        for (int mt = 0; mt < MT; ++mt) {
          mma_tf32(acc[mt], a[mt][ks], h0, h1);
          mma_tf32(acc[mt], a[mt][ks], l0, l1);
        }
      }
      // D fragment: (row g, cols 2 tq, 2 tq + 1) and (row g + 8, same cols) of each 16 x 8 tile
#pragma unroll
      for (int mt = 0; mt < MT; ++mt) {
        const int col = c0 + nt * 8 + 2 * tq;
        const int r0 = mt * 16 + g, r1 = r0 + 8;
        if (r0 < M) *reinterpret_cast<float2*>(slot + (e * M + r0) * R + col) = make_float2(acc[mt][0], acc[mt][1]);
        if (r1 < M) *reinterpret_cast<float2*>(slot + (e * M + r1) * R + col) = make_float2(acc[mt][2], acc[mt][3]);
      }
    }
  }
}

// ------------------------------------------------------------------ per-column Krylov kernels
// Vector entries t = entry * R + column; with a grid stride that is a multiple of R (256
// threads per block, R | 256) every thread keeps one column, so per-thread accumulators
// are per column. Block partials: part[blk][R]; column scalars are reduced in fixed order.
template <typename TV>
struct MAcc;
template <>
struct MAcc<float> {
  Acc2 a;
  __device__ __forceinline__ void dot(float x, float y) { a.dot(x, y); }
  __device__ __forceinline__ double value() const { return a.value(); }
};
template <>
struct MAcc<double> {
  double s = 0.0;
  __device__ __forceinline__ void dot(double x, double y) { s += x * y; }
  __device__ __forceinline__ double value() const { return s; }
};

// per-column block sum of one value per thread (thread t holds column t % R); result in red[0..R)
__device__ __forceinline__ void block_cols(double v, int R, double* red /*[256]*/) {
  __syncthreads();
  red[threadIdx.x] = v;
  __syncthreads();
  for (int w = 128; w >= R; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
}

// Per-column sums of block partials part[(b0 + b) * R + j] (b < nb) by the whole block (256
// threads, R a power of two <= 256): 256 / R threads per column, each with four accumulators
// (so four independent loads are in flight: one dependent chain of nb / G loads made the
// single-block scalar kernels latency-bound), fixed partition, order and tree, so the sums are
// deterministic; column j's sum is left in red[j].
__device__ __forceinline__ void col_partials(const double* __restrict__ part, int nb, int R, int64_t b0,
                                             double* red /*[256]*/) {
  const int G = 256 / R, j = threadIdx.x & (R - 1), g = threadIdx.x / R;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  int b = g;
  for (; b + 3 * G < nb; b += 4 * G) {
    s0 += part[(b0 + b) * R + j];
    s1 += part[(b0 + b + G) * R + j];
    s2 += part[(b0 + b + 2 * G) * R + j];
    s3 += part[(b0 + b + 3 * G) * R + j];
  }
  for (; b < nb; b += G) s0 += part[(b0 + b) * R + j];
  block_cols((s0 + s1) + (s2 + s3), R, red);
}

// Per-column least-squares initial guess over stored pairs (b_i, lam_i), i < q, ring
// [q][n R] (column innermost). mdots_ring_kernel: block partials of (b_i, w)_j and (w, w)_j
// per column, part[blk][q + 1][R]; the grid stride is a multiple of R, so each thread keeps
// one column.
static __global__ void mdots_ring_kernel(int64_t n, int R, int q, int64_t stride, const double* __restrict__ ring,
                                         const double* __restrict__ w, double* __restrict__ part) {
  __shared__ double red[256];
  double acc[9];
  for (int i = 0; i <= q; ++i) acc[i] = 0.0;
  for (int64_t t = blockIdx.x * 256 + threadIdx.x; t < n; t += (int64_t)gridDim.x * 256) {
    const double wv = w[t];
    for (int i = 0; i < q; ++i) acc[i] += ring[i * stride + t] * wv;
    acc[q] += wv * wv;
  }
  for (int i = 0; i <= q; ++i) {
    block_cols(acc[i], R, red);
    if (threadIdx.x < R) part[((int64_t)blockIdx.x * (q + 1) + i) * R + threadIdx.x] = red[threadIdx.x];
  }
}

static __global__ void mdots_final_kernel(int nb, int R, int q, const double* __restrict__ part,
                                          double* __restrict__ out) {
  __shared__ double red[256];
  for (int i = 0; i <= q; ++i) {
    // column sums of part[b][i][j] over b: stride (q + 1) R between blocks
    const int G = 256 / R, j = threadIdx.x & (R - 1), g = threadIdx.x / R;
    double s = 0.0;
    for (int b = g; b < nb; b += G) s += part[((int64_t)b * (q + 1) + i) * R + j];
    block_cols(s, R, red);
    if (threadIdx.x < R) out[i * R + threadIdx.x] = red[threadIdx.x];
  }
}

// out[t] = sum_i coef[i][j] ring[i][t] (j = t mod R) on interior entries (mask per trace entry);
// a column whose coef[0][j] is NaN (no usable history) keeps its current values
static __global__ void mlincomb_ring_kernel(int64_t n, int R, int q, int64_t stride, const double* __restrict__ ring,
                                            const double* __restrict__ coef, const uint8_t* __restrict__ mask,
                                            double* __restrict__ out) {
  const int lg = __ffs(R) - 1;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    if (!mask[t >> lg]) continue;
    const int j = (int)(t & (R - 1));
    if (isnan(coef[j])) continue;
    double s = 0.0;
    for (int i = 0; i < q; ++i) s += coef[i * R + j] * ring[i * stride + t];
    out[t] = s;
  }
}

struct MScal {              // per-column Krylov scalars, arrays of R entries
  double *rho0, *rho1, *alpha, *rr, *bb, *tol2;
  int* conv;                // per column: converged
  int* done;                // all columns converged (or maxit)
  int* iters;               // iterations executed
};

// q = (-K) p; partial p.q per column
template <int DIM, int K, typename TV>
__global__ void __launch_bounds__(256) mface_q_kernel(int nf, int R, const int32_t* __restrict__ face_slot,
                                                      const int32_t* __restrict__ face_bnd, const TV* __restrict__ slot,
                                                      const TV* __restrict__ p, TV* __restrict__ q,
                                                      double* __restrict__ part, const int* __restrict__ done) {
  constexpr int NF = Dims<DIM, K>::NF;
  if (*done) return;
  __shared__ double red[256];
  MAcc<TV> acc;
  const int lg = __ffs(R) - 1;   // R is a power of two
  const int64_t n = (int64_t)nf * NF * R;
  for (int64_t t = blockIdx.x * 256 + threadIdx.x; t < n; t += (int64_t)gridDim.x * 256) {
    const int j = (int)(t & (R - 1));
    const uint32_t fe = (uint32_t)(t >> lg);
    const uint32_t f = fe / NF;
    const int mm = (int)(fe - f * NF);
    TV qv = TV(0);
    if (face_bnd[f] < 0)
      qv = -(slot[((int64_t)face_slot[2 * f] * NF + mm) * R + j] + slot[((int64_t)face_slot[2 * f + 1] * NF + mm) * R + j]);
    q[t] = qv;
    acc.dot(p[t], qv);
  }
  block_cols(acc.value(), R, red);
  if (threadIdx.x < R) part[(int64_t)blockIdx.x * R + threadIdx.x] = red[threadIdx.x];
}

// alpha_j = rho_j / pq_j (0 for converged columns)
static __global__ void mcols_alpha(int nb, int R, int parity, const double* __restrict__ part, MScal sc) {
  __shared__ double red[256];
  if (*sc.done) return;
  col_partials(part, nb, R, 0, red);
  for (int j = threadIdx.x; j < R; j += blockDim.x) {
    const double s = red[j];
    const double rho = parity ? sc.rho1[j] : sc.rho0[j];
    sc.alpha[j] = (sc.conv[j] || s == 0.0) ? 0.0 : rho / s;
  }
}

template <typename TV>
__global__ void __launch_bounds__(256) mupdate_kernel(int64_t n, int R, const TV* __restrict__ p, const TV* __restrict__ q,
                                                      const TV* __restrict__ dinv, TV* __restrict__ x, TV* __restrict__ r,
                                                      TV* __restrict__ z, double* __restrict__ part, MScal sc) {
  if (*sc.done) return;
  __shared__ double red[256];
  MAcc<TV> rz, rr;
  const int j = threadIdx.x % R;
  const int lg = __ffs(R) - 1;
  const TV al = (TV)sc.alpha[j];
  for (int64_t t = blockIdx.x * 256 + threadIdx.x; t < n; t += (int64_t)gridDim.x * 256) {
    x[t] += al * p[t];
    const TV rv = r[t] - al * q[t];
    const TV zv = dinv[t >> lg] * rv;
    r[t] = rv; z[t] = zv;
    rz.dot(rv, zv); rr.dot(rv, rv);
  }
  block_cols(rz.value(), R, red);
  if (threadIdx.x < R) part[(int64_t)blockIdx.x * R + threadIdx.x] = red[threadIdx.x];
  block_cols(rr.value(), R, red);
  if (threadIdx.x < R) part[(int64_t)(gridDim.x + blockIdx.x) * R + threadIdx.x] = red[threadIdx.x];
}

// rho_new, rr per column; convergence; beta. Single block: the iteration counter lives on the
// device (read by every thread before thread 0 advances it), so launches carry no host index.
// dev != 0 (device-driven loop): thread 0 also sets the loop condition h (continue while not
// done), including when the solve had already finished.
static __global__ void mcols_beta(int nb, int R, int parity, int maxit, const double* __restrict__ part, MScal sc,
                           double* __restrict__ beta, int dev, cudaGraphConditionalHandle h) {
  __shared__ int notconv;
  if (threadIdx.x == 0) notconv = 0;
  __syncthreads();
  if (*sc.done) {
    if (dev && threadIdx.x == 0) cudaGraphSetConditional(h, 0u);
    return;
  }
  const int iter = *sc.iters;
  __shared__ double red[256], rzs[256];
  col_partials(part, nb, R, 0, red);
  if (threadIdx.x < R) rzs[threadIdx.x] = red[threadIdx.x];
  col_partials(part, nb, R, nb, red);   // starts with a barrier: rzs is complete
  for (int j = threadIdx.x; j < R; j += blockDim.x) {
    const double rz = rzs[j], rr = red[j];
    const double rho = parity ? sc.rho1[j] : sc.rho0[j];
    const int c = sc.conv[j] || rr <= sc.tol2[j];
    beta[j] = c ? 0.0 : rz / rho;
    if (parity) sc.rho0[j] = rz; else sc.rho1[j] = rz;
    sc.rr[j] = rr;
    sc.conv[j] = c;
    if (!c) atomicAdd(&notconv, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    *sc.iters = iter + 1;
    const int done = (notconv == 0 || iter + 1 >= maxit) ? (notconv == 0 ? 1 : 2) : 0;
    if (done) *sc.done = done;
    if (dev) cudaGraphSetConditional(h, done ? 0u : 1u);
  }
}

// Sweep control of the device-driven multi-column refinement, one thread: records the last
// inner solve's iterations, stops when every column has converged (nconv == 0) or after
// max_sweeps, and sets the sweep and inner-loop conditions.
static __global__ void msweep_ctl_kernel(const int* __restrict__ nconv, const int* __restrict__ iters, LoopCtl* L,
                                         int max_sweeps, cudaGraphConditionalHandle h_sweep,
                                         cudaGraphConditionalHandle h_in) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (L->sweep > 0) L->total_it += *iters;
  const int stop = *nconv == 0 ? 1 : (L->sweep >= max_sweeps ? 3 : 0);
  if (!stop) L->sweep += 1;
  L->stop = stop;
  cudaGraphSetConditional(h_sweep, stop ? 0u : 1u);
  cudaGraphSetConditional(h_in, stop ? 0u : 1u);
}

// End of a device-driven multi-column FP64 solve, one thread: iterations and stop code.
static __global__ void mcg_finish_kernel(const int* __restrict__ done, const int* __restrict__ iters, LoopCtl* L) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  L->total_it = *iters;
  L->sweep = 1;
  L->rel = 0.0;
  L->stop = *done == 1 ? 1 : 4;
}

template <typename TV>
__global__ void __launch_bounds__(256) mdirection_kernel(int64_t n, int R, const TV* __restrict__ z, TV* __restrict__ p,
                                                         const double* __restrict__ beta, const int* __restrict__ done) {
  if (*done) return;
  const TV be = (TV)beta[threadIdx.x % R];
  for (int64_t t = blockIdx.x * 256 + threadIdx.x; t < n; t += (int64_t)gridDim.x * 256) p[t] = z[t] + be * p[t];
}

// ---- column-block Krylov kernels with NV columns per thread (R a multiple of NV)
// Vectors are read NV columns at a time (float4 for the FP32 inner solve, double2 for the FP64
// refinement residual): thread t holds entry t >> lg and columns NV (t & (R/NV - 1)) + 0..NV-1.
// The grid stride (gridDim.x * 256 vector elements) is a multiple of R/NV (R/NV <= 64 divides
// 256), so a thread keeps its columns, and several independent vector loads per trip keep
// enough bytes in flight per SM to stream at HBM rate (one 4-byte load per thread and trip
// does not). In the FP32 inner solve z = D^{-1} r is not stored: the direction kernel forms it
// again from r, with the same rounding as the one-column-per-thread kernels that store it.

// per-column block sums of NV values per thread (thread t: columns NV (t mod R/NV) + c), written
// to part[row][R]; fixed partition and tree, so the sums are deterministic
template <int NV>
__device__ __forceinline__ void block_cols_v(const double (&v)[NV], int R, double* red /*[256]*/,
                                             double* __restrict__ part, int64_t row) {
  const int RV = R / NV;
#pragma unroll
  for (int c = 0; c < NV; ++c) {
    block_cols(v[c], RV, red);
    if (threadIdx.x < RV) part[row * R + NV * threadIdx.x + c] = red[threadIdx.x];
  }
}

// q = (-K) p from the two slots of each interior entry; partial p.q per column. The reducing
// kernels of this family are bounded to 64 registers, so four 256-thread CTAs are resident per
// SM and the reduction grid (a multiple of the SM count) runs in whole waves.
template <int DIM, int K>
__global__ void __launch_bounds__(256, 4) mface_q4_kernel(int nf, int R, const int2* __restrict__ face_slot2,
                                                       const int32_t* __restrict__ face_bnd,
                                                       const float4* __restrict__ slot, const float4* __restrict__ p,
                                                       float4* __restrict__ q, double* __restrict__ part,
                                                       const int* __restrict__ done) {
  constexpr int NF = Dims<DIM, K>::NF, U = 4;
  if (*done) return;
  __shared__ double red[256];
  const int R4 = R >> 2, lg = __ffs(R4) - 1, jq = threadIdx.x & (R4 - 1);
  const int64_t n4 = (int64_t)nf * NF * R4, S = (int64_t)gridDim.x * 256;
  Acc2 acc[4];
  for (int64_t t = blockIdx.x * 256 + threadIdx.x; t < n4; t += U * S) {
    float4 s0[U], s1[U], pv[U];
    bool in[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t tu = t + u * S;
      in[u] = false;
      s0[u] = s1[u] = pv[u] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (tu < n4) {
        const uint32_t fe = (uint32_t)(tu >> lg);
        const uint32_t f = fe / NF;
        const int mm = (int)(fe - f * NF);
        const int fb = face_bnd[f];
        const int2 fs = face_slot2[f];
        pv[u] = p[tu];
        if (fb < 0) {
          in[u] = true;
          s0[u] = slot[((int64_t)fs.x * NF + mm) * R4 + jq];
          s1[u] = slot[((int64_t)fs.y * NF + mm) * R4 + jq];
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t tu = t + u * S;
      if (tu >= n4) break;
      float4 qv = make_float4(0.f, 0.f, 0.f, 0.f);
      if (in[u]) qv = make_float4(-(s0[u].x + s1[u].x), -(s0[u].y + s1[u].y), -(s0[u].z + s1[u].z), -(s0[u].w + s1[u].w));
      q[tu] = qv;
      acc[0].dot(pv[u].x, qv.x); acc[1].dot(pv[u].y, qv.y); acc[2].dot(pv[u].z, qv.z); acc[3].dot(pv[u].w, qv.w);
    }
  }
  const double v[4] = {acc[0].value(), acc[1].value(), acc[2].value(), acc[3].value()};
  block_cols_v<4>(v, R, red, part, blockIdx.x);
}

// x += alpha p, r -= alpha q; partials (r, D^{-1} r) and (r, r) per column (z is not stored)
static __global__ void __launch_bounds__(256, 4) mupdate4_kernel(int64_t n4, int R, const float4* __restrict__ p,
                                                              const float4* __restrict__ q, const float* __restrict__ dinv,
                                                              float4* __restrict__ x, float4* __restrict__ r,
                                                              double* __restrict__ part, MScal sc) {
  constexpr int U = 2;
  if (*sc.done) return;
  __shared__ double red[256];
  const int R4 = R >> 2, lg = __ffs(R4) - 1, jq = threadIdx.x & (R4 - 1);
  const int64_t S = (int64_t)gridDim.x * 256;
  float al[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) al[c] = (float)sc.alpha[4 * jq + c];
  Acc2 rz[4], rr[4];
  for (int64_t t = blockIdx.x * 256 + threadIdx.x; t < n4; t += U * S) {
    float4 pv[U], qv[U], xv[U], rv[U];
    float d[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t tu = t + u * S;
      if (tu < n4) { pv[u] = p[tu]; qv[u] = q[tu]; xv[u] = x[tu]; rv[u] = r[tu]; d[u] = dinv[tu >> lg]; }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t tu = t + u * S;
      if (tu >= n4) break;
      x[tu] = make_float4(fmaf(al[0], pv[u].x, xv[u].x), fmaf(al[1], pv[u].y, xv[u].y), fmaf(al[2], pv[u].z, xv[u].z),
                          fmaf(al[3], pv[u].w, xv[u].w));
      const float4 rn = make_float4(fmaf(-al[0], qv[u].x, rv[u].x), fmaf(-al[1], qv[u].y, rv[u].y),
                                    fmaf(-al[2], qv[u].z, rv[u].z), fmaf(-al[3], qv[u].w, rv[u].w));
      r[tu] = rn;
      rz[0].dot(rn.x, __fmul_rn(d[u], rn.x)); rr[0].dot(rn.x, rn.x);
      rz[1].dot(rn.y, __fmul_rn(d[u], rn.y)); rr[1].dot(rn.y, rn.y);
      rz[2].dot(rn.z, __fmul_rn(d[u], rn.z)); rr[2].dot(rn.z, rn.z);
      rz[3].dot(rn.w, __fmul_rn(d[u], rn.w)); rr[3].dot(rn.w, rn.w);
    }
  }
  const double vz[4] = {rz[0].value(), rz[1].value(), rz[2].value(), rz[3].value()};
  block_cols_v<4>(vz, R, red, part, blockIdx.x);
  const double vr[4] = {rr[0].value(), rr[1].value(), rr[2].value(), rr[3].value()};
  block_cols_v<4>(vr, R, red, part, (int64_t)gridDim.x + blockIdx.x);
}

// Persistent form of apply_tc_kernel for exactly NC = R columns (32 or 64) inside the FP32
// Krylov iteration, with the iteration's p.q and step length in its epilogue. With
// K = sum_K P_K^T S_K P_K and q = -K p, (p, q)_j = -sum_K sum_r X_K[r][j] (S_K X_K)[r][j] (the
// gathered block is zero on boundary faces), so the face pass that formed q before alpha is not
// needed: the update kernel forms q from the two slots of each entry itself.
// Each CTA loops over groups of WPB elements (one per warp) with two stages per warp: after
// the A fragments of the current group are in registers, the packed S_K of the next group
// (all threads) and each warp's next trace block are copied by cp.async while the current
// block is multiplied. Per-lane p.q partials (columns 8 g + 2 tq, + 1 of n-tile g) are summed
// over the warp's rows by shuffles, over the CTA's warps in warp order, and the last CTA to
// finish (ticket counter, no waiting) sums the CTA partials in index order and writes
// alpha_j = rho_j / (p, q)_j (0 for converged columns).
template <int DIM, int K>
struct ApplyTcPCfg {
  using C = ApplyTcCfg<DIM, K>;
  static constexpr int WPB = 4;
  static constexpr int XB = C::KS * 8 * C::XS;   // floats of one staged trace block
  static constexpr size_t SMEM = (size_t)WPB * C::P4 * 16 + (size_t)2 * WPB * XB * 4 + (size_t)WPB * 64 * 8;
};

struct MPqOut {
  double* part;       // [gridDim.x][R] CTA partials of (p, q) per column
  unsigned* ticket;   // zero between launches
  MScal sc;           // alpha is written by the last CTA
  int parity;         // selects rho0 / rho1 as mcols_alpha does
};

template <int DIM, int K, int NC>
__global__ void __launch_bounds__(32 * ApplyTcPCfg<DIM, K>::WPB) apply_tc_pq_kernel(
    int64_t ne, const int32_t* __restrict__ elem_face, const int32_t* __restrict__ face_bnd,
    const float4* __restrict__ S32m, const float* __restrict__ x, float* __restrict__ slot, MPqOut o) {
  using C = ApplyTcCfg<DIM, K>;
  using CP = ApplyTcPCfg<DIM, K>;
  using Dm = Dims<DIM, K>;
  constexpr int M = C::M, NF = Dm::NF, NFC = Dm::NFC, P4 = C::P4, MT = C::MT, KS = C::KS, WPB = CP::WPB,
                XS = C::XS, XB = CP::XB, R = NC;
  constexpr int Q = NC / 4, NLD = KS * 8 * Q, LPL = (NLD + 31) / 32;   // float4 copies of X: total, per lane
  static_assert(NC == 32 || NC == 64, "one n-tile of 8 columns per lane group g");
  if (*o.sc.done) return;
  extern __shared__ float4 smem4[];
  float* sS = reinterpret_cast<float*>(smem4);                       // [WPB][P4 * 4] packed S_K
  float* sX = sS + WPB * P4 * 4;                                     // [2][WPB][XB] trace blocks
  double* sPq = reinterpret_cast<double*>(sX + 2 * WPB * XB);         // [WPB][NC]
  __shared__ bool last;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int g = lane >> 2, tq = lane & 3;
  const int64_t nq = (ne + WPB - 1) / WPB;
  const unsigned ss = (unsigned)__cvta_generic_to_shared(sS);
  // copies of group qd: the packed S_K of its elements (all threads) and warp w's trace block
  // (rows of boundary faces and rows M..KS*8 zero-filled: source size 0 reads no memory)
  auto stage = [&](int64_t qd, int b) {
    const int64_t e0 = qd * WPB;
    const int nel = (int)((ne - e0) < WPB ? (ne - e0) : WPB);
    for (int t = threadIdx.x; t < nel * P4; t += blockDim.x)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(ss + 16u * (unsigned)t), "l"(S32m + e0 * P4 + t)
                   : "memory");
    const bool act = w < nel;
    int64_t fo = -1;
    if (act && lane < NFC) {
      const int f = elem_face[(e0 + w) * NFC + lane];
      fo = face_bnd[f] < 0 ? (int64_t)f * NF * R : -1;
    }
    const unsigned xs = (unsigned)__cvta_generic_to_shared(sX + ((size_t)b * WPB + w) * XB);
#pragma unroll 4
    for (int i = 0; i < LPL; ++i) {
      const int t = lane + 32 * i;
      const int r = (t < NLD ? t : 0) / Q, q = t % Q;
      const int64_t off = __shfl_sync(0xffffffffu, fo, (r < M ? r : 0) / NF);
      if (t < NLD) {
        const bool rd = act && r < M && off >= 0;
        const float* src = rd ? x + off + (int64_t)(r % NF) * R + 4 * q : x;
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(xs + 4u * (unsigned)(r * XS + 4 * q)),
                     "l"(src), "r"(rd ? 16 : 0)
                     : "memory");
      }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  double pq0 = 0.0, pq1 = 0.0;   // lanes of n-tile g: columns 8 g + 2 tq and 8 g + 2 tq + 1
  int b = 0;
  if ((int64_t)blockIdx.x < nq) stage(blockIdx.x, 0);
  for (int64_t qd = blockIdx.x; qd < nq; qd += gridDim.x, b ^= 1) {
    const int64_t e0 = qd * WPB;
    const int nel = (int)((ne - e0) < WPB ? (ne - e0) : WPB);
    const bool act = w < nel;
    const int64_t e = e0 + (act ? w : 0);
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");   // this group's copies (the only ones in flight)
    __syncthreads();                                          // S_K copied by all threads is visible
    uint32_t a[MT][KS][4];
    if (act) {
      const float* Se = sS + w * P4 * 4;
#pragma unroll
      for (int mt = 0; mt < MT; ++mt)
#pragma unroll
        for (int ks = 0; ks < KS; ++ks)
#pragma unroll
          for (int h = 0; h < 4; ++h) {
            const int r = mt * 16 + g + (h & 1) * 8, cc = ks * 8 + tq + (h >> 1) * 4;
            float sv = 0.f;
            if (r < M && cc < M) sv = Se[r <= cc ? packed_index(M, r, cc) : packed_index(M, cc, r)];
            a[mt][ks][h] = to_tf32(sv);
          }
    }
    __syncthreads();   // every warp holds its A fragments: the S_K stage may be refilled
    if (qd + gridDim.x < nq) stage(qd + gridDim.x, b ^ 1);
    if (!act) continue;
    const float* Xe = sX + ((size_t)b * WPB + w) * XB;
#pragma unroll 2
    for (int nt = 0; nt < NC / 8; ++nt) {
      float acc[MT][4];
#pragma unroll
      for (int mt = 0; mt < MT; ++mt) acc[mt][0] = acc[mt][1] = acc[mt][2] = acc[mt][3] = 0.f;
#pragma unroll
      for (int ks = 0; ks < KS; ++ks) {
        const float x0 = Xe[(ks * 8 + tq) * XS + nt * 8 + g];
        const float x1 = Xe[(ks * 8 + tq + 4) * XS + nt * 8 + g];
        const uint32_t h0 = to_tf32(x0), h1 = to_tf32(x1);
        const uint32_t l0 = to_tf32(x0 - __uint_as_float(h0)), l1 = to_tf32(x1 - __uint_as_float(h1));
#pragma unroll
        for (int mt = 0; mt < MT; ++mt) {
          mma_tf32(acc[mt], a[mt][ks], h0, h1);
          mma_tf32(acc[mt], a[mt][ks], l0, l1);
        }
      }
      const int col = nt * 8 + 2 * tq;
      float v0 = 0.f, v1 = 0.f;
#pragma unroll
      for (int mt = 0; mt < MT; ++mt) {
        const int r0 = mt * 16 + g, r1 = r0 + 8;
        if (r0 < M) {
          *reinterpret_cast<float2*>(slot + (e * M + r0) * R + col) = make_float2(acc[mt][0], acc[mt][1]);
          v0 = fmaf(Xe[r0 * XS + col], acc[mt][0], v0);
          v1 = fmaf(Xe[r0 * XS + col + 1], acc[mt][1], v1);
        }
        if (r1 < M) {
          *reinterpret_cast<float2*>(slot + (e * M + r1) * R + col) = make_float2(acc[mt][2], acc[mt][3]);
          v0 = fmaf(Xe[r1 * XS + col], acc[mt][2], v0);
          v1 = fmaf(Xe[r1 * XS + col + 1], acc[mt][3], v1);
        }
      }
      // rows of the 8 lanes with this tq (g = 0..7)
      v0 += __shfl_xor_sync(0xffffffffu, v0, 4);
      v1 += __shfl_xor_sync(0xffffffffu, v1, 4);
      v0 += __shfl_xor_sync(0xffffffffu, v0, 8);
      v1 += __shfl_xor_sync(0xffffffffu, v1, 8);
      v0 += __shfl_xor_sync(0xffffffffu, v0, 16);
      v1 += __shfl_xor_sync(0xffffffffu, v1, 16);
      if (g == nt) { pq0 += (double)v0; pq1 += (double)v1; }
    }
  }
  // CTA partial per column (warps in order), then the last CTA's column sums in CTA order
  if (g < NC / 8) {
    sPq[w * NC + 8 * g + 2 * tq] = pq0;
    sPq[w * NC + 8 * g + 2 * tq + 1] = pq1;
  }
  __syncthreads();
  if (threadIdx.x < NC) {
    double v = 0.0;
#pragma unroll
    for (int w2 = 0; w2 < WPB; ++w2) v += sPq[w2 * NC + threadIdx.x];
    o.part[(int64_t)blockIdx.x * NC + threadIdx.x] = v;
    __threadfence();
  }
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(o.ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  {
    // column j = t mod NC; the blockDim / NC threads of a column take every (blockDim / NC)-th CTA
    constexpr int G = 32 * WPB / NC;
    const int j = threadIdx.x % NC, h = threadIdx.x / NC;
    double v = 0.0;
    for (unsigned bk = h; bk < gridDim.x; bk += G) v += __ldcg(o.part + (int64_t)bk * NC + j);
    __syncthreads();
    sPq[h * NC + j] = v;
    __syncthreads();
    if (threadIdx.x < NC) {
      double sum = 0.0;
#pragma unroll
      for (int h2 = 0; h2 < G; ++h2) sum += sPq[h2 * NC + j];
      const double pq = -sum;
      const double rho = o.parity ? o.sc.rho1[j] : o.sc.rho0[j];
      o.sc.alpha[j] = (o.sc.conv[j] || pq == 0.0) ? 0.0 : rho / pq;
    }
    if (threadIdx.x == 0) *o.ticket = 0u;
  }
}

// mupdate4_kernel with q = -K p formed from the two slots of each interior entry (after
// apply_tc_pq_kernel, which leaves no q vector)
template <int DIM, int K>
__global__ void __launch_bounds__(256, 4) mupdate4s_kernel(int nf, int R, const int2* __restrict__ face_slot2,
                                                        const int32_t* __restrict__ face_bnd,
                                                        const float4* __restrict__ slot, const float4* __restrict__ p,
                                                        const float* __restrict__ dinv, float4* __restrict__ x,
                                                        float4* __restrict__ r, double* __restrict__ part, MScal sc) {
  constexpr int NF = Dims<DIM, K>::NF, U = 2;
  if (*sc.done) return;
  __shared__ double red[256];
  const int R4 = R >> 2, lg = __ffs(R4) - 1, jq = threadIdx.x & (R4 - 1);
  const int64_t n4 = (int64_t)nf * NF * R4, S = (int64_t)gridDim.x * 256;
  float al[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) al[c] = (float)sc.alpha[4 * jq + c];
  Acc2 rz[4], rr[4];
  for (int64_t t = blockIdx.x * 256 + threadIdx.x; t < n4; t += U * S) {
    float4 pv[U], s0[U], s1[U], xv[U], rv[U];
    float d[U];
    bool in[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t tu = t + u * S;
      in[u] = false;
      s0[u] = s1[u] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (tu < n4) {
        const uint32_t fe = (uint32_t)(tu >> lg);
        const uint32_t f = fe / NF;
        const int mm = (int)(fe - f * NF);
        const int fb = face_bnd[f];
        const int2 fs = face_slot2[f];
        pv[u] = p[tu]; xv[u] = x[tu]; rv[u] = r[tu]; d[u] = dinv[fe];
        if (fb < 0) {
          in[u] = true;
          s0[u] = slot[((int64_t)fs.x * NF + mm) * R4 + jq];
          s1[u] = slot[((int64_t)fs.y * NF + mm) * R4 + jq];
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t tu = t + u * S;
      if (tu >= n4) break;
      float4 qv = make_float4(0.f, 0.f, 0.f, 0.f);
      if (in[u]) qv = make_float4(-(s0[u].x + s1[u].x), -(s0[u].y + s1[u].y), -(s0[u].z + s1[u].z), -(s0[u].w + s1[u].w));
      x[tu] = make_float4(fmaf(al[0], pv[u].x, xv[u].x), fmaf(al[1], pv[u].y, xv[u].y), fmaf(al[2], pv[u].z, xv[u].z),
                          fmaf(al[3], pv[u].w, xv[u].w));
      const float4 rn = make_float4(fmaf(-al[0], qv.x, rv[u].x), fmaf(-al[1], qv.y, rv[u].y), fmaf(-al[2], qv.z, rv[u].z),
                                    fmaf(-al[3], qv.w, rv[u].w));
      r[tu] = rn;
      rz[0].dot(rn.x, __fmul_rn(d[u], rn.x)); rr[0].dot(rn.x, rn.x);
      rz[1].dot(rn.y, __fmul_rn(d[u], rn.y)); rr[1].dot(rn.y, rn.y);
      rz[2].dot(rn.z, __fmul_rn(d[u], rn.z)); rr[2].dot(rn.z, rn.z);
      rz[3].dot(rn.w, __fmul_rn(d[u], rn.w)); rr[3].dot(rn.w, rn.w);
    }
  }
  const double vz[4] = {rz[0].value(), rz[1].value(), rz[2].value(), rz[3].value()};
  block_cols_v<4>(vz, R, red, part, blockIdx.x);
  const double vr[4] = {rr[0].value(), rr[1].value(), rr[2].value(), rr[3].value()};
  block_cols_v<4>(vr, R, red, part, (int64_t)gridDim.x + blockIdx.x);
}

// p = D^{-1} r + beta p
static __global__ void __launch_bounds__(256) mdirection4_kernel(int64_t n4, int R, const float4* __restrict__ r,
                                                                 const float* __restrict__ dinv, float4* __restrict__ p,
                                                                 const double* __restrict__ beta,
                                                                 const int* __restrict__ done) {
  constexpr int U = 4;
  if (*done) return;
  const int R4 = R >> 2, lg = __ffs(R4) - 1, jq = threadIdx.x & (R4 - 1);
  const int64_t S = (int64_t)gridDim.x * 256;
  float be[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) be[c] = (float)beta[4 * jq + c];
  for (int64_t t = blockIdx.x * 256 + threadIdx.x; t < n4; t += U * S) {
    float4 rv[U], pv[U];
    float d[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t tu = t + u * S;
      if (tu < n4) { rv[u] = r[tu]; pv[u] = p[tu]; d[u] = dinv[tu >> lg]; }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t tu = t + u * S;
      if (tu >= n4) break;
      p[tu] = make_float4(fmaf(be[0], pv[u].x, __fmul_rn(d[u], rv[u].x)), fmaf(be[1], pv[u].y, __fmul_rn(d[u], rv[u].y)),
                          fmaf(be[2], pv[u].z, __fmul_rn(d[u], rv[u].z)), fmaf(be[3], pv[u].w, __fmul_rn(d[u], rv[u].w)));
    }
  }
}

// FP64 refinement residual, two columns per thread: rho = b + sum of the two slots (interior
// entries), partials |rho|^2 and |b|^2 per column
template <int DIM, int K>
__global__ void __launch_bounds__(256) mrefine_residual2_kernel(int nf, int R, const int2* __restrict__ face_slot2,
                                                                const int32_t* __restrict__ face_bnd,
                                                                const double2* __restrict__ slot,
                                                                const double2* __restrict__ b, double2* __restrict__ res,
                                                                double* __restrict__ part) {
  constexpr int NF = Dims<DIM, K>::NF, U = 4;
  __shared__ double red[256];
  const int R2 = R >> 1, lg = __ffs(R2) - 1, jh = threadIdx.x & (R2 - 1);
  const int64_t n2 = (int64_t)nf * NF * R2, S = (int64_t)gridDim.x * 256;
  double rr[2] = {0.0, 0.0}, bb[2] = {0.0, 0.0};
  for (int64_t t = blockIdx.x * 256 + threadIdx.x; t < n2; t += U * S) {
    double2 bv[U], s0[U], s1[U];
    bool in[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t tu = t + u * S;
      in[u] = false;
      bv[u] = s0[u] = s1[u] = make_double2(0.0, 0.0);
      if (tu < n2) {
        const uint32_t fe = (uint32_t)(tu >> lg);
        const uint32_t f = fe / NF;
        const int mm = (int)(fe - f * NF);
        const int fb = face_bnd[f];
        const int2 fs = face_slot2[f];
        if (fb < 0) {
          in[u] = true;
          bv[u] = b[tu];
          s0[u] = slot[((int64_t)fs.x * NF + mm) * R2 + jh];
          s1[u] = slot[((int64_t)fs.y * NF + mm) * R2 + jh];
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t tu = t + u * S;
      if (tu >= n2) break;
      double2 v = make_double2(0.0, 0.0);
      if (in[u]) {
        v = make_double2(bv[u].x + s0[u].x + s1[u].x, bv[u].y + s0[u].y + s1[u].y);
        bb[0] += bv[u].x * bv[u].x;
        bb[1] += bv[u].y * bv[u].y;
      }
      res[tu] = v;
      rr[0] += v.x * v.x;
      rr[1] += v.y * v.y;
    }
  }
  block_cols_v<2>(rr, R, red, part, blockIdx.x);
  block_cols_v<2>(bb, R, red, part, (int64_t)gridDim.x + blockIdx.x);
}

// inner right-hand side of a sweep, four columns per thread: b32 = fl32(rho * scale_j)
static __global__ void mto32_scaled4_kernel(int64_t n4, int R, const double2* __restrict__ res,
                                            const double* __restrict__ scale, float4* __restrict__ b32) {
  const int R4 = R >> 2, jq = threadIdx.x & (R4 - 1);
  double s[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) s[c] = scale[4 * jq + c];
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n4; t += (int64_t)gridDim.x * blockDim.x) {
    const double2 a = res[2 * t], b = res[2 * t + 1];
    b32[t] = make_float4((float)(a.x * s[0]), (float)(a.y * s[1]), (float)(b.x * s[2]), (float)(b.y * s[3]));
  }
}

// lam += delta |rho|_j (|rho|_j = 1 / scale_j) on interior entries of the columns still refined
// (scale_j != 0), four columns per thread. The reciprocal is taken once per thread: an FP64
// division per entry made this kernel FP64-ALU-bound (8x its streaming time).
static __global__ void mrefine_update4_kernel(int64_t n4, int R, int NF, const int32_t* __restrict__ face_bnd,
                                              const float4* __restrict__ delta, const double* __restrict__ scale,
                                              double2* __restrict__ lam) {
  const int R4 = R >> 2, lg = __ffs(R4) - 1, jq = threadIdx.x & (R4 - 1);
  double s[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const double sc = scale[4 * jq + c];
    s[c] = sc != 0.0 ? 1.0 / sc : 0.0;
  }
  if (s[0] == 0.0 && s[1] == 0.0 && s[2] == 0.0 && s[3] == 0.0) return;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n4; t += (int64_t)gridDim.x * blockDim.x) {
    if (face_bnd[(uint32_t)(t >> lg) / (uint32_t)NF] >= 0) continue;
    const float4 d = delta[t];
    double2 a = lam[2 * t], b = lam[2 * t + 1];
    if (s[0] != 0.0) a.x += (double)d.x * s[0];
    if (s[1] != 0.0) a.y += (double)d.y * s[1];
    if (s[2] != 0.0) b.x += (double)d.z * s[2];
    if (s[3] != 0.0) b.y += (double)d.w * s[3];
    lam[2 * t] = a;
    lam[2 * t + 1] = b;
  }
}

// PCG start: r = b - (-K) x0 (x0 given; slot holds S x0 or zero), z = Dinv r, p = z; partials rz, rr, bb
template <int DIM, int K, typename TV>
__global__ void __launch_bounds__(256) minit_kernel(int nf, int R, const int32_t* __restrict__ face_slot,
                                                    const int32_t* __restrict__ face_bnd, const TV* __restrict__ slot,
                                                    const TV* __restrict__ bvec, const TV* __restrict__ dinv,
                                                    TV* __restrict__ r, TV* __restrict__ z, TV* __restrict__ p,
                                                    double* __restrict__ part) {
  constexpr int NF = Dims<DIM, K>::NF;
  __shared__ double red[256];
  MAcc<TV> rz, rr, bb;
  const int lg = __ffs(R) - 1;
  const int64_t n = (int64_t)nf * NF * R;
  for (int64_t t = blockIdx.x * 256 + threadIdx.x; t < n; t += (int64_t)gridDim.x * 256) {
    const int j = (int)(t & (R - 1));
    const uint32_t fe = (uint32_t)(t >> lg);
    const uint32_t f = fe / NF;
    const int mm = (int)(fe - f * NF);
    TV rv = TV(0), zv = TV(0);
    if (face_bnd[f] < 0) {
      TV q = TV(0);
      if (slot)
        q = -(slot[((int64_t)face_slot[2 * f] * NF + mm) * R + j] + slot[((int64_t)face_slot[2 * f + 1] * NF + mm) * R + j]);
      const TV bv = bvec[t];
      rv = bv - q;
      zv = dinv[fe] * rv;
      bb.dot(bv, bv);
    }
    r[t] = rv; z[t] = zv; p[t] = zv;
    rz.dot(rv, zv); rr.dot(rv, rv);
  }
  block_cols(rz.value(), R, red);
  if (threadIdx.x < R) part[(int64_t)blockIdx.x * R + threadIdx.x] = red[threadIdx.x];
  block_cols(rr.value(), R, red);
  if (threadIdx.x < R) part[(int64_t)(gridDim.x + blockIdx.x) * R + threadIdx.x] = red[threadIdx.x];
  block_cols(bb.value(), R, red);
  if (threadIdx.x < R) part[(int64_t)(2 * gridDim.x + blockIdx.x) * R + threadIdx.x] = red[threadIdx.x];
}

// column scalars after minit: rho0 = rz, rr, bb, tol2 = rtol^2 * (bb or rr when bb_from_rr)
// With outer_rr / outer_bb (the columns' refinement residual and right-hand side norms, the
// inner solve of a refinement sweep), a column's inner tolerance is relaxed to
// min(0.5, max(rtol, 0.25 outer_rtol / |r|/|b|)): the last sweep gains only what is left.
static __global__ void mcols_init(int nb, int R, double rtol, int tol_from_rr, const double* __restrict__ part, MScal sc,
                                  const double* __restrict__ outer_rr = nullptr,
                                  const double* __restrict__ outer_bb = nullptr, double outer_rtol = 0.0) {
  __shared__ int notconv;
  if (threadIdx.x == 0) notconv = 0;
  __syncthreads();
  __shared__ double red[256], rzs[256], rrs[256];
  col_partials(part, nb, R, 0, red);
  if (threadIdx.x < R) rzs[threadIdx.x] = red[threadIdx.x];
  col_partials(part, nb, R, nb, red);
  if (threadIdx.x < R) rrs[threadIdx.x] = red[threadIdx.x];
  col_partials(part, nb, R, 2 * (int64_t)nb, red);
  for (int j = threadIdx.x; j < R; j += blockDim.x) {
    const double rz = rzs[j], rr = rrs[j], bb = red[j];
    sc.rho0[j] = rz; sc.rho1[j] = 0.0; sc.rr[j] = rr; sc.bb[j] = bb;
    double tol = rtol;
    if (outer_rr && outer_bb[j] > 0.0 && outer_rr[j] > 0.0)
      tol = fmin(0.5, fmax(rtol, 0.25 * outer_rtol / sqrt(outer_rr[j] / outer_bb[j])));
    sc.tol2[j] = tol * tol * (tol_from_rr ? rr : bb);
    const int c = rr <= sc.tol2[j];
    sc.conv[j] = c;
    if (!c) atomicAdd(&notconv, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    *sc.done = notconv == 0 ? 1 : 0;
    *sc.iters = 0;
  }
}

// FP64 refinement (per column): rho = b + sum slots64; partial |rho|^2, |b|^2 per column
template <int DIM, int K>
__global__ void __launch_bounds__(256) mrefine_residual_kernel(int nf, int R, const int32_t* __restrict__ face_slot,
                                                               const int32_t* __restrict__ face_bnd,
                                                               const double* __restrict__ slot, const double* __restrict__ b,
                                                               double* __restrict__ res, double* __restrict__ part) {
  constexpr int NF = Dims<DIM, K>::NF;
  __shared__ double red[256];
  double rr = 0.0, bb = 0.0;
  const int lg = __ffs(R) - 1;
  const int64_t n = (int64_t)nf * NF * R;
  for (int64_t t = blockIdx.x * 256 + threadIdx.x; t < n; t += (int64_t)gridDim.x * 256) {
    const int j = (int)(t & (R - 1));
    const uint32_t fe = (uint32_t)(t >> lg);
    const uint32_t f = fe / NF;
    const int mm = (int)(fe - f * NF);
    double v = 0.0;
    if (face_bnd[f] < 0) {
      const double bv = b[t];
      v = bv + slot[((int64_t)face_slot[2 * f] * NF + mm) * R + j] + slot[((int64_t)face_slot[2 * f + 1] * NF + mm) * R + j];
      bb += bv * bv;
    }
    res[t] = v;
    rr += v * v;
  }
  block_cols(rr, R, red);
  if (threadIdx.x < R) part[(int64_t)blockIdx.x * R + threadIdx.x] = red[threadIdx.x];
  block_cols(bb, R, red);
  if (threadIdx.x < R) part[(int64_t)(gridDim.x + blockIdx.x) * R + threadIdx.x] = red[threadIdx.x];
}

// per column: rr, bb, scale = 1/|rho| (0 -> column converged: its inner right-hand side is zero)
static __global__ void mrefine_scalars(int nb, int R, double rtol, const double* __restrict__ part, double* __restrict__ rr,
                                double* __restrict__ bb, double* __restrict__ scale, int* __restrict__ nconv) {
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  __shared__ double red[256], as[256];
  col_partials(part, nb, R, 0, red);
  if (threadIdx.x < R) as[threadIdx.x] = red[threadIdx.x];
  col_partials(part, nb, R, nb, red);
  for (int j = threadIdx.x; j < R; j += blockDim.x) {
    const double a = as[j], c = red[j];
    rr[j] = a; bb[j] = c;
    const bool ok = a <= rtol * rtol * c;
    scale[j] = (ok || a == 0.0) ? 0.0 : 1.0 / sqrt(a);
    if (!ok) atomicAdd(&cnt, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) *nconv = cnt;
}

static __global__ void mto32_scaled_kernel(int64_t n, int R, const double* __restrict__ res, const double* __restrict__ scale,
                                    float* __restrict__ b32) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    b32[t] = (float)(res[t] * scale[t & (R - 1)]);
}

static __global__ void mrefine_update_kernel(int64_t n, int R, int NF, const int32_t* __restrict__ face_bnd,
                                      const float* __restrict__ delta, const double* __restrict__ scale,
                                      double* __restrict__ lam) {
  // the grid stride (a multiple of 256) is a multiple of R: a thread keeps its column j
  const int lg = __ffs(R) - 1;
  const double sc = scale[(blockIdx.x * (int64_t)blockDim.x + threadIdx.x) & (R - 1)];
  if (sc == 0.0) return;
  const double inv = 1.0 / sc;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    if (face_bnd[(uint32_t)(t >> lg) / (uint32_t)NF] < 0) lam[t] += (double)delta[t] * inv;
}

// boundary entries of lam (all columns) <- coef[b] * fac
static __global__ void mdirichlet_kernel(int64_t nb, int NF, int R, const int64_t* __restrict__ bnd_faces,
                                  const double* __restrict__ coef, double fac, double* __restrict__ lam) {
  const int64_t n = nb * NF * R;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t bf = t / R;
    const int64_t b = bf / NF;
    lam[(bnd_faces[b] * NF + bf % NF) * R + t % R] = coef ? coef[bf] * fac : 0.0;
  }
}

// faces from slots (all columns): out = scale * (slot0 + slot1) on interior faces, 0 on boundary
template <int DIM, int K>
__global__ void mface_gather_kernel(int nf, int R, const int32_t* __restrict__ face_slot,
                                    const int32_t* __restrict__ face_bnd, const double* __restrict__ slot, double scale,
                                    double* __restrict__ out) {
  constexpr int NF = Dims<DIM, K>::NF;
  const int lg = __ffs(R) - 1;
  const int64_t n = (int64_t)nf * NF * R;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(t & (R - 1));
    const uint32_t fe = (uint32_t)(t >> lg);
    const uint32_t f = fe / NF;
    const int mm = (int)(fe - f * NF);
    double v = 0.0;
    if (face_bnd[f] < 0)
      v = scale * (slot[((int64_t)face_slot[2 * f] * NF + mm) * R + j] + slot[((int64_t)face_slot[2 * f + 1] * NF + mm) * R + j]);
    out[t] = v;
  }
}

// interior entries (all columns) <- 0
static __global__ void mzero_interior_kernel(int64_t n, int R, int NF, const int32_t* __restrict__ face_bnd,
                                      double* __restrict__ x) {
  const int lg = __ffs(R) - 1;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    if (face_bnd[(uint32_t)(t >> lg) / (uint32_t)NF] < 0) x[t] = 0.0;
}

// volume projection replicated over R columns: u[e][c*NP+i][j] = sum_q w_q vals[e][q][c] phi_i(xi_q)
static __global__ void mproject_volume_kernel(int64_t ne, int NP, int nq, int ncomp, int R, const double* __restrict__ w,
                                       const double* __restrict__ phi, const double* __restrict__ vals,
                                       double* __restrict__ u) {
  const int64_t n = ne * ncomp * NP * R;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = t / R;
    const int64_t e = row / (ncomp * NP);
    const int c = (int)((row / NP) % ncomp), i = (int)(row % NP);
    double s = 0.0;
    for (int q = 0; q < nq; ++q) s += w[q] * vals[(e * nq + q) * ncomp + c] * phi[q * NP + i];
    u[t] = s;
  }
}

}  // namespace hdg

namespace hdg {
// column j of an [count][R] array <- 0
static __global__ void zero_column_kernel(int64_t count, int R, int j, double* __restrict__ a) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x)
    a[t * R + j] = 0.0;
}
}  // namespace hdg
