// Variable-degree elastodynamics (per-element k_K, face degree k_F = max over the face's
// elements) on the GPU: the scheme of elastic.cuh with the spaces of Sec. 2.2 chosen per
// element and per face.
//
// Elements are grouped in classes (K, KT): volume degree K and KT = the largest degree of
// the element's faces. A class computes with the face tables of degree KT ("padded" local
// trace layout [face][component][N_f(KT) modes]); a face of lower degree k_F uses only the
// modes of total degree <= k_F, which are a subset of the degree-KT modes (the Dubiner
// functions do not depend on the maximal degree). Restricting S_K = D - C A^{-1} B to those
// rows and columns is exactly the Schur complement of the smaller trace space, so each
// element stores the compact active block (m_e x m_e) and the matrix-free apply, the face
// sums and the Krylov vectors work on compact indices:
//   gidx[m_off[e] + a]  global trace entry of compact local entry a (all faces),
//   gint[...]           the same, -1 on boundary faces (the applies skip them),
//   pidx[...]           padded local index (class layout) of compact entry a,
//   dslot[2 d + s]      the two slot positions summed into trace entry d (-1: boundary).
#pragma once
#include "elastic.cuh"

namespace hdg {

template <int DIM, int K, int KT>
struct VdDims {
  static constexpr int NP = Dims<DIM, K>::NP;
  static constexpr int NFP = Dims<DIM, KT>::NF;   // scalar face modes of the padded layout
  static constexpr int NF = DIM * NFP;
  static constexpr int NFC = DIM + 1;
  static constexpr int NT = DIM * (DIM + 1) / 2;
  static constexpr int NV = DIM * NP;
  static constexpr int N = (DIM + NT) * NP;
  static constexpr int M = NFC * NF;
  static constexpr int OJF = 1 + DIM * DIM;
  static constexpr int ON = 1 + DIM * DIM + DIM + 1;
};

struct VdIndex {
  const int32_t* elist;   // elements of the class
  const int64_t* u_off;   // [ne + 1] field offsets
  const int64_t* h_off;   // [ne + 1] H^{-1} offsets
  const int64_t* s_off;   // [ne + 1] S_K offsets
  const int32_t* m_off;   // [ne + 1] compact trace offsets
  const int32_t* gidx;
  const int16_t* pidx;
};

// H and L^{-1} stay in shared memory unless the class is too large for it; then they live
// in a per-block global scratch (L2-resident), and W alone uses shared memory.
template <int DIM, int K, int KT>
struct CondVdCfg {
  using D = VdDims<DIM, K, KT>;
  static constexpr size_t FULL = sizeof(double) * ((size_t)2 * D::NV * D::NV + (size_t)D::NV * D::M);
  static constexpr bool GH = FULL > (size_t)200 * 1024;
  static constexpr size_t SMEM = GH ? sizeof(double) * (size_t)D::NV * D::M : FULL;
  static constexpr size_t SCR = GH ? (size_t)2 * D::NV * D::NV : 0;   // doubles per block
};

template <int DIM, int K, int KT>
__global__ void __launch_bounds__(256) condense_vd_kernel(DevMesh mesh, Tabs T, const double* __restrict__ lamv,
                                                           const double* __restrict__ muv, double alpha, VdIndex X,
                                                           double* __restrict__ S, double* __restrict__ Hinv,
                                                           double* __restrict__ scratch, int* __restrict__ err) {
  using D = VdDims<DIM, K, KT>;
  using C = CondVdCfg<DIM, K, KT>;
  constexpr int NP = D::NP, NFP = D::NFP, NF = D::NF, NFC = D::NFC, NT = D::NT, NV = D::NV, M = D::M;
  constexpr int NTH = 256;
  extern __shared__ double dyn[];
  double* H = C::GH ? scratch + (size_t)blockIdx.x * C::SCR : dyn;
  double* Li = H + NV * NV;
  double* W = C::GH ? dyn : Li + NV * NV;
  __shared__ double g[GEO_STRIDE];
  __shared__ double Xi[DIM * DIM * DIM * DIM];
  __shared__ double Psi[DIM * DIM * NFC * DIM];
  __shared__ double Phi[NFC * DIM * NFC * DIM];
  const int64_t e = X.elist[blockIdx.x];
  const int tid = threadIdx.x;
  if (tid < GEO_STRIDE) g[tid] = mesh.geo[e * GEO_STRIDE + tid];
  __syncthreads();
  const double dJ = g[0];
  const double rho = mesh.rho[e], lam = lamv[e], mu = muv[e];
  const double s = 2.0 * sqrt(rho * mu);
  for (int t = tid; t < DIM * DIM * DIM * DIM + DIM * DIM * NFC * DIM + NFC * DIM * NFC * DIM; t += NTH) {
    double v = 0.0;
    if (t < DIM * DIM * DIM * DIM) {
      const int i = t / (DIM * DIM * DIM), j = (t / (DIM * DIM)) % DIM, r = (t / DIM) % DIM, s2 = t % DIM;
      for (int a = 0; a < NT; ++a) {
        const int q = qa<DIM>(a, i);
        if (q < 0) continue;
        for (int b = 0; b < NT; ++b) {
          const int q2 = qa<DIM>(b, j);
          if (q2 < 0) continue;
          v += cm_entry<DIM>(a, b, lam, mu) * g[1 + r * DIM + q] * g[1 + s2 * DIM + q2];
        }
      }
      Xi[t] = v;
    } else if (t < DIM * DIM * DIM * DIM + DIM * DIM * NFC * DIM) {
      const int u = t - DIM * DIM * DIM * DIM;
      const int i = u / (DIM * NFC * DIM), p = (u / (NFC * DIM)) % DIM, f = (u / DIM) % NFC, r = u % DIM;
      for (int a = 0; a < NT; ++a) {
        const int q = qa<DIM>(a, i);
        if (q < 0) continue;
        for (int b = 0; b < NT; ++b) {
          const int q2 = qa<DIM>(b, p);
          if (q2 < 0) continue;
          v += cm_entry<DIM>(a, b, lam, mu) * g[1 + r * DIM + q] * g[D::ON + f * DIM + q2];
        }
      }
      Psi[u] = v;
    } else {
      const int u = t - DIM * DIM * DIM * DIM - DIM * DIM * NFC * DIM;
      const int f = u / (DIM * NFC * DIM), p = (u / (NFC * DIM)) % DIM, gg = (u / DIM) % NFC, p2 = u % DIM;
      for (int a = 0; a < NT; ++a) {
        const int q = qa<DIM>(a, p);
        if (q < 0) continue;
        for (int b = 0; b < NT; ++b) {
          const int q2 = qa<DIM>(b, p2);
          if (q2 < 0) continue;
          v += cm_entry<DIM>(a, b, lam, mu) * g[D::ON + f * DIM + q] * g[D::ON + gg * DIM + q2];
        }
      }
      Phi[u] = v;
    }
  }
  __syncthreads();
  for (int idx = tid; idx < NV * NV; idx += NTH) {
    const int row = idx / NV, col = idx % NV;
    const int i = row / NP, l = row % NP, j = col / NP, m = col % NP;
    double v = 0.0;
    for (int rs = 0; rs < DIM * DIM; ++rs) v += Xi[(i * DIM + j) * DIM * DIM + rs] * T.Trs[(rs * NP + l) * NP + m];
    v *= dJ / alpha;
    if (i == j) {
      double fe = 0.0;
      for (int f = 0; f < NFC; ++f) fe += g[D::OJF + f] * T.Ef[(f * NP + l) * NP + m];
      v += s * fe + (l == m ? alpha * rho * dJ : 0.0);
    }
    H[idx] = v;
    Li[idx] = row == col ? 1.0 : 0.0;
  }
  for (int idx = tid; idx < NV * M; idx += NTH) {
    const int row = idx / M, col = idx % M;
    const int i = row / NP, l = row % NP;
    const int f = col / NF, p = (col % NF) / NFP, mm = col % NFP;
    double v = 0.0;
    for (int r = 0; r < DIM; ++r) v += Psi[((i * DIM + p) * NFC + f) * DIM + r] * T.DFrf[((r * NFC + f) * NP + l) * NFP + mm];
    v = -(g[D::OJF + f] / alpha) * v;
    if (i == p) v -= s * g[D::OJF + f] * T.Ff[(f * NP + l) * NFP + mm];
    W[idx] = v;
  }
  __syncthreads();
  for (int j = 0; j < NV; ++j) {
    if (tid == 0) {
      double d = H[j * NV + j];
      if (!(d > 0.0)) { atomicExch(err, 1); d = 1.0; }
      H[j * NV + j] = sqrt(d);
    }
    __syncthreads();
    for (int i = j + 1 + tid; i < NV; i += NTH) H[i * NV + j] /= H[j * NV + j];
    __syncthreads();
    const int w = NV - j - 1;
    for (int idx = tid; idx < w * w; idx += NTH) {
      const int i = j + 1 + idx / w, l = j + 1 + idx % w;
      if (l <= i) H[i * NV + l] -= H[i * NV + j] * H[l * NV + j];
    }
    __syncthreads();
  }
  for (int col = tid; col < M + NV; col += NTH) {
    if (col < M) {
      for (int i = 0; i < NV; ++i) {
        double sacc = W[i * M + col];
        for (int l = 0; l < i; ++l) sacc -= H[i * NV + l] * W[l * M + col];
        W[i * M + col] = sacc / H[i * NV + i];
      }
    } else {
      const int c2 = col - M;
      for (int i = c2; i < NV; ++i) {
        double sacc = (i == c2) ? 1.0 : 0.0;
        for (int l = c2; l < i; ++l) sacc -= H[i * NV + l] * Li[l * NV + c2];
        Li[i * NV + c2] = sacc / H[i * NV + i];
      }
    }
  }
  __syncthreads();
  // compact active block of S_K
  const int m0 = X.m_off[e], me = X.m_off[e + 1] - m0;
  const int16_t* pi = X.pidx + m0;
  double* Se = S + X.s_off[e];
  const double ia = 1.0 / (alpha * dJ);
  for (int idx = tid; idx < me * me; idx += NTH) {
    const int c1 = pi[idx / me], c2 = pi[idx % me];
    const int f = c1 / NF, p = (c1 % NF) / NFP, a1 = c1 % NFP;
    const int gg = c2 / NF, p2 = (c2 % NF) / NFP, b1 = c2 % NFP;
    double v = 0.0;
    for (int i = 0; i < NV; ++i) v -= W[i * M + c1] * W[i * M + c2];
    v += ia * g[D::OJF + f] * g[D::OJF + gg] * Phi[((f * DIM + p) * NFC + gg) * DIM + p2] *
         T.Pfg[((f * NFC + gg) * NFP + a1) * NFP + b1];
    if (c1 == c2) v += s * g[D::OJF + f];
    Se[idx] = v;
  }
  double* He = Hinv + X.h_off[e];
  for (int idx = tid; idx < NV * NV; idx += NTH) {
    const int i = idx / NV, l = idx % NV;
    const int q0 = i > l ? i : l;
    double sacc = 0.0;
    for (int q = q0; q < NV; ++q) sacc += Li[q * NV + i] * Li[q * NV + l];
    He[idx] = sacc;
  }
}

// Shared workspace of one element of class (K, KT) in the local solves (offsets in doubles).
template <int DIM, int K, int KT>
struct LocalVdSmem {
  using D = VdDims<DIM, K, KT>;
  static constexpr int G = 0, LL = G + GEO_STRIDE, FL = LL + D::M, RV = FL + D::NFC * DIM * D::NP,
                       RS = RV + D::NV, Y = RS + D::NT * D::NP, TT = Y + D::NT * D::NP,
                       RHS = TT + DIM * DIM * D::NP, V = RHS + D::NV, Z = V + D::NV, W = Z + DIM * DIM * D::NP,
                       SG = W + D::NT * D::NP, CM = SG + D::NT * D::NP, QM = CM + D::NT * D::NT,
                       FUSE = QM + D::NT * D::NT, TOTAL = FUSE + 4;
};

// Element-local solves of one element of class (K, KT), NTH threads. MODE 0:
// out[m_off[e] + a] = (C_K A_K^{-1}(F_K - B_K lamD_K)) at the compact entries; MODE 1:
// out[u_off[e] ..] = A_K^{-1}(F_K - B_K lam_K). F_K = F[u_off[e] ..] or alpha Mw_K hist[u_off[e] ..].
template <int DIM, int K, int KT, int MODE, int NTH>
__device__ __forceinline__ void local_vd_body(const DevMesh& mesh, const Tabs& T, const double* __restrict__ lamv,
                                              const double* __restrict__ muv, const double* __restrict__ Hinv,
                                              double alpha, const VdIndex& X, int64_t e, const double* __restrict__ F,
                                              const double* __restrict__ hist, const double* __restrict__ lamt,
                                              double* __restrict__ out, double* sm) {
  using D = VdDims<DIM, K, KT>;
  using SM = LocalVdSmem<DIM, K, KT>;
  constexpr int NP = D::NP, NFP = D::NFP, NF = D::NF, NFC = D::NFC, NT = D::NT, NV = D::NV, M = D::M, N = D::N;
  double* g = sm + SM::G;
  double* ll = sm + SM::LL;
  double* Fl = sm + SM::FL;
  double *rv = sm + SM::RV, *rs = sm + SM::RS, *y = sm + SM::Y, *tt = sm + SM::TT, *rhs = sm + SM::RHS,
         *v = sm + SM::V, *z = sm + SM::Z, *w = sm + SM::W, *sg = sm + SM::SG, *Cm = sm + SM::CM, *Qm = sm + SM::QM;
  int* fuse = reinterpret_cast<int*>(sm + SM::FUSE);
  const int tid = threadIdx.x;
  const double rho = mesh.rho[e], lam = lamv[e], mu = muv[e];
  const double s = 2.0 * sqrt(rho * mu);
  const int64_t u0 = X.u_off[e];
  const int m0 = X.m_off[e], me = X.m_off[e + 1] - m0;
  if (tid < GEO_STRIDE) g[tid] = mesh.geo[e * GEO_STRIDE + tid];
  if (tid < NFC) {
    int use = 0;
    if (lamt) {
      const int f = mesh.elem_face[e * NFC + tid];
      use = (MODE == 1) || (mesh.face_bnd[f] >= 0);
    }
    fuse[tid] = use;
  }
  for (int t = tid; t < NT * NT; t += NTH) {
    Cm[t] = cm_entry<DIM>(t / NT, t % NT, lam, mu);
    Qm[t] = q_entry<DIM>(t / NT, t % NT, lam, mu);
  }
  for (int t = tid; t < M; t += NTH) ll[t] = 0.0;
  __syncthreads();
  for (int a = tid; a < me; a += NTH) {
    const int pc = X.pidx[m0 + a];
    if (fuse[pc / NF]) ll[pc] = lamt[X.gidx[m0 + a]];
  }
  __syncthreads();
  const double dJ = g[0];
  for (int t = tid; t < NFC * DIM * NP; t += NTH) {
    const int f = t / (DIM * NP), p = (t / NP) % DIM, l = t % NP;
    double acc = 0.0;
    if (fuse[f])
      for (int mm = 0; mm < NFP; ++mm) acc += T.Ff[(f * NP + l) * NFP + mm] * ll[f * NF + p * NFP + mm];
    Fl[t] = acc;
  }
  __syncthreads();
  for (int t = tid; t < N; t += NTH) {
    const int comp = t / NP, l = t % NP;
    if (comp < DIM) {
      double val = hist ? alpha * rho * dJ * hist[u0 + t] : F[u0 + t];
      double bl = 0.0;
      for (int f = 0; f < NFC; ++f) bl += g[D::OJF + f] * Fl[(f * DIM + comp) * NP + l];
      rv[t] = val + s * bl;
    } else {
      const int a = comp - DIM;
      double val;
      if (hist) {
        val = 0.0;
        for (int b = 0; b < NT; ++b) val += Qm[a * NT + b] * hist[u0 + (DIM + b) * NP + l];
        val *= alpha * dJ;
      } else {
        val = F[u0 + t];
      }
      int ai, aj;
      sym_ij<DIM>(a, ai, aj);
      double bl = 0.0;
      for (int f = 0; f < NFC; ++f) {
        bl += g[D::ON + f * DIM + aj] * g[D::OJF + f] * Fl[(f * DIM + ai) * NP + l];
        if (ai != aj) bl += g[D::ON + f * DIM + ai] * g[D::OJF + f] * Fl[(f * DIM + aj) * NP + l];
      }
      rs[a * NP + l] = val + bl;
    }
  }
  __syncthreads();
  for (int t = tid; t < NT * NP; t += NTH) {
    const int a = t / NP, l = t % NP;
    double acc = 0.0;
    for (int b = 0; b < NT; ++b) acc += Cm[a * NT + b] * rs[b * NP + l];
    y[t] = acc;
  }
  __syncthreads();
  for (int t = tid; t < DIM * DIM * NP; t += NTH) {
    const int i = t / (DIM * NP), r = (t / NP) % DIM, l = t % NP;
    double acc = 0.0;
    for (int a = 0; a < NT; ++a) {
      const int q = qa<DIM>(a, i);
      if (q >= 0) acc += g[1 + r * DIM + q] * y[a * NP + l];
    }
    tt[t] = acc;
  }
  __syncthreads();
  for (int t = tid; t < NV; t += NTH) {
    const int i = t / NP, l = t % NP;
    double acc = 0.0;
    for (int r = 0; r < DIM; ++r)
      for (int m = 0; m < NP; ++m) acc += T.Dr[(r * NP + l) * NP + m] * tt[(i * DIM + r) * NP + m];
    rhs[t] = rv[t] + acc / alpha;
  }
  __syncthreads();
  const double* He = Hinv + X.h_off[e];
  for (int t = tid; t < NV; t += NTH) {
    double acc = 0.0;
    for (int l = 0; l < NV; ++l) acc += He[l * NV + t] * rhs[l];
    v[t] = acc;
  }
  __syncthreads();
  for (int t = tid; t < DIM * DIM * NP; t += NTH) {
    const int r = t / (DIM * NP), p = (t / NP) % DIM, l = t % NP;
    double acc = 0.0;
    for (int m = 0; m < NP; ++m) acc += T.Dr[(r * NP + m) * NP + l] * v[p * NP + m];
    z[t] = acc;
  }
  __syncthreads();
  for (int t = tid; t < NT * NP; t += NTH) {
    const int b = t / NP, l = t % NP;
    double acc = 0.0;
    for (int p = 0; p < DIM; ++p) {
      const int q = qa<DIM>(b, p);
      if (q < 0) continue;
      for (int r = 0; r < DIM; ++r) acc += g[1 + r * DIM + q] * z[(r * DIM + p) * NP + l];
    }
    w[t] = acc;
  }
  __syncthreads();
  for (int t = tid; t < NT * NP; t += NTH) {
    const int a = t / NP, l = t % NP;
    double acc = 0.0;
    for (int b = 0; b < NT; ++b) acc += Cm[a * NT + b] * w[b * NP + l];
    sg[t] = y[t] / (alpha * dJ) - acc / alpha;
  }
  __syncthreads();
  if (MODE == 1) {
    for (int t = tid; t < N; t += NTH) out[u0 + t] = t < NV ? v[t] : sg[t - NV];
    return;
  }
  for (int t = tid; t < NFC * DIM * NP; t += NTH) {
    const int f = t / (DIM * NP), i = (t / NP) % DIM, l = t % NP;
    double acc = -s * v[i * NP + l];
    for (int j = 0; j < DIM; ++j) acc += g[D::ON + f * DIM + j] * sg[sym_index<DIM>(i, j) * NP + l];
    Fl[t] = acc;
  }
  __syncthreads();
  for (int a = tid; a < me; a += NTH) {
    const int t = X.pidx[m0 + a];
    const int f = t / NF, i = (t % NF) / NFP, mm = t % NFP;
    double acc = 0.0;
    for (int l = 0; l < NP; ++l) acc += T.Ff[(f * NP + l) * NFP + mm] * Fl[(f * DIM + i) * NP + l];
    out[m0 + a] = g[D::OJF + f] * acc;
  }
}

// All classes of a variable-degree mesh in one launch: block b handles element elist[b]; the
// element list is grouped by class, heaviest classes first, and the class ranges are
// [start[c], start[c + 1]). The shared workspace is the largest class's (dynamic).
struct VdClassTable {
  int n;
  int64_t start[11];
  int key[10];     // 10 K + KT
  Tabs tabs[10];
};

template <int MODE, int NTH>
__global__ void __launch_bounds__(NTH) local_vd_all_kernel(DevMesh mesh, VdClassTable C, const double* __restrict__ lamv,
                                                           const double* __restrict__ muv,
                                                           const double* __restrict__ Hinv, double alpha, VdIndex X,
                                                           const double* __restrict__ F, const double* __restrict__ hist,
                                                           const double* __restrict__ lamt, double* __restrict__ out) {
  extern __shared__ double sm[];
  const int64_t b = blockIdx.x;
  int c = 0;
  while (c + 1 < C.n && b >= C.start[c + 1]) ++c;
  const int64_t e = X.elist[b];
#define HDG_VD_BODY(KK, KKT)                                                                                      \
  case KK * 10 + KKT:                                                                                             \
    local_vd_body<3, KK, KKT, MODE, NTH>(mesh, C.tabs[c], lamv, muv, Hinv, alpha, X, e, F, hist, lamt, out, sm); \
    break;
  switch (C.key[c]) {
    HDG_VD_BODY(4, 4)
    HDG_VD_BODY(3, 4)
    HDG_VD_BODY(3, 3)
    HDG_VD_BODY(2, 4)
    HDG_VD_BODY(2, 3)
    HDG_VD_BODY(2, 2)
    HDG_VD_BODY(1, 4)
    HDG_VD_BODY(1, 3)
    HDG_VD_BODY(1, 2)
    HDG_VD_BODY(1, 1)
    default: break;
  }
#undef HDG_VD_BODY
}

// slot[m_off[e] + r] = sum_c S_e[r][c] x[gint[m_off[e] + c]] (boundary entries read as 0).
// Warp per element, WPB warps per block, lane handles rows lane + 32 q; S_e is symmetric, so
// column r is read as row r (coalesced); UNR columns are in flight per step. MMAX bounds m_e.
// (WPB, UNR) is the tile the autotuner picks per context.
__device__ __forceinline__ double vd_val(double s) { return s; }
__device__ __forceinline__ float vd_val(float s) { return s; }
__device__ __forceinline__ float vd_val(__half s) { return __half2float(s); }

// ST: storage type of S_K (double, float, or __half with a per-element scale sc[e]).
template <typename TV, typename ST, int MMAX, int WPB, int UNR>
__global__ void __launch_bounds__(32 * WPB) apply_vd_kernel(int64_t ne, const int64_t* __restrict__ s_off,
                                                            const int32_t* __restrict__ m_off,
                                                            const int32_t* __restrict__ gint, const ST* __restrict__ S,
                                                            const float* __restrict__ sc, const TV* __restrict__ x,
                                                            TV* __restrict__ slot, const int* __restrict__ done) {
  constexpr int RPL = (MMAX + 31) / 32;
  __shared__ TV lx[WPB][MMAX];
  if (done && *done) return;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t e = (int64_t)blockIdx.x * WPB + w;
  if (e >= ne) return;
  const int m0 = m_off[e], me = m_off[e + 1] - m0;
  for (int c = lane; c < me; c += 32) {
    const int gi = gint[m0 + c];
    lx[w][c] = gi >= 0 ? x[gi] : TV(0);
  }
  __syncwarp();
  TV acc[RPL];
#pragma unroll
  for (int q = 0; q < RPL; ++q) acc[q] = TV(0);
  const ST* Se = S + s_off[e];
#pragma unroll UNR
  for (int c = 0; c < me; ++c) {
    const TV xc = lx[w][c];
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
      const int r = lane + 32 * q;
      if (r < me) acc[q] += (TV)vd_val(__ldcs(Se + (int64_t)c * me + r)) * xc;
    }
  }
  const TV scl = sc ? (TV)sc[e] : TV(1);
#pragma unroll
  for (int q = 0; q < RPL; ++q) {
    const int r = lane + 32 * q;
    if (r < me) slot[m0 + r] = scl * acc[q];
  }
}

// FP16 copy of the compact S_K blocks with one scale per element (max |S_K|, rounded up so
// every stored value lies in [-1, 1]). Warp per element.
static __global__ void pack16_vd_kernel(int64_t ne, const int64_t* __restrict__ s_off, const double* __restrict__ S,
                                        float* __restrict__ sc, __half* __restrict__ S16) {
  const int lane = threadIdx.x & 31;
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t e = w; e < ne; e += nw) {
    const int64_t a = s_off[e], b = s_off[e + 1];
    double m = 0.0;
    for (int64_t t = a + lane; t < b; t += 32) m = fmax(m, fabs(S[t]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    const float s = m > 0.0 ? __double2float_ru(m) : 1.f;
    if (lane == 0) sc[e] = s;
    for (int64_t t = a + lane; t < b; t += 32) S16[t] = __float2half_rn((float)(S[t] / (double)s));
  }
}

// FP64-accurate refinement apply on the FP32 pipe: S_e = hi + lo (hi = the FP32 copy, lo =
// fl32(S - hi)), x split into double-floats, compensated accumulation (same tile structure as
// apply_vd_kernel; the FP64 slot is written).
template <int MMAX, int WPB, int UNR>
__global__ void __launch_bounds__(32 * WPB) apply_vd_df_kernel(int64_t ne, const int64_t* __restrict__ s_off,
                                                               const int32_t* __restrict__ m_off,
                                                               const int32_t* __restrict__ gint,
                                                               const float* __restrict__ Shi,
                                                               const float* __restrict__ Slo,
                                                               const double* __restrict__ x, double* __restrict__ slot) {
  constexpr int RPL = (MMAX + 31) / 32;
  __shared__ df2 lx[WPB][MMAX];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t e = (int64_t)blockIdx.x * WPB + w;
  if (e >= ne) return;
  const int m0 = m_off[e], me = m_off[e + 1] - m0;
  for (int c = lane; c < me; c += 32) {
    const int gi = gint[m0 + c];
    lx[w][c] = df_from(gi >= 0 ? x[gi] : 0.0);
  }
  __syncwarp();
  DfAcc acc[RPL];
  const int64_t so = s_off[e];
#pragma unroll UNR
  for (int c = 0; c < me; ++c) {
    const df2 xc = lx[w][c];
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
      const int r = lane + 32 * q;
      if (r < me) {
        const int64_t o = so + (int64_t)c * me + r;
        acc[q].fma(df2{__ldcs(Shi + o), __ldcs(Slo + o)}, xc);
      }
    }
  }
#pragma unroll
  for (int q = 0; q < RPL; ++q) {
    const int r = lane + 32 * q;
    if (r < me) slot[m0 + r] = acc[q].value();
  }
}

// lo = fl32(S - hi): the part of each FP64 entry that its FP32 copy does not hold
static __global__ void lo32_kernel(int64_t n, const double* __restrict__ S, const float* __restrict__ hi,
                                   float* __restrict__ lo) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    lo[t] = __double2float_rn(S[t] - (double)hi[t]);
}

// L2 projection of point values at each element's own volume rule (degree k_K, (k_K + 2)^3
// points): u_K[c][i] = sum_q w_q vals[q][c] phi_i(xi_q) (orthonormal basis: the mass |J| I
// cancels |J| in the load). Block per element; tables per degree at qw[k], qphi[k].
struct VdQuad {
  const double* qw[5];
  const double* qphi[5];
  int nq[5], np[5];
};

static __global__ void project_vd_kernel(int64_t ne, int ncomp, const int32_t* __restrict__ ek,
                                         const int64_t* __restrict__ q_off, const int64_t* __restrict__ u_off,
                                         VdQuad Q, const double* __restrict__ vals, double* __restrict__ u) {
  for (int64_t e = blockIdx.x; e < ne; e += gridDim.x) {
    const int k = ek[e], nq = Q.nq[k], np = Q.np[k];
    const double* w = Q.qw[k];
    const double* phi = Q.qphi[k];
    const double* v = vals + q_off[e] * ncomp;
    for (int t = threadIdx.x; t < ncomp * np; t += blockDim.x) {
      const int c = t / np, i = t % np;
      double s = 0.0;
      for (int q = 0; q < nq; ++q) s += w[q] * v[q * ncomp + c] * phi[q * np + i];
      u[u_off[e] + t] = s;
    }
  }
}

// ---- trace-entry passes through the slot map (generic over the per-face size)
template <typename TV>
__device__ __forceinline__ TV vd_sum(const int32_t* __restrict__ dslot, const TV* __restrict__ slot, int64_t d) {
  return slot[dslot[2 * d]] + slot[dslot[2 * d + 1]];
}

static __global__ void vd_face_gather_kernel(int64_t n, const int32_t* __restrict__ dslot, const double* __restrict__ slot,
                                      double scale, double* __restrict__ out) {
  for (int64_t d = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; d < n; d += (int64_t)gridDim.x * blockDim.x)
    out[d] = dslot[2 * d] >= 0 ? scale * vd_sum(dslot, slot, d) : 0.0;
}

static __global__ void vd_cg_init_kernel(int64_t n, double sgn, const int32_t* __restrict__ dslot,
                                  const double* __restrict__ slot, const double* __restrict__ bvec,
                                  const double* __restrict__ dinv, double* __restrict__ r, double* __restrict__ z,
                                  double* __restrict__ p, double* __restrict__ part) {
  __shared__ double red[8];
  double rz = 0, rr = 0, bb = 0;
  for (int64_t d = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; d < n; d += (int64_t)gridDim.x * blockDim.x) {
    double rv = 0, zv = 0;
    if (dslot[2 * d] >= 0) {
      const double bv = bvec[d];
      rv = bv - sgn * vd_sum(dslot, slot, d);
      zv = dinv[d] * rv;
      bb += bv * bv;
    }
    r[d] = rv; z[d] = zv; p[d] = zv;
    rz += rv * zv; rr += rv * rv;
  }
  double s;
  s = block_sum256(rz, red); if (threadIdx.x == 0) part[blockIdx.x * 3 + 0] = s;
  s = block_sum256(rr, red); if (threadIdx.x == 0) part[blockIdx.x * 3 + 1] = s;
  s = block_sum256(bb, red); if (threadIdx.x == 0) part[blockIdx.x * 3 + 2] = s;
}

// q = sgn K p through the slots; partial p.q (FP64, or compensated FP32 for float vectors)
template <typename TV>
__global__ void __launch_bounds__(256) vd_face_q_kernel(int64_t n, TV sgn, const int32_t* __restrict__ dslot,
                                                        const TV* __restrict__ slot, const TV* __restrict__ p,
                                                        TV* __restrict__ q, double* __restrict__ part,
                                                        const CgScal* __restrict__ sc) {
  if (sc->done) return;
  __shared__ double red[8];
  double pq = 0.0;
  Acc2 pq32;
  for (int64_t d = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; d < n; d += (int64_t)gridDim.x * blockDim.x) {
    const TV qv = dslot[2 * d] >= 0 ? sgn * vd_sum(dslot, slot, d) : TV(0);
    q[d] = qv;
    if (sizeof(TV) == 8) pq += (double)p[d] * (double)qv;
    else pq32.dot((float)p[d], (float)qv);
  }
  const double s = block_sum256(sizeof(TV) == 8 ? pq : pq32.value(), red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

static __global__ void vd_refine_residual_kernel(int64_t n, double sgn, const int32_t* __restrict__ dslot,
                                          const double* __restrict__ slot, const double* __restrict__ b,
                                          double* __restrict__ rho, double* __restrict__ part) {
  __shared__ double red[8];
  double rr = 0, bb = 0;
  for (int64_t d = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; d < n; d += (int64_t)gridDim.x * blockDim.x) {
    double v = 0.0;
    if (dslot[2 * d] >= 0) {
      const double bv = b[d];
      v = bv - sgn * vd_sum(dslot, slot, d);
      bb += bv * bv;
    }
    rho[d] = v;
    rr += v * v;
  }
  double s;
  s = block_sum256(rr, red); if (threadIdx.x == 0) part[blockIdx.x * 2 + 0] = s;
  s = block_sum256(bb, red); if (threadIdx.x == 0) part[blockIdx.x * 2 + 1] = s;
}

static __global__ void vd_refine_update_kernel(int64_t n, const int32_t* __restrict__ dslot, const float* __restrict__ delta,
                                        const RefScal* __restrict__ rs, double* __restrict__ lam) {
  const double inv = 1.0 / rs->scale;
  for (int64_t d = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; d < n; d += (int64_t)gridDim.x * blockDim.x)
    if (dslot[2 * d] >= 0) lam[d] += (double)delta[d] * inv;
}

static __global__ void vd_zero_interior_kernel(int64_t n, const int32_t* __restrict__ dslot, double* __restrict__ x) {
  for (int64_t d = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; d < n; d += (int64_t)gridDim.x * blockDim.x)
    if (dslot[2 * d] >= 0) x[d] = 0.0;
}

// Jacobi: dinv[d] = sgn / (sum of the two slots' diagonal entries of S_K); sdiag[slot] is
// the offset of that diagonal entry in S.
static __global__ void vd_diag_kernel(int64_t n, double sgn, const int32_t* __restrict__ dslot,
                               const int64_t* __restrict__ sdiag, const double* __restrict__ S,
                               double* __restrict__ dinv) {
  for (int64_t d = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; d < n; d += (int64_t)gridDim.x * blockDim.x) {
    const int32_t a = dslot[2 * d], b = dslot[2 * d + 1];
    dinv[d] = a >= 0 ? sgn / (S[sdiag[a]] + S[sdiag[b]]) : 0.0;
  }
}

}  // namespace hdg
