// Nonlinear (Saint Venant-Kirchhoff) elastodynamics, Sec. 4.4 (Eqs. UNEL, eq:HDG_nelas1-5), 3D:
// the element kernels of one Newton iteration of an implicit stage.
//
// Unknowns per element: v (3 N_p), H = F - I (9 N_p, row-major (i, J)), P (9 N_p), each a block
// of orthonormal-basis coefficients (mass matrix |det J| I); the trace v_hat has 3 N_f
// coefficients per face, component-major. The stage equations at (u, v_hat) are
//   (alpha rho (v - h_v), w) + (P, grad w) - <P n - s (v - v_hat), w> = (f, w)
//   (alpha (H - h_H), G) + (v, div G) - <v_hat, G n> = 0
//   (P, Q) - (F S(F), Q) = 0,      S(F) = lam tr(E) I + 2 mu E,  E = (F^T F - I) / 2
// with s = 2 sqrt(rho mu) (Eq. eq:stab_matrix_lin) and, on the faces, the conservation of
// P_hat n = P n - s (v - v_hat). Newton's matrix of one element is
//   A = [alpha rho d I + s E      0        -Dx   ]      B = [ -s Fm   ]
//       [ Dx^T                alpha d I     0   ]          [ -N Fm   ]
//       [ 0                      -T        d I  ]          [   0     ]
//   C = [ -s Fm^T   0   (N Fm)^T ],   D = s J_F I,
// where d = |det J|, Dx_J[a][b] = (phi_a, d_J phi_b), Fm_f = J_F Ff_f (face moments), N the
// normal components and T[(iJ) a, (kL) b] = sum_q w_q A_q[iJ, kL] phi_a phi_b the tangent
// dP/dF at the quadrature points. (The v-row block of P, Dx_J^T - sum_f n_J E_f, equals -Dx_J
// by integration by parts.) H and P are eliminated through their diagonal mass blocks:
//   S_v = alpha rho d I + s E + Dx T Dx^T / (alpha d^2)           (3 N_p x 3 N_p, SPD)
//   W   = Bv + Dx T BH / (alpha d^2)                              (3 N_p x m)
//   S_K = D - C A^{-1} B = D - W^T S_v^{-1} W + BH^T T BH / (alpha d^2)
// and, for the residual R = (R_v, R_H, R_P), y = R_P / d + T R_H / (alpha d^2):
//   A^{-1} R = (z_v, (R_H - Dx^T z_v) / (alpha d), (R_P + T z_H) / d),  z_v = S_v^{-1} (R_v + Dx y)
//   C A^{-1} R = W^T z_v - BH^T y.
// The three products Dx T Dx^T, Dx T BH and BH^T T BH are sums over the quadrature points of
// outer products (one CTA per element, accumulators in registers); T is never formed.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace hdg {

// Precision: the residual R, Rh (and so the solution Newton converges to) is FP64. The
// Jacobian pipeline (tangent, the three accumulations, the Cholesky of S_v, S_K, and the
// tangent applies of A^{-1} R and of the recovery) runs in TJ: double, or float for the
// mixed mode, where Newton converges to the same stage solution with an approximate Jacobian.
template <int K>
struct SvkDims {
  static constexpr int NP = (K + 1) * (K + 2) * (K + 3) / 6;
  static constexpr int NFP = (K + 1) * (K + 2) / 2;   // scalar face modes
  static constexpr int NF = 3 * NFP;                  // trace entries per face
  static constexpr int NV = 3 * NP;
  static constexpr int N = 21 * NP;
  static constexpr int M = 4 * NF;
  static constexpr int QR = 2 * K + 2;               // residual rule: points per direction
  static constexpr int NQR = QR * QR * QR;
  static constexpr int QJ = 2 * K + 1;               // Jacobian rule (exact for degree 4k)
  static constexpr int NQJ = QJ * QJ * QJ;
  static constexpr int QC = 8;                        // Jacobian points per chunk
  static constexpr int NT = 256;
  // chunk area: per-point S and F F^T (18), tangent (81), g_J (3 N_p), psi_f (4 N_fp), weight,
  // and the largest per-pass precompute (27 N_p, 36 N_p + 108 or 144 per point)
  static constexpr int PRE = 36 * NP + 108;
  static constexpr int CHJ = QC * (18 + 81 + 3 * NP + 4 * NFP + 1 + PRE);
  static constexpr int CHR = 9 * NQR;                 // P(F) at every residual point (double)
  static constexpr int CHT = 9 * NQJ;                 // T-apply: values at the Jacobian points
  // condensation kernel: double arena | scratch (double CHR or TJ chunk / T-apply) | TJ arena
  static constexpr int SMD = 32 + N + M + 3 * NP * NP + N + M + 4 * 9 * NP + 3 * NV;
  template <typename TJ>
  __host__ __device__ static constexpr size_t scr_bytes() {
    const size_t a = sizeof(double) * CHR, b = sizeof(TJ) * (CHJ > CHT ? CHJ : CHT);
    return ((a > b ? a : b) + 15) / 16 * 16;
  }
  template <typename TJ>
  __host__ __device__ static constexpr size_t cond_bytes() {
    return sizeof(double) * SMD + scr_bytes<TJ>() + sizeof(TJ) * (NV * NV + NV * M + 9 * NQJ);
  }
  // recovery kernel: double arena | TJ arena (L, F at the points, T-apply scratch)
  static constexpr int SMD_REC = 32 + N + M + 3 * NP * NP + 4 * 9 * NP + 3 * NV;
  template <typename TJ>
  __host__ __device__ static constexpr size_t rec_bytes() {
    return sizeof(double) * SMD_REC + sizeof(TJ) * (NV * NV + 9 * NQJ + CHT);
  }
};

// reference tables of one degree (device pointers into one buffer)
struct SvkTabs {
  const double* Dr;    // [3][Np][Np]   (phi_i, d_r phi_l) at [r][i][l]
  const double* Ff;    // [4][Np][Nfp]  reference face moments
  const double* Ef;    // [4][Np][Np]   Ff Ff^T
  const double* phiR;  // [NQR][Np]     residual rule
  const double* wR;    // [NQR]
  const double* muF;   // [NQF][Nfp]    face rule: face basis values
  const double* wF;    // [NQF]
  int nqf;
};

// Jacobian-rule tables in the Jacobian precision
template <typename T>
struct SvkJT {
  const T* phiJ;   // [NQJ][Np]
  const T* wJ;     // [NQJ]
  const T* GJ;     // [NQJ][3][Np]  sum_b Dr[r][a][b] phi_b(x_q)
  const T* PSJ;    // [NQJ][4][Nfp] sum_a Ff[f][a][m] phi_a(x_q)
};

struct SvkArgs {
  int64_t ne;
  const double* geo;
  const double* rho;
  const double* lam;
  const double* mu;
  const int32_t* elem_face;
  const int32_t* face_bnd;   // < 0: face carries unknowns (interior or traction face)
  double alpha;
  const double* u;           // [ne][N] Newton iterate (updated by the recovery kernel)
  const double* lamv;        // [nf][NF] traces of the iterate
  const double* h;           // [ne][N] stage history
  const double* fq;          // [ne][NQR][3] body force at the residual points, or null
  double* S;                 // [ne][M][M]
  double* L;                 // [ne][NV][NV] Cholesky factor of S_v (lower)
  double* zR;                // [ne][N] A^{-1} R
  double* slot;              // [ne][M] element part of the condensed right-hand side
  int* err;                  // set when S_v is not positive definite
};

__device__ __forceinline__ double tsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float tsqrt(float x) { return sqrtf(x); }

// ------------------------------------------------------------------ pointwise material law
// P = F S(F) and the tangent A[iJ][kL] = dP_iJ / dF_kL
//   = delta_ik S_LJ + lam F_iJ F_kL + mu F_iL F_kJ + mu (F F^T)_ik delta_JL.
template <typename T>
__device__ __forceinline__ void svk_stress(const T* F, T lam, T mu, T* Sout, T* FFt) {
  T C[9];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) C[a * 3 + b] = F[a] * F[b] + F[3 + a] * F[3 + b] + F[6 + a] * F[6 + b];
  const T trE = T(0.5) * (C[0] + C[4] + C[8] - T(3));
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) Sout[a * 3 + b] = mu * (C[a * 3 + b] - (a == b ? T(1) : T(0))) + (a == b ? lam * trE : T(0));
  if (FFt) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int k = 0; k < 3; ++k) FFt[i * 3 + k] = F[i * 3] * F[k * 3] + F[i * 3 + 1] * F[k * 3 + 1] + F[i * 3 + 2] * F[k * 3 + 2];
  }
}

template <typename T>
__device__ __forceinline__ T svk_tangent_entry(const T* F, const T* S, const T* FFt, T lam, T mu, int iJ, int kL) {
  const int i = iJ / 3, J = iJ % 3, k = kL / 3, L = kL % 3;
  T v = lam * F[iJ] * F[kL] + mu * F[i * 3 + L] * F[k * 3 + J];
  if (i == k) v += S[L * 3 + J];
  if (J == L) v += mu * FFt[i * 3 + k];
  return v;
}

// F = I + H at a point with basis values phi [Np] (H: [9][Np] FP64 coefficients)
template <int NP, typename PT>
__device__ __forceinline__ void svk_deformation(const PT* __restrict__ phi, const double* H, double* F) {
#pragma unroll
  for (int c = 0; c < 9; ++c) {
    double v = (c == 0 || c == 4 || c == 8) ? 1.0 : 0.0;
    for (int a = 0; a < NP; ++a) v += H[c * NP + a] * (double)phi[a];
    F[c] = v;
  }
}

// y = T x (x, y: [9][Np] FP64 in shared memory) on the Jacobian rule in precision TJ; FJ
// [NQJ][9] the deformation gradient at its points; scratch CHT entries. Ends with a barrier.
template <int K, typename TJ>
__device__ void svk_T_apply(const SvkJT<TJ>& tj, const TJ* FJ, TJ lam, TJ mu, TJ dJ, const double* x, double* y,
                            TJ* scr) {
  using D = SvkDims<K>;
  constexpr int NP = D::NP, NQJ = D::NQJ, NT = D::NT;
  const int tid = threadIdx.x;
  for (int q = tid; q < NQJ; q += NT) {
    const TJ* ph = tj.phiJ + (int64_t)q * NP;
    TJ xv[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) {
      TJ v = TJ(0);
      for (int a = 0; a < NP; ++a) v += (TJ)x[c * NP + a] * ph[a];
      xv[c] = v;
    }
    const TJ* F = FJ + q * 9;
    TJ S[9], FFt[9];
    svk_stress<TJ>(F, lam, mu, S, FFt);
    const TJ w = tj.wJ[q] * dJ;
#pragma unroll
    for (int r = 0; r < 9; ++r) {
      TJ v = TJ(0);
#pragma unroll
      for (int c = 0; c < 9; ++c) v += svk_tangent_entry<TJ>(F, S, FFt, lam, mu, r, c) * xv[c];
      scr[q * 9 + r] = w * v;
    }
  }
  __syncthreads();
  for (int idx = tid; idx < 9 * NP; idx += NT) {
    const int c = idx / NP, a = idx % NP;
    TJ v = TJ(0);
    for (int q = 0; q < NQJ; ++q) v += tj.phiJ[(int64_t)q * NP + a] * scr[q * 9 + c];
    y[idx] = (double)v;
  }
  __syncthreads();
}

// deformation gradient at every Jacobian-rule point from H (shared [9][Np], FP64)
template <int K, typename TJ>
__device__ void svk_F_at_jac(const SvkJT<TJ>& tj, const double* H, TJ* FJ) {
  using D = SvkDims<K>;
  for (int q = threadIdx.x; q < D::NQJ; q += D::NT) {
    double F[9];
    svk_deformation<D::NP, TJ>(tj.phiJ + (int64_t)q * D::NP, H, F);
#pragma unroll
    for (int c = 0; c < 9; ++c) FJ[q * 9 + c] = (TJ)F[c];
  }
  __syncthreads();
}

// upper-triangle index t -> (row, col) of an n x n matrix, row-major rows of n - r entries
__device__ __forceinline__ void tri_decode(int t, int n, int& r, int& c) {
  r = 0;
  while (t >= n - r) { t -= n - r; ++r; }
  c = r + t;
}

// CTAs per SM the register budget is cut for: two for the FP32 Jacobian up to k = 2
template <int K, typename TJ>
struct SvkMinBlocks { static constexpr int value = sizeof(TJ) == 4 && K <= 2 ? 2 : 1; };

// One Newton iteration's condensation of one element: residual, S_K, the factor of S_v,
// A^{-1} R and the element part g_K = -Rh + C A^{-1} R of the condensed right-hand side.
template <int K, typename TJ>
__global__ void __launch_bounds__(256, SvkMinBlocks<K, TJ>::value) svk_condense_kernel(SvkArgs a, SvkTabs tb, SvkJT<TJ> tj) {
  using D = SvkDims<K>;
  constexpr int NP = D::NP, NFP = D::NFP, NF = D::NF, NV = D::NV, N = D::N, M = D::M, NT = D::NT;
  constexpr int NQR = D::NQR, NQJ = D::NQJ, QC = D::QC;
  extern __shared__ __align__(16) unsigned char smraw[];
  double* g = reinterpret_cast<double*>(smraw);
  double* ue = g + 32;
  double* lk = ue + N;
  double* Dx = lk + M;       // [3][Np][Np]
  double* R = Dx + 3 * NP * NP;
  double* Rh = R + N;
  double* y = Rh + M;        // [9][Np]
  double* zH = y + 9 * NP;
  double* t1 = zH + 9 * NP;  // [9][Np] T-apply results
  double* t2 = t1 + 9 * NP;  // [9][Np]
  double* rv = t2 + 9 * NP;  // [NV]
  double* w1 = rv + NV;
  double* zv = w1 + NV;
  unsigned char* scr = smraw + sizeof(double) * D::SMD;
  double* CHR = reinterpret_cast<double*>(scr);   // residual phase
  TJ* CH = reinterpret_cast<TJ*>(scr);             // Jacobian phase
  TJ* Sv = reinterpret_cast<TJ*>(scr + D::template scr_bytes<TJ>());   // [NV][NV] -> L
  TJ* W = Sv + NV * NV;      // [NV][M] -> Z = L^{-1} W
  TJ* FJ = W + NV * M;       // [NQJ][9]
  const int64_t e = blockIdx.x;
  const int tid = threadIdx.x;
  if (tid < 32) g[tid] = a.geo[e * 32 + tid];
  for (int i = tid; i < N; i += NT) ue[i] = a.u[e * N + i];
  for (int i = tid; i < M; i += NT) {
    const int f = i / NF;
    const int fid = a.elem_face[e * 4 + f];
    lk[i] = a.face_bnd[fid] < 0 ? a.lamv[(int64_t)fid * NF + i % NF] : 0.0;
  }
  __syncthreads();
  const double dJ = g[0];
  const double rho = a.rho[e], lam = a.lam[e], mu = a.mu[e];
  const double s = 2.0 * sqrt(rho * mu);
  const double alpha = a.alpha;
  const double iad2 = 1.0 / (alpha * dJ * dJ);
  const TJ lamj = (TJ)lam, muj = (TJ)mu, dJj = (TJ)dJ;
  const double* Ji = g + 1;          // Jinv[r][j]
  const double* JF = g + 10;         // face Jacobians
  const double* nrm = g + 14;        // outward normals [4][3]
  for (int idx = tid; idx < 3 * NP * NP; idx += NT) {
    const int J = idx / (NP * NP), ab = idx % (NP * NP);
    double v = 0.0;
#pragma unroll
    for (int r = 0; r < 3; ++r) v += Ji[r * 3 + J] * tb.Dr[r * NP * NP + ab];
    Dx[idx] = dJ * v;
  }
  const double* Hc = ue + 3 * NP;
  const double* Pc = ue + 12 * NP;
  // ---- residual (FP64): P(F) at the residual points, then the volume and face terms
  for (int q = tid; q < NQR; q += NT) {
    double F[9], S[9];
    svk_deformation<NP, double>(tb.phiR + (int64_t)q * NP, Hc, F);
    svk_stress<double>(F, lam, mu, S, nullptr);
    const double w = tb.wR[q];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int J = 0; J < 3; ++J) CHR[q * 9 + i * 3 + J] = w * (F[i * 3] * S[J] + F[i * 3 + 1] * S[3 + J] + F[i * 3 + 2] * S[6 + J]);
  }
  __syncthreads();
  const double* hv = a.h + e * N;
  for (int idx = tid; idx < N; idx += NT) {
    double v;
    if (idx < 3 * NP) {
      const int i = idx / NP, aa = idx % NP;
      v = alpha * rho * dJ * (ue[idx] - hv[idx]);
      for (int f = 0; f < 4; ++f) {
        double ev = 0.0, fl = 0.0;
        for (int b = 0; b < NP; ++b) ev += tb.Ef[(f * NP + aa) * NP + b] * ue[i * NP + b];
        for (int m = 0; m < NFP; ++m) fl += tb.Ff[(f * NP + aa) * NFP + m] * lk[f * NF + i * NFP + m];
        v += s * JF[f] * (ev - fl);
      }
      if (a.fq) {
        double b = 0.0;
        for (int q = 0; q < NQR; ++q) b += tb.wR[q] * a.fq[((int64_t)e * NQR + q) * 3 + i] * tb.phiR[(int64_t)q * NP + aa];
        v -= dJ * b;
      }
      for (int J = 0; J < 3; ++J) {
        double dp = 0.0;
        for (int b = 0; b < NP; ++b) dp += Dx[(J * NP + aa) * NP + b] * Pc[(i * 3 + J) * NP + b];
        v -= dp;
      }
    } else if (idx < 12 * NP) {
      const int c = idx / NP - 3, aa = idx % NP, i = c / 3, J = c % 3;
      v = alpha * dJ * (ue[idx] - hv[idx]);
      double dv = 0.0;
      for (int b = 0; b < NP; ++b) dv += Dx[(J * NP + b) * NP + aa] * ue[i * NP + b];
      v += dv;
      for (int f = 0; f < 4; ++f) {
        double fl = 0.0;
        for (int m = 0; m < NFP; ++m) fl += tb.Ff[(f * NP + aa) * NFP + m] * lk[f * NF + i * NFP + m];
        v -= nrm[f * 3 + J] * JF[f] * fl;
      }
    } else {
      const int c = idx / NP - 12, aa = idx % NP;
      double sq = 0.0;
      for (int q = 0; q < NQR; ++q) sq += CHR[q * 9 + c] * tb.phiR[(int64_t)q * NP + aa];
      v = dJ * (ue[idx] - sq);
    }
    R[idx] = v;
  }
  for (int idx = tid; idx < M; idx += NT) {
    const int f = idx / NF, i = (idx % NF) / NFP, m = idx % NFP;
    double fv = 0.0;
    for (int b = 0; b < NP; ++b) fv += tb.Ff[(f * NP + b) * NFP + m] * ue[i * NP + b];
    double v = -s * JF[f] * fv + s * JF[f] * lk[idx];
    for (int J = 0; J < 3; ++J) {
      double fp = 0.0;
      for (int b = 0; b < NP; ++b) fp += tb.Ff[(f * NP + b) * NFP + m] * Pc[(i * 3 + J) * NP + b];
      v += nrm[f * 3 + J] * JF[f] * fp;
    }
    Rh[idx] = v;
  }
  __syncthreads();   // the residual scratch is reused below
  svk_F_at_jac<K, TJ>(tj, Hc, FJ);   // barrier inside
  // chunk layout
  TJ* cS = CH;                         // [QC][9]  S
  TJ* cFF = cS + QC * 9;               // [QC][9]  F F^T
  TJ* cA = cFF + QC * 9;               // [QC][81] tangent
  TJ* cg = cA + QC * 81;               // [QC][3][Np] g_J
  TJ* cps = cg + QC * 3 * NP;          // [QC][4][Nfp] psi_f
  TJ* cw = cps + QC * 4 * NFP;         // [QC] physical weights
  TJ* cpre = cw + QC;                  // per-pass precompute
  __shared__ TJ Jij[9], nj[12];   // J^{-1} and the normals in the Jacobian precision
  if (tid < 9) Jij[tid] = (TJ)Ji[tid];
  else if (tid < 21) nj[tid - 9] = (TJ)nrm[tid - 9];
  __syncthreads();
  // per chunk: S, F F^T, tangent, g_J, psi_f, weights of points q0 .. q0 + nq
  auto load_chunk = [&](int q0, int nq) {
    for (int t = tid; t < nq; t += NT) {
      svk_stress<TJ>(FJ + (q0 + t) * 9, lamj, muj, cS + t * 9, cFF + t * 9);
      cw[t] = tj.wJ[q0 + t] * dJj;
    }
    __syncthreads();
    for (int t = tid; t < nq * 81; t += NT) {
      const int qq = t / 81, r = t % 81;
      cA[t] = svk_tangent_entry<TJ>(FJ + (q0 + qq) * 9, cS + qq * 9, cFF + qq * 9, lamj, muj, r / 9, r % 9);
    }
    for (int t = tid; t < nq * 3 * NP; t += NT) {
      const int qq = t / (3 * NP), J = (t / NP) % 3, aa = t % NP;
      const TJ* G = tj.GJ + (int64_t)(q0 + qq) * 3 * NP;
      cg[t] = dJj * (Jij[J] * G[aa] + Jij[3 + J] * G[NP + aa] + Jij[6 + J] * G[2 * NP + aa]);
    }
    for (int t = tid; t < nq * 4 * NFP; t += NT) {
      const int qq = t / (4 * NFP), f = (t / NFP) % 4;
      cps[t] = (TJ)JF[f] * tj.PSJ[(int64_t)(q0 + qq) * 4 * NFP + t % (4 * NFP)];
    }
    __syncthreads();
  };
  // ---- (a) Dx T Dx^T, upper triangle: [(i,a),(k,b)] = sum_q w sum_L t[i][k][L][a] g_L(q)_b,
  //      t[i][k][L][a] = sum_J g_J(q)_a A[iJ][kL]
  {
    constexpr int NE = NV * (NV + 1) / 2, NS = (NE + NT - 1) / NT;
    TJ acc[NS];
    int rc[NS];
#pragma unroll
    for (int u = 0; u < NS; ++u) {
      acc[u] = TJ(0);
      const int t = tid + u * NT;
      int r = 0, c = 0;
      if (t < NE) tri_decode(t, NV, r, c);
      rc[u] = (r << 16) | c;
    }
    for (int q0 = 0; q0 < NQJ; q0 += QC) {
      const int nq = NQJ - q0 < QC ? NQJ - q0 : QC;
      load_chunk(q0, nq);
      for (int t = tid; t < nq * 27 * NP; t += NT) {
        const int qq = t / (27 * NP), ikL = (t / NP) % 27, aa = t % NP;
        const int i = ikL / 9, k = (ikL / 3) % 3, L = ikL % 3;
        const TJ* A = cA + qq * 81;
        const TJ* gg = cg + qq * 3 * NP;
        cpre[t] = gg[aa] * A[(i * 3) * 9 + k * 3 + L] + gg[NP + aa] * A[(i * 3 + 1) * 9 + k * 3 + L] +
                  gg[2 * NP + aa] * A[(i * 3 + 2) * 9 + k * 3 + L];
      }
      __syncthreads();
#pragma unroll
      for (int u = 0; u < NS; ++u) {
        if (tid + u * NT < NE) {
          const int r = rc[u] >> 16, c = rc[u] & 0xffff;
          const int i = r / NP, aa = r % NP, k = c / NP, b = c % NP;
          TJ v = acc[u];
          for (int qq = 0; qq < nq; ++qq) {
            const TJ* tt = cpre + ((qq * 27) + i * 9 + k * 3) * NP + aa;
            const TJ* gg = cg + qq * 3 * NP + b;
            v += cw[qq] * (tt[0] * gg[0] + tt[NP] * gg[NP] + tt[2 * NP] * gg[2 * NP]);
          }
          acc[u] = v;
        }
      }
      __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < NS; ++u) {
      if (tid + u * NT < NE) {
        const int r = rc[u] >> 16, c = rc[u] & 0xffff;
        const int i = r / NP, aa = r % NP, k = c / NP, b = c % NP;
        double v = iad2 * (double)acc[u];
        if (i == k) {
          double ev = 0.0;
          for (int f = 0; f < 4; ++f) ev += JF[f] * tb.Ef[(f * NP + aa) * NP + b];
          v += s * ev + (aa == b ? alpha * rho * dJ : 0.0);
        }
        Sv[r * NV + c] = (TJ)v;
        Sv[c * NV + r] = (TJ)v;
      }
    }
  }
  // ---- (b) Dx T BH: [(i,a),(f,i2,m)] = -sum_q w u[i][i2][f][a] psi_f(q)_m,
  //      u[i][i2][f][a] = sum_J g_J(q)_a sum_L A[iJ][i2 L] n_fL;   W = Bv + Dx T BH / (alpha d^2)
  {
    constexpr int NE = NV * M, NS = (NE + NT - 1) / NT;
    TJ acc[NS];
#pragma unroll
    for (int u = 0; u < NS; ++u) acc[u] = TJ(0);
    for (int q0 = 0; q0 < NQJ; q0 += QC) {
      const int nq = NQJ - q0 < QC ? NQJ - q0 : QC;
      load_chunk(q0, nq);
      // c_J[i][i2][f] = sum_L A[iJ][i2 L] n_fL, then u = sum_J g_J c_J
      TJ* ccj = cpre + QC * 36 * NP;
      for (int t = tid; t < nq * 108; t += NT) {
        const int qq = t / 108, r = t % 108;
        const int i = r / 36, i2 = (r / 12) % 3, f = (r / 3) % 4, J = r % 3;
        const TJ* A = cA + qq * 81 + (i * 3 + J) * 9 + i2 * 3;
        ccj[t] = A[0] * nj[f * 3] + A[1] * nj[f * 3 + 1] + A[2] * nj[f * 3 + 2];
      }
      __syncthreads();
      for (int t = tid; t < nq * 36 * NP; t += NT) {
        const int qq = t / (36 * NP), c36 = (t / NP) % 36, aa = t % NP;
        const TJ* cj = ccj + qq * 108 + c36 * 3;
        const TJ* gg = cg + qq * 3 * NP + aa;
        cpre[t] = gg[0] * cj[0] + gg[NP] * cj[1] + gg[2 * NP] * cj[2];
      }
      __syncthreads();
#pragma unroll
      for (int u = 0; u < NS; ++u) {
        const int t = tid + u * NT;
        if (t < NE) {
          const int r = t / M, col = t % M;
          const int i = r / NP, aa = r % NP, f = col / NF, i2 = (col % NF) / NFP, m = col % NFP;
          TJ v = acc[u];
          for (int qq = 0; qq < nq; ++qq)
            v += cw[qq] * cpre[((qq * 36) + i * 12 + i2 * 4 + f) * NP + aa] * cps[(qq * 4 + f) * NFP + m];
          acc[u] = v;
        }
      }
      __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < NS; ++u) {
      const int t = tid + u * NT;
      if (t < NE) {
        const int r = t / M, col = t % M;
        const int i = r / NP, aa = r % NP, f = col / NF, i2 = (col % NF) / NFP, m = col % NFP;
        double v = -iad2 * (double)acc[u];
        if (i == i2) v -= s * JF[f] * tb.Ff[(f * NP + aa) * NFP + m];
        W[t] = (TJ)v;
      }
    }
  }
  __syncthreads();
  // ---- Cholesky S_v = L L^T (in place, lower), then Z = L^{-1} W
  for (int j = 0; j < NV; ++j) {
    if (tid == 0) {
      TJ dd = Sv[j * NV + j];
      if (!(dd > TJ(0))) { atomicExch(a.err, 1); dd = TJ(1); }
      Sv[j * NV + j] = tsqrt(dd);
    }
    __syncthreads();
    for (int i = j + 1 + tid; i < NV; i += NT) Sv[i * NV + j] /= Sv[j * NV + j];
    __syncthreads();
    const int w = NV - j - 1;
    for (int idx = tid; idx < w * w; idx += NT) {
      const int i = j + 1 + idx / w, l = j + 1 + idx % w;
      if (l <= i) Sv[i * NV + l] -= Sv[i * NV + j] * Sv[l * NV + j];
    }
    __syncthreads();
  }
  for (int col = tid; col < M; col += NT) {
    for (int i = 0; i < NV; ++i) {
      TJ v = W[i * M + col];
      for (int l = 0; l < i; ++l) v -= Sv[i * NV + l] * W[l * M + col];
      W[i * M + col] = v / Sv[i * NV + i];
    }
  }
  __syncthreads();
  // ---- (c) BH^T T BH, upper triangle: [(f,i,m),(f2,i2,m2)] = sum_q w c[f][i][f2][i2] psi_f(q)_m psi_f2(q)_m2,
  //      c = n_f^T A^{(i,i2)} n_f2;   S_K = D - Z^T Z + BH^T T BH / (alpha d^2)
  {
    constexpr int NE = M * (M + 1) / 2, NS = (NE + NT - 1) / NT;
    TJ acc[NS];
    int rc[NS];
#pragma unroll
    for (int u = 0; u < NS; ++u) {
      acc[u] = TJ(0);
      const int t = tid + u * NT;
      int r = 0, c = 0;
      if (t < NE) tri_decode(t, M, r, c);
      rc[u] = (r << 16) | c;
    }
    for (int q0 = 0; q0 < NQJ; q0 += QC) {
      const int nq = NQJ - q0 < QC ? NQJ - q0 : QC;
      load_chunk(q0, nq);
      for (int t = tid; t < nq * 144; t += NT) {
        const int qq = t / 144, c144 = t % 144;
        const int f = c144 / 36, i = (c144 / 12) % 3, f2 = (c144 / 3) % 4, i2 = c144 % 3;
        const TJ* A = cA + qq * 81;
        TJ v = TJ(0);
#pragma unroll
        for (int J = 0; J < 3; ++J)
#pragma unroll
          for (int L = 0; L < 3; ++L) v += nj[f * 3 + J] * A[(i * 3 + J) * 9 + i2 * 3 + L] * nj[f2 * 3 + L];
        cpre[t] = cw[qq] * v;
      }
      __syncthreads();
#pragma unroll
      for (int u = 0; u < NS; ++u) {
        if (tid + u * NT < NE) {
          const int c1 = rc[u] >> 16, c2 = rc[u] & 0xffff;
          const int f = c1 / NF, i = (c1 % NF) / NFP, m = c1 % NFP;
          const int f2 = c2 / NF, i2 = (c2 % NF) / NFP, m2 = c2 % NFP;
          TJ v = acc[u];
          for (int qq = 0; qq < nq; ++qq)
            v += cpre[qq * 144 + f * 36 + i * 12 + f2 * 3 + i2] * cps[(qq * 4 + f) * NFP + m] * cps[(qq * 4 + f2) * NFP + m2];
          acc[u] = v;
        }
      }
      __syncthreads();
    }
    double* Se = a.S + e * (int64_t)(M * M);
#pragma unroll
    for (int u = 0; u < NS; ++u) {
      if (tid + u * NT < NE) {
        const int c1 = rc[u] >> 16, c2 = rc[u] & 0xffff;
        TJ zz = TJ(0);
        for (int r = 0; r < NV; ++r) zz += W[r * M + c1] * W[r * M + c2];
        double v = iad2 * (double)acc[u] - (double)zz;
        if (c1 == c2) v += s * JF[c1 / NF];
        Se[c1 * M + c2] = v;
        Se[c2 * M + c1] = v;
      }
    }
  }
  // ---- condensed right-hand side and A^{-1} R (FP64 vectors; the Jacobian factors in TJ)
  svk_T_apply<K, TJ>(tj, FJ, lamj, muj, dJj, R + 3 * NP, t1, CH);           // T R_H
  for (int idx = tid; idx < 9 * NP; idx += NT) y[idx] = R[12 * NP + idx] / dJ + iad2 * t1[idx];
  __syncthreads();
  for (int idx = tid; idx < NV; idx += NT) {
    const int i = idx / NP, aa = idx % NP;
    double v = R[idx];
    for (int J = 0; J < 3; ++J)
      for (int b = 0; b < NP; ++b) v += Dx[(J * NP + aa) * NP + b] * y[(i * 3 + J) * NP + b];
    rv[idx] = v;
  }
  __syncthreads();
  if (tid == 0) {
    for (int i = 0; i < NV; ++i) {
      double v = rv[i];
      for (int l = 0; l < i; ++l) v -= (double)Sv[i * NV + l] * w1[l];
      w1[i] = v / (double)Sv[i * NV + i];
    }
    for (int i = NV - 1; i >= 0; --i) {
      double v = w1[i];
      for (int l = i + 1; l < NV; ++l) v -= (double)Sv[l * NV + i] * zv[l];
      zv[i] = v / (double)Sv[i * NV + i];
    }
  }
  __syncthreads();
  double* gK = a.slot + e * (int64_t)M;
  for (int idx = tid; idx < M; idx += NT) {
    const int f = idx / NF, i = (idx % NF) / NFP, m = idx % NFP;
    double v = -Rh[idx];
    for (int r = 0; r < NV; ++r) v += (double)W[r * M + idx] * w1[r];
    for (int J = 0; J < 3; ++J) {
      double fy = 0.0;
      for (int b = 0; b < NP; ++b) fy += tb.Ff[(f * NP + b) * NFP + m] * y[(i * 3 + J) * NP + b];
      v += nrm[f * 3 + J] * JF[f] * fy;
    }
    gK[idx] = v;
  }
  for (int idx = tid; idx < 9 * NP; idx += NT) {
    const int c = idx / NP, aa = idx % NP, i = c / 3, J = c % 3;
    double v = R[3 * NP + idx];
    for (int b = 0; b < NP; ++b) v -= Dx[(J * NP + b) * NP + aa] * zv[i * NP + b];
    zH[idx] = v / (alpha * dJ);
  }
  __syncthreads();
  svk_T_apply<K, TJ>(tj, FJ, lamj, muj, dJj, zH, t2, CH);                    // T z_H
  double* zr = a.zR + e * (int64_t)N;
  for (int idx = tid; idx < N; idx += NT) {
    double v;
    if (idx < NV) v = zv[idx];
    else if (idx < 12 * NP) v = zH[idx - NV];
    else v = (R[idx] + t2[idx - 12 * NP]) / dJ;
    zr[idx] = v;
  }
  double* Le = a.L + e * (int64_t)(NV * NV);
  for (int idx = tid; idx < NV * NV; idx += NT) Le[idx] = (double)Sv[idx];
}

struct SvkRecArgs {
  int64_t ne;
  const double* geo;
  const double* rho;
  const double* lam;
  const double* mu;
  const int32_t* elem_face;
  const int32_t* face_bnd;
  double alpha;
  double* u;                 // [ne][N], updated in place: u -= A^{-1} R + A^{-1} B dlam
  const double* dl;          // [nf][NF] trace increment
  const double* L;
  const double* zR;
  unsigned long long* umax;  // [2] max |du|, max |u_new| (bit patterns of non-negative doubles)
};

// Local recovery of the Newton increment (Eq. LS): du = -A^{-1} R - A^{-1} B dlam, u += du.
template <int K, typename TJ>
__global__ void __launch_bounds__(256, SvkMinBlocks<K, TJ>::value) svk_recover_kernel(SvkRecArgs a, SvkTabs tb, SvkJT<TJ> tj) {
  using D = SvkDims<K>;
  constexpr int NP = D::NP, NFP = D::NFP, NF = D::NF, NV = D::NV, N = D::N, M = D::M, NT = D::NT, NQJ = D::NQJ;
  extern __shared__ __align__(16) unsigned char smraw[];
  double* g = reinterpret_cast<double*>(smraw);
  double* ue = g + 32;
  double* dk = ue + N;
  double* Dx = dk + M;
  double* rH = Dx + 3 * NP * NP;   // [9][Np]
  double* t1 = rH + 9 * NP;
  double* zH = t1 + 9 * NP;
  double* t2 = zH + 9 * NP;
  double* rv = t2 + 9 * NP;
  double* w1 = rv + NV;
  double* zv = w1 + NV;
  TJ* Ls = reinterpret_cast<TJ*>(smraw + sizeof(double) * D::SMD_REC);
  TJ* FJ = Ls + NV * NV;
  TJ* CH = FJ + 9 * NQJ;
  __shared__ double red[2][8];
  const int64_t e = blockIdx.x;
  const int tid = threadIdx.x;
  if (tid < 32) g[tid] = a.geo[e * 32 + tid];
  for (int i = tid; i < N; i += NT) ue[i] = a.u[e * N + i];
  for (int i = tid; i < NV * NV; i += NT) Ls[i] = (TJ)a.L[e * (int64_t)(NV * NV) + i];
  for (int i = tid; i < M; i += NT) {
    const int fid = a.elem_face[e * 4 + i / NF];
    dk[i] = a.face_bnd[fid] < 0 ? a.dl[(int64_t)fid * NF + i % NF] : 0.0;
  }
  __syncthreads();
  const double dJ = g[0];
  const double rho = a.rho[e], lam = a.lam[e], mu = a.mu[e];
  const double s = 2.0 * sqrt(rho * mu);
  const double alpha = a.alpha;
  const double iad2 = 1.0 / (alpha * dJ * dJ);
  const double* Ji = g + 1;
  const double* JF = g + 10;
  const double* nrm = g + 14;
  for (int idx = tid; idx < 3 * NP * NP; idx += NT) {
    const int J = idx / (NP * NP), ab = idx % (NP * NP);
    double v = 0.0;
#pragma unroll
    for (int r = 0; r < 3; ++r) v += Ji[r * 3 + J] * tb.Dr[r * NP * NP + ab];
    Dx[idx] = dJ * v;
  }
  // B dlam: v rows -s Fm dlam_i, H rows -n_J Fm dlam_i
  for (int idx = tid; idx < 12 * NP; idx += NT) {
    if (idx < NV) {
      const int i = idx / NP, aa = idx % NP;
      double v = 0.0;
      for (int f = 0; f < 4; ++f) {
        double fl = 0.0;
        for (int m = 0; m < NFP; ++m) fl += tb.Ff[(f * NP + aa) * NFP + m] * dk[f * NF + i * NFP + m];
        v -= s * JF[f] * fl;
      }
      rv[idx] = v;
    } else {
      const int c = idx / NP - 3, aa = idx % NP, i = c / 3, J = c % 3;
      double v = 0.0;
      for (int f = 0; f < 4; ++f) {
        double fl = 0.0;
        for (int m = 0; m < NFP; ++m) fl += tb.Ff[(f * NP + aa) * NFP + m] * dk[f * NF + i * NFP + m];
        v -= nrm[f * 3 + J] * JF[f] * fl;
      }
      rH[c * NP + aa] = v;
    }
  }
  __syncthreads();
  const TJ lamj = (TJ)lam, muj = (TJ)mu, dJj = (TJ)dJ;
  svk_F_at_jac<K, TJ>(tj, ue + 3 * NP, FJ);
  svk_T_apply<K, TJ>(tj, FJ, lamj, muj, dJj, rH, t1, CH);   // T (BH dlam)
  // z_v = S_v^{-1} (Bv dlam + Dx T BH dlam / (alpha d^2))
  for (int idx = tid; idx < NV; idx += NT) {
    const int i = idx / NP, aa = idx % NP;
    double v = rv[idx];
    for (int J = 0; J < 3; ++J)
      for (int b = 0; b < NP; ++b) v += iad2 * Dx[(J * NP + aa) * NP + b] * t1[(i * 3 + J) * NP + b];
    w1[idx] = v;
  }
  __syncthreads();
  if (tid == 0) {
    for (int i = 0; i < NV; ++i) {
      double v = w1[i];
      for (int l = 0; l < i; ++l) v -= (double)Ls[i * NV + l] * w1[l];
      w1[i] = v / (double)Ls[i * NV + i];
    }
    for (int i = NV - 1; i >= 0; --i) {
      double v = w1[i];
      for (int l = i + 1; l < NV; ++l) v -= (double)Ls[l * NV + i] * zv[l];
      zv[i] = v / (double)Ls[i * NV + i];
    }
  }
  __syncthreads();
  for (int idx = tid; idx < 9 * NP; idx += NT) {
    const int c = idx / NP, aa = idx % NP, i = c / 3, J = c % 3;
    double v = rH[idx];
    for (int b = 0; b < NP; ++b) v -= Dx[(J * NP + b) * NP + aa] * zv[i * NP + b];
    zH[idx] = v / (alpha * dJ);
  }
  __syncthreads();
  svk_T_apply<K, TJ>(tj, FJ, lamj, muj, dJj, zH, t2, CH);   // T z_H
  const double* zr = a.zR + e * (int64_t)N;
  double mdu = 0.0, mu_ = 0.0;
  double* uo = a.u + e * (int64_t)N;
  for (int idx = tid; idx < N; idx += NT) {
    double z;
    if (idx < NV) z = zv[idx];
    else if (idx < 12 * NP) z = zH[idx - NV];
    else z = t2[idx - 12 * NP] / dJ;
    const double du = -zr[idx] - z;
    const double un = ue[idx] + du;
    uo[idx] = un;
    mdu = fmax(mdu, fabs(du));
    mu_ = fmax(mu_, fabs(un));
  }
  for (int o = 16; o > 0; o >>= 1) {
    mdu = fmax(mdu, __shfl_xor_sync(0xffffffffu, mdu, o));
    mu_ = fmax(mu_, __shfl_xor_sync(0xffffffffu, mu_, o));
  }
  if ((tid & 31) == 0) { red[0][tid >> 5] = mdu; red[1][tid >> 5] = mu_; }
  __syncthreads();
  if (tid == 0) {
    double m0 = 0.0, m1 = 0.0;
    for (int w = 0; w < NT / 32; ++w) { m0 = fmax(m0, red[0][w]); m1 = fmax(m1, red[1][w]); }
    atomicMax(&a.umax[0], (unsigned long long)__double_as_longlong(m0));
    atomicMax(&a.umax[1], (unsigned long long)__double_as_longlong(m1));
  }
}

// lam += dlam on the faces with unknowns; max |dlam| into umax[0]
static __global__ void svk_trace_update_kernel(int64_t nf, int NF, const int32_t* __restrict__ face_bnd,
                                               const double* __restrict__ dl, double* __restrict__ lamv,
                                               unsigned long long* umax) {
  double m = 0.0;
  const int64_t n = nf * NF;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    if (face_bnd[t / NF] < 0) {
      lamv[t] += dl[t];
      m = fmax(m, fabs(dl[t]));
    }
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0.0) atomicMax(umax, (unsigned long long)__double_as_longlong(m));
}

// Jacobi diagonal of the assembled trace system; a traction face has one element (its
// second slot is the zero sentinel past the last element)
static __global__ void svk_diag_kernel(int64_t nf, int NF, int M, int64_t nslots, const int32_t* __restrict__ face_slot,
                                       const int32_t* __restrict__ face_bnd, const double* __restrict__ S,
                                       double* __restrict__ dinv) {
  const int64_t n = nf * NF;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t f = t / NF;
    const int mm = (int)(t % NF);
    double d = 0.0;
    if (face_bnd[f] < 0) {
      for (int sd = 0; sd < 2; ++sd) {
        const int64_t slot = face_slot[2 * f + sd];
        if (slot < 0 || slot >= nslots) continue;
        const int64_t e = slot / 4;
        const int r = (int)(slot % 4) * NF + mm;
        d += S[e * (int64_t)M * M + (int64_t)r * M + r];
      }
      dinv[t] = 1.0 / d;
    } else {
      dinv[t] = 0.0;
    }
  }
}

// traction load on the traction faces: b[f][i][m] += J_F sum_q w_q g_i(x_q) mu_m(x_q)
static __global__ void svk_traction_kernel(int64_t nb, int NFP, const int64_t* __restrict__ bnd_faces,
                                           const int32_t* __restrict__ face_slot0, const uint8_t* __restrict__ neu,
                                           const double* __restrict__ geo, const double* __restrict__ gq,
                                           const double* __restrict__ muF, const double* __restrict__ wF, int nqf,
                                           double* __restrict__ b) {
  const int64_t n = nb * 3 * NFP;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t bi = t / (3 * NFP);
    if (!neu[bi]) continue;
    const int i = (int)((t / NFP) % 3), m = (int)(t % NFP);
    const int64_t f = bnd_faces[bi];
    const int32_t slot = face_slot0[2 * f];
    const double jf = geo[(int64_t)(slot / 4) * 32 + 10 + slot % 4];
    double v = 0.0;
    for (int q = 0; q < nqf; ++q) v += wF[q] * gq[(bi * nqf + q) * 3 + i] * muF[q * NFP + m];
    b[f * 3 * NFP + i * NFP + m] += jf * v;
  }
}

}  // namespace hdg
