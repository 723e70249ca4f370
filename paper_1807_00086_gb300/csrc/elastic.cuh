// Linear elastodynamics (Sec. 4.1, velocity / symmetric-stress form) on the GPU.
//
// Unknowns per element: v_i (i < d) then sigma_a (a < NT, components (11,22,33,23,13,12) in
// 3D, (11,22,12) in 2D), N_p coefficients each; trace v_hat per face, d components x N_f
// (component-major). Flux sigma_hat n = sigma n - s (v - v_hat), s = 2 rho c_s
// (Eq. eq:stab_matrix_lin with the paper's experiment factor). Per element, with
// G_q = (d_q phi_l, phi_m)^T-type derivative blocks from the reference tables:
//   v rows:     alpha rho |J| v + s E v - sum_j (G_j^T) sigma_ij - s F v_hat = r_v
//   sigma rows: alpha |J| Q sigma + sum G_q v_p - sum n_q F v_hat_p = r_sigma      (Q: compliance)
// The compliance mass is block-diagonal with inverse Cm = [[2 mu I + lam 1 1^T, 0], [0, mu I]],
// so sigma is eliminated analytically and the velocity block
//   H = alpha rho |J| I + s sum_f J_f E^_f + (|J|/alpha) sum_rs Xi_ij,rs T^_rs
// is SPD; then S_K = s J_f I + (J_f J_g/(alpha |J|)) Phi P^_fg - Bt^T H^{-1} Bt with
//   Bt = -s J_f F^_f delta_ip - (J_f/alpha) sum_r Psi_ipfr (D^_r F^_f),
// where Xi, Psi, Phi contract Cm with J^{-1} and the face normals.
#pragma once
#include "kernels.cuh"

namespace hdg {

template <int DIM, int K>
struct ElDims {
  static constexpr int NP = Dims<DIM, K>::NP;
  static constexpr int NFP = Dims<DIM, K>::NF;   // scalar face basis
  static constexpr int NF = DIM * NFP;            // trace DOFs per face
  static constexpr int NFC = DIM + 1;
  static constexpr int NT = DIM * (DIM + 1) / 2;
  static constexpr int NV = DIM * NP;
  static constexpr int N = (DIM + NT) * NP;
  static constexpr int M = NFC * NF;
  static constexpr int OJF = 1 + DIM * DIM;
  static constexpr int ON = 1 + DIM * DIM + DIM + 1;
};

// symmetric component a -> (i, j)
template <int DIM>
__device__ __forceinline__ void sym_ij(int a, int& i, int& j) {
  if (DIM == 2) {
    const int ti[3] = {0, 1, 0}, tj[3] = {0, 1, 1};
    i = ti[a]; j = tj[a];
  } else {
    const int ti[6] = {0, 1, 2, 1, 0, 0}, tj[6] = {0, 1, 2, 2, 2, 1};
    i = ti[a]; j = tj[a];
  }
}
// component index of (i, j) or (j, i)
template <int DIM>
__device__ __forceinline__ int sym_index(int i, int j) {
  if (i > j) { const int t = i; i = j; j = t; }
  if (i == j) return i;
  if (DIM == 2) return 2;
  return (i == 1 && j == 2) ? 3 : (i == 0 && j == 2) ? 4 : 5;
}
// q with (i, q) in the symmetric pair set of component a, or -1
template <int DIM>
__device__ __forceinline__ int qa(int a, int i) {
  int ai, aj;
  sym_ij<DIM>(a, ai, aj);
  if (i == ai) return aj;
  if (i == aj && ai != aj) return ai;
  return -1;
}
// Cm = compliance^{-1} in the component basis; Q = compliance (for the mass term)
template <int DIM>
__device__ __forceinline__ double cm_entry(int a, int b, double lam, double mu) {
  int ai, aj, bi, bj;
  sym_ij<DIM>(a, ai, aj);
  sym_ij<DIM>(b, bi, bj);
  if (ai == aj && bi == bj) return lam + (a == b ? 2.0 * mu : 0.0);
  return a == b ? mu : 0.0;
}
template <int DIM>
__device__ __forceinline__ double q_entry(int a, int b, double lam, double mu) {
  int ai, aj, bi, bj;
  sym_ij<DIM>(a, ai, aj);
  sym_ij<DIM>(b, bi, bj);
  double v = 0.0;
  if (a == b) v += (ai == aj ? 1.0 : 2.0) / (2.0 * mu);
  if (ai == aj && bi == bj) v -= lam / ((DIM * lam + 2.0 * mu) * 2.0 * mu);
  return v;
}

// ------------------------------------------------------------------ condensation
template <int DIM, int K>
struct CondElCfg {
  using D = ElDims<DIM, K>;
  static constexpr size_t SMEM = sizeof(double) * ((size_t)2 * D::NV * D::NV + (size_t)D::NV * D::M);
};

template <int DIM, int K>
__global__ void __launch_bounds__(256) condense_el_kernel(DevMesh mesh, Tabs T, const double* __restrict__ lamv,
                                                           const double* __restrict__ muv, double alpha,
                                                           double* __restrict__ S, double* __restrict__ Hinv,
                                                           int* __restrict__ err) {
  using D = ElDims<DIM, K>;
  constexpr int NP = D::NP, NFP = D::NFP, NF = D::NF, NFC = D::NFC, NT = D::NT, NV = D::NV, M = D::M;
  constexpr int NTH = 256;
  extern __shared__ double dyn[];
  double* H = dyn;
  double* Li = H + NV * NV;
  double* W = Li + NV * NV;
  __shared__ double g[GEO_STRIDE];
  __shared__ double Xi[DIM * DIM * DIM * DIM];
  __shared__ double Psi[DIM * DIM * NFC * DIM];
  __shared__ double Phi[NFC * DIM * NFC * DIM];
  const int64_t e = blockIdx.x;
  const int tid = threadIdx.x;
  if (tid < GEO_STRIDE) g[tid] = mesh.geo[e * GEO_STRIDE + tid];
  __syncthreads();
  const double dJ = g[0];
  const double rho = mesh.rho[e], lam = lamv[e], mu = muv[e];
  const double s = 2.0 * sqrt(rho * mu);
  // coefficient tensors
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
  double* Se = S + e * (int64_t)(M * M);
  const double ia = 1.0 / (alpha * dJ);
  for (int idx = tid; idx < M * M; idx += NTH) {
    const int c1 = idx / M, c2 = idx % M;
    const int f = c1 / NF, p = (c1 % NF) / NFP, a1 = c1 % NFP;
    const int gg = c2 / NF, p2 = (c2 % NF) / NFP, b1 = c2 % NFP;
    double v = 0.0;
    for (int i = 0; i < NV; ++i) v -= W[i * M + c1] * W[i * M + c2];
    v += ia * g[D::OJF + f] * g[D::OJF + gg] * Phi[((f * DIM + p) * NFC + gg) * DIM + p2] *
         T.Pfg[((f * NFC + gg) * NFP + a1) * NFP + b1];
    if (c1 == c2) v += s * g[D::OJF + f];
    Se[idx] = v;
  }
  double* He = Hinv + e * (int64_t)(NV * NV);
  for (int idx = tid; idx < NV * NV; idx += NTH) {
    const int i = idx / NV, l = idx % NV;
    const int q0 = i > l ? i : l;
    double sacc = 0.0;
    for (int q = q0; q < NV; ++q) sacc += Li[q * NV + i] * Li[q * NV + l];
    He[idx] = sacc;
  }
}

// ------------------------------------------------------------------ element-local solves
// MODE 0: out = C_K A_K^{-1} (F_K - B_K lamD_K) [ne][M];  MODE 1: out = A_K^{-1} (F_K - B_K lam_K) [ne][N].
// F_K = F[e] or alpha Mw_K hist[e] (no sources in the elastic path).
template <int DIM, int K, int MODE>
__global__ void __launch_bounds__(128) local_el_kernel(DevMesh mesh, Tabs T, const double* __restrict__ lamv,
                                                        const double* __restrict__ muv, const double* __restrict__ Hinv,
                                                        double alpha, const double* __restrict__ F,
                                                        const double* __restrict__ hist, const double* __restrict__ lamt,
                                                        double* __restrict__ out) {
  using D = ElDims<DIM, K>;
  constexpr int NP = D::NP, NFP = D::NFP, NF = D::NF, NFC = D::NFC, NT = D::NT, NV = D::NV, M = D::M, N = D::N;
  constexpr int NTH = 128;
  __shared__ double g[GEO_STRIDE];
  __shared__ double ll[M];
  __shared__ int fuse[NFC];
  __shared__ double Fl[NFC * DIM * NP];
  __shared__ double rv[NV], rs[NT * NP], y[NT * NP], tt[DIM * DIM * NP], rhs[NV], v[NV], z[DIM * DIM * NP];
  __shared__ double w[NT * NP], sg[NT * NP];
  __shared__ double Cm[NT * NT], Qm[NT * NT];
  const int64_t e = blockIdx.x;
  const int tid = threadIdx.x;
  const double rho = mesh.rho[e], lam = lamv[e], mu = muv[e];
  const double s = 2.0 * sqrt(rho * mu);
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
  __syncthreads();
  for (int t = tid; t < M; t += NTH) {
    const int f = mesh.elem_face[e * NFC + t / NF];
    ll[t] = fuse[t / NF] ? lamt[(int64_t)f * NF + t % NF] : 0.0;
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
  // right-hand sides r_v, r_sigma
  for (int t = tid; t < N; t += NTH) {
    const int comp = t / NP, l = t % NP;
    if (comp < DIM) {
      double val = hist ? alpha * rho * dJ * hist[e * N + t] : F[e * N + t];
      double bl = 0.0;
      for (int f = 0; f < NFC; ++f) bl += g[D::OJF + f] * Fl[(f * DIM + comp) * NP + l];
      rv[t] = val + s * bl;
    } else {
      const int a = comp - DIM;
      double val;
      if (hist) {
        val = 0.0;
        for (int b = 0; b < NT; ++b) val += Qm[a * NT + b] * hist[e * N + (DIM + b) * NP + l];
        val *= alpha * dJ;
      } else {
        val = F[e * N + t];
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
  const double* He = Hinv + e * (int64_t)(NV * NV);
  for (int t = tid; t < NV; t += NTH) {
    double acc = 0.0;
    for (int l = 0; l < NV; ++l) acc += He[l * NV + t] * rhs[l];   // H^{-1} symmetric: column read
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
    for (int t = tid; t < N; t += NTH) out[e * N + t] = t < NV ? v[t] : sg[t - NV];
    return;
  }
  // g[f][i][mm] = J_f sum_l F^_f[l][mm] (-s v_i[l] + sum_j n_fj sigma_ij[l]); Fl reused for the weights
  for (int t = tid; t < NFC * DIM * NP; t += NTH) {
    const int f = t / (DIM * NP), i = (t / NP) % DIM, l = t % NP;
    double acc = -s * v[i * NP + l];
    for (int j = 0; j < DIM; ++j) acc += g[D::ON + f * DIM + j] * sg[sym_index<DIM>(i, j) * NP + l];
    Fl[t] = acc;
  }
  __syncthreads();
  for (int t = tid; t < M; t += NTH) {
    const int f = t / NF, i = (t % NF) / NFP, mm = t % NFP;
    double acc = 0.0;
    for (int l = 0; l < NP; ++l) acc += T.Ff[(f * NP + l) * NFP + mm] * Fl[(f * DIM + i) * NP + l];
    out[e * M + t] = g[D::OJF + f] * acc;
  }
}

// ------------------------------------------------------------------ FP32 apply for large blocks
// warp per element, full FP32 S_K [e][M][M]; lane handles rows lane + 32 q; column c of the
// symmetric S_K is read as row c (coalesced).
template <class L>
__global__ void __launch_bounds__(128) apply32f_kernel(int64_t ne, const int32_t* __restrict__ elem_face,
                                                       const int32_t* __restrict__ face_bnd, const float* __restrict__ S32,
                                                       const float* __restrict__ x, float* __restrict__ slot,
                                                       const int* __restrict__ done) {
  constexpr int NF = L::NF, M = L::M, NFC = L::NFC;
  constexpr int RPL = (M + 31) / 32;
  __shared__ float lx[4][M];
  if (done && *done) return;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t e = (int64_t)blockIdx.x * 4 + w;
  if (e < ne) {
    for (int r = lane; r < M; r += 32) {
      const int f = elem_face[e * NFC + r / NF];
      lx[w][r] = face_bnd[f] < 0 ? x[(int64_t)f * NF + r % NF] : 0.f;
    }
  }
  __syncwarp();
  if (e >= ne) return;
  float acc[RPL];
#pragma unroll
  for (int q = 0; q < RPL; ++q) acc[q] = 0.f;
  const float* Se = S32 + e * (int64_t)(M * M);
#pragma unroll 4
  for (int c = 0; c < M; ++c) {
    const float xc = lx[w][c];
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
      const int r = lane + 32 * q;
      if (r < M) acc[q] = fmaf(__ldcs(Se + c * M + r), xc, acc[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < RPL; ++q) {
    const int r = lane + 32 * q;
    if (r < M) slot[e * M + r] = acc[q];
  }
}

static __global__ void to32_copy_kernel(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    b[t] = (float)a[t];
}

}  // namespace hdg
