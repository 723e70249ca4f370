// Element-local post-processing of the acoustic pressure into P_{k+1} (the local, superconvergent
// post-processing step of HDG methods named in Sec. 1; acoustic reading of the standard one).
//
// Per element K with fields p (degree k, orthonormal phi) and traces lam_f on its faces:
//   q_h in [P_k(K)]^d is the discrete gradient of the local momentum equation,
//     (q_h, r)_K = -(p, div r)_K + <lam, r.n>_dK, mass |det J| I, so
//     q^j = -sum_r Jinv[r][j] Dr[r]^T p + (1/|det J|) sum_f n_f,j J_F,f Ff[f] lam_f;
//   p* in P_{k+1}(K) (orthonormal psi) solves (grad p*, grad psi_i)_K = (q_h, grad psi_i)_K for
//   i >= 1, both sides divided by |det J|:
//     A_il = sum_{r,s} (Jinv Jinv^T)[r][s] K1[r][s][i][l],  b_i = sum_{j,r} Jinv[r][j] (E1[r] q^j)_i;
//   the mean condition (p*, 1)_K = (p, 1)_K fixes the constant mode: p*_0 = p_0 (psi_0 = phi_0),
//   and psi_0 has no gradient, so A' c' = b' on the modes 1..Np1-1 (SPD) gives the rest.
// One warp per element, A' in shared memory, right-looking Cholesky and the two triangular
// solves by the same warp. FP64 throughout: the step runs once per output time.
#pragma once

#include "kernels.cuh"

namespace hdg {

struct PostTabs {
  const double* K1;   // [dim][dim][Np1][Np1]
  const double* E1;   // [dim][Np1][Np]
};

template <int DIM, int K>
struct PostCfg {
  static constexpr int NP = Dims<DIM, K>::NP;
  static constexpr int NP1 = Dims<DIM, K + 1>::NP;
  static constexpr int NA = NP1 - 1;
  // per-warp shared memory (doubles): A' [NA][NA+1], geometry, p, traces, q, b, metric
  static constexpr int SM_W = NA * (NA + 1) + GEO_STRIDE + NP + (DIM + 1) * Dims<DIM, K>::NF + DIM * NP + NA + DIM * DIM;
  static constexpr int WPB = SM_W * 8 * 4 <= 46 * 1024 ? 4 : (SM_W * 8 * 2 <= 46 * 1024 ? 2 : 1);
  static constexpr int NT = 32 * WPB;
  // CTAs per SM the registers are budgeted for (the shared memory admits at least this many)
  static constexpr int MINB = WPB == 4 ? 3 : 2;
};

// One warp per element (WPB independent warps per CTA, warp-stride over the elements), all
// synchronisation by __syncwarp, so many elements are in flight per SM.
template <int DIM, int K>
__global__ void __launch_bounds__(PostCfg<DIM, K>::NT, PostCfg<DIM, K>::MINB) post_kernel(DevMesh mesh, Tabs T, PostTabs P,
                                                                   const double* __restrict__ u,
                                                                   const double* __restrict__ lam,
                                                                   double* __restrict__ pstar) {
  using D = Dims<DIM, K>;
  using C = PostCfg<DIM, K>;
  constexpr int NP = C::NP, NF = D::NF, NFC = D::NFC, N = D::N, NP1 = C::NP1, NA = C::NA;
  __shared__ double smem[C::WPB][C::SM_W];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  double(*A)[NA + 1] = reinterpret_cast<double(*)[NA + 1]>(smem[w]);
  double* g = smem[w] + NA * (NA + 1);
  double* p = g + GEO_STRIDE;
  double* lf = p + NP;
  double* q = lf + NFC * NF;
  double* b = q + DIM * NP;
  double* gm = b + NA;
  const int64_t nw = (int64_t)gridDim.x * C::WPB;
  for (int64_t e = (int64_t)blockIdx.x * C::WPB + w; e < mesh.ne; e += nw) {
    for (int t = lane; t < GEO_STRIDE; t += 32) g[t] = mesh.geo[e * GEO_STRIDE + t];
    for (int t = lane; t < NP; t += 32) p[t] = u[e * N + t];
    for (int t = lane; t < NFC * NF; t += 32) {
      const int f = mesh.elem_face[e * NFC + t / NF];
      lf[t] = lam[(int64_t)f * NF + t % NF];
    }
    __syncwarp();
    if (lane < DIM * DIM) {
      const int r = lane / DIM, s = lane % DIM;
      double v = 0.0;
      for (int j = 0; j < DIM; ++j) v += g[1 + r * DIM + j] * g[1 + s * DIM + j];
      gm[lane] = v;
    }
    // discrete gradient q_h
    for (int t = lane; t < DIM * NP; t += 32) {
      const int j = t / NP, i = t % NP;
      double vol = 0.0;
      for (int r = 0; r < DIM; ++r) {
        double d = 0.0;
        for (int l = 0; l < NP; ++l) d += T.Dr[(r * NP + l) * NP + i] * p[l];
        vol += g[1 + r * DIM + j] * d;
      }
      double fc = 0.0;
      for (int f = 0; f < NFC; ++f) {
        double s = 0.0;
        for (int m = 0; m < NF; ++m) s += T.Ff[(f * NP + i) * NF + m] * lf[f * NF + m];
        fc += g[D::ON + f * DIM + j] * g[D::OJF + f] * s;
      }
      q[t] = fc / g[0] - vol;
    }
    __syncwarp();
    // right-hand side and the lower triangle of A' (modes 1..NP1-1)
    for (int t = lane; t < NA; t += 32) {
      double s = 0.0;
      for (int j = 0; j < DIM; ++j)
        for (int r = 0; r < DIM; ++r) {
          double d = 0.0;
          for (int l = 0; l < NP; ++l) d += P.E1[(r * NP1 + t + 1) * NP + l] * q[j * NP + l];
          s += g[1 + r * DIM + j] * d;
        }
      b[t] = s;
    }
    for (int t = lane; t < NA * (NA + 1) / 2; t += 32) {
      // t -> (i, l), l <= i, row by row
      int i = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
      while ((i + 1) * (i + 2) / 2 <= t) ++i;
      while (i * (i + 1) / 2 > t) --i;
      const int l = t - i * (i + 1) / 2;
      double s = 0.0;
#pragma unroll
      for (int rs = 0; rs < DIM * DIM; ++rs) s += gm[rs] * P.K1[(rs * NP1 + i + 1) * NP1 + l + 1];
      A[i][l] = s;
    }
    __syncwarp();
    // Cholesky A' = L L^T in place (lower triangle)
    for (int c = 0; c < NA; ++c) {
      const double dc = sqrt(A[c][c]);
      __syncwarp();
      if (lane == 0) A[c][c] = dc;
      for (int i = c + 1 + lane; i < NA; i += 32) A[i][c] /= dc;
      __syncwarp();
      for (int i = c + 1; i < NA; ++i)
        for (int l = c + 1 + lane; l <= i; l += 32) A[i][l] -= A[i][c] * A[l][c];
      __syncwarp();
    }
    // L y = b, then L^T c' = y (b is overwritten)
    for (int i = 0; i < NA; ++i) {
      double s = 0.0;
      for (int l = lane; l < i; l += 32) s += A[i][l] * b[l];
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      const double bi = (b[i] - s) / A[i][i];
      __syncwarp();
      if (lane == 0) b[i] = bi;
      __syncwarp();
    }
    for (int i = NA - 1; i >= 0; --i) {
      double s = 0.0;
      for (int l = i + 1 + lane; l < NA; l += 32) s += A[l][i] * b[l];
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      const double bi = (b[i] - s) / A[i][i];
      __syncwarp();
      if (lane == 0) b[i] = bi;
      __syncwarp();
    }
    for (int t = lane; t < NP1; t += 32) pstar[e * NP1 + t] = t == 0 ? p[0] : b[t - 1];
    __syncwarp();
  }
}

}  // namespace hdg
