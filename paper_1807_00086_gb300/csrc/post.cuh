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
// One CTA per element (grid-stride), A' in shared memory, right-looking Cholesky, then the two
// triangular solves by one warp. FP64 throughout: the step runs once per output time.
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
  static constexpr int NT = 128;
};

template <int DIM, int K>
__global__ void __launch_bounds__(PostCfg<DIM, K>::NT) post_kernel(DevMesh mesh, Tabs T, PostTabs P,
                                                                   const double* __restrict__ u,
                                                                   const double* __restrict__ lam,
                                                                   double* __restrict__ pstar) {
  using D = Dims<DIM, K>;
  using C = PostCfg<DIM, K>;
  constexpr int NP = C::NP, NF = D::NF, NFC = D::NFC, N = D::N, NP1 = C::NP1, NA = C::NA, NT = C::NT;
  __shared__ double A[NA][NA + 1];
  __shared__ double g[GEO_STRIDE], p[NP], lf[NFC * NF], q[DIM * NP], b[NA], gm[DIM * DIM];
  const int tid = threadIdx.x;
  for (int64_t e = blockIdx.x; e < mesh.ne; e += gridDim.x) {
    if (tid < GEO_STRIDE) g[tid] = mesh.geo[e * GEO_STRIDE + tid];
    for (int t = tid; t < NP; t += NT) p[t] = u[e * N + t];
    for (int t = tid; t < NFC * NF; t += NT) {
      const int f = mesh.elem_face[e * NFC + t / NF];
      lf[t] = lam[(int64_t)f * NF + t % NF];
    }
    __syncthreads();
    if (tid < DIM * DIM) {
      const int r = tid / DIM, s = tid % DIM;
      double v = 0.0;
      for (int j = 0; j < DIM; ++j) v += g[1 + r * DIM + j] * g[1 + s * DIM + j];
      gm[tid] = v;
    }
    // discrete gradient q_h
    for (int t = tid; t < DIM * NP; t += NT) {
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
    __syncthreads();
    // right-hand side and the lower triangle of A' (modes 1..NP1-1)
    for (int t = tid; t < NA; t += NT) {
      double s = 0.0;
      for (int j = 0; j < DIM; ++j)
        for (int r = 0; r < DIM; ++r) {
          double d = 0.0;
          for (int l = 0; l < NP; ++l) d += P.E1[(r * NP1 + t + 1) * NP + l] * q[j * NP + l];
          s += g[1 + r * DIM + j] * d;
        }
      b[t] = s;
    }
    for (int t = tid; t < NA * NA; t += NT) {
      const int i = t / NA, l = t % NA;
      if (l > i) continue;
      double s = 0.0;
#pragma unroll
      for (int rs = 0; rs < DIM * DIM; ++rs) s += gm[rs] * P.K1[(rs * NP1 + i + 1) * NP1 + l + 1];
      A[i][l] = s;
    }
    __syncthreads();
    // Cholesky A' = L L^T in place (lower triangle)
    for (int c = 0; c < NA; ++c) {
      if (tid == 0) A[c][c] = sqrt(A[c][c]);
      __syncthreads();
      for (int i = c + 1 + tid; i < NA; i += NT) A[i][c] /= A[c][c];
      __syncthreads();
      const int nt = NA - c - 1;
      for (int t = tid; t < nt * nt; t += NT) {
        const int i = c + 1 + t / nt, l = c + 1 + t % nt;
        if (l <= i) A[i][l] -= A[i][c] * A[l][c];
      }
      __syncthreads();
    }
    // L y = b, then L^T c' = y, by warp 0 (b is overwritten)
    if (tid < 32) {
      for (int i = 0; i < NA; ++i) {
        double s = 0.0;
        for (int l = tid; l < i; l += 32) s += A[i][l] * b[l];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (tid == 0) b[i] = (b[i] - s) / A[i][i];
        __syncwarp();
      }
      for (int i = NA - 1; i >= 0; --i) {
        double s = 0.0;
        for (int l = i + 1 + tid; l < NA; l += 32) s += A[l][i] * b[l];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (tid == 0) b[i] = (b[i] - s) / A[i][i];
        __syncwarp();
      }
    }
    __syncthreads();
    for (int t = tid; t < NP1; t += NT) pstar[e * NP1 + t] = t == 0 ? p[0] : b[t - 1];
    __syncthreads();
  }
}

}  // namespace hdg
