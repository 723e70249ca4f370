// Block ILU(0) of the assembled trace system (Sec. 2.4: the paper's GMRES preconditioner).
// One block row per interior face (N_f x N_f blocks, N_f <= 32), the pattern of the face
// adjacency (faces sharing an element), rows in increasing face id. The factorisation and the
// two block substitutions run one warp per block row, level by level: a level holds the rows
// whose lower (forward) or upper (backward) neighbours are all in earlier levels.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace hdg {

struct BiluDev {
  int Nf;
  const int32_t* rowface;   // [nr] face of each block row
  const int32_t* rptr;      // [nr + 1] block row pointers
  const int32_t* col;       // [nnzb] block column (row index), ascending per row
  const int32_t* dpos;      // [nr] position of the diagonal block
  const int32_t* uptr;      // [nnzb + 1] updates triggered by a lower block (factorisation)
  const int2* upd;          // (q, t): A_t -= L_p A_q
  double* val;              // [nnzb][Nf][Nf]: A, then L (below the diagonal) and U
  double* dinv;             // [nr][Nf][Nf] inverses of the diagonal blocks of U
};

// A_p = sgn sum over the (one or two) elements holding both faces of the block of S_K
static __global__ void bilu_assemble_kernel(int64_t nnzb, int Nf, int m, const int32_t* __restrict__ ce,
                                            const int8_t* __restrict__ ca, const int8_t* __restrict__ cb,
                                            const double* __restrict__ S, double sgn, double* __restrict__ val) {
  const int64_t nb2 = (int64_t)Nf * Nf;
  const int64_t n = nnzb * nb2;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = t / nb2;
    const int rr = (int)((t % nb2) / Nf), cc = (int)(t % Nf);
    double v = 0.0;
    for (int s = 0; s < 2; ++s) {
      const int32_t e = ce[2 * p + s];
      if (e < 0) continue;
      const int a = ca[2 * p + s], b = cb[2 * p + s];
      v += S[(int64_t)e * m * m + (int64_t)(a * Nf + rr) * m + (b * Nf + cc)];
    }
    val[t] = sgn * v;
  }
}

// C = A B for Nf x Nf blocks, the warp's lanes over the entries of C
__device__ __forceinline__ void bilu_warp_gemm(int Nf, const double* A, const double* B, double* C, int lane) {
  for (int e = lane; e < Nf * Nf; e += 32) {
    const int r = e / Nf, c = e % Nf;
    double v = 0.0;
    for (int k = 0; k < Nf; ++k) v += A[r * Nf + k] * B[k * Nf + c];
    C[e] = v;
  }
}

// One level of the factorisation: warp w handles row rows[w]. For each lower block p (in
// increasing column order): L_p = A_p U_kk^{-1}, then A_t -= L_p A_q for its updates; last, the
// inverse of the diagonal block by Gauss-Jordan with partial pivoting (a zero pivot sets err).
static __global__ void __launch_bounds__(128) bilu_factor_kernel(BiluDev d, const int32_t* __restrict__ rows, int nrows,
                                                                int* __restrict__ err) {
  extern __shared__ double bsm[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int Nf = d.Nf, nb2 = Nf * Nf;
  double* Lb = bsm + wid * (nb2 + 2 * nb2);   // [Nf][Nf] L block, then [Nf][2 Nf] Gauss-Jordan
  double* G = Lb + nb2;
  const int w = blockIdx.x * 4 + wid;
  if (w >= nrows) return;
  const int r = rows[w];
  for (int p = d.rptr[r]; p < d.dpos[r]; ++p) {
    const int k = d.col[p];
    double* Ap = d.val + (int64_t)p * nb2;
    bilu_warp_gemm(Nf, Ap, d.dinv + (int64_t)k * nb2, Lb, lane);
    __syncwarp();
    for (int e = lane; e < nb2; e += 32) Ap[e] = Lb[e];
    for (int u = d.uptr[p]; u < d.uptr[p + 1]; ++u) {
      const int2 qt = d.upd[u];
      const double* Aq = d.val + (int64_t)qt.x * nb2;
      double* At = d.val + (int64_t)qt.y * nb2;
      for (int e = lane; e < nb2; e += 32) {
        const int rr = e / Nf, cc = e % Nf;
        double v = 0.0;
        for (int kk = 0; kk < Nf; ++kk) v += Lb[rr * Nf + kk] * Aq[kk * Nf + cc];
        At[e] -= v;
      }
    }
    __syncwarp();
  }
  // [U_rr | I] -> [I | U_rr^{-1}]
  const double* D = d.val + (int64_t)d.dpos[r] * nb2;
  for (int e = lane; e < 2 * nb2; e += 32) {
    const int rr = e / (2 * Nf), cc = e % (2 * Nf);
    G[e] = cc < Nf ? D[rr * Nf + cc] : (cc - Nf == rr ? 1.0 : 0.0);
  }
  __syncwarp();
  for (int j = 0; j < Nf; ++j) {
    // pivot row: the largest |G[i][j]|, i >= j
    double best = -1.0;
    int bi = j;
    for (int i = j + lane; i < Nf; i += 32) {
      const double a = fabs(G[i * 2 * Nf + j]);
      if (a > best) { best = a; bi = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (!(best > 0.0)) {
      if (lane == 0) atomicExch(err, 1);
      return;
    }
    if (bi != j)
      for (int c = lane; c < 2 * Nf; c += 32) {
        const double t = G[j * 2 * Nf + c];
        G[j * 2 * Nf + c] = G[bi * 2 * Nf + c];
        G[bi * 2 * Nf + c] = t;
      }
    __syncwarp();
    const double inv = 1.0 / G[j * 2 * Nf + j];
    __syncwarp();
    for (int c = lane; c < 2 * Nf; c += 32) G[j * 2 * Nf + c] *= inv;
    __syncwarp();
    for (int i = 0; i < Nf; ++i) {
      if (i == j) continue;
      const double f = G[i * 2 * Nf + j];
      __syncwarp();
      for (int c = lane; c < 2 * Nf; c += 32) G[i * 2 * Nf + c] -= f * G[j * 2 * Nf + c];
      __syncwarp();
    }
  }
  double* Di = d.dinv + (int64_t)r * nb2;
  for (int e = lane; e < nb2; e += 32) Di[e] = G[(e / Nf) * 2 * Nf + Nf + e % Nf];
}

// forward substitution, one level: y_r = b_r - sum_{p < diag} L_p y_col(p) (face-major vectors)
static __global__ void __launch_bounds__(128) bilu_fwd_kernel(BiluDev d, const int32_t* __restrict__ rows, int nrows,
                                                             const double* __restrict__ b, double* __restrict__ y) {
  const int lane = threadIdx.x & 31;
  const int w = blockIdx.x * 4 + (threadIdx.x >> 5);
  if (w >= nrows) return;
  const int r = rows[w], Nf = d.Nf, nb2 = Nf * Nf;
  const int64_t f = d.rowface[r];
  double s = lane < Nf ? b[f * Nf + lane] : 0.0;
  for (int p = d.rptr[r]; p < d.dpos[r]; ++p) {
    const double* Lp = d.val + (int64_t)p * nb2;
    const double* yk = y + (int64_t)d.rowface[d.col[p]] * Nf;
    if (lane < Nf)
      for (int c = 0; c < Nf; ++c) s -= Lp[lane * Nf + c] * yk[c];
  }
  if (lane < Nf) y[f * Nf + lane] = s;
}

// backward substitution, one level: z_r = U_rr^{-1} (y_r - sum_{p > diag} U_p z_col(p))
static __global__ void __launch_bounds__(128) bilu_bwd_kernel(BiluDev d, const int32_t* __restrict__ rows, int nrows,
                                                             const double* __restrict__ y, double* __restrict__ z) {
  const int lane = threadIdx.x & 31;
  const int w = blockIdx.x * 4 + (threadIdx.x >> 5);
  if (w >= nrows) return;
  const int r = rows[w], Nf = d.Nf, nb2 = Nf * Nf;
  const int64_t f = d.rowface[r];
  double s = lane < Nf ? y[f * Nf + lane] : 0.0;
  for (int p = d.dpos[r] + 1; p < d.rptr[r + 1]; ++p) {
    const double* Up = d.val + (int64_t)p * nb2;
    const double* zj = z + (int64_t)d.rowface[d.col[p]] * Nf;
    if (lane < Nf)
      for (int c = 0; c < Nf; ++c) s -= Up[lane * Nf + c] * zj[c];
  }
  const double* Di = d.dinv + (int64_t)r * nb2;
  double v = 0.0;
  for (int c = 0; c < Nf; ++c) {
    const double sc = __shfl_sync(0xffffffffu, s, c);
    if (lane < Nf) v += Di[lane * Nf + c] * sc;
  }
  if (lane < Nf) z[f * Nf + lane] = v;
}

// out = sum_j y_j V_j (j < k), the Krylov combination before the preconditioner
static __global__ void bilu_vcombine_kernel(int64_t n, int k, const double* __restrict__ V, const double* __restrict__ y,
                                            double* __restrict__ out) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    double v = 0.0;
    for (int j = 0; j < k; ++j) v += y[j] * V[(int64_t)j * n + t];
    out[t] = v;
  }
}

// x += z on the entries with mask != 0
static __global__ void bilu_add_masked_kernel(int64_t n, const uint8_t* __restrict__ mask, const double* __restrict__ z,
                                              double* __restrict__ x) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    if (mask[t]) x[t] += z[t];
}

}  // namespace hdg
