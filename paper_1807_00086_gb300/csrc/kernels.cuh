// Device kernels of the FP64 HDG hot path (sm_103a).
//
// Per element K with affine map x = X0 + J xi, |det J| = dJ, the acoustic local blocks
// are (Sec. 2.4, Eq. LS, acoustic specialisation of Eqs. eq:HDG_linelas1-5):
//   A_K = [ a dJ I + tau sum_f E_f    Dx_1 .. Dx_d ]      a = alpha/(rho c^2)
//         [ -Dx_j^T                   b dJ I       ]      b = alpha rho
//   B_K: p rows -tau F_f, v_j rows n_fj F_f;   C_K = [tau F_f^T, n_fj F_f^T];
//   D_K = -tau J_f I per face,
// with Dx_j = dJ sum_r Jinv[r][j] Dr_r, F_f = J_f Ff_f, E_f = J_f Ff_f Ff_f^T from the
// reference tables. The diagonal velocity block is eliminated analytically, leaving the
// SPD pressure block
//   H = a dJ I + tau sum_f J_f E^_f + (dJ/b) sum_{r,s} (Jinv Jinv^T)_{rs} Dr_r Dr_s^T,
// so A_K^{-1} costs one H^{-1} mat-vec plus derivative-table products, and
//   S_K = Bt^T H^{-1} Bt + D_K - (1/(b dJ)) [J_f J_g (n_f . n_g) Ff_f^T Ff_g]_{fg},
//   Bt_f = -J_f (tau Ff_f + (1/b) sum_r (n_f . Jinv[r]) Dr_r Ff_f).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "mesh.h"

namespace hdg {

struct Tabs {
  const double *Dr, *Ff, *Ef, *Trs, *DFrf, *Pfg;
};

struct DevMesh {
  int64_t ne, nf;
  const double* geo;
  const double* rho;
  const double* c;
  const int32_t* elem_face;
  const int32_t* face_slot;
  const int32_t* face_bnd;
};

template <int DIM, int K>
struct Dims {
  static constexpr int NP = (DIM == 2) ? (K + 1) * (K + 2) / 2 : (K + 1) * (K + 2) * (K + 3) / 6;
  static constexpr int NF = (DIM == 2) ? (K + 1) : (K + 1) * (K + 2) / 2;
  static constexpr int NFC = DIM + 1;
  static constexpr int N = NFC * NP;
  static constexpr int M = NFC * NF;
  static constexpr int OJF = 1 + DIM * DIM;
  static constexpr int ON = 1 + DIM * DIM + DIM + 1;
};

// ---------------------------------------------------------------- condensation (a)(b)(c)
// One CTA per element: assemble H, Cholesky H = L L^T, W = L^{-1} Bt, S = W^T W + ...,
// H^{-1} = L^{-T} L^{-1}. Writes S [ne][M][M] and Hinv [ne][NP][NP].
template <int DIM, int K, int NT>
__global__ void __launch_bounds__(NT) condense_kernel(DevMesh mesh, Tabs T, double alpha, double tau,
                                                      double* __restrict__ S, double* __restrict__ Hinv,
                                                      int* __restrict__ err) {
  using D = Dims<DIM, K>;
  constexpr int NP = D::NP, NF = D::NF, M = D::M, NFC = D::NFC;
  __shared__ double H[NP * NP];
  __shared__ double W[NP * M];
  __shared__ double Li[NP * NP];
  __shared__ double g[GEO_STRIDE];
  __shared__ double Grs[DIM * DIM], Bfr[NFC * DIM], nn[NFC * NFC];
  const int64_t e = blockIdx.x;
  const int tid = threadIdx.x;
  if (tid < GEO_STRIDE) g[tid] = mesh.geo[e * GEO_STRIDE + tid];
  __syncthreads();
  const double dJ = g[0];
  const double rho = mesh.rho[e], cc = mesh.c[e];
  const double a = alpha / (rho * cc * cc), b = alpha * rho;
  if (tid < DIM * DIM) {
    int r = tid / DIM, s = tid % DIM;
    double v = 0.0;
    for (int j = 0; j < DIM; ++j) v += g[1 + r * DIM + j] * g[1 + s * DIM + j];
    Grs[tid] = v;
  } else if (tid < DIM * DIM + NFC * DIM) {
    int t = tid - DIM * DIM, f = t / DIM, r = t % DIM;
    double v = 0.0;
    for (int j = 0; j < DIM; ++j) v += g[D::ON + f * DIM + j] * g[1 + r * DIM + j];
    Bfr[t] = v;
  } else if (tid < DIM * DIM + NFC * DIM + NFC * NFC) {
    int t = tid - DIM * DIM - NFC * DIM, f = t / NFC, h = t % NFC;
    double v = 0.0;
    for (int j = 0; j < DIM; ++j) v += g[D::ON + f * DIM + j] * g[D::ON + h * DIM + j];
    nn[t] = v;
  }
  __syncthreads();
  for (int idx = tid; idx < NP * NP; idx += NT) {
    const int i = idx / NP, l = idx % NP;
    double v = (i == l) ? a * dJ : 0.0;
    double fe = 0.0;
    for (int f = 0; f < NFC; ++f) fe += g[D::OJF + f] * T.Ef[(f * NP + i) * NP + l];
    double dd = 0.0;
    for (int rs = 0; rs < DIM * DIM; ++rs) dd += Grs[rs] * T.Trs[(rs * NP + i) * NP + l];
    H[idx] = v + tau * fe + (dJ / b) * dd;
    Li[idx] = (i == l) ? 1.0 : 0.0;
  }
  for (int idx = tid; idx < NP * M; idx += NT) {
    const int i = idx / M, col = idx % M, f = col / NF, mm = col % NF;
    double v = tau * T.Ff[(f * NP + i) * NF + mm];
    double d2 = 0.0;
    for (int r = 0; r < DIM; ++r) d2 += Bfr[f * DIM + r] * T.DFrf[((r * NFC + f) * NP + i) * NF + mm];
    W[idx] = -g[D::OJF + f] * (v + d2 / b);
  }
  __syncthreads();
  // Cholesky, right-looking, lower triangle in place
  for (int j = 0; j < NP; ++j) {
    if (tid == 0) {
      double d = H[j * NP + j];
      if (!(d > 0.0)) { atomicExch(err, 1); d = 1.0; }
      H[j * NP + j] = sqrt(d);
    }
    __syncthreads();
    for (int i = j + 1 + tid; i < NP; i += NT) H[i * NP + j] /= H[j * NP + j];
    __syncthreads();
    const int w = NP - j - 1;
    for (int idx = tid; idx < w * w; idx += NT) {
      const int i = j + 1 + idx / w, l = j + 1 + idx % w;
      if (l <= i) H[i * NP + l] -= H[i * NP + j] * H[l * NP + j];
    }
    __syncthreads();
  }
  // forward substitution, one column per thread: W <- L^{-1} Bt, Li <- L^{-1}
  for (int col = tid; col < M + NP; col += NT) {
    if (col < M) {
      for (int i = 0; i < NP; ++i) {
        double s = W[i * M + col];
        for (int l = 0; l < i; ++l) s -= H[i * NP + l] * W[l * M + col];
        W[i * M + col] = s / H[i * NP + i];
      }
    } else {
      const int c2 = col - M;
      for (int i = c2; i < NP; ++i) {
        double s = (i == c2) ? 1.0 : 0.0;
        for (int l = c2; l < i; ++l) s -= H[i * NP + l] * Li[l * NP + c2];
        Li[i * NP + c2] = s / H[i * NP + i];
      }
    }
  }
  __syncthreads();
  double* Se = S + e * (int64_t)(M * M);
  const double ib = 1.0 / (b * dJ);
  for (int idx = tid; idx < M * M; idx += NT) {
    const int ra = idx / M, cb = idx % M;
    const int f = ra / NF, aa = ra % NF, h = cb / NF, bb = cb % NF;
    double s = 0.0;
    for (int i = 0; i < NP; ++i) s += W[i * M + ra] * W[i * M + cb];
    if (ra == cb) s -= tau * g[D::OJF + f];
    s -= ib * g[D::OJF + f] * g[D::OJF + h] * nn[f * NFC + h] * T.Pfg[((f * NFC + h) * NF + aa) * NF + bb];
    Se[idx] = s;
  }
  double* He = Hinv + e * (int64_t)(NP * NP);
  for (int idx = tid; idx < NP * NP; idx += NT) {
    const int i = idx / NP, l = idx % NP;
    const int q0 = i > l ? i : l;
    double s = 0.0;
    for (int q = q0; q < NP; ++q) s += Li[q * NP + i] * Li[q * NP + l];
    He[idx] = s;
  }
}

// Jacobi preconditioner of -K: dinv = -1 / (sum over the face's slots of diag S_K).
template <int DIM, int K>
__global__ void diag_kernel(DevMesh mesh, const double* __restrict__ S, double* __restrict__ dinv) {
  using D = Dims<DIM, K>;
  constexpr int NF = D::NF, M = D::M;
  const int64_t n = mesh.nf * NF;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t f = t / NF;
    const int mm = (int)(t % NF);
    double d = 0.0;
    if (mesh.face_bnd[f] < 0) {
      for (int s = 0; s < 2; ++s) {
        const int64_t slot = mesh.face_slot[2 * f + s];
        const int64_t e = slot / D::NFC;
        const int r = (int)(slot % D::NFC) * NF + mm;
        d += S[e * (int64_t)(M * M) + (int64_t)r * M + r];
      }
      dinv[t] = -1.0 / d;
    } else {
      dinv[t] = 0.0;
    }
  }
}

// ---------------------------------------------------------------- element-local solves
// MODE 0 (condensed rhs): out = gslot [ne][M] = C_K A_K^{-1} (F_K - B_K lamD_K)
// MODE 1 (recovery):      out = u     [ne][N] = A_K^{-1} (F_K - B_K lam_K)
// F_K is F[e] when hist == nullptr, else alpha Mw_K hist[e] + r(t) sum_src phi(x_s).
template <int DIM, int K, int MODE, int NT>
__global__ void __launch_bounds__(NT) local_kernel(DevMesh mesh, Tabs T, const double* __restrict__ Hinv,
                                                   double alpha, double tau, const double* __restrict__ F,
                                                   const double* __restrict__ hist, const int32_t* __restrict__ src_ptr,
                                                   const double* __restrict__ src_phi, double src_rt,
                                                   const double* __restrict__ lam, double* __restrict__ out) {
  using D = Dims<DIM, K>;
  constexpr int NP = D::NP, NF = D::NF, M = D::M, NFC = D::NFC, N = D::N;
  __shared__ double g[GEO_STRIDE];
  __shared__ double ll[M];
  __shared__ double Fl[NFC * NP];
  __shared__ double Fu[N];          // p block then v blocks
  __shared__ double Tr[DIM * NP];
  __shared__ double rp[NP], pp[NP];
  __shared__ double qd[DIM * NP];
  __shared__ double vv[DIM * NP];
  const int64_t e = blockIdx.x;
  const int tid = threadIdx.x;
  if (tid < GEO_STRIDE) g[tid] = mesh.geo[e * GEO_STRIDE + tid];
  for (int t = tid; t < M; t += NT) {
    const int f = mesh.elem_face[e * NFC + t / NF];
    const bool use = (MODE == 1) || (mesh.face_bnd[f] >= 0);
    ll[t] = (use && lam) ? lam[(int64_t)f * NF + t % NF] : 0.0;
  }
  __syncthreads();
  const double dJ = g[0];
  const double rho = mesh.rho[e], cc = mesh.c[e];
  const double b = alpha * rho;
  for (int t = tid; t < NFC * NP; t += NT) {
    const int f = t / NP, i = t % NP;
    double s = 0.0;
    for (int mm = 0; mm < NF; ++mm) s += T.Ff[(f * NP + i) * NF + mm] * ll[f * NF + mm];
    Fl[t] = s;
  }
  __syncthreads();
  for (int t = tid; t < N; t += NT) {
    const int comp = t / NP, i = t % NP;
    double v;
    if (hist) {
      v = (comp == 0 ? alpha * dJ / (rho * cc * cc) : alpha * rho * dJ) * hist[e * N + t];
      if (comp == 0 && src_ptr)
        for (int s = src_ptr[e]; s < src_ptr[e + 1]; ++s) v += src_rt * src_phi[(int64_t)s * NP + i];
    } else {
      v = F[e * N + t];
    }
    double bl = 0.0;
    if (comp == 0) {
      for (int f = 0; f < NFC; ++f) bl += g[D::OJF + f] * Fl[f * NP + i];
      v += tau * bl;
    } else {
      for (int f = 0; f < NFC; ++f) bl += g[D::ON + f * DIM + comp - 1] * g[D::OJF + f] * Fl[f * NP + i];
      v -= bl;
    }
    Fu[t] = v;
  }
  __syncthreads();
  for (int t = tid; t < DIM * NP; t += NT) {
    const int r = t / NP, l = t % NP;
    double s = 0.0;
    for (int j = 0; j < DIM; ++j) s += g[1 + r * DIM + j] * Fu[(j + 1) * NP + l];
    Tr[t] = s;
  }
  __syncthreads();
  for (int i = tid; i < NP; i += NT) {
    double s = 0.0;
    for (int r = 0; r < DIM; ++r)
      for (int l = 0; l < NP; ++l) s += T.Dr[(r * NP + i) * NP + l] * Tr[r * NP + l];
    rp[i] = Fu[i] - s / b;
  }
  __syncthreads();
  const double* He = Hinv + e * (int64_t)(NP * NP);
  for (int i = tid; i < NP; i += NT) {
    double s = 0.0;
    for (int l = 0; l < NP; ++l) s += He[i * NP + l] * rp[l];
    pp[i] = s;
  }
  __syncthreads();
  for (int t = tid; t < DIM * NP; t += NT) {
    const int r = t / NP, i = t % NP;
    double s = 0.0;
    for (int l = 0; l < NP; ++l) s += T.Dr[(r * NP + l) * NP + i] * pp[l];
    qd[t] = s;
  }
  __syncthreads();
  for (int t = tid; t < DIM * NP; t += NT) {
    const int j = t / NP, i = t % NP;
    double s = 0.0;
    for (int r = 0; r < DIM; ++r) s += g[1 + r * DIM + j] * qd[r * NP + i];
    vv[t] = Fu[(j + 1) * NP + i] / (b * dJ) + s / b;
  }
  __syncthreads();
  if (MODE == 1) {
    for (int t = tid; t < N; t += NT) out[e * N + t] = (t < NP) ? pp[t] : vv[t - NP];
  } else {
    // reuse Fl as w_f = tau p + sum_j n_fj v_j per face
    for (int t = tid; t < NFC * NP; t += NT) {
      const int f = t / NP, i = t % NP;
      double s = tau * pp[i];
      for (int j = 0; j < DIM; ++j) s += g[D::ON + f * DIM + j] * vv[j * NP + i];
      Fl[t] = s;
    }
    __syncthreads();
    for (int t = tid; t < M; t += NT) {
      const int f = t / NF, mm = t % NF;
      double s = 0.0;
      for (int i = 0; i < NP; ++i) s += T.Ff[(f * NP + i) * NF + mm] * Fl[f * NP + i];
      out[e * M + t] = g[D::OJF + f] * s;
    }
  }
}

// ---------------------------------------------------------------- matrix-free trace apply (d)
// zslot[e][r] = sum_c S_K[r][c] x_K[c], x gathered from faces (boundary faces read as 0).
// S_K is symmetric, so thread r reads column r (coalesced across the element's threads).
template <int DIM, int K>
struct ApplyCfg {
  static constexpr int M = Dims<DIM, K>::M;
  static constexpr int EPB = (128 / M) > 0 ? (128 / M) : 1;
  static constexpr int NT = EPB * M;
};

template <int DIM, int K>
__global__ void __launch_bounds__(ApplyCfg<DIM, K>::NT) apply_kernel(DevMesh mesh, const double* __restrict__ S,
                                                                     const double* __restrict__ x,
                                                                     double* __restrict__ zslot,
                                                                     const int* __restrict__ done) {
  using D = Dims<DIM, K>;
  using C = ApplyCfg<DIM, K>;
  constexpr int NF = D::NF, M = D::M, NFC = D::NFC;
  if (done && *done) return;
  __shared__ double lx[C::EPB][M];
  const int el = threadIdx.x / M, r = threadIdx.x % M;
  const int64_t e = (int64_t)blockIdx.x * C::EPB + el;
  if (e < mesh.ne) {
    const int f = mesh.elem_face[e * NFC + r / NF];
    lx[el][r] = mesh.face_bnd[f] < 0 ? x[(int64_t)f * NF + r % NF] : 0.0;
  }
  __syncthreads();
  if (e < mesh.ne) {
    const double* Se = S + e * (int64_t)(M * M);
    double s = 0.0;
#pragma unroll 8
    for (int c = 0; c < M; ++c) s += Se[c * M + r] * lx[el][c];
    zslot[e * M + r] = s;
  }
}

// ---------------------------------------------------------------- face passes and PCG
struct CgScal {
  double rho[2];
  double bb, rr, tol2;
  int done, iters, pad0, pad1;
};

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic block sum of one value per thread (blockDim = 256); result in thread 0.
__device__ __forceinline__ double block_sum256(double v, double* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < 8; ++i) s += red[i];
  return s;
}

// Deterministic sum of a partials array (same order in every block); result in all threads.
__device__ __forceinline__ double reduce_partials(const double* __restrict__ part, int n, int stride, double* red) {
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v += part[(int64_t)i * stride];
  v = block_sum256(v, red);
  __shared__ double bc;
  if (threadIdx.x == 0) bc = v;
  __syncthreads();
  return bc;
}

// sum of the two slot contributions of each face entry (interior faces), 0 on boundary.
__device__ __forceinline__ double face_sum(const int32_t* __restrict__ face_slot, const double* __restrict__ zslot,
                                           int64_t f, int mm, int NF) {
  const int64_t s0 = face_slot[2 * f], s1 = face_slot[2 * f + 1];
  return zslot[s0 * NF + mm] + zslot[s1 * NF + mm];
}

// b = sum of slots (interior), 0 on boundary; optional scale.
__global__ void face_gather_kernel(int64_t nf, int NF, const int32_t* __restrict__ face_slot,
                                   const int32_t* __restrict__ face_bnd, const double* __restrict__ zslot,
                                   double scale, double* __restrict__ out) {
  const int64_t n = nf * NF;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t f = t / NF;
    const int mm = (int)(t % NF);
    out[t] = face_bnd[f] < 0 ? scale * face_sum(face_slot, zslot, f, mm, NF) : 0.0;
  }
}

// r = b - (-K) x0, z = Dinv r, p = z; partials (rz, rr, bb) per block.
__global__ void cg_init_kernel(int64_t nf, int NF, const int32_t* __restrict__ face_slot,
                               const int32_t* __restrict__ face_bnd, const double* __restrict__ zslot,
                               const double* __restrict__ bvec, const double* __restrict__ dinv, double* __restrict__ r,
                               double* __restrict__ z, double* __restrict__ p, double* __restrict__ part) {
  __shared__ double red[8];
  const int64_t n = nf * NF;
  double rz = 0, rr = 0, bb = 0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t f = t / NF;
    const int mm = (int)(t % NF);
    double rv = 0, zv = 0;
    if (face_bnd[f] < 0) {
      const double q = -face_sum(face_slot, zslot, f, mm, NF);
      const double bv = bvec[t];
      rv = bv - q;
      zv = dinv[t] * rv;
      bb += bv * bv;
    }
    r[t] = rv; z[t] = zv; p[t] = zv;
    rz += rv * zv; rr += rv * rv;
  }
  double s;
  s = block_sum256(rz, red); if (threadIdx.x == 0) part[blockIdx.x * 3 + 0] = s;
  s = block_sum256(rr, red); if (threadIdx.x == 0) part[blockIdx.x * 3 + 1] = s;
  s = block_sum256(bb, red); if (threadIdx.x == 0) part[blockIdx.x * 3 + 2] = s;
}

__global__ void cg_init_scalars(int nb, const double* __restrict__ part, double rtol, CgScal* sc) {
  __shared__ double red[8];
  const double rz = reduce_partials(part + 0, nb, 3, red);
  const double rr = reduce_partials(part + 1, nb, 3, red);
  const double bb = reduce_partials(part + 2, nb, 3, red);
  if (threadIdx.x == 0) {
    sc->rho[0] = rz; sc->rho[1] = 0; sc->bb = bb; sc->rr = rr;
    sc->tol2 = rtol * rtol * bb;
    sc->iters = 0;
    sc->done = (rr <= sc->tol2) ? 1 : 0;
  }
}

// q = (-K) p on faces; partial p.q
__global__ void cg_face_q_kernel(int64_t nf, int NF, const int32_t* __restrict__ face_slot,
                                 const int32_t* __restrict__ face_bnd, const double* __restrict__ zslot,
                                 const double* __restrict__ p, double* __restrict__ q, double* __restrict__ part,
                                 const CgScal* __restrict__ sc) {
  if (sc->done) return;
  __shared__ double red[8];
  const int64_t n = nf * NF;
  double pq = 0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t f = t / NF;
    const int mm = (int)(t % NF);
    double qv = 0;
    if (face_bnd[f] < 0) qv = -face_sum(face_slot, zslot, f, mm, NF);
    q[t] = qv;
    pq += p[t] * qv;
  }
  const double s = block_sum256(pq, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// alpha = rho/pq; x += alpha p; r -= alpha q; z = Dinv r; partials (rz, rr)
__global__ void cg_update_kernel(int64_t n, int nb, int parity, const double* __restrict__ part_pq,
                                 const double* __restrict__ p, const double* __restrict__ q,
                                 const double* __restrict__ dinv, double* __restrict__ x, double* __restrict__ r,
                                 double* __restrict__ z, double* __restrict__ part, const CgScal* __restrict__ sc) {
  if (sc->done) return;
  __shared__ double red[8];
  const double pq = reduce_partials(part_pq, nb, 1, red);
  const double al = sc->rho[parity] / pq;
  double rz = 0, rr = 0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const double pv = p[t];
    x[t] += al * pv;
    const double rv = r[t] - al * q[t];
    const double zv = dinv[t] * rv;
    r[t] = rv; z[t] = zv;
    rz += rv * zv; rr += rv * rv;
  }
  double s;
  s = block_sum256(rz, red); if (threadIdx.x == 0) part[blockIdx.x * 2 + 0] = s;
  s = block_sum256(rr, red); if (threadIdx.x == 0) part[blockIdx.x * 2 + 1] = s;
}

// beta = rz_new / rho; p = z + beta p; convergence test.
__global__ void cg_direction_kernel(int64_t n, int nb, int parity, int iter, const double* __restrict__ part,
                                    const double* __restrict__ z, double* __restrict__ p, CgScal* sc, int maxit) {
  if (sc->done) return;
  __shared__ double red[8];
  const double rz = reduce_partials(part + 0, nb, 2, red);
  const double rr = reduce_partials(part + 1, nb, 2, red);
  const bool conv = rr <= sc->tol2;
  const int it = iter + 1;  // iteration index from the host: no block reads what block 0 writes
  if (!conv && it < maxit) {
    const double be = rz / sc->rho[parity];
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
      p[t] = z[t] + be * p[t];
  }
  // every block has read sc->rho[parity] above; block 0 alone writes the other slot
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    sc->rho[parity ^ 1] = rz;
    sc->rr = rr;
    sc->iters = it;
    if (conv || it >= maxit) sc->done = conv ? 1 : 2;
  }
}

// out = sum_q c_q in_q (up to four inputs), elementwise.
__global__ void combine_kernel(int64_t n, double c0, const double* __restrict__ i0, double c1,
                               const double* __restrict__ i1, double c2, const double* __restrict__ i2, double c3,
                               const double* __restrict__ i3, double* __restrict__ out) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    double v = c0 * i0[t];
    if (i1) v += c1 * i1[t];
    if (i2) v += c2 * i2[t];
    if (i3) v += c3 * i3[t];
    out[t] = v;
  }
}

// boundary entries of lam <- coef[b] * fac (Dirichlet trace at the current time).
__global__ void dirichlet_kernel(int64_t nb, int NF, const int64_t* __restrict__ bnd_faces,
                                 const double* __restrict__ coef, double fac, double* __restrict__ lam) {
  const int64_t n = nb * NF;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = t / NF;
    lam[bnd_faces[b] * NF + t % NF] = coef ? coef[t] * fac : 0.0;
  }
}

// interior entries of x <- 0
__global__ void zero_interior_kernel(int64_t nf, int NF, const int32_t* __restrict__ face_bnd, double* __restrict__ x) {
  const int64_t n = nf * NF;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    if (face_bnd[t / NF] < 0) x[t] = 0.0;
}

// volume projection: u[e][c*NP+i] = sum_q w_q vals[e][q][c] phi_i(xi_q)  (mass = dJ I cancels dJ)
__global__ void project_volume_kernel(int64_t ne, int NP, int nq, int ncomp, const double* __restrict__ w,
                                      const double* __restrict__ phi, const double* __restrict__ vals,
                                      double* __restrict__ u) {
  const int64_t n = ne * ncomp * NP;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = t / (ncomp * NP);
    const int c = (int)((t / NP) % ncomp), i = (int)(t % NP);
    double s = 0.0;
    for (int q = 0; q < nq; ++q) s += w[q] * vals[(e * nq + q) * ncomp + c] * phi[q * NP + i];
    u[t] = s;
  }
}

}  // namespace hdg
