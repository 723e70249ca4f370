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

#include <cuda_fp16.h>
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

// Point sources: CSR by element (ptr[e]..ptr[e+1]), per source the basis values at the
// point times its amplitude (phi), its right-hand-side column and its time delay; the
// Ricker wavelet r(t - delay) = (1 - 2a) exp(-a), a = (pi f0 (t - delay - t0))^2.
struct SrcArgs {
  const int32_t* ptr;
  const double* phi;
  const int32_t* col;
  const double* delay;
  double f0, t0, t;
};

__device__ __forceinline__ double ricker_at(const SrcArgs& s, int q) {
  const double x = 3.14159265358979323846 * s.f0 * (s.t - s.delay[q] - s.t0);
  const double a = x * x;
  return (1.0 - 2.0 * a) * exp(-a);
}

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

// Jacobi preconditioner: dinv = sgn / (sum over the face's slots of diag S_K), sgn = -1 for the
// acoustic convention (K negative definite), +1 for the elastic one (K positive definite).
template <class D>
__global__ void diag_kernel(DevMesh mesh, const double* __restrict__ S, double sgn, double* __restrict__ dinv) {
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
      dinv[t] = sgn / d;
    } else {
      dinv[t] = 0.0;
    }
  }
}

// ---------------------------------------------------------------- element-local solves
// MODE 0 (condensed rhs): out = gslot [ne][M] = C_K A_K^{-1} (F_K - B_K lamD_K)
// MODE 1 (recovery):      out = u     [ne][N] = A_K^{-1} (F_K - B_K lam_K)
// F_K is F[e] when hist == nullptr, else alpha Mw_K hist[e] + r(t) sum_src phi(x_s).
// EPB elements per CTA, one thread per (element, row i < NP); only three block-wide
// barriers, the rest of each element's work is row-local.
template <int DIM, int K>
struct LocalCfg {
  static constexpr int NP = Dims<DIM, K>::NP;
  static constexpr int EPB = NP <= 10 ? 16 : (NP <= 20 ? 8 : 4);
  static constexpr int NT = EPB * NP;
};

template <int DIM, int K, int MODE>
__global__ void __launch_bounds__(LocalCfg<DIM, K>::NT) local_kernel(DevMesh mesh, Tabs T, const double* __restrict__ Hinv,
                                                                    double alpha, double tau, const double* __restrict__ F,
                                                                    const double* __restrict__ hist, SrcArgs src,
                                                                    const double* __restrict__ lam, double* __restrict__ out) {
  using D = Dims<DIM, K>;
  using L = LocalCfg<DIM, K>;
  constexpr int NP = D::NP, NF = D::NF, M = D::M, NFC = D::NFC, N = D::N, EPB = L::EPB, NT = L::NT;
  __shared__ double g[EPB][GEO_STRIDE];
  __shared__ double ll[EPB][M];
  __shared__ double Tr[EPB][DIM * NP];   // reused for the face weights w_f in MODE 0
  __shared__ double rp[EPB][NP];
  __shared__ double pp[EPB][NP];
  __shared__ double co[EPB][2];          // b = alpha rho, a' = alpha dJ / (rho c^2) (hist mode)
  __shared__ int fuse[EPB][NFC];         // face contributes a trace (nonzero lam) to this element
  const int tid = threadIdx.x;
  const int64_t e0 = (int64_t)blockIdx.x * EPB;
  for (int t = tid; t < EPB * GEO_STRIDE; t += NT) {
    const int64_t e = e0 + t / GEO_STRIDE;
    g[t / GEO_STRIDE][t % GEO_STRIDE] = e < mesh.ne ? mesh.geo[e * GEO_STRIDE + t % GEO_STRIDE] : (t % GEO_STRIDE == 0 ? 1.0 : 0.0);
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
    ll[t / M][r] = v;
  }
  if (tid < EPB) {
    const int64_t e = e0 + tid;
    const double rho = e < mesh.ne ? mesh.rho[e] : 1.0, cc = e < mesh.ne ? mesh.c[e] : 1.0;
    co[tid][0] = alpha * rho;
    co[tid][1] = alpha / (rho * cc * cc);
  }
  __syncthreads();
  const int el = tid / NP, i = tid % NP;
  const int64_t e = e0 + el;
  const bool live = e < mesh.ne;
  const double* ge = g[el];
  const double dJ = ge[0];
  const double b = co[el][0];
  // row i of F~ for all components (+ the F^ lam face products it needs)
  double Fu[DIM + 1];
  {
    double Fl[NFC];
#pragma unroll
    for (int f = 0; f < NFC; ++f) {
      double s = 0.0;
      if (fuse[el][f])
        for (int mm = 0; mm < NF; ++mm) s += T.Ff[(f * NP + i) * NF + mm] * ll[el][f * NF + mm];
      Fl[f] = s;
    }
#pragma unroll
    for (int comp = 0; comp <= DIM; ++comp) {
      double v = 0.0;
      if (live) {
        if (hist) {
          const double sc = comp == 0 ? co[el][1] * dJ : b * dJ;
          v = sc * hist[e * N + comp * NP + i];
          if (comp == 0 && src.ptr)
            for (int q = src.ptr[e]; q < src.ptr[e + 1]; ++q) v += ricker_at(src, q) * src.phi[(int64_t)q * NP + i];
        } else {
          v = F[e * N + comp * NP + i];
        }
      }
      double bl = 0.0;
      if (comp == 0) {
#pragma unroll
        for (int f = 0; f < NFC; ++f) bl += ge[D::OJF + f] * Fl[f];
        v += tau * bl;
      } else {
#pragma unroll
        for (int f = 0; f < NFC; ++f) bl += ge[D::ON + f * DIM + comp - 1] * ge[D::OJF + f] * Fl[f];
        v -= bl;
      }
      Fu[comp] = v;
    }
  }
  // Tr[r][i] = sum_j Jinv[r][j] F~v_j[i]
#pragma unroll
  for (int r = 0; r < DIM; ++r) {
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < DIM; ++j) s += ge[1 + r * DIM + j] * Fu[j + 1];
    Tr[el][r * NP + i] = s;
  }
  __syncthreads();
  {
    double s = 0.0;
#pragma unroll
    for (int r = 0; r < DIM; ++r)
      for (int l = 0; l < NP; ++l) s += T.Dr[(r * NP + i) * NP + l] * Tr[el][r * NP + l];
    rp[el][i] = Fu[0] - s / b;
  }
  __syncthreads();
  {
    // p = H^{-1} rp; H^{-1} is symmetric, so row i is read as column i (coalesced)
    const double* He = Hinv + (live ? e : 0) * (int64_t)(NP * NP);
    double s = 0.0;
    for (int l = 0; l < NP; ++l) s += He[l * NP + i] * rp[el][l];
    pp[el][i] = s;
  }
  __syncthreads();
  double vv[DIM];
  {
    double qd[DIM];
#pragma unroll
    for (int r = 0; r < DIM; ++r) {
      double s = 0.0;
      for (int l = 0; l < NP; ++l) s += T.Dr[(r * NP + l) * NP + i] * pp[el][l];
      qd[r] = s;
    }
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      double s = 0.0;
#pragma unroll
      for (int r = 0; r < DIM; ++r) s += ge[1 + r * DIM + j] * qd[r];
      vv[j] = Fu[j + 1] / (b * dJ) + s / b;
    }
  }
  if (MODE == 1) {
    if (live) {
      out[e * N + i] = pp[el][i];
#pragma unroll
      for (int j = 0; j < DIM; ++j) out[e * N + (j + 1) * NP + i] = vv[j];
    }
    return;
  }
  // MODE 0: w_f[i] = tau p[i] + sum_j n_fj v_j[i]  (Tr reused: NFC*NP <= DIM*NP + NP)
  double* w = &Tr[el][0];
  __syncthreads();   // every thread is done reading Tr
#pragma unroll
  for (int f = 0; f < NFC; ++f) {
    double s = tau * pp[el][i];
#pragma unroll
    for (int j = 0; j < DIM; ++j) s += ge[D::ON + f * DIM + j] * vv[j];
    if (f < DIM) w[f * NP + i] = s;
    else rp[el][i] = s;                   // last face's weights live in rp (no longer needed)
  }
  __syncthreads();
  for (int t = tid; t < EPB * M; t += NT) {
    const int el2 = t / M, r = t % M, f = r / NF, mm = r % NF;
    const int64_t e2 = e0 + el2;
    if (e2 >= mesh.ne) continue;
    const double* wf = f < DIM ? &Tr[el2][f * NP] : &rp[el2][0];
    double s = 0.0;
    for (int q = 0; q < NP; ++q) s += T.Ff[(f * NP + q) * NF + mm] * wf[q];
    out[e2 * M + r] = g[el2][D::OJF + f] * s;
  }
}

// ---------------------------------------------------------------- matrix-free trace apply (d)
// zslot[e][r] = sum_c S_K[r][c] x_K[c], x gathered from faces (boundary faces read as 0).
// S_K is symmetric, so thread r reads column r (coalesced across the element's threads).
template <class L>
struct ApplyCfg {
  static constexpr int M = L::M;
  static constexpr int EPB = (128 / M) > 0 ? (128 / M) : 1;
  static constexpr int NT = EPB * M;
};

template <class D>
__global__ void __launch_bounds__(ApplyCfg<D>::NT) apply_kernel(DevMesh mesh, const double* __restrict__ S,
                                                                const double* __restrict__ x,
                                                                double* __restrict__ zslot,
                                                                const int* __restrict__ done) {
  using C = ApplyCfg<D>;
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

// Inner products of FP32 vectors, accurate to FP64 level but evaluated on the FP32 pipe
// (GB300's FP64 rate is 1/58 of FP32): each product is split exactly into p + e with an
// FMA, and the terms are accumulated in a compensated (s, c) float pair (TwoSum). Only
// the per-thread result is widened to FP64 for the block/grid reduction.
struct Acc2 {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float t = s + x;
    const float bb = t - s;
    c += (s - (t - bb)) + (x - bb);
    s = t;
  }
  __device__ __forceinline__ void dot(float a, float b) {
    const float p = a * b;
    c += fmaf(a, b, -p);
    add(p);
  }
  __device__ __forceinline__ void dot4(float4 a, float4 b) { dot(a.x, b.x); dot(a.y, b.y); dot(a.z, b.z); dot(a.w, b.w); }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

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
static __global__ void face_gather_kernel(int64_t nf, int NF, const int32_t* __restrict__ face_slot,
                                   const int32_t* __restrict__ face_bnd, const double* __restrict__ zslot,
                                   double scale, double* __restrict__ out) {
  const int64_t n = nf * NF;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t f = t / NF;
    const int mm = (int)(t % NF);
    out[t] = face_bnd[f] < 0 ? scale * face_sum(face_slot, zslot, f, mm, NF) : 0.0;
  }
}

// r = b - (sgn K) x0, z = Dinv r, p = z; partials (rz, rr, bb) per block.
static __global__ void cg_init_kernel(int64_t nf, int NF, double sgn, const int32_t* __restrict__ face_slot,
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
      const double q = sgn * face_sum(face_slot, zslot, f, mm, NF);
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

static __global__ void cg_init_scalars(int nb, const double* __restrict__ part, double rtol, CgScal* sc) {
  __shared__ double red[8];
  const double rz = reduce_partials(part + 0, nb, 3, red);
  const double rr = reduce_partials(part + 1, nb, 3, red);
  const double bb = reduce_partials(part + 2, nb, 3, red);
  if (threadIdx.x == 0) {
    sc->rho[0] = rz; sc->rho[1] = 0; sc->bb = bb; sc->rr = rr;
    sc->tol2 = rtol * rtol * bb;
    sc->iters = 0;
    // a zero right-hand side ends the solve here (its solution is zero on interior faces)
    sc->done = (bb == 0.0 || rr <= sc->tol2) ? 1 : 0;
  }
}

// q = (-K) p on faces (sgn = -1; +K for sgn = +1); partial p.q (NF compile-time)
template <class LD>
__global__ void __launch_bounds__(256) cg_face_q_kernel(int nf, double sgn, const int32_t* __restrict__ face_slot,
                                                        const int32_t* __restrict__ face_bnd,
                                                        const double* __restrict__ zslot, const double* __restrict__ p,
                                                        double* __restrict__ q, double* __restrict__ part,
                                                        const CgScal* __restrict__ sc) {
  constexpr int NF = LD::NF;
  if (sc->done) return;
  __shared__ double red[8];
  double pq = 0;
  for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < nf; f += gridDim.x * blockDim.x) {
    double qv[NF];
    if (face_bnd[f] < 0) {
      const double* s0 = zslot + (int64_t)face_slot[2 * f] * NF;
      const double* s1 = zslot + (int64_t)face_slot[2 * f + 1] * NF;
#pragma unroll
      for (int mm = 0; mm < NF; ++mm) qv[mm] = sgn * (s0[mm] + s1[mm]);
    } else {
#pragma unroll
      for (int mm = 0; mm < NF; ++mm) qv[mm] = 0.0;
    }
#pragma unroll
    for (int mm = 0; mm < NF; ++mm) {
      q[(int64_t)f * NF + mm] = qv[mm];
      pq += p[(int64_t)f * NF + mm] * qv[mm];
    }
  }
  const double s = block_sum256(pq, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// alpha = rho/pq; x += alpha p; r -= alpha q; z = Dinv r; partials (rz, rr)
static __global__ void cg_update_kernel(int64_t n, int nb, int parity, const double* __restrict__ part_pq,
                                 const double* __restrict__ p, const double* __restrict__ q,
                                 const double* __restrict__ dinv, double* __restrict__ x, double* __restrict__ r,
                                 double* __restrict__ z, double* __restrict__ part, const CgScal* __restrict__ sc) {
  if (sc->done) return;
  __shared__ double red[8];
  const double pq = reduce_partials(part_pq, nb, 1, red);
  const double al = sc->rho[parity] / pq;
  double rz = 0, rr = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (; t + 3 * stride < n; t += 4 * stride) {
    double pv[4], qv[4], xv[4], rv[4], dv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      pv[u] = p[t + u * stride]; qv[u] = q[t + u * stride]; xv[u] = x[t + u * stride];
      rv[u] = r[t + u * stride]; dv[u] = dinv[t + u * stride];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      x[t + u * stride] = xv[u] + al * pv[u];
      const double rn = rv[u] - al * qv[u];
      const double zn = dv[u] * rn;
      r[t + u * stride] = rn; z[t + u * stride] = zn;
      rz += rn * zn; rr += rn * rn;
    }
  }
  for (; t < n; t += stride) {
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

// beta = rz_new / rho; p = z + beta p; convergence test. iter >= 0: the iteration index from the
// host, h unused. iter < 0 (device-driven loop): block 0 counts the iterations in sc->iters and
// sets the loop condition h (continue while not done), also when the solve had already finished.
static __global__ void cg_direction_kernel(int64_t n, int nb, int parity, int iter, const double* __restrict__ part,
                                    const double* __restrict__ z, double* __restrict__ p, CgScal* sc, int maxit,
                                    cudaGraphConditionalHandle h) {
  if (sc->done) {
    if (iter < 0 && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(h, 0u);
    return;
  }
  __shared__ double red[8];
  const double rz = reduce_partials(part + 0, nb, 2, red);
  const double rr = reduce_partials(part + 1, nb, 2, red);
  const bool conv = rr <= sc->tol2;
  // with a host index no block reads what block 0 writes; on the device only block 0 uses it
  const int it = iter >= 0 ? iter + 1 : sc->iters + 1;
  if (!conv && (iter < 0 || it < maxit)) {
    const double be = rz / sc->rho[parity];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (; t + 3 * stride < n; t += 4 * stride) {
      double pv[4], zv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) { pv[u] = p[t + u * stride]; zv[u] = z[t + u * stride]; }
#pragma unroll
      for (int u = 0; u < 4; ++u) p[t + u * stride] = zv[u] + be * pv[u];
    }
    for (; t < n; t += stride) p[t] = z[t] + be * p[t];
  }
  // every block has read sc->rho[parity] above; block 0 alone writes the other slot
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    sc->rho[parity ^ 1] = rz;
    sc->rr = rr;
    sc->iters = it;
    const int done = conv ? 1 : (it >= maxit ? 2 : 0);
    if (done) sc->done = done;
    if (iter < 0) cudaGraphSetConditional(h, done ? 0u : 1u);
  }
}

// Least-squares initial guess over stored stage solutions. ring: [Q][n] contiguous.
// dots_ring_kernel: block partials of (v_i, w) for i < q and of (w, w), part[blk][q + 1].
static __global__ void dots_ring_kernel(int64_t n, int q, int64_t stride, const double* __restrict__ ring,
                                        const double* __restrict__ w, double* __restrict__ part) {
  __shared__ double red[8];
  double acc[9];
  for (int i = 0; i <= q; ++i) acc[i] = 0.0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const double wv = w[t];
    for (int i = 0; i < q; ++i) acc[i] += ring[i * stride + t] * wv;
    acc[q] += wv * wv;
  }
  for (int i = 0; i <= q; ++i) {
    const double s = block_sum256(acc[i], red);
    if (threadIdx.x == 0) part[blockIdx.x * (q + 1) + i] = s;
  }
}

static __global__ void dots_final_kernel(int nb, int q, const double* __restrict__ part, double* __restrict__ out) {
  __shared__ double red[8];
  for (int i = 0; i <= q; ++i) {
    const double s = reduce_partials(part + i, nb, q + 1, red);
    if (threadIdx.x == 0) out[i] = s;
  }
}

struct Coef8 {
  double c[8];
};

// out[t] = sum_i c_i ring[i][t] on interior trace entries (mask != 0); boundary entries untouched
static __global__ void lincomb_ring_kernel(int64_t n, int q, int64_t stride, const double* __restrict__ ring, Coef8 c,
                                           const uint8_t* __restrict__ mask, double* __restrict__ out) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    if (!mask[t]) continue;
    double s = 0.0;
    for (int i = 0; i < q; ++i) s += c.c[i] * ring[i * stride + t];
    out[t] = s;
  }
}

// out = sum_q c_q in_q (up to four inputs), elementwise.
static __global__ void combine_kernel(int64_t n, double c0, const double* __restrict__ i0, double c1,
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
static __global__ void dirichlet_kernel(int64_t nb, int NF, const int64_t* __restrict__ bnd_faces,
                                 const double* __restrict__ coef, double fac, double* __restrict__ lam) {
  const int64_t n = nb * NF;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = t / NF;
    lam[bnd_faces[b] * NF + t % NF] = coef ? coef[t] * fac : 0.0;
  }
}

// interior entries of x <- 0
static __global__ void zero_interior_kernel(int64_t nf, int NF, const int32_t* __restrict__ face_bnd, double* __restrict__ x) {
  const int64_t n = nf * NF;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    if (face_bnd[t / NF] < 0) x[t] = 0.0;
}

// volume projection: u[e][c*NP+i] = sum_q w_q vals[e][q][c] phi_i(xi_q)  (mass = dJ I cancels dJ)
static __global__ void project_volume_kernel(int64_t ne, int NP, int nq, int ncomp, const double* __restrict__ w,
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

namespace hdg {

// ================================================================ mixed precision (FP32 inner solve)
// S32: the upper triangle (row-major, c >= r) of every S_K rounded to FP32, stored for groups
// of 32 elements as [group][P4][32][4] floats, P4 = ceil(M(M+1)/2 / 4): one warp handles a
// group, lane = element, each lane reads float4s and the warp's loads are contiguous.
template <int DIM, int K>
struct Packed {
  static constexpr int M = Dims<DIM, K>::M;
  static constexpr int P = M * (M + 1) / 2;
  static constexpr int P4 = (P + 3) / 4;
};

__host__ __device__ constexpr int packed_index(int M, int r, int c) { return r * M - r * (r - 1) / 2 + (c - r); }

template <int DIM, int K>
__global__ void pack32_kernel(int64_t ne, const double* __restrict__ S, float* __restrict__ S32) {
  using PK = Packed<DIM, K>;
  constexpr int M = PK::M, P4 = PK::P4;
  const int64_t ngroups = (ne + 31) / 32;
  const int64_t n = ngroups * P4 * 32 * 4;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(t & 3);
    const int lane = (int)((t >> 2) & 31);
    const int64_t q = (t >> 7) % P4;
    const int64_t g = (t >> 7) / P4;
    const int64_t e = g * 32 + lane;
    const int p = (int)(q * 4 + j);
    float v = 0.f;
    if (e < ne && p < PK::P) {
      // invert the packed index: row r holds entries [packed_index(r, r), packed_index(r, M-1)]
      int r = 0;
      while (packed_index(M, r, M - 1) < p) ++r;
      const int c = r + (p - packed_index(M, r, r));
      v = (float)S[e * (int64_t)(M * M) + r * M + c];
    }
    S32[t] = v;
  }
}

// p.q of the Krylov iteration, formed inside the element apply: with q = sgn K p and K the
// sum of the element blocks, p.q = sgn sum_K p_K . (S_K p_K) (boundary entries of p are zero
// on both sides). Each 4-warp block writes its partial; the last block to finish (ticket
// counter, no waiting) sums the partials in index order and resets the counter.
// Launch timing on the device (also inside CUDA graphs): the first CTA to start lowers
// start_ns, the last CTA to finish (the one that sums the partials) adds the elapsed
// %globaltimer time to ms and counts the launch. Launches that return early (solve converged)
// are not counted.
struct DevTiming {
  unsigned long long start_ns;   // ULLONG_MAX between launches
  unsigned long long count;
  double ms;
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

struct PqOut {
  double* part;       // [gridDim.x] block partials
  unsigned* ticket;   // zero between launches
  double* pq;         // result
  float sgn;
  DevTiming* timing;  // may be null
};

__device__ __forceinline__ void timing_start(const PqOut& o) {
  if (o.timing && o.part && threadIdx.x == 0) atomicMin(&o.timing->start_ns, global_ns());
}

__device__ __forceinline__ void pq_epilogue(const PqOut& o, double v) {
  __shared__ double wsum[4];
  __shared__ bool last;
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) wsum[wid] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    o.part[blockIdx.x] = ((wsum[0] + wsum[1]) + (wsum[2] + wsum[3]));
    __threadfence();
    last = atomicAdd(o.ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double s = 0.0;
  for (unsigned i = threadIdx.x; i < gridDim.x; i += blockDim.x) s += __ldcg(o.part + i);
  s = warp_sum(s);
  if (lane == 0) wsum[wid] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    *o.pq = (double)o.sgn * ((wsum[0] + wsum[1]) + (wsum[2] + wsum[3]));
    *o.ticket = 0u;
    if (o.timing) {
      const unsigned long long t1 = global_ns();
      const unsigned long long t0 = *(volatile unsigned long long*)&o.timing->start_ns;
      if (t1 > t0) {
        o.timing->ms += 1e-6 * (double)(t1 - t0);
        o.timing->count += 1;
      }
      o.timing->start_ns = ~0ull;
    }
  }
}

// slot32 layout: [e][M] floats (element-major, like the FP64 slots); the warp transposes
// its 32 x M products through shared memory so that the stores are contiguous float4s.
template <int DIM, int K>
__global__ void __launch_bounds__(128, 4) apply32_kernel(int64_t ne, const int32_t* __restrict__ elem_face,
                                                      const int32_t* __restrict__ face_bnd,
                                                      const float* __restrict__ S32, const float* __restrict__ x,
                                                      float* __restrict__ slot, const int* __restrict__ done, PqOut pqo) {
  using D = Dims<DIM, K>;
  using PK = Packed<DIM, K>;
  constexpr int NF = D::NF, M = D::M, NFC = D::NFC, P4 = PK::P4;
  constexpr int MP = M + 1;   // padded row: conflict-free transposed writes
  __shared__ float tr[4][32 * MP];
  if (done && *done) return;
  timing_start(pqo);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t g0 = (int64_t)blockIdx.x * 4 + wid;
  const bool wact = g0 * 32 < ne;                 // the last block may hold idle warps
  const int64_t g = wact ? g0 : 0;
  const int64_t e = g0 * 32 + lane;
  float xl[M], y[M];
#pragma unroll
  for (int f = 0; f < NFC; ++f) {
    int fid = -1;
    if (e < ne) fid = elem_face[e * NFC + f];
    const bool use = fid >= 0 && face_bnd[fid] < 0;
#pragma unroll
    for (int mm = 0; mm < NF; ++mm) xl[f * NF + mm] = use ? x[(int64_t)fid * NF + mm] : 0.f;
  }
#pragma unroll
  for (int r = 0; r < M; ++r) y[r] = 0.f;
  const float4* Sg = reinterpret_cast<const float4*>(S32) + g * (int64_t)P4 * 32 + lane;
  float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int r = 0; r < M; ++r) {
#pragma unroll
    for (int c = r; c < M; ++c) {
      const int p = packed_index(M, r, c);
      if ((p & 3) == 0) v = __ldcs(Sg + (p >> 2) * 32);
      const float s = (p & 3) == 0 ? v.x : (p & 3) == 1 ? v.y : (p & 3) == 2 ? v.z : v.w;
      y[r] = fmaf(s, xl[c], y[r]);
      if (c != r) y[c] = fmaf(s, xl[r], y[c]);
    }
  }
  float* t = tr[wid];
#pragma unroll
  for (int r = 0; r < M; ++r) t[lane * MP + r] = y[r];
  __syncwarp();
  if (wact) {
    const int64_t nvalid = (ne - g * 32) < 32 ? (ne - g * 32) : 32;
    float* dst = slot + g * 32 * (int64_t)M;
    for (int idx = lane; idx < nvalid * M; idx += 32) dst[idx] = t[(idx / M) * MP + idx % M];
  }
  if (pqo.part) {
    Acc2 a;
#pragma unroll
    for (int r = 0; r < M; ++r) a.dot(xl[r], y[r]);
    pq_epilogue(pqo, a.value());
  }
}

// ---------------------------------------------------------------- FP16 operator copy
// Packed symmetric S_K in binary16 with one FP32 scale per element: S_K ~ sc16[e] * S16,
// sc16[e] = max |S_K| (so every stored value lies in [-1, 1]). Layout [group][P8][lane][8]:
// one 16-byte load per lane carries 8 consecutive packed entries.
template <int DIM, int K>
struct Packed16 {
  static constexpr int M = Dims<DIM, K>::M;
  static constexpr int P = M * (M + 1) / 2;
  static constexpr int P8 = (P + 7) / 8;
};

template <int DIM, int K>
__global__ void scale16_kernel(int64_t ne, const double* __restrict__ S, float* __restrict__ sc16) {
  constexpr int M = Dims<DIM, K>::M;
  const int lane = threadIdx.x & 31;
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t e = w; e < ne; e += nw) {
    double m = 0.0;
    for (int i = lane; i < M * M; i += 32) m = fmax(m, fabs(S[e * (int64_t)(M * M) + i]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    // round the scale up so that |S / sc| <= 1 holds after the FP32 rounding of sc
    if (lane == 0) sc16[e] = m > 0.0 ? __double2float_ru(m) : 1.f;
  }
}

template <int DIM, int K>
__global__ void pack16_kernel(int64_t ne, const double* __restrict__ S, const float* __restrict__ sc16,
                              __half* __restrict__ S16) {
  using PK = Packed16<DIM, K>;
  constexpr int M = PK::M, P8 = PK::P8;
  const int64_t ngroups = (ne + 31) / 32;
  const int64_t n = ngroups * P8 * 32 * 8;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(t & 7);
    const int lane = (int)((t >> 3) & 31);
    const int64_t q = (t >> 8) % P8;
    const int64_t g = (t >> 8) / P8;
    const int64_t e = g * 32 + lane;
    const int p = (int)(q * 8 + j);
    float v = 0.f;
    if (e < ne && p < PK::P) {
      int r = 0;
      while (packed_index(M, r, M - 1) < p) ++r;
      const int c = r + (p - packed_index(M, r, r));
      v = (float)(S[e * (int64_t)(M * M) + r * M + c] / (double)sc16[e]);
    }
    S16[t] = __float2half_rn(v);
  }
}

// Trace gather table of the FP16 apply: gface[e][f] = the id of face f of element e where it
// carries trace unknowns (an interior face), else -1; rows past the last element are -1
// (n = whole 32-element groups x NFC).
static __global__ void gface_kernel(int64_t n, int64_t nval, const int32_t* __restrict__ elem_face,
                                    const int32_t* __restrict__ face_bnd, int32_t* __restrict__ gface) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    int v = -1;
    if (t < nval) {
      const int f = elem_face[t];
      if (f >= 0 && face_bnd[f] < 0) v = f;
    }
    gface[t] = v;
  }
}

// Shared memory of the FP16 apply, per warp: the staged traces of the next group (row stride
// XS floats; each face run is copied by 8-byte asynchronous copies when NF is even, else
// 4-byte ones) and the transpose buffer of the slot write (row stride MP).
template <int DIM, int K>
struct Apply16Cfg {
  static constexpr int NF = Dims<DIM, K>::NF, M = Dims<DIM, K>::M;
  static constexpr int CPB = NF % 2 == 0 ? 8 : 4;
  static constexpr int XS = CPB == 8 ? M + 2 : M + 1;
  static constexpr int MP = M + 1;
  static constexpr int WARPS = 4;
  static constexpr size_t SMEM = sizeof(float) * WARPS * 32 * (XS + MP);
};

// slot = S_K x_K with the FP16 copy (FP32 accumulation, the element scale applied once at the
// end), one thread per element, one warp per group of 32 elements. Persistent: warps stride
// over the groups, and the traces of a warp's next group are gathered into shared memory by
// asynchronous copies (from gface, read one more group ahead) while the current group's S16
// streams in, so the gather latency is off the streaming path.
template <int DIM, int K>
__global__ void __launch_bounds__(128, 4) apply16_kernel(int64_t ne, const int32_t* __restrict__ gface,
                                                      const __half* __restrict__ S16, const float* __restrict__ sc16,
                                                      const float* __restrict__ x, float* __restrict__ slot,
                                                      const int* __restrict__ done, PqOut pqo) {
  using D = Dims<DIM, K>;
  using PK = Packed16<DIM, K>;
  using C = Apply16Cfg<DIM, K>;
  constexpr int NF = D::NF, M = D::M, NFC = D::NFC, P8 = PK::P8, XS = C::XS, MP = C::MP, CPB = C::CPB;
  extern __shared__ __align__(16) float a16sm[];
  if (done && *done) return;
  timing_start(pqo);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  float* t = a16sm + wid * 32 * (XS + MP) + 32 * XS;
  const unsigned xrow = (unsigned)__cvta_generic_to_shared(a16sm + wid * 32 * (XS + MP) + lane * XS);
  const float* xrow_g = a16sm + wid * 32 * (XS + MP) + lane * XS;
  const int64_t ngroups = (ne + 31) / 32;
  const int64_t nw = (int64_t)gridDim.x * C::WARPS;
  int gf[NFC];
  auto load_gf = [&](int64_t gg) {
#pragma unroll
    for (int f = 0; f < NFC; ++f) gf[f] = gg < ngroups ? gface[(gg * 32 + lane) * NFC + f] : -1;
  };
  // this lane's traces into its own row (zeros where gf < 0); only this lane reads the row
  auto issue = [&]() {
#pragma unroll
    for (int f = 0; f < NFC; ++f) {
      const float* src = gf[f] >= 0 ? x + (int64_t)gf[f] * NF : x;
      const unsigned nb = gf[f] >= 0 ? CPB : 0;
#pragma unroll
      for (int j = 0; j < NF * 4 / CPB; ++j)
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(xrow + 4 * f * NF + CPB * j),
                     "l"(src + (CPB / 4) * j), "n"(CPB), "r"(nb)
                     : "memory");
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  int64_t g = (int64_t)blockIdx.x * C::WARPS + wid;
  load_gf(g);
  issue();
  load_gf(g + nw);
  Acc2 a;
  for (; g < ngroups; g += nw) {
    const int64_t e = g * 32 + lane;
    const float scl = e < ne ? sc16[e] : 0.f;
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    float xl[M], y[M];
#pragma unroll
    for (int r = 0; r < M; ++r) xl[r] = xrow_g[r];
    issue();              // the next group's traces
    load_gf(g + 2 * nw);  // and the group after it's gather table
#pragma unroll
    for (int r = 0; r < M; ++r) y[r] = 0.f;
    const uint4* Sg = reinterpret_cast<const uint4*>(S16) + g * (int64_t)P8 * 32 + lane;
    float sv[8];
#pragma unroll
    for (int r = 0; r < M; ++r) {
#pragma unroll
      for (int c = r; c < M; ++c) {
        const int p = packed_index(M, r, c);
        if ((p & 7) == 0) {
          const uint4 u = __ldcs(Sg + (p >> 3) * 32);
          const unsigned w4[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
          for (int h = 0; h < 4; ++h) {
            const float2 f2 = __half22float2(*reinterpret_cast<const __half2*>(&w4[h]));
            sv[2 * h] = f2.x;
            sv[2 * h + 1] = f2.y;
          }
        }
        const float s = sv[p & 7];
        y[r] = fmaf(s, xl[c], y[r]);
        if (c != r) y[c] = fmaf(s, xl[r], y[c]);
      }
    }
#pragma unroll
    for (int r = 0; r < M; ++r) {
      y[r] *= scl;
      t[lane * MP + r] = y[r];
      a.dot(xl[r], y[r]);
    }
    __syncwarp();
    const int64_t nvalid = (ne - g * 32) < 32 ? (ne - g * 32) : 32;
    float* dst = slot + g * 32 * (int64_t)M;
    for (int idx = lane; idx < nvalid * M; idx += 32) dst[idx] = t[(idx / M) * MP + idx % M];
    __syncwarp();   // the transpose buffer is rewritten by the next group
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  if (pqo.part) pq_epilogue(pqo, a.value());
}

// q = sgn K32 p on faces; partial p.q in FP64. NF is compile-time (no integer division).
template <class LD>
__global__ void __launch_bounds__(256) cg32_face_q_kernel(int nf, float sgn, const int32_t* __restrict__ face_slot,
                                                          const int32_t* __restrict__ face_bnd,
                                                          const float* __restrict__ slot, const float* __restrict__ p,
                                                          float* __restrict__ q, double* __restrict__ part,
                                                          const CgScal* __restrict__ sc) {
  constexpr int NF = LD::NF;
  if (sc->done) return;
  __shared__ double red[8];
  Acc2 pq;
  for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < nf; f += gridDim.x * blockDim.x) {
    float qv[NF];
    if (face_bnd[f] < 0) {
      const float* s0 = slot + (int64_t)face_slot[2 * f] * NF;
      const float* s1 = slot + (int64_t)face_slot[2 * f + 1] * NF;
#pragma unroll
      for (int mm = 0; mm < NF; ++mm) qv[mm] = sgn * (s0[mm] + s1[mm]);
    } else {
#pragma unroll
      for (int mm = 0; mm < NF; ++mm) qv[mm] = 0.f;
    }
#pragma unroll
    for (int mm = 0; mm < NF; ++mm) {
      q[(int64_t)f * NF + mm] = qv[mm];
      pq.dot(p[(int64_t)f * NF + mm], qv[mm]);
    }
  }
  const double s = block_sum256(pq.value(), red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// FP32 vectors are padded to a multiple of 4 entries (padding: zero, dinv = 0) and
// processed as float4.
__device__ __forceinline__ float4 f4fma(float a, float4 x, float4 y) {
  return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
}
__device__ __forceinline__ float4 f4mul(float4 a, float4 b) { return make_float4(a.x * b.x, a.y * b.y, a.z * b.z, a.w * b.w); }


// inner solve start from x = 0: r = b, z = Dinv r, p = z; partials (rz, rr)
static __global__ void cg32_init_kernel(int64_t n4, const float4* __restrict__ b, const float4* __restrict__ dinv,
                                 float4* __restrict__ x, float4* __restrict__ r, float4* __restrict__ z,
                                 float4* __restrict__ p, double* __restrict__ part) {
  __shared__ double red[8];
  Acc2 rz, rr;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n4; t += (int64_t)gridDim.x * blockDim.x) {
    const float4 rv = b[t];
    const float4 zv = f4mul(dinv[t], rv);
    x[t] = make_float4(0.f, 0.f, 0.f, 0.f); r[t] = rv; z[t] = zv; p[t] = zv;
    rz.dot4(rv, zv); rr.dot4(rv, rv);
  }
  double s;
  s = block_sum256(rz.value(), red); if (threadIdx.x == 0) part[blockIdx.x * 2 + 0] = s;
  s = block_sum256(rr.value(), red); if (threadIdx.x == 0) part[blockIdx.x * 2 + 1] = s;
}

// rtol_dev (may be null): the relative tolerance read on the device instead of rtol
static __global__ void cg32_init_scalars(int nb, const double* __restrict__ part, double rtol, CgScal* sc,
                                         const double* __restrict__ rtol_dev) {
  __shared__ double red[8];
  const double rz = reduce_partials(part + 0, nb, 2, red);
  const double rr = reduce_partials(part + 1, nb, 2, red);
  if (threadIdx.x == 0) {
    const double tol = rtol_dev ? *rtol_dev : rtol;
    sc->rho[0] = rz; sc->rho[1] = 0; sc->bb = rr; sc->rr = rr;
    sc->tol2 = tol * tol * rr;
    sc->iters = 0;
    sc->done = (rr == 0.0) ? 1 : 0;
  }
}

static __global__ void cg32_update_kernel(int64_t n4, int nb, int parity, const double* __restrict__ part_pq,
                                   const float4* __restrict__ p, const float4* __restrict__ q,
                                   const float4* __restrict__ dinv, float4* __restrict__ x, float4* __restrict__ r,
                                   float4* __restrict__ z, double* __restrict__ part, const CgScal* __restrict__ sc) {
  if (sc->done) return;
  __shared__ double red[8];
  const double pq = reduce_partials(part_pq, nb, 1, red);
  const float al = (float)(sc->rho[parity] / pq);
  Acc2 rz, rr;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (; t + 3 * stride < n4; t += 4 * stride) {
    float4 pv[4], qv[4], xv[4], rv[4], dv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      pv[u] = p[t + u * stride]; qv[u] = q[t + u * stride]; xv[u] = x[t + u * stride];
      rv[u] = r[t + u * stride]; dv[u] = dinv[t + u * stride];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      x[t + u * stride] = f4fma(al, pv[u], xv[u]);
      const float4 rn = f4fma(-al, qv[u], rv[u]);
      const float4 zn = f4mul(dv[u], rn);
      r[t + u * stride] = rn; z[t + u * stride] = zn;
      rz.dot4(rn, zn); rr.dot4(rn, rn);
    }
  }
  for (; t < n4; t += stride) {
    x[t] = f4fma(al, p[t], x[t]);
    const float4 rv1 = f4fma(-al, q[t], r[t]);
    const float4 zv1 = f4mul(dinv[t], rv1);
    r[t] = rv1; z[t] = zv1;
    rz.dot4(rv1, zv1); rr.dot4(rv1, rv1);
  }
  double s;
  s = block_sum256(rz.value(), red); if (threadIdx.x == 0) part[blockIdx.x * 2 + 0] = s;
  s = block_sum256(rr.value(), red); if (threadIdx.x == 0) part[blockIdx.x * 2 + 1] = s;
}

// The update of the Krylov iteration with q = sgn K p formed from the slots (the face pass
// is folded in): q = sgn (slot0 + slot1) on interior faces (0 on the boundary),
// x += alpha p, r -= alpha q, z = Dinv r; partials (r.z, r.r). alpha = rho / pq with pq
// from the apply's reduction. Vectors are processed as float4 (coalesced); the two slot
// values of each entry are gathered per entry (runs of NF consecutive floats). Two float4
// per trip, and the face flags and slot pairs loaded before the branch on them, keep two
// independent load chains in flight per thread; a thread visits its entries in the same order
// as with one float4 per trip, so the sums are the same.
template <class LD>
__device__ __forceinline__ float4 q_entries4(int64_t t, int64_t nfe, float sgn, const int2* __restrict__ face_slot2,
                                             const int32_t* __restrict__ face_bnd, const float* __restrict__ slot) {
  constexpr int NF = LD::NF;
  const int64_t d0 = 4 * t;
  uint32_t f = (uint32_t)(d0 / NF);   // n_faces * NF < 2^32
  int mm = (int)(d0 - (int64_t)f * NF);
  uint32_t fi[4];
  int mi[4], fb[4];
  int2 fs[4];
  bool ok[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    fi[i] = f;
    mi[i] = mm;
    if (++mm == NF) { mm = 0; ++f; }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    ok[i] = d0 + i < nfe;
    fb[i] = ok[i] ? face_bnd[fi[i]] : 0;
    fs[i] = ok[i] ? face_slot2[fi[i]] : make_int2(0, 0);
  }
  float q[4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
    q[i] = (ok[i] && fb[i] < 0)
               ? sgn * (slot[(int64_t)fs[i].x * NF + mi[i]] + slot[(int64_t)fs[i].y * NF + mi[i]])
               : 0.f;
  return make_float4(q[0], q[1], q[2], q[3]);
}

template <class LD>
__global__ void __launch_bounds__(256) cg32_update_f_kernel(int64_t n4, int64_t nfe, float sgn, int parity,
                                                            const int32_t* __restrict__ face_slot,
                                                            const int32_t* __restrict__ face_bnd,
                                                            const float* __restrict__ slot,
                                                            const float4* __restrict__ p,
                                                            const float4* __restrict__ dinv, float4* __restrict__ x,
                                                            float4* __restrict__ r, float4* __restrict__ z,
                                                            const double* __restrict__ pq_in,
                                                            double* __restrict__ part, const CgScal* __restrict__ sc) {
  constexpr int U = 2;
  if (sc->done) return;
  __shared__ double red[8];
  const float al = (float)(sc->rho[parity] / *pq_in);
  const int2* face_slot2 = reinterpret_cast<const int2*>(face_slot);
  Acc2 rz, rr;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n4; t += U * stride) {
    float4 pv[U], xv[U], rv[U], dv[U], qv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t tu = t + u * stride;
      if (tu < n4) {
        pv[u] = p[tu]; xv[u] = x[tu]; rv[u] = r[tu]; dv[u] = dinv[tu];
        qv[u] = q_entries4<LD>(tu, nfe, sgn, face_slot2, face_bnd, slot);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t tu = t + u * stride;
      if (tu >= n4) break;
      x[tu] = f4fma(al, pv[u], xv[u]);
      const float4 rn = f4fma(-al, qv[u], rv[u]);
      const float4 zn = f4mul(dv[u], rn);
      r[tu] = rn;
      z[tu] = zn;
      rz.dot4(rn, zn);
      rr.dot4(rn, rn);
    }
  }
  double s;
  s = block_sum256(rz.value(), red); if (threadIdx.x == 0) part[blockIdx.x * 2 + 0] = s;
  s = block_sum256(rr.value(), red); if (threadIdx.x == 0) part[blockIdx.x * 2 + 1] = s;
}

// as cg_direction_kernel, FP32 vectors (float4)
static __global__ void cg32_direction_kernel(int64_t n4, int nb, int parity, int iter, const double* __restrict__ part,
                                      const float4* __restrict__ z, float4* __restrict__ p, CgScal* sc, int maxit,
                                      cudaGraphConditionalHandle h) {
  if (sc->done) {
    if (iter < 0 && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(h, 0u);
    return;
  }
  __shared__ double red[8];
  const double rz = reduce_partials(part + 0, nb, 2, red);
  const double rr = reduce_partials(part + 1, nb, 2, red);
  const bool conv = rr <= sc->tol2;
  const int it = iter >= 0 ? iter + 1 : sc->iters + 1;
  if (!conv && (iter < 0 || it < maxit)) {
    const float be = (float)(rz / sc->rho[parity]);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (; t + 3 * stride < n4; t += 4 * stride) {
      float4 pv[4], zv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) { pv[u] = p[t + u * stride]; zv[u] = z[t + u * stride]; }
#pragma unroll
      for (int u = 0; u < 4; ++u) p[t + u * stride] = f4fma(be, pv[u], zv[u]);
    }
    for (; t < n4; t += stride) p[t] = f4fma(be, p[t], z[t]);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    sc->rho[parity ^ 1] = rz;
    sc->rr = rr;
    sc->iters = it;
    const int done = conv ? 1 : (it >= maxit ? 2 : 0);
    if (done) sc->done = done;
    if (iter < 0) cudaGraphSetConditional(h, done ? 0u : 1u);
  }
}

// FP64 refinement residual rho = b - (sgn K) lam = b - sgn sum slots64 (interior), partials |rho|^2, |b|^2
static __global__ void refine_residual_kernel(int64_t nf, int NF, double sgn, const int32_t* __restrict__ face_slot,
                                       const int32_t* __restrict__ face_bnd, const double* __restrict__ zslot,
                                       const double* __restrict__ b, double* __restrict__ rho,
                                       double* __restrict__ part, const int* __restrict__ skip) {
  if (skip && *skip) return;   // rho and the partials are already in place
  __shared__ double red[8];
  const int64_t n = nf * NF;
  double rr = 0, bb = 0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t f = t / NF;
    const int mm = (int)(t % NF);
    double v = 0.0;
    if (face_bnd[f] < 0) {
      const double bv = b[t];
      v = bv - sgn * face_sum(face_slot, zslot, f, mm, NF);
      bb += bv * bv;
    }
    rho[t] = v;
    rr += v * v;
  }
  double s;
  s = block_sum256(rr, red); if (threadIdx.x == 0) part[blockIdx.x * 2 + 0] = s;
  s = block_sum256(bb, red); if (threadIdx.x == 0) part[blockIdx.x * 2 + 1] = s;
}

struct RefScal {
  double rr, bb, scale;
};

static __global__ void refine_scalars(int nb, const double* __restrict__ part, RefScal* rs) {
  __shared__ double red[8];
  const double rr = reduce_partials(part + 0, nb, 2, red);
  const double bb = reduce_partials(part + 1, nb, 2, red);
  if (threadIdx.x == 0) {
    rs->rr = rr; rs->bb = bb;
    rs->scale = rr > 0.0 ? 1.0 / sqrt(rr) : 1.0;
  }
}

// b32 = rho * scale (inner right-hand side of unit norm)
static __global__ void to32_scaled_kernel(int64_t n, const double* __restrict__ rho, const RefScal* __restrict__ rs,
                                   float* __restrict__ b32) {
  const double s = rs->scale;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    b32[t] = (float)(rho[t] * s);
}

// lam += delta / scale on interior faces (delta is zero on boundary faces)
static __global__ void refine_update_kernel(int64_t nf, int NF, const int32_t* __restrict__ face_bnd,
                                     const float* __restrict__ delta, const RefScal* __restrict__ rs,
                                     double* __restrict__ lam) {
  const double inv = 1.0 / rs->scale;
  const int64_t n = nf * NF;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    if (face_bnd[t / NF] < 0) lam[t] += (double)delta[t] * inv;
}

static __global__ void to32_kernel(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    b[t] = (float)a[t];
}

}  // namespace hdg

namespace hdg {

// ================================================================ double-float (FP64-class on the FP32 pipe)
// A value is the unevaluated sum h + l of two floats (|l| <= ulp(h)/2): about 48 significant
// bits. Products use the exact FMA error of h*h, sums the TwoSum error, so dot products keep
// the accuracy of FP64 evaluation to ~1e-14 relative on GB300's 58x faster FP32 pipe.
struct df2 {
  float h, l;
};

__device__ __forceinline__ df2 df_from(double x) {
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ double df_to(df2 a) { return (double)a.h + (double)a.l; }

// compensated accumulator of sum_i a_i b_i with a_i, b_i double-floats
struct DfAcc {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void fma(df2 a, df2 b) {
    const float p = a.h * b.h;
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, fmaf(a.l, b.h, e));
    const float t = s + p;
    const float bb = t - s;
    c += ((s - (t - bb)) + (p - bb)) + e;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// Double-float copy of S_K for the refinement apply, element-contiguous and diagonal-major:
// element e holds [hi | lo], each PD = 4 * P4 floats, entry (r, r + s) of the upper triangle at
// off(s) + r with off(s) = packed_index(M, s, s) (the s-th superdiagonal follows the first s
// ones). hi = fl32(S), lo = fl32(S - hi).
__host__ __device__ constexpr int diag_off(int M, int s) { return packed_index(M, s, s); }

template <int DIM, int K>
__global__ void packdf_kernel(int64_t ne, const double* __restrict__ S, float* __restrict__ Sdf) {
  using PK = Packed<DIM, K>;
  constexpr int M = PK::M, PD = PK::P4 * 4;
  const int64_t n = ne * PD;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = t / PD;
    const int pos = (int)(t - e * PD);
    float hi = 0.f, lo = 0.f;
    if (pos < PK::P) {
      int s = 0;
      while (s < M - 1 && diag_off(M, s + 1) <= pos) ++s;
      const int r = pos - diag_off(M, s);
      const double v = S[e * (int64_t)(M * M) + r * M + r + s];
      hi = __double2float_rn(v);
      lo = __double2float_rn(v - (double)hi);
    }
    Sdf[e * 2 * PD + pos] = hi;
    Sdf[e * 2 * PD + PD + pos] = lo;
  }
}

// FP64-accurate refinement apply on the FP32 pipe: zslot[e][r] = sum_c S_K[r][c] x_K[c] with
// S_K = hi + lo from the diagonal-major copy and x split into double-floats. CTA = EPB
// elements, one thread per (element, row); persistent over groups of EPB elements, the
// copies of the next group staged in shared memory with 16-byte asynchronous copies while the
// current one is computed (two stages). At step s thread r takes column c = (r + s) mod M: the
// superdiagonal s at row r when c >= r, else the superdiagonal M - s at row c, so the threads
// of an element read two runs of consecutive words.
template <int DIM, int K>
struct ApplyDfCfg {
  static constexpr int M = Dims<DIM, K>::M;
  static constexpr int EPB = 4;
  static constexpr int NT = EPB * M;
  static constexpr int PD = Packed<DIM, K>::P4 * 4;
  static constexpr int CH = EPB * 2 * PD / 4;                   // 16-byte chunks per group
  static constexpr int STAGE = EPB * 2 * PD;                     // floats per stage
  static constexpr size_t SMEM = sizeof(float) * 2 * STAGE + sizeof(df2) * EPB * M;
};

template <int DIM, int K>
__global__ void __launch_bounds__(ApplyDfCfg<DIM, K>::NT) apply_df_kernel(DevMesh mesh, const float* __restrict__ Sdf,
                                                                         const double* __restrict__ x,
                                                                         double* __restrict__ zslot, int64_t ngroups,
                                                                         const int* __restrict__ skip) {
  using D = Dims<DIM, K>;
  using C = ApplyDfCfg<DIM, K>;
  if (skip && *skip) return;   // the residual this apply serves is already in place
  constexpr int NF = D::NF, M = D::M, NFC = D::NFC, EPB = C::EPB, PD = C::PD;
  extern __shared__ __align__(16) float dsm[];
  df2* lx = reinterpret_cast<df2*>(dsm + 2 * C::STAGE);   // [EPB][M]
  const unsigned sbase = (unsigned)__cvta_generic_to_shared(dsm);
  // the copy is padded to whole 32-element groups, so every chunk of a group is in bounds
  auto issue = [&](int64_t g, int stage) {
    const char* src = reinterpret_cast<const char*>(Sdf + g * EPB * 2 * PD);
    const unsigned dst = sbase + (unsigned)(stage * C::STAGE * sizeof(float));
    for (int i = threadIdx.x; i < C::CH; i += C::NT)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst + 16 * i), "l"(src + 16 * i) : "memory");
  };
  int64_t g = blockIdx.x;
  if (g >= ngroups) return;
  issue(g, 0);
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  const int el = threadIdx.x / M, r = threadIdx.x % M;
  // this thread's trace entry of group gg (gathered one group ahead, off the compute path)
  auto gather = [&](int64_t gg) {
    double v = 0.0;
    const int64_t ee = gg * EPB + el;
    if (gg < ngroups && ee < mesh.ne) {
      const int f = mesh.elem_face[ee * NFC + r / NF];
      if (mesh.face_bnd[f] < 0) v = x[(int64_t)f * NF + r % NF];
    }
    return v;
  };
  double vnext = gather(g);
  for (int it = 0; g < ngroups; ++it, g += gridDim.x) {
    const int cur = it & 1;
    if (g + gridDim.x < ngroups) issue(g + gridDim.x, cur ^ 1);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    const int64_t e = g * EPB + el;
    lx[el * M + r] = df_from(vnext);
    vnext = gather(g + gridDim.x);
    asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    __syncthreads();
    if (e < mesh.ne) {
      const float* hi = dsm + cur * C::STAGE + el * 2 * PD;
      const float* lo = hi + PD;
      const df2* ex = lx + el * M;
      DfAcc acc;
#pragma unroll
      for (int s = 0; s < M; ++s) {
        const int c = r + s;
        const bool up = c < M;
        const int pos = up ? diag_off(M, s) + r : diag_off(M, M - s) + (c - M);
        acc.fma(df2{hi[pos], lo[pos]}, ex[up ? c : c - M]);
      }
      zslot[e * M + r] = acc.value();
    }
    __syncthreads();   // the stage just read is the next prefetch target
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

}  // namespace hdg
