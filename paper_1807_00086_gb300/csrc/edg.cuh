// Continuous trace spaces (Sec. 2.2, Eq. e:spaces2): EDG (all faces continuous) and IEDG
// (interior faces continuous). The element blocks and S_K are those of HDG; the global unknowns
// are the values mu at the degree-k equispaced nodes shared between faces, and the face modal
// traces are lam_F = V^{-1} mu(nodes of F) (the same V^{-1} on every face, since each face is
// parametrised from its vertices in ascending global id). The trace system is the Galerkin
// restriction R^T K R mu = R^T r of the HDG one.
//
// Device layout: face_node [n_faces][Nf] free node of each face node (-1: a fixed node or a face
// outside the continuous set); vinv [Nf][Nf] (row m: modal coefficient, column a: node); the
// node-owned incidence list node_ptr [n_free + 1] / node_inc [..] of face entries f * Nf + a, so
// that every sum over a node's faces runs in a fixed order (deterministic, no atomics).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.cuh"

namespace hdg {

// The 10-term sums below are FP32 on the FP32 path and double-float (FP64-class accuracy on the
// FP32 pipe; GB300 issues FP64 at 1/58 of the FP32 rate) on the FP64 path.
template <typename T>
struct VTab;
template <>
struct VTab<float> {
  float v;
  __device__ static VTab from(double x) { return VTab{(float)x}; }
};
template <>
struct VTab<double> {
  df2 v;
  __device__ static VTab from(double x) { return VTab{df_from(x)}; }
};

template <typename T>
struct VSum;
template <>
struct VSum<float> {
  float s = 0.f;
  __device__ __forceinline__ void add(const VTab<float>& a, float x) { s = fmaf(a.v, x, s); }
  __device__ __forceinline__ float value() const { return s; }
};
template <>
struct VSum<double> {
  DfAcc acc;
  __device__ __forceinline__ void add(const VTab<double>& a, double x) { acc.fma(a.v, df_from(x)); }
  __device__ __forceinline__ double value() const { return acc.value(); }
};

// lam[f][m] = sum_a vinv[m][a] mu[face_node[f][a]] on interior faces. Boundary faces: 0 when
// zero_bnd (Krylov work vectors), left as they are otherwise (the step's Dirichlet traces).
// One thread per face: its NF nodal values are gathered once.
template <typename T, int NF>
__global__ void edg_expand_kernel(int64_t nf, const int32_t* __restrict__ face_bnd, const int32_t* __restrict__ face_node,
                                  const double* __restrict__ vinv, const T* __restrict__ mu, T* __restrict__ lam,
                                  int zero_bnd) {
  __shared__ VTab<T> V[NF * NF];
  for (int i = threadIdx.x; i < NF * NF; i += blockDim.x) V[i] = VTab<T>::from(vinv[i]);
  __syncthreads();
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nf; f += (int64_t)gridDim.x * blockDim.x) {
    if (face_bnd[f] >= 0) {
      if (zero_bnd) {
#pragma unroll
        for (int m = 0; m < NF; ++m) lam[f * NF + m] = T(0);
      }
      continue;
    }
    T mv[NF];
#pragma unroll
    for (int a = 0; a < NF; ++a) {
      const int32_t node = face_node[f * NF + a];
      mv[a] = node >= 0 ? mu[node] : T(0);
    }
#pragma unroll
    for (int m = 0; m < NF; ++m) {
      VSum<T> v;
#pragma unroll
      for (int a = 0; a < NF; ++a) v.add(V[m * NF + a], mv[a]);
      lam[f * NF + m] = v.value();
    }
  }
}

// Nodal weights of each interior face, w[f][a] = sum_m vinv[m][a] y_f[m], with y_f the face's
// slot sum (slot != null: both elements' slot products) or the face array itself (slot == null);
// 0 on boundary faces. One thread per face.
template <typename T, int NF>
__global__ void edg_face_w_kernel(int64_t nf, const int32_t* __restrict__ face_slot, const int32_t* __restrict__ face_bnd,
                                  const double* __restrict__ vinv, const T* __restrict__ slot, const T* __restrict__ yface,
                                  T* __restrict__ w) {
  __shared__ VTab<T> V[NF * NF];
  for (int i = threadIdx.x; i < NF * NF; i += blockDim.x) V[i] = VTab<T>::from(vinv[i]);
  __syncthreads();
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nf; f += (int64_t)gridDim.x * blockDim.x) {
    if (face_bnd[f] >= 0) {
#pragma unroll
      for (int a = 0; a < NF; ++a) w[f * NF + a] = T(0);
      continue;
    }
    T y[NF];
    if (slot) {
      const T* s0 = slot + (int64_t)face_slot[2 * f] * NF;
      const T* s1 = slot + (int64_t)face_slot[2 * f + 1] * NF;
#pragma unroll
      for (int m = 0; m < NF; ++m) y[m] = s0[m] + s1[m];
    } else {
#pragma unroll
      for (int m = 0; m < NF; ++m) y[m] = yface[f * NF + m];
    }
#pragma unroll
    for (int a = 0; a < NF; ++a) {
      VSum<T> v;
#pragma unroll
      for (int m = 0; m < NF; ++m) v.add(V[m * NF + a], y[m]);
      w[f * NF + a] = v.value();
    }
  }
}

__device__ __forceinline__ double node_sum(const int32_t* __restrict__ ptr, const int32_t* __restrict__ inc,
                                           const double* __restrict__ w, int64_t i) {
  double v = 0.0;
  for (int32_t k = ptr[i]; k < ptr[i + 1]; ++k) v += w[inc[k]];
  return v;
}
__device__ __forceinline__ float node_sum(const int32_t* __restrict__ ptr, const int32_t* __restrict__ inc,
                                          const float* __restrict__ w, int64_t i) {
  float v = 0.f;
  for (int32_t k = ptr[i]; k < ptr[i + 1]; ++k) v += w[inc[k]];
  return v;
}

// out[i] = scale * sum of w over node i's face entries (R^T applied to face nodal weights)
static __global__ void edg_node_gather_kernel(int64_t n, const int32_t* __restrict__ ptr, const int32_t* __restrict__ inc,
                                              const double* __restrict__ w, double scale, double* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = scale * node_sum(ptr, inc, w, i);
}

// FP64 CG start on the nodes: q0 = sgn R^T K R x0 from the face weights, r = b - q0, z = Dinv r,
// p = z; partials (rz, rr, bb).
static __global__ void edg_cg_init_kernel(int64_t n, double sgn, const int32_t* __restrict__ ptr,
                                          const int32_t* __restrict__ inc, const double* __restrict__ w,
                                          const double* __restrict__ b, const double* __restrict__ dinv,
                                          double* __restrict__ r, double* __restrict__ z, double* __restrict__ p,
                                          double* __restrict__ part) {
  __shared__ double red[8];
  double rz = 0, rr = 0, bb = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double bv = b[i];
    const double rv = bv - sgn * node_sum(ptr, inc, w, i);
    const double zv = dinv[i] * rv;
    r[i] = rv; z[i] = zv; p[i] = zv;
    rz += rv * zv; rr += rv * rv; bb += bv * bv;
  }
  double s;
  s = block_sum256(rz, red); if (threadIdx.x == 0) part[blockIdx.x * 3 + 0] = s;
  s = block_sum256(rr, red); if (threadIdx.x == 0) part[blockIdx.x * 3 + 1] = s;
  s = block_sum256(bb, red); if (threadIdx.x == 0) part[blockIdx.x * 3 + 2] = s;
}

// q = sgn R^T K R p on the nodes; partial p.q
static __global__ void edg_q64_kernel(int64_t n, double sgn, const int32_t* __restrict__ ptr,
                                      const int32_t* __restrict__ inc, const double* __restrict__ w,
                                      const double* __restrict__ p, double* __restrict__ q, double* __restrict__ part,
                                      const CgScal* __restrict__ sc) {
  if (sc->done) return;
  __shared__ double red[8];
  double pq = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double qv = sgn * node_sum(ptr, inc, w, i);
    q[i] = qv;
    pq += p[i] * qv;
  }
  const double s = block_sum256(pq, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// FP32 Krylov update on the nodes with q = sgn R^T (slot sums) gathered from the face weights:
// alpha = rho / pq (pq from the apply's epilogue), x += alpha p, r -= alpha q, z = Dinv r;
// partials (r.z, r.r) accurate to FP64 level.
static __global__ void edg_update32_kernel(int64_t n, float sgn, const int32_t* __restrict__ ptr,
                                           const int32_t* __restrict__ inc, const float* __restrict__ w,
                                           const float* __restrict__ p, const float* __restrict__ dinv,
                                           float* __restrict__ x, float* __restrict__ r, float* __restrict__ z,
                                           int parity, const double* __restrict__ pq_in, double* __restrict__ part,
                                           const CgScal* __restrict__ sc) {
  if (sc->done) return;
  __shared__ double red[8];
  const float al = (float)(sc->rho[parity] / *pq_in);
  Acc2 rz, rr;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float qv = sgn * node_sum(ptr, inc, w, i);
    x[i] = fmaf(al, p[i], x[i]);
    const float rn = fmaf(-al, qv, r[i]);
    const float zn = dinv[i] * rn;
    r[i] = rn; z[i] = zn;
    rz.dot(rn, zn); rr.dot(rn, rn);
  }
  double s;
  s = block_sum256(rz.value(), red); if (threadIdx.x == 0) part[blockIdx.x * 2 + 0] = s;
  s = block_sum256(rr.value(), red); if (threadIdx.x == 0) part[blockIdx.x * 2 + 1] = s;
}

// FP64-accurate refinement residual on the nodes, res = b - sgn R^T K R x; partials |res|^2, |b|^2
static __global__ void edg_residual_kernel(int64_t n, double sgn, const int32_t* __restrict__ ptr,
                                           const int32_t* __restrict__ inc, const double* __restrict__ w,
                                           const double* __restrict__ b, double* __restrict__ res,
                                           double* __restrict__ part) {
  __shared__ double red[8];
  double rr = 0, bb = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double bv = b[i];
    const double v = bv - sgn * node_sum(ptr, inc, w, i);
    res[i] = v;
    rr += v * v; bb += bv * bv;
  }
  double s;
  s = block_sum256(rr, red); if (threadIdx.x == 0) part[blockIdx.x * 2 + 0] = s;
  s = block_sum256(bb, red); if (threadIdx.x == 0) part[blockIdx.x * 2 + 1] = s;
}

// x += delta / scale (every node is an unknown)
static __global__ void flat_refine_update_kernel(int64_t n, const float* __restrict__ delta, const RefScal* __restrict__ rs,
                                                 double* __restrict__ x) {
  const double inv = 1.0 / rs->scale;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] += (double)delta[i] * inv;
}

// Jacobi diagonal of R^T K R, element part: for element slot (e, local face a) and face node j,
// c[(e NFC + a) NF + j] = sum over the element's face nodes (b, l) at the same global node of
// (V^{-1}[:, j])^T S_K[a-block, b-block] V^{-1}[:, l]. Summed over a node's incidences (both
// elements of each face) this is w_K^T S_K w_K summed over the elements, w_K = R_K e_node.
template <int DIM, int NF>
__global__ void edg_diag_elem_kernel(int64_t ne, const int32_t* __restrict__ elem_face, const int32_t* __restrict__ face_node,
                                     const double* __restrict__ vinv, const double* __restrict__ S, double* __restrict__ c) {
  constexpr int NFC = DIM + 1, M = NFC * NF;
  const int64_t n = ne * M;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = t / M;
    const int a = (int)((t - e * M) / NF), j = (int)(t % NF);
    const int32_t node = face_node[(int64_t)elem_face[e * NFC + a] * NF + j];
    double v = 0.0;
    if (node >= 0) {
      const double* Se = S + e * (int64_t)(M * M);
      for (int b = 0; b < NFC; ++b) {
        const int64_t fb = elem_face[e * NFC + b];
        for (int l = 0; l < NF; ++l) {
          if (face_node[fb * NF + l] != node) continue;
          for (int mm = 0; mm < NF; ++mm) {
            double row = 0.0;
            for (int nn = 0; nn < NF; ++nn) row += Se[(a * NF + mm) * M + b * NF + nn] * vinv[nn * NF + l];
            v += vinv[mm * NF + j] * row;
          }
        }
      }
    }
    c[t] = v;
  }
}

// dinv[i] = sgn / (sum of the element parts over node i's face entries, both sides of each face)
static __global__ void edg_diag_node_kernel(int64_t n, int NF, const int32_t* __restrict__ ptr,
                                            const int32_t* __restrict__ inc, const int32_t* __restrict__ face_slot,
                                            const double* __restrict__ c, double sgn, double* __restrict__ dinv,
                                            float* __restrict__ dinv32) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double d = 0.0;
    for (int32_t k = ptr[i]; k < ptr[i + 1]; ++k) {
      const int64_t f = inc[k] / NF;
      const int a = inc[k] % NF;
      d += c[(int64_t)face_slot[2 * f] * NF + a] + c[(int64_t)face_slot[2 * f + 1] * NF + a];
    }
    dinv[i] = sgn / d;
    if (dinv32) dinv32[i] = (float)(sgn / d);
  }
}

}  // namespace hdg
