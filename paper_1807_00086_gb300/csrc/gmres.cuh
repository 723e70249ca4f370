// Restarted GMRES with iterated classical Gram-Schmidt (Sec. 2.4: the paper solves the trace
// system with GMRES, orthogonalised by ICGS): vector kernels over the trace entries. The basis
// V is [m + 1][n] (n entries per vector, interior faces; boundary entries stay zero). All sums
// are block partials reduced in a fixed order (deterministic).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.cuh"

namespace hdg {

// part[i][blk] = block partial of (V_i, w) for i < q and of (w, w) for i = q; grid (nbx, q + 1)
static __global__ void gm_dots_kernel(int64_t n, int q, const double* __restrict__ V, const double* __restrict__ w,
                                      double* __restrict__ part) {
  __shared__ double red[8];
  const int i = blockIdx.y;
  const double* a = i < q ? V + (int64_t)i * n : w;
  double s = 0.0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    s += a[t] * w[t];
  s = block_sum256(s, red);
  if (threadIdx.x == 0) part[(int64_t)i * gridDim.x + blockIdx.x] = s;
}

// out[i] = sum of part[i][0..nbx), one block per i
static __global__ void gm_dots_final_kernel(int nbx, const double* __restrict__ part, double* __restrict__ out) {
  __shared__ double red[8];
  const double s = reduce_partials(part + (int64_t)blockIdx.x * nbx, nbx, 1, red);
  if (threadIdx.x == 0) out[blockIdx.x] = s;
}

// w -= sum_{i<q} h_i V_i
static __global__ void gm_orth_kernel(int64_t n, int q, const double* __restrict__ V, const double* __restrict__ h,
                                      double* __restrict__ w) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    double s = w[t];
    for (int i = 0; i < q; ++i) s -= h[i] * V[(int64_t)i * n + t];
    w[t] = s;
  }
}

// x += Dinv (sum_{i<q} y_i V_i) on interior entries (right preconditioning)
static __global__ void gm_update_kernel(int64_t n, int q, const double* __restrict__ V, const double* __restrict__ y,
                                       const double* __restrict__ dinv, const uint8_t* __restrict__ mask,
                                       double* __restrict__ x) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    if (!mask[t]) continue;
    double s = 0.0;
    for (int i = 0; i < q; ++i) s += y[i] * V[(int64_t)i * n + t];
    x[t] += dinv[t] * s;
  }
}

// out = a * b (elementwise)
static __global__ void vmul_kernel(int64_t n, const double* __restrict__ a, const double* __restrict__ b,
                                   double* __restrict__ out) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    out[t] = a[t] * b[t];
}

// out = s * a with s read on the device (1 / norm)
static __global__ void vscale_inv_kernel(int64_t n, const double* __restrict__ norm2, const double* __restrict__ a,
                                         double* __restrict__ out) {
  const double s = 1.0 / sqrt(*norm2);
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    out[t] = s * a[t];
}

}  // namespace hdg
