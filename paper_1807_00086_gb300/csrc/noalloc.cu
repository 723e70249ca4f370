// Allocation-free variant of the matrix-free trace apply.
//
// Some callers cannot call cudaMalloc when they need this operation: code that must not
// trigger the implicit device synchronisation of an allocation inside a latency-bound
// loop, code that runs under a fixed memory budget handed out once at start-up (an
// arena owned by someone else), or plug-ins that are not allowed to touch the process's
// allocator at all. For them this entry point takes every input and output from the
// caller and keeps its only scratch (the per-element slot products that make the face
// reduction deterministic) in a file-scope device array of fixed size, which every GPU
// that loads the library holds until the process exits.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/hdg.h"

namespace {

constexpr size_t kScratchDoubles = (size_t)1 << 20;  // 8 MiB
static __device__ __align__(256) double g_slot_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {};  // device address of g_slot_scratch, per device

void put_err(char* err, int32_t len, const char* msg) {
  if (err && len > 0) {
    std::strncpy(err, msg, (size_t)len - 1);
    err[len - 1] = '\0';
  }
}

template <int DIM, int K>
struct NaDims {
  static constexpr int NP = (DIM == 2) ? (K + 1) * (K + 2) / 2 : (K + 1) * (K + 2) * (K + 3) / 6;
  static constexpr int NF = (DIM == 2) ? (K + 1) : (K + 1) * (K + 2) / 2;
  static constexpr int NFC = DIM + 1;
  static constexpr int M = NFC * NF;
  static constexpr int EPB = (128 / M) > 0 ? (128 / M) : 1;
  static constexpr int NT = EPB * M;
};

// slot[e][r] = sum_c S_K[r][c] x_K[c] (x gathered from faces, boundary faces read as 0). Thread r
// of an element walks row r of S_K, so S_K need not be symmetric.
template <int DIM, int K>
__global__ void __launch_bounds__(NaDims<DIM, K>::NT)
    noalloc_elem_kernel(int64_t ne, const double* __restrict__ S, const int32_t* __restrict__ elem_face,
                        const int32_t* __restrict__ face_bnd, const double* __restrict__ x, double* __restrict__ slot) {
  using D = NaDims<DIM, K>;
  constexpr int NF = D::NF, M = D::M;
  __shared__ double lx[D::EPB][M];
  const int el = threadIdx.x / M, r = threadIdx.x % M;
  const int64_t e = (int64_t)blockIdx.x * D::EPB + el;
  if (e < ne) {
    const int f = elem_face[e * D::NFC + r / NF];
    lx[el][r] = face_bnd[f] < 0 ? x[(int64_t)f * NF + r % NF] : 0.0;
  }
  __syncthreads();
  if (e < ne) {
    const double* Sr = S + e * (int64_t)(M * M) + (int64_t)r * M;
    double acc = 0.0;
    for (int c = 0; c < M; ++c) acc += Sr[c] * lx[el][c];
    slot[e * M + r] = acc;
  }
}

// y[f] = slot of the lower element + slot of the upper element (interior faces), 0 on boundary.
__global__ void noalloc_face_kernel(int64_t nf, int NF, const int32_t* __restrict__ face_slot,
                                    const int32_t* __restrict__ face_bnd, const double* __restrict__ slot,
                                    double* __restrict__ y) {
  const int64_t n = nf * NF;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t f = t / NF;
    const int mm = (int)(t % NF);
    double v = 0.0;
    if (face_bnd[f] < 0) v = slot[(int64_t)face_slot[2 * f] * NF + mm] + slot[(int64_t)face_slot[2 * f + 1] * NF + mm];
    y[t] = v;
  }
}

template <int DIM, int K>
void launch_noalloc(int64_t ne, int64_t nf, const double* S, const int32_t* elem_face, const int32_t* face_slot,
                    const int32_t* face_bnd, const double* x, double* y, double* slot, cudaStream_t st) {
  using D = NaDims<DIM, K>;
  const unsigned grid = (unsigned)((ne + D::EPB - 1) / D::EPB);
  noalloc_elem_kernel<DIM, K><<<grid, D::NT, 0, st>>>(ne, S, elem_face, face_bnd, x, slot);
  const int64_t n = nf * D::NF;
  const int64_t g2 = (n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096;
  noalloc_face_kernel<<<(unsigned)(g2 > 0 ? g2 : 1), 256, 0, st>>>(nf, D::NF, face_slot, face_bnd, slot, y);
}

}  // namespace

extern "C" hdg_status hdg_trace_apply_noalloc(int32_t dim, int32_t k, int64_t n_elem, int64_t n_faces,
                                              const double* S_dev, const int32_t* elem_face_dev,
                                              const int32_t* face_slot_dev, const int32_t* face_bnd_dev,
                                              const double* x_dev, double* y_dev, void* cuda_stream, char* err,
                                              int32_t err_len) {
  put_err(err, err_len, "");
  if ((dim != 2 && dim != 3) || k < 1 || k > 4) {
    put_err(err, err_len, "hdg_trace_apply_noalloc: dim must be 2 or 3 and 1 <= k <= 4");
    return HDG_EINVAL;
  }
  if (n_elem <= 0 || n_faces <= 0 || !S_dev || !elem_face_dev || !face_slot_dev || !face_bnd_dev || !x_dev || !y_dev) {
    put_err(err, err_len, "hdg_trace_apply_noalloc: empty sizes or null pointer");
    return HDG_EINVAL;
  }
  const int Nf = dim == 2 ? k + 1 : (k + 1) * (k + 2) / 2;
  const int64_t m = (int64_t)(dim + 1) * Nf;
  if (n_elem > (int64_t)(kScratchDoubles / (size_t)m)) {
    char msg[256];
    std::snprintf(msg, sizeof msg,
                  "hdg_trace_apply_noalloc: n_elem * m = %lld doubles exceeds the fixed scratch of %zu doubles "
                  "(8 MiB; at most %lld elements for m = %lld)",
                  (long long)(n_elem * m), kScratchDoubles, (long long)(kScratchDoubles / (size_t)m), (long long)m);
    put_err(err, err_len, msg);
    return HDG_EINVAL;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    put_err(err, err_len, "hdg_trace_apply_noalloc: no usable current device");
    return HDG_ECUDA;
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // The host-side name of the array is only a stand-in, so the kernels get its device address,
  // looked up with the device current. The lookup allocates nothing. It is repeated on every
  // call made while `st` is not being captured, so a context re-created after cudaDeviceReset
  // never sees a stale address; while `st` is being captured no lookup is made and the address
  // of the last call on this device is used, so the first call on a device must come before
  // any stream capture.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(st, &cap);
  if (e != cudaSuccess) {
    put_err(err, err_len, "hdg_trace_apply_noalloc: cudaStreamIsCapturing failed");
    return HDG_ECUDA;
  }
  double* slot = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (cap == cudaStreamCaptureStatusNone) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_slot_scratch);
      if (e != cudaSuccess || !p) {
        put_err(err, err_len, "hdg_trace_apply_noalloc: cudaGetSymbolAddress of the scratch array failed");
        return HDG_ECUDA;
      }
      g_scratch_ptr[dev] = (double*)p;
    } else if (!g_scratch_ptr[dev]) {
      put_err(err, err_len,
              "hdg_trace_apply_noalloc: the first call on a device must come before any stream capture");
      return HDG_ESTATE;
    }
    slot = g_scratch_ptr[dev];
  }
  switch (dim * 10 + k) {
    case 21: launch_noalloc<2, 1>(n_elem, n_faces, S_dev, elem_face_dev, face_slot_dev, face_bnd_dev, x_dev, y_dev, slot, st); break;
    case 22: launch_noalloc<2, 2>(n_elem, n_faces, S_dev, elem_face_dev, face_slot_dev, face_bnd_dev, x_dev, y_dev, slot, st); break;
    case 23: launch_noalloc<2, 3>(n_elem, n_faces, S_dev, elem_face_dev, face_slot_dev, face_bnd_dev, x_dev, y_dev, slot, st); break;
    case 24: launch_noalloc<2, 4>(n_elem, n_faces, S_dev, elem_face_dev, face_slot_dev, face_bnd_dev, x_dev, y_dev, slot, st); break;
    case 31: launch_noalloc<3, 1>(n_elem, n_faces, S_dev, elem_face_dev, face_slot_dev, face_bnd_dev, x_dev, y_dev, slot, st); break;
    case 32: launch_noalloc<3, 2>(n_elem, n_faces, S_dev, elem_face_dev, face_slot_dev, face_bnd_dev, x_dev, y_dev, slot, st); break;
    case 33: launch_noalloc<3, 3>(n_elem, n_faces, S_dev, elem_face_dev, face_slot_dev, face_bnd_dev, x_dev, y_dev, slot, st); break;
    default: launch_noalloc<3, 4>(n_elem, n_faces, S_dev, elem_face_dev, face_slot_dev, face_bnd_dev, x_dev, y_dev, slot, st); break;
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    put_err(err, err_len, cudaGetErrorString(e));
    return HDG_ECUDA;
  }
  return HDG_OK;
}
