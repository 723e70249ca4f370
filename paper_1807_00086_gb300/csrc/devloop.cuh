// Device-driven trace solves: the Krylov iterations and the refinement sweeps of Sec. 2.4's
// condensed solve run as CUDA-graph WHILE loops whose conditions the kernels set on the device,
// and the least-squares initial guess over earlier stage solutions is formed on the device,
// so a whole trace solve is one graph launch with no host round trip.
//
// Termination of every loop is decided on the device and bounded: an inner Krylov loop stops
// at convergence or at maxit (the direction kernel counts the iterations), the sweep loop at
// convergence, a zero right-hand side or max_sweeps (the control kernel counts the sweeps).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "kernels.cuh"

namespace hdg {

// Control block of one device-driven solve.
struct LoopCtl {
  double rel, rel_prev;   // relative FP64 residual of the current / previous sweep
  double tol;             // relative tolerance of the current sweep's inner solve
  int sweep;              // inner solves started
  int use16;              // inner operator of the next sweep: 1 FP16 copy, 0 FP32 copy
  int stop;               // 0 running, 1 converged, 2 zero right-hand side, 3 max_sweeps, 4 maxit
  int total_it;           // inner iterations summed over the finished sweeps
  int skip_res;           // the next residual is already in place (taken from the guess's pairs)
};

// Refinement sweep control, one thread, after the FP64 residual of a sweep (rs): records the
// previous inner solve's iterations, decides whether to stop, switches the inner operator to the
// FP32 copy when an FP16 sweep gained less than a factor 10, sets the next inner tolerance and the
// loop conditions (sweep loop, FP16 inner loop when has16, FP32 inner loop). A handle value of
// 0 may be valid, so has16 and not the handle says whether the FP16 loop exists.
static __global__ void sweep_ctl_kernel(const RefScal* __restrict__ rs, const CgScal* __restrict__ sc, LoopCtl* L,
                                        double rtol, double inner_rtol, int max_sweeps, cudaGraphConditionalHandle h_sweep,
                                        int has16, cudaGraphConditionalHandle h16, cudaGraphConditionalHandle h32) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (L->sweep > 0) L->total_it += sc->iters;
  int stop = 0;
  if (rs->bb == 0.0) {
    L->rel = 0.0;
    stop = 2;
  } else {
    L->rel_prev = L->rel;
    L->rel = sqrt(rs->rr / rs->bb);
    if (L->use16 && L->sweep > 0 && L->rel > 0.1 * L->rel_prev) L->use16 = 0;
    // a residual taken from the guess's pairs is accurate only to the tolerance the pairs
    // were solved to, so it never ends the solve: the stop test waits for a computed one
    if (L->rel <= rtol && !L->skip_res) stop = 1;
    else if (L->sweep >= max_sweeps) stop = 3;
  }
  L->skip_res = 0;
  if (!stop) {
    L->tol = fmin(0.5, fmax(inner_rtol, 0.25 * rtol / L->rel));
    L->sweep += 1;
  }
  L->stop = stop;
  cudaGraphSetConditional(h_sweep, stop ? 0u : 1u);
  if (has16) cudaGraphSetConditional(h16, (!stop && L->use16) ? 1u : 0u);
  cudaGraphSetConditional(h32, (!stop && !L->use16) ? 1u : 0u);
}

// FP64 CG epilogue, one thread: the stop code from the CG scalars.
static __global__ void cg_ctl_finish_kernel(const CgScal* __restrict__ sc, LoopCtl* L) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  L->total_it = sc->iters;
  L->sweep = 1;
  L->rel = sc->bb > 0.0 ? sqrt(fmax(0.0, sc->rr) / sc->bb) : 0.0;
  L->stop = sc->bb == 0.0 ? 2 : (sc->done == 1 ? 1 : 4);
}

// x[t] = 0 on interior entries (mask != 0; null mask: every entry) when the solve found a zero
// right-hand side.
static __global__ void zero_masked_if_kernel(int64_t n, const uint8_t* __restrict__ mask, const LoopCtl* __restrict__ L,
                                             double* __restrict__ x) {
  if (L->stop != 2) return;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    if (!mask || mask[t]) x[t] = 0.0;
}

static __global__ void loopctl_init_kernel(LoopCtl* L, int use16) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  L->rel = 0.0; L->rel_prev = 0.0; L->tol = 0.5;
  L->sweep = 0; L->use16 = use16; L->stop = 0; L->total_it = 0; L->skip_res = 0;
}

// Totals of the trace solves inside one graph-launched time step.
struct StepAcc {
  double rel;       // relative residual of the last solve
  int iters;        // Krylov iterations summed over the stage solves
  int sweeps;       // refinement sweeps (or solves) summed
  int bad;          // stop code of a solve that did not converge (3 max_sweeps, 4 maxit), else 0
  int pad;
};

static __global__ void step_acc_reset_kernel(StepAcc* A) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  A->rel = 0.0; A->iters = 0; A->sweeps = 0; A->bad = 0;
}

// after a stage solve: add its counts, keep the first failure
static __global__ void step_acc_kernel(const LoopCtl* __restrict__ L, StepAcc* A) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  A->iters += L->total_it;
  A->sweeps += L->sweep;
  A->rel = L->rel;
  if (!A->bad && L->stop != 1 && L->stop != 2) A->bad = L->stop;
}

// ---------------------------------------------------------------- least-squares initial guess
// Ring of the last q stage right-hand sides b_i and solutions lam_i of the same operator
// (K lam_i = b_i to the solver tolerance). With the Gram matrix G_ij = (b_i, b_j) kept on the
// device, lam0 = sum c_i lam_i minimising |b - K lam0| solves (G + mu I) c = g, g_i = (b_i, b),
// mu = 1e-13 max_i G_ii.
struct GuessDev {
  double gram[8][8];
  double dots[9];    // (b_i, b) for i < n, then (b, b)
  double coef[8];
  int q, n, next, ok;   // capacity, stored pairs, next slot, coefficients valid
};

// block partials of (ring_i, w) for i < n and of (w, w): part[blk][9]
static __global__ void gdots_kernel(int64_t n, const GuessDev* __restrict__ g, const double* __restrict__ ring,
                                    const double* __restrict__ w, double* __restrict__ part) {
  __shared__ double red[8];
  const int m = g->n;
  double acc[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) acc[i] = 0.0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const double wv = w[t];
#pragma unroll
    for (int i = 0; i < 8; ++i)
      if (i < m) acc[i] += ring[i * n + t] * wv;
    acc[8] += wv * wv;
  }
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    if (i < m || i == 8) {
      const double s = block_sum256(acc[i], red);
      if (threadIdx.x == 0) part[blockIdx.x * 9 + i] = s;
    }
  }
}

// sums the partials into g->dots (one block of 256 threads), then thread 0 solves the damped
// normal equations by Cholesky; g->ok = 0 when there is no usable history
static __global__ void gsolve_kernel(int nb, const double* __restrict__ part, GuessDev* g) {
  __shared__ double red[8];
  const int m = g->n;
  for (int i = 0; i <= m; ++i) {
    const int col = i < m ? i : 8;
    const double v = reduce_partials(part + col, nb, 9, red);
    if (threadIdx.x == 0) g->dots[i] = v;
  }
  if (threadIdx.x != 0) return;
  g->ok = 0;
  if (m == 0) return;
  double L[8][8], y[8], dmax = 0.0;
  for (int i = 0; i < m; ++i) dmax = fmax(dmax, g->gram[i][i]);
  if (!(dmax > 0.0)) return;
  for (int j = 0; j < m; ++j) {
    double d = g->gram[j][j] + 1e-13 * dmax;
    for (int k = 0; k < j; ++k) d -= L[j][k] * L[j][k];
    if (!(d > 0.0)) return;
    L[j][j] = sqrt(d);
    for (int i = j + 1; i < m; ++i) {
      double v = g->gram[i][j];
      for (int k = 0; k < j; ++k) v -= L[i][k] * L[j][k];
      L[i][j] = v / L[j][j];
    }
  }
  for (int i = 0; i < m; ++i) {
    double v = g->dots[i];
    for (int k = 0; k < i; ++k) v -= L[i][k] * y[k];
    y[i] = v / L[i][i];
  }
  for (int i = m - 1; i >= 0; --i) {
    double v = y[i];
    for (int k = i + 1; k < m; ++k) v -= L[k][i] * g->coef[k];
    g->coef[i] = v / L[i][i];
  }
  g->ok = 1;
}

// lam[t] = sum_i c_i ring_l[i][t] on interior entries (null mask: every entry) when the
// coefficients are valid
static __global__ void glincomb_kernel(int64_t n, const GuessDev* __restrict__ g, const double* __restrict__ ring,
                                       const uint8_t* __restrict__ mask, double* __restrict__ lam) {
  if (!g->ok) return;
  const int m = g->n;
  double c[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) c[i] = i < m ? g->coef[i] : 0.0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    if (mask && !mask[t]) continue;
    double v = 0.0;
#pragma unroll
    for (int i = 0; i < 8; ++i)
      if (i < m) v += c[i] * ring[i * n + t];
    lam[t] = v;
  }
}

// The refinement's first residual without an apply, when lam0 = sum c_i lam_i came from the
// guess: K lam_i = b_i up to the pairs' solve tolerance, so b - K lam0 = b - sum c_i b_i on
// interior entries (0 on the others). Same output and block partials (|rho|^2, |b|^2) as
// refine_residual_kernel; sets L->skip_res so that the sweep's own residual kernels stand
// aside. Does nothing when the coefficients are not valid.
static __global__ void gresidual_kernel(int64_t nf, int NF, const int32_t* __restrict__ face_bnd,
                                        const GuessDev* __restrict__ g, const double* __restrict__ ring,
                                        const double* __restrict__ b, double* __restrict__ rho,
                                        double* __restrict__ part, LoopCtl* L) {
  if (!g->ok) return;
  __shared__ double red[8];
  const int m = g->n;
  const int64_t n = nf * NF;
  double c[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) c[i] = i < m ? g->coef[i] : 0.0;
  double rr = 0, bb = 0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    double v = 0.0;
    if (face_bnd[t / NF] < 0) {
      const double bv = b[t];
      double s = 0.0;
#pragma unroll
      for (int i = 0; i < 8; ++i)
        if (i < m) s += c[i] * ring[i * n + t];
      v = bv - s;
      bb += bv * bv;
    }
    rho[t] = v;
    rr += v * v;
  }
  double s;
  s = block_sum256(rr, red); if (threadIdx.x == 0) part[blockIdx.x * 2 + 0] = s;
  s = block_sum256(bb, red); if (threadIdx.x == 0) part[blockIdx.x * 2 + 1] = s;
  if (blockIdx.x == 0 && threadIdx.x == 0) L->skip_res = 1;
}

// stores (b, lam) of the solve just finished in ring slot g->next
static __global__ void gstore_kernel(int64_t n, const GuessDev* __restrict__ g, const double* __restrict__ b,
                                     const double* __restrict__ lam, double* __restrict__ ring_b,
                                     double* __restrict__ ring_l) {
  const int64_t s = g->next;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    ring_b[s * n + t] = b[t];
    ring_l[s * n + t] = lam[t];
  }
}

// one thread: the new pair's Gram row from the dots of this solve's b, then advance the ring
static __global__ void gupdate_kernel(GuessDev* g) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int s = g->next, m = g->n;
  for (int i = 0; i < m; ++i)
    if (i != s) g->gram[s][i] = g->gram[i][s] = g->dots[i];
  g->gram[s][s] = g->dots[m];
  g->next = (s + 1) % g->q;
  g->n = m + 1 < g->q ? m + 1 : g->q;
}

static __global__ void guess_reset_kernel(GuessDev* g, int q) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  g->q = q; g->n = 0; g->next = 0; g->ok = 0;
  for (int i = 0; i < 8; ++i)
    for (int j = 0; j < 8; ++j) g->gram[i][j] = 0.0;
}

}  // namespace hdg

// ---------------------------------------------------------------- host: graph construction
// Builds a graph section by section: straight-line work is captured from a private stream into
// the graph after the current sink nodes; a WHILE node is added with a handle created on the
// graph that holds it, and its body is captured in turn. Every CUDA error is kept in `err`.
struct GraphBuild {
  cudaStream_t st = nullptr;
  cudaError_t err = cudaSuccess;

  template <class F>
  void seq(cudaGraph_t g, std::vector<cudaGraphNode_t>& deps, F issue) {
    if (err != cudaSuccess) return;
    err = cudaStreamBeginCaptureToGraph(st, g, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(),
                                        cudaStreamCaptureModeThreadLocal);
    if (err != cudaSuccess) return;
    issue();
    const cudaError_t le = cudaGetLastError();
    cudaStreamCaptureStatus cs;
    const cudaGraphNode_t* d = nullptr;
    size_t nd = 0;
    cudaError_t ie = cudaStreamGetCaptureInfo(st, &cs, nullptr, nullptr, &d, nullptr, &nd);
    std::vector<cudaGraphNode_t> sinks;
    if (ie == cudaSuccess) sinks.assign(d, d + nd);
    cudaGraph_t out = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(st, &out);
    err = le != cudaSuccess ? le : (ie != cudaSuccess ? ie : ee);
    if (err == cudaSuccess) deps = sinks;
  }

  // WHILE node after deps; returns its body graph (deps becomes the node)
  cudaGraph_t loop(cudaGraph_t g, std::vector<cudaGraphNode_t>& deps, cudaGraphConditionalHandle h) {
    if (err != cudaSuccess) return nullptr;
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    err = cudaGraphAddNode(&node, g, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(), &p);
    if (err != cudaSuccess) return nullptr;
    deps.assign(1, node);
    return p.conditional.phGraph_out[0];
  }

  cudaGraphConditionalHandle handle(cudaGraph_t g, unsigned dflt, bool assign_default) {
    cudaGraphConditionalHandle h = 0;
    if (err != cudaSuccess) return 0;
    err = cudaGraphConditionalHandleCreate(&h, g, dflt, assign_default ? cudaGraphCondAssignDefault : 0);
    return h;
  }
};
