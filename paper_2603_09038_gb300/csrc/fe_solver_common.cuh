// Shared pieces of the CG solvers (fe_pcg.cu, fe_pcg_batched.cu): deterministic block
// reductions of FP64 partials, the device-state conventions and the CUDA-graph capture of an
// iteration batch.  Included into an anonymous namespace of each
// solver translation unit.
#pragma once

#include <cuda_runtime.h>

#include "fe_f2.h"
#include "fe_internal.h"

constexpr int kReduceBlocks = 1024;
constexpr int kReduceThreads = 256;
constexpr int kBatch = 8;  // iterations queued between two host reads of the stop flag

// scalar slots in d_red after the two partial arrays
enum { S_RZ = 0, S_BB, S_PQ, S_ALPHA, S_BETA, S_REL, S_RR, S_TRUE, kScalars = 16 };
// flags[0]: 0 running, 1 converged, 2 breakdown, 3 NaN/Inf, 4 maxit; flags[1]: iterations
enum { F_STATE = 0, F_ITERS = 1 };
enum { ST_RUN = 0, ST_CONV = 1, ST_BREAK = 2, ST_NAN = 3, ST_MAXIT = 4 };

// Deterministic block sum of two values; thread 0 writes them to part0/part1[blockIdx.x].
__device__ __forceinline__ void block_sum2(double a, double b, double* part0, double* part1) {
  __shared__ double sa[kReduceThreads / 32], sb[kReduceThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  if (l == 0) {
    sa[w] = a;
    sb[w] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ta = 0.0, tb = 0.0;
    for (int i = 0; i < kReduceThreads / 32; ++i) {
      ta += sa[i];
      tb += sb[i];
    }
    part0[blockIdx.x] = ta;
    if (part1) part1[blockIdx.x] = tb;
  }
}

// Deterministic sum of the kReduceBlocks partials by one block of kReduceBlocks threads (fixed
// shuffle tree, then the warp sums in order); every thread returns the total.
constexpr int kFinishThreads = kReduceBlocks;

__device__ __forceinline__ double ordered_sum(const double* part) {
  __shared__ double ws[kFinishThreads / 32];
  __shared__ double total;
  double v = part[threadIdx.x];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double w = ws[threadIdx.x];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w += __shfl_down_sync(0xffffffffu, w, o);
    if (threadIdx.x == 0) total = w;
  }
  __syncthreads();
  const double t = total;
  __syncthreads();
  return t;
}


// One batch of PCG iterations captured as a CUDA graph (on a private stream: the caller's may be
// the legacy stream, which cannot be captured) and replayed on the caller's stream with one
// launch.  The captured kernels read every scalar from device memory, so the same graph serves
// all batches of a solve.  A capture that fails leaves `failed` set and the caller enqueues
// kernels one by one instead (same kernels, same results).
struct GraphBatch {
  cudaGraphExec_t exec = nullptr;
  int kernels = 0;
  bool failed = false;
  template <typename Fn>
  void capture(Fn&& enqueue) {
    cudaStream_t cs = nullptr;
    cudaGraph_t g = nullptr;
    failed = true;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      const int st = enqueue(cs);
      const cudaError_t e = cudaStreamEndCapture(cs, &g);
      if (st == FE_OK && e == cudaSuccess && g &&
          cudaGraphInstantiate(&exec, g, 0) == cudaSuccess)
        failed = false;
      else
        exec = nullptr;
    }
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    cudaGetLastError();  // a failed capture is not an error of the solve
    clear_error();
  }
  ~GraphBatch() {
    if (exec) cudaGraphExecDestroy(exec);
  }
};

