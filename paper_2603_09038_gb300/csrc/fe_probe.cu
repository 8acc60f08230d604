// Throughput probes behind the roofline denominators (measurement utility, not the hot path):
// independent FMA / DMMA chains per thread on every SM, timed with CUDA events.  GB300's FP64
// rate is not in the measured peaks (those are an HBM copy and a BF16 GEMM), so the FP64
// roofline of the FP64 apply is derived from the DFMA rate these kernels measure.
#include <cuda_runtime.h>

#include "fe_f2.h"
#include "fe_internal.h"

namespace {

constexpr int kChains = 8;

__global__ void k_probe_dfma(double* out, int iters, double b, double c) {
  double a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = threadIdx.x * 1e-3 + i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = fma(a[i], b, c);
  }
  double s = 0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  if (s == 12345.678) out[0] = s;  // keeps the chains live
}

__global__ void k_probe_ffma(float* out, int iters, float b, float c) {
  float a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = threadIdx.x * 1e-3f + i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = fmaf(a[i], b, c);
  }
  float s = 0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  if (s == 12345.678f) out[0] = s;
}

__global__ void k_probe_dmma(double* out, int iters) {
  double a = threadIdx.x * 1e-3, b = 0.999;
  double c[kChains][2];
#pragma unroll
  for (int i = 0; i < kChains; ++i) c[i][0] = c[i][1] = i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                   : "+d"(c[i][0]), "+d"(c[i][1])
                   : "d"(a), "d"(b));
  }
  double s = 0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += c[i][0] + c[i][1];
  if (s == 12345.678) out[0] = s;
}

// DFMA chains in the even warps and DMMA chains in the odd ones, at the same time: whether the two
// FP64 instruction kinds share one datapath (the combined rate stays at the DFMA rate) or not
// (the rates add).  The chain lengths make each half run about equally long on its own unit.
__global__ void k_probe_dfma_dmma(double* out, int iters_f, int iters_m) {
  const int warp = threadIdx.x >> 5;
  double s = 0;
  if ((warp & 1) == 0) {
    double a[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = threadIdx.x * 1e-3 + i;
    for (int it = 0; it < iters_f; ++it) {
#pragma unroll
      for (int i = 0; i < kChains; ++i) a[i] = fma(a[i], 0.9999, 1e-3);
    }
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += a[i];
  } else {
    double a = threadIdx.x * 1e-3, b = 0.999;
    double c[kChains][2];
#pragma unroll
    for (int i = 0; i < kChains; ++i) c[i][0] = c[i][1] = i;
    for (int it = 0; it < iters_m; ++it) {
#pragma unroll
      for (int i = 0; i < kChains; ++i)
        asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                     : "+d"(c[i][0]), "+d"(c[i][1])
                     : "d"(a), "d"(b));
    }
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += c[i][0] + c[i][1];
  }
  if (s == 12345.678) out[0] = s;
}

// BF16 m16n8k16 tensor-core MMA chains with FP32 accumulation (the instruction of the learned
// preconditioner's kernels), 4096 flops each per warp
__global__ void k_probe_hmma(float* out, int iters, uint32_t av, uint32_t bv) {
  float c[kChains][4];
#pragma unroll
  for (int i = 0; i < kChains; ++i) c[i][0] = c[i][1] = c[i][2] = c[i][3] = (float)i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i)
      asm volatile(
          "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
          "{%8,%9}, {%0,%1,%2,%3};"
          : "+f"(c[i][0]), "+f"(c[i][1]), "+f"(c[i][2]), "+f"(c[i][3])
          : "r"(av), "r"(av), "r"(av), "r"(av), "r"(bv), "r"(bv));
  }
  float s = 0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += c[i][0] + c[i][1] + c[i][2] + c[i][3];
  if (s == 12345.678f) out[0] = s;
}

// anchored float-float multiply-add chains (the apply's inner step), counted as 2 flops each
__global__ void k_probe_f2(float* out, int iters, float ah, float al) {
  fe::Anch acc[kChains];
  fe::f2 x[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) {
    acc[i] = fe::anch_begin(1024.0f);
    x[i] = fe::f2{threadIdx.x * 1e-3f + i, 1e-9f * i};
  }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) fe::anch_mad(acc[i], ah, al, x[i]);
  }
  float s = 0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += acc[i].A + acc[i].L;
  if (s == 12345.678f) out[0] = s;
}

}  // namespace

extern "C" int fe_probe_throughput(int unit, double* tflops) {
  fe::clear_error();
  if (!tflops) return fe::set_error(FE_ERR_ARG, "fe_probe_throughput: tflops is NULL");
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int threads = 256, blocks = sms * 8;
  const double nthreads = (double)threads * blocks;
  void* buf = nullptr;
  cudaError_t err = cudaMalloc(&buf, 64);
  if (err != cudaSuccess) return fe::cuda_error(err, "fe_probe_throughput: cudaMalloc");
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int iters = 0;
  double flops_per_iter = 0;
  auto launch = [&]() {
    switch (unit) {
      case FE_PROBE_FP64_FMA:
        iters = 4096;
        flops_per_iter = 2.0 * kChains * nthreads;
        k_probe_dfma<<<blocks, threads>>>((double*)buf, iters, 0.9999, 1e-3);
        break;
      case FE_PROBE_FP64_DMMA:
        iters = 2048;
        flops_per_iter = 512.0 * kChains * (nthreads / 32);
        k_probe_dmma<<<blocks, threads>>>((double*)buf, iters);
        break;
      case FE_PROBE_FP32_FMA:
        iters = 65536;
        flops_per_iter = 2.0 * kChains * nthreads;
        k_probe_ffma<<<blocks, threads>>>((float*)buf, iters, 0.9999f, 1e-3f);
        break;
      case FE_PROBE_BF16_MMA:
        iters = 4096;
        flops_per_iter = 4096.0 * kChains * (nthreads / 32);
        k_probe_hmma<<<blocks, threads>>>((float*)buf, iters, 0x3F803F80u, 0x3F7F3F7Fu);
        break;
      case FE_PROBE_FP64_DFMA_DMMA: {
        // half the warps each: 2 flops x 8 chains x 32 lanes per DFMA iteration, 512 x 8 per
        // DMMA iteration; 1/8 the DMMA iterations gives each half the same flop count
        iters = 4096;
        const int iters_m = iters / 8;
        flops_per_iter = (2.0 * kChains * 32 + 512.0 * kChains / 8) * (nthreads / 64);
        k_probe_dfma_dmma<<<blocks, threads>>>((double*)buf, iters, iters_m);
        break;
      }
      default:
        iters = 8192;
        flops_per_iter = 2.0 * kChains * nthreads;
        k_probe_f2<<<blocks, threads>>>((float*)buf, iters, 0.999f, 1e-9f);
        break;
    }
  };
  int st = FE_OK;
  if (unit < FE_PROBE_FP64_FMA || unit > FE_PROBE_FP64_DFMA_DMMA) {
    st = fe::set_error(FE_ERR_ARG, "fe_probe_throughput: unknown unit");
  } else {
    launch();  // warm-up
    cudaEventRecord(e0);
    for (int r = 0; r < 3; ++r) launch();
    cudaEventRecord(e1);
    err = cudaEventSynchronize(e1);
    if (err == cudaSuccess) err = cudaGetLastError();
    if (err != cudaSuccess) {
      st = fe::cuda_error(err, "fe_probe_throughput");
    } else {
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      *tflops = 3.0 * flops_per_iter * iters / (ms * 1e-3) / 1e12;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  return st;
}
