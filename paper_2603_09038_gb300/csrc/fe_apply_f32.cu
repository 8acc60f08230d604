// Plain FP32 instantiations of the fused apply kernel (inner solves of iterative refinement),
// and the conversion of the stored quadrature data to its FP32 copy.
#include "fe_apply_launch.cuh"

namespace fe {

int launch_apply_f32(int op, const ApplyArgs& a, cudaStream_t s) {
  return dispatch_order<ArF32>(op, a, s);
}

// FP32 vectors in and out (a.x, a.y point to float arrays): the inner solves of fe_pcg_ir.
int launch_apply_f32_vec32(int op, const ApplyArgs& a, cudaStream_t s) {
  return dispatch_order<ArF32, float>(op, a, s);
}

// Largest biased FP64 exponent of n values, into *emax (atomicMax; the caller zeroes it).
__global__ void k_max_exponent(const double* __restrict__ src, int64_t n, int* emax) {
  int m = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    m = max(m, f64_exponent(src[i]));
  m = __reduce_max_sync(0xffffffffu, m);
  if ((threadIdx.x & 31) == 0) atomicMax(emax, m);
}

// FP32 copy of n quadrature values times 2^-shift (exact scaling in FP64, then rounded).
__global__ void k_qd_to_f32(const double* __restrict__ src, float* __restrict__ dst, int64_t n,
                            int shift) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    dst[i] = __double2float_rn(ldexp(src[i], -shift));
}

int make_qd_f32(const double* src, float* dst, int64_t n, int* shift, cudaStream_t s) {
  *shift = 0;
  if (n == 0 || src == nullptr) return FE_OK;
  int* d_emax = nullptr;
  cudaError_t err = cudaMalloc(&d_emax, sizeof(int));
  if (err != cudaSuccess) return cuda_error(err, "qdata FP32 copy: cudaMalloc");
  int emax = 0;
  cudaMemsetAsync(d_emax, 0, sizeof(int), s);
  k_max_exponent<<<4 * 152, 256, 0, s>>>(src, n, d_emax);
  err = cudaMemcpyAsync(&emax, d_emax, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  cudaFree(d_emax);
  if (err != cudaSuccess) return cuda_error(err, "qdata FP32 copy: exponent");
  *shift = emax > 0 ? emax - 1023 : 0;
  k_qd_to_f32<<<4 * 152, 256, 0, s>>>(src, dst, n, *shift);
  return cuda_error(cudaGetLastError(), "qdata FP32 copy launch");
}

}  // namespace fe
