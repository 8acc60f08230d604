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

// FP32 copy of n quadrature values: from FP64 data, or from (hi, lo) pairs (hi is already the
// rounded float).
__global__ void k_qd_to_f32(const double* __restrict__ src, float* __restrict__ dst, int64_t n,
                            int pairs) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    dst[i] = pairs ? reinterpret_cast<const float2*>(src)[i].x : __double2float_rn(src[i]);
}

int make_qd_f32(const double* src, float* dst, int64_t n, bool pairs, cudaStream_t s) {
  if (n == 0 || src == nullptr) return FE_OK;
  k_qd_to_f32<<<4 * 152, 256, 0, s>>>(src, dst, n, pairs ? 1 : 0);
  return cuda_error(cudaGetLastError(), "qdata FP32 copy launch");
}

}  // namespace fe
