// Float-float (FP64-accurate on the FP32 pipe) instantiations of the fused apply kernel.
#include "fe_apply_launch.cuh"

namespace fe {

int launch_apply_f32x2(int op, const ApplyArgs& a, cudaStream_t s) {
  return dispatch_order<ArF32x2>(op, a, s);
}

// In-place re-encoding of FP64 quadrature data as (hi, lo) float pairs and back.  The pair is
// produced on the host-independent path: hi = round-to-nearest float of v, lo = float of the
// remainder v - hi (exact in FP64), so hi + lo carries ~48 significant bits.
__global__ void k_encode_f32x2(double* __restrict__ data, int64_t n, int to_pairs) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    if (to_pairs) {
      const double v = data[i];
      const float h = __double2float_rn(v);
      const float l = __double2float_rn(v - (double)h);
      reinterpret_cast<float2*>(data)[i] = make_float2(h, l);
    } else {
      const float2 p = reinterpret_cast<const float2*>(data)[i];
      data[i] = (double)p.x + (double)p.y;
    }
  }
}

int encode_f32x2(double* data, int64_t n, bool to_pairs, cudaStream_t s) {
  if (n == 0 || data == nullptr) return FE_OK;
  k_encode_f32x2<<<4 * 152, 256, 0, s>>>(data, n, to_pairs ? 1 : 0);
  return cuda_error(cudaGetLastError(), "encode_f32x2 launch");
}

}  // namespace fe
