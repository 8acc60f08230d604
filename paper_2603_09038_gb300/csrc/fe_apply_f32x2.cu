// Float-float (FP64-accurate on the FP32 pipe) fused apply: the order dispatch, the persistent
// multi-order kernel and the float-pair encoding of the quadrature data.
#include "fe_apply_launch.cuh"

namespace fe {

// The per-order kernels live in fe_apply_f32x2_p*.cu.
extern template int apply_order<ArF32x2, 1>(int, const ApplyArgs&, cudaStream_t);
extern template int apply_order<ArF32x2, 2>(int, const ApplyArgs&, cudaStream_t);
extern template int apply_order<ArF32x2, 3>(int, const ApplyArgs&, cudaStream_t);
extern template int apply_order<ArF32x2, 4>(int, const ApplyArgs&, cudaStream_t);
extern template int apply_order<ArF32x2, 5>(int, const ApplyArgs&, cudaStream_t);
extern template int apply_order<ArF32x2, 6>(int, const ApplyArgs&, cudaStream_t);
extern template int apply_order<ArF32x2, 7>(int, const ApplyArgs&, cudaStream_t);
extern template int apply_order<ArF32x2, 8>(int, const ApplyArgs&, cudaStream_t);

int launch_apply_f32x2(int op, const ApplyArgs& a, cudaStream_t s) {
  if (a.Q != a.p + 2) return set_error(FE_ERR_UNSUPPORTED, "only q1d = order + 2 is built");
  switch (a.p) {
    case 1: return apply_order<ArF32x2, 1>(op, a, s);
    case 2: return apply_order<ArF32x2, 2>(op, a, s);
    case 3: return apply_order<ArF32x2, 3>(op, a, s);
    case 4: return apply_order<ArF32x2, 4>(op, a, s);
    case 5: return apply_order<ArF32x2, 5>(op, a, s);
    case 6: return apply_order<ArF32x2, 6>(op, a, s);
    case 7: return apply_order<ArF32x2, 7>(op, a, s);
    case 8: return apply_order<ArF32x2, 8>(op, a, s);
    default: return set_error(FE_ERR_UNSUPPORTED, "order out of range 1..8");
  }
}

int multi_elems_f32x2(int op, int order) {
  using SH = ApplyShape<ArF32x2, 0>;
  return op == FE_DIFFUSION ? multi_elems<ArF32x2, true, SH::SMEM>(order)
                            : multi_elems<ArF32x2, false, SH::SMEM>(order);
}

int launch_apply_multi_f32x2(int op, const MultiGroups& g, const Basis1D* const* basis,
                           const double* x, double* y, int* counter, int nrhs, int64_t ldx,
                           int64_t ldy, cudaStream_t s) {
  return op == FE_DIFFUSION ? launch_multi<ArF32x2, true>(g, basis, x, y, counter, nrhs, ldx, ldy, s)
                            : launch_multi<ArF32x2, false>(g, basis, x, y, counter, nrhs, ldx, ldy, s);
}

// Float-pair copy of the FP64 quadrature data, one warp per element: the element's largest
// biased exponent e_max gives its scale s = e_max - 1023 (0 for an all-zero element), and each
// entry v becomes the pair hi = rn(v 2^-s), lo = rn(v 2^-s - hi) (v 2^-s exact in FP64), so
// the element's largest entry lies in [1, 2) and hi + lo carries ~48 significant bits whatever
// the magnitude of the coefficient.
__global__ void k_encode_f32x2(const double* __restrict__ src, double* __restrict__ dst,
                               int32_t* __restrict__ scale, int64_t ne, int per_elem) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
  for (int64_t e = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32; e < ne;
       e += warps) {
    const double* v = src + e * per_elem;
    int emax = 0;
    for (int i = lane; i < per_elem; i += 32) emax = max(emax, f64_exponent(v[i]));
    emax = __reduce_max_sync(0xffffffffu, emax);
    const int sc = emax > 0 ? emax - 1023 : 0;
    if (lane == 0) scale[e] = sc;
    float2* out = reinterpret_cast<float2*>(dst + e * per_elem);
    for (int i = lane; i < per_elem; i += 32) {
      const double w = ldexp(v[i], -sc);
      const float h = __double2float_rn(w);
      out[i] = make_float2(h, __double2float_rn(w - (double)h));
    }
  }
}

int encode_f32x2(const double* src, double* dst, int32_t* scale, int64_t ne, int per_elem,
                 cudaStream_t s) {
  if (ne == 0 || src == nullptr) return FE_OK;
  k_encode_f32x2<<<8 * 152, 256, 0, s>>>(src, dst, scale, ne, per_elem);
  return cuda_error(cudaGetLastError(), "encode_f32x2 launch");
}

}  // namespace fe
