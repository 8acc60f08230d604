// FP64 (DFMA) instantiations of the fused apply kernel, orders 1..8 with Q = p + 2.
#include "fe_apply_launch.cuh"

namespace fe {

int launch_apply_f64(int op, const ApplyArgs& a, cudaStream_t s) {
  return dispatch_order<ArF64>(op, a, s);
}

int multi_elems_f64(int op, int order) {
  using SH = ApplyShape<ArF64, 0>;
  return op == FE_DIFFUSION ? multi_elems<ArF64, true, SH::SMEM>(order)
                            : multi_elems<ArF64, false, SH::SMEM>(order);
}

int launch_apply_multi_f64(int op, const MultiGroups& g, const Basis1D* const* basis,
                           const double* x, double* y, int* counter, int nrhs, int64_t ldx,
                           int64_t ldy, cudaStream_t s) {
  return op == FE_DIFFUSION ? launch_multi<ArF64, true>(g, basis, x, y, counter, nrhs, ldx, ldy, s)
                            : launch_multi<ArF64, false>(g, basis, x, y, counter, nrhs, ldx, ldy, s);
}

}  // namespace fe
