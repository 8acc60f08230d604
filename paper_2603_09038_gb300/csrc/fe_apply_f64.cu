// FP64 (DFMA) instantiations of the fused apply kernel, orders 1..8 with Q = p + 2.
#include "fe_apply_launch.cuh"

namespace fe {

int launch_apply_f64(int op, const ApplyArgs& a, cudaStream_t s) {
  return dispatch_order<ArF64>(op, a, s);
}

}  // namespace fe
