// Float-float fused apply, orders 5..6 (one of several translation units, so that the float-float
// kernels compile in parallel).
#include "fe_apply_launch.cuh"

namespace fe {

template int apply_order<ArF32x2, 5>(int, const ApplyArgs&, cudaStream_t);
template int apply_order<ArF32x2, 6>(int, const ApplyArgs&, cudaStream_t);

}  // namespace fe
