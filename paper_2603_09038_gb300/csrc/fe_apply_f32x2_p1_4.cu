// Float-float fused apply, orders 1..4 (one of several translation units, so that the float-float
// kernels compile in parallel).
#include "fe_apply_launch.cuh"

namespace fe {

template int apply_order<ArF32x2, 1>(int, const ApplyArgs&, cudaStream_t);
template int apply_order<ArF32x2, 2>(int, const ApplyArgs&, cudaStream_t);
template int apply_order<ArF32x2, 3>(int, const ApplyArgs&, cudaStream_t);
template int apply_order<ArF32x2, 4>(int, const ApplyArgs&, cudaStream_t);

}  // namespace fe
