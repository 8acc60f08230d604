// Float-float fused apply, order 7 (one of several translation units, so that the float-float
// kernels compile in parallel).
#include "fe_apply_launch.cuh"

namespace fe {

template int apply_order<ArF32x2, 7>(int, const ApplyArgs&, cudaStream_t);

}  // namespace fe
