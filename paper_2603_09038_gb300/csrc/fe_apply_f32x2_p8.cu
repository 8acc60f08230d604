// Float-float fused apply, order 8 (one of several translation units, so that the float-float
// kernels compile in parallel).
#include "fe_apply_launch.cuh"

namespace fe {

template int apply_order<ArF32x2, 8>(int, const ApplyArgs&, cudaStream_t);

}  // namespace fe
