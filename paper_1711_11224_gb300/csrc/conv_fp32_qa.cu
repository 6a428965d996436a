// Instantiations of the FP32 engine for template widths (along the contiguous axis): 1 3 5 7.
#include "conv_fp32.cuh"

namespace cdv {
CDV_INSTANTIATE_FP32(1)
CDV_INSTANTIATE_FP32(3)
CDV_INSTANTIATE_FP32(5)
CDV_INSTANTIATE_FP32(7)
}  // namespace cdv
