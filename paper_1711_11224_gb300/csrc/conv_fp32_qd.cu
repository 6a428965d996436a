// Instantiations of the FP32 engine for template widths (along the contiguous axis): 25 27 29 31.
#include "conv_fp32.cuh"

namespace cdv {
CDV_INSTANTIATE_FP32(25)
CDV_INSTANTIATE_FP32(27)
CDV_INSTANTIATE_FP32(29)
CDV_INSTANTIATE_FP32(31)
}  // namespace cdv
