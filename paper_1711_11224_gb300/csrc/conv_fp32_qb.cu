// Instantiations of the FP32 engine for template widths (along the contiguous axis): 9 11 13 15.
#include "conv_fp32.cuh"

namespace cdv {
CDV_INSTANTIATE_FP32(9)
CDV_INSTANTIATE_FP32(11)
CDV_INSTANTIATE_FP32(13)
CDV_INSTANTIATE_FP32(15)
}  // namespace cdv
