// Instantiations of the FP32 engine for template widths (along the contiguous axis): 17 19 21 23.
#include "conv_fp32.cuh"

namespace cdv {
CDV_INSTANTIATE_FP32(17)
CDV_INSTANTIATE_FP32(19)
CDV_INSTANTIATE_FP32(21)
CDV_INSTANTIATE_FP32(23)
}  // namespace cdv
