// Instantiations of the separable-template passes for tap counts 25, 27, 29, 31.
#include "sep.cuh"

namespace cdv {
template cudaError_t sep_launch_q<25, false>(const SepPass&, int, cudaStream_t);
template cudaError_t sep_launch_q<25, true>(const SepPass&, int, cudaStream_t);
template cudaError_t sep_launch_q<27, false>(const SepPass&, int, cudaStream_t);
template cudaError_t sep_launch_q<27, true>(const SepPass&, int, cudaStream_t);
template cudaError_t sep_launch_q<29, false>(const SepPass&, int, cudaStream_t);
template cudaError_t sep_launch_q<29, true>(const SepPass&, int, cudaStream_t);
template cudaError_t sep_launch_q<31, false>(const SepPass&, int, cudaStream_t);
template cudaError_t sep_launch_q<31, true>(const SepPass&, int, cudaStream_t);
}  // namespace cdv
