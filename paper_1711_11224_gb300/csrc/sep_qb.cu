// Instantiations of the separable-template passes for tap counts 9, 11, 13, 15.
#include "sep.cuh"

namespace cdv {
template cudaError_t sep_launch_q<9, false>(const SepPass&, int, cudaStream_t);
template cudaError_t sep_launch_q<9, true>(const SepPass&, int, cudaStream_t);
template cudaError_t sep_launch_q<11, false>(const SepPass&, int, cudaStream_t);
template cudaError_t sep_launch_q<11, true>(const SepPass&, int, cudaStream_t);
template cudaError_t sep_launch_q<13, false>(const SepPass&, int, cudaStream_t);
template cudaError_t sep_launch_q<13, true>(const SepPass&, int, cudaStream_t);
template cudaError_t sep_launch_q<15, false>(const SepPass&, int, cudaStream_t);
template cudaError_t sep_launch_q<15, true>(const SepPass&, int, cudaStream_t);
}  // namespace cdv
