// Instantiations of the separable-template passes for tap counts 1, 3, 5, 7.
#include "sep.cuh"

namespace cdv {
template cudaError_t sep_launch_q<1, false>(const SepPass&, int, cudaStream_t);
template cudaError_t sep_launch_q<1, true>(const SepPass&, int, cudaStream_t);
template cudaError_t sep_launch_q<3, false>(const SepPass&, int, cudaStream_t);
template cudaError_t sep_launch_q<3, true>(const SepPass&, int, cudaStream_t);
template cudaError_t sep_launch_q<5, false>(const SepPass&, int, cudaStream_t);
template cudaError_t sep_launch_q<5, true>(const SepPass&, int, cudaStream_t);
template cudaError_t sep_launch_q<7, false>(const SepPass&, int, cudaStream_t);
template cudaError_t sep_launch_q<7, true>(const SepPass&, int, cudaStream_t);
}  // namespace cdv
