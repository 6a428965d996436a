// Instantiations of the separable-template passes for tap counts 17, 19, 21, 23.
#include "sep.cuh"

namespace cdv {
template cudaError_t sep_launch_q<17, false>(const SepPass&, int, cudaStream_t);
template cudaError_t sep_launch_q<17, true>(const SepPass&, int, cudaStream_t);
template cudaError_t sep_launch_q<19, false>(const SepPass&, int, cudaStream_t);
template cudaError_t sep_launch_q<19, true>(const SepPass&, int, cudaStream_t);
template cudaError_t sep_launch_q<21, false>(const SepPass&, int, cudaStream_t);
template cudaError_t sep_launch_q<21, true>(const SepPass&, int, cudaStream_t);
template cudaError_t sep_launch_q<23, false>(const SepPass&, int, cudaStream_t);
template cudaError_t sep_launch_q<23, true>(const SepPass&, int, cudaStream_t);
}  // namespace cdv
