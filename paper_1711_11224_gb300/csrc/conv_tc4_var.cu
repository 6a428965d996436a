// Instantiations of the narrow tensor-core kernel with the step-rule variants of the iteration in the
// adjoint epilogue; compiled apart from the default ones in conv_tc4.cu.
#include "conv_tc4.cuh"

namespace cdv {

cudaError_t tc4_prepare_var(int kind) { return tc4_prepare_kinds<true>(kind); }

cudaError_t tc4_launch_var(const TcArgs& t, const CUtensorMap* maps, cudaStream_t s)
{
    return tc4_launch_kinds<true>(t, maps, s);
}

}  // namespace cdv
