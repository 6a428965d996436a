// Instantiations of the tensor-core engine with the step-rule variants of the iteration in the
// adjoint epilogue (Tikhonov term, Armijo slope, Barzilai-Borwein inner product); compiled apart from
// the default instantiations in conv_tc.cu.
#include "conv_tc.cuh"

namespace cdv {

cudaError_t tc_prepare_var(int kind) { return tc_prepare_kinds<true>(kind); }

cudaError_t tc_launch_var(const TcArgs& t, const CUtensorMap* maps, cudaStream_t s)
{
    return tc_launch_kinds<true>(t, maps, s);
}

}  // namespace cdv
