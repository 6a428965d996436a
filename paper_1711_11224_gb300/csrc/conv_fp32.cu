// Tile selection and template-width dispatch of the FP32 engine.
#include <algorithm>

#include "conv_fp32.cuh"

namespace cdv {

CDV_EXTERN_FP32(1) CDV_EXTERN_FP32(3) CDV_EXTERN_FP32(5) CDV_EXTERN_FP32(7)
CDV_EXTERN_FP32(9) CDV_EXTERN_FP32(11) CDV_EXTERN_FP32(13) CDV_EXTERN_FP32(15)
CDV_EXTERN_FP32(17) CDV_EXTERN_FP32(19) CDV_EXTERN_FP32(21) CDV_EXTERN_FP32(23)
CDV_EXTERN_FP32(25) CDV_EXTERN_FP32(27) CDV_EXTERN_FP32(29) CDV_EXTERN_FP32(31)

bool conv_fp32_supported(int q3) { return q3 >= 1 && q3 <= 31 && (q3 & 1); }

ConvTile conv_fp32_tile(const ConvGeom& g)
{
    ConvTile t;
    const int64_t cols = (g.b3 + kR3 - 1) / kR3;                 // thread columns needed
    t.tiles3 = (int)((cols + 31) / 32);
    t.ntx = (int)((cols + t.tiles3 - 1) / t.tiles3);
    int nty = std::max(1, kMaxThreads / t.ntx);
    nty = (int)std::min<int64_t>(nty, g.b2);
    // two CTAs per SM: at most 110 KB of shared memory each
    while (nty > 1 && ConvSmem::make(t.ntx, nty, g.q2, g.q3).bytes() > 110 * 1024) nty--;
    t.nty = nty;
    t.tiles2 = (int)((g.b2 + nty - 1) / nty);
    t.tiles1 = (int)((g.b1 + kT1 - 1) / kT1);
    t.grid = t.tiles1 * t.tiles2 * t.tiles3;
    t.smem = ConvSmem::make(t.ntx, t.nty, g.q2, g.q3).bytes();
    return t;
}

cudaError_t conv_fp32_batch_launch(int q3, const ConvBatchVol* vols, const int2* items, int nitems, size_t smem,
                                   cudaStream_t s)
{
    switch (q3) {
#define CDV_CASE(Q) \
    case Q: return conv_fp32_batch_launch_q<Q>(vols, items, nitems, smem, s);
        CDV_CASE(1) CDV_CASE(3) CDV_CASE(5) CDV_CASE(7) CDV_CASE(9) CDV_CASE(11) CDV_CASE(13) CDV_CASE(15)
        CDV_CASE(17) CDV_CASE(19) CDV_CASE(21) CDV_CASE(23) CDV_CASE(25) CDV_CASE(27) CDV_CASE(29) CDV_CASE(31)
#undef CDV_CASE
    default:
        return cudaErrorInvalidValue;
    }
}

// Tile of the FP32 engine with a given number of thread rows (nty <= 0: the default choice).
ConvTile conv_fp32_tile_shape(const ConvGeom& g, int nty)
{
    ConvTile t = conv_fp32_tile(g);
    if (nty <= 0) return t;
    nty = (int)std::min<int64_t>(std::max(1, std::min(nty, kMaxThreads / t.ntx)), g.b2);
    t.nty = nty;
    t.tiles2 = (int)((g.b2 + nty - 1) / nty);
    t.grid = t.tiles1 * t.tiles2 * t.tiles3;
    t.smem = ConvSmem::make(t.ntx, t.nty, g.q2, g.q3).bytes();
    return t;
}

cudaError_t conv_fp32_prepare(int q3)
{
    ConvLaunch L{};
    L.g.q3 = q3;
    L.batch = 0;
    ConvTile t{};
    return conv_fp32_launch(L, t, nullptr);
}

cudaError_t conv_fp32_launch(const ConvLaunch& L, const ConvTile& t, cudaStream_t s)
{
    switch (L.g.q3) {
#define CDV_CASE(Q) \
    case Q: return conv_fp32_launch_q<Q>(L, t, s);
        CDV_CASE(1) CDV_CASE(3) CDV_CASE(5) CDV_CASE(7) CDV_CASE(9) CDV_CASE(11) CDV_CASE(13) CDV_CASE(15)
        CDV_CASE(17) CDV_CASE(19) CDV_CASE(21) CDV_CASE(23) CDV_CASE(25) CDV_CASE(27) CDV_CASE(29) CDV_CASE(31)
#undef CDV_CASE
    default:
        return cudaErrorInvalidValue;
    }
}

}  // namespace cdv
