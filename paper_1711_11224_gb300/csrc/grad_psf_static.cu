// Allocation-free template gradient: cdv_grad_psf without a plan.
//
// Some callers cannot call cudaMalloc: code that runs while a CUDA graph is
// being captured in global mode (where allocation calls are not permitted),
// plug-ins and callbacks hosted by a framework that owns all device memory
// through its own pool, and real-time loops that must not touch the
// allocator after start-up.  This entry point takes only the caller's input
// and output arrays; the FP64 block partials that cdv_grad_psf keeps in a
// plan's workspace live here in one file-scope __device__ array.
//
// Properties of that array:
//  * Its size is fixed at build time (kScratchDoubles doubles, 4 MiB).  Every
//    GPU that loads this library holds it until the process exits.
//  * All calls share it and it keeps the contents of the last call.  Each
//    call writes every partial it later reads, so nothing has to start at
//    zero; but calls whose kernels overlap on the GPU (different streams, or
//    different host threads without ordering) race on it and give wrong
//    results.  Order such calls on one stream.
//  * Host code cannot use the array's name as a device address, so the first
//    call on each device looks the address up with cudaGetSymbolAddress (and
//    sets the kernel's shared-memory attribute).  Make that first call
//    before any stream capture begins.
#include <stdarg.h>
#include <stdio.h>

#include <algorithm>
#include <mutex>

#include "cdv_internal.h"

namespace {

constexpr size_t kScratchDoubles = (size_t)1 << 19;      // 4 MiB of FP64 partials
__device__ __align__(256) double g_grad_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
double* g_scratch_ptr[kMaxDevices] = {};

cdv_status fail(cdv_status s, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    cdv::set_last_error(buf);
    return s;
}

// Once per device, with that device current: the array's device address.
cdv_status scratch_for_current_device(double** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(CDV_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(CDV_ERR_UNSUPPORTED, "device index %d", dev);
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_grad_scratch);
        if (e != cudaSuccess || !p)
            return fail(CDV_ERR_CUDA, "cudaGetSymbolAddress(static scratch): %s", cudaGetErrorString(e));
        e = cdv::grad_psf_prepare();
        if (e != cudaSuccess) return fail(CDV_ERR_CUDA, "kernel attribute: %s", cudaGetErrorString(e));
        g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_ptr[dev];
    return CDV_OK;
}

}  // namespace

extern "C" cdv_status cdv_grad_psf_static(int n, const int64_t* m, const int32_t* p, int batch, const float* X,
                                          const float* dY, float* dH, void* stream)
{
    if (!m || !p || !X || !dY || !dH) return fail(CDV_ERR_INVALID_ARG, "NULL argument");
    if (n < 1 || n > 3) return fail(CDV_ERR_SHAPE, "n = %d, must be 1, 2 or 3", n);
    if (batch < 1) return fail(CDV_ERR_INVALID_ARG, "batch = %d", batch);
    int64_t mm[3] = {1, 1, 1};
    int pp[3] = {0, 0, 0};
    for (int i = 0; i < n; i++) {
        if (m[i] < 1 || m[i] > (1LL << 31)) return fail(CDV_ERR_SHAPE, "m[%d] = %lld", i, (long long)m[i]);
        if (p[i] < 0 || p[i] > (1 << 20)) return fail(CDV_ERR_SHAPE, "p[%d] = %d", i, (int)p[i]);
        mm[3 - n + i] = m[i];
        pp[3 - n + i] = p[i];
    }
    const int q1 = 2 * pp[0] + 1, q2 = 2 * pp[1] + 1, q3 = 2 * pp[2] + 1;
    const size_t nh = (size_t)q1 * q2 * q3;
    if (nh > kScratchDoubles)
        return fail(CDV_ERR_UNSUPPORTED,
                    "template of %zu samples: the static scratch holds partials for at most %zu samples",
                    nh, kScratchDoubles);
    if ((size_t)q2 * ((q3 + 3) / 4) > 1024)
        return fail(CDV_ERR_UNSUPPORTED, "template rows too wide for one block (q2 = %d, q3 = %d)", q2, q3);
    int chunks = std::max(1, (152 * 4 + q1 - 1) / q1);
    chunks = (int)std::min<size_t>((size_t)chunks, kScratchDoubles / nh);
    cdv::GradPsfPlan g{mm[0], mm[1], mm[2], q1, q2, q3, batch, chunks};
    const size_t smem = cdv::grad_psf_smem_bytes(g);
    if (smem == 0 || smem > cdv::kGradPsfMaxSmem)
        return fail(CDV_ERR_UNSUPPORTED, "template rows need %zu bytes of shared memory per block (at most %zu)",
                    smem, cdv::kGradPsfMaxSmem);
    double* scratch = nullptr;
    cdv_status st = scratch_for_current_device(&scratch);
    if (st != CDV_OK) return st;
    cudaError_t e = cdv::launch_grad_psf(g, X, dY, scratch, dH, (cudaStream_t)stream);
    if (e != cudaSuccess) return fail(CDV_ERR_CUDA, "grad_psf (static scratch): %s", cudaGetErrorString(e));
    return CDV_OK;
}
