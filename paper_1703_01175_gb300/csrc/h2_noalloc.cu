// h2_matvec_noalloc: the single-RHS FP32 H^2 product with its coefficient
// scratch in a static device array instead of memory the handle allocated.
//
// Who needs it: code that runs where the CUDA allocator must not be called.
// Examples are a solver step embedded in another framework whose caching
// allocator has reserved all device memory, or a control loop with a
// real-time budget where cudaMalloc's implicit device synchronisation is not
// allowed. Such a caller loads the operator once at initialisation (h2_load
// allocates) and from then on only passes x and y.
//
// The scratch holds the forward-transform coefficients xh and the backward
// coefficients yh (2 * sum of ranks complex64 entries). It is one array per
// GPU that loads the library, kept until the process exits.
#include <cuda_runtime.h>

#include <string>

#include "h2_internal.h"

static __device__ __align__(256) float2 g_h2_noalloc_scratch[H2_NOALLOC_MAX_COEF];

namespace {

// Device address of the scratch array in the current context. The host-side
// symbol is only a stand-in and must never reach a kernel; the address is
// looked up with the handle's device current and kept in the handle, whose
// memory lives in that same context.
h2_status scratch_address(h2_handle *h, float2 **out)
{
    if (!h->noalloc_coef) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_h2_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            h2::set_error(std::string("h2_matvec_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            return H2_ERR_CUDA;
        }
        h->noalloc_coef = reinterpret_cast<float2 *>(p);
    }
    *out = h->noalloc_coef;
    return H2_OK;
}

}  // namespace

#define NA_CUDA(call)                                                                  \
    do {                                                                               \
        cudaError_t e__ = (call);                                                      \
        if (e__ != cudaSuccess) {                                                      \
            h2::set_error(std::string(#call) + ": " + cudaGetErrorString(e__));        \
            return H2_ERR_CUDA;                                                        \
        }                                                                              \
    } while (0)

extern "C" h2_status h2_matvec_noalloc(h2_handle *h, const void *x, void *y, void *stream)
{
    using namespace h2;
    if (!h || !x || !y) {
        set_error("h2_matvec_noalloc: NULL argument");
        return H2_ERR_ARG;
    }
    if (x == y) {
        set_error("h2_matvec_noalloc: x and y must not overlap");
        return H2_ERR_ARG;
    }
    const int64_t need = 2 * h->ktot;
    if (need > (int64_t)H2_NOALLOC_MAX_COEF) {
        set_error("h2_matvec_noalloc: the operator needs " + std::to_string(need) +
                  " scratch coefficients (2 x sum of ranks), above the limit of " +
                  std::to_string((long long)H2_NOALLOC_MAX_COEF));
        return H2_ERR_ARG;
    }
    DeviceGuard dev_guard(h->device);
    NA_CUDA(dev_guard.err);
    float2 *coef = nullptr;
    h2_status s = scratch_address(h, &coef);
    if (s != H2_OK) return s;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const float2 *xx = reinterpret_cast<const float2 *>(x);
    float2 *yy = reinterpret_cast<float2 *>(y);
    const float2 *mat = h->d_mat;
    const Seg *segs = h->d_segs;
    // the array keeps the previous call's values: the coefficients start at zero
    NA_CUDA(cudaMemsetAsync(coef, 0, sizeof(float2) * (size_t)std::max<int64_t>(1, need), st));
    NA_CUDA(cudaEventRecord(h->ev_fork, st));
    NA_CUDA(cudaStreamWaitEvent(h->s_aux, h->ev_fork, 0));
    NA_CUDA(launch_phase_f32(h->near, mat, segs, xx, coef, yy, 0, h->s_aux));
    NA_CUDA(cudaEventRecord(h->ev_near, h->s_aux));
    NA_CUDA(launch_phase_f32(h->upleaf, mat, segs, xx, coef, coef, 0, st));
    for (int l = h->nlev - 1; l >= 0; --l) NA_CUDA(launch_phase_f32(h->up[l], mat, segs, xx, coef, coef, 0, st));
    NA_CUDA(launch_phase_f32(h->couple, mat, segs, xx, coef, coef, 0, st));
    for (int l = 0; l < h->nlev; ++l) NA_CUDA(launch_phase_f32(h->down[l], mat, segs, xx, coef, coef, 1, st));
    NA_CUDA(cudaStreamWaitEvent(st, h->ev_near, 0));
    NA_CUDA(launch_phase_f32(h->leafexp, mat, segs, xx, coef, yy, 1, st));
    return H2_OK;
}
