// gl_noalloc.cu -- the photometric loss for callers that must not allocate
// device memory during the call.
//
// gl_photometric_loss keeps its per-tile partial sums in scratch owned by a
// gl_ctx, which grows with cudaMalloc.  Here the same kernels write their
// partials into one fixed, file-scope device array instead.  The array is
// part of the library image: every GPU that loads the library holds it until
// the process exits, and every call shares it.
#include <mutex>

#include "gl_internal.h"

namespace gl {
namespace {

// Partial sums: 14 floats per 32x32 output tile; 16,384 tiles cover up to
// 4096 x 4096 pixels (any width x height with that many tiles or fewer).
constexpr int kNoallocMaxTiles = 16384;
constexpr int kNoallocFloats = kNoallocMaxTiles * 14;   // 917,504 bytes

static __device__ __align__(256) float g_loss_scratch[kNoallocFloats];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
float* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (host code cannot use the symbol itself as a device address).
gl_status scratch_on_current_device(float** out)
{
    int dev = 0;
    GL_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("device ordinal out of range for the fixed-scratch loss");
        return GL_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        GL_CUDA_TRY(cudaGetSymbolAddress(&p, g_loss_scratch));
        g_scratch_addr[dev] = static_cast<float*>(p);
    }
    *out = g_scratch_addr[dev];
    return GL_OK;
}

}  // namespace
}  // namespace gl

using namespace gl;

extern "C" gl_status gl_photometric_loss_noalloc(const float* rgb, const float* target, const float* E34,
                                                 int32_t width, int32_t height, float lambda_dssim,
                                                 float* loss_out, float* dL_drgb, float* dL_dE,
                                                 void* cuda_stream)
{
    if (!rgb || !target || !E34 || !dL_drgb) { set_error("null argument"); return GL_ERR_INVALID; }
    if (width <= 0 || height <= 0) { set_error("bad image size"); return GL_ERR_INVALID; }
    if (!(lambda_dssim >= 0.f && lambda_dssim <= 1.f)) { set_error("lambda must be in [0,1]"); return GL_ERR_INVALID; }
    const int64_t need = (int64_t)loss_partials_needed(width, height);
    if (need > kNoallocFloats) {
        set_error("image too large for the fixed loss scratch: at most 16384 tiles of 32x32 pixels "
                  "(for example 4096 x 4096)");
        return GL_ERR_INVALID;
    }
    float* part = nullptr;
    GL_TRY(scratch_on_current_device(&part));
    // Every partial the reduction reads is written by this call's tile pass,
    // so nothing in the shared array needs clearing first.
    return photometric_loss(rgb, target, E34, width, height, lambda_dssim, dL_drgb, part, loss_out, dL_dE,
                            static_cast<cudaStream_t>(cuda_stream));
}
