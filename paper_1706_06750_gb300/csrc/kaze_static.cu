// kaze_static.cu -- one AOS step that allocates no memory.
//
// Some callers cannot let a library call cudaMalloc: a framework whose
// caching allocator owns all device memory, or a processing loop that must
// not allocate once it is running.  kaze_aos_step_static serves them: the
// caller passes its inputs and output, and the one intermediate the step
// needs -- the row solution of the splitting, read back by the column pass --
// lives in a file-scope device array of fixed size instead of a handle's
// buffers.  Every GPU that loads the library holds that array (16 MiB) until
// the process exits.
#include <mutex>

#include "kaze_internal.h"

#define KAZE_API extern "C" __attribute__((visibility("default")))

namespace {

constexpr long long kStaticMaxPixels = 4ll * 1024 * 1024;  // pitch * h limit (16 MiB of floats)
constexpr int kMaxDevices = 64;

// Row-solution scratch and the status word of the bounded device waits,
// shared by every call on a device.
static __device__ __align__(256) float g_static_ux[kStaticMaxPixels];
static __device__ __align__(256) int g_static_status[1];

struct DeviceScratch {
    bool ready = false;
    float* ux = nullptr;
    int* status = nullptr;
};
DeviceScratch g_scratch[kMaxDevices];
std::mutex g_scratch_mu;

// First use on a device (which must be current): device addresses of the
// file-scope arrays and the kernels' shared-memory limits.  The addresses are
// cached per device ordinal for the life of the process; a cudaDeviceReset
// invalidates them and is not supported.
kaze_status setup_current_device(DeviceScratch** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return KAZE_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    DeviceScratch& s = g_scratch[dev];
    if (!s.ready) {
        if (cudaGetSymbolAddress((void**)&s.ux, g_static_ux) != cudaSuccess) return KAZE_ERR_CUDA;
        if (cudaGetSymbolAddress((void**)&s.status, g_static_status) != cudaSuccess) return KAZE_ERR_CUDA;
        if (kz::configure_aos_kernels() != cudaSuccess) return KAZE_ERR_CUDA;
        s.ready = true;
    }
    *out = &s;
    return KAZE_OK;
}

}  // namespace

KAZE_API kaze_status kaze_aos_step_static(const float* d_Lprev, const float* d_g, float* d_Lnext, int pitch, int w,
                                          int h, float tau, void* cuda_stream)
{
    if (!d_Lprev || !d_g || !d_Lnext) return KAZE_ERR_INVALID_ARG;
    if (w < 3 || h < 3 || pitch < w || pitch % 4) return KAZE_ERR_INVALID_ARG;
    if ((long long)pitch * h > kStaticMaxPixels) return KAZE_ERR_INVALID_ARG;
    if (kz::aos_rows_smem_bytes(w) == 0 || kz::aos_cols_smem_bytes(h) == 0) return KAZE_ERR_INVALID_ARG;
    if (((uintptr_t)d_Lprev | (uintptr_t)d_g | (uintptr_t)d_Lnext) & 15) return KAZE_ERR_INVALID_ARG;
    // the planes span pitch * (h - 1) + w floats; the output may not overlap
    // either input anywhere (the column pass writes while it still reads)
    const size_t span = sizeof(float) * ((size_t)pitch * (h - 1) + w);
    if (kz::ranges_overlap(d_Lnext, d_Lprev, span) || kz::ranges_overlap(d_Lnext, d_g, span))
        return KAZE_ERR_INVALID_ARG;
    if (!(tau >= 0.f)) return KAZE_ERR_INVALID_ARG;
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    // the scratch address belongs to the current device: the stream must too
    int cur = 0, sdev = 0;
    if (cudaGetDevice(&cur) != cudaSuccess || cudaStreamGetDevice(stream, &sdev) != cudaSuccess)
        return KAZE_ERR_CUDA;
    if (sdev != cur) return KAZE_ERR_INVALID_ARG;
    DeviceScratch* s = nullptr;
    const kaze_status st = setup_current_device(&s);
    if (st != KAZE_OK) return st;
    // the array keeps the previous call's contents: the status word must
    // start at zero, the row solution is overwritten before it is read
    if (cudaMemsetAsync(s->status, 0, sizeof(int), stream) != cudaSuccess) return KAZE_ERR_CUDA;
    if (kz::launch_aos_rows(d_Lprev, d_g, s->ux, nullptr, pitch, w, h, tau, s->status, stream) != cudaSuccess)
        return KAZE_ERR_CUDA;
    if (kz::launch_aos_cols(d_Lprev, d_g, s->ux, d_Lnext, pitch, w, h, tau, s->status, stream) != cudaSuccess)
        return KAZE_ERR_CUDA;
    int host_status = 0;
    if (cudaMemcpyAsync(&host_status, s->status, sizeof(int), cudaMemcpyDeviceToHost, stream) != cudaSuccess)
        return KAZE_ERR_CUDA;
    if (cudaStreamSynchronize(stream) != cudaSuccess) return KAZE_ERR_CUDA;
    return host_status ? KAZE_ERR_TIMEOUT : KAZE_OK;
}
