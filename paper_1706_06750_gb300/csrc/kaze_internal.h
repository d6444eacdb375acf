// kaze_internal.h -- declarations shared by the CUDA translation units of
// libkaze.so (kernels and the C ABI host runtime).  Not part of the ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kaze.h"

namespace kz {

constexpr int kMaxLevels = 64;     // N = O*S upper bound
constexpr int kMaxGaussR = 16;     // presmoothing radius bound (sigma <= 5.33)
constexpr int kMaxGradR = 6;       // gradient-smoothing radius bound (sigma_d <= 2)
constexpr int kMaxBins = 4096;
constexpr int kMaxDynSmem = 227 * 1024;  // opt-in dynamic shared memory per CTA

// Sampled, normalised Gaussian taps w[0..2r] for offsets -r..r.
struct GaussTaps {
    int r;
    float w[2 * kMaxGaussR + 1];
};

// Per-level constants of the detector (Eq. 6-8), passed by value.
struct LevelTable {
    int n;                       // number of levels in the table
    int step[kMaxLevels];        // derivative step s_i
    float norm[kMaxLevels];      // DoH normalisation factor
    float sigma[kMaxLevels];     // sigma_i
    int sublevels;               // S (octave = i / S, sublevel = i % S)
};

// Half-sample symmetric reflection of i into [0, n).
__host__ __device__ __forceinline__ int reflect_index(int i, int n)
{
    if (i >= 0 && i < n) return i;
    int p = 2 * n;
    int r = i % p;
    if (r < 0) r += p;
    return r < n ? r : p - 1 - r;
}

// Raises a kernel's dynamic shared-memory limit to what the device allows
// beside the kernel's static shared memory.
template <typename F>
inline cudaError_t allow_max_dynamic_smem(F* func)
{
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, (const void*)func);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute((const void*)func, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                optin - (int)fa.sharedSizeBytes);
}

// Raise every kernel's dynamic shared-memory limit once (outside any stream
// capture); launches then pass their actual size.
cudaError_t configure_filter_kernels();
cudaError_t configure_aos_kernels();
const char* aos_config_error();  // why configure_aos_kernels failed, if it did
cudaError_t configure_detector_kernels();

// ---- launchers (all asynchronous on `st`; return the launch error) ----

cudaError_t launch_gaussian(const float* in, int in_pitch, float* out, int out_pitch,
                            int w, int h, const GaussTaps& taps, cudaStream_t st);

cudaError_t launch_conductance(const float* L, float* g, int pitch, int w, int h,
                               const GaussTaps& taps, const float* d_k, int diffusivity,
                               cudaStream_t st);

// Contrast factor: hmax pass, histogram pass, percentile pick.  hmax is kept
// as the bit pattern of a non-negative float (ordered like an unsigned int).
cudaError_t launch_grad_max(const float* L, int pitch, int w, int h, const GaussTaps& taps,
                            unsigned int* d_hmax_bits, cudaStream_t st);
cudaError_t launch_grad_hist(const float* L, int pitch, int w, int h, const GaussTaps& taps,
                             const unsigned int* d_hmax_bits, unsigned int* d_hist, int nbins,
                             cudaStream_t st);
cudaError_t launch_percentile(const unsigned int* d_hist, int nbins,
                              const unsigned int* d_hmax_bits, double pct, float* d_k,
                              cudaStream_t st);
cudaError_t launch_set_scalar(float* d_dst, float value, cudaStream_t st);

// AOS step of Eq. 4: rows (writes ux), then columns + average (writes Lnext).
// Rows need 16-byte aligned rows (pitch % 4 == 0); columns are staged by TMA
// tensor copies.  A bounded wait that runs out sets bit 0 of *d_status.
cudaError_t launch_aos_rows(const float* L, const float* g, float* ux, int pitch,
                            int w, int h, float tau, int* d_status, cudaStream_t st);
cudaError_t launch_aos_cols(const float* L, const float* g, const float* ux, float* Lnext,
                            int pitch, int w, int h, float tau, int* d_status, cudaStream_t st);
size_t aos_rows_smem_bytes(int w);
size_t aos_cols_smem_bytes(int h);

// Detector response of Eq. 8 for levels [l0, l0 + nl) of a level stack.
cudaError_t launch_doh(const float* L, float* D, int pitch, long long plane_stride,
                       int w, int h, int l0, int nl, const LevelTable& tab, cudaStream_t st);

// 3x3x3 maxima on levels [1, n-2] of a response stack.
cudaError_t launch_extrema(const float* D, int pitch, long long plane_stride, int w, int h,
                           int n, const LevelTable& tab, float dthreshold, float edge_r,
                           kaze_keypoint* d_kp, int cap, unsigned int* d_count,
                           cudaStream_t st);

// Handle runtime helpers used by the batch API (kaze_api.cu).
kaze_status handle_enqueue_into(kaze_handle* h, const float* d_img, int w, int hh, int pitch, float* levels,
                                float* doh, kaze_keypoint* d_kp, unsigned int* d_count, int cap);
int* handle_status_ptr(kaze_handle* h);

}  // namespace kz
