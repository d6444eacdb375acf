// kaze_internal.h -- declarations shared by the CUDA translation units of
// libkaze.so (kernels and the C ABI host runtime).  Not part of the ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "kaze.h"

namespace kz {

constexpr int kMaxLevels = 64;     // N = O*S upper bound
constexpr int kMaxGaussR = 16;     // presmoothing radius bound (sigma <= 5.33)
constexpr int kMaxGradR = 6;       // gradient-smoothing radius bound (sigma_d <= 2)
constexpr int kMaxBins = 4096;
constexpr int kMaxDynSmem = 227 * 1024;  // opt-in dynamic shared memory per CTA
constexpr int kKeypointsWithCount = 4096;  // keypoint slots copied to the host with the count

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
    int xr[kMaxLevels];          // cross-level radius of the maximum test (1: 3x3x3)
    float doh_scale[kMaxLevels]; // norm / (1024 s^2)^2, filled by launch_doh
};

// Per-level constants of keypoint description (Sec. II-C), passed by value.
// single != 0: one caller-supplied level (entry 0) serves every keypoint.
struct DescTable {
    int n;
    int single;
    float sigma[kMaxLevels];
    int step[kMaxLevels];
};

// True when the byte ranges [a, a + bytes) and [b, b + bytes) intersect.
inline bool ranges_overlap(const void* a, const void* b, size_t bytes)
{
    const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
    return x < y + bytes && y < x + bytes;
}

// Half-sample symmetric reflection of i into [0, n).
__host__ __device__ __forceinline__ int reflect_index(int i, int n)
{
    if (i >= 0 && i < n) return i;
    int p = 2 * n;
    int r = i % p;
    if (r < 0) r += p;
    return r < n ? r : p - 1 - r;
}

// Response arithmetic of Eq. 8 shared by the single-image and batched
// kernels (explicit fmaf, so both give the same bits).  One lattice row
// (taps at -2s .. 2s): the x-derivative pair [1 0 -2 0 1], the smoothing
// [9 60 118 60 9] and the first derivative [-3 -10 0 10 3].
__device__ __forceinline__ void doh_lattice_row(float v0, float v1, float v2, float v3, float v4, float& hd,
                                                float& hs, float& hx)
{
    hd = fmaf(-2.f, v2, v0 + v4);
    hs = fmaf(118.f, v2, fmaf(60.f, v1 + v3, 9.f * (v0 + v4)));
    hx = fmaf(10.f, v3 - v1, 3.f * (v4 - v0));
}

// The determinant from five consecutive filtered lattice rows a[0..4].
__device__ __forceinline__ float doh_value(const float* hd, const float* hs, const float* hx, float scale)
{
    const float lxx = fmaf(118.f, hd[2], fmaf(60.f, hd[1] + hd[3], 9.f * (hd[0] + hd[4])));
    const float lyy = fmaf(-2.f, hs[2], hs[0] + hs[4]);
    const float lxy = fmaf(10.f, hx[3] - hx[1], 3.f * (hx[4] - hx[0]));
    return scale * fmaf(lxx, lyy, -(lxy * lxy));
}

// Contrast factor k from the histogram of gradient magnitudes (Sec. III-1,
// reading R4), on one full warp: lane l owns a contiguous slice of bins, the
// slice sums are prefix-summed with shuffles, and the lane whose slice
// crosses pct * n walks its bins; k = hmax (b + 1) / nbins for the first bin
// b where the cumulative count reaches pct * n, 0.03 when nothing was binned.
// Returns k to every lane.
__device__ __forceinline__ float percentile_k(const unsigned int* hist, int nbins, float hmax, double pct, int lane)
{
    const int per = (nbins + 31) / 32;
    const int b0 = min(lane * per, nbins), b1 = min(b0 + per, nbins);
    unsigned long long s = 0;
    for (int b = b0; b < b1; ++b) s += hist[b];
    unsigned long long inc = s;
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    const unsigned long long n = __shfl_sync(0xffffffffu, inc, 31);
    if (n == 0 || !(hmax > 0.f)) return 0.03f;
    const double target = pct * (double)n;
    const unsigned ballot = __ballot_sync(0xffffffffu, (double)inc >= target);
    if (ballot == 0u) return 0.03f;
    const int src = __ffs(ballot) - 1;
    float k = 0.03f;
    if (lane == src) {
        unsigned long long cum = inc - s;
        for (int b = b0; b < b1; ++b) {
            cum += hist[b];
            if ((double)cum >= target) {
                k = hmax * (float)(b + 1) / (float)nbins;
                break;
            }
        }
    }
    return __shfl_sync(0xffffffffu, k, src);
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

// g of Eq. 3 from L; if zero_out is not null it also receives zeros at the
// same pixels (the accumulation target of the next AOS step).
cudaError_t launch_conductance(const float* L, float* g, float* zero_out, int pitch, int w, int h,
                               const GaussTaps& taps, const float* d_k, int diffusivity,
                               cudaStream_t st);

// Contrast factor: hmax pass, histogram pass, percentile pick.  hmax is kept
// as the bit pattern of a non-negative float (ordered like an unsigned int).
// m2_out (optional): receives |grad|^2 of every pixel, for launch_hist_m2
// and launch_cond_m2 (the same values the gradient kernels compute).
cudaError_t launch_grad_max(const float* L, int pitch, int w, int h, const GaussTaps& taps,
                            unsigned int* d_hmax_bits, cudaStream_t st, float* m2_out = nullptr);
// The histogram pass and the conductance (in place, zeroing zero_out) from
// such a plane; rows 16-byte aligned, pitch % 4 == 0.
// launch_hist_m2 also picks the percentile (its last block): d_hist holds
// nbins + 1 counters, all zero before the launch, and k lands in d_k.
cudaError_t launch_hist_m2(const float* m2, int pitch, int w, int h, const unsigned int* d_hmax_bits,
                           unsigned int* d_hist, int nbins, double pct, float* d_k, cudaStream_t st);
cudaError_t launch_cond_m2(float* gm, float* zero_out, int pitch, int w, int h, const float* d_k, int diffusivity,
                           cudaStream_t st);
cudaError_t launch_grad_hist(const float* L, int pitch, int w, int h, const GaussTaps& taps,
                             const unsigned int* d_hmax_bits, unsigned int* d_hist, int nbins,
                             cudaStream_t st);
cudaError_t launch_percentile(const unsigned int* d_hist, int nbins,
                              const unsigned int* d_hmax_bits, double pct, float* d_k,
                              cudaStream_t st);
cudaError_t launch_set_scalar(float* d_dst, float value, cudaStream_t st);

// AOS step of Eq. 4, L_next = (u_x + u_y) / 2.  Either sequentially: rows
// write u_x to ux (acc == nullptr), then columns read it and write Lnext; or
// as two independent halves that may run concurrently: with Lnext zeroed
// beforehand, rows add u_x / 2 into acc == Lnext and columns (ux == nullptr)
// add u_y / 2 into Lnext (two addends onto zero: the same sum in either
// order).  Rows need 16-byte aligned rows (pitch % 4 == 0); columns are
// staged by TMA tensor copies.  A bounded wait that runs out sets bit 0 of
// *d_status.
cudaError_t launch_aos_rows(const float* L, const float* g, float* ux, float* acc, int pitch,
                            int w, int h, float tau, int* d_status, cudaStream_t st);
// cols: columns per CTA (4 or 8); 0 picks the widest that fits.
cudaError_t launch_aos_cols(const float* L, const float* g, const float* ux, float* Lnext,
                            int pitch, int w, int h, float tau, int* d_status, cudaStream_t st, int cols = 0);
size_t aos_rows_smem_bytes(int w);
size_t aos_cols_smem_bytes(int h);

// The whole AOS evolution (levels 1..n_levels-1 from level 0) in one
// cooperative launch with each 128 x 120 tile resident in shared memory
// (k_evolve.cu).  evolve_fits: whether a w x h image with a gradient
// smoothing radius `radius` can take it on the current device (tiles one per
// SM); `exchange` holds evolve_exchange_floats(max_tiles) floats, `barrier`
// one counter (zeroed by the launch unless zero_barrier is false: the
// caller did); a timed-out grid barrier sets bit 0 of *status.  wait_limit:
// SM cycles a barrier wait may take (0: 2^31); stall_tile >= 0 (a test
// hook) makes that tile never arrive, so every wait runs out.
// The front of the pipeline inside the same launch: with `img`, level 0 is
// the presmoothing of the image (radius taps0->r == 5, sigma0 in (4/3, 5/3])
// instead of being read;
// with `hist` too (nbins counters and hmax_bits zeroed beforehand, nbins <=
// 1030), the contrast factor is measured inside (maximum and histogram of
// step 1's gradient magnitudes, the percentile pct) and written to d_k.
struct EvolveFront {
    const float* img = nullptr;
    int img_pitch = 0;
    const GaussTaps* taps0 = nullptr;
    unsigned int* hmax_bits = nullptr;
    unsigned int* hist = nullptr;
    int nbins = 0;
    double pct = 0.0;
};
// The batched form: one cooperative launch of evolve_batch_grid() CTAs (one
// per SM) evolving many images, each image's tiles on distinct CTAs of one
// wave (work: (image, tile) pairs, CTA b taking work[off[b] .. off[b + 1])
// in order; every image's tiles fit the grid).  The parameters of image i
// are the evolve_params_bytes() bytes at d_params + i * that size, made by
// evolve_batch_params (false: the image does not take the resident
// evolution).  Each image has its own exchange (evolve_exchange_floats of its
// tiles) and barrier counter, zeroed before the launch; hist null takes k
// from k_fixed > 0 (written to d_k), else from d_k.
struct EvolveImage {
    float* levels = nullptr;
    long long plane = 0;
    int pitch = 0, w = 0, h = 0;
    const float* img = nullptr;  // presmoothed into level 0 inside the launch
    int img_pitch = 0;
    const GaussTaps* taps0 = nullptr;
    float* d_k = nullptr;
    unsigned int* hmax_bits = nullptr;
    unsigned int* hist = nullptr;
    int nbins = 0;
    double pct = 0.0;
    float k_fixed = 0.f;
    float* exchange = nullptr;
    unsigned int* barrier = nullptr;
};
// The streamed form for images whose tiles exceed one per SM (up to 64 x 64
// tiles): each step as three launches, pass 0 (conductance and records of
// every tile; g to the plane `g`), pass 1 (every segment's outside
// neighbours from its line's records), pass 2 (the re-solves, L_lev to its
// plane), for lev = 1 .. n_levels - 1 in order.  `scratch` holds
// evolve_stream_floats(w, h) floats; *d_k holds the contrast factor.
size_t evolve_stream_floats(int max_w, int max_h);
bool evolve_stream_fits(int w, int h, int radius);
cudaError_t launch_stream_pass(int pass, int lev, float* levels, long long plane, int pitch, int w, int h,
                               int n_levels, const double* t, float* d_k, const GaussTaps& taps, int diffusivity,
                               float* g, float* scratch, cudaStream_t st);
size_t evolve_params_bytes();
bool evolve_batch_params(void* out, const EvolveImage& im, int n_levels, const double* t, const GaussTaps& taps,
                         int diffusivity, int* status, long long wait_limit, int stall_tile);
int evolve_batch_grid();
cudaError_t launch_evolve_batch(const void* d_params, const int2* d_work, const int* d_off, int grid,
                                cudaStream_t st);
cudaError_t configure_evolve_kernel();
size_t evolve_exchange_floats(int max_tiles);
bool evolve_fits(int w, int h, int radius, int* tiles);
bool evolve_front_fits(int r0, int nbins);
cudaError_t launch_evolve(float* levels, long long plane, int pitch, int w, int h, int n_levels, const double* t,
                          float* d_k, const GaussTaps& taps, int diffusivity, float* exchange, int max_tiles,
                          unsigned int* barrier, int* status, cudaStream_t st, const EvolveFront* front = nullptr,
                          long long wait_limit = 0, int stall_tile = -1, bool zero_barrier = true);

// The pixels the extremum test of Sec. III-2 can accept: response above the
// threshold, on a level in [lo, hi] (1 .. N-2), one pixel or more inside the
// image.  The response kernel appends them as (level << 48 | y << 24 | x);
// the extremum kernel then visits only those, and scans every pixel when more
// than `cap` were found (*count > cap).  *count is zeroed before the response
// launch.
struct Candidates {
    unsigned long long* list = nullptr;
    unsigned int* count = nullptr;
    unsigned int cap = 0;
    float thr = 0.f;
    int lo = 1, hi = 0;
};

// Detector response of Eq. 8 for levels [l0, l0 + nl) of a level stack.
// Number of kernels launch_doh issues for levels l0 .. l0 + nl - 1.
int doh_launches(const LevelTable& tab, int l0, int nl);
cudaError_t launch_doh(const float* L, float* D, int pitch, long long plane_stride,
                       int w, int h, int l0, int nl, const LevelTable& tab, cudaStream_t st,
                       const Candidates* cand = nullptr);

// 3x3x3 maxima on levels [1, n-2] of a response stack (with `cand`: the
// pixels the response launch listed).
cudaError_t launch_extrema(const float* D, int pitch, long long plane_stride, int w, int h,
                           int n, const LevelTable& tab, float dthreshold, float edge_r,
                           kaze_keypoint* d_kp, int cap, unsigned int* d_count,
                           cudaStream_t st, const Candidates* cand = nullptr);

// FED (Eq. 5): the step sizes of one cycle reaching stopping time dt with
// stability limit tau_max (the smallest n whose cycle time tau_max (n^2+n)/3
// reaches dt, sizes scaled to sum to dt); writes min(n, cap), returns n.
int fed_cycle(double dt, double tau_max, double* tau, int cap);
// The same sizes in the step order the library takes them (kappa cycle of
// the smallest worst-case rounding amplification).
std::vector<double> fed_ordered_steps(double dt, double tau_max);
// One explicit step L_out = L_in + tau div(g grad L_in) (flux form, no flux
// through the border); rows 16-byte aligned, pitch % 4 == 0.
cudaError_t launch_fed_step(const float* Lin, const float* g, float* Lout, int pitch, int w, int h, float tau,
                            cudaStream_t st);
// k <= fed_max_fused() consecutive explicit steps (sizes tau[0..k-1]) in one
// launch, bit-identical to k one-step launches; Lout must not alias Lin or g
// (a timed-out staging wait sets bit 0 of *status)
cudaError_t launch_fed_steps(const float* Lin, const float* g, float* Lout, int pitch, int w, int h, const float* tau,
                             int k, int* status, cudaStream_t st);
cudaError_t configure_fed_kernels();
int fed_max_fused();
// a cycle of n steps split into launches of fed_max_fused() steps and the remainder
std::vector<int> fed_chunks(int n);

// Orientation and 64-D M-SURF descriptor of n device keypoints (angle
// written back into d_kps, descriptors to d_desc, n x 64); keypoint k lies on
// level kps[k].level of the stack (or on the single level).  Tables are
// uploaded by configure_describe_kernels.
cudaError_t configure_describe_kernels();
cudaError_t launch_describe(const float* levels, long long plane_stride, int pitch, int w, int h,
                            const DescTable& tab, kaze_keypoint* d_kps, int n, float* d_desc, int upright,
                            cudaStream_t st);

// Handle runtime helpers used by the batch API (kaze_api.cu).
kaze_status handle_enqueue_into(kaze_handle* h, const float* d_img, int w, int hh, int pitch, float* levels,
                                float* doh, kaze_keypoint* d_kp, unsigned int* d_count, int cap);
int* handle_status_ptr(kaze_handle* h);

}  // namespace kz
