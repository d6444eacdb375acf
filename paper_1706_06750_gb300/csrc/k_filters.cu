// k_filters.cu -- stencil kernels of the nonlinear scale space (Sec. III-1):
//   * Gaussian presmoothing of the input image,
//   * the fused "smooth -> Scharr -> conductance" kernel (Eq. 2-3),
//   * the two gradient-statistics passes and the percentile pick that give
//     the contrast factor k from the gradient histogram.
//
// All three stencil kernels share one tiling: a CTA of 32x8 threads owns a
// 32x32 output tile, stages its input tile plus halo in shared memory with
// half-sample symmetric borders (index reflection on load), runs the
// separable Gaussian rows-then-columns in shared memory and finishes with a
// 3x3 Scharr stencil where needed.  The inputs are read once from HBM/L2;
// halo re-reads come from neighbouring tiles and hit L2.
#include "kaze_internal.h"

namespace kz {
namespace {

constexpr int TX = 32;  // output tile width
constexpr int TY = 32;  // output tile height
constexpr int BX = 32;  // threads per CTA, x
constexpr int BY = 8;   // threads per CTA, y

// Separable Gaussian: rows first, then columns (same order as the method's
// definition of the presmoothing).
__global__ void __launch_bounds__(BX* BY)
k_gaussian(const float* __restrict__ in, int in_pitch, float* __restrict__ out, int out_pitch,
           int w, int h, const __grid_constant__ GaussTaps taps)
{
    extern __shared__ float sm[];
    const int r = taps.r;
    const int SW = TX + 2 * r;
    const int SH = TY + 2 * r;
    float* A = sm;            // SH x SW input tile
    float* B = sm + SH * SW;  // SH x TX row-filtered tile
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int tid = threadIdx.y * BX + threadIdx.x;
    constexpr int NT = BX * BY;

    for (int i = tid; i < SH * SW; i += NT) {
        int sy = i / SW, sx = i - sy * SW;
        int gy = reflect_index(y0 - r + sy, h), gx = reflect_index(x0 - r + sx, w);
        A[i] = __ldg(in + (size_t)gy * in_pitch + gx);
    }
    __syncthreads();
    for (int i = tid; i < SH * TX; i += NT) {
        int sy = i / TX, sx = i - sy * TX;
        const float* a = A + sy * SW + sx;
        float acc = 0.f;
        for (int j = 0; j <= 2 * r; ++j) acc = fmaf(taps.w[j], a[j], acc);
        B[i] = acc;
    }
    __syncthreads();
    for (int ty = threadIdx.y; ty < TY; ty += BY) {
        int gx = x0 + threadIdx.x, gy = y0 + ty;
        if (gx >= w || gy >= h) continue;
        const float* b = B + ty * TX + threadIdx.x;
        float acc = 0.f;
        for (int j = 0; j <= 2 * r; ++j) acc = fmaf(taps.w[j], b[j * TX], acc);
        out[(size_t)gy * out_pitch + gx] = acc;
    }
}

enum GradMode { MODE_COND = 0, MODE_MAX = 1, MODE_HIST = 2 };

// Smoothed Scharr gradient of a 32x32 tile.  Stages L with a halo of r+1,
// smooths with G(sigma_d) on a (32+2)^2 region, then applies the 3x3 Scharr
// pair ([-1 0 1]/2 x [3 10 3]/16 and its transpose).  MODE_COND writes the
// conductance g of Eq. 3; MODE_MAX folds |grad| of interior pixels into a
// global maximum; MODE_HIST bins the non-zero interior magnitudes.
template <int MODE>
__global__ void __launch_bounds__(BX* BY)
k_gradient(const float* __restrict__ L, float* __restrict__ g, int pitch, int w, int h,
           const __grid_constant__ GaussTaps taps, const float* __restrict__ d_k, int diffusivity,
           unsigned int* __restrict__ d_hmax_bits, unsigned int* __restrict__ d_hist, int nbins)
{
    extern __shared__ float sm[];
    const int r = taps.r;
    constexpr int CW = TX + 2, CH = TY + 2;  // smoothed region (halo 1 for Scharr)
    const int SW = CW + 2 * r, SH = CH + 2 * r;
    float* A = sm;                 // SH x SW   raw L
    float* B = A + SH * SW;        // SH x CW   row-smoothed
    float* C = B + SH * CW;        // CH x CW   smoothed
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int tid = threadIdx.y * BX + threadIdx.x;
    constexpr int NT = BX * BY;

    unsigned int* hist_s = reinterpret_cast<unsigned int*>(C + CH * CW);
    if (MODE == MODE_HIST) {
        for (int i = tid; i < nbins; i += NT) hist_s[i] = 0u;
    }
    for (int i = tid; i < SH * SW; i += NT) {
        int sy = i / SW, sx = i - sy * SW;
        int gy = reflect_index(y0 - 1 - r + sy, h), gx = reflect_index(x0 - 1 - r + sx, w);
        A[i] = __ldg(L + (size_t)gy * pitch + gx);
    }
    __syncthreads();
    for (int i = tid; i < SH * CW; i += NT) {
        int sy = i / CW, sx = i - sy * CW;
        const float* a = A + sy * SW + sx;
        float acc = 0.f;
        for (int j = 0; j <= 2 * r; ++j) acc = fmaf(taps.w[j], a[j], acc);
        B[i] = acc;
    }
    __syncthreads();
    for (int i = tid; i < CH * CW; i += NT) {
        int sy = i / CW, sx = i - sy * CW;
        const float* b = B + sy * CW + sx;
        float acc = 0.f;
        for (int j = 0; j <= 2 * r; ++j) acc = fmaf(taps.w[j], b[j * CW], acc);
        C[i] = acc;
    }
    __syncthreads();

    float kk = 0.f, hmax = 0.f;
    if (MODE == MODE_COND) kk = *d_k;
    if (MODE == MODE_HIST) hmax = __uint_as_float(*d_hmax_bits);
    float local_max = 0.f;
    const float c0 = 3.f / 16.f, c1 = 10.f / 16.f;

    for (int ty = threadIdx.y; ty < TY; ty += BY) {
        const int tx = threadIdx.x;
        const int gx = x0 + tx, gy = y0 + ty;
        if (gx >= w || gy >= h) continue;
        // C(cx, cy) holds the smoothed value at (x0 - 1 + cx, y0 - 1 + cy).
        const float* c = C + (ty + 1) * CW + (tx + 1);
        float lx = c0 * 0.5f * (c[-CW + 1] - c[-CW - 1]);
        lx += c1 * 0.5f * (c[1] - c[-1]);
        lx += c0 * 0.5f * (c[CW + 1] - c[CW - 1]);
        float ly = c0 * 0.5f * (c[CW - 1] - c[-CW - 1]);
        ly += c1 * 0.5f * (c[CW] - c[-CW]);
        ly += c0 * 0.5f * (c[CW + 1] - c[-CW + 1]);
        if (MODE == MODE_COND) {
            float q = (lx * lx + ly * ly) / (kk * kk);
            g[(size_t)gy * pitch + gx] = diffusivity == KAZE_G1 ? expf(-q) : 1.f / (1.f + q);
        } else {
            bool interior = gx >= 1 && gx <= w - 2 && gy >= 1 && gy <= h - 2;
            if (!interior) continue;
            float m = sqrtf(lx * lx + ly * ly);
            if (MODE == MODE_MAX) {
                local_max = fmaxf(local_max, m);
            } else if (m > 0.f) {
                int b = (int)floorf((float)nbins * m / hmax);
                b = min(b, nbins - 1);
                atomicAdd(&hist_s[b], 1u);
            }
        }
    }
    if (MODE == MODE_MAX) {
        for (int o = 16; o > 0; o >>= 1) local_max = fmaxf(local_max, __shfl_xor_sync(0xffffffffu, local_max, o));
        // non-negative floats order like their bit patterns
        if (threadIdx.x == 0 && local_max > 0.f) atomicMax(d_hmax_bits, __float_as_uint(local_max));
    }
    if (MODE == MODE_HIST) {
        __syncthreads();
        for (int i = tid; i < nbins; i += NT) {
            unsigned int v = hist_s[i];
            if (v) atomicAdd(&d_hist[i], v);
        }
    }
}

// Percentile pick on one warp: lane l owns a contiguous slice of bins, the
// slice sums are prefix-summed with shuffles, and the lane whose slice
// crosses pct * n walks its bins.  k = hmax * (b + 1) / nbins; 0.03 when no
// pixel was binned.
__global__ void k_percentile(const unsigned int* __restrict__ hist, int nbins,
                             const unsigned int* __restrict__ d_hmax_bits, double pct,
                             float* __restrict__ d_k)
{
    const int lane = threadIdx.x;
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
    const float hmax = __uint_as_float(*d_hmax_bits);
    if (n == 0 || !(hmax > 0.f)) {
        if (lane == 0) *d_k = 0.03f;
        return;
    }
    const double target = pct * (double)n;
    const unsigned ballot = __ballot_sync(0xffffffffu, (double)inc >= target);
    if (ballot == 0u) {
        if (lane == 0) *d_k = 0.03f;
        return;
    }
    if (lane == __ffs(ballot) - 1) {
        unsigned long long cum = inc - s;
        for (int b = b0; b < b1; ++b) {
            cum += hist[b];
            if ((double)cum >= target) {
                *d_k = hmax * (float)(b + 1) / (float)nbins;
                break;
            }
        }
    }
}

__global__ void k_set_scalar(float* d, float v) { *d = v; }

size_t gradient_smem(int r, int nbins, int mode)
{
    const int CW = TX + 2, CH = TY + 2;
    const int SW = CW + 2 * r, SH = CH + 2 * r;
    size_t f = (size_t)SH * SW + (size_t)SH * CW + (size_t)CH * CW;
    return f * sizeof(float) + (mode == MODE_HIST ? (size_t)nbins * sizeof(unsigned int) : 0);
}

template <int MODE>
cudaError_t launch_gradient(const float* L, float* g, int pitch, int w, int h, const GaussTaps& taps,
                            const float* d_k, int diffusivity, unsigned int* hmax_bits,
                            unsigned int* hist, int nbins, cudaStream_t st)
{
    dim3 grid((w + TX - 1) / TX, (h + TY - 1) / TY);
    size_t smem = gradient_smem(taps.r, nbins, MODE);
    k_gradient<MODE><<<grid, dim3(BX, BY), smem, st>>>(L, g, pitch, w, h, taps, d_k, diffusivity,
                                                       hmax_bits, hist, nbins);
    return cudaGetLastError();
}

}  // namespace

cudaError_t configure_filter_kernels()
{
    const int cap = kMaxDynSmem;
    cudaError_t e = cudaFuncSetAttribute(k_gaussian, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gradient<MODE_COND>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gradient<MODE_MAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gradient<MODE_HIST>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
    return e;
}

cudaError_t launch_gaussian(const float* in, int in_pitch, float* out, int out_pitch, int w, int h,
                            const GaussTaps& taps, cudaStream_t st)
{
    const int r = taps.r;
    size_t smem = ((size_t)(TY + 2 * r) * (TX + 2 * r) + (size_t)(TY + 2 * r) * TX) * sizeof(float);
    dim3 grid((w + TX - 1) / TX, (h + TY - 1) / TY);
    k_gaussian<<<grid, dim3(BX, BY), smem, st>>>(in, in_pitch, out, out_pitch, w, h, taps);
    return cudaGetLastError();
}

cudaError_t launch_conductance(const float* L, float* g, int pitch, int w, int h, const GaussTaps& taps,
                               const float* d_k, int diffusivity, cudaStream_t st)
{
    return launch_gradient<MODE_COND>(L, g, pitch, w, h, taps, d_k, diffusivity, nullptr, nullptr, 0, st);
}

cudaError_t launch_grad_max(const float* L, int pitch, int w, int h, const GaussTaps& taps,
                            unsigned int* d_hmax_bits, cudaStream_t st)
{
    return launch_gradient<MODE_MAX>(L, nullptr, pitch, w, h, taps, nullptr, 0, d_hmax_bits, nullptr, 0, st);
}

cudaError_t launch_grad_hist(const float* L, int pitch, int w, int h, const GaussTaps& taps,
                             const unsigned int* d_hmax_bits, unsigned int* d_hist, int nbins,
                             cudaStream_t st)
{
    return launch_gradient<MODE_HIST>(L, nullptr, pitch, w, h, taps, nullptr, 0,
                                      const_cast<unsigned int*>(d_hmax_bits), d_hist, nbins, st);
}

cudaError_t launch_percentile(const unsigned int* d_hist, int nbins, const unsigned int* d_hmax_bits,
                              double pct, float* d_k, cudaStream_t st)
{
    k_percentile<<<1, 32, 0, st>>>(d_hist, nbins, d_hmax_bits, pct, d_k);
    return cudaGetLastError();
}

cudaError_t launch_set_scalar(float* d_dst, float value, cudaStream_t st)
{
    k_set_scalar<<<1, 1, 0, st>>>(d_dst, value);
    return cudaGetLastError();
}

}  // namespace kz
