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

// Separable Gaussian of radius R: rows first, then columns (the order of the
// method's definition of the presmoothing).  Loops have compile-time trip
// counts so each thread issues all of its staging loads before storing.
template <int R>
__global__ void __launch_bounds__(BX* BY)
k_gaussian(const float* __restrict__ in, int in_pitch, float* __restrict__ out, int out_pitch,
           int w, int h, const __grid_constant__ GaussTaps taps)
{
    constexpr int SW = TX + 2 * R, SH = TY + 2 * R;
    __shared__ float A[SH][SW + 1];  // input tile
    __shared__ float B[SH][TX + 1];  // row-filtered tile
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int tx = threadIdx.x, ty = threadIdx.y;

    int gx[(SW + BX - 1) / BX];
#pragma unroll
    for (int k = 0; k < (SW + BX - 1) / BX; ++k) gx[k] = reflect_index(x0 - R + tx + k * BX, w);
#pragma unroll
    for (int sy = ty; sy < SH; sy += BY) {
        const float* row = in + (size_t)reflect_index(y0 - R + sy, h) * in_pitch;
#pragma unroll
        for (int k = 0; k < (SW + BX - 1) / BX; ++k)
            if (tx + k * BX < SW) A[sy][tx + k * BX] = __ldg(row + gx[k]);
    }
    __syncthreads();
#pragma unroll
    for (int sy = ty; sy < SH; sy += BY) {
        float acc = 0.f;
#pragma unroll
        for (int j = 0; j <= 2 * R; ++j) acc = fmaf(taps.w[j], A[sy][tx + j], acc);
        B[sy][tx] = acc;
    }
    __syncthreads();
    const int ox = x0 + tx;
#pragma unroll
    for (int oy = ty; oy < TY; oy += BY) {
        float acc = 0.f;
#pragma unroll
        for (int j = 0; j <= 2 * R; ++j) acc = fmaf(taps.w[j], B[oy + j][tx], acc);
        if (ox < w && y0 + oy < h) out[(size_t)(y0 + oy) * out_pitch + ox] = acc;
    }
}

enum GradMode { MODE_COND = 0, MODE_MAX = 1, MODE_HIST = 2 };

// Smoothed Scharr gradient of a 32x32 tile.  Stages L with a halo of R+1,
// smooths with G(sigma_d) (radius R) on the (32+2)^2 region around the tile,
// then applies the 3x3 Scharr pair ([-1 0 1]/2 x [3 10 3]/16 and its
// transpose).  MODE_COND writes the conductance g of Eq. 3; MODE_MAX folds
// |grad| of interior pixels into a global maximum; MODE_HIST bins the
// non-zero interior magnitudes.
// Every pass works on runs of 4 consecutive outputs per thread so each
// shared-memory value loaded feeds several taps from registers.
template <int MODE, int R>
__global__ void __launch_bounds__(BX* BY)
k_gradient(const float* __restrict__ L, float* __restrict__ g, int pitch, int w, int h,
           const __grid_constant__ GaussTaps taps, const float* __restrict__ d_k, int diffusivity,
           unsigned int* __restrict__ d_hmax_bits, unsigned int* __restrict__ d_hist, int nbins)
{
    constexpr int CW = TX + 2, CH = TY + 2;      // smoothed region (halo 1 for Scharr)
    constexpr int SW = CW + 2 * R, SH = CH + 2 * R;
    constexpr int KX = (SW + BX - 1) / BX;
    constexpr int CWR = (CW + 3) / 4;            // 4-wide runs per row of B / C
    constexpr int CHR = (CH + 3) / 4;            // 4-high runs per column of C
    __shared__ float A[SH][SW + 4];  // raw L (+4: runs may read past the edge)
    __shared__ float B[SH + 4][CW + 4];  // row-smoothed
    __shared__ float C[CH + 4][CW + 1];  // smoothed
    extern __shared__ unsigned int hist_s[];
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * BX + tx;
    constexpr int NT = BX * BY;

    if (MODE == MODE_HIST) {
        for (int i = tid; i < nbins; i += NT) hist_s[i] = 0u;
    }
    int gx[KX];
#pragma unroll
    for (int k = 0; k < KX; ++k) gx[k] = reflect_index(x0 - 1 - R + tx + k * BX, w);
#pragma unroll
    for (int sy = ty; sy < SH; sy += BY) {
        const float* row = L + (size_t)reflect_index(y0 - 1 - R + sy, h) * pitch;
#pragma unroll
        for (int k = 0; k < KX; ++k)
            if (tx + k * BX < SW) A[sy][tx + k * BX] = __ldg(row + gx[k]);
    }
    __syncthreads();
    // rows: B[sy][4u .. 4u+3]
#pragma unroll
    for (int t = tid; t < SH * CWR; t += NT) {
        const int sy = t / CWR, u = t - sy * CWR;
        float v[4 + 2 * R];
#pragma unroll
        for (int j = 0; j < 4 + 2 * R; ++j) v[j] = A[sy][4 * u + j];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float acc = 0.f;
#pragma unroll
            for (int j = 0; j <= 2 * R; ++j) acc = fmaf(taps.w[j], v[q + j], acc);
            B[sy][4 * u + q] = acc;
        }
    }
    __syncthreads();
    // columns: C[4u .. 4u+3][sx]
#pragma unroll
    for (int t = tid; t < CW * CHR; t += NT) {
        const int u = t / CW, sx = t - u * CW;
        float v[4 + 2 * R];
#pragma unroll
        for (int j = 0; j < 4 + 2 * R; ++j) v[j] = B[4 * u + j][sx];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float acc = 0.f;
#pragma unroll
            for (int j = 0; j <= 2 * R; ++j) acc = fmaf(taps.w[j], v[q + j], acc);
            C[4 * u + q][sx] = acc;
        }
    }
    __syncthreads();

    float kk = 0.f, hmax = 0.f;
    if (MODE == MODE_COND) kk = *d_k;
    if (MODE == MODE_HIST) hmax = __uint_as_float(*d_hmax_bits);
    float local_max = 0.f;
    const float c0 = 3.f / 16.f, c1 = 10.f / 16.f;
    const int gxo = x0 + tx;
    const int oy0 = 4 * ty;  // this thread's 4 output rows
    // C[cy][cx] holds the smoothed value at (x0 - 1 + cx, y0 - 1 + cy)
    float cm[6], cc[6], cp[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        cm[j] = C[oy0 + j][tx];
        cc[j] = C[oy0 + j][tx + 1];
        cp[j] = C[oy0 + j][tx + 2];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int gy = y0 + oy0 + q;
        float lx = c0 * 0.5f * (cp[q] - cm[q]);
        lx += c1 * 0.5f * (cp[q + 1] - cm[q + 1]);
        lx += c0 * 0.5f * (cp[q + 2] - cm[q + 2]);
        float ly = c0 * 0.5f * (cm[q + 2] - cm[q]);
        ly += c1 * 0.5f * (cc[q + 2] - cc[q]);
        ly += c0 * 0.5f * (cp[q + 2] - cp[q]);
        if (gxo >= w || gy >= h) continue;
        if (MODE == MODE_COND) {
            const float qv = (lx * lx + ly * ly) / (kk * kk);
            g[(size_t)gy * pitch + gxo] = diffusivity == KAZE_G1 ? expf(-qv) : 1.f / (1.f + qv);
        } else {
            const bool interior = gxo >= 1 && gxo <= w - 2 && gy >= 1 && gy <= h - 2;
            if (!interior) continue;
            const float m = sqrtf(lx * lx + ly * ly);
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
        if (tx == 0 && local_max > 0.f) atomicMax(d_hmax_bits, __float_as_uint(local_max));
    }
    if (MODE == MODE_HIST) {
        __syncthreads();
        for (int i = tid; i < nbins; i += NT) {
            const unsigned int v = hist_s[i];
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

template <int MODE, int R>
cudaError_t launch_gradient_r(const float* L, float* g, int pitch, int w, int h, const GaussTaps& taps,
                              const float* d_k, int diffusivity, unsigned int* hmax_bits, unsigned int* hist,
                              int nbins, cudaStream_t st)
{
    dim3 grid((w + TX - 1) / TX, (h + TY - 1) / TY);
    const size_t smem = MODE == MODE_HIST ? (size_t)nbins * sizeof(unsigned int) : 0;
    k_gradient<MODE, R><<<grid, dim3(BX, BY), smem, st>>>(L, g, pitch, w, h, taps, d_k, diffusivity, hmax_bits,
                                                         hist, nbins);
    return cudaGetLastError();
}

template <int MODE>
cudaError_t launch_gradient(const float* L, float* g, int pitch, int w, int h, const GaussTaps& taps,
                            const float* d_k, int diffusivity, unsigned int* hmax_bits, unsigned int* hist,
                            int nbins, cudaStream_t st)
{
    switch (taps.r) {
#define KZ_GRAD_CASE(RR) \
    case RR: return launch_gradient_r<MODE, RR>(L, g, pitch, w, h, taps, d_k, diffusivity, hmax_bits, hist, nbins, st);
        KZ_GRAD_CASE(1) KZ_GRAD_CASE(2) KZ_GRAD_CASE(3) KZ_GRAD_CASE(4) KZ_GRAD_CASE(5) KZ_GRAD_CASE(6)
#undef KZ_GRAD_CASE
        default: return cudaErrorInvalidValue;
    }
}

template <int R>
cudaError_t launch_gaussian_r(const float* in, int in_pitch, float* out, int out_pitch, int w, int h,
                              const GaussTaps& taps, cudaStream_t st)
{
    dim3 grid((w + TX - 1) / TX, (h + TY - 1) / TY);
    k_gaussian<R><<<grid, dim3(BX, BY), 0, st>>>(in, in_pitch, out, out_pitch, w, h, taps);
    return cudaGetLastError();
}

}  // namespace

cudaError_t configure_filter_kernels()
{
    // static shared memory only (the histogram's dynamic part is <= 16 KB)
    return cudaSuccess;
}

cudaError_t launch_gaussian(const float* in, int in_pitch, float* out, int out_pitch, int w, int h,
                            const GaussTaps& taps, cudaStream_t st)
{
    switch (taps.r) {
#define KZ_GAUSS_CASE(RR) \
    case RR: return launch_gaussian_r<RR>(in, in_pitch, out, out_pitch, w, h, taps, st);
        KZ_GAUSS_CASE(1) KZ_GAUSS_CASE(2) KZ_GAUSS_CASE(3) KZ_GAUSS_CASE(4) KZ_GAUSS_CASE(5) KZ_GAUSS_CASE(6)
        KZ_GAUSS_CASE(7) KZ_GAUSS_CASE(8) KZ_GAUSS_CASE(9) KZ_GAUSS_CASE(10) KZ_GAUSS_CASE(11) KZ_GAUSS_CASE(12)
        KZ_GAUSS_CASE(13) KZ_GAUSS_CASE(14) KZ_GAUSS_CASE(15) KZ_GAUSS_CASE(16)
#undef KZ_GAUSS_CASE
        default: return cudaErrorInvalidValue;
    }
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
