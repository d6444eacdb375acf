// k_filters.cu -- stencil kernels of the nonlinear scale space (Sec. III-1):
//   * Gaussian presmoothing of the input image,
//   * the fused "smooth -> Scharr -> conductance" kernel (Eq. 2-3),
//   * the gradient-statistics passes (maximum, histogram of the kept |grad|^2
//     plane) and the percentile pick that give the contrast factor k.
//
// Presmoothing: a CTA of 32x8 threads owns a 32x32 output tile, stages its
// input tile plus halo in shared memory with half-sample symmetric borders
// (index reflection on load) and runs the separable Gaussian rows-then-
// columns.  The gradient kernels walk down columns instead: a warp stages
// each needed row in a small shared-memory row for the horizontal taps,
// keeps the vertical filter window in registers and trades neighbouring
// smoothed values by warp shuffles -- one column a lane (k_gradient) or four
// (k_gradient4, used wherever the planes allow 16-byte access), with the
// same arithmetic.
#include <algorithm>

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

constexpr int GK = 16;     // output rows per thread
constexpr int GWARPS = 8;  // warps per CTA
constexpr int GCOLS = 30;  // output columns per warp (lanes 1..30; 0 and 31 are halo)
constexpr int GPD = 4;     // rows of loads kept in flight

// Smoothed Scharr gradient, walking down columns.  Lane l of a warp owns
// column x = x_w + l - 1 (x_w: the warp's first output column) and the GK
// output rows y0 .. y0 + GK - 1.  Each needed row of L is staged per warp
// (columns x_w - 1 - R .. x_w + GCOLS + R, two coalesced loads per lane,
// issued GPD rows ahead) in a small shared-memory row from which every lane
// filters its column horizontally with G(sigma_d) (radius R, reflected
// borders); the last 2R + 1 filtered rows stay in registers for the vertical
// pass, and the smoothed values S of neighbouring columns come from warp
// shuffles for the 3x3 Scharr pair ([-1 0 1]/2 x [3 10 3]/16 and its
// transpose):
//   Lx(y) = (3 D(y-1) + 10 D(y) + 3 D(y+1)) / 32,  D = S(x+1) - S(x-1)
//   Ly(y) = (E(y+1) - E(y-1)) / 32,  E = 3 S(x-1) + 10 S(x) + 3 S(x+1).
// Lanes 0 and 31 only supply S to their neighbours.  MODE_COND writes the
// conductance g of Eq. 3 (and zeros to `zero` if given); MODE_MAX folds
// |grad| of interior pixels into a global maximum; MODE_HIST bins the
// non-zero interior magnitudes.
template <int MODE, int R>
__global__ void __launch_bounds__(GWARPS * 32)
k_gradient(const float* __restrict__ L, float* __restrict__ g, float* __restrict__ zero, int pitch, int w, int h,
           const __grid_constant__ GaussTaps taps, const float* __restrict__ d_k, int diffusivity,
           unsigned int* __restrict__ d_hmax_bits, unsigned int* __restrict__ d_hist, int nbins)
{
    constexpr int RW = GCOLS + 2 + 2 * R;  // staged columns per row (<= 64)
    __shared__ float srow[GWARPS][2][64];
    extern __shared__ unsigned int hist_s[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int xw = (blockIdx.x * GWARPS + warp) * GCOLS;
    const int x = xw + lane - 1;
    const int y0 = blockIdx.y * GK;
    constexpr int NT = GWARPS * 32;
    if (MODE == MODE_HIST) {
        for (int i = threadIdx.x; i < nbins; i += NT) hist_s[i] = 0u;
        __syncthreads();
    }
    // the two staged columns of this lane, reflected into the image
    const int c0 = reflect_index(xw - 1 - R + lane, w);
    const bool has1 = lane + 32 < RW;
    const int c1 = reflect_index(xw - 1 - R + lane + 32, w);
    float wt[R + 1];
#pragma unroll
    for (int j = 0; j <= R; ++j) wt[j] = taps.w[R + j];

    float inv_k2 = 0.f, hmax_scale = 0.f;
    if (MODE == MODE_COND) {
        const float kk = *d_k;
        inv_k2 = 1.f / (kk * kk);
    }
    if (MODE == MODE_HIST) hmax_scale = (float)nbins / __uint_as_float(*d_hmax_bits);
    float local_max = 0.f;
    const bool out_col = lane >= 1 && lane <= GCOLS && x < w;

    // H rows y0 - 1 - R .. y0 + GK + R; S rows y0 - 1 .. y0 + GK
    constexpr int NI = GK + 2 + 2 * R;
    float pre[GPD + 1][2];
#pragma unroll
    for (int i = 0; i < GPD && i < NI; ++i) {
        const int ro = reflect_index(y0 - 1 - R + i, h) * pitch;  // plane offsets fit 32 bits
        pre[i][0] = __ldg(L + (unsigned)(ro + c0));
        pre[i][1] = has1 ? __ldg(L + (unsigned)(ro + c1)) : 0.f;
    }
    float hw[2 * R + 1];      // last 2R + 1 horizontally filtered rows
    float dm = 0.f, d0 = 0.f, em = 0.f, e0 = 0.f;  // D, E of the two previous S rows
#pragma unroll
    for (int i = 0; i < NI; ++i) {
        if (i + GPD < NI) {
            const int ro = reflect_index(y0 - 1 - R + i + GPD, h) * pitch;
            pre[(i + GPD) % (GPD + 1)][0] = __ldg(L + (unsigned)(ro + c0));
            pre[(i + GPD) % (GPD + 1)][1] = has1 ? __ldg(L + (unsigned)(ro + c1)) : 0.f;
        }
        float* sr_ = srow[warp][i & 1];
        sr_[lane] = pre[i % (GPD + 1)][0];
        if (has1) sr_[lane + 32] = pre[i % (GPD + 1)][1];
        __syncwarp();
        const float* v = sr_ + lane;  // v[R] is this lane's column
        float hv = wt[0] * v[R];
#pragma unroll
        for (int j = 1; j <= R; ++j) hv = fmaf(wt[j], v[R - j] + v[R + j], hv);
#pragma unroll
        for (int j = 0; j < 2 * R; ++j) hw[j] = hw[j + 1];
        hw[2 * R] = hv;
        if (i < 2 * R) continue;
        // S at row y0 - 1 + (i - 2R)
        float sv = wt[0] * hw[R];
#pragma unroll
        for (int j = 1; j <= R; ++j) sv = fmaf(wt[j], hw[R - j] + hw[R + j], sv);
        const float sl = __shfl_up_sync(0xffffffffu, sv, 1);
        const float sr = __shfl_down_sync(0xffffffffu, sv, 1);
        // explicit fmaf: the batched kernel (k_batch.cu) repeats this
        // arithmetic operation for operation, so both paths agree bit for bit
        const float dp = sr - sl;
        const float ep = fmaf(10.f, sv, 3.f * (sl + sr));
        const int si = i - 2 * R;
        if (si >= 2) {
            const int y = y0 + si - 2;  // output row: S rows y - 1, y, y + 1
            const float lx = fmaf(10.f, d0, 3.f * (dm + dp)) * (1.f / 32.f);
            const float ly = (ep - em) * (1.f / 32.f);
            const float m2 = fmaf(ly, ly, lx * lx);
            if (out_col && y < h) {
                if (MODE == MODE_COND) {
                    const unsigned o = (unsigned)(y * pitch + x);
                    g[o] = diffusivity == KAZE_G1 ? expf(-(m2 * inv_k2)) : __fdividef(1.f, fmaf(m2, inv_k2, 1.f));
                    if (zero) zero[o] = 0.f;
                } else {
                    // the max pass may keep |grad|^2 for the histogram and the
                    // first conductance (g is then an m2 plane)
                    if (MODE == MODE_MAX && g) g[(unsigned)(y * pitch + x)] = m2;
                    if (x >= 1 && x <= w - 2 && y >= 1 && y <= h - 2) {
                        const float m = sqrtf(m2);
                        if (MODE == MODE_MAX) {
                            local_max = fmaxf(local_max, m);
                        } else if (m > 0.f) {
                            int b = (int)floorf(m * hmax_scale);
                            b = min(b, nbins - 1);
                            atomicAdd(&hist_s[b], 1u);
                        }
                    }
                }
            }
        }
        dm = d0;
        d0 = dp;
        em = e0;
        e0 = ep;
    }
    if (MODE == MODE_MAX) {
        for (int o = 16; o > 0; o >>= 1) local_max = fmaxf(local_max, __shfl_xor_sync(0xffffffffu, local_max, o));
        // non-negative floats order like their bit patterns
        if (lane == 0 && local_max > 0.f) atomicMax(d_hmax_bits, __float_as_uint(local_max));
    }
    if (MODE == MODE_HIST) {
        __syncthreads();
        for (int i = threadIdx.x; i < nbins; i += NT) {
            const unsigned int v = hist_s[i];
            if (v) atomicAdd(&d_hist[i], v);
        }
    }
}

// The same smoothed Scharr gradient, four columns a lane.  A warp stages
// 128 columns (X - 4 .. X + 123, float4 loads, reflected into the image) of
// each needed row in a padded shared-memory row, reads its neighbours
// there with two 16-byte loads, and writes the 120 columns X .. X + 119
// (lanes 1..30); lanes 0 and 31 only supply the smoothed values S at X - 1
// and X + 120.  The radius of G(sigma_d) must be <= 3 so that S(X - 1)
// only needs the staged columns.  Every value is formed with the
// arithmetic of k_gradient, operation for operation, so the two kernels
// (and the batched kernel, which repeats it) agree bit for bit.
constexpr int C4W = 8;     // warps per CTA
constexpr int C4K = 8;    // output rows per warp
constexpr int C4MW = 120;  // output columns per warp
constexpr int C4PD = 4;    // rows of loads in flight

template <int MODE, int R>
__global__ void __launch_bounds__(C4W * 32)
k_gradient4(const float* __restrict__ L, float* __restrict__ g, float* __restrict__ zero, int pitch, int w, int h,
            const __grid_constant__ GaussTaps taps, const float* __restrict__ d_k, int diffusivity,
            unsigned int* __restrict__ d_hmax_bits)
{
    static_assert(R >= 1 && R <= 3, "S(X - 1) must come from the staged columns");
    static_assert(MODE == MODE_COND || MODE == MODE_MAX, "conductance or maximum pass");
    __shared__ __align__(16) float srow[C4W][2][136];  // 4 pad + 128 + 4 pad
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int X = (blockIdx.x * C4W + warp) * C4MW;
    if (X >= w) return;  // whole warp beyond the image (warps never wait on each other)
    const int x0 = X - 4 + 4 * lane;
    const int y0 = blockIdx.y * C4K;
    if (lane == 0 || lane == 31) {  // the pads only feed unused halo columns; keep them finite
        const int o = lane == 0 ? 0 : 132;
        *reinterpret_cast<float4*>(&srow[warp][0][o]) = make_float4(0.f, 0.f, 0.f, 0.f);
        *reinterpret_cast<float4*>(&srow[warp][1][o]) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const bool vec = x0 >= 0 && x0 + 4 <= w;
    int cx[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) cx[q] = reflect_index(x0 + q, w);
    float wt[R + 1];
#pragma unroll
    for (int j = 0; j <= R; ++j) wt[j] = taps.w[R + j];
    float inv_k2 = 0.f;
    if (MODE == MODE_COND) {
        const float kk = *d_k;
        inv_k2 = 1.f / (kk * kk);
    }
    float local_max = 0.f;
    const bool out_lane = lane >= 1 && lane <= 30 && x0 < w;

    auto load_row = [&](int i) {
        const int ro = reflect_index(y0 - 1 - R + i, h) * pitch;  // plane offsets fit 32 bits
        if (vec) return __ldg(reinterpret_cast<const float4*>(L + (unsigned)(ro + x0)));
        return make_float4(__ldg(L + (unsigned)(ro + cx[0])), __ldg(L + (unsigned)(ro + cx[1])),
                           __ldg(L + (unsigned)(ro + cx[2])), __ldg(L + (unsigned)(ro + cx[3])));
    };
    // H rows y0 - 1 - R .. y0 + C4K + R; S rows y0 - 1 .. y0 + C4K
    constexpr int NI = C4K + 2 + 2 * R;
    float4 pre[C4PD + 1];
#pragma unroll
    for (int i = 0; i < C4PD && i < NI; ++i) pre[i] = load_row(i);
    float hw[2 * R + 1][4];  // last 2R + 1 horizontally filtered rows
    float dm[4], d0[4], em[4], e0[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) dm[q] = d0[q] = em[q] = e0[q] = 0.f;
#pragma unroll
    for (int i = 0; i < NI; ++i) {
        if (i + C4PD < NI) pre[(i + C4PD) % (C4PD + 1)] = load_row(i + C4PD);
        float* sr_ = srow[warp][i & 1];
        const float4 c = pre[i % (C4PD + 1)];
        *reinterpret_cast<float4*>(sr_ + 4 + 4 * lane) = c;
        __syncwarp();
        const float4 a = *reinterpret_cast<const float4*>(sr_ + 4 * lane);
        const float4 b = *reinterpret_cast<const float4*>(sr_ + 8 + 4 * lane);
        const float v[12] = {a.x, a.y, a.z, a.w, c.x, c.y, c.z, c.w, b.x, b.y, b.z, b.w};  // columns x0 - 4 ..
#pragma unroll
        for (int j = 0; j < 2 * R; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) hw[j][q] = hw[j + 1][q];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float hv = wt[0] * v[4 + q];
#pragma unroll
            for (int j = 1; j <= R; ++j) hv = fmaf(wt[j], v[4 + q - j] + v[4 + q + j], hv);
            hw[2 * R][q] = hv;
        }
        if (i < 2 * R) continue;
        // S at row y0 - 1 + (i - 2R)
        float sv[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            sv[q] = wt[0] * hw[R][q];
#pragma unroll
            for (int j = 1; j <= R; ++j) sv[q] = fmaf(wt[j], hw[R - j][q] + hw[R + j][q], sv[q]);
        }
        const float s_l = __shfl_up_sync(0xffffffffu, sv[3], 1);
        const float s_r = __shfl_down_sync(0xffffffffu, sv[0], 1);
        float dp[4], ep[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float sl = q == 0 ? s_l : sv[q - 1];
            const float sr = q == 3 ? s_r : sv[q + 1];
            dp[q] = sr - sl;
            ep[q] = fmaf(10.f, sv[q], 3.f * (sl + sr));
        }
        const int si = i - 2 * R;
        if (si >= 2) {
            const int y = y0 + si - 2;  // output row: S rows y - 1, y, y + 1
            float m2[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float lx = fmaf(10.f, d0[q], 3.f * (dm[q] + dp[q])) * (1.f / 32.f);
                const float ly = (ep[q] - em[q]) * (1.f / 32.f);
                m2[q] = fmaf(ly, ly, lx * lx);
            }
            if (out_lane && y < h) {
                const unsigned o = (unsigned)(y * pitch + x0);
                float4 r;
                if (MODE == MODE_COND) {
                    float* rr = &r.x;
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        rr[q] = diffusivity == KAZE_G1 ? expf(-(m2[q] * inv_k2))
                                                       : __fdividef(1.f, fmaf(m2[q], inv_k2, 1.f));
                } else {
                    r = make_float4(m2[0], m2[1], m2[2], m2[3]);
                    if (y >= 1 && y <= h - 2) {
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            if (x0 + q >= 1 && x0 + q <= w - 2) local_max = fmaxf(local_max, sqrtf(m2[q]));
                    }
                }
                if (MODE == MODE_COND || g) {
                    if (x0 + 4 <= w) {
                        *reinterpret_cast<float4*>(g + o) = r;
                        if (MODE == MODE_COND && zero) *reinterpret_cast<float4*>(zero + o) = make_float4(0.f, 0.f, 0.f, 0.f);
                    } else {
                        const float* rr = &r.x;
                        for (int q = 0; q < 4 && x0 + q < w; ++q) {
                            g[o + q] = rr[q];
                            if (MODE == MODE_COND && zero) zero[o + q] = 0.f;
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            dm[q] = d0[q];
            d0[q] = dp[q];
            em[q] = e0[q];
            e0[q] = ep[q];
        }
    }
    if (MODE == MODE_MAX) {
        for (int o = 16; o > 0; o >>= 1) local_max = fmaxf(local_max, __shfl_xor_sync(0xffffffffu, local_max, o));
        // non-negative floats order like their bit patterns
        if (lane == 0 && local_max > 0.f) atomicMax(d_hmax_bits, __float_as_uint(local_max));
    }
}

// Percentile pick of the contrast factor on one warp (percentile_k), k to d_k.
__device__ __forceinline__ void percentile_pick(const unsigned int* hist, int nbins,
                                                const unsigned int* d_hmax_bits, double pct, float* d_k, int lane)
{
    const float k = percentile_k(hist, nbins, __uint_as_float(*d_hmax_bits), pct, lane);
    if (lane == 0) *d_k = k;
}

__global__ void k_percentile(const unsigned int* __restrict__ hist, int nbins,
                             const unsigned int* __restrict__ d_hmax_bits, double pct,
                             float* __restrict__ d_k)
{
    percentile_pick(hist, nbins, d_hmax_bits, pct, d_k, threadIdx.x);
}

__global__ void k_set_scalar(float* d, float v) { *d = v; }

// Histogram pass from the |grad|^2 plane the max pass kept: interior
// pixels, the same binning as k_gradient<MODE_HIST>.  Four pixels a thread.
__global__ void __launch_bounds__(256)
k_hist_m2(const float* __restrict__ m2p, int pitch, int w, int h, const unsigned int* __restrict__ d_hmax_bits,
          unsigned int* __restrict__ d_hist, int nbins, double pct, float* __restrict__ d_k)
{
    __shared__ bool s_last;
    extern __shared__ unsigned int hist_s[];
    for (int i = threadIdx.x; i < nbins; i += blockDim.x) hist_s[i] = 0u;
    __syncthreads();
    const float hmax_scale = (float)nbins / __uint_as_float(*d_hmax_bits);
    const int x4 = (blockIdx.x * blockDim.x + threadIdx.x) * 4;
    // rows blockIdx.y, + gridDim.y, ...: a few CTAs an SM each flush their
    // shared histogram once, HB rows of loads in flight at a time
    constexpr int HB = 4;
    for (int y0 = blockIdx.y; y0 < h; y0 += HB * gridDim.y) {
        float4 v4[HB];
#pragma unroll
        for (int k = 0; k < HB; ++k) {
            const int y = y0 + k * gridDim.y;
            v4[k] = (y >= 1 && y <= h - 2 && x4 < w)
                        ? __ldg(reinterpret_cast<const float4*>(m2p + (unsigned)(y * pitch + x4)))
                        : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int k = 0; k < HB; ++k) {
            const float v[4] = {v4[k].x, v4[k].y, v4[k].z, v4[k].w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int x = x4 + q;
                if (x < 1 || x > w - 2) continue;
                const float m = sqrtf(v[q]);  // rows outside 1..h-2 read as 0: not binned
                if (m > 0.f) {
                    int b = (int)floorf(m * hmax_scale);
                    b = min(b, nbins - 1);
                    atomicAdd(&hist_s[b], 1u);
                }
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nbins; i += blockDim.x) {
        const unsigned int c = hist_s[i];
        if (c) atomicAdd(&d_hist[i], c);
    }
    // the last block to finish picks the percentile (d_hist[nbins] counts
    // finished blocks): no separate launch, no block waits for another
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0)
        s_last = atomicAdd(&d_hist[nbins], 1u) == gridDim.x * gridDim.y - 1u;
    __syncthreads();
    if (s_last && threadIdx.x < 32) {
        __threadfence();
        percentile_pick(d_hist, nbins, d_hmax_bits, pct, d_k, threadIdx.x);
    }
}

// Conductance of Eq. 3 from the |grad|^2 plane, in place (the arithmetic of
// k_gradient<MODE_COND>), zeroing `zero` at the same pixels if given.
__global__ void __launch_bounds__(256)
k_cond_m2(float* __restrict__ gm, float* __restrict__ zero, int pitch, int w, int h, const float* __restrict__ d_k,
          int diffusivity)
{
    const float kk = *d_k;
    const float inv_k2 = 1.f / (kk * kk);
    const int y = blockIdx.y;
    const int x4 = (blockIdx.x * blockDim.x + threadIdx.x) * 4;
    if (y >= h || x4 >= w) return;
    const unsigned o = (unsigned)(y * pitch + x4);
    float4 v = *reinterpret_cast<const float4*>(gm + o);
    float* c = &v.x;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        c[q] = diffusivity == KAZE_G1 ? expf(-(c[q] * inv_k2)) : __fdividef(1.f, fmaf(c[q], inv_k2, 1.f));
    }
    if (x4 + 4 <= w) {
        *reinterpret_cast<float4*>(gm + o) = v;
        if (zero) *reinterpret_cast<float4*>(zero + o) = make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
        for (int q = 0; q < 4 && x4 + q < w; ++q) {
            gm[o + q] = c[q];
            if (zero) zero[o + q] = 0.f;
        }
    }
}

template <int MODE, int R>
cudaError_t launch_gradient_r(const float* L, float* g, float* zero, int pitch, int w, int h, const GaussTaps& taps,
                              const float* d_k, int diffusivity, unsigned int* hmax_bits, unsigned int* hist,
                              int nbins, cudaStream_t st)
{
    dim3 grid((w + GWARPS * GCOLS - 1) / (GWARPS * GCOLS), (h + GK - 1) / GK);
    const size_t smem = MODE == MODE_HIST ? (size_t)nbins * sizeof(unsigned int) : 0;
    k_gradient<MODE, R><<<grid, GWARPS * 32, smem, st>>>(L, g, zero, pitch, w, h, taps, d_k, diffusivity,
                                                         hmax_bits, hist, nbins);
    return cudaGetLastError();
}

template <int MODE, int R>
cudaError_t launch_gradient4_r(const float* L, float* g, float* zero, int pitch, int w, int h, const GaussTaps& taps,
                               const float* d_k, int diffusivity, unsigned int* hmax_bits, cudaStream_t st)
{
    dim3 grid((w + C4W * C4MW - 1) / (C4W * C4MW), (h + C4K - 1) / C4K);
    k_gradient4<MODE, R><<<grid, C4W * 32, 0, st>>>(L, g, zero, pitch, w, h, taps, d_k, diffusivity, hmax_bits);
    return cudaGetLastError();
}

template <int MODE>
cudaError_t launch_gradient(const float* L, float* g, float* zero, int pitch, int w, int h, const GaussTaps& taps,
                            const float* d_k, int diffusivity, unsigned int* hmax_bits, unsigned int* hist,
                            int nbins, cudaStream_t st)
{
    // four columns a lane where the radius allows it and the planes take
    // 16-byte accesses
    const bool aligned = (pitch & 3) == 0 && (((uintptr_t)L | (uintptr_t)g | (uintptr_t)zero) & 15) == 0;
    if constexpr (MODE != MODE_HIST) {
        if (aligned && taps.r >= 1 && taps.r <= 3) {
            switch (taps.r) {
            case 1: return launch_gradient4_r<MODE, 1>(L, g, zero, pitch, w, h, taps, d_k, diffusivity, hmax_bits, st);
            case 2: return launch_gradient4_r<MODE, 2>(L, g, zero, pitch, w, h, taps, d_k, diffusivity, hmax_bits, st);
            default: return launch_gradient4_r<MODE, 3>(L, g, zero, pitch, w, h, taps, d_k, diffusivity, hmax_bits, st);
            }
        }
    }
    switch (taps.r) {
#define KZ_GRAD_CASE(RR) \
    case RR: return launch_gradient_r<MODE, RR>(L, g, zero, pitch, w, h, taps, d_k, diffusivity, hmax_bits, hist, nbins, st);
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

cudaError_t launch_conductance(const float* L, float* g, float* zero_out, int pitch, int w, int h,
                               const GaussTaps& taps, const float* d_k, int diffusivity, cudaStream_t st)
{
    return launch_gradient<MODE_COND>(L, g, zero_out, pitch, w, h, taps, d_k, diffusivity, nullptr, nullptr, 0, st);
}

cudaError_t launch_grad_max(const float* L, int pitch, int w, int h, const GaussTaps& taps,
                            unsigned int* d_hmax_bits, cudaStream_t st, float* m2_out)
{
    return launch_gradient<MODE_MAX>(L, m2_out, nullptr, pitch, w, h, taps, nullptr, 0, d_hmax_bits, nullptr, 0, st);
}

cudaError_t launch_hist_m2(const float* m2, int pitch, int w, int h, const unsigned int* d_hmax_bits,
                           unsigned int* d_hist, int nbins, double pct, float* d_k, cudaStream_t st)
{
    if ((pitch & 3) || ((uintptr_t)m2 & 15)) return cudaErrorInvalidValue;
    const int tx = (w + 3) / 4;
    const int gx = (tx + 255) / 256;
    const int gy = std::max(1, std::min(h, 608 / gx));  // about four CTAs an SM
    dim3 grid(gx, gy);
    k_hist_m2<<<grid, 256, (size_t)nbins * sizeof(unsigned int), st>>>(m2, pitch, w, h, d_hmax_bits, d_hist, nbins,
                                                                        pct, d_k);
    return cudaGetLastError();
}

cudaError_t launch_cond_m2(float* gm, float* zero_out, int pitch, int w, int h, const float* d_k, int diffusivity,
                           cudaStream_t st)
{
    if ((pitch & 3) || (((uintptr_t)gm | (uintptr_t)zero_out) & 15)) return cudaErrorInvalidValue;
    const int tx = (w + 3) / 4;
    dim3 grid((tx + 255) / 256, h);
    k_cond_m2<<<grid, 256, 0, st>>>(gm, zero_out, pitch, w, h, d_k, diffusivity);
    return cudaGetLastError();
}

cudaError_t launch_grad_hist(const float* L, int pitch, int w, int h, const GaussTaps& taps,
                             const unsigned int* d_hmax_bits, unsigned int* d_hist, int nbins,
                             cudaStream_t st)
{
    return launch_gradient<MODE_HIST>(L, nullptr, nullptr, pitch, w, h, taps, nullptr, 0,
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
