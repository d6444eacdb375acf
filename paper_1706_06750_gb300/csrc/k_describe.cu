// k_describe.cu -- keypoint description (Sec. II-C): the dominant orientation
// and the 64-D M-SURF descriptor of each keypoint on its scale level.
//
// One CTA of 512 threads per keypoint; all levels are served by the same
// launch (the level index comes with the keypoint), so keypoints of every
// scale are described concurrently.  First derivatives are evaluated where
// they are needed, from the level itself: the step-s Scharr pair of the
// detector (s = max(1, round(sigma_i))) on the half-sample symmetric
// extension,
//     L_x = sum_b c_b (L(x+s, y+bs) - L(x-s, y+bs)) / (2s),  c = (3,10,3)/16,
// and L_y its transpose, so no derivative planes are written.  Values
// between pixels come by bilinear interpolation of the four surrounding
// pixels' derivatives (taps clamped into the image).
//
// Orientation: threads 0..108 each take one sample of the disc a^2 + b^2 <
// 36 around the keypoint (step sigma_i), weighted by a Gaussian of std
// 2.5 sigma_i, and place it in one of 72 five-degree sectors; 72 threads sum
// their sector in sample order, then the 72 windows of 12 sectors (pi/3);
// one warp picks the longest window sum (the first on ties), whose angle is
// the orientation.
// Descriptor: 16 subregions of 9 x 9 samples (centres 5 sigma_i apart,
// spacing sigma_i) in the keypoint's rotated frame; a warp per subregion
// accumulates (sum r_x', sum r_y', sum |r_x'|, sum |r_y'|) with the
// subregion's Gaussian (std 2.5 sigma_i), reduce by shuffles, apply the 4 x
// 4 mask weight (std 1.5 grid units) and the vector is normalised to unit
// length.  Every memory access is clamped into its buffer.
#include <cmath>

#include "kaze_internal.h"

namespace kz {
namespace {

constexpr int DT = 512;
constexpr int kOriN = 109;
constexpr int kSectors = 72;
constexpr int kWindow = 12;
constexpr float kTwoPi = 6.28318530717958647692f;

__constant__ signed char c_ori_a[kOriN];
__constant__ signed char c_ori_b[kOriN];
__constant__ float c_ori_w[kOriN];
__constant__ float c_sub_w[81];  // per sample of a subregion, offsets (j % 9 - 4, j / 9 - 4)
__constant__ float c_grid_w[16];  // per subregion r = 4 q + p

// L_x, L_y at pixel (xa, ya) (inside the image) with step s; inv = 1 / (32 s).
__device__ __forceinline__ void scharr_at(const float* __restrict__ L, int pitch, int w, int h, int xa, int ya, int s,
                                          float inv, float& gx, float& gy)
{
    const int xm = reflect_index(xa - s, w), xp = reflect_index(xa + s, w);
    const int ym = reflect_index(ya - s, h), yp = reflect_index(ya + s, h);
    const float* rm = L + (size_t)ym * pitch;
    const float* r0 = L + (size_t)ya * pitch;
    const float* rp = L + (size_t)yp * pitch;
    const float mm = __ldg(rm + xm), m0 = __ldg(rm + xa), mp = __ldg(rm + xp);
    const float zm = __ldg(r0 + xm), zp = __ldg(r0 + xp);
    const float pm = __ldg(rp + xm), p0 = __ldg(rp + xa), pp = __ldg(rp + xp);
    gx = fmaf(10.f, zp - zm, 3.f * ((mp - mm) + (pp - pm))) * inv;
    gy = fmaf(10.f, p0 - m0, 3.f * ((pm - mm) + (pp - mp))) * inv;
}

// Bilinearly interpolated (L_x, L_y) at (px, py).
__device__ __forceinline__ void sample_at(const float* __restrict__ L, int pitch, int w, int h, int s, float inv,
                                          float px, float py, float& gx, float& gy)
{
    float fx0 = floorf(px), fy0 = floorf(py);
    const float fx = px - fx0, fy = py - fy0;
    // taps beyond the image clamp to its edge; clamping the corner first keeps
    // the integer conversion in range (and NaN positions fall on the edge)
    fx0 = fminf(fmaxf(fx0, -1.f), (float)w);
    fy0 = fminf(fmaxf(fy0, -1.f), (float)h);
    const int x0 = (int)fx0, y0 = (int)fy0;
    const int xa = min(max(x0, 0), w - 1), xb = min(max(x0 + 1, 0), w - 1);
    const int ya = min(max(y0, 0), h - 1), yb = min(max(y0 + 1, 0), h - 1);
    float ax, ay, bx, by, cx, cy, dx, dy;
    scharr_at(L, pitch, w, h, xa, ya, s, inv, ax, ay);
    scharr_at(L, pitch, w, h, xb, ya, s, inv, bx, by);
    scharr_at(L, pitch, w, h, xa, yb, s, inv, cx, cy);
    scharr_at(L, pitch, w, h, xb, yb, s, inv, dx, dy);
    const float w00 = (1.f - fx) * (1.f - fy), w10 = fx * (1.f - fy), w01 = (1.f - fx) * fy, w11 = fx * fy;
    gx = fmaf(w11, dx, fmaf(w01, cx, fmaf(w10, bx, w00 * ax)));
    gy = fmaf(w11, dy, fmaf(w01, cy, fmaf(w10, by, w00 * ay)));
}

__global__ void __launch_bounds__(DT) k_describe(const float* __restrict__ levels, long long plane_stride, int pitch,
                                                 int w, int h, const __grid_constant__ DescTable tab,
                                                 kaze_keypoint* __restrict__ kps, int n, float* __restrict__ desc,
                                                 int upright)
{
    __shared__ float s_rx[kOriN + 3], s_ry[kOriN + 3];
    __shared__ int s_sec[kOriN + 3];
    __shared__ float s_sx[kSectors], s_sy[kSectors];
    __shared__ float s_wx[kSectors], s_wy[kSectors], s_n2[kSectors];
    __shared__ float s_desc[64];
    __shared__ float s_theta;
    const int k = blockIdx.x;
    if (k >= n) return;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const float x = kps[k].x, y = kps[k].y;
    int lev = tab.single ? 0 : kps[k].level;
    const bool valid = lev >= 0 && lev < tab.n;
    if (!valid) {  // not a level of this stack: zero descriptor
        if (t < 64) desc[(size_t)k * 64 + t] = 0.f;
        if (t == 0) kps[k].angle = 0.f;
        return;
    }
    const float* L = levels + (tab.single ? 0 : (long long)lev * plane_stride);
    const float sigma = tab.sigma[lev];
    const int s = tab.step[lev];
    const float inv = 1.f / (32.f * (float)s);

    if (!upright) {
        if (t < kOriN) {
            float gx, gy;
            sample_at(L, pitch, w, h, s, inv, fmaf((float)c_ori_a[t], sigma, x), fmaf((float)c_ori_b[t], sigma, y),
                      gx, gy);
            const float rx = c_ori_w[t] * gx, ry = c_ori_w[t] * gy;
            float phi = atan2f(ry, rx);
            if (phi < 0.f) phi += kTwoPi;
            s_rx[t] = rx;
            s_ry[t] = ry;
            s_sec[t] = min((int)(phi * ((float)kSectors / kTwoPi)), kSectors - 1);
        }
        __syncthreads();
        if (t < kSectors) {
            float sx = 0.f, sy = 0.f;
            for (int j = 0; j < kOriN; ++j)
                if (s_sec[j] == t) {
                    sx += s_rx[j];
                    sy += s_ry[j];
                }
            s_sx[t] = sx;
            s_sy[t] = sy;
        }
        __syncthreads();
        if (t < kSectors) {
            float wx = 0.f, wy = 0.f;
#pragma unroll
            for (int m = 0; m < kWindow; ++m) {
                const int q = t + m < kSectors ? t + m : t + m - kSectors;
                wx += s_sx[q];
                wy += s_sy[q];
            }
            s_wx[t] = wx;
            s_wy[t] = wy;
            s_n2[t] = fmaf(wx, wx, wy * wy);
        }
        __syncthreads();
        if (warp == 0) {
            float best = -1.f;
            int bk = 0;
            for (int q = lane; q < kSectors; q += 32)
                if (s_n2[q] > best) {
                    best = s_n2[q];
                    bk = q;
                }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int ok = __shfl_xor_sync(0xffffffffu, bk, o);
                if (ob > best || (ob == best && ok < bk)) {
                    best = ob;
                    bk = ok;
                }
            }
            if (lane == 0) {
                float th = 0.f;
                if (best > 0.f) {
                    th = atan2f(s_wy[bk], s_wx[bk]);
                    if (th < 0.f) th += kTwoPi;
                }
                s_theta = th;
            }
        }
        __syncthreads();
    } else if (t == 0) {
        s_theta = 0.f;
    }
    __syncthreads();
    const float theta = s_theta;
    float si, co;
    sincosf(theta, &si, &co);

    // descriptor: subregion r = t / 32 (p = r % 4 along x', q = r / 4 along y'),
    // one warp per subregion
    const int r = t >> 5, l32 = lane;
    const float cp = ((float)(r & 3) - 1.5f) * 5.f, cq = ((float)(r >> 2) - 1.5f) * 5.f;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    for (int j = l32; j < 81; j += 32) {
        const float du = cp + (float)(j % 9 - 4), dv = cq + (float)(j / 9 - 4);
        const float ox = sigma * fmaf(du, co, -dv * si), oy = sigma * fmaf(du, si, dv * co);
        float gx, gy;
        sample_at(L, pitch, w, h, s, inv, x + ox, y + oy, gx, gy);
        const float rxp = fmaf(gx, co, gy * si), ryp = fmaf(-gx, si, gy * co);
        const float w1 = c_sub_w[j];
        a0 = fmaf(w1, rxp, a0);
        a1 = fmaf(w1, ryp, a1);
        a2 = fmaf(w1, fabsf(rxp), a2);
        a3 = fmaf(w1, fabsf(ryp), a3);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a0 += __shfl_xor_sync(0xffffffffu, a0, o);
        a1 += __shfl_xor_sync(0xffffffffu, a1, o);
        a2 += __shfl_xor_sync(0xffffffffu, a2, o);
        a3 += __shfl_xor_sync(0xffffffffu, a3, o);
    }
    if (l32 == 0) {
        const float w2 = c_grid_w[r];
        s_desc[4 * r + 0] = w2 * a0;
        s_desc[4 * r + 1] = w2 * a1;
        s_desc[4 * r + 2] = w2 * a2;
        s_desc[4 * r + 3] = w2 * a3;
    }
    __syncthreads();
    if (warp < 2) {
        const float v0 = s_desc[lane], v1 = s_desc[lane + 32];
        float ss = fmaf(v0, v0, v1 * v1);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
        const float sc = ss > 0.f ? 1.f / sqrtf(ss) : 0.f;
        const int i = t;  // warps 0 and 1 write entries 0..63
        desc[(size_t)k * 64 + i] = s_desc[i] * sc;
    }
    if (t == 0) kps[k].angle = theta;
}

}  // namespace

cudaError_t configure_describe_kernels()
{
    signed char a[kOriN], b[kOriN];
    float wo[kOriN], ws[81], wg[16];
    int m = 0;
    for (int bb = -6; bb <= 6; ++bb)
        for (int aa = -6; aa <= 6; ++aa)
            if (aa * aa + bb * bb < 36) {
                a[m] = (signed char)aa;
                b[m] = (signed char)bb;
                wo[m] = (float)std::exp(-(double)(aa * aa + bb * bb) / (2.0 * 2.5 * 2.5));
                ++m;
            }
    if (m != kOriN) return cudaErrorInvalidValue;
    for (int j = 0; j < 81; ++j) {
        const int u = j % 9 - 4, v = j / 9 - 4;
        ws[j] = (float)std::exp(-(double)(u * u + v * v) / (2.0 * 2.5 * 2.5));
    }
    for (int r = 0; r < 16; ++r) {
        const double p = (r & 3) - 1.5, q = (r >> 2) - 1.5;
        wg[r] = (float)std::exp(-(p * p + q * q) / (2.0 * 1.5 * 1.5));
    }
    cudaError_t e = cudaMemcpyToSymbol(c_ori_a, a, sizeof(a));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_ori_b, b, sizeof(b));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_ori_w, wo, sizeof(wo));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_sub_w, ws, sizeof(ws));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_grid_w, wg, sizeof(wg));
    return e;
}

cudaError_t launch_describe(const float* levels, long long plane_stride, int pitch, int w, int h,
                            const DescTable& tab, kaze_keypoint* d_kps, int n, float* d_desc, int upright,
                            cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_describe<<<n, DT, 0, st>>>(levels, plane_stride, pitch, w, h, tab, d_kps, n, d_desc, upright);
    return cudaGetLastError();
}

}  // namespace kz
