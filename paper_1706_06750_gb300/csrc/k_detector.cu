// k_detector.cu -- feature detection of Sec. II-B / Sec. III-2:
//   * the normalised Hessian determinant of Eq. 8, with second derivatives
//     built from two concatenated step-s Scharr operators, and
//   * the 3x3x3 maximum test with sub-pixel quadratic fit and the edge test
//     of Eq. 9-12.
//
// Second derivatives.  With D_x = [-1 0 1]/(2s) along x (taps at -s, 0, s)
// times [3 10 3]/16 along y and D_y its transpose, the composed operators are
// separable on the sparse lattice {-2s, -s, 0, s, 2s}^2:
//   Lxx: x-taps [1 0 -2 0 1]/(4 s^2),   y-taps [9 60 118 60 9]/256
//   Lyy: the transpose of Lxx
//   Lxy: x-taps [-3 -10 0 10 3]/(32 s), y-taps [-3 -10 0 10 3]/(32 s)
// All three share the denominator 1024 s^2, so the kernel filters with the
// integer taps and applies norm / (1024 s^2)^2 once to the determinant.
// Borders reflect coordinates into the image (half-sample symmetric).
//
// GB300 mapping (one launch per level, its own step s): a CTA stages the
// level's (64 + 4s)^2 input tile in shared memory (reflection on load), then
// each thread computes a vertical run of up to 8 outputs that share one
// residue modulo s.  Consecutive outputs of a run reuse 4 of their 5
// horizontally filtered lattice rows, which stay in registers: per output
// ~5 (K+4)/K shared loads and ~30 FP32 operations instead of 25 loads.
#include "kaze_internal.h"

namespace kz {
namespace {

constexpr int DT = 64;       // output tile edge (DT x DT)
constexpr int DTHREADS = 256;
constexpr int RUN = 8;       // outputs per vertical run

__global__ void __launch_bounds__(DTHREADS)
k_doh(const float* __restrict__ L, float* __restrict__ D, int pitch, long long plane_stride, int w, int h,
      int l0, const __grid_constant__ LevelTable tab)
{
    extern __shared__ float T[];  // [R][C] input tile, C odd
    const int level = l0 + blockIdx.z;
    const int s = tab.step[level];
    const double dd = 1024.0 * s * s;
    const float scale = tab.norm[level] / (float)(dd * dd);
    L += (size_t)level * plane_stride;
    D += (size_t)level * plane_stride;
    const int R = DT + 4 * s;
    const int C = (DT + 4 * s) | 1;
    const int x0 = blockIdx.x * DT, y0 = blockIdx.y * DT;
    const int tid = threadIdx.x;

    // stage rows y0-2s .. y0+DT+2s-1, columns x0-2s .. x0+DT+2s-1: each
    // thread owns up to 3 columns (reflected once) and every 4th row; four
    // rows of loads are issued before their stores
    {
        const int cw = DT + 4 * s;  // <= 3 * DT for s <= 32
        const int tc = tid & (DT - 1), tr = tid / DT;
        int gxs[3];
        bool okc[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            okc[k] = tc + k * DT < cw;
            gxs[k] = reflect_index(x0 - 2 * s + tc + k * DT, w);
        }
        for (int r0 = tr; r0 < R; r0 += 16) {
            float v[4][3];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int r = r0 + 4 * q;
                const float* row = L + (size_t)reflect_index(y0 - 2 * s + min(r, R - 1), h) * pitch;
#pragma unroll
                for (int k = 0; k < 3; ++k) v[q][k] = okc[k] ? __ldg(row + gxs[k]) : 0.f;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int r = r0 + 4 * q;
                if (r < R) {
#pragma unroll
                    for (int k = 0; k < 3; ++k)
                        if (okc[k]) T[r * C + tc + k * DT] = v[q][k];
                }
            }
        }
    }
    __syncthreads();

    // runs: residue q in [0, s), segment j; rows q + s (RUN j + k), k < RUN
    const int col = tid & (DT - 1);          // output column in the tile
    const int lane_row = tid / DT;           // 0..3
    const int per_class = (DT / s + (DT % s ? 1 : 0) + RUN - 1) / RUN;  // >= 1
    const int nruns = s * per_class;
    const int gx = x0 + col;
    for (int ri = lane_row; ri < nruns; ri += DTHREADS / DT) {
        const int q = ri / per_class, j = ri - q * per_class;
        const int base = q + s * RUN * j;    // first output row of the run (tile coords)
        if (base >= DT) continue;
        float hd[RUN + 4], hs[RUN + 4], hx[RUN + 4];
#pragma unroll
        for (int m = 0; m < RUN + 4; ++m) {
            const int tr = base + s * m;      // tile row of lattice row m (offset -2s folded in)
            if (tr < R) {
                const float* t = T + tr * C + col;
                const float v0 = t[0], v1 = t[s], v2 = t[2 * s], v3 = t[3 * s], v4 = t[4 * s];
                hd[m] = (v0 + v4) - 2.f * v2;
                hs[m] = 9.f * (v0 + v4) + 60.f * (v1 + v3) + 118.f * v2;
                hx[m] = 3.f * (v4 - v0) + 10.f * (v3 - v1);
            } else {
                hd[m] = hs[m] = hx[m] = 0.f;
            }
        }
#pragma unroll
        for (int k = 0; k < RUN; ++k) {
            const int ty = base + s * k;
            if (ty >= DT) break;
            const int gy = y0 + ty;
            if (gy >= h || gx >= w) continue;
            const float lxx = 9.f * (hd[k] + hd[k + 4]) + 60.f * (hd[k + 1] + hd[k + 3]) + 118.f * hd[k + 2];
            const float lyy = (hs[k] + hs[k + 4]) - 2.f * hs[k + 2];
            const float lxy = 3.f * (hx[k + 4] - hx[k]) + 10.f * (hx[k + 3] - hx[k + 1]);
            D[(size_t)gy * pitch + gx] = scale * (lxx * lyy - lxy * lxy);
        }
    }
}

// Each thread tests 4 adjacent pixels (one 16-byte load) of one row of
// level 1 + blockIdx.z.  Most fail the threshold; survivors read their 26
// neighbours, fit the quadratic and apply the edge test.
__global__ void __launch_bounds__(256)
k_extrema(const float* __restrict__ D, int pitch, long long plane_stride, int w, int h,
          const __grid_constant__ LevelTable tab, float thr, float edge_r,
          kaze_keypoint* __restrict__ kp, int cap, unsigned int* __restrict__ count)
{
    const int level = 1 + blockIdx.z;
    const int y = blockIdx.y;
    const int x4 = (blockIdx.x * blockDim.x + threadIdx.x) * 4;
    if (y < 1 || y > h - 2 || x4 >= w) return;
    const float* Dc = D + (size_t)level * plane_stride;
    const float4 c4 = __ldg(reinterpret_cast<const float4*>(Dc + (size_t)y * pitch + x4));
    const float cv[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int x = x4 + q;
        const float v = cv[q];
        if (!(v > thr) || x < 1 || x > w - 2) continue;
        const size_t p = (size_t)y * pitch + x;
        bool is_max = true;
        for (int l = -1; l <= 1 && is_max; ++l) {
            const float* Dl = Dc + (long long)l * plane_stride;
            for (int dy = -1; dy <= 1 && is_max; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    if (l == 0 && dx == 0 && dy == 0) continue;
                    if (!(v > Dl[(long long)p + (long long)dy * pitch + dx])) {
                        is_max = false;
                        break;
                    }
                }
        }
        if (!is_max) continue;
        // 3x3 quadratic model of the response around the maximum
        const float dxp = Dc[p + 1], dxm = Dc[p - 1], dyp = Dc[p + pitch], dym = Dc[p - pitch];
        const float gxv = 0.5f * (dxp - dxm);
        const float gyv = 0.5f * (dyp - dym);
        const float hxx = dxp - 2.f * v + dxm;
        const float hyy = dyp - 2.f * v + dym;
        const float hxy = 0.25f * (Dc[p + pitch + 1] - Dc[p + pitch - 1] - Dc[p - pitch + 1] + Dc[p - pitch - 1]);
        const float det = hxx * hyy - hxy * hxy;
        const float tr = hxx + hyy;
        // Eq. 12: keep Tr^2 / Det < (r+1)^2 / r with Det > 0
        if (edge_r > 0.f) {
            if (!(det > 0.f)) continue;
            if (!(tr * tr * edge_r < (edge_r + 1.f) * (edge_r + 1.f) * det)) continue;
        }
        if (det == 0.f) continue;
        const float ox = -(hyy * gxv - hxy * gyv) / det;
        const float oy = -(hxx * gyv - hxy * gxv) / det;
        if (fabsf(ox) > 1.f || fabsf(oy) > 1.f) continue;
        const unsigned idx = atomicAdd(count, 1u);
        if (idx < (unsigned)cap) {
            kaze_keypoint k;
            k.x = (float)x + ox;
            k.y = (float)y + oy;
            k.sigma = tab.sigma[level];
            k.response = v;
            k.angle = 0.f;
            k.level = level;
            k.octave = level / tab.sublevels;
            k.sublevel = level % tab.sublevels;
            k.ix = x;
            k.iy = y;
            kp[idx] = k;
        }
    }
}

size_t doh_smem(int s)
{
    const int R = DT + 4 * s;
    const int C = (DT + 4 * s) | 1;
    return (size_t)R * C * sizeof(float);
}

}  // namespace

cudaError_t configure_detector_kernels()
{
    return allow_max_dynamic_smem(k_doh);
}

cudaError_t launch_doh(const float* L, float* D, int pitch, long long plane_stride, int w, int h,
                       int l0, int nl, const LevelTable& tab, cudaStream_t st)
{
    // levels with similar steps share a launch (shared memory sized for the
    // largest step of the group)
    int i = l0;
    while (i < l0 + nl) {
        int j = i + 1;
        while (j < l0 + nl && doh_smem(tab.step[j]) <= doh_smem(tab.step[i]) * 3 / 2) ++j;
        int smax = 1;
        for (int k = i; k < j; ++k) smax = tab.step[k] > smax ? tab.step[k] : smax;
        if (smax > 32) return cudaErrorInvalidValue;
        const size_t smem = doh_smem(smax);
        if (smem > (size_t)kMaxDynSmem) return cudaErrorInvalidValue;
        dim3 grid((w + DT - 1) / DT, (h + DT - 1) / DT, j - i);
        k_doh<<<grid, DTHREADS, smem, st>>>(L, D, pitch, plane_stride, w, h, i, tab);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        i = j;
    }
    return cudaSuccess;
}

cudaError_t launch_extrema(const float* D, int pitch, long long plane_stride, int w, int h, int n,
                           const LevelTable& tab, float dthreshold, float edge_r,
                           kaze_keypoint* d_kp, int cap, unsigned int* d_count, cudaStream_t st)
{
    if (n < 3) return cudaSuccess;
    const int threads_x = (w + 3) / 4;  // one thread per 4 pixels of a row
    const int bx = threads_x < 256 ? (threads_x + 31) / 32 * 32 : 256;
    dim3 grid((threads_x + bx - 1) / bx, h, n - 2);
    k_extrema<<<grid, bx, 0, st>>>(D, pitch, plane_stride, w, h, tab, dthreshold, edge_r, d_kp, cap, d_count);
    return cudaGetLastError();
}

}  // namespace kz
