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
// Borders reflect coordinates into the image (half-sample symmetric).
// A CTA computes a 32 x 32 tile: one pass of 5 horizontal taps per needed
// row writes three row-filtered planes to shared memory, one pass of 5
// vertical taps combines them into Lxx, Lyy, Lxy and the response.  One
// launch covers a range of levels (grid.z), each with its own step.
#include "kaze_internal.h"

namespace kz {
namespace {

constexpr int TX = 32, TY = 32, BX = 32, BY = 8;

__global__ void __launch_bounds__(BX* BY)
k_doh(const float* __restrict__ L, float* __restrict__ D, int pitch, long long plane_stride,
      int w, int h, int l0, const __grid_constant__ LevelTable tab)
{
    extern __shared__ float sm[];
    const int level = l0 + blockIdx.z;
    const int s = tab.step[level];
    const float norm = tab.norm[level];
    const float* Li = L + (size_t)level * plane_stride;
    float* Di = D + (size_t)level * plane_stride;
    const int NR = TY + 4 * s;  // rows y0-2s .. y0+TY-1+2s
    float* Hdd = sm;
    float* Hss = Hdd + NR * TX;
    float* Hds = Hss + NR * TX;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int tx = threadIdx.x;
    const int gx = x0 + tx;
    const float inv4s2 = 1.f / (4.f * s * s);
    const float inv32s = 1.f / (32.f * s);

    if (gx < w) {
        const int xm2 = reflect_index(gx - 2 * s, w), xm1 = reflect_index(gx - s, w);
        const int xp1 = reflect_index(gx + s, w), xp2 = reflect_index(gx + 2 * s, w);
        for (int ry = threadIdx.y; ry < NR; ry += BY) {
            const int gy = reflect_index(y0 - 2 * s + ry, h);
            const float* row = Li + (size_t)gy * pitch;
            const float v0 = __ldg(row + xm2), v1 = __ldg(row + xm1), v2 = __ldg(row + gx);
            const float v3 = __ldg(row + xp1), v4 = __ldg(row + xp2);
            Hdd[ry * TX + tx] = (v0 - 2.f * v2 + v4) * inv4s2;
            Hss[ry * TX + tx] = (9.f * (v0 + v4) + 60.f * (v1 + v3) + 118.f * v2) * (1.f / 256.f);
            Hds[ry * TX + tx] = (3.f * (v4 - v0) + 10.f * (v3 - v1)) * inv32s;
        }
    }
    __syncthreads();
    if (gx >= w) return;
    for (int ty = threadIdx.y; ty < TY; ty += BY) {
        const int gy = y0 + ty;
        if (gy >= h) break;
        const int r0 = ty, r1 = ty + s, r2 = ty + 2 * s, r3 = ty + 3 * s, r4 = ty + 4 * s;
        const float lxx = (9.f * (Hdd[r0 * TX + tx] + Hdd[r4 * TX + tx]) +
                           60.f * (Hdd[r1 * TX + tx] + Hdd[r3 * TX + tx]) + 118.f * Hdd[r2 * TX + tx]) *
                          (1.f / 256.f);
        const float lyy = (Hss[r0 * TX + tx] - 2.f * Hss[r2 * TX + tx] + Hss[r4 * TX + tx]) * inv4s2;
        const float lxy = (3.f * (Hds[r4 * TX + tx] - Hds[r0 * TX + tx]) +
                           10.f * (Hds[r3 * TX + tx] - Hds[r1 * TX + tx])) * inv32s;
        Di[(size_t)gy * pitch + gx] = norm * (lxx * lyy - lxy * lxy);
    }
}

// One thread per pixel of levels 1..n-2 (blockIdx.z + 1).  Most pixels fail
// the threshold on their first load; survivors read their 26 neighbours.
__global__ void __launch_bounds__(BX* BY)
k_extrema(const float* __restrict__ D, int pitch, long long plane_stride, int w, int h,
          const __grid_constant__ LevelTable tab, float thr, float edge_r,
          kaze_keypoint* __restrict__ kp, int cap, unsigned int* __restrict__ count)
{
    const int level = 1 + blockIdx.z;
    const int x = blockIdx.x * BX + threadIdx.x;
    const int y = blockIdx.y * BY + threadIdx.y;
    if (x < 1 || y < 1 || x > w - 2 || y > h - 2) return;
    const float* Dc = D + (size_t)level * plane_stride;
    const size_t p = (size_t)y * pitch + x;
    const float v = Dc[p];
    if (!(v > thr)) return;
    for (int l = -1; l <= 1; ++l) {
        const float* Dl = Dc + (long long)l * plane_stride;
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                if (l == 0 && dx == 0 && dy == 0) continue;
                if (!(v > Dl[(long long)p + (long long)dy * pitch + dx])) return;
            }
    }
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
        if (!(det > 0.f)) return;
        if (!(tr * tr * edge_r < (edge_r + 1.f) * (edge_r + 1.f) * det)) return;
    }
    if (det == 0.f) return;
    const float ox = -(hyy * gxv - hxy * gyv) / det;
    const float oy = -(hxx * gyv - hxy * gxv) / det;
    if (fabsf(ox) > 1.f || fabsf(oy) > 1.f) return;
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

}  // namespace

cudaError_t configure_detector_kernels()
{
    return allow_max_dynamic_smem(k_doh);
}

cudaError_t launch_doh(const float* L, float* D, int pitch, long long plane_stride, int w, int h,
                       int l0, int nl, const LevelTable& tab, cudaStream_t st)
{
    if (nl <= 0) return cudaSuccess;
    int smax = 1;
    for (int i = l0; i < l0 + nl; ++i) smax = tab.step[i] > smax ? tab.step[i] : smax;
    size_t smem = (size_t)3 * (TY + 4 * smax) * TX * sizeof(float);
    if (smem > (size_t)kMaxDynSmem) return cudaErrorInvalidValue;
    dim3 grid((w + TX - 1) / TX, (h + TY - 1) / TY, nl);
    k_doh<<<grid, dim3(BX, BY), smem, st>>>(L, D, pitch, plane_stride, w, h, l0, tab);
    return cudaGetLastError();
}

cudaError_t launch_extrema(const float* D, int pitch, long long plane_stride, int w, int h, int n,
                           const LevelTable& tab, float dthreshold, float edge_r,
                           kaze_keypoint* d_kp, int cap, unsigned int* d_count, cudaStream_t st)
{
    if (n < 3) return cudaSuccess;
    dim3 grid((w + BX - 1) / BX, (h + BY - 1) / BY, n - 2);
    k_extrema<<<grid, dim3(BX, BY), 0, st>>>(D, pitch, plane_stride, w, h, tab, dthreshold, edge_r,
                                             d_kp, cap, d_count);
    return cudaGetLastError();
}

}  // namespace kz
