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
// GB300 mapping: one launch for a group of levels (grid.z), no shared
// memory.  A thread owns one column x and walks DOH_WK consecutive lattice
// rows y = py + s k of one residue py of the level's step s (doh_walk.cuh).
// Its five column taps x - 2s .. x + 2s are reflected once; each lattice row
// costs five loads (coalesced across the warp, L1/L2-resident) and the three
// horizontal filters, and each output then combines five consecutive lattice
// rows held in registers: ~(WK + 4) / WK x 5 loads and ~30 FP32 operations
// per output.
#include "doh_walk.cuh"

namespace kz {
namespace {

constexpr int WTX = 128;  // threads per CTA (consecutive columns)

// blockIdx.y = py * nseg + seg for the level's step s: residue py, segment
// seg of DOH_WK lattice rows; blocks past the level's residues return.
__global__ void __launch_bounds__(WTX)
k_doh(const float* __restrict__ L, float* __restrict__ D, int pitch, long long plane_stride, int w, int h,
      int l0, const __grid_constant__ LevelTable tab)
{
    const int level = l0 + blockIdx.z;
    const int s = tab.step[level];
    const int nseg = doh_segments(h, s);
    const int py = blockIdx.y / nseg, seg = blockIdx.y - py * nseg;
    const int x = blockIdx.x * WTX + threadIdx.x;
    const int k0 = seg * DOH_WK;
    if (py >= s || x >= w || py + s * k0 >= h) return;
    doh_walk(L + (size_t)level * plane_stride, D + (size_t)level * plane_stride, pitch, w, h, s,
             tab.doh_scale[level], x, py, k0, [](const float* q) { return __ldg(q); });
}

// Each thread tests 4 adjacent pixels (one 16-byte load) of one row of
// level 1 + blockIdx.z.  Most fail the threshold; survivors read their 8
// neighbours and the (2r+1)^2 responses below and above (r = 1: the 26
// neighbours of the 3x3x3 test), fit the quadratic and apply the edge test.
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
        for (int dy = -1; dy <= 1 && is_max; ++dy)  // the 8 neighbours on the level
            for (int dx = -1; dx <= 1; ++dx) {
                if (dx == 0 && dy == 0) continue;
                if (!(v > Dc[(long long)p + (long long)dy * pitch + dx])) {
                    is_max = false;
                    break;
                }
            }
        // levels i - 1 and i + 1 within |dx|, |dy| <= r (r = 1: the 3x3x3
        // test; wider for the sigma x sigma window), pixels outside skipped
        const int r = tab.xr[level];
        for (int l = -1; l <= 1 && is_max; l += 2) {
            const float* Dl = Dc + (long long)l * plane_stride;
            for (int dy = -r; dy <= r && is_max; ++dy) {
                const int yy = y + dy;
                if (yy < 0 || yy >= h) continue;
                for (int dx = -r; dx <= r; ++dx) {
                    const int xx = x + dx;
                    if (xx < 0 || xx >= w) continue;
                    if (!(v > Dl[(long long)yy * pitch + xx])) {
                        is_max = false;
                        break;
                    }
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

}  // namespace

cudaError_t configure_detector_kernels() { return cudaSuccess; }

// All levels of a response go to one launch (no shared memory to size).
int doh_launches(const LevelTable&, int, int nl) { return nl > 0 ? 1 : 0; }

cudaError_t launch_doh(const float* L, float* D, int pitch, long long plane_stride, int w, int h,
                       int l0, int nl, const LevelTable& tab, cudaStream_t st)
{
    if (nl <= 0) return cudaSuccess;
    int gy = 1;
    for (int i = l0; i < l0 + nl; ++i) {
        const int s = tab.step[i];
        if (s < 1 || s > 4096) return cudaErrorInvalidValue;
        const int nseg = doh_segments(h, s);
        gy = s * nseg > gy ? s * nseg : gy;
    }
    if (gy > 65535) return cudaErrorInvalidValue;
    // the determinant's scale in double on the host (the batched path forms
    // it the same way): a double division per thread would keep the GPU's
    // slow FP64 pipe busy for a third of the launch
    LevelTable t = tab;
    for (int i = l0; i < l0 + nl; ++i) {
        const double dd = 1024.0 * t.step[i] * t.step[i];
        t.doh_scale[i] = (float)((double)t.norm[i] / (dd * dd));
    }
    dim3 grid((w + WTX - 1) / WTX, gy, nl);
    k_doh<<<grid, WTX, 0, st>>>(L, D, pitch, plane_stride, w, h, l0, t);
    return cudaGetLastError();
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
