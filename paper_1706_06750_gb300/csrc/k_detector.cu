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
// seg of DOH_WK lattice rows; blocks past the level's residues return.  With
// a candidate list, each response the extremum test can accept sets a bit of
// the walker's mask (no branch in the walk: code there costs instruction-
// cache misses), and the walker's bits are appended after the walk, one
// atomic per warp.
__global__ void __launch_bounds__(WTX)
k_doh(const float* __restrict__ L, float* __restrict__ D, int pitch, long long plane_stride, int w, int h,
      int l0, const __grid_constant__ LevelTable tab, const Candidates cand)
{
    static_assert(DOH_WK <= 32, "one mask bit per output");
    const int level = l0 + blockIdx.z;
    const int s = tab.step[level];
    const int nseg = doh_segments(h, s);
    const int py = blockIdx.y / nseg, seg = blockIdx.y - py * nseg;
    const int x = blockIdx.x * WTX + threadIdx.x;
    const int k0 = seg * DOH_WK;
    if (py >= s || x >= w || py + s * k0 >= h) return;
    // the threshold this column's responses are listed above: +inf off the
    // listed levels and on the first and last columns
    const bool listing = cand.list != nullptr && level >= cand.lo && level <= cand.hi;  // uniform
    const float thr = listing && x >= 1 && x <= w - 2 ? cand.thr : __int_as_float(0x7f800000);
    unsigned cm = 0u;
    doh_walk(L + (size_t)level * plane_stride, D + (size_t)level * plane_stride, pitch, w, h, s,
             tab.doh_scale[level], x, py, k0, [](const float* q) { return __ldg(q); },
             [&](int j, float v) { cm |= (v > thr ? 1u : 0u) << j; });
    if (!listing) return;
    // rows 0 and h - 1 are not tested
    if (py + s * k0 == 0) cm &= ~1u;
    const int jl = (h - 1 - py) / s - k0;  // the output on row h - 1, if any
    if (jl >= 0 && jl < DOH_WK && py + s * (k0 + jl) == h - 1) cm &= ~(1u << jl);
    // the warp's lanes with a column inside the image: a prefix of the warp
    const unsigned lane = threadIdx.x & 31u;
    const int nv = min(32, w - (x - (int)lane));
    const unsigned act = nv >= 32 ? 0xffffffffu : (1u << nv) - 1u;
    if (__ballot_sync(act, cm != 0u) == 0u) return;
    const unsigned n = (unsigned)__popc(cm);
    unsigned incl = n;  // inclusive prefix of the counts over the lanes
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned t = __shfl_up_sync(act, incl, o);
        if (lane >= (unsigned)o) incl += t;
    }
    const int last = 31 - __clz(act);
    unsigned base = 0u;
    if ((int)lane == last) base = atomicAdd(cand.count, incl);
    base = __shfl_sync(act, base, last) + incl - n;
    for (unsigned i = base; cm; cm &= cm - 1u, ++i) {
        const int jj = __ffs(cm) - 1;
        const int y = py + s * (k0 + jj);
        if (i < cand.cap)
            cand.list[i] = ((unsigned long long)level << 48) | ((unsigned long long)y << 24) | (unsigned)x;
    }
}

// The extremum test of one pixel (x, y) of `level` whose response v passed
// the threshold, 1 <= x <= w-2, 1 <= y <= h-2: larger than its 8 neighbours
// on the level and than the (2r+1)^2 responses below and above (r = 1: the
// 26 neighbours of the 3x3x3 test; wider for the sigma x sigma window), then
// the quadratic fit and the edge test; appends the keypoint.
__device__ __forceinline__ void extremum_test(const float* __restrict__ Dc, int pitch, long long plane_stride, int w,
                                              int h, int level, int x, int y, float v, const LevelTable& tab,
                                              float edge_r, kaze_keypoint* __restrict__ kp, int cap,
                                              unsigned int* __restrict__ count)
{
    const size_t p = (size_t)y * pitch + x;
    // the 8 neighbours on the level, loaded together
    float nb[9];
#pragma unroll
    for (int j = 0; j < 9; ++j) nb[j] = Dc[(long long)p + (long long)(j / 3 - 1) * pitch + (j % 3 - 1)];
#pragma unroll
    for (int j = 0; j < 9; ++j)
        if (j != 4 && !(v > nb[j])) return;
    // levels i - 1 and i + 1 within |dx|, |dy| <= r, pixels outside skipped
    // (r = 1: all 18 inside the image, loaded together)
    const int r = tab.xr[level];
    if (r == 1) {
        float ab[18];
#pragma unroll
        for (int j = 0; j < 18; ++j)
            ab[j] = Dc[(long long)(j < 9 ? -plane_stride : plane_stride) + (long long)p +
                       (long long)((j % 9) / 3 - 1) * pitch + ((j % 9) % 3 - 1)];
#pragma unroll
        for (int j = 0; j < 18; ++j)
            if (!(v > ab[j])) return;
    } else for (int l = -1; l <= 1; l += 2) {
        const float* Dl = Dc + (long long)l * plane_stride;
        for (int dy = -r; dy <= r; ++dy) {
            const int yy = y + dy;
            if (yy < 0 || yy >= h) continue;
            for (int dx = -r; dx <= r; ++dx) {
                const int xx = x + dx;
                if (xx < 0 || xx >= w) continue;
                if (!(v > Dl[(long long)yy * pitch + xx])) return;
            }
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

// The 4 pixels (one 16-byte load) at x4 of row y of `level`: most fail the
// threshold; survivors take the extremum test.
__device__ __forceinline__ void extrema_quad(const float* __restrict__ D, int pitch, long long plane_stride, int w,
                                             int h, int level, int x4, int y, const LevelTable& tab, float thr,
                                             float edge_r, kaze_keypoint* __restrict__ kp, int cap,
                                             unsigned int* __restrict__ count)
{
    const float* Dc = D + (size_t)level * plane_stride;
    const float4 c4 = __ldg(reinterpret_cast<const float4*>(Dc + (size_t)y * pitch + x4));
    const float cv[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int x = x4 + q;
        if (!(cv[q] > thr) || x < 1 || x > w - 2) continue;
        extremum_test(Dc, pitch, plane_stride, w, h, level, x, y, cv[q], tab, edge_r, kp, cap, count);
    }
}

// Each thread tests 4 adjacent pixels of one row of level 1 + blockIdx.z.
__global__ void __launch_bounds__(256)
k_extrema(const float* __restrict__ D, int pitch, long long plane_stride, int w, int h,
          const __grid_constant__ LevelTable tab, float thr, float edge_r,
          kaze_keypoint* __restrict__ kp, int cap, unsigned int* __restrict__ count)
{
    const int y = blockIdx.y;
    const int x4 = (blockIdx.x * blockDim.x + threadIdx.x) * 4;
    if (y < 1 || y > h - 2 || x4 >= w) return;
    extrema_quad(D, pitch, plane_stride, w, h, 1 + blockIdx.z, x4, y, tab, thr, edge_r, kp, cap, count);
}

// The pixels the response launch listed, one a thread (grid-stride); when the
// list overflowed, every row quad of levels 1 .. n-2 instead.
__global__ void __launch_bounds__(256)
k_extrema_cand(const float* __restrict__ D, int pitch, long long plane_stride, int w, int h, int n,
               const __grid_constant__ LevelTable tab, float thr, float edge_r,
               kaze_keypoint* __restrict__ kp, int cap, unsigned int* __restrict__ count, const Candidates cand)
{
    const unsigned nc = *(volatile const unsigned*)cand.count;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t t0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (nc <= cand.cap) {
        for (size_t i = t0; i < nc; i += stride) {
            const unsigned long long e = cand.list[i];
            const int level = (int)(e >> 48), y = (int)((e >> 24) & 0xffffffu), x = (int)(e & 0xffffffu);
            const float* Dc = D + (size_t)level * plane_stride;
            extremum_test(Dc, pitch, plane_stride, w, h, level, x, y, Dc[(size_t)y * pitch + x], tab, edge_r, kp,
                          cap, count);
        }
        return;
    }
    const size_t qx = (size_t)(w + 3) / 4, per_level = qx * (size_t)h;
    for (size_t u = t0; u < per_level * (size_t)(n - 2); u += stride) {
        const int level = 1 + (int)(u / per_level);
        const size_t r = u - (size_t)(level - 1) * per_level;
        const int y = (int)(r / qx), x4 = (int)(r - (size_t)y * qx) * 4;
        if (y < 1 || y > h - 2) continue;
        extrema_quad(D, pitch, plane_stride, w, h, level, x4, y, tab, thr, edge_r, kp, cap, count);
    }
}

}  // namespace

cudaError_t configure_detector_kernels() { return cudaSuccess; }

// All levels of a response go to one launch (no shared memory to size).
int doh_launches(const LevelTable&, int, int nl) { return nl > 0 ? 1 : 0; }

cudaError_t launch_doh(const float* L, float* D, int pitch, long long plane_stride, int w, int h,
                       int l0, int nl, const LevelTable& tab, cudaStream_t st, const Candidates* cand)
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
    Candidates c;
    if (cand) {
        if (!cand->count || (cand->cap > 0 && !cand->list) || w > (1 << 24) || h > (1 << 24))
            return cudaErrorInvalidValue;
        c = *cand;
    }
    k_doh<<<grid, WTX, 0, st>>>(L, D, pitch, plane_stride, w, h, l0, t, c);
    return cudaGetLastError();
}

cudaError_t launch_extrema(const float* D, int pitch, long long plane_stride, int w, int h, int n,
                           const LevelTable& tab, float dthreshold, float edge_r,
                           kaze_keypoint* d_kp, int cap, unsigned int* d_count, cudaStream_t st,
                           const Candidates* cand)
{
    if (n < 3) return cudaSuccess;
    if (cand) {
        if (!cand->count || (cand->cap > 0 && !cand->list)) return cudaErrorInvalidValue;
        int dev = 0, sms = 0;  // the grid only sizes the grid-stride loop
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        k_extrema_cand<<<4 * sms, 256, 0, st>>>(D, pitch, plane_stride, w, h, n, tab, dthreshold, edge_r, d_kp, cap,
                                                d_count, *cand);
        return cudaGetLastError();
    }
    const int threads_x = (w + 3) / 4;  // one thread per 4 pixels of a row
    const int bx = threads_x < 256 ? (threads_x + 31) / 32 * 32 : 256;
    dim3 grid((threads_x + bx - 1) / bx, h, n - 2);
    k_extrema<<<grid, bx, 0, st>>>(D, pitch, plane_stride, w, h, tab, dthreshold, edge_r, d_kp, cap, d_count);
    return cudaGetLastError();
}

}  // namespace kz
