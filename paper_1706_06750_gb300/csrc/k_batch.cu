// k_batch.cu -- the whole detection of many images of uneven sizes in ONE
// persistent launch.
//
// The host flattens the batch into an ordered list of work items, stage-major
// across images:
//   presmooth tiles, gradient-max tiles, histogram tiles, percentile, level-0
//   response tiles, then for every level l = 1..N-1: conductance tiles, row
//   groups, column strips, level-l response tiles, extrema bands of level l-1.
// Resident CTAs pop items in that order from a device counter.  Before it
// runs, an item waits until the stages it reads from are complete for its own
// image (per-image, per-stage completion counters, acquire loads); after it
// runs it publishes (fence + counter increment).  Every wait targets items
// that were popped earlier by running CTAs, so the schedule cannot deadlock,
// and while one image waits the CTAs work on the other images.  Every wait is
// bounded; a wait that runs out (or sees another CTA's failure) sets bit 0 of
// *status and the CTA leaves, so the kernel always terminates.
//
// The arithmetic is the same as the single-image kernels (Sec. III-1/III-2:
// presmoothing, contrast factor, Eq. 2-4 AOS steps, Eq. 8 response, Eq. 9-12
// extrema).  The line solver here takes its chunk length at run time (one
// kernel serves every image size): a' lives in shared memory beside c' and d'.
#include "aos_solver.cuh"
#include "kaze_batch.h"

namespace kz {
namespace batch {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int NT = kBatchThreads;  // 256 threads, 8 warps

__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// ------------------------------------------------------------- stencils --

// Separable Gaussian of radius r on a 32x32 tile: rows then columns.  RC > 0
// fixes the radius at compile time (unrolled taps); RC = 0 reads it from taps.
template <int RC>
__device__ void gauss_tile(const float* __restrict__ in, int in_pitch, float* __restrict__ out, int out_pitch,
                           int w, int h, const GaussTaps& taps, int tx0, int ty0, float* sm)
{
    const int r = RC > 0 ? RC : taps.r;
    const int SW = 32 + 2 * r, SH = 32 + 2 * r;
    float* A = sm;            // SH x (SW)
    float* B = sm + SH * SW;  // SH x 32
    const int tid = threadIdx.x;
    const int x0 = tx0 * 32, y0 = ty0 * 32;
    for (int i = tid; i < SH * SW; i += NT) {
        const int sy = i / SW, sx = i - sy * SW;
        A[i] = __ldg(in + (size_t)reflect_index(y0 - r + sy, h) * in_pitch + reflect_index(x0 - r + sx, w));
    }
    __syncthreads();
    for (int i = tid; i < SH * 32; i += NT) {
        const int sy = i >> 5, sx = i & 31;
        float acc = 0.f;
        if (RC > 0) {
#pragma unroll
            for (int j = 0; j <= 2 * RC; ++j) acc = fmaf(taps.w[j], A[sy * SW + sx + j], acc);
        } else {
            for (int j = 0; j <= 2 * r; ++j) acc = fmaf(taps.w[j], A[sy * SW + sx + j], acc);
        }
        B[i] = acc;
    }
    __syncthreads();
    for (int i = tid; i < 32 * 32; i += NT) {
        const int oy = i >> 5, ox = i & 31;
        float acc = 0.f;
        if (RC > 0) {
#pragma unroll
            for (int j = 0; j <= 2 * RC; ++j) acc = fmaf(taps.w[j], B[(oy + j) * 32 + ox], acc);
        } else {
            for (int j = 0; j <= 2 * r; ++j) acc = fmaf(taps.w[j], B[(oy + j) * 32 + ox], acc);
        }
        if (x0 + ox < w && y0 + oy < h) out[(size_t)(y0 + oy) * out_pitch + x0 + ox] = acc;
    }
    __syncthreads();  // the next tile of the same item reuses the shared memory
}

enum { GM_COND = 0, GM_MAX = 1, GM_HIST = 2 };

// Smoothed Scharr gradient of a 32x32 tile (radius r smoothing, halo r+1),
// then the conductance of Eq. 3, the maximum magnitude or the histogram.
// The arithmetic repeats the single-image kernel (k_filters.cu) operation
// for operation -- symmetric tap pairs, the D / E form of the Scharr pair,
// explicit fmaf -- so the batched and single-image paths agree bit for bit.
template <int RC>
__device__ void gradient_tile(int mode, const float* __restrict__ L, float* __restrict__ g, int pitch, int w, int h,
                              const GaussTaps& taps, float k, int diffusivity, unsigned* hmax_bits, unsigned* hist,
                              int nbins, int tx0, int ty0, float* sm)
{
    const int r = RC > 0 ? RC : taps.r;
    constexpr int CW = 34, CH = 34;
    const int SW = CW + 2 * r, SH = CH + 2 * r;
    float* A = sm;                 // SH x SW
    float* B = A + SH * SW;        // SH x CW
    float* C = B + SH * CW;        // CH x CW
    unsigned* hs = reinterpret_cast<unsigned*>(C + CH * CW);
    const int tid = threadIdx.x;
    const int x0 = tx0 * 32, y0 = ty0 * 32;
    if (mode == GM_HIST)
        for (int i = tid; i < nbins; i += NT) hs[i] = 0u;
    for (int i = tid; i < SH * SW; i += NT) {
        const int sy = i / SW, sx = i - sy * SW;
        A[i] = __ldcg(L + (size_t)reflect_index(y0 - 1 - r + sy, h) * pitch + reflect_index(x0 - 1 - r + sx, w));
    }
    __syncthreads();
    for (int i = tid; i < SH * CW; i += NT) {
        const int sy = i / CW, sx = i - sy * CW;
        const float* a = A + sy * SW + sx;
        float acc = taps.w[r] * a[r];
        if (RC > 0) {
#pragma unroll
            for (int j = 1; j <= RC; ++j) acc = fmaf(taps.w[RC + j], a[RC - j] + a[RC + j], acc);
        } else {
            for (int j = 1; j <= r; ++j) acc = fmaf(taps.w[r + j], a[r - j] + a[r + j], acc);
        }
        B[i] = acc;
    }
    __syncthreads();
    for (int i = tid; i < CH * CW; i += NT) {
        const int sy = i / CW, sx = i - sy * CW;
        const float* b = B + sy * CW + sx;
        float acc = taps.w[r] * b[r * CW];
        if (RC > 0) {
#pragma unroll
            for (int j = 1; j <= RC; ++j) acc = fmaf(taps.w[RC + j], b[(RC - j) * CW] + b[(RC + j) * CW], acc);
        } else {
            for (int j = 1; j <= r; ++j) acc = fmaf(taps.w[r + j], b[(r - j) * CW] + b[(r + j) * CW], acc);
        }
        C[i] = acc;
    }
    __syncthreads();
    const float inv_k2 = mode == GM_COND ? 1.f / (k * k) : 0.f;
    const float hmax_scale = mode == GM_HIST ? (float)nbins / __uint_as_float(__ldcg(hmax_bits)) : 0.f;
    float local_max = 0.f;
    for (int i = tid; i < 32 * 32; i += NT) {
        const int oy = i >> 5, ox = i & 31;
        const int gx = x0 + ox, gy = y0 + oy;
        const float* c = C + (oy + 1) * CW + (ox + 1);
        const float dm = c[-CW + 1] - c[-CW - 1];
        const float d0 = c[1] - c[-1];
        const float dp = c[CW + 1] - c[CW - 1];
        const float em = fmaf(10.f, c[-CW], 3.f * (c[-CW - 1] + c[-CW + 1]));
        const float ep = fmaf(10.f, c[CW], 3.f * (c[CW - 1] + c[CW + 1]));
        const float lx = fmaf(10.f, d0, 3.f * (dm + dp)) * (1.f / 32.f);
        const float ly = (ep - em) * (1.f / 32.f);
        const float m2 = fmaf(ly, ly, lx * lx);
        if (gx >= w || gy >= h) continue;
        if (mode == GM_COND) {
            // explicit fmaf: the single-image kernels write the same operations
            g[(size_t)gy * pitch + gx] =
                diffusivity == KAZE_G1 ? expf(-(m2 * inv_k2)) : __fdividef(1.f, fmaf(m2, inv_k2, 1.f));
        } else if (gx >= 1 && gx <= w - 2 && gy >= 1 && gy <= h - 2) {
            const float m = sqrtf(m2);
            if (mode == GM_MAX) {
                local_max = fmaxf(local_max, m);
            } else if (m > 0.f) {
                const int b = min((int)floorf(m * hmax_scale), nbins - 1);
                atomicAdd(&hs[b], 1u);
            }
        }
    }
    if (mode == GM_MAX) {
        for (int o = 16; o > 0; o >>= 1) local_max = fmaxf(local_max, __shfl_xor_sync(FULL, local_max, o));
        if ((tid & 31) == 0 && local_max > 0.f) atomicMax(hmax_bits, __float_as_uint(local_max));
    }
    if (mode == GM_HIST) {
        __syncthreads();
        for (int i = tid; i < nbins; i += NT)
            if (hs[i]) atomicAdd(&hist[i], hs[i]);
    }
    __syncthreads();  // the next tile of the same item reuses the shared memory
}

// Percentile pick of Sec. III-1 (first warp of the CTA).
__device__ void percentile_item(const unsigned* hist, int nbins, const unsigned* hmax_bits, double pct, float* k_out)
{
    const int lane = threadIdx.x & 31;
    const int per = (nbins + 31) / 32;
    const int b0 = min(lane * per, nbins), b1 = min(b0 + per, nbins);
    unsigned long long s = 0;
    for (int b = b0; b < b1; ++b) s += __ldcg(hist + b);
    unsigned long long inc = s;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long t = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += t;
    }
    const unsigned long long n = __shfl_sync(FULL, inc, 31);
    const float hmax = __uint_as_float(__ldcg(hmax_bits));
    if (n == 0 || !(hmax > 0.f)) {
        if (lane == 0) *k_out = 0.03f;
        return;
    }
    const double target = pct * (double)n;
    const unsigned ballot = __ballot_sync(FULL, (double)inc >= target);
    if (ballot == 0u) {
        if (lane == 0) *k_out = 0.03f;
        return;
    }
    if (lane == __ffs(ballot) - 1) {
        unsigned long long cum = inc - s;
        for (int b = b0; b < b1; ++b) {
            cum += __ldcg(hist + b);
            if ((double)cum >= target) {
                *k_out = hmax * (float)(b + 1) / (float)nbins;
                break;
            }
        }
    }
}

// Eq. 8 response of a 64x64 tile (same lattice-run scheme as the
// single-image response kernel).
__device__ void doh_tile(const float* __restrict__ L, float* __restrict__ D, int pitch, int w, int h, int s,
                         float scale, int tx0, int ty0, float* T)
{
    constexpr int DT = 64, RUN = 8;
    const int R = DT + 4 * s;
    const int C = (DT + 4 * s) | 1;
    const int x0 = tx0 * DT, y0 = ty0 * DT;
    const int tid = threadIdx.x;
    const int cw = DT + 4 * s;
    for (int i = tid; i < R * cw; i += NT) {
        const int r = i / cw, c = i - r * cw;
        T[r * C + c] =
            __ldcg(L + (size_t)reflect_index(y0 - 2 * s + r, h) * pitch + reflect_index(x0 - 2 * s + c, w));
    }
    __syncthreads();
    const int col = tid & (DT - 1), lane_row = tid / DT;
    const int per_class = (DT / s + (DT % s ? 1 : 0) + RUN - 1) / RUN;
    const int nruns = s * per_class;
    const int gx = x0 + col;
    for (int ri = lane_row; ri < nruns; ri += NT / DT) {
        const int q = ri / per_class, j = ri - q * per_class;
        const int base = q + s * RUN * j;
        if (base >= DT) continue;
        float hd[RUN + 4], hs[RUN + 4], hx[RUN + 4];
#pragma unroll
        for (int m = 0; m < RUN + 4; ++m) {
            const int tr = base + s * m;
            if (tr < R) {
                const float* t = T + tr * C + col;
                doh_lattice_row(t[0], t[s], t[2 * s], t[3 * s], t[4 * s], hd[m], hs[m], hx[m]);
            } else {
                hd[m] = hs[m] = hx[m] = 0.f;
            }
        }
#pragma unroll
        for (int kk = 0; kk < RUN; ++kk) {
            const int ty = base + s * kk;
            if (ty >= DT) break;
            const int gy = y0 + ty;
            if (gy >= h || gx >= w) continue;
            D[(size_t)gy * pitch + gx] = doh_value(hd + kk, hs + kk, hx + kk, scale);
        }
    }
}

// 3x3x3 maxima, sub-pixel fit and edge test on rows [y0, y0 + rows) of one
// level (Sec. II-B, Eq. 9-12); keypoints go to the image's own buffer.
__device__ void extrema_band(const float* __restrict__ D, int pitch, long long plane, int w, int h, int level,
                             int y0, int rows, const BatchParams& P, const ImageDesc& im)
{
    const float* Dc = D + (size_t)level * plane;
    const int nvec = (w + 3) / 4;
    for (int e = threadIdx.x; e < rows * nvec; e += NT) {
        const int y = y0 + e / nvec;
        const int x4 = 4 * (e % nvec);
        if (y < 1 || y > h - 2) continue;
        const float4 c4 = __ldcg(reinterpret_cast<const float4*>(Dc + (size_t)y * pitch + x4));
        const float cv[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int x = x4 + q;
            const float v = cv[q];
            if (!(v > P.thr) || x < 1 || x > w - 2) continue;
            const size_t p = (size_t)y * pitch + x;
            bool is_max = true;
            for (int l = -1; l <= 1 && is_max; ++l) {
                const float* Dl = Dc + (long long)l * plane;
                for (int dy = -1; dy <= 1 && is_max; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        if (l == 0 && dx == 0 && dy == 0) continue;
                        if (!(v > __ldcg(Dl + (long long)p + (long long)dy * pitch + dx))) {
                            is_max = false;
                            break;
                        }
                    }
            }
            if (!is_max) continue;
            const float dxp = __ldcg(Dc + p + 1), dxm = __ldcg(Dc + p - 1);
            const float dyp = __ldcg(Dc + p + pitch), dym = __ldcg(Dc + p - pitch);
            const float gxv = 0.5f * (dxp - dxm), gyv = 0.5f * (dyp - dym);
            const float hxx = dxp - 2.f * v + dxm, hyy = dyp - 2.f * v + dym;
            const float hxy = 0.25f * (__ldcg(Dc + p + pitch + 1) - __ldcg(Dc + p + pitch - 1) -
                                       __ldcg(Dc + p - pitch + 1) + __ldcg(Dc + p - pitch - 1));
            const float det = hxx * hyy - hxy * hxy, tr = hxx + hyy;
            if (P.edge_r > 0.f) {
                if (!(det > 0.f)) continue;
                if (!(tr * tr * P.edge_r < (P.edge_r + 1.f) * (P.edge_r + 1.f) * det)) continue;
            }
            if (det == 0.f) continue;
            const float ox = -(hyy * gxv - hxy * gyv) / det;
            const float oy = -(hxx * gyv - hxy * gxv) / det;
            if (fabsf(ox) > 1.f || fabsf(oy) > 1.f) continue;
            const unsigned idx = atomicAdd(im.kp_count, 1u);
            if (idx < (unsigned)im.kp_cap) {
                kaze_keypoint kpt;
                kpt.x = (float)x + ox;
                kpt.y = (float)y + oy;
                kpt.sigma = P.tab.sigma[level];
                kpt.response = v;
                kpt.angle = 0.f;
                kpt.level = level;
                kpt.octave = level / P.tab.sublevels;
                kpt.sublevel = level % P.tab.sublevels;
                kpt.ix = x;
                kpt.iy = y;
                im.kp[idx] = kpt;
            }
        }
    }
}

// ----------------------------------------------------------- line solver --
// Same elimination as the single-image solver (modified Thomas on chunks,
// PCR on the interface), with the chunk length m known only at run time: a'
// is kept in shared memory at the stride of g and d.

struct ChunkEqs {
    float aL, cL, dL, aF, cF, dF;
};

__device__ ChunkEqs chunk_reduce_rt(float* g, float* d, float* ap, int S, float g_prev, float g_next, int j0,
                                    int m, int n, float tau)
{
    ChunkEqs q;
    float cprev = 0.f, dprev = 0.f, aprev = 0.f;
    float gcur = g[0];
    float a = (j0 > 0 && j0 < n) ? -tau * (g_prev + gcur) : 0.f;
    for (int i = 0; i < m; ++i) {
        const int j = j0 + i;
        const float gn = (i + 1 < m) ? g[(i + 1) * S] : g_next;
        const float c = (j + 1 < n) ? -tau * (gcur + gn) : 0.f;
        const float di = (j < n) ? d[i * S] : 0.f;
        const float b = 1.f - a - c;
        float r, apv, dp;
        if (i < 2) {
            r = rcp_approx(b);
            apv = a * r;
            dp = di * r;
        } else {
            r = rcp_approx(b - a * cprev);
            apv = -a * aprev * r;
            dp = (di - a * dprev) * r;
        }
        const float cp = c * r;
        g[i * S] = cp;
        d[i * S] = dp;
        ap[i * S] = apv;
        cprev = cp;
        dprev = dp;
        aprev = apv;
        a = c;
        gcur = gn;
    }
    q.aL = aprev;
    q.cL = cprev;
    q.dL = dprev;
    float cn = g[(m - 2) * S], dn = d[(m - 2) * S], an = ap[(m - 2) * S];
    for (int i = m - 3; i >= 1; --i) {
        const float ci = g[i * S];
        const float di = d[i * S] - ci * dn;
        const float ai = ap[i * S] - ci * an;
        const float cc = -ci * cn;
        g[i * S] = cc;
        d[i * S] = di;
        ap[i * S] = ai;
        cn = cc;
        dn = di;
        an = ai;
    }
    const float c0 = g[0], d0 = d[0];
    const float r = rcp_approx(1.f - c0 * an);
    q.dF = r * (d0 - c0 * dn);
    q.aF = r * ap[0];
    q.cF = -r * c0 * cn;
    return q;
}

__device__ __forceinline__ void interface_solve(const ChunkEqs& e, int lane, float& xfirst, float& xlast)
{
    float aFn = __shfl_down_sync(FULL, e.aF, 1);
    float cFn = __shfl_down_sync(FULL, e.cF, 1);
    float dFn = __shfl_down_sync(FULL, e.dF, 1);
    if (lane == 31) aFn = cFn = dFn = 0.f;
    float A = -e.aL * e.aF;
    float B = 1.f - e.aL * e.cF - e.cL * aFn;
    float C = -e.cL * cFn;
    float D = e.dL - e.aL * e.dF - e.cL * dFn;
    if (lane == 0) A = 0.f;
    if (lane == 31) C = 0.f;
#pragma unroll
    for (int s = 1; s < 32; s <<= 1) {
        float Am = __shfl_up_sync(FULL, A, s), Bm = __shfl_up_sync(FULL, B, s);
        float Cm = __shfl_up_sync(FULL, C, s), Dm = __shfl_up_sync(FULL, D, s);
        float Ap = __shfl_down_sync(FULL, A, s), Bp = __shfl_down_sync(FULL, B, s);
        float Cp = __shfl_down_sync(FULL, C, s), Dp = __shfl_down_sync(FULL, D, s);
        if (lane < s) {
            Am = 0.f;
            Bm = 1.f;
            Cm = 0.f;
            Dm = 0.f;
        }
        if (lane + s > 31) {
            Ap = 0.f;
            Bp = 1.f;
            Cp = 0.f;
            Dp = 0.f;
        }
        const float k1 = A * rcp_approx(Bm), k2 = C * rcp_approx(Bp);
        const float nA = -Am * k1, nC = -Cp * k2;
        const float nB = B - Cm * k1 - Ap * k2;
        const float nD = D - Dm * k1 - Dp * k2;
        A = nA;
        B = nB;
        C = nC;
        D = nD;
    }
    xlast = D * rcp_approx(B);
    float xprev = __shfl_up_sync(FULL, xlast, 1);
    if (lane == 0) xprev = 0.f;
    xfirst = e.dF - e.aF * xprev - e.cF * xlast;
}

// Interface of P = 32 NW chunks (NW = 1 or 2) held in eq[6][P]; one warp.
__device__ void interface_line(const float* eq, float* xs, int P, int lane)
{
    auto load = [&](int p) {
        ChunkEqs e;
        e.aL = eq[0 * P + p];
        e.cL = eq[1 * P + p];
        e.dL = eq[2 * P + p];
        e.aF = eq[3 * P + p];
        e.cF = eq[4 * P + p];
        e.dF = eq[5 * P + p];
        return e;
    };
    if (P == 32) {
        float xf, xl;
        interface_solve(load(lane), lane, xf, xl);
        xs[lane] = xf;
        xs[P + lane] = xl;
        return;
    }
    const int p0 = 2 * lane, p1 = p0 + 1, p2 = p0 + 2;
    const ChunkEqs e0 = load(p0), e1 = load(p1);
    const float aF2 = p2 < P ? eq[3 * P + p2] : 0.f;
    const float cF2 = p2 < P ? eq[4 * P + p2] : 0.f;
    const float dF2 = p2 < P ? eq[5 * P + p2] : 0.f;
    const float A0 = -e0.aL * e0.aF, B0 = 1.f - e0.aL * e0.cF - e0.cL * e1.aF;
    const float C0 = -e0.cL * e1.cF, D0 = e0.dL - e0.aL * e0.dF - e0.cL * e1.dF;
    const float A1 = -e1.aL * e1.aF, B1 = 1.f - e1.aL * e1.cF - e1.cL * aF2;
    const float C1 = -e1.cL * cF2, D1 = e1.dL - e1.aL * e1.dF - e1.cL * dF2;
    const float r0 = rcp_approx(B0), r1 = rcp_approx(B1);
    ChunkEqs q;
    q.aF = lane ? A0 * r0 : 0.f;
    q.cF = C0 * r0;
    q.dF = D0 * r0;
    q.aL = A1 * r1;
    q.cL = lane < 31 ? C1 * r1 : 0.f;
    q.dL = D1 * r1;
    float L0, L1;
    interface_solve(q, lane, L0, L1);
    float Lm = __shfl_up_sync(FULL, L1, 1);
    if (lane == 0) Lm = 0.f;
    xs[p0] = e0.dF - e0.aF * Lm - e0.cF * L0;
    xs[p1] = e1.dF - e1.aF * L0 - e1.cF * L1;
    xs[P + p0] = L0;
    xs[P + p1] = L1;
}

// Row group: 4 rows, 2 warps (64 chunks) per row.
__device__ void rows_item(const ImageDesc& im, const float* __restrict__ L, float tau, int y0, float* sm)
{
    constexpr int P = 64;
    const int w = im.w, h = im.h, pitch = im.pitch, m = im.mrow;
    const int ls = (P * m + 3) / 4 * 4;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = warp >> 1, part = warp & 1;
    const int y = y0 + r;
    const bool active = y < h;
    float* sg = sm + (size_t)r * (3 * ls + 8 * P);
    float* sd = sg + ls;
    float* sa = sd + ls;
    float* eq = sa + ls;
    float* xs = eq + 6 * P;
    const int p = part * 32 + lane;
    if (active) {
        const float* grow = im.g + (size_t)y * pitch;
        const float* lrow = L + (size_t)y * pitch;
        const int w4 = w & ~3;
        for (int x = p * 4; x < w4; x += 4 * P) {
            *reinterpret_cast<float4*>(sg + x) = __ldcg(reinterpret_cast<const float4*>(grow + x));
            *reinterpret_cast<float4*>(sd + x) = __ldcg(reinterpret_cast<const float4*>(lrow + x));
        }
        for (int x = w4 + p; x < w; x += P) {
            sg[x] = __ldcg(grow + x);
            sd[x] = __ldcg(lrow + x);
        }
    }
    __syncthreads();
    const int j0 = p * m;
    const float g_prev = (j0 > 0 && j0 - 1 < w) ? sg[j0 - 1] : 0.f;
    const float g_next = (j0 + m < w) ? sg[j0 + m] : 0.f;
    __syncthreads();
    if (active) {
        const ChunkEqs q = chunk_reduce_rt(sg + j0, sd + j0, sa + j0, 1, g_prev, g_next, j0, m, w, tau);
        eq[0 * P + p] = q.aL;
        eq[1 * P + p] = q.cL;
        eq[2 * P + p] = q.dL;
        eq[3 * P + p] = q.aF;
        eq[4 * P + p] = q.cF;
        eq[5 * P + p] = q.dF;
    }
    __syncthreads();
    if (active && part == 0) interface_line(eq, xs, P, lane);
    __syncthreads();
    if (active) {
        const float xf = xs[p], xl = xs[P + p];
        float* cd = sd + j0;
        const float* cc = sg + j0;
        const float* ca = sa + j0;
        cd[0] = xf;
        for (int i = 1; i < m - 1; ++i) cd[i] = cd[i] - ca[i] * xf - cc[i] * xl;
        cd[m - 1] = xl;
    }
    __syncthreads();
    if (active) {
        float* urow = im.ux + (size_t)y * pitch;
        const int w4 = w & ~3;
        for (int x = p * 4; x < w4; x += 4 * P)
            *reinterpret_cast<float4*>(urow + x) = *reinterpret_cast<const float4*>(sd + x);
        for (int x = w4 + p; x < w; x += P) urow[x] = sd[x];
    }
}

// Column strip of `cols` columns (4 or 8): 256 / cols threads per column
// (P = 64 or 32 chunks), a thread per (column, chunk).
__device__ void cols_item(const ImageDesc& im, const float* __restrict__ L, float* __restrict__ Ln, float tau,
                          int x0, int cols, float* sm)
{
    const int P = NT / cols;
    const int w = im.w, h = im.h, pitch = im.pitch;
    const int m = cols == 4 ? im.mcol : im.mcol32;
    const int rs = P * m;  // rows held (>= h)
    float* tg = sm;
    float* td = tg + (size_t)rs * cols;
    float* ta = td + (size_t)rs * cols;
    float* eq0 = ta + (size_t)rs * cols;
    const int tid = threadIdx.x;
    const int c = tid % cols, p = tid / cols;
    const bool full = x0 + cols <= w;
    // stage the strip: one 16-byte load per 4 columns of a row
    const int vper = cols / 4;
    for (int e = tid; e < rs * vper; e += NT) {
        const int j = e / vper, q = e - j * vper;
        float4 gv = make_float4(0.f, 0.f, 0.f, 0.f), lv = gv;
        if (j < h) {
            const size_t gi = (size_t)j * pitch + x0 + 4 * q;
            if (full) {
                gv = __ldcg(reinterpret_cast<const float4*>(im.g + gi));
                lv = __ldcg(reinterpret_cast<const float4*>(L + gi));
            } else {
                float* gp = &gv.x;
                float* lp = &lv.x;
                for (int k = 0; k < 4; ++k)
                    if (x0 + 4 * q + k < w) {
                        gp[k] = __ldcg(im.g + gi + k);
                        lp[k] = __ldcg(L + gi + k);
                    }
            }
        }
        *reinterpret_cast<float4*>(tg + (size_t)j * cols + 4 * q) = gv;
        *reinterpret_cast<float4*>(td + (size_t)j * cols + 4 * q) = lv;
    }
    __syncthreads();
    const int j0 = p * m;
    float* ce = tg + (size_t)j0 * cols + c;
    float* cd = td + (size_t)j0 * cols + c;
    float* ca = ta + (size_t)j0 * cols + c;
    const float g_prev = (j0 > 0 && j0 - 1 < h) ? ce[-cols] : 0.f;
    const float g_next = (j0 + m < h) ? ce[m * cols] : 0.f;
    __syncthreads();
    float* eqc = eq0 + (size_t)c * 8 * P;
    const ChunkEqs q = chunk_reduce_rt(ce, cd, ca, cols, g_prev, g_next, j0, m, h, tau);
    eqc[0 * P + p] = q.aL;
    eqc[1 * P + p] = q.cL;
    eqc[2 * P + p] = q.dL;
    eqc[3 * P + p] = q.aF;
    eqc[4 * P + p] = q.cF;
    eqc[5 * P + p] = q.dF;
    __syncthreads();
    const int warp = tid >> 5, lane = tid & 31;
    if (warp < cols) {
        float* eqw = eq0 + (size_t)warp * 8 * P;
        interface_line(eqw, eqw + 6 * P, P, lane);
    }
    __syncthreads();
    {
        const float xf = eqc[6 * P + p], xl = eqc[7 * P + p];
        cd[0] = xf;
        for (int i = 1; i < m - 1; ++i) cd[i * cols] = cd[i * cols] - ca[i * cols] * xf - ce[i * cols] * xl;
        cd[(m - 1) * cols] = xl;
    }
    __syncthreads();
    for (int e = tid; e < h * vper; e += NT) {
        const int j = e / vper, qq = e - j * vper;
        const size_t gi = (size_t)j * pitch + x0 + 4 * qq;
        const float* uy = td + (size_t)j * cols + 4 * qq;
        if (full) {
            const float4 a = __ldcg(reinterpret_cast<const float4*>(im.ux + gi));
            float4 rr;
            rr.x = 0.5f * (a.x + uy[0]);
            rr.y = 0.5f * (a.y + uy[1]);
            rr.z = 0.5f * (a.z + uy[2]);
            rr.w = 0.5f * (a.w + uy[3]);
            *reinterpret_cast<float4*>(Ln + gi) = rr;
        } else {
            for (int k = 0; k < 4; ++k)
                if (x0 + 4 * qq + k < w) Ln[gi + k] = 0.5f * (__ldcg(im.ux + gi + k) + uy[k]);
        }
    }
}

// Row group with a compile-time chunk length: the register-resident solver
// of the single-image path (aos_solver.cuh), 4 rows x 2 warps.
template <int M>
__device__ void rows_item_m(const ImageDesc& im, const float* __restrict__ L, float tau, int y0, float* sm)
{
    constexpr int P = 64;
    constexpr int LS = aos::row_stride_floats(P, M);
    const int w = im.w, h = im.h, pitch = im.pitch;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = warp >> 1, part = warp & 1;
    const int y = y0 + r;
    const bool active = y < h;
    float* sg = sm + (size_t)r * (2 * LS + 8 * P);
    float* sd = sg + LS;
    float* eq = sd + LS;
    float* xs = eq + 6 * P;
    const int p = part * 32 + lane;
    const int w4 = w & ~3;
    if (active) {
        const float* grow = im.g + (size_t)y * pitch;
        const float* lrow = L + (size_t)y * pitch;
        for (int x = p * 4; x < w4; x += 4 * P) {
            *reinterpret_cast<float4*>(sg + x) = __ldcg(reinterpret_cast<const float4*>(grow + x));
            *reinterpret_cast<float4*>(sd + x) = __ldcg(reinterpret_cast<const float4*>(lrow + x));
        }
        for (int x = w4 + p; x < w; x += P) {
            sg[x] = __ldcg(grow + x);
            sd[x] = __ldcg(lrow + x);
        }
    }
    __syncthreads();
    const int j0 = p * M;
    float* ce = sg + j0;
    float* cd = sd + j0;
    const float g_prev = (j0 > 0 && j0 - 1 < w) ? ce[-1] : 0.f;
    const float g_next = (j0 + M < w) ? ce[M] : 0.f;
    __syncthreads();
    float ap[M];
    if (active) {
        const aos::ChunkEqs q = aos::chunk_reduce<1, M>(ce, cd, g_prev, g_next, j0, w, tau, ap);
        eq[0 * P + p] = q.aL;
        eq[1 * P + p] = q.cL;
        eq[2 * P + p] = q.dL;
        eq[3 * P + p] = q.aF;
        eq[4 * P + p] = q.cF;
        eq[5 * P + p] = q.dF;
    }
    __syncthreads();
    if (active && part == 0) aos::interface_line<2>(eq, xs, lane);
    __syncthreads();
    if (active) aos::chunk_solution<1, M>(ce, cd, ap, xs[p], xs[P + p]);
    __syncthreads();
    if (active) {
        float* urow = im.ux + (size_t)y * pitch;
        for (int x = p * 4; x < w4; x += 4 * P)
            *reinterpret_cast<float4*>(urow + x) = *reinterpret_cast<const float4*>(sd + x);
        for (int x = w4 + p; x < w; x += P) urow[x] = sd[x];
    }
    __syncthreads();
}

// Column strip of 4 columns, 64 chunks, compile-time chunk length.
template <int M>
__device__ void cols_item_m(const ImageDesc& im, const float* __restrict__ L, float* __restrict__ Ln, float tau,
                            int x0, float* sm)
{
    constexpr int COLS = 4, P = 64;
    constexpr int RS = P * M;
    const int w = im.w, h = im.h, pitch = im.pitch;
    float* tg = sm;
    float* td = tg + (size_t)RS * COLS;
    float* eq0 = td + (size_t)RS * COLS;
    const int tid = threadIdx.x;
    const int c = tid % COLS, p = tid / COLS;
    const bool full = x0 + COLS <= w;
    for (int j = tid; j < RS; j += NT) {
        float4 gv = make_float4(0.f, 0.f, 0.f, 0.f), lv = gv;
        if (j < h) {
            const size_t gi = (size_t)j * pitch + x0;
            if (full) {
                gv = __ldcg(reinterpret_cast<const float4*>(im.g + gi));
                lv = __ldcg(reinterpret_cast<const float4*>(L + gi));
            } else {
                float* gp = &gv.x;
                float* lp = &lv.x;
                for (int k = 0; k < 4; ++k)
                    if (x0 + k < w) {
                        gp[k] = __ldcg(im.g + gi + k);
                        lp[k] = __ldcg(L + gi + k);
                    }
            }
        }
        *reinterpret_cast<float4*>(tg + (size_t)j * COLS) = gv;
        *reinterpret_cast<float4*>(td + (size_t)j * COLS) = lv;
    }
    __syncthreads();
    const int j0 = p * M;
    float* ce = tg + (size_t)j0 * COLS + c;
    float* cd = td + (size_t)j0 * COLS + c;
    const float g_prev = (j0 > 0 && j0 - 1 < h) ? ce[-COLS] : 0.f;
    const float g_next = (j0 + M < h) ? ce[M * COLS] : 0.f;
    __syncthreads();
    float ap[M];
    const aos::ChunkEqs q = aos::chunk_reduce<COLS, M>(ce, cd, g_prev, g_next, j0, h, tau, ap);
    float* eqc = eq0 + (size_t)c * 8 * P;
    eqc[0 * P + p] = q.aL;
    eqc[1 * P + p] = q.cL;
    eqc[2 * P + p] = q.dL;
    eqc[3 * P + p] = q.aF;
    eqc[4 * P + p] = q.cF;
    eqc[5 * P + p] = q.dF;
    __syncthreads();
    const int warp = tid >> 5, lane = tid & 31;
    if (warp < COLS) {
        float* eqw = eq0 + (size_t)warp * 8 * P;
        aos::interface_line<2>(eqw, eqw + 6 * P, lane);
    }
    __syncthreads();
    aos::chunk_solution<COLS, M>(ce, cd, ap, eqc[6 * P + p], eqc[7 * P + p]);
    __syncthreads();
    for (int j = tid; j < h; j += NT) {
        const size_t gi = (size_t)j * pitch + x0;
        const float* uy = td + (size_t)j * COLS;
        if (full) {
            const float4 a = __ldcg(reinterpret_cast<const float4*>(im.ux + gi));
            float4 rr;
            rr.x = 0.5f * (a.x + uy[0]);
            rr.y = 0.5f * (a.y + uy[1]);
            rr.z = 0.5f * (a.z + uy[2]);
            rr.w = 0.5f * (a.w + uy[3]);
            *reinterpret_cast<float4*>(Ln + gi) = rr;
        } else {
            for (int k = 0; k < 4; ++k)
                if (x0 + k < w) Ln[gi + k] = 0.5f * (__ldcg(im.ux + gi + k) + uy[k]);
        }
    }
    __syncthreads();
}

// Chunk lengths with compiled solvers (the sizes of the mixed-size
// workload); other lengths use the run-time solver.
#define KZ_BATCH_ROW_M(X) X(11) X(21) X(31)
#define KZ_BATCH_COL_M(X) X(9) X(13) X(17) X(19)

__device__ void rows_dispatch(const ImageDesc& im, const float* L, float tau, int y0, float* sm)
{
    switch (im.mrow) {
#define KZ_R(M)                              \
    case M:                                  \
        rows_item_m<M>(im, L, tau, y0, sm);  \
        return;
        KZ_BATCH_ROW_M(KZ_R)
#undef KZ_R
        default: rows_item(im, L, tau, y0, sm); __syncthreads();
    }
}

__device__ void cols_dispatch(const ImageDesc& im, const float* L, float* Ln, float tau, int x0, int cols, float* sm)
{
    if (cols == 4) {
        switch (im.mcol) {
#define KZ_C(M)                                  \
    case M:                                      \
        cols_item_m<M>(im, L, Ln, tau, x0, sm);  \
        return;
            KZ_BATCH_COL_M(KZ_C)
#undef KZ_C
            default: break;
        }
    }
    cols_item(im, L, Ln, tau, x0, cols, sm);
    __syncthreads();
}

// ------------------------------------------------------ the persistent kernel

// Waits (thread 0) until counter[slot] reaches need[slot]; false on timeout
// or when another CTA has already failed.
__device__ bool wait_stage(const BatchParams& P, int image, int slot)
{
    if (slot < 0) return true;
    const size_t k = (size_t)image * P.slots + slot;
    const unsigned need = P.need[k];
    const long long t0 = clock64();
    while (ld_acquire(P.done + k) < need) {
        if (*(volatile int*)P.status) return false;
        if (clock64() - t0 > P.spin_limit) {
            atomicOr(P.status, 1);
            return false;
        }
        __nanosleep(64);
    }
    return true;
}

__global__ void __launch_bounds__(NT, 2) k_batch(const __grid_constant__ BatchParams P)
{
    extern __shared__ __align__(16) float sm[];
    __shared__ unsigned s_item, s_next;
    __shared__ int s_ok;
    // stages this CTA has already seen complete: one bit per (image, slot)
    // for the first kMaxCachedImages images
    constexpr int kMaxCachedImages = 64;
    __shared__ unsigned s_seen[kMaxCachedImages * kSlotWords];
    const int tid = threadIdx.x;
    for (int i = tid; i < kMaxCachedImages * kSlotWords; i += NT) s_seen[i] = 0u;
    if (tid == 0) s_next = atomicAdd(P.next, 1u);
    __syncthreads();
    auto wait_cached = [&](int image, int slot) -> bool {
        if (image < kMaxCachedImages) {
            unsigned& word = s_seen[image * kSlotWords + (slot >> 5)];
            const unsigned bit = 1u << (slot & 31);
            if (word & bit) return true;
            if (!wait_stage(P, image, slot)) return false;
            word |= bit;
            return true;
        }
        return wait_stage(P, image, slot);
    };
    while (true) {
        // the next item was fetched while the previous one ran
        if (tid == 0) {
            s_item = s_next;
            if (s_item < (unsigned)P.n_items) s_next = atomicAdd(P.next, 1u);
        }
        __syncthreads();
        const unsigned it = s_item;
        if (it >= (unsigned)P.n_items) return;
        const Item item = P.items[it];
        const ImageDesc& im = P.imgs[item.image];
        const int lv = item.level;
        // dependencies of this item's stage, for its own image
        if (tid == 0) {
            bool ok = true;
            switch (item.kind) {
                case IT_GMAX: ok = wait_cached(item.image, slot_presmooth()); break;
                case IT_GHIST: ok = wait_cached(item.image, slot_gmax()); break;
                case IT_PCT: ok = wait_cached(item.image, slot_ghist()); break;
                case IT_COND:
                    ok = wait_cached(item.image, lv == 1 ? slot_pct() : slot_cols(lv - 1)) &&
                         wait_cached(item.image, slot_presmooth());
                    break;
                case IT_ROWS: ok = wait_cached(item.image, slot_cond(lv)); break;
                case IT_COLS: ok = wait_cached(item.image, slot_rows(lv)); break;
                case IT_DOH: ok = wait_cached(item.image, lv == 0 ? slot_presmooth() : slot_cols(lv)); break;
                case IT_EXTREMA:
                    ok = wait_cached(item.image, slot_doh(lv - 1)) && wait_cached(item.image, slot_doh(lv)) &&
                         wait_cached(item.image, slot_doh(lv + 1));
                    break;
                default: break;
            }
            s_ok = ok;
        }
        __syncthreads();
        if (!s_ok) return;
        const float* Lprev = im.levels + (size_t)(lv > 0 ? lv - 1 : 0) * im.plane;
        int slot = -1;
        switch (item.kind) {
            case IT_PRESMOOTH: {
                const int gx = item.index % im.groups32_x, ty = item.index / im.groups32_x;
                for (int tx = gx * kTilesPerItem; tx < min(im.tiles32_x, (gx + 1) * kTilesPerItem); ++tx) {
                    if (P.taps0.r == 5)
                        gauss_tile<5>(im.img, im.img_pitch, im.levels, im.pitch, im.w, im.h, P.taps0, tx, ty, sm);
                    else
                        gauss_tile<0>(im.img, im.img_pitch, im.levels, im.pitch, im.w, im.h, P.taps0, tx, ty, sm);
                }
                slot = slot_presmooth();
                break;
            }
            case IT_GMAX:
            case IT_GHIST: {
                const int gx = item.index % im.groups32_x, ty = item.index / im.groups32_x;
                const int mode = item.kind == IT_GMAX ? GM_MAX : GM_HIST;
                for (int tx = gx * kTilesPerItem; tx < min(im.tiles32_x, (gx + 1) * kTilesPerItem); ++tx) {
                    if (P.tapsd.r == 3)
                        gradient_tile<3>(mode, im.levels, nullptr, im.pitch, im.w, im.h, P.tapsd, 0.f, 0, im.hmax,
                                         im.hist, P.nbins, tx, ty, sm);
                    else
                        gradient_tile<0>(mode, im.levels, nullptr, im.pitch, im.w, im.h, P.tapsd, 0.f, 0, im.hmax,
                                         im.hist, P.nbins, tx, ty, sm);
                }
                slot = item.kind == IT_GMAX ? slot_gmax() : slot_ghist();
                break;
            }
            case IT_PCT:
                if (tid < 32) {
                    if (P.k_override > 0.f) {
                        if (tid == 0) *im.k = P.k_override;
                    } else {
                        percentile_item(im.hist, P.nbins, im.hmax, P.pct, im.k);
                    }
                }
                slot = slot_pct();
                break;
            case IT_COND: {
                const int gx = item.index % im.groups32_x, ty = item.index / im.groups32_x;
                const float k = __ldcg(im.k);
                for (int tx = gx * kTilesPerItem; tx < min(im.tiles32_x, (gx + 1) * kTilesPerItem); ++tx) {
                    if (P.tapsd.r == 3)
                        gradient_tile<3>(GM_COND, Lprev, im.g, im.pitch, im.w, im.h, P.tapsd, k, P.diffusivity,
                                         nullptr, nullptr, 0, tx, ty, sm);
                    else
                        gradient_tile<0>(GM_COND, Lprev, im.g, im.pitch, im.w, im.h, P.tapsd, k, P.diffusivity,
                                         nullptr, nullptr, 0, tx, ty, sm);
                }
                slot = slot_cond(lv);
                break;
            }
            case IT_ROWS:
                rows_dispatch(im, Lprev, P.tau[lv], 4 * item.index, sm);
                slot = slot_rows(lv);
                break;
            case IT_COLS:
                cols_dispatch(im, Lprev, im.levels + (size_t)lv * im.plane, P.tau[lv], P.cols * item.index, P.cols,
                              sm);
                slot = slot_cols(lv);
                break;
            case IT_DOH: {
                const int tx = item.index % im.tiles64_x, ty = item.index / im.tiles64_x;
                doh_tile(im.levels + (size_t)lv * im.plane, im.doh + (size_t)lv * im.plane, im.pitch, im.w, im.h,
                         P.tab.step[lv], P.doh_scale[lv], tx, ty, sm);
                slot = slot_doh(lv);
                break;
            }
            case IT_EXTREMA:
                extrema_band(im.doh, im.pitch, im.plane, im.w, im.h, lv, kExtremaRows * item.index, kExtremaRows,
                             P, im);
                slot = slot_extrema(lv);
                break;
            default: break;
        }
        __syncthreads();  // every thread's stores are issued before the release
        if (tid == 0) {
            __threadfence();
            atomicAdd(P.done + (size_t)item.image * P.slots + slot, 1u);
        }
    }
}

}  // namespace

cudaError_t configure_batch_kernel(int smem)
{
    return cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

cudaError_t batch_occupancy(int smem, int* blocks_per_sm)
{
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_batch, NT, smem);
}

cudaError_t launch_batch(const BatchParams& p, int grid, int smem, cudaStream_t st)
{
    k_batch<<<grid, NT, smem, st>>>(p);
    return cudaGetLastError();
}

}  // namespace batch
}  // namespace kz
