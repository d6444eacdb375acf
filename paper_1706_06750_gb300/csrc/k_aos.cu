// k_aos.cu -- the semi-implicit step of Eq. 4 by additive operator splitting
// (Weickert, ter Haar Romeny & Viergever 1998), m = 2:
//
//     L_next = 1/2 [ (I - 2 tau A_x(g))^-1 + (I - 2 tau A_y(g))^-1 ] L_prev
//
// Each line operator is tridiagonal, symmetric and strictly diagonally
// dominant: between neighbours j, j+1 the off-diagonal is -tau (g_j + g_j+1),
// the diagonal is 1 minus the two off-diagonals, and the borders are Neumann
// (no coupling past the first / last pixel).
//
// GB300 mapping.  A line is solved by ONE WARP out of shared memory:
//   * the line (conductance g and right-hand side d) is staged in shared
//     memory, split into 32 contiguous chunks of m = max(2, ceil(n/32)) rows,
//     chunk p at offset p*ms with ms = m rounded up to an odd number so the
//     32 lanes walking their chunks hit 32 different banks;
//   * phase 1: every lane eliminates the interior of its chunk twice, top
//     down and bottom up (two independent recurrences, interleaved for ILP),
//     leaving two equations that couple only the chunk's first and last
//     unknowns to the neighbouring chunks (the partition method of Wang 1981
//     in the "modified Thomas" form);
//   * phase 2: the 64-unknown interface system is reduced to 32 unknowns
//     (one per lane) and solved by parallel cyclic reduction with warp
//     shuffles (5 steps);
//   * phase 3: every lane solves its chunk's interior by Thomas with the two
//     now-known end values, overwriting g and d in place.
// Rows are contiguous in memory: a CTA holds several rows, one per warp, and
// stages each with 128-bit loads.  Columns are strided: a CTA holds a strip
// of COLS adjacent columns (row segments of COLS floats, sector-aligned
// loads), one warp per column, and fuses the final average with the row
// solution.
#include "kaze_internal.h"

namespace kz {
namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

struct LineGeom {
    int n;       // line length
    int m;       // chunk length (>= 2); 32*m >= n
    int ms;      // chunk stride in shared memory (odd, >= m)
    float inv_m; // 1/m for the index split in the staging loops
};

__host__ __device__ inline LineGeom make_geom(int n)
{
    LineGeom g;
    g.n = n;
    g.m = (n + 31) / 32;
    if (g.m < 2) g.m = 2;
    g.ms = g.m | 1;
    g.inv_m = 1.0f / (float)g.m;
    return g;
}

// Shared-memory slot of line element j (0 <= j < 32*m).
__device__ __forceinline__ int slot(int j, const LineGeom& G)
{
    // exact for j < 2^21: (j + 0.5)/m is at least 0.5/m away from an integer
    int p = (int)(((float)j + 0.5f) * G.inv_m);
    return p * G.ms + (j - p * G.m);
}

// Solves (I - 2 tau A(g)) x = d for one line held in shared memory by the
// calling warp.  sg[] holds g, sd[] holds d (chunked layout); on return sd[]
// holds x and sg[] is clobbered.
__device__ __forceinline__ void solve_line_warp(float* sg, float* sd, const LineGeom& G, float tau)
{
    const int lane = threadIdx.x & 31;
    const int n = G.n, m = G.m, ms = G.ms;
    const int j0 = lane * m;           // first line index of this chunk
    float* cg = sg + lane * ms;        // this chunk's g
    float* cd = sd + lane * ms;        // this chunk's d

    // g at chunk-local index i in [-1, m]; zero beyond the line.
    auto gl = [&](int i) -> float {
        int j = j0 + i;
        if (j < 0 || j >= n) return 0.f;
        if (i < 0) return sg[(lane - 1) * ms + (m - 1)];
        if (i >= m) return sg[(lane + 1) * ms];
        return cg[i];
    };
    auto dl = [&](int i) -> float { return (j0 + i < n) ? cd[i] : 0.f; };
    // off-diagonals of local row i given g_{i-1}, g_i, g_{i+1}
    auto lower = [&](int i, float gm, float g0) -> float {
        int j = j0 + i;
        return (j >= 1 && j < n) ? -tau * (gm + g0) : 0.f;
    };
    auto upper = [&](int i, float g0, float gp) -> float {
        int j = j0 + i;
        return (j + 1 < n) ? -tau * (g0 + gp) : 0.f;
    };

    // ---- phase 1: two eliminations per chunk ----
    // down: rows 1..m-1 with x_0 as the known left end ->
    //       aL x_0 + x_{m-1} + cL x_m = dL
    // up:   rows m-2..0 with x_{m-1} as the known right end ->
    //       aF x_{-1} + x_0 + cF x_{m-1} = dF
    float aL, cL, dL, aF, cF, dF;
    {
        // down state
        float gdA = gl(0), gdB = gl(1);
        float ap = 0.f, cp = 0.f, dp = 0.f;
        // up state
        float guB = gl(m - 2), guC = gl(m - 1);
        float au = 0.f, cu = 0.f, du = 0.f;
        for (int t = 0; t < m - 1; ++t) {
            // down row i = 1 + t
            {
                const int i = 1 + t;
                float gdC = gl(i + 1);
                float a = lower(i, gdA, gdB), c = upper(i, gdB, gdC);
                float b = 1.f - a - c, d = dl(i);
                if (t == 0) {
                    float r = rcp_approx(b);
                    ap = a * r; cp = c * r; dp = d * r;
                } else {
                    float r = rcp_approx(b - a * cp);
                    ap = -a * ap * r;
                    dp = (d - a * dp) * r;
                    cp = c * r;
                }
                gdA = gdB; gdB = gdC;
            }
            // up row i = m - 2 - t
            {
                const int i = m - 2 - t;
                float guA = gl(i - 1);
                float a = lower(i, guA, guB), c = upper(i, guB, guC);
                float b = 1.f - a - c, d = dl(i);
                if (t == 0) {
                    float r = rcp_approx(b);
                    au = a * r; cu = c * r; du = d * r;
                } else {
                    float r = rcp_approx(b - c * au);
                    cu = -c * cu * r;
                    du = (d - c * du) * r;
                    au = a * r;
                }
                guC = guB; guB = guA;
            }
        }
        aL = ap; cL = cp; dL = dp;
        aF = au; cF = cu; dF = du;
    }
    __syncwarp();

    // ---- phase 2: interface system ----
    // Eliminate the first unknowns F_p = dF - aF Lst_{p-1} - cF Lst_p from
    // the last-row equations: A Lst_{p-1} + B Lst_p + C Lst_{p+1} = D.
    float aFn = __shfl_down_sync(FULL, aF, 1);
    float cFn = __shfl_down_sync(FULL, cF, 1);
    float dFn = __shfl_down_sync(FULL, dF, 1);
    if (lane == 31) { aFn = 0.f; cFn = 0.f; dFn = 0.f; }
    float A = -aL * aF;
    float B = 1.f - aL * cF - cL * aFn;
    float C = -cL * cFn;
    float D = dL - aL * dF - cL * dFn;
    if (lane == 0) A = 0.f;
    if (lane == 31) C = 0.f;
    // parallel cyclic reduction over the 32 lanes
#pragma unroll
    for (int s = 1; s < 32; s <<= 1) {
        float Am = __shfl_up_sync(FULL, A, s), Bm = __shfl_up_sync(FULL, B, s);
        float Cm = __shfl_up_sync(FULL, C, s), Dm = __shfl_up_sync(FULL, D, s);
        float Ap = __shfl_down_sync(FULL, A, s), Bp = __shfl_down_sync(FULL, B, s);
        float Cp = __shfl_down_sync(FULL, C, s), Dp = __shfl_down_sync(FULL, D, s);
        if (lane < s) { Am = 0.f; Bm = 1.f; Cm = 0.f; Dm = 0.f; }
        if (lane + s > 31) { Ap = 0.f; Bp = 1.f; Cp = 0.f; Dp = 0.f; }
        float k1 = A * rcp_approx(Bm);
        float k2 = C * rcp_approx(Bp);
        float nA = -Am * k1;
        float nC = -Cp * k2;
        float nB = B - Cm * k1 - Ap * k2;
        float nD = D - Dm * k1 - Dp * k2;
        A = nA; B = nB; C = nC; D = nD;
    }
    const float xlast = D * rcp_approx(B);
    float xprev = __shfl_up_sync(FULL, xlast, 1);
    if (lane == 0) xprev = 0.f;
    const float xfirst = dF - aF * xprev - cF * xlast;

    // ---- phase 3: chunk interior by Thomas with both ends known ----
    // (each lane now touches only its own chunk)
    if (m >= 3) {
        float gA = cg[0], gB = cg[1];
        float cp = 0.f, dp = 0.f;
        for (int i = 1; i <= m - 2; ++i) {
            float gC = cg[i + 1];
            float a = lower(i, gA, gB), c = upper(i, gB, gC);
            float b = 1.f - a - c;
            float rhs = dl(i);
            if (i == 1) { rhs -= a * xfirst; a = 0.f; }
            if (i == m - 2) { rhs -= c * xlast; c = 0.f; }
            float r = rcp_approx(b - a * cp);
            dp = (rhs - a * dp) * r;
            cp = c * r;
            cg[i] = cp;
            cd[i] = dp;
            gA = gB; gB = gC;
        }
        float x = xlast;
        for (int i = m - 2; i >= 1; --i) {
            x = cd[i] - cg[i] * x;
            cd[i] = x;
        }
    }
    cd[0] = xfirst;
    cd[m - 1] = xlast;
    __syncwarp();
}

// ---------------------------------------------------------------- rows ----
// One warp per row; blockDim = 32 * rows_per_cta.
__global__ void k_aos_rows(const float* __restrict__ L, const float* __restrict__ g,
                           float* __restrict__ ux, int pitch, int w, int h, float tau,
                           LineGeom G)
{
    extern __shared__ float sm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int y = blockIdx.x * (blockDim.x >> 5) + warp;
    if (y >= h) return;  // no CTA-wide barrier below
    float* sg = sm + (size_t)warp * 2 * 32 * G.ms;
    float* sd = sg + 32 * G.ms;
    const float* grow = g + (size_t)y * pitch;
    const float* lrow = L + (size_t)y * pitch;

    const int w4 = w & ~3;
    for (int x = lane * 4; x < w4; x += 128) {
        float4 gv = __ldg(reinterpret_cast<const float4*>(grow + x));
        float4 lv = __ldg(reinterpret_cast<const float4*>(lrow + x));
        sg[slot(x, G)] = gv.x; sd[slot(x, G)] = lv.x;
        sg[slot(x + 1, G)] = gv.y; sd[slot(x + 1, G)] = lv.y;
        sg[slot(x + 2, G)] = gv.z; sd[slot(x + 2, G)] = lv.z;
        sg[slot(x + 3, G)] = gv.w; sd[slot(x + 3, G)] = lv.w;
    }
    for (int x = w4 + lane; x < w; x += 32) {
        sg[slot(x, G)] = __ldg(grow + x);
        sd[slot(x, G)] = __ldg(lrow + x);
    }
    __syncwarp();
    solve_line_warp(sg, sd, G, tau);

    float* urow = ux + (size_t)y * pitch;
    for (int x = lane * 4; x < w4; x += 128) {
        float4 v;
        v.x = sd[slot(x, G)];
        v.y = sd[slot(x + 1, G)];
        v.z = sd[slot(x + 2, G)];
        v.w = sd[slot(x + 3, G)];
        *reinterpret_cast<float4*>(urow + x) = v;
    }
    for (int x = w4 + lane; x < w; x += 32) urow[x] = sd[slot(x, G)];
}

// ------------------------------------------------------------- columns ----
// A strip of `cols` adjacent columns per CTA, one warp per column;
// blockDim = 32 * cols.  Column c's arrays start at c * line_stride floats,
// line_stride = 64 ms + 4 so the staging stores of 4 rows x 8 columns fall
// in 32 different banks.
__global__ void k_aos_cols(const float* __restrict__ L, const float* __restrict__ g,
                           const float* __restrict__ ux, float* __restrict__ Lnext,
                           int pitch, int w, int h, float tau, LineGeom G, int cols,
                           int line_stride)
{
    extern __shared__ float sm[];
    const int warp = threadIdx.x >> 5;
    const int x0 = blockIdx.x * cols;
    const int nthreads = blockDim.x;
    const int ncols = min(cols, w - x0);
    const int total = h * cols;

    for (int e = threadIdx.x; e < total; e += nthreads) {
        int y = e / cols, c = e - y * cols;
        if (c < ncols) {
            size_t gi = (size_t)y * pitch + x0 + c;
            float* base = sm + (size_t)c * line_stride;
            int s = slot(y, G);
            base[s] = __ldg(g + gi);
            base[32 * G.ms + s] = __ldg(L + gi);
        }
    }
    __syncthreads();
    if (warp < ncols) {
        float* base = sm + (size_t)warp * line_stride;
        solve_line_warp(base, base + 32 * G.ms, G, tau);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < total; e += nthreads) {
        int y = e / cols, c = e - y * cols;
        if (c < ncols) {
            size_t gi = (size_t)y * pitch + x0 + c;
            const float* base = sm + (size_t)c * line_stride;
            Lnext[gi] = 0.5f * (__ldg(ux + gi) + base[32 * G.ms + slot(y, G)]);
        }
    }
}

constexpr size_t kSmemCap = 220 * 1024;

int rows_per_cta(int w)
{
    LineGeom G = make_geom(w);
    size_t per = (size_t)2 * 32 * G.ms * sizeof(float);
    int r = (int)(kSmemCap / per);
    return r < 1 ? 0 : (r > 4 ? 4 : r);
}

int cols_per_cta(int h, int* stride)
{
    LineGeom G = make_geom(h);
    int ls = 64 * G.ms + 4;
    *stride = ls;
    size_t per = (size_t)ls * sizeof(float);
    for (int c = 8; c >= 1; c >>= 1)
        if ((size_t)c * per <= kSmemCap) return c;
    return 0;
}

}  // namespace

cudaError_t configure_aos_kernels()
{
    cudaError_t e = cudaFuncSetAttribute(k_aos_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_aos_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
    return e;
}

size_t aos_rows_smem_bytes(int w)
{
    int r = rows_per_cta(w);
    if (r == 0) return 0;
    return (size_t)r * 2 * 32 * make_geom(w).ms * sizeof(float);
}

size_t aos_cols_smem_bytes(int h)
{
    int ls;
    int c = cols_per_cta(h, &ls);
    if (c == 0) return 0;
    return (size_t)c * ls * sizeof(float);
}

cudaError_t launch_aos_rows(const float* L, const float* g, float* ux, int pitch, int w, int h,
                            float tau, cudaStream_t st)
{
    int r = rows_per_cta(w);
    if (r == 0) return cudaErrorInvalidValue;
    LineGeom G = make_geom(w);
    size_t smem = aos_rows_smem_bytes(w);
    k_aos_rows<<<(h + r - 1) / r, 32 * r, smem, st>>>(L, g, ux, pitch, w, h, tau, G);
    return cudaGetLastError();
}

cudaError_t launch_aos_cols(const float* L, const float* g, const float* ux, float* Lnext, int pitch,
                            int w, int h, float tau, cudaStream_t st)
{
    int ls;
    int c = cols_per_cta(h, &ls);
    if (c == 0) return cudaErrorInvalidValue;
    LineGeom G = make_geom(h);
    size_t smem = (size_t)c * ls * sizeof(float);
    k_aos_cols<<<(w + c - 1) / c, 32 * c, smem, st>>>(L, g, ux, Lnext, pitch, w, h, tau, G, c, ls);
    return cudaGetLastError();
}

}  // namespace kz
