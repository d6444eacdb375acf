// aos_solver.cuh -- line solver and kernels of the semi-implicit step of
// Eq. 4 by additive operator splitting (Weickert, ter Haar Romeny &
// Viergever 1998), m = 2:
//
//     L_next = 1/2 [ (I - 2 tau A_x(g))^-1 + (I - 2 tau A_y(g))^-1 ] L_prev
//
// Each line operator is tridiagonal, symmetric and strictly diagonally
// dominant: between neighbours j, j+1 the off-diagonal is -tau (g_j + g_j+1),
// the diagonal is 1 minus the two off-diagonals, and the borders are Neumann
// (no coupling past the first / last pixel).
//
// Line solver (partition method of Wang 1981 in the "modified Thomas" form of
// Laszlo, Giles & Appleyard 2016).  A line of n unknowns is padded with
// identity rows to P chunks of M rows (P = 32 NW, M odd, compile-time).
//   phase 1  per chunk, a forward sweep (one reciprocal per row) and a
//            multiply-only backward sweep leave every row coupled only to the
//            chunk's first and last unknowns, and two equations that tie those
//            to the neighbouring chunks;
//   phase 2  the interface system (one unknown per chunk after eliminating
//            the first unknowns) is solved by one warp with parallel cyclic
//            reduction over shuffles;
//   phase 3  every interior unknown follows independently from the two ends.
// The off-diagonals are formed on the fly from g; a' stays in registers
// (loops fully unrolled over the compile-time M), c' and d' overwrite g and d
// in shared memory.  M odd puts the chunks' i-th rows in distinct banks.
//
// GB300 mapping.
//   rows:    NW warps per row (chunk p = lane + 32 * warp-in-row).  The row's g
//            and L are staged with two TMA bulk copies (cp.async.bulk,
//            mbarrier completion); the solution leaves in 128-bit stores.
//   columns: a CTA per strip of COLS adjacent columns, a thread per (column,
//            chunk).  The strip of g and L is staged by TMA 2-D tensor copies
//            (boxes of COLS x 256, zero fill past the image) into a
//            [row][COLS] tile; the interface systems are solved by one warp
//            per column; the row solution is averaged in with 128-bit loads
//            and stores.
// Every mbarrier wait is bounded; on timeout the kernel raises bit 0 of
// *status and returns.
#pragma once

#include <cuda.h>

#include "kaze_internal.h"

namespace kz {
namespace aos {

constexpr unsigned FULL = 0xffffffffu;

// ------------------------------------------------------------ geometry ----

// Chunks per line: 64 (two warps) once 32 chunks would exceed 17 rows.
__host__ __device__ inline int warps_per_line(int n) { return (n + 31) / 32 > 17 ? 2 : 1; }

// Compile-time chunk lengths, per warps-per-line.
constexpr int kChunks1[] = {3, 5, 7, 9, 11, 13, 15, 17};
constexpr int kChunks2[] = {9, 11, 13, 15, 17, 19, 21, 23, 25, 27, 29, 31, 33, 37, 41, 45,
                            49, 57, 65, 73, 81, 97, 113, 129};

inline int chunk_len(int n)
{
    const int nw = warps_per_line(n);
    const int P = 32 * nw;
    if (nw == 1) {
        for (int m : kChunks1)
            if (P * m >= n) return m;
    } else {
        for (int m : kChunks2)
            if (P * m >= n) return m;
    }
    return 0;  // line too long
}

__host__ __device__ constexpr int row_stride_floats(int P, int M) { return (P * M + 3) / 4 * 4; }
__host__ __device__ constexpr int rows_staged(int P, int M) { return (P * M + 255) / 256 * 256; }

// ------------------------------------------------------------- helpers ----

__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Waits for phase `parity` of the barrier; gives up after ~2^31 cycles.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity)
{
    const long long t0 = clock64();
    while (true) {
        unsigned ok;
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
        if (clock64() - t0 > (1ll << 31)) return false;
    }
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// ------------------------------------------------------------ the solver --

// Two equations per chunk after phase 1:
//   aL x_0 + x_{M-1} + cL x_M  = dL     (last row, x_M = next chunk's first)
//   aF x_-1 + x_0 + cF x_{M-1} = dF     (first row, x_-1 = previous chunk's last)
struct ChunkEqs {
    float aL, cL, dL, aF, cF, dF;
};

// Phase 1 on one chunk of rows j0 .. j0+M-1 of a line of length n.  g and d
// hold the chunk's conductances and right-hand side at stride S and are
// overwritten by c' and d'; g_prev = g_{j0-1} and g_next = g_{j0+M} were read
// before any chunk was overwritten (0 outside the line).  Rows j >= n are
// identity rows.  After the forward sweep every row i >= 1 reads
//   a'_i x_0 + x_i + c'_i x_{i+1} = d'_i;
// the backward sweep turns rows 1..M-2 into a'_i x_0 + x_i + c'_i x_{M-1} =
// d'_i and row 0 into a'_0 x_{-1} + x_0 + c'_0 x_{M-1} = d'_0.
template <int S, int M>
__device__ __forceinline__ ChunkEqs chunk_reduce(float* g, float* d, float g_prev, float g_next, int j0, int n,
                                                 float tau, float (&ap)[M])
{
    static_assert(M >= 3, "the elimination needs chunks of at least 3 rows");
    ChunkEqs q;
    float cprev = 0.f, dprev = 0.f, aprev = 0.f;
    auto row = [&](int i, float a, float c, float di) {
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
        ap[i] = apv;
        cprev = cp;
        dprev = dp;
        aprev = apv;
    };
    float gcur = g[0];
    if (j0 > 0 && j0 + M < n) {  // every row has both neighbours in the line
        float a = -tau * (g_prev + gcur);
#pragma unroll
        for (int i = 0; i < M; ++i) {
            const float gn = (i + 1 < M) ? g[(i + 1) * S] : g_next;
            const float c = -tau * (gcur + gn);
            row(i, a, c, d[i * S]);
            a = c;
            gcur = gn;
        }
    } else {
        float a = (j0 > 0 && j0 < n) ? -tau * (g_prev + gcur) : 0.f;
#pragma unroll
        for (int i = 0; i < M; ++i) {
            const int j = j0 + i;
            const float gn = (i + 1 < M) ? g[(i + 1) * S] : g_next;
            const float c = (j + 1 < n) ? -tau * (gcur + gn) : 0.f;
            row(i, a, c, (j < n) ? d[i * S] : 0.f);
            a = c;
            gcur = gn;
        }
    }
    q.aL = aprev;
    q.cL = cprev;
    q.dL = dprev;
    float cn = g[(M - 2) * S], dn = d[(M - 2) * S], an = ap[M - 2];
#pragma unroll
    for (int i = M - 3; i >= 1; --i) {
        const float ci = g[i * S];
        const float di = d[i * S] - ci * dn;
        const float ai = ap[i] - ci * an;
        const float cc = -ci * cn;
        g[i * S] = cc;
        d[i * S] = di;
        ap[i] = ai;
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

// Phase 2 for 32 chunks, one per lane: returns the chunk's first and last
// unknowns.  The first unknowns are eliminated,
//   F_p = dF - aF Lst_{p-1} - cF Lst_p,
// leaving A Lst_{p-1} + B Lst_p + C Lst_{p+1} = D, solved by PCR.
__device__ __forceinline__ void interface_solve(const ChunkEqs& e, int lane, float& xfirst, float& xlast)
{
    float aFn = __shfl_down_sync(FULL, e.aF, 1);
    float cFn = __shfl_down_sync(FULL, e.cF, 1);
    float dFn = __shfl_down_sync(FULL, e.dF, 1);
    if (lane == 31) {
        aFn = 0.f;
        cFn = 0.f;
        dFn = 0.f;
    }
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
        const float k1 = A * rcp_approx(Bm);
        const float k2 = C * rcp_approx(Bp);
        const float nA = -Am * k1;
        const float nC = -Cp * k2;
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

// Phase 2 for one line of P = 32 NW chunks whose equations sit in shared
// memory (eq[k P + p] for k = aL, cL, dL, aF, cF, dF), run by one full warp;
// lane l owns chunks NW l .. NW l + NW - 1.  Writes each chunk's first
// unknown to xs[p] and its last unknown to xs[P + p].  For NW = 2 the last
// unknowns satisfy a P-row tridiagonal system; lane l's two normalised rows
// are the first/last equations of a chunk of length 2, so interface_solve
// applies unchanged.
template <int NW>
__device__ __forceinline__ void interface_line(const float* eq, float* xs, int lane)
{
    constexpr int P = 32 * NW;
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
    if constexpr (NW == 1) {
        float xf, xl;
        interface_solve(load(lane), lane, xf, xl);
        xs[lane] = xf;
        xs[P + lane] = xl;
    } else {
        const int p0 = 2 * lane, p1 = p0 + 1, p2 = p0 + 2;
        const ChunkEqs e0 = load(p0), e1 = load(p1);
        const float aF2 = p2 < P ? eq[3 * P + p2] : 0.f;
        const float cF2 = p2 < P ? eq[4 * P + p2] : 0.f;
        const float dF2 = p2 < P ? eq[5 * P + p2] : 0.f;
        const float A0 = -e0.aL * e0.aF;
        const float B0 = 1.f - e0.aL * e0.cF - e0.cL * e1.aF;
        const float C0 = -e0.cL * e1.cF;
        const float D0 = e0.dL - e0.aL * e0.dF - e0.cL * e1.dF;
        const float A1 = -e1.aL * e1.aF;
        const float B1 = 1.f - e1.aL * e1.cF - e1.cL * aF2;
        const float C1 = -e1.cL * cF2;
        const float D1 = e1.dL - e1.aL * e1.dF - e1.cL * dF2;
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
}

// Phase 3: x_i = d'_i - a'_i x_0 - c'_i x_{M-1} for the interior rows; the
// solution overwrites d.
template <int S, int M>
__device__ __forceinline__ void chunk_solution(const float* c, float* d, const float (&ap)[M], float xfirst,
                                               float xlast)
{
    d[0] = xfirst;
#pragma unroll
    for (int i = 1; i < M - 1; ++i) d[i * S] = d[i * S] - ap[i] * xfirst - c[i * S] * xlast;
    d[(M - 1) * S] = xlast;
}

// ---------------------------------------------------------------- rows ----
// NW warps per row, 128 threads per CTA (4 / NW rows).  Shared memory per
// row: g and L (ls floats each), the chunk equations (6 P), the chunk end
// values (2 P).  Output: u_x to `ux`, or, with acc != nullptr, u_x / 2 added
// into acc (the other half of the step is the column kernel's).
template <int M, int NW>
__global__ void __launch_bounds__(128) k_aos_rows(const float* __restrict__ L, const float* __restrict__ g,
                                                  float* __restrict__ ux, float* __restrict__ acc, int pitch, int w,
                                                  int h, float tau, int* __restrict__ status)
{
    constexpr int P = 32 * NW;
    constexpr int ROWS = 4 / NW;
    constexpr int LS = row_stride_floats(P, M);
    extern __shared__ __align__(128) float sm[];
    __shared__ __align__(8) uint64_t bars[ROWS];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = warp / NW, part = warp - r * NW;
    const int y = blockIdx.x * ROWS + r;
    const bool active = y < h;
    float* sg = sm + (size_t)r * (2 * LS + 8 * P);
    float* sd = sg + LS;
    float* eq = sd + LS;
    float* xs = eq + 6 * P;
    const float* grow = g + (size_t)(active ? y : 0) * pitch;
    const float* lrow = L + (size_t)(active ? y : 0) * pitch;
    const int w4 = w & ~3;

    if (active && part == 0 && lane == 0) mbar_init(&bars[r], 1);
    __syncthreads();
    if (active && part == 0) {
        if (lane == 0) {
            mbar_expect_tx(&bars[r], 2u * 4u * (unsigned)w4);
            if (w4 > 0) {
                bulk_load(sg, grow, 4u * w4, &bars[r]);
                bulk_load(sd, lrow, 4u * w4, &bars[r]);
            }
        }
        for (int x = w4 + lane; x < w; x += 32) {
            sg[x] = __ldg(grow + x);
            sd[x] = __ldg(lrow + x);
        }
    }
    const bool ok = !active || mbar_wait_bounded(&bars[r], 0);
    if (!__syncthreads_and(ok)) {  // same decision in every thread
        if (threadIdx.x == 0) atomicOr(status, 1);
        // the row's copies still in flight land (bounded wait) before the CTA
        // gives up its shared memory
        if (active && part == 0 && lane == 0) mbar_wait_bounded(&bars[r], 0);
        __syncthreads();
        return;
    }

    const int p = part * 32 + lane;
    const int j0 = p * M;
    float* ce = sg + j0;
    float* cd = sd + j0;
    const float g_prev = (j0 > 0 && j0 - 1 < w) ? ce[-1] : 0.f;
    const float g_next = (j0 + M < w) ? ce[M] : 0.f;
    __syncthreads();
    float ap[M];
    if (active) {
        const ChunkEqs q = chunk_reduce<1, M>(ce, cd, g_prev, g_next, j0, w, tau, ap);
        eq[0 * P + p] = q.aL;
        eq[1 * P + p] = q.cL;
        eq[2 * P + p] = q.dL;
        eq[3 * P + p] = q.aF;
        eq[4 * P + p] = q.cF;
        eq[5 * P + p] = q.dF;
    }
    __syncthreads();
    if (active && part == 0) interface_line<NW>(eq, xs, lane);
    __syncthreads();
    if (active) chunk_solution<1, M>(ce, cd, ap, xs[p], xs[P + p]);
    __syncthreads();
    if (!active) return;
    if (acc) {
        // two halves added onto zero in either order give the same sum
        float* arow = acc + (size_t)y * pitch;
        for (int x = p * 4; x < w4; x += 4 * P) {
            float4 v = *reinterpret_cast<const float4*>(sd + x);
            v.x *= 0.5f;
            v.y *= 0.5f;
            v.z *= 0.5f;
            v.w *= 0.5f;
            atomicAdd(reinterpret_cast<float4*>(arow + x), v);
        }
        for (int x = w4 + p; x < w; x += P) atomicAdd(arow + x, 0.5f * sd[x]);
        return;
    }
    float* urow = ux + (size_t)y * pitch;
    for (int x = p * 4; x < w4; x += 4 * P)
        *reinterpret_cast<float4*>(urow + x) = *reinterpret_cast<const float4*>(sd + x);
    for (int x = w4 + p; x < w; x += P) urow[x] = sd[x];
}

// ------------------------------------------------------------- columns ----
// A strip of COLS columns per CTA, P = 32 NW chunks per column, blockDim =
// COLS P; thread t owns column t % COLS and chunk t / COLS.  Shared memory:
// the g and L tiles ([RS][COLS], RS = P M rounded up to whole 256-row boxes)
// and per column the chunk equations (6 P) and end values (2 P).  Output:
// Lnext = (u_x + u_y) / 2 with u_x read from `ux`, or, with ux == nullptr,
// u_y / 2 added into Lnext (the row kernel adds the other half).
template <int COLS, int M, int NW>
__global__ void __launch_bounds__(COLS * 32 * NW)
    k_aos_cols(const __grid_constant__ CUtensorMap tmL, const __grid_constant__ CUtensorMap tmG,
               const float* __restrict__ gsrc, const float* __restrict__ ux, float* __restrict__ Lnext, int pitch,
               int w, int h, float tau, int* __restrict__ status)
{
    constexpr int P = 32 * NW;
    constexpr int NT = COLS * P;
    constexpr int RS = rows_staged(P, M);
    constexpr int V = COLS / 4;                  // float4 per strip row
    constexpr int EPI = (RS * V + NT - 1) / NT;  // epilogue vectors per thread
    constexpr int NB = RS / 256;  // 256-row boxes, one barrier each
    extern __shared__ __align__(128) float sm[];
    __shared__ __align__(8) uint64_t bars[NB];
    const int tid = threadIdx.x;
    const int c = tid % COLS, p = tid / COLS;
    const int x0 = blockIdx.x * COLS;
    float* tg = sm;
    float* td = sm + (size_t)RS * COLS;
    float* eq0 = td + (size_t)RS * COLS;
    float* eqc = eq0 + (size_t)c * 8 * P;  // this column's equations

    __shared__ int s_fail;
    if (tid == 0) {
        s_fail = 0;
#pragma unroll
        for (int b = 0; b < NB; ++b) mbar_init(&bars[b], 1);
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            mbar_expect_tx(&bars[b], 2u * 256u * COLS * 4u);
            tma_load_2d(tg + (size_t)b * 256 * COLS, &tmG, x0, 256 * b, &bars[b]);
            tma_load_2d(td + (size_t)b * 256 * COLS, &tmL, x0, 256 * b, &bars[b]);
        }
    }
    __syncthreads();
    // a chunk starts as soon as the boxes holding its rows (and the row on
    // either side) have landed, while later boxes are still in flight
    const int j0 = p * M;
    bool ok = true;
    {
        const int b_lo = (j0 > 0 ? j0 - 1 : 0) / 256;
        const int b_hi = min(j0 + M, RS - 1) / 256;
        for (int b = b_lo; b <= b_hi && ok; ++b) ok = mbar_wait_bounded(&bars[b], 0);
    }
    if (!__all_sync(FULL, ok)) {  // a wait ran out: every warp still meets the barrier below
        if ((tid & 31) == 0) {
            atomicOr(status, 1);
            s_fail = 1;
        }
    }
    float* ce = tg + (size_t)j0 * COLS + c;
    float* cd = td + (size_t)j0 * COLS + c;
    // the neighbouring chunks' edge conductances come from global memory (L2):
    // their shared copies are overwritten by those chunks' own sweeps, which
    // no block-wide barrier orders against this read
    const int xc = x0 + c;
    const float g_prev = (j0 > 0 && j0 - 1 < h && xc < w) ? __ldg(gsrc + (unsigned)((j0 - 1) * pitch + xc)) : 0.f;
    const float g_next = (j0 + M < h && xc < w) ? __ldg(gsrc + (unsigned)((j0 + M) * pitch + xc)) : 0.f;
    float ap[M];
    const ChunkEqs q = chunk_reduce<COLS, M>(ce, cd, g_prev, g_next, j0, h, tau, ap);
    eqc[0 * P + p] = q.aL;
    eqc[1 * P + p] = q.cL;
    eqc[2 * P + p] = q.dL;
    eqc[3 * P + p] = q.aF;
    eqc[4 * P + p] = q.cF;
    eqc[5 * P + p] = q.dF;

    __syncthreads();
    if (s_fail) {
        // a staging wait ran out (the status is set): the boxes still in
        // flight land (bounded wait) before the CTA gives up its shared memory
        if (tid == 0)
            for (int b = 0; b < NB; ++b) mbar_wait_bounded(&bars[b], 0);
        __syncthreads();
        return;
    }
    const int warp = tid >> 5, lane = tid & 31;
    if (warp < COLS) {  // warp `warp` solves column `warp`
        float* eqw = eq0 + (size_t)warp * 8 * P;
        interface_line<NW>(eqw, eqw + 6 * P, lane);
    }
    __syncthreads();
    chunk_solution<COLS, M>(ce, cd, ap, eqc[6 * P + p], eqc[7 * P + p]);
    __syncthreads();

    const bool full = x0 + COLS <= w;
    if (ux == nullptr) {
        for (int e = tid; e < h * V; e += NT) {
            const int j = e / V, qq = e - j * V;
            const unsigned gi = (unsigned)(j * pitch + x0 + 4 * qq);  // plane offsets fit 32 bits
            const float* uy = td + (size_t)j * COLS + 4 * qq;
            if (full) {
                atomicAdd(reinterpret_cast<float4*>(Lnext + gi),
                          make_float4(0.5f * uy[0], 0.5f * uy[1], 0.5f * uy[2], 0.5f * uy[3]));
            } else {
                for (int kk = 0; kk < 4; ++kk)
                    if (x0 + 4 * qq + kk < w) atomicAdd(Lnext + gi + kk, 0.5f * uy[kk]);
            }
        }
        return;
    }
    // L_next = (u_x + u_y) / 2 over the strip: the 16-byte loads of the row
    // solution are all issued before the stores
    float4 pre[EPI];
#pragma unroll
    for (int k = 0; k < EPI; ++k) {
        const int e = tid + k * NT;
        const int j = e / V, qq = e - j * V;
        pre[k] = (full && j < h)
                     ? __ldg(reinterpret_cast<const float4*>(ux + (size_t)j * pitch + x0 + 4 * qq))
                     : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int k = 0; k < EPI; ++k) {
        const int e = tid + k * NT;
        const int j = e / V, qq = e - j * V;
        if (j >= h) break;
        const size_t gi = (size_t)j * pitch + x0 + 4 * qq;
        const float* uy = td + (size_t)j * COLS + 4 * qq;
        if (full) {
            float4 rr;
            rr.x = 0.5f * (pre[k].x + uy[0]);
            rr.y = 0.5f * (pre[k].y + uy[1]);
            rr.z = 0.5f * (pre[k].z + uy[2]);
            rr.w = 0.5f * (pre[k].w + uy[3]);
            *reinterpret_cast<float4*>(Lnext + gi) = rr;
        } else {
            for (int kk = 0; kk < 4; ++kk)
                if (x0 + 4 * qq + kk < w) Lnext[gi + kk] = 0.5f * (__ldg(ux + gi + kk) + uy[kk]);
        }
    }
}

// ------------------------------------------------------ launch plumbing ----

struct RowsArgs {
    const float* L;
    const float* g;
    float* ux;
    float* acc;
    int pitch, w, h;
    float tau;
    int* status;
    size_t smem;
    cudaStream_t st;
};

struct ColsArgs {
    CUtensorMap mL, mG;
    const float* g;
    const float* ux;
    float* Lnext;
    int pitch, w, h;
    float tau;
    int* status;
    size_t smem;
    int cols;
    cudaStream_t st;
};

template <int M, int NW>
cudaError_t launch_rows_m(const RowsArgs& a)
{
    constexpr int ROWS = 4 / NW;
    k_aos_rows<M, NW><<<(a.h + ROWS - 1) / ROWS, 128, a.smem, a.st>>>(a.L, a.g, a.ux, a.acc, a.pitch, a.w, a.h,
                                                                        a.tau, a.status);
    return cudaGetLastError();
}

template <int M, int NW>
cudaError_t launch_cols_m(const ColsArgs& a)
{
    if (a.cols == 16)
        k_aos_cols<16, M, NW><<<(a.w + 15) / 16, 16 * 32 * NW, a.smem, a.st>>>(a.mL, a.mG, a.g, a.ux, a.Lnext,
                                                                              a.pitch, a.w, a.h, a.tau, a.status);
    else if (a.cols == 8)
        k_aos_cols<8, M, NW><<<(a.w + 7) / 8, 8 * 32 * NW, a.smem, a.st>>>(a.mL, a.mG, a.g, a.ux, a.Lnext,
                                                                           a.pitch, a.w, a.h, a.tau, a.status);
    else
        k_aos_cols<4, M, NW><<<(a.w + 3) / 4, 4 * 32 * NW, a.smem, a.st>>>(a.mL, a.mG, a.g, a.ux, a.Lnext,
                                                                           a.pitch, a.w, a.h, a.tau, a.status);
    return cudaGetLastError();
}

template <int M, int NW>
cudaError_t configure_m()
{
    cudaError_t e = allow_max_dynamic_smem(k_aos_rows<M, NW>);
    if (e == cudaSuccess) e = allow_max_dynamic_smem(k_aos_cols<16, M, NW>);
    if (e == cudaSuccess) e = allow_max_dynamic_smem(k_aos_cols<8, M, NW>);
    if (e == cudaSuccess) e = allow_max_dynamic_smem(k_aos_cols<4, M, NW>);
    return e;
}

// Every (M, NW) variant; X(M, NW) is expanded once per variant.
#define KZ_AOS_VARIANTS_A(X) X(3, 1) X(5, 1) X(7, 1) X(9, 1) X(11, 1) X(13, 1) X(15, 1) X(17, 1)
#define KZ_AOS_VARIANTS_B(X) X(9, 2) X(11, 2) X(13, 2) X(15, 2) X(17, 2) X(19, 2) X(21, 2) X(23, 2)
#define KZ_AOS_VARIANTS_C(X) X(25, 2) X(27, 2) X(29, 2) X(31, 2) X(33, 2) X(37, 2) X(41, 2) X(45, 2)
#define KZ_AOS_VARIANTS_D(X) X(49, 2) X(57, 2) X(65, 2) X(73, 2) X(81, 2) X(97, 2) X(113, 2) X(129, 2)
#define KZ_AOS_VARIANTS(X) KZ_AOS_VARIANTS_A(X) KZ_AOS_VARIANTS_B(X) KZ_AOS_VARIANTS_C(X) KZ_AOS_VARIANTS_D(X)

#define KZ_AOS_DECLARE(M, NW)                                  \
    extern template cudaError_t launch_rows_m<M, NW>(const RowsArgs&); \
    extern template cudaError_t launch_cols_m<M, NW>(const ColsArgs&); \
    extern template cudaError_t configure_m<M, NW>();
#define KZ_AOS_INSTANTIATE(M, NW)                                \
    template cudaError_t launch_rows_m<M, NW>(const RowsArgs&);  \
    template cudaError_t launch_cols_m<M, NW>(const ColsArgs&);  \
    template cudaError_t configure_m<M, NW>();

}  // namespace aos

// 2-D tensor map of a w x h FP32 plane (row pitch in elements) with a
// box_x x box_y box; reads past the plane's edges fill with zeros.
bool make_plane_map(CUtensorMap* map, const float* base, int pitch, int w, int h, int box_x, int box_y);

}  // namespace kz
