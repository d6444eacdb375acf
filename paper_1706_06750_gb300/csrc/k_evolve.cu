// k_evolve.cu -- the whole AOS evolution of Sec. II-A (levels 1..N-1, one
// semi-implicit step of Eq. 4 per level, tau_i = t_i - t_{i-1} of Eq. 7) in
// ONE persistent cooperative launch, with every tile of the image resident in
// shared memory for all N-1 steps.
//
// The image is cut into tiles of TW x TH pixels, one CTA (one SM) per tile.
// A CTA keeps its tile of L (with a HALO-pixel ring) and of the conductance
// g (with a 1-pixel ring) in shared memory.  Per step:
//   1. g = g2(|grad(G_sigma_d * L)|) of Eq. 2-3 on the tile and its ring,
//      from the tile of L: a row-walking horizontal pass into a scratch
//      tile, then column walkers for the vertical pass, the 3x3 Scharr pair
//      (D = S(x+1) - S(x-1), E = 3 S(x-1) + 10 S(x) + 3 S(x+1), neighbours by
//      warp shuffles) and g -- the operations of the line-kernel path, in
//      the same order;
//   2. every row and column of the tile is cut into chunks (8 per segment);
//      each chunk's tridiagonal system, its couplings to the neighbouring
//      chunks removed, is solved (Thomas) for its right-hand side and for
//      the unit vectors at its two ends.  The ends of a chunk's solution
//      then follow as  x = y - V x_left - W x_right  in its two external
//      neighbours ("spike" form, as in the SPIKE algorithm of Polizzi &
//      Sameh 2006);
//   3. adjacent spike records merge into the record of their union (a 2x2
//      solve at the joint); the 8 chunk records of a line segment merge into
//      the segment's record, which goes to global memory;
//   4. grid barrier; each line's thread reads the records of its line from
//      every tile, merges those left and right of its own segment and solves
//      for the segment's two external neighbours, then walks the chunk merges
//      back to every chunk's external neighbours;
//   5. each chunk is solved again with its external terms moved to the
//      right-hand side: rows give u_x (shared memory), columns u_y and
//      L_i = (u_x + u_y) / 2, written to the tile and to the level plane;
//   6. grid barrier; the CTA reads the HALO ring of L_i from the level plane.
// Borders: the lines have Neumann ends (no coupling past the image), every
// stencil reflects coordinates into the image (half-sample symmetric).  Line
// elements past the image inside a ragged tile are identity rows.
//
// Shared memory is laid out with odd row strides: the row solves give a lane
// a row (lanes 32 rows apart in bank terms), the column solves a column.
// Every grid-barrier wait is bounded; a timeout (or another CTA's) sets bit 0
// of *status and the CTA returns.
#include "kaze_internal.h"

namespace kz {
namespace ev {

constexpr int TW = 128, TH = 120;  // tile
constexpr int RMAX = 3;            // radius of G(sigma_d) this kernel takes
constexpr int HALO = RMAX + 2;     // L ring: smoothing, Scharr, g ring
constexpr int NT = 512, NWARP = NT / 32;
constexpr int MR = 16, KR = TW / MR;  // row chunks: 8 of 16 elements
constexpr int MC = 15, KC = TH / MC;  // column chunks: 8 of 15 elements
constexpr int TMAX = 16;              // tiles along a line

constexpr int LROWS = TH + 2 * HALO, LCOLS = TW + 2 * HALO, LS = LCOLS + 1;  // 130 x 138, stride 139
constexpr int GROWS = TH + 2, GCOLS = TW + 2, GS = GCOLS + 1;                  // 122 x 130, stride 131
constexpr int HROWS = LROWS, HCOLS = TW + 4, HS = HCOLS + 1;                   // 130 x 132, stride 133
constexpr int US = TW + 1;                                                     // u_x, stride 129
constexpr int REC = 6;
constexpr int RREC = KR * REC * TH;  // row chunk records [k][f][r]
constexpr int CREC = KC * REC * TW;  // column chunk records [k][f][c]
constexpr int SROWS = TH + 4, SCOLS = TW + 4, SS = SCOLS + 1;  // smoothed S: 124 x 132, stride 133
constexpr int cmax(int a, int b) { return a > b ? a : b; }
// Shared memory: LH | A | XE | B.  During the conductance pass B holds the
// horizontal pass H, A the smoothed S, and g is written into B (H is dead by
// then); the line solves then use A for the chunk records, the staged
// segment records (which also reach into XE) and u_x.
constexpr int OFF_L = 0;
constexpr int OFF_A = (OFF_L + LROWS * LS + 3) & ~3;
constexpr int A_SIZE = cmax(cmax(SROWS * SS, TH * US), RREC + CREC);
constexpr int OFF_X = OFF_A + A_SIZE;
constexpr int X_SIZE = KR * 2 * TH + KC * 2 * TW;  // chunk externals
constexpr int OFF_B = OFF_X + X_SIZE;
constexpr int B_SIZE = cmax(HROWS * HS, GROWS * GS);
constexpr int SMEM_FLOATS = OFF_B + B_SIZE;
constexpr size_t SMEM_BYTES = (size_t)SMEM_FLOATS * sizeof(float);
static_assert((OFF_A * 4) % 16 == 0, "the staging copies land on a 16-byte boundary");
// Presmoothing inside the launch (radius R0MAX): the input tile over LH and A,
// the row pass over XE and B.
constexpr int R0MAX = 5;
constexpr int IS = TW + 2 * (HALO + R0MAX) + 1;  // staged input, stride 149
constexpr int PS = LCOLS + 1;                     // row pass, stride 139
constexpr int OFF_I = OFF_L, OFF_P = OFF_X;
static_assert((TH + 2 * (HALO + R0MAX)) * IS <= OFF_X, "the staged input fits LH and A");
static_assert(OFF_P + (TH + 2 * (HALO + R0MAX)) * PS <= SMEM_FLOATS, "the row pass fits XE and B");
static_assert(SMEM_BYTES <= 227 * 1024, "tile state must fit one SM's shared memory");

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

__device__ __forceinline__ int ld_relaxed(const int* p)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned smem_u32(const void* q) { return (unsigned)__cvta_generic_to_shared(q); }

__device__ __forceinline__ void mbar_init(uint64_t* bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// One bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned)
// from global to shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Waits for phase `parity` of `bar`, giving up after `limit` cycles.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, long long limit)
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
        if (clock64() - t0 > limit) return false;
    }
}

// Spike record of a block of consecutive line elements: its first and last
// unknowns as  x = y - V x_left - W x_right  in the block's two external
// neighbours.
struct Rec {
    float yF, VF, WF, yL, VL, WL;
};
// One unknown in the same form.
struct Pt {
    float y, V, W;
};

// Union of adjacent blocks A (left) and B (right).  P and Q receive A's last
// and B's first unknowns in terms of the union's external neighbours.
__device__ __forceinline__ Rec merge(const Rec& A, const Rec& B, Pt& P, Pt& Q)
{
    // the joint: xA_l + WA_l xB_f = yA_l - VA_l xl,  VB_f xA_l + xB_f = yB_f - WB_f xr
    const float s = rcp_approx(fmaf(-A.WL, B.VF, 1.f));
    P.y = s * fmaf(-A.WL, B.yF, A.yL);
    P.V = s * A.VL;
    P.W = -s * (A.WL * B.WF);
    Q.y = s * fmaf(-B.VF, A.yL, B.yF);
    Q.V = -s * (B.VF * A.VL);
    Q.W = s * B.WF;
    Rec M;
    M.yF = fmaf(-A.WF, Q.y, A.yF);
    M.VF = fmaf(-A.WF, Q.V, A.VF);
    M.WF = -(A.WF * Q.W);
    M.yL = fmaf(-B.VL, P.y, B.yL);
    M.VL = -(B.VL * P.V);
    M.WL = fmaf(-B.VL, P.W, B.WL);
    return M;
}

__device__ __forceinline__ Rec merge(const Rec& A, const Rec& B)
{
    Pt P, Q;
    return merge(A, B, P, Q);
}

__device__ __forceinline__ float eval(const Pt& p, float xl, float xr) { return p.y - p.V * xl - p.W * xr; }

// One chunk of M consecutive elements of a line (Eq. 4 with the AOS
// splitting): c_i = -tau (g_i + g_i+1) couples element i to i+1, a_i = c_i-1,
// b_i = 1 - a_i - c_i.  The conductance past the image holds ghost values
// (+-g of the last pixel, alternating) that make every coupling across the
// image border exactly zero, so elements past the border are decoupled rows
// and the chunk needs no masks.
template <int M>
struct Chunk {
    // d[i * ds]: right-hand side, g[i * gs]: conductance (g[-gs], g[M * gs]:
    // the neighbours' values)
    const float* d;
    const float* g;
    int ds, gs;
    float tau;

    // Thomas on the chunk with its couplings a_0, c_M-1 removed, for the
    // right-hand side d (dl, dr subtracted at the first / last element) and,
    // if wanted, for e_0.
    template <bool WANT_V>
    __device__ __forceinline__ void factor(float (&q)[M], float (&dy)[M], float (&dv)[M], float dl, float dr,
                                           float& a0, float& clast, float& rlast) const
    {
        float gc = g[0];
        a0 = -tau * (g[-gs] + gc);
        float a = a0;
#pragma unroll
        for (int i = 0; i < M; ++i) {
            const float gn = g[(i + 1) * gs];
            const float c = -tau * (gc + gn);
            const float b = 1.f - a - c;
            float di = d[i * ds];
            if (i == 0) di -= dl;
            if (i == M - 1) {
                di -= dr;
                clast = c;
            }
            float r;
            if (i == 0) {
                r = rcp_approx(b);
                dy[0] = di * r;
                if (WANT_V) dv[0] = r;
            } else {
                r = rcp_approx(fmaf(-a, q[i - 1], b));
                dy[i] = fmaf(-a, dy[i - 1], di) * r;
                if (WANT_V) dv[i] = -a * dv[i - 1] * r;
            }
            q[i] = c * r;
            if (i == M - 1) rlast = r;
            a = c;
            gc = gn;
        }
    }

    // The chunk's spike record.
    __device__ __forceinline__ Rec record() const
    {
        float q[M], dy[M], dv[M];
        float a0, cl, rl;
        factor<true>(q, dy, dv, 0.f, 0.f, a0, cl, rl);
        float y = dy[M - 1], v = dv[M - 1];
#pragma unroll
        for (int i = M - 2; i >= 0; --i) {
            y = fmaf(-q[i], y, dy[i]);
            v = fmaf(-q[i], v, dv[i]);
        }
        // (A^-1)_{0,M-1} = (A^-1)_{M-1,0} = dv[M-1]: the chunk matrix is symmetric
        Rec R;
        R.yF = y;
        R.VF = a0 * v;
        R.WF = cl * dv[M - 1];
        R.yL = dy[M - 1];
        R.VL = a0 * dv[M - 1];
        R.WL = cl * rl;
        return R;
    }

    // The chunk's solution given its external neighbours; x[i] receives
    // element i.
    __device__ __forceinline__ void solve(float xl, float xr, float (&x)[M]) const
    {
        float q[M], dv[M];
        float a0, cl, rl;
        // the external terms a_0 xl and c_M-1 xr move to the right-hand side
        const float a0v = -tau * (g[-gs] + g[0]);
        const float clv = -tau * (g[(M - 1) * gs] + g[M * gs]);
        factor<false>(q, x, dv, a0v * xl, clv * xr, a0, cl, rl);
#pragma unroll
        for (int i = M - 2; i >= 0; --i) x[i] = fmaf(-q[i], x[i + 1], x[i]);
    }
};

struct Params {
    float* levels;    // N planes of pitch * h floats, plane stride `plane`
    long long plane;
    int pitch, w, h, n_levels;
    int tiles_x, tiles_y;
    float* d_k;  // contrast factor (read, or written when computed here)
    float wt[RMAX + 1];  // G(sigma_d) taps for offsets 0..RMAX (0 past the radius)
    int diffusivity;
    float tau[kMaxLevels];
    float* xrow;  // row segment records [y][tiles_x][6]
    float* xcol;  // column segment records [x][tiles_y][6] (16-byte aligned)
    unsigned int* barrier;
    int* status;
    // presmoothing inside the launch (img != null): the input image and the
    // Gaussian taps w[0 .. 2 r0] of offsets -r0 .. r0; level 0 is written here
    const float* img;
    int img_pitch, r0;
    float pw[2 * R0MAX + 1];
    // contrast factor inside the launch (hist != null): maximum and histogram
    // of the interior gradient magnitudes of step 1, percentile; k to d_k
    unsigned int* hmax_bits;
    unsigned int* hist;
    int nbins;
    double pct;
    float k_fixed;         // > 0: the contrast factor (hist null), also written to d_k
    long long wait_limit;  // SM cycles a grid-barrier wait may take
    int stall_tile;        // test hook: this tile never arrives (-1: none)
};

// Grid-wide barrier in two halves: every CTA arrives once per barrier, and
// `target` is the count once every CTA has arrived.  The wait is bounded: on
// timeout, or when another CTA has already flagged one, it sets bit 0 of
// *status and returns false.
__device__ __forceinline__ void grid_arrive(const Params& p, int tile)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (tile != p.stall_tile) atomicAdd(p.barrier, 1u);
    }
}

__device__ __forceinline__ bool grid_wait(const Params& p, unsigned target, volatile int* s_abort)
{
    if (threadIdx.x == 0) {
        const long long t0 = clock64();
        while (ld_acquire(p.barrier) < target) {
            if (ld_relaxed(p.status) != 0 || clock64() - t0 > p.wait_limit) {
                atomicOr(p.status, 1);
                *s_abort = 1;
                break;
            }
        }
    }
    __syncthreads();
    return *s_abort == 0;
}

__device__ __forceinline__ bool grid_barrier(const Params& p, int tile, unsigned target, volatile int* s_abort)
{
    grid_arrive(p, tile);
    return grid_wait(p, target, s_abort);
}

// Asynchronous 4-byte copy from global to shared memory (cp.async); a
// cp_async_wait_all makes this thread's copies complete.
__device__ __forceinline__ void cp_async4(float* dst, const float* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// Copies n elements from global to shared memory: element e goes from
// src(e) to dst(e).  Loads are issued in batches of B before their stores
// (the cache-global loads are ordered asm statements).
template <int B, typename Src, typename Dst>
__device__ __forceinline__ void copy_batched(int n, Src src, Dst dst)
{
    for (int e0 = threadIdx.x; e0 < n; e0 += B * NT) {
        float v[B];
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const int e = e0 + b * NT;
            v[b] = e < n ? __ldcg(src(e)) : 0.f;
        }
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const int e = e0 + b * NT;
            if (e < n) *dst(e) = v[b];
        }
    }
}

// Every LH position (r, c), r in [-HALO, TH + HALO), c in [-HALO, TW + HALO),
// from plane `src` at the reflected image position.
__device__ __forceinline__ void load_all(float* LH, const float* src, const Params& p, int x0, int y0)
{
    copy_batched<8>(
        LROWS * LCOLS,
        [&](int e) {
            const int rr = e / LCOLS, cc = e - rr * LCOLS;
            return src + (size_t)reflect_index(y0 + rr - HALO, p.h) * p.pitch + reflect_index(x0 + cc - HALO, p.w);
        },
        [&](int e) {
            const int rr = e / LCOLS, cc = e - rr * LCOLS;
            return LH + rr * LS + cc;
        });
}

// The LH positions outside the tile's own image pixels [0, th) x [0, tw):
// the bands above and below (whole width, a warp per row, lanes along it),
// then left and right of them.  A full tile's side bands are HALO columns
// each (element e: row e / 10, a compile-time division); a ragged tile's
// right band is wider and takes the general enumeration.
__device__ __forceinline__ void load_halo(float* LH, const float* src, const Params& p, int x0, int y0, int tw,
                                          int th)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nb = TH + HALO - th;  // rows below
    const int wr = TW + HALO - tw;  // columns right of the image part
    auto col = [&](int cc) { return reflect_index(x0 + cc - HALO, p.w); };
    constexpr int NCI = (LCOLS + 31) / 32;
    for (int q = warp; q < HALO + nb; q += NWARP) {
        const int rr = q < HALO ? q : th + HALO + (q - HALO);
        const float* srow = src + (size_t)reflect_index(y0 + rr - HALO, p.h) * p.pitch;
        float v[NCI];
#pragma unroll
        for (int i = 0; i < NCI; ++i) {
            const int cc = lane + 32 * i;
            v[i] = cc < LCOLS ? __ldcg(srow + col(cc)) : 0.f;
        }
#pragma unroll
        for (int i = 0; i < NCI; ++i) {
            const int cc = lane + 32 * i;
            if (cc < LCOLS) LH[rr * LS + cc] = v[i];
        }
    }
    const int nside = HALO + wr;
    if (nside == 2 * HALO) {
        copy_batched<4>(
            th * 2 * HALO,
            [&](int e) {
                const int r = e / (2 * HALO), q = e - r * (2 * HALO);
                const int cc = q < HALO ? q : tw + q;
                return src + (size_t)(y0 + r) * p.pitch + col(cc);
            },
            [&](int e) {
                const int r = e / (2 * HALO), q = e - r * (2 * HALO);
                const int cc = q < HALO ? q : tw + q;
                return LH + (r + HALO) * LS + cc;
            });
    } else {
        copy_batched<4>(
            th * nside,
            [&](int e) {
                const int r = e / nside, q = e - r * nside;
                const int cc = q < HALO ? q : tw + HALO + (q - HALO);
                return src + (size_t)(y0 + r) * p.pitch + col(cc);
            },
            [&](int e) {
                const int r = e / nside, q = e - r * nside;
                const int cc = q < HALO ? q : tw + HALO + (q - HALO);
                return LH + (r + HALO) * LS + cc;
            });
    }
}

// Ghost conductance past the image (see Chunk): along rows, columns
// x >= w take (-1)^(x - w + 1) g(w - 1) and x = -1 takes -g(0); along
// columns the same with y.  Runs after the conductance pass; the two
// directions in turn (their writes meet only at unused corners).
__device__ __forceinline__ void ghost_conductance(float* G, int x0, int y0, int w, int h)
{
    const int cw = w - x0, rh = h - y0;  // first tile column / row past the image
    if (x0 == 0)
        for (int rr = threadIdx.x; rr < GROWS; rr += NT) G[rr * GS] = -G[rr * GS + 1];
    if (cw <= TW) {
        const int nc = TW + 1 - cw;  // ghost columns cw .. TW (index c + 1)
        for (int e = threadIdx.x; e < GROWS * nc; e += NT) {
            const int rr = e / nc, c = cw + (e - rr * nc);
            float* row = G + rr * GS;
            row[c + 1] = ((c - cw) & 1) ? row[cw] : -row[cw];  // row[cw]: column cw - 1
        }
    }
    __syncthreads();
    if (y0 == 0)
        for (int cc = threadIdx.x; cc < GCOLS; cc += NT) G[cc] = -G[GS + cc];
    if (rh <= TH) {
        const int nr = TH + 1 - rh;  // ghost rows rh .. TH (index r + 1)
        for (int e = threadIdx.x; e < nr * GCOLS; e += NT) {
            const int q = e / GCOLS, cc = e - q * GCOLS, r = rh + q;
            G[(r + 1) * GS + cc] = ((r - rh) & 1) ? G[rh * GS + cc] : -G[rh * GS + cc];
        }
    }
}

// g of Eq. 2-3 on tile rows -1..TH, columns -1..TW (into G) from LH in three
// passes, each thread taking two lines half the tile apart with packed FP32x2
// arithmetic (each half rounds exactly as the scalar operation, so the
// results are those of the line-kernel path bit for bit): the horizontal
// Gaussian pass H(r, c) = sum_j w_j L(r, c + j), r in [-HALO, TH + HALO),
// c in [-2, TW + 2), by threads walking 22 columns of rows r and r + 65
// (lanes: consecutive rows) ...
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

__device__ __forceinline__ void h_pass(const float* __restrict__ LH, float* __restrict__ H, const Params& p)
{
    const float2 w0 = f2(p.wt[0], p.wt[0]), w1 = f2(p.wt[1], p.wt[1]), w2 = f2(p.wt[2], p.wt[2]),
                 w3 = f2(p.wt[3], p.wt[3]);
    constexpr int HALF = HROWS / 2, SEG = HCOLS / 6;
    static_assert(HALF * 2 == HROWS && SEG * 6 == HCOLS && HALF * 6 <= NT, "two rows, six segments, one job a thread");
    const int job = threadIdx.x;
    if (job >= HALF * 6) return;
    const int s = job / HALF, rr = job - s * HALF;
    const int cb = -2 + SEG * s;
    const float* a = LH + rr * LS + (cb + HALO);
    const float* b = a + HALF * LS;
    float* da = H + rr * HS + (cb + 2);
    float* db = da + HALF * HS;
    float2 v0 = f2(a[-3], b[-3]), v1 = f2(a[-2], b[-2]), v2 = f2(a[-1], b[-1]), v3 = f2(a[0], b[0]),
           v4 = f2(a[1], b[1]), v5 = f2(a[2], b[2]);
#pragma unroll 2
    for (int q = 0; q < SEG; ++q) {
        const float2 v6 = f2(a[q + 3], b[q + 3]);
        float2 hv = __fmul2_rn(w0, v3);
        hv = __ffma2_rn(w1, __fadd2_rn(v2, v4), hv);
        hv = __ffma2_rn(w2, __fadd2_rn(v1, v5), hv);
        hv = __ffma2_rn(w3, __fadd2_rn(v0, v6), hv);
        da[q] = hv.x;
        db[q] = hv.y;
        v0 = v1;
        v1 = v2;
        v2 = v3;
        v3 = v4;
        v4 = v5;
        v5 = v6;
    }
}

// ... then the vertical pass S, r in [-2, TH + 2), c in [-2, TW + 2), by
// threads walking 21 rows of columns c and c + 66 with the 7 H values of
// each in registers (lanes: consecutive columns) ...
__device__ __forceinline__ void v_pass(const float* __restrict__ H, float* __restrict__ S, const Params& p)
{
    const float2 w0 = f2(p.wt[0], p.wt[0]), w1 = f2(p.wt[1], p.wt[1]), w2 = f2(p.wt[2], p.wt[2]),
                 w3 = f2(p.wt[3], p.wt[3]);
    constexpr int HALF = SCOLS / 2, RG = (SROWS + 5) / 6;  // 66 column pairs, 21 rows a job
    static_assert(HALF * 2 == SCOLS && HALF * 6 <= NT, "two columns, six segments, one job a thread");
    const int job = threadIdx.x;
    if (job >= HALF * 6) return;
    const int q = job / HALF, c = job - q * HALF;  // c: column + 2
    const int r0 = q * RG, r1 = min(r0 + RG, SROWS);  // S rows r0 - 2 .. r1 - 3
    // S row index i needs H row indices i .. i + 6
    const float* ha = H + c;
    const float* hb = ha + HALF;
    auto ld = [&](int i) { return f2(ha[i * HS], hb[i * HS]); };
    float2 h0 = ld(r0), h1 = ld(r0 + 1), h2 = ld(r0 + 2), h3 = ld(r0 + 3), h4 = ld(r0 + 4), h5 = ld(r0 + 5);
    float* oa = S + c;
    float* ob = oa + HALF;
#pragma unroll 2
    for (int i = r0; i < r1; ++i) {
        const float2 h6 = ld(i + 6);
        float2 sv = __fmul2_rn(w0, h3);
        sv = __ffma2_rn(w1, __fadd2_rn(h2, h4), sv);
        sv = __ffma2_rn(w2, __fadd2_rn(h1, h5), sv);
        sv = __ffma2_rn(w3, __fadd2_rn(h0, h6), sv);
        oa[i * SS] = sv.x;
        ob[i * SS] = sv.y;
        h0 = h1;
        h1 = h2;
        h2 = h3;
        h3 = h4;
        h4 = h5;
        h5 = h6;
    }
}

// ... and the 3x3 Scharr pair and g (Eq. 3) at rows -1..TH, columns -1..TW:
// a thread walks 21 rows of columns c and c + 65 with the D, E values of the
// rows above in registers (the operations of the line-kernel path, in
// order; b - a as b + (-a), the same rounding).  MODE_G2 / MODE_G1 write g of
// Eq. 3; MODE_M2 writes |grad|^2 and returns this thread's maximum of |grad|
// over the tile's own interior image pixels (the contrast factor's maximum
// pass).
enum { MODE_G2 = 0, MODE_G1 = 1, MODE_M2 = 2 };

template <int MODE>
__device__ __forceinline__ float scharr_pass(const float* __restrict__ S, float* __restrict__ G, float inv_k2, int x0,
                                             int y0, int tw, int th, int w, int h)
{
    constexpr int HALF = GCOLS / 2, RG = (GROWS + 5) / 6;  // 65 column pairs, 21 rows a job
    static_assert(HALF * 2 == GCOLS && HALF * 6 <= NT, "two columns, six segments, one job a thread");
    float mx = 0.f;
    const int job = threadIdx.x;
    if (job >= HALF * 6) return mx;
    const int q = job / HALF, cc = job - q * HALF;  // cc: column + 1
    const int r0 = q * RG, r1 = min(r0 + RG, GROWS);  // g rows r0 - 1 .. r1 - 2
    // g row gr (index gr + 1) uses S rows gr - 1 .. gr + 1 (index gr + 1 .. gr + 3)
    const float* sa = S + cc;  // S column (cc - 1) - 1 + 2 = cc: the left neighbour
    const float* sb = sa + HALF;
    const float2 c10 = f2(10.f, 10.f), c3 = f2(3.f, 3.f), c32 = f2(1.f / 32.f, 1.f / 32.f);
    auto de = [&](int si, float2& d, float2& e) {
        const float2 sl = f2(sa[si * SS], sb[si * SS]), sv = f2(sa[si * SS + 1], sb[si * SS + 1]),
                     sr = f2(sa[si * SS + 2], sb[si * SS + 2]);
        d = __fadd2_rn(sr, f2(-sl.x, -sl.y));
        e = __ffma2_rn(c10, sv, __fmul2_rn(c3, __fadd2_rn(sl, sr)));
    };
    float2 dm, em, d0, e0;
    de(r0, dm, em);
    de(r0 + 1, d0, e0);
    float* oa = G + cc;
    float* ob = oa + HALF;
    // interior image pixels of the tile's own columns, if any (MODE_M2)
    const int gca = cc - 1, gcb = cc - 1 + HALF;
    const bool in_a = gca >= 0 && gca < tw && x0 + gca >= 1 && x0 + gca <= w - 2;
    const bool in_b = gcb >= 0 && gcb < tw && x0 + gcb >= 1 && x0 + gcb <= w - 2;
    const int ilo = max(1 - y0, 0) + 1, ihi = min(h - 2 - y0, th - 1) + 1;  // g row index range
#pragma unroll 2
    for (int i = r0; i < r1; ++i) {
        float2 dp, ep;
        de(i + 2, dp, ep);
        const float2 lx = __fmul2_rn(__ffma2_rn(c10, d0, __fmul2_rn(c3, __fadd2_rn(dm, dp))), c32);
        const float2 ly = __fmul2_rn(__fadd2_rn(ep, f2(-em.x, -em.y)), c32);
        const float2 m2 = __ffma2_rn(ly, ly, __fmul2_rn(lx, lx));
        if (MODE == MODE_M2) {
            oa[i * GS] = m2.x;
            ob[i * GS] = m2.y;
            if (i >= ilo && i <= ihi) {
                if (in_a) mx = fmaxf(mx, sqrtf(m2.x));
                if (in_b) mx = fmaxf(mx, sqrtf(m2.y));
            }
        } else if (MODE == MODE_G1) {
            oa[i * GS] = expf(-(m2.x * inv_k2));
            ob[i * GS] = expf(-(m2.y * inv_k2));
        } else {
            oa[i * GS] = __fdividef(1.f, fmaf(m2.x, inv_k2, 1.f));
            ob[i * GS] = __fdividef(1.f, fmaf(m2.y, inv_k2, 1.f));
        }
        dm = d0;
        d0 = dp;
        em = e0;
        e0 = ep;
    }
    return mx;
}

// The Gaussian presmoothing of Sec. III-1 of the input image on the tile and
// its HALO ring into LH, the operations of the presmoothing kernel in order
// (rows first, taps accumulated left to right from zero, reflected input):
// the input tile with an R0 + HALO ring is staged in shared memory (over LH
// and A), the row pass goes into P (over XE and B) by threads walking 46
// columns of one row, then the column pass into LH by threads walking 44 rows
// of one column, each with the 11 inputs in registers.  Positions outside the
// image then take the value of their reflection (the half-sample symmetric
// extension of L_0), and the tile's own pixels go to the level plane.
__device__ __forceinline__ void presmooth_tile(float* __restrict__ sm, const Params& p, int x0, int y0, int tw,
                                               int th, float* __restrict__ L0)
{
    constexpr int R0 = R0MAX, IR = TH + 2 * (HALO + R0), IC = TW + 2 * (HALO + R0);
    float* I = sm + OFF_I;
    float* P = sm + OFF_P;
    float* LH = sm + OFF_L;
    // every copy in flight at once: one round trip to memory
    for (int rr = threadIdx.x >> 5; rr < IR; rr += NWARP) {
        const float* in = p.img + (size_t)reflect_index(y0 + rr - HALO - R0, p.h) * p.img_pitch;
        for (int cc = threadIdx.x & 31; cc < IC; cc += 32)
            cp_async4(I + rr * IS + cc, in + reflect_index(x0 + cc - HALO - R0, p.w));
    }
    cp_async_wait_all();
    __syncthreads();
    float wj[2 * R0 + 1];
#pragma unroll
    for (int j = 0; j <= 2 * R0; ++j) wj[j] = p.pw[j];
    // row pass: P(r, c) for rows -HALO - R0 .. TH + HALO + R0 - 1, columns
    // -HALO .. TW + HALO - 1 (three walks of 46 columns a row, unrolled: the
    // window shifts by register renaming)
    static_assert(3 * 46 == LCOLS && 3 * 44 >= LROWS, "walk lengths");
    for (int job = threadIdx.x; job < IR * 3; job += NT) {
        const int sg = job / IR, rr = job - sg * IR;
        const float* in = I + rr * IS + 46 * sg;  // P column c reads staged columns c .. c + 2 R0
        float* dst = P + rr * PS + 46 * sg;
        float v[46 + 2 * R0];
#pragma unroll
        for (int j = 0; j < 46 + 2 * R0; ++j) v[j] = in[j];
#pragma unroll
        for (int c = 0; c < 46; ++c) {
            float acc = 0.f;
#pragma unroll
            for (int j = 0; j <= 2 * R0; ++j) acc = fmaf(wj[j], v[c + j], acc);
            dst[c] = acc;
        }
    }
    __syncthreads();
    // column pass: L_0(r, c) for rows -HALO .. TH + HALO - 1 into LH (over the
    // dead input tile), three walks of up to 44 rows a column
    for (int job = threadIdx.x; job < LCOLS * 3; job += NT) {
        const int sg = job / LCOLS, cc = job - sg * LCOLS;
        const int rb = 44 * sg, n = min(44, LROWS - rb);  // LH row index; P row index + j
        const float* col = P + rb * PS + cc;
        float v[2 * R0 + 1];
#pragma unroll
        for (int j = 0; j < 2 * R0; ++j) v[j + 1] = col[j * PS];
#pragma unroll
        for (int r = 0; r < 44; ++r) {
            if (r < n) {
#pragma unroll
                for (int j = 0; j < 2 * R0; ++j) v[j] = v[j + 1];
                v[2 * R0] = col[(r + 2 * R0) * PS];
                float acc = 0.f;
#pragma unroll
                for (int j = 0; j <= 2 * R0; ++j) acc = fmaf(wj[j], v[j], acc);
                LH[(rb + r) * LS + cc] = acc;
            }
        }
    }
    __syncthreads();
    // the reflected extension past the image, from positions inside it.
    // Every position the stencils of image pixels reach lies within four
    // pixels of the border and reflects into this tile's window; positions
    // farther out (deep in a ragged tile) only feed ghost conductances and
    // decoupled line elements, and take 0 when their reflection falls
    // outside the window (any finite value serves).  Positions past the image
    // lie in the rows above -y0 and from h - y0 on, and in the columns left
    // of -x0 and from w - x0 on.
    const int rin0 = max(0, HALO - y0), rin1 = min(LROWS, p.h - y0 + HALO);  // LH rows inside the image
    const int cin0 = max(0, HALO - x0), cin1 = min(LCOLS, p.w - x0 + HALO);
    auto fill = [&](int rr, int cc) {
        const int sy = reflect_index(y0 + rr - HALO, p.h) - y0 + HALO;
        const int sx = reflect_index(x0 + cc - HALO, p.w) - x0 + HALO;
        LH[rr * LS + cc] = (sy >= 0 && sy < LROWS && sx >= 0 && sx < LCOLS) ? LH[sy * LS + sx] : 0.f;
    };
    const int nout_r = rin0 + (LROWS - rin1);  // whole rows outside
    for (int e = threadIdx.x; e < nout_r * LCOLS; e += NT) {
        const int q = e / LCOLS, cc = e - q * LCOLS;
        fill(q < rin0 ? q : rin1 + (q - rin0), cc);
    }
    const int nout_c = cin0 + (LCOLS - cin1);  // columns outside, on the rows inside
    for (int e = threadIdx.x; e < (rin1 - rin0) * nout_c; e += NT) {
        const int r = rin0 + e / nout_c, q = e % nout_c;
        fill(r, q < cin0 ? q : cin1 + (q - cin0));
    }
    // own pixels to the level plane
    for (int e = threadIdx.x; e < th * tw; e += NT) {
        const int r = e / tw, c = e - r * tw;
        L0[(size_t)(y0 + r) * p.pitch + x0 + c] = LH[(r + HALO) * LS + (c + HALO)];
    }
}

// g of Eq. 3 in place from |grad|^2 on the tile and its ring.
template <bool G1>
__device__ __forceinline__ void g_from_m2(float* G, float inv_k2)
{
    for (int rr = threadIdx.x >> 5; rr < GROWS; rr += NWARP)
        for (int cc = threadIdx.x & 31; cc < GCOLS; cc += 32) {
            float* q = G + rr * GS + cc;
            const float m2 = *q;
            *q = G1 ? expf(-(m2 * inv_k2)) : __fdividef(1.f, fmaf(m2, inv_k2, 1.f));
        }
}

__device__ __forceinline__ Rec load_rec(const float* s, int st)
{
    return Rec{s[0 * st], s[1 * st], s[2 * st], s[3 * st], s[4 * st], s[5 * st]};
}

__device__ __forceinline__ void store_rec(float* d, int st, const Rec& R)
{
    d[0 * st] = R.yF;
    d[1 * st] = R.VF;
    d[2 * st] = R.WF;
    d[3 * st] = R.yL;
    d[4 * st] = R.VL;
    d[5 * st] = R.WL;
}

// ------------------------------------------------ the phases of a tile's step
// (shared by the resident launch and the streamed passes)

// 2. Every line of the tile cut into chunks, each chunk's spike record into
// RRc (rows, [k][f][r]) and CRc (columns, [k][f][c]); warp jobs of 32 lines
// and one chunk.
__device__ __forceinline__ void chunk_records(const float* __restrict__ LH, const float* __restrict__ G,
                                              float* __restrict__ RRc, float* __restrict__ CRc, int tw, int th,
                                              float tau)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int job = warp; job < 4 * KR + 4 * KC; job += NWARP) {
        if (job < 4 * KR) {
            const int r = (job / KR) * 32 + lane, k = job % KR;
            if (r < th) {
                const Chunk<MR> ch{LH + (r + HALO) * LS + (k * MR + HALO), G + (r + 1) * GS + (k * MR + 1), 1, 1,
                                   tau};
                store_rec(RRc + (k * REC) * TH + r, TH, ch.record());
            }
        } else {
            const int jb = job - 4 * KR;
            const int c = (jb / KC) * 32 + lane, k = jb % KC;
            if (c < tw) {
                const Chunk<MC> ch{LH + (k * MC + HALO) * LS + (c + HALO), G + (k * MC + 1) * GS + (c + 1), LS, GS,
                                   tau};
                store_rec(CRc + (k * REC) * TW + c, TW, ch.record());
            }
        }
    }
}

// 3. The segment record of the thread's line (row li, or column li) from its
// 8 chunk records; the joints of the merges go to P, Q.
__device__ __forceinline__ Rec segment_record(const float* __restrict__ RRc, const float* __restrict__ CRc,
                                              bool row_line, int li, Pt (&P)[8], Pt (&Q)[8])
{
    const float* src = row_line ? RRc + li : CRc + li;
    const int st = row_line ? TH : TW;
    Rec S = load_rec(src, st);
#pragma unroll
    for (int k = 1; k < 8; ++k) S = merge(S, load_rec(src + k * REC * st, st), P[k], Q[k]);
    return S;
}

// Every chunk's external neighbours from the segment's (xl, xr), walking the
// joints back from the segment's right end, into XR / XC ([k][2][line]).
__device__ __forceinline__ void chunk_externals(float* __restrict__ XR, float* __restrict__ XC, bool row_line, int li,
                                                const Pt (&P)[8], const Pt (&Q)[8], float xl, float xr)
{
    float* xe = row_line ? XR + li : XC + li;
    const int st = row_line ? TH : TW;
    float right = xr;
#pragma unroll
    for (int k = 7; k >= 1; --k) {
        const float first_k = eval(Q[k], xl, right);
        xe[(k * 2 + 0) * st] = eval(P[k], xl, right);
        xe[(k * 2 + 1) * st] = right;
        right = first_k;
    }
    xe[0] = xl;
    xe[st] = right;
}

// 5. The chunks solved again with their external terms on the right-hand
// side: rows give u_x (U), columns u_y and L = (u_x + u_y) / 2, into the tile
// and the level plane.
__device__ __forceinline__ void resolve_tile(float* __restrict__ LH, const float* __restrict__ G, float* __restrict__ U,
                                             const float* __restrict__ XR, const float* __restrict__ XC,
                                             float* __restrict__ Lout, int pitch, int x0, int y0, int tw, int th,
                                             float tau)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int job = warp; job < 4 * KR; job += NWARP) {
        const int r = (job / KR) * 32 + lane, k = job % KR;
        if (r < th) {
            const Chunk<MR> ch{LH + (r + HALO) * LS + (k * MR + HALO), G + (r + 1) * GS + (k * MR + 1), 1, 1, tau};
            float x[MR];
            ch.solve(XR[(k * 2 + 0) * TH + r], XR[(k * 2 + 1) * TH + r], x);
            float* u = U + r * US + k * MR;
#pragma unroll
            for (int i = 0; i < MR; ++i) u[i] = x[i];
        }
    }
    __syncthreads();
    for (int job = warp; job < 4 * KC; job += NWARP) {
        const int c = (job / KC) * 32 + lane, k = job % KC;
        if (c < tw) {
            const Chunk<MC> ch{LH + (k * MC + HALO) * LS + (c + HALO), G + (k * MC + 1) * GS + (c + 1), LS, GS,
                               tau};
            float x[MC];
            ch.solve(XC[(k * 2 + 0) * TW + c], XC[(k * 2 + 1) * TW + c], x);
#pragma unroll
            for (int i = 0; i < MC; ++i) {
                const int r = k * MC + i;
                const float v = 0.5f * (U[r * US + c] + x[i]);
                LH[(r + HALO) * LS + (c + HALO)] = v;
                if (r < th) Lout[(size_t)(y0 + r) * pitch + (x0 + c)] = v;
            }
        }
    }
}

// Shared state of a tile's run besides the tile arrays.
struct TileShared {
    int abort;
    float k;
    unsigned max;
};

// The whole evolution of one tile of the image `p` describes (tile index
// tile = ty * tiles_x + tx); every tile of the image runs it on its own CTA
// at the same time.  `bar` is the CTA's mbarrier of the record staging
// copies and mphase the number of its phases completed so far.  False when a
// bounded wait ran out (bit 0 of *p.status is set).
__device__ __forceinline__ bool evolve_tile(const Params& p, int tile, TileShared& S, uint64_t* bar,
                                            unsigned& mphase)
{
    extern __shared__ __align__(16) float sm[];
    float* LH = sm + OFF_L;
    float* SC = sm + OFF_A;  // S, then chunk records, staged records, u_x
    float* XE = sm + OFF_X;
    float* G = sm + OFF_B;   // H, then g
    float* RRc = SC;         // row chunk records [k][f][r]
    float* CRc = SC + RREC;  // column chunk records [k][f][c]
    float* XR = XE;          // row chunk externals [k][2][r]
    float* XC = XE + KR * 2 * TH;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tx = tile % p.tiles_x, ty = tile / p.tiles_x;
    const int x0 = tx * TW, y0 = ty * TH;
    const int tw = min(TW, p.w - x0), th = min(TH, p.h - y0);
    const unsigned ntiles = (unsigned)(p.tiles_x * p.tiles_y);
    unsigned nbar = 0;
    // lines: threads 0..TH-1 own the tile's rows, threads 128..128+TW-1 its columns
    const bool row_line = tid < th;
    const bool col_line = tid >= 128 && tid - 128 < tw;
    const int li = row_line ? tid : tid - 128;
    __syncthreads();  // the previous tile's run is done with shared memory

    if (p.img)
        presmooth_tile(sm, p, x0, y0, tw, th, p.levels);
    else
        load_all(LH, p.levels, p, x0, y0);
    if (tid == 0) S.max = 0u;
    __syncthreads();
    float inv_k2 = 0.f;
    if (!p.hist) {
        const float kk = p.k_fixed > 0.f ? p.k_fixed : *p.d_k;
        if (p.k_fixed > 0.f && tile == 0 && tid == 0) *p.d_k = kk;
        inv_k2 = 1.f / (kk * kk);
    }

    for (int lev = 1; lev < p.n_levels; ++lev) {
        const float tau = p.tau[lev];
        float* Lout = p.levels + (size_t)lev * p.plane;

        // 1. conductance of L_{lev-1} on the tile and its ring, ghosts past
        // the image
        h_pass(LH, G, p);
        __syncthreads();
        v_pass(G, SC, p);
        __syncthreads();
        if (lev == 1 && p.hist) {
            // the contrast factor: |grad|^2 of L_0 into G, the maximum of |grad|
            // over the interior, the histogram, the percentile; then g from
            // |grad|^2 in place
            float mx = scharr_pass<MODE_M2>(SC, G, 0.f, x0, y0, tw, th, p.w, p.h);
            for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            // non-negative floats order like their bit patterns
            if (lane == 0 && mx > 0.f) atomicMax(&S.max, __float_as_uint(mx));
            __syncthreads();
            if (tid == 0 && S.max) atomicMax(p.hmax_bits, S.max);
            nbar += ntiles;
            if (!grid_barrier(p, tile, nbar, &S.abort)) return false;
            const float hmax = __uint_as_float(ld_relaxed(reinterpret_cast<const int*>(p.hmax_bits)));
            // the tile's interior image pixels binned into one histogram per
            // warp (in SC, free after the smoothing), each thread counting a
            // run of up to 32 consecutive pixels of a row and adding a count
            // when the bin changes
            unsigned* wh = reinterpret_cast<unsigned*>(SC) + warp * p.nbins;
            for (int b = lane; b < p.nbins; b += 32) wh[b] = 0u;
            __syncthreads();
            const float hmax_scale = (float)p.nbins / hmax;
            const int ylo = max(1, y0), yhi = min(p.h - 2, y0 + th - 1), xlo = max(1, x0), xhi = min(p.w - 2, x0 + tw - 1);
            {
                const int yy = ylo + (tid >> 2), xs = xlo + 32 * (tid & 3), xe = min(xs + 32, xhi + 1);
                if (yy <= yhi) {
                    const float* grow = G + (yy - y0 + 1) * GS + (1 - x0);
                    int cur = -1;
                    unsigned cnt = 0;
                    for (int xx = xs; xx < xe; ++xx) {
                        const float m = sqrtf(grow[xx]);
                        if (!(m > 0.f)) continue;
                        const int b = min((int)floorf(m * hmax_scale), p.nbins - 1);
                        if (b != cur) {
                            if (cnt) atomicAdd(&wh[cur], cnt);
                            cur = b;
                            cnt = 0;
                        }
                        ++cnt;
                    }
                    if (cnt) atomicAdd(&wh[cur], cnt);
                }
            }
            __syncthreads();
            for (int b = tid; b < p.nbins; b += NT) {
                unsigned c = 0;
                const unsigned* wb = reinterpret_cast<const unsigned*>(SC) + b;
#pragma unroll 4
                for (int q = 0; q < NWARP; ++q) c += wb[q * p.nbins];
                if (c) atomicAdd(&p.hist[b], c);
            }
            nbar += ntiles;
            if (!grid_barrier(p, tile, nbar, &S.abort)) return false;
            // the whole histogram into shared memory, then the percentile
            unsigned* hs = reinterpret_cast<unsigned*>(XE);
            for (int b = tid; b < p.nbins; b += NT) hs[b] = __ldcg(p.hist + b);
            __syncthreads();
            if (warp == 0) {
                const float kk = percentile_k(hs, p.nbins, hmax, p.pct, lane);
                if (lane == 0) {
                    S.k = kk;
                    if (tile == 0) *p.d_k = kk;
                }
            }
            __syncthreads();
            inv_k2 = 1.f / (S.k * S.k);
            if (p.diffusivity == KAZE_G1)
                g_from_m2<true>(G, inv_k2);
            else
                g_from_m2<false>(G, inv_k2);
        } else if (p.diffusivity == KAZE_G1) {
            scharr_pass<MODE_G1>(SC, G, inv_k2, x0, y0, tw, th, p.w, p.h);
        } else {
            scharr_pass<MODE_G2>(SC, G, inv_k2, x0, y0, tw, th, p.w, p.h);
        }
        __syncthreads();
        ghost_conductance(G, x0, y0, p.w, p.h);
        __syncthreads();

        // 2. chunk records (warp jobs: 32 lines x one chunk)
        chunk_records(LH, G, RRc, CRc, tw, th, tau);
        __syncthreads();

        // 3. segment records (one thread per line) to global memory; the
        // joints of the chunk merges stay in registers for step 4
        Pt P[8], Q[8];
        if (row_line || col_line) {
            const Rec seg = segment_record(RRc, CRc, row_line, li, P, Q);
            float* dst = row_line ? p.xrow + ((size_t)(y0 + li) * p.tiles_x + tx) * REC
                                  : p.xcol + ((size_t)(x0 + li) * p.tiles_y + ty) * REC;
            store_rec(dst, 1, seg);
        }
        nbar += ntiles;
        if (!grid_barrier(p, tile, nbar, &S.abort)) return false;

        // 4. the records of the tile's lines from every tile (rows, then
        // columns: two contiguous blocks of global memory), staged into shared
        // memory by two bulk copies
        const int nrow = th * p.tiles_x * REC, ncol = tw * p.tiles_y * REC;
        const int nrow4 = (nrow + 3) & ~3;
        if (tid == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            const unsigned brow = (unsigned)nrow4 * 4u, bcol = (unsigned)((ncol + 3) & ~3) * 4u;
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                         "r"(brow + bcol)
                         : "memory");
            bulk_load(SC, p.xrow + (size_t)y0 * p.tiles_x * REC, brow, bar);
            bulk_load(SC + nrow4, p.xcol + (size_t)x0 * p.tiles_y * REC, bcol, bar);
        }
        if (!__syncthreads_and(mbar_wait(bar, mphase & 1u, p.wait_limit))) {
            if (tid == 0) {
                atomicOr(p.status, 1);
                mbar_wait(bar, mphase & 1u, p.wait_limit);  // copies still in flight
            }
            __syncthreads();
            return false;
        }
        ++mphase;
        // the line's own segment: merge the records left and right of it and
        // solve for its two external neighbours
        float xl = 0.f, xr = 0.f;
        if (row_line || col_line) {
            const int T = row_line ? p.tiles_x : p.tiles_y;
            const int t = row_line ? tx : ty;
            const float* rs = SC + (row_line ? li * T * REC : nrow4 + li * T * REC);
            Rec Lb = load_rec(rs, 1), Rb = Lb;
            for (int s = 1; s < t; ++s) Lb = merge(Lb, load_rec(rs + s * REC, 1));
            if (t + 1 < T) Rb = load_rec(rs + (t + 1) * REC, 1);
            for (int s = t + 2; s < T; ++s) Rb = merge(Rb, load_rec(rs + s * REC, 1));
            const Rec own = load_rec(rs + t * REC, 1);
            Pt P1{0.f, 0.f, 0.f}, Q1;
            Rec Mx = own;
            if (t > 0) Mx = merge(Lb, own, P1, Q1);
            if (t + 1 < T) {
                Pt P2, Q2;
                merge(Mx, Rb, P2, Q2);
                xr = Q2.y;
            }
            if (t > 0) xl = P1.y - P1.W * xr;
        }
        __syncthreads();  // the staged records are dead: XE is written next
        // every chunk's external neighbours, walking the chunk joints back
        // from the segment's right end
        if (row_line || col_line) chunk_externals(XR, XC, row_line, li, P, Q, xl, xr);
        __syncthreads();

        // 5. rows: u_x into SC; columns: L = (u_x + u_y) / 2 into the tile and
        // the level plane
        resolve_tile(LH, G, SC, XR, XC, Lout, p.pitch, x0, y0, tw, th, tau);
        if (lev + 1 < p.n_levels) {
            // 6. every tile's L_lev is in the level plane: read the ring
            nbar += ntiles;
            if (!grid_barrier(p, tile, nbar, &S.abort)) return false;
            load_halo(LH, Lout, p, x0, y0, tw, th);
            __syncthreads();
        }
    }
    return true;
}

__global__ void __launch_bounds__(NT, 1) k_evolve(const __grid_constant__ Params p)
{
    __shared__ TileShared S;
    __shared__ __align__(8) uint64_t s_bar;  // completion of the record staging copies
    if (threadIdx.x == 0) {
        S.abort = 0;
        mbar_init(&s_bar);
    }
    unsigned mphase = 0;
    evolve_tile(p, (int)blockIdx.x, S, &s_bar, mphase);
}

// The evolution of a batch of images of any sizes in one cooperative launch:
// CTA b runs the tiles work[off[b] .. off[b + 1]) in turn, each an (image,
// tile) pair.  The host packs the images into waves of at most gridDim.x
// tiles and gives an image's tiles to distinct CTAs of one wave, each CTA
// taking the waves in order: the tiles of an image run at the same time, and
// a CTA waits only for the CTAs of its own image, which reach it once they
// are done with the earlier waves (no cycle of waits).
__global__ void __launch_bounds__(NT, 1)
k_evolve_batch(const Params* __restrict__ ps, const int2* __restrict__ work, const int* __restrict__ off)
{
    __shared__ TileShared S;
    __shared__ __align__(8) uint64_t s_bar;
    if (threadIdx.x == 0) {
        S.abort = 0;
        mbar_init(&s_bar);
    }
    unsigned mphase = 0;
    for (int a = off[blockIdx.x]; a < off[blockIdx.x + 1]; ++a) {
        const int2 wk = work[a];
        if (!evolve_tile(ps[wk.x], wk.y, S, &s_bar, mphase)) return;
    }
}

// ------------------------------------------------------- the streamed form
// Images whose tiles exceed one per SM take each AOS step in three launches
// over all tiles, the tiles streaming through the SMs:
//   A: the tile of L_{lev-1} with its ring from the level plane, g on the
//      tile and its ring (ghosts past the image) -- the tile's own g to the
//      conductance plane --, the chunk and segment records to global memory;
//   X: one thread per line merges the records of the line's segments (prefix
//      from the left, suffix from the right) and solves every segment's two
//      outside neighbours;
//   B: the tile's L and g (own pixels and ring from the planes, ghosts past
//      the image), the chunk records again (for the joints), the chunk
//      externals from the segment's neighbours, the re-solves, L_lev to the
//      level plane.
// The arithmetic is the resident launch's, the launch boundaries replacing
// its grid barriers.

__global__ void __launch_bounds__(NT, 1) k_stream_a(const __grid_constant__ Params p, int lev, float* __restrict__ gpl)
{
    extern __shared__ __align__(16) float sm[];
    float* LH = sm + OFF_L;
    float* SC = sm + OFF_A;
    float* G = sm + OFF_B;
    float* RRc = SC;
    float* CRc = SC + RREC;
    const int tid = threadIdx.x;
    const int tile = blockIdx.x;
    const int tx = tile % p.tiles_x, ty = tile / p.tiles_x;
    const int x0 = tx * TW, y0 = ty * TH;
    const int tw = min(TW, p.w - x0), th = min(TH, p.h - y0);
    const bool row_line = tid < th;
    const bool col_line = tid >= 128 && tid - 128 < tw;
    const int li = row_line ? tid : tid - 128;
    const float tau = p.tau[lev];
    const float kk = *p.d_k;
    const float inv_k2 = 1.f / (kk * kk);
    load_all(LH, p.levels + (size_t)(lev - 1) * p.plane, p, x0, y0);
    __syncthreads();
    h_pass(LH, G, p);
    __syncthreads();
    v_pass(G, SC, p);
    __syncthreads();
    if (p.diffusivity == KAZE_G1)
        scharr_pass<MODE_G1>(SC, G, inv_k2, x0, y0, tw, th, p.w, p.h);
    else
        scharr_pass<MODE_G2>(SC, G, inv_k2, x0, y0, tw, th, p.w, p.h);
    __syncthreads();
    // the tile's own g to the plane (pass B reads its ring from the neighbours')
    for (int e = tid; e < th * tw; e += NT) {
        const int r = e / tw, c = e - r * tw;
        gpl[(size_t)(y0 + r) * p.pitch + (x0 + c)] = G[(r + 1) * GS + (c + 1)];
    }
    ghost_conductance(G, x0, y0, p.w, p.h);
    __syncthreads();
    chunk_records(LH, G, RRc, CRc, tw, th, tau);
    __syncthreads();
    if (row_line || col_line) {
        Pt P[8], Q[8];
        const Rec seg = segment_record(RRc, CRc, row_line, li, P, Q);
        float* dst = row_line ? p.xrow + ((size_t)(y0 + li) * p.tiles_x + tx) * REC
                              : p.xcol + ((size_t)(x0 + li) * p.tiles_y + ty) * REC;
        store_rec(dst, 1, seg);
    }
}

constexpr int STREAM_TMAX = 64;  // segments of a line the line pass takes

// One thread per line (rows 0..h-1, then columns 0..w-1): the outside
// neighbours (xl, xr) of every segment of the line, to ext[line][t][2].
__global__ void __launch_bounds__(128) k_stream_x(const __grid_constant__ Params p, float* __restrict__ erow,
                                                  float* __restrict__ ecol)
{
    const int line = blockIdx.x * blockDim.x + threadIdx.x;
    if (line >= p.h + p.w) return;
    const bool row = line < p.h;
    const int li = row ? line : line - p.h;
    const int T = row ? p.tiles_x : p.tiles_y;
    const float* rec = row ? p.xrow + (size_t)li * T * REC : p.xcol + (size_t)li * T * REC;
    float* ext = row ? erow + (size_t)li * T * 2 : ecol + (size_t)li * T * 2;
    // prefix records: pre[t] = the union of segments 0 .. t - 1
    Rec pre[STREAM_TMAX];
    if (T > 1) pre[1] = load_rec(rec, 1);
    for (int t = 2; t < T; ++t) pre[t] = merge(pre[t - 1], load_rec(rec + (t - 1) * REC, 1));
    // from the right: suf = the union of segments t + 1 .. T - 1
    Rec suf{};
    for (int t = T - 1; t >= 0; --t) {
        const Rec own = load_rec(rec + t * REC, 1);
        Pt P1{0.f, 0.f, 0.f}, Q1;
        Rec Mx = own;
        if (t > 0) Mx = merge(pre[t], own, P1, Q1);
        float xl = 0.f, xr = 0.f;
        if (t + 1 < T) {
            Pt P2, Q2;
            merge(Mx, suf, P2, Q2);
            xr = Q2.y;
        }
        if (t > 0) xl = P1.y - P1.W * xr;
        ext[t * 2 + 0] = xl;
        ext[t * 2 + 1] = xr;
        suf = t + 1 < T ? merge(own, suf) : own;
    }
}

__global__ void __launch_bounds__(NT, 1) k_stream_b(const __grid_constant__ Params p, int lev,
                                                    const float* __restrict__ gpl, const float* __restrict__ erow,
                                                    const float* __restrict__ ecol)
{
    extern __shared__ __align__(16) float sm[];
    float* LH = sm + OFF_L;
    float* SC = sm + OFF_A;
    float* XE = sm + OFF_X;
    float* G = sm + OFF_B;
    float* RRc = SC;
    float* CRc = SC + RREC;
    float* XR = XE;
    float* XC = XE + KR * 2 * TH;
    const int tid = threadIdx.x;
    const int tile = blockIdx.x;
    const int tx = tile % p.tiles_x, ty = tile / p.tiles_x;
    const int x0 = tx * TW, y0 = ty * TH;
    const int tw = min(TW, p.w - x0), th = min(TH, p.h - y0);
    const bool row_line = tid < th;
    const bool col_line = tid >= 128 && tid - 128 < tw;
    const int li = row_line ? tid : tid - 128;
    const float tau = p.tau[lev];
    const float* Lp = p.levels + (size_t)(lev - 1) * p.plane;
    // the tile's L with its ring (the chunk solves read the tile's own pixels;
    // a ragged tile's elements past the image must hold finite values: the
    // reflected ones) and g on the tile and its ring inside the image,
    // ghosts past it
    load_all(LH, Lp, p, x0, y0);
    for (int e = tid; e < (th + 2) * (tw + 2); e += NT) {
        const int r = e / (tw + 2) - 1, c = e - (r + 1) * (tw + 2) - 1;
        const int y = y0 + r, x = x0 + c;
        if (y >= 0 && y < p.h && x >= 0 && x < p.w) G[(r + 1) * GS + (c + 1)] = __ldcg(gpl + (size_t)y * p.pitch + x);
    }
    __syncthreads();
    ghost_conductance(G, x0, y0, p.w, p.h);
    __syncthreads();
    chunk_records(LH, G, RRc, CRc, tw, th, tau);
    __syncthreads();
    Pt P[8], Q[8];
    if (row_line || col_line) {
        segment_record(RRc, CRc, row_line, li, P, Q);
        const float* e = row_line ? erow + ((size_t)(y0 + li) * p.tiles_x + tx) * 2
                                  : ecol + ((size_t)(x0 + li) * p.tiles_y + ty) * 2;
        chunk_externals(XR, XC, row_line, li, P, Q, __ldcg(e), __ldcg(e + 1));
    }
    __syncthreads();
    resolve_tile(LH, G, SC, XR, XC, p.levels + (size_t)lev * p.plane, p.pitch, x0, y0, tw, th, tau);
}

}  // namespace ev

cudaError_t configure_evolve_kernel()
{
    cudaError_t e = cudaFuncSetAttribute(ev::k_evolve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ev::SMEM_BYTES);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(ev::k_stream_a, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ev::SMEM_BYTES);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(ev::k_stream_b, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ev::SMEM_BYTES);
    return e;
}

bool evolve_front_fits(int r0, int nbins) { return r0 == ev::R0MAX && nbins * ev::NWARP <= ev::A_SIZE; }

size_t evolve_exchange_floats(int max_tiles)
{
    // segment records of every line of every tile (rows, then columns from a
    // 16-byte boundary), and slack for the 16-byte rounding of the copies
    return (size_t)(ev::TH + ev::TW) * max_tiles * ev::REC + 64;
}

bool evolve_fits(int w, int h, int radius, int* tiles)
{
    if (radius < 1 || radius > ev::RMAX) return false;
    const int tx = (w + ev::TW - 1) / ev::TW, ty = (h + ev::TH - 1) / ev::TH;
    if (tx > ev::TMAX || ty > ev::TMAX) return false;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return false;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ev::k_evolve, ev::NT, ev::SMEM_BYTES) != cudaSuccess)
        return false;
    if (per_sm < 1 || tx * ty > sms * per_sm) return false;
    if (tiles) *tiles = tx * ty;
    return true;
}

namespace {

// The launch parameters of one image; false when it does not fit.
bool make_params(ev::Params& p, float* levels, long long plane, int pitch, int w, int h, int n_levels,
                 const double* t, float* d_k, const GaussTaps& taps, int diffusivity, float* exchange,
                 unsigned int* barrier, int* status, const EvolveFront* front, long long wait_limit, int stall_tile,
                 float k_fixed)
{
    if (n_levels > kMaxLevels || taps.r < 1 || taps.r > ev::RMAX) return false;
    p.levels = levels;
    p.plane = plane;
    p.pitch = pitch;
    p.w = w;
    p.h = h;
    p.n_levels = n_levels;
    p.tiles_x = (w + ev::TW - 1) / ev::TW;
    p.tiles_y = (h + ev::TH - 1) / ev::TH;
    p.d_k = d_k;
    for (int j = 0; j <= ev::RMAX; ++j) p.wt[j] = j <= taps.r ? taps.w[taps.r + j] : 0.f;
    p.diffusivity = diffusivity;
    for (int i = 0; i < kMaxLevels; ++i) p.tau[i] = (i >= 1 && i < n_levels) ? (float)(t[i] - t[i - 1]) : 0.f;
    p.xrow = exchange;
    p.xcol = exchange + (((size_t)h * p.tiles_x * ev::REC + 3) & ~(size_t)3);
    p.barrier = barrier;
    p.status = status;
    p.img = nullptr;
    p.img_pitch = 0;
    p.r0 = 0;
    for (int j = 0; j <= 2 * ev::R0MAX; ++j) p.pw[j] = 0.f;
    p.hmax_bits = nullptr;
    p.hist = nullptr;
    p.nbins = 0;
    p.pct = 0.0;
    if (front && front->img) {
        if (front->taps0->r != ev::R0MAX) return false;
        p.img = front->img;
        p.img_pitch = front->img_pitch;
        p.r0 = front->taps0->r;
        for (int j = 0; j <= 2 * p.r0; ++j) p.pw[j] = front->taps0->w[j];
        if (front->hist) {
            if (front->nbins < 1 || front->nbins * ev::NWARP > ev::A_SIZE) return false;
            p.hmax_bits = front->hmax_bits;
            p.hist = front->hist;
            p.nbins = front->nbins;
            p.pct = front->pct;
        }
    }
    p.k_fixed = p.hist ? 0.f : k_fixed;
    p.wait_limit = wait_limit > 0 ? wait_limit : (1ll << 31);
    p.stall_tile = stall_tile;
    return true;
}

}  // namespace

cudaError_t launch_evolve(float* levels, long long plane, int pitch, int w, int h, int n_levels, const double* t,
                          float* d_k, const GaussTaps& taps, int diffusivity, float* exchange, int max_tiles,
                          unsigned int* barrier, int* status, cudaStream_t st, const EvolveFront* front,
                          long long wait_limit, int stall_tile, bool zero_barrier)
{
    int tiles = 0;
    if (!evolve_fits(w, h, taps.r, &tiles) || tiles > max_tiles) return cudaErrorInvalidValue;
    ev::Params p;
    if (!make_params(p, levels, plane, pitch, w, h, n_levels, t, d_k, taps, diffusivity, exchange, barrier, status,
                     front, wait_limit, stall_tile, 0.f))
        return cudaErrorInvalidValue;
    if (zero_barrier) {
        const cudaError_t e = cudaMemsetAsync(barrier, 0, sizeof(unsigned int), st);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(tiles);
    cfg.blockDim = dim3(ev::NT);
    cfg.dynamicSmemBytes = ev::SMEM_BYTES;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, ev::k_evolve, p);
}

size_t evolve_stream_floats(int max_w, int max_h)
{
    const size_t tx = (size_t)(max_w + ev::TW - 1) / ev::TW, ty = (size_t)(max_h + ev::TH - 1) / ev::TH;
    auto r4 = [](size_t n) { return (n + 3) & ~(size_t)3; };
    return r4(max_h * tx * ev::REC) + r4(max_w * ty * ev::REC) + r4(max_h * tx * 2) + r4(max_w * ty * 2) + 64;
}

bool evolve_stream_fits(int w, int h, int radius)
{
    if (radius < 1 || radius > ev::RMAX || w < 1 || h < 1) return false;
    const int tx = (w + ev::TW - 1) / ev::TW, ty = (h + ev::TH - 1) / ev::TH;
    return tx <= ev::STREAM_TMAX && ty <= ev::STREAM_TMAX;
}

cudaError_t launch_stream_pass(int pass, int lev, float* levels, long long plane, int pitch, int w, int h,
                               int n_levels, const double* t, float* d_k, const GaussTaps& taps, int diffusivity,
                               float* g, float* scratch, cudaStream_t st)
{
    if (!evolve_stream_fits(w, h, taps.r) || lev < 1 || lev >= n_levels || !scratch || !g)
        return cudaErrorInvalidValue;
    const int tx = (w + ev::TW - 1) / ev::TW, ty = (h + ev::TH - 1) / ev::TH;
    auto r4 = [](size_t n) { return (n + 3) & ~(size_t)3; };
    float* xrow = scratch;
    float* xcol = xrow + r4((size_t)h * tx * ev::REC);
    float* erow = xcol + r4((size_t)w * ty * ev::REC);
    float* ecol = erow + r4((size_t)h * tx * 2);
    ev::Params p;
    if (!make_params(p, levels, plane, pitch, w, h, n_levels, t, d_k, taps, diffusivity, scratch, nullptr, nullptr,
                     nullptr, 0, -1, 0.f))
        return cudaErrorInvalidValue;
    p.xrow = xrow;
    p.xcol = xcol;
    if (pass == 0)
        ev::k_stream_a<<<tx * ty, ev::NT, ev::SMEM_BYTES, st>>>(p, lev, g);
    else if (pass == 1)
        ev::k_stream_x<<<(h + w + 127) / 128, 128, 0, st>>>(p, erow, ecol);
    else
        ev::k_stream_b<<<tx * ty, ev::NT, ev::SMEM_BYTES, st>>>(p, lev, g, erow, ecol);
    return cudaGetLastError();
}

size_t evolve_params_bytes() { return sizeof(ev::Params); }

bool evolve_batch_params(void* out, const EvolveImage& im, int n_levels, const double* t, const GaussTaps& taps,
                         int diffusivity, int* status, long long wait_limit, int stall_tile)
{
    int tiles = 0;
    if (!evolve_fits(im.w, im.h, taps.r, &tiles)) return false;
    EvolveFront f;
    f.img = im.img;
    f.img_pitch = im.img_pitch;
    f.taps0 = im.taps0;
    f.hmax_bits = im.hmax_bits;
    f.hist = im.hist;
    f.nbins = im.nbins;
    f.pct = im.pct;
    return make_params(*static_cast<ev::Params*>(out), im.levels, im.plane, im.pitch, im.w, im.h, n_levels, t,
                       im.d_k, taps, diffusivity, im.exchange, im.barrier, status, &f, wait_limit, stall_tile,
                       im.k_fixed);
}

int evolve_batch_grid()
{
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaFuncSetAttribute(ev::k_evolve_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ev::SMEM_BYTES) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ev::k_evolve_batch, ev::NT, ev::SMEM_BYTES) !=
            cudaSuccess)
        return 0;
    return per_sm < 1 ? 0 : sms * per_sm;
}

cudaError_t launch_evolve_batch(const void* d_params, const int2* d_work, const int* d_off, int grid,
                                cudaStream_t st)
{
    if (grid < 1 || !d_params || !d_work || !d_off) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(ev::NT);
    cfg.dynamicSmemBytes = ev::SMEM_BYTES;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, ev::k_evolve_batch, static_cast<const ev::Params*>(d_params), d_work, d_off);
}

}  // namespace kz
