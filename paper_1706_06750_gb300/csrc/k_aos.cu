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
// Line solver (partition method of Wang 1981 in "modified Thomas" form).  A
// line of n unknowns is cut into 32 chunks of m rows, m odd and >= 3 with
// 32 m >= n (rows past n are identity rows).  Then
//   phase 1  every chunk eliminates its interior twice -- top down and
//            bottom up, two independent recurrences interleaved for ILP --
//            leaving two equations that tie its first and last unknowns to
//            the neighbouring chunks;
//   phase 2  the 64-unknown interface system is reduced to the 32 last
//            unknowns and solved by parallel cyclic reduction with warp
//            shuffles (one lane per chunk, 5 steps);
//   phase 3  every chunk solves its interior by Thomas with both ends known.
// Because m is odd, a line stored contiguously puts the 32 chunks' i-th
// elements in 32 different shared-memory banks.
//
// GB300 mapping.
//   rows:    a warp per row.  The row's g and L are staged into shared memory
//            with two TMA bulk copies (cp.async.bulk, mbarrier completion);
//            lane p owns chunk p.  Output rows are written with 128-bit
//            stores.
//   columns: a CTA per strip of COLS adjacent columns, a thread per (column,
//            chunk).  The strip of g and L is staged by TMA 2-D tensor copies
//            (boxes of COLS x 256, zero fill past the image) into a
//            [row][COLS] tile, so thread (c, p) walks its chunk at stride COLS
//            without bank conflicts (m odd).  The interface systems are
//            solved by one warp per column; the final average with the row
//            solution is fused into the back substitution.
// Every mbarrier wait is bounded; on timeout the kernel raises a flag in
// *status and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <dlfcn.h>

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

// ---------------------------------------------------------- TMA helpers --

__device__ __forceinline__ unsigned smem_u32(const void* p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

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
//   aL x_0 + x_{m-1} + cL x_m  = dL     (last row, x_m = next chunk's first)
//   aF x_-1 + x_0 + cF x_{m-1} = dF     (first row, x_-1 = previous chunk's last)
struct ChunkEqs {
    float aL, cL, dL, aF, cF, dF;
};

// Phase 1 on one chunk.  g, d point at the chunk's element 0; element i is at
// [i*S]; [-S] and [m*S] are the neighbouring chunks' end elements.  j0 is the
// chunk's first line index, n the line length.
template <int S>
__device__ __forceinline__ ChunkEqs chunk_reduce(const float* g, const float* d, int j0, int m, int n, float tau)
{
    auto gl = [&](int i) -> float {
        const int j = j0 + i;
        return (j >= 0 && j < n) ? g[i * S] : 0.f;
    };
    auto dl = [&](int i) -> float { return (j0 + i < n) ? d[i * S] : 0.f; };
    auto lower = [&](int i, float gm, float g0) -> float {
        const int j = j0 + i;
        return (j >= 1 && j < n) ? -tau * (gm + g0) : 0.f;
    };
    auto upper = [&](int i, float g0, float gp) -> float { return (j0 + i + 1 < n) ? -tau * (g0 + gp) : 0.f; };

    float gdA = gl(0), gdB = gl(1);
    float ap = 0.f, cp = 0.f, dp = 0.f;
    float guB = gl(m - 2), guC = gl(m - 1);
    float au = 0.f, cu = 0.f, du = 0.f;
#pragma unroll 2
    for (int t = 0; t < m - 1; ++t) {
        {  // top-down row i = 1 + t, x_0 treated as known
            const int i = 1 + t;
            const float gdC = gl(i + 1);
            const float a = lower(i, gdA, gdB), c = upper(i, gdB, gdC);
            const float b = 1.f - a - c, dd = dl(i);
            if (t == 0) {
                const float r = rcp_approx(b);
                ap = a * r;
                cp = c * r;
                dp = dd * r;
            } else {
                const float r = rcp_approx(b - a * cp);
                ap = -a * ap * r;
                dp = (dd - a * dp) * r;
                cp = c * r;
            }
            gdA = gdB;
            gdB = gdC;
        }
        {  // bottom-up row i = m - 2 - t, x_{m-1} treated as known
            const int i = m - 2 - t;
            const float guA = gl(i - 1);
            const float a = lower(i, guA, guB), c = upper(i, guB, guC);
            const float b = 1.f - a - c, dd = dl(i);
            if (t == 0) {
                const float r = rcp_approx(b);
                au = a * r;
                cu = c * r;
                du = dd * r;
            } else {
                const float r = rcp_approx(b - c * au);
                cu = -c * cu * r;
                du = (dd - c * du) * r;
                au = a * r;
            }
            guC = guB;
            guB = guA;
        }
    }
    return ChunkEqs{ap, cp, dp, au, cu, du};
}

// Phase 2: lane p holds chunk p's equations; returns that chunk's first and
// last unknowns.  The first unknowns are eliminated,
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

// Phase 3: interior rows 1..m-2 of the chunk by Thomas with x_0 = xfirst and
// x_{m-1} = xlast known.  The forward sweep overwrites g[i*S] with c'_i and
// d[i*S] with d'_i; the backward sweep hands every solution value to
// emit(i, x_i), including both ends.
template <int S, typename Emit>
__device__ __forceinline__ void chunk_interior(float* g, float* d, int j0, int m, int n, float tau, float xfirst,
                                               float xlast, Emit emit)
{
    auto lower = [&](int i, float gm, float g0) -> float {
        const int j = j0 + i;
        return (j >= 1 && j < n) ? -tau * (gm + g0) : 0.f;
    };
    auto upper = [&](int i, float g0, float gp) -> float { return (j0 + i + 1 < n) ? -tau * (g0 + gp) : 0.f; };
    emit(m - 1, xlast);
    if (m >= 3) {
        float gA = g[0], gB = g[S];
        float cp = 0.f, dp = 0.f;
#pragma unroll 2
        for (int i = 1; i <= m - 2; ++i) {
            const float gC = g[(i + 1) * S];
            float a = lower(i, gA, gB), c = upper(i, gB, gC);
            const float b = 1.f - a - c;
            float rhs = (j0 + i < n) ? d[i * S] : 0.f;
            if (i == 1) {
                rhs -= a * xfirst;
                a = 0.f;
            }
            if (i == m - 2) {
                rhs -= c * xlast;
                c = 0.f;
            }
            const float r = rcp_approx(b - a * cp);
            dp = (rhs - a * dp) * r;
            cp = c * r;
            g[i * S] = cp;
            d[i * S] = dp;
            gA = gB;
            gB = gC;
        }
        float x = xlast;
#pragma unroll 4
        for (int i = m - 2; i >= 1; --i) {
            x = d[i * S] - g[i * S] * x;
            emit(i, x);
        }
    }
    emit(0, xfirst);
}

// ---------------------------------------------------------------- rows ----
// One warp per row; blockDim = 32 * rows per CTA.  Shared memory per warp:
// g and L of the row, each ls floats (ls = 32 m rounded up to 4).
__global__ void __launch_bounds__(256) k_aos_rows(const float* __restrict__ L, const float* __restrict__ g,
                                                  float* __restrict__ ux, int pitch, int w, int h, float tau, int m,
                                                  int ls, int* __restrict__ status)
{
    extern __shared__ __align__(128) float sm[];
    __shared__ __align__(8) uint64_t bars[8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int y = blockIdx.x * (blockDim.x >> 5) + warp;
    if (y >= h) return;  // no CTA-wide barrier below
    float* sg = sm + (size_t)warp * 2 * ls;
    float* sd = sg + ls;
    const float* grow = g + (size_t)y * pitch;
    const float* lrow = L + (size_t)y * pitch;
    const int w4 = w & ~3;

    if (lane == 0) {
        mbar_init(&bars[warp], 1);
        mbar_expect_tx(&bars[warp], 2u * 4u * (unsigned)w4);
        if (w4 > 0) {
            bulk_load(sg, grow, 4u * w4, &bars[warp]);
            bulk_load(sd, lrow, 4u * w4, &bars[warp]);
        }
    }
    for (int x = w4 + lane; x < w; x += 32) {
        sg[x] = __ldg(grow + x);
        sd[x] = __ldg(lrow + x);
    }
    __syncwarp();
    const bool ok = mbar_wait_bounded(&bars[warp], 0);
    if (!__all_sync(FULL, ok)) {  // same decision in every lane
        if (lane == 0) atomicOr(status, 1);
        return;
    }

    const int j0 = lane * m;
    const ChunkEqs e = chunk_reduce<1>(sg + j0, sd + j0, j0, m, w, tau);
    __syncwarp();  // all neighbours' reads done before phase 3 writes
    float xf, xl;
    interface_solve(e, lane, xf, xl);
    float* cd = sd + j0;
    chunk_interior<1>(sg + j0, cd, j0, m, w, tau, xf, xl, [&](int i, float x) { cd[i] = x; });
    __syncwarp();

    float* urow = ux + (size_t)y * pitch;
    for (int x = lane * 4; x < w4; x += 128)
        *reinterpret_cast<float4*>(urow + x) = *reinterpret_cast<const float4*>(sd + x);
    for (int x = w4 + lane; x < w; x += 32) urow[x] = sd[x];
}

// ------------------------------------------------------------- columns ----
// A strip of COLS columns per CTA, blockDim = 32 * COLS, thread t owns
// column t % COLS and chunk t / COLS.  Shared memory: the g and L tiles
// ([rows][COLS], rows = 32 m rounded up to whole 256-row boxes) and the
// interface equations.
template <int COLS>
__global__ void __launch_bounds__(COLS * 32)
    k_aos_cols(const __grid_constant__ CUtensorMap tmL, const __grid_constant__ CUtensorMap tmG,
               const float* __restrict__ ux, float* __restrict__ Lnext, int pitch, int w, int h, float tau, int m,
               int rows_staged, int* __restrict__ status)
{
    extern __shared__ __align__(128) float sm[];
    __shared__ __align__(8) uint64_t bar;
    const int tid = threadIdx.x;
    const int c = tid % COLS, p = tid / COLS;
    const int x0 = blockIdx.x * COLS;
    float* tg = sm;
    float* td = sm + (size_t)rows_staged * COLS;
    float* eq = td + (size_t)rows_staged * COLS;  // [6][COLS][32]

    if (tid == 0) {
        mbar_init(&bar, 1);
        const int nb = rows_staged / 256;
        mbar_expect_tx(&bar, 2u * nb * 256u * COLS * 4u);
        for (int b = 0; b < nb; ++b) {
            tma_load_2d(tg + (size_t)b * 256 * COLS, &tmG, x0, 256 * b, &bar);
            tma_load_2d(td + (size_t)b * 256 * COLS, &tmL, x0, 256 * b, &bar);
        }
    }
    __syncthreads();
    const bool ok = mbar_wait_bounded(&bar, 0);
    if (!__syncthreads_and(ok)) {  // same decision in every thread
        if (tid == 0) atomicOr(status, 1);
        return;
    }

    const int j0 = p * m;
    float* cg = tg + (size_t)j0 * COLS + c;
    float* cdd = td + (size_t)j0 * COLS + c;
    const ChunkEqs e = chunk_reduce<COLS>(cg, cdd, j0, m, h, tau);
    eq[(0 * COLS + c) * 32 + p] = e.aL;
    eq[(1 * COLS + c) * 32 + p] = e.cL;
    eq[(2 * COLS + c) * 32 + p] = e.dL;
    eq[(3 * COLS + c) * 32 + p] = e.aF;
    eq[(4 * COLS + c) * 32 + p] = e.cF;
    eq[(5 * COLS + c) * 32 + p] = e.dF;
    __syncthreads();
    const int warp = tid >> 5, lane = tid & 31;
    if (warp < COLS) {  // warp `warp` solves column `warp`; lane = chunk
        ChunkEqs f;
        f.aL = eq[(0 * COLS + warp) * 32 + lane];
        f.cL = eq[(1 * COLS + warp) * 32 + lane];
        f.dL = eq[(2 * COLS + warp) * 32 + lane];
        f.aF = eq[(3 * COLS + warp) * 32 + lane];
        f.cF = eq[(4 * COLS + warp) * 32 + lane];
        f.dF = eq[(5 * COLS + warp) * 32 + lane];
        float xf, xl;
        interface_solve(f, lane, xf, xl);
        __syncwarp();
        eq[(0 * COLS + warp) * 32 + lane] = xf;
        eq[(1 * COLS + warp) * 32 + lane] = xl;
    }
    __syncthreads();
    const float xf = eq[(0 * COLS + c) * 32 + p];
    const float xl = eq[(1 * COLS + c) * 32 + p];
    const int x = x0 + c;
    const bool active = x < w;
    chunk_interior<COLS>(cg, cdd, j0, m, h, tau, xf, xl, [&](int i, float v) {
        const int j = j0 + i;
        if (active && j < h) {
            const size_t gi = (size_t)j * pitch + x;
            Lnext[gi] = 0.5f * (__ldg(ux + gi) + v);
        }
    });
}

constexpr size_t kSmemBudget = 220 * 1024;

int chunk_len(int n)
{
    int m = (n + 31) / 32;
    m |= 1;
    return m < 3 ? 3 : m;
}

int row_stride_floats(int w) { return (32 * chunk_len(w) + 3) / 4 * 4; }

int rows_per_cta(int w)
{
    const size_t per = (size_t)2 * row_stride_floats(w) * sizeof(float);
    int r = (int)(kSmemBudget / per);
    return r < 1 ? 0 : (r > 4 ? 4 : r);
}

int rows_staged(int h) { return (32 * chunk_len(h) + 255) / 256 * 256; }

size_t cols_smem(int h, int cols)
{
    return ((size_t)2 * rows_staged(h) * cols + (size_t)6 * cols * 32) * sizeof(float);
}

int cols_per_cta(int h)
{
    if (cols_smem(h, 8) <= kSmemBudget) return 8;
    if (cols_smem(h, 4) <= kSmemBudget) return 4;
    return 0;
}

const char* g_encode_err = "";

// cuTensorMapEncodeTiled from the driver: through the runtime's entry-point
// query, else straight from libcuda.so.1 (no link-time driver dependency).
PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (fn) return fn;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
    if (e == cudaSuccess && q == cudaDriverEntryPointSuccess && p) {
        fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
        return fn;
    }
    void* lib = dlopen("libcuda.so.1", RTLD_NOW | RTLD_NOLOAD);
    if (!lib) lib = dlopen("libcuda.so.1", RTLD_NOW);
    if (lib) p = dlsym(lib, "cuTensorMapEncodeTiled");
    if (p) {
        fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
        return fn;
    }
    g_encode_err = e != cudaSuccess ? "cudaGetDriverEntryPointByVersion failed and libcuda.so.1 has no cuTensorMapEncodeTiled"
                                    : "cuTensorMapEncodeTiled not found in the driver";
    return nullptr;
}

// 2-D map of a w x h FP32 plane with the given pitch, box COLS x 256.
bool make_strip_map(CUtensorMap* map, const float* base, int pitch, int w, int h, int cols)
{
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)w, (cuuint64_t)h};
    cuuint64_t strides[1] = {(cuuint64_t)pitch * sizeof(float)};
    cuuint32_t box[2] = {(cuuint32_t)cols, 256u};
    cuuint32_t estr[2] = {1u, 1u};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

}  // namespace

const char* aos_config_error() { return g_encode_err; }

cudaError_t configure_aos_kernels()
{
    cudaError_t e = allow_max_dynamic_smem(k_aos_rows);
    if (e == cudaSuccess) e = allow_max_dynamic_smem(k_aos_cols<8>);
    if (e == cudaSuccess) e = allow_max_dynamic_smem(k_aos_cols<4>);
    if (e == cudaSuccess && !encode_fn()) e = cudaErrorNotSupported;
    return e;
}

size_t aos_rows_smem_bytes(int w)
{
    const int r = rows_per_cta(w);
    return r == 0 ? 0 : (size_t)r * 2 * row_stride_floats(w) * sizeof(float);
}

size_t aos_cols_smem_bytes(int h)
{
    const int c = cols_per_cta(h);
    return c == 0 ? 0 : cols_smem(h, c);
}

cudaError_t launch_aos_rows(const float* L, const float* g, float* ux, int pitch, int w, int h, float tau,
                            int* d_status, cudaStream_t st)
{
    const int r = rows_per_cta(w);
    if (r == 0) return cudaErrorInvalidValue;
    const size_t smem = aos_rows_smem_bytes(w);
    k_aos_rows<<<(h + r - 1) / r, 32 * r, smem, st>>>(L, g, ux, pitch, w, h, tau, chunk_len(w), row_stride_floats(w),
                                                       d_status);
    return cudaGetLastError();
}

cudaError_t launch_aos_cols(const float* L, const float* g, const float* ux, float* Lnext, int pitch, int w, int h,
                            float tau, int* d_status, cudaStream_t st)
{
    const int c = cols_per_cta(h);
    if (c == 0) return cudaErrorInvalidValue;
    CUtensorMap mL, mG;
    if (!make_strip_map(&mL, L, pitch, w, h, c) || !make_strip_map(&mG, g, pitch, w, h, c))
        return cudaErrorInvalidValue;
    const size_t smem = cols_smem(h, c);
    const int m = chunk_len(h), rs = rows_staged(h);
    if (c == 8)
        k_aos_cols<8><<<(w + 7) / 8, 256, smem, st>>>(mL, mG, ux, Lnext, pitch, w, h, tau, m, rs, d_status);
    else
        k_aos_cols<4><<<(w + 3) / 4, 128, smem, st>>>(mL, mG, ux, Lnext, pitch, w, h, tau, m, rs, d_status);
    return cudaGetLastError();
}

}  // namespace kz
