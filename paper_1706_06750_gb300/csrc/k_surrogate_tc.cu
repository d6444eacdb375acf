// k_surrogate_tc.cu -- the whole surrogate network in one persistent kernel
// on the 5th-generation tensor cores (tcgen05.mma, accumulators in tensor
// memory).  Same contract as the other surrogate kernels: x0 = [dx, dy, g, s,
// c], three 3x3 conv + ReLU layers of 32 channels, a last 3x3 conv to one
// channel z, L_next = L + z / 256; BF16 operands, FP32 accumulation, zero
// padding at the image border.
//
// A CTA computes a 24 x 24 tile of L_next on a 32 x 32 pixel frame (the
// tile plus a 4-pixel border).  Activations live in shared memory in the
// canonical K-major layout of the tensor cores without swizzling: for every
// group of 8 channels, the frame's pixels in row-major order, 16 bytes each,
// so 8 consecutive pixels form one 8 x 16-byte core matrix.  Layer l (1..4)
// is an implicit GEMM over the frame pixels of rows l .. 31 - l, all 32
// columns, in tiles of M = 128 consecutive pixels: tap (ky, kx) of the 3x3
// kernel reads the source pixels shifted by (ky - 1) * 32 + (kx - 1), i.e.
// the same operand descriptor with its start address moved by 16 bytes per
// pixel.  The columns that wrap around a frame row produce garbage that no
// later valid output reads (each layer's valid region shrinks by one pixel a
// side, as the convolutions do).  N = 32 output channels (16 for the last
// layer, whose channels 1..15 are zero weights), K = 16 input channels per
// instruction.  One thread issues every MMA of a layer into its own TMEM
// columns per M tile and commits each tile to its own mbarrier; the 8 warps
// read finished tiles back while later tiles still compute (tcgen05.ld, each
// warp its quarter of the 128 TMEM lanes, the two warp groups alternating
// tiles), add the bias, apply the ReLU and zero padding, and write the next
// layer's operand.  The next frame's input is staged while the last layer
// computes.  All weights stay in shared memory for the CTA's life.
// Every wait is bounded: on a timeout the kernel raises bit 0 of *status,
// waits (bounded) for its MMAs, frees its tensor memory and returns.
#include "kaze_internal.h"
#include "surrogate.h"

namespace kz {
namespace sg {
namespace {

constexpr int TC_T = 24;                  // output tile edge
constexpr int TC_F = TC_T + 8;            // frame edge (32)
constexpr int TC_FP = TC_F * TC_F;        // frame pixels (1024)
constexpr int TC_FS = 64;                 // front slack pixels (taps read up to 33 before)
constexpr int TC_BP = TC_FS + TC_FP + 192;  // pixels per channel group incl. slack (1280)
constexpr int TC_THREADS = 256;
constexpr int TC_TMEM_COLS = 256;         // 8 M tiles x 32 columns
constexpr uint32_t TC_LBO_ACT = TC_BP * 16;   // bytes between channel groups of an activation buffer

// weight buffers: [K/8][N][8] BF16
constexpr int W1_BYTES = (9 * kC0 / 8) * 32 * 16;
constexpr int WH_BYTES = (9 * kC / 8) * 32 * 16;
constexpr int W4_BYTES = (9 * kC / 8) * 16 * 16;
constexpr int ACT_BYTES = 4 * TC_BP * 16;     // 32 channels
constexpr int OFF_W1 = 0;
constexpr int OFF_W2 = OFF_W1 + W1_BYTES;
constexpr int OFF_W3 = OFF_W2 + WH_BYTES;
constexpr int OFF_W4 = OFF_W3 + WH_BYTES;
constexpr int OFF_BIAS = OFF_W4 + W4_BYTES;
constexpr int OFF_ACTA = OFF_BIAS + 128 * 4;
constexpr int OFF_ACTB = OFF_ACTA + ACT_BYTES;
constexpr int TC_SMEM = OFF_ACTB + ACT_BYTES;
static_assert(OFF_ACTA % 128 == 0 && OFF_ACTB % 128 == 0 && OFF_W2 % 128 == 0 && OFF_W3 % 128 == 0 &&
                  OFF_W4 % 128 == 0,
              "operand bases 128-byte aligned");
static_assert(TC_SMEM <= 227 * 1024, "fits one CTA per SM");
static_assert(TC_LBO_ACT < (1u << 18), "descriptor offsets are 14 bits of 16-byte units");

__device__ __forceinline__ uint32_t s_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: K-major, no swizzle, core matrices of
// 8 rows x 16 bytes; lbo = bytes between K-adjacent core matrices, sbo =
// bytes between M/N-adjacent ones.
__device__ __forceinline__ uint64_t mat_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, shape M x N.
__host__ __device__ constexpr uint32_t instr_desc(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile("{ .reg .pred p; setp.ne.b32 p, %4, 0; tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(
                     tmem),
                 "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(s_addr(bar))
                 : "memory");
}

__device__ __forceinline__ bool bar_wait(uint64_t* bar, uint32_t parity, long long limit)
{
    const long long t0 = clock64();
    while (true) {
        uint32_t ok;
        asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                     : "=r"(ok)
                     : "r"(s_addr(bar)), "r"(parity)
                     : "memory");
        if (ok) return true;
        if (clock64() - t0 > limit) return false;
    }
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
        "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t tmem_ld1(uint32_t taddr)
{
    uint32_t r;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r) : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    return r;
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

// Issues layer l's MMAs, output frame rows l .. TC_F - 1 - l in tiles of 128
// pixels, tile m into TMEM columns m * NOUT, and commits tile m to bars[m].
// The descriptors are formed once; an MMA only adds its operand offset (in
// 16-byte units) to the address field.
template <int CIN, int NOUT>
__device__ __forceinline__ void issue_layer(int l, uint32_t src, uint32_t wsm, uint32_t tmem, uint64_t* bars)
{
    constexpr uint32_t LBO_W = NOUT * 16;
    const int p0 = l * TC_F;
    const int tiles = ((TC_F - 2 * l) * TC_F + 127) / 128;
    const uint32_t idesc = instr_desc(128, NOUT);
    const uint64_t abase = mat_desc(src + (uint32_t)(TC_FS + p0) * 16u, TC_LBO_ACT, 128);
    const uint64_t bbase = mat_desc(wsm, LBO_W, 128);
    for (int m = 0; m < tiles; ++m) {
        const uint64_t am = abase + (uint64_t)(128 * m);  // 128 pixels of 16 bytes
#pragma unroll
        for (int t = 0; t < 9; ++t) {
            constexpr int F = TC_F;
            const int delta = (t / 3 - 1) * F + (t % 3 - 1);
#pragma unroll
            for (int kb = 0; kb < CIN / 16; ++kb) {
                const uint64_t da = am + (uint64_t)(int64_t)(delta + (int)(2 * kb * (TC_LBO_ACT >> 4)));
                const uint64_t db = bbase + (uint64_t)((t * CIN / 8 + 2 * kb) * (LBO_W >> 4));
                mma_f16(tmem + (uint32_t)(m * NOUT), da, db, idesc, (t > 0 || kb > 0) ? 1u : 0u);
            }
        }
        mma_commit(&bars[m]);
    }
}

// x0 = [dx, dy, g, s, c] on the frame at image origin (fy0, fx0), channel
// groups 0 and 1 of `buf`.
__device__ __forceinline__ void stage_x0(uint4* buf, const Samples& S, int n, int fy0, int fx0)
{
    const float* Ln = S.L[n];
    const float* gn = S.g[n];
    const float sv = S.s[n];
    for (int p = threadIdx.x; p < TC_FP; p += TC_THREADS) {
        const int gy = fy0 + p / TC_F, gx = fx0 + p % TC_F;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (gy >= 0 && gy < S.h && gx >= 0 && gx < S.w) {
            const size_t gi = (size_t)gy * S.pitch + gx;
            const float c = __ldg(Ln + gi);
            const float dx = gx + 1 < S.w ? kDiffScale * (__ldg(Ln + gi + 1) - c) : 0.f;
            const float dy = gy + 1 < S.h ? kDiffScale * (__ldg(Ln + gi + S.pitch) - c) : 0.f;
            v.x = pack_bf16x2(dx, dy);
            v.y = pack_bf16x2(__ldg(gn + gi), sv);
            v.z = pack_bf16x2(1.f, 0.f);
        }
        buf[TC_FS + p] = v;
        buf[TC_BP + TC_FS + p] = make_uint4(0u, 0u, 0u, 0u);
    }
}

__global__ void __launch_bounds__(TC_THREADS, 1)
k_surrogate_tc(const __nv_bfloat16* __restrict__ wpad, const float* __restrict__ ppad, Samples S, int* status,
               long long spin_limit)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t bars[9];  // one per M tile, [8]: drain after a timeout
    __shared__ uint32_t tmem_base;
    __shared__ int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    float* bias = reinterpret_cast<float*>(smem + OFF_BIAS);  // b1 | b2 | b3 | b4 at 0, 32, 64, 96

    // weights: global [co][t][ci] -> shared [(t CIN + ci) / 8][co][8]
    {
        auto stage = [&](int l, int off, int nout) {
            const int cin = cin_of(l), cout = cout_of(l), K = 9 * cin;
            __nv_bfloat16* dst = reinterpret_cast<__nv_bfloat16*>(smem + off);
            const __nv_bfloat16* src = wpad + w_offset(l);
            for (int e = tid; e < nout * K; e += TC_THREADS) {
                const int n = e / K, k = e - n * K;
                dst[(k / 8) * nout * 8 + n * 8 + (k % 8)] = n < cout ? src[(size_t)n * K + k] : __float2bfloat16(0.f);
            }
        };
        stage(0, OFF_W1, 32);
        stage(1, OFF_W2, 32);
        stage(2, OFF_W3, 32);
        stage(3, OFF_W4, 16);
        for (int e = tid; e < 128; e += TC_THREADS) {
            const int l = e >> 5, c = e & 31;
            bias[e] = c < cout_of(l) ? ppad[b_offset(l) + c] : 0.f;
        }
    }
    if (tid == 0) {
        for (int i = 0; i < 9; ++i) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s_addr(&bars[i])));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fail = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_addr(&tmem_base)),
                     "r"(TC_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    const uint32_t actA = s_addr(smem + OFF_ACTA), actB = s_addr(smem + OFF_ACTB);
    const uint32_t w1 = s_addr(smem + OFF_W1), w2 = s_addr(smem + OFF_W2), w3 = s_addr(smem + OFF_W3),
                   w4 = s_addr(smem + OFF_W4);
    uint4* bufA = reinterpret_cast<uint4*>(smem + OFF_ACTA);
    uint4* bufB = reinterpret_cast<uint4*>(smem + OFF_ACTB);
    const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;  // this warp's TMEM lane quarter
    const int group = warp >> 2;                                   // handles the M tiles m = group (mod 2)
    uint32_t phases = 0;                                           // parity bit per barrier
    bool failed = false;

    const int tiles_x = (S.w + TC_T - 1) / TC_T, tiles_y = (S.h + TC_T - 1) / TC_T;
    const int per_sample = tiles_x * tiles_y;
    const int n_tiles = per_sample * S.n;
    if ((int)blockIdx.x < n_tiles) {
        const int r = (int)blockIdx.x % per_sample;
        stage_x0(bufA, S, (int)blockIdx.x / per_sample, (r / tiles_x) * TC_T - 4, (r % tiles_x) * TC_T - 4);
    }
    for (int tile = blockIdx.x; tile < n_tiles && !failed; tile += gridDim.x) {
        const int n = tile / per_sample;
        const int r = tile - n * per_sample;
        const int fy0 = (r / tiles_x) * TC_T - 4, fx0 = (r % tiles_x) * TC_T - 4;  // image coords of frame pixel 0
#pragma unroll 1
        for (int l = 1; l <= kLayers; ++l) {
            // the previous writes of the operand become visible to the tensor cores
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
            const bool odd = (l & 1) != 0;  // l = 1, 3: A -> B; l = 2: B -> A; l = 4: B -> global
            uint4* dst = odd ? bufB : bufA;
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t src = odd ? actA : actB;
                if (l == 1)
                    issue_layer<kC0, 32>(l, src, w1, tmem, bars);
                else if (l == 2)
                    issue_layer<kC, 32>(l, src, w2, tmem, bars);
                else if (l == 3)
                    issue_layer<kC, 32>(l, src, w3, tmem, bars);
                else
                    issue_layer<kC, 16>(l, src, w4, tmem, bars);
            }
            if (l == kLayers) {
                // the last layer reads buffer B only: stage the next tile's x0
                // into A while its MMAs run
                const int nt = tile + (int)gridDim.x;
                if (nt < n_tiles) {
                    const int nn = nt / per_sample, rr = nt - nn * per_sample;
                    stage_x0(bufA, S, nn, (rr / tiles_x) * TC_T - 4, (rr % tiles_x) * TC_T - 4);
                }
            }
            const int tiles = ((TC_F - 2 * l) * TC_F + 127) / 128;
            const int p0 = l * TC_F;
            for (int m = group; m < tiles; m += 2) {
                if (!bar_wait(&bars[m], (phases >> m) & 1u, spin_limit)) {
                    if (lane == 0) atomicOr(status, 1);
                    s_fail = 1;
                    break;
                }
                phases ^= 1u << m;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const int p = p0 + 128 * m + 32 * (warp & 3) + lane;  // this thread's frame pixel
                const int py = p / TC_F, px = p - py * TC_F;
                const int gy = fy0 + py, gx = fx0 + px;
                const bool inside = gy >= 0 && gy < S.h && gx >= 0 && gx < S.w && p < TC_FP;
                if (l < kLayers) {
                    uint32_t v[32];
                    tmem_ld32(tmem + lane_base + (uint32_t)(m * 32), v);
                    const float* b = bias + 32 * (l - 1);
#pragma unroll
                    for (int gq = 0; gq < 4; ++gq) {
                        uint4 o;
                        uint32_t* ow = &o.x;
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const int c = 8 * gq + 2 * j;
                            const float a0 = inside ? fmaxf(__uint_as_float(v[c]) + b[c], 0.f) : 0.f;
                            const float a1 = inside ? fmaxf(__uint_as_float(v[c + 1]) + b[c + 1], 0.f) : 0.f;
                            ow[j] = pack_bf16x2(a0, a1);
                        }
                        dst[gq * TC_BP + TC_FS + p] = o;
                    }
                } else {
                    const float z = __uint_as_float(tmem_ld1(tmem + lane_base + (uint32_t)(m * 16))) + bias[96];
                    if (inside && py >= 4 && py < TC_F - 4 && px >= 4 && px < TC_F - 4)
                        S.out[n][(size_t)gy * S.opitch + gx] = S.L[n][(size_t)gy * S.pitch + gx] + kOutScale * z;
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
            if (s_fail) {
                failed = true;
                break;
            }
        }
    }
    if (failed && tid == 0) {
        // every MMA this thread issued completes before the tensor memory goes
        mma_commit(&bars[8]);
        bar_wait(&bars[8], 0, spin_limit);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS));
}

int g_tc_grid = 0;

}  // namespace

cudaError_t configure_surrogate_tc()
{
    cudaError_t e = cudaFuncSetAttribute((const void*)k_surrogate_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         TC_SMEM);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    g_tc_grid = sms;  // one CTA per SM (shared memory), so tensor-memory allocation never waits
    return cudaSuccess;
}

cudaError_t launch_forward_tc(const __nv_bfloat16* wpad, const float* ppad, const Samples& S, int* status,
                              cudaStream_t st)
{
    const int tiles = ((S.w + TC_T - 1) / TC_T) * ((S.h + TC_T - 1) / TC_T) * S.n;
    int grid = g_tc_grid > 0 ? g_tc_grid : 152;
    if (grid > tiles) grid = tiles;
    k_surrogate_tc<<<grid, TC_THREADS, TC_SMEM, st>>>(wpad, ppad, S, status, 1ll << 31);
    return cudaGetLastError();
}

}  // namespace sg
}  // namespace kz
