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
// is an implicit GEMM over the frame pixels of rows l .. 31 - l in tiles of
// M = 128 consecutive pixels (four frame rows).  The three horizontal taps
// of the 3x3 kernel sit in the N dimension: for kernel row ky the A operand
// is the source shifted by (ky - 1) frame rows (the same descriptor with its
// start moved by 32 pixels x 16 bytes) and B holds W[ky, kx, c, :] in row
// kx * C + c, so the accumulator gets
//     D[p, kx C + c] = sum_ky sum_ci W[c, ky, kx, ci] x[p + 32 (ky - 1), ci]
// and the epilogue adds D[p - 1, c] + D[p, C + c] + D[p + 1, 2C + c] with
// warp shuffles: a frame row is exactly one warp's 32 tensor-memory lanes,
// and the lanes a shuffle cannot reach (frame columns 0 and 31) are columns
// no valid output reads (each layer's valid region shrinks by one pixel a
// side).  N = 96 (48 for the last layer, whose channels 1..15 are zero
// weights); an instruction of N = 96 costs little more than one of N = 32,
// so a layer takes a third of the instructions of a tap-by-tap GEMM.
//
// Warp roles: warp 16 allocates 512 columns of tensor memory and one of its
// threads issues every MMA into a ring of five 96-column slots, committing
// each M tile to the slot's "full" barrier; warps 0-15 (four groups of four
// taking every fourth tile, each warp its quarter of the 128 lanes) read a full
// slot (tcgen05.ld), release it on its "empty" barrier, add bias and ReLU,
// zero the padding outside the image and write the next layer's operand (or
// L_next).  A layer's MMAs start once every epilogue warp has finished the
// previous layer ("layer" barrier, with a proxy fence for the tensor
// cores' view of shared memory); the next frame's input is staged while the
// last layer computes.  All weights stay in shared memory for the CTA's
// life.  Every wait is bounded: on a timeout the kernel raises bit 0 of
// *status, every warp leaves its loop, the MMAs are drained (bounded) and
// the tensor memory is freed before the kernel returns.
#include "kaze_internal.h"
#include "surrogate.h"

namespace kz {
namespace sg {
namespace {

constexpr int TC_T = 24;                  // output tile edge
constexpr int TC_F = TC_T + 8;            // frame edge (32)
constexpr int TC_FP = TC_F * TC_F;        // frame pixels (1024)
constexpr int TC_FS = 64;                 // front slack pixels (operands start up to 32 before)
constexpr int TC_BP = TC_FS + TC_FP + 192;  // pixels per channel group incl. slack (1280)
constexpr int TC_EPI_WARPS = 16;           // four groups of four
constexpr int TC_GROUPS = TC_EPI_WARPS / 4;
constexpr int TC_THREADS = 32 * (TC_EPI_WARPS + 1);
constexpr int TC_SLOTS = 5;               // tensor-memory ring
constexpr int TC_SLOT_COLS = 96;
constexpr int TC_TMEM_COLS = 512;
constexpr uint32_t TC_LBO_ACT = TC_BP * 16;   // bytes between channel groups of an activation buffer
static_assert(TC_SLOTS * TC_SLOT_COLS <= TC_TMEM_COLS, "ring fits the allocation");
static_assert(TC_SLOTS > TC_GROUPS, "every group can hold a slot while the next tile fills");

// weight buffers: per kernel row ky, [CIN/8][N][8] BF16 with N = 3 C
constexpr int W1_BYTES = 3 * (kC0 / 8) * 96 * 16;
constexpr int WH_BYTES = 3 * (kC / 8) * 96 * 16;
constexpr int W4_BYTES = 3 * (kC / 8) * 48 * 16;
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

__device__ __forceinline__ void bar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(s_addr(bar)) : "memory");
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

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* r)
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

// bar_wait for a whole warp: one lane polls, then every lane observes the
// completed phase itself (acquire for each thread).  Same result in all lanes.
__device__ __forceinline__ bool warp_bar_wait(uint64_t* bar, uint32_t parity, long long limit, int lane)
{
    bool ok = true;
    if (lane == 0) ok = bar_wait(bar, parity, limit);
    ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
    if (ok) ok = bar_wait(bar, parity, limit);
    return __all_sync(0xffffffffu, ok);
}

__device__ __forceinline__ uint32_t tmem_ld1(uint32_t taddr)
{
    uint32_t r;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r) : "r"(taddr));
    return r;
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ int tiles_of(int l) { return ((TC_F - 2 * l) * TC_F + 127) / 128; }

// Shared state of the CTA's barriers.
struct TcBars {
    uint64_t full[TC_SLOTS];   // MMA -> epilogue: slot holds a finished tile
    uint64_t empty[TC_SLOTS];  // epilogue -> MMA: slot read out (4 warps)
    uint64_t layer;            // epilogue -> MMA: a layer's outputs are written (8 warps)
    uint64_t drain;            // MMAs finished before the tensor memory is freed
};

// Issues layer l's MMAs: output frame rows l .. TC_F - 1 - l in tiles of 128
// pixels; global tile T goes to slot T % TC_SLOTS once the slot's previous
// tile has been read out.  Returns false if a wait ran out.
template <int CIN, int NW>
__device__ __forceinline__ bool issue_layer(int l, uint32_t src, uint32_t wsm, uint32_t tmem, TcBars& b,
                                            uint32_t& T, long long limit)
{
    constexpr uint32_t LBO_W = NW * 16;
    constexpr uint32_t KY_BYTES = (CIN / 8) * NW * 16;
    const uint32_t idesc = instr_desc(128, NW);
    const uint32_t a0 = src + (uint32_t)(TC_FS + l * TC_F - TC_F) * 16u;  // tile 0, kernel row 0
    const uint64_t abase = mat_desc(a0, TC_LBO_ACT, 128);
    const uint64_t bbase = mat_desc(wsm, LBO_W, 128);
    const int tiles = tiles_of(l);
    for (int m = 0; m < tiles; ++m, ++T) {
        const uint32_t slot = T % TC_SLOTS, use = T / TC_SLOTS;
        if (use > 0 && !bar_wait(&b.empty[slot], (use - 1) & 1u, limit)) return false;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d = tmem + slot * TC_SLOT_COLS;
#pragma unroll
        for (int ky = 0; ky < 3; ++ky) {
            // 128 pixels per tile and one frame row per kernel row, 16 bytes each
            const uint64_t am = abase + (uint64_t)(8 * m + 2 * ky) * 16u;
#pragma unroll
            for (int kb = 0; kb < CIN / 16; ++kb) {
                const uint64_t da = am + (uint64_t)(2 * kb * (TC_LBO_ACT >> 4));
                const uint64_t db = bbase + (uint64_t)((ky * KY_BYTES + 2 * kb * LBO_W) >> 4);
                mma_f16(d, da, db, idesc, (ky > 0 || kb > 0) ? 1u : 0u);
            }
        }
        mma_commit(&b.full[slot]);
    }
    return true;
}

// x0 = [dx, dy, g, s, c] on the frame at image origin (fy0, fx0), channel
// groups 0 and 1 of `buf`, written by the 256 epilogue threads.
__device__ __forceinline__ void stage_x0(uint4* buf, const Samples& S, int n, int fy0, int fx0, int et)
{
    const float* Ln = S.L[n];
    const float* gn = S.g[n];
    const float sv = S.s[n];
    for (int p = et; p < TC_FP; p += 32 * TC_EPI_WARPS) {
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
    __shared__ __align__(8) TcBars bars;
    __shared__ uint32_t tmem_base;
    __shared__ volatile int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    float* bias = reinterpret_cast<float*>(smem + OFF_BIAS);  // b1 | b2 | b3 | b4 at 0, 32, 64, 96

    // weights: global [co][t][ci] -> shared, per kernel row ky: [ci / 8][kx C + co][8]
    {
        auto stage = [&](int l, int off, int C) {
            const int cin = cin_of(l), cout = cout_of(l), K = 9 * cin, NW = 3 * C;
            __nv_bfloat16* dst = reinterpret_cast<__nv_bfloat16*>(smem + off);
            const __nv_bfloat16* src = wpad + w_offset(l);
            for (int e = tid; e < NW * 3 * cin; e += TC_THREADS) {
                const int n = e / (3 * cin), rest = e - n * (3 * cin);
                const int ky = rest / cin, ci = rest - ky * cin;
                const int kx = n / C, c = n - kx * C, t = 3 * ky + kx;
                dst[ky * (cin / 8) * NW * 8 + (ci / 8) * NW * 8 + n * 8 + (ci % 8)] =
                    c < cout ? src[(size_t)c * K + t * cin + ci] : __float2bfloat16(0.f);
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
        for (int i = 0; i < TC_SLOTS; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s_addr(&bars.full[i])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(s_addr(&bars.empty[i])));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s_addr(&bars.layer)), "r"(TC_EPI_WARPS));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s_addr(&bars.drain)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fail = 0;
    }
    if (warp == TC_EPI_WARPS) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_addr(&tmem_base)),
                     "r"(TC_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }

    const int tiles_x = (S.w + TC_T - 1) / TC_T, tiles_y = (S.h + TC_T - 1) / TC_T;
    const int per_sample = tiles_x * tiles_y;
    const int n_tiles = per_sample * S.n;
    uint4* bufA = reinterpret_cast<uint4*>(smem + OFF_ACTA);
    uint4* bufB = reinterpret_cast<uint4*>(smem + OFF_ACTB);
    if (warp < TC_EPI_WARPS && (int)blockIdx.x < n_tiles) {
        const int r = (int)blockIdx.x % per_sample;
        stage_x0(bufA, S, (int)blockIdx.x / per_sample, (r / tiles_x) * TC_T - 4, (r % tiles_x) * TC_T - 4, tid);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    const uint32_t actA = s_addr(smem + OFF_ACTA), actB = s_addr(smem + OFF_ACTB);

    if (warp == TC_EPI_WARPS) {
        // ---- MMA issuer ----
        if (lane == 0) {
            const uint32_t w1 = s_addr(smem + OFF_W1), w2 = s_addr(smem + OFF_W2), w3 = s_addr(smem + OFF_W3),
                           w4 = s_addr(smem + OFF_W4);
            uint32_t T = 0, layers_seen = 0;
            bool first = true;
            for (int tile = blockIdx.x; tile < n_tiles && !s_fail; tile += gridDim.x) {
                for (int l = 1; l <= kLayers; ++l) {
                    if (!first) {
                        if (!bar_wait(&bars.layer, layers_seen & 1u, spin_limit)) {
                            atomicOr(status, 1);
                            s_fail = 1;
                            break;
                        }
                        ++layers_seen;
                    }
                    first = false;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    bool ok;
                    if (l == 1)
                        ok = issue_layer<kC0, 96>(l, actA, w1, tmem, bars, T, spin_limit);
                    else if (l == 2)
                        ok = issue_layer<kC, 96>(l, actB, w2, tmem, bars, T, spin_limit);
                    else if (l == 3)
                        ok = issue_layer<kC, 96>(l, actA, w3, tmem, bars, T, spin_limit);
                    else
                        ok = issue_layer<kC, 48>(l, actB, w4, tmem, bars, T, spin_limit);
                    if (!ok) {
                        atomicOr(status, 1);
                        s_fail = 1;
                        break;
                    }
                }
            }
            // every MMA issued by this thread completes before the memory goes
            mma_commit(&bars.drain);
            bar_wait(&bars.drain, 0, spin_limit);
        }
        __syncwarp();
    } else {
        // ---- epilogue warps ----
        const int group = warp >> 2;  // handles the M tiles T = group (mod TC_GROUPS)
        const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;  // this warp's TMEM lane quarter
        uint32_t T = 0;
        int frame = 0;
        for (int tile = blockIdx.x; tile < n_tiles && !s_fail; tile += gridDim.x, ++frame) {
            const int n = tile / per_sample;
            const int r = tile - n * per_sample;
            const int fy0 = (r / tiles_x) * TC_T - 4, fx0 = (r % tiles_x) * TC_T - 4;  // image coords of pixel 0
            for (int l = 1; l <= kLayers && !s_fail; ++l) {
                uint4* dst = (l & 1) ? bufB : bufA;  // l = 1, 3: A -> B; l = 2: B -> A; l = 4: B -> L_next
                const int tiles = tiles_of(l);
                const int p0 = l * TC_F;
                for (int m = 0; m < tiles; ++m, ++T) {
                    if ((int)(T % TC_GROUPS) != group) continue;
                    const uint32_t slot = T % TC_SLOTS, use = T / TC_SLOTS;
                    if (!warp_bar_wait(&bars.full[slot], use & 1u, spin_limit, lane)) {
                        if (lane == 0) atomicOr(status, 1);
                        s_fail = 1;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t ta = tmem + lane_base + slot * TC_SLOT_COLS;
                    const int p = p0 + 128 * m + 32 * (warp & 3) + lane;  // this thread's frame pixel
                    const int py = p / TC_F, px = p - py * TC_F;
                    const int gy = fy0 + py, gx = fx0 + px;
                    const bool inside = gy >= 0 && gy < S.h && gx >= 0 && gx < S.w && p < TC_FP;
                    if (l < kLayers) {
                        // two halves of 16 channels: D[p - 1, c], D[p, 32 + c], D[p + 1, 64 + c]
                        const float* bb = bias + 32 * (l - 1);
#pragma unroll
                        for (int hf = 0; hf < 2; ++hf) {
                            uint32_t v[48];
                            tmem_ld16(ta + 16 * hf, v);
                            tmem_ld16(ta + 32 + 16 * hf, v + 16);
                            tmem_ld16(ta + 64 + 16 * hf, v + 32);
                            tmem_wait_ld();
                            if (hf == 1) {
                                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                                __syncwarp();
                                if (lane == 0) bar_arrive(&bars.empty[slot]);
                            }
#pragma unroll
                            for (int gq = 0; gq < 2; ++gq) {
                                uint4 o;
                                uint32_t* ow = &o.x;
#pragma unroll
                                for (int j = 0; j < 4; ++j) {
                                    const int c = 8 * gq + 2 * j;  // channel 16 hf + c
                                    const float s0 = __shfl_up_sync(0xffffffffu, __uint_as_float(v[c]), 1) +
                                                     __uint_as_float(v[16 + c]) +
                                                     __shfl_down_sync(0xffffffffu, __uint_as_float(v[32 + c]), 1);
                                    const float s1 = __shfl_up_sync(0xffffffffu, __uint_as_float(v[c + 1]), 1) +
                                                     __uint_as_float(v[17 + c]) +
                                                     __shfl_down_sync(0xffffffffu, __uint_as_float(v[33 + c]), 1);
                                    // ReLU after the BF16 rounding (the same values: rounding
                                    // keeps signs), one select per packed pair
                                    __nv_bfloat162 pr = __floats2bfloat162_rn(s0 + bb[16 * hf + c],
                                                                              s1 + bb[16 * hf + c + 1]);
                                    pr = __hmax2(pr, __floats2bfloat162_rn(0.f, 0.f));
                                    ow[j] = inside ? *reinterpret_cast<uint32_t*>(&pr) : 0u;
                                }
                                dst[(2 * hf + gq) * TC_BP + TC_FS + p] = o;
                            }
                        }
                    } else {
                        const uint32_t z0 = tmem_ld1(ta), z1 = tmem_ld1(ta + 16), z2 = tmem_ld1(ta + 32);
                        tmem_wait_ld();
                        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                        __syncwarp();
                        if (lane == 0) bar_arrive(&bars.empty[slot]);
                        const float z = __shfl_up_sync(0xffffffffu, __uint_as_float(z0), 1) + __uint_as_float(z1) +
                                        __shfl_down_sync(0xffffffffu, __uint_as_float(z2), 1) + bias[96];
                        if (inside && py >= 4 && py < TC_F - 4 && px >= 4 && px < TC_F - 4)
                            S.out[n][(size_t)gy * S.opitch + gx] = S.L[n][(size_t)gy * S.pitch + gx] + kOutScale * z;
                    }
                }
                // this warp's writes of the layer become visible to the tensor cores
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) bar_arrive(&bars.layer);
                if (l == 3 && !s_fail) {
                    // layer 3 read buffer A: once every warp is past it, stage the
                    // next frame's input there while layer 4 runs on buffer B
                    if (!warp_bar_wait(&bars.layer, (uint32_t)(4 * frame + 2) & 1u, spin_limit, lane)) {
                        if (lane == 0) atomicOr(status, 1);
                        s_fail = 1;
                        break;
                    }
                    const int nt = tile + (int)gridDim.x;
                    if (nt < n_tiles) {
                        const int nn = nt / per_sample, rr = nt - nn * per_sample;
                        stage_x0(bufA, S, nn, (rr / tiles_x) * TC_T - 4, (rr % tiles_x) * TC_T - 4, tid);
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == TC_EPI_WARPS)
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
