// k_surrogate_fused.cu -- the whole surrogate network in one persistent
// kernel (inference).  Same contract as the layer kernels of k_surrogate.cu:
// x0 = [dx, dy, g, s, c], three 3x3 conv + ReLU layers of 32 channels, a last
// 3x3 conv to one channel z, L_next = L + z / 256; BF16 operands, FP32
// accumulation, zero padding at the image border.
//
// A CTA computes a 16 x 16 tile of L_next.  It builds x0 on the tile's 24 x 24
// neighbourhood in shared memory, then evaluates layer l on the (16 + 8 - 2l)^2
// pixels the following layers need: no activation ever goes to HBM.  The
// price is recomputation of the halos (about 1.5x the MACs of the layer-wise
// kernels for the hidden layers).  Activations that fall outside the image
// are stored as zeros, which is the zero padding of the next layer.
//
// All four layers' weights and the biases stay resident in shared memory for
// the CTA's lifetime; the CTA walks over tiles with a grid stride.  Two
// activation buffers alternate: x0 -> B, B -> A, A -> B, B -> L_next.
//
// Each layer is an implicit GEMM on mma.sync m16n8k16: M = the region's
// pixels in row-major order (16 per m16 tile, each lane computing its own row
// addresses, so the region width need not be a multiple of 16), N = output
// channels, K = 9 taps x input channels.  Operands are fetched with
// ldmatrix; pixel and weight rows carry 8 BF16 of padding so that the eight
// 16-byte rows of each 8x8 matrix land in distinct bank groups.
#include "kaze_internal.h"
#include "surrogate.h"

namespace kz {
namespace sg {
namespace {

constexpr int FT = 16;               // output tile edge
constexpr int FWARPS = 8;
constexpr int FTHREADS = FWARPS * 32;
constexpr int R0 = FT + 8;           // x0 region edge (24)
constexpr int CS0 = kC0 + 8;         // x0 pixel stride (BF16)
constexpr int CSH = kC + 8;          // hidden pixel stride
constexpr int KS1 = 9 * kC0 + 8;     // weight row strides
constexpr int KSH = 9 * kC + 8;

// shared-memory carve-up (bytes)
constexpr int OFF_W1 = 0;
constexpr int OFF_W2 = OFF_W1 + kC * KS1 * 2;
constexpr int OFF_W3 = OFF_W2 + kC * KSH * 2;
constexpr int OFF_W4 = OFF_W3 + kC * KSH * 2;
constexpr int OFF_B = OFF_W4 + kC4 * KSH * 2;
constexpr int OFF_A = OFF_B + 128 * 4;
constexpr int BUF_A_BYTES = ((R0 * R0 * CS0 > (FT + 4) * (FT + 4) * CSH) ? R0 * R0 * CS0 : (FT + 4) * (FT + 4) * CSH) * 2;
constexpr int OFF_BUFB = OFF_A + BUF_A_BYTES;
constexpr int BUF_B_BYTES = (FT + 6) * (FT + 6) * CSH * 2;
constexpr int FUSED_SMEM = OFF_BUFB + BUF_B_BYTES;
static_assert(OFF_A % 16 == 0 && OFF_BUFB % 16 == 0 && OFF_W2 % 16 == 0 && OFF_W3 % 16 == 0 && OFF_W4 % 16 == 0,
              "16-byte aligned smem regions");

__device__ __forceinline__ unsigned pack2(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<unsigned*>(&v);
}

__device__ __forceinline__ void mma16816(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void ldsm_x4(unsigned (&r)[4], uint32_t addr)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr));
}

__device__ __forceinline__ void ldsm_x2(unsigned& r0, unsigned& r1, uint32_t addr)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];" : "=r"(r0), "=r"(r1) : "r"(addr));
}

// One layer over a region of RW x RW destination pixels whose source region
// (RW + 2)^2 starts one pixel further up-left.  (gy0, gx0): image coordinates
// of the destination region's origin.
template <int CIN, int COUT, int RW, int MW, bool LAST>
__device__ __forceinline__ void layer(const __nv_bfloat16* src, const __nv_bfloat16* wsm, const float* bsm,
                                      __nv_bfloat16* dst, int gy0, int gx0, const Samples& S, int n)
{
    constexpr int SW = RW + 2;
    constexpr int CSI = CIN + 8, CSO = COUT + 8;
    constexpr int KS = 9 * CIN + 8;
    constexpr int NPX = RW * RW;
    constexpr int NM = (NPX + 15) / 16;
    constexpr int NB = COUT / 8;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gid = lane >> 2, tig = lane & 3;
    const uint32_t src_s = (uint32_t)__cvta_generic_to_shared(src);
    const uint32_t w_s = (uint32_t)__cvta_generic_to_shared(wsm);
    // B operand rows: matrix (lane >> 3) of an n16 x k16 block
    const int bm = lane >> 3;
    const uint32_t b_lane = w_s + (uint32_t)((((bm >> 1) * 8 + (lane & 7)) * KS + (bm & 1) * 8) * 2);

    for (int base = warp * MW; base < NM; base += FWARPS * MW) {
        float acc[MW][NB][4];
        uint32_t a_lane[MW];
#pragma unroll
        for (int i = 0; i < MW; ++i) {
#pragma unroll
            for (int nb = 0; nb < NB; ++nb)
#pragma unroll
                for (int r = 0; r < 4; ++r) acc[i][nb][r] = 0.f;
            int q = (base + i) * 16 + (lane & 15);
            q = q < NPX ? q : NPX - 1;  // rows past the region compute garbage that is not stored
            const int qy = q / RW, qx = q - qy * RW;
            a_lane[i] = src_s + (uint32_t)(((qy * SW + qx) * CSI + (lane >> 4) * 8) * 2);
        }
#pragma unroll
        for (int t = 0; t < 9; ++t) {
            const uint32_t tap = (uint32_t)((((t / 3) * SW + (t % 3)) * CSI) * 2);
#pragma unroll
            for (int c0 = 0; c0 < CIN; c0 += 16) {
                unsigned b[NB][2];
                if constexpr (NB == 1) {
                    ldsm_x2(b[0][0], b[0][1], b_lane + (uint32_t)((t * CIN + c0) * 2));
                } else {
#pragma unroll
                    for (int p = 0; p < NB / 2; ++p) {
                        unsigned r[4];
                        ldsm_x4(r, b_lane + (uint32_t)(((p * 16) * KS + t * CIN + c0) * 2));
                        b[2 * p][0] = r[0];
                        b[2 * p][1] = r[1];
                        b[2 * p + 1][0] = r[2];
                        b[2 * p + 1][1] = r[3];
                    }
                }
#pragma unroll
                for (int i = 0; i < MW; ++i) {
                    unsigned a[4];
                    ldsm_x4(a, a_lane[i] + tap + (uint32_t)(c0 * 2));
#pragma unroll
                    for (int nb = 0; nb < NB; ++nb) mma16816(acc[i][nb], a, b[nb][0], b[nb][1]);
                }
            }
        }
        // epilogue: accumulator rows gid / gid + 8 of m16 tile base + i
#pragma unroll
        for (int i = 0; i < MW; ++i) {
            if (base + i >= NM) break;
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                const int q = (base + i) * 16 + gid + 8 * half;
                if (q >= NPX) continue;
                const int qy = q / RW, qx = q - qy * RW;
                const int gy = gy0 + qy, gx = gx0 + qx;
                const bool inside = gy >= 0 && gy < S.h && gx >= 0 && gx < S.w;
                if constexpr (!LAST) {
#pragma unroll
                    for (int nb = 0; nb < NB; ++nb) {
                        const int co = nb * 8 + 2 * tig;
                        const float v0 = inside ? fmaxf(acc[i][nb][2 * half] + bsm[co], 0.f) : 0.f;
                        const float v1 = inside ? fmaxf(acc[i][nb][2 * half + 1] + bsm[co + 1], 0.f) : 0.f;
                        *reinterpret_cast<unsigned*>(dst + q * CSO + co) = pack2(v0, v1);
                    }
                } else {
                    if (tig == 0 && inside)
                        S.out[n][(size_t)gy * S.opitch + gx] =
                            S.L[n][(size_t)gy * S.pitch + gx] + kOutScale * (acc[i][0][2 * half] + bsm[0]);
                }
            }
        }
    }
}

__global__ void __launch_bounds__(FTHREADS, 1)
k_surrogate_fused(const __nv_bfloat16* __restrict__ wpad, const float* __restrict__ ppad, Samples S)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __nv_bfloat16* W1 = reinterpret_cast<__nv_bfloat16*>(smem + OFF_W1);
    __nv_bfloat16* W2 = reinterpret_cast<__nv_bfloat16*>(smem + OFF_W2);
    __nv_bfloat16* W3 = reinterpret_cast<__nv_bfloat16*>(smem + OFF_W3);
    __nv_bfloat16* W4 = reinterpret_cast<__nv_bfloat16*>(smem + OFF_W4);
    float* bs = reinterpret_cast<float*>(smem + OFF_B);  // b1 | b2 | b3 | b4 at 0, 32, 64, 96
    __nv_bfloat16* bufA = reinterpret_cast<__nv_bfloat16*>(smem + OFF_A);
    __nv_bfloat16* bufB = reinterpret_cast<__nv_bfloat16*>(smem + OFF_BUFB);

    // weights: global rows of 9*CIN BF16 -> shared rows of 9*CIN + 8
    {
        __nv_bfloat16* dsts[4] = {W1, W2, W3, W4};
#pragma unroll
        for (int l = 0; l < kLayers; ++l) {
            const int K = 9 * cin_of(l), KS = K + 8, V = K / 8;
            const uint4* src = reinterpret_cast<const uint4*>(wpad + w_offset(l));
            for (int e = threadIdx.x; e < cout_of(l) * V; e += FTHREADS) {
                const int co = e / V, qv = e - co * V;
                *reinterpret_cast<uint4*>(dsts[l] + co * KS + 8 * qv) = src[e];
            }
        }
        for (int e = threadIdx.x; e < 128; e += FTHREADS) {
            const int l = e >> 5, c = e & 31;
            bs[e] = c < cout_of(l) ? ppad[b_offset(l) + c] : 0.f;
        }
    }

    const int tiles_x = (S.w + FT - 1) / FT, tiles_y = (S.h + FT - 1) / FT;
    const int per_sample = tiles_x * tiles_y;
    const int n_tiles = per_sample * S.n;
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int n = tile / per_sample;
        const int r = tile - n * per_sample;
        const int y0 = (r / tiles_x) * FT, x0 = (r % tiles_x) * FT;
        __syncthreads();  // previous tile's readers of bufA are done (and weights staged)
        // x0 on the 24 x 24 neighbourhood, zero outside the image
        {
            const float* Ln = S.L[n];
            const float* gn = S.g[n];
            const float sv = S.s[n];
            for (int e = threadIdx.x; e < R0 * R0; e += FTHREADS) {
                const int ry = e / R0, rx = e - ry * R0;
                const int gy = y0 - 4 + ry, gx = x0 - 4 + rx;
                uint4 v = make_uint4(0u, 0u, 0u, 0u);
                if (gy >= 0 && gy < S.h && gx >= 0 && gx < S.w) {
                    const size_t gi = (size_t)gy * S.pitch + gx;
                    const float c = __ldg(Ln + gi);
                    const float dx = gx + 1 < S.w ? kDiffScale * (__ldg(Ln + gi + 1) - c) : 0.f;
                    const float dy = gy + 1 < S.h ? kDiffScale * (__ldg(Ln + gi + S.pitch) - c) : 0.f;
                    v.x = pack2(dx, dy);
                    v.y = pack2(__ldg(gn + gi), sv);
                    v.z = pack2(1.f, 0.f);
                }
                uint4* o = reinterpret_cast<uint4*>(bufA + e * CS0);
                o[0] = v;
                o[1] = make_uint4(0u, 0u, 0u, 0u);
            }
        }
        __syncthreads();
        layer<kC0, kC, FT + 6, 4, false>(bufA, W1, bs, bufB, y0 - 3, x0 - 3, S, n);
        __syncthreads();
        layer<kC, kC, FT + 4, 4, false>(bufB, W2, bs + 32, bufA, y0 - 2, x0 - 2, S, n);
        __syncthreads();
        layer<kC, kC, FT + 2, 4, false>(bufA, W3, bs + 64, bufB, y0 - 1, x0 - 1, S, n);
        __syncthreads();
        layer<kC, kC4, FT, 2, true>(bufB, W4, bs + 96, nullptr, y0, x0, S, n);
    }
}

int g_fused_grid = 0;

}  // namespace

cudaError_t configure_surrogate_kernels()
{
    cudaError_t e = cudaFuncSetAttribute((const void*)k_surrogate_fused,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, FUSED_SMEM);
    if (e != cudaSuccess) return e;
    if ((e = configure_surrogate_tc()) != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_surrogate_fused, FTHREADS, FUSED_SMEM)) !=
        cudaSuccess)
        return e;
    g_fused_grid = sms * (per_sm > 0 ? per_sm : 1);
    return cudaSuccess;
}

cudaError_t launch_forward_fused(const __nv_bfloat16* wpad, const float* ppad, const Samples& S, cudaStream_t st)
{
    const int tiles = ((S.w + FT - 1) / FT) * ((S.h + FT - 1) / FT) * S.n;
    int grid = g_fused_grid > 0 ? g_fused_grid : 152;
    if (grid > tiles) grid = tiles;
    k_surrogate_fused<<<grid, FTHREADS, FUSED_SMEM, st>>>(wpad, ppad, S);
    return cudaGetLastError();
}

}  // namespace sg
}  // namespace kz
