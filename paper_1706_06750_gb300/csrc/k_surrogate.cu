// k_surrogate.cu -- layer kernels of the learned AOS surrogate: features,
// convolution forward, input gradient (dX), weight gradient (dW), loss,
// deterministic reductions and Adam.
//
// The surrogate is not in the paper: it stands in for one AOS step (Eq. 4).
// Network and precision contract:
//   x0 = [dx, dy, g, s, c], BF16: dx = 16 (L[y][x+1] - L[y][x]) and
//        dy = 16 (L[y+1][x] - L[y][x]) (0 in the last column / row),
//        s = log(1 + tau)/5, c = 1 inside the image;
//   h_l = relu(conv3x3(h_{l-1}) + b_l) for l = 1..3, BF16, 32 channels;
//   z = conv3x3(h3) + b4;  L_next = L + z / 256 (FP32).
// Convolutions pad with zeros.  Weights are BF16 copies of FP32 masters,
// biases FP32, every product is accumulated in FP32 by the tensor cores.
//
// Tensor cores: each convolution is an implicit GEMM on mma.sync m16n8k16
// (BF16 operands, FP32 accumulators).
//   forward  M = pixels (a row of 16 pixels per m16 tile), N = output
//            channels, K = 9 taps x input channels;
//   dX       the same GEMM with mirrored taps and transposed weights; the
//            ReLU derivative of the layer below is applied in its epilogue;
//   dW       M = output channels, N = taps x input channels, K = pixels.
// A CTA owns a tile of 8 x 16 pixels (4 warps, 2 pixel rows each).  Its input
// tile with a one-pixel halo and the layer's weights are staged in shared
// memory with 8 BF16 of padding per pixel / weight row, which spreads the
// fragment loads of a warp over all 32 banks.
#include <math.h>

#include "kaze_internal.h"
#include "surrogate.h"

namespace kz {
namespace sg {
namespace {

constexpr int TH = 8, TW = 16;  // pixel tile
constexpr int NT = 128;         // threads per CTA
constexpr int HALO = (TH + 2) * (TW + 2);

__device__ __forceinline__ unsigned pack_bf16(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<unsigned*>(&v);
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ unsigned ld32(const __nv_bfloat16* p) { return *reinterpret_cast<const unsigned*>(p); }

__device__ __forceinline__ unsigned ld2x16(const __nv_bfloat16* p0, const __nv_bfloat16* p1)
{
    const unsigned short lo = *reinterpret_cast<const unsigned short*>(p0);
    const unsigned short hi = *reinterpret_cast<const unsigned short*>(p1);
    return (unsigned)lo | ((unsigned)hi << 16);
}

// Stages the halo tile (TH+2) x (TW+2) of an NHWC BF16 tensor with C
// channels into shared memory with a pixel stride of C + 8 (zero outside the
// image).
template <int C>
__device__ void stage_halo(const __nv_bfloat16* __restrict__ src, __nv_bfloat16* tile, int n, int w, int h, int y0,
                           int x0)
{
    constexpr int V = C / 8;  // 16-byte vectors per pixel
    constexpr int CS = C + 8;
    const __nv_bfloat16* base = src + (size_t)n * h * w * C;
    for (int e = threadIdx.x; e < HALO * V; e += NT) {
        const int hp = e / V, q = e - hp * V;
        const int ty = hp / (TW + 2), tx = hp - ty * (TW + 2);
        const int y = y0 + ty - 1, x = x0 + tx - 1;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (y >= 0 && y < h && x >= 0 && x < w)
            v = *reinterpret_cast<const uint4*>(base + ((size_t)y * w + x) * C + 8 * q);
        *reinterpret_cast<uint4*>(tile + (size_t)hp * CS + 8 * q) = v;
    }
}

// ------------------------------------------------------------- features --
__global__ void k_features(Samples S, __nv_bfloat16* __restrict__ x0)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    const int n = blockIdx.z;
    if (x >= S.w) return;
    const float* Ln = S.L[n];
    const size_t gi = (size_t)y * S.pitch + x;
    const float c = Ln[gi];
    const float dx = x + 1 < S.w ? kDiffScale * (Ln[gi + 1] - c) : 0.f;
    const float dy = y + 1 < S.h ? kDiffScale * (Ln[gi + S.pitch] - c) : 0.f;
    uint4 lo;
    lo.x = pack_bf16(dx, dy);
    lo.y = pack_bf16(S.g[n][gi], S.s[n]);
    lo.z = pack_bf16(1.f, 0.f);
    lo.w = 0u;
    uint4* o = reinterpret_cast<uint4*>(x0 + (((size_t)n * S.h + y) * S.w + x) * kC0);
    o[0] = lo;
    o[1] = make_uint4(0u, 0u, 0u, 0u);
}

// ------------------------------------------------------------- forward --
// MODE 0: out = relu(conv + b) as BF16 NHWC.  MODE 1 (last layer):
// S.out[n] = S.L[n] + (conv + b)[channel 0] / 256, FP32.
template <int CIN, int COUT, int MODE>
__global__ void __launch_bounds__(NT)
k_conv_fwd(const __nv_bfloat16* __restrict__ in, const __nv_bfloat16* __restrict__ wgt,
           const float* __restrict__ bias, __nv_bfloat16* __restrict__ out, Samples S)
{
    constexpr int K = 9 * CIN;
    constexpr int KS = K + 8;  // weight row stride
    constexpr int CS = CIN + 8;
    constexpr int NB = COUT / 8;
    __shared__ __align__(16) __nv_bfloat16 s_in[HALO * CS];
    __shared__ __align__(16) __nv_bfloat16 s_w[COUT * KS];
    const int w = S.w, h = S.h;
    const int n = blockIdx.z;
    const int y0 = blockIdx.y * TH, x0 = blockIdx.x * TW;
    stage_halo<CIN>(in, s_in, n, w, h, y0, x0);
    for (int e = threadIdx.x; e < COUT * K / 8; e += NT) {
        const int co = e / (K / 8), q = e - co * (K / 8);
        *reinterpret_cast<uint4*>(s_w + (size_t)co * KS + 8 * q) = reinterpret_cast<const uint4*>(wgt)[e];
    }
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gid = lane >> 2, tig = lane & 3;
    float acc[2][NB][4];
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int nb = 0; nb < NB; ++nb)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[mi][nb][r] = 0.f;

#pragma unroll
    for (int t = 0; t < 9; ++t) {
        const int ky = t / 3, kx = t % 3;
#pragma unroll
        for (int c0 = 0; c0 < CIN; c0 += 16) {
            unsigned b[NB][2];
#pragma unroll
            for (int nb = 0; nb < NB; ++nb) {
                const __nv_bfloat16* wr = s_w + (size_t)(nb * 8 + gid) * KS + t * CIN + c0 + 2 * tig;
                b[nb][0] = ld32(wr);
                b[nb][1] = ld32(wr + 8);
            }
#pragma unroll
            for (int mi = 0; mi < 2; ++mi) {
                const int ty = 2 * warp + mi;  // tile row of this m16 tile
                const __nv_bfloat16* r0 = s_in + ((size_t)(ty + ky) * (TW + 2) + gid + kx) * CS + c0 + 2 * tig;
                const __nv_bfloat16* r1 = r0 + 8 * CS;  // pixel gid + 8
                unsigned a[4] = {ld32(r0), ld32(r1), ld32(r0 + 8), ld32(r1 + 8)};
#pragma unroll
                for (int nb = 0; nb < NB; ++nb) mma_bf16(acc[mi][nb], a, b[nb][0], b[nb][1]);
            }
        }
    }
    // accumulator rows gid / gid + 8 = pixels x0 + gid / x0 + gid + 8
#pragma unroll
    for (int mi = 0; mi < 2; ++mi) {
        const int y = y0 + 2 * warp + mi;
        if (y >= h) continue;
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int x = x0 + gid + 8 * half;
            if (x >= w) continue;
            if (MODE == 0) {
                __nv_bfloat16* o = out + (((size_t)n * h + y) * w + x) * COUT;
#pragma unroll
                for (int nb = 0; nb < NB; ++nb) {
                    const int co = nb * 8 + 2 * tig;
                    const float v0 = fmaxf(acc[mi][nb][2 * half] + bias[co], 0.f);
                    const float v1 = fmaxf(acc[mi][nb][2 * half + 1] + bias[co + 1], 0.f);
                    *reinterpret_cast<unsigned*>(o + co) = pack_bf16(v0, v1);
                }
            } else if (tig == 0) {  // output channel 0 sits in the lanes with tig 0
                S.out[n][(size_t)y * S.opitch + x] =
                    S.L[n][(size_t)y * S.pitch + x] + kOutScale * (acc[mi][0][2 * half] + bias[0]);
            }
        }
    }
}

// ---------------------------------------------------------------- loss ---
// dz4 channel 0 = dloss/dz = 2 (L_next - T) / (256 count), channels 1..7 = 0; each CTA writes
// the sum of its squared errors to partials[cta].
__global__ void k_loss(Samples S, __nv_bfloat16* __restrict__ dz, double* __restrict__ partials, float scale)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, n = blockIdx.z;
    double sq = 0.0;
    if (x < S.w) {
        const float e = S.out[n][(size_t)y * S.opitch + x] - S.T[n][(size_t)y * S.pitch + x];
        sq = (double)e * (double)e;
        const uint4 v = make_uint4(pack_bf16(scale * e, 0.f), 0u, 0u, 0u);
        *reinterpret_cast<uint4*>(dz + (((size_t)n * S.h + y) * S.w + x) * kC4) = v;
    }
    __shared__ double s_part[4];
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = sq;
    __syncthreads();
    if (threadIdx.x == 0) {
        const size_t b = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        partials[b] = ((s_part[0] + s_part[1]) + s_part[2]) + s_part[3];
    }
}

// Sums partials[0..count) in a fixed order into *out (scaled).
__global__ void k_sum_partials(const double* __restrict__ partials, int count, double scale, double* __restrict__ out)
{
    __shared__ double s[256];
    double a = 0.0;
    for (int i = threadIdx.x; i < count; i += 256) a += partials[i];
    s[threadIdx.x] = a;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = s[0] * scale;
}

// ----------------------------------------------------------------- dX ----
// dact[p][ci] = relu'(act[p][ci]) * sum_{t, co} W[co][t][ci] dz[p - off(t)][co]:
// the convolution of dz with the mirrored taps and the transposed weights
// (zero outside the image).  act is the layer input, itself a ReLU output.
template <int CIN, int COUT>
__global__ void __launch_bounds__(NT)
k_conv_dx(const __nv_bfloat16* __restrict__ dz, const __nv_bfloat16* __restrict__ wgt,
          const __nv_bfloat16* __restrict__ act, __nv_bfloat16* __restrict__ dact, int w, int h)
{
    constexpr int NB = CIN / 8;
    constexpr int CP = COUT < 16 ? 16 : COUT;  // dz channels per pixel, padded to k16
    constexpr int CS = CP + 8;
    constexpr int KP = 9 * CP;
    constexpr int KS = KP + 8;
    __shared__ __align__(16) __nv_bfloat16 s_dz[HALO * CS];
    __shared__ __align__(16) __nv_bfloat16 s_wt[CIN * KS];  // [ci][t'][co]
    const int n = blockIdx.z;
    const int y0 = blockIdx.y * TH, x0 = blockIdx.x * TW;
    {
        const __nv_bfloat16* base = dz + (size_t)n * h * w * COUT;
        for (int e = threadIdx.x; e < HALO * (CP / 8); e += NT) {
            const int hp = e / (CP / 8), q = e - hp * (CP / 8);
            const int ty = hp / (TW + 2), tx = hp - ty * (TW + 2);
            const int y = y0 + ty - 1, x = x0 + tx - 1;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (8 * q < COUT && y >= 0 && y < h && x >= 0 && x < w)
                v = *reinterpret_cast<const uint4*>(base + ((size_t)y * w + x) * COUT + 8 * q);
            *reinterpret_cast<uint4*>(s_dz + (size_t)hp * CS + 8 * q) = v;
        }
    }
    // s_wt[ci][t'][co] = W[co][8 - t'][ci]: tap t' reads dz at p + off(t')
    for (int e = threadIdx.x; e < CIN * KP; e += NT) {
        const int ci = e / KP, rem = e - ci * KP, tp = rem / CP, co = rem - tp * CP;
        s_wt[(size_t)ci * KS + rem] =
            co < COUT ? wgt[((size_t)co * 9 + (8 - tp)) * CIN + ci] : __float2bfloat16(0.f);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gid = lane >> 2, tig = lane & 3;
    float acc[2][NB][4];
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int nb = 0; nb < NB; ++nb)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[mi][nb][r] = 0.f;
#pragma unroll
    for (int t = 0; t < 9; ++t) {
        const int ky = t / 3, kx = t % 3;
#pragma unroll
        for (int c0 = 0; c0 < CP; c0 += 16) {
            unsigned b[NB][2];
#pragma unroll
            for (int nb = 0; nb < NB; ++nb) {
                const __nv_bfloat16* wr = s_wt + (size_t)(nb * 8 + gid) * KS + t * CP + c0 + 2 * tig;
                b[nb][0] = ld32(wr);
                b[nb][1] = ld32(wr + 8);
            }
#pragma unroll
            for (int mi = 0; mi < 2; ++mi) {
                const int ty = 2 * warp + mi;
                const __nv_bfloat16* r0 = s_dz + ((size_t)(ty + ky) * (TW + 2) + gid + kx) * CS + c0 + 2 * tig;
                const __nv_bfloat16* r1 = r0 + 8 * CS;
                unsigned a[4] = {ld32(r0), ld32(r1), ld32(r0 + 8), ld32(r1 + 8)};
#pragma unroll
                for (int nb = 0; nb < NB; ++nb) mma_bf16(acc[mi][nb], a, b[nb][0], b[nb][1]);
            }
        }
    }
#pragma unroll
    for (int mi = 0; mi < 2; ++mi) {
        const int y = y0 + 2 * warp + mi;
        if (y >= h) continue;
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int x = x0 + gid + 8 * half;
            if (x >= w) continue;
            const size_t pi = (((size_t)n * h + y) * w + x) * CIN;
#pragma unroll
            for (int nb = 0; nb < NB; ++nb) {
                const int ci = nb * 8 + 2 * tig;
                const __nv_bfloat162 av = *reinterpret_cast<const __nv_bfloat162*>(act + pi + ci);
                const float m0 = __low2float(av) > 0.f ? 1.f : 0.f;
                const float m1 = __high2float(av) > 0.f ? 1.f : 0.f;
                *reinterpret_cast<unsigned*>(dact + pi + ci) =
                    pack_bf16(acc[mi][nb][2 * half] * m0, acc[mi][nb][2 * half + 1] * m1);
            }
        }
    }
}

// ----------------------------------------------------------------- dW ----
// partial[cta][co][t][ci] = sum over the CTA's tiles of dz[p][co] x[p + off(t)][ci]
// and partial[cta][COUT*9*CIN + co] = sum of dz[p][co]; tiles are dealt to
// the kDwCtas CTAs round-robin, so the sums are reproducible.
template <int CIN, int COUT>
__global__ void __launch_bounds__(NT)
k_conv_dw(const __nv_bfloat16* __restrict__ dz, const __nv_bfloat16* __restrict__ x, float* __restrict__ partial,
          int w, int h, int n_samples)
{
    constexpr int NCOL = 9 * CIN;                   // GEMM N
    constexpr int MT = COUT < 16 ? 1 : COUT / 16;   // m16 tiles (COUT 8: half of one)
    constexpr int NB_ALL = NCOL / 8;
    constexpr int NBW = (NB_ALL + 3) / 4;           // n8 tiles per warp
    constexpr int CS = CIN + 8;
    constexpr int DS = TH * TW + 8;                 // s_dzt row stride
    constexpr int NPAR = COUT * NCOL + COUT;
    __shared__ __align__(16) __nv_bfloat16 s_dzt[16 * MT * DS];  // [co][pixel]
    __shared__ __align__(16) __nv_bfloat16 s_x[HALO * CS];
    __shared__ float s_db[16 * MT];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gid = lane >> 2, tig = lane & 3;
    const int tiles_x = (w + TW - 1) / TW, tiles_y = (h + TH - 1) / TH;
    const int n_tiles = tiles_x * tiles_y * n_samples;
    float acc[MT][NBW][4];
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
        for (int j = 0; j < NBW; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[mt][j][r] = 0.f;
    for (int i = threadIdx.x; i < 16 * MT; i += NT) s_db[i] = 0.f;

    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int n = tile / (tiles_x * tiles_y);
        const int r = tile - n * tiles_x * tiles_y;
        const int y0 = (r / tiles_x) * TH, x0 = (r % tiles_x) * TW;
        __syncthreads();
        stage_halo<CIN>(x, s_x, n, w, h, y0, x0);
        for (int e = threadIdx.x; e < 16 * MT * TH * TW; e += NT) {
            const int co = e / (TH * TW), p = e - co * (TH * TW);
            const int py = p / TW, px = p - py * TW;
            const int y = y0 + py, xx = x0 + px;
            __nv_bfloat16 v = __float2bfloat16(0.f);
            if (co < COUT && y < h && xx < w) v = dz[(((size_t)n * h + y) * w + xx) * COUT + co];
            s_dzt[co * DS + p] = v;
        }
        __syncthreads();
        for (int co = warp; co < COUT; co += 4) {
            float s = 0.f;
            for (int p = lane; p < TH * TW; p += 32) s += __bfloat162float(s_dzt[co * DS + p]);
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) s_db[co] += s;
        }
        // K = the 128 pixels in 8 chunks of 16 (one tile row each)
#pragma unroll 1
        for (int kc = 0; kc < TH; ++kc) {
            unsigned a[MT][4];
#pragma unroll
            for (int mt = 0; mt < MT; ++mt) {
                const __nv_bfloat16* r0 = s_dzt + (size_t)(16 * mt + gid) * DS + kc * TW + 2 * tig;
                const __nv_bfloat16* r1 = r0 + 8 * DS;
                a[mt][0] = ld32(r0);
                a[mt][1] = ld32(r1);
                a[mt][2] = ld32(r0 + 8);
                a[mt][3] = ld32(r1 + 8);
            }
#pragma unroll
            for (int j = 0; j < NBW; ++j) {
                const int nb = warp * NBW + j;
                if (nb >= NB_ALL) break;
                const int col = nb * 8 + gid;  // GEMM column = t * CIN + ci
                const int t = col / CIN, ci = col - t * CIN;
                const int ky = t / 3, kx = t % 3;
                // pixel k of the chunk: halo row kc + ky, halo column k + kx
                const __nv_bfloat16* xb = s_x + ((size_t)(kc + ky) * (TW + 2) + kx) * CS + ci;
                const int k0 = 2 * tig;
                const unsigned b0 = ld2x16(xb + (size_t)k0 * CS, xb + (size_t)(k0 + 1) * CS);
                const unsigned b1 = ld2x16(xb + (size_t)(k0 + 8) * CS, xb + (size_t)(k0 + 9) * CS);
#pragma unroll
                for (int mt = 0; mt < MT; ++mt) mma_bf16(acc[mt][j], a[mt], b0, b1);
            }
        }
    }
    __syncthreads();
    float* out = partial + (size_t)blockIdx.x * NPAR;
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
        for (int j = 0; j < NBW; ++j) {
            const int nb = warp * NBW + j;
            if (nb >= NB_ALL) break;
            const int col = nb * 8 + 2 * tig;
            const int co0 = 16 * mt + gid, co1 = co0 + 8;
            if (co0 < COUT) {
                out[(size_t)co0 * NCOL + col] = acc[mt][j][0];
                out[(size_t)co0 * NCOL + col + 1] = acc[mt][j][1];
            }
            if (co1 < COUT) {
                out[(size_t)co1 * NCOL + col] = acc[mt][j][2];
                out[(size_t)co1 * NCOL + col + 1] = acc[mt][j][3];
            }
        }
    for (int co = threadIdx.x; co < COUT; co += NT) out[(size_t)COUT * NCOL + co] = s_db[co];
}

// grad[i] = sum over the CTAs, in order, of partial[cta][i]
__global__ void k_reduce_dw(const float* __restrict__ partial, int npar, int ctas, float* __restrict__ grad)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npar) return;
    float s = 0.f;
    for (int b = 0; b < ctas; ++b) s += partial[(size_t)b * npar + i];
    grad[i] = s;
}

// Adam (Kingma and Ba, 2015) on the FP32 masters; refreshes the BF16 copies.
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ grad, float* __restrict__ m,
                       float* __restrict__ v, __nv_bfloat16* __restrict__ pb, int count, float lr, float b1,
                       float b2, float eps, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const float gr = grad[i];
    const float mm = b1 * m[i] + (1.f - b1) * gr;
    const float vv = b2 * v[i] + (1.f - b2) * gr * gr;
    m[i] = mm;
    v[i] = vv;
    const float np = p[i] - lr * (mm * c1) / (sqrtf(vv * c2) + eps);
    p[i] = np;
    pb[i] = __float2bfloat16(np);
}

__global__ void k_to_bf16(const float* __restrict__ p, __nv_bfloat16* __restrict__ pb, int count)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) pb[i] = __float2bfloat16(p[i]);
}

template <int CIN, int COUT>
constexpr int dw_npar()
{
    return COUT * 9 * CIN + COUT;
}

}  // namespace

size_t dw_partial_floats() { return (size_t)kDwCtas * dw_npar<kC, kC>(); }

cudaError_t launch_features(const Samples& S, __nv_bfloat16* x0, cudaStream_t st)
{
    dim3 grid((S.w + 127) / 128, S.h, S.n);
    k_features<<<grid, 128, 0, st>>>(S, x0);
    return cudaGetLastError();
}

cudaError_t launch_forward(const Net& net, const Samples& S, const __nv_bfloat16* x0, __nv_bfloat16* a1,
                           __nv_bfloat16* a2, __nv_bfloat16* a3, cudaStream_t st)
{
    dim3 grid((S.w + TW - 1) / TW, (S.h + TH - 1) / TH, S.n);
    k_conv_fwd<kC0, kC, 0><<<grid, NT, 0, st>>>(x0, net.w[0], net.b[0], a1, S);
    k_conv_fwd<kC, kC, 0><<<grid, NT, 0, st>>>(a1, net.w[1], net.b[1], a2, S);
    k_conv_fwd<kC, kC, 0><<<grid, NT, 0, st>>>(a2, net.w[2], net.b[2], a3, S);
    k_conv_fwd<kC, kC4, 1><<<grid, NT, 0, st>>>(a3, net.w[3], net.b[3], nullptr, S);
    return cudaGetLastError();
}

int loss_blocks(int w, int h, int n) { return ((w + 127) / 128) * h * n; }

cudaError_t launch_loss(const Samples& S, __nv_bfloat16* dz4, double* partials, double* d_loss, cudaStream_t st)
{
    const double count = (double)S.w * S.h * S.n;
    dim3 grid((S.w + 127) / 128, S.h, S.n);
    k_loss<<<grid, 128, 0, st>>>(S, dz4, partials, (float)(kOutScale * 2.0 / count));
    k_sum_partials<<<1, 256, 0, st>>>(partials, loss_blocks(S.w, S.h, S.n), 1.0 / count, d_loss);
    return cudaGetLastError();
}

template <int CIN, int COUT>
static void dw_and_reduce(const __nv_bfloat16* dz, const __nv_bfloat16* x, float* partial, float* grad_w,
                          const Samples& S, cudaStream_t st)
{
    constexpr int npar = dw_npar<CIN, COUT>();
    k_conv_dw<CIN, COUT><<<kDwCtas, NT, 0, st>>>(dz, x, partial, S.w, S.h, S.n);
    k_reduce_dw<<<(npar + 255) / 256, 256, 0, st>>>(partial, npar, kDwCtas, grad_w);
}

cudaError_t launch_backward(const Net& net, const Samples& S, const __nv_bfloat16* x0, const __nv_bfloat16* a1,
                            const __nv_bfloat16* a2, const __nv_bfloat16* a3, __nv_bfloat16* dz4,
                            __nv_bfloat16* dz3, __nv_bfloat16* dz2, __nv_bfloat16* dz1, float* partial,
                            float* grad, cudaStream_t st)
{
    dim3 grid((S.w + TW - 1) / TW, (S.h + TH - 1) / TH, S.n);
    // the weight block of layer l is followed by its bias block in `grad`
    dw_and_reduce<kC, kC4>(dz4, a3, partial, grad + w_offset(3), S, st);
    k_conv_dx<kC, kC4><<<grid, NT, 0, st>>>(dz4, net.w[3], a3, dz3, S.w, S.h);
    dw_and_reduce<kC, kC>(dz3, a2, partial, grad + w_offset(2), S, st);
    k_conv_dx<kC, kC><<<grid, NT, 0, st>>>(dz3, net.w[2], a2, dz2, S.w, S.h);
    dw_and_reduce<kC, kC>(dz2, a1, partial, grad + w_offset(1), S, st);
    k_conv_dx<kC, kC><<<grid, NT, 0, st>>>(dz2, net.w[1], a1, dz1, S.w, S.h);
    dw_and_reduce<kC0, kC>(dz1, x0, partial, grad + w_offset(0), S, st);
    return cudaGetLastError();
}

cudaError_t launch_adam(float* p, const float* grad, float* m, float* v, __nv_bfloat16* pb, int count, float lr,
                        long long step, cudaStream_t st)
{
    const double b1 = 0.9, b2 = 0.999;
    const float c1 = (float)(1.0 / (1.0 - pow(b1, (double)step)));
    const float c2 = (float)(1.0 / (1.0 - pow(b2, (double)step)));
    k_adam<<<(count + 255) / 256, 256, 0, st>>>(p, grad, m, v, pb, count, lr, (float)b1, (float)b2, 1e-8f, c1, c2);
    return cudaGetLastError();
}

cudaError_t launch_to_bf16(const float* p, __nv_bfloat16* pb, int count, cudaStream_t st)
{
    k_to_bf16<<<(count + 255) / 256, 256, 0, st>>>(p, pb, count);
    return cudaGetLastError();
}

}  // namespace sg
}  // namespace kz
