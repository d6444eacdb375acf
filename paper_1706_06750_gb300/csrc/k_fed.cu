// k_fed.cu -- the FED evolution of Sec. II-A (Eq. 5): each level is reached
// from the previous one by a cycle of n explicit diffusion steps of varying
// size tau_j, with the conductance g of the previous level held fixed:
//     L <- L + tau_j * sum over the 4-neighbours q of (g_p + g_q)/2 (L_q - L_p),
// a neighbour outside the image contributing nothing (no flux through the
// border, the Neumann condition of the AOS step).
//
// The steps of a cycle are taken in a kappa-cycle order (Grewenig, Weickert
// & Bruhn 2010): the cycle is exact in any order, but in FP32 the natural
// increasing order lets the last, largest steps amplify early rounding errors
// by up to ~1e13 for n = 29; the kappa with the smallest worst-case
// amplification (~1e2 there) is taken.
//
// The one-step kernel: a warp owns 128 consecutive columns (four per lane,
// 16-byte loads) and walks FR consecutive rows, keeping the rows above, at
// and below the current one of L and g in registers (each row is loaded once
// per walk, FDP rows ahead); horizontal neighbours come from the adjacent
// lanes by shuffles, the two columns beyond the warp's ends by scalar loads
// of the end lanes.  Planes need 16-byte aligned rows (pitch % 4 == 0).
#include <algorithm>
#include <cmath>
#include <vector>

#include "aos_solver.cuh"
#include "kaze_internal.h"

namespace kz {
namespace {

constexpr int FR = 16;        // rows per warp
constexpr int FW = 4;         // warps per CTA, side by side
constexpr int FDP = 2;        // rows of loads in flight ahead of the arithmetic

struct Row {
    float4 L, g;
    float lL, lg, rL, rg;     // the columns left of lane 0 / right of lane 31
};

__device__ __forceinline__ Row load_row(const float* __restrict__ L, const float* __restrict__ g, int pitch, int w,
                                        int h, int y, int x0, int lane)
{
    Row r;
    const int yy = min(max(y, 0), h - 1);  // rows outside carry no flux; any valid row will do
    const size_t o = (size_t)yy * pitch + x0;
    if (x0 < w) {
        r.L = __ldg(reinterpret_cast<const float4*>(L + o));
        r.g = __ldg(reinterpret_cast<const float4*>(g + o));
    } else {
        r.L = make_float4(0.f, 0.f, 0.f, 0.f);
        r.g = r.L;
    }
    r.lL = r.lg = r.rL = r.rg = 0.f;
    if (lane == 0 && x0 > 0 && x0 - 1 < w) {
        r.lL = __ldg(L + o - 1);
        r.lg = __ldg(g + o - 1);
    }
    if (lane == 31 && x0 + 4 < w) {
        r.rL = __ldg(L + o + 4);
        r.rg = __ldg(g + o + 4);
    }
    return r;
}

// flux of one pixel: c = centre, (l, r, u, d) neighbours with their g, masks
// for the neighbours that exist
__device__ __forceinline__ float fed_flux(float Lc, float gc, float Ll, float gl, float Lr, float gr, float Lu,
                                          float gu, float Ld, float gd, bool hl, bool hr, bool hu, bool hd)
{
    float f = 0.f;
    if (hl) f = fmaf(0.5f * (gc + gl), Ll - Lc, f);
    if (hr) f = fmaf(0.5f * (gc + gr), Lr - Lc, f);
    if (hu) f = fmaf(0.5f * (gc + gu), Lu - Lc, f);
    if (hd) f = fmaf(0.5f * (gc + gd), Ld - Lc, f);
    return f;
}

__global__ void __launch_bounds__(FW * 32) k_fed_step(const float* __restrict__ Lin, const float* __restrict__ g,
                                                      float* __restrict__ Lout, int pitch, int w, int h, float tau)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int x0 = (blockIdx.x * FW + warp) * 128 + 4 * lane;
    const int y0 = blockIdx.y * FR;
    if ((blockIdx.x * FW + warp) * 128 >= w) return;  // whole warp beyond the image
    // rows y0 - 1 .. y0 + FR: a ring of FDP + 3 rows
    Row ring[FDP + 3];
#pragma unroll
    for (int i = 0; i < FDP + 2; ++i) ring[i] = load_row(Lin, g, pitch, w, h, y0 - 1 + i, x0, lane);
#pragma unroll
    for (int k = 0; k < FR; ++k) {
        if (k + FDP + 2 <= FR + 1) ring[(k + FDP + 2) % (FDP + 3)] = load_row(Lin, g, pitch, w, h, y0 + k + FDP + 1, x0, lane);
        const int y = y0 + k;
        if (y >= h) break;
        const Row& U = ring[k % (FDP + 3)];
        const Row& C = ring[(k + 1) % (FDP + 3)];
        const Row& D = ring[(k + 2) % (FDP + 3)];
        // left neighbour of component x: the previous lane's w (lane 0: the scalar load)
        float Ll = __shfl_up_sync(0xffffffffu, C.L.w, 1), gl = __shfl_up_sync(0xffffffffu, C.g.w, 1);
        float Lr = __shfl_down_sync(0xffffffffu, C.L.x, 1), gr = __shfl_down_sync(0xffffffffu, C.g.x, 1);
        if (lane == 0) {
            Ll = C.lL;
            gl = C.lg;
        }
        if (lane == 31) {
            Lr = C.rL;
            gr = C.rg;
        }
        if (x0 >= w) continue;
        const bool hu = y > 0, hd = y < h - 1;
        float4 o;
        o.x = fmaf(tau, fed_flux(C.L.x, C.g.x, Ll, gl, C.L.y, C.g.y, U.L.x, U.g.x, D.L.x, D.g.x, x0 > 0, x0 + 1 < w, hu,
                                 hd),
                   C.L.x);
        o.y = fmaf(tau, fed_flux(C.L.y, C.g.y, C.L.x, C.g.x, C.L.z, C.g.z, U.L.y, U.g.y, D.L.y, D.g.y, true, x0 + 2 < w,
                                 hu, hd),
                   C.L.y);
        o.z = fmaf(tau, fed_flux(C.L.z, C.g.z, C.L.y, C.g.y, C.L.w, C.g.w, U.L.z, U.g.z, D.L.z, D.g.z, true, x0 + 3 < w,
                                 hu, hd),
                   C.L.z);
        o.w = fmaf(tau, fed_flux(C.L.w, C.g.w, C.L.z, C.g.z, Lr, gr, U.L.w, U.g.w, D.L.w, D.g.w, true, x0 + 4 < w, hu,
                                 hd),
                   C.L.w);
        float* out = Lout + (size_t)y * pitch + x0;
        if (x0 + 4 <= w) {
            *reinterpret_cast<float4*>(out) = o;
        } else {
            out[0] = o.x;
            if (x0 + 1 < w) out[1] = o.y;
            if (x0 + 2 < w) out[2] = o.z;
        }
    }
}

// ---- K steps in one launch ---------------------------------------------------
//
// A warp stages 128 columns, X - 4 .. X + 123, and writes the 120 in the
// middle.  Each step spoils one more column at each end of what the warp
// holds (its outermost columns have no neighbour there; they get a zero-flux
// edge), so the 4 columns of halo on each side absorb up to FMAX steps.  The
// warp's input rows y0 - K .. y0 + FRF + K - 1 of L and g arrive in shared
// memory by TMA tensor copies (boxes of 128 x 8, zeros past the image), all
// requested at the start, one mbarrier per box row.  Rows then go by as a
// wavefront in registers: input row i arrives, then step s is taken on row
// i - s for s = 1..K, each from the three rows of step s - 1 around it; the
// last step's rows y0 .. y0 + FRF - 1 are written.  The edge weights
// (g_p + g_q)/2 are formed once per row and reused by every step, a weight of
// zero standing for a neighbour that does not exist; the sums are taken in
// the same order as the one-step kernel's, so the two agree bit for bit.
// Warps are independent (no block-wide barrier).  A wait that runs out sets
// bit 0 of *status.
constexpr int FMAX = 4;   // steps per fused launch
constexpr int MW = 120;   // columns written per warp
constexpr int TW = 128;   // columns staged per warp
constexpr int CH = 8;     // rows per staged box
constexpr int FRF = 16;   // rows written per warp
constexpr int NCH = (FRF + 2 * FMAX + CH - 1) / CH;  // boxes per warp and plane
constexpr size_t FUSED_SMEM = (size_t)FW * NCH * CH * TW * 2 * sizeof(float);

struct FedTaus {
    float t[FMAX];
};

__device__ __forceinline__ float half_sum(float a, float b) { return 0.5f * (a + b); }

// one pixel: f = sum of w_q (L_q - L_c) in the order left, right, up, down
__device__ __forceinline__ float fused_px(float tau, float c, float l, float wl, float r, float wr, float u, float wu,
                                          float d, float wd)
{
    float f = fmaf(wl, l - c, 0.f);
    f = fmaf(wr, r - c, f);
    f = fmaf(wu, u - c, f);
    f = fmaf(wd, d - c, f);
    return fmaf(tau, f, c);
}

template <int K>
__global__ void __launch_bounds__(FW * 32) k_fed_fused(const __grid_constant__ CUtensorMap tmL,
                                                       const __grid_constant__ CUtensorMap tmG,
                                                       float* __restrict__ Lout, int pitch, int w, int h,
                                                       FedTaus taus, int* __restrict__ status)
{
    static_assert(K >= 2 && K <= FMAX, "the halo holds FMAX steps");
    constexpr int NI = FRF + 2 * K;         // input rows y0 - K .. y0 + FRF + K - 1
    constexpr int NB = (NI + CH - 1) / CH;  // boxes this K needs
    constexpr int NW = K + 2;               // weight rows kept
    extern __shared__ __align__(128) float fsm[];
    __shared__ __align__(8) uint64_t bars[FW][NCH];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int X = (blockIdx.x * FW + warp) * MW;
    if (X >= w) return;  // whole warp beyond the image
    const int y0 = blockIdx.y * FRF;
    float* sL = fsm + (size_t)warp * (NCH * CH * TW * 2);
    float* sG = sL + NCH * CH * TW;
    if (lane == 0) {
#pragma unroll
        for (int b = 0; b < NB; ++b) aos::mbar_init(&bars[warp][b], 1);
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            aos::mbar_expect_tx(&bars[warp][b], 2u * CH * TW * sizeof(float));
            aos::tma_load_2d(sL + b * CH * TW, &tmL, X - 4, y0 - K + b * CH, &bars[warp][b]);
            aos::tma_load_2d(sG + b * CH * TW, &tmG, X - 4, y0 - K + b * CH, &bars[warp][b]);
        }
    }
    __syncwarp();
    const int x0 = X - 4 + 4 * lane;
    // horizontal edge weight to the right of each of the lane's columns: zero
    // where that edge leaves the image or the warp
    const bool e0 = x0 >= 0 && x0 + 1 < w, e1 = x0 + 1 >= 0 && x0 + 2 < w, e2 = x0 + 2 >= 0 && x0 + 3 < w,
               e3 = x0 + 3 >= 0 && x0 + 4 < w && lane != 31;
    const bool store_lane = lane >= 1 && lane <= 30 && x0 < w;

    float4 lv[K][3];  // step s (0..K-1) values, rows by index mod 3
    float4 wr[NW], wd[NW];
    float wl[NW];
    float4 gprev = make_float4(0.f, 0.f, 0.f, 0.f);
    bool ok = true;
#pragma unroll
    for (int i = 0; i < NI; ++i) {
        if (i % CH == 0) {
            ok = aos::mbar_wait_bounded(&bars[warp][i / CH], 0) && ok;
            if (!ok && lane == 0) atomicOr(status, 1);
        }
        const float4 G = *reinterpret_cast<const float4*>(sG + i * TW + 4 * lane);
        const int yi = y0 - K + i;
        // weights of row i: to the right of each column, and of row i - 1 downwards
        {
            const float gn = __shfl_down_sync(0xffffffffu, G.x, 1);
            float4 r;
            r.x = e0 ? half_sum(G.x, G.y) : 0.f;
            r.y = e1 ? half_sum(G.y, G.z) : 0.f;
            r.z = e2 ? half_sum(G.z, G.w) : 0.f;
            r.w = e3 ? half_sum(G.w, gn) : 0.f;
            const float l = __shfl_up_sync(0xffffffffu, r.w, 1);
            wr[i % NW] = r;
            wl[i % NW] = lane == 0 ? 0.f : l;
            if (i > 0) {
                const bool v = yi - 1 >= 0 && yi - 1 < h - 1;
                float4 d;
                d.x = v ? half_sum(gprev.x, G.x) : 0.f;
                d.y = v ? half_sum(gprev.y, G.y) : 0.f;
                d.z = v ? half_sum(gprev.z, G.z) : 0.f;
                d.w = v ? half_sum(gprev.w, G.w) : 0.f;
                wd[(i - 1) % NW] = d;
            }
            gprev = G;
        }
        lv[0][i % 3] = *reinterpret_cast<const float4*>(sL + i * TW + 4 * lane);
#pragma unroll
        for (int s = 1; s <= K; ++s) {
            if (i < 2 * s) continue;  // step s - 1 has no three rows around row i - s yet
            const int j = i - s;
            const float4 U = lv[s - 1][(j - 1) % 3], C = lv[s - 1][j % 3], D = lv[s - 1][(j + 1) % 3];
            const float4 R4 = wr[j % NW], WU = wd[(j - 1) % NW], WD = wd[j % NW];
            const float WL = wl[j % NW];
            const float Ll = __shfl_up_sync(0xffffffffu, C.w, 1), Lr = __shfl_down_sync(0xffffffffu, C.x, 1);
            const float tau = taus.t[s - 1];
            float4 o;
            o.x = fused_px(tau, C.x, Ll, WL, C.y, R4.x, U.x, WU.x, D.x, WD.x);
            o.y = fused_px(tau, C.y, C.x, R4.x, C.z, R4.y, U.y, WU.y, D.y, WD.y);
            o.z = fused_px(tau, C.z, C.y, R4.y, C.w, R4.z, U.z, WU.z, D.z, WD.z);
            o.w = fused_px(tau, C.w, C.z, R4.z, Lr, R4.w, U.w, WU.w, D.w, WD.w);
            if (s < K) {
                lv[s][j % 3] = o;
            } else {
                const int y = y0 - K + j;
                if (j >= K && j < K + FRF && y < h && store_lane) {
                    float* out = Lout + (size_t)y * pitch + x0;
                    if (x0 + 4 <= w) {
                        *reinterpret_cast<float4*>(out) = o;
                    } else {
                        out[0] = o.x;
                        if (x0 + 1 < w) out[1] = o.y;
                        if (x0 + 2 < w) out[2] = o.z;
                    }
                }
            }
        }
    }
    // a staging wait ran out (the status is set): the warp's boxes still in
    // flight land (bounded wait) before it leaves its shared memory
    if (__any_sync(0xffffffffu, !ok) && lane == 0)
        for (int b = 0; b < NB; ++b) aos::mbar_wait_bounded(&bars[warp][b], 0);
}

}  // namespace

int fed_cycle(double dt, double tau_max, double* tau, int cap)
{
    if (!(dt > 0.0) || !(tau_max > 0.0)) return 0;
    auto T = [&](int n) { return tau_max * ((double)n * n + n) / 3.0; };
    int n = (int)std::ceil(std::sqrt(3.0 * dt / tau_max + 0.25) - 0.5);
    if (n < 1) n = 1;
    while (T(n) < dt) ++n;
    while (n > 1 && T(n - 1) >= dt) --n;
    const double sc = dt / T(n);
    for (int j = 0; j < n && j < cap; ++j) {
        const double c = std::cos(3.14159265358979323846 * (2.0 * j + 1.0) / (4.0 * n + 2.0));
        tau[j] = sc * tau_max / (2.0 * c * c);
    }
    return n;
}

namespace {

bool prime(int q)
{
    if (q < 2) return false;
    for (int d = 2; d * d <= q; ++d)
        if (q % d == 0) return false;
    return true;
}

// Position l of the kappa cycle takes step (kappa (l + 1) mod p) - 1 (p the
// smallest prime above n; indices outside 0..n-1 are skipped).
std::vector<int> kappa_order(int n, int kappa)
{
    int p = n + 1;
    while (!prime(p)) ++p;
    std::vector<int> o;
    o.reserve((size_t)n);
    for (long long l = 1; (int)o.size() < n; ++l) {
        const int i = (int)((l * kappa) % p) - 1;
        if (i >= 0 && i < n) o.push_back(i);
    }
    return o;
}

// sum over positions j of max_x |prod_{k<=j} (1 - tau x)| * max_x |prod_{k>j} (1 - tau x)|,
// x over 2001 points of [0, 8]: how far later steps can amplify a rounding
// error made at step j, times the size the iterate can reach there.
double amplification(const std::vector<double>& tau, const std::vector<int>& o)
{
    const int n = (int)o.size();
    std::vector<double> hm((size_t)n, 0.0), tm((size_t)n, 0.0);
    for (int gi = 0; gi <= 2000; ++gi) {
        const double x = 8.0 * gi / 2000;
        double a = 1.0;
        for (int j = 0; j < n; ++j) {
            a *= std::fabs(1.0 - tau[(size_t)o[(size_t)j]] * x);
            hm[(size_t)j] = std::max(hm[(size_t)j], a);
        }
        double b = 1.0;
        for (int j = n - 1; j >= 0; --j) {
            tm[(size_t)j] = std::max(tm[(size_t)j], b);
            b *= std::fabs(1.0 - tau[(size_t)o[(size_t)j]] * x);
        }
    }
    double sum = 0.0;
    for (int j = 0; j < n; ++j) sum += hm[(size_t)j] * tm[(size_t)j];
    return sum;
}

}  // namespace

std::vector<double> fed_ordered_steps(double dt, double tau_max)
{
    const int n = fed_cycle(dt, tau_max, nullptr, 0);
    std::vector<double> tau((size_t)n);
    fed_cycle(dt, tau_max, tau.data(), n);
    if (n <= 1) return tau;
    double best = 0.0;
    std::vector<int> pick;
    for (int kappa = 1; kappa <= n; ++kappa) {
        std::vector<int> o = kappa_order(n, kappa);
        const double a = amplification(tau, o);
        if (pick.empty() || a < best) {
            best = a;
            pick = o;
        }
    }
    std::vector<double> out((size_t)n);
    for (int j = 0; j < n; ++j) out[(size_t)j] = tau[(size_t)pick[(size_t)j]];
    return out;
}

cudaError_t launch_fed_step(const float* Lin, const float* g, float* Lout, int pitch, int w, int h, float tau,
                            cudaStream_t st)
{
    if ((pitch & 3) || (((uintptr_t)Lin | (uintptr_t)g | (uintptr_t)Lout) & 15)) return cudaErrorInvalidValue;
    dim3 grid((w + FW * 128 - 1) / (FW * 128), (h + FR - 1) / FR);
    k_fed_step<<<grid, FW * 32, 0, st>>>(Lin, g, Lout, pitch, w, h, tau);
    return cudaGetLastError();
}

namespace {
template <int K>
cudaError_t fused(const float* Lin, const float* g, float* Lout, int pitch, int w, int h, const FedTaus& t,
                  int* status, cudaStream_t st)
{
    CUtensorMap mL, mG;
    if (!make_plane_map(&mL, Lin, pitch, w, h, TW, CH) || !make_plane_map(&mG, g, pitch, w, h, TW, CH))
        return cudaErrorInvalidValue;
    dim3 grid((w + FW * MW - 1) / (FW * MW), (h + FRF - 1) / FRF);
    k_fed_fused<K><<<grid, FW * 32, FUSED_SMEM, st>>>(mL, mG, Lout, pitch, w, h, t, status);
    return cudaGetLastError();
}
}  // namespace

cudaError_t configure_fed_kernels()
{
    cudaError_t e = cudaFuncSetAttribute(k_fed_fused<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FUSED_SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fed_fused<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FUSED_SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fed_fused<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FUSED_SMEM);
    return e;
}

int fed_max_fused() { return FMAX; }

cudaError_t launch_fed_steps(const float* Lin, const float* g, float* Lout, int pitch, int w, int h, const float* tau,
                             int k, int* status, cudaStream_t st)
{
    if (k < 1 || k > FMAX || !tau || !status) return cudaErrorInvalidValue;
    if (k == 1) return launch_fed_step(Lin, g, Lout, pitch, w, h, tau[0], st);
    if ((pitch & 3) || (((uintptr_t)Lin | (uintptr_t)g | (uintptr_t)Lout) & 15)) return cudaErrorInvalidValue;
    FedTaus t;
    for (int j = 0; j < FMAX; ++j) t.t[j] = j < k ? tau[j] : 0.f;
    switch (k) {
    case 2: return fused<2>(Lin, g, Lout, pitch, w, h, t, status, st);
    case 3: return fused<3>(Lin, g, Lout, pitch, w, h, t, status, st);
    default: return fused<4>(Lin, g, Lout, pitch, w, h, t, status, st);
    }
}

std::vector<int> fed_chunks(int n)
{
    // a launch costs about the same for 2, 3 or 4 steps (it waits on its
    // loads), so take full launches and leave the remainder (a single step
    // goes to the one-step kernel)
    std::vector<int> c((size_t)(n > 0 ? n / FMAX : 0), FMAX);
    if (n > 0 && n % FMAX) c.push_back(n % FMAX);
    return c;
}

}  // namespace kz
