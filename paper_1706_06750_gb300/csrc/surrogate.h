// surrogate.h -- layouts of the learned AOS surrogate shared by its kernels
// (k_surrogate.cu) and its host runtime (kaze_surrogate_api.cu).  Not part of
// the ABI.
//
// Logical network: inputs (dx, dy, g, s, c), four 3x3 convolutions of widths
// 5-32-32-32-1 with ReLU after the first three, L_next = L + z / 256.  On the
// device the first layer reads 16 input channels (5 used) and the last one
// writes 8 output channels (1 used), the k16 / n8 granularity of the BF16
// tensor-core MMA; the padded weights are zero and stay zero in training
// because their gradients are identically zero.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "kaze.h"

namespace kz {
namespace sg {

constexpr int kIn = 5;     // logical input channels
constexpr int kC0 = 16;    // stored input channels
constexpr int kC = 32;     // hidden width
constexpr int kC4 = 8;     // computed output channels of the last layer
constexpr int kLayers = 4;
constexpr int kMaxSamples = 64;
constexpr float kDiffScale = 16.f;        // dx, dy = 16 x forward differences of L
constexpr float kOutScale = 1.f / 256.f;  // L_next = L + kOutScale z

// Device (padded) parameter layout, FP32 masters and BF16 copies alike:
//   W1 [32][9][16] b1[32] | W2 [32][9][32] b2[32] | W3 [32][9][32] b3[32] | W4 [8][9][32] b4[8]
__host__ __device__ constexpr int cin_of(int l) { return l == 0 ? kC0 : kC; }
__host__ __device__ constexpr int cout_of(int l) { return l == kLayers - 1 ? kC4 : kC; }
__host__ __device__ constexpr int logical_cin(int l) { return l == 0 ? kIn : kC; }
__host__ __device__ constexpr int logical_cout(int l) { return l == kLayers - 1 ? 1 : kC; }

__host__ __device__ constexpr int w_count(int l) { return cout_of(l) * 9 * cin_of(l); }
// offset of layer l's block: layer 0, then up to two hidden layers, then the last
__host__ __device__ constexpr int w_offset(int l)
{
    return (l >= 1 ? w_count(0) + kC : 0) + (l >= 2 ? (l - 1 < 2 ? l - 1 : 2) * (w_count(1) + kC) : 0) +
           (l >= 4 ? w_count(3) + kC4 : 0);
}
__host__ __device__ constexpr int b_offset(int l) { return w_offset(l) + w_count(l); }
constexpr int kParamsPadded = w_offset(kLayers);  // 25448

__host__ __device__ constexpr int logical_w_count(int l) { return logical_cout(l) * 9 * logical_cin(l); }
__host__ __device__ constexpr int logical_w_offset(int l)
{
    return (l >= 1 ? logical_w_count(0) + kC : 0) + (l >= 2 ? (l - 1 < 2 ? l - 1 : 2) * (logical_w_count(1) + kC) : 0) +
           (l >= 4 ? logical_w_count(3) + 1 : 0);
}
static_assert(w_offset(4) == 25448 && logical_w_offset(4) == 20257, "parameter counts");
constexpr int kParamsLogical = logical_w_offset(kLayers);  // 20257

struct Net {
    const __nv_bfloat16* w[kLayers];
    const float* b[kLayers];
};

// Per-call sample table, passed by value to the kernels (graph-capturable).
struct Samples {
    const float* L[kMaxSamples];  // previous level, FP32 plane with `pitch`
    const float* g[kMaxSamples];  // conductance of L
    const float* T[kMaxSamples];  // target level (training only)
    float* out[kMaxSamples];      // L_next
    float s[kMaxSamples];         // BF16 value of log(1 + tau) / 5
    int n, w, h;
    int pitch;                    // floats per row of L, g, T
    int opitch;                   // floats per row of out
};

// Fixed number of CTAs of the weight-gradient kernels: each writes one
// partial sum, reduced afterwards in a fixed order (deterministic training).
constexpr int kDwCtas = 296;

size_t dw_partial_floats();  // floats of the partial-sum buffer

cudaError_t launch_features(const Samples& S, __nv_bfloat16* x0, cudaStream_t st);
cudaError_t launch_forward(const Net& net, const Samples& S, const __nv_bfloat16* x0, __nv_bfloat16* a1,
                           __nv_bfloat16* a2, __nv_bfloat16* a3, cudaStream_t st);
// One kernel for the whole network (inference): no activations in HBM.
// wpad / ppad: padded BF16 and FP32 parameter vectors.  launch_forward_tc
// runs it on the tcgen05 tensor cores (a bounded wait that runs out sets bit
// 0 of *status); launch_forward_fused on mma.sync.
cudaError_t launch_forward_tc(const __nv_bfloat16* wpad, const float* ppad, const Samples& S, int* status,
                              cudaStream_t st);
cudaError_t launch_forward_fused(const __nv_bfloat16* wpad, const float* ppad, const Samples& S, cudaStream_t st);
cudaError_t configure_surrogate_tc();
cudaError_t configure_surrogate_kernels();
// Loss partials per CTA (double) and dL/dy (BF16, 8 channels).
int loss_blocks(int w, int h, int n);
cudaError_t launch_loss(const Samples& S, __nv_bfloat16* dz4, double* partials, double* d_loss, cudaStream_t st);
cudaError_t launch_backward(const Net& net, const Samples& S, const __nv_bfloat16* x0, const __nv_bfloat16* a1,
                            const __nv_bfloat16* a2, const __nv_bfloat16* a3, __nv_bfloat16* dz4,
                            __nv_bfloat16* dz3, __nv_bfloat16* dz2, __nv_bfloat16* dz1, float* partial,
                            float* grad, cudaStream_t st);
cudaError_t launch_adam(float* p, const float* grad, float* m, float* v, __nv_bfloat16* pb, int count, float lr,
                        long long step, cudaStream_t st);
cudaError_t launch_to_bf16(const float* p, __nv_bfloat16* pb, int count, cudaStream_t st);

// The network's step input s = log(1 + tau) / 5, rounded to BF16 on the host.
float input_scale(double tau);
// One fused surrogate step of the detection pipeline (kaze_api.cu); a
// device-side timeout sets bit 0 of *status.
cudaError_t enqueue_pipeline_step(const kaze_surrogate* s, const Samples& S, int* status, cudaStream_t st);

}  // namespace sg
}  // namespace kz
