// kaze_surrogate_api.cu -- host runtime of the learned AOS surrogate behind
// the kaze_surrogate_* entry points of include/kaze.h.
//
// The surrogate owns its parameters in the padded device layout of
// surrogate.h (FP32 masters, Adam moments, gradients and BF16 copies) and,
// when created for training, one device arena for the activations and
// gradients of max_samples images of max_w x max_h.  Host-visible parameter
// vectors, gradients and checkpoints use the logical layout (widths
// 5-32-32-32-1); packing between the two happens here on the host.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "kaze_internal.h"
#include "surrogate.h"

#define KAZE_API extern "C" __attribute__((visibility("default")))

using kz::sg::kParamsLogical;
using kz::sg::kParamsPadded;

static_assert(kParamsLogical == KAZE_SURROGATE_PARAMS, "header parameter count");
static_assert(kz::sg::kMaxSamples == KAZE_SURROGATE_MAX_SAMPLES, "header sample bound");

struct kaze_surrogate {
    int max_w = 0, max_h = 0, max_n = 0;
    bool training = false;
    cudaStream_t stream = nullptr;

    float* p = nullptr;       // FP32 masters (padded layout)
    float* grad = nullptr;
    float* m = nullptr;
    float* v = nullptr;
    __nv_bfloat16* pb = nullptr;  // BF16 copies
    long long steps = 0;

    // training arena
    void* arena = nullptr;
    __nv_bfloat16 *x0 = nullptr, *a1 = nullptr, *a2 = nullptr, *a3 = nullptr;
    __nv_bfloat16 *dz4 = nullptr, *dz3 = nullptr, *dz2 = nullptr, *dz1 = nullptr;
    float* lnext = nullptr;
    float* partial = nullptr;
    double* loss_part = nullptr;
    double* d_loss = nullptr;
    double* h_loss = nullptr;  // pinned
    int* d_status = nullptr;   // bit 0: a bounded device wait of the tcgen05 kernel ran out
    int* h_status = nullptr;   // pinned

    int launches = 0;
    std::string err;
};

namespace {

thread_local std::string g_sg_create_err;

kaze_status sfail(kaze_surrogate* s, kaze_status st, const std::string& msg)
{
    if (s && s->err.empty()) s->err = msg;
    return st;
}

kaze_status scuda(kaze_surrogate* s, cudaError_t e, const char* what)
{
    return sfail(s, KAZE_ERR_CUDA, std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}

#define SG_TRY(s, call)                                              \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) return scuda((s), e_, #call);         \
    } while (0)

#define SG_LAUNCH(s, count, call)   \
    do {                            \
        SG_TRY(s, call);            \
        (s)->launches += (count);   \
    } while (0)

// splitmix64 (Steele, Lea and Flood, 2014): a counter-based generator.
uint64_t splitmix64(uint64_t x)
{
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

// Nearest bfloat16 value of x (8 significant bits, ties to even).
float bf16_value(double x)
{
    if (x == 0.0 || !std::isfinite(x)) return (float)x;
    int e = 0;
    const double m = std::frexp(x, &e);  // x = m 2^e, 0.5 <= |m| < 1
    return (float)std::ldexp(std::nearbyint(m * 256.0), e - 8);
}

int padded_index(int l, int co, int t, int ci)
{
    return kz::sg::w_offset(l) + (co * 9 + t) * kz::sg::cin_of(l) + ci;
}

int logical_index(int l, int co, int t, int ci)
{
    return kz::sg::logical_w_offset(l) + (co * 9 + t) * kz::sg::logical_cin(l) + ci;
}

void pack_params(const float* logical, std::vector<float>& padded)
{
    using namespace kz::sg;
    padded.assign(kParamsPadded, 0.f);
    for (int l = 0; l < kLayers; ++l) {
        for (int co = 0; co < logical_cout(l); ++co) {
            for (int t = 0; t < 9; ++t)
                for (int ci = 0; ci < logical_cin(l); ++ci)
                    padded[padded_index(l, co, t, ci)] = logical[logical_index(l, co, t, ci)];
            padded[b_offset(l) + co] = logical[logical_w_offset(l) + logical_w_count(l) + co];
        }
    }
}

void unpack_params(const std::vector<float>& padded, float* logical)
{
    using namespace kz::sg;
    for (int l = 0; l < kLayers; ++l) {
        for (int co = 0; co < logical_cout(l); ++co) {
            for (int t = 0; t < 9; ++t)
                for (int ci = 0; ci < logical_cin(l); ++ci)
                    logical[logical_index(l, co, t, ci)] = padded[padded_index(l, co, t, ci)];
            logical[logical_w_offset(l) + logical_w_count(l) + co] = padded[b_offset(l) + co];
        }
    }
}

// Uploads FP32 masters (logical layout), zeroes the Adam state.
kaze_status upload_params(kaze_surrogate* s, const float* logical)
{
    std::vector<float> padded;
    pack_params(logical, padded);
    SG_TRY(s, cudaMemcpyAsync(s->p, padded.data(), sizeof(float) * kParamsPadded, cudaMemcpyHostToDevice, s->stream));
    SG_TRY(s, cudaMemsetAsync(s->m, 0, sizeof(float) * kParamsPadded, s->stream));
    SG_TRY(s, cudaMemsetAsync(s->v, 0, sizeof(float) * kParamsPadded, s->stream));
    SG_TRY(s, cudaMemsetAsync(s->grad, 0, sizeof(float) * kParamsPadded, s->stream));
    SG_LAUNCH(s, 1, kz::sg::launch_to_bf16(s->p, s->pb, kParamsPadded, s->stream));
    SG_TRY(s, cudaStreamSynchronize(s->stream));  // `padded` is pageable and goes out of scope
    s->steps = 0;
    return KAZE_OK;
}

kaze_status download(kaze_surrogate* s, const float* d_padded, float* logical)
{
    std::vector<float> padded(kParamsPadded);
    SG_TRY(s, cudaMemcpyAsync(padded.data(), d_padded, sizeof(float) * kParamsPadded, cudaMemcpyDeviceToHost,
                              s->stream));
    SG_TRY(s, cudaStreamSynchronize(s->stream));
    unpack_params(padded, logical);
    return KAZE_OK;
}

// Validates one call's samples and fills the kernels' table.
kaze_status make_samples(kaze_surrogate* s, const float* const* L, const float* const* g, const float* tau,
                         const float* const* T, float* const* out, int n, int w, int h, int pitch, bool need_arena,
                         kz::sg::Samples* S)
{
    if (!s) return KAZE_ERR_INVALID_ARG;
    if (!L || !g || !tau) return sfail(s, KAZE_ERR_INVALID_ARG, "NULL sample array");
    if (n < 1 || n > kz::sg::kMaxSamples) return sfail(s, KAZE_ERR_INVALID_ARG, "sample count out of range");
    if (w < 1 || h < 1 || pitch < w) return sfail(s, KAZE_ERR_INVALID_ARG, "bad image size or pitch");
    if (need_arena) {
        if (!s->training) return sfail(s, KAZE_ERR_STATE, "surrogate was created without KAZE_SURROGATE_TRAIN");
        if (w > s->max_w || h > s->max_h || n > s->max_n)
            return sfail(s, KAZE_ERR_INVALID_ARG, "samples exceed the surrogate's maximum");
    }
    std::memset(S, 0, sizeof(*S));
    for (int i = 0; i < n; ++i) {
        if (!L[i] || !g[i]) return sfail(s, KAZE_ERR_INVALID_ARG, "NULL sample pointer");
        if (!(tau[i] >= 0.f) || !std::isfinite(tau[i])) return sfail(s, KAZE_ERR_INVALID_ARG, "bad tau");
        S->L[i] = L[i];
        S->g[i] = g[i];
        S->s[i] = kz::sg::input_scale(tau[i]);
        if (T) {
            if (!T[i]) return sfail(s, KAZE_ERR_INVALID_ARG, "NULL target pointer");
            S->T[i] = T[i];
        }
        if (out) {
            if (!out[i]) return sfail(s, KAZE_ERR_INVALID_ARG, "NULL output pointer");
            if ((const float*)out[i] == L[i] || (const float*)out[i] == g[i])
                return sfail(s, KAZE_ERR_INVALID_ARG, "output aliases an input");
            S->out[i] = out[i];
        }
    }
    S->n = n;
    S->w = w;
    S->h = h;
    S->pitch = pitch;
    S->opitch = pitch;
    return KAZE_OK;
}

kz::sg::Net net_of(const kaze_surrogate* s)
{
    kz::sg::Net net;
    for (int l = 0; l < kz::sg::kLayers; ++l) {
        net.w[l] = s->pb + kz::sg::w_offset(l);
        net.b[l] = s->p + kz::sg::b_offset(l);
    }
    return net;
}

// Forward (layer kernels) + loss + backward into s->grad; the outputs go to
// the internal lnext planes.
kaze_status enqueue_gradients(kaze_surrogate* s, kz::sg::Samples& S)
{
    for (int i = 0; i < S.n; ++i) S.out[i] = s->lnext + (size_t)i * S.w * S.h;
    S.opitch = S.w;
    const kz::sg::Net net = net_of(s);
    SG_LAUNCH(s, 1, kz::sg::launch_features(S, s->x0, s->stream));
    SG_LAUNCH(s, 4, kz::sg::launch_forward(net, S, s->x0, s->a1, s->a2, s->a3, s->stream));
    SG_LAUNCH(s, 2, kz::sg::launch_loss(S, s->dz4, s->loss_part, s->d_loss, s->stream));
    SG_LAUNCH(s, 11, kz::sg::launch_backward(net, S, s->x0, s->a1, s->a2, s->a3, s->dz4, s->dz3, s->dz2, s->dz1,
                                             s->partial, s->grad, s->stream));
    return KAZE_OK;
}

kaze_status read_loss(kaze_surrogate* s, double* h_loss)
{
    if (!h_loss) return KAZE_OK;
    SG_TRY(s, cudaMemcpyAsync(s->h_loss, s->d_loss, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    SG_TRY(s, cudaStreamSynchronize(s->stream));
    *h_loss = *s->h_loss;
    return KAZE_OK;
}

constexpr char kMagic[4] = {'K', 'Z', 'S', 'G'};
constexpr uint32_t kVersion = 1;

}  // namespace

namespace kz {
namespace sg {

float input_scale(double tau) { return bf16_value(std::log1p(tau) / 5.0); }

// The detection pipeline's hook (kaze_api.cu): one surrogate step of the
// fused kernel on the given stream.
cudaError_t enqueue_pipeline_step(const kaze_surrogate* s, const Samples& S, int* status, cudaStream_t st)
{
    return launch_forward_tc(s->pb, s->p, S, status, st);
}

}  // namespace sg
}  // namespace kz

KAZE_API kaze_status kaze_surrogate_create(int max_w, int max_h, int max_samples, int flags,
                                           unsigned long long seed, void* cuda_stream, kaze_surrogate** out)
{
    if (!out) return KAZE_ERR_INVALID_ARG;
    *out = nullptr;
    if (flags & ~KAZE_SURROGATE_TRAIN) {
        g_sg_create_err = "unknown flags";
        return KAZE_ERR_INVALID_ARG;
    }
    const bool training = (flags & KAZE_SURROGATE_TRAIN) != 0;
    if (training && (max_w < 1 || max_h < 1 || max_samples < 1 || max_samples > kz::sg::kMaxSamples ||
                     (double)max_w * max_h * max_samples > 2.0e9)) {
        g_sg_create_err = "bad training size";
        return KAZE_ERR_INVALID_ARG;
    }
    kaze_surrogate* s = new (std::nothrow) kaze_surrogate;
    if (!s) return KAZE_ERR_OOM;
    s->max_w = max_w;
    s->max_h = max_h;
    s->max_n = max_samples;
    s->training = training;
    s->stream = (cudaStream_t)cuda_stream;
    auto bail = [&](kaze_status st, const std::string& msg) {
        g_sg_create_err = msg;
        kaze_surrogate_destroy(s);
        return st;
    };
    cudaError_t e = kz::sg::configure_surrogate_kernels();
    if (e != cudaSuccess) return bail(KAZE_ERR_CUDA, std::string("configure: ") + cudaGetErrorString(e));
    if (cudaMalloc(&s->d_status, sizeof(int)) != cudaSuccess || cudaMemset(s->d_status, 0, sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&s->h_status, sizeof(int)) != cudaSuccess)
        return bail(KAZE_ERR_OOM, "status allocation failed");
    if (cudaMalloc(&s->p, sizeof(float) * kParamsPadded) != cudaSuccess ||
        cudaMalloc(&s->grad, sizeof(float) * kParamsPadded) != cudaSuccess ||
        cudaMalloc(&s->m, sizeof(float) * kParamsPadded) != cudaSuccess ||
        cudaMalloc(&s->v, sizeof(float) * kParamsPadded) != cudaSuccess ||
        cudaMalloc(&s->pb, sizeof(__nv_bfloat16) * kParamsPadded) != cudaSuccess)
        return bail(KAZE_ERR_OOM, "parameter allocation failed");
    if (training) {
        const size_t px = (size_t)max_w * max_h * max_samples;
        const size_t nloss = (size_t)kz::sg::loss_blocks(max_w, max_h, max_samples);
        size_t off = 0;
        auto take = [&](size_t bytes) {
            const size_t o = off;
            off += (bytes + 255) / 256 * 256;
            return o;
        };
        const size_t o_x0 = take(px * kz::sg::kC0 * 2);
        const size_t o_a1 = take(px * kz::sg::kC * 2), o_a2 = take(px * kz::sg::kC * 2),
                     o_a3 = take(px * kz::sg::kC * 2);
        const size_t o_dz4 = take(px * kz::sg::kC4 * 2);
        const size_t o_dz3 = take(px * kz::sg::kC * 2), o_dz2 = take(px * kz::sg::kC * 2),
                     o_dz1 = take(px * kz::sg::kC * 2);
        const size_t o_ln = take(px * 4);
        const size_t o_part = take(kz::sg::dw_partial_floats() * 4);
        const size_t o_lp = take(nloss * 8);
        const size_t o_loss = take(8);
        if (cudaMalloc(&s->arena, off) != cudaSuccess) return bail(KAZE_ERR_OOM, "training arena allocation failed");
        char* a = (char*)s->arena;
        s->x0 = (__nv_bfloat16*)(a + o_x0);
        s->a1 = (__nv_bfloat16*)(a + o_a1);
        s->a2 = (__nv_bfloat16*)(a + o_a2);
        s->a3 = (__nv_bfloat16*)(a + o_a3);
        s->dz4 = (__nv_bfloat16*)(a + o_dz4);
        s->dz3 = (__nv_bfloat16*)(a + o_dz3);
        s->dz2 = (__nv_bfloat16*)(a + o_dz2);
        s->dz1 = (__nv_bfloat16*)(a + o_dz1);
        s->lnext = (float*)(a + o_ln);
        s->partial = (float*)(a + o_part);
        s->loss_part = (double*)(a + o_lp);
        s->d_loss = (double*)(a + o_loss);
        if (cudaMallocHost(&s->h_loss, sizeof(double)) != cudaSuccess)
            return bail(KAZE_ERR_OOM, "pinned allocation failed");
    }
    // Initial parameters: layers 1-3 uniform in +-sqrt(6 / fan_in) (fan_in =
    // 9 x input width), the last layer and every bias zero, so the untrained
    // network maps L to itself.
    std::vector<float> init(kParamsLogical, 0.f);
    for (int l = 0; l < kz::sg::kLayers - 1; ++l) {
        const double bound = std::sqrt(6.0 / (9.0 * kz::sg::logical_cin(l)));
        const int o = kz::sg::logical_w_offset(l);
        for (int i = 0; i < kz::sg::logical_w_count(l); ++i) {
            const uint64_t r = splitmix64(seed * 0x100000001B3ull + (uint64_t)(o + i));
            const double u = (double)(r >> 11) * (1.0 / 9007199254740992.0);  // [0, 1)
            init[o + i] = (float)((2.0 * u - 1.0) * bound);
        }
    }
    kaze_status st = upload_params(s, init.data());
    if (st != KAZE_OK) return bail(st, s->err);
    *out = s;
    return KAZE_OK;
}

KAZE_API kaze_status kaze_surrogate_set_stream(kaze_surrogate* s, void* cuda_stream)
{
    if (!s) return KAZE_ERR_INVALID_ARG;
    s->stream = (cudaStream_t)cuda_stream;
    return KAZE_OK;
}

KAZE_API kaze_status kaze_surrogate_get_params(kaze_surrogate* s, float* h_params, int count)
{
    if (!s || !h_params) return KAZE_ERR_INVALID_ARG;
    if (count != kParamsLogical) return sfail(s, KAZE_ERR_INVALID_ARG, "count must be KAZE_SURROGATE_PARAMS");
    return download(s, s->p, h_params);
}

KAZE_API kaze_status kaze_surrogate_set_params(kaze_surrogate* s, const float* h_params, int count)
{
    if (!s || !h_params) return KAZE_ERR_INVALID_ARG;
    if (count != kParamsLogical) return sfail(s, KAZE_ERR_INVALID_ARG, "count must be KAZE_SURROGATE_PARAMS");
    for (int i = 0; i < count; ++i)
        if (!std::isfinite(h_params[i])) return sfail(s, KAZE_ERR_INVALID_ARG, "non-finite parameter");
    s->launches = 0;
    return upload_params(s, h_params);
}

KAZE_API kaze_status kaze_surrogate_step(kaze_surrogate* s, const float* const* d_L, const float* const* d_g,
                                         const float* h_tau, float* const* d_out, int n, int w, int h_, int pitch,
                                         int path)
{
    if (!s) return KAZE_ERR_INVALID_ARG;
    if (path != KAZE_SURROGATE_FUSED && path != KAZE_SURROGATE_LAYERED && path != KAZE_SURROGATE_FUSED_SYNC)
        return sfail(s, KAZE_ERR_INVALID_ARG, "unknown path");
    if (!d_out) return sfail(s, KAZE_ERR_INVALID_ARG, "NULL output array");
    kz::sg::Samples S;
    const bool layered = path == KAZE_SURROGATE_LAYERED;
    kaze_status st = make_samples(s, d_L, d_g, h_tau, nullptr, d_out, n, w, h_, pitch, layered, &S);
    if (st != KAZE_OK) return st;
    s->launches = 0;
    if (layered) {
        const kz::sg::Net net = net_of(s);
        SG_LAUNCH(s, 1, kz::sg::launch_features(S, s->x0, s->stream));
        SG_LAUNCH(s, 4, kz::sg::launch_forward(net, S, s->x0, s->a1, s->a2, s->a3, s->stream));
    } else if (path == KAZE_SURROGATE_FUSED_SYNC) {
        SG_LAUNCH(s, 1, kz::sg::launch_forward_fused(s->pb, s->p, S, s->stream));
    } else {
        SG_LAUNCH(s, 1, kz::sg::launch_forward_tc(s->pb, s->p, S, s->d_status, s->stream));
    }
    return KAZE_OK;
}

KAZE_API kaze_status kaze_surrogate_gradients(kaze_surrogate* s, const float* const* d_L, const float* const* d_g,
                                              const float* h_tau, const float* const* d_T, int n, int w, int h_,
                                              int pitch, double* h_loss, float* h_grad)
{
    if (!s) return KAZE_ERR_INVALID_ARG;
    if (!d_T || !h_grad) return sfail(s, KAZE_ERR_INVALID_ARG, "NULL target array or gradient output");
    kz::sg::Samples S;
    kaze_status st = make_samples(s, d_L, d_g, h_tau, d_T, nullptr, n, w, h_, pitch, true, &S);
    if (st != KAZE_OK) return st;
    s->launches = 0;
    if ((st = enqueue_gradients(s, S)) != KAZE_OK) return st;
    if ((st = read_loss(s, h_loss)) != KAZE_OK) return st;
    return download(s, s->grad, h_grad);
}

KAZE_API kaze_status kaze_surrogate_train_step(kaze_surrogate* s, const float* const* d_L, const float* const* d_g,
                                               const float* h_tau, const float* const* d_T, int n, int w, int h_,
                                               int pitch, float lr, double* h_loss)
{
    if (!s) return KAZE_ERR_INVALID_ARG;
    if (!d_T) return sfail(s, KAZE_ERR_INVALID_ARG, "NULL target array");
    if (!(lr > 0.f) || !std::isfinite(lr)) return sfail(s, KAZE_ERR_INVALID_ARG, "bad learning rate");
    kz::sg::Samples S;
    kaze_status st = make_samples(s, d_L, d_g, h_tau, d_T, nullptr, n, w, h_, pitch, true, &S);
    if (st != KAZE_OK) return st;
    s->launches = 0;
    if ((st = enqueue_gradients(s, S)) != KAZE_OK) return st;
    s->steps += 1;
    SG_LAUNCH(s, 1, kz::sg::launch_adam(s->p, s->grad, s->m, s->v, s->pb, kParamsPadded, lr, s->steps, s->stream));
    return read_loss(s, h_loss);
}

KAZE_API kaze_status kaze_surrogate_sync(kaze_surrogate* s)
{
    if (!s) return KAZE_ERR_INVALID_ARG;
    SG_TRY(s, cudaMemcpyAsync(s->h_status, s->d_status, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    SG_TRY(s, cudaStreamSynchronize(s->stream));
    if (*s->h_status) {
        SG_TRY(s, cudaMemsetAsync(s->d_status, 0, sizeof(int), s->stream));
        return sfail(s, KAZE_ERR_TIMEOUT, "a bounded device-side wait ran out");
    }
    return KAZE_OK;
}

KAZE_API kaze_status kaze_surrogate_steps_taken(const kaze_surrogate* s, long long* steps)
{
    if (!s || !steps) return KAZE_ERR_INVALID_ARG;
    *steps = s->steps;
    return KAZE_OK;
}

KAZE_API int kaze_surrogate_last_launch_count(const kaze_surrogate* s) { return s ? s->launches : -1; }

KAZE_API kaze_status kaze_surrogate_save(kaze_surrogate* s, const char* path)
{
    if (!s || !path) return KAZE_ERR_INVALID_ARG;
    std::vector<float> p(kParamsLogical), m(kParamsLogical), v(kParamsLogical);
    kaze_status st;
    if ((st = download(s, s->p, p.data())) != KAZE_OK) return st;
    if ((st = download(s, s->m, m.data())) != KAZE_OK) return st;
    if ((st = download(s, s->v, v.data())) != KAZE_OK) return st;
    FILE* f = std::fopen(path, "wb");
    if (!f) return sfail(s, KAZE_ERR_INVALID_ARG, std::string("cannot open for writing: ") + path);
    const uint32_t hdr[3] = {kVersion, (uint32_t)kParamsLogical, 0u};
    const int64_t steps = s->steps;
    bool ok = std::fwrite(kMagic, 1, 4, f) == 4 && std::fwrite(hdr, 4, 3, f) == 3 &&
              std::fwrite(&steps, 8, 1, f) == 1 &&
              std::fwrite(p.data(), 4, kParamsLogical, f) == (size_t)kParamsLogical &&
              std::fwrite(m.data(), 4, kParamsLogical, f) == (size_t)kParamsLogical &&
              std::fwrite(v.data(), 4, kParamsLogical, f) == (size_t)kParamsLogical;
    ok = (std::fclose(f) == 0) && ok;
    return ok ? KAZE_OK : sfail(s, KAZE_ERR_INVALID_ARG, std::string("write failed: ") + path);
}

KAZE_API kaze_status kaze_surrogate_load(kaze_surrogate* s, const char* path)
{
    if (!s || !path) return KAZE_ERR_INVALID_ARG;
    FILE* f = std::fopen(path, "rb");
    if (!f) return sfail(s, KAZE_ERR_INVALID_ARG, std::string("cannot open: ") + path);
    char magic[4];
    uint32_t hdr[3];
    int64_t steps = 0;
    std::vector<float> p(kParamsLogical), m(kParamsLogical), v(kParamsLogical);
    bool ok = std::fread(magic, 1, 4, f) == 4 && std::memcmp(magic, kMagic, 4) == 0 &&
              std::fread(hdr, 4, 3, f) == 3 && hdr[0] == kVersion && hdr[1] == (uint32_t)kParamsLogical &&
              std::fread(&steps, 8, 1, f) == 1 && steps >= 0 &&
              std::fread(p.data(), 4, kParamsLogical, f) == (size_t)kParamsLogical &&
              std::fread(m.data(), 4, kParamsLogical, f) == (size_t)kParamsLogical &&
              std::fread(v.data(), 4, kParamsLogical, f) == (size_t)kParamsLogical;
    std::fclose(f);
    if (!ok) return sfail(s, KAZE_ERR_INVALID_ARG, std::string("not a surrogate checkpoint: ") + path);
    for (int i = 0; i < kParamsLogical; ++i)
        if (!std::isfinite(p[i]) || !std::isfinite(m[i]) || !(v[i] >= 0.f))
            return sfail(s, KAZE_ERR_INVALID_ARG, "checkpoint holds non-finite values");
    kaze_status st = upload_params(s, p.data());
    if (st != KAZE_OK) return st;
    std::vector<float> padded;
    pack_params(m.data(), padded);
    SG_TRY(s, cudaMemcpyAsync(s->m, padded.data(), sizeof(float) * kParamsPadded, cudaMemcpyHostToDevice, s->stream));
    SG_TRY(s, cudaStreamSynchronize(s->stream));
    pack_params(v.data(), padded);
    SG_TRY(s, cudaMemcpyAsync(s->v, padded.data(), sizeof(float) * kParamsPadded, cudaMemcpyHostToDevice, s->stream));
    SG_TRY(s, cudaStreamSynchronize(s->stream));
    s->steps = steps;
    return KAZE_OK;
}

KAZE_API const char* kaze_surrogate_last_error(const kaze_surrogate* s)
{
    return s ? s->err.c_str() : g_sg_create_err.c_str();
}

KAZE_API void kaze_surrogate_destroy(kaze_surrogate* s)
{
    if (!s) return;
    cudaFree(s->p);
    cudaFree(s->grad);
    cudaFree(s->m);
    cudaFree(s->v);
    cudaFree(s->pb);
    cudaFree(s->arena);
    cudaFree(s->d_status);
    if (s->h_loss) cudaFreeHost(s->h_loss);
    if (s->h_status) cudaFreeHost(s->h_status);
    delete s;
}
