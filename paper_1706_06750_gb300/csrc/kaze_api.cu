// kaze_api.cu -- host runtime behind the C ABI of include/kaze.h.
//
// The handle owns one device arena, carved into: the N evolution levels, the
// N detector responses, the conductance and row-solution scratch planes, a
// staging plane for host input, the contrast statistics and the keypoint
// buffer.  Every plane of a w x h image uses pitch = w rounded up to 32
// floats (128-byte rows, 16-byte aligned vector access), planes packed
// back to back.  All work is stream-ordered on the handle's stream; the
// contrast factor stays on the device so a whole detection can be recorded
// once as a CUDA graph and replayed.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "kaze_internal.h"
#include "surrogate.h"

#define KAZE_API extern "C" __attribute__((visibility("default")))

namespace {
// Kernel kinds, in pipeline order, for launch counting and profiling.
enum KernelKind {
    KK_PRESMOOTH = 0, KK_GRAD_MAX, KK_GRAD_HIST, KK_PERCENTILE, KK_SET_SCALAR,
    KK_CONDUCTANCE, KK_AOS_ROWS, KK_AOS_COLS, KK_DOH, KK_EXTREMA, KK_SURROGATE, KK_DESCRIBE, KK_FED, KK_EVOLVE,
    KK_FRONT_EVOLVE, KK_STREAM_A, KK_STREAM_X, KK_STREAM_B, KK_COUNT
};
const char* const kKindNames[KK_COUNT] = {
    "presmooth", "grad_max", "grad_hist", "percentile", "set_scalar",
    "conductance", "aos_rows", "aos_cols", "doh", "extrema", "surrogate", "describe", "fed", "aos_evolve",
    "front_evolve", "stream_a", "stream_x", "stream_b"};
}  // namespace

struct kaze_handle {
    kaze_options opt;
    int max_w = 0, max_h = 0, N = 0;
    cudaStream_t stream = nullptr;
    // second stream for the column half of each AOS step, with the events
    // that fork it off and join it back to `stream`
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;

    // device arena and its parts
    void* arena = nullptr;
    size_t plane_max = 0;          // floats per plane at max size
    float* levels = nullptr;       // N planes
    float* doh = nullptr;          // N planes
    float* g = nullptr;            // conductance scratch
    float* ux = nullptr;           // row-solution scratch
    float* staging = nullptr;      // device copy of a host input image
    float* staging2 = nullptr;     // a second one: the next host image arrives here while one is detected
    float* d_k = nullptr;          // contrast factor
    unsigned int* d_hmax = nullptr;
    unsigned int* d_hist = nullptr;
    // control block: keypoint count, status word, contrast maximum, candidate
    // count, grid-barrier counter, histogram (+ block counter); one memset
    // clears it at the start of a whole detection (in_detect)
    unsigned int* d_ctl = nullptr;
    size_t ctl_bytes = 0;
    bool in_detect = false;
    unsigned int* d_count = nullptr;
    unsigned long long* d_cand = nullptr;  // pixels the response launch found above the threshold
    unsigned int* d_cand_count = nullptr;
    unsigned int cand_cap = 0;
    const float* cand_doh = nullptr;  // the response stack the list was made from
    int* d_status = nullptr;         // bit 0: a bounded device wait ran out
    float* d_exchange = nullptr;     // segment records of the resident evolution
    float* d_stream = nullptr;       // records and segment neighbours of the streamed evolution
    unsigned int* d_barrier = nullptr;  // its grid-barrier counter
    int max_tiles = 0;               // tiles the exchange buffer serves (the SM count)
    long long evolve_wait_limit = 0;  // test hook of the resident evolution's barrier waits
    int evolve_stall_tile = -1;
    kaze_keypoint* d_kp = nullptr;
    kaze_keypoint* d_dkp = nullptr;  // keypoints uploaded for description
    float* d_desc = nullptr;         // their descriptors, max_keypoints x 64
    unsigned int* h_count = nullptr;  // pinned
    int* h_status = nullptr;          // pinned
    kaze_keypoint* h_kp_pre = nullptr;  // pinned: the first kp_pre keypoints, copied with the count
    int kp_pre = 0;

    // current image geometry
    int cur_w = 0, cur_h = 0, cur_pitch = 0;
    long long cur_plane = 0;
    bool built = false, responded = false;
    bool pending = false;  // a kaze_detect_enqueue awaits its kaze_detect_collect

    // scale table (Eq. 6-7) and filter taps
    double sigma[kz::kMaxLevels];
    double t[kz::kMaxLevels];
    std::vector<float> fed_tau[kz::kMaxLevels];  // FED step sizes of level i's cycle
    kz::GaussTaps taps0, tapsd;
    kz::LevelTable tab;

    // learned stand-in for the AOS step (borrowed; NULL: AOS), and the one
    // the handle owns when it loaded the checkpoint itself
    const kaze_surrogate* surrogate = nullptr;
    kaze_surrogate* own_surrogate = nullptr;
    // the batch kaze_build_batch runs, kept while the image sizes repeat
    kaze_batch* batch = nullptr;
    std::vector<int> batch_w, batch_h;
    float sg_s[kz::kMaxLevels];  // BF16 value of log(1 + tau_i) / 5 per level

    // recorded detection graphs, one per (input plane, size): two slots, so
    // that the two staging planes of a stream of host images both keep theirs
    struct GraphSlot {
        cudaGraphExec_t exec = nullptr;
        const float* img = nullptr;
        int w = 0, h = 0, pitch = 0, launches = 0;
    } gslot[2];
    int g_last = 0;  // slot used last

    // the next host image, copied on `copy` while the current one is detected
    cudaStream_t copy = nullptr;
    cudaEvent_t ev_copied = nullptr;
    const float* pre_src = nullptr;
    int pre_slot = -1, pre_w = 0, pre_h = 0, pre_pitch = 0;
    bool pre_issued = false;  // a copy was issued on `copy` (the main stream waits for it before reusing a plane)

    // launch accounting: kernels enqueued by the current pipeline call, and
    // optional event pairs around each launch (kaze_profile)
    int launches = 0;
    bool profiling = false;
    struct ProfEntry {
        int kind, kernels;
        cudaEvent_t start, stop;
    };
    std::vector<ProfEntry> prof;

    std::vector<kaze_keypoint> hkp;
    std::string err;
};

namespace {

// Message of the last kaze_create that failed on this thread.
thread_local std::string g_create_err;

kaze_status fail(kaze_handle* h, kaze_status s, const std::string& msg)
{
    if (h && h->err.empty()) h->err = msg;
    return s;
}

kaze_status create_fail(kaze_status s, const std::string& msg)
{
    g_create_err = msg;
    return s;
}

kaze_status cuda_fail(kaze_handle* h, cudaError_t e, const char* what)
{
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return fail(h, KAZE_ERR_CUDA, m);
}

#define KZ_TRY(h, call)                                               \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess) return cuda_fail((h), e_, #call);      \
    } while (0)

// Enqueue `nk` kernels of the given kind with one launcher call, counting
// them and, while profiling, bracketing the call with an event pair on the
// handle's stream (external records: inside a stream capture they become
// event-record nodes of the graph, which is what timing needs).
#define KZ_LAUNCH_N(h, kind, nk, call)                                             \
    do {                                                                           \
        cudaEvent_t ev0_ = nullptr, ev1_ = nullptr;                                \
        if ((h)->profiling) {                                                      \
            KZ_TRY(h, cudaEventCreate(&ev0_));                                     \
            KZ_TRY(h, cudaEventCreate(&ev1_));                                     \
            KZ_TRY(h, cudaEventRecordWithFlags(ev0_, (h)->stream, cudaEventRecordExternal)); \
        }                                                                          \
        KZ_TRY(h, call);                                                           \
        (h)->launches += (nk);                                                     \
        if ((h)->profiling) {                                                      \
            KZ_TRY(h, cudaEventRecordWithFlags(ev1_, (h)->stream, cudaEventRecordExternal)); \
            (h)->prof.push_back({(kind), (nk), ev0_, ev1_});                       \
        }                                                                          \
    } while (0)
#define KZ_LAUNCH(h, kind, call) KZ_LAUNCH_N(h, kind, 1, call)

#define KZ_CHECK(st) \
    do {                                   \
        kaze_status s_ = (st);             \
        if (s_ != KAZE_OK) return s_;      \
    } while (0)

int pitch_for(int w) { return (w + 31) / 32 * 32; }

// Sampled normalised Gaussian, radius ceil(3 sigma) (presmoothing and
// gradient smoothing of Sec. III-1).
bool make_taps(double sigma, int rmax, kz::GaussTaps* t)
{
    int r = (int)std::ceil(3.0 * sigma);
    if (r < 1) r = 1;
    if (r > rmax) return false;
    double w[2 * kz::kMaxGaussR + 1];
    double sum = 0.0;
    for (int j = -r; j <= r; ++j) {
        w[j + r] = std::exp(-(double)j * j / (2.0 * sigma * sigma));
        sum += w[j + r];
    }
    t->r = r;
    for (int j = 0; j <= 2 * r; ++j) t->w[j] = (float)(w[j] / sum);
    return true;
}

// Cross-level radius of the maximum test: 1 (3x3x3), or the sigma x sigma
// window max(1, floor(s / 2)) for the step s of the level.
int cross_radius(const kaze_options& o, int step)
{
    if (o.extrema_window != KAZE_EXTREMA_SIGMA_WINDOW) return 1;
    return step / 2 > 1 ? step / 2 : 1;
}

int step_of(double sigma)
{
    int s = (int)std::floor(sigma + 0.5);
    return s < 1 ? 1 : s;
}

kaze_status check_image(kaze_handle* h, int w, int hh)
{
    if (w < 3 || hh < 3) return fail(h, KAZE_ERR_INVALID_ARG, "image smaller than 3x3");
    if (w > h->max_w || hh > h->max_h) return fail(h, KAZE_ERR_INVALID_ARG, "image larger than the handle's maximum");
    return KAZE_OK;
}

void set_geometry(kaze_handle* h, int w, int hh)
{
    h->cur_w = w;
    h->cur_h = hh;
    h->cur_pitch = pitch_for(w);
    h->cur_plane = (long long)h->cur_pitch * hh;
}

float* level_ptr(kaze_handle* h, int i) { return h->levels + (size_t)i * h->cur_plane; }
float* doh_ptr(kaze_handle* h, int i) { return h->doh + (size_t)i * h->cur_plane; }

// Contrast factor k of the base image into h->d_k (device only).  With
// m2_out (a plane of the handle's pitch) the max pass keeps |grad|^2 there
// and the histogram is taken from it instead of recomputing the gradient.
kaze_status enqueue_contrast(kaze_handle* h, const float* L0, int pitch, int w, int hh, float* m2_out = nullptr)
{
    cudaStream_t st = h->stream;
    if (h->opt.k_override > 0.f) {
        KZ_LAUNCH(h, KK_SET_SCALAR, kz::launch_set_scalar(h->d_k, h->opt.k_override, st));
        return KAZE_OK;
    }
    if (!h->in_detect) {  // a whole detection cleared the control block
        KZ_TRY(h, cudaMemsetAsync(h->d_hmax, 0, sizeof(unsigned int), st));
        KZ_TRY(h, cudaMemsetAsync(h->d_hist, 0, sizeof(unsigned int) * (h->opt.nbins + 1), st));
    }
    KZ_LAUNCH(h, KK_GRAD_MAX, kz::launch_grad_max(L0, pitch, w, hh, h->tapsd, h->d_hmax, st, m2_out));
    if (m2_out) {  // histogram and percentile in one launch
        KZ_LAUNCH(h, KK_GRAD_HIST, kz::launch_hist_m2(m2_out, pitch, w, hh, h->d_hmax, h->d_hist, h->opt.nbins,
                                                      h->opt.k_percentile, h->d_k, st));
    } else {
        KZ_LAUNCH(h, KK_GRAD_HIST,
                  kz::launch_grad_hist(L0, pitch, w, hh, h->tapsd, h->d_hmax, h->d_hist, h->opt.nbins, st));
        KZ_LAUNCH(h, KK_PERCENTILE,
                  kz::launch_percentile(h->d_hist, h->opt.nbins, h->d_hmax, h->opt.k_percentile, h->d_k, st));
    }
    return KAZE_OK;
}

// Sec. II-A: presmoothing, k, then N-1 AOS steps (Eq. 4, tau from Eq. 7).
kaze_status enqueue_build(kaze_handle* h, const float* d_img, int w, int hh, int pitch_elems)
{
    cudaStream_t st = h->stream;
    set_geometry(h, w, hh);
    const int P = h->cur_pitch;
    if (h->in_detect)  // count, status, contrast statistics, barrier: one memset
        KZ_TRY(h, cudaMemsetAsync(h->d_ctl, 0, h->ctl_bytes, st));
    else
        KZ_TRY(h, cudaMemsetAsync(h->d_status, 0, sizeof(int), st));
    const bool resident = h->N > 1 && !h->surrogate && h->opt.scheme == KAZE_SCHEME_AOS &&
                          h->opt.aos_solver == KAZE_AOS_AUTO && h->d_exchange &&
                          kz::evolve_fits(w, hh, h->tapsd.r, nullptr);
    if (resident && kz::evolve_front_fits(h->taps0.r, h->opt.nbins)) {
        // presmoothing, the contrast factor and every AOS step in one
        // cooperative launch, the tiles resident in shared memory
        kz::EvolveFront f;
        f.img = d_img;
        f.img_pitch = pitch_elems;
        f.taps0 = &h->taps0;
        if (h->opt.k_override > 0.f) {
            KZ_LAUNCH(h, KK_SET_SCALAR, kz::launch_set_scalar(h->d_k, h->opt.k_override, st));
        } else {
            if (!h->in_detect) {
                KZ_TRY(h, cudaMemsetAsync(h->d_hmax, 0, sizeof(unsigned int), st));
                KZ_TRY(h, cudaMemsetAsync(h->d_hist, 0, sizeof(unsigned int) * h->opt.nbins, st));
            }
            f.hmax_bits = h->d_hmax;
            f.hist = h->d_hist;
            f.nbins = h->opt.nbins;
            f.pct = h->opt.k_percentile;
        }
        KZ_LAUNCH(h, KK_FRONT_EVOLVE,
                  kz::launch_evolve(h->levels, h->cur_plane, P, w, hh, h->N, h->t, h->d_k, h->tapsd,
                                    h->opt.diffusivity, h->d_exchange, h->max_tiles, h->d_barrier, h->d_status, st,
                                    &f, h->evolve_wait_limit, h->evolve_stall_tile, !h->in_detect));
        h->built = true;
        h->responded = false;
        return KAZE_OK;
    }
    KZ_LAUNCH(h, KK_PRESMOOTH, kz::launch_gaussian(d_img, pitch_elems, level_ptr(h, 0), P, w, hh, h->taps0, st));
    // the streamed tile passes when asked for (the line kernels are faster
    // for the images beyond one tile per SM)
    const bool streamed = !resident && h->N > 1 && !h->surrogate && h->opt.scheme == KAZE_SCHEME_AOS &&
                          h->opt.aos_solver == KAZE_AOS_STREAMED && kz::evolve_stream_fits(w, hh, h->tapsd.r);
    // with k measured here and the line kernels, |grad(G * L_0)|^2 stays in
    // the conductance plane and the first conductance is computed from it
    const bool m2 = h->opt.k_override <= 0.f && !streamed;
    KZ_CHECK(enqueue_contrast(h, level_ptr(h, 0), P, w, hh, m2 ? h->g : nullptr));
    if (streamed) {
        for (int i = 1; i < h->N; ++i) {
            KZ_LAUNCH(h, KK_STREAM_A, kz::launch_stream_pass(0, i, h->levels, h->cur_plane, P, w, hh, h->N, h->t,
                                                             h->d_k, h->tapsd, h->opt.diffusivity, h->g,
                                                             h->d_stream, st));
            KZ_LAUNCH(h, KK_STREAM_X, kz::launch_stream_pass(1, i, h->levels, h->cur_plane, P, w, hh, h->N, h->t,
                                                             h->d_k, h->tapsd, h->opt.diffusivity, h->g,
                                                             h->d_stream, st));
            KZ_LAUNCH(h, KK_STREAM_B, kz::launch_stream_pass(2, i, h->levels, h->cur_plane, P, w, hh, h->N, h->t,
                                                             h->d_k, h->tapsd, h->opt.diffusivity, h->g,
                                                             h->d_stream, st));
        }
        h->built = true;
        h->responded = false;
        return KAZE_OK;
    }
    auto conductance = [&](int i, const float* Lp, float* zero) -> kaze_status {
        if (i == 1 && m2)
            KZ_LAUNCH(h, KK_CONDUCTANCE, kz::launch_cond_m2(h->g, zero, P, w, hh, h->d_k, h->opt.diffusivity, st));
        else
            KZ_LAUNCH(h, KK_CONDUCTANCE,
                      kz::launch_conductance(Lp, h->g, zero, P, w, hh, h->tapsd, h->d_k, h->opt.diffusivity, st));
        return KAZE_OK;
    };
    if (resident) {
        // every AOS step in one cooperative launch from level 0 in its plane
        KZ_LAUNCH(h, KK_EVOLVE,
                  kz::launch_evolve(h->levels, h->cur_plane, P, w, hh, h->N, h->t, h->d_k, h->tapsd,
                                    h->opt.diffusivity, h->d_exchange, h->max_tiles, h->d_barrier, h->d_status, st,
                                    nullptr, h->evolve_wait_limit, h->evolve_stall_tile, !h->in_detect));
        h->built = true;
        h->responded = false;
        return KAZE_OK;
    }
    for (int i = 1; i < h->N; ++i) {
        const float* Lp = level_ptr(h, i - 1);
        float* Li = level_ptr(h, i);
        const float tau = (float)(h->t[i] - h->t[i - 1]);
        if (h->surrogate) {
            KZ_CHECK(conductance(i, Lp, nullptr));
            kz::sg::Samples S;
            std::memset(&S, 0, sizeof(S));
            S.L[0] = Lp;
            S.g[0] = h->g;
            S.out[0] = Li;
            S.s[0] = h->sg_s[i];
            S.n = 1;
            S.w = w;
            S.h = hh;
            S.pitch = P;
            S.opitch = P;
            KZ_LAUNCH(h, KK_SURROGATE, kz::sg::enqueue_pipeline_step(h->surrogate, S, h->d_status, st));
            continue;
        }
        if (h->opt.scheme == KAZE_SCHEME_FED) {
            // one FED cycle: n explicit steps from L_{i-1}, alternating between
            // the row-solution scratch plane and L_i so that the last lands in L_i
            KZ_CHECK(conductance(i, Lp, nullptr));
            // (up to four steps per launch)
            const std::vector<float>& tj = h->fed_tau[i];
            const std::vector<int> ch = kz::fed_chunks((int)tj.size());
            const int q = (int)ch.size();
            const float* src = Lp;
            for (int c = 0, j = 0; c < q; j += ch[(size_t)c], ++c) {
                float* dst = ((q - 1 - c) % 2 == 0) ? Li : h->ux;
                KZ_LAUNCH(h, KK_FED, kz::launch_fed_steps(src, h->g, dst, P, w, hh, tj.data() + j, ch[(size_t)c],
                                                          h->d_status, st));
                src = dst;
            }
            continue;
        }
        // conductance also zeroes L_i; the row and column halves of the AOS
        // step then add into it, concurrently on two streams (one stream
        // while profiling, so that events bracket single kernels)
        KZ_CHECK(conductance(i, Lp, Li));
        const bool fork = !h->profiling && h->side != nullptr;
        if (fork) {
            KZ_TRY(h, cudaEventRecord(h->ev_fork, st));
            KZ_TRY(h, cudaStreamWaitEvent(h->side, h->ev_fork, 0));
        }
        KZ_LAUNCH(h, KK_AOS_ROWS, kz::launch_aos_rows(Lp, h->g, nullptr, Li, P, w, hh, tau, h->d_status, st));
        KZ_LAUNCH(h, KK_AOS_COLS,
                  kz::launch_aos_cols(Lp, h->g, nullptr, Li, P, w, hh, tau, h->d_status, fork ? h->side : st));
        if (fork) {
            KZ_TRY(h, cudaEventRecord(h->ev_join, h->side));
            KZ_TRY(h, cudaStreamWaitEvent(st, h->ev_join, 0));
        }
    }
    h->built = true;
    h->responded = false;
    return KAZE_OK;
}

// The candidate list the response launch fills for the extremum launch.
kz::Candidates candidates(const kaze_handle* h)
{
    kz::Candidates c;
    c.list = h->d_cand;
    c.count = h->d_cand_count;
    c.cap = h->cand_cap;
    c.thr = h->opt.dthreshold;
    c.lo = 1;
    c.hi = h->N - 2;
    return c;
}

kaze_status enqueue_response(kaze_handle* h)
{
    const kz::Candidates c = candidates(h);
    if (!h->in_detect) KZ_TRY(h, cudaMemsetAsync(c.count, 0, sizeof(unsigned int), h->stream));
    KZ_LAUNCH_N(h, KK_DOH, kz::doh_launches(h->tab, 0, h->N),
                kz::launch_doh(h->levels, h->doh, h->cur_pitch, h->cur_plane, h->cur_w, h->cur_h, 0, h->N, h->tab,
                               h->stream, &c));
    h->cand_doh = h->doh;
    h->responded = true;
    return KAZE_OK;
}

// With `listed`, D is the handle's response stack just computed by
// enqueue_response, whose candidate list the extremum launch visits.
kaze_status enqueue_extrema(kaze_handle* h, const float* D, int pitch, long long plane, int w, int hh, int n,
                            const kz::LevelTable& tab, bool listed)
{
    const kz::Candidates c = candidates(h);
    if (!h->in_detect) KZ_TRY(h, cudaMemsetAsync(h->d_count, 0, sizeof(unsigned int), h->stream));
    KZ_LAUNCH_N(h, KK_EXTREMA, n >= 3 ? 1 : 0, kz::launch_extrema(D, pitch, plane, w, hh, n, tab, h->opt.dthreshold, h->opt.edge_r, h->d_kp,
                                 h->opt.max_keypoints, h->d_count, h->stream,
                                 listed && D == h->cand_doh ? &c : nullptr));
    // the count and the status word (adjacent on both sides) in one copy
    static_assert(sizeof(unsigned int) == sizeof(int), "count and status words");
    KZ_TRY(h, cudaMemcpyAsync(h->h_count, h->d_count, 2 * sizeof(unsigned int), cudaMemcpyDeviceToHost, h->stream));
    // the first kp_pre keypoint slots go with the count, so that a detection
    // with no more keypoints than that needs no second round trip to the host
    KZ_TRY(h, cudaMemcpyAsync(h->h_kp_pre, h->d_kp, sizeof(kaze_keypoint) * h->kp_pre, cudaMemcpyDeviceToHost,
                              h->stream));
    return KAZE_OK;
}

// After enqueue_extrema: wait, take the keypoints (from the slots copied with
// the count, or by a second copy when there are more), sort by (level, iy, ix).
kaze_status collect_keypoints(kaze_handle* h, kaze_keypoint* out, int capacity, int* count)
{
    KZ_TRY(h, cudaStreamSynchronize(h->stream));
    if (*h->h_status) return fail(h, KAZE_ERR_TIMEOUT, "a bounded device-side wait ran out");
    const unsigned total = *h->h_count;
    const unsigned have = std::min<unsigned>(total, (unsigned)h->opt.max_keypoints);
    h->hkp.resize(have);
    if (have && have <= (unsigned)h->kp_pre) {
        std::memcpy(h->hkp.data(), h->h_kp_pre, sizeof(kaze_keypoint) * have);
    } else if (have) {
        KZ_TRY(h, cudaMemcpyAsync(h->hkp.data(), h->d_kp, sizeof(kaze_keypoint) * have, cudaMemcpyDeviceToHost,
                                  h->stream));
        KZ_TRY(h, cudaStreamSynchronize(h->stream));
    }
    std::sort(h->hkp.begin(), h->hkp.end(), [](const kaze_keypoint& a, const kaze_keypoint& b) {
        if (a.level != b.level) return a.level < b.level;
        if (a.iy != b.iy) return a.iy < b.iy;
        return a.ix < b.ix;
    });
    const unsigned cap = capacity > 0 ? (unsigned)capacity : 0u;
    const unsigned nout = std::min(have, cap);
    if (nout && out) std::memcpy(out, h->hkp.data(), sizeof(kaze_keypoint) * nout);
    if (count) *count = (int)total;
    if (total > cap || total > (unsigned)h->opt.max_keypoints)
        return fail(h, KAZE_ERR_CAPACITY, "more keypoints than the output capacity");
    return KAZE_OK;
}

void drop_graph(kaze_handle* h)
{
    for (auto& g : h->gslot) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        g = kaze_handle::GraphSlot();
    }
}

// Records build + response + extrema once per (input pointer, size) and
// replays it.
kaze_status run_detect_graph(kaze_handle* h, const float* d_img, int w, int hh, int pitch)
{
    if (h->stream == nullptr || h->stream == cudaStreamLegacy || h->stream == cudaStreamPerThread) {
        // the default streams cannot be captured: launch the same kernels directly
        h->launches = 0;
        h->in_detect = true;
        kaze_status s = enqueue_build(h, d_img, w, hh, pitch);
        if (s == KAZE_OK) s = enqueue_response(h);
        if (s == KAZE_OK) s = enqueue_extrema(h, h->doh, h->cur_pitch, h->cur_plane, w, hh, h->N, h->tab, true);
        h->in_detect = false;
        return s;
    }
    int slot = -1;
    for (int i = 0; i < 2; ++i) {
        const kaze_handle::GraphSlot& g = h->gslot[i];
        if (g.exec && g.img == d_img && g.w == w && g.h == hh && g.pitch == pitch) slot = i;
    }
    if (slot < 0) {
        slot = 1 - h->g_last;  // replace the slot used less recently
        kaze_handle::GraphSlot& g = h->gslot[slot];
        if (g.exec) cudaGraphExecDestroy(g.exec);
        g = kaze_handle::GraphSlot();
        cudaGraph_t graph = nullptr;
        h->launches = 0;
        KZ_TRY(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
        h->in_detect = true;
        kaze_status s = enqueue_build(h, d_img, w, hh, pitch);
        if (s == KAZE_OK) s = enqueue_response(h);
        if (s == KAZE_OK) s = enqueue_extrema(h, h->doh, h->cur_pitch, h->cur_plane, w, hh, h->N, h->tab, true);
        h->in_detect = false;
        cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
        if (s != KAZE_OK) {
            if (graph) cudaGraphDestroy(graph);
            return s;
        }
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&g.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            g.exec = nullptr;
            return cuda_fail(h, e, "cudaGraphInstantiate");
        }
        g.launches = h->launches;
        g.img = d_img;
        g.w = w;
        g.h = hh;
        g.pitch = pitch;
    }
    h->g_last = slot;
    set_geometry(h, w, hh);
    KZ_TRY(h, cudaGraphLaunch(h->gslot[slot].exec, h->stream));
    h->launches = h->gslot[slot].launches;
    h->built = true;
    h->responded = true;
    return KAZE_OK;
}

}  // namespace

// ------------------------------------------------- internal (batch API) ----

namespace kz {

// Enqueues the whole detection of one image on the handle's stream with the
// levels, responses and keypoints going to caller-provided device buffers
// (planes of the handle's pitch for w, packed); the handle lends only its
// scratch (conductance, row solution, contrast statistics, status word).
kaze_status handle_enqueue_into(kaze_handle* h, const float* d_img, int w, int hh, int pitch, float* levels,
                                float* doh, kaze_keypoint* d_kp, unsigned int* d_count, int cap)
{
    KZ_CHECK(check_image(h, w, hh));
    float* own_levels = h->levels;
    float* own_doh = h->doh;
    h->levels = levels;
    h->doh = doh;
    kaze_status s = enqueue_build(h, d_img, w, hh, pitch);
    if (s == KAZE_OK) s = enqueue_response(h);
    h->levels = own_levels;
    h->doh = own_doh;
    KZ_CHECK(s);
    const kz::Candidates c = candidates(h);  // filled by enqueue_response from `doh`
    KZ_TRY(h, cudaMemsetAsync(d_count, 0, sizeof(unsigned int), h->stream));
    KZ_LAUNCH_N(h, KK_EXTREMA, h->N >= 3 ? 1 : 0, kz::launch_extrema(doh, h->cur_pitch, h->cur_plane, w, hh, h->N, h->tab,
                                                h->opt.dthreshold, h->opt.edge_r, d_kp, cap, d_count, h->stream, &c));
    h->built = false;  // the handle's own buffers were not written
    h->responded = false;
    return KAZE_OK;
}

int* handle_status_ptr(kaze_handle* h) { return h->d_status; }

}  // namespace kz

// ------------------------------------------------------------------ ABI ----

KAZE_API void kaze_default_options(kaze_options* o)
{
    if (!o) return;
    o->octaves = 4;
    o->sublevels = 4;
    o->sigma0 = 1.6f;
    o->sigma_d = 1.0f;
    o->k_percentile = 0.7;
    o->nbins = 300;
    o->diffusivity = KAZE_G2;
    o->dthreshold = 0.001f;
    o->edge_r = 10.0f;
    o->doh_norm = KAZE_DOH_SIGMA4;
    o->k_override = 0.0f;
    o->max_keypoints = 65536;
    o->scheme = KAZE_SCHEME_AOS;
    o->fed_tau_max = 0.25f;
    o->extrema_window = KAZE_EXTREMA_3X3;
    o->aos_solver = KAZE_AOS_AUTO;
}

KAZE_API kaze_status kaze_create(const kaze_options* opt, int max_w, int max_h, void* cuda_stream,
                                 kaze_handle** out)
{
    if (!out) return create_fail(KAZE_ERR_INVALID_ARG, "null output pointer");
    *out = nullptr;
    g_create_err.clear();
    kaze_options o;
    if (opt) o = *opt; else kaze_default_options(&o);
    const int N = o.octaves * o.sublevels;
    if (o.octaves < 1 || o.sublevels < 1 || N > kz::kMaxLevels)
        return create_fail(KAZE_ERR_INVALID_ARG, "octaves, sublevels must be >= 1 with octaves*sublevels <= 64");
    if (!(o.sigma0 > 0.f) || !(o.sigma_d > 0.f)) return create_fail(KAZE_ERR_INVALID_ARG, "sigma0 and sigma_d must be > 0");
    if (!(o.k_percentile > 0.0 && o.k_percentile <= 1.0)) return create_fail(KAZE_ERR_INVALID_ARG, "k_percentile must be in (0, 1]");
    if (o.nbins < 1 || o.nbins > kz::kMaxBins) return create_fail(KAZE_ERR_INVALID_ARG, "nbins must be in 1..4096");
    if (o.diffusivity != KAZE_G1 && o.diffusivity != KAZE_G2) return create_fail(KAZE_ERR_INVALID_ARG, "unknown diffusivity");
    if (o.doh_norm != KAZE_DOH_SIGMA4 && o.doh_norm != KAZE_DOH_PAPER_LITERAL)
        return create_fail(KAZE_ERR_INVALID_ARG, "unknown doh_norm");
    if (o.max_keypoints < 1) return create_fail(KAZE_ERR_INVALID_ARG, "max_keypoints must be >= 1");
    if (o.scheme != KAZE_SCHEME_AOS && o.scheme != KAZE_SCHEME_FED)
        return create_fail(KAZE_ERR_INVALID_ARG, "unknown evolution scheme");
    if (!(o.fed_tau_max > 0.f && o.fed_tau_max <= 0.25f))
        return create_fail(KAZE_ERR_INVALID_ARG, "fed_tau_max must lie in (0, 0.25]");
    if (o.extrema_window != KAZE_EXTREMA_3X3 && o.extrema_window != KAZE_EXTREMA_SIGMA_WINDOW)
        return create_fail(KAZE_ERR_INVALID_ARG, "unknown extrema window");
    if (o.aos_solver != KAZE_AOS_AUTO && o.aos_solver != KAZE_AOS_LINES && o.aos_solver != KAZE_AOS_STREAMED)
        return create_fail(KAZE_ERR_INVALID_ARG, "unknown AOS solver");
    if (max_w < 3 || max_h < 3 || max_w > 16384 || max_h > 16384)
        return create_fail(KAZE_ERR_INVALID_ARG, "max_w and max_h must be in 3..16384");
    if (kz::aos_rows_smem_bytes(max_w) == 0 || kz::aos_cols_smem_bytes(max_h) == 0)
        return create_fail(KAZE_ERR_INVALID_ARG, "image lines too long for the shared-memory line solver");

    kaze_handle* h = new (std::nothrow) kaze_handle();
    if (!h) return create_fail(KAZE_ERR_OOM, "host allocation failed");
    h->opt = o;
    h->N = N;
    h->max_w = max_w;
    h->max_h = max_h;
    h->stream = (cudaStream_t)cuda_stream;
    if (!make_taps(o.sigma0, kz::kMaxGaussR, &h->taps0) || !make_taps(o.sigma_d, kz::kMaxGradR, &h->tapsd)) {
        delete h;
        return create_fail(KAZE_ERR_INVALID_ARG, "Gaussian radius too large (sigma0 <= 5.33, sigma_d <= 2)");
    }
    // Eq. 6 (sigma_i = sigma0 2^(o + s/S)) and Eq. 7 (t_i = sigma_i^2 / 2)
    h->tab.n = N;
    h->tab.sublevels = o.sublevels;
    for (int oc = 0; oc < o.octaves; ++oc)
        for (int s = 0; s < o.sublevels; ++s) {
            const int i = oc * o.sublevels + s;
            h->sigma[i] = (double)o.sigma0 * std::pow(2.0, (double)oc + (double)s / o.sublevels);
            h->t[i] = 0.5 * h->sigma[i] * h->sigma[i];
            const int st = step_of(h->sigma[i]);
            h->tab.step[i] = st;
            h->tab.sigma[i] = (float)h->sigma[i];
            h->tab.xr[i] = cross_radius(o, st);
            if (o.doh_norm == KAZE_DOH_PAPER_LITERAL) {
                const double kn = h->sigma[i] / std::pow(2.0, (double)oc);
                h->tab.norm[i] = (float)(kn * kn);
            } else {
                h->tab.norm[i] = (float)((double)st * st * st * st);
            }
        }

    for (int i = 1; i < N; ++i) {
        const std::vector<double> tj = kz::fed_ordered_steps(h->t[i] - h->t[i - 1], (double)o.fed_tau_max);
        h->fed_tau[i].assign(tj.begin(), tj.end());
    }
    {
        cudaError_t ce = kz::configure_filter_kernels();
        const char* what = "configure_filter_kernels";
        if (ce == cudaSuccess) {
            ce = kz::configure_aos_kernels();
            what = "configure_aos_kernels";
        }
        if (ce == cudaSuccess) {
            ce = kz::configure_detector_kernels();
            what = "configure_detector_kernels";
        }
        if (ce == cudaSuccess) {
            ce = kz::configure_describe_kernels();
            what = "configure_describe_kernels";
        }
        if (ce == cudaSuccess) {
            ce = kz::configure_fed_kernels();
            what = "configure_fed_kernels";
        }
        if (ce == cudaSuccess) {
            ce = kz::configure_evolve_kernel();
            what = "configure_evolve_kernel";
        }
        if (ce != cudaSuccess) {
            delete h;
            return create_fail(KAZE_ERR_CUDA, std::string(what) + ": " + cudaGetErrorName(ce) + " " +
                                                  kz::aos_config_error());
        }
    }
    const size_t pm = (size_t)pitch_for(max_w) * max_h;
    h->plane_max = pm;
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    size_t bytes = 0;
    const size_t off_levels = bytes; bytes += al(sizeof(float) * pm * N);
    const size_t off_doh = bytes;    bytes += al(sizeof(float) * pm * N);
    const size_t off_g = bytes;      bytes += al(sizeof(float) * pm);
    const size_t off_ux = bytes;     bytes += al(sizeof(float) * pm);
    const size_t off_stage = bytes;  bytes += al(sizeof(float) * pm);
    const size_t off_stage2 = bytes; bytes += al(sizeof(float) * pm);
    const size_t off_k = bytes;      bytes += al(sizeof(float));
    // the control block (words): [0] keypoint count, [1] status, [2] contrast
    // maximum, [3] candidate count, [8] grid barrier, [32 ..] histogram and
    // its block counter
    const size_t ctl_bytes = sizeof(unsigned int) * (32 + (size_t)o.nbins + 1);
    const size_t off_ctl = bytes;    bytes += al(ctl_bytes);
    // candidates of the extremum test: a sixteenth of the pixels of all
    // levels (more falls back to the full scan)
    const unsigned cand_cap = (unsigned)std::min<size_t>(std::max<size_t>((size_t)N * pm / 16, 65536), 1u << 30);
    const size_t off_cand = bytes;   bytes += al(sizeof(unsigned long long) * cand_cap);
    const size_t off_kp = bytes;     bytes += al(sizeof(kaze_keypoint) * (size_t)o.max_keypoints);
    const size_t off_dkp = bytes;    bytes += al(sizeof(kaze_keypoint) * (size_t)o.max_keypoints);
    const size_t off_desc = bytes;   bytes += al(sizeof(float) * 64 * (size_t)o.max_keypoints);
    int sms = 0, dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t off_xchg = bytes;   bytes += al(sizeof(float) * kz::evolve_exchange_floats(sms));
    const size_t off_strm = bytes;   bytes += al(sizeof(float) * kz::evolve_stream_floats(max_w, max_h));
    cudaError_t e = cudaMalloc(&h->arena, bytes);
    if (e != cudaSuccess) {
        delete h;
        return create_fail(e == cudaErrorMemoryAllocation ? KAZE_ERR_OOM : KAZE_ERR_CUDA,
                           std::string("cudaMalloc of the device arena: ") + cudaGetErrorName(e));
    }
    char* a = (char*)h->arena;
    h->levels = (float*)(a + off_levels);
    h->doh = (float*)(a + off_doh);
    h->g = (float*)(a + off_g);
    h->ux = (float*)(a + off_ux);
    h->staging = (float*)(a + off_stage);
    h->staging2 = (float*)(a + off_stage2);
    h->d_k = (float*)(a + off_k);
    h->d_ctl = (unsigned int*)(a + off_ctl);
    h->ctl_bytes = ctl_bytes;
    h->d_count = h->d_ctl;
    h->d_status = (int*)(h->d_ctl + 1);
    h->d_hmax = h->d_ctl + 2;
    h->d_cand_count = h->d_ctl + 3;
    h->d_barrier = h->d_ctl + 8;
    h->d_hist = h->d_ctl + 32;
    h->d_cand = (unsigned long long*)(a + off_cand);
    h->cand_cap = cand_cap;
    h->d_kp = (kaze_keypoint*)(a + off_kp);
    h->d_dkp = (kaze_keypoint*)(a + off_dkp);
    h->d_desc = (float*)(a + off_desc);
    h->d_exchange = sms > 0 ? (float*)(a + off_xchg) : nullptr;
    h->d_stream = (float*)(a + off_strm);
    h->max_tiles = sms;
    e = cudaMallocHost(&h->h_count, 2 * sizeof(unsigned int));
    if (e != cudaSuccess) {
        cudaFree(h->arena);
        delete h;
        return create_fail(KAZE_ERR_CUDA, std::string("cudaMallocHost: ") + cudaGetErrorName(e));
    }
    *h->h_count = 0;
    h->h_status = (int*)(h->h_count + 1);
    *h->h_status = 0;
    h->kp_pre = std::min(o.max_keypoints, kz::kKeypointsWithCount);
    e = cudaMallocHost(&h->h_kp_pre, sizeof(kaze_keypoint) * h->kp_pre);
    if (e != cudaSuccess) {
        cudaFreeHost(h->h_count);
        cudaFree(h->arena);
        delete h;
        return create_fail(KAZE_ERR_CUDA, std::string("cudaMallocHost: ") + cudaGetErrorName(e));
    }
    if ((e = cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&h->copy, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&h->ev_copied, cudaEventDisableTiming)) != cudaSuccess) {
        kaze_destroy(h);
        return create_fail(KAZE_ERR_CUDA, std::string("stream / event creation: ") + cudaGetErrorName(e));
    }
    *out = h;
    return KAZE_OK;
}

KAZE_API kaze_status kaze_set_stream(kaze_handle* h, void* cuda_stream)
{
    if (!h) return KAZE_ERR_INVALID_ARG;
    h->stream = (cudaStream_t)cuda_stream;
    return KAZE_OK;
}

KAZE_API kaze_status kaze_build_scale_space(kaze_handle* h, const float* d_img, int w, int hh, int pitch_elems)
{
    if (!h || !d_img) return fail(h, KAZE_ERR_INVALID_ARG, "null argument");
    KZ_CHECK(check_image(h, w, hh));
    if (pitch_elems < w) return fail(h, KAZE_ERR_INVALID_ARG, "pitch smaller than width");
    h->launches = 0;
    return enqueue_build(h, d_img, w, hh, pitch_elems);
}

KAZE_API kaze_status kaze_get_level(kaze_handle* h, int i, const float** d_level, int* pitch_elems, float* t_i)
{
    if (!h) return KAZE_ERR_INVALID_ARG;
    if (i < 0 || i >= h->N) return fail(h, KAZE_ERR_INVALID_ARG, "level index out of range");
    if (!h->built) return fail(h, KAZE_ERR_STATE, "no scale space built yet");
    if (d_level) *d_level = level_ptr(h, i);
    if (pitch_elems) *pitch_elems = h->cur_pitch;
    if (t_i) *t_i = (float)h->t[i];
    return KAZE_OK;
}

KAZE_API kaze_status kaze_set_evolve_wait_limit(kaze_handle* h, long long cycles, int stall_tile)
{
    if (!h) return KAZE_ERR_INVALID_ARG;
    if (cycles < 0) return fail(h, KAZE_ERR_INVALID_ARG, "negative wait limit");
    h->evolve_wait_limit = cycles;
    h->evolve_stall_tile = stall_tile < 0 ? -1 : stall_tile;
    drop_graph(h);  // recorded graphs hold the old launch parameters
    return KAZE_OK;
}

KAZE_API kaze_status kaze_get_level_scale(kaze_handle* h, int i, float* sigma_i, float* t_i)
{
    if (!h) return KAZE_ERR_INVALID_ARG;
    if (i < 0 || i >= h->N) return fail(h, KAZE_ERR_INVALID_ARG, "level index out of range");
    if (sigma_i) *sigma_i = h->tab.sigma[i];  // Eq. 6, the value the kernels use
    if (t_i) *t_i = (float)h->t[i];          // Eq. 7
    return KAZE_OK;
}

KAZE_API kaze_status kaze_get_contrast(kaze_handle* h, float* k)
{
    if (!h || !k) return KAZE_ERR_INVALID_ARG;
    if (!h->built) return fail(h, KAZE_ERR_STATE, "no scale space built yet");
    KZ_TRY(h, cudaMemcpyAsync(k, h->d_k, sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    KZ_TRY(h, cudaMemcpyAsync(h->h_status, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    KZ_TRY(h, cudaStreamSynchronize(h->stream));
    if (*h->h_status) return fail(h, KAZE_ERR_TIMEOUT, "a bounded device-side wait ran out");
    return KAZE_OK;
}

KAZE_API kaze_status kaze_detector_response(kaze_handle* h)
{
    if (!h) return KAZE_ERR_INVALID_ARG;
    if (!h->built) return fail(h, KAZE_ERR_STATE, "no scale space built yet");
    return enqueue_response(h);
}

KAZE_API kaze_status kaze_get_response(kaze_handle* h, int i, const float** d_doh, int* pitch_elems)
{
    if (!h) return KAZE_ERR_INVALID_ARG;
    if (i < 0 || i >= h->N) return fail(h, KAZE_ERR_INVALID_ARG, "level index out of range");
    if (!h->responded) return fail(h, KAZE_ERR_STATE, "no detector response computed yet");
    if (d_doh) *d_doh = doh_ptr(h, i);
    if (pitch_elems) *pitch_elems = h->cur_pitch;
    return KAZE_OK;
}

KAZE_API kaze_status kaze_find_extrema(kaze_handle* h, kaze_keypoint* h_out, int capacity, int* count)
{
    if (!h || capacity < 0 || (capacity > 0 && !h_out)) return fail(h, KAZE_ERR_INVALID_ARG, "bad output");
    if (!h->responded) return fail(h, KAZE_ERR_STATE, "no detector response computed yet");
    KZ_CHECK(enqueue_extrema(h, h->doh, h->cur_pitch, h->cur_plane, h->cur_w, h->cur_h, h->N, h->tab, true));
    return collect_keypoints(h, h_out, capacity, count);
}

KAZE_API kaze_status kaze_detect(kaze_handle* h, const float* d_img, int w, int hh, int pitch_elems,
                                 kaze_keypoint* h_out, int capacity, int* count)
{
    if (!h || !d_img || capacity < 0 || (capacity > 0 && !h_out))
        return fail(h, KAZE_ERR_INVALID_ARG, "null argument");
    KZ_CHECK(check_image(h, w, hh));
    if (pitch_elems < w) return fail(h, KAZE_ERR_INVALID_ARG, "pitch smaller than width");
    KZ_CHECK(run_detect_graph(h, d_img, w, hh, pitch_elems));
    return collect_keypoints(h, h_out, capacity, count);
}

KAZE_API kaze_status kaze_detect_enqueue(kaze_handle* h, const float* d_img, int w, int hh, int pitch_elems)
{
    if (!h || !d_img) return fail(h, KAZE_ERR_INVALID_ARG, "null argument");
    KZ_CHECK(check_image(h, w, hh));
    if (pitch_elems < w) return fail(h, KAZE_ERR_INVALID_ARG, "pitch smaller than width");
    KZ_CHECK(run_detect_graph(h, d_img, w, hh, pitch_elems));
    h->pending = true;
    return KAZE_OK;
}

KAZE_API kaze_status kaze_detect_collect(kaze_handle* h, kaze_keypoint* h_out, int capacity, int* count)
{
    if (!h || capacity < 0 || (capacity > 0 && !h_out)) return fail(h, KAZE_ERR_INVALID_ARG, "null argument");
    if (!h->pending) return fail(h, KAZE_ERR_STATE, "no detection enqueued");
    h->pending = false;
    return collect_keypoints(h, h_out, capacity, count);
}

namespace {
// Detection of a host image through the staging planes: the image is the
// one copied ahead by the previous call (same pointer, size and pitch), or
// is copied now; with h_next, the next image is copied into the other plane
// on the copy stream while this one is detected.
kaze_status detect_host_impl(kaze_handle* h, const float* h_img, const float* h_next, int w, int hh,
                             int pitch_elems, kaze_keypoint* h_out, int capacity, int* count)
{
    if (!h || !h_img || capacity < 0 || (capacity > 0 && !h_out))
        return fail(h, KAZE_ERR_INVALID_ARG, "null argument");
    KZ_CHECK(check_image(h, w, hh));
    if (pitch_elems < w) return fail(h, KAZE_ERR_INVALID_ARG, "pitch smaller than width");
    const int sp = pitch_for(w);
    float* planes[2] = {h->staging, h->staging2};
    // the main stream never touches a plane before a copy issued into it has landed
    if (h->pre_issued) KZ_TRY(h, cudaStreamWaitEvent(h->stream, h->ev_copied, 0));
    int slot;
    if (h->pre_slot >= 0 && h->pre_src == h_img && h->pre_w == w && h->pre_h == hh && h->pre_pitch == pitch_elems) {
        slot = h->pre_slot;
    } else {
        slot = h->pre_slot >= 0 ? 1 - h->pre_slot : 0;
        KZ_TRY(h, cudaMemcpy2DAsync(planes[slot], sizeof(float) * sp, h_img, sizeof(float) * pitch_elems,
                                    sizeof(float) * w, hh, cudaMemcpyHostToDevice, h->stream));
    }
    h->pre_slot = -1;
    h->pre_src = nullptr;
    KZ_CHECK(run_detect_graph(h, planes[slot], w, hh, sp));
    if (h_next) {
        // the other plane was last read by the previous detection, which the
        // previous call waited for (collect_keypoints synchronises)
        const int other = 1 - slot;
        KZ_TRY(h, cudaMemcpy2DAsync(planes[other], sizeof(float) * sp, h_next, sizeof(float) * pitch_elems,
                                    sizeof(float) * w, hh, cudaMemcpyHostToDevice, h->copy));
        KZ_TRY(h, cudaEventRecord(h->ev_copied, h->copy));
        h->pre_issued = true;
        h->pre_src = h_next;
        h->pre_slot = other;
        h->pre_w = w;
        h->pre_h = hh;
        h->pre_pitch = pitch_elems;
    }
    return collect_keypoints(h, h_out, capacity, count);
}
}  // namespace

KAZE_API kaze_status kaze_detect_host(kaze_handle* h, const float* h_img, int w, int hh, int pitch_elems,
                                      kaze_keypoint* h_out, int capacity, int* count)
{
    return detect_host_impl(h, h_img, nullptr, w, hh, pitch_elems, h_out, capacity, count);
}

KAZE_API kaze_status kaze_detect_host_next(kaze_handle* h, const float* h_img, const float* h_next, int w, int hh,
                                           int pitch_elems, kaze_keypoint* h_out, int capacity, int* count)
{
    return detect_host_impl(h, h_img, h_next, w, hh, pitch_elems, h_out, capacity, count);
}

namespace {
// waits for the stream and reports a bounded device-side wait that ran out
kaze_status sync_status(kaze_handle* h)
{
    KZ_TRY(h, cudaMemcpyAsync(h->h_status, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    KZ_TRY(h, cudaStreamSynchronize(h->stream));
    if (*h->h_status) return fail(h, KAZE_ERR_TIMEOUT, "a bounded device-side wait ran out");
    return KAZE_OK;
}
}  // namespace

KAZE_API kaze_status kaze_op_fed_cycle(kaze_handle* h, const float* d_Lprev, const float* d_g, float* d_scratch,
                                       float* d_Lnext, int pitch, int w, int hh, float dt, int* n_steps)
{
    if (!h || !d_Lprev || !d_g || !d_scratch || !d_Lnext) return fail(h, KAZE_ERR_INVALID_ARG, "null argument");
    KZ_CHECK(check_image(h, w, hh));
    if (pitch < w || pitch % 4) return fail(h, KAZE_ERR_INVALID_ARG, "pitch must be >= w and a multiple of 4");
    const uintptr_t al = (uintptr_t)d_Lprev | (uintptr_t)d_g | (uintptr_t)d_scratch | (uintptr_t)d_Lnext;
    if (al & 15) return fail(h, KAZE_ERR_INVALID_ARG, "buffers must be 16-byte aligned");
    if (d_Lnext == d_Lprev || d_Lnext == d_g || d_scratch == d_Lprev || d_scratch == d_g || d_scratch == d_Lnext)
        return fail(h, KAZE_ERR_INVALID_ARG, "outputs alias inputs");
    if (!(dt >= 0.f) || !std::isfinite(dt)) return fail(h, KAZE_ERR_INVALID_ARG, "bad stopping time");
    const std::vector<double> tj = kz::fed_ordered_steps((double)dt, (double)h->opt.fed_tau_max);
    const int n = (int)tj.size();
    h->launches = 0;
    KZ_TRY(h, cudaMemsetAsync(h->d_status, 0, sizeof(int), h->stream));
    if (n == 0) {
        KZ_TRY(h, cudaMemcpy2DAsync(d_Lnext, sizeof(float) * pitch, d_Lprev, sizeof(float) * pitch, sizeof(float) * w,
                                    hh, cudaMemcpyDeviceToDevice, h->stream));
    }
    std::vector<float> tf(tj.begin(), tj.end());
    const std::vector<int> ch = kz::fed_chunks(n);
    const int q = (int)ch.size();
    const float* src = d_Lprev;
    for (int c = 0, j = 0; c < q; j += ch[(size_t)c], ++c) {
        float* dst = ((q - 1 - c) % 2 == 0) ? d_Lnext : d_scratch;
        KZ_LAUNCH(h, KK_FED,
                  kz::launch_fed_steps(src, d_g, dst, pitch, w, hh, tf.data() + j, ch[(size_t)c], h->d_status,
                                       h->stream));
        src = dst;
    }
    if (n_steps) *n_steps = n;
    return sync_status(h);
}

KAZE_API kaze_status kaze_op_fed_steps(kaze_handle* h, const float* d_Lprev, const float* d_g, float* d_Lnext,
                                       int pitch, int w, int hh, const float* h_tau, int k)
{
    if (!h || !d_Lprev || !d_g || !d_Lnext || !h_tau) return fail(h, KAZE_ERR_INVALID_ARG, "null argument");
    KZ_CHECK(check_image(h, w, hh));
    if (pitch < w || pitch % 4) return fail(h, KAZE_ERR_INVALID_ARG, "pitch must be >= w and a multiple of 4");
    if (((uintptr_t)d_Lprev | (uintptr_t)d_g | (uintptr_t)d_Lnext) & 15)
        return fail(h, KAZE_ERR_INVALID_ARG, "buffers must be 16-byte aligned");
    if (d_Lnext == d_Lprev || d_Lnext == d_g) return fail(h, KAZE_ERR_INVALID_ARG, "output aliases an input");
    if (k < 1 || k > kz::fed_max_fused()) return fail(h, KAZE_ERR_INVALID_ARG, "k must be 1..4");
    for (int j = 0; j < k; ++j)
        if (!std::isfinite(h_tau[j])) return fail(h, KAZE_ERR_INVALID_ARG, "step size not finite");
    h->launches = 0;
    KZ_TRY(h, cudaMemsetAsync(h->d_status, 0, sizeof(int), h->stream));
    KZ_LAUNCH(h, KK_FED, kz::launch_fed_steps(d_Lprev, d_g, d_Lnext, pitch, w, hh, h_tau, k, h->d_status, h->stream));
    return sync_status(h);
}

// ---- description (Sec. II-C) -------------------------------------------------

namespace {

kz::DescTable desc_table(const kaze_handle* h)
{
    kz::DescTable t;
    std::memset(&t, 0, sizeof(t));
    t.n = h->N;
    t.single = 0;
    for (int i = 0; i < h->N; ++i) {
        t.sigma[i] = (float)h->sigma[i];
        t.step[i] = h->tab.step[i];
    }
    return t;
}

kaze_status check_host_keypoints(kaze_handle* h, const kaze_keypoint* kps, int n, bool need_level)
{
    for (int i = 0; i < n; ++i) {
        if (!std::isfinite(kps[i].x) || !std::isfinite(kps[i].y))
            return fail(h, KAZE_ERR_INVALID_ARG, "keypoint position is not finite");
        if (need_level && (kps[i].level < 0 || kps[i].level >= h->N))
            return fail(h, KAZE_ERR_INVALID_ARG, "keypoint level out of range");
    }
    return KAZE_OK;
}

// Upload, describe, download; synchronises.
kaze_status describe_host(kaze_handle* h, const float* levels, long long plane, int pitch, int w, int hh,
                          const kz::DescTable& tab, kaze_keypoint* kps, int n, float* desc, int upright)
{
    h->launches = 0;
    if (n == 0) return KAZE_OK;
    KZ_TRY(h, cudaMemcpyAsync(h->d_dkp, kps, sizeof(kaze_keypoint) * (size_t)n, cudaMemcpyHostToDevice, h->stream));
    KZ_LAUNCH(h, KK_DESCRIBE, kz::launch_describe(levels, plane, pitch, w, hh, tab, h->d_dkp, n, h->d_desc, upright,
                                                  h->stream));
    KZ_TRY(h, cudaMemcpyAsync(desc, h->d_desc, sizeof(float) * 64 * (size_t)n, cudaMemcpyDeviceToHost, h->stream));
    KZ_TRY(h, cudaMemcpyAsync(kps, h->d_dkp, sizeof(kaze_keypoint) * (size_t)n, cudaMemcpyDeviceToHost, h->stream));
    KZ_TRY(h, cudaStreamSynchronize(h->stream));
    return KAZE_OK;
}

}  // namespace

KAZE_API kaze_status kaze_describe(kaze_handle* h, kaze_keypoint* kps, int n, float* desc, int upright)
{
    if (!h || n < 0 || (n > 0 && (!kps || !desc))) return fail(h, KAZE_ERR_INVALID_ARG, "null argument");
    if (!h->built) return fail(h, KAZE_ERR_STATE, "no scale space built yet");
    if (n > h->opt.max_keypoints) return fail(h, KAZE_ERR_CAPACITY, "more keypoints than max_keypoints");
    KZ_CHECK(check_host_keypoints(h, kps, n, true));
    return describe_host(h, h->levels, h->cur_plane, h->cur_pitch, h->cur_w, h->cur_h, desc_table(h), kps, n, desc,
                         upright);
}

KAZE_API kaze_status kaze_describe_device(kaze_handle* h, kaze_keypoint* d_kps, int n, float* d_desc, int upright)
{
    if (!h || n < 0 || (n > 0 && (!d_kps || !d_desc))) return fail(h, KAZE_ERR_INVALID_ARG, "null argument");
    if (!h->built) return fail(h, KAZE_ERR_STATE, "no scale space built yet");
    h->launches = 0;
    if (n == 0) return KAZE_OK;
    KZ_LAUNCH(h, KK_DESCRIBE, kz::launch_describe(h->levels, h->cur_plane, h->cur_pitch, h->cur_w, h->cur_h,
                                                  desc_table(h), d_kps, n, d_desc, upright, h->stream));
    return KAZE_OK;
}

KAZE_API kaze_status kaze_op_describe(kaze_handle* h, const float* d_L, int pitch, int w, int hh, float sigma,
                                      kaze_keypoint* kps, int n, float* desc, int upright)
{
    if (!h || !d_L || n < 0 || (n > 0 && (!kps || !desc))) return fail(h, KAZE_ERR_INVALID_ARG, "null argument");
    KZ_CHECK(check_image(h, w, hh));
    if (pitch < w) return fail(h, KAZE_ERR_INVALID_ARG, "pitch smaller than width");
    if (!(sigma > 0.f) || !std::isfinite(sigma) || sigma > 1e4f) return fail(h, KAZE_ERR_INVALID_ARG, "bad sigma");
    if (n > h->opt.max_keypoints) return fail(h, KAZE_ERR_CAPACITY, "more keypoints than max_keypoints");
    KZ_CHECK(check_host_keypoints(h, kps, n, false));
    kz::DescTable t;
    std::memset(&t, 0, sizeof(t));
    t.n = 1;
    t.single = 1;
    t.sigma[0] = sigma;
    t.step[0] = step_of(sigma);
    return describe_host(h, d_L, 0, pitch, w, hh, t, kps, n, desc, upright);
}

// ---- single steps ----------------------------------------------------------

KAZE_API kaze_status kaze_op_gaussian(kaze_handle* h, const float* d_in, int in_pitch, float* d_out, int out_pitch,
                                      int w, int hh, float sigma)
{
    if (!h || !d_in || !d_out || d_in == d_out) return fail(h, KAZE_ERR_INVALID_ARG, "bad buffers");
    KZ_CHECK(check_image(h, w, hh));
    if (in_pitch < w || out_pitch < w) return fail(h, KAZE_ERR_INVALID_ARG, "pitch smaller than width");
    kz::GaussTaps t;
    if (!(sigma > 0.f) || !make_taps(sigma, kz::kMaxGaussR, &t)) return fail(h, KAZE_ERR_INVALID_ARG, "bad sigma");
    KZ_TRY(h, kz::launch_gaussian(d_in, in_pitch, d_out, out_pitch, w, hh, t, h->stream));
    return KAZE_OK;
}

KAZE_API kaze_status kaze_op_contrast(kaze_handle* h, const float* d_L0, int pitch, int w, int hh, float* h_k,
                                      float* h_hmax, unsigned int* h_hist)
{
    if (!h || !d_L0) return fail(h, KAZE_ERR_INVALID_ARG, "null argument");
    KZ_CHECK(check_image(h, w, hh));
    if (pitch < w) return fail(h, KAZE_ERR_INVALID_ARG, "pitch smaller than width");
    const float ko = h->opt.k_override;
    h->opt.k_override = 0.f;  // this op always measures
    kaze_status s = enqueue_contrast(h, d_L0, pitch, w, hh);
    h->opt.k_override = ko;
    KZ_CHECK(s);
    float k = 0.f;
    unsigned int hm = 0;
    KZ_TRY(h, cudaMemcpyAsync(&k, h->d_k, sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    KZ_TRY(h, cudaMemcpyAsync(&hm, h->d_hmax, sizeof(unsigned int), cudaMemcpyDeviceToHost, h->stream));
    if (h_hist)
        KZ_TRY(h, cudaMemcpyAsync(h_hist, h->d_hist, sizeof(unsigned int) * h->opt.nbins, cudaMemcpyDeviceToHost,
                                  h->stream));
    KZ_TRY(h, cudaStreamSynchronize(h->stream));
    if (h_k) *h_k = k;
    if (h_hmax) {
        float f;
        std::memcpy(&f, &hm, sizeof(float));
        *h_hmax = f;
    }
    return KAZE_OK;
}

KAZE_API kaze_status kaze_op_conductance(kaze_handle* h, const float* d_L, float* d_g, int pitch, int w, int hh,
                                         float k)
{
    if (!h || !d_L || !d_g || d_L == d_g) return fail(h, KAZE_ERR_INVALID_ARG, "bad buffers");
    KZ_CHECK(check_image(h, w, hh));
    if (pitch < w || !(k > 0.f)) return fail(h, KAZE_ERR_INVALID_ARG, "bad pitch or k");
    KZ_TRY(h, kz::launch_set_scalar(h->d_k, k, h->stream));
    KZ_TRY(h, kz::launch_conductance(d_L, d_g, nullptr, pitch, w, hh, h->tapsd, h->d_k, h->opt.diffusivity, h->stream));
    return KAZE_OK;
}

KAZE_API kaze_status kaze_op_aos_step(kaze_handle* h, const float* d_Lprev, const float* d_g, float* d_ux,
                                      float* d_Lnext, int pitch, int w, int hh, float tau)
{
    if (!h || !d_Lprev || !d_g || !d_ux || !d_Lnext) return fail(h, KAZE_ERR_INVALID_ARG, "null argument");
    KZ_CHECK(check_image(h, w, hh));
    if (pitch < w || pitch % 4) return fail(h, KAZE_ERR_INVALID_ARG, "pitch must be >= w and a multiple of 4");
    const uintptr_t al = (uintptr_t)d_Lprev | (uintptr_t)d_g | (uintptr_t)d_ux | (uintptr_t)d_Lnext;
    if (al & 15) return fail(h, KAZE_ERR_INVALID_ARG, "buffers must be 16-byte aligned");
    {
        // planes span pitch * (h - 1) + w floats: no output may overlap an
        // input or the other output anywhere (the column pass writes while
        // it still reads)
        const size_t span = sizeof(float) * ((size_t)pitch * (hh - 1) + w);
        if (kz::ranges_overlap(d_Lnext, d_Lprev, span) || kz::ranges_overlap(d_Lnext, d_g, span) ||
            kz::ranges_overlap(d_ux, d_Lprev, span) || kz::ranges_overlap(d_ux, d_g, span) ||
            kz::ranges_overlap(d_ux, d_Lnext, span))
            return fail(h, KAZE_ERR_INVALID_ARG, "outputs overlap inputs");
    }
    if (!(tau >= 0.f)) return fail(h, KAZE_ERR_INVALID_ARG, "negative tau");
    KZ_TRY(h, cudaMemsetAsync(h->d_status, 0, sizeof(int), h->stream));
    KZ_TRY(h, kz::launch_aos_rows(d_Lprev, d_g, d_ux, nullptr, pitch, w, hh, tau, h->d_status, h->stream));
    KZ_TRY(h, kz::launch_aos_cols(d_Lprev, d_g, d_ux, d_Lnext, pitch, w, hh, tau, h->d_status, h->stream));
    KZ_TRY(h, cudaMemcpyAsync(h->h_status, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    KZ_TRY(h, cudaStreamSynchronize(h->stream));
    if (*h->h_status) return fail(h, KAZE_ERR_TIMEOUT, "a bounded device-side wait ran out");
    return KAZE_OK;
}

KAZE_API kaze_status kaze_op_doh(kaze_handle* h, const float* d_L, float* d_D, int pitch, int w, int hh,
                                 float sigma_i, int octave)
{
    if (!h || !d_L || !d_D || d_L == d_D) return fail(h, KAZE_ERR_INVALID_ARG, "bad buffers");
    KZ_CHECK(check_image(h, w, hh));
    if (pitch < w || !(sigma_i > 0.f) || octave < 0) return fail(h, KAZE_ERR_INVALID_ARG, "bad pitch/sigma/octave");
    kz::LevelTable t = h->tab;
    t.n = 1;
    t.step[0] = step_of(sigma_i);
    t.sigma[0] = sigma_i;
    if (h->opt.doh_norm == KAZE_DOH_PAPER_LITERAL) {
        const double kn = (double)sigma_i / std::pow(2.0, (double)octave);
        t.norm[0] = (float)(kn * kn);
    } else {
        const double s = t.step[0];
        t.norm[0] = (float)(s * s * s * s);
    }
    KZ_TRY(h, kz::launch_doh(d_L, d_D, pitch, 0, w, hh, 0, 1, t, h->stream));
    return KAZE_OK;
}

KAZE_API kaze_status kaze_op_extrema(kaze_handle* h, const float* d_D, int pitch, long long plane_stride, int w,
                                     int hh, int n, const float* h_sigma, kaze_keypoint* h_out, int capacity,
                                     int* count)
{
    if (!h || !d_D || !h_sigma || capacity < 0 || (capacity > 0 && !h_out))
        return fail(h, KAZE_ERR_INVALID_ARG, "null argument");
    KZ_CHECK(check_image(h, w, hh));
    if (pitch < w || plane_stride < (long long)pitch * hh || n < 1 || n > kz::kMaxLevels)
        return fail(h, KAZE_ERR_INVALID_ARG, "bad pitch, plane stride or level count");
    if (pitch % 4 || plane_stride % 4 || ((uintptr_t)d_D & 15))
        return fail(h, KAZE_ERR_INVALID_ARG, "responses must be 16-byte aligned with pitch and plane stride % 4 == 0");
    kz::LevelTable t = h->tab;
    t.n = n;
    for (int i = 0; i < n; ++i) {
        t.sigma[i] = h_sigma[i];
        t.xr[i] = cross_radius(h->opt, step_of(h_sigma[i]));
    }
    KZ_CHECK(enqueue_extrema(h, d_D, pitch, plane_stride, w, hh, n, t, false));
    return collect_keypoints(h, h_out, capacity, count);
}

KAZE_API kaze_status kaze_load_surrogate(kaze_handle* h, const char* path)
{
    if (!h) return KAZE_ERR_INVALID_ARG;
    if (!path) {  // back to AOS
        kaze_set_surrogate(h, nullptr);
        if (h->own_surrogate) kaze_surrogate_destroy(h->own_surrogate);
        h->own_surrogate = nullptr;
        return KAZE_OK;
    }
    kaze_surrogate* s = nullptr;
    kaze_status st = kaze_surrogate_create(0, 0, 0, 0, 0ull, (void*)h->stream, &s);
    if (st != KAZE_OK) return fail(h, st, std::string("kaze_surrogate_create: ") + kaze_surrogate_last_error(nullptr));
    st = kaze_surrogate_load(s, path);
    if (st != KAZE_OK) {
        const std::string msg = std::string("kaze_surrogate_load: ") + kaze_surrogate_last_error(s);
        kaze_surrogate_destroy(s);
        return fail(h, st, msg);
    }
    kaze_set_surrogate(h, s);
    if (h->own_surrogate) kaze_surrogate_destroy(h->own_surrogate);
    h->own_surrogate = s;
    return KAZE_OK;
}

KAZE_API kaze_status kaze_build_batch(kaze_handle* h, const float* const* d_imgs, const int* w, const int* hh, int n,
                                      kaze_keypoint* h_out, int capacity, int* counts)
{
    if (!h || !d_imgs || !w || !hh || n < 1 || capacity < 0 || (capacity > 0 && !h_out) || !counts)
        return fail(h, KAZE_ERR_INVALID_ARG, "bad batch arguments");
    const std::vector<int> ws(w, w + n), hs(hh, hh + n);
    if (!h->batch || ws != h->batch_w || hs != h->batch_h) {
        if (h->batch) kaze_batch_destroy(h->batch);
        h->batch = nullptr;
        kaze_batch* b = nullptr;
        const kaze_status st = kaze_batch_create(&h->opt, n, w, hh, (void*)h->stream, &b);
        if (st != KAZE_OK) return fail(h, st, "kaze_batch_create refused the batch (sizes 3..4096; AOS, 3x3x3 maxima)");
        h->batch = b;
        h->batch_w = ws;
        h->batch_h = hs;
    }
    const kaze_status st = kaze_batch_detect(h->batch, d_imgs, nullptr, h_out, capacity, counts);
    if (st != KAZE_OK && st != KAZE_ERR_CAPACITY)
        return fail(h, st, std::string("kaze_batch_detect: ") + kaze_batch_last_error(h->batch));
    return st;
}

KAZE_API kaze_status kaze_set_surrogate(kaze_handle* h, kaze_surrogate* s)
{
    if (!h) return KAZE_ERR_INVALID_ARG;
    drop_graph(h);
    h->surrogate = s;
    if (s) {
        for (int i = 1; i < h->N; ++i)
            h->sg_s[i] = kz::sg::input_scale(h->t[i] - h->t[i - 1]);
    }
    h->built = false;
    h->responded = false;
    return KAZE_OK;
}

KAZE_API int kaze_kernel_kinds(void) { return KK_COUNT; }

KAZE_API const char* kaze_kernel_name(int kind)
{
    return (kind >= 0 && kind < KK_COUNT) ? kKindNames[kind] : "";
}

KAZE_API int kaze_last_launch_count(const kaze_handle* h) { return h ? h->launches : -1; }

KAZE_API kaze_status kaze_profile(kaze_handle* h, const float* d_img, int w, int hh, int pitch_elems,
                                  double* h_ms, int* h_launches)
{
    if (!h || !d_img || !h_ms || !h_launches) return fail(h, KAZE_ERR_INVALID_ARG, "null argument");
    KZ_CHECK(check_image(h, w, hh));
    if (pitch_elems < w) return fail(h, KAZE_ERR_INVALID_ARG, "pitch smaller than width");
    for (int k = 0; k < KK_COUNT; ++k) {
        h_ms[k] = 0.0;
        h_launches[k] = 0;
    }
    // The launch sequence with an event pair around every kernel; on a
    // capturable stream it is recorded as a graph and replayed twice (the
    // events keep the second replay's times), so the kernels are timed as a
    // detection runs them.  The default streams replay nothing: eager timing.
    const bool capture = !(h->stream == nullptr || h->stream == cudaStreamLegacy || h->stream == cudaStreamPerThread);
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    h->profiling = true;
    h->launches = 0;
    if (capture) KZ_TRY(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    kaze_status s = enqueue_build(h, d_img, w, hh, pitch_elems);
    if (s == KAZE_OK) s = enqueue_response(h);
    if (s == KAZE_OK) s = enqueue_extrema(h, h->doh, h->cur_pitch, h->cur_plane, w, hh, h->N, h->tab, true);
    h->profiling = false;
    cudaError_t e = cudaSuccess;
    if (capture) {
        e = cudaStreamEndCapture(h->stream, &graph);
        if (s == KAZE_OK && e == cudaSuccess) e = cudaGraphInstantiate(&gexec, graph, 0);
        for (int r = 0; r < 2 && s == KAZE_OK && e == cudaSuccess; ++r) e = cudaGraphLaunch(gexec, h->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
    for (auto& p : h->prof) {
        float ms = 0.f;
        if (s == KAZE_OK && e == cudaSuccess) {
            e = cudaEventElapsedTime(&ms, p.start, p.stop);
            h_ms[p.kind] += ms;
            h_launches[p.kind] += p.kernels;
        }
        cudaEventDestroy(p.start);
        cudaEventDestroy(p.stop);
    }
    h->prof.clear();
    if (s != KAZE_OK) return s;
    if (e != cudaSuccess) return cuda_fail(h, e, "kaze_profile (graph replay or event timing)");
    return KAZE_OK;
}

KAZE_API const char* kaze_status_string(kaze_status s)
{
    switch (s) {
        case KAZE_OK: return "ok";
        case KAZE_ERR_INVALID_ARG: return "invalid argument";
        case KAZE_ERR_CUDA: return "CUDA error";
        case KAZE_ERR_OOM: return "out of device memory";
        case KAZE_ERR_CAPACITY: return "keypoint capacity exceeded";
        case KAZE_ERR_TIMEOUT: return "device-side wait timed out";
        case KAZE_ERR_STATE: return "call out of order";
    }
    return "unknown status";
}

KAZE_API const char* kaze_last_error(const kaze_handle* h)
{
    if (!h) return g_create_err.c_str();
    return h->err.c_str();
}

KAZE_API void kaze_destroy(kaze_handle* h)
{
    if (!h) return;
    if (h->copy) cudaStreamSynchronize(h->copy);  // a copy of the next host image may still be landing
    drop_graph(h);
    if (h->arena) cudaFree(h->arena);
    if (h->h_count) cudaFreeHost(h->h_count);
    if (h->h_kp_pre) cudaFreeHost(h->h_kp_pre);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    if (h->ev_copied) cudaEventDestroy(h->ev_copied);
    if (h->own_surrogate) kaze_surrogate_destroy(h->own_surrogate);
    if (h->batch) kaze_batch_destroy(h->batch);
    if (h->side) cudaStreamDestroy(h->side);
    if (h->copy) cudaStreamDestroy(h->copy);
    delete h;
}
