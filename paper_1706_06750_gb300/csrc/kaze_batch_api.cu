// kaze_batch_api.cu -- host runtime of the batched detection: one handle for
// a fixed set of image sizes, its device arena, the ordered work list of the
// persistent kernel (k_batch.cu), the captured CUDA graph around it and the
// autotuner of its solve-tile shapes.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "kaze_batch.h"

#define KAZE_API extern "C" __attribute__((visibility("default")))

using kz::batch::ImageDesc;
using kz::batch::Item;

struct kaze_batch {
    kaze_options opt;
    int n = 0, N = 0;
    cudaStream_t stream = nullptr;
    std::vector<int> w, h, pitch;
    std::vector<long long> plane;

    void* arena = nullptr;           // device: planes, scratch, statistics, keypoints
    ImageDesc* d_desc = nullptr;     // device descriptors
    ImageDesc* h_desc = nullptr;     // pinned host copy (image pointers updated per call)
    unsigned* d_count_status = nullptr;  // per-image keypoint counts then status word (device)
    unsigned* h_count_status = nullptr;  // pinned host copy
    unsigned* d_next = nullptr;
    unsigned* d_done = nullptr;
    unsigned* d_need = nullptr;
    Item* d_items = nullptr;
    size_t items_cap = 0;
    void* stats_base = nullptr;      // per-image k / hmax / hist block, cleared per call
    size_t stats_bytes = 0;

    kz::batch::BatchParams params;
    kaze_batch_tuning tuning{KAZE_BATCH_RESIDENT, 4, 2, 8};

    // concurrent mode: single-image kernel sequences on parallel branches
    std::vector<kaze_handle*> branch_h;
    std::vector<cudaStream_t> branch_s;
    std::vector<cudaEvent_t> branch_ev;  // [0] fork, [1..] joins
    int* h_branch_status = nullptr;      // pinned, one word per branch
    int grid = 0, smem = 0;
    int n_items = 0;
    long long spin_limit = 1ll << 31;
    int stall_image = -1;            // test hook: a stage that never completes

    // resident mode: every image evolved by one cooperative launch with its
    // tiles resident (k_evolve.cu), then each image's response and extrema
    std::vector<double> t;           // t_i of Eq. 7
    int egrid = 0;                   // CTAs of the launch (one per SM)
    int2* d_work = nullptr;          // (image, tile) per CTA, wave after wave
    int* d_off = nullptr;            // CTA b's work: d_work[d_off[b] .. d_off[b + 1])
    size_t work_cap = 0;
    void* d_resident = nullptr;      // exchange buffers, barrier counters, candidate list
    std::vector<float*> exchange;    // per image
    unsigned* d_ebar = nullptr;      // per image barrier counter
    // the images' response and extrema launches run on kResBranches graph
    // branches, each with its own candidate list
    static constexpr int kResBranches = 4;
    unsigned long long* d_cand = nullptr;  // kResBranches lists of cand_cap entries
    unsigned* d_cand_count = nullptr;      // kResBranches counters
    unsigned cand_cap = 0;
    cudaStream_t res_s[kResBranches] = {};
    cudaEvent_t res_ev[kResBranches + 1] = {};  // [0] fork, [1..] joins
    size_t eparams_bytes = 0;
    void* d_eparams = nullptr;       // per image launch parameters
    void* h_eparams = nullptr;       // pinned copy, refreshed with the input pointers
    int waves = 0;

    cudaGraphExec_t gexec = nullptr;
    std::vector<kaze_keypoint> hkp;
    std::string err;
};

namespace {

kaze_status bfail(kaze_batch* b, kaze_status s, const std::string& m)
{
    if (b && b->err.empty()) b->err = m;
    return s;
}

#define KB_TRY(b, call)                                                                                  \
    do {                                                                                                 \
        cudaError_t e_ = (call);                                                                         \
        if (e_ != cudaSuccess)                                                                           \
            return bfail((b), KAZE_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorName(e_));          \
    } while (0)

int odd_chunk(int n, int P)
{
    int m = (n + P - 1) / P;
    m |= 1;
    return m < 3 ? 3 : m;
}

bool make_taps(double sigma, int rmax, kz::GaussTaps* t)
{
    int r = (int)std::ceil(3.0 * sigma);
    if (r < 1) r = 1;
    if (r > rmax) return false;
    double w[2 * kz::kMaxGaussR + 1], sum = 0.0;
    for (int j = -r; j <= r; ++j) {
        w[j + r] = std::exp(-(double)j * j / (2.0 * sigma * sigma));
        sum += w[j + r];
    }
    t->r = r;
    for (int j = 0; j <= 2 * r; ++j) t->w[j] = (float)(w[j] / sum);
    return true;
}

// Shared memory the persistent kernel needs for the batch's largest item.
int pool_floats(const kaze_batch* b, int cols)
{
    using namespace kz::batch;
    size_t need = 0;
    const int r0 = b->params.taps0.r, rd = b->params.tapsd.r;
    need = std::max(need, (size_t)(32 + 2 * r0) * (32 + 2 * r0) + (size_t)(32 + 2 * r0) * 32);
    need = std::max(need, (size_t)(34 + 2 * rd) * (34 + 2 * rd) + (size_t)(34 + 2 * rd) * 34 + 34 * 34 +
                              (size_t)b->opt.nbins);
    int smax = 1;
    for (int i = 0; i < b->N; ++i) smax = std::max(smax, b->params.tab.step[i]);
    need = std::max(need, (size_t)(64 + 4 * smax) * ((64 + 4 * smax) | 1));
    auto in = [](int m, const int* set, int n) { return std::find(set, set + n, m) != set + n; };
    for (int i = 0; i < b->n; ++i) {
        // compiled solvers keep a' in registers (2 arrays), the run-time one
        // in shared memory (3 arrays)
        const int mr = odd_chunk(b->w[i], 64);
        const int ra = in(mr, kRowCompiledM, 3) ? 2 : 3;
        const int ls = (64 * mr + 3) / 4 * 4;
        need = std::max(need, (size_t)4 * (ra * ls + 8 * 64));
        const int P = kBatchThreads / cols;
        const int mc = odd_chunk(b->h[i], P);
        const int ca = (cols == 4 && in(mc, kColCompiledM, 4)) ? 2 : 3;
        const int rs = P * mc;
        need = std::max(need, (size_t)ca * rs * cols + (size_t)8 * P * cols);
    }
    return (int)need;
}

// The ordered work list (stage-major across images) and the per-stage
// item counts.
void build_items(const kaze_batch* b, int cols, std::vector<Item>& items, std::vector<unsigned>& need)
{
    using namespace kz::batch;
    const int S = slots_per_image();
    need.assign((size_t)b->n * S, 0u);
    items.clear();
    auto add = [&](ItemKind kind, int level, int img, unsigned count, int slot) {
        for (unsigned t = 0; t < count; ++t) items.push_back(Item{(uint8_t)kind, (uint8_t)level, (uint16_t)img, t});
        need[(size_t)img * S + slot] += count;
    };
    auto t32 = [&](int i) {
        const int tx = (b->w[i] + 31) / 32;
        return (unsigned)(((tx + kTilesPerItem - 1) / kTilesPerItem) * ((b->h[i] + 31) / 32));
    };
    auto t64 = [&](int i) { return (unsigned)(((b->w[i] + 63) / 64) * ((b->h[i] + 63) / 64)); };
    for (int i = 0; i < b->n; ++i) add(IT_PRESMOOTH, 0, i, t32(i), slot_presmooth());
    for (int i = 0; i < b->n; ++i) add(IT_GMAX, 0, i, t32(i), slot_gmax());
    for (int i = 0; i < b->n; ++i) add(IT_GHIST, 0, i, t32(i), slot_ghist());
    for (int i = 0; i < b->n; ++i) add(IT_PCT, 0, i, 1, slot_pct());
    for (int i = 0; i < b->n; ++i) add(IT_DOH, 0, i, t64(i), slot_doh(0));
    for (int l = 1; l < b->N; ++l) {
        for (int i = 0; i < b->n; ++i) add(IT_COND, l, i, t32(i), slot_cond(l));
        for (int i = 0; i < b->n; ++i) add(IT_ROWS, l, i, (unsigned)((b->h[i] + 3) / 4), slot_rows(l));
        for (int i = 0; i < b->n; ++i) add(IT_COLS, l, i, (unsigned)((b->w[i] + cols - 1) / cols), slot_cols(l));
        for (int i = 0; i < b->n; ++i) add(IT_DOH, l, i, t64(i), slot_doh(l));
        if (l >= 2)
            for (int i = 0; i < b->n; ++i)
                add(IT_EXTREMA, l - 1, i, (unsigned)((b->h[i] + kExtremaRows - 1) / kExtremaRows),
                    slot_extrema(l - 1));
    }
}

void drop_graph(kaze_batch* b)
{
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
}

void drop_branches(kaze_batch* b)
{
    for (auto* h : b->branch_h) kaze_destroy(h);
    for (auto s : b->branch_s) cudaStreamDestroy(s);
    for (auto e : b->branch_ev) cudaEventDestroy(e);
    b->branch_h.clear();
    b->branch_s.clear();
    b->branch_ev.clear();
}

// Concurrent mode: one single-image handle and stream per branch.
kaze_status prepare_branches(kaze_batch* b)
{
    const int nb = std::max(1, std::min(b->tuning.streams, b->n));
    if ((int)b->branch_h.size() == nb) return KAZE_OK;
    drop_branches(b);
    const int mw = *std::max_element(b->w.begin(), b->w.end());
    const int mh = *std::max_element(b->h.begin(), b->h.end());
    kaze_options o = b->opt;
    o.max_keypoints = 1;  // keypoints go to the batch's own buffers
    o.aos_solver = KAZE_AOS_LINES;  // branches run side by side: no launch may claim every SM
    for (int i = 0; i < nb; ++i) {
        cudaStream_t st = nullptr;
        KB_TRY(b, cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        b->branch_s.push_back(st);
        kaze_handle* h = nullptr;
        const kaze_status s = kaze_create(&o, mw, mh, st, &h);
        if (s != KAZE_OK) return bfail(b, s, "branch handle creation failed");
        b->branch_h.push_back(h);
    }
    for (int i = 0; i < nb + 1; ++i) {
        cudaEvent_t e = nullptr;
        KB_TRY(b, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        b->branch_ev.push_back(e);
    }
    return KAZE_OK;
}

// The resident mode's launch parameters of every image from the current
// input pointers (pinned: the recorded graph copies them at each replay).
kaze_status refresh_resident(kaze_batch* b)
{
    const kz::batch::BatchParams& P = b->params;
    for (int i = 0; i < b->n; ++i) {
        const ImageDesc& d = b->h_desc[i];
        kz::EvolveImage im;
        im.levels = d.levels;
        im.plane = d.plane;
        im.pitch = d.pitch;
        im.w = d.w;
        im.h = d.h;
        im.img = d.img;
        im.img_pitch = d.img_pitch;
        im.taps0 = &P.taps0;
        im.d_k = d.k;
        if (b->opt.k_override > 0.f) {
            im.k_fixed = b->opt.k_override;
        } else {
            im.hmax_bits = d.hmax;
            im.hist = d.hist;
            im.nbins = b->opt.nbins;
            im.pct = b->opt.k_percentile;
        }
        im.exchange = b->exchange[i];
        im.barrier = b->d_ebar + i;
        if (!kz::evolve_batch_params((char*)b->h_eparams + b->eparams_bytes * i, im, b->N, b->t.data(), P.tapsd,
                                     b->opt.diffusivity, P.status, b->spin_limit, i == b->stall_image ? 0 : -1))
            return bfail(b, KAZE_ERR_INVALID_ARG, "image does not take the resident evolution");
    }
    return KAZE_OK;
}

// Resident mode: the images packed into waves of at most one tile per CTA
// (largest first, each into the first wave with room), the work lists of
// the CTAs, and the buffers of the launch.
kaze_status prepare_resident(kaze_batch* b)
{
    const kz::batch::BatchParams& P = b->params;
    if (!kz::evolve_front_fits(P.taps0.r, b->opt.nbins))
        return bfail(b, KAZE_ERR_INVALID_ARG, "presmoothing radius or bins outside the resident evolution");
    KB_TRY(b, kz::configure_evolve_kernel());  // evolve_fits asks the occupancy of the configured kernel
    const int grid = kz::evolve_batch_grid();
    if (grid < 1) return bfail(b, KAZE_ERR_CUDA, "resident evolution does not fit an SM");
    std::vector<int> tiles(b->n);
    for (int i = 0; i < b->n; ++i)
        if (!kz::evolve_fits(b->w[i], b->h[i], P.tapsd.r, &tiles[i]) || tiles[i] > grid)
            return bfail(b, KAZE_ERR_INVALID_ARG, "an image does not take the resident evolution");
    std::vector<int> order(b->n);
    for (int i = 0; i < b->n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return tiles[x] > tiles[y]; });
    std::vector<std::vector<int>> wave_imgs;
    std::vector<int> wave_load;
    for (int i : order) {
        size_t wv = 0;
        while (wv < wave_load.size() && wave_load[wv] + tiles[i] > grid) ++wv;
        if (wv == wave_load.size()) {
            wave_load.push_back(0);
            wave_imgs.emplace_back();
        }
        wave_load[wv] += tiles[i];
        wave_imgs[wv].push_back(i);
    }
    std::vector<std::vector<int2>> lists(grid);
    for (const auto& wi : wave_imgs) {
        int cta = 0;
        for (int i : wi)
            for (int t = 0; t < tiles[i]; ++t) lists[cta++].push_back(make_int2(i, t));
    }
    std::vector<int2> work;
    std::vector<int> off(grid + 1, 0);
    for (int c = 0; c < grid; ++c) {
        off[c] = (int)work.size();
        work.insert(work.end(), lists[c].begin(), lists[c].end());
    }
    off[grid] = (int)work.size();
    if (work.size() > b->work_cap || !b->d_off) {
        if (b->d_work) cudaFree(b->d_work);
        if (b->d_off) cudaFree(b->d_off);
        b->d_work = nullptr;
        b->d_off = nullptr;
        KB_TRY(b, cudaMalloc(&b->d_work, sizeof(int2) * work.size()));
        KB_TRY(b, cudaMalloc(&b->d_off, sizeof(int) * (grid + 1)));
        b->work_cap = work.size();
    }
    KB_TRY(b, cudaMemcpy(b->d_work, work.data(), sizeof(int2) * work.size(), cudaMemcpyHostToDevice));
    KB_TRY(b, cudaMemcpy(b->d_off, off.data(), sizeof(int) * (grid + 1), cudaMemcpyHostToDevice));
    b->egrid = grid;
    b->waves = (int)wave_imgs.size();
    if (!b->d_resident || !b->h_eparams) {
        auto al = [](size_t x) { return (x + 255) / 256 * 256; };
        size_t bytes = 0, max_plane = 0;
        std::vector<size_t> xoff(b->n);
        for (int i = 0; i < b->n; ++i) {
            xoff[i] = bytes;
            bytes += al(sizeof(float) * kz::evolve_exchange_floats(tiles[i]));
            max_plane = std::max(max_plane, (size_t)b->plane[i]);
        }
        const size_t off_bar = bytes;
        bytes += al(sizeof(unsigned) * b->n);
        const unsigned cand_cap =
            (unsigned)std::min<size_t>(std::max<size_t>((size_t)b->N * max_plane / 16, 65536), 1u << 30);
        const size_t off_cand = bytes;
        bytes += al(sizeof(unsigned long long) * cand_cap) * kaze_batch::kResBranches;
        const size_t off_ccnt = bytes;
        bytes += al(sizeof(unsigned) * kaze_batch::kResBranches);
        const size_t pbytes = (kz::evolve_params_bytes() + 15) / 16 * 16;
        const size_t off_par = bytes;
        bytes += al(pbytes * b->n);
        // allocated together, kept only when both succeed
        void* dres = nullptr;
        void* hpar = nullptr;
        cudaError_t e = cudaMalloc(&dres, bytes);
        if (e == cudaSuccess) e = cudaMallocHost(&hpar, pbytes * b->n);
        if (e != cudaSuccess) {
            if (dres) cudaFree(dres);
            return bfail(b, e == cudaErrorMemoryAllocation ? KAZE_ERR_OOM : KAZE_ERR_CUDA,
                         std::string("resident batch buffers: ") + cudaGetErrorName(e));
        }
        if (b->d_resident) cudaFree(b->d_resident);
        if (b->h_eparams) cudaFreeHost(b->h_eparams);
        b->d_resident = dres;
        b->h_eparams = hpar;
        b->eparams_bytes = pbytes;
        b->cand_cap = cand_cap;
        char* a = (char*)b->d_resident;
        b->exchange.resize(b->n);
        for (int i = 0; i < b->n; ++i) b->exchange[i] = (float*)(a + xoff[i]);
        b->d_ebar = (unsigned*)(a + off_bar);
        b->d_cand = (unsigned long long*)(a + off_cand);
        b->d_cand_count = (unsigned*)(a + off_ccnt);
        b->d_eparams = a + off_par;
    }
    for (int k = 0; k < kaze_batch::kResBranches; ++k)
        if (!b->res_s[k]) KB_TRY(b, cudaStreamCreateWithFlags(&b->res_s[k], cudaStreamNonBlocking));
    for (int k = 0; k <= kaze_batch::kResBranches; ++k)
        if (!b->res_ev[k]) KB_TRY(b, cudaEventCreateWithFlags(&b->res_ev[k], cudaEventDisableTiming));
    return refresh_resident(b);
}

kaze_status enqueue_resident(kaze_batch* b)
{
    const kz::batch::BatchParams& P = b->params;
    cudaStream_t st = b->stream;
    KB_TRY(b, cudaMemsetAsync(b->d_count_status, 0, sizeof(unsigned) * (b->n + 1), st));
    KB_TRY(b, cudaMemsetAsync(b->stats_base, 0, b->stats_bytes, st));
    KB_TRY(b, cudaMemsetAsync(b->d_ebar, 0, sizeof(unsigned) * b->n, st));
    KB_TRY(b, cudaMemcpyAsync(b->d_eparams, b->h_eparams, b->eparams_bytes * b->n, cudaMemcpyHostToDevice, st));
    KB_TRY(b, kz::launch_evolve_batch(b->d_eparams, b->d_work, b->d_off, b->egrid, st));
    // each image's response and extrema on branch i % kResBranches, so that
    // the small images' launches run side by side
    constexpr int NB = kaze_batch::kResBranches;
    KB_TRY(b, cudaEventRecord(b->res_ev[0], st));
    for (int k = 0; k < NB; ++k) KB_TRY(b, cudaStreamWaitEvent(b->res_s[k], b->res_ev[0], 0));
    const size_t list_stride = (sizeof(unsigned long long) * b->cand_cap + 255) / 256 * 256 / sizeof(unsigned long long);
    for (int i = 0; i < b->n; ++i) {
        const ImageDesc& d = b->h_desc[i];
        const int k = i % NB;
        cudaStream_t sk = b->res_s[k];
        kz::Candidates c;
        c.list = b->d_cand + list_stride * k;
        c.count = b->d_cand_count + k;
        c.cap = b->cand_cap;
        c.thr = b->opt.dthreshold;
        c.lo = 1;
        c.hi = b->N - 2;
        KB_TRY(b, cudaMemsetAsync(c.count, 0, sizeof(unsigned), sk));
        KB_TRY(b, kz::launch_doh(d.levels, d.doh, d.pitch, d.plane, d.w, d.h, 0, b->N, P.tab, sk, &c));
        KB_TRY(b, kz::launch_extrema(d.doh, d.pitch, d.plane, d.w, d.h, b->N, P.tab, b->opt.dthreshold,
                                     b->opt.edge_r, d.kp, d.kp_cap, d.kp_count, sk, &c));
    }
    for (int k = 0; k < NB; ++k) {
        KB_TRY(b, cudaEventRecord(b->res_ev[1 + k], b->res_s[k]));
        KB_TRY(b, cudaStreamWaitEvent(st, b->res_ev[1 + k], 0));
    }
    KB_TRY(b, cudaMemcpyAsync(b->h_count_status, b->d_count_status, sizeof(unsigned) * (b->n + 1),
                              cudaMemcpyDeviceToHost, st));
    return KAZE_OK;
}

// Prepares the work list, shared memory and grid for the current tuning.
kaze_status prepare(kaze_batch* b)
{
    using namespace kz::batch;
    if (b->tuning.mode == KAZE_BATCH_CONCURRENT) {
        drop_graph(b);
        return prepare_branches(b);
    }
    if (b->tuning.mode == KAZE_BATCH_RESIDENT) {
        drop_graph(b);
        return prepare_resident(b);
    }
    const int cols = b->tuning.cols_per_strip;
    std::vector<Item> items;
    std::vector<unsigned> need;
    build_items(b, cols, items, need);
    if (b->stall_image >= 0 && b->stall_image < b->n)  // test hook: unreachable count
        need[(size_t)b->stall_image * slots_per_image() + slot_rows(1)] += 1;
    if (items.size() > b->items_cap) {
        if (b->d_items) cudaFree(b->d_items);
        b->d_items = nullptr;
        KB_TRY(b, cudaMalloc(&b->d_items, sizeof(Item) * items.size()));
        b->items_cap = items.size();
    }
    KB_TRY(b, cudaMemcpy(b->d_items, items.data(), sizeof(Item) * items.size(), cudaMemcpyHostToDevice));
    KB_TRY(b, cudaMemcpy(b->d_need, need.data(), sizeof(unsigned) * need.size(), cudaMemcpyHostToDevice));
    b->n_items = (int)items.size();
    b->smem = pool_floats(b, cols) * (int)sizeof(float);
    int optin = 0, dev = 0;
    KB_TRY(b, cudaGetDevice(&dev));
    KB_TRY(b, cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    if (b->smem + 64 > optin) return bfail(b, KAZE_ERR_INVALID_ARG, "images too large for the batched kernel");
    KB_TRY(b, configure_batch_kernel(b->smem));
    int per_sm = 0, sms = 0;
    KB_TRY(b, batch_occupancy(b->smem, &per_sm));
    KB_TRY(b, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (per_sm < 1) return bfail(b, KAZE_ERR_INVALID_ARG, "batched kernel does not fit on an SM");
    b->grid = sms * std::min(per_sm, std::max(1, b->tuning.ctas_per_sm));
    b->params.items = b->d_items;
    b->params.n_items = b->n_items;
    b->params.cols = cols;
    b->params.spin_limit = b->spin_limit;
    drop_graph(b);
    return KAZE_OK;
}

kaze_status enqueue_concurrent(kaze_batch* b)
{
    cudaStream_t st = b->stream;
    const int nb = (int)b->branch_h.size();
    KB_TRY(b, cudaMemsetAsync(b->d_count_status, 0, sizeof(unsigned) * (b->n + 1), st));
    KB_TRY(b, cudaEventRecord(b->branch_ev[0], st));
    for (int k = 0; k < nb; ++k) {
        KB_TRY(b, cudaStreamWaitEvent(b->branch_s[k], b->branch_ev[0], 0));
        KB_TRY(b, kaze_set_stream(b->branch_h[k], b->branch_s[k]) == KAZE_OK ? cudaSuccess : cudaErrorUnknown);
    }
    for (int i = 0; i < b->n; ++i) {
        const ImageDesc& d = b->h_desc[i];
        const kaze_status s = kz::handle_enqueue_into(b->branch_h[i % nb], d.img, d.w, d.h, d.img_pitch, d.levels,
                                                      d.doh, d.kp, d.kp_count, d.kp_cap);
        if (s != KAZE_OK)
            return bfail(b, s, std::string("branch enqueue: ") + kaze_last_error(b->branch_h[i % nb]));
    }
    for (int k = 0; k < nb; ++k) {
        KB_TRY(b, cudaMemcpyAsync(b->h_branch_status + k, kz::handle_status_ptr(b->branch_h[k]), sizeof(int),
                                  cudaMemcpyDeviceToHost, b->branch_s[k]));
        KB_TRY(b, cudaEventRecord(b->branch_ev[1 + k], b->branch_s[k]));
        KB_TRY(b, cudaStreamWaitEvent(st, b->branch_ev[1 + k], 0));
    }
    KB_TRY(b, cudaMemcpyAsync(b->h_count_status, b->d_count_status, sizeof(unsigned) * (b->n + 1),
                              cudaMemcpyDeviceToHost, st));
    return KAZE_OK;
}

kaze_status enqueue(kaze_batch* b)
{
    using namespace kz::batch;
    if (b->tuning.mode == KAZE_BATCH_CONCURRENT) return enqueue_concurrent(b);
    if (b->tuning.mode == KAZE_BATCH_RESIDENT) return enqueue_resident(b);
    cudaStream_t st = b->stream;
    KB_TRY(b, cudaMemsetAsync(b->d_next, 0, sizeof(unsigned), st));
    KB_TRY(b, cudaMemsetAsync(b->d_done, 0, sizeof(unsigned) * (size_t)b->n * slots_per_image(), st));
    KB_TRY(b, cudaMemsetAsync(b->d_count_status, 0, sizeof(unsigned) * (b->n + 1), st));
    KB_TRY(b, cudaMemsetAsync(b->stats_base, 0, b->stats_bytes, st));
    KB_TRY(b, cudaMemcpyAsync(b->d_desc, b->h_desc, sizeof(ImageDesc) * b->n, cudaMemcpyHostToDevice, st));
    KB_TRY(b, launch_batch(b->params, b->grid, b->smem, st));
    KB_TRY(b, cudaMemcpyAsync(b->h_count_status, b->d_count_status, sizeof(unsigned) * (b->n + 1),
                              cudaMemcpyDeviceToHost, st));
    return KAZE_OK;
}

kaze_status run(kaze_batch* b)
{
    const bool capturable = b->stream && b->stream != cudaStreamLegacy && b->stream != cudaStreamPerThread;
    if (!capturable) return enqueue(b);
    if (!b->gexec) {
        cudaGraph_t graph = nullptr;
        KB_TRY(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        const kaze_status s = enqueue(b);
        const cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
        if (s != KAZE_OK) {
            if (graph) cudaGraphDestroy(graph);
            return s;
        }
        if (e != cudaSuccess) return bfail(b, KAZE_ERR_CUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorName(e));
        const cudaError_t ei = cudaGraphInstantiate(&b->gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) {
            b->gexec = nullptr;
            return bfail(b, KAZE_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorName(ei));
        }
    }
    KB_TRY(b, cudaGraphLaunch(b->gexec, b->stream));
    return KAZE_OK;
}

kaze_status set_inputs(kaze_batch* b, const float* const* d_imgs, const int* pitches)
{
    if (!d_imgs) return bfail(b, KAZE_ERR_INVALID_ARG, "null image list");
    for (int i = 0; i < b->n; ++i) {
        const int p = pitches ? pitches[i] : b->w[i];
        if (!d_imgs[i] || p < b->w[i]) return bfail(b, KAZE_ERR_INVALID_ARG, "bad image pointer or pitch");
        b->h_desc[i].img = d_imgs[i];
        b->h_desc[i].img_pitch = p;
    }
    return KAZE_OK;
}

}  // namespace

KAZE_API kaze_status kaze_batch_create(const kaze_options* opt, int n, const int* w, const int* h, void* cuda_stream,
                                       kaze_batch** out)
{
    using namespace kz::batch;
    if (!out || !w || !h || n < 1 || n > 65535) return KAZE_ERR_INVALID_ARG;
    *out = nullptr;
    kaze_options o;
    if (opt) o = *opt; else kaze_default_options(&o);
    const int N = o.octaves * o.sublevels;
    if (o.octaves < 1 || o.sublevels < 1 || N > kz::kMaxLevels || N > 255) return KAZE_ERR_INVALID_ARG;
    if (!(o.sigma0 > 0.f) || !(o.sigma_d > 0.f) || !(o.k_percentile > 0.0 && o.k_percentile <= 1.0))
        return KAZE_ERR_INVALID_ARG;
    if (o.nbins < 1 || o.nbins > kz::kMaxBins || o.max_keypoints < 1) return KAZE_ERR_INVALID_ARG;
    if (o.diffusivity != KAZE_G1 && o.diffusivity != KAZE_G2) return KAZE_ERR_INVALID_ARG;
    if (o.doh_norm != KAZE_DOH_SIGMA4 && o.doh_norm != KAZE_DOH_PAPER_LITERAL) return KAZE_ERR_INVALID_ARG;
    // the persistent batch kernel evolves by AOS and tests 3x3x3 maxima
    if (o.scheme != KAZE_SCHEME_AOS || o.extrema_window != KAZE_EXTREMA_3X3) return KAZE_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i)
        if (w[i] < 3 || h[i] < 3 || w[i] > 4096 || h[i] > 4096) return KAZE_ERR_INVALID_ARG;

    kaze_batch* b = new (std::nothrow) kaze_batch();
    if (!b) return KAZE_ERR_OOM;
    b->opt = o;
    b->n = n;
    b->N = N;
    b->stream = (cudaStream_t)cuda_stream;
    b->w.assign(w, w + n);
    b->h.assign(h, h + n);
    BatchParams& P = b->params;
    std::memset(&P, 0, sizeof(P));
    if (!make_taps(o.sigma0, kz::kMaxGaussR, &P.taps0) || !make_taps(o.sigma_d, kz::kMaxGradR, &P.tapsd)) {
        delete b;
        return KAZE_ERR_INVALID_ARG;
    }
    // Eq. 6-8: scales, evolution steps, derivative steps and normalisation
    double sig[kz::kMaxLevels], t[kz::kMaxLevels];
    P.tab.n = N;
    P.tab.sublevels = o.sublevels;
    for (int oc = 0; oc < o.octaves; ++oc)
        for (int s = 0; s < o.sublevels; ++s) {
            const int i = oc * o.sublevels + s;
            sig[i] = (double)o.sigma0 * std::pow(2.0, (double)oc + (double)s / o.sublevels);
            t[i] = 0.5 * sig[i] * sig[i];
            int st = (int)std::floor(sig[i] + 0.5);
            st = st < 1 ? 1 : st;
            P.tab.step[i] = st;
            P.tab.sigma[i] = (float)sig[i];
            P.tab.xr[i] = 1;  // the 3x3x3 test
            double norm;
            if (o.doh_norm == KAZE_DOH_PAPER_LITERAL) {
                const double kn = sig[i] / std::pow(2.0, (double)oc);
                norm = kn * kn;
            } else {
                norm = (double)st * st * st * st;
            }
            P.tab.norm[i] = (float)norm;
            const double d = 1024.0 * st * st;
            P.doh_scale[i] = (float)((double)P.tab.norm[i] / (d * d));  // as the single-image kernel does
            P.tau[i] = i > 0 ? (float)(t[i] - t[i - 1]) : 0.f;
        }
    P.pct = o.k_percentile;
    P.nbins = o.nbins;
    P.diffusivity = o.diffusivity;
    P.thr = o.dthreshold;
    P.edge_r = o.edge_r;
    P.k_override = o.k_override;
    P.N = N;
    P.slots = slots_per_image();
    b->t.assign(t, t + N);

    // arena: per image N levels, N responses, g, ux; then statistics, keypoints
    auto al = [](size_t x) { return (x + 255) / 256 * 256; };
    size_t planes = 0;
    b->pitch.resize(n);
    b->plane.resize(n);
    for (int i = 0; i < n; ++i) {
        b->pitch[i] = (w[i] + 31) / 32 * 32;
        b->plane[i] = (long long)b->pitch[i] * h[i];
        planes += al(sizeof(float) * (size_t)b->plane[i] * (2 * N + 2));
    }
    const size_t stat_per = al(sizeof(float)) + al(sizeof(unsigned)) + al(sizeof(unsigned) * o.nbins);
    b->stats_bytes = stat_per * n;
    const size_t kp_bytes = al(sizeof(kaze_keypoint) * (size_t)o.max_keypoints) * n;
    const size_t ctl = al(sizeof(ImageDesc) * n) + al(sizeof(unsigned) * (n + 1)) + al(sizeof(unsigned)) +
                       2 * al(sizeof(unsigned) * (size_t)n * slots_per_image());
    cudaError_t e = cudaMalloc(&b->arena, planes + b->stats_bytes + kp_bytes + ctl);
    if (e != cudaSuccess) {
        delete b;
        return e == cudaErrorMemoryAllocation ? KAZE_ERR_OOM : KAZE_ERR_CUDA;
    }
    char* a = (char*)b->arena;
    if (cudaMallocHost(&b->h_desc, sizeof(ImageDesc) * n) != cudaSuccess ||
        cudaMallocHost(&b->h_count_status, sizeof(unsigned) * (n + 1)) != cudaSuccess ||
        cudaMallocHost(&b->h_branch_status, sizeof(int) * 64) != cudaSuccess) {
        kaze_batch_destroy(b);
        return KAZE_ERR_CUDA;
    }
    char* stats = a + planes;
    b->stats_base = stats;
    char* kps = stats + b->stats_bytes;
    char* c = kps + kp_bytes;
    b->d_desc = (ImageDesc*)c;
    c += al(sizeof(ImageDesc) * n);
    b->d_count_status = (unsigned*)c;
    c += al(sizeof(unsigned) * (n + 1));
    b->d_next = (unsigned*)c;
    c += al(sizeof(unsigned));
    b->d_done = (unsigned*)c;
    c += al(sizeof(unsigned) * (size_t)n * slots_per_image());
    b->d_need = (unsigned*)c;

    for (int i = 0; i < n; ++i) {
        ImageDesc& d = b->h_desc[i];
        std::memset(&d, 0, sizeof(d));
        d.w = w[i];
        d.h = h[i];
        d.pitch = b->pitch[i];
        d.plane = b->plane[i];
        d.levels = (float*)a;
        d.doh = d.levels + (size_t)N * d.plane;
        d.g = d.doh + (size_t)N * d.plane;
        d.ux = d.g + d.plane;
        a += al(sizeof(float) * (size_t)d.plane * (2 * N + 2));
        d.k = (float*)(stats + stat_per * i);
        d.hmax = (unsigned*)(stats + stat_per * i + al(sizeof(float)));
        d.hist = (unsigned*)(stats + stat_per * i + al(sizeof(float)) + al(sizeof(unsigned)));
        d.kp = (kaze_keypoint*)(kps + al(sizeof(kaze_keypoint) * (size_t)o.max_keypoints) * i);
        d.kp_count = b->d_count_status + i;
        d.kp_cap = o.max_keypoints;
        d.mrow = odd_chunk(w[i], 64);
        d.mcol = odd_chunk(h[i], 64);
        d.mcol32 = odd_chunk(h[i], 32);
        d.tiles32_x = (w[i] + 31) / 32;
        d.groups32_x = (d.tiles32_x + kz::batch::kTilesPerItem - 1) / kz::batch::kTilesPerItem;
        d.tiles64_x = (w[i] + 63) / 64;
    }
    P.imgs = b->d_desc;
    P.next = b->d_next;
    P.done = b->d_done;
    P.need = b->d_need;
    P.status = (int*)(b->d_count_status + n);
    // the resident evolution where every image takes it, else the work queue
    kaze_status s = prepare(b);
    if (s != KAZE_OK && b->tuning.mode == KAZE_BATCH_RESIDENT) {
        b->err.clear();
        b->tuning.mode = KAZE_BATCH_PERSISTENT;
        s = prepare(b);
    }
    if (s != KAZE_OK) {
        kaze_batch_destroy(b);
        return s;
    }
    *out = b;
    return KAZE_OK;
}

KAZE_API kaze_status kaze_batch_detect(kaze_batch* b, const float* const* d_imgs, const int* pitches,
                                       kaze_keypoint* h_out, int capacity_per_image, int* counts)
{
    if (!b || capacity_per_image < 0 || (capacity_per_image > 0 && !h_out) || !counts)
        return bfail(b, KAZE_ERR_INVALID_ARG, "bad output arguments");
    kaze_status s = set_inputs(b, d_imgs, pitches);
    if (s != KAZE_OK) return s;
    if (b->tuning.mode == KAZE_BATCH_RESIDENT && (s = refresh_resident(b)) != KAZE_OK) return s;
    s = run(b);
    if (s != KAZE_OK) return s;
    KB_TRY(b, cudaStreamSynchronize(b->stream));
    bool timed_out = b->h_count_status[b->n] != 0;
    if (b->tuning.mode == KAZE_BATCH_CONCURRENT)
        for (size_t k = 0; k < b->branch_h.size(); ++k) timed_out |= b->h_branch_status[k] != 0;
    if (timed_out) return bfail(b, KAZE_ERR_TIMEOUT, "a bounded device-side wait ran out");
    kaze_status result = KAZE_OK;
    const unsigned cap = (unsigned)capacity_per_image;
    for (int i = 0; i < b->n; ++i) {
        const unsigned total = b->h_count_status[i];
        const unsigned have = std::min(total, (unsigned)b->opt.max_keypoints);
        b->hkp.resize(have);
        if (have) {
            KB_TRY(b, cudaMemcpyAsync(b->hkp.data(), b->h_desc[i].kp, sizeof(kaze_keypoint) * have,
                                      cudaMemcpyDeviceToHost, b->stream));
            KB_TRY(b, cudaStreamSynchronize(b->stream));
        }
        std::sort(b->hkp.begin(), b->hkp.end(), [](const kaze_keypoint& x, const kaze_keypoint& y) {
            if (x.level != y.level) return x.level < y.level;
            if (x.iy != y.iy) return x.iy < y.iy;
            return x.ix < y.ix;
        });
        const unsigned nout = std::min(have, cap);
        if (nout) std::memcpy(h_out + (size_t)i * cap, b->hkp.data(), sizeof(kaze_keypoint) * nout);
        counts[i] = (int)total;
        if (total > cap || total > (unsigned)b->opt.max_keypoints) result = KAZE_ERR_CAPACITY;
    }
    if (result != KAZE_OK) return bfail(b, result, "more keypoints than the output capacity");
    return KAZE_OK;
}

KAZE_API kaze_status kaze_batch_get_level(kaze_batch* b, int image, int level, const float** d_level, int* pitch)
{
    if (!b || image < 0 || image >= b->n || level < 0 || level >= b->N) return KAZE_ERR_INVALID_ARG;
    if (d_level) *d_level = b->h_desc[image].levels + (size_t)level * b->plane[image];
    if (pitch) *pitch = b->pitch[image];
    return KAZE_OK;
}

KAZE_API kaze_status kaze_batch_get_response(kaze_batch* b, int image, int level, const float** d_doh, int* pitch)
{
    if (!b || image < 0 || image >= b->n || level < 0 || level >= b->N) return KAZE_ERR_INVALID_ARG;
    if (d_doh) *d_doh = b->h_desc[image].doh + (size_t)level * b->plane[image];
    if (pitch) *pitch = b->pitch[image];
    return KAZE_OK;
}

KAZE_API kaze_status kaze_batch_set_tuning(kaze_batch* b, const kaze_batch_tuning* t)
{
    if (!b || !t) return KAZE_ERR_INVALID_ARG;
    if ((t->mode != KAZE_BATCH_PERSISTENT && t->mode != KAZE_BATCH_CONCURRENT && t->mode != KAZE_BATCH_RESIDENT) ||
        (t->cols_per_strip != 4 && t->cols_per_strip != 8) || t->ctas_per_sm < 1 || t->ctas_per_sm > 8 ||
        t->streams < 1 || t->streams > 64)
        return bfail(b, KAZE_ERR_INVALID_ARG, "tuning out of range");
    const kaze_batch_tuning old = b->tuning;
    b->tuning = *t;
    const kaze_status s = prepare(b);
    if (s != KAZE_OK) {
        b->tuning = old;
        prepare(b);
    }
    return s;
}

KAZE_API kaze_status kaze_batch_get_tuning(const kaze_batch* b, kaze_batch_tuning* t)
{
    if (!b || !t) return KAZE_ERR_INVALID_ARG;
    *t = b->tuning;
    return KAZE_OK;
}

KAZE_API kaze_status kaze_batch_autotune(kaze_batch* b, const float* const* d_imgs, const int* pitches, int reps,
                                         kaze_batch_tuning* best, double* best_ms)
{
    if (!b || reps < 1) return KAZE_ERR_INVALID_ARG;
    kaze_status s = set_inputs(b, d_imgs, pitches);
    if (s != KAZE_OK) return s;
    const kaze_batch_tuning start = b->tuning;
    kaze_batch_tuning winner = start;
    double winner_ms = 1e30;
    cudaEvent_t e0, e1;
    KB_TRY(b, cudaEventCreate(&e0));
    KB_TRY(b, cudaEventCreate(&e1));
    std::vector<kaze_batch_tuning> cands;
    cands.push_back(kaze_batch_tuning{KAZE_BATCH_RESIDENT, 4, 1, 8});
    for (int cols : {4, 8})
        for (int ctas : {1, 2}) cands.push_back(kaze_batch_tuning{KAZE_BATCH_PERSISTENT, cols, ctas, 8});
    for (int streams : {4, 8, 16}) cands.push_back(kaze_batch_tuning{KAZE_BATCH_CONCURRENT, 4, 2, streams});
    for (const kaze_batch_tuning& cand : cands) {
        {
            b->tuning = cand;
            if (prepare(b) != KAZE_OK) {
                b->err.clear();
                continue;
            }
            if (run(b) != KAZE_OK || cudaStreamSynchronize(b->stream) != cudaSuccess || b->h_count_status[b->n]) {
                b->err.clear();
                continue;
            }
            float total = 0.f;
            bool ok = true;
            for (int r = 0; r < reps && ok; ++r) {
                ok = cudaEventRecord(e0, b->stream) == cudaSuccess && run(b) == KAZE_OK &&
                     cudaEventRecord(e1, b->stream) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess;
                float ms = 0.f;
                ok = ok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && !b->h_count_status[b->n];
                total += ms;
            }
            if (ok && total / reps < winner_ms) {
                winner_ms = total / reps;
                winner = cand;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->tuning = winner;
    s = prepare(b);
    if (s != KAZE_OK) return s;
    if (winner_ms >= 1e30) return bfail(b, KAZE_ERR_CUDA, "no tuning candidate ran");
    if (best) *best = winner;
    if (best_ms) *best_ms = winner_ms;
    return KAZE_OK;
}

KAZE_API kaze_status kaze_batch_set_wait_limit(kaze_batch* b, long long cycles, int stall_image)
{
    if (!b || cycles < 1000) return KAZE_ERR_INVALID_ARG;
    b->spin_limit = cycles;
    b->stall_image = stall_image;
    return prepare(b);
}

KAZE_API const char* kaze_batch_last_error(const kaze_batch* b) { return b ? b->err.c_str() : "null batch"; }

KAZE_API void kaze_batch_destroy(kaze_batch* b)
{
    if (!b) return;
    drop_graph(b);
    drop_branches(b);
    if (b->h_branch_status) cudaFreeHost(b->h_branch_status);
    if (b->d_items) cudaFree(b->d_items);
    if (b->d_work) cudaFree(b->d_work);
    if (b->d_off) cudaFree(b->d_off);
    if (b->d_resident) cudaFree(b->d_resident);
    for (auto sres : b->res_s)
        if (sres) cudaStreamDestroy(sres);
    for (auto e : b->res_ev)
        if (e) cudaEventDestroy(e);
    if (b->h_eparams) cudaFreeHost(b->h_eparams);
    if (b->arena) cudaFree(b->arena);
    if (b->h_desc) cudaFreeHost(b->h_desc);
    if (b->h_count_status) cudaFreeHost(b->h_count_status);
    delete b;
}
