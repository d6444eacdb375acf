/*
 * kaze.h -- C ABI of the GB300 (sm_103a) KAZE scale-space and detector
 * library, libkaze.so.
 *
 * Method: "GPGPU Acceleration of the KAZE Image Feature Extraction Algorithm"
 * (arXiv 1706.06750).  The library computes, for one FP32 grayscale image:
 *   - the nonlinear scale space of Sec. II-A: Gaussian presmoothing, the
 *     contrast factor k from the gradient histogram (Sec. III-1), the
 *     Perona-Malik conductance of Eq. 2-3 and the semi-implicit step of
 *     Eq. 4 solved by additive operator splitting (one tridiagonal solve per
 *     row and per column), with evolution times from Eq. 6-7;
 *   - the normalised Hessian-determinant detector response of Eq. 8;
 *   - 3x3x3 maxima with sub-pixel refinement and the edge test of
 *     Eq. 9-12 (Sec. II-B, Sec. III-2).
 *
 * Conventions shared by every entry point:
 *   - Images are FP32, row-major, element (x, y) at ptr[y * pitch + x];
 *     pitch is given in elements (pitch_elems >= w).
 *   - "d_" pointers are DEVICE pointers (e.g. torch.empty(..., device='cuda')
 *     .data_ptr()); "h_" pointers are HOST pointers.  The caller owns every
 *     pointer it passes; the library never frees them.
 *   - The handle owns its scratch, its level and response buffers.  Pointers
 *     it hands out (kaze_get_level, kaze_get_response) are borrowed and stay
 *     valid until the next kaze_build_scale_space / kaze_detect* call on the
 *     handle or until kaze_destroy.
 *   - All work is enqueued on the handle's CUDA stream (cudaStream_t passed
 *     as void*; NULL = legacy default stream).  Only calls that return host
 *     data synchronise that stream: kaze_get_contrast, kaze_find_extrema,
 *     kaze_detect, kaze_detect_host and kaze_op_contrast / kaze_op_extrema.
 *   - Every call returns a kaze_status.  The first CUDA error seen by a
 *     handle is kept and reported by kaze_last_error; after a KAZE_ERR_CUDA
 *     the handle should be destroyed.
 *   - Images smaller than 3x3 or larger than the handle's max_w x max_h give
 *     KAZE_ERR_INVALID_ARG.
 */
#ifndef KAZE_H
#define KAZE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    KAZE_OK = 0,
    KAZE_ERR_INVALID_ARG = 1,  /* a size, pointer, pitch or option is invalid   */
    KAZE_ERR_CUDA = 2,         /* a CUDA call or kernel launch failed             */
    KAZE_ERR_OOM = 3,          /* device allocation failed in kaze_create         */
    KAZE_ERR_CAPACITY = 4,     /* more keypoints than the output holds            */
    KAZE_ERR_TIMEOUT = 5,      /* a bounded device-side wait ran out              */
    KAZE_ERR_STATE = 6         /* call out of order (e.g. response before build)  */
} kaze_status;

/* Conductance functions of Eq. 3. */
#define KAZE_G1 1  /* g1 = exp(-|grad L_sigma|^2 / k^2)         */
#define KAZE_G2 2  /* g2 = 1 / (1 + |grad L_sigma|^2 / k^2)     */

/* Evolution scheme of each level (Sec. II-A). */
#define KAZE_SCHEME_AOS 0  /* one AOS step of Eq. 4 per level (default)                    */
#define KAZE_SCHEME_FED 1  /* one FED cycle of explicit steps per level (Eq. 5): the n with
                              cycle time fed_tau_max (n^2 + n) / 3 >= t_i - t_{i-1}, steps
                              tau_j of Eq. 5 scaled to sum to t_i - t_{i-1}, conductance of
                              the previous level held fixed over the cycle                 */

/* Cross-level neighbourhood of the maximum test (Sec. II-B, Sec. IV).  A
 * candidate is above the threshold and above its 8 neighbours on its level;
 * it must also lie above every response of levels i-1 and i+1 within |dx|,
 * |dy| <= r_i (pixels outside the image skipped):                         */
#define KAZE_EXTREMA_3X3 0           /* r_i = 1, the 3x3x3 test (default)    */
#define KAZE_EXTREMA_SIGMA_WINDOW 1  /* the sigma_i x sigma_i window:
                                        r_i = max(1, floor(s_i / 2)),
                                        s_i = max(1, round(sigma_i)); single-
                                        image handles only                  */

/* How the AOS steps of Eq. 4 are solved (the same method; the solutions
 * agree to FP32 rounding). */
#define KAZE_AOS_AUTO 0   /* the resident evolution when the image's 128 x 120
                             tiles fit one per SM (at most 16 along a line) and
                             sigma_d <= 1: all N-1 steps in one cooperative
                             launch, each tile of L and g held in shared memory,
                             lines solved in chunks coupled through their end
                             values; the line kernels otherwise (default)      */
#define KAZE_AOS_LINES 1  /* always the line kernels: per step a conductance
                             pass, then every row and every column solved by
                             one CTA strip each (no cooperative launch)         */
#define KAZE_AOS_STREAMED 2 /* the streamed tile passes where they fit (at most
                             64 tiles along a line; the line kernels beyond):
                             per step three launches over all tiles
                             (conductance and chunk records of every tile;
                             every segment's outside neighbours from its line;
                             the re-solves, L_i written once), the resident
                             evolution's tile arithmetic without its residency
                             (slower than the line kernels on large images)   */

/* Normalisation of the Hessian determinant, Eq. 8. */
#define KAZE_DOH_SIGMA4 0         /* s_i^4 det, s_i = max(1, round(sigma_i)) (default) */
#define KAZE_DOH_PAPER_LITERAL 1  /* (sigma_i / 2^o_i)^2 det, as Eq. 8 is printed      */

typedef struct kaze_options {
    int octaves;          /* O of Eq. 6 (>= 1)                                   */
    int sublevels;        /* S of Eq. 6 (>= 1); N = O*S levels, N <= 64           */
    float sigma0;         /* base scale of Eq. 6 and presmoothing std (1.6)       */
    float sigma_d;        /* std of the Gaussian before the gradient (1.0), <= 2  */
    double k_percentile;  /* percentile of the gradient histogram, (0, 1] (0.7)   */
    int nbins;            /* histogram bins (300), 1..4096                        */
    int diffusivity;      /* KAZE_G1 or KAZE_G2 (default)                         */
    float dthreshold;     /* detector threshold (0.001)                           */
    float edge_r;         /* edge ratio r of Eq. 12 (10); <= 0 disables the test  */
    int doh_norm;         /* KAZE_DOH_*                                           */
    float k_override;     /* > 0: use this contrast factor, skip the histogram    */
    int max_keypoints;    /* capacity of the device keypoint buffer (65536)       */
    int scheme;           /* KAZE_SCHEME_AOS (default) or KAZE_SCHEME_FED         */
    float fed_tau_max;    /* FED stability limit, (0, 0.25] (0.25)                */
    int extrema_window;   /* KAZE_EXTREMA_3X3 (default) or _SIGMA_WINDOW          */
    int aos_solver;       /* KAZE_AOS_AUTO (default), _LINES or _STREAMED           */
} kaze_options;

/* One detected keypoint (Sec. II-B). */
typedef struct kaze_keypoint {
    float x, y;       /* sub-pixel position in full-resolution pixels          */
    float sigma;      /* sigma_i of the level (Eq. 6)                          */
    float response;   /* DoH_i at the detected pixel (Eq. 8)                   */
    float angle;      /* dominant orientation; 0 until described             */
    int level;        /* i = o*S + s                                           */
    int octave;       /* o                                                     */
    int sublevel;     /* s                                                     */
    int ix, iy;       /* integer pixel at which the 3x3x3 maximum was found    */
} kaze_keypoint;

typedef struct kaze_handle kaze_handle;

/* Fills *opt with the defaults listed beside each field. */
void kaze_default_options(kaze_options* opt);

/* Creates a handle for images up to max_w x max_h (3 <= max_w, max_h <= 4128:
 * each row and column is solved by 32 chunks whose coefficients must fit in
 * registers and shared memory).
 * Allocates all device buffers up front (about (2N + 4) * max_w * max_h * 4
 * bytes -- levels, responses, conductance, row solution, two input planes
 * -- plus 336 bytes per keypoint of max_keypoints).  cuda_stream: the
 * cudaStream_t all work goes to.  On error *out is NULL.  Errors:
 * INVALID_ARG (bad options or sizes), OOM, CUDA. */
kaze_status kaze_create(const kaze_options* opt, int max_w, int max_h,
                        void* cuda_stream, kaze_handle** out);

/* Replaces the handle's stream (work already enqueued stays where it is). */
kaze_status kaze_set_stream(kaze_handle* h, void* cuda_stream);

/* Builds the nonlinear scale space of Sec. II-A / Sec. III-1 from the device
 * image d_img (w x h, pitch_elems): L_0 = G_sigma0 * I, k on the device
 * (no host sync), then for i = 1..N-1 one AOS step of Eq. 4 with
 * tau = t_i - t_{i-1} (Eq. 7).  Asynchronous. */
kaze_status kaze_build_scale_space(kaze_handle* h, const float* d_img, int w, int h_,
                                   int pitch_elems);

/* Borrowed pointer to level L_i (0 <= i < N) of the last build, its pitch in
 * elements and its evolution time t_i.  Any output pointer may be NULL. */
kaze_status kaze_get_level(kaze_handle* h, int i, const float** d_level,
                           int* pitch_elems, float* t_i);

/* Test hook for failure detection of the resident AOS evolution
 * (KAZE_AOS_AUTO): sets how many SM cycles one of its grid-barrier waits may
 * take (0 restores the default, 2^31) and, if stall_tile >= 0, makes that
 * tile never arrive at a barrier, so every wait runs out, the kernel returns
 * early and the detection reports KAZE_ERR_TIMEOUT.  stall_tile < 0 clears
 * the stall.  Drops the handle's recorded graphs. */
kaze_status kaze_set_evolve_wait_limit(kaze_handle* h, long long cycles, int stall_tile);

/* Scale of level i (0 <= i < N) from the handle's options, available
 * without a build: sigma_i = sigma0 2^(o + s/S) of Eq. 6 (i = o S + s) and
 * t_i = sigma_i^2 / 2 of Eq. 7, both as FP32 -- the values the kernels use
 * (sigma_i sets the derivative step of Eq. 8 and the sampling of the
 * descriptor).  Either output may be NULL.  INVALID_ARG for a bad index. */
kaze_status kaze_get_level_scale(kaze_handle* h, int i, float* sigma_i, float* t_i);

/* Contrast factor k used by the last build (synchronises the stream). */
kaze_status kaze_get_contrast(kaze_handle* h, float* k);

/* Detector response of Eq. 8 for all N levels of the last build.  Async. */
kaze_status kaze_detector_response(kaze_handle* h);

/* Borrowed pointer to DoH_i of the last kaze_detector_response. */
kaze_status kaze_get_response(kaze_handle* h, int i, const float** d_doh, int* pitch_elems);

/* 3x3x3 maxima of the responses (levels 1..N-2, 1-pixel border), sub-pixel
 * fit and edge test (Sec. II-B, Eq. 9-12).  Copies the keypoints to h_out
 * sorted by (level, iy, ix) and their total number to *count.  If the total
 * exceeds capacity (or the handle's max_keypoints), the first entries of the
 * sorted order that fit are written, *count holds the true total and the
 * call returns KAZE_ERR_CAPACITY.  h_out may be NULL when capacity is 0.
 * Synchronises the stream. */
kaze_status kaze_find_extrema(kaze_handle* h, kaze_keypoint* h_out, int capacity, int* count);

/* kaze_build_scale_space + kaze_detector_response + kaze_find_extrema on a
 * device image.  The fixed launch sequence is recorded once per image size
 * and input pointer as a CUDA graph and replayed afterwards; on the legacy
 * or per-thread default stream, which cannot be captured, the same kernels
 * are launched one by one.  Synchronises the stream.  The keypoint count
 * travels to the host with the first min(4096, max_keypoints) keypoint slots
 * (40 bytes each, in one copy), so a detection with no more keypoints than
 * that takes one round trip; more take a second copy. */
kaze_status kaze_detect(kaze_handle* h, const float* d_img, int w, int h_, int pitch_elems,
                        kaze_keypoint* h_out, int capacity, int* count);

/* kaze_detect in two halves, so that the host can work while the GPU
 * detects: kaze_detect_enqueue replays the recorded detection (with the
 * count and the keypoint slots copied to pinned host memory) on the handle's
 * stream and returns without waiting; kaze_detect_collect waits for it and
 * fills h_out, capacity and count as kaze_detect does.  Every enqueue must be
 * collected before the handle's next build or detection (STATE otherwise);
 * collect without an enqueue returns KAZE_ERR_STATE. */
kaze_status kaze_detect_enqueue(kaze_handle* h, const float* d_img, int w, int h_, int pitch_elems);
kaze_status kaze_detect_collect(kaze_handle* h, kaze_keypoint* h_out, int capacity, int* count);

/* kaze_detect on a HOST image: copies h_img to the device on the handle's
 * stream, runs the pipeline, copies the keypoints back.  For overlap the
 * host buffer should be page-locked (e.g. torch pinned memory). */
kaze_status kaze_detect_host(kaze_handle* h, const float* h_img, int w, int h_, int pitch_elems,
                             kaze_keypoint* h_out, int capacity, int* count);

/* kaze_detect_host for a stream of host images: also starts copying h_next
 * (the next image: same w, h_ and pitch; NULL for none) to the device on a
 * second stream while h_img is detected, into the other of the handle's
 * two input planes.  A following kaze_detect_host or kaze_detect_host_next
 * whose h_img is that h_next (same size and pitch) then detects the copy
 * already on the device instead of copying again.  h_next must stay valid
 * and unchanged until that call, and be page-locked for the copy to
 * overlap.  Keypoints, count and errors as kaze_detect_host; synchronises
 * the handle's stream (the copy of h_next may still be in flight). */
kaze_status kaze_detect_host_next(kaze_handle* h, const float* h_img, const float* h_next, int w, int h_,
                                  int pitch_elems, kaze_keypoint* h_out, int capacity, int* count);

/* ---- description (Sec. II-C) --------------------------------------------- *
 * Dominant orientation and 64-D M-SURF descriptor of keypoints on the levels
 * of the last kaze_build_scale_space (any level of the stack, all in one
 * launch).  Per keypoint: first derivatives of its level L_i by the step-s_i
 * Scharr pair of the detector, sampled bilinearly (taps clamped into the
 * image); the orientation is the angle of the longest response sum over pi/3
 * windows (72 five-degree sectors) of 109 samples within 6 sigma_i, weighted
 * by a Gaussian of std 2.5 sigma_i; the descriptor sums (r_x', r_y', |r_x'|,
 * |r_y'|) in the rotated frame over 4 x 4 subregions of 9 x 9 samples spaced
 * sigma_i (centres 5 sigma_i apart, 24 sigma_i window) with Gaussian weights
 * of std 2.5 sigma_i per subregion and 1.5 grid units over the 4 x 4 mask;
 * entry 4 (4 q + p) + c holds component c of subregion (p, q) (p along the
 * orientation, q across it) and the 64 entries have unit Euclidean norm.
 * upright != 0 skips the orientation (angle 0).  The keypoint's x, y (sub-
 * pixel, full resolution) and level are read; its sigma field is not (the
 * level's sigma_i is used); angle receives the orientation in radians, in
 * [0, 2 pi). */

/* Host arrays: kps (n keypoints, angle written back) and desc (n x 64
 * floats, row k for kps[k]).  Synchronises.  Errors: INVALID_ARG (NULL
 * arrays with n > 0, a level outside 0..N-1, a non-finite position), STATE
 * (no build yet), CAPACITY (n > max_keypoints), CUDA. */
kaze_status kaze_describe(kaze_handle* h, kaze_keypoint* kps, int n, float* desc, int upright);

/* Device arrays d_kps (n keypoints, angle written back) and d_desc (n x 64
 * floats); asynchronous on the handle's stream, no size limit beyond the
 * caller's buffers.  A keypoint whose level is outside 0..N-1 gets a zero
 * descriptor and angle 0. */
kaze_status kaze_describe_device(kaze_handle* h, kaze_keypoint* d_kps, int n, float* d_desc, int upright);

/* Description on one caller-supplied level image d_L (w x h_, pitch) of scale
 * sigma: every keypoint is taken to lie on it (its level is ignored).  Host
 * kps / desc as kaze_describe; synchronises. */
kaze_status kaze_op_describe(kaze_handle* h, const float* d_L, int pitch, int w, int h_, float sigma,
                             kaze_keypoint* kps, int n, float* desc, int upright);

/* ---- single steps, for testing each kernel on given inputs -------------- *
 * These run one step of the method on caller-owned device buffers on the
 * handle's stream.  Sizes obey the same limits as kaze_build_scale_space.   */

/* Separable Gaussian (sampled, normalised, radius ceil(3 sigma) <= 16) with
 * half-sample symmetric borders; in and out may not alias.  Async. */
kaze_status kaze_op_gaussian(kaze_handle* h, const float* d_in, int in_pitch,
                             float* d_out, int out_pitch, int w, int h_, float sigma);

/* Contrast factor of Sec. III-1 from base image d_L0 with the handle's
 * sigma_d, k_percentile and nbins; returns k, hmax and (if h_hist != NULL)
 * the nbins histogram counts.  Synchronises. */
kaze_status kaze_op_contrast(kaze_handle* h, const float* d_L0, int pitch, int w, int h_,
                             float* h_k, float* h_hmax, unsigned int* h_hist);

/* Conductance of Eq. 2-3 (handle's sigma_d and diffusivity) of d_L with
 * contrast factor k into d_g (same pitch).  Async. */
kaze_status kaze_op_conductance(kaze_handle* h, const float* d_L, float* d_g, int pitch,
                                int w, int h_, float k);

/* One AOS step of Eq. 4 with step tau: d_ux receives the row solution,
 * d_Lnext = (row solution + column solution) / 2.  All buffers share pitch,
 * which must be a multiple of 4, and start on 16-byte boundaries; outputs
 * must not alias inputs.  Synchronises the stream (it reports a timed-out
 * device wait as KAZE_ERR_TIMEOUT). */
kaze_status kaze_op_aos_step(kaze_handle* h, const float* d_Lprev, const float* d_g,
                             float* d_ux, float* d_Lnext, int pitch, int w, int h_, float tau);

/* One FED cycle (Eq. 5) from d_Lprev to stopping time dt with the
 * conductance d_g held fixed: n explicit steps of the handle's scheme
 * (fed_tau_max), up to four per launch, alternating between d_scratch and
 * d_Lnext and ending in d_Lnext.  All buffers share pitch (a multiple of 4)
 * and start on 16-byte boundaries; outputs must not alias inputs or each
 * other.  *n_steps (may be NULL) receives n.  Synchronises the stream (it
 * reports a timed-out device wait as KAZE_ERR_TIMEOUT). */
kaze_status kaze_op_fed_cycle(kaze_handle* h, const float* d_Lprev, const float* d_g, float* d_scratch,
                              float* d_Lnext, int pitch, int w, int h_, float dt, int* n_steps);

/* k explicit steps of Eq. 5 (1 <= k <= 4), of sizes h_tau[0..k-1] in that
 * order, from d_Lprev into d_Lnext with d_g held fixed, in one launch (the
 * steps are taken as a wavefront over the rows of tiles staged in shared
 * memory, with a 4-column halo per warp); the result equals k single steps
 * bit for bit.  Same layout rules as kaze_op_fed_cycle; d_Lnext may not
 * alias d_Lprev or d_g.  Synchronises the stream, as kaze_op_fed_cycle
 * does. */
kaze_status kaze_op_fed_steps(kaze_handle* h, const float* d_Lprev, const float* d_g, float* d_Lnext,
                              int pitch, int w, int h_, const float* h_tau, int k);

/* Detector response of Eq. 8 of one level: step s = max(1, round(sigma_i)),
 * normalisation by the handle's doh_norm.  Async. */
kaze_status kaze_op_doh(kaze_handle* h, const float* d_L, float* d_D, int pitch,
                        int w, int h_, float sigma_i, int octave);

/* Extrema of a caller-supplied response stack of n levels (level l at
 * d_D + l * plane_stride, each with the given pitch); level l has scale
 * sigma[l] (host array).  d_D must be 16-byte aligned and pitch and
 * plane_stride multiples of 4 (rows are read 4 values at a time).  Output as
 * kaze_find_extrema.  Synchronises. */
kaze_status kaze_op_extrema(kaze_handle* h, const float* d_D, int pitch, long long plane_stride,
                            int w, int h_, int n, const float* h_sigma,
                            kaze_keypoint* h_out, int capacity, int* count);

/* ---- batches of images: one persistent launch -------------------------- *
 * A batch handle serves a fixed list of n images of (possibly different)
 * sizes w[i] x h[i] (3..4096 each), all with the same options.  One call
 * runs the whole detection of every image -- presmoothing, contrast
 * factor, the N-1 AOS steps, the responses of all levels and the extrema --
 * as ONE persistent kernel whose CTAs pop work items (tiles, row groups,
 * column strips) from an ordered device queue; an item waits, with a
 * bounded spin, until the stages it reads are complete for its image.  The
 * launch and its set-up are recorded once as a CUDA graph and replayed
 * (except on the legacy or per-thread default stream).  Results match the
 * single-image path.  Batches evolve by AOS and test 3x3x3 maxima: options
 * with scheme KAZE_SCHEME_FED or extrema_window KAZE_EXTREMA_SIGMA_WINDOW are
 * refused (INVALID_ARG). */
typedef struct kaze_batch kaze_batch;

/* Execution of a batch.
 *   KAZE_BATCH_PERSISTENT: the one persistent launch described above;
 *     cols_per_strip (4: 64 chunks per column, 8: 32 chunks) and
 *     ctas_per_sm (capped by occupancy) shape it.
 *   KAZE_BATCH_CONCURRENT: each image runs the single-image kernel
 *     sequence; `streams` sequences run side by side as parallel branches
 *     of one recorded graph.
 *   KAZE_BATCH_RESIDENT (the default where every image takes it: at most
 *     16 x 16 tiles of 128 x 120 and no more tiles than SMs, sigma0 in
 *     (4/3, 5/3], sigma_d <= 2): the presmoothing, contrast factor and every
 *     AOS step of every image in ONE cooperative launch of one CTA per SM,
 *     each image's tiles resident in shared memory on the CTAs of one wave
 *     (images packed into waves largest first); then, per image, one
 *     response launch and one launch of the extremum test on the pixels it
 *     lists.  The other fields are not used. */
#define KAZE_BATCH_PERSISTENT 0
#define KAZE_BATCH_CONCURRENT 1
#define KAZE_BATCH_RESIDENT 2
typedef struct kaze_batch_tuning {
    int mode;
    int cols_per_strip;
    int ctas_per_sm;
    int streams;
} kaze_batch_tuning;

/* Allocates every plane of every image (2N + 2 planes each), the keypoint
 * buffers (max_keypoints per image) and the work list.  Errors:
 * INVALID_ARG (options, n outside 1..65535, sizes), OOM, CUDA. */
kaze_status kaze_batch_create(const kaze_options* opt, int n, const int* w, const int* h_, void* cuda_stream,
                              kaze_batch** out);

/* Detects keypoints in the n device images d_imgs[i] (row pitch pitches[i]
 * elements, or w[i] when pitches is NULL).  Image i's keypoints, sorted by
 * (level, iy, ix), go to h_out + i * capacity_per_image and their true
 * number to counts[i]; KAZE_ERR_CAPACITY if any image had more than fit.
 * KAZE_ERR_TIMEOUT if a bounded device wait ran out.  Synchronises. */
kaze_status kaze_batch_detect(kaze_batch* b, const float* const* d_imgs, const int* pitches,
                              kaze_keypoint* h_out, int capacity_per_image, int* counts);

/* Borrowed pointers to level / response `level` of image `image` after the
 * last kaze_batch_detect, with their pitch. */
kaze_status kaze_batch_get_level(kaze_batch* b, int image, int level, const float** d_level, int* pitch_elems);
kaze_status kaze_batch_get_response(kaze_batch* b, int image, int level, const float** d_doh, int* pitch_elems);

/* Current / new solve-tile shape (a new shape re-plans and re-records). */
kaze_status kaze_batch_get_tuning(const kaze_batch* b, kaze_batch_tuning* t);
kaze_status kaze_batch_set_tuning(kaze_batch* b, const kaze_batch_tuning* t);

/* Autotuner: times every candidate (resident; persistent with cols_per_strip
 * in {4, 8} x ctas_per_sm in {1, 2}; concurrent with 4, 8 or 16 streams) on
 * the given images, `reps` runs each (CUDA events), keeps the fastest and
 * reports it and its mean time in ms. */
kaze_status kaze_batch_autotune(kaze_batch* b, const float* const* d_imgs, const int* pitches, int reps,
                                kaze_batch_tuning* best, double* best_ms);

/* Test hook for failure detection (persistent mode): sets how many SM
 * cycles a device-side wait may take (default 2^31) and, if stall_image >=
 * 0, makes one stage of that image wait for an item that never exists, so
 * the wait runs out and kaze_batch_detect returns KAZE_ERR_TIMEOUT.
 * stall_image < 0 clears the hook. */
kaze_status kaze_batch_set_wait_limit(kaze_batch* b, long long cycles, int stall_image);

/* Message of the batch's first error ("" if none). */
const char* kaze_batch_last_error(const kaze_batch* b);

void kaze_batch_destroy(kaze_batch* b);

/* ---- a step that allocates nothing ------------------------------------- *
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot let a library allocate device memory (a framework whose
 * caching allocator owns the GPU's memory, a processing loop that must not
 * allocate once running).
 *
 * kaze_aos_step_static computes d_Lnext from d_Lprev and the conductance
 * d_g exactly as kaze_op_aos_step does (one AOS step of Eq. 4 with step
 * tau), without a handle and without allocating: the row solution it needs
 * internally lives in a file-scope device array that every GPU loading the
 * library holds until the process exits.  Limits: pitch * h <= 4,194,304
 * (16 MiB of scratch), 3 <= w, h <= 4128, pitch >= w and a multiple of 4,
 * all three buffers 16-byte aligned, d_Lnext overlapping neither input
 * (each plane spans pitch * (h - 1) + w floats), cuda_stream belonging to
 * the current device; anything else returns KAZE_ERR_INVALID_ARG before
 * touching the GPU.
 * The first call on a device looks up the array's device address and sets
 * the kernels' shared-memory limits for the current device, so make that
 * first call before any stream capture.  The address is kept for the life
 * of the process: a cudaDeviceReset in between is not supported.  All calls
 * share the one array: calls that overlap on the GPU (different streams, or
 * another thread) race on it and must be serialised by the caller.
 * The call is synchronous: its work goes to cuda_stream (cudaStream_t) and
 * the call waits for that stream before it returns KAZE_OK,
 * KAZE_ERR_TIMEOUT (a bounded device wait ran out) or KAZE_ERR_CUDA. */
kaze_status kaze_aos_step_static(const float* d_Lprev, const float* d_g, float* d_Lnext, int pitch, int w,
                                 int h_, float tau, void* cuda_stream);

/* ---- learned AOS surrogate ---------------------------------------------- *
 * Not in the paper: a small convolutional network that stands in for one
 * AOS step of Eq. 4.  From the previous level L, its conductance g
 * (Eq. 2-3, as kaze_op_conductance computes it) and the step
 * tau = t_i - t_{i-1} (Eq. 7) it predicts the next level:
 *   x0 = (dx, dy, g, s, c) per pixel: dx = 16 (L(x+1, y) - L(x, y)) and
 *        dy = 16 (L(x, y+1) - L(x, y)) (0 in the last column / row),
 *        s = log(1 + tau) / 5, c = 1; all zero outside the image.  L enters
 *        through its differences only, as the AOS step commutes with adding
 *        a constant to L;
 *   h1 = relu(conv(x0)), h2 = relu(conv(h1)), h3 = relu(conv(h2)),
 *   z = conv(h3), every conv 3x3 with zero padding and a bias, widths
 *   5-32-32-32-1;  L_next = L + z / 256.
 * Weights, every layer input (x0, h1, h2, h3) and every back-propagated
 * layer gradient are BF16 (nearest, ties to even); biases are FP32; all sums
 * are accumulated in FP32 on the tensor cores.  Training minimises the mean
 * over all pixels of all samples of (L_next - T)^2 with Adam (beta1 0.9,
 * beta2 0.999, eps 1e-8, bias-corrected) on FP32 master weights.  Training
 * kernels add their partial sums in a fixed order: the same calls from the
 * same state give bit-identical results, so a run resumed from a checkpoint
 * repeats the uninterrupted one.
 *
 * Parameter vectors (KAZE_SURROGATE_PARAMS FP32 values, host memory): for
 * each layer in order, W[out][3][3][in] (the two 3s: dy, dx = -1, 0, 1),
 * then b[out].  Tap (dy, dx) of W multiplies the input at (x + dx, y + dy).
 *
 * Sample arrays: d_L[i], d_g[i], d_T[i], d_out[i] are DEVICE pointers to
 * FP32 planes of w x h with the given pitch (elements); the arrays holding
 * them and h_tau are HOST arrays of n entries, 1 <= n <=
 * KAZE_SURROGATE_MAX_SAMPLES.  The sample table travels in the kernels'
 * parameters, so steps can be recorded in a CUDA graph. */
#define KAZE_SURROGATE_PARAMS 20257
#define KAZE_SURROGATE_MAX_SAMPLES 64
#define KAZE_SURROGATE_TRAIN 1   /* create flag: allocate training buffers      */
#define KAZE_SURROGATE_FUSED 0      /* step path: whole network in one kernel, tcgen05 */
#define KAZE_SURROGATE_LAYERED 1    /* step path: one kernel per layer (TRAIN)         */
#define KAZE_SURROGATE_FUSED_SYNC 2 /* step path: one kernel on mma.sync (cross-check)  */

typedef struct kaze_surrogate kaze_surrogate;

/* Creates a surrogate with seeded initial parameters: layers 1-3 uniform in
 * +-sqrt(6 / (9 in)) from splitmix64 draws, the last layer and all biases 0
 * (the untrained network returns L).  With KAZE_SURROGATE_TRAIN in flags it
 * also allocates activations and gradients for max_samples images of up to
 * max_w x max_h (about 440 bytes per pixel); without it the surrogate can
 * only run the fused step, for any image size.  Returns KAZE_ERR_OOM or
 * KAZE_ERR_INVALID_ARG (message: kaze_surrogate_last_error(NULL)). */
kaze_status kaze_surrogate_create(int max_w, int max_h, int max_samples, int flags, unsigned long long seed,
                                  void* cuda_stream, kaze_surrogate** out);
kaze_status kaze_surrogate_set_stream(kaze_surrogate* s, void* cuda_stream);

/* Copies the FP32 master parameters out / in (count must equal
 * KAZE_SURROGATE_PARAMS).  set_params also zeroes the Adam moments and the
 * step count.  Both synchronise the stream. */
kaze_status kaze_surrogate_get_params(kaze_surrogate* s, float* h_params, int count);
kaze_status kaze_surrogate_set_params(kaze_surrogate* s, const float* h_params, int count);

/* d_out[i] = L_next of sample i (asynchronous).  path KAZE_SURROGATE_FUSED
 * runs one persistent kernel on the tcgen05 tensor cores (accumulators in
 * tensor memory); KAZE_SURROGATE_FUSED_SYNC the same network in one kernel
 * on mma.sync; KAZE_SURROGATE_LAYERED the layer kernels of training (needs
 * KAZE_SURROGATE_TRAIN and sizes within the maximum).  The three agree to
 * FP32 summation order.  d_out[i] must not overlap d_L[j] or d_g[j] (equal
 * pointers are rejected). */
kaze_status kaze_surrogate_step(kaze_surrogate* s, const float* const* d_L, const float* const* d_g,
                                const float* h_tau, float* const* d_out, int n, int w, int h_, int pitch,
                                int path);

/* Waits for the surrogate's stream; KAZE_ERR_TIMEOUT (and the flag cleared)
 * if a bounded device-side wait of a fused step ran out since the last
 * call. */
kaze_status kaze_surrogate_sync(kaze_surrogate* s);

/* Loss and its gradient with respect to the parameters (h_grad: host,
 * KAZE_SURROGATE_PARAMS values) for targets d_T; h_loss may be NULL.
 * Parameters are not changed.  Synchronises. */
kaze_status kaze_surrogate_gradients(kaze_surrogate* s, const float* const* d_L, const float* const* d_g,
                                     const float* h_tau, const float* const* d_T, int n, int w, int h_,
                                     int pitch, double* h_loss, float* h_grad);

/* One Adam step with learning rate lr on the batch.  *h_loss (if h_loss is
 * not NULL) receives the loss before the update, which synchronises. */
kaze_status kaze_surrogate_train_step(kaze_surrogate* s, const float* const* d_L, const float* const* d_g,
                                      const float* h_tau, const float* const* d_T, int n, int w, int h_,
                                      int pitch, float lr, double* h_loss);

/* Number of Adam steps applied so far (restored by kaze_surrogate_load).
 * KAZE_ERR_INVALID_ARG for a NULL surrogate or steps.  Host only. */
kaze_status kaze_surrogate_steps_taken(const kaze_surrogate* s, long long* steps);

/* Checkpoint: "KZSG", uint32 version 1, uint32 KAZE_SURROGATE_PARAMS,
 * uint32 0, int64 steps taken, then parameters, Adam first and second
 * moments (FP32, parameter-vector layout), all little-endian.  load
 * restores all of it; a file that is not such a checkpoint gives
 * KAZE_ERR_INVALID_ARG and leaves the surrogate unchanged. */
kaze_status kaze_surrogate_save(kaze_surrogate* s, const char* path);
kaze_status kaze_surrogate_load(kaze_surrogate* s, const char* path);

/* Kernels the surrogate's last call enqueued; -1 for NULL. */
int kaze_surrogate_last_launch_count(const kaze_surrogate* s);
/* First error the surrogate recorded; with s == NULL, why the calling
 * thread's last kaze_surrogate_create failed. */
const char* kaze_surrogate_last_error(const kaze_surrogate* s);
void kaze_surrogate_destroy(kaze_surrogate* s);

/* Makes the handle's scale space evolve with the surrogate's fused step
 * instead of the AOS row and column solves (s = NULL restores AOS, the
 * default).  The surrogate is borrowed: keep it alive while it is set.
 * Drops the handle's recorded detection graph. */
kaze_status kaze_set_surrogate(kaze_handle* h, kaze_surrogate* s);

/* Loads a surrogate checkpoint (the format of kaze_surrogate_save) into a
 * surrogate the handle owns and evolves the scale space with it from then
 * on, as kaze_set_surrogate does; path NULL restores AOS and frees it.  A
 * file that is not a checkpoint gives KAZE_ERR_INVALID_ARG and leaves the
 * handle as it was.  Synchronises. */
kaze_status kaze_load_surrogate(kaze_handle* h, const char* path);

/* The whole detection of n images of (possibly different) sizes w[i] x h[i]
 * (3..4096, rows contiguous: pitch = w[i]) on device memory d_imgs[i], with
 * the handle's options, through one batch (kaze_batch_create /
 * kaze_batch_detect, which the handle keeps while the size list repeats).
 * Image i's keypoints, sorted by (level, iy, ix), go to h_out + i *
 * capacity and their true number to counts[i]; KAZE_ERR_CAPACITY when one
 * exceeds capacity.  Batches evolve by AOS and test 3x3x3 maxima.
 * Synchronises. */
kaze_status kaze_build_batch(kaze_handle* h, const float* const* d_imgs, const int* w, const int* h_, int n,
                             kaze_keypoint* h_out, int capacity, int* counts);

/* ---- instrumentation ---------------------------------------------------- */

/* Number of kernel kinds the pipeline launches, and the name of kind k
 * (presmooth, grad_max, grad_hist, percentile, set_scalar, conductance,
 * aos_rows, aos_cols, doh, extrema); "" for an unknown kind. */
int kaze_kernel_kinds(void);
const char* kaze_kernel_name(int kind);

/* Kernels enqueued by the handle's last pipeline call (kaze_build_scale_space,
 * kaze_detect, kaze_detect_host or kaze_profile; a replayed graph counts the
 * kernels it holds); -1 for a NULL handle. */
int kaze_last_launch_count(const kaze_handle* h);

/* Times kaze_build_scale_space + kaze_detector_response + the extrema
 * kernel with a CUDA event pair recorded on the handle's stream around every
 * kernel (the two halves of each AOS step run one after the other here).
 * On a capturable stream the sequence is recorded as a CUDA graph and
 * replayed twice, the times taken from the second replay, as a detection
 * runs; on the legacy or per-thread default stream it runs once, launch by
 * launch.  h_ms[k] receives the summed device time in ms of kind k,
 * h_launches[k] its number of kernels; both arrays hold kaze_kernel_kinds()
 * entries.  Synchronises the stream. */
kaze_status kaze_profile(kaze_handle* h, const float* d_img, int w, int h_, int pitch_elems,
                         double* h_ms, int* h_launches);

/* Static description of a status code. */
const char* kaze_status_string(kaze_status s);

/* Message of the first error the handle recorded ("" if none).  With
 * h == NULL: why the calling thread's last failed kaze_create failed. */
const char* kaze_last_error(const kaze_handle* h);

/* Frees every device buffer and the handle.  NULL is ignored. */
void kaze_destroy(kaze_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* KAZE_H */
