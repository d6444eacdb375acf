/*
 * kaze_oracle.h -- plain FP64 CPU oracle of the KAZE scale space and detector.
 *
 * TEST INFRASTRUCTURE ONLY.  This file and kaze_oracle.c are the slow,
 * obviously-correct restatement of the method against which the CUDA path is
 * checked.  Only the test suite, the smoke check and the CPU-baseline leg of
 * the benchmark may build, load or call it.  It shares no code, header, table
 * or constant with the CUDA library (include/kaze.h, paper_1706_06750_gb300/).
 *
 * Paper: "GPGPU Acceleration of the KAZE Image Feature Extraction Algorithm"
 * (arXiv 1706.06750).  Each function names the section / equation it follows.
 *
 * Conventions: images are row-major double arrays of W*H values, element
 * (x, y) at [y*W + x].  Borders use half-sample symmetric extension.
 */
#ifndef KAZE_ORACLE_H
#define KAZE_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Diffusivity selector, Eq. 3. */
#define KO_G1 1   /* exp(-|grad|^2 / k^2) */
#define KO_G2 2   /* 1 / (1 + |grad|^2 / k^2)  (default) */

/* Evolution scheme of each level (Sec. II-A). */
#define KO_SCHEME_AOS 0         /* one AOS step of Eq. 4 per level             */
#define KO_SCHEME_FED 1         /* one FED cycle of explicit steps, Eq. 5      */

/* Cross-level neighbourhood of the maximum test (Sec. II-B, Sec. IV). */
#define KO_EXTREMA_3X3 0           /* 3x3 at levels i-1 and i+1 (26 neighbours)  */
#define KO_EXTREMA_SIGMA_WINDOW 1  /* the sigma x sigma window at levels i +- 1  */

/* Hessian normalisation selector, Eq. 8 (see ko_doh). */
#define KO_DOH_SIGMA4 0         /* s_i^4 * det, s_i = max(1, round(sigma_i)) */
#define KO_DOH_PAPER_LITERAL 1  /* (sigma_i / 2^o_i)^2 * det                 */

typedef struct {
    int octaves, sublevels;     /* O, S of Eq. 6                               */
    double sigma0;              /* base scale of Eq. 6 and of the presmoothing */
    double sigma_d;             /* std of the smoothing before the gradient    */
    double k_percentile;        /* percentile of the gradient histogram        */
    int nbins;                  /* histogram bins                              */
    int diffusivity;            /* KO_G1 / KO_G2                               */
    double dthreshold;          /* detector threshold                          */
    double edge_r;              /* edge ratio r of Eq. 12; <= 0 disables       */
    int doh_norm;               /* KO_DOH_*                                    */
    double k_override;          /* > 0: use this k instead of the histogram    */
    int scheme;                 /* KO_SCHEME_AOS (default) or KO_SCHEME_FED    */
    double fed_tau_max;         /* FED stability limit tau_max (0.25)          */
    int extrema_window;         /* KO_EXTREMA_3X3 (default) or _SIGMA_WINDOW  */
} ko_options;

typedef struct {
    double x, y;        /* sub-pixel position (full-resolution pixels)       */
    double sigma;       /* sigma_i of the level                               */
    double response;    /* DoH_i at the detected pixel                        */
    int level, octave, sublevel;
    int ix, iy;         /* integer pixel at which the maximum was found       */
} ko_keypoint;

/* Half-sample symmetric index reflection into [0, n). */
/* Host threads for the loops over independent pixels and lines (the
 * results do not depend on it); ko_threads: the count in use. */
void ko_set_threads(int n);
int ko_threads(void);

long ko_reflect(long i, long n);

/* Eq. 6 / Eq. 7: sigma_i = sigma0 * 2^(o + s/S), t_i = sigma_i^2 / 2, N = O*S. */
void ko_scale_table(int O, int S, double sigma0, double* sigma, double* t);

/* Sampled normalised Gaussian of radius ceil(3 sigma); writes 2r+1 weights,
 * returns r (or -1 if cap is too small). */
int ko_gaussian_weights(double sigma, double* w, int cap);

/* Separable Gaussian convolution (rows, then columns). */
void ko_gaussian(const double* in, double* out, int W, int H, double sigma);

/* 3x3 Scharr first derivatives (step 1). */
void ko_scharr(const double* L, double* Lx, double* Ly, int W, int H);

/* Contrast factor k from the gradient histogram of the base image.
 * Returns k; optionally reports hmax, the histogram and the binned count. */
double ko_contrast_k(const double* L0, int W, int H, double sigma_d,
                     double pct, int nbins, double* hmax_out,
                     long long* hist_out, long long* nbinned_out);

/* Conductance g = g(|grad (G_sigma_d * L)|), Eq. 2 and Eq. 3. */
void ko_conductance(const double* L, int W, int H, double sigma_d, double k,
                    int diffusivity, double* g);

/* Thomas algorithm for a_j x_{j-1} + b_j x_j + c_j x_{j+1} = d_j. */
void ko_thomas(int n, const double* a, const double* b, const double* c,
               const double* d, double* x);

/* One AOS step of Eq. 4 (m = 2 directions): writes the row solution ux,
 * the column solution uy (either may be NULL) and Lnext = (ux + uy) / 2. */
void ko_aos_step(const double* Lprev, const double* g, int W, int H,
                 double tau, double* ux, double* uy, double* Lnext);

/* Eq. 5, readings F1-F3: the step sizes of one FED cycle that reaches the
 * stopping time dt.  n is the smallest cycle length whose stopping time
 * tau_max (n^2 + n) / 3 reaches dt; tau_j = tau_max / (2 cos^2(pi (2j + 1) /
 * (4n + 2))) for j = 0..n-1, all scaled by dt / (tau_max (n^2 + n) / 3) so
 * that they sum to dt.  Writes min(n, cap) sizes and returns n (0 when
 * dt <= 0). */
int ko_fed_tau(double dt, double tau_max, double* tau, int cap);

/* Reading F5: the order of the steps of one cycle.  The cycle is exact in
 * any order (the operator is fixed), but rounding errors of early steps are
 * amplified by the later ones; the kappa-cycle orders of Grewenig, Weickert
 * & Bruhn (2010) take step (kappa (l + 1) mod p) - 1 at position l (p the
 * smallest prime above n, values outside 0..n-1 skipped).  Of kappa = 1..n
 * the one whose worst-case amplification sum_j max|prod_{k<=j} (1 - tau_k x)|
 * * max|prod_{k>j} (1 - tau_k x)| over x in [0, 8] (the spectrum of the
 * operator for g <= 1, sampled at 2001 points) is smallest is taken, the
 * smallest kappa on ties.  Writes the permutation of 0..n-1 to order and
 * returns kappa. */
int ko_fed_order(int n, const double* tau, int* order);

/* One explicit diffusion step with the conductance g held fixed (F4):
 * out = L + tau * sum over the 4-neighbours q of (g_p + g_q)/2 (L_q - L_p);
 * a neighbour outside the image contributes nothing (no flux through the
 * border, the Neumann condition of the AOS step).  out may not alias L. */
void ko_fed_step(const double* L, const double* g, int W, int H, double tau, double* out);

/* One FED cycle: the steps of ko_fed_tau(dt, tau_max) in the order of
 * ko_fed_order from L.
 * Returns the number of steps. */
int ko_fed_evolve(const double* L, const double* g, int W, int H, double dt, double tau_max,
                  double* out);

/* Whole nonlinear scale space (Sec. II-A): presmoothing, k, N-1 AOS steps
 * (or FED cycles with opt->scheme == KO_SCHEME_FED).
 * levels holds N*W*H doubles.  Returns 0 on success. */
int ko_build_scale_space(const double* img, int W, int H, const ko_options* opt,
                         double* levels, double* k_used);

/* Derivative step s_i = max(1, round(sigma_i)). */
int ko_step_size(double sigma);

/* Concatenated step-s Scharr second derivatives (Sec. II-B). */
void ko_hessian(const double* L, int W, int H, int s,
                double* Lxx, double* Lyy, double* Lxy);

/* Normalised Hessian determinant of one level, Eq. 8 (reading in ko_doh). */
void ko_doh(const double* L, int W, int H, double sigma_i, int octave,
            int doh_norm, double* D);

/* Maxima with sub-pixel fit and edge test (Sec. II-B, Eq. 9-12): above the
 * threshold, strictly above the 8 neighbours at level i and above every
 * response of levels i-1 and i+1 within |dx|, |dy| <= r_i: r_i = 1 (the 3x3x3
 * test), or with window = KO_EXTREMA_SIGMA_WINDOW (reading W1) the sigma_i x
 * sigma_i window r_i = max(1, floor(s_i / 2)), s_i = max(1, round(sigma_i)),
 * pixels outside the image skipped.  D holds N*W*H responses.  Writes at most
 * cap keypoints, returns the total number found (which may exceed cap). */
int ko_find_extrema(const double* D, int W, int H, int N, int S,
                    const double* sigma, double dthreshold, double edge_r,
                    int window, ko_keypoint* out, int cap);

#ifdef __cplusplus
}
#endif
#endif
