/*
 * kaze_oracle.c -- plain FP64 CPU oracle of the KAZE scale space and detector.
 *
 * TEST INFRASTRUCTURE ONLY: used by the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark; never by the product path.  Written for
 * readability, not speed: one function per step of the method, in the order
 * the paper describes them, with no fusion or blocking.  Loops over
 * independent pixels or lines may run on several host threads (OpenMP, when
 * the compiler offers it; ko_set_threads): each output is computed by the
 * same operations either way, so the results do not depend on the thread
 * count.
 *
 * Readings of passages where the paper is silent or garbled (each also listed
 * in the design notes):
 *   R1 borders: half-sample symmetric extension everywhere (the Neumann
 *      condition of the diffusion); the paper is silent.
 *   R2 Gaussian: sampled, normalised, radius ceil(3 sigma).
 *   R3 Eq. 6 prints 2^((o+s)/S); read as sigma0 * 2^(o + s/S) (octaves double
 *      sigma, no two levels coincide).  N = O*S levels, indices 0..N-1.
 *   R4 k (Sec. III-1 takes k from a gradient histogram, procedure not given): smooth
 *      L0 with G(sigma_d = 1), 3x3 Scharr, magnitude over interior pixels,
 *      hmax = max, histogram of the non-zero magnitudes in nbins bins,
 *      k = hmax * (b+1)/nbins for the smallest bin b whose cumulative count
 *      reaches pct * n; fallback k = 0.03 when nothing is binned.
 *   R5 Eq. 4 is solved by AOS (additive operator splitting, Weickert et al.
 *      1998) with m = 2: L_{i+1} = 1/2 sum_l (I - 2 tau A_l(L_i))^-1 L_i,
 *      tau = t_{i+1} - t_i from Eq. 7, one step per level.
 *   R6 Eq. 8 is garbled; default normalisation s_i^4 with derivative step
 *      s_i = max(1, round(sigma_i)); the literal (sigma_i/2^o)^2 form is a
 *      flag.
 *   R7 extrema: maxima only, strict, level 1..N-2, 1-pixel border,
 *      3x3 neighbourhood on levels i-1, i, i+1 (the approximate check).
 *   R8 sub-pixel: Newton step on the 3x3 quadratic of the response; rejected
 *      when the Hessian is singular or the offset exceeds one pixel.
 *   R9 Eq. 10 prints Tr = Dxx + Dxy; read as Dxx + Dyy.  r = 10.
 */
#include "kaze_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Host threads for the loops over independent pixels and lines (1: serial). */
void ko_set_threads(int n)
{
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : 1);
#else
    (void)n;
#endif
}

int ko_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* R1: index i reflected into [0, n) by half-sample symmetric extension
 * (... 2 1 0 | 0 1 2 ... n-1 | n-1 n-2 ...), repeated for tiny n. */
long ko_reflect(long i, long n)
{
    long p = 2 * n;
    long r = i % p;
    if (r < 0) r += p;
    return r < n ? r : p - 1 - r;
}

static double at(const double* img, int W, int H, long x, long y)
{
    return img[ko_reflect(y, H) * (long)W + ko_reflect(x, W)];
}

/* Eq. 6 (reading R3) and Eq. 7. */
void ko_scale_table(int O, int S, double sigma0, double* sigma, double* t)
{
    for (int o = 0; o < O; ++o)
        for (int s = 0; s < S; ++s) {
            int i = o * S + s;
            sigma[i] = sigma0 * pow(2.0, (double)o + (double)s / (double)S);
            t[i] = 0.5 * sigma[i] * sigma[i];
        }
}

/* R2: w_j = exp(-j^2 / (2 sigma^2)), |j| <= r = ceil(3 sigma), sum 1. */
int ko_gaussian_weights(double sigma, double* w, int cap)
{
    int r = (int)ceil(3.0 * sigma);
    if (r < 1) r = 1;
    if (2 * r + 1 > cap) return -1;
    double sum = 0.0;
    for (int j = -r; j <= r; ++j) {
        w[j + r] = exp(-(double)(j * j) / (2.0 * sigma * sigma));
        sum += w[j + r];
    }
    for (int j = 0; j < 2 * r + 1; ++j) w[j] /= sum;
    return r;
}

/* Presmoothing and gradient smoothing (Sec. III-1): separable Gaussian,
 * along rows first, then along columns. */
void ko_gaussian(const double* in, double* out, int W, int H, double sigma)
{
    double w[512];
    int r = ko_gaussian_weights(sigma, w, 512);
    double* tmp = (double*)malloc(sizeof(double) * (size_t)W * H);
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            double acc = 0.0;
            for (int j = -r; j <= r; ++j) acc += w[j + r] * at(in, W, H, x + j, y);
            tmp[(long)y * W + x] = acc;
        }
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            double acc = 0.0;
            for (int j = -r; j <= r; ++j) acc += w[j + r] * at(tmp, W, H, x, y + j);
            out[(long)y * W + x] = acc;
        }
    free(tmp);
}

/* Scharr first derivatives (Sec. III-1, Weickert & Scharr 2002):
 * Lx = central difference [-1 0 1]/2 along x, smoothed by [3 10 3]/16
 * along y; Ly is the transpose. */
void ko_scharr(const double* L, double* Lx, double* Ly, int W, int H)
{
    const double c[3] = {3.0 / 16.0, 10.0 / 16.0, 3.0 / 16.0};
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            double gx = 0.0, gy = 0.0;
            for (int k = -1; k <= 1; ++k) {
                gx += c[k + 1] * 0.5 * (at(L, W, H, x + 1, y + k) - at(L, W, H, x - 1, y + k));
                gy += c[k + 1] * 0.5 * (at(L, W, H, x + k, y + 1) - at(L, W, H, x + k, y - 1));
            }
            Lx[(long)y * W + x] = gx;
            Ly[(long)y * W + x] = gy;
        }
}

/* Contrast factor k, reading R4. */
double ko_contrast_k(const double* L0, int W, int H, double sigma_d,
                     double pct, int nbins, double* hmax_out,
                     long long* hist_out, long long* nbinned_out)
{
    size_t P = (size_t)W * H;
    double* Ls = (double*)malloc(sizeof(double) * P);
    double* Lx = (double*)malloc(sizeof(double) * P);
    double* Ly = (double*)malloc(sizeof(double) * P);
    long long* hist = (long long*)calloc((size_t)nbins, sizeof(long long));
    ko_gaussian(L0, Ls, W, H, sigma_d);
    ko_scharr(Ls, Lx, Ly, W, H);

    double hmax = 0.0;
    for (int y = 1; y < H - 1; ++y)
        for (int x = 1; x < W - 1; ++x) {
            size_t p = (size_t)y * W + x;
            double m = sqrt(Lx[p] * Lx[p] + Ly[p] * Ly[p]);
            if (m > hmax) hmax = m;
        }

    long long n = 0;
    if (hmax > 0.0) {
        for (int y = 1; y < H - 1; ++y)
            for (int x = 1; x < W - 1; ++x) {
                size_t p = (size_t)y * W + x;
                double m = sqrt(Lx[p] * Lx[p] + Ly[p] * Ly[p]);
                if (m > 0.0) {
                    long b = (long)floor((double)nbins * m / hmax);
                    if (b > nbins - 1) b = nbins - 1;
                    hist[b] += 1;
                    n += 1;
                }
            }
    }

    double k = 0.03;
    if (n > 0) {
        long long cum = 0;
        for (int b = 0; b < nbins; ++b) {
            cum += hist[b];
            if ((double)cum >= pct * (double)n) {
                k = hmax * (double)(b + 1) / (double)nbins;
                break;
            }
        }
    }
    if (hmax_out) *hmax_out = hmax;
    if (hist_out) memcpy(hist_out, hist, sizeof(long long) * (size_t)nbins);
    if (nbinned_out) *nbinned_out = n;
    free(Ls); free(Lx); free(Ly); free(hist);
    return k;
}

/* Eq. 2 and Eq. 3: conductance of the Gaussian-smoothed gradient. */
void ko_conductance(const double* L, int W, int H, double sigma_d, double k,
                    int diffusivity, double* g)
{
    size_t P = (size_t)W * H;
    double* Ls = (double*)malloc(sizeof(double) * P);
    double* Lx = (double*)malloc(sizeof(double) * P);
    double* Ly = (double*)malloc(sizeof(double) * P);
    ko_gaussian(L, Ls, W, H, sigma_d);
    ko_scharr(Ls, Lx, Ly, W, H);
#pragma omp parallel for schedule(static)
    for (size_t p = 0; p < P; ++p) {
        double q = (Lx[p] * Lx[p] + Ly[p] * Ly[p]) / (k * k);
        g[p] = diffusivity == KO_G1 ? exp(-q) : 1.0 / (1.0 + q);
    }
    free(Ls); free(Lx); free(Ly);
}

/* Thomas algorithm (tridiagonal LU without pivoting): forward elimination,
 * then back substitution.  a[0] and c[n-1] are not used. */
void ko_thomas(int n, const double* a, const double* b, const double* c,
               const double* d, double* x)
{
    if (n <= 0) return;
    double* cp = (double*)malloc(sizeof(double) * (size_t)n);
    double* dp = (double*)malloc(sizeof(double) * (size_t)n);
    cp[0] = n > 1 ? c[0] / b[0] : 0.0;
    dp[0] = d[0] / b[0];
    for (int j = 1; j < n; ++j) {
        double den = b[j] - a[j] * cp[j - 1];
        cp[j] = j < n - 1 ? c[j] / den : 0.0;
        dp[j] = (d[j] - a[j] * dp[j - 1]) / den;
    }
    x[n - 1] = dp[n - 1];
    for (int j = n - 2; j >= 0; --j) x[j] = dp[j] - cp[j] * x[j + 1];
    free(cp); free(dp);
}

/* One line of the AOS operator (I - 2 tau A_l(g)) v = d with Neumann ends
 * (R5).  Between neighbours j and j+1 the diffusivity is the mean
 * w = (g_j + g_{j+1}) / 2, so the off-diagonal is -2 tau w and the diagonal
 * is 1 plus 2 tau times the sum of the diffusivities to existing neighbours. */
static void aos_line(int n, const double* gl, const double* dl, double tau, double* v)
{
    double* a = (double*)malloc(sizeof(double) * (size_t)n);
    double* b = (double*)malloc(sizeof(double) * (size_t)n);
    double* c = (double*)malloc(sizeof(double) * (size_t)n);
    for (int j = 0; j < n; ++j) {
        double wl = j > 0 ? 0.5 * (gl[j - 1] + gl[j]) : 0.0;
        double wr = j < n - 1 ? 0.5 * (gl[j] + gl[j + 1]) : 0.0;
        a[j] = -2.0 * tau * wl;
        c[j] = -2.0 * tau * wr;
        b[j] = 1.0 + 2.0 * tau * (wl + wr);
    }
    ko_thomas(n, a, b, c, dl, v);
    free(a); free(b); free(c);
}

/* Eq. 4 by AOS (R5): solve every row and every column, average. */
void ko_aos_step(const double* Lprev, const double* g, int W, int H,
                 double tau, double* ux, double* uy, double* Lnext)
{
    size_t P = (size_t)W * H;
    int n = W > H ? W : H;
    double* vx = (double*)malloc(sizeof(double) * P);
    double* vy = (double*)malloc(sizeof(double) * P);

#pragma omp parallel
    {
        /* one line's conductance, right-hand side and solution per thread */
        double* gl = (double*)malloc(sizeof(double) * (size_t)n);
        double* dl = (double*)malloc(sizeof(double) * (size_t)n);
        double* vl = (double*)malloc(sizeof(double) * (size_t)n);
#pragma omp for schedule(static)
        for (int y = 0; y < H; ++y) {          /* x direction: every row */
            for (int x = 0; x < W; ++x) {
                gl[x] = g[(size_t)y * W + x];
                dl[x] = Lprev[(size_t)y * W + x];
            }
            aos_line(W, gl, dl, tau, vl);
            for (int x = 0; x < W; ++x) vx[(size_t)y * W + x] = vl[x];
        }
#pragma omp for schedule(static)
        for (int x = 0; x < W; ++x) {          /* y direction: every column */
            for (int y = 0; y < H; ++y) {
                gl[y] = g[(size_t)y * W + x];
                dl[y] = Lprev[(size_t)y * W + x];
            }
            aos_line(H, gl, dl, tau, vl);
            for (int y = 0; y < H; ++y) vy[(size_t)y * W + x] = vl[y];
        }
        free(gl); free(dl); free(vl);
    }
    for (size_t p = 0; p < P; ++p) {
        if (Lnext) Lnext[p] = 0.5 * (vx[p] + vy[p]);
        if (ux) ux[p] = vx[p];
        if (uy) uy[p] = vy[p];
    }
    free(vx); free(vy);
}

/* Stopping time of one FED cycle of n steps with limit tau_max. */
static double fed_cycle_time(int n, double tau_max)
{
    return tau_max * ((double)n * n + n) / 3.0;
}

/* Eq. 5 with readings F1-F3 (see the header). */
int ko_fed_tau(double dt, double tau_max, double* tau, int cap)
{
    if (!(dt > 0.0) || !(tau_max > 0.0)) return 0;
    int n = (int)ceil(sqrt(3.0 * dt / tau_max + 0.25) - 0.5);
    if (n < 1) n = 1;
    while (fed_cycle_time(n, tau_max) < dt) ++n;
    while (n > 1 && fed_cycle_time(n - 1, tau_max) >= dt) --n;
    const double scale = dt / fed_cycle_time(n, tau_max);
    const double pi = 3.14159265358979323846;
    for (int j = 0; j < n && j < cap; ++j) {
        const double c = cos(pi * (2.0 * j + 1.0) / (4.0 * n + 2.0));
        tau[j] = scale * tau_max / (2.0 * c * c);
    }
    return n;
}

static int is_prime(int q)
{
    if (q < 2) return 0;
    for (int d = 2; d * d <= q; ++d)
        if (q % d == 0) return 0;
    return 1;
}

/* The kappa-cycle permutation: position l takes step (kappa (l+1) mod p) - 1. */
static void kappa_cycle(int n, int kappa, int* order)
{
    int p = n + 1;
    while (!is_prime(p)) ++p;
    int m = 0;
    for (int l = 0; m < n; ++l) {
        int idx = (int)(((long long)(l + 1) * kappa) % p) - 1;
        if (idx >= 0 && idx < n) order[m++] = idx;
    }
}

/* Worst-case rounding amplification of the steps in this order (F5). */
static double order_amplification(int n, const double* tau, const int* order)
{
    const int G = 2000;
    double* head = (double*)malloc(sizeof(double) * (size_t)n);
    double* tail = (double*)malloc(sizeof(double) * (size_t)n);
    for (int j = 0; j < n; ++j) head[j] = tail[j] = 0.0;
    for (int gi = 0; gi <= G; ++gi) {
        const double x = 8.0 * gi / G;
        double pr = 1.0;
        for (int j = 0; j < n; ++j) {          /* steps 0..j */
            pr *= fabs(1.0 - tau[order[j]] * x);
            if (pr > head[j]) head[j] = pr;
        }
        pr = 1.0;
        for (int j = n - 1; j >= 0; --j) {     /* steps j+1..n-1 */
            if (pr > tail[j]) tail[j] = pr;
            pr *= fabs(1.0 - tau[order[j]] * x);
        }
    }
    double b = 0.0;
    for (int j = 0; j < n; ++j) b += head[j] * tail[j];
    free(head); free(tail);
    return b;
}

int ko_fed_order(int n, const double* tau, int* order)
{
    if (n <= 0) return 0;
    int* cand = (int*)malloc(sizeof(int) * (size_t)n);
    double best = -1.0;
    int bk = 1;
    for (int kappa = 1; kappa <= n; ++kappa) {
        kappa_cycle(n, kappa, cand);
        const double b = order_amplification(n, tau, cand);
        if (best < 0.0 || b < best) {
            best = b;
            bk = kappa;
        }
    }
    kappa_cycle(n, bk, order);
    free(cand);
    return bk;
}

/* F4: explicit step of div(g grad L) in the flux form of the AOS operator. */
void ko_fed_step(const double* L, const double* g, int W, int H, double tau, double* out)
{
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            const size_t p = (size_t)y * W + x;
            double flux = 0.0;
            if (x > 0) flux += 0.5 * (g[p] + g[p - 1]) * (L[p - 1] - L[p]);
            if (x < W - 1) flux += 0.5 * (g[p] + g[p + 1]) * (L[p + 1] - L[p]);
            if (y > 0) flux += 0.5 * (g[p] + g[p - W]) * (L[p - W] - L[p]);
            if (y < H - 1) flux += 0.5 * (g[p] + g[p + W]) * (L[p + W] - L[p]);
            out[p] = L[p] + tau * flux;
        }
}

int ko_fed_evolve(const double* L, const double* g, int W, int H, double dt, double tau_max,
                  double* out)
{
    size_t P = (size_t)W * H;
    int n = ko_fed_tau(dt, tau_max, NULL, 0);
    double* tau = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    ko_fed_tau(dt, tau_max, tau, n);
    int* order = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    ko_fed_order(n, tau, order);
    double* a = (double*)malloc(sizeof(double) * P);
    double* b = (double*)malloc(sizeof(double) * P);
    memcpy(a, L, sizeof(double) * P);
    for (int j = 0; j < n; ++j) {
        ko_fed_step(a, g, W, H, tau[order[j]], b);
        double* t = a;
        a = b;
        b = t;
    }
    memcpy(out, a, sizeof(double) * P);
    free(a); free(b); free(tau); free(order);
    return n;
}

/* Sec. II-A / III-1: presmoothing with sigma0, k from the base image, then
 * one AOS step (or one FED cycle) per level with tau_i = t_i - t_{i-1}
 * (Eq. 7). */
int ko_build_scale_space(const double* img, int W, int H, const ko_options* opt,
                         double* levels, double* k_used)
{
    int N = opt->octaves * opt->sublevels;
    if (N < 1 || W < 1 || H < 1) return -1;
    size_t P = (size_t)W * H;
    double* sigma = (double*)malloc(sizeof(double) * (size_t)N);
    double* t = (double*)malloc(sizeof(double) * (size_t)N);
    double* g = (double*)malloc(sizeof(double) * P);
    ko_scale_table(opt->octaves, opt->sublevels, opt->sigma0, sigma, t);

    ko_gaussian(img, levels, W, H, opt->sigma0);               /* L_0 */
    double k = opt->k_override > 0.0
                   ? opt->k_override
                   : ko_contrast_k(levels, W, H, opt->sigma_d, opt->k_percentile,
                                   opt->nbins, NULL, NULL, NULL);
    if (k_used) *k_used = k;

    for (int i = 1; i < N; ++i) {
        const double* Lp = levels + (size_t)(i - 1) * P;
        double* Li = levels + (size_t)i * P;
        ko_conductance(Lp, W, H, opt->sigma_d, k, opt->diffusivity, g);
        if (opt->scheme == KO_SCHEME_FED)
            ko_fed_evolve(Lp, g, W, H, t[i] - t[i - 1], opt->fed_tau_max, Li);
        else
            ko_aos_step(Lp, g, W, H, t[i] - t[i - 1], NULL, NULL, Li);
    }
    free(sigma); free(t); free(g);
    return 0;
}

/* R6: derivative step, rounded half away from zero, at least 1. */
int ko_step_size(double sigma)
{
    int s = (int)floor(sigma + 0.5);
    return s < 1 ? 1 : s;
}

/* Second derivatives as the concatenation of two step-s Scharr operators
 * (Sec. II-B, Sec. III-2), applied to the symmetrically extended level:
 *   D_x = [-1 0 1]/(2s) along x (taps at -s, 0, s) times [3 10 3]/16 along y,
 *   D_y = the transpose,
 *   Lxx = D_x D_x, Lyy = D_y D_y, Lxy = D_x D_y.
 * The composed taps lie on the lattice {-2s, -s, 0, s, 2s}^2. */
void ko_hessian(const double* L, int W, int H, int s,
                double* Lxx, double* Lyy, double* Lxy)
{
    /* 1-D factors of the first derivatives, taps at -s, 0, s. */
    const double dif[3] = {-1.0 / (2.0 * s), 0.0, 1.0 / (2.0 * s)};
    const double smo[3] = {3.0 / 16.0, 10.0 / 16.0, 3.0 / 16.0};
    /* Compose two 3-tap factors into a 5-tap one (taps -2s .. 2s). */
    double dd[5] = {0}, ss[5] = {0}, ds[5] = {0};
    for (int p = 0; p < 3; ++p)
        for (int q = 0; q < 3; ++q) {
            dd[p + q] += dif[p] * dif[q];
            ss[p + q] += smo[p] * smo[q];
            ds[p + q] += dif[p] * smo[q];
        }
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            double xx = 0.0, yy = 0.0, xy = 0.0;
            for (int v = -2; v <= 2; ++v)
                for (int u = -2; u <= 2; ++u) {
                    double l = at(L, W, H, x + (long)u * s, y + (long)v * s);
                    xx += dd[u + 2] * ss[v + 2] * l;
                    yy += ss[u + 2] * dd[v + 2] * l;
                    xy += ds[u + 2] * ds[v + 2] * l;
                }
            size_t p = (size_t)y * W + x;
            Lxx[p] = xx;
            Lyy[p] = yy;
            Lxy[p] = xy;
        }
}

/* Eq. 8 (reading R6): normalised determinant of the Hessian. */
void ko_doh(const double* L, int W, int H, double sigma_i, int octave,
            int doh_norm, double* D)
{
    size_t P = (size_t)W * H;
    int s = ko_step_size(sigma_i);
    double* xx = (double*)malloc(sizeof(double) * P);
    double* yy = (double*)malloc(sizeof(double) * P);
    double* xy = (double*)malloc(sizeof(double) * P);
    ko_hessian(L, W, H, s, xx, yy, xy);
    double norm;
    if (doh_norm == KO_DOH_PAPER_LITERAL) {
        double kn = sigma_i / pow(2.0, (double)octave);
        norm = kn * kn;
    } else {
        norm = (double)s * s * s * s;
    }
#pragma omp parallel for schedule(static)
    for (size_t p = 0; p < P; ++p) D[p] = norm * (xx[p] * yy[p] - xy[p] * xy[p]);
    free(xx); free(yy); free(xy);
}

/* Sec. II-B and Sec. III-2 (readings R7, R8, R9, W1). */
int ko_find_extrema(const double* D, int W, int H, int N, int S,
                    const double* sigma, double dthreshold, double edge_r,
                    int window, ko_keypoint* out, int cap)
{
    size_t P = (size_t)W * H;
    int count = 0;
    for (int i = 1; i <= N - 2; ++i) {
        const double* Dc = D + (size_t)i * P;
        int r = 1;
        if (window == KO_EXTREMA_SIGMA_WINDOW) {
            r = ko_step_size(sigma[i]) / 2;
            if (r < 1) r = 1;
        }
        for (int y = 1; y <= H - 2; ++y)
            for (int x = 1; x <= W - 2; ++x) {
                double v = Dc[(size_t)y * W + x];
                if (!(v > dthreshold)) continue;
                int is_max = 1;
                /* the 8 neighbours on the level itself */
                for (int dy = -1; dy <= 1 && is_max; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        if (dx == 0 && dy == 0) continue;
                        if (!(v > Dc[(size_t)(y + dy) * W + (x + dx)])) {
                            is_max = 0;
                            break;
                        }
                    }
                /* the window directly below and above */
                for (int l = i - 1; l <= i + 1 && is_max; l += 2)
                    for (int dy = -r; dy <= r && is_max; ++dy)
                        for (int dx = -r; dx <= r; ++dx) {
                            int xx = x + dx, yy = y + dy;
                            if (xx < 0 || xx >= W || yy < 0 || yy >= H) continue;
                            if (!(v > D[(size_t)l * P + (size_t)yy * W + xx])) {
                                is_max = 0;
                                break;
                            }
                        }
                if (!is_max) continue;

                /* Hessian and gradient of the response on its 3x3 patch. */
#define DV(ox, oy) Dc[(size_t)(y + (oy)) * W + (x + (ox))]
                double gx = 0.5 * (DV(1, 0) - DV(-1, 0));
                double gy = 0.5 * (DV(0, 1) - DV(0, -1));
                double hxx = DV(1, 0) - 2.0 * v + DV(-1, 0);
                double hyy = DV(0, 1) - 2.0 * v + DV(0, -1);
                double hxy = 0.25 * (DV(1, 1) - DV(-1, 1) - DV(1, -1) + DV(-1, -1));
#undef DV
                double det = hxx * hyy - hxy * hxy;
                double tr = hxx + hyy;
                /* Eq. 12 edge test: keep only Tr^2/Det < (r+1)^2/r, Det > 0. */
                if (edge_r > 0.0) {
                    if (!(det > 0.0)) continue;
                    if (!(tr * tr * edge_r < (edge_r + 1.0) * (edge_r + 1.0) * det)) continue;
                }
                /* Quadratic fit: offset = -H^-1 grad. */
                if (det == 0.0) continue;
                double ox = -(hyy * gx - hxy * gy) / det;
                double oy = -(hxx * gy - hxy * gx) / det;
                if (fabs(ox) > 1.0 || fabs(oy) > 1.0) continue;

                if (count < cap && out) {
                    ko_keypoint* k = &out[count];
                    k->x = x + ox;
                    k->y = y + oy;
                    k->sigma = sigma[i];
                    k->response = v;
                    k->level = i;
                    k->octave = i / S;
                    k->sublevel = i % S;
                    k->ix = x;
                    k->iy = y;
                }
                count += 1;
            }
    }
    return count;
}
