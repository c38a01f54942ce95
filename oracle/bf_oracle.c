/*
 * FP64 CPU oracle for the trigonometric O(1) bilateral filter
 * (Chaudhury, Sage, Unser, "Fast O(1) bilateral filtering using trigonometric
 * range kernels").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file: only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no code, header, table or constant
 * with the CUDA library; the two meet only through seeded synthetic inputs.
 *
 * Everything here is written out from the paper's definitions, slowly and in
 * double precision:
 *   - or_bf_brute*     : the bilateral filter in its unbiased form,
 *                        eq. (BF) and eq. (normalization), summed directly
 *                        over the support of the spatial kernel;
 *   - or_bf_trig       : Algorithm 1, steps 3-5, with the N+1 complex
 *                        auxiliary images of the raised-cosine expansion
 *                        (Section 2.3) and eq. (final-form);
 *   - or_bf_grad       : the exact derivative of eq. (BF) with respect to
 *                        every input pixel and to sigma_r (not in the paper;
 *                        the chain rule applied to the definition);
 *   - or_bf_fd_grad_f  : central finite differences of or_bf_brute for the
 *                        same gradient;
 *   - or_rg_* / or_bf_trig_rg : the recursive O(1) Gaussian of Young and van
 *                        Vliet (the spatial filter of the paper's experiments,
 *                        Section 3) and Algorithm 1 with it as the averaging
 *                        of step 4; or_rg_matrix, the same line filter as a
 *                        matrix, and or_bf_brute_mat / or_bf_grad_mat, the
 *                        filter and its exact gradient with explicit per-axis
 *                        weight matrices;
 *   - or_bf_brute_sv   : the space-variant extension (Section 4): at each
 *                        pixel its own box (or, or_bf_brute_sv_shape, hat)
 *                        of half-width r(x), eq. (BF) summed directly over it;
 *   - or_bf_*_cos      : the same filter, gradient and differences for a
 *                        general trigonometric range kernel of Section 2.2,
 *                        phi(s) = a_0 + a_1 cos(gamma s) + ... + a_N cos(N gamma s),
 *                        evaluated term by term as written.
 *
 * Readings of the paper used here (each one also listed in the design notes):
 *   - Degree rule (Algorithm 1 step 2, Table 1 last row):
 *       N = max(1, ceil((gamma*sigma_r)^-2)), gamma = pi/(2T).
 *   - Range kernel (Algorithm 1 step 3 with rho = gamma*sigma_r):
 *       phi(s) = cos(gamma*s/(rho*sqrt(N)))^N = cos(s/(sigma_r*sqrt(N)))^N,
 *     evaluated directly as a power, never through its expansion.
 *     Mode 1 is the Gaussian exp(-s^2/(2 sigma_r^2)) that eq. (convergence1)
 *     approximates.
 *   - Boundary: the paper integrates over Omega and is silent about image
 *     borders; the image is extended by clamping each coordinate to the
 *     nearest edge pixel.
 *   - Spatial kernels: a truncated Gaussian normalised over [-R, R]
 *     (the experiments use the support [-3 sigma, 3 sigma]), or an iterated
 *     box b*b*...*b with b = 1/(2r+1) on [-r, r].  Both are separable
 *     w(y1, y2) = w1(y1) w1(y2) and have unit mass (eq. (averaging)).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <complex.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846

static int or_clamp(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Degree rule: Algorithm 1 step 2 ("set N = (gamma sigma_r)^-2"), rounded up
 * as in the last row of Table 1.  A relative guard of 1e-12 keeps a value that
 * is an integer in exact arithmetic from being pushed up by rounding. */
int or_n_rule(double sigma_r, double T)
{
    double gamma = OR_PI / (2.0 * T);
    double x = 1.0 / ((gamma * sigma_r) * (gamma * sigma_r));
    double n = ceil(x * (1.0 - 1e-12));
    if (n < 1.0) n = 1.0;
    if (n > 1e7) n = 1e7;
    return (int)n;
}

/* One-dimensional spatial weights w1[0 .. 2R] (index k <-> offset k - R).
 * kind 0: truncated Gaussian exp(-i^2 / (2 sigma_s^2)) on |i| <= R,
 *         R = radius_override > 0 ? radius_override : ceil(3 sigma_s),
 *         normalised to unit sum.
 * kind 1: iterated box, `passes` boxes of half-width r
 *         (r = radius_override > 0 ? radius_override : the r whose
 *          variance passes*((2r+1)^2-1)/12 is closest to sigma_s^2),
 *         built as exact integer counts divided by (2r+1)^passes.
 * Returns R (support half-width), or -1 when cap is too small. */
int or_spatial_w1(int kind, double sigma_s, int radius_override, int passes,
                  double *w1, int cap)
{
    if (kind == 0) {
        int R = radius_override > 0 ? radius_override : (int)ceil(3.0 * sigma_s);
        if (R < 0) R = 0;
        if (2 * R + 1 > cap) return -1;
        double s = 0.0;
        for (int i = -R; i <= R; i++) {
            double v = exp(-(double)i * i / (2.0 * sigma_s * sigma_s));
            w1[i + R] = v;
            s += v;
        }
        for (int k = 0; k <= 2 * R; k++) w1[k] /= s;
        return R;
    } else {
        if (passes <= 0) passes = 3;
        int r = radius_override;
        if (r <= 0) {
            double L = sqrt(12.0 * sigma_s * sigma_s / passes + 1.0);
            r = (int)floor((L - 1.0) / 2.0 + 0.5);
            if (r < 1) r = 1;
        }
        int R = passes * r;
        if (2 * R + 1 > cap) return -1;
        /* counts[k] = number of ways offsets of `passes` boxes sum to k - R */
        double *cnt = (double *)calloc((size_t)(2 * R + 1), sizeof(double));
        double *tmp = (double *)calloc((size_t)(2 * R + 1), sizeof(double));
        int cur = 0; /* current half-width */
        cnt[R] = 1.0;
        for (int p = 0; p < passes; p++) {
            memset(tmp, 0, sizeof(double) * (size_t)(2 * R + 1));
            for (int k = -cur; k <= cur; k++)
                for (int d = -r; d <= r; d++) tmp[k + d + R] += cnt[k + R];
            memcpy(cnt, tmp, sizeof(double) * (size_t)(2 * R + 1));
            cur += r;
        }
        double denom = pow(2.0 * r + 1.0, passes);
        for (int k = 0; k <= 2 * R; k++) w1[k] = cnt[k] / denom;
        free(cnt);
        free(tmp);
        return R;
    }
}

/* Range kernel and its derivatives.  mode 0: raised cosine of degree N with
 * k = 1/(sigma_r sqrt N); mode 1: Gaussian of standard deviation sigma_r;
 * mode 2: the cosine polynomial sum_{n=0..N} a[n] cos(n gamma s) of
 * Section 2.2 (a has N+1 entries). */
typedef struct {
    int mode; int N; double k; double sigma_r;
    const double *a; double gamma;
} or_range;

static or_range or_make_range(int mode, double sigma_r, int N)
{
    or_range r;
    r.mode = mode;
    r.N = N < 1 ? 1 : N;
    r.sigma_r = sigma_r;
    r.k = 1.0 / (sigma_r * sqrt((double)r.N));
    r.a = NULL;
    r.gamma = 0.0;
    return r;
}

static or_range or_make_cos_range(double gamma, const double *a, int n_coef)
{
    or_range r;
    r.mode = 2;
    r.N = n_coef - 1;
    r.sigma_r = 0.0;
    r.k = 0.0;
    r.a = a;
    r.gamma = gamma;
    return r;
}

static double or_phi(const or_range *r, double s)
{
    if (r->mode == 1) return exp(-s * s / (2.0 * r->sigma_r * r->sigma_r));
    if (r->mode == 2) {
        double v = 0.0;
        for (int n = 0; n <= r->N; n++) v += r->a[n] * cos((double)n * r->gamma * s);
        return v;
    }
    return pow(cos(r->k * s), r->N);
}

/* d phi / d s */
static double or_dphi(const or_range *r, double s)
{
    if (r->mode == 1) return -s / (r->sigma_r * r->sigma_r) * or_phi(r, s);
    if (r->mode == 2) {
        double v = 0.0;
        for (int n = 1; n <= r->N; n++)
            v -= r->a[n] * (double)n * r->gamma * sin((double)n * r->gamma * s);
        return v;
    }
    double c = cos(r->k * s);
    double cn1 = r->N == 1 ? 1.0 : pow(c, r->N - 1);
    return -(double)r->N * r->k * cn1 * sin(r->k * s);
}

/* d phi / d sigma_r at fixed N (N is piecewise constant in sigma_r). */
static double or_dphi_dsigma(const or_range *r, double s)
{
    return -(s / r->sigma_r) * or_dphi(r, s);
}

/* eq. (BF) and eq. (normalization) at one pixel (i, j) of an H x W image. */
static void or_pq_at(const double *f, int H, int W, const double *w1, int R,
                     const or_range *rg, int i, int j, double *P, double *Q)
{
    double fx = f[(size_t)i * W + j];
    double p = 0.0, q = 0.0;
    for (int a = -R; a <= R; a++) {
        int zi = or_clamp(i - a, 0, H - 1);
        for (int b = -R; b <= R; b++) {
            int zj = or_clamp(j - b, 0, W - 1);
            double wt = w1[a + R] * w1[b + R];
            double v = f[(size_t)zi * W + zj];
            double ph = or_phi(rg, v - fx);
            p += wt * ph * v;
            q += wt * ph;
        }
    }
    *P = p;
    *Q = q;
}

static void or_brute_rg(const double *f, int H, int W, const double *w1, int R,
                        const or_range *rg, double *out, double *q_out)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int i = 0; i < H; i++) {
        for (int j = 0; j < W; j++) {
            double P, Q;
            or_pq_at(f, H, W, w1, R, rg, i, j, &P, &Q);
            out[(size_t)i * W + j] = P / Q;
            if (q_out) q_out[(size_t)i * W + j] = Q;
        }
    }
}

static void or_brute_at_rg(const double *f, int H, int W, const double *w1, int R,
                           const or_range *rg, const long long *idx, long long n_idx,
                           double *out, double *q_out)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (long long t = 0; t < n_idx; t++) {
        int i = (int)(idx[t] / W), j = (int)(idx[t] % W);
        double P, Q;
        or_pq_at(f, H, W, w1, R, rg, i, j, &P, &Q);
        out[t] = P / Q;
        if (q_out) q_out[t] = Q;
    }
}

/* Brute-force filter of a whole single-channel image.  q_out may be NULL. */
void or_bf_brute(const double *f, int H, int W, const double *w1, int R,
                 int mode, double sigma_r, int N, double *out, double *q_out)
{
    or_range rg = or_make_range(mode, sigma_r, N);
    or_brute_rg(f, H, W, w1, R, &rg, out, q_out);
}

/* Space-variant extension (Section 4): the spatial kernel at pixel (i, j) is
 * centred there with half-width r = radius[i * W + j] clamped into
 * [0, r_max]: the (2 r + 1) x (2 r + 1) box (hat = 0), or the separable hat
 * (hat = 1), weight (r + 1 - |a|) (r + 1 - |b|) at offset (a, b).  The
 * kernel's total weight cancels in the ratio, so eq. (BF) is summed directly
 * with these weights over the clamp-extended image.  q_out (may be NULL)
 * receives the normaliser with unit-mass weights. */
static void or_sv_at(const double *f, int H, int W, const int *radius, int r_max, int hat,
                     const or_range *rg, int i, int j, double *out, double *q_out)
{
    int r = or_clamp(radius[(size_t)i * W + j], 0, r_max);
    double fx = f[(size_t)i * W + j];
    double p = 0.0, q = 0.0, mass = 0.0;
    for (int a = -r; a <= r; a++) {
        int zi = or_clamp(i + a, 0, H - 1);
        double wa = hat ? (double)(r + 1 - abs(a)) : 1.0;
        for (int b = -r; b <= r; b++) {
            int zj = or_clamp(j + b, 0, W - 1);
            double w = wa * (hat ? (double)(r + 1 - abs(b)) : 1.0);
            double v = f[(size_t)zi * W + zj];
            double ph = w * or_phi(rg, v - fx);
            p += ph * v;
            q += ph;
            mass += w;
        }
    }
    *out = p / q;
    if (q_out) *q_out = q / mass;
}

void or_bf_brute_sv(const double *f, int H, int W, const int *radius, int r_max, int mode,
                    double sigma_r, int N, double *out, double *q_out)
{
    or_range rg = or_make_range(mode, sigma_r, N);
#pragma omp parallel for schedule(dynamic, 4)
    for (int i = 0; i < H; i++)
        for (int j = 0; j < W; j++)
            or_sv_at(f, H, W, radius, r_max, 0, &rg, i, j, out + (size_t)i * W + j,
                     q_out ? q_out + (size_t)i * W + j : NULL);
}

/* The space-variant filter with the hat (hat = 1) or the box (hat = 0). */
void or_bf_brute_sv_shape(const double *f, int H, int W, const int *radius, int r_max, int hat,
                          int mode, double sigma_r, int N, double *out, double *q_out)
{
    or_range rg = or_make_range(mode, sigma_r, N);
#pragma omp parallel for schedule(dynamic, 4)
    for (int i = 0; i < H; i++)
        for (int j = 0; j < W; j++)
            or_sv_at(f, H, W, radius, r_max, hat, &rg, i, j, out + (size_t)i * W + j,
                     q_out ? q_out + (size_t)i * W + j : NULL);
}

/* The space-variant filter with a general cosine kernel (Section 2.2),
 * phi(s) = sum_n a[n] cos(n gamma s), evaluated term by term. */
void or_bf_brute_sv_cos(const double *f, int H, int W, const int *radius, int r_max,
                        double gamma, const double *a, int n_coef, double *out)
{
    or_range rg = or_make_cos_range(gamma, a, n_coef);
#pragma omp parallel for schedule(dynamic, 4)
    for (int i = 0; i < H; i++)
        for (int j = 0; j < W; j++)
            or_sv_at(f, H, W, radius, r_max, 0, &rg, i, j, out + (size_t)i * W + j, NULL);
}

/* The space-variant filter at a list of flat pixel indices only. */
void or_bf_brute_sv_at(const double *f, int H, int W, const int *radius, int r_max, int mode,
                       double sigma_r, int N, const long long *idx, long long n_idx,
                       double *out)
{
    or_range rg = or_make_range(mode, sigma_r, N);
#pragma omp parallel for schedule(dynamic, 16)
    for (long long t = 0; t < n_idx; t++)
        or_sv_at(f, H, W, radius, r_max, 0, &rg, (int)(idx[t] / W), (int)(idx[t] % W), out + t,
                 NULL);
}

/* The same at a list of flat pixel indices, box (hat = 0) or hat (hat = 1). */
void or_bf_brute_sv_shape_at(const double *f, int H, int W, const int *radius, int r_max,
                             int hat, int mode, double sigma_r, int N, const long long *idx,
                             long long n_idx, double *out)
{
    or_range rg = or_make_range(mode, sigma_r, N);
#pragma omp parallel for schedule(dynamic, 16)
    for (long long t = 0; t < n_idx; t++)
        or_sv_at(f, H, W, radius, r_max, hat, &rg, (int)(idx[t] / W), (int)(idx[t] % W),
                 out + t, NULL);
}

/* Brute-force filter at a list of flat pixel indices only. */
void or_bf_brute_at(const double *f, int H, int W, const double *w1, int R,
                    int mode, double sigma_r, int N, const long long *idx,
                    long long n_idx, double *out, double *q_out)
{
    or_range rg = or_make_range(mode, sigma_r, N);
    or_brute_at_rg(f, H, W, w1, R, &rg, idx, n_idx, out, q_out);
}

/* The same two with the cosine polynomial of Section 2.2,
 * phi(s) = sum_{n=0..n_coef-1} a[n] cos(n gamma s). */
void or_bf_brute_cos(const double *f, int H, int W, const double *w1, int R,
                     double gamma, const double *a, int n_coef, double *out, double *q_out)
{
    or_range rg = or_make_cos_range(gamma, a, n_coef);
    or_brute_rg(f, H, W, w1, R, &rg, out, q_out);
}

void or_bf_brute_cos_at(const double *f, int H, int W, const double *w1, int R,
                        double gamma, const double *a, int n_coef, const long long *idx,
                        long long n_idx, double *out, double *q_out)
{
    or_range rg = or_make_cos_range(gamma, a, n_coef);
    or_brute_at_rg(f, H, W, w1, R, &rg, idx, n_idx, out, q_out);
}

/* Separable filtering of a complex image with clamp-to-edge extension:
 * y(i,j) = sum_a sum_b w1(a) w1(b) x(clamp(i-a), clamp(j-b)). */
static void or_filter_c(const double complex *x, int H, int W, const double *w1,
                        int R, double complex *tmp, double complex *y)
{
#pragma omp parallel for schedule(static)
    for (int i = 0; i < H; i++)
        for (int j = 0; j < W; j++) {
            double complex s = 0.0;
            for (int b = -R; b <= R; b++)
                s += w1[b + R] * x[(size_t)i * W + or_clamp(j - b, 0, W - 1)];
            tmp[(size_t)i * W + j] = s;
        }
#pragma omp parallel for schedule(static)
    for (int i = 0; i < H; i++)
        for (int j = 0; j < W; j++) {
            double complex s = 0.0;
            for (int a = -R; a <= R; a++)
                s += w1[a + R] * tmp[(size_t)or_clamp(i - a, 0, H - 1) * W + j];
            y[(size_t)i * W + j] = s;
        }
}

/* Algorithm 1, steps 1-5, in the paper's complex notation:
 *   gamma = pi/(2T), rho = gamma sigma_r                          (step 1)
 *   h_n = exp(j gamma (2n-N) f / (rho sqrt N)), g_n = f h_n,
 *   d_n = 2^-N C(N,n) exp(-j gamma (2n-N) f / (rho sqrt N))       (step 3)
 *   filter h_n and g_n with the spatial kernel                    (step 4)
 *   out = sum_n d_n gbar_n / sum_n d_n hbar_n                      (step 5)
 * The degree N is passed in (the caller applies the rule of step 2).
 * Returns the largest |Im| / |Re| of numerator and denominator seen. */
double or_bf_trig(const double *f, int H, int W, const double *w1, int R,
                  double sigma_r, double T, int N, double *out, double *q_out)
{
    size_t n = (size_t)H * W;
    double gamma = OR_PI / (2.0 * T);
    double rho = gamma * sigma_r;
    double complex *h = (double complex *)malloc(n * sizeof(double complex));
    double complex *g = (double complex *)malloc(n * sizeof(double complex));
    double complex *hb = (double complex *)malloc(n * sizeof(double complex));
    double complex *gb = (double complex *)malloc(n * sizeof(double complex));
    double complex *tmp = (double complex *)malloc(n * sizeof(double complex));
    double complex *num = (double complex *)calloc(n, sizeof(double complex));
    double complex *den = (double complex *)calloc(n, sizeof(double complex));
    for (int k = 0; k <= N; k++) {
        /* 2^-N C(N,k), through log-gamma to stay finite for large N */
        double cn = exp(lgamma(N + 1.0) - lgamma(k + 1.0) - lgamma(N - k + 1.0) -
                        N * log(2.0));
        double freq = gamma * (double)(2 * k - N) / (rho * sqrt((double)N));
        for (size_t p = 0; p < n; p++) {
            h[p] = cexp(I * freq * f[p]);
            g[p] = f[p] * h[p];
        }
        or_filter_c(h, H, W, w1, R, tmp, hb);
        or_filter_c(g, H, W, w1, R, tmp, gb);
        for (size_t p = 0; p < n; p++) {
            double complex d = cn * cexp(-I * freq * f[p]);
            num[p] += d * gb[p];
            den[p] += d * hb[p];
        }
    }
    double worst = 0.0;
    for (size_t p = 0; p < n; p++) {
        out[p] = creal(num[p]) / creal(den[p]);
        if (q_out) q_out[p] = creal(den[p]);
        double e1 = fabs(cimag(num[p])) / (fabs(creal(num[p])) + 1e-300);
        double e2 = fabs(cimag(den[p])) / (fabs(creal(den[p])) + 1e-300);
        if (e1 > worst) worst = e1;
        if (e2 > worst) worst = e2;
    }
    free(h); free(g); free(hb); free(gb); free(tmp); free(num); free(den);
    return worst;
}

/* Exact gradient of L = sum_x u(x) out(x) with respect to every pixel of f
 * and to sigma_r (N held fixed).  Chain rule on eq. (BF):
 *   dL/df(p) = sum_x alpha(x) [ dP(x)/df(p) - out(x) dQ(x)/df(p) ],
 *   alpha = u / Q,
 * where each neighbour z of x contributes through its clamped pixel
 * clamp(z) (value and range-kernel argument) and through x itself (the
 * argument f(z) - f(x)). */
static void or_grad_rg(const double *f, const double *u, int H, int W, const double *w1,
                       int R, const or_range *rgp, double *grad_f, double *grad_sigma_r)
{
    const or_range rg = *rgp;
    size_t n = (size_t)H * W;
    int nt = or_num_threads();
    double *buf = (double *)calloc(n * (size_t)nt, sizeof(double));
    double *gs = (double *)calloc((size_t)nt, sizeof(double));
#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *g = buf + n * (size_t)tid;
        double gsl = 0.0;
#pragma omp for schedule(dynamic, 4)
        for (int i = 0; i < H; i++) {
            for (int j = 0; j < W; j++) {
                double P, Q;
                or_pq_at(f, H, W, w1, R, &rg, i, j, &P, &Q);
                double o = P / Q;
                double alpha = u[(size_t)i * W + j] / Q;
                double fx = f[(size_t)i * W + j];
                for (int a = -R; a <= R; a++) {
                    int zi = or_clamp(i - a, 0, H - 1);
                    for (int b = -R; b <= R; b++) {
                        int zj = or_clamp(j - b, 0, W - 1);
                        double wt = w1[a + R] * w1[b + R];
                        double v = f[(size_t)zi * W + zj];
                        double s = v - fx;
                        double ph = or_phi(&rg, s);
                        double dph = or_dphi(&rg, s);
                        g[(size_t)zi * W + zj] += alpha * wt * (ph + dph * (v - o));
                        g[(size_t)i * W + j] -= alpha * wt * dph * (v - o);
                        if (grad_sigma_r) gsl += alpha * wt * or_dphi_dsigma(&rg, s) * (v - o);
                    }
                }
            }
        }
        gs[tid] = gsl;
    }
    for (size_t p = 0; p < n; p++) {
        double s = 0.0;
        for (int t = 0; t < nt; t++) s += buf[n * (size_t)t + p];
        grad_f[p] = s;
    }
    double s = 0.0;
    for (int t = 0; t < nt; t++) s += gs[t];
    if (grad_sigma_r) *grad_sigma_r = s;
    free(buf);
    free(gs);
}

void or_bf_grad(const double *f, const double *u, int H, int W, const double *w1,
                int R, int mode, double sigma_r, int N, double *grad_f,
                double *grad_sigma_r)
{
    or_range rg = or_make_range(mode, sigma_r, N);
    or_grad_rg(f, u, H, W, w1, R, &rg, grad_f, grad_sigma_r);
}

/* Image gradient for the cosine polynomial of Section 2.2 (no sigma_r). */
void or_bf_grad_cos(const double *f, const double *u, int H, int W, const double *w1,
                    int R, double gamma, const double *a, int n_coef, double *grad_f)
{
    or_range rg = or_make_cos_range(gamma, a, n_coef);
    or_grad_rg(f, u, H, W, w1, R, &rg, grad_f, NULL);
}

/* Central finite differences of L = sum_x u(x) out(x) with respect to the
 * listed pixels.  Only outputs within R of the perturbed pixel change, so only
 * those are recomputed (with clamping, a neighbour that maps onto p lies
 * within R of every output that sees it). */
static void or_fd_rg(const double *f, const double *u, int H, int W,
                     const double *w1, int R, const or_range *rgp,
                     const long long *idx, long long n_idx, double h, double *out)
{
    const or_range rg = *rgp;
    size_t n = (size_t)H * W;
#pragma omp parallel
    {
        double *fl = (double *)malloc(n * sizeof(double));
        memcpy(fl, f, n * sizeof(double));
#pragma omp for schedule(dynamic, 1)
        for (long long t = 0; t < n_idx; t++) {
            int pi = (int)(idx[t] / W), pj = (int)(idx[t] % W);
            int i0 = pi - R < 0 ? 0 : pi - R, i1 = pi + R > H - 1 ? H - 1 : pi + R;
            int j0 = pj - R < 0 ? 0 : pj - R, j1 = pj + R > W - 1 ? W - 1 : pj + R;
            double orig = fl[idx[t]];
            double L[2];
            for (int sgn = 0; sgn < 2; sgn++) {
                fl[idx[t]] = orig + (sgn == 0 ? h : -h);
                double acc = 0.0;
                for (int i = i0; i <= i1; i++)
                    for (int j = j0; j <= j1; j++) {
                        double P, Q;
                        or_pq_at(fl, H, W, w1, R, &rg, i, j, &P, &Q);
                        acc += u[(size_t)i * W + j] * (P / Q);
                    }
                L[sgn] = acc;
            }
            fl[idx[t]] = orig;
            out[t] = (L[0] - L[1]) / (2.0 * h);
        }
        free(fl);
    }
}

void or_bf_fd_grad_f(const double *f, const double *u, int H, int W,
                     const double *w1, int R, int mode, double sigma_r, int N,
                     const long long *idx, long long n_idx, double h, double *out)
{
    or_range rg = or_make_range(mode, sigma_r, N);
    or_fd_rg(f, u, H, W, w1, R, &rg, idx, n_idx, h, out);
}

void or_bf_fd_grad_f_cos(const double *f, const double *u, int H, int W,
                         const double *w1, int R, double gamma, const double *a, int n_coef,
                         const long long *idx, long long n_idx, double h, double *out)
{
    or_range rg = or_make_cos_range(gamma, a, n_coef);
    or_fd_rg(f, u, H, W, w1, R, &rg, idx, n_idx, h, out);
}

/* L = sum_x u(x) out(x) for the whole image (used for sigma_r differences). */
double or_bf_loss(const double *f, const double *u, int H, int W, const double *w1,
                  int R, int mode, double sigma_r, int N)
{
    or_range rg = or_make_range(mode, sigma_r, N);
    double total = 0.0;
#pragma omp parallel for reduction(+ : total) schedule(dynamic, 4)
    for (int i = 0; i < H; i++)
        for (int j = 0; j < W; j++) {
            double P, Q;
            or_pq_at(f, H, W, w1, R, &rg, i, j, &P, &Q);
            total += u[(size_t)i * W + j] * (P / Q);
        }
    return total;
}

/* The cosine polynomial itself. */
void or_phi_cos_table(double gamma, const double *a, int n_coef, const double *s, long long n,
                      double *out)
{
    or_range rg = or_make_cos_range(gamma, a, n_coef);
    for (long long t = 0; t < n; t++) out[t] = or_phi(&rg, s[t]);
}

/* The range kernel itself, for tests of the convergence claim. */
void or_phi_table(int mode, double sigma_r, int N, const double *s, long long n,
                  double *out)
{
    or_range rg = or_make_range(mode, sigma_r, N);
    for (long long t = 0; t < n; t++) out[t] = or_phi(&rg, s[t]);
}


/* ------------------------------------------------------------------------
 * Recursive Gaussian (Young and van Vliet, "Recursive implementation of the
 * Gaussian filter", Signal Processing 44, 1995): a causal and an anticausal
 * third-order recursion whose cascade approximates a Gaussian of standard
 * deviation sigma (valid for sigma >= 0.5).  Published design:
 *   q  = 0.98711 sigma - 0.96330                    (sigma >= 2.5)
 *   q  = 3.97156 - 4.14554 sqrt(1 - 0.26891 sigma)  (0.5 <= sigma < 2.5)
 *   b0 = 1.57825 + 2.44413 q + 1.4281 q^2 + 0.422205 q^3
 *   b1 = 2.44413 q + 2.85619 q^2 + 1.26661 q^3
 *   b2 = -(1.4281 q^2 + 1.26661 q^3)
 *   b3 = 0.422205 q^3
 *   B  = 1 - (b1 + b2 + b3) / b0
 *   causal:     w[n] = B x[n] + (b1 w[n-1] + b2 w[n-2] + b3 w[n-3]) / b0
 *   anticausal: y[n] = B w[n] + (b1 y[n+1] + b2 y[n+2] + b3 y[n+3]) / b0
 * Boundary (the image extended by clamping, as everywhere here): the causal
 * pass starts from its steady state for the constant x[0] (exact for a
 * constant extension, the recursion having unit gain at DC); it then runs P
 * further samples into the constant extension x[n-1], and the anticausal pass
 * starts there from its steady state w[n-1+P].  P = ceil(6 sigma).
 * coef[] = { B, b1/b0, b2/b0, b3/b0 }.  Returns P. */
int or_rg_coefs(double sigma, double *coef)
{
    double q = sigma >= 2.5 ? 0.98711 * sigma - 0.96330
                            : 3.97156 - 4.14554 * sqrt(1.0 - 0.26891 * sigma);
    double b0 = 1.57825 + 2.44413 * q + 1.4281 * q * q + 0.422205 * q * q * q;
    double b1 = 2.44413 * q + 2.85619 * q * q + 1.26661 * q * q * q;
    double b2 = -(1.4281 * q * q + 1.26661 * q * q * q);
    double b3 = 0.422205 * q * q * q;
    coef[0] = 1.0 - (b1 + b2 + b3) / b0;
    coef[1] = b1 / b0;
    coef[2] = b2 / b0;
    coef[3] = b3 / b0;
    return (int)ceil(6.0 * sigma);
}

/* One line x[0 .. n-1] (stride `st`) -> y (stride `st`), work buffer of n + P. */
static void or_rg_line(const double complex *x, long st, int n, const double *c, int P,
                       double complex *w, double complex *y)
{
    double complex w1 = x[0], w2 = x[0], w3 = x[0];
    for (int k = 0; k < n + P; k++) {
        double complex xin = k < n ? x[(long)k * st] : x[(long)(n - 1) * st];
        double complex v = c[0] * xin + c[1] * w1 + c[2] * w2 + c[3] * w3;
        w[k] = v;
        w3 = w2; w2 = w1; w1 = v;
    }
    double complex y1 = w[n + P - 1], y2 = y1, y3 = y1;
    for (int k = n + P - 1; k >= 0; k--) {
        double complex v = c[0] * w[k] + c[1] * y1 + c[2] * y2 + c[3] * y3;
        if (k < n) y[(long)k * st] = v;
        y3 = y2; y2 = y1; y1 = v;
    }
}

/* Separable recursive Gaussian of a complex H x W image: columns, then rows. */
static void or_rg_filter_c(const double complex *x, int H, int W, double sigma,
                           double complex *tmp, double complex *y)
{
    double c[4];
    int P = or_rg_coefs(sigma, c);
#pragma omp parallel
    {
        double complex *w = (double complex *)malloc(sizeof(double complex) * (size_t)((H > W ? H : W) + P));
#pragma omp for schedule(static)
        for (int j = 0; j < W; j++) or_rg_line(x + j, W, H, c, P, w, tmp + j);
#pragma omp for schedule(static)
        for (int i = 0; i < H; i++) or_rg_line(tmp + (size_t)i * W, 1, W, c, P, w, y + (size_t)i * W);
        free(w);
    }
}

/* The recursive Gaussian of a real image (the spatial averaging alone). */
void or_rg_filter(const double *x, int H, int W, double sigma, double *y)
{
    size_t n = (size_t)H * W;
    double complex *a = (double complex *)malloc(n * sizeof(double complex));
    double complex *t = (double complex *)malloc(n * sizeof(double complex));
    double complex *b = (double complex *)malloc(n * sizeof(double complex));
    for (size_t p = 0; p < n; p++) a[p] = x[p];
    or_rg_filter_c(a, H, W, sigma, t, b);
    for (size_t p = 0; p < n; p++) y[p] = creal(b[p]);
    free(a); free(t); free(b);
}

/* The recursive Gaussian of one line of n samples as an n x n matrix:
 * M[a n + b] is the weight of input b in output a (column b is the line's
 * response to the unit vector e_b, both recursions and their starts and the
 * extension past the end included).  The filter is linear, so these weights
 * are the whole filter. */
void or_rg_matrix(int n, double sigma, double *M)
{
    double c[4];
    int P = or_rg_coefs(sigma, c);
    double complex *e = (double complex *)malloc(sizeof(double complex) * (size_t)n);
    double complex *w = (double complex *)malloc(sizeof(double complex) * (size_t)(n + P));
    double complex *y = (double complex *)malloc(sizeof(double complex) * (size_t)n);
    for (int b = 0; b < n; b++) {
        for (int k = 0; k < n; k++) e[k] = k == b ? 1.0 : 0.0;
        or_rg_line(e, 1, n, c, P, w, y);
        for (int a = 0; a < n; a++) M[(size_t)a * n + b] = creal(y[a]);
    }
    free(e); free(w); free(y);
}

/* P and Q of eq. (BF) at pixel (i, j) with explicit per-axis weights: pixel
 * (zi, zj) weighs Mv[i][zi] Mh[j][zj] (any separable linear spatial filter,
 * its border handling folded into the matrices). */
static void or_pq_mat(const double *f, int H, int W, const double *Mv, const double *Mh,
                      const or_range *rg, int i, int j, double *P, double *Q)
{
    double fx = f[(size_t)i * W + j], num = 0.0, den = 0.0;
    for (int zi = 0; zi < H; zi++) {
        double wv = Mv[(size_t)i * H + zi];
        if (wv == 0.0) continue;
        for (int zj = 0; zj < W; zj++) {
            double weight = wv * Mh[(size_t)j * W + zj];
            double val = f[(size_t)zi * W + zj];
            double k = or_phi(rg, val - fx);
            num += weight * k * val;
            den += weight * k;
        }
    }
    *P = num;
    *Q = den;
}

/* eq. (BF) summed over every pixel with the weights of or_pq_mat. */
void or_bf_brute_mat(const double *f, int H, int W, const double *Mv, const double *Mh,
                     int mode, double sigma_r, int N, double *out)
{
    or_range rg = or_make_range(mode, sigma_r, N);
#pragma omp parallel for schedule(dynamic, 4)
    for (int i = 0; i < H; i++)
        for (int j = 0; j < W; j++) {
            double P, Q;
            or_pq_mat(f, H, W, Mv, Mh, &rg, i, j, &P, &Q);
            out[(size_t)i * W + j] = P / Q;
        }
}

/* Exact gradient of L = sum_x u(x) out(x) with respect to every pixel of f
 * and to sigma_r (N held fixed) with the weights of or_pq_mat: the chain rule
 * of or_grad_rg, each pixel z of the image contributing with its weight in
 * the output at x (through its value and the argument f(z) - f(x)) and x
 * through the argument. */
void or_bf_grad_mat(const double *f, const double *u, int H, int W, const double *Mv,
                    const double *Mh, int mode, double sigma_r, int N, double *grad_f,
                    double *grad_sigma_r)
{
    or_range rg = or_make_range(mode, sigma_r, N);
    size_t n = (size_t)H * W;
    int nt = or_num_threads();
    double *buf = (double *)calloc(n * (size_t)nt, sizeof(double));
    double *gs = (double *)calloc((size_t)nt, sizeof(double));
#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *g = buf + n * (size_t)tid;
        double gsl = 0.0;
#pragma omp for schedule(dynamic, 4)
        for (int i = 0; i < H; i++) {
            for (int j = 0; j < W; j++) {
                double P, Q;
                or_pq_mat(f, H, W, Mv, Mh, &rg, i, j, &P, &Q);
                double o = P / Q;
                double alpha = u[(size_t)i * W + j] / Q;
                double fx = f[(size_t)i * W + j];
                const size_t px = (size_t)i * W + j;
                for (int zi = 0; zi < H; zi++) {
                    double wv = Mv[(size_t)i * H + zi];
                    if (wv == 0.0) continue;
                    for (int zj = 0; zj < W; zj++) {
                        const size_t pz = (size_t)zi * W + zj;
                        double aw = alpha * wv * Mh[j * (size_t)W + zj];
                        double dv = f[pz] - o;
                        double arg = f[pz] - fx;
                        double dk = or_dphi(&rg, arg);
                        g[pz] += aw * (or_phi(&rg, arg) + dk * dv);
                        g[px] -= aw * dk * dv;
                        if (grad_sigma_r) gsl += aw * or_dphi_dsigma(&rg, arg) * dv;
                    }
                }
            }
        }
        gs[tid] = gsl;
    }
    for (size_t p = 0; p < n; p++) {
        double s = 0.0;
        for (int t = 0; t < nt; t++) s += buf[n * (size_t)t + p];
        grad_f[p] = s;
    }
    double s = 0.0;
    for (int t = 0; t < nt; t++) s += gs[t];
    if (grad_sigma_r) *grad_sigma_r = s;
    free(buf);
    free(gs);
}

/* Algorithm 1, steps 1-5, in the paper's complex notation (as or_bf_trig),
 * with the recursive Gaussian as the O(1) averaging of step 4 (Section 3). */
double or_bf_trig_rg(const double *f, int H, int W, double sigma_s, double sigma_r,
                     double T, int N, double *out, double *q_out)
{
    size_t n = (size_t)H * W;
    double gamma = OR_PI / (2.0 * T);
    double rho = gamma * sigma_r;
    double complex *h = (double complex *)malloc(n * sizeof(double complex));
    double complex *g = (double complex *)malloc(n * sizeof(double complex));
    double complex *hb = (double complex *)malloc(n * sizeof(double complex));
    double complex *gb = (double complex *)malloc(n * sizeof(double complex));
    double complex *tmp = (double complex *)malloc(n * sizeof(double complex));
    double complex *num = (double complex *)calloc(n, sizeof(double complex));
    double complex *den = (double complex *)calloc(n, sizeof(double complex));
    for (int k = 0; k <= N; k++) {
        double cn = exp(lgamma(N + 1.0) - lgamma(k + 1.0) - lgamma(N - k + 1.0) -
                        N * log(2.0));
        double freq = gamma * (double)(2 * k - N) / (rho * sqrt((double)N));
        for (size_t p = 0; p < n; p++) {
            h[p] = cexp(I * freq * f[p]);
            g[p] = f[p] * h[p];
        }
        or_rg_filter_c(h, H, W, sigma_s, tmp, hb);
        or_rg_filter_c(g, H, W, sigma_s, tmp, gb);
        for (size_t p = 0; p < n; p++) {
            double complex d = cn * cexp(-I * freq * f[p]);
            num[p] += d * gb[p];
            den[p] += d * hb[p];
        }
    }
    double worst = 0.0;
    for (size_t p = 0; p < n; p++) {
        out[p] = creal(num[p]) / creal(den[p]);
        if (q_out) q_out[p] = creal(den[p]);
        double e1 = fabs(cimag(num[p])) / (fabs(creal(num[p])) + 1e-300);
        double e2 = fabs(cimag(den[p])) / (fabs(creal(den[p])) + 1e-300);
        if (e1 > worst) worst = e1;
        if (e2 > worst) worst = e2;
    }
    free(h); free(g); free(hb); free(gb); free(tmp); free(num); free(den);
    return worst;
}
