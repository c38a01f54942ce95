// Host-side plan: Algorithm 1 steps 1-3 in double precision.
//
//   step 1: gamma = pi / (2T), rho = gamma sigma_r
//   step 2: N = (gamma sigma_r)^-2 rounded up (last row of Table 1), N >= 1
//   step 3: the raised cosine cos^N of Section 2.3 expanded by the binomial
//           theorem into N+1 exponentials with weights 2^-N C(N,n) and
//           frequencies gamma (2n - N) / (rho sqrt N) = (2n - N) / (sigma_r sqrt N).
//
// Terms n and N-n are complex conjugates with equal weights (the c_n of
// eq. (kernel) are real and symmetric), so each pair folds into one real
// cosine term of weight 2 * 2^-N C(N,n) at frequency m / (sigma_r sqrt N),
// m = N - 2n > 0; for even N the middle term n = N/2 is the constant
// 2^-N C(N, N/2) (Section 2.3).  A term whose FP32 weight rounds to exactly 0
// contributes exactly 0 in the kernels' FP32 arithmetic and is dropped.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include "bf_internal.h"

namespace {

constexpr double kPi = 3.14159265358979323846;

// Degree rule with a relative guard so that a value that is an integer in
// exact arithmetic is not pushed up by rounding.
int degree_rule(double sigma_r, double T) {
    double gamma = kPi / (2.0 * T);
    double x = 1.0 / ((gamma * sigma_r) * (gamma * sigma_r));
    if (!(x < 1e9)) return 1 << 30;
    double n = std::ceil(x * (1.0 - 1e-12));
    return n < 1.0 ? 1 : (int)n;
}

// Table 1: empirical minimum degrees N_0 for T = 255, by decreasing sigma.
constexpr double kTable1Sigma[] = {200.0, 150.0, 100.0, 80.0, 60.0, 50.0, 40.0};
constexpr int kTable1N0[] = {1, 2, 3, 4, 5, 7, 9};

// Degree from Table 1 at sigma' = 255 sigma_r / T: the N_0 of the largest
// tabulated sigma not above sigma', capped by the estimate; the estimate
// below the table's smallest sigma.
int degree_table1(double sigma_r, double T) {
    const double sp = sigma_r * 255.0 / T;
    const int est = degree_rule(sigma_r, T);
    for (int k = 0; k < 7; ++k)
        if (sp >= kTable1Sigma[k]) return kTable1N0[k] < est ? kTable1N0[k] : est;
    return est;
}

// p[n] = 2^-N C(N, n), n = 0..N, by the ratio C(N,n-1)/C(N,n) = n/(N-n+1)
// walked outward from the middle and normalised to unit sum (the binomial
// weights sum to 1).  Tails below the double range become 0.
std::vector<double> binomial_weights(int N) {
    std::vector<double> u(N + 1, 0.0);
    int mid = N / 2;
    u[mid] = 1.0;
    for (int n = mid; n >= 1; --n) u[n - 1] = u[n] * (double)n / (double)(N - n + 1);
    for (int n = mid; n < N; ++n) u[n + 1] = u[n] * (double)(N - n) / (double)(n + 1);
    double s = 0.0;
    for (int n = 0; n <= N; ++n) s += u[n];
    for (int n = 0; n <= N; ++n) u[n] /= s;
    return u;
}

}  // namespace

// Spatial kernel of a plan (the 1-D taps w1, support radius, achieved sigma
// and the box normaliser).  On failure nothing needs freeing; the caller
// deletes the plan.
static bf_status set_spatial(bf_plan *p, double sigma_s, bf_spatial_kind kind,
                             const bf_plan_opts &o, const std::string &who) {
    if (kind == BF_SPATIAL_GAUSS_RECURSIVE) {
        // Young and van Vliet (1995), published design (valid for sigma >= 0.5)
        if (sigma_s < 0.5 || sigma_s > 256.0)
            return bf::fail(BF_EUNSUPPORTED, who + ": the recursive Gaussian takes "
                                                   "0.5 <= sigma_s <= 256");
        if (o.radius_override != 0 || o.box_passes != 0)
            return bf::fail(BF_EINVAL, who + ": radius and passes do not apply to the "
                                             "recursive Gaussian");
        const double q = sigma_s >= 2.5 ? 0.98711 * sigma_s - 0.96330
                                        : 3.97156 - 4.14554 * std::sqrt(1.0 - 0.26891 * sigma_s);
        const double q2 = q * q, q3 = q2 * q;
        const double b0 = 1.57825 + 2.44413 * q + 1.4281 * q2 + 0.422205 * q3;
        const double b1 = 2.44413 * q + 2.85619 * q2 + 1.26661 * q3;
        const double b2 = -(1.4281 * q2 + 1.26661 * q3);
        const double b3 = 0.422205 * q3;
        p->rg[0] = 1.0 - (b1 + b2 + b3) / b0;
        p->rg[1] = b1 / b0;
        p->rg[2] = b2 / b0;
        p->rg[3] = b3 / b0;
        p->rg_P = (int)std::ceil(6.0 * sigma_s);
        p->R = p->rg_P;
        // standard deviation of the cascade's impulse response, from the
        // cumulants of the causal part: mean S'/B, variance S''/B + (S'/B)^2
        // with S' = sum k a_k, S'' = sum k^2 a_k, doubled for the cascade
        const double s1 = p->rg[1] + 2 * p->rg[2] + 3 * p->rg[3];
        const double s2 = p->rg[1] + 4 * p->rg[2] + 9 * p->rg[3];
        const double B = p->rg[0];
        p->achieved_sigma = std::sqrt(2.0 * (s2 / B + (s1 / B) * (s1 / B)));
        p->q_scale = 1.f;
        return BF_OK;
    }
    if (kind == BF_SPATIAL_GAUSS_TRUNC) {
        int R = o.radius_override > 0 ? o.radius_override : (int)std::ceil(3.0 * sigma_s);
        if (R > BF_MAX_TAPS_R) {
            return bf::fail(BF_EUNSUPPORTED, who + ": Gaussian support radius " +
                                                 std::to_string(R) + " exceeds " +
                                                 std::to_string(BF_MAX_TAPS_R));
        }
        p->R = R;
        p->w1.resize(2 * R + 1);
        double s = 0.0;
        for (int i = -R; i <= R; ++i) {
            double v = std::exp(-(double)i * i / (2.0 * sigma_s * sigma_s));
            p->w1[i + R] = v;
            s += v;
        }
        double var = 0.0;
        for (int i = -R; i <= R; ++i) {
            p->w1[i + R] /= s;
            var += p->w1[i + R] * (double)i * i;
        }
        p->achieved_sigma = std::sqrt(var);
        p->q_scale = 1.f;
    } else {
        int passes = o.box_passes > 0 ? o.box_passes : 3;
        if (passes != 3) {
            return bf::fail(BF_EUNSUPPORTED, who + ": only 3 box passes are implemented");
        }
        int r = o.radius_override;
        if (r <= 0) {
            // passes boxes of width 2r+1 have variance passes ((2r+1)^2 - 1) / 12
            double L = std::sqrt(12.0 * sigma_s * sigma_s / passes + 1.0);
            r = (int)std::floor((L - 1.0) / 2.0 + 0.5);
            if (r < 1) r = 1;
        }
        if (r > 64) {
            return bf::fail(BF_EUNSUPPORTED, who + ": box half-width " +
                                                 std::to_string(r) + " exceeds 64");
        }
        p->passes = passes;
        p->r_box = r;
        p->R = passes * r;
        // taps: convolution of `passes` boxes, exact integer counts / (2r+1)^passes
        std::vector<double> c(1, 1.0);
        for (int k = 0; k < passes; ++k) {
            std::vector<double> n(c.size() + 2 * r, 0.0);
            for (size_t i = 0; i < c.size(); ++i)
                for (int d = 0; d <= 2 * r; ++d) n[i + d] += c[i];
            c.swap(n);
        }
        double denom = std::pow(2.0 * r + 1.0, passes);
        p->w1.resize(c.size());
        for (size_t i = 0; i < c.size(); ++i) p->w1[i] = c[i] / denom;
        double L = 2.0 * r + 1.0;
        p->achieved_sigma = std::sqrt(passes * (L * L - 1.0) / 12.0);
        // the kernels sum the 2-D box cascade without dividing: scale = L^(-2 passes)
        p->q_scale = (float)std::pow(L, -2.0 * passes);
    }
    p->w1f.assign(p->w1.begin(), p->w1.end());
    return BF_OK;
}

// FP32 copies of the term table; BF_EUNSUPPORTED above the kernels' limit.
static bf_status finish_terms(bf_plan *p, const std::string &who) {
    if ((int)p->a.size() > BF_MAX_TERMS)
        return bf::fail(BF_EUNSUPPORTED, who + ": too many terms");
    for (size_t k = 0; k < p->a.size(); ++k) {
        p->a32.push_back((float)p->a[k]);
        p->turns32.push_back((float)(p->omega[k] / (2.0 * kPi)));
    }
    return BF_OK;
}

extern "C" bf_status bf_plan_create(bf_plan **out, double sigma_s, double sigma_r, double T,
                                    bf_spatial_kind kind, const bf_plan_opts *opts) {
    if (!out) return bf::fail(BF_EINVAL, "bf_plan_create: out is NULL");
    *out = nullptr;
    if (!(sigma_s > 0) || !std::isfinite(sigma_s))
        return bf::fail(BF_EINVAL, "bf_plan_create: sigma_s must be finite and > 0");
    if (!(sigma_r > 0) || !std::isfinite(sigma_r))
        return bf::fail(BF_EINVAL, "bf_plan_create: sigma_r must be finite and > 0");
    if (!(T > 0) || !std::isfinite(T))
        return bf::fail(BF_EINVAL, "bf_plan_create: T must be finite and > 0");
    if (kind != BF_SPATIAL_GAUSS_TRUNC && kind != BF_SPATIAL_BOX_ITER &&
        kind != BF_SPATIAL_GAUSS_RECURSIVE)
        return bf::fail(BF_EINVAL, "bf_plan_create: unknown spatial kind");
    bf_plan_opts o{};
    if (opts) o = *opts;
    if (o.N_override < 0 || o.radius_override < 0 || o.box_passes < 0)
        return bf::fail(BF_EINVAL, "bf_plan_create: negative option");
    if (o.degree_rule != BF_DEGREE_ESTIMATE && o.degree_rule != BF_DEGREE_TABLE1)
        return bf::fail(BF_EINVAL, "bf_plan_create: unknown degree_rule");

    bf_plan *p = new (std::nothrow) bf_plan();
    if (!p) return bf::fail(BF_ENOMEM, "bf_plan_create: out of host memory");
    p->sigma_s = sigma_s;
    p->sigma_r = sigma_r;
    p->T = T;
    p->kind = (int)kind;

    int N = o.N_override > 0                        ? o.N_override
            : o.degree_rule == BF_DEGREE_TABLE1 ? degree_table1(sigma_r, T)
                                                : degree_rule(sigma_r, T);
    if (N > BF_MAX_N) {
        delete p;
        return bf::fail(BF_EUNSUPPORTED, "bf_plan_create: degree N = " + std::to_string(N) +
                                             " exceeds " + std::to_string(BF_MAX_N) +
                                             " (sigma_r too small for T)");
    }
    p->N = N;

    {
        const bf_status st = set_spatial(p, sigma_s, kind, o, "bf_plan_create");
        if (st != BF_OK) {
            delete p;
            return st;
        }
    }

    // ---- range kernel terms (folded conjugate pairs)
    std::vector<double> bw = binomial_weights(N);
    double delta = 1.0 / (sigma_r * std::sqrt((double)N));  // gamma / (rho sqrt N)
    for (int n = 0; 2 * n < N; ++n) {  // m = N - 2n > 0, largest m (smallest weight) first
        int m = N - 2 * n;
        double a = 2.0 * bw[n];
        if ((float)a == 0.0f) continue;
        double w = m * delta;
        p->a.push_back(a);
        p->omega.push_back(w);
    }
    if (N % 2 == 0) {
        p->a.push_back(bw[N / 2]);
        p->omega.push_back(0.0);
        p->has_center = true;
    }
    {
        const bf_status st = finish_terms(p, "bf_plan_create");
        if (st != BF_OK) {
            delete p;
            return st;
        }
    }
    *out = p;
    return BF_OK;
}

extern "C" bf_status bf_plan_create_cosine(bf_plan **out, double sigma_s, double gamma,
                                           const double *a, int n_coef, bf_spatial_kind kind,
                                           const bf_plan_opts *opts) {
    const std::string who = "bf_plan_create_cosine";
    if (!out) return bf::fail(BF_EINVAL, who + ": out is NULL");
    *out = nullptr;
    if (!a) return bf::fail(BF_EINVAL, who + ": coefficients are NULL");
    if (!(sigma_s > 0) || !std::isfinite(sigma_s))
        return bf::fail(BF_EINVAL, who + ": sigma_s must be finite and > 0");
    if (!(gamma > 0) || !std::isfinite(gamma))
        return bf::fail(BF_EINVAL, who + ": gamma must be finite and > 0");
    if (n_coef < 1) return bf::fail(BF_EINVAL, who + ": n_coef must be >= 1");
    if (n_coef > BF_MAX_N + 1)
        return bf::fail(BF_EUNSUPPORTED, who + ": degree above " + std::to_string(BF_MAX_N));
    for (int n = 0; n < n_coef; ++n)
        if (!std::isfinite(a[n])) return bf::fail(BF_EINVAL, who + ": non-finite coefficient");
    if (kind != BF_SPATIAL_GAUSS_TRUNC && kind != BF_SPATIAL_BOX_ITER &&
        kind != BF_SPATIAL_GAUSS_RECURSIVE)
        return bf::fail(BF_EINVAL, who + ": unknown spatial kind");
    bf_plan_opts o{};
    if (opts) o = *opts;
    if (o.N_override != 0 || o.degree_rule != 0)
        return bf::fail(BF_EINVAL, who + ": N_override and degree_rule do not apply");
    if (o.radius_override < 0 || o.box_passes < 0)
        return bf::fail(BF_EINVAL, who + ": negative option");

    bf_plan *p = new (std::nothrow) bf_plan();
    if (!p) return bf::fail(BF_ENOMEM, who + ": out of host memory");
    p->sigma_s = sigma_s;
    p->sigma_r = 0.0;  // no sigma_r: the kernel is given by its coefficients
    p->T = 0.0;
    p->kind = (int)kind;
    p->cosine = true;
    p->gamma = gamma;
    {
        const bf_status st = set_spatial(p, sigma_s, kind, o, who);
        if (st != BF_OK) {
            delete p;
            return st;
        }
    }
    // Terms cos(n gamma s) with a nonzero FP32 weight, smallest |a_n| first
    // (a zero weight adds exactly 0 in the kernels), the constant a_0 last.
    std::vector<int> order;
    int degree = 0;
    for (int n = 1; n < n_coef; ++n)
        if ((float)a[n] != 0.0f) {
            order.push_back(n);
            degree = n;
        }
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return std::fabs(a[x]) < std::fabs(a[y]); });
    for (int n : order) {
        p->a.push_back(a[n]);
        p->omega.push_back((double)n * gamma);
    }
    if ((float)a[0] != 0.0f) {
        p->a.push_back(a[0]);
        p->omega.push_back(0.0);
        p->has_center = true;
    }
    if (p->a.empty()) {
        delete p;
        return bf::fail(BF_EINVAL, who + ": every coefficient is 0 in FP32");
    }
    p->N = degree;
    {
        const bf_status st = finish_terms(p, who);
        if (st != BF_OK) {
            delete p;
            return st;
        }
    }
    *out = p;
    return BF_OK;
}

extern "C" void bf_plan_destroy(bf_plan *plan) { delete plan; }

extern "C" bf_status bf_plan_info(const bf_plan *p, int *N, int *n_freq, int *radius,
                                  double *achieved_sigma_s) {
    if (!p) return bf::fail(BF_EINVAL, "bf_plan_info: plan is NULL");
    if (N) *N = p->N;
    if (n_freq) *n_freq = (int)p->a.size();
    if (radius) *radius = p->R;
    if (achieved_sigma_s) *achieved_sigma_s = p->achieved_sigma;
    return BF_OK;
}

extern "C" bf_status bf_plan_terms(const bf_plan *p, double *a, double *omega, int cap,
                                   int *count) {
    if (!p) return bf::fail(BF_EINVAL, "bf_plan_terms: plan is NULL");
    int n = (int)p->a.size();
    if (count) *count = n;
    if (a || omega) {
        if (cap < n) return bf::fail(BF_EINVAL, "bf_plan_terms: cap too small");
        for (int k = 0; k < n; ++k) {
            if (a) a[k] = p->a[k];
            if (omega) omega[k] = p->omega[k];
        }
    }
    return BF_OK;
}

extern "C" bf_status bf_plan_weights(const bf_plan *p, double *w1, int cap, int *count) {
    if (!p) return bf::fail(BF_EINVAL, "bf_plan_weights: plan is NULL");
    int n = (int)p->w1.size();
    if (count) *count = n;
    if (w1) {
        if (cap < n) return bf::fail(BF_EINVAL, "bf_plan_weights: cap too small");
        std::memcpy(w1, p->w1.data(), sizeof(double) * n);
    }
    return BF_OK;
}

namespace bf {

void fill_terms(const bf_plan *p, BfTerms *t) {
    t->n_terms = (int)p->a32.size();
    for (int k = 0; k < t->n_terms; ++k) {
        t->a[k] = p->a32[k];
        t->t[k] = p->turns32[k];
    }
}

void fill_taps(const bf_plan *p, BfTaps *t) {
    std::memset(t, 0, sizeof(*t));
    int n = (int)p->w1f.size();
    for (int k = 0; k < n && k < 2 * BF_MAX_TAPS_R + 1; ++k) t->w[k] = p->w1f[k];
    pair_taps(t);
}

void pair_taps(BfTaps *t) {
    for (int k = 0; k < 2 * BF_MAX_TAPS_R + 1; ++k) t->w2[k] = make_float2(t->w[k], t->w[k]);
}

}  // namespace bf
