/*
 * cfust_oracle.c -- plain FP64 CPU oracle for the FM-CFUST EM algorithm.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg, never by the CUDA library.  It is written to
 * be checked by eye against the paper (Lee, Leemaqz & McLachlan,
 * arXiv:1606.02054): every step below names the equation it evaluates, runs
 * one observation and one component at a time, and uses no blocking or
 * fusion.  The special functions are its own (continued fractions, series,
 * Newton/Halley iterations); libm supplies only exp/log/lgamma/erfc.
 *
 * Readings of the paper taken here (the paper is silent or garbled there):
 *  - eq (3): the constant is (nu*pi)^(-p/2) and the exponent -(nu+p)/2;
 *  - eq (13): "nu d" under both square roots is nu + d;
 *  - eqs (16)-(17): U|y follows the W-tilted truncated t of Sec. 3.1, so
 *    e2 = u E[U], e3 = u E[U U^T]; the truncated-t moments use the identity
 *    x t_v(x; S) = -(v/(v-2)) S grad t_{v-2}(x; v S/(v-2)), which needs one
 *    T_{q-1} (dof nu+p+1) per coordinate and one T_{q-2} (dof nu+p) per
 *    ordered coordinate pair;
 *  - eq (22): the sum runs over j and the sign of the second term is +;
 *    nu is bracketed in [nu_min, nu_max] and found by bisection;
 *  - M-step order pi -> mu (with Delta^(k)) -> Delta (with mu^(k+1)) ->
 *    Sigma (with mu^(k+1), Delta^(k+1)) -> nu, as eqs (19)-(21) state;
 *  - T_q is not specified by the paper: T_0 = 1, T_1 by the incomplete beta
 *    function, T_2 by adaptive Gauss-Legendre quadrature of the conditional
 *    one-dimensional integral, T_k (k >= 3) by Genz's separation of
 *    variables for the multivariate t (chi variable first, fixed variable
 *    order) on a randomised rank-1 Korobov lattice with the baker's
 *    transform.
 */
#include "cfust_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORA_PI 3.14159265358979323846
#define ORA_MAXP 64
#define ORA_MAXQ 8

/* ------------------------------------------------------------------ */
/* digamma: recurrence psi(x) = psi(x+1) - 1/x up to x >= 10, then the   */
/* asymptotic series ln x - 1/(2x) - sum_k B_2k / (2k x^2k).             */
/* ------------------------------------------------------------------ */
double ora_digamma(double x)
{
    if (x <= 0.0 && floor(x) == x) return NAN;
    if (x < 0.0) return ora_digamma(1.0 - x) - ORA_PI / tan(ORA_PI * x);
    double acc = 0.0;
    while (x < 10.0) { acc -= 1.0 / x; x += 1.0; }
    double f = 1.0 / (x * x);
    /* B2/2=1/12, B4/4=-1/120, B6/6=1/252, B8/8=-1/240, B10/10=1/132,
       B12/12=-691/32760, B14/14=1/12 */
    double t = f * (1.0 / 12 - f * (1.0 / 120 - f * (1.0 / 252 - f * (1.0 / 240
               - f * (1.0 / 132 - f * (691.0 / 32760 - f / 12.0))))));
    return acc + log(x) - 0.5 / x - t;
}

/* ------------------------------------------------------------------ */
/* Standard normal CDF and its inverse.                                  */
/* ------------------------------------------------------------------ */
double ora_phi(double x) { return 0.5 * erfc(-x / sqrt(2.0)); }

/* Inverse normal CDF: Abramowitz & Stegun 26.2.23 starting value
 * (|error| < 4.5e-4), then Halley steps on Phi(x) = p, which converge
 * cubically to full double precision. */
double ora_phi_inv(double p)
{
    if (!(p > 0.0)) return -INFINITY;
    if (!(p < 1.0)) return INFINITY;
    double pt = p < 0.5 ? p : 1.0 - p; /* exact for p >= 0.5 (Sterbenz) */
    double t = sqrt(-2.0 * log(pt));
    double x = -(t - (2.515517 + 0.802853 * t + 0.010328 * t * t)
                 / (1.0 + 1.432788 * t + 0.189269 * t * t + 0.001308 * t * t * t));
    for (int it = 0; it < 3; ++it) {
        double e = ora_phi(x) - pt;
        double u = e * sqrt(2.0 * ORA_PI) * exp(0.5 * x * x);
        x = x - u / (1.0 + 0.5 * x * u);
    }
    return p < 0.5 ? x : -x;
}

/* ------------------------------------------------------------------ */
/* Regularised incomplete beta I_x(a, b) by its continued fraction        */
/* 1/(1+ d1/(1+ d2/(1+ ...))), d_{2m+1} = -(a+m)(a+b+m)x/((a+2m)(a+2m+1)), */
/* d_{2m} = m(b-m)x/((a+2m-1)(a+2m)), evaluated by the modified Lentz      */
/* method.  x and y = 1 - x are both passed so neither loses precision.  */
/* ------------------------------------------------------------------ */
static double betacf(double a, double b, double x)
{
    const double tiny = 1e-300;
    double c = 1.0, d = 1.0 - (a + b) * x / (a + 1.0);
    if (fabs(d) < tiny) d = tiny;
    d = 1.0 / d;
    double h = d;
    for (int m = 1; m <= 20000; ++m) {
        double m2 = 2.0 * m;
        double aa = m * (b - m) * x / ((a - 1.0 + m2) * (a + m2));
        d = 1.0 + aa * d; if (fabs(d) < tiny) d = tiny;
        c = 1.0 + aa / c; if (fabs(c) < tiny) c = tiny;
        d = 1.0 / d; h *= d * c;
        aa = -(a + m) * (a + b + m) * x / ((a + m2) * (a + 1.0 + m2));
        d = 1.0 + aa * d; if (fabs(d) < tiny) d = tiny;
        c = 1.0 + aa / c; if (fabs(c) < tiny) c = tiny;
        d = 1.0 / d;
        double del = d * c;
        h *= del;
        if (fabs(del - 1.0) < 1e-16) break;
    }
    return h;
}

/* lgb = lgamma(a+b) - lgamma(a) - lgamma(b) */
static double incbeta2c(double a, double b, double x, double y, double lgb)
{
    if (x <= 0.0) return 0.0;
    if (y <= 0.0) return 1.0;
    double lbt = lgb + a * log(x) + b * log(y);
    if (x < (a + 1.0) / (a + b + 2.0)) return exp(lbt) * betacf(a, b, x) / a;
    return 1.0 - exp(lbt) * betacf(b, a, y) / b;
}

static double incbeta2(double a, double b, double x, double y)
{
    return incbeta2c(a, b, x, y, lgamma(a + b) - lgamma(a) - lgamma(b));
}

double ora_incbeta(double a, double b, double x) { return incbeta2(a, b, x, 1.0 - x); }

/* ------------------------------------------------------------------ */
/* Regularised incomplete gamma P(a, x), Q = 1 - P: power series for     */
/* x < a + 1, Legendre continued fraction for Q otherwise.               */
/* ------------------------------------------------------------------ */
static void incgamma_pq(double a, double x, double* P, double* Q)
{
    if (x <= 0.0) { *P = 0.0; *Q = 1.0; return; }
    if (isinf(x)) { *P = 1.0; *Q = 0.0; return; }
    double lpre = -x + a * log(x) - lgamma(a);
    if (x < a + 1.0) {
        double ap = a, del = 1.0 / a, sum = del;
        for (int n = 1; n < 100000; ++n) {
            ap += 1.0; del *= x / ap; sum += del;
            if (fabs(del) < fabs(sum) * 1e-17) break;
        }
        *P = sum * exp(lpre);
        *Q = 1.0 - *P;
    } else {
        const double tiny = 1e-300;
        double b = x + 1.0 - a, c = 1.0 / tiny, d = 1.0 / b, h = d;
        for (int i = 1; i < 100000; ++i) {
            double an = -i * (i - a);
            b += 2.0;
            d = an * d + b; if (fabs(d) < tiny) d = tiny;
            c = b + an / c; if (fabs(c) < tiny) c = tiny;
            d = 1.0 / d;
            double del = d * c;
            h *= del;
            if (fabs(del - 1.0) < 1e-16) break;
        }
        *Q = exp(lpre) * h;
        *P = 1.0 - *Q;
    }
}

double ora_incgamma_p(double a, double x)
{
    double P, Q;
    incgamma_pq(a, x, &P, &Q);
    return P;
}

/* Chi-square quantile: x with P(nu/2, x/2) = w (lower half) or
 * Q(nu/2, x/2) = wc (upper half), wc = 1 - w supplied separately.
 * Newton's method on the log tail probability with a bisection safeguard;
 * Wilson-Hilferty start. */
double ora_chi2_quantile(double w, double wc, double nu)
{
    if (!(w > 0.0)) return 0.0;
    if (!(wc > 0.0)) return INFINITY;
    const double a = 0.5 * nu;
    const int upper = w > 0.5;
    double z = upper ? -ora_phi_inv(wc) : ora_phi_inv(w);
    double cwh = 2.0 / (9.0 * nu);
    double base = 1.0 - cwh + z * sqrt(cwh);
    double x = nu * base * base * base;
    if (!(x > 0.0) || (!upper && w < 1e-3)) {
        /* small-x start from P(a, x/2) ~ (x/2)^a / Gamma(a+1) */
        double xs = 2.0 * exp((log(w) + lgamma(a + 1.0)) / a);
        if (!(x > 0.0) || xs < x) x = xs;
    }
    /* Newton on G(x) = log P(a, x/2) - log w (or log wc - log Q(a, x/2)),
     * increasing in x, G' = density / P (or density / Q). */
    double lo = 0.0, hi = INFINITY;
    const double lt = upper ? log(wc) : log(w);
    for (int it = 0; it < 400; ++it) {
        double P, Q;
        incgamma_pq(a, 0.5 * x, &P, &Q);
        double tailv = upper ? Q : P;
        double G = upper ? (lt - log(tailv)) : (log(tailv) - lt);
        if (G == 0.0) return x;
        if (G > 0.0) hi = x; else lo = x;
        double ldens = log(0.5) + (a - 1.0) * log(0.5 * x) - 0.5 * x - lgamma(a);
        double xn = x - G * exp(log(tailv) - ldens);
        if (!(xn > lo && xn < hi)) xn = isinf(hi) ? 2.0 * x : 0.5 * (lo + hi);
        if (fabs(xn - x) <= 1e-15 * x) { x = xn; break; }
        if (isfinite(hi) && hi - lo <= 1e-15 * hi) { x = 0.5 * (lo + hi); break; }
        x = xn;
    }
    return x;
}

/* ------------------------------------------------------------------ */
/* Univariate t density and CDF (standard location 0, scale 1).          */
/* ------------------------------------------------------------------ */
double ora_t1pdf(double x, double nu)
{
    if (isinf(nu)) return exp(-0.5 * x * x) / sqrt(2.0 * ORA_PI);  /* the normal limit */
    return exp(lgamma(0.5 * (nu + 1.0)) - lgamma(0.5 * nu) - 0.5 * log(nu * ORA_PI)
               - 0.5 * (nu + 1.0) * log1p(x * x / nu));
}

/* T_1(x; nu): P(T > |x|) = 1/2 I_{nu/(nu+x^2)}(nu/2, 1/2). */
double ora_t1cdf(double x, double nu)
{
    if (isinf(nu)) return ora_phi(x);  /* the normal limit */
    if (x == 0.0) return 0.5;
    if (isinf(x)) return x > 0 ? 1.0 : 0.0;
    double x2 = x * x;
    double tail = 0.5 * incbeta2(0.5 * nu, 0.5, nu / (nu + x2), x2 / (nu + x2));
    return x > 0.0 ? 1.0 - tail : tail;
}

/* ------------------------------------------------------------------ */
/* Gauss-Legendre rule of order 20 (nodes by Newton on P_20).            */
/* ------------------------------------------------------------------ */
#define GL_N 20
static double gl_x[GL_N], gl_w[GL_N];

__attribute__((constructor)) static void gl_init(void)
{
    const int n = GL_N;
    for (int i = 0; i < n; ++i) {
        double x = cos(ORA_PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int j = 1; j < n; ++j) {
                double p2 = ((2.0 * j + 1.0) * x * p1 - j * p0) / (j + 1.0);
                p0 = p1; p1 = p2;
            }
            dp = n * (x * p1 - p0) / (x * x - 1.0);
            double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        /* recompute derivative at the converged node */
        double p0 = 1.0, p1 = x;
        for (int j = 1; j < n; ++j) {
            double p2 = ((2.0 * j + 1.0) * x * p1 - j * p0) / (j + 1.0);
            p0 = p1; p1 = p2;
        }
        dp = n * (x * p1 - p0) / (x * x - 1.0);
        gl_x[i] = x;
        gl_w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
}

typedef double (*ora_fn)(double s, const void* ctx);

static double gl_rule(ora_fn f, const void* ctx, double a, double b)
{
    double half = 0.5 * (b - a), mid = 0.5 * (a + b), sum = 0.0;
    for (int i = 0; i < GL_N; ++i) sum += gl_w[i] * f(mid + half * gl_x[i], ctx);
    return sum * half;
}

/* Recursive bisection: accept [a, b] when the 20-point rule on the whole
 * interval and on its halves agree to tol, or to a rounding floor
 * (floor = 1e-16 of the whole integral, so the recursion always ends). */
static double adapt_rec(ora_fn f, const void* ctx, double a, double b,
                        double whole, double tol, double floor_abs, int depth)
{
    double m = 0.5 * (a + b);
    double L = gl_rule(f, ctx, a, m), R = gl_rule(f, ctx, m, b);
    double err = fabs(L + R - whole);
    if (depth >= 40 || err <= tol || err <= floor_abs) return L + R;
    return adapt_rec(f, ctx, a, m, L, 0.5 * tol, floor_abs, depth + 1)
         + adapt_rec(f, ctx, m, b, R, 0.5 * tol, floor_abs, depth + 1);
}

/* Adaptive integral over [a, b] to relative accuracy ~1e-14. */
static double integrate(ora_fn f, const void* ctx, double a, double b)
{
    const int k0 = 4;
    double crude = 0.0, parts[4];
    for (int i = 0; i < k0; ++i) {
        parts[i] = gl_rule(f, ctx, a + (b - a) * i / k0, a + (b - a) * (i + 1) / k0);
        crude += parts[i];
    }
    double tol = 1e-15 * fabs(crude) + 1e-300;
    double floor_abs = 1e-17 * fabs(crude) + 1e-300;
    double sum = 0.0;
    for (int i = 0; i < k0; ++i)
        sum += adapt_rec(f, ctx, a + (b - a) * i / k0, a + (b - a) * (i + 1) / k0,
                         parts[i], tol / k0, floor_abs, 0);
    return sum;
}

/* ------------------------------------------------------------------ */
/* Bivariate t CDF T_2(h, k; rho, nu) of the standard bivariate t:       */
/* T_2 = int_{-inf}^{h} t_nu(x) T_1((k - rho x) / sqrt((1-rho^2)(nu+x^2)/ */
/* (nu+1)); nu+1) dx (the conditional law of X2 given X1 = x), with the   */
/* map x = h - (1-s)/s, s in (0, 1].                                      */
/* ------------------------------------------------------------------ */
typedef struct { double h, k, rho, nu, lpdf, lgb; } t2ctx;

static double t2_integrand(double s, const void* vctx)
{
    const t2ctx* c = (const t2ctx*)vctx;
    if (s <= 0.0) return 0.0;
    double x = c->h - (1.0 - s) / s;
    /* t_nu(x), constant hoisted */
    double pdf = exp(c->lpdf - 0.5 * (c->nu + 1.0) * log1p(x * x / c->nu));
    /* T_1(z; nu+1), same formula as ora_t1cdf with the log-beta constant hoisted */
    double z = (c->k - c->rho * x) / sqrt((1.0 - c->rho * c->rho) * (c->nu + x * x) / (c->nu + 1.0));
    double cdf;
    if (z == 0.0) cdf = 0.5;
    else {
        double n1 = c->nu + 1.0, z2 = z * z;
        double tail = 0.5 * incbeta2c(0.5 * n1, 0.5, n1 / (n1 + z2), z2 / (n1 + z2), c->lgb);
        cdf = z > 0.0 ? 1.0 - tail : tail;
    }
    return pdf * cdf / (s * s);
}

/* Standard bivariate normal CDF (the nu -> infinity limit of T_2):
 * Phi_2(h, k; rho) = Phi(h) Phi(k) + int_0^rho phi_2(h, k; r) dr, and with r = sin(theta)
 * the integrand exp(-(h^2 - 2 h k sin(theta) + k^2) / (2 cos^2(theta))) / (2 pi) is bounded
 * on [0, asin(rho)]. */
typedef struct { double h, k; } phi2_ctx;
static double phi2_integrand(double th, const void* vctx)
{
    const phi2_ctx* c = (const phi2_ctx*)vctx;
    const double st = sin(th), ct = cos(th);
    if (ct <= 0.0) return 0.0;
    return exp(-(c->h * c->h - 2.0 * c->h * c->k * st + c->k * c->k) / (2.0 * ct * ct)) / (2.0 * ORA_PI);
}

double ora_phi2(double h, double k, double rho)
{
    if (rho >= 1.0) return ora_phi(h < k ? h : k);
    /* Phi_2 at rho = -1: P(-k < X <= h) = P(-h <= X < k), taken in the form whose larger
       endpoint is the one nearer the lower tail, where Phi keeps its relative precision */
    double lower = 0.0;
    if (h + k > 0.0) lower = h - k < 0.0 ? ora_phi(h) - ora_phi(-k) : ora_phi(k) - ora_phi(-h);
    if (rho <= -1.0) return lower;
    phi2_ctx c = {h, k};
    /* the integrand is positive: from rho = 0 for rho >= 0, and from rho = -1 (the lower
       Frechet bound) for rho < 0, so small values are not differences of large ones */
    if (rho >= 0.0) return ora_phi(h) * ora_phi(k) + integrate(phi2_integrand, &c, 0.0, asin(rho));
    return lower + integrate(phi2_integrand, &c, -0.5 * ORA_PI, asin(rho));
}

double ora_t2cdf(double h, double k, double rho, double nu)
{
    if (isinf(nu)) return ora_phi2(h, k, rho);
    if (h == -INFINITY || k == -INFINITY) return 0.0;
    if (h == INFINITY) return ora_t1cdf(k, nu);
    if (k == INFINITY) return ora_t1cdf(h, nu);
    if (rho >= 1.0) return ora_t1cdf(h < k ? h : k, nu);
    if (rho <= -1.0) {
        double v = ora_t1cdf(h, nu) + ora_t1cdf(k, nu) - 1.0;
        return v > 0.0 ? v : 0.0;
    }
    t2ctx c = {h, k, rho, nu,
               lgamma(0.5 * (nu + 1.0)) - lgamma(0.5 * nu) - 0.5 * log(nu * ORA_PI),
               lgamma(0.5 * (nu + 1.0) + 0.5) - lgamma(0.5 * (nu + 1.0)) - lgamma(0.5)};
    return integrate(t2_integrand, &c, 0.0, 1.0);
}

/* ------------------------------------------------------------------ */
/* Randomised rank-1 lattice.                                            */
/* ------------------------------------------------------------------ */
double ora_splitmix64_u01(uint64_t key)
{
    /* SplitMix64 (Steele, Lea & Flood 2014), one output from state = key */
    uint64_t z = key + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z ^= z >> 31;
    return (double)(z >> 11) * 0x1.0p-53;
}

double ora_qmc_shift(const ora_qmc* qmc, int m, int d)
{
    uint64_t key = qmc->seed ^ ((uint64_t)(m + 1) << 32) ^ (uint64_t)(d + 1);
    return ora_splitmix64_u01(key);
}

/* generator z_d = a^d mod N */
static uint64_t korobov_z(const ora_qmc* qmc, int d)
{
    uint64_t z = 1, N = (uint64_t)qmc->npoints;
    for (int i = 0; i < d; ++i) z = (z * (uint64_t)qmc->korobov_a) % N;
    return z % N;
}

/* lattice coordinate after the baker's transform: w and 1 - w */
static void lattice_w(const ora_qmc* qmc, int i, int m, int d, double* w, double* wc)
{
    uint64_t N = (uint64_t)qmc->npoints;
    uint64_t r = ((uint64_t)i * korobov_z(qmc, d)) % N;
    double x = (double)r / (double)N + ora_qmc_shift(qmc, m, d);
    x -= floor(x);
    double t = fabs(2.0 * x - 1.0);
    *w = 1.0 - t;
    *wc = t;
}

/* s = sqrt(chi2_nu^{-1}(w_0) / nu) at every lattice point (shift-major). */
static void chi_table(const ora_qmc* qmc, double nu, double* tab)
{
    if (isinf(nu)) {  /* the normal limit: no chi variable, s = 1 */
        for (size_t t = 0; t < (size_t)qmc->npoints * qmc->nshifts; ++t) tab[t] = 1.0;
        return;
    }
    for (int m = 0; m < qmc->nshifts; ++m)
        for (int i = 0; i < qmc->npoints; ++i) {
            double w, wc;
            lattice_w(qmc, i, m, 0, &w, &wc);
            tab[(size_t)m * qmc->npoints + i] = sqrt(ora_chi2_quantile(w, wc, nu) / nu);
        }
}

/* Cholesky factor L (lower, row-major) of an n x n SPD matrix; 0 on success. */
static int chol(int n, const double* A, double* L)
{
    memset(L, 0, sizeof(double) * n * n);
    for (int j = 0; j < n; ++j) {
        double s = A[j * n + j];
        for (int k = 0; k < j; ++k) s -= L[j * n + k] * L[j * n + k];
        if (!(s > 0.0)) return 1;
        L[j * n + j] = sqrt(s);
        for (int i = j + 1; i < n; ++i) {
            double t = A[i * n + j];
            for (int k = 0; k < j; ++k) t -= L[i * n + k] * L[j * n + k];
            L[i * n + j] = t / L[j * n + j];
        }
    }
    return 0;
}

/* Genz separation of variables for T_k(b; 0, V, nu), k >= 3, on the
 * randomised lattice.  stab (shift-major chi table for this nu) may be NULL,
 * in which case the chi quantile is evaluated at every point. */
static double tk_qmc(int k, const double* b, const double* V, double nu,
                     const ora_qmc* qmc, const double* stab, double* se)
{
    double R[ORA_MAXQ * ORA_MAXQ], L[ORA_MAXQ * ORA_MAXQ], bt[ORA_MAXQ], dsc[ORA_MAXQ];
    for (int i = 0; i < k; ++i) dsc[i] = 1.0 / sqrt(V[i * k + i]);
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) R[i * k + j] = V[i * k + j] * dsc[i] * dsc[j];
    for (int i = 0; i < k; ++i) bt[i] = b[i] * dsc[i];
    if (chol(k, R, L)) { if (se) *se = NAN; return NAN; }
    const int N = qmc->npoints, M = qmc->nshifts;
    if (M < 1 || M > 64 || N < 1) { if (se) *se = NAN; return NAN; }
    double shift_mean[64];
    double total = 0.0;
    for (int m = 0; m < M; ++m) {
        double sum = 0.0;
        for (int i = 0; i < N; ++i) {
            double w, wc;
            double s;
            if (stab) s = stab[(size_t)m * N + i];
            else if (isinf(nu)) s = 1.0;
            else { lattice_w(qmc, i, m, 0, &w, &wc); s = sqrt(ora_chi2_quantile(w, wc, nu) / nu); }
            double y[ORA_MAXQ];
            double f = 1.0;
            for (int r = 0; r < k; ++r) {
                double acc = bt[r] * s;
                for (int l = 0; l < r; ++l) acc -= L[r * k + l] * y[l];
                double e = ora_phi(acc / L[r * k + r]);
                if (e <= 1e-300) { f = 0.0; break; }
                f *= e;
                if (r < k - 1) {
                    lattice_w(qmc, i, m, r + 1, &w, &wc);
                    double v = w * e;
                    if (v >= 1.0) v = 1.0 - 0x1.0p-53;
                    y[r] = ora_phi_inv(v);
                }
            }
            sum += f;
        }
        shift_mean[m] = sum / N;
        total += shift_mean[m];
    }
    double mean = total / M;
    if (se) {
        double ss = 0.0;
        for (int m = 0; m < M; ++m) ss += (shift_mean[m] - mean) * (shift_mean[m] - mean);
        *se = M > 1 ? sqrt(ss / (M - 1) / M) : 0.0;
    }
    return mean;
}

/* Truncated moments of X ~ t_k(0, V, nu) given X <= b from one lattice pass.
 * The separation of variables is run to the last coordinate as well
 * (y_k = Phi^{-1}(w_k e_k), lattice dimension k), so every point gives a
 * draw X = diag(V)^{1/2} L y / s inside the truncation region with weight
 * f = prod e_i:  alpha = mean f,  E[X | X <= b] = sum f X / sum f,
 * E[X X^T | X <= b] = sum f X X^T / sum f  (ratio estimators). */
static double tk_moments_qmc(int k, const double* b, const double* V, double nu,
                             const ora_qmc* qmc, const double* stab, double* m1, double* m2)
{
    double R[ORA_MAXQ * ORA_MAXQ], L[ORA_MAXQ * ORA_MAXQ], bt[ORA_MAXQ], dsc[ORA_MAXQ];
    for (int i = 0; i < k; ++i) dsc[i] = 1.0 / sqrt(V[i * k + i]);
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) R[i * k + j] = V[i * k + j] * dsc[i] * dsc[j];
    for (int i = 0; i < k; ++i) bt[i] = b[i] * dsc[i];
    if (chol(k, R, L)) return NAN;
    const int N = qmc->npoints, M = qmc->nshifts;
    double sf = 0.0, sx[ORA_MAXQ], sxx[ORA_MAXQ * ORA_MAXQ];
    memset(sx, 0, sizeof(sx));
    memset(sxx, 0, sizeof(sxx));
    for (int m = 0; m < M; ++m) {
        for (int i = 0; i < N; ++i) {
            double w, wc, s;
            if (stab) s = stab[(size_t)m * N + i];
            else if (isinf(nu)) s = 1.0;
            else { lattice_w(qmc, i, m, 0, &w, &wc); s = sqrt(ora_chi2_quantile(w, wc, nu) / nu); }
            double y[ORA_MAXQ];
            double f = 1.0;
            for (int r = 0; r < k; ++r) {
                double acc = bt[r] * s;
                for (int l = 0; l < r; ++l) acc -= L[r * k + l] * y[l];
                double e = ora_phi(acc / L[r * k + r]);
                if (e <= 1e-300) { f = 0.0; break; }
                f *= e;
                lattice_w(qmc, i, m, r + 1, &w, &wc);
                double v = w * e;
                if (v >= 1.0) v = 1.0 - 0x1.0p-53;
                y[r] = ora_phi_inv(v);
            }
            if (f == 0.0) continue;
            /* X (standardised) = L y / s */
            double x[ORA_MAXQ];
            for (int r = 0; r < k; ++r) {
                double z = 0.0;
                for (int l = 0; l <= r; ++l) z += L[r * k + l] * y[l];
                x[r] = z / s;
            }
            sf += f;
            for (int a = 0; a < k; ++a) {
                sx[a] += f * x[a];
                for (int c2 = 0; c2 < k; ++c2) sxx[a * k + c2] += f * x[a] * x[c2];
            }
        }
    }
    const double alpha = sf / ((double)N * M);
    for (int a = 0; a < k; ++a) {
        m1[a] = sf > 0.0 ? sx[a] / sf / dsc[a] : 0.0;
        for (int c2 = 0; c2 < k; ++c2)
            m2[a * k + c2] = sf > 0.0 ? sxx[a * k + c2] / sf / (dsc[a] * dsc[c2]) : 0.0;
    }
    return alpha;
}

/* The single-pass reading of eqs (13), (16), (17), sharing the lattice pass of alpha_s.
 * Each point of the pass at k1 = nu + p dof carries its chi-square(k1) variate W through
 * s = sqrt(W/k1), which scales the standardised limits of alpha_s.  The chi-square density at
 * k2 = k1 + 2 dof is the one at k1 times w/k1, so weighting every point by s^2 = W/k1 turns
 * the pass into one at k2: the weighted mean is alpha = T_q(c sqrt(k2/(nu+d)); 0, Lambda, k2)
 * of eq (13), and the weighted means of X = diag(S2)^{1/2} L y / s2, s2 = sqrt(W/k2),
 * S2 = ((nu+d)/k2) Lambda, are the moments of the truncated t_q(0, S2, k2) of eqs (16)-(17).
 * The unweighted mean of the same points is alpha_s (eq 4).  Returns alpha; m1 (k) and
 * m2 (k x k) in the units of X.  stab: chi table at k1 dof (optional). */
static double tk_joint_qmc(int k, const double* c, const double* Lam, double nud, double k1,
                           const ora_qmc* qmc, const double* stab, double* m1, double* m2, double* elogw)
{
    const double k2 = k1 + 2.0;
    double R[ORA_MAXQ * ORA_MAXQ], L[ORA_MAXQ * ORA_MAXQ], bt[ORA_MAXQ], dl[ORA_MAXQ];
    for (int i = 0; i < k; ++i) dl[i] = sqrt(Lam[i * k + i]);
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) R[i * k + j] = Lam[i * k + j] / (dl[i] * dl[j]);
    for (int i = 0; i < k; ++i) bt[i] = c[i] * sqrt(k1 / nud) / dl[i];
    if (chol(k, R, L)) return NAN;
    const double ratio = sqrt(k1 / k2);
    const int N = qmc->npoints, M = qmc->nshifts;
    double sw = 0.0, sx[ORA_MAXQ], sxx[ORA_MAXQ * ORA_MAXQ];
    double sf = 0.0, sfl = 0.0;  /* sum f and sum f log(s^2) over the points (elogw) */
    memset(sx, 0, sizeof(sx));
    memset(sxx, 0, sizeof(sxx));
    for (int m = 0; m < M; ++m) {
        for (int i = 0; i < N; ++i) {
            double w, wc, s;
            if (stab) s = stab[(size_t)m * N + i];
            else { lattice_w(qmc, i, m, 0, &w, &wc); s = sqrt(ora_chi2_quantile(w, wc, k1) / k1); }
            double y[ORA_MAXQ];
            double f = 1.0;
            for (int r = 0; r < k; ++r) {
                double acc = bt[r] * s;
                for (int l = 0; l < r; ++l) acc -= L[r * k + l] * y[l];
                double e = ora_phi(acc / L[r * k + r]);
                if (e <= 1e-300) { f = 0.0; break; }
                f *= e;
                lattice_w(qmc, i, m, r + 1, &w, &wc);
                double v = w * e;
                if (v >= 1.0) v = 1.0 - 0x1.0p-53;
                y[r] = ora_phi_inv(v);
            }
            if (f == 0.0) continue;
            if (elogw) {
                /* W = k1 s^2 / nud, so log W = log(s^2) + log(k1/nud) */
                sf += f;
                sfl += f * log(s * s);
            }
            const double fw = f * s * s, s2 = s * ratio;
            double x[ORA_MAXQ];
            for (int r = 0; r < k; ++r) {
                double z = 0.0;
                for (int l = 0; l <= r; ++l) z += L[r * k + l] * y[l];
                x[r] = z / s2;
            }
            sw += fw;
            for (int a = 0; a < k; ++a) {
                sx[a] += fw * x[a];
                for (int c2 = 0; c2 < k; ++c2) sxx[a * k + c2] += fw * x[a] * x[c2];
            }
        }
    }
    const double alpha = sw / ((double)N * M);
    if (elogw) *elogw = sf > 0.0 ? sfl / sf + log(k1 / nud) : NAN;
    for (int a = 0; a < k; ++a) {
        const double sa = sqrt(nud / k2) * dl[a];
        m1[a] = sw > 0.0 ? sx[a] / sw * sa : 0.0;
        for (int c2 = 0; c2 < k; ++c2)
            m2[a * k + c2] = sw > 0.0 ? sxx[a * k + c2] / sw * sa * sqrt(nud / k2) * dl[c2] : 0.0;
    }
    return alpha;
}

double ora_tk_joint(int k, const double* c, const double* Lam, double nud, double k1, const ora_qmc* qmc,
                    double* m1, double* m2)
{
    if (k < 1 || k > ORA_MAXQ || !(k1 > 0.0) || !(nud > 0.0)) return NAN;
    return tk_joint_qmc(k, c, Lam, nud, k1, qmc, NULL, m1, m2, NULL);
}

double ora_tk_moments(int k, const double* b, const double* V, double nu, const ora_qmc* qmc,
                      double* m1, double* m2)
{
    if (k < 1 || k > ORA_MAXQ) return NAN;
    return tk_moments_qmc(k, b, V, nu, qmc, NULL, m1, m2);
}

/* T_k(b; 0, V, nu) dispatcher; stab optional chi table for k >= 3. */
static double tk_any(int k, const double* b, const double* V, double nu,
                     const ora_qmc* qmc, const double* stab, double* se)
{
    if (se) *se = 0.0;
    if (k == 0) return 1.0;
    if (k == 1) return ora_t1cdf(b[0] / sqrt(V[0]), nu);
    if (k == 2) {
        double s0 = sqrt(V[0]), s1 = sqrt(V[3]);
        return ora_t2cdf(b[0] / s0, b[1] / s1, V[1] / (s0 * s1), nu);
    }
    return tk_qmc(k, b, V, nu, qmc, stab, se);
}

double ora_tkcdf(int k, const double* b, const double* V, double nu,
                 const ora_qmc* qmc, double* se)
{
    if (k < 0 || k > ORA_MAXQ) return NAN;
    return tk_any(k, b, V, nu, qmc, NULL, se);
}

/* ------------------------------------------------------------------ */
/* Per-component quantities (definitions under eq (4)).                  */
/* ------------------------------------------------------------------ */
typedef struct {
    int p, q;
    double nu;
    const double* mu;
    const double* Delta;
    double Lo[ORA_MAXP * ORA_MAXP];      /* chol(Omega), Omega = Sigma + Delta Delta^T */
    double logdet;                       /* log |Omega| */
    double Lambda[ORA_MAXQ * ORA_MAXQ];  /* I_q - Delta^T Omega^{-1} Delta */
    double logtp_const;                  /* log of the constant of eq (3) */
    const double* stab[3];               /* chi tables for dof nu+p, nu+p+1, nu+p+2 */
} comp_t;

/* solve L L^T x = r */
static void chol_solve(int n, const double* L, const double* r, double* x)
{
    double z[ORA_MAXP];
    for (int i = 0; i < n; ++i) {
        double s = r[i];
        for (int k = 0; k < i; ++k) s -= L[i * n + k] * z[k];
        z[i] = s / L[i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = z[i];
        for (int k = i + 1; k < n; ++k) s -= L[k * n + i] * x[k];
        x[i] = s / L[i * n + i];
    }
}

static int comp_init(comp_t* C, int p, int q, const double* mu, const double* Sigma,
                     const double* Delta, double nu)
{
    C->p = p; C->q = q; C->nu = nu; C->mu = mu; C->Delta = Delta;
    C->stab[0] = C->stab[1] = C->stab[2] = NULL;
    double Omega[ORA_MAXP * ORA_MAXP];
    for (int i = 0; i < p; ++i)
        for (int j = 0; j < p; ++j) {
            double s = Sigma[i * p + j];
            for (int k = 0; k < q; ++k) s += Delta[i * q + k] * Delta[j * q + k];
            Omega[i * p + j] = s;
        }
    if (chol(p, Omega, C->Lo)) return 1;
    C->logdet = 0.0;
    for (int i = 0; i < p; ++i) C->logdet += 2.0 * log(C->Lo[i * p + i]);
    /* Lambda = I - Delta^T Omega^{-1} Delta */
    double col[ORA_MAXP], sol[ORA_MAXP], OiD[ORA_MAXP * ORA_MAXQ];
    for (int k = 0; k < q; ++k) {
        for (int i = 0; i < p; ++i) col[i] = Delta[i * q + k];
        chol_solve(p, C->Lo, col, sol);
        for (int i = 0; i < p; ++i) OiD[i * q + k] = sol[i];
    }
    for (int a = 0; a < q; ++a)
        for (int b = 0; b < q; ++b) {
            double s = 0.0;
            for (int i = 0; i < p; ++i) s += Delta[i * q + a] * OiD[i * q + b];
            C->Lambda[a * q + b] = (a == b ? 1.0 : 0.0) - s;
        }
    /* eq (3): Gamma((nu+p)/2) / Gamma(nu/2) (nu pi)^{-p/2} |Omega|^{-1/2};
       nu = infinity: the normal density of eq (2), (2 pi)^{-p/2} |Omega|^{-1/2} */
    if (isinf(nu)) C->logtp_const = -0.5 * p * log(2.0 * ORA_PI) - 0.5 * C->logdet;
    else C->logtp_const = lgamma(0.5 * (nu + p)) - lgamma(0.5 * nu)
                        - 0.5 * p * log(nu * ORA_PI) - 0.5 * C->logdet;
    return 0;
}

/* density of the univariate t with location 0, scale^2 v, dof nu at x */
static double t1pdf_scaled(double x, double v, double nu)
{
    return ora_t1pdf(x / sqrt(v), nu) / sqrt(v);
}

/* Drop coordinate r: conditional location coefficient and Schur complement
 * of a t law with scale S (dimension k) given X_r = x_r.
 * Out: mvec (k-1) = S_{-r,r}/S_rr, schur ((k-1)x(k-1)). */
static void condition_on(int k, const double* S, int r, double* mvec, double* schur)
{
    int ii = 0;
    for (int i = 0; i < k; ++i) {
        if (i == r) continue;
        mvec[ii] = S[i * k + r] / S[r * k + r];
        int jj = 0;
        for (int j = 0; j < k; ++j) {
            if (j == r) continue;
            schur[ii * (k - 1) + jj] = S[i * k + j] - S[i * k + r] * S[r * k + j] / S[r * k + r];
            ++jj;
        }
        ++ii;
    }
}

/* A pair whose T_q is 0 in FP64 (the observation lies beyond the range of the arithmetic
 * on this component's skewing side): log f = -inf there, so tau = 0 (eq 12), and the
 * conditional expectations, which enter eqs (18)-(22) only multiplied by tau, are set to
 * u = 1, E[log w] = 0, e2 = 0, e3 = 0 instead of the 0/0 of eqs (13)-(17). */
static int pair_null(int q, int density_only, double* u_out, double* elogu_out, double* eu, double* euu)
{
    if (density_only) return 0;
    *u_out = 1.0;
    *elogu_out = 0.0;
    for (int a = 0; a < q; ++a) eu[a] = 0.0;
    for (int a = 0; a < q * q; ++a) euu[a] = 0.0;
    return 0;
}

/* One (observation, component) pair: eqs (3), (4), (13), (15), (16), (17). */
/* The pair quantities of the nu -> infinity limit, the CFUSN model of eq (5):
 * f = 2^q phi_p(y; mu, Omega) Phi_q(c; 0, Lambda); the latent scale W is 1, so u = 1
 * (eq 13), eq (15) is not needed (no nu step), and eqs (16)-(17) are the moments of
 * U = c - X with X ~ N_q(0, Lambda) truncated to X <= c.  Every scaling of the t case
 * ((nu+d)/(nu+p), the conditional-scale factors, nu/(nu-2)) is 1 here. */
static int pair_core_normal(const comp_t* C, const ora_qmc* qmc, const double* y, int density_only,
                            double* logf, double* u_out, double* elogu_out, double* eu,
                            double* euu, double* se_out)
{
    const int p = C->p, q = C->q;
    const double inf = INFINITY;
    double r[ORA_MAXP], Oir[ORA_MAXP];
    for (int i = 0; i < p; ++i) r[i] = y[i] - C->mu[i];
    chol_solve(p, C->Lo, r, Oir);
    double d = 0.0;
    for (int i = 0; i < p; ++i) d += r[i] * Oir[i];
    double c[ORA_MAXQ];
    for (int k = 0; k < q; ++k) {
        double sum = 0.0;
        for (int i = 0; i < p; ++i) sum += C->Delta[i * q + k] * Oir[i];
        c[k] = sum;
    }
    /* eq (5): log 2^q + log phi_p(y; mu, Omega) + log Phi_q(c; 0, Lambda) */
    double se_a = 0.0;
    const double alpha = tk_any(q, c, C->Lambda, inf, qmc, C->stab[0], &se_a);
    *logf = q * log(2.0) + C->logtp_const - 0.5 * d + log(alpha);
    if (se_out) *se_out = se_a;
    if (!(alpha > 0.0)) return pair_null(q, density_only, u_out, elogu_out, eu, euu);
    if (density_only) return 0;
    *u_out = 1.0;
    *elogu_out = 0.0;
    if (qmc->moments && q >= 3) {
        double m1[ORA_MAXQ], m2[ORA_MAXQ * ORA_MAXQ];
        tk_moments_qmc(q, c, C->Lambda, inf, qmc, C->stab[2], m1, m2);
        for (int a = 0; a < q; ++a) eu[a] = c[a] - m1[a];
        for (int a = 0; a < q; ++a)
            for (int bb = 0; bb < q; ++bb)
                euu[a * q + bb] = c[a] * c[bb] - c[a] * m1[bb] - m1[a] * c[bb]
                                + 0.5 * (m2[a * q + bb] + m2[bb * q + a]);
        return 0;
    }
    /* x phi(x; S) = -S grad phi(x; S): E[X 1(X <= c)] = -Lambda xi with
     * xi_r = phi_1(c_r; Lambda_rr) Phi_{q-1}(c_{-r} - m_r c_r; V_r) */
    const double* S = C->Lambda;
    double xi[ORA_MAXQ], H[ORA_MAXQ * ORA_MAXQ];
    memset(H, 0, sizeof(H));
    for (int rr = 0; rr < q; ++rr) {
        const int k1 = q - 1;
        double mvec[ORA_MAXQ], Vr[ORA_MAXQ * ORA_MAXQ], cp[ORA_MAXQ], mr[ORA_MAXQ];
        double tq1 = 1.0;
        if (k1 > 0) {
            condition_on(q, S, rr, mvec, Vr);
            int ii = 0;
            for (int i = 0; i < q; ++i) {
                if (i == rr) continue;
                mr[ii] = mvec[ii] * c[rr];
                cp[ii] = c[i] - mr[ii];
                ++ii;
            }
            tq1 = tk_any(k1, cp, Vr, inf, qmc, C->stab[1], NULL);
        }
        xi[rr] = t1pdf_scaled(c[rr], S[rr * q + rr], inf) * tq1;
        H[rr * q + rr] = c[rr] * xi[rr];
        if (k1 == 0 || xi[rr] == 0.0) continue;
        /* E[X_{-r} | X_r = c_r, X_{-r} <= c_{-r}] = m_r + E[Y | Y <= c'], Y ~ N(0, V_r) */
        double xip[ORA_MAXQ];
        for (int s2 = 0; s2 < k1; ++s2) {
            const int k2 = k1 - 1;
            double tq2 = 1.0;
            if (k2 > 0) {
                double mv2[ORA_MAXQ], Vs[ORA_MAXQ * ORA_MAXQ], cpp[ORA_MAXQ];
                condition_on(k1, Vr, s2, mv2, Vs);
                int ii = 0;
                for (int i = 0; i < k1; ++i) {
                    if (i == s2) continue;
                    cpp[ii] = cp[i] - mv2[ii] * cp[s2];
                    ++ii;
                }
                tq2 = tk_any(k2, cpp, Vs, inf, qmc, C->stab[0], NULL);
            }
            xip[s2] = t1pdf_scaled(cp[s2], Vr[s2 * k1 + s2], inf) * tq2;
        }
        int ii = 0;
        for (int bcol = 0; bcol < q; ++bcol) {
            if (bcol == rr) continue;
            double ey = 0.0;
            for (int s2 = 0; s2 < k1; ++s2) ey += Vr[ii * k1 + s2] * xip[s2];
            H[rr * q + bcol] = xi[rr] * (mr[ii] - ey / tq1);
            ++ii;
        }
    }
    /* e2 = c + Lambda xi / alpha; e3 = c c^T + c (Lambda xi)^T/alpha + (Lambda xi) c^T/alpha
     * + Lambda - Lambda H / alpha */
    double Lxi[ORA_MAXQ];
    for (int a = 0; a < q; ++a) {
        double sum = 0.0;
        for (int k = 0; k < q; ++k) sum += S[a * q + k] * xi[k];
        Lxi[a] = sum;
        eu[a] = c[a] + sum / alpha;
    }
    double E3[ORA_MAXQ * ORA_MAXQ];
    for (int a = 0; a < q; ++a)
        for (int bb = 0; bb < q; ++bb) {
            double LH = 0.0;
            for (int k = 0; k < q; ++k) LH += S[a * q + k] * H[k * q + bb];
            E3[a * q + bb] = c[a] * c[bb] + (c[a] * Lxi[bb] + Lxi[a] * c[bb]) / alpha
                           + S[a * q + bb] - LH / alpha;
        }
    for (int a = 0; a < q; ++a)
        for (int bb = 0; bb < q; ++bb)
            euu[a * q + bb] = 0.5 * (E3[a * q + bb] + E3[bb * q + a]);
    return 0;
}

static int pair_core(const comp_t* C, const ora_qmc* qmc, const double* y, int density_only,
                     double* logf, double* u_out, double* elogu_out, double* eu,
                     double* euu, double* se_out)
{
    if (isinf(C->nu))
        return pair_core_normal(C, qmc, y, density_only, logf, u_out, elogu_out, eu, euu, se_out);
    const int p = C->p, q = C->q;
    const double nu = C->nu;
    double r[ORA_MAXP], Oir[ORA_MAXP];
    for (int i = 0; i < p; ++i) r[i] = y[i] - C->mu[i];
    chol_solve(p, C->Lo, r, Oir);
    /* d(y) = (y-mu)^T Omega^{-1} (y-mu);  c(y) = Delta^T Omega^{-1} (y-mu) */
    double d = 0.0;
    for (int i = 0; i < p; ++i) d += r[i] * Oir[i];
    double c[ORA_MAXQ];
    for (int k = 0; k < q; ++k) {
        double s = 0.0;
        for (int i = 0; i < p; ++i) s += C->Delta[i * q + k] * Oir[i];
        c[k] = s;
    }
    /* eq (3) corrected: log t_p(y; mu, Omega, nu) */
    double logtp = C->logtp_const - 0.5 * (nu + p) * log1p(d / nu);
    /* eq (4): T_q(c sqrt((nu+p)/(nu+d)); 0, Lambda, nu+p) */
    double b[ORA_MAXQ], se_s = 0.0;
    double fs = sqrt((nu + p) / (nu + d));
    for (int k = 0; k < q; ++k) b[k] = c[k] * fs;
    double alpha_s = tk_any(q, b, C->Lambda, nu + p, qmc, C->stab[0], &se_s);
    *logf = q * log(2.0) + logtp + log(alpha_s);
    if (se_out) *se_out = se_s;
    if (!(alpha_s > 0.0)) return pair_null(q, density_only, u_out, elogu_out, eu, euu);
    if (density_only) return 0;

    if (qmc->moments && q >= 3) {
        /* eqs (13), (16), (17) from the lattice pass of alpha_s (points weighted by W/(nu+p)):
         * X ~ t_q(0, S2, nu+p+2), S2 = ((nu+d)/(nu+p+2)) Lambda, truncated to X <= c; U = c - X. */
        double m1[ORA_MAXQ], m2[ORA_MAXQ * ORA_MAXQ], ew = NAN;
        const int exact = qmc->elogw && !isinf(nu);
        double alpha = tk_joint_qmc(q, c, C->Lambda, nu + d, nu + p, qmc, C->stab[0], m1, m2, exact ? &ew : NULL);
        double u = (nu + p) / (nu + d) * alpha / alpha_s;
        *u_out = u;
        /* eq (15) (one-step-late), or the exact E[log W | y] of the same pass */
        *elogu_out = exact ? ew : u - log(0.5 * (nu + d)) - (nu + p) / (nu + d) + ora_digamma(0.5 * (nu + p));
        for (int a = 0; a < q; ++a) eu[a] = u * (c[a] - m1[a]);
        for (int a = 0; a < q; ++a)
            for (int bb = 0; bb < q; ++bb) {
                double e3 = c[a] * c[bb] - c[a] * m1[bb] - m1[a] * c[bb]
                          + 0.5 * (m2[a * q + bb] + m2[bb * q + a]);
                euu[a * q + bb] = u * e3;
            }
        return 0;
    }
    /* eq (13): u = ((nu+p)/(nu+d)) T_q(c sqrt((nu+p+2)/(nu+d)); Lambda, nu+p+2) / alpha_s */
    double f2 = sqrt((nu + p + 2.0) / (nu + d));
    for (int k = 0; k < q; ++k) b[k] = c[k] * f2;
    double alpha = tk_any(q, b, C->Lambda, nu + p + 2.0, qmc, C->stab[2], NULL);
    double u = (nu + p) / (nu + d) * alpha / alpha_s;
    /* eq (15): one-step-late E[log W] */
    double elogu = u - log(0.5 * (nu + d)) - (nu + p) / (nu + d) + ora_digamma(0.5 * (nu + p));
    *u_out = u;
    *elogu_out = elogu;

    /* eqs (16)-(17): moments of the truncated t.  S = ((nu+d)/(nu+p)) Lambda
     * is the scale of the t law whose CDF at c is alpha_s. */
    const double nu1 = nu + p;
    double S[ORA_MAXQ * ORA_MAXQ];
    for (int i = 0; i < q * q; ++i) S[i] = (nu + d) / nu1 * C->Lambda[i];
    double xi[ORA_MAXQ], H[ORA_MAXQ * ORA_MAXQ];
    memset(H, 0, sizeof(H));
    for (int rr = 0; rr < q; ++rr) {
        const int k1 = q - 1;
        double mvec[ORA_MAXQ], Vr[ORA_MAXQ * ORA_MAXQ], cp[ORA_MAXQ], mr[ORA_MAXQ];
        double tq1 = 1.0;
        if (k1 > 0) {
            condition_on(q, S, rr, mvec, Vr);
            double scal = (nu1 + c[rr] * c[rr] / S[rr * q + rr]) / (nu1 + 1.0);
            for (int i = 0; i < k1 * k1; ++i) Vr[i] *= scal;
            int ii = 0;
            for (int i = 0; i < q; ++i) {
                if (i == rr) continue;
                mr[ii] = mvec[ii] * c[rr];
                cp[ii] = c[i] - mr[ii];
                ++ii;
            }
            tq1 = tk_any(k1, cp, Vr, nu1 + 1.0, qmc, C->stab[1], NULL);
        }
        /* xi_r = t_1(c_r; 0, S_rr, nu+p) T_{q-1}(c_{-r} - m_r; 0, V_r, nu+p+1) */
        xi[rr] = t1pdf_scaled(c[rr], S[rr * q + rr], nu1) * tq1;
        H[rr * q + rr] = c[rr] * xi[rr];
        if (k1 == 0 || xi[rr] == 0.0) continue;
        /* E[X_{-r} | X_r = c_r, X_{-r} <= c_{-r}] = m_r + E[Y | Y <= c'],
         * Y ~ t_{q-1}(0, V_r, nu2), nu2 = nu+p+1; E[Y 1(Y<=c')] = -(nu2/(nu2-2)) V_r xi'. */
        const double nu2 = nu1 + 1.0;
        double Vp[ORA_MAXQ * ORA_MAXQ], xip[ORA_MAXQ];
        for (int i = 0; i < k1 * k1; ++i) Vp[i] = nu2 * Vr[i] / (nu2 - 2.0);
        for (int s = 0; s < k1; ++s) {
            const int k2 = k1 - 1;
            double tq2 = 1.0;
            if (k2 > 0) {
                double mv2[ORA_MAXQ], Vs[ORA_MAXQ * ORA_MAXQ], cpp[ORA_MAXQ];
                condition_on(k1, Vp, s, mv2, Vs);
                double scal2 = (nu2 - 2.0 + cp[s] * cp[s] / Vp[s * k1 + s]) / (nu2 - 1.0);
                for (int i = 0; i < k2 * k2; ++i) Vs[i] *= scal2;
                int ii = 0;
                for (int i = 0; i < k1; ++i) {
                    if (i == s) continue;
                    cpp[ii] = cp[i] - mv2[ii] * cp[s];
                    ++ii;
                }
                tq2 = tk_any(k2, cpp, Vs, nu2 - 1.0, qmc, C->stab[0], NULL);
            }
            xip[s] = t1pdf_scaled(cp[s], Vp[s * k1 + s], nu2 - 2.0) * tq2;
        }
        int ii = 0;
        for (int bcol = 0; bcol < q; ++bcol) {
            if (bcol == rr) continue;
            double ey = 0.0;
            for (int s = 0; s < k1; ++s) ey += Vr[ii * k1 + s] * xip[s];
            ey = -(nu2 / (nu2 - 2.0)) * ey / tq1;
            H[rr * q + bcol] = xi[rr] * (mr[ii] + ey);
            ++ii;
        }
    }
    /* e2 = u c + Lambda xi / alpha_s */
    double Lxi[ORA_MAXQ];
    for (int a = 0; a < q; ++a) {
        double s = 0.0;
        for (int k = 0; k < q; ++k) s += C->Lambda[a * q + k] * xi[k];
        Lxi[a] = s;
        eu[a] = u * c[a] + s / alpha_s;
    }
    /* e3 = u c c^T + c (Lambda xi)^T/alpha_s + (Lambda xi) c^T/alpha_s + Lambda - Lambda H/alpha_s */
    double E3[ORA_MAXQ * ORA_MAXQ];
    for (int a = 0; a < q; ++a)
        for (int bb = 0; bb < q; ++bb) {
            double LH = 0.0;
            for (int k = 0; k < q; ++k) LH += C->Lambda[a * q + k] * H[k * q + bb];
            E3[a * q + bb] = u * c[a] * c[bb] + (c[a] * Lxi[bb] + Lxi[a] * c[bb]) / alpha_s
                           + C->Lambda[a * q + bb] - LH / alpha_s;
        }
    for (int a = 0; a < q; ++a)
        for (int bb = 0; bb < q; ++bb)
            euu[a * q + bb] = 0.5 * (E3[a * q + bb] + E3[bb * q + a]);
    return 0;
}

int ora_pair(int p, int q, const double* y, const double* mu, const double* Sigma,
             const double* Delta, double nu, const ora_qmc* qmc, double* logf,
             double* u, double* elogu, double* eu, double* euu, double* se_alpha_s)
{
    if (p < 1 || p > ORA_MAXP || q < 1 || q > ORA_MAXQ) return 1;
    comp_t C;
    if (comp_init(&C, p, q, mu, Sigma, Delta, nu)) return 2;
    return pair_core(&C, qmc, y, 0, logf, u, elogu, eu, euu, se_alpha_s);
}

/* ------------------------------------------------------------------ */
/* E-step over all pairs (eqs 12-17) and the log-likelihood (eq 27).    */
/* ------------------------------------------------------------------ */
static int estep_impl(int n, int p, int q, int g, const double* y, const double* pi,
                      const double* mu, const double* Sigma, const double* Delta,
                      const double* nu, const ora_qmc* qmc, int nthreads, int density_only,
                      double* logf, double* tau, double* u, double* elogu, double* eu,
                      double* euu, double* se, double* loglik)
{
    if (p < 1 || p > ORA_MAXP || q < 1 || q > ORA_MAXQ || g < 1 || n < 0) return 1;
    comp_t* C = (comp_t*)malloc(sizeof(comp_t) * g);
    double* tabs = NULL;
    const size_t NM = (size_t)qmc->npoints * qmc->nshifts;
    int need_tabs = q >= 3;
    if (need_tabs) tabs = (double*)malloc(sizeof(double) * NM * 3 * g);
    for (int h = 0; h < g; ++h) {
        if (comp_init(&C[h], p, q, mu + (size_t)h * p, Sigma + (size_t)h * p * p,
                      Delta + (size_t)h * p * q, nu[h])) {
            free(C); free(tabs); return 2 + h;
        }
    }
    if (need_tabs) {
        #pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
        for (int t = 0; t < 3 * g; ++t) {
            int h = t / 3, k = t % 3;
            chi_table(qmc, nu[h] + p + k, tabs + NM * t);
        }
        for (int h = 0; h < g; ++h)
            for (int k = 0; k < 3; ++k) C[h].stab[k] = tabs + NM * (3 * h + k);
    }
    double* lf = (double*)malloc(sizeof(double) * (size_t)n * g);
    double* lj = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    int err = 0;
    #pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads)
    for (int j = 0; j < n; ++j) {
        for (int h = 0; h < g; ++h) {
            size_t idx = (size_t)h * n + j;
            double lfv, uv = 0, ev = 0, sev = 0;
            double euv[ORA_MAXQ], euuv[ORA_MAXQ * ORA_MAXQ];
            pair_core(&C[h], qmc, y + (size_t)j * p, density_only, &lfv, &uv, &ev, euv,
                      euuv, &sev);
            lf[idx] = lfv;
            if (logf) logf[idx] = lfv;
            if (se) se[idx] = sev;
            if (!density_only) {
                if (u) u[idx] = uv;
                if (elogu) elogu[idx] = ev;
                if (eu) memcpy(eu + idx * q, euv, sizeof(double) * q);
                if (euu) memcpy(euu + idx * q * q, euuv, sizeof(double) * q * q);
            }
        }
        /* eq (12) via log-sum-exp; the denominator is f(y_j; Psi) of eq (27) */
        double mx = -INFINITY;
        for (int h = 0; h < g; ++h) {
            double v = log(pi[h]) + lf[(size_t)h * n + j];
            if (v > mx) mx = v;
        }
        double s = 0.0;
        for (int h = 0; h < g; ++h) s += exp(log(pi[h]) + lf[(size_t)h * n + j] - mx);
        lj[j] = mx + log(s);
        if (tau)
            for (int h = 0; h < g; ++h)
                tau[(size_t)h * n + j] = exp(log(pi[h]) + lf[(size_t)h * n + j] - mx) / s;
    }
    double L = 0.0;
    for (int j = 0; j < n; ++j) L += lj[j];
    if (loglik) *loglik = L;
    if (!isfinite(L)) err = 100;
    free(lf); free(lj); free(C); free(tabs);
    return err;
}

int ora_estep(int n, int p, int q, int g, const double* y, const double* pi,
              const double* mu, const double* Sigma, const double* Delta, const double* nu,
              const ora_qmc* qmc, int nthreads, double* logf, double* tau, double* u,
              double* elogu, double* eu, double* euu, double* se, double* loglik)
{
    return estep_impl(n, p, q, g, y, pi, mu, Sigma, Delta, nu, qmc, nthreads, 0, logf, tau,
                      u, elogu, eu, euu, se, loglik);
}

int ora_loglik(int n, int p, int q, int g, const double* y, const double* pi,
               const double* mu, const double* Sigma, const double* Delta, const double* nu,
               const ora_qmc* qmc, int nthreads, double* loglik)
{
    return estep_impl(n, p, q, g, y, pi, mu, Sigma, Delta, nu, qmc, nthreads, 1, NULL, NULL,
                      NULL, NULL, NULL, NULL, NULL, loglik);
}

/* ------------------------------------------------------------------ */
/* M-step (eqs 18-22).                                                   */
/* ------------------------------------------------------------------ */
double ora_nu_root(double n_h, double s_h, double nu_min, double nu_max, int* flag)
{
    /* F(nu) = n_h [log(nu/2) - psi(nu/2) + 1] + s_h, decreasing in nu */
#define ORA_NUF(v) (n_h * (log(0.5 * (v)) - ora_digamma(0.5 * (v)) + 1.0) + s_h)
    double flo = ORA_NUF(nu_min), fhi = ORA_NUF(nu_max);
    if (flag) *flag = 0;
    if (!(flo > 0.0)) { if (flag) *flag = -1; return nu_min; }
    if (!(fhi < 0.0)) { if (flag) *flag = 1; return nu_max; }
    double lo = nu_min, hi = nu_max;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        double fm = ORA_NUF(mid);
        if (fm > 0.0) lo = mid; else hi = mid;
        if (hi - lo <= 1e-14 * mid) break;
    }
#undef ORA_NUF
    return 0.5 * (lo + hi);
}

int ora_mstep(int n, int p, int q, int g, const double* y, const double* tau,
              const double* u, const double* elogu, const double* eu, const double* euu,
              double nu_min, double nu_max, double* pi, double* mu, double* Sigma,
              double* Delta, double* nu, int* nu_flag)
{
    return ora_mstep_hold(n, p, q, g, y, tau, u, elogu, eu, euu, nu_min, nu_max, pi, mu, Sigma,
                          Delta, nu, nu_flag, 0);
}

int ora_mstep_hold(int n, int p, int q, int g, const double* y, const double* tau,
                   const double* u, const double* elogu, const double* eu, const double* euu,
                   double nu_min, double nu_max, double* pi, double* mu, double* Sigma,
                   double* Delta, double* nu, int* nu_flag, int hold)
{
    if (p < 1 || p > ORA_MAXP || q < 1 || q > ORA_MAXQ) return -1;
    for (int h = 0; h < g; ++h) {
        const double* th = tau + (size_t)h * n;
        const double* uh = u + (size_t)h * n;
        const double* lh = elogu + (size_t)h * n;
        const double* e2 = eu + (size_t)h * n * q;
        const double* e3 = euu + (size_t)h * n * q * q;
        double* muh = mu + (size_t)h * p;
        double* Sh = Sigma + (size_t)h * p * p;
        double* Dh = Delta + (size_t)h * p * q;
        /* eq (18) */
        double N = 0.0;
        for (int j = 0; j < n; ++j) N += th[j];
        if (!(N > 0.0)) return 1 + h;
        pi[h] = N / n;
        /* eq (19), with Delta^(k) */
        double stu = 0.0, stuy[ORA_MAXP], ste[ORA_MAXQ];
        memset(stuy, 0, sizeof(stuy)); memset(ste, 0, sizeof(ste));
        for (int j = 0; j < n; ++j) {
            stu += th[j] * uh[j];
            for (int i = 0; i < p; ++i) stuy[i] += th[j] * uh[j] * y[(size_t)j * p + i];
            for (int k = 0; k < q; ++k) ste[k] += th[j] * e2[(size_t)j * q + k];
        }
        double mun[ORA_MAXP];
        for (int i = 0; i < p; ++i) {
            double s = stuy[i];
            for (int k = 0; k < q; ++k) s -= Dh[i * q + k] * ste[k];
            mun[i] = s / stu;
        }
        /* eq (20), with mu^(k+1) */
        double A[ORA_MAXP * ORA_MAXQ], B[ORA_MAXQ * ORA_MAXQ], LB[ORA_MAXQ * ORA_MAXQ];
        memset(A, 0, sizeof(A)); memset(B, 0, sizeof(B));
        for (int j = 0; j < n; ++j) {
            for (int i = 0; i < p; ++i)
                for (int k = 0; k < q; ++k)
                    A[i * q + k] += th[j] * (y[(size_t)j * p + i] - mun[i]) * e2[(size_t)j * q + k];
            for (int a = 0; a < q * q; ++a) B[a] += th[j] * e3[(size_t)j * q * q + a];
        }
        double Dn[ORA_MAXP * ORA_MAXQ];
        if (hold & ORA_HOLD_DELTA) {
            /* Delta held at Delta^(k): eq (21) below uses it in place of Delta^(k+1) */
            memcpy(Dn, Dh, sizeof(double) * p * q);
        } else {
        if (chol(q, B, LB)) return 1 + h;
        for (int i = 0; i < p; ++i) {
            /* row i of A B^{-1}: solve B x = A_i^T (B symmetric) */
            double rhs[ORA_MAXQ], sol[ORA_MAXQ];
            for (int k = 0; k < q; ++k) rhs[k] = A[i * q + k];
            chol_solve(q, LB, rhs, sol);
            for (int k = 0; k < q; ++k) Dn[i * q + k] = sol[k];
        }
        }
        /* eq (21), with mu^(k+1) and Delta^(k+1) */
        double Sn[ORA_MAXP * ORA_MAXP];
        memset(Sn, 0, sizeof(Sn));
        for (int j = 0; j < n; ++j) {
            double rr[ORA_MAXP], De2[ORA_MAXP], De3D[ORA_MAXP * ORA_MAXP];
            for (int i = 0; i < p; ++i) rr[i] = y[(size_t)j * p + i] - mun[i];
            for (int i = 0; i < p; ++i) {
                double s = 0.0;
                for (int k = 0; k < q; ++k) s += Dn[i * q + k] * e2[(size_t)j * q + k];
                De2[i] = s;
            }
            for (int i = 0; i < p; ++i)
                for (int l = 0; l < p; ++l) {
                    double s = 0.0;
                    for (int a = 0; a < q; ++a)
                        for (int b = 0; b < q; ++b)
                            s += Dn[i * q + a] * e3[(size_t)j * q * q + b * q + a] * Dn[l * q + b];
                    De3D[i * p + l] = s;
                }
            for (int i = 0; i < p; ++i)
                for (int l = 0; l < p; ++l)
                    Sn[i * p + l] += th[j] * (uh[j] * rr[i] * rr[l] - De2[i] * rr[l]
                                              - rr[i] * De2[l] + De3D[i * p + l]);
        }
        for (int i = 0; i < p; ++i)
            for (int l = 0; l < p; ++l) Sn[i * p + l] /= N;
        for (int i = 0; i < p; ++i)
            for (int l = i + 1; l < p; ++l) {
                double s = 0.5 * (Sn[i * p + l] + Sn[l * p + i]);
                Sn[i * p + l] = Sn[l * p + i] = s;
            }
        double LS[ORA_MAXP * ORA_MAXP];
        if (chol(p, Sn, LS)) return 1 + h;
        /* eq (22) */
        double snu = 0.0;
        for (int j = 0; j < n; ++j) snu += th[j] * (lh[j] - uh[j]);
        int fl = 0;
        double nun = (hold & ORA_HOLD_NU) ? nu[h] : ora_nu_root(N, snu, nu_min, nu_max, &fl);
        if (nu_flag) nu_flag[h] = fl;
        memcpy(muh, mun, sizeof(double) * p);
        memcpy(Dh, Dn, sizeof(double) * p * q);
        memcpy(Sh, Sn, sizeof(double) * p * p);
        nu[h] = nun;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Aitken rule (eqs 24-26) and the EM loop.                              */
/* ------------------------------------------------------------------ */
int ora_aitken_converged(double l_km1, double l_k, double l_kp1, double eps, double* l_inf)
{
    double den = l_k - l_km1;
    if (den == 0.0) { if (l_inf) *l_inf = l_kp1; return 1; }
    double a = (l_kp1 - l_k) / den;                       /* eq (26) */
    double linf = l_k + (l_kp1 - l_k) / (1.0 - a);        /* eq (25) */
    if (l_inf) *l_inf = linf;
    return fabs(linf - l_kp1) < eps;                      /* eq (24) */
}

int ora_fit(int n, int p, int q, int g, const double* y, double* pi, double* mu,
            double* Sigma, double* Delta, double* nu, const ora_qmc* qmc, int max_iter,
            double tol, double nu_min, double nu_max, int nthreads, int* iters_done,
            double* loglik_hist)
{
    return ora_fit_hold(n, p, q, g, y, pi, mu, Sigma, Delta, nu, qmc, max_iter, tol, nu_min, nu_max,
                        nthreads, iters_done, loglik_hist, 0);
}

int ora_fit_hold(int n, int p, int q, int g, const double* y, double* pi, double* mu,
            double* Sigma, double* Delta, double* nu, const ora_qmc* qmc, int max_iter,
            double tol, double nu_min, double nu_max, int nthreads, int* iters_done,
            double* loglik_hist, int hold)
{
    size_t ng = (size_t)n * g;
    double* tau = (double*)malloc(sizeof(double) * ng);
    double* u = (double*)malloc(sizeof(double) * ng);
    double* el = (double*)malloc(sizeof(double) * ng);
    double* eu = (double*)malloc(sizeof(double) * ng * q);
    double* euu = (double*)malloc(sizeof(double) * ng * q * q);
    int rc = 0, it;
    for (it = 0; it < max_iter; ++it) {
        double L;
        rc = ora_estep(n, p, q, g, y, pi, mu, Sigma, Delta, nu, qmc, nthreads, NULL, tau, u,
                       el, eu, euu, NULL, &L);
        if (rc) break;
        if (loglik_hist) loglik_hist[it] = L;
        if (tol > 0.0 && it >= 2 && loglik_hist &&
            ora_aitken_converged(loglik_hist[it - 2], loglik_hist[it - 1], L, tol, NULL))
            break;
        rc = ora_mstep_hold(n, p, q, g, y, tau, u, el, eu, euu, nu_min, nu_max, pi, mu, Sigma,
                            Delta, nu, NULL, hold);
        if (rc) break;
    }
    if (!rc && it == max_iter) {
        double L;
        rc = ora_loglik(n, p, q, g, y, pi, mu, Sigma, Delta, nu, qmc, nthreads, &L);
        if (loglik_hist) loglik_hist[max_iter] = L;
    }
    if (iters_done) *iters_done = it;
    free(tau); free(u); free(el); free(eu); free(euu);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Initialisation: Algorithm 1 with the moment starts of eq (23)       */
/* (Sec. 3.3).                                                          */
/* ------------------------------------------------------------------ */
void ora_random_partition(int n, int g, uint64_t seed, int start, int* labels)
{
    /* one SplitMix64 draw per observation, label = floor(u g) */
    for (int j = 0; j < n; ++j) {
        uint64_t key = seed ^ ((uint64_t)(start + 1) << 40) ^ (uint64_t)(j + 1);
        int h = (int)(ora_splitmix64_u01(key) * g);
        labels[j] = h < g ? h : g - 1;
    }
}

int ora_kmeans(int n, int p, int g, const double* y, int nstarts, uint64_t seed, int max_iter,
               int* labels, int* iters, double* centres)
{
    if (n < g) return 1;
    double* c = (double*)malloc(sizeof(double) * (size_t)g * p);
    double* sum = (double*)malloc(sizeof(double) * (size_t)g * p);
    long* cnt = (long*)malloc(sizeof(long) * (size_t)g);
    int* idx = (int*)malloc(sizeof(int) * (size_t)g);
    for (int s = 0; s < nstarts; ++s) {
        int* lab = labels + (size_t)s * n;
        /* starting centres: g distinct observations */
        for (int h = 0; h < g; ++h) {
            for (uint64_t a = 0;; ++a) {
                uint64_t key = seed ^ ((uint64_t)(s + 1) << 40) ^ ((uint64_t)1 << 36) ^ (uint64_t)(h + 1 + (uint64_t)g * a);
                int j = (int)(ora_splitmix64_u01(key) * n);
                if (j > n - 1) j = n - 1;
                int dup = 0;
                for (int l = 0; l < h; ++l) dup |= idx[l] == j;
                if (!dup) { idx[h] = j; break; }
            }
            for (int d = 0; d < p; ++d) c[(size_t)h * p + d] = y[(size_t)idx[h] * p + d];
        }
        for (int j = 0; j < n; ++j) lab[j] = -1;
        int it = 0;
        while (it < max_iter) {
            /* assignment */
            long changes = 0;
            for (int j = 0; j < n; ++j) {
                double best = INFINITY;
                int hb = 0;
                for (int h = 0; h < g; ++h) {
                    double dist = 0.0;
                    for (int d = 0; d < p; ++d) {
                        double t = y[(size_t)j * p + d] - c[(size_t)h * p + d];
                        dist += t * t;
                    }
                    if (dist < best) { best = dist; hb = h; }
                }
                if (lab[j] != hb) { ++changes; lab[j] = hb; }
            }
            ++it;
            if (changes == 0 || it == max_iter) break;
            /* update: cluster means */
            for (int t = 0; t < g * p; ++t) sum[t] = 0.0;
            for (int h = 0; h < g; ++h) cnt[h] = 0;
            for (int j = 0; j < n; ++j) {
                ++cnt[lab[j]];
                for (int d = 0; d < p; ++d) sum[(size_t)lab[j] * p + d] += y[(size_t)j * p + d];
            }
            for (int h = 0; h < g; ++h)
                if (cnt[h] > 0)
                    for (int d = 0; d < p; ++d) c[(size_t)h * p + d] = sum[(size_t)h * p + d] / (double)cnt[h];
        }
        if (iters) iters[s] = it;
        if (centres) memcpy(centres + (size_t)s * g * p, c, sizeof(double) * (size_t)g * p);
    }
    free(c); free(sum); free(cnt); free(idx);
    return 0;
}

int ora_moment_start(int n, int p, int q, int g, const double* y, const int* labels,
                     double alpha, double nu0, double* pi, double* mu, double* Sigma,
                     double* Delta, double* nu)
{
    const double PI = 3.14159265358979323846;
    double* ybar = (double*)calloc((size_t)p, sizeof(double));
    double* S = (double*)calloc((size_t)p * p, sizeof(double));
    double* m3 = (double*)calloc((size_t)p, sizeof(double));
    double* L = (double*)malloc(sizeof(double) * p * p);
    int rc = 0;
    for (int h = 0; h < g && !rc; ++h) {
        /* sample mean, covariance S and its diagonal s* of cluster h */
        long long nh = 0;
        for (int i = 0; i < p; ++i) ybar[i] = m3[i] = 0.0;
        for (int i = 0; i < p * p; ++i) S[i] = 0.0;
        for (int j = 0; j < n; ++j)
            if (labels[j] == h) {
                ++nh;
                for (int i = 0; i < p; ++i) ybar[i] += y[(size_t)j * p + i];
            }
        if (nh < 2) { rc = 1 + h; break; }
        for (int i = 0; i < p; ++i) ybar[i] /= (double)nh;
        for (int j = 0; j < n; ++j)
            if (labels[j] == h) {
                const double* yj = y + (size_t)j * p;
                for (int a = 0; a < p; ++a) {
                    const double ra = yj[a] - ybar[a];
                    for (int b = 0; b < p; ++b) S[a * p + b] += ra * (yj[b] - ybar[b]);
                    m3[a] += ra * ra * ra;
                }
            }
        for (int i = 0; i < p * p; ++i) S[i] /= (double)(nh - 1);
        /* pi from the partition */
        pi[h] = (double)nh / n;
        /* eq (23): delta = sign(m3) sqrt(pi (1 - alpha) s* / (pi - 2)) element-wise,
           Sigma = S - (1 - alpha) diag(s*), mu = ybar - sqrt(2/pi) delta, nu = nu0.
           Delta (p x q): diag(delta) for q = p, the column delta for q = 1, otherwise delta
           on the leading diagonal; only the coordinates that carry a delta are skewed. */
        double* Dh = Delta + (size_t)h * p * q;
        double* Sh = Sigma + (size_t)h * p * p;
        for (int i = 0; i < p * q; ++i) Dh[i] = 0.0;
        for (int a = 0; a < p; ++a) {
            const int skewed = (q == 1 || q >= p || a < q);
            const double sa = S[a * p + a];
            const double d = skewed ? (m3[a] >= 0.0 ? 1.0 : -1.0) *
                                          sqrt(PI * (1.0 - alpha) * sa / (PI - 2.0))
                                    : 0.0;
            if (q == 1) Dh[a * q] = d;
            else if (a < q) Dh[a * q + a] = d;
            mu[(size_t)h * p + a] = ybar[a] - sqrt(2.0 / PI) * d;
            for (int b = 0; b < p; ++b)
                Sh[a * p + b] = S[a * p + b] - (a == b && skewed ? (1.0 - alpha) * sa : 0.0);
        }
        nu[h] = nu0;
        if (chol(p, Sh, L)) rc = 1 + h;   /* Sigma^(0) not positive definite */
    }
    free(ybar); free(S); free(m3); free(L);
    return rc;
}

int ora_init(int n, int p, int q, int g, const double* y, int nstarts, const int* labels,
             uint64_t seed, int nalpha, const double* alphas, double nu0, const ora_qmc* qmc,
             int nthreads, double* loglik_out, int* best, double* pi, double* mu,
             double* Sigma, double* Delta, double* nu)
{
    double* cp = (double*)malloc(sizeof(double) * g);
    double* cm = (double*)malloc(sizeof(double) * g * p);
    double* cS = (double*)malloc(sizeof(double) * g * p * p);
    double* cD = (double*)malloc(sizeof(double) * g * p * q);
    double* cn = (double*)malloc(sizeof(double) * g);
    int* lab = (int*)malloc(sizeof(int) * (n > 0 ? n : 1));
    double lbest = -INFINITY;       /* the best log-likelihood so far */
    int ibest = -1, rc = 0;         /* no candidate kept yet */
    for (int s = 0; s < nstarts && !rc; ++s) {              /* each start */
        if (labels) memcpy(lab, labels + (size_t)s * n, sizeof(int) * n);
        else ora_random_partition(n, g, seed, s, lab);       /* its partition */
        for (int a = 0; a < nalpha && !rc; ++a) {            /* each alpha */
            double L = -INFINITY;
            if (ora_moment_start(n, p, q, g, y, lab, alphas[a], nu0, cp, cm, cS, cD, cn) == 0) {
                rc = ora_loglik(n, p, q, g, y, cp, cm, cS, cD, cn, qmc, nthreads, &L);  /* its log-likelihood */
                if (rc || !isfinite(L)) { rc = 0; L = -INFINITY; }
            }
            if (loglik_out) loglik_out[(size_t)s * nalpha + a] = L;
            if (L > lbest) {                                 /* keep the best (first maximum) */
                lbest = L;
                ibest = s * nalpha + a;
                memcpy(pi, cp, sizeof(double) * g);
                memcpy(mu, cm, sizeof(double) * g * p);
                memcpy(Sigma, cS, sizeof(double) * g * p * p);
                memcpy(Delta, cD, sizeof(double) * g * p * q);
                memcpy(nu, cn, sizeof(double) * g);
            }
        }
    }
    if (best) *best = ibest;
    free(cp); free(cm); free(cS); free(cD); free(cn); free(lab);
    return rc ? rc : (ibest < 0 ? 1 : 0);
}
