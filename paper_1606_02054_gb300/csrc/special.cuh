// special.cuh -- device special functions and the warp-cooperative T_k
// integrators of the E-step.
//
// T_q(b; 0, V, nu), the multivariate t CDF in eq (4) (dof nu+p), eq (13)
// (dof nu+p+2) and in the truncated-t moments of eqs (16)-(17), is not
// specified by the paper.  Here:
//   k = 0: 1;
//   k = 1: regularised incomplete beta, continued fraction (modified Lentz);
//   k = 2: x = sqrt(nu) tan(theta) turns the conditional integral
//          int_{-inf}^{h} t_nu(x) T_1((k - rho x)/sqrt((1-rho^2)(nu+x^2)/(nu+1)); nu+1) dx
//          into C_nu int cos^{nu-1}(theta) T_1(...) dtheta on a finite interval
//          with a smooth integrand; fixed Gauss-Legendre nodes, split where the
//          inner argument changes sign, nodes spread over the 32 lanes;
//   k >= 3: Genz's separation of variables for the multivariate t (chi
//          variable first, fixed order) on a randomised rank-1 Korobov
//          lattice with the baker's transform; lattice points spread over the
//          32 lanes, one warp-shuffle reduction per random shift.
// Every warp-cooperative routine must be called by all 32 lanes with the
// same arguments; it returns the same value in every lane.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "internal.cuh"

#define CF_PI 3.141592653589793238462643383279502884
#define CF_LN2 0.693147180559945309417232121458176568
#define CF_FULL 0xffffffffu

// ---------------------------------------------------------------------------
// precision-generic wrappers
// ---------------------------------------------------------------------------
__device__ __forceinline__ float m_exp(float x) { return expf(x); }
__device__ __forceinline__ double m_exp(double x) { return exp(x); }
__device__ __forceinline__ float m_log(float x) { return logf(x); }
__device__ __forceinline__ double m_log(double x) { return log(x); }
__device__ __forceinline__ float m_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double m_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float m_abs(float x) { return fabsf(x); }
__device__ __forceinline__ double m_abs(double x) { return fabs(x); }
// ---------------------------------------------------------------------------
// FP32 normal CDF and inverse of the lattice integrators: this project's own
// near-minimax polynomial fits (csrc/fit_special_f32.py derives every constant
// below), evaluated with the approximate PTX reciprocal, exp2 and log2.
//   Phi(a) = tau 2^(P(t) - z^2 log2 e), z = |a|/sqrt 2, tau = 1/(1 + z/2), a <= 0;
//            1 - Phi(-a) for a > 0.  Error (measured on the device against FP64):
//            2.5e-6 relative for a >= -5, 1.3e-5 at the bottom of FP32's normal
//            range (a = -13); it comes from the FP32 rounding of z sqrt(log2 e)
//            and of the exponent, and stays far below the lattice's QMC error.
//   Phi^-1(p) = x Q(t), x = log2(-log2 pm), t affine in x, pm = min(p, 1 - p); negated for
//            p > 1/2.  Error (measured on the device): 7.6e-7 absolute for
//            |y| <= 1 (the approximate log2 near p = 1/2), 5.7e-7 relative
//            beyond, on p in [1e-37, 1 - 6e-8].  No branch: every lane runs one
//            polynomial.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float ptx_rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float ptx_ex2_approx(float x)
{
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float ptx_lg2_approx(float x)
{
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float cf_ncdf_f32(float a)
{
    const float zs = fabsf(a) * 0.8493218f;  // z sqrt(log2 e)
    const float tau = ptx_rcp_approx(fmaf(zs, 0.41627732f, 1.0f));
    const float t = fmaf(tau, 2.4210527f, -1.4210526f);
    float P = 9.749631e-05f;
    P = fmaf(P, t, -0.00055511825f);
    P = fmaf(P, t, -0.00034124474f);
    P = fmaf(P, t, 0.0049820864f);
    P = fmaf(P, t, -0.0012651688f);
    P = fmaf(P, t, -0.041432276f);
    P = fmaf(P, t, 0.021236187f);
    P = fmaf(P, t, 0.81600434f);
    P = fmaf(P, t, -1.7987266f);
    const float h = tau * ptx_ex2_approx(fmaf(-zs, zs, P));
    return a > 0.0f ? 1.0f - h : h;
}

__device__ __forceinline__ float cf_ncdfinv_f32(float p)
{
    const float pm = fminf(p, 1.0f - p);
    const float x = ptx_lg2_approx(-ptx_lg2_approx(pm));
    const float t = fmaf(x, 0.2857142984867096f, -1.0f);
    float Q = -6.053980087017408e-06f;
    Q = fmaf(Q, t, -0.0001364098279736936f);
    Q = fmaf(Q, t, -0.0008223482873290777f);
    Q = fmaf(Q, t, -0.004026791080832481f);
    Q = fmaf(Q, t, -0.020278355106711388f);
    Q = fmaf(Q, t, -0.08408169448375702f);
    Q = fmaf(Q, t, -0.25317469239234924f);
    Q = fmaf(Q, t, -0.5432434678077698f);
    Q = fmaf(Q, t, -0.9593654870986938f);
    Q *= x;  // Phi^-1(1/2) = 0 exactly
    return p > 0.5f ? -Q : Q;
}

// sin(x) for |x| <= pi (the arguments of the FP32 T_2 quadrature): |x| folded onto
// [0, pi/2] by pi - |x| (pi in two FP32 parts), then r S(r^2) with S a degree-4
// near-minimax fit (csrc/fit_special_f32.py); error 1.2e-7 relative where
// |sin x| > 1e-3, 1.7e-7 absolute near +-pi.
__device__ __forceinline__ float cf_sin_pi(float x)
{
    const float ax = fabsf(x);
    const float r = ax > 1.57079637f ? (3.14159274f - ax) + -8.74227766e-08f : ax;
    const float r2 = r * r;
    float S = 2.605247118e-06f;
    S = fmaf(S, r2, -1.980908564e-04f);
    S = fmaf(S, r2, 8.333051577e-03f);
    S = fmaf(S, r2, -1.666665822e-01f);
    S = fmaf(S, r2, 1.0f);
    return copysignf(r * S, x);
}

// FP32 reciprocal and division by the approximate PTX reciprocal (relative
// error ~1 ulp); the FP64 versions stay exact IEEE operations.
__device__ __forceinline__ float m_rcp(float x) { return ptx_rcp_approx(x); }
__device__ __forceinline__ double m_rcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float m_div(float a, float b) { return a * ptx_rcp_approx(b); }
__device__ __forceinline__ double m_div(double a, double b) { return a / b; }
__device__ __forceinline__ float m_ncdf(float x) { return cf_ncdf_f32(x); }
__device__ __forceinline__ double m_ncdf(double x) { return normcdf(x); }
__device__ __forceinline__ float m_ncdfinv(float x) { return cf_ncdfinv_f32(x); }
__device__ __forceinline__ double m_ncdfinv(double x) { return normcdfinv(x); }
__device__ __forceinline__ float m_sin(float x) { return sinf(x); }
__device__ __forceinline__ double m_sin(double x) { return sin(x); }
__device__ __forceinline__ float m_cos(float x) { return cosf(x); }
__device__ __forceinline__ double m_cos(double x) { return cos(x); }
__device__ __forceinline__ float m_atan2(float y, float x) { return atan2f(y, x); }
__device__ __forceinline__ double m_atan2(double y, double x) { return atan2(y, x); }

template <typename R> struct Lim;
template <> struct Lim<float> {
    static __device__ __forceinline__ float tiny() { return 1e-30f; }
    static __device__ __forceinline__ float eps() { return 6e-8f; }
    static __device__ __forceinline__ float one_minus_ulp() { return 0.99999994f; }
    static __device__ __forceinline__ float vmin() { return 1e-37f; }
    static constexpr int cf_iters = 200;
};
template <> struct Lim<double> {
    static __device__ __forceinline__ double tiny() { return 1e-300; }
    static __device__ __forceinline__ double eps() { return 1e-16; }
    static __device__ __forceinline__ double one_minus_ulp() { return 1.0 - 0x1.0p-53; }
    static __device__ __forceinline__ double vmin() { return 1e-300; }
    static constexpr int cf_iters = 600;
};

// ---------------------------------------------------------------------------
// warp helpers
// ---------------------------------------------------------------------------
// Sum over the warp; the result is lane 0's butterfly total, broadcast, so
// every lane holds a bitwise-identical value (keeps later branches uniform).
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(CF_FULL, v, o);
    return __shfl_sync(CF_FULL, v, 0);
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(CF_FULL, v, o);
    return __shfl_sync(CF_FULL, v, 0);
}

__device__ __forceinline__ void m_sincos(float x, float* s, float* c) { sincosf(x, s, c); }
__device__ __forceinline__ void m_sincos(double x, double* s, double* c) { sincos(x, s, c); }
__device__ __forceinline__ float m_atan(float x) { return atanf(x); }
__device__ __forceinline__ double m_atan(double x) { return atan(x); }

// ---------------------------------------------------------------------------
// digamma (FP64): psi(x) = psi(x + k) - sum 1/(x+i) up to x >= 12, then
// psi(x) ~ ln x - 1/(2x) - sum_{k>=1} B_{2k} / (2k x^{2k}).
// ---------------------------------------------------------------------------
__device__ inline double cf_digamma(double x)
{
    double s = 0.0;
    while (x < 12.0) { s -= 1.0 / x; x += 1.0; }
    const double r = 1.0 / x, r2 = r * r;
    // coefficients B_{2k}/(2k) for k = 1..6
    double ser = r2 * (1.0 / 12 + r2 * (-1.0 / 120 + r2 * (1.0 / 252 + r2 * (-1.0 / 240
                 + r2 * (1.0 / 132 + r2 * (-691.0 / 32760))))));
    return s + log(x) - 0.5 * r - ser;
}

// trigamma (FP64) for Newton steps on eq (22): psi'(x) = sum 1/(x+i)^2 + asymptotic
__device__ inline double cf_trigamma(double x)
{
    double s = 0.0;
    while (x < 12.0) { s += 1.0 / (x * x); x += 1.0; }
    const double r = 1.0 / x, r2 = r * r;
    // psi'(x) ~ 1/x + 1/(2x^2) + sum_k B_{2k} / x^{2k+1}
    double ser = r * (1.0 + r * (0.5 + r * (1.0 / 6 + r2 * (-1.0 / 30 + r2 * (1.0 / 42
                 + r2 * (-1.0 / 30 + r2 * (5.0 / 66)))))));
    return s + ser;
}

// log of the univariate t density at x with scale^2 v and dof nu (FP64);
// lc = lgamma((nu+1)/2) - lgamma(nu/2) - log(nu pi)/2
// log of the N(0, v) density at x (the nu -> infinity limit of cf_logt1)
__device__ inline double cf_lognorm1(double x, double v)
{
    return -0.5 * log(2.0 * CF_PI * v) - 0.5 * x * x / v;
}

__device__ inline double cf_logt1(double x, double v, double nu, double lc)
{
    return lc - 0.5 * log(v) - 0.5 * (nu + 1.0) * log1p(x * x / (nu * v));
}

// ---------------------------------------------------------------------------
// T_1: P(T <= t), T ~ t_nu, from I_x(nu/2, 1/2) with x = nu/(nu+t^2).
// lgb = lgamma((nu+1)/2) - lgamma(nu/2) - lgamma(1/2), precomputed per dof.
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ R betacf_dev(R a, R b, R x)
{
    const R tiny = Lim<R>::tiny();
    R c = R(1), d = R(1) - m_div((a + b) * x, a + R(1));
    if (m_abs(d) < tiny) d = tiny;
    d = m_rcp(d);
    R h = d;
    for (int m = 1; m <= Lim<R>::cf_iters; ++m) {
        const R mm = R(m), m2 = R(2 * m);
        R aa = m_div(mm * (b - mm) * x, (a - R(1) + m2) * (a + m2));
        d = R(1) + aa * d; if (m_abs(d) < tiny) d = tiny;
        c = R(1) + m_div(aa, c); if (m_abs(c) < tiny) c = tiny;
        d = m_rcp(d); h *= d * c;
        aa = m_div(-(a + mm) * (a + b + mm) * x, (a + m2) * (a + R(1) + m2));
        d = R(1) + aa * d; if (m_abs(d) < tiny) d = tiny;
        c = R(1) + m_div(aa, c); if (m_abs(c) < tiny) c = tiny;
        d = m_rcp(d);
        const R del = d * c;
        h *= del;
        if (m_abs(del - R(1)) < Lim<R>::eps()) break;
    }
    return h;
}

template <typename R>
__device__ __forceinline__ R t1cdf_dev(R t, R nu, R lgb)
{
    if (t == R(0)) return R(0.5);
    const R t2 = t * t, den = nu + t2;
    const R x = m_div(nu, den), y = m_div(t2, den);
    const R a = R(0.5) * nu, b = R(0.5);
    const R ld = m_log(den);
    const R lbt = lgb + a * (m_log(nu) - ld) + b * (R(2) * m_log(m_abs(t)) - ld);
    // one continued fraction per lane: I_x(a,b) directly, or 1 - I_y(b,a)
    // (arguments selected first, so divergent lanes do not run both)
    const bool direct = x < (a + R(1)) / (a + b + R(2));
    const R cf = betacf_dev<R>(direct ? a : b, direct ? b : a, direct ? x : y);
    const R pre = m_exp(lbt) * cf;
    const R I = direct ? m_div(pre, a) : R(1) - m_div(pre, b);
    const R tail = R(0.5) * I;
    return t > R(0) ? R(1) - tail : tail;
}

__device__ __forceinline__ double t1_lgb(double nu)
{
    return lgamma(0.5 * (nu + 1.0)) - lgamma(0.5 * nu) - 0.5723649429247001 /* lgamma(1/2) */;
}

// ---------------------------------------------------------------------------
// T_1(z; nu + 1) inside an FP32 T_2 from its per-dof table (IntegArgs::t1tab):
// cubic Hermite interpolation of log2 T_1(-|z|) in v = log2(1 + |z|) (values
// and derivatives tabulated in FP64, see t1_table_kernel), continued linearly
// beyond the grid, where log2 T_1 approaches its asymptote -(nu+1) v + const.
// T_1(z) = 1 - T_1(-z) for z > 0.  Interpolation error ~1e-8 in log2 T_1;
// the FP32 table values bound the result at ~5e-6 relative in the far tail.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float t1cdf_table(float z, const float2* __restrict__ tab)
{
    constexpr float hv = T1TAB_V / (T1TAB_N - 1);
    const float w = fabsf(z);
    const float v = ptx_lg2_approx(1.0f + w);
    const float pos = fminf(v * (1.0f / hv), (float)(T1TAB_N - 1));
    const int i = min((int)pos, T1TAB_N - 2);
    const float t = pos - (float)i;
    const float2 a = __ldg(tab + i), b = __ldg(tab + i + 1);
    const float m0 = hv * a.y, m1 = hv * b.y, dl = b.x - a.x;
    const float c2 = 3.0f * dl - 2.0f * m0 - m1, c3 = m0 + m1 - 2.0f * dl;
    float lg = fmaf(fmaf(fmaf(c3, t, c2), t, m0), t, a.x);
    lg = v > T1TAB_V ? fmaf(v - T1TAB_V, b.y, b.x) : lg;
    const float T = ptx_ex2_approx(lg);
    return z > 0.0f ? 1.0f - T : T;
}

// ---------------------------------------------------------------------------
// T_2(h, k; rho, nu), standard bivariate t, warp-cooperative.
// With theta = phi - pi/2 (phi in (0, pi)): cos theta = sin phi and
// sin theta = -cos phi, so
//   T_2 = C_nu int_0^{phi_h} sin^{nu-1}(phi) T_1((k sin phi + rho sqrt(nu) cos phi) s_r; nu+1) dphi
// with C_nu = Gamma((nu+1)/2)/(Gamma(nu/2) sqrt(pi)), s_r = sqrt((nu+1)/((1-rho^2) nu)),
// phi_h = pi/2 + atan(h/sqrt(nu)).  The inner argument changes sign at phi*,
// (sin, cos)(phi*) = (|rho| sqrt(nu), -k sign(rho)) / R with R = sqrt(k^2 + rho^2 nu),
// and equals -sign(rho) R sin(phi - phi*) exactly (rho = 0 counts as negative);
// that form is used, with phi - phi* taken from the node's offset, so nothing
// cancels near phi*.  The interval is split at phi*.  For |rho| > 0.99 the
// nodes are graded (phi = anchor + L t^3) toward the split point (or toward
// phi_h when there is no split) to resolve the boundary layer of width
// ~ sqrt(1 - rho^2), and glxh/glwh (nh nodes) replace glx/glw (n nodes).  With nlo > 0
// (FP32), a piece with 4 <= nu <= 64 and |rho| < 0.9 takes the node set of its
// t2_lo_class from glxl/glwl (the classes' sets packed in order).
// The second piece's length phi_h - phi* is computed directly (not as a
// difference of the two angles, which can be far shorter than FP32 resolves
// them), and it also places the upper end, so the split point and the upper
// end move together.  Inputs are the records' FP64 values; 1 - rho^2 is
// formed as (1 - rho)(1 + rho) in FP64.
// t1tab (FP32 only, may be NULL): this record's table of T_1 at dof nu + 1.
// ---------------------------------------------------------------------------
template <typename T>
struct T2Setup {
    T phis, anc0, L0, L1, d0, zs;
    bool split;
};

// omr2 = 1 - rho^2 and cr = h |rho| - sign(rho) k come formed in FP64 (the
// rounding of h, k and rho to FP32 would otherwise dominate both near |rho| = 1).
template <typename T>
__device__ __forceinline__ T2Setup<T> t2_setup(T h, T k, T rho, T nu, T omr2, T cr)
{
    T2Setup<T> o;
    const T sn = m_sqrt(nu);
    const T sg = rho > T(0) ? T(1) : T(-1);  // sign(rho), rho = 0 counting as negative
    const T ar = m_abs(rho);
    // phi_h = pi/2 + atan(h/sqrt(nu)), accurate for h << 0 as atan(sqrt(nu)/(-h))
    const T phi_h = h < T(0) ? m_atan(sn / (-h)) : T(0.5 * CF_PI) + m_atan(h / sn);
    o.phis = m_atan2(ar * sn, -sg * k);
    // D = phi_h - phi*: the angle between (-h, sqrt nu) and (-sign(rho) k, |rho| sqrt nu)
    const T D = m_atan2(sn * cr, sg * h * k + ar * nu);
    o.split = rho != T(0) && D > T(0);
    o.anc0 = o.split ? o.phis : phi_h;  // pieces run from the anchor to the far end
    o.L0 = -o.anc0;                     // piece 0: anchor -> 0
    o.L1 = D;                           // piece 1: phi* -> phi* + D
    o.d0 = o.split ? T(0) : D;          // phi - phi* at piece 0's anchor
    const T Rr = m_sqrt(rho * rho * nu + k * k);
    o.zs = -sg * Rr * m_sqrt((nu + T(1)) / (omr2 * nu));
    return o;
}

template <typename R>
__device__ double t2cdf_warp(R h, R k, R rho, R nu, R omr2, R cr, R lgb, R lgb1, R C2, int n,
                             const R* __restrict__ glx, const R* __restrict__ glw, int nh,
                             const R* __restrict__ glxh, const R* __restrict__ glwh, int lane,
                             const float2* __restrict__ t1tab = nullptr, int* nodes_out = nullptr,
                             int nlo = 0, const R* __restrict__ glxl = nullptr, const R* __restrict__ glwl = nullptr)
{
    if (nodes_out) *nodes_out = 0;
    if (rho >= R(1)) {
        const R m = h < k ? h : k;
        return (double)t1cdf_dev<R>(m, nu, lgb);
    }
    if (rho <= R(-1)) {
        const R v = t1cdf_dev<R>(h, nu, lgb) + t1cdf_dev<R>(k, nu, lgb) - R(1);
        return v > R(0) ? (double)v : 0.0;
    }
    const bool graded = m_abs(rho) > R(0.99);
    // fewer nodes where the integrand is smooth enough (nlo > 0: FP32, t2_lo_class per piece)
    const bool lo = nlo > 0 && !graded && m_abs(rho) < R(T2_LO_RHO) && nu >= R(T2_LO_DOF_MIN) &&
                    nu <= R(T2_LO_DOF_MAX);
    const T2Setup<R> S = t2_setup<R>(h, k, rho, nu, omr2, cr);
    const int npieces = S.split ? 2 : 1;
    // node set of each piece: its class's Gauss-Legendre set, else n nodes, else nh graded
    const R* __restrict__ gx0 = graded ? glxh : glx;
    const R* __restrict__ gw0 = graded ? glwh : glw;
    const R* __restrict__ gx1 = gx0;
    const R* __restrict__ gw1 = gw0;
    int n0 = graded ? nh : n, n1 = n0;
    if (lo) {
        const int c0 = t2_lo_class((float)S.L0, (float)nu, (float)S.zs);
        const int c1 = t2_lo_class((float)S.L1, (float)nu, (float)S.zs);
        if (c0 < T2_LO_NCLS) { n0 = t2_lo_nodes(c0); gx0 = glxl + t2_lo_off(c0); gw0 = glwl + t2_lo_off(c0); }
        if (c1 < T2_LO_NCLS) { n1 = t2_lo_nodes(c1); gx1 = glxl + t2_lo_off(c1); gw1 = glwl + t2_lo_off(c1); }
    }
    if (npieces == 1) n1 = 0;
    if (nodes_out) *nodes_out = n0 + n1;
    const R nu1 = nu + R(1), num1 = nu - R(1);
    R acc = R(0);
    for (int t = lane; t < n0 + n1; t += CF_WARP) {
        const bool p1 = t >= n0;
        const int i = p1 ? t - n0 : t;
        const R anc = p1 ? S.phis : S.anc0;
        const R L = p1 ? S.L1 : S.L0;
        const R u = p1 ? gx1[i] : gx0[i];
        const R um = graded ? u * u * u : u;
        const R jac = graded ? R(3) * u * u : R(1);
        const R off = L * um;
        R sp, sd;
        if constexpr (sizeof(R) == sizeof(float)) {
            sp = cf_sin_pi(anc + off);  // both arguments lie in [-pi, pi]
            sd = cf_sin_pi((p1 ? R(0) : S.d0) + off);
        } else {
            sp = m_sin(anc + off);
            sd = m_sin((p1 ? R(0) : S.d0) + off);
        }
        const R z = S.zs * sd;
        R f;
        if constexpr (sizeof(R) == sizeof(float)) {
            // sin^(nu-1) by the approximate log2/exp2 (~5e-6 relative at nu ~ 40)
            f = ptx_ex2_approx(num1 * ptx_lg2_approx(sp)) *
                (t1tab ? t1cdf_table(z, t1tab) : t1cdf_dev<R>(z, nu1, lgb1));
        } else {
            f = m_exp(num1 * m_log(sp)) * t1cdf_dev<R>(z, nu1, lgb1);
        }
        acc += (p1 ? gw1[i] : gw0[i]) * jac * f * m_abs(L);
    }
    acc = warp_sum(acc);
    return (double)(C2 * acc);
}

// Sum over aligned groups of L lanes (L a power of two <= 32); every lane of a group
// gets the group's total, bitwise identical (the group's first lane's value).  All 32
// lanes must execute it.
template <int L>
__device__ __forceinline__ float group_sum(float v)
{
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) v += __shfl_xor_sync(CF_FULL, v, o);
    return __shfl_sync(CF_FULL, v, (threadIdx.x & (CF_WARP - 1)) & ~(L - 1));
}

// ---------------------------------------------------------------------------
// Phi_2(h, k; rho), the nu -> infinity limit of T_2 (the CFUSN model of eq 5),
// warp-cooperative.  With e(theta) = exp(-(h^2 - 2 h k sin theta + k^2) / (2 cos^2 theta)),
// which is positive (Sheppard's integral, r = sin theta):
//   rho >= 0:  Phi(h) Phi(k) + (1/2pi) int_0^{asin rho} e,
//   rho < 0:   P(-k < X <= h) + (1/2pi) int_{-pi/2}^{asin rho} e   (Phi_2 at rho = -1 plus
//              the rest),
// so small values are never differences of large ones.  In the tails e is concentrated
// at one end of the interval, and for rho < 0 it rises over a width ~|h + k| at -pi/2:
// the interval is split in halves, each with n nodes graded (t^3) toward its own end.
// P(-k < X <= h) by 4-point Gauss-Legendre where the interval is narrow against the
// Gaussian's scale there, else as a difference of Phi values in the lower tail.
// ---------------------------------------------------------------------------
template <typename R>
__device__ double phi2_warp(R h, R k, R rho, int n, const R* __restrict__ glx, const R* __restrict__ glw,
                            int lane)
{
    if (rho >= R(1)) return (double)m_ncdf(h < k ? h : k);
    const R hk = h + k;
    R lower = R(0);
    if (hk > R(0)) {
        const R mid = R(0.5) * (h - k), half = R(0.5) * hk;  // the interval (-k, h]
        if (hk * (R(1) + fabs(mid)) < R(0.5)) {
            // narrow against the Gaussian's scale there: 4-point Gauss-Legendre
            const R x4[2] = {R(0.8611363115940526), R(0.3399810435848563)};
            const R w4[2] = {R(0.3478548451374538), R(0.6521451548625461)};
            R s4 = R(0);
            for (int i = 0; i < 2; ++i) {
                const R xa = mid + half * x4[i], xb = mid - half * x4[i];
                s4 += w4[i] * (m_exp(R(-0.5) * xa * xa) + m_exp(R(-0.5) * xb * xb));
            }
            lower = s4 * half * R(0.3989422804014327);  // 1/sqrt(2 pi)
        } else {
            // P(-k < X <= h) = P(-h <= X < k): the form whose endpoints are nearer the lower
            // tail, where Phi keeps its relative precision; outside the Gauss-Legendre range
            // the smaller term is at most about 2/3 of the larger, so at most a few ulps go
            lower = mid < R(0) ? m_ncdf(h) - m_ncdf(-k) : m_ncdf(k) - m_ncdf(-h);
        }
    }
    if (rho <= R(-1)) return (double)lower;
    const bool neg = rho < R(0);
    const R b = asin(rho);
    const R a = neg ? R(-0.5 * CF_PI) : R(0);
    const R hL = R(0.5) * (b - a);
    R acc = R(0);
    for (int t = lane; t < 2 * n; t += CF_WARP) {
        const bool top = t >= n;  // second half: anchored at b, running down
        const R u = glx[top ? t - n : t];
        const R th = top ? b - hL * u * u * u : a + hL * u * u * u;
        R sn;
        if constexpr (sizeof(R) == sizeof(float)) sn = cf_sin_pi(th);
        else sn = sin(th);
        const R c2 = (R(1) - sn) * (R(1) + sn);
        const R e = c2 > R(0) ? m_exp(-(h * h - R(2) * h * k * sn + k * k) / (R(2) * c2)) : R(0);
        acc += glw[top ? t - n : t] * R(3) * u * u * e;
    }
    acc = warp_sum(acc);
    const R base = neg ? lower : m_ncdf(h) * m_ncdf(k);
    return (double)(base + acc * hL * R(0.15915494309189535));  // 1/(2 pi)
}

// ---------------------------------------------------------------------------
// Regularised incomplete gamma and the chi-square quantile (FP64), used to
// tabulate s = sqrt(chi2_nu^{-1}(w_0)/nu) at every lattice point.
// ---------------------------------------------------------------------------
// lga = lgamma(a)
__device__ inline void cf_gamma_pq(double a, double lga, double x, double* P, double* Q)
{
    if (x <= 0.0) { *P = 0.0; *Q = 1.0; return; }
    const double lpre = a * log(x) - x - lga;
    if (x < a + 1.0) {
        // series: P = x^a e^-x / Gamma(a+1) * sum_n x^n / ((a+1)...(a+n))
        double term = 1.0, sum = 1.0, ap = a;
        for (int n = 0; n < 2000; ++n) {
            ap += 1.0;
            term *= x / ap;
            sum += term;
            if (term < sum * 1e-17) break;
        }
        *P = exp(lpre) * sum / a;
        *Q = 1.0 - *P;
    } else {
        // Legendre continued fraction for Q, modified Lentz
        const double tiny = 1e-300;
        double b = x + 1.0 - a, c = 1.0 / tiny, d = 1.0 / b, hh = d;
        for (int i = 1; i < 2000; ++i) {
            const double an = -i * (i - a);
            b += 2.0;
            d = an * d + b; if (fabs(d) < tiny) d = tiny;
            c = b + an / c; if (fabs(c) < tiny) c = tiny;
            d = 1.0 / d;
            const double del = d * c;
            hh *= del;
            if (fabs(del - 1.0) < 1e-16) break;
        }
        *Q = exp(lpre) * hh;
        *P = 1.0 - *Q;
    }
}

// x with P(nu/2, x/2) = w (w <= 1/2) or Q(nu/2, x/2) = wc (w > 1/2):
// safeguarded Newton on the log of the smaller tail probability.
// lga = lgamma(nu/2); Newton stops at relative change rtol (1e-15 for FP64 tables).
__device__ inline double cf_chi2_quantile(double w, double wc, double nu, double lga, double rtol)
{
    if (!(w > 0.0)) return 0.0;
    if (!(wc > 0.0)) return INFINITY;
    const double a = 0.5 * nu;
    const bool upper = w > 0.5;
    const double target = upper ? log(wc) : log(w);
    // start: Wilson-Hilferty, or the small-x expansion in the far lower tail
    const double z = upper ? -normcdfinv(wc) : normcdfinv(w);
    const double c9 = 2.0 / (9.0 * nu);
    const double base = 1.0 - c9 + z * sqrt(c9);
    double x = nu * base * base * base;
    const double xs = 2.0 * exp((log(w) + lga + log(a)) / a);
    if (!(x > 0.0) || (!upper && xs < x)) x = xs;
    double lo = 0.0, hi = INFINITY;
    for (int it = 0; it < 200; ++it) {
        double P, Q;
        cf_gamma_pq(a, lga, 0.5 * x, &P, &Q);
        const double tv = upper ? Q : P;
        const double G = upper ? (target - log(tv)) : (log(tv) - target);  // increasing in x
        if (G == 0.0) break;
        if (G > 0.0) hi = x; else lo = x;
        const double ldens = (a - 1.0) * log(0.5 * x) - 0.5 * x - lga - 0.6931471805599453;
        double xn = x - G * exp(log(tv) - ldens);
        if (!(xn > lo && xn < hi)) xn = isinf(hi) ? 2.0 * x : 0.5 * (lo + hi);
        const bool done = fabs(xn - x) <= rtol * x || (isfinite(hi) && hi - lo <= rtol * hi);
        x = xn;
        if (done) break;
    }
    return x;
}

// ---------------------------------------------------------------------------
// Lattice T_k, k = K >= 3, warp-cooperative.
//   bt:   standardised limits b_i / sqrt(V_ii) (K values, FP64)
//   Lc:   Cholesky factor of the correlation matrix of V (K x K, row-major, FP64)
//   chi:  s at every lattice point for this dof, [m][i] (N per shift)
//   shf:  shifts [m][d], d < CF_MAXDIM, in precision R
// Returns the mean over shifts of the shift means; *se the standard error.
// ---------------------------------------------------------------------------
template <typename R, int K>
__device__ double tk_lattice_warp(const double* bt, const double* Lc, const R* __restrict__ chi,
                                  const R* __restrict__ shf, const Lattice& lat, int lane, double* se)
{
    R b[K], invd[K], Lo[K][K];
#pragma unroll
    for (int r = 0; r < K; ++r) {
        b[r] = (R)bt[r];
        invd[r] = R(1) / (R)Lc[r * K + r];
#pragma unroll
        for (int l = 0; l < K; ++l) Lo[r][l] = l < r ? (R)Lc[r * K + l] : R(0);
    }
    const int N = lat.N, M = lat.M;
    const R invN = R(1) / (R)N;
    // lattice coordinates x_d = frac(i z_d / N + shift_d), advanced by dx_d = frac(32 z_d / N)
    // per point of this lane: x - (1 - dx) when that is >= 0 (exact), else x + dx (exact but
    // for one rounding when x enters a higher binade: a few ulp over a lane's points)
    R x0[K], dx[K], omdx[K];
#pragma unroll
    for (int d = 1; d < K; ++d) {
        dx[d] = (R)(((long long)CF_WARP * lat.z[d]) % N) * invN;
        omdx[d] = R(1) - dx[d];
        x0[d] = (R)(((long long)lane * lat.z[d]) % N) * invN;
    }
    R mean = R(0), m2 = R(0);  // Welford over the shift means
    for (int m = 0; m < M; ++m) {
        R xs[K];
#pragma unroll
        for (int d = 1; d < K; ++d) {
            xs[d] = x0[d] + shf[m * CF_MAXDIM + d];
            if (xs[d] >= R(1)) xs[d] -= R(1);
        }
        R acc = R(0), comp = R(0);  // compensated sum
        const R* __restrict__ crow = chi + (size_t)m * N;
        for (int i = lane; i < N; i += CF_WARP) {
            const R s = crow[i];
            R y[K];
            R f = R(1);
#pragma unroll
            for (int r = 0; r < K; ++r) {
                R a = b[r] * s;
#pragma unroll
                for (int l = 0; l < r; ++l) a -= Lo[r][l] * y[l];
                const R e = m_ncdf(a * invd[r]);
                f *= e;
                if (r < K - 1) {
                    const R w = R(1) - m_abs(R(2) * xs[r + 1] - R(1));
                    R v = w * e;
                    v = v < Lim<R>::vmin() ? Lim<R>::vmin() : v;
                    v = v > Lim<R>::one_minus_ulp() ? Lim<R>::one_minus_ulp() : v;
                    y[r] = m_ncdfinv(v);
                }
                if (e <= Lim<R>::tiny()) f = R(0);
            }
            // Kahan step
            const R yk = f - comp;
            const R tk = acc + yk;
            comp = (tk - acc) - yk;
            acc = tk;
#pragma unroll
            for (int d = 1; d < K; ++d) {
                const R t = xs[d] - omdx[d];
                xs[d] = t >= R(0) ? t : xs[d] + dx[d];
            }
        }
        const R smean = warp_sum(acc) * invN;
        const R delta = smean - mean;
        mean += delta / R(m + 1);
        m2 += delta * (smean - mean);
    }
    if (se) *se = M > 1 ? (double)m_sqrt(m2 / R(M - 1) / R(M)) : 0.0;
    return (double)mean;
}

// ---------------------------------------------------------------------------
// Lattice T_K with the truncated moments, warp-cooperative: the pass of
// alpha_s at k1 dof (chi table chi, limits bt) that also yields alpha and the
// moments at k2 = k1 + 2 dof.  Each point carries s = sqrt(W/k1), W its
// chi-square(k1) variate; the chi-square(k2) density is the chi-square(k1)
// density times W/k1, so weighting a point by s^2 moves the pass to k2 dof.
// The separation of variables also samples the last coordinate (lattice
// dimension K), so every point gives the draw X = L y / s2 (standardised at
// k2 dof, s2 = s sqrt(k1/k2); rk = sqrt(k2/k1), 1 in the normal limit) inside
// the truncation region with weight f = prod e_i.  Returns alpha = mean f s^2;
// *alpha_s = mean f (as tk_lattice_warp: the same points) and *se its standard
// error over the shifts (all lanes).  Leaves the ratio estimators in
// acc_sm[1..K] (m1 = sum f s^2 X / sum f s^2) and acc_sm[1+K..K+K(K+1)/2]
// (m2, lower triangle), visible to the whole warp until the next call; they are
// accumulated in the whitened coordinates y and mapped through L once per record.
// ---------------------------------------------------------------------------
template <typename R, int K>
__device__ double tk_lattice_mom_warp(const double* bt, const double* Lc, const R* __restrict__ chi,
                                      const R* __restrict__ shf, const Lattice& lat, int lane,
                                      double* acc_sm, R rk, double* alpha_s, double* se,
                                      const R* __restrict__ lchi = nullptr, double* lw_out = nullptr)
{
    // lchi (exact E[log W], may be null): log(s^2) at every point; *lw_out receives the
    // f-weighted mean of it over the points (all lanes)
    double lw_acc = 0.0;
    // acc_sm: this warp's shared-memory slot of K + K(K+1)/2 + 3 + CF_MAXSHIFT doubles
    // that lane 0 uses for the running totals and the per-shift sums of f
    constexpr int K2 = K * (K + 1) / 2;
    R b[K], invd[K], Lf[K][K];
#pragma unroll
    for (int r = 0; r < K; ++r) {
        b[r] = (R)bt[r];
        invd[r] = R(1) / (R)Lc[r * K + r];
#pragma unroll
        for (int l = 0; l < K; ++l) Lf[r][l] = l <= r ? (R)Lc[r * K + l] : R(0);
    }
    const int N = lat.N, M = lat.M;
    const R invN = R(1) / (R)N;
    R x0[K + 1], dx[K + 1], omdx[K + 1];  // lattice coordinates as in tk_lattice_warp
#pragma unroll
    for (int d = 1; d <= K; ++d) {
        dx[d] = (R)(((long long)CF_WARP * lat.z[d]) % N) * invN;
        omdx[d] = R(1) - dx[d];
        x0[d] = (R)(((long long)lane * lat.z[d]) % N) * invN;
    }
    for (int r = lane; r <= K + K2; r += CF_WARP) acc_sm[r] = 0.0;
    __syncwarp();
    for (int m = 0; m < M; ++m) {
        R xs[K + 1];
#pragma unroll
        for (int d = 1; d <= K; ++d) {
            xs[d] = x0[d] + shf[m * CF_MAXDIM + d];
            if (xs[d] >= R(1)) xs[d] -= R(1);
        }
        R af = R(0), aw = R(0), al = R(0), a1[K], a2[K2];
#pragma unroll
        for (int r = 0; r < K; ++r) a1[r] = R(0);
#pragma unroll
        for (int r = 0; r < K2; ++r) a2[r] = R(0);
        const R* __restrict__ crow = chi + (size_t)m * N;
        R s_next = lane < N ? crow[lane] : R(1);  // the chi value one point ahead
        for (int i = lane; i < N; i += CF_WARP) {
            const R s = s_next;
            if (i + CF_WARP < N) s_next = crow[i + CF_WARP];
            R y[K];
            R f = R(1);
#pragma unroll
            for (int r = 0; r < K; ++r) {
                R a = b[r] * s;
#pragma unroll
                for (int l = 0; l < r; ++l) a -= Lf[r][l] * y[l];
                const R e = m_ncdf(a * invd[r]);
                f *= e;
                const R w = R(1) - m_abs(R(2) * xs[r + 1] - R(1));
                R v = w * e;
                v = v < Lim<R>::vmin() ? Lim<R>::vmin() : v;
                v = v > Lim<R>::one_minus_ulp() ? Lim<R>::one_minus_ulp() : v;
                y[r] = m_ncdfinv(v);
                if (e <= Lim<R>::tiny()) f = R(0);
            }
            // weight f s^2; X = L y / s2 is linear in y: accumulate f s^2 y / s2 =
            // f s rk y and f s^2 y y^T / s2^2 = f rk^2 y y^T, and apply L once per record
            const R fs = f * s;
            const R w1 = fs * rk, w2 = f * (rk * rk);
            af += f;
            aw += fs * s;
            if (lchi) al += f * lchi[(size_t)m * N + i];
#pragma unroll
            for (int r = 0; r < K; ++r) {
                a1[r] += w1 * y[r];
                const R t = w2 * y[r];
#pragma unroll
                for (int c = 0; c <= r; ++c) a2[r * (r + 1) / 2 + c] += t * y[c];
            }
#pragma unroll
            for (int d = 1; d <= K; ++d) {
                const R t = xs[d] - omdx[d];
                xs[d] = t >= R(0) ? t : xs[d] + dx[d];
            }
        }
        af = warp_sum(af);
        aw = warp_sum(aw);
        if (lchi) lw_acc += (double)warp_sum(al);
#pragma unroll
        for (int r = 0; r < K; ++r) a1[r] = warp_sum(a1[r]);
#pragma unroll
        for (int r = 0; r < K2; ++r) a2[r] = warp_sum(a2[r]);
        if (lane == 0) {
            acc_sm[3 + K + K2 + m] = (double)af;  // alpha_s: this shift's sum
            acc_sm[0] += (double)aw;
#pragma unroll
            for (int r = 0; r < K; ++r) acc_sm[1 + r] += (double)a1[r];
#pragma unroll
            for (int r = 0; r < K2; ++r) acc_sm[1 + K + r] += (double)a2[r];
        }
    }
    __syncwarp();
    if (lw_out) {  // sum f over all shifts (every lane reads the per-shift sums)
        double sf = 0.0;
        for (int m = 0; m < M; ++m) sf += acc_sm[3 + K + K2 + m];
        *lw_out = sf > 0.0 ? lw_acc / sf : NAN;
    }
    const double Sf = acc_sm[0];
    const double inv = Sf > 0.0 ? 1.0 / Sf : 0.0;
    // m1 = L E[y/s], m2 = L E[y y^T / s^2] L^T in FP64 (Lc is the full lower
    // factor), one output per lane, written back over the totals
    double o[2] = {0.0, 0.0};
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int t = lane + u * CF_WARP;
        if (t >= K + K2) break;
        double v = 0.0;
        if (t < K) {
            for (int l = 0; l <= t; ++l) v += Lc[t * K + l] * acc_sm[1 + l];
        } else {
            const int e = t - K;
            int r = 0;
            while ((r + 1) * (r + 2) / 2 <= e) ++r;
            const int c = e - r * (r + 1) / 2;
            for (int i = 0; i <= r; ++i) {
                double w = 0.0;
                for (int j = 0; j <= c; ++j)
                    w += acc_sm[1 + K + (i >= j ? i * (i + 1) / 2 + j : j * (j + 1) / 2 + i)] * Lc[c * K + j];
                v += Lc[r * K + i] * w;
            }
        }
        o[u] = v * inv;
    }
    __syncwarp();
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int t = lane + u * CF_WARP;
        if (t < K + K2) acc_sm[1 + t] = o[u];
    }
    __syncwarp();
    __syncwarp();
    if (lane == 0) {  // alpha_s: mean of the shift means and its standard error (Welford)
        double mean = 0.0, m2 = 0.0;
        for (int m = 0; m < M; ++m) {
            const double smean = acc_sm[3 + K + K2 + m] / (double)N;
            const double delta = smean - mean;
            mean += delta / (double)(m + 1);
            m2 += delta * (smean - mean);
        }
        acc_sm[1 + K + K2] = mean;
        acc_sm[2 + K + K2] = M > 1 ? sqrt(m2 / (double)(M - 1) / (double)M) : 0.0;
    }
    __syncwarp();
    *alpha_s = acc_sm[1 + K + K2];
    *se = acc_sm[2 + K + K2];
    return Sf / ((double)N * M);
}

// ---------------------------------------------------------------------------
// tk_lattice_mom_warp with the baker-transformed coordinates of each point read from
// wtab (IntegArgs::wtab, one float4 per (shift, point), K <= 4) instead of advanced in
// floating point, and without the cut-off of factors below Lim::tiny (an underflowed
// factor zeroes the product by itself): the same estimator up to the coordinates'
// rounding.  A separate function, so that the code generated for the other dimensions
// stays as it was.
// ---------------------------------------------------------------------------
template <typename R, int K, bool TAB = true>
__device__ double tk_lattice_mom_tab_warp(const double* bt, const double* Lc, const R* __restrict__ chi,
                                      const R* __restrict__ shf, const Lattice& lat, int lane,
                                      double* acc_sm, R rk, double* alpha_s, double* se,
                                      const float4* __restrict__ wtab = nullptr)
{
    constexpr int WQ = (K + 3) / 4;
    // acc_sm: this warp's shared-memory slot of K + K(K+1)/2 + 3 + CF_MAXSHIFT doubles
    // that lane 0 uses for the running totals and the per-shift sums of f
    constexpr int K2 = K * (K + 1) / 2;
    R b[K], invd[K], Lf[K][K];
#pragma unroll
    for (int r = 0; r < K; ++r) {
        b[r] = (R)bt[r];
        invd[r] = R(1) / (R)Lc[r * K + r];
#pragma unroll
        for (int l = 0; l < K; ++l) Lf[r][l] = l <= r ? (R)Lc[r * K + l] : R(0);
    }
    const int N = lat.N, M = lat.M;
    const R invN = R(1) / (R)N;
    R x0[K + 1], dx[K + 1], omdx[K + 1];  // lattice coordinates as in tk_lattice_warp
#pragma unroll
    for (int d = 1; d <= K; ++d) {
        dx[d] = (R)(((long long)CF_WARP * lat.z[d]) % N) * invN;
        omdx[d] = R(1) - dx[d];
        x0[d] = (R)(((long long)lane * lat.z[d]) % N) * invN;
    }
    for (int r = lane; r <= K + K2; r += CF_WARP) acc_sm[r] = 0.0;
    __syncwarp();
    for (int m = 0; m < M; ++m) {
        R xs[K + 1];
#pragma unroll
        for (int d = 1; d <= K; ++d) {
            xs[d] = x0[d] + shf[m * CF_MAXDIM + d];
            if (xs[d] >= R(1)) xs[d] -= R(1);
        }
        R af = R(0), aw = R(0), a1[K], a2[K2];
#pragma unroll
        for (int r = 0; r < K; ++r) a1[r] = R(0);
#pragma unroll
        for (int r = 0; r < K2; ++r) a2[r] = R(0);
        const R* __restrict__ crow = chi + (size_t)m * N;
        R s_next = lane < N ? crow[lane] : R(1);  // the chi value one point ahead
        const float4* __restrict__ wrow = TAB ? wtab + (size_t)m * N * WQ : nullptr;
        float4 w_next[WQ];  // TAB: the coordinates one point ahead
        if constexpr (TAB) {
#pragma unroll
            for (int u = 0; u < WQ; ++u) w_next[u] = lane < N ? wrow[(size_t)lane * WQ + u] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        for (int i = lane; i < N; i += CF_WARP) {
            const R s = s_next;
            if (i + CF_WARP < N) s_next = crow[i + CF_WARP];
            float wc[4 * WQ];
            if constexpr (TAB) {
#pragma unroll
                for (int u = 0; u < WQ; ++u) {
                    wc[4 * u] = w_next[u].x; wc[4 * u + 1] = w_next[u].y;
                    wc[4 * u + 2] = w_next[u].z; wc[4 * u + 3] = w_next[u].w;
                }
                if (i + CF_WARP < N) {
#pragma unroll
                    for (int u = 0; u < WQ; ++u) w_next[u] = wrow[(size_t)(i + CF_WARP) * WQ + u];
                }
            }
            R y[K];
            R f = R(1);
#pragma unroll
            for (int r = 0; r < K; ++r) {
                R a = b[r] * s;
#pragma unroll
                for (int l = 0; l < r; ++l) a -= Lf[r][l] * y[l];
                const R e = m_ncdf(a * invd[r]);
                f *= e;
                R w;
                if constexpr (TAB) w = (R)wc[r];
                else w = R(1) - m_abs(R(2) * xs[r + 1] - R(1));
                R v = w * e;
                v = v < Lim<R>::vmin() ? Lim<R>::vmin() : v;
                v = v > Lim<R>::one_minus_ulp() ? Lim<R>::one_minus_ulp() : v;
                y[r] = m_ncdfinv(v);
                // no cut-off at Lim::tiny: a factor that underflows zeroes f by itself, and
                // the clamped v keeps y finite
            }
            // weight f s^2; X = L y / s2 is linear in y: accumulate f s^2 y / s2 =
            // f s rk y and f s^2 y y^T / s2^2 = f rk^2 y y^T, and apply L once per record
            const R fs = f * s;
            const R w1 = fs * rk, w2 = f * (rk * rk);
            af += f;
            aw += fs * s;
#pragma unroll
            for (int r = 0; r < K; ++r) {
                a1[r] += w1 * y[r];
                const R t = w2 * y[r];
#pragma unroll
                for (int c = 0; c <= r; ++c) a2[r * (r + 1) / 2 + c] += t * y[c];
            }
            if constexpr (!TAB) {
#pragma unroll
                for (int d = 1; d <= K; ++d) {
                    const R t = xs[d] - omdx[d];
                    xs[d] = t >= R(0) ? t : xs[d] + dx[d];
                }
            }
        }
        af = warp_sum(af);
        aw = warp_sum(aw);
#pragma unroll
        for (int r = 0; r < K; ++r) a1[r] = warp_sum(a1[r]);
#pragma unroll
        for (int r = 0; r < K2; ++r) a2[r] = warp_sum(a2[r]);
        if (lane == 0) {
            acc_sm[3 + K + K2 + m] = (double)af;  // alpha_s: this shift's sum
            acc_sm[0] += (double)aw;
#pragma unroll
            for (int r = 0; r < K; ++r) acc_sm[1 + r] += (double)a1[r];
#pragma unroll
            for (int r = 0; r < K2; ++r) acc_sm[1 + K + r] += (double)a2[r];
        }
    }
    __syncwarp();
    const double Sf = acc_sm[0];
    const double inv = Sf > 0.0 ? 1.0 / Sf : 0.0;
    // m1 = L E[y/s], m2 = L E[y y^T / s^2] L^T in FP64 (Lc is the full lower
    // factor), one output per lane, written back over the totals
    double o[2] = {0.0, 0.0};
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int t = lane + u * CF_WARP;
        if (t >= K + K2) break;
        double v = 0.0;
        if (t < K) {
            for (int l = 0; l <= t; ++l) v += Lc[t * K + l] * acc_sm[1 + l];
        } else {
            const int e = t - K;
            int r = 0;
            while ((r + 1) * (r + 2) / 2 <= e) ++r;
            const int c = e - r * (r + 1) / 2;
            for (int i = 0; i <= r; ++i) {
                double w = 0.0;
                for (int j = 0; j <= c; ++j)
                    w += acc_sm[1 + K + (i >= j ? i * (i + 1) / 2 + j : j * (j + 1) / 2 + i)] * Lc[c * K + j];
                v += Lc[r * K + i] * w;
            }
        }
        o[u] = v * inv;
    }
    __syncwarp();
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int t = lane + u * CF_WARP;
        if (t < K + K2) acc_sm[1 + t] = o[u];
    }
    __syncwarp();
    __syncwarp();
    if (lane == 0) {  // alpha_s: mean of the shift means and its standard error (Welford)
        double mean = 0.0, m2 = 0.0;
        for (int m = 0; m < M; ++m) {
            const double smean = acc_sm[3 + K + K2 + m] / (double)N;
            const double delta = smean - mean;
            mean += delta / (double)(m + 1);
            m2 += delta * (smean - mean);
        }
        acc_sm[1 + K + K2] = mean;
        acc_sm[2 + K + K2] = M > 1 ? sqrt(m2 / (double)(M - 1) / (double)M) : 0.0;
    }
    __syncwarp();
    *alpha_s = acc_sm[1 + K + K2];
    *se = acc_sm[2 + K + K2];
    return Sf / ((double)N * M);
}

// ---------------------------------------------------------------------------
// FP32 single-pass lattice pass of T_K with the truncated moments: the estimator of
// tk_lattice_mom_warp / tk_lattice_mom_tab_warp (same points, same weights), arranged
// for a GPU whose FP64 rate is a small fraction of its FP32 rate:
//   - every sum except the per-shift sums of f (alpha_s's standard error needs those)
//     stays in per-lane FP32 registers over all shifts, and the warp reduces each one
//     once per record instead of once per shift;
//   - the epilogue (the L-mapping of the moments, the mean and standard error of
//     alpha_s over the shifts) runs in FP32 on every lane; only the record's outputs
//     are widened to FP64;
//   - TAB: the baker-transformed coordinates of each point come from wtab (K <= 4);
//     P points per lane are in flight at once (independent chains of the separation
//     of variables), P = 1 without the table.
// Output protocol as tk_lattice_mom_warp: returns alpha (all lanes), *alpha_s, *se,
// and acc_sm[1 .. K + K(K+1)/2] the standardised moments (FP64, visible to the warp).
// acc_sm is this warp's slot of K + K(K+1)/2 + 3 + CF_MAXSHIFT doubles; its tail holds
// the per-shift sums as floats.
// ---------------------------------------------------------------------------
template <int K, bool TAB, int P, bool LW = false>
__device__ double tk_lattice_mom_f32(const double* bt, const double* Lc, const float* __restrict__ chi,
                                     const float* __restrict__ shf, const Lattice& lat, int lane,
                                     double* acc_sm, float rk, double* alpha_s, double* se,
                                     const float4* __restrict__ wtab, const float* __restrict__ lchi = nullptr,
                                     double* lw_out = nullptr)
{
    // LW (exact E[log W]): lchi holds log(s^2) at every point; *lw_out receives its
    // f-weighted mean over the points
    static_assert(TAB || P == 1, "P > 1 needs the coordinate table");
    static_assert(!TAB || K <= 4, "the coordinate table holds 4 coordinates");
    constexpr int K2 = K * (K + 1) / 2;
    constexpr int W = K + K2;
    float b[K], invd[K], Lf[K][K];
#pragma unroll
    for (int r = 0; r < K; ++r) {
        b[r] = (float)bt[r];
        invd[r] = 1.0f / (float)Lc[r * K + r];
#pragma unroll
        for (int l = 0; l < K; ++l) Lf[r][l] = l <= r ? (float)Lc[r * K + l] : 0.0f;
    }
    const int N = lat.N, M = lat.M;
    float* fshift = (float*)(acc_sm + W + 3);  // M per-shift sums of f
    float x0[K + 1], dx[K + 1], omdx[K + 1];   // coordinates advanced in floating point (!TAB)
    if constexpr (!TAB) {
        const float invN = 1.0f / (float)N;
#pragma unroll
        for (int d = 1; d <= K; ++d) {
            dx[d] = (float)(((long long)CF_WARP * lat.z[d]) % N) * invN;
            omdx[d] = 1.0f - dx[d];
            x0[d] = (float)(((long long)lane * lat.z[d]) % N) * invN;
        }
    }
    float aw = 0.0f, al = 0.0f, a1[K], a2[K2];
#pragma unroll
    for (int r = 0; r < K; ++r) a1[r] = 0.0f;
#pragma unroll
    for (int r = 0; r < K2; ++r) a2[r] = 0.0f;
    const float rk2 = rk * rk;
    for (int m = 0; m < M; ++m) {
        const float* __restrict__ crow = chi + (size_t)m * N;
        const float* __restrict__ lrow = LW ? lchi + (size_t)m * N : nullptr;
        float af = 0.0f;
        float xs[K + 1];
        if constexpr (!TAB) {
#pragma unroll
            for (int d = 1; d <= K; ++d) {
                xs[d] = x0[d] + shf[m * CF_MAXDIM + d];
                if (xs[d] >= 1.0f) xs[d] -= 1.0f;
            }
        }
        const float4* __restrict__ wrow = TAB ? wtab + (size_t)m * N : nullptr;
        for (int i0 = lane; i0 < N; i0 += CF_WARP * P) {
            float s[P], wc[P][4], ls[P];
            bool ok[P];
#pragma unroll
            for (int p = 0; p < P; ++p) {
                const int i = i0 + CF_WARP * p;
                ok[p] = i < N;
                s[p] = ok[p] ? crow[i] : 0.0f;
                if constexpr (LW) ls[p] = ok[p] ? lrow[i] : 0.0f;
                if constexpr (TAB) {
                    const float4 t = ok[p] ? wrow[i] : make_float4(0.f, 0.f, 0.f, 0.f);
                    wc[p][0] = t.x; wc[p][1] = t.y; wc[p][2] = t.z; wc[p][3] = t.w;
                }
            }
            float y[P][K], f[P];
#pragma unroll
            for (int p = 0; p < P; ++p) f[p] = 1.0f;
#pragma unroll
            for (int r = 0; r < K; ++r) {
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    float a = b[r] * s[p];
#pragma unroll
                    for (int l = 0; l < r; ++l) a -= Lf[r][l] * y[p][l];
                    const float e = cf_ncdf_f32(a * invd[r]);
                    f[p] *= e;
                    float w;
                    if constexpr (TAB) w = wc[p][r];
                    else w = 1.0f - fabsf(2.0f * xs[r + 1] - 1.0f);
                    float v = w * e;
                    v = v < Lim<float>::vmin() ? Lim<float>::vmin() : v;
                    v = v > Lim<float>::one_minus_ulp() ? Lim<float>::one_minus_ulp() : v;
                    y[p][r] = cf_ncdfinv_f32(v);
                }
            }
            // weight f s^2 (alpha at k2 dof); X = L y / s2 is linear in y: accumulate
            // f s rk y and f rk^2 y y^T and map through L once per record
#pragma unroll
            for (int p = 0; p < P; ++p) {
                const float fp = ok[p] ? f[p] : 0.0f;
                const float fs = fp * s[p];
                const float w1 = fs * rk, w2 = fp * rk2;
                af += fp;
                aw = fmaf(fs, s[p], aw);
                if constexpr (LW) al = fmaf(fp, ls[p], al);
#pragma unroll
                for (int r = 0; r < K; ++r) {
                    a1[r] = fmaf(w1, y[p][r], a1[r]);
                    const float t = w2 * y[p][r];
#pragma unroll
                    for (int c = 0; c <= r; ++c) a2[r * (r + 1) / 2 + c] = fmaf(t, y[p][c], a2[r * (r + 1) / 2 + c]);
                }
            }
            if constexpr (!TAB) {
#pragma unroll
                for (int d = 1; d <= K; ++d) {
                    const float t = xs[d] - omdx[d];
                    xs[d] = t >= 0.0f ? t : xs[d] + dx[d];
                }
            }
        }
        af = warp_sum(af);
        if (lane == 0) fshift[m] = af;
    }
    aw = warp_sum(aw);
    if constexpr (LW) al = warp_sum(al);
#pragma unroll
    for (int r = 0; r < K; ++r) a1[r] = warp_sum(a1[r]);
#pragma unroll
    for (int r = 0; r < K2; ++r) a2[r] = warp_sum(a2[r]);
    __syncwarp();
    // alpha_s: mean of the shift means and its standard error, shifts over lanes
    const float invN = 1.0f / (float)N;
    float sm0 = lane < M ? fshift[lane] * invN : 0.0f;
    float sm1 = lane + CF_WARP < M ? fshift[lane + CF_WARP] * invN : 0.0f;
    const float mean = warp_sum(sm0 + sm1) / (float)M;
    if constexpr (LW) {  // sum f = mean x N x M
        const float sf = mean * (float)N * (float)M;
        *lw_out = sf > 0.0f ? (double)(al / sf) : NAN;
    }
    const float d0 = lane < M ? sm0 - mean : 0.0f, d1 = lane + CF_WARP < M ? sm1 - mean : 0.0f;
    const float ss = warp_sum(d0 * d0 + d1 * d1);
    // the moments: m1 = L a1 / aw, m2 = L A L^T / aw (A the symmetric matrix of a2), on every
    // lane; lane t keeps output t
    const float inv = aw > 0.0f ? 1.0f / aw : 0.0f;
    float mine[2] = {0.0f, 0.0f};
#pragma unroll
    for (int t = 0; t < K; ++t) {
        float v = 0.0f;
#pragma unroll
        for (int l = 0; l <= t; ++l) v = fmaf(Lf[t][l], a1[l], v);
        if (lane == t) mine[0] = v * inv;
        if (lane + CF_WARP == t) mine[1] = v * inv;
    }
    float B[K][K];  // B = A L^T
#pragma unroll
    for (int i = 0; i < K; ++i)
#pragma unroll
        for (int c = 0; c < K; ++c) {
            float v = 0.0f;
#pragma unroll
            for (int j = 0; j <= c; ++j) v = fmaf(a2[i >= j ? i * (i + 1) / 2 + j : j * (j + 1) / 2 + i], Lf[c][j], v);
            B[i][c] = v;
        }
#pragma unroll
    for (int r = 0; r < K; ++r)
#pragma unroll
        for (int c = 0; c <= r; ++c) {
            float v = 0.0f;
#pragma unroll
            for (int i = 0; i <= r; ++i) v = fmaf(Lf[r][i], B[i][c], v);
            const int t = K + r * (r + 1) / 2 + c;
            if (lane == t) mine[0] = v * inv;
            if (lane + CF_WARP == t) mine[1] = v * inv;
        }
    __syncwarp();  // every lane has read the per-shift sums before the slot is overwritten
    if (lane < W) acc_sm[1 + lane] = (double)mine[0];
    if (lane + CF_WARP < W) acc_sm[1 + lane + CF_WARP] = (double)mine[1];
    __syncwarp();
    *alpha_s = (double)mean;
    *se = M > 1 ? (double)sqrtf(ss / (float)(M - 1) / (float)M) : 0.0;
    return (double)aw / ((double)N * M);
}
