// estep_common.cuh -- per-pair arithmetic of the E-step shared by the
// plan / combine kernels and the fused FP64 fix-up routine (FP64 throughout).
//
//   whiten        r = y - mu, z = Linv r, d = z^T z, c = A^T z, log t_p   (eqs 3-4)
//   limits_l0     standardised limits of alpha_s (eq 4, dof nu+p) and alpha
//                 (eq 13, dof nu+p+2):  c_i sqrt(nu'/(nu+d)) / sqrt(Lambda_ii)
//   limits_l1     T_{q-1}(c_{-r} - m_r; 0, V_r, nu+p+1) of xi_r, with
//                 S = ((nu+d)/(nu+p)) Lambda, m_r = S_{-r,r} c_r / S_rr,
//                 V_r = ((nu+p + c_r^2/S_rr)/(nu+p+1)) (S_{-r,-r} - S_{-r,r} S_{r,-r}/S_rr)
//   limits_l2     T_{q-2} at dof nu+p of the conditional mean
//                 E[X_s | X_r = c_r, X_{-r} <= c_{-r}] (same construction one level down
//                 with V' = nu2 V_r / (nu2 - 2), nu2 = nu+p+1)
//   assemble      eqs (4), (13), (15), (16), (17) from the integrals
#pragma once

#include "internal.cuh"
#include "special.cuh"

struct PairOut {
    double logf, u, elogu, se;
    double eu[CF_MAXQ];
    double euu[CF_MAXQ * CF_MAXQ];
};

// The mixed form's pair: log f in FP64, the conditional expectations in FP32 as assembled.
struct PairOutF {
    double logf;
    float u, elogu;
    float eu[CF_MAXQ];
    float euu[CF_MAXQ * CF_MAXQ];
};

// Mixed form: one FP32 row per pair, [u, E log w, eu (q), euu (q x q)], the layout the
// statistics kernel stages (widened to the FP64 pair buffers only when read back).

__device__ inline void store_pr32(float* row, int q, const PairOutF& o)
{
    row[0] = o.u;
    row[1] = o.elogu;
    for (int k = 0; k < q; ++k) row[2 + k] = o.eu[k];
    for (int k = 0; k < q * q; ++k) row[2 + q + k] = o.euu[k];
}

__device__ inline void store_pr32(float* row, int q, const PairOut& o)
{
    row[0] = (float)o.u;
    row[1] = (float)o.elogu;
    for (int k = 0; k < q; ++k) row[2 + k] = (float)o.eu[k];
    for (int k = 0; k < q * q; ++k) row[2 + q + k] = (float)o.euu[k];
}

__device__ inline void pair_whiten(const double* F, const Layout& Ly, int p, int q,
                                   const double* yj, double* d_out, double* c, double* logtp)
{
    double rr[CF_MAXP];
    for (int i = 0; i < p; ++i) rr[i] = yj[i] - F[Ly.mu + i];
    double d = 0.0;
    double z[CF_MAXP];
    for (int i = 0; i < p; ++i) {
        double s = 0.0;
        for (int l = 0; l <= i; ++l) s += F[Ly.Linv + i * p + l] * rr[l];
        z[i] = s;
        d += s * s;
    }
    for (int k = 0; k < q; ++k) {
        double s = 0.0;
        for (int i = 0; i < p; ++i) s += F[Ly.A + i * q + k] * z[i];
        c[k] = s;
    }
    const double nu = F[Ly.scal + SC_NU];
    *d_out = d;
    *logtp = isinf(nu) ? F[Ly.scal + SC_LOGTP] - 0.5 * d  // the normal limit (eq 2)
                       : F[Ly.scal + SC_LOGTP] - 0.5 * (nu + p) * log1p(d / nu);
}

// Mixed precision: the same whitening and log t_p in FP32 from FP32 copies of y
// and of the factor block.
// P > 0: p known at compile time (= P), the loops unrolled and the vectors in registers;
// P = 0: any p.  P a multiple of 4: y_j, mu and the rows of Linv read four values per
// load (F32 and yj 16-byte aligned; mu, Linv and A then start on 16-byte boundaries).
// The same operations in the same order in every case.
template <int P = 0>
__device__ inline void pair_whiten_f32(const float* F32, const Layout& Ly, int p_rt, int q, const float* yj,
                                       float* d_out, float* c, float* logtp)
{
    constexpr int NA = P > 0 ? P : CF_MAXP;
    const int p = P > 0 ? P : p_rt;
    float rr[NA], z[NA];
    if constexpr (P > 0 && P % 4 == 0) {
#pragma unroll
        for (int i = 0; i < P; i += 4) {
            const float4 y4 = *reinterpret_cast<const float4*>(yj + i);
            const float4 m4 = *reinterpret_cast<const float4*>(F32 + Ly.mu + i);
            rr[i] = y4.x - m4.x; rr[i + 1] = y4.y - m4.y; rr[i + 2] = y4.z - m4.z; rr[i + 3] = y4.w - m4.w;
        }
    } else {
#pragma unroll
        for (int i = 0; i < NA; ++i)
            if (i < p) rr[i] = yj[i] - F32[Ly.mu + i];
    }
    float d = 0.0f;
#pragma unroll
    for (int i = 0; i < NA; ++i) {
        if (i >= p) break;
        float s = 0.0f;
        if constexpr (P > 0 && P % 4 == 0) {
#pragma unroll
            for (int l4 = 0; l4 <= i; l4 += 4) {
                const float4 w = *reinterpret_cast<const float4*>(F32 + Ly.Linv + i * P + l4);
                s = fmaf(w.x, rr[l4], s);
                if (l4 + 1 <= i) s = fmaf(w.y, rr[l4 + 1], s);
                if (l4 + 2 <= i) s = fmaf(w.z, rr[l4 + 2], s);
                if (l4 + 3 <= i) s = fmaf(w.w, rr[l4 + 3], s);
            }
        } else {
#pragma unroll
            for (int l = 0; l <= i; ++l) s = fmaf(F32[Ly.Linv + i * p + l], rr[l], s);
        }
        z[i] = s;
        d = fmaf(s, s, d);
    }
    for (int k = 0; k < q; ++k) {
        float s = 0.0f;
#pragma unroll
        for (int i = 0; i < NA; ++i)
            if (i < p) s = fmaf(F32[Ly.A + i * q + k], z[i], s);
        c[k] = s;
    }
    const float nu = F32[Ly.scal + SC_NU];
    *d_out = d;
    *logtp = isinf(nu) ? F32[Ly.scal + SC_LOGTP] - 0.5f * d
                       : F32[Ly.scal + SC_LOGTP] - 0.5f * (nu + p) * log1pf(d / nu);
}

// Limits of the records, in T = double (F the factor block) or, in the mixed
// form, T = float (F its FP32 copy).
// which = 0: alpha_s (dof nu+p); which = 1: alpha (dof nu+p+2)
template <typename T>
__device__ inline void limits_l0(const T* F, const Layout& Ly, int p, int q, const T* c, T d, int which, T* bt)
{
    const T nu = F[Ly.scal + SC_NU], nu1 = nu + p;
    const T f = isinf(nu) ? T(1) : m_sqrt((nu1 + T(2) * which) / (nu + d));  // 1 in the normal limit
    for (int k = 0; k < q; ++k) bt[k] = c[k] * f * F[Ly.dq + k];
}

// Level-1 limits for coordinate r; returns the scale factor sc1 (V_r = sc1 schur_r).
template <typename T>
__device__ inline T limits_l1(const T* F, const Layout& Ly, int p, int q, const T* c, T d, int r, T* bt)
{
    const int q1 = q - 1;
    const T nu = F[Ly.scal + SC_NU], nu1 = nu + p;
    const bool nrm = isinf(nu);  // the normal limit: every t scaling is 1
    const T k0 = nrm ? T(1) : (nu + d) / nu1;
    const T Srr = k0 * F[Ly.Lam + r * q + r];
    const T* blk = F + Ly.l1 + r * Ly.l1s;
    const T* mvec = blk;
    const T* dsc = blk + q1 + q1 * q1;
    const T kap1 = nrm ? T(1) : (nu1 + c[r] * c[r] / Srr) / (nu1 + T(1));
    const T sc1 = kap1 * k0;
    const T isc = T(1) / m_sqrt(sc1);
    for (int i = 0; i < q1; ++i) {
        const int b = i < r ? i : i + 1;
        bt[i] = (c[b] - mvec[i] * c[r]) * dsc[i] * isc;
    }
    return sc1;
}

template <typename T>
__device__ inline void limits_l2(const T* F, const Layout& Ly, int p, int q, const T* c, T d, int r, int s, T* bt)
{
    const int q1 = q - 1, q2 = q - 2;
    const T nu = F[Ly.scal + SC_NU], nu1 = nu + p, nu2 = nu1 + T(1);
    const bool nrm = isinf(nu);  // the normal limit: every t scaling is 1
    const T k0 = nrm ? T(1) : (nu + d) / nu1;
    const T Srr = k0 * F[Ly.Lam + r * q + r];
    const T* blk = F + Ly.l1 + r * Ly.l1s;
    const T* mvec = blk;
    const T* sch = blk + q1;
    T cp[CF_MAXQ];
    for (int i = 0; i < q1; ++i) {
        const int b = i < r ? i : i + 1;
        cp[i] = c[b] - mvec[i] * c[r];
    }
    const T sc1 = nrm ? T(1) : (nu1 + c[r] * c[r] / Srr) / (nu1 + T(1)) * k0;
    const T kp = nrm ? T(1) : nu2 / (nu2 - T(2)) * sc1;
    const T Vss = kp * sch[s * q1 + s];
    const T* b2 = F + Ly.l2 + (r * q1 + s) * Ly.l2s;
    const T* mv2 = b2;
    const T* ds2 = b2 + q2;
    const T kap2 = nrm ? T(1) : (nu2 - T(2) + cp[s] * cp[s] / Vss) / (nu2 - T(1));
    const T isc2 = T(1) / m_sqrt(kap2 * kp);
    for (int i = 0; i < q2; ++i) {
        const int b = i < s ? i : i + 1;
        bt[i] = (cp[b] - mv2[i] * cp[s]) * ds2[i] * isc2;
    }
}

// Offsets of the correlation Cholesky factors used by each level.
__device__ inline int fac_l0(const Layout& Ly) { return Ly.Lq; }
__device__ inline int fac_l1(const Layout& Ly, int q, int r)
{
    const int q1 = q - 1;
    return Ly.l1 + r * Ly.l1s + 2 * q1 + q1 * q1;
}
__device__ inline int fac_l2(const Layout& Ly, int q, int r, int s)
{
    const int q1 = q - 1, q2 = q - 2;
    return Ly.l2 + (r * q1 + s) * Ly.l2s + 2 * q2;
}

// A pair whose T_q is 0 in the working precision (beyond the range of the
// arithmetic on this component's skewing side): log f = -inf, so tau = 0 (eq 12),
// and the conditional expectations, which enter eqs (18)-(22) only multiplied by
// tau, are set to u = 1, E[log w] = 0, e2 = 0, e3 = 0 instead of a 0/0.
template <typename O>
__device__ inline void pair_null(int q, int density_only, O& o)
{
    o.logf = -INFINITY;
    if (density_only) return;
    o.u = 1;
    o.elogu = 0;
    for (int a = 0; a < q; ++a) o.eu[a] = 0;
    for (int a = 0; a < q * q; ++a) o.euu[a] = 0;
}

// tq1[r] = T_{q-1} of level 1 (1 when q = 1); tq2[r*(q-1)+s] = T_{q-2} of
// level 2 (1 when q <= 2).
// cst: per-dof constants of this component's dof nu+p (table index 3h)
__device__ inline void pair_assemble(const double* F, const Layout& Ly, int p, int q,
                                     const double* c, double d, double logtp, double alpha_s,
                                     double alpha, const double* tq1, const double* tq2,
                                     int density_only, const double* cst, PairOut& o)
{
    const double nu = F[Ly.scal + SC_NU], nu1 = nu + p;
    const bool nrm = isinf(nu);  // the normal limit (eq 5): u = 1, every t scaling is 1
    if (!(alpha_s > 0.0)) return pair_null(q, density_only, o);
    o.logf = q * 0.6931471805599453 + logtp + log(alpha_s);  // eq (4)
    if (density_only) return;
    const double u = nrm ? 1.0 : nu1 / (nu + d) * alpha / alpha_s;  // eq (13)
    o.u = u;
    o.elogu = nrm ? 0.0 : u - log(0.5 * (nu + d)) - nu1 / (nu + d) + F[Ly.scal + SC_PSI];  // eq (15)
    const double* Lam = F + Ly.Lam;
    const double k0 = nrm ? 1.0 : (nu + d) / nu1;
    const int q1 = q - 1;
    double xi[CF_MAXQ], H[CF_MAXQ * CF_MAXQ];
    for (int i = 0; i < q * q; ++i) H[i] = 0.0;
    for (int r = 0; r < q; ++r) {
        const double Srr = k0 * Lam[r * q + r];
        const double t1q = q1 > 0 ? tq1[r] : 1.0;
        xi[r] = exp(nrm ? cf_lognorm1(c[r], Srr) : cf_logt1(c[r], Srr, nu1, cst[CST_LT1])) * t1q;
        H[r * q + r] = c[r] * xi[r];
        if (q1 == 0 || xi[r] == 0.0) continue;
        const double* blk = F + Ly.l1 + r * Ly.l1s;
        const double* mvec = blk;
        const double* sch = blk + q1;
        double cp[CF_MAXQ];
        for (int i = 0; i < q1; ++i) {
            const int b = i < r ? i : i + 1;
            cp[i] = c[b] - mvec[i] * c[r];
        }
        const double nu2 = nu1 + 1.0;
        const double sc1 = nrm ? 1.0 : (nu1 + c[r] * c[r] / Srr) / (nu1 + 1.0) * k0;
        const double kp = nrm ? 1.0 : nu2 / (nu2 - 2.0) * sc1;
        double xip[CF_MAXQ];
        for (int s = 0; s < q1; ++s) {
            const double Vss = kp * sch[s * q1 + s];
            const double t2q = q1 > 1 ? tq2[r * q1 + s] : 1.0;
            xip[s] = exp(nrm ? cf_lognorm1(cp[s], Vss) : cf_logt1(cp[s], Vss, nu2 - 2.0, cst[CST_LT1M])) * t2q;
        }
        // E[Y 1(Y <= c')] = -(nu2/(nu2-2)) V_r xi', V_r = sc1 schur_r (-V_r xi' when normal)
        // divided last: t1q may be subnormal while s / t1q (a Mills-type ratio) is moderate
        const double fac = nrm ? -1.0 : -(nu2 / (nu2 - 2.0)) * sc1;
        for (int i = 0; i < q1; ++i) {
            double s = 0.0;
            for (int t = 0; t < q1; ++t) s += sch[i * q1 + t] * xip[t];
            const int b = i < r ? i : i + 1;
            H[r * q + b] = xi[r] * (mvec[i] * c[r] + fac * s / t1q);
        }
    }
    double Lxi[CF_MAXQ];
    for (int a = 0; a < q; ++a) {
        double s = 0.0;
        for (int k = 0; k < q; ++k) s += Lam[a * q + k] * xi[k];
        Lxi[a] = s;
        o.eu[a] = u * c[a] + s / alpha_s;  // eq (16)
    }
    for (int a = 0; a < q; ++a)
        for (int b = 0; b <= a; ++b) {  // eq (17), symmetrised
            double lh1 = 0.0, lh2 = 0.0;
            for (int k = 0; k < q; ++k) {
                lh1 += Lam[a * q + k] * H[k * q + b];
                lh2 += Lam[b * q + k] * H[k * q + a];
            }
            const double v = u * c[a] * c[b] + (c[a] * Lxi[b] + Lxi[a] * c[b]) / alpha_s + Lam[a * q + b]
                           - 0.5 * (lh1 + lh2) / alpha_s;
            o.euu[a * q + b] = v;
            o.euu[b * q + a] = v;
        }
}

// Single-pass reading of eqs (13), (16), (17): alpha and the standardised
// moments m = (E[X~], lower triangle of E[X~ X~^T]) of the truncated
// X ~ t_q(0, S2, nu+p+2), S2 = ((nu+d)/(nu+p+2)) Lambda, X <= c, come from one
// lattice pass; X = sigma * X~ with sigma_i = sqrt(S2_ii); U = c - X.
// lw: the f-weighted mean of log(s^2) over the pass (exact E[log W]), or NaN for the
// one-step-late form of eq (15)
__device__ inline void pair_assemble_sp(const double* F, const Layout& Ly, int p, int q,
                                        const double* c, double d, double logtp, double alpha_s,
                                        double alpha, const double* m, PairOut& o, double lw = NAN)
{
    const double nu = F[Ly.scal + SC_NU], nu1 = nu + p;
    const bool nrm = isinf(nu);  // the normal limit (eq 5): u = 1, X ~ N(0, Lambda)
    if (!(alpha_s > 0.0)) return pair_null(q, 0, o);
    o.logf = q * 0.6931471805599453 + logtp + log(alpha_s);  // eq (4)
    const double u = nrm ? 1.0 : nu1 / (nu + d) * alpha / alpha_s;  // eq (13)
    o.u = u;
    // eq (15), or the exact E[log W | y]: W = s^2 (nu+p)/(nu+d) at every point of the pass
    o.elogu = nrm ? 0.0 : !isnan(lw) ? lw + log(nu1 / (nu + d))
                                     : u - log(0.5 * (nu + d)) - nu1 / (nu + d) + F[Ly.scal + SC_PSI];
    const double sc = nrm ? 1.0 : sqrt((nu + d) / (nu1 + 2.0));
    double sig[CF_MAXQ], m1[CF_MAXQ];
    for (int a = 0; a < q; ++a) {
        sig[a] = sc / F[Ly.dq + a];
        m1[a] = sig[a] * m[a];
        o.eu[a] = u * (c[a] - m1[a]);  // eq (16)
    }
    for (int a = 0; a < q; ++a)
        for (int b = 0; b <= a; ++b) {  // eq (17)
            const double m2 = sig[a] * sig[b] * m[q + a * (a + 1) / 2 + b];
            const double v = u * (c[a] * c[b] - c[a] * m1[b] - m1[a] * c[b] + m2);
            o.euu[a * q + b] = v;
            o.euu[b * q + a] = v;
        }
}

// Mixed precision: the assembly of pair_assemble in FP32 (log f keeps the
// FP64 log t_p and adds log alpha_s computed in FP32).
// F: the component's FP32 factor block, cst its FP32 per-dof constants (conversions from
// FP64 run on GB300's FP64 pipe, 1/64 of the FP32 rate: the per-component values are read
// from their FP32 copies).
__device__ inline void pair_assemble_f32(const float* F, const Layout& Ly, int p, int q,
                                         const float* cf, float d, float logtp, float alpha_s,
                                         float alpha, const float* tq1, const float* tq2,
                                         int density_only, const float* cst, PairOutF& o)
{
    if (!(alpha_s > 0.0f)) return pair_null(q, density_only, o);
    // eq (4): log t_p + log alpha_s in FP32 (both FP32 quantities), q log 2 added in FP64
    o.logf = q * 0.6931471805599453 + (double)(logtp + logf(alpha_s));
    if (density_only) return;
    const float nu = F[Ly.scal + SC_NU], nu1 = nu + (float)p;
    float c[CF_MAXQ];
    for (int k = 0; k < q; ++k) c[k] = cf[k];
    const bool nrm = isinf(nu);  // the normal limit (eq 5): u = 1, every t scaling is 1
    const float u = nrm ? 1.0f : nu1 / (nu + d) * alpha / alpha_s;  // eq (13)
    o.u = u;
    o.elogu = nrm ? 0.0f : u - logf(0.5f * (nu + d)) - nu1 / (nu + d) + F[Ly.scal + SC_PSI];  // eq (15)
    float Lam[CF_MAXQ * CF_MAXQ];
    for (int i = 0; i < q * q; ++i) Lam[i] = F[Ly.Lam + i];
    const float k0 = nrm ? 1.0f : (nu + d) / nu1;
    const float lt1 = cst[CST_LT1], lt1m = cst[CST_LT1M];
    const int q1 = q - 1;
    float xi[CF_MAXQ], H[CF_MAXQ * CF_MAXQ];
    for (int i = 0; i < q * q; ++i) H[i] = 0.0f;
    for (int r = 0; r < q; ++r) {
        const float Srr = k0 * Lam[r * q + r];
        const float t1q = q1 > 0 ? tq1[r] : 1.0f;
        xi[r] = expf(nrm ? -0.5f * logf(2.0f * (float)CF_PI * Srr) - 0.5f * c[r] * c[r] / Srr
                         : lt1 - 0.5f * logf(Srr) - 0.5f * (nu1 + 1.0f) * log1pf(c[r] * c[r] / (nu1 * Srr))) * t1q;
        H[r * q + r] = c[r] * xi[r];
        if (q1 == 0 || xi[r] == 0.0f) continue;
        const float* blk = F + Ly.l1 + r * Ly.l1s;
        float mvec[CF_MAXQ], sch[CF_MAXQ * CF_MAXQ], cp[CF_MAXQ];
        for (int i = 0; i < q1; ++i) mvec[i] = blk[i];
        for (int i = 0; i < q1 * q1; ++i) sch[i] = blk[q1 + i];
        for (int i = 0; i < q1; ++i) {
            const int b = i < r ? i : i + 1;
            cp[i] = c[b] - mvec[i] * c[r];
        }
        const float nu2 = nu1 + 1.0f;
        const float sc1 = nrm ? 1.0f : (nu1 + c[r] * c[r] / Srr) / (nu1 + 1.0f) * k0;
        const float kp = nrm ? 1.0f : nu2 / (nu2 - 2.0f) * sc1;
        float xip[CF_MAXQ];
        for (int s = 0; s < q1; ++s) {
            const float Vss = kp * sch[s * q1 + s];
            const float t2q = q1 > 1 ? tq2[r * q1 + s] : 1.0f;
            const float nuv = nu2 - 2.0f;
            xip[s] = expf(nrm ? -0.5f * logf(2.0f * (float)CF_PI * Vss) - 0.5f * cp[s] * cp[s] / Vss
                              : lt1m - 0.5f * logf(Vss) - 0.5f * (nuv + 1.0f) * log1pf(cp[s] * cp[s] / (nuv * Vss))) * t2q;
        }
        const float fac = nrm ? -1.0f : -(nu2 / (nu2 - 2.0f)) * sc1;  // divided last, as above
        for (int i = 0; i < q1; ++i) {
            float s = 0.0f;
            for (int t = 0; t < q1; ++t) s += sch[i * q1 + t] * xip[t];
            const int b = i < r ? i : i + 1;
            H[r * q + b] = xi[r] * (mvec[i] * c[r] + fac * s / t1q);
        }
    }
    float Lxi[CF_MAXQ];
    for (int a = 0; a < q; ++a) {
        float s = 0.0f;
        for (int k = 0; k < q; ++k) s += Lam[a * q + k] * xi[k];
        Lxi[a] = s;
        o.eu[a] = u * c[a] + s / alpha_s;  // eq (16)
    }
    for (int a = 0; a < q; ++a)
        for (int b = 0; b <= a; ++b) {  // eq (17), symmetrised
            float lh1 = 0.0f, lh2 = 0.0f;
            for (int k = 0; k < q; ++k) {
                lh1 += Lam[a * q + k] * H[k * q + b];
                lh2 += Lam[b * q + k] * H[k * q + a];
            }
            const float v = u * c[a] * c[b] + (c[a] * Lxi[b] + Lxi[a] * c[b]) / alpha_s + Lam[a * q + b]
                          - 0.5f * (lh1 + lh2) / alpha_s;
            o.euu[a * q + b] = v;
            o.euu[b * q + a] = v;
        }
}
