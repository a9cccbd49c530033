// setup.cu -- per-component factors (S0) and the chi table (S1).
//
// S0, one warp per component, FP64 (definitions under eq (4)):
//   Omega = Sigma + Delta Delta^T, L = chol(Omega), Linv = L^{-1},
//   log|Omega|, A = Linv Delta (so c = A^T Linv (y - mu), d = |Linv (y-mu)|^2),
//   Lambda = I - Delta^T Omega^{-1} Delta = I - A^T A,
//   the constant of the log t_p density (eq 3) and psi((nu+p)/2) of eq (15),
//   and for the truncated-t moments the correlation Cholesky factors of
//   Lambda, of its Schur complements at each r, and of theirs at each s.
// S1: s = sqrt(chi2_nu'^{-1}(w_0)/nu') at every (shift, lattice point) for
//   each tabulated dof nu'; independent of the observations.
#include "internal.cuh"
#include "special.cuh"

namespace {

// Cholesky (lower, row-major, n x n); returns false if not positive definite.
__device__ bool chol_dev(int n, const double* A, double* L)
{
    for (int j = 0; j < n; ++j) {
        double s = A[j * n + j];
        for (int k = 0; k < j; ++k) s -= L[j * n + k] * L[j * n + k];
        if (!(s > 0.0)) return false;
        const double dj = sqrt(s);
        L[j * n + j] = dj;
        for (int i = j + 1; i < n; ++i) {
            double t = A[i * n + j];
            for (int k = 0; k < j; ++k) t -= L[i * n + k] * L[j * n + k];
            L[i * n + j] = t / dj;
        }
        for (int i = 0; i < j; ++i) L[i * n + j] = 0.0;
    }
    return true;
}

// Correlation Cholesky and 1/sqrt(diag) of an n x n scale matrix S.
__device__ bool corr_chol_dev(int n, const double* S, double* dsc, double* Lc)
{
    double R[CF_MAXQ * CF_MAXQ];
    for (int i = 0; i < n; ++i) {
        if (!(S[i * n + i] > 0.0)) return false;
        dsc[i] = 1.0 / sqrt(S[i * n + i]);
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) R[i * n + j] = S[i * n + j] * dsc[i] * dsc[j];
    for (int i = 0; i < n; ++i) R[i * n + i] = 1.0;
    return chol_dev(n, R, Lc);
}

// Schur complement of an n x n matrix S at index r: (n-1) x (n-1), and the
// regression coefficients S_{-r,r}/S_rr.
__device__ void schur_dev(int n, const double* S, int r, double* out, double* mvec)
{
    const double srr = S[r * n + r];
    int ii = 0;
    for (int i = 0; i < n; ++i) {
        if (i == r) continue;
        mvec[ii] = S[i * n + r] / srr;
        int jj = 0;
        for (int j = 0; j < n; ++j) {
            if (j == r) continue;
            out[ii * (n - 1) + jj] = S[i * n + j] - S[i * n + r] * S[r * n + j] / srr;
            ++jj;
        }
        ++ii;
    }
}

}  // namespace

__global__ void __launch_bounds__(32) setup_components_kernel(Dims D, Layout Ly, const double* mu,
                                                              const double* Sigma, const double* Delta,
                                                              const double* nu, double* F, int* flags)
{
    // one warp per component (blockIdx.x); lane i owns row i (Cholesky, A) or column i
    // (L^{-1}); every element is summed in the same order as a serial loop would
    __shared__ double W[CF_MAXP * CF_MAXP];
    __shared__ double Li[CF_MAXP * CF_MAXP];
    const int h = blockIdx.x, lane = threadIdx.x;
    if (h >= D.g) return;
    const int p = D.p, q = D.q;
    const double* Sg = Sigma + (size_t)h * p * p;
    const double* Dl = Delta + (size_t)h * p * q;
    double* Fh = F + (size_t)h * Ly.stride;

    for (int i = lane; i < p; i += 32) Fh[Ly.mu + i] = mu[(size_t)h * p + i];
    // Omega = Sigma + Delta Delta^T (lower triangle of W)
    for (int e = lane; e < p * p; e += 32) {
        const int i = e / p, j = e % p;
        if (j > i) continue;
        double s = Sg[i * p + j];
        for (int k = 0; k < q; ++k) s += Dl[i * q + k] * Dl[j * q + k];
        W[i * p + j] = s;
    }
    __syncwarp();
    // L = chol(Omega) in place, column j at step j: lane i >= j forms its row's entry
    double logdet = 0.0;
    for (int j = 0; j < p; ++j) {
        double t = 0.0;
        if (lane >= j && lane < p) {
            t = W[lane * p + j];
            for (int k = 0; k < j; ++k) t -= W[lane * p + k] * W[j * p + k];
        }
        const double sjj = __shfl_sync(0xffffffffu, t, j);
        if (!(sjj > 0.0)) {
            if (lane == 0) atomicOr(flags, KF_NOTPD_OMEGA);
            return;
        }
        const double dj = sqrt(sjj);
        logdet += 2.0 * log(dj);
        __syncwarp();
        if (lane == j) W[j * p + j] = dj;
        else if (lane > j && lane < p) W[lane * p + j] = t / dj;
        __syncwarp();
    }
    // Linv = L^{-1}: lane c forward-substitutes column c
    for (int c = lane; c < p; c += 32)
        for (int i = 0; i < p; ++i) {
            if (i < c) { Li[i * p + c] = 0.0; continue; }
            double s = (i == c) ? 1.0 : 0.0;
            for (int k = c; k < i; ++k) s -= W[i * p + k] * Li[k * p + c];
            Li[i * p + c] = s / W[i * p + i];
        }
    __syncwarp();
    for (int e = lane; e < p * p; e += 32) Fh[Ly.Linv + e] = Li[e];
    // A = Linv Delta (lane i: row i), into W's upper part is not needed: A goes to Fh and smem
    __shared__ double As[CF_MAXP * CF_MAXQ];
    __shared__ double Lam[CF_MAXQ * CF_MAXQ];
    for (int i = lane; i < p; i += 32)
        for (int k = 0; k < q; ++k) {
            double s = 0.0;
            for (int l = 0; l <= i; ++l) s += Li[i * p + l] * Dl[l * q + k];
            As[i * q + k] = s;
            Fh[Ly.A + i * q + k] = s;
        }
    __syncwarp();
    // Lambda = I - A^T A
    for (int e = lane; e < q * q; e += 32) {
        const int a = e / q, b = e % q;
        double s = (a == b) ? 1.0 : 0.0;
        for (int i = 0; i < p; ++i) s -= As[i * q + a] * As[i * q + b];
        Lam[e] = s;
        Fh[Ly.Lam + e] = s;
    }
    __syncwarp();
    const double v = nu[h];
    if (lane == 0) {
        Fh[Ly.scal + SC_NU] = v;
        if (isinf(v)) {  // nu = infinity: the normal density of eq (2) (CFUSN, eq 5); no eq (15)
            Fh[Ly.scal + SC_LOGTP] = -0.5 * p * log(2.0 * CF_PI) - 0.5 * logdet;
            Fh[Ly.scal + SC_PSI] = 0.0;
        } else {
            Fh[Ly.scal + SC_LOGTP] = lgamma(0.5 * (v + p)) - lgamma(0.5 * v) - 0.5 * p * log(v * CF_PI)
                                   - 0.5 * logdet;
            Fh[Ly.scal + SC_PSI] = cf_digamma(0.5 * (v + p));
        }
        Fh[Ly.scal + 3] = 0.0;
        if (!corr_chol_dev(q, Lam, Fh + Ly.dq, Fh + Ly.Lq)) atomicOr(flags, KF_NOTPD_LAMBDA);
    }
    // level 1: Schur complement of Lambda at each r (lane r), level 2 inside
    const int q1 = q - 1, q2 = q - 2;
    if (lane < q && q1 > 0) {
        const int r = lane;
        double* blk = Fh + Ly.l1 + r * Ly.l1s;
        double* mvec = blk;
        double* sch = blk + q1;
        double* dsc = sch + q1 * q1;
        double* Lc = dsc + q1;
        schur_dev(q, Lam, r, sch, mvec);
        if (!corr_chol_dev(q1, sch, dsc, Lc)) {
            atomicOr(flags, KF_NOTPD_LAMBDA);
            return;
        }
        for (int s2 = 0; s2 < q1 && q2 > 0; ++s2) {
            double* b2 = Fh + Ly.l2 + (r * q1 + s2) * Ly.l2s;
            double sch2[CF_MAXQ * CF_MAXQ];
            schur_dev(q1, sch, s2, sch2, b2);
            if (!corr_chol_dev(q2, sch2, b2 + q2, b2 + 2 * q2)) {
                atomicOr(flags, KF_NOTPD_LAMBDA);
                return;
            }
        }
    }
}

// s = sqrt(chi2_{dof}^{-1}(w_0)/dof) for every dof in `dofs`, shift m and point i.
// Lattice coordinate 0: x = frac(i/N + shift(m, 0)), w = 1 - |2x - 1|.
// rtol: Newton tolerance of the quantile (1e-15 when the FP64 table is used, 1e-9 when only
// the FP32 table is); cst: the per-dof constants (lgamma(dof/2) at CST_LGA).
// Tables k = 0, every, 2 every, ... < ndof (every = 3: only the dof nu+p tables,
// all that the single-pass E-step reads).
__global__ void chi_table_kernel(int ndof, int every, const double* __restrict__ dofs, const double* __restrict__ cst,
                                 Lattice lat, const double* __restrict__ shf, double rtol,
                                 double* __restrict__ t64, float* __restrict__ t32,
                                 double* __restrict__ l64, float* __restrict__ l32)
{
    const long long NM = (long long)lat.M * lat.N;
    const long long total = (long long)((ndof + every - 1) / every) * NM;
    for (long long te = blockIdx.x * (long long)blockDim.x + threadIdx.x; te < total;
         te += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(te % lat.N);
        const int m = (int)((te / lat.N) % lat.M);
        const int k = (int)(te / NM) * every;
        const long long t = k * NM + (te % NM);
        const double dof = dofs[k];
        double x = (double)(((long long)i * lat.z[0]) % lat.N) / (double)lat.N + shf[m * CF_MAXDIM];
        if (x >= 1.0) x -= 1.0;
        const double wc = fabs(2.0 * x - 1.0);
        const double w = 1.0 - wc;
        // dof = infinity (the normal limit): no chi variable, s = 1
        const double x2 = isinf(dof) ? 1.0 : cf_chi2_quantile(w, wc, dof, cst[k * CST_STRIDE + CST_LGA], rtol) / dof;
        const double s = sqrt(x2);
        t64[t] = s;
        t32[t] = (float)s;
        if (l64) {  // log(s^2) (exact E[log W])
            const double ls = log(x2);
            l64[t] = ls;
            l32[t] = (float)ls;
        }
    }
}

// Degrees of freedom and T_1/T_2 constants for every table index t:
// E-step tables t = 3h + j have dof nu_h + p + j (j = 0: T_q and T_{q-2},
// j = 1: T_{q-1}, j = 2: T_q at nu+p+2); with F == nullptr the dofs are
// already given (cfust_tk_eval, one index per case).
__global__ void dof_consts_kernel(Dims D, Layout Ly, const double* __restrict__ F, int ndof,
                                  double* dofs, double* c64, float* c32)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ndof; t += gridDim.x * blockDim.x) {
        double v;
        if (F) {
            const int h = t / 3, j = t % 3;
            v = F[(size_t)h * Ly.stride + Ly.scal + SC_NU] + D.p + j;
            dofs[t] = v;
        } else {
            v = dofs[t];
        }
        if (isinf(v)) {  // the normal limit uses none of these constants
            for (int k = 0; k < CST_STRIDE; ++k) {
                c64[t * CST_STRIDE + k] = 0.0;
                c32[t * CST_STRIDE + k] = 0.0f;
            }
            continue;
        }
        const double lt = lgamma(0.5 * (v + 1.0)) - lgamma(0.5 * v) - 0.5 * log(v * CF_PI);
        const double ltm = lgamma(0.5 * v) - lgamma(0.5 * (v - 1.0)) - 0.5 * log((v - 1.0) * CF_PI);
        const double c[CST_STRIDE] = {t1_lgb(v), t1_lgb(v + 1.0),
                                      exp(lgamma(0.5 * (v + 1.0)) - lgamma(0.5 * v)) / sqrt(CF_PI),
                                      lt, v > 1.0 ? ltm : 0.0, lgamma(0.5 * v), 0.0, 0.0};
        for (int k = 0; k < CST_STRIDE; ++k) {
            c64[t * CST_STRIDE + k] = c[k];
            c32[t * CST_STRIDE + k] = (float)c[k];
        }
    }
}

// FP32 observations widened to FP64 (row stride ld).
__global__ void widen_kernel(const float* __restrict__ src, long long ld, Dims D,
                             double* __restrict__ dst)
{
    const long long total = D.n * D.p;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long j = t / D.p;
        const int i = (int)(t % D.p);
        dst[t] = (double)src[j * ld + i];
    }
}

// FP64 observations narrowed to FP32 (mixed precision copy).
__global__ void narrow_kernel(const double* __restrict__ src, Dims D, float* __restrict__ dst)
{
    const long long total = D.n * D.p;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x)
        dst[t] = (float)src[t];
}

// log T_1(-w; nu) for w >= 0 in FP64, without underflow: with x = nu/(nu+w^2),
// T_1(-w) = I_x(nu/2, 1/2)/2 from the continued fraction in log form; lbeta =
// lgamma((nu+1)/2) - lgamma(nu/2) - lgamma(1/2), the table's constant.
static __device__ double log_t1_lower(double w, double nu, double lbeta)
{
    if (w == 0.0) return -CF_LN2;
    const double w2 = w * w, den = nu + w2;
    const double x = nu / den, y = w2 / den;
    const double a = 0.5 * nu, b = 0.5;
    const double lbt = lbeta + a * log(x) + b * log(y);
    if (x < (a + 1.0) / (a + b + 2.0))
        return lbt + log(betacf_dev<double>(a, b, x)) - log(a) - CF_LN2;
    return log1p(-exp(lbt) * betacf_dev<double>(b, a, y) / b) - CF_LN2;
}

// Tables of log2 T_1(-|z|; dofs[t] + 1) and d/dv on the grid uniform in v = log2(1 + |z|)
// (see IntegArgs::t1tab).
// jmask: the tables t with bit (t mod 3) set are built (E-step tables t = 3h + j; the
// others are left as they are: no record reads them); 7 builds every table.
// cst: the per-dof constants of dof_consts_kernel (CST_LGB1: lbeta at dofs[t] + 1).
__global__ void t1_table_kernel(int ndof, const double* __restrict__ dofs, const double* __restrict__ cst,
                                float2* __restrict__ tab, int jmask)
{
    const long long total = (long long)ndof * T1TAB_N;
    const double hv = (double)T1TAB_V / (T1TAB_N - 1);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int t = (int)(e / T1TAB_N), i = (int)(e % T1TAB_N);
        if (!((jmask >> (t % 3)) & 1)) continue;
        const double nu = dofs[t] + 1.0;
        if (isinf(nu)) {  // the normal limit evaluates Phi_2 directly, not through this table
            tab[e] = make_float2(0.0f, 0.0f);
            continue;
        }
        const double v = i * hv;
        const double w = expm1(v * CF_LN2);
        const double lbeta = cst[t * CST_STRIDE + CST_LGB1];
        const double lT = log_t1_lower(w, nu, lbeta);
        // d/dv log2 T_1(-w(v)) = -t_nu(w) (1 + w) / T_1(-w)   (dw/dv = (1 + w) ln 2); the
        // density's constant lgamma((nu+1)/2) - lgamma(nu/2) - log(nu pi)/2 is lbeta - log(nu)/2
        const double lt = lbeta - 0.5 * log(nu) - 0.5 * (nu + 1.0) * log1p(w * w / nu);
        const double d = -exp(lt - lT) * (1.0 + w);
        tab[e] = make_float2((float)(lT / CF_LN2), (float)d);
    }
}
