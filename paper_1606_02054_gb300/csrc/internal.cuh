// internal.cuh -- shared definitions of the CUDA library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define CF_MAXP 32
#define CF_MAXQ 8
#define CF_MAXG 16
#define CF_MAXSHIFT 64
#define CF_MAXDIM 9     // lattice dimensions (largest T_k plus the sampled last coordinate)
#define CF_WARP 32

// Sizes of one problem.
struct Dims {
    int p, q, g;
    long long n;
};

// Offsets (in doubles) inside one component's factor block, written by the
// set-up kernel from Psi and read by the E-step.  Definitions under eq (4):
// Omega = Sigma + Delta Delta^T, c = Delta^T Omega^{-1} (y - mu),
// Lambda = I - Delta^T Omega^{-1} Delta, d = (y-mu)^T Omega^{-1} (y-mu).
struct Layout {
    int mu;     // p
    int Linv;   // p x p, lower-triangular inverse Cholesky factor of Omega
    int A;      // p x q, Linv * Delta: c = A^T z with z = Linv (y - mu)
    int scal;   // SC_COUNT scalars
    int Lam;    // q x q, Lambda
    int dq;     // q, 1 / sqrt(diag Lambda)
    int Lq;     // q x q, Cholesky factor of the correlation matrix of Lambda
    int l1;     // q blocks (one per coordinate r) of size l1s:
    int l1s;    //   mvec (q-1) = Lambda_{-r,r} / Lambda_rr, schur ((q-1)^2),
                //   dsc (q-1) = 1/sqrt(diag schur), L ((q-1)^2) chol of corr(schur)
    int l2;     // q*(q-1) blocks (pairs r, s) of size l2s, for the Schur
    int l2s;    //   complement of schur_r at s: mvec (q-2), dsc (q-2), L ((q-2)^2)
    int stride; // doubles per component
};

enum { SC_NU = 0, SC_LOGTP = 1, SC_PSI = 2, SC_COUNT = 4 };

__host__ __device__ inline Layout make_layout(int p, int q)
{
    Layout L;
    int o = 0;
    L.mu = o; o += p;
    L.Linv = o; o += p * p;
    L.A = o; o += p * q;
    L.scal = o; o += SC_COUNT;
    L.Lam = o; o += q * q;
    L.dq = o; o += q;
    L.Lq = o; o += q * q;
    int q1 = q - 1, q2 = q - 2 > 0 ? q - 2 : 0;
    L.l1s = q1 > 0 ? (2 * q1 + 2 * q1 * q1) : 0;
    L.l1 = o; o += q * L.l1s;
    L.l2s = q2 > 0 ? (2 * q2 + q2 * q2) : 0;
    L.l2 = o; o += q * (q - 1) * L.l2s;
    L.stride = (o + 1) & ~1;
    return L;
}

// Rank-1 lattice of the T_k integrator (k >= 3): z_d = a^d mod N.
struct Lattice {
    int N, M;
    int z[CF_MAXDIM];
};

// Error flags written by kernels (bitwise OR into one device int).
enum {
    KF_NOTPD_OMEGA = 1 << 0,
    KF_NOTPD_LAMBDA = 1 << 1,
    KF_NOTPD_SEE = 1 << 2,
    KF_NOTPD_SIGMA = 1 << 3,
    KF_EMPTY = 1 << 4,
    KF_NUROOT = 1 << 5,
    KF_NAN = 1 << 6,
    KF_TIMEOUT = 1 << 7,  // a bounded device wait gave up
};

// Number of statistics per component (see cfust_get_stats).
__host__ __device__ inline int stats_per_comp(int p, int q)
{
    return 3 + p + q + p * q + q * q + p * p;
}

// ---------------------------------------------------------------------------
// E-step pipeline.  Every T_k of a pair depends only on (c, d) of that pair,
// so a plan kernel writes one record per integral, integrator kernels
// evaluate all records of one dimension, and a combine kernel assembles the
// E-step quantities.  Records per pair and level:
//   level 0, dim q:    alpha_s (eq 4) and alpha (eq 13)   [1 when density-only]
//   level 1, dim q-1:  T_{q-1} of xi_r, r = 0..q-1
//   level 2, dim q-2:  T_{q-2} of the conditional mean, (r, s), s over the q-1 others
// ---------------------------------------------------------------------------
struct RecSet {
    int k;             // dimension of every integral in the set (0 = none)
    double* mom;       // moment records only: nrec x (k + k(k+1)/2) standardised
                       // E[X], E[X X^T] (lower triangle, row-major) given X <= limits
    long long nrec;    // number of records
    double* bt;        // nrec x k standardised upper limits
    int* fac;          // offset in F of the k x k correlation Cholesky factor
    int* tab;          // chi table index 3h + j (dof nu_h + p + j)
    double* dof;       // degrees of freedom
    double* res;       // T_k
    double* se;        // standard error over the lattice shifts (may be null)
    float4* t2f;       // FP32 modes, k = 2 only (else null): per record two float4,
                       // (h, k, rho, dof) and (1 - rho^2, h|rho| - sign(rho) k, 0, 0),
                       // the last two formed in FP64, so the T_2 kernel runs no FP64
    double* res0;      // moment records: alpha_s of the same pair from the shared pass (level 0
    double* se0;       //   results and standard error; may be null)
    const int* sel;    // lattice kernels (k >= 3): if set, only records sel[0 .. *nsel)
    const int* nsel;   //   (the learned surrogate's fallback list; device count)
    double* lw;        // moment records, exact E[log W] only (else null): the f-weighted mean of
                       // log(s^2) over the points of the pass (s the chi variate of alpha_s)
    float* res32 = nullptr;  // FP32 T_2 records of the mixed form at q = 2 (else null): the
                             // results in FP32, written instead of res
};

// Record index t of a set: every record, or (SEL: a kernel instantiated for
// selection lists) the t-th selected one.
template <bool SEL>
__device__ __forceinline__ long long rec_count(const RecSet& r) { return SEL ? (long long)*r.nsel : r.nrec; }
template <bool SEL>
__device__ __forceinline__ long long rec_index(const RecSet& r, long long t) { return SEL ? (long long)r.sel[t] : t; }

// FP32 inputs of one T_2 record (see RecSet::t2f); rho = 0 counts as negative.
__host__ __device__ inline void t2_record_f32(double h, double k, double rho, double dof, float4* out)
{
    out[0] = make_float4((float)h, (float)k, (float)rho, (float)dof);
    out[1] = make_float4((float)((1.0 - rho) * (1.0 + rho)),
                         (float)(h * (rho > 0.0 ? rho : -rho) - (rho > 0.0 ? k : -k)), 0.0f, 0.0f);
}

struct PlanArgs {
    Dims D;
    Layout Ly;
    const double* y;
    const double* F;
    const float* y32;      // mixed precision: FP32 observations and factor blocks
    const float* F32;      //   (whitening in FP32), else null
    int density_only;
    int single_pass;       // moments by ratio estimators (q >= 3): records LM instead of alpha/L1/L2
    double* pd;        // per pair: d, log t_p
    double* pc;        // per pair: c (q)
    float* pd32;       // mixed form: the same in FP32 (written instead of pd, pc)
    float* pc32;
    int fuse_l1;       // mixed form at q = 2: no level-1 records (combine evaluates the T_1s)
    int blocks = 0;    // mixed form: blocks of the plan (resident on the device; each takes
                       // tiles of 128 observations of one component), 0: one per tile
    RecSet L0, L1, L2, LM;
};

// Per-dof constants of the T_1 / T_2 integrators, 4 per table index
// (3h + j for the E-step, the case index for cfust_tk_eval):
//   [0] lgamma((v+1)/2) - lgamma(v/2) - lgamma(1/2)   (T_1 at dof v)
//   [1] the same at dof v + 1                          (inner T_1 of T_2)
//   [2] Gamma((v+1)/2) / (Gamma(v/2) sqrt(pi))         (T_2 at dof v)
//   [3] lgamma((v+1)/2) - lgamma(v/2) - log(v pi)/2    (log t_1 density at dof v)
//   [4] the same at dof v - 1
//   [5] lgamma(v/2)                                    (chi-square quantile at dof v)
enum { CST_LGB = 0, CST_LGB1 = 1, CST_C2 = 2, CST_LT1 = 3, CST_LT1M = 4, CST_LGA = 5, CST_STRIDE = 8 };

struct IntegArgs {
    const double* cst64;   // [tab][CST_STRIDE]
    const float* cst32;
    const double* F;
    Lattice lat;
    const double* chi64;   // [(3h + j)][M][N] (or per case for cfust_tk_eval)
    const float* chi32;
    const double* shf64;   // [M][CF_MAXDIM]
    const float* shf32;
    const double* glx64;   // Gauss-Legendre nodes/weights on [0, 1]
    const double* glw64;
    const float* glx32;
    const float* glw32;
    int t2n;
    // nodes of the graded T_2 pieces (|rho| > 0.99): T2_NH per piece
    const float* glx32h;
    const float* glw32h;
    // FP32: > 0 where pieces with 4 <= dof <= 64 and |rho| < 0.9 take 8-32 nodes by
    // t2_lo_class (T2_LO_* below), glx32l / glw32l the node sets of classes 0-4 packed
    int t2n_lo;
    const float* glx32l;
    const float* glw32l;
    // FP32 T_2: per tab, log2 T_1(-|z|; dof + 1) on the grid of T1TAB_N points
    // uniform in v = log2(1 + |z|) over [0, T1TAB_V], with d/dv (float2 each);
    // NULL: the continued fraction is used instead
    const float2* t1tab;
    // FP32 single-pass moments at q <= 4 (else null): per shift m and lattice point i, the
    // baker-transformed coordinates w_d = 1 - |2 frac(i z_d / N + shift_md) - 1|, d = 1..q,
    // in one float4 (computed in FP64 at creation; they are the same for every record)
    const float4* wtab;
    // T_2 records only (may be null): quadrature nodes evaluated, added once per warp
    // (the profiler's algorithmic work count)
    unsigned long long* nodes;
    // lanes per FP32 T_2 quadrature piece of finite dof: 2, 4, 8, 16 (a warp's pieces dealt
    // to its 32/L groups) or 32 (a warp per record; always for the CFUSN model's Phi_2 records)
    int t2_group;
    // lattice points in flight per lane in the FP32 moment pass with the coordinate table
    // (K <= 4): 1 or 2
    int mom_p;
    // exact E[log W] (else null): log(s^2) at every point of the chi tables, same layout
    const double* lchi64;
    const float* lchi32;
};

constexpr int T1TAB_N = 2048;
constexpr int T2_NH = 64;
// FP32 T_2 pieces where 4 <= dof <= 64 and |rho| < 0.9: Gauss-Legendre with 8, 12, 16, 20,
// 24 or t2n (32) nodes by the piece's length L in units of the integrand's two widths: the
// peak of sin^(dof-1) (~ 1/sqrt(dof - 1)) and the rise of the inner T_1 at the split point
// (~ 1/|zs|, zs the slope of its argument there).  Class c <= 4 serves a piece with
//   s^2 = L^2 (dof - 1 + 0.2 zs^2) <= T2_LO_S2_c  (and dof <= T2_LO_DMAX_c for c = 0, 1:
// a piece that ends at phi = 0 carries the factor phi^(dof-1), integrated exactly only by
// enough nodes), class 5 (the t2n set) the rest.  The bounds were fitted on the host
// (fit_t2_classes.py, which derives them and checks them on held-out records)
// against 1024-node graded quadrature over 2.2e5 pieces (dof log-uniform, tails of h and k
// down to T_1 = 1e-12, h up to 40) with the largest admissible error 5e-6 relative to T_2,
// and 0.85 of each fitted bound is kept; on held-out samples of two other distributions
// (4.4e5 pieces) the pieces of classes 0-4 stay within 1.9e-6, and whole records with
// |k| <= 8 within 2.5e-6 (one 24-node set for every piece reached 2.9e-4 there, at large h
// and dof).  The FP32 integrators' error floor is 5e-5.
constexpr int T2_LO_NCLS = 5;            // classes with a node set of their own (0-4)
constexpr int T2_LO_TOTAL = 80;            // 8 + 12 + 16 + 20 + 24 nodes, packed by class
__host__ __device__ constexpr int t2_lo_nodes(int c) { return 8 + 4 * c; }
__host__ __device__ constexpr int t2_lo_off(int c) { return 2 * c * c + 6 * c; }  // sum of the counts below c
// bounds on s^2 = L^2 (dof - 1 + T2_LO_ZW zs^2) of the classes 0-4, and the dof caps
constexpr float T2_LO_S2_0 = 1.54f * 1.54f, T2_LO_S2_1 = 4.12f * 4.12f, T2_LO_S2_2 = 7.58f * 7.58f,
                T2_LO_S2_3 = 11.32f * 11.32f, T2_LO_S2_4 = 15.5f * 15.5f;
constexpr float T2_LO_DMAX_0 = 20.0f, T2_LO_DMAX_1 = 40.0f;
constexpr float T2_LO_ZW = 0.2f;
constexpr float T2_LO_DOF_MIN = 4.0f, T2_LO_DOF_MAX = 64.0f, T2_LO_RHO = 0.9f;

// class of an FP32 T_2 piece of length L (either sign) in the region above: 0-4, or 5 for
// the t2n nodes
__device__ __forceinline__ int t2_lo_class(float L, float nu, float zs)
{
    const float s2 = L * L * fmaf(T2_LO_ZW * zs, zs, nu - 1.0f);
    return (s2 <= T2_LO_S2_0 && nu <= T2_LO_DMAX_0)   ? 0
           : (s2 <= T2_LO_S2_1 && nu <= T2_LO_DMAX_1) ? 1
           : s2 <= T2_LO_S2_2                         ? 2
           : s2 <= T2_LO_S2_3                         ? 3
           : s2 <= T2_LO_S2_4                         ? 4
                                                      : T2_LO_NCLS;
}

constexpr float T1TAB_V = 48.0f;

struct CombineArgs {
    Dims D;
    Layout Ly;
    const double* cst64;   // per-dof constants, [3h + j][CST_STRIDE]
    const float* cst32;    //   (FP32 copies, read by the mixed form's assembly)
    const double* F;
    const float* F32;      // mixed form: FP32 copies of the factor blocks (else null)
    const double* pd;
    const double* pc;
    const float* pd32;     // mixed form: d, log t_p and c in FP32 (read instead of pd, pc)
    const float* pc32;
    const float2* t1tab;   // mixed form at q = 2 with fuse_l1: the level-1 T_1 from the tables
    int fuse_l1;
    RecSet L0, L1, L2, LM;
    int density_only;
    int single_pass;
    int mixed;             // assemble the moments in FP32 (mixed precision)
    int fp32;              // records evaluated in FP32: pairs with alpha_s < 1e-35 go to the fix-up list
    double* logf;
    double* u;
    double* elogu;
    double* eu;
    double* euu;
    float* pr32;           // mixed form: FP32 pair rows (pr32_width(q) floats) instead of u..euu
    double* se;
    int* fix_count;
    int* fix_list;
    int* flags;
};

// Arguments of the fused FP64 pair routine (fix-up of FP32 pairs in the far
// tail of T_q, and the reference path of cfust_tk_eval).
struct EstepArgs {
    Dims D;
    Layout Ly;
    Lattice lat;
    const double* cst64;
    const double* y;        // n x p
    const double* F;        // g x stride factor blocks
    const double* chi64;    // [(3h + k)][M][N]
    const float* chi32;
    const double* shf64;    // [M][CF_MAXDIM]
    const float* shf32;
    const double* glx64;    // Gauss-Legendre nodes/weights on [0,1]
    const double* glw64;
    const float* glx32;
    const float* glw32;
    int t2n;
    int density_only;
    int single_pass;
    const double* lchi64;   // exact E[log W]: log(s^2) beside chi64 (else null)
    double* logf;           // g*n
    double* u;
    double* elogu;
    double* eu;             // g*n*q
    double* euu;            // g*n*q*q
    float* pr32;            // mixed form: FP32 pair rows in place of u..euu (else null)
    double* se;
    int* flags;
};

// message returned by cfust_last_error(NULL) (calls without a context)
// Device-side state of one EM fit run as a single CUDA graph (fit_graph.cu):
// the iteration counter and the stopping decision live on the device so the
// whole loop runs without host round trips.
struct FitState {
    int it;          // completed EM iterations (E-step + committed M-step)
    int done;        // the loop has stopped
    int converged;   // stopped by the Aitken rule
    int status;      // cfust_status of the fit
    int comp;        // component named by a failing M-step, else -1
    int nuroot;      // M-steps whose nu was clamped at a bound
    int final_pass;  // the loop ran max_iter iterations: evaluate l(Psi^(K))
    int pad;
};

#include <string>
void cf_set_global_error(const std::string& msg);

// initialisation (init.cu)
size_t cluster_moments_smem(int pass, int p, int g, int chunk);
cudaError_t launch_random_partition(long long n, int g, uint64_t seed, int start, int* labels,
                                    cudaStream_t st);
cudaError_t launch_kmeans_assign(const Dims& D, const double* y, const double* centres, int* labels,
                                 int* changes, int nsm, cudaStream_t st);
cudaError_t launch_cluster_moments(int pass, const Dims& D, const double* y, const int* labels,
                                   const double* mean, int chunk, int blocks, double* partial,
                                   cudaStream_t st);

// host launchers (each issues on `st`; *launches counts kernels issued)
cudaError_t launch_plan(const PlanArgs& a, cudaStream_t st, long long* launches);
cudaError_t launch_integrals(const RecSet& r, const IntegArgs& a, int fp32, int nsm,
                             cudaStream_t st, long long* launches);
cudaError_t launch_combine(const CombineArgs& a, cudaStream_t st, long long* launches);
cudaError_t launch_fixup(const EstepArgs& a, const int* count, const int* list, int nsm,
                         cudaStream_t st, long long* launches);
cudaError_t launch_tk_eval(int k, int count, const double* b, const double* V, const double* nu,
                           const IntegArgs& a, int fp32, double* out, double* se, cudaStream_t st,
                           long long* launches);
cudaError_t launch_lattice32(int k, const RecSet& r, const IntegArgs& a, int blocks, cudaStream_t st);
cudaError_t launch_lattice64(int k, const RecSet& r, const IntegArgs& a, int blocks, cudaStream_t st);
cudaError_t launch_t2(const RecSet& r, const IntegArgs& a, int fp32, int blocks, cudaStream_t st);
cudaError_t launch_factors_f32(const double* F, float* F32, long long count, cudaStream_t st,
                               long long* launches);
cudaError_t launch_moments(const RecSet& r, const IntegArgs& a, int fp32, int nsm, cudaStream_t st,
                           long long* launches);
cudaError_t launch_mom32(int k, const RecSet& r, const IntegArgs& a, int blocks, cudaStream_t st);
cudaError_t launch_mom64(int k, const RecSet& r, const IntegArgs& a, int blocks, cudaStream_t st);

// Arguments of the statistics reduction (reduce.cu).
struct ReduceArgs {
    Dims D;
    const double* y;
    const double* pi;
    const double* mu;
    const double* logf;
    const double* u;
    const double* elogu;
    const double* eu;
    const double* euu;
    const float* pr32;  // mixed form: FP32 pair rows (read in place of u..euu when set)
    double* tau;       // g*n
    double* partial;   // nblocks x (g*S + 1)
    int chunk;         // observations per block (<= blockDim.x)
    int row;           // values per staged observation row
    const float* y32;  // FP32 observations (FP32 statistics kernel only)
    int small_only;    // 1: N, U, Snu, Se, See only (Sr, Sre, Srr from the tensor-core kernel)
};

// floats per pair in the mixed form's FP32 pair rows: u, E log w, eu (q), euu (q x q)
__host__ __device__ inline int pr32_width(int q) { return 2 + q + q * q; }

size_t reduce_tc_smem(int p, int q, int g);
bool reduce_tc_fits(int p, int q, int g);
cudaError_t launch_reduce_tc(const ReduceArgs& a, int* flags, int nsm, cudaStream_t st);
cudaError_t launch_reduce_f32(const ReduceArgs& a, int nblocks, size_t smem, cudaStream_t st);
void reduce_set_smem_limits(int bytes);

// ---------------------------------------------------------------------------
// Learned surrogate (not part of the paper): a 3 x 256 tanh MLP mapping a
// record's features (standardised limits, correlations of Lambda, 1/dof) to
// log T_q and the standardised truncated moments of the single-pass form.
// Parameters: FP32 master vector W1 b1 W2 b2 W3 b3 W4 b4 (matrices row-major,
// input index first); BF16 copies for the GEMMs.
// ---------------------------------------------------------------------------
constexpr int MLP_IN = 48, MLP_H = 256, MLP_OUT = 48;
constexpr long long MLP_W1 = 0, MLP_B1 = MLP_W1 + MLP_IN * MLP_H, MLP_W2 = MLP_B1 + MLP_H,
                    MLP_B2 = MLP_W2 + MLP_H * MLP_H, MLP_W3 = MLP_B2 + MLP_H, MLP_B3 = MLP_W3 + MLP_H * MLP_H,
                    MLP_W4 = MLP_B3 + MLP_H, MLP_B4 = MLP_W4 + MLP_H * MLP_OUT, MLP_NPARAM = MLP_B4 + MLP_OUT;
// feature / target statistics: fmean, fstd, zlo, zhi (MLP_IN each), tmean, tstd (MLP_OUT each)
constexpr int MLP_NSTAT = 4 * MLP_IN + 2 * MLP_OUT;

struct SurOpts {
    int epochs, batch;
    long long samples_per_epoch;
    float lr, margin;
    unsigned long long seed;
};

struct Surrogate {
    int q = 0, nin = 0, nout = 0;
    bool trained = false, on = false;
    long long step = 0;          // Adam steps taken
    long long cap = 0;           // records per set the buffers hold
    float margin = 0.25f;
    float *theta = nullptr, *grad = nullptr, *am = nullptr, *av = nullptr, *stats = nullptr;
    void* wb = nullptr;          // BF16 row-major copy of theta
    void* wf = nullptr;          // BF16 weights in mma fragment order
    void* wtc = nullptr;         // BF16 W^T per layer in the tensor-core operand layout (inference)
    // training set
    long long ns = 0, ns_cap = 0;
    float *X = nullptr, *T = nullptr;
    unsigned char* type = nullptr;   // 0: log T only (dof nu + p); 1: log T and moments; 2: unused
    unsigned long long* count = nullptr;
    // minibatch buffers
    int bcap = 0;
    void *xb = nullptr, *h1 = nullptr, *h2 = nullptr, *h3 = nullptr, *dz = nullptr, *dz2 = nullptr, *one = nullptr;
    float *y = nullptr, *tb = nullptr, *mb = nullptr, *part = nullptr;
    double* lpart = nullptr;
    double* host_part = nullptr;
    // fallback lists of the E-step
    int *fall0 = nullptr, *fallM = nullptr, *nfall = nullptr;
    unsigned char* mark = nullptr;  // per pair: its moment record is in fallM
    long long last_records = 0;
    float hstats[MLP_NSTAT] = {};  // host copy of stats (standardisation fixed at the first training)
};

cudaError_t sur_reserve(Surrogate& s, int q, long long records, cudaStream_t st);
void sur_free(Surrogate& s);
cudaError_t sur_collect(Surrogate& s, const RecSet& L0, const RecSet& LM, const double* F, cudaStream_t st);
cudaError_t sur_train(Surrogate& s, const SurOpts& o, cudaStream_t st, double* losses);
// mark (optional): with moments = 1 records which pairs went to the fallback list;
// with moments = 0 a level-0 record whose pair is marked is not appended again
// err: device flags, KF_TIMEOUT set if a barrier wait of the kernel ran out
cudaError_t sur_infer(const Surrogate& s, const RecSet& r, const double* F, int moments, int* fall, int* nfall,
                      int* err, cudaStream_t st, unsigned char* mark = nullptr);
