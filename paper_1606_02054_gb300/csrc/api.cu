// api.cu -- the C ABI of include/cfust.h: context, device buffers, kernel
// launches and the EM loop (Sec. 3; Aitken rule of Sec. 3.4, eqs (24)-(26)).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "cfust.h"
#include "internal.cuh"

// kernels (defined in the other translation units)
__global__ void setup_components_kernel(Dims, Layout, const double*, const double*, const double*,
                                        const double*, double*, int*);
__global__ void chi_table_kernel(int, int, const double*, const double*, Lattice, const double*, double, double*,
                                 float*, double*, float*);
__global__ void dof_consts_kernel(Dims, Layout, const double*, int, double*, double*, float*);
__global__ void t1_table_kernel(int, const double*, const double*, float2*, int);
__global__ void widen_kernel(const float*, long long, Dims, double*);
__global__ void widen_pairs_kernel(const float*, long long, int, double*, double*, double*, double*);
__global__ void narrow_kernel(const double*, Dims, float*);


__global__ void estep_reduce_kernel(ReduceArgs);
__global__ void reduce_partials_kernel(const double*, int, int, double*, int*);
__global__ void segment_partials_kernel(const double*, int, int, int, double*, long long);
__global__ void loglik_partial_kernel(Dims, const double*, const double*, double*);
__global__ void mstep_kernel(Dims, const double*, double, double, const double*, const double*,
                             const double*, double*, double*, double*, double*, double*, int*, int*,
                             const int*, int);

struct cfust_ctx {
    int p = 0, q = 0, g = 0;
    long long n = 0;
    cfust_opts opts{};
    cudaStream_t st = nullptr;
    Dims D{};
    Layout Ly{};
    Lattice lat{};
    int t2n = 0;
    int nsm = 0;
    int chunk = 0, row = 0, nblocks_red = 0, nblocks_ll = 0;
    // device buffers
    double* y = nullptr;
    double *pi = nullptr, *mu = nullptr, *Sigma = nullptr, *Delta = nullptr, *nu = nullptr;
    double *pi_n = nullptr, *mu_n = nullptr, *Sigma_n = nullptr, *Delta_n = nullptr, *nu_n = nullptr;
    double* F = nullptr;
    double* dofs = nullptr;
    double* cst64 = nullptr;
    float* cst32 = nullptr;
    double* chi64 = nullptr;
    float* chi32 = nullptr;
    double* lchi64 = nullptr;  // exact E[log W]: log(s^2) beside the chi tables
    float* lchi32 = nullptr;
    double* shf64 = nullptr;
    float* shf32 = nullptr;
    float4* wtab = nullptr;  // FP32 single pass: lattice coordinates of every (shift, point)
    double *glx64 = nullptr, *glw64 = nullptr;
    float *glx32 = nullptr, *glw32 = nullptr;
    float *glx32h = nullptr, *glw32h = nullptr;  // T2_NH nodes for graded T_2 pieces
    float *glx32l = nullptr, *glw32l = nullptr;  // node sets of the FP32 T_2 piece classes (t2_lo_class)
    int t2n_lo = 0;
    double *logf = nullptr, *u = nullptr, *elogu = nullptr, *eu = nullptr, *euu = nullptr,
           *se = nullptr, *tau = nullptr;
    double *partial = nullptr, *stats = nullptr;
    int tune_t2_group = 0;  // launch shapes of the integrators chosen by cfust_autotune on this
    int tune_mom_p = 0;     // context (0: the process-wide choice for its shape, else the default)
    double* seg = nullptr;  // segment sums of the block partials (nseg x width)
    long long nseg = 0;
    long long n_stats = 0;  // observations behind the current statistics (all shards'), the n of eq (18)
    int *flags = nullptr, *comp_status = nullptr;
    float* stage32 = nullptr;
    float2* t1tab = nullptr;  // FP32 T_2: per-dof tables of T_1 at dof + 1
    // mixed precision: FP32 copies of the observations and factor blocks
    bool mixed = false;
    bool tc_stats = false;  // mixed form: cross statistics on the tensor cores (reduce_tc.cu)
    float* y32 = nullptr;
    float* F32 = nullptr;
    float* pr32 = nullptr;  // FP32 pair rows (u, E log w, eu, euu) written by the mixed E-step
    float *pd32 = nullptr, *pc32 = nullptr;  // mixed form: d, log t_p and c in FP32
    float* res32_l0 = nullptr;  // mixed form at q = 2: the level-0 T_2 results in FP32
    // E-step pipeline: per-pair (d, log t_p) and c, integral records per level
    double *pd = nullptr, *pc = nullptr;
    RecSet rec[4]{};  // levels 0, 1, 2 and the single-pass moment records
    Surrogate sur;    // learned surrogate of the level-0 and moment records
    bool single_pass = false;
    int *fix_count = nullptr, *fix_list = nullptr;
    // optional per-kernel-class timing (opts.profile)
    cudaEvent_t ev[CFUST_NPROF][2]{};
    bool pending[CFUST_NPROF]{};
    double prof_ms[CFUST_NPROF]{};
    long long prof_n[CFUST_NPROF]{};
    double prof_units[CFUST_NPROF]{};            // algorithmic work (cfust_profile_work)
    unsigned long long* work_dev = nullptr;      // device counts of T_2 quadrature nodes per class
    // pinned host scratch
    double* h_ll = nullptr;
    int* h_flags = nullptr;
    int* h_comp = nullptr;
    bool have_data = false, have_params = false, have_stats = false;
    long long launches = 0;
    std::string err;
    // whole-fit CUDA graph (cfust_fit_batch): captured on gst, cached per (max_iter, tol, flags)
    bool capturing = false;
    cudaStream_t gst = nullptr;
    // the T_1 tables are built on a side stream while the plan runs: forked after the dof
    // constants, joined before the first kernel that reads them (t1_pending in between)
    cudaStream_t st2 = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    bool t1_pending = false;
    cudaGraph_t fgraph = nullptr;
    cudaGraphExec_t fexec = nullptr;
    int fg_max_iter = -1, fg_flags = -1;
    double fg_tol = 0.0;
    long long fg_body_kernels = 0, fg_final_kernels = 0;
    FitState* fstate = nullptr;
    double* fhist = nullptr;
    int fhist_cap = 0;
    FitState* h_fstate = nullptr;
    double* h_fhist = nullptr;
};

namespace {
void tune_lookup(const cfust_ctx* c, int* t2_group, int* mom_p);  // shapes in force (below)
}

static thread_local std::string g_create_err;

void cf_set_global_error(const std::string& msg) { g_create_err = msg; }

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
static cfust_status fail(cfust_ctx* c, cfust_status s, const std::string& msg)
{
    if (c) c->err = msg;
    else g_create_err = msg;
    return s;
}

#define CU(call)                                                                            \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return fail(c, CFUST_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define LAUNCHED()                                                                          \
    do {                                                                                    \
        c->launches++;                                                                      \
        cudaError_t e_ = cudaGetLastError();                                                \
        if (e_ != cudaSuccess)                                                              \
            return fail(c, CFUST_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e_)); \
    } while (0)

template <typename T>
static cudaError_t dalloc(T** p, size_t count)
{
    *p = nullptr;
    if (count == 0) count = 1;
    return cudaMalloc((void**)p, sizeof(T) * count);
}

// SplitMix64 (Steele, Lea & Flood 2014): one output from state = key, as a
// double in [0, 1).
static double splitmix_u01(uint64_t key)
{
    uint64_t z = key + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z = z ^ (z >> 31);
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

// n-point Gauss-Legendre rule mapped to [0, 1] (Newton iteration on P_n).
static void gauss_legendre01(int n, std::vector<double>& x, std::vector<double>& w)
{
    x.resize(n);
    w.resize(n);
    for (int i = 0; i < n; ++i) {
        double t = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = t;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (t * p1 - p0) / (t * t - 1.0);
            const double step = p1 / dp;
            t -= step;
            if (std::fabs(step) < 1e-16) {
                // derivative at the converged node
                p0 = 1.0; p1 = t;
                for (int k = 2; k <= n; ++k) {
                    const double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
                    p0 = p1;
                    p1 = p2;
                }
                dp = n * (t * p1 - p0) / (t * t - 1.0);
                break;
            }
        }
        x[i] = 0.5 * (t + 1.0);
        w[i] = 1.0 / ((1.0 - t * t) * dp * dp);  // (2/((1-t^2) P'^2)) / 2
    }
}

static cfust_status check_flags(cfust_ctx* c, int f, const char* where)
{
    if (f & (KF_NOTPD_OMEGA | KF_NOTPD_LAMBDA))
        return fail(c, CFUST_ENOTPD, std::string(where) + ": Sigma, Omega or Lambda not positive definite");
    if (f & KF_NAN) return fail(c, CFUST_ENAN, std::string(where) + ": non-finite density or statistic");
    if (f & KF_TIMEOUT) return fail(c, CFUST_ETIMEOUT, std::string(where) + ": a bounded device wait gave up");
    return CFUST_OK;
}

// Observations per block of the statistics reduction: rows of 4 + p + q + q^2 values
// (FP32 in the mixed form) plus g posterior weights staged in at most ~64 KB of
// shared memory, chunk <= 256.  Depends on the sizes and the precision only, not on n.
// values per staged row of the statistics kernel (FP32 rows also hold tau u r: p more, and
// an odd length, so that the threads of a warp staging consecutive rows write to distinct
// shared-memory banks)
static int reduce_row(int p, int q, bool mixed) { return mixed ? (4 + 2 * p + q + q * q) | 1 : 4 + p + q + q * q; }

static int reduce_chunk(int p, int q, int g, bool mixed)
{
    const int row = reduce_row(p, q, mixed);
    const size_t rowbytes = mixed ? sizeof(float) : sizeof(double);
    int chunk = 256;
    while (chunk > 32 && (size_t)chunk * ((row + g) * rowbytes + sizeof(double)) + CF_MAXG * sizeof(double) > 64 * 1024)
        chunk -= 32;
    return chunk;
}

// Blocks per segment of the two-level statistics reduction (segment_partials_kernel).
constexpr int SEG_BLOCKS = 32;

// Aitken's acceleration (eqs 24-26) on l^(k-1), l^k, l^(k+1): converged when
// |l_inf^(k+1) - l^(k+1)| < tol; equal consecutive values count as converged.
static bool aitken_converged(double l_km1, double l_k, double l_kp1, double tol)
{
    const double den = l_k - l_km1;
    if (den == 0.0) return true;
    const double acc = (l_kp1 - l_k) / den;
    const double linf = l_k + (l_kp1 - l_k) / (1.0 - acc);
    return std::fabs(linf - l_kp1) < tol;
}

// kernel-class timing: events bracket each class on the context stream and
// are read after the next stream synchronisation
// A class entered again before its events were read (the two levels of the statistics
// reduction) keeps its first begin event, so its time spans both.
static void prof_begin(cfust_ctx* c, int k)
{
    if (c->opts.profile && !c->capturing && !c->pending[k]) cudaEventRecord(c->ev[k][0], c->st);
}
static void prof_end(cfust_ctx* c, int k, long long launches)
{
    if (c->capturing) return;  // graph nodes are counted when the graph runs
    c->prof_n[k] += launches;
    if (!c->opts.profile) return;
    cudaEventRecord(c->ev[k][1], c->st);
    c->pending[k] = true;
}
static void prof_collect(cfust_ctx* c)
{
    if (!c->opts.profile) return;
    if (c->work_dev) {  // device-counted work (T_2 nodes), after the stream synchronised
        unsigned long long w[CFUST_NPROF];
        if (cudaMemcpy(w, c->work_dev, sizeof(w), cudaMemcpyDeviceToHost) == cudaSuccess) {
            for (int k = 0; k < CFUST_NPROF; ++k) c->prof_units[k] += (double)w[k];
            cudaMemset(c->work_dev, 0, sizeof(w));
        }
    }
    for (int k = 0; k < CFUST_NPROF; ++k)
        if (c->pending[k]) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, c->ev[k][0], c->ev[k][1]) == cudaSuccess) c->prof_ms[k] += ms;
            c->pending[k] = false;
        }
}

// ---------------------------------------------------------------------------
// ABI
// ---------------------------------------------------------------------------
extern "C" void cfust_default_opts(cfust_opts* o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = CFUST_PREC_FP64;
    o->tensor_stats = 0;
    o->qmc_points = 1024;
    o->qmc_shifts = 8;
    o->qmc_korobov_a = 119;
    o->seed = 0;
    o->nu_min = 1.0;
    o->nu_max = 200.0;
    o->device = 0;
    o->cuda_stream = nullptr;
    o->t2_nodes = 0;
}

extern "C" const char* cfust_last_error(const cfust_ctx* c)
{
    return c ? c->err.c_str() : g_create_err.c_str();
}

extern "C" int64_t cfust_launch_count(const cfust_ctx* c) { return c ? c->launches : 0; }

extern "C" cfust_status cfust_debug_read(cfust_ctx* c, int what, void* dst, int64_t bytes,
                                         int64_t* written)
{
    if (!c) return fail(nullptr, CFUST_EINVAL, "cfust_debug_read: ctx is NULL");
    if (!dst || bytes < 0) return fail(c, CFUST_EINVAL, "cfust_debug_read: bad buffer");
    const size_t ng = (size_t)c->n * c->g;
    const void* src = nullptr;
    size_t avail = 0;
    switch (what) {
    case 0: src = c->F; avail = sizeof(double) * (size_t)c->g * c->Ly.stride; break;
    case 1: src = c->pd; avail = sizeof(double) * 2 * ng; break;
    case 2: src = c->pc; avail = sizeof(double) * ng * c->q; break;
    case 3: case 4: case 5: {
        const RecSet& r = c->rec[what - 3];
        src = r.bt; avail = sizeof(double) * (size_t)r.nrec * r.k; break;
    }
    case 6: case 7: case 8: {
        const RecSet& r = c->rec[what - 6];
        src = r.res; avail = sizeof(double) * (size_t)r.nrec; break;
    }
    case 9: src = c->flags; avail = sizeof(int); break;
    default: return fail(c, CFUST_EINVAL, "cfust_debug_read: unknown buffer");
    }
    const size_t nb = std::min(avail, (size_t)bytes);
    CU(cudaSetDevice(c->opts.device));
    if (nb) CU(cudaMemcpyAsync(dst, src, nb, cudaMemcpyDeviceToHost, c->st));
    CU(cudaStreamSynchronize(c->st));
    if (written) *written = (int64_t)nb;
    return CFUST_OK;
}

extern "C" cfust_status cfust_profile(cfust_ctx* c, double* ms, int64_t* launches, int reset)
{
    if (!c) return fail(nullptr, CFUST_EINVAL, "cfust_profile: ctx is NULL");
    if (!c->opts.profile) return fail(c, CFUST_ESTATE, "cfust_profile: context created without opts.profile");
    for (int k = 0; k < CFUST_NPROF; ++k) {
        if (ms) ms[k] = c->prof_ms[k];
        if (launches) launches[k] = c->prof_n[k];
        if (reset) { c->prof_ms[k] = 0.0; c->prof_n[k] = 0; c->prof_units[k] = 0.0; }
    }
    return CFUST_OK;
}

extern "C" cfust_status cfust_profile_work(cfust_ctx* c, double* units)
{
    if (!c) return fail(nullptr, CFUST_EINVAL, "cfust_profile_work: ctx is NULL");
    if (!units) return fail(c, CFUST_EINVAL, "cfust_profile_work: units is NULL");
    if (!c->opts.profile) return fail(c, CFUST_ESTATE, "cfust_profile_work: context created without opts.profile");
    for (int k = 0; k < CFUST_NPROF; ++k) units[k] = c->prof_units[k];
    return CFUST_OK;
}

static void free_all(cfust_ctx* c)
{
    sur_free(c->sur);
    void* bufs[] = {c->y, c->pi, c->mu, c->Sigma, c->Delta, c->nu, c->pi_n, c->mu_n, c->Sigma_n,
                    c->Delta_n, c->nu_n, c->F, c->dofs, c->cst64, c->cst32, c->chi64, c->chi32, c->shf64, c->shf32, c->wtab,
                    c->glx64, c->glw64, c->glx32, c->glw32, c->glx32h, c->glw32h, c->glx32l, c->glw32l,
                    c->logf, c->u, c->elogu, c->eu,
                    c->euu, c->se, c->tau, c->partial, c->stats, c->flags, c->comp_status,
                    c->stage32, c->pd, c->pc, c->fix_count, c->fix_list, c->y32, c->F32, c->pr32, c->pd32, c->pc32, c->res32_l0, c->t1tab,
                    c->work_dev, c->seg, c->lchi64, c->lchi32};
    for (void* b : bufs)
        if (b) cudaFree(b);
    for (RecSet& r : c->rec) {
        void* rb[] = {r.bt, r.fac, r.tab, r.dof, r.res, r.se, r.mom, r.t2f, r.lw};
        for (void* b : rb)
            if (b) cudaFree(b);
    }
    for (int k = 0; k < CFUST_NPROF; ++k)
        for (int i = 0; i < 2; ++i)
            if (c->ev[k][i]) cudaEventDestroy(c->ev[k][i]);
    if (c->h_ll) cudaFreeHost(c->h_ll);
    if (c->h_flags) cudaFreeHost(c->h_flags);
    if (c->h_comp) cudaFreeHost(c->h_comp);
    if (c->fexec) cudaGraphExecDestroy(c->fexec);
    if (c->fgraph) cudaGraphDestroy(c->fgraph);
    if (c->gst) cudaStreamDestroy(c->gst);
    if (c->st2) cudaStreamDestroy(c->st2);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->fstate) cudaFree(c->fstate);
    if (c->fhist) cudaFree(c->fhist);
    if (c->h_fstate) cudaFreeHost(c->h_fstate);
    if (c->h_fhist) cudaFreeHost(c->h_fhist);
}

extern "C" cfust_status cfust_destroy(cfust_ctx* c)
{
    if (!c) return CFUST_OK;
    cudaSetDevice(c->opts.device);
    if (c->st) cudaStreamSynchronize(c->st);
    if (c->gst) cudaStreamSynchronize(c->gst);
    if (c->st2) cudaStreamSynchronize(c->st2);
    free_all(c);
    delete c;
    return CFUST_OK;
}

extern "C" cfust_status cfust_create(cfust_ctx** out, int p, int q, int g, int64_t n,
                                     const cfust_opts* opts)
{
    cfust_ctx* c = nullptr;
    if (!out) return fail(nullptr, CFUST_EINVAL, "cfust_create: out is NULL");
    *out = nullptr;
    if (p < 1 || p > CF_MAXP || q < 1 || q > CF_MAXQ || g < 1 || g > CF_MAXG || n < 1 ||
        n >= (int64_t(1) << 31))
        return fail(nullptr, CFUST_EINVAL, "cfust_create: sizes out of range (1<=p<=32, 1<=q<=8, 1<=g<=16, 1<=n<2^31)");
    cfust_opts o;
    cfust_default_opts(&o);
    if (opts) o = *opts;
    if (o.precision != CFUST_PREC_FP64 && o.precision != CFUST_PREC_FP32 &&
        o.precision != CFUST_PREC_MIXED)
        return fail(nullptr, CFUST_EINVAL, "cfust_create: precision must be CFUST_PREC_FP64, _FP32 or _MIXED");
    if (o.qmc_points < 32 || o.qmc_points > (1 << 20) || o.qmc_shifts < 2 ||
        o.qmc_shifts > CF_MAXSHIFT || o.qmc_korobov_a < 1)
        return fail(nullptr, CFUST_EINVAL, "cfust_create: lattice needs 32 <= N <= 2^20, 2 <= M <= 64, a >= 1");
    if (!(o.nu_min > 0.0) || !(o.nu_max >= o.nu_min))
        return fail(nullptr, CFUST_EINVAL, "cfust_create: need 0 < nu_min <= nu_max");
    if (o.t2_nodes != 0 && (o.t2_nodes < 8 || o.t2_nodes > 64))
        return fail(nullptr, CFUST_EINVAL, "cfust_create: t2_nodes must be 0 or in [8, 64]");
    if (o.moments != 0 && o.moments != 1)
        return fail(nullptr, CFUST_EINVAL, "cfust_create: moments must be 0 or 1");
    if (o.hold & ~(CFUST_HOLD_DELTA | CFUST_HOLD_NU))
        return fail(nullptr, CFUST_EINVAL, "cfust_create: hold must combine CFUST_HOLD_DELTA and CFUST_HOLD_NU");
    if (o.model != CFUST_MODEL_CFUST && o.model != CFUST_MODEL_CFUSN)
        return fail(nullptr, CFUST_EINVAL, "cfust_create: model must be CFUST_MODEL_CFUST or CFUST_MODEL_CFUSN");
    if (o.tensor_stats != 0 && o.tensor_stats != 1)
        return fail(nullptr, CFUST_EINVAL, "cfust_create: tensor_stats must be 0 or 1");
    if (o.elogw != CFUST_ELOGW_OSL && o.elogw != CFUST_ELOGW_EXACT)
        return fail(nullptr, CFUST_EINVAL, "cfust_create: elogw must be CFUST_ELOGW_OSL or CFUST_ELOGW_EXACT");
    if (o.elogw == CFUST_ELOGW_EXACT && (o.moments != 1 || q < 3 || o.model != CFUST_MODEL_CFUST))
        return fail(nullptr, CFUST_EINVAL, "cfust_create: exact E[log W] needs moments = 1, q >= 3 and the CFUST model");
    if (o.model == CFUST_MODEL_CFUSN) o.hold |= CFUST_HOLD_NU;  // no nu step in the normal limit
    cudaError_t e = cudaSetDevice(o.device);
    if (e != cudaSuccess)
        return fail(nullptr, CFUST_ECUDA, std::string("cfust_create: cudaSetDevice: ") + cudaGetErrorString(e));

    c = new cfust_ctx();
    c->p = p; c->q = q; c->g = g; c->n = n;
    c->single_pass = o.moments == 1 && q >= 3;
    c->opts = o;
    c->st = (cudaStream_t)o.cuda_stream;
    c->D = Dims{p, q, g, (long long)n};
    c->Ly = make_layout(p, q);
    c->lat.N = o.qmc_points;
    c->lat.M = o.qmc_shifts;
    {
        long long z = 1;
        for (int d = 0; d < CF_MAXDIM; ++d) {
            c->lat.z[d] = (int)(z % o.qmc_points);
            z = (z * o.qmc_korobov_a) % o.qmc_points;
        }
    }
    c->mixed = o.precision == CFUST_PREC_MIXED;
    c->tc_stats = c->mixed && o.tensor_stats && reduce_tc_fits(p, q, g);
    // a warp evaluates 32 nodes at a time: fewer than 32 per piece saves nothing
    c->t2n = o.t2_nodes ? o.t2_nodes : (o.precision == CFUST_PREC_FP64 ? 64 : 32);
    // FP32 modes by default: 8-24 nodes by t2_lo_class where the integrand is smooth enough
    // (a node count set in the options holds for every piece)
    c->t2n_lo = (o.precision != CFUST_PREC_FP64 && o.t2_nodes == 0) ? 1 : 0;
    cudaDeviceProp prop;
    if ((e = cudaGetDeviceProperties(&prop, o.device)) != cudaSuccess) {
        cfust_status s = fail(nullptr, CFUST_ECUDA, std::string("cfust_create: ") + cudaGetErrorString(e));
        delete c;
        return s;
    }
    c->nsm = prop.multiProcessorCount;
    const size_t ng = (size_t)n * g;
    const int S = stats_per_comp(p, q);
    // reduction staging: rows of 4 + p + q + q^2 doubles, chunk <= 256 observations,
    // at most ~64 KB of shared memory
    c->row = reduce_row(p, q, c->mixed);
    const int chunk = reduce_chunk(p, q, g, c->mixed);
    c->chunk = chunk;
    c->nblocks_red = (int)((n + chunk - 1) / chunk);
    c->nseg = (c->nblocks_red + SEG_BLOCKS - 1) / SEG_BLOCKS;
    c->nblocks_ll = (int)((n + 255) / 256);
    const size_t NM = (size_t)o.qmc_points * o.qmc_shifts;
    const int ntab = q >= 3 ? 3 * g : 0;
    const size_t part = (size_t)std::max(c->nblocks_red * (g * S + 1), c->nblocks_ll);

#define ALLOC(ptr, cnt)                                                                      \
    if ((e = dalloc(&c->ptr, (cnt))) != cudaSuccess) {                                       \
        free_all(c);                                                                         \
        delete c;                                                                            \
        return fail(nullptr, CFUST_ENOMEM, std::string("cfust_create: cudaMalloc " #ptr ": ") + \
                                               cudaGetErrorString(e));                       \
    }
    ALLOC(y, (size_t)n * p);
    ALLOC(pi, g); ALLOC(mu, (size_t)g * p); ALLOC(Sigma, (size_t)g * p * p);
    ALLOC(Delta, (size_t)g * p * q); ALLOC(nu, g);
    ALLOC(pi_n, g); ALLOC(mu_n, (size_t)g * p); ALLOC(Sigma_n, (size_t)g * p * p);
    ALLOC(Delta_n, (size_t)g * p * q); ALLOC(nu_n, g);
    ALLOC(F, (size_t)g * c->Ly.stride);
    ALLOC(dofs, 3 * g);
    ALLOC(cst64, 3 * g * CST_STRIDE);
    ALLOC(cst32, 3 * g * CST_STRIDE);
    ALLOC(chi64, ntab * NM);
    ALLOC(chi32, ntab * NM);
    if (o.elogw == CFUST_ELOGW_EXACT) {
        ALLOC(lchi64, ntab * NM);
        ALLOC(lchi32, ntab * NM);
    }
    ALLOC(shf64, (size_t)o.qmc_shifts * CF_MAXDIM);
    ALLOC(shf32, (size_t)o.qmc_shifts * CF_MAXDIM);
    ALLOC(glx64, c->t2n); ALLOC(glw64, c->t2n); ALLOC(glx32, c->t2n); ALLOC(glw32, c->t2n);
    ALLOC(glx32h, T2_NH); ALLOC(glw32h, T2_NH);
    ALLOC(glx32l, T2_LO_TOTAL); ALLOC(glw32l, T2_LO_TOTAL);
    ALLOC(logf, ng); ALLOC(u, ng); ALLOC(elogu, ng); ALLOC(se, ng); ALLOC(tau, ng);
    ALLOC(eu, ng * q); ALLOC(euu, ng * q * q);
    ALLOC(partial, part);
    ALLOC(seg, (size_t)c->nseg * (g * S + 1));
    ALLOC(stats, (size_t)g * S + 1);
    ALLOC(flags, 1); ALLOC(comp_status, g);
    ALLOC(pd, 2 * ng); ALLOC(pc, ng * q);
    if (c->mixed) {
        ALLOC(y32, (size_t)n * p);
        ALLOC(F32, (size_t)g * c->Ly.stride);
        ALLOC(pr32, ng * pr32_width(q));
        ALLOC(pd32, 2 * ng); ALLOC(pc32, ng * q);
        if (q == 2) ALLOC(res32_l0, 2 * ng);
    }
    ALLOC(fix_count, 1); ALLOC(fix_list, ng);
    // T_2 records exist at q = 2 (level 0) and, in the recursion form, at q = 3, 4 (levels 1, 2)
    if (o.precision != CFUST_PREC_FP64 && (q == 2 || (!c->single_pass && (q == 3 || q == 4)))) {
        ALLOC(t1tab, (size_t)3 * g * T1TAB_N);
    }
    {
        const bool sp = c->single_pass;
        const int kdim[4] = {q, q - 1, q - 2, q};
        const long long mult[4] = {2, (!sp && q >= 2) ? q : 0,
                                   (!sp && q >= 3) ? (long long)q * (q - 1) : 0, sp ? 1 : 0};
        for (int l = 0; l < 4; ++l) {
            RecSet& r = c->rec[l];
            r.k = kdim[l] > 0 ? kdim[l] : 0;
            r.nrec = r.k > 0 ? (long long)ng * mult[l] : 0;
            const size_t nr = (size_t)r.nrec;
            ALLOC(rec[l].bt, nr * (r.k > 0 ? r.k : 1));
            ALLOC(rec[l].fac, nr); ALLOC(rec[l].tab, nr);
            ALLOC(rec[l].dof, nr); ALLOC(rec[l].res, nr);
            if (l == 0) { ALLOC(rec[l].se, nr); }
            if (r.k == 2 && o.precision != CFUST_PREC_FP64) { ALLOC(rec[l].t2f, 2 * nr); }
            if (l == 3) { ALLOC(rec[l].mom, nr * (q + q * (q + 1) / 2)); }
            if (l == 3 && o.elogw == CFUST_ELOGW_EXACT) { ALLOC(rec[l].lw, nr); }
        }
    }
#undef ALLOC
    if (cudaMallocHost((void**)&c->h_ll, sizeof(double) * 4) != cudaSuccess ||
        cudaMallocHost((void**)&c->h_flags, sizeof(int) * 4) != cudaSuccess ||
        cudaMallocHost((void**)&c->h_comp, sizeof(int) * CF_MAXG) != cudaSuccess) {
        free_all(c);
        delete c;
        return fail(nullptr, CFUST_ENOMEM, "cfust_create: cudaMallocHost failed");
    }
    // lattice shifts and Gauss-Legendre nodes
    std::vector<double> s64((size_t)o.qmc_shifts * CF_MAXDIM);
    std::vector<float> s32(s64.size());
    for (int m = 0; m < o.qmc_shifts; ++m)
        for (int d = 0; d < CF_MAXDIM; ++d) {
            const uint64_t key = o.seed ^ ((uint64_t)(m + 1) << 32) ^ (uint64_t)(d + 1);
            s64[m * CF_MAXDIM + d] = splitmix_u01(key);
            s32[m * CF_MAXDIM + d] = (float)s64[m * CF_MAXDIM + d];
            if (s32[m * CF_MAXDIM + d] >= 1.0f) s32[m * CF_MAXDIM + d] = 0.0f;
        }
    std::vector<double> gx, gw;
    gauss_legendre01(c->t2n, gx, gw);
    std::vector<float> gx32(gx.begin(), gx.end()), gw32(gw.begin(), gw.end());
    std::vector<double> gxh, gwh;
    gauss_legendre01(T2_NH, gxh, gwh);
    std::vector<float> gxh32(gxh.begin(), gxh.end()), gwh32(gwh.begin(), gwh.end());
    std::vector<float> gxl32, gwl32;  // the node sets of the classes of t2_lo_class, packed
    for (int cl = 0; cl < T2_LO_NCLS; ++cl) {
        std::vector<double> gxl, gwl;
        gauss_legendre01(t2_lo_nodes(cl), gxl, gwl);
        gxl32.insert(gxl32.end(), gxl.begin(), gxl.end());
        gwl32.insert(gwl32.end(), gwl.begin(), gwl.end());
    }
    cfust_status s = CFUST_OK;
    auto cp = [&](void* dst, const void* src, size_t bytes) {
        cudaError_t ee = cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
        if (ee != cudaSuccess && s == CFUST_OK)
            s = fail(nullptr, CFUST_ECUDA, std::string("cfust_create: cudaMemcpy: ") + cudaGetErrorString(ee));
    };
    cp(c->shf64, s64.data(), sizeof(double) * s64.size());
    cp(c->shf32, s32.data(), sizeof(float) * s32.size());
    if (c->single_pass && o.precision != CFUST_PREC_FP64 && q <= 4) {
        // baker-transformed lattice coordinates d = 1..q of every (shift, point), FP64 -> FP32
        // (read by the FP32 moment pass at q <= 4)
        const int N = o.qmc_points, M = o.qmc_shifts, WQ = (q + 3) / 4;
        std::vector<float> wt((size_t)M * N * 4 * WQ, 0.0f);
        for (int m = 0; m < M; ++m)
            for (int i = 0; i < N; ++i)
                for (int d = 1; d <= q; ++d) {
                    double x = (double)(((long long)i * c->lat.z[d]) % N) / (double)N + s64[m * CF_MAXDIM + d];
                    if (x >= 1.0) x -= 1.0;
                    wt[((size_t)m * N + i) * 4 * WQ + (d - 1)] = (float)(1.0 - std::fabs(2.0 * x - 1.0));
                }
        if (cudaMalloc((void**)&c->wtab, sizeof(float) * wt.size()) != cudaSuccess) {
            free_all(c);
            delete c;
            return fail(nullptr, CFUST_ENOMEM, "cfust_create: cudaMalloc failed (lattice coordinates)");
        }
        cp(c->wtab, wt.data(), sizeof(float) * wt.size());
    }
    cp(c->glx64, gx.data(), sizeof(double) * gx.size());
    cp(c->glw64, gw.data(), sizeof(double) * gw.size());
    cp(c->glx32, gx32.data(), sizeof(float) * gx32.size());
    cp(c->glw32, gw32.data(), sizeof(float) * gw32.size());
    cp(c->glx32h, gxh32.data(), sizeof(float) * gxh32.size());
    cp(c->glw32h, gwh32.data(), sizeof(float) * gwh32.size());
    cp(c->glx32l, gxl32.data(), sizeof(float) * gxl32.size());
    cp(c->glw32l, gwl32.data(), sizeof(float) * gwl32.size());
    if (s != CFUST_OK) {
        free_all(c);
        delete c;
        return s;
    }
    reduce_set_smem_limits(96 * 1024);
    if (o.profile &&
        (cudaMalloc((void**)&c->work_dev, sizeof(unsigned long long) * CFUST_NPROF) != cudaSuccess ||
         cudaMemset(c->work_dev, 0, sizeof(unsigned long long) * CFUST_NPROF) != cudaSuccess)) {
        free_all(c);
        delete c;
        return fail(nullptr, CFUST_ENOMEM, "cfust_create: profiler counters");
    }
    if (o.profile)
        for (int k = 0; k < CFUST_NPROF; ++k)
            for (int i = 0; i < 2; ++i)
                if (cudaEventCreate(&c->ev[k][i]) != cudaSuccess) {
                    free_all(c);
                    delete c;
                    return fail(nullptr, CFUST_ECUDA, "cfust_create: cudaEventCreate failed");
                }
    if (c->t1tab && (cudaStreamCreateWithFlags(&c->st2, cudaStreamNonBlocking) != cudaSuccess ||
                     cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
                     cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess)) {
        free_all(c);
        delete c;
        return fail(nullptr, CFUST_ECUDA, "cfust_create: side stream or events");
    }
    *out = c;
    return CFUST_OK;
}

extern "C" cfust_status cfust_set_data(cfust_ctx* c, const void* y, int dtype, int64_t ld, int on_device)
{
    if (!c) return fail(nullptr, CFUST_EINVAL, "cfust_set_data: ctx is NULL");
    if (!y || ld < c->p || (dtype != CFUST_F32 && dtype != CFUST_F64))
        return fail(c, CFUST_EINVAL, "cfust_set_data: need y != NULL, ld >= p, dtype F32 or F64");
    CU(cudaSetDevice(c->opts.device));
    const size_t rows = (size_t)c->n, pitch = (size_t)c->p;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    // contiguous rows: one linear copy (a pitched copy of n short rows is far slower)
    auto copy_rows = [&](void* dst, size_t elem) -> cudaError_t {
        if ((size_t)ld == pitch) return cudaMemcpyAsync(dst, y, rows * pitch * elem, kind, c->st);
        return cudaMemcpy2DAsync(dst, pitch * elem, y, (size_t)ld * elem, pitch * elem, rows, kind, c->st);
    };
    const long long total = (long long)rows * pitch;
    const int blocks = (int)std::min<long long>((total + 255) / 256, 4LL * c->nsm * 8);
    if (dtype == CFUST_F64) {
        CU(copy_rows(c->y, sizeof(double)));
        if (c->mixed) {  // the FP32 copy, narrowed from the FP64 rows
            narrow_kernel<<<blocks, 256, 0, c->st>>>(c->y, c->D, c->y32);
            LAUNCHED();
        }
    } else {
        // FP32 rows: into the mixed form's FP32 copy (exact) or a staging buffer, then widened
        float* dst = c->mixed ? c->y32 : nullptr;
        if (!dst) {
            if (!c->stage32) CU(dalloc(&c->stage32, rows * pitch));
            dst = c->stage32;
        }
        CU(copy_rows(dst, sizeof(float)));
        widen_kernel<<<blocks, 256, 0, c->st>>>(dst, c->p, c->D, c->y);
        LAUNCHED();
    }
    c->have_data = true;
    c->have_stats = false;
    return CFUST_OK;
}

extern "C" cfust_status cfust_set_params(cfust_ctx* c, const cfust_params* P)
{
    if (!c) return fail(nullptr, CFUST_EINVAL, "cfust_set_params: ctx is NULL");
    if (!P || !P->pi || !P->mu || !P->Sigma || !P->Delta || !P->nu)
        return fail(c, CFUST_EINVAL, "cfust_set_params: NULL parameter buffer");
    const int p = c->p, q = c->q, g = c->g;
    for (int h = 0; h < g; ++h) {
        if (!(P->pi[h] > 0.0 && P->pi[h] <= 1.0))
            return fail(c, CFUST_EINVAL, "cfust_set_params: pi[" + std::to_string(h) + "] not in (0, 1]");
        if (c->opts.model != CFUST_MODEL_CFUSN && !(P->nu[h] >= c->opts.nu_min && P->nu[h] <= c->opts.nu_max))
            return fail(c, CFUST_EINVAL, "cfust_set_params: nu[" + std::to_string(h) + "] outside [nu_min, nu_max]");
    }
    for (size_t i = 0; i < (size_t)g * p; ++i)
        if (!std::isfinite(P->mu[i])) return fail(c, CFUST_EINVAL, "cfust_set_params: non-finite mu");
    for (size_t i = 0; i < (size_t)g * p * p; ++i)
        if (!std::isfinite(P->Sigma[i])) return fail(c, CFUST_EINVAL, "cfust_set_params: non-finite Sigma");
    for (size_t i = 0; i < (size_t)g * p * q; ++i)
        if (!std::isfinite(P->Delta[i])) return fail(c, CFUST_EINVAL, "cfust_set_params: non-finite Delta");
    CU(cudaSetDevice(c->opts.device));
    CU(cudaMemcpyAsync(c->pi, P->pi, sizeof(double) * g, cudaMemcpyHostToDevice, c->st));
    CU(cudaMemcpyAsync(c->mu, P->mu, sizeof(double) * g * p, cudaMemcpyHostToDevice, c->st));
    CU(cudaMemcpyAsync(c->Sigma, P->Sigma, sizeof(double) * g * p * p, cudaMemcpyHostToDevice, c->st));
    CU(cudaMemcpyAsync(c->Delta, P->Delta, sizeof(double) * g * p * q, cudaMemcpyHostToDevice, c->st));
    if (c->opts.model == CFUST_MODEL_CFUSN) {
        // the normal limit: nu = +infinity selects it in every kernel
        const std::vector<double> inf(g, INFINITY);
        CU(cudaMemcpyAsync(c->nu, inf.data(), sizeof(double) * g, cudaMemcpyHostToDevice, c->st));
    } else {
        CU(cudaMemcpyAsync(c->nu, P->nu, sizeof(double) * g, cudaMemcpyHostToDevice, c->st));
    }
    CU(cudaStreamSynchronize(c->st));
    c->have_params = true;
    c->have_stats = false;
    return CFUST_OK;
}

extern "C" cfust_status cfust_get_params(cfust_ctx* c, cfust_params* P)
{
    if (!c) return fail(nullptr, CFUST_EINVAL, "cfust_get_params: ctx is NULL");
    if (!P || !P->pi || !P->mu || !P->Sigma || !P->Delta || !P->nu)
        return fail(c, CFUST_EINVAL, "cfust_get_params: NULL parameter buffer");
    if (!c->have_params) return fail(c, CFUST_ESTATE, "cfust_get_params: no parameters set");
    const int p = c->p, q = c->q, g = c->g;
    CU(cudaSetDevice(c->opts.device));
    CU(cudaMemcpyAsync(P->pi, c->pi, sizeof(double) * g, cudaMemcpyDeviceToHost, c->st));
    CU(cudaMemcpyAsync(P->mu, c->mu, sizeof(double) * g * p, cudaMemcpyDeviceToHost, c->st));
    CU(cudaMemcpyAsync(P->Sigma, c->Sigma, sizeof(double) * g * p * p, cudaMemcpyDeviceToHost, c->st));
    CU(cudaMemcpyAsync(P->Delta, c->Delta, sizeof(double) * g * p * q, cudaMemcpyDeviceToHost, c->st));
    CU(cudaMemcpyAsync(P->nu, c->nu, sizeof(double) * g, cudaMemcpyDeviceToHost, c->st));
    CU(cudaStreamSynchronize(c->st));
    return CFUST_OK;
}

// S0 + S1: per-component factors and (q >= 3) the chi tables.
static cfust_status launch_setup(cfust_ctx* c)
{
    prof_begin(c, CFUST_PROF_SETUP);
    setup_components_kernel<<<c->g, 32, 0, c->st>>>(c->D, c->Ly, c->mu, c->Sigma, c->Delta, c->nu,
                                                 c->F, c->flags);
    LAUNCHED();
    dof_consts_kernel<<<1, 64, 0, c->st>>>(c->D, c->Ly, c->F, 3 * c->g, c->dofs, c->cst64, c->cst32);
    LAUNCHED();
    if (c->t1tab) {
        // tables t = 3h + j hold T_1 at dof nu_h + p + j + 1: the FP32 T_2 records read those of
        // their own dof, the q = 2 level-1 T_1 records (dof nu + p + 1) the j = 0 table
        int jmask = 0;
        for (int l = 0; l < 3; ++l) {
            const RecSet& r = c->rec[l];
            if (r.nrec == 0) continue;
            if (r.k == 2) jmask |= l == 0 ? 5 : l == 1 ? 2 : 1;  // dofs nu+p (+2), nu+p+1, nu+p
            if (r.k == 1 && l == 1) jmask |= 1;
        }
        const int total = 3 * c->g * T1TAB_N;
        CU(cudaEventRecord(c->ev_fork, c->st));
        CU(cudaStreamWaitEvent(c->st2, c->ev_fork, 0));
        t1_table_kernel<<<(total + 255) / 256, 256, 0, c->st2>>>(3 * c->g, c->dofs, c->cst64, c->t1tab, jmask);
        LAUNCHED();
        CU(cudaEventRecord(c->ev_join, c->st2));
        c->t1_pending = true;
    }
    if (c->mixed) {
        cudaError_t e = launch_factors_f32(c->F, c->F32, (long long)c->g * c->Ly.stride, c->st, &c->launches);
        if (e != cudaSuccess) return fail(c, CFUST_ECUDA, std::string("factor copy: ") + cudaGetErrorString(e));
    }
    prof_end(c, CFUST_PROF_SETUP, 2 + (c->mixed ? 1 : 0) + (c->t1tab ? 1 : 0));
    if (c->q >= 3) {
        prof_begin(c, CFUST_PROF_CHI);
        // the single-pass E-step reads only the dof nu+p tables (index 3h)
        const int every = c->single_pass ? 3 : 1;
        const long long total = 3LL * c->g / every * c->lat.N * c->lat.M;
        const int blocks = (int)std::min<long long>((total + 127) / 128, 64LL * c->nsm);
        // the FP64 table serves the FP64 integrators; in the FP32 modes only the rare FP64
        // fix-up reads it, and 1e-9 is far inside what a pair sent there needs
        const double rtol = c->opts.precision == CFUST_PREC_FP64 ? 1e-15 : 1e-9;
        chi_table_kernel<<<blocks, 128, 0, c->st>>>(3 * c->g, every, c->dofs, c->cst64, c->lat, c->shf64, rtol,
                                                     c->chi64, c->chi32, c->lchi64, c->lchi32);
        LAUNCHED();
        prof_end(c, CFUST_PROF_CHI, 1);
    }
    return CFUST_OK;
}

static IntegArgs integ_args(const cfust_ctx* c)
{
    IntegArgs ia;
    ia.cst64 = c->cst64; ia.cst32 = c->cst32;
    ia.F = c->F; ia.lat = c->lat;
    ia.chi64 = c->chi64; ia.chi32 = c->chi32; ia.shf64 = c->shf64; ia.shf32 = c->shf32;
    ia.glx64 = c->glx64; ia.glw64 = c->glw64; ia.glx32 = c->glx32; ia.glw32 = c->glw32;
    ia.t2n = c->t2n;
    ia.glx32h = c->glx32h; ia.glw32h = c->glw32h;
    ia.t2n_lo = c->t2n_lo; ia.glx32l = c->glx32l; ia.glw32l = c->glw32l;
    ia.t1tab = c->t1tab;
    ia.wtab = c->wtab;
    ia.nodes = nullptr;
    int t2g = 0, mp = 0;
    tune_lookup(c, &t2g, &mp);
    ia.t2_group = c->opts.model == CFUST_MODEL_CFUSN ? CF_WARP : t2g;
    ia.mom_p = mp;
    ia.lchi64 = c->lchi64;
    ia.lchi32 = c->lchi32;
    return ia;
}

// S2-S7: plan, integrals of each level, combine, FP64 fix-up of far-tail pairs.
static cfust_status launch_pairs(cfust_ctx* c, int density_only)
{
    const int fp32 = c->opts.precision != CFUST_PREC_FP64;
    const int sp = c->single_pass ? 1 : 0;
    PlanArgs pa;
    pa.D = c->D; pa.Ly = c->Ly; pa.y = c->y; pa.F = c->F; pa.density_only = density_only;
    pa.y32 = c->mixed ? c->y32 : nullptr;
    pa.F32 = c->mixed ? c->F32 : nullptr;
    pa.single_pass = sp;
    pa.pd = c->pd; pa.pc = c->pc;
    pa.pd32 = c->mixed ? c->pd32 : nullptr; pa.pc32 = c->mixed ? c->pc32 : nullptr;
    // mixed form at q = 2: the level-1 T_1s are table lookups done by combine, not records
    const int fuse_l1 = c->mixed && c->q == 2 && !c->single_pass && c->t1tab != nullptr;
    pa.fuse_l1 = fuse_l1;
    pa.blocks = 16 * c->nsm;
    pa.L0 = c->rec[0]; pa.L1 = c->rec[1]; pa.L2 = c->rec[2]; pa.LM = c->rec[3];
    if (fuse_l1 && c->res32_l0) {
        // the level-0 T_2 results in FP32 for combine; no standard errors (quadrature: 0)
        pa.L0.res32 = c->res32_l0;
        pa.L0.se = nullptr;
    }
    if (density_only || sp) pa.L0.nrec = c->n * c->g;
    cudaError_t e;
    long long n0 = c->launches;
    prof_begin(c, CFUST_PROF_PLAN);
    if ((e = launch_plan(pa, c->st, &c->launches)) != cudaSuccess)
        return fail(c, CFUST_ECUDA, std::string("plan kernel: ") + cudaGetErrorString(e));
    if (c->t1_pending) {  // the T_1 tables of this E-step, built beside the plan
        CU(cudaStreamWaitEvent(c->st, c->ev_join, 0));
        c->t1_pending = false;
    }
    prof_end(c, CFUST_PROF_PLAN, c->launches - n0);
    const IntegArgs ia = integ_args(c);
    // learned surrogate: the network evaluates the level-0 and moment records, the
    // lattice only those outside its training range (selection lists)
    const bool sur = c->sur.on && sp;
    if (sur) {
        CU(cudaMemsetAsync(c->sur.nfall, 0, 2 * sizeof(int), c->st));
        c->sur.last_records = pa.L0.nrec + (density_only ? 0 : c->rec[3].nrec);
        n0 = c->launches;
        prof_begin(c, CFUST_PROF_SURROGATE);
        if (density_only) {
            if ((e = sur_infer(c->sur, pa.L0, c->F, 0, c->sur.fall0, c->sur.nfall, c->flags, c->st)) != cudaSuccess)
                return fail(c, CFUST_ECUDA, std::string("surrogate kernel: ") + cudaGetErrorString(e));
            ++c->launches;
        } else {
            // moment records first (marking the pairs they leave to the lattice); a level-0
            // record out of range sends its pair to the same list, since the shared lattice
            // pass gives alpha_s as well
            if ((e = sur_infer(c->sur, c->rec[3], c->F, 1, c->sur.fallM, c->sur.nfall + 1, c->flags, c->st,
                               c->sur.mark)) != cudaSuccess ||
                (e = sur_infer(c->sur, pa.L0, c->F, 0, c->sur.fallM, c->sur.nfall + 1, c->flags, c->st,
                               c->sur.mark)) != cudaSuccess)
                return fail(c, CFUST_ECUDA, std::string("surrogate kernel: ") + cudaGetErrorString(e));
            c->launches += 2;
        }
        prof_end(c, CFUST_PROF_SURROGATE, c->launches - n0);
    }
    for (int l = 0; l < (density_only || sp ? 1 : 3); ++l) {
        // single-pass E-step: alpha_s comes from the moment pass (the same lattice points),
        // also for the surrogate's out-of-range pairs; level 0 runs only in density passes
        if (l == 0 && sp && !density_only) continue;
        if (l == 1 && fuse_l1) continue;  // evaluated inside combine
        RecSet r = l == 0 ? pa.L0 : c->rec[l];
        n0 = c->launches;
        prof_begin(c, CFUST_PROF_LEVEL0 + l);
        if (sur && l == 0) {  // the records outside the network's training range
            r.sel = c->sur.fall0;
            r.nsel = c->sur.nfall;
        }
        IntegArgs il = ia;
        if (c->opts.profile && !c->capturing) {
            // algorithmic work: T_2 nodes counted on the device; lattice points (records x
            // N x M) and T_1 records here (selection lists: counted by the surrogate's info)
            if (r.k == 2) il.nodes = c->work_dev + CFUST_PROF_LEVEL0 + l;
            else if (r.k >= 3 && !(sur && l == 0)) c->prof_units[CFUST_PROF_LEVEL0 + l] += (double)r.nrec * c->lat.N * c->lat.M;
            else if (r.k == 1) c->prof_units[CFUST_PROF_LEVEL0 + l] += (double)r.nrec;
        }
        if ((e = launch_integrals(r, il, fp32, c->nsm, c->st, &c->launches)) != cudaSuccess)
            return fail(c, CFUST_ECUDA, std::string("integral kernel: ") + cudaGetErrorString(e));
        prof_end(c, CFUST_PROF_LEVEL0 + l, c->launches - n0);
    }
    if (sp && !density_only) {
        n0 = c->launches;
        prof_begin(c, CFUST_PROF_MOMENTS);
        RecSet rm = c->rec[3];
        rm.res0 = pa.L0.res;  // alpha_s and its standard error from the same pass
        rm.se0 = pa.L0.se;
        if (sur) {
            rm.sel = c->sur.fallM;
            rm.nsel = c->sur.nfall + 1;
        } else if (c->opts.profile && !c->capturing) {
            c->prof_units[CFUST_PROF_MOMENTS] += (double)rm.nrec * c->lat.N * c->lat.M;
        }
        if ((e = launch_moments(rm, ia, fp32, c->nsm, c->st, &c->launches)) != cudaSuccess)
            return fail(c, CFUST_ECUDA, std::string("moment kernel: ") + cudaGetErrorString(e));
        prof_end(c, CFUST_PROF_MOMENTS, c->launches - n0);
    }
    if (fp32) CU(cudaMemsetAsync(c->fix_count, 0, sizeof(int), c->st));
    CombineArgs ca;
    ca.D = c->D; ca.Ly = c->Ly; ca.cst64 = c->cst64; ca.cst32 = c->cst32; ca.F = c->F; ca.pd = c->pd; ca.pc = c->pc;
    ca.pd32 = c->mixed ? c->pd32 : nullptr; ca.pc32 = c->mixed ? c->pc32 : nullptr;
    ca.t1tab = c->t1tab; ca.fuse_l1 = fuse_l1;
    ca.F32 = c->mixed ? c->F32 : nullptr;
    ca.L0 = pa.L0; ca.L1 = c->rec[1]; ca.L2 = c->rec[2]; ca.LM = c->rec[3];
    ca.density_only = density_only; ca.single_pass = sp; ca.fp32 = fp32;
    ca.mixed = c->mixed ? 1 : 0;
    ca.logf = c->logf; ca.u = c->u; ca.elogu = c->elogu; ca.eu = c->eu; ca.euu = c->euu; ca.se = c->se;
    ca.pr32 = c->mixed ? c->pr32 : nullptr;
    ca.fix_count = c->fix_count; ca.fix_list = c->fix_list; ca.flags = c->flags;
    n0 = c->launches;
    prof_begin(c, CFUST_PROF_COMBINE);
    if ((e = launch_combine(ca, c->st, &c->launches)) != cudaSuccess)
        return fail(c, CFUST_ECUDA, std::string("combine kernel: ") + cudaGetErrorString(e));
    prof_end(c, CFUST_PROF_COMBINE, c->launches - n0);
    if (fp32) {
        EstepArgs a;
        a.D = c->D; a.Ly = c->Ly; a.lat = c->lat; a.cst64 = c->cst64;
        a.y = c->y; a.F = c->F;
        a.chi64 = c->chi64; a.chi32 = c->chi32;
        a.shf64 = c->shf64; a.shf32 = c->shf32;
        a.glx64 = c->glx64; a.glw64 = c->glw64; a.glx32 = c->glx32; a.glw32 = c->glw32;
        a.t2n = c->t2n;
        a.density_only = density_only;
        a.single_pass = sp;
        a.lchi64 = c->lchi64;
        a.logf = c->logf; a.u = c->u; a.elogu = c->elogu; a.eu = c->eu; a.euu = c->euu; a.se = c->se;
        a.pr32 = c->mixed ? c->pr32 : nullptr;
        a.flags = c->flags;
        n0 = c->launches;
        prof_begin(c, CFUST_PROF_FIXUP);
        if ((e = launch_fixup(a, c->fix_count, c->fix_list, c->nsm, c->st, &c->launches)) != cudaSuccess)
            return fail(c, CFUST_ECUDA, std::string("fix-up kernel: ") + cudaGetErrorString(e));
        prof_end(c, CFUST_PROF_FIXUP, c->launches - n0);
    }
    return CFUST_OK;
}

// S0-S9 for every pair and the segment sums of the block partials (the first level
// of S10) into seg (nseg_out segments, those past this context's own count zero),
// enqueued on c->st without any host synchronisation.
static cfust_status enqueue_estep_segments(cfust_ctx* c, double* seg, long long nseg_out)
{
    CU(cudaMemsetAsync(c->flags, 0, sizeof(int), c->st));
    cfust_status s;
    if ((s = launch_setup(c)) != CFUST_OK) return s;
    if ((s = launch_pairs(c, 0)) != CFUST_OK) return s;
    ReduceArgs r;
    r.D = c->D; r.y = c->y; r.pi = c->pi; r.mu = c->mu; r.logf = c->logf; r.u = c->u;
    r.elogu = c->elogu; r.eu = c->eu; r.euu = c->euu; r.tau = c->tau; r.partial = c->partial;
    r.pr32 = c->mixed ? c->pr32 : nullptr;
    r.chunk = c->chunk; r.row = c->row;
    r.y32 = c->y32;
    r.small_only = c->tc_stats ? 1 : 0;
    const size_t smem = (c->mixed ? sizeof(float) : sizeof(double)) * ((size_t)c->chunk * c->row + (size_t)c->g * c->chunk) +
                        sizeof(double) * ((size_t)c->chunk + CF_MAXG);
    prof_begin(c, CFUST_PROF_REDUCE);
    if (c->mixed) launch_reduce_f32(r, c->nblocks_red, smem, c->st);
    else estep_reduce_kernel<<<c->nblocks_red, 256, smem, c->st>>>(r);
    LAUNCHED();
    if (c->tc_stats) {  // Sr, Sre, Srr of the same blocks (reads the tau just written)
        cudaError_t e = launch_reduce_tc(r, c->flags, c->nsm, c->st);
        if (e != cudaSuccess) return fail(c, CFUST_ECUDA, std::string("tensor-core statistics: ") + cudaGetErrorString(e));
        c->launches++;
    }
    const int width = c->g * stats_per_comp(c->p, c->q) + 1;
    const long long tot = nseg_out * width;
    segment_partials_kernel<<<(int)std::min<long long>((tot + 255) / 256, 8LL * c->nsm), 256, 0, c->st>>>(
        c->partial, c->nblocks_red, SEG_BLOCKS, width, seg, nseg_out);
    LAUNCHED();
    prof_end(c, CFUST_PROF_REDUCE, c->tc_stats ? 3 : 2);
    return CFUST_OK;
}

// Second level of S10: stats = sum of nseg segment rows in order, and the flag of a
// non-finite sum.
static cfust_status enqueue_reduce_segments(cfust_ctx* c, const double* seg, long long nseg)
{
    const int width = c->g * stats_per_comp(c->p, c->q) + 1;
    prof_begin(c, CFUST_PROF_REDUCE);
    reduce_partials_kernel<<<(width + 127) / 128, 128, 0, c->st>>>(seg, (int)nseg, width, c->stats, c->flags);
    LAUNCHED();
    prof_end(c, CFUST_PROF_REDUCE, 1);
    return CFUST_OK;
}

// S0-S10 for every pair, enqueued on c->st without any host synchronisation
// (also captured into the whole-fit graph).  l(Psi) lands in stats[width - 1].
static cfust_status enqueue_estep(cfust_ctx* c)
{
    cfust_status s;
    c->n_stats = c->n;
    if ((s = enqueue_estep_segments(c, c->seg, c->nseg)) != CFUST_OK) return s;
    return enqueue_reduce_segments(c, c->seg, c->nseg);
}

extern "C" cfust_status cfust_estep(cfust_ctx* c, double* loglik_out)
{
    if (!c) return fail(nullptr, CFUST_EINVAL, "cfust_estep: ctx is NULL");
    if (!c->have_data || !c->have_params)
        return fail(c, CFUST_ESTATE, "cfust_estep: set_data and set_params must come first");
    CU(cudaSetDevice(c->opts.device));
    cfust_status s;
    if ((s = enqueue_estep(c)) != CFUST_OK) return s;
    const int width = c->g * stats_per_comp(c->p, c->q) + 1;
    CU(cudaMemcpyAsync(c->h_ll, c->stats + (width - 1), sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CU(cudaMemcpyAsync(c->h_flags, c->flags, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    CU(cudaStreamSynchronize(c->st));
    prof_collect(c);
    if ((s = check_flags(c, *c->h_flags, "cfust_estep")) != CFUST_OK) return s;
    if (!std::isfinite(*c->h_ll)) return fail(c, CFUST_ENAN, "cfust_estep: non-finite log-likelihood");
    if (loglik_out) *loglik_out = *c->h_ll;
    c->have_stats = true;
    return CFUST_OK;
}

extern "C" cfust_status cfust_get_pairs(cfust_ctx* c, double* logf, double* tau, double* u,
                                        double* elogu, double* eu, double* euu, double* se)
{
    if (!c) return fail(nullptr, CFUST_EINVAL, "cfust_get_pairs: ctx is NULL");
    if (!c->have_stats) return fail(c, CFUST_ESTATE, "cfust_get_pairs: no E-step results");
    const size_t ng = (size_t)c->n * c->g;
    CU(cudaSetDevice(c->opts.device));
    if (c->mixed && (u || elogu || eu || euu)) {  // the mixed E-step keeps these in its FP32 rows
        widen_pairs_kernel<<<(int)std::min<size_t>((ng + 255) / 256, 64 * (size_t)c->nsm), 256, 0, c->st>>>(
            c->pr32, (long long)ng, c->q, c->u, c->elogu, c->eu, c->euu);
        c->launches++;
        CU(cudaGetLastError());
    }
    if (logf) CU(cudaMemcpyAsync(logf, c->logf, sizeof(double) * ng, cudaMemcpyDeviceToHost, c->st));
    if (tau) CU(cudaMemcpyAsync(tau, c->tau, sizeof(double) * ng, cudaMemcpyDeviceToHost, c->st));
    if (u) CU(cudaMemcpyAsync(u, c->u, sizeof(double) * ng, cudaMemcpyDeviceToHost, c->st));
    if (elogu) CU(cudaMemcpyAsync(elogu, c->elogu, sizeof(double) * ng, cudaMemcpyDeviceToHost, c->st));
    if (eu) CU(cudaMemcpyAsync(eu, c->eu, sizeof(double) * ng * c->q, cudaMemcpyDeviceToHost, c->st));
    if (euu) CU(cudaMemcpyAsync(euu, c->euu, sizeof(double) * ng * c->q * c->q, cudaMemcpyDeviceToHost, c->st));
    if (se) CU(cudaMemcpyAsync(se, c->se, sizeof(double) * ng, cudaMemcpyDeviceToHost, c->st));
    CU(cudaStreamSynchronize(c->st));
    return CFUST_OK;
}

extern "C" cfust_status cfust_get_stats(cfust_ctx* c, double* stats)
{
    if (!c) return fail(nullptr, CFUST_EINVAL, "cfust_get_stats: ctx is NULL");
    if (!stats) return fail(c, CFUST_EINVAL, "cfust_get_stats: stats is NULL");
    if (!c->have_stats) return fail(c, CFUST_ESTATE, "cfust_get_stats: no E-step results");
    CU(cudaSetDevice(c->opts.device));
    CU(cudaMemcpyAsync(stats, c->stats, sizeof(double) * c->g * stats_per_comp(c->p, c->q),
                       cudaMemcpyDeviceToHost, c->st));
    CU(cudaStreamSynchronize(c->st));
    return CFUST_OK;
}

// S11 into the *_n buffers; gate (device flag, may be NULL) skips it.
static cfust_status enqueue_mstep(cfust_ctx* c, const int* gate)
{
    CU(cudaMemsetAsync(c->flags, 0, sizeof(int), c->st));
    prof_begin(c, CFUST_PROF_MSTEP);
    Dims Dm = c->D;
    Dm.n = c->n_stats;  // pi_h = N_h / n over every observation the statistics cover
    mstep_kernel<<<c->g, 32, 0, c->st>>>(Dm, c->stats, c->opts.nu_min, c->opts.nu_max, c->mu, c->Delta,
                                      c->nu, c->pi_n, c->mu_n, c->Sigma_n, c->Delta_n, c->nu_n,
                                      c->flags, c->comp_status, gate, c->opts.hold);
    LAUNCHED();
    prof_end(c, CFUST_PROF_MSTEP, 1);
    return CFUST_OK;
}

extern "C" cfust_status cfust_mstep(cfust_ctx* c)
{
    if (!c) return fail(nullptr, CFUST_EINVAL, "cfust_mstep: ctx is NULL");
    if (!c->have_stats) return fail(c, CFUST_ESTATE, "cfust_mstep: run cfust_estep first");
    CU(cudaSetDevice(c->opts.device));
    cfust_status s;
    if ((s = enqueue_mstep(c, nullptr)) != CFUST_OK) return s;
    CU(cudaMemcpyAsync(c->h_flags, c->flags, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    CU(cudaMemcpyAsync(c->h_comp, c->comp_status, sizeof(int) * c->g, cudaMemcpyDeviceToHost, c->st));
    CU(cudaStreamSynchronize(c->st));
    prof_collect(c);
    const int f = *c->h_flags;
    auto first = [&](int bit) {
        for (int h = 0; h < c->g; ++h)
            if (c->h_comp[h] & bit) return h;
        return -1;
    };
    if (f & KF_EMPTY)
        return fail(c, CFUST_EEMPTY, "cfust_mstep: component " + std::to_string(first(KF_EMPTY)) +
                                         " has no weight (sum tau = 0)");
    if (f & KF_NOTPD_SEE)
        return fail(c, CFUST_ENOTPD, "cfust_mstep: component " + std::to_string(first(KF_NOTPD_SEE)) +
                                         ": sum tau e3 not positive definite");
    if (f & KF_NOTPD_SIGMA)
        return fail(c, CFUST_ENOTPD, "cfust_mstep: component " + std::to_string(first(KF_NOTPD_SIGMA)) +
                                         ": updated Sigma not positive definite");
    const int p = c->p, q = c->q, g = c->g;
    CU(cudaMemcpyAsync(c->pi, c->pi_n, sizeof(double) * g, cudaMemcpyDeviceToDevice, c->st));
    CU(cudaMemcpyAsync(c->mu, c->mu_n, sizeof(double) * g * p, cudaMemcpyDeviceToDevice, c->st));
    CU(cudaMemcpyAsync(c->Sigma, c->Sigma_n, sizeof(double) * g * p * p, cudaMemcpyDeviceToDevice, c->st));
    CU(cudaMemcpyAsync(c->Delta, c->Delta_n, sizeof(double) * g * p * q, cudaMemcpyDeviceToDevice, c->st));
    CU(cudaMemcpyAsync(c->nu, c->nu_n, sizeof(double) * g, cudaMemcpyDeviceToDevice, c->st));
    c->have_stats = false;
    if (f & KF_NUROOT)
        return fail(c, CFUST_ENUROOT, "cfust_mstep: component " + std::to_string(first(KF_NUROOT)) +
                                          ": eq (22) has no root in [nu_min, nu_max]; nu clamped");
    return CFUST_OK;
}

// density-only pass (eq 27); l(Psi) lands in stats[0]
static cfust_status enqueue_loglik(cfust_ctx* c)
{
    CU(cudaMemsetAsync(c->flags, 0, sizeof(int), c->st));
    cfust_status s;
    if ((s = launch_setup(c)) != CFUST_OK) return s;
    if ((s = launch_pairs(c, 1)) != CFUST_OK) return s;
    prof_begin(c, CFUST_PROF_REDUCE);
    loglik_partial_kernel<<<c->nblocks_ll, 256, 0, c->st>>>(c->D, c->pi, c->logf, c->partial);
    LAUNCHED();
    reduce_partials_kernel<<<1, 32, 0, c->st>>>(c->partial, c->nblocks_ll, 1, c->stats, c->flags);
    LAUNCHED();
    prof_end(c, CFUST_PROF_REDUCE, 2);
    return CFUST_OK;
}

extern "C" cfust_status cfust_loglik(cfust_ctx* c, double* out)
{
    if (!c) return fail(nullptr, CFUST_EINVAL, "cfust_loglik: ctx is NULL");
    if (!out) return fail(c, CFUST_EINVAL, "cfust_loglik: out is NULL");
    if (!c->have_data || !c->have_params)
        return fail(c, CFUST_ESTATE, "cfust_loglik: set_data and set_params must come first");
    CU(cudaSetDevice(c->opts.device));
    cfust_status s;
    if ((s = enqueue_loglik(c)) != CFUST_OK) return s;
    CU(cudaMemcpyAsync(c->h_ll, c->stats, sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CU(cudaMemcpyAsync(c->h_flags, c->flags, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    CU(cudaStreamSynchronize(c->st));
    prof_collect(c);
    c->have_stats = false;
    if ((s = check_flags(c, *c->h_flags, "cfust_loglik")) != CFUST_OK) return s;
    *out = *c->h_ll;
    return std::isfinite(*out) ? CFUST_OK : fail(c, CFUST_ENAN, "cfust_loglik: non-finite log-likelihood");
}

extern "C" cfust_status cfust_fit(cfust_ctx* c, int max_iter, double tol, int* iters_out,
                                  double* loglik_hist)
{
    if (!c) return fail(nullptr, CFUST_EINVAL, "cfust_fit: ctx is NULL");
    if (max_iter < 0) return fail(c, CFUST_EINVAL, "cfust_fit: max_iter < 0");
    std::vector<double> hist((size_t)max_iter + 1, NAN);
    int it = 0;
    cfust_status s = CFUST_OK;
    bool converged = false;
    for (it = 0; it < max_iter; ++it) {
        double L;
        if ((s = cfust_estep(c, &L)) != CFUST_OK) break;
        hist[it] = L;
        if (tol > 0.0 && it >= 2 && aitken_converged(hist[it - 2], hist[it - 1], L, tol)) {
            converged = true;  // Aitken (eqs 24-26)
            break;
        }
        s = cfust_mstep(c);
        if (s == CFUST_ENUROOT) s = CFUST_OK;  // nu clamped: keep iterating
        if (s != CFUST_OK) break;
    }
    if (s == CFUST_OK && !converged) {
        double L = NAN;
        s = cfust_loglik(c, &L);
        if (s == CFUST_OK) hist[max_iter] = L;
        it = max_iter;
    }
    if (iters_out) *iters_out = it;
    if (loglik_hist) std::memcpy(loglik_hist, hist.data(), sizeof(double) * ((size_t)it + 1));
    return s;
}

// ---------------------------------------------------------------------------
// Autotuner of the integrators' launch shapes.  Choices are kept per (kernel, record
// dimension, precision) for the process, and every context of that shape without a tuning
// of its own uses them from its next E-step on (a CUDA graph keeps the shape in force when
// it was built).  The lanes per T_2 piece set the order in which a record's nodes are
// added, so one choice per shape -- not per problem size -- keeps the shards of one
// problem (which differ in size) bitwise equal to the whole problem.
// ---------------------------------------------------------------------------
namespace {
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, int> g_tune;  // (kind, k, precision) -> choice
enum { TUNE_T2 = 0, TUNE_MOM = 1 };
// the level of the context's T_2 records (FP32, finite dof), or -1
int t2_level(const cfust_ctx* c)
{
    if (c->opts.precision == CFUST_PREC_FP64 || c->opts.model == CFUST_MODEL_CFUSN) return -1;
    for (int l = 0; l < 3; ++l)
        if (c->rec[l].k == 2 && c->rec[l].nrec > 0) return l;
    return -1;
}
bool mom_tunable(const cfust_ctx* c)
{
    return c->single_pass && c->opts.precision != CFUST_PREC_FP64 && c->q <= 4 && c->rec[3].nrec > 0;
}
// The shapes in force: this context's tuning, else the process-wide choice for its
// shape, else the defaults (2 lanes per T_2 piece, 2 points per lane)
void tune_lookup(const cfust_ctx* c, int* t2_group, int* mom_p)
{
    *t2_group = c->tune_t2_group ? c->tune_t2_group : 2;
    *mom_p = c->tune_mom_p ? c->tune_mom_p : 2;
    if (c->tune_t2_group && c->tune_mom_p) return;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    const int l = t2_level(c);
    if (!c->tune_t2_group && l >= 0) {
        auto it = g_tune.find({TUNE_T2, 2, c->opts.precision});
        if (it != g_tune.end()) *t2_group = it->second;
    }
    if (!c->tune_mom_p && mom_tunable(c)) {
        auto it = g_tune.find({TUNE_MOM, c->q, c->opts.precision});
        if (it != g_tune.end()) *mom_p = it->second;
    }
}
}  // namespace

extern "C" cfust_status cfust_autotune(cfust_ctx* c, int reps, int* choices, double* ms)
{
    if (!c) return fail(nullptr, CFUST_EINVAL, "cfust_autotune: ctx is NULL");
    if (reps < 1 || reps > 100) return fail(c, CFUST_EINVAL, "cfust_autotune: reps must lie in [1, 100]");
    if (!c->have_data || !c->have_params)
        return fail(c, CFUST_ESTATE, "cfust_autotune: set_data and set_params must come first");
    CU(cudaSetDevice(c->opts.device));
    static const int t2c[5] = {2, 4, 8, 16, 32};
    static const int mpc[2] = {1, 2};
    double t[7];
    for (int i = 0; i < 7; ++i) t[i] = -1.0;
    // one E-step leaves the records of the current Psi on the device
    cfust_status s;
    if ((s = enqueue_estep(c)) != CFUST_OK) return s;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CU(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(c, CFUST_ECUDA, "cfust_autotune: cudaEventCreate failed");
    }
    auto timeit = [&](auto launch, double* best) -> cudaError_t {
        cudaError_t e = launch();  // warm-up
        *best = 1e30;
        for (int r = 0; r < reps && e == cudaSuccess; ++r) {
            if ((e = cudaEventRecord(e0, c->st)) != cudaSuccess) break;
            if ((e = launch()) != cudaSuccess) break;
            if ((e = cudaEventRecord(e1, c->st)) != cudaSuccess) break;
            if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
            float f = 0.f;
            if ((e = cudaEventElapsedTime(&f, e0, e1)) != cudaSuccess) break;
            *best = std::min(*best, (double)f);
        }
        return e;
    };
    cudaError_t e = cudaSuccess;
    IntegArgs ia = integ_args(c);
    long long dummy = 0;
    const int l = t2_level(c);
    if (l >= 0) {
        int bi = 0;
        for (int i = 0; i < 5 && e == cudaSuccess; ++i) {
            ia.t2_group = t2c[i];
            e = timeit([&] { return launch_integrals(c->rec[l], ia, 1, c->nsm, c->st, &dummy); }, &t[i]);
            if (t[i] < t[bi]) bi = i;
        }
        if (e == cudaSuccess) c->tune_t2_group = t2c[bi];
    }
    if (e == cudaSuccess && mom_tunable(c)) {
        RecSet rm = c->rec[3];
        rm.res0 = c->rec[0].res;
        rm.se0 = c->rec[0].se;
        int bi = 0;
        for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
            ia = integ_args(c);
            ia.mom_p = mpc[i];
            e = timeit([&] { return launch_moments(rm, ia, 1, c->nsm, c->st, &dummy); }, &t[5 + i]);
            if (t[5 + i] < t[5 + bi]) bi = i;
        }
        if (e == cudaSuccess) c->tune_mom_p = mpc[bi];
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return fail(c, CFUST_ECUDA, std::string("cfust_autotune: ") + cudaGetErrorString(e));
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        if (l >= 0) g_tune[{TUNE_T2, 2, c->opts.precision}] = c->tune_t2_group;
        if (mom_tunable(c)) g_tune[{TUNE_MOM, c->q, c->opts.precision}] = c->tune_mom_p;
    }
    c->launches += dummy;
    c->have_stats = false;  // the timing runs overwrote the integral records
    if (choices) {
        choices[0] = l >= 0 ? c->tune_t2_group : 0;
        choices[1] = mom_tunable(c) ? c->tune_mom_p : 0;
    }
    if (ms)
        for (int i = 0; i < 7; ++i) ms[i] = t[i];
    return CFUST_OK;
}

// ---------------------------------------------------------------------------
// Row-sharded E-step (Sec. 4's collection step over processes instead of threads):
// each process holds a contiguous range of observations that starts on a segment
// boundary, computes the segment sums of its statistics, the caller gathers the
// segments of every process in rank order, and each process reduces them in that
// order and runs the same M-step.
// ---------------------------------------------------------------------------
extern "C" cfust_status cfust_rows_per_segment(int p, int q, int g, int precision, int64_t* rows)
{
    if (!rows || p < 1 || p > CF_MAXP || q < 1 || q > CF_MAXQ || g < 1 || g > CF_MAXG ||
        precision < CFUST_PREC_FP64 || precision > CFUST_PREC_MIXED)
        return fail(nullptr, CFUST_EINVAL, "cfust_rows_per_segment: sizes or precision out of range");
    *rows = (int64_t)reduce_chunk(p, q, g, precision == CFUST_PREC_MIXED) * SEG_BLOCKS;
    return CFUST_OK;
}

extern "C" cfust_status cfust_segment_count(cfust_ctx* c, int64_t* nseg, int* width)
{
    if (!c) return fail(nullptr, CFUST_EINVAL, "cfust_segment_count: ctx is NULL");
    if (nseg) *nseg = c->nseg;
    if (width) *width = c->g * stats_per_comp(c->p, c->q) + 1;
    return CFUST_OK;
}

extern "C" cfust_status cfust_estep_segments(cfust_ctx* c, double* seg, int64_t nseg_out)
{
    if (!c) return fail(nullptr, CFUST_EINVAL, "cfust_estep_segments: ctx is NULL");
    if (!seg || nseg_out < c->nseg)
        return fail(c, CFUST_EINVAL, "cfust_estep_segments: need a device buffer of at least " +
                                         std::to_string(c->nseg) + " segments");
    if (!c->have_data || !c->have_params)
        return fail(c, CFUST_ESTATE, "cfust_estep_segments: set_data and set_params must come first");
    CU(cudaSetDevice(c->opts.device));
    c->have_stats = false;
    return enqueue_estep_segments(c, seg, nseg_out);
}

extern "C" cfust_status cfust_reduce_segments(cfust_ctx* c, const double* seg, int64_t nseg, int64_t n_total,
                                              double* loglik_out)
{
    if (!c) return fail(nullptr, CFUST_EINVAL, "cfust_reduce_segments: ctx is NULL");
    if (!seg || nseg < 1 || nseg > INT32_MAX) return fail(c, CFUST_EINVAL, "cfust_reduce_segments: bad segments");
    if (n_total < c->n) return fail(c, CFUST_EINVAL, "cfust_reduce_segments: n_total below this shard's rows");
    c->n_stats = n_total;
    CU(cudaSetDevice(c->opts.device));
    cfust_status s;
    if ((s = enqueue_reduce_segments(c, seg, nseg)) != CFUST_OK) return s;
    const int width = c->g * stats_per_comp(c->p, c->q) + 1;
    CU(cudaMemcpyAsync(c->h_ll, c->stats + (width - 1), sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CU(cudaMemcpyAsync(c->h_flags, c->flags, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    CU(cudaStreamSynchronize(c->st));
    prof_collect(c);
    if ((s = check_flags(c, *c->h_flags, "cfust_reduce_segments")) != CFUST_OK) return s;
    if (!std::isfinite(*c->h_ll)) return fail(c, CFUST_ENAN, "cfust_reduce_segments: non-finite log-likelihood");
    if (loglik_out) *loglik_out = *c->h_ll;
    c->have_stats = true;
    return CFUST_OK;
}

extern "C" int cfust_aitken_converged(double l_km1, double l_k, double l_kp1, double tol)
{
    return aitken_converged(l_km1, l_k, l_kp1, tol) ? 1 : 0;
}

// ---------------------------------------------------------------------------
// Whole-fit CUDA graph: the loop of cfust_fit with its control on the device
// (fit_graph.cu), so a batch of fits runs concurrently without host round trips.
// ---------------------------------------------------------------------------
__global__ void fit_init_kernel(FitState*, int);
__global__ void fit_gate_kernel(FitState*, const double*, const int*, double*, double);
__global__ void fit_commit_kernel(Dims, FitState*, const int*, const int*, const double*, const double*,
                                  const double*, const double*, const double*, double*, double*, double*,
                                  double*, double*, int, cudaGraphConditionalHandle);
__global__ void fit_final_gate_kernel(const FitState*, cudaGraphConditionalHandle);
__global__ void fit_final_kernel(FitState*, const double*, const int*, double*, int);

static void drop_fit_graph(cfust_ctx* c)
{
    if (c->fexec) cudaGraphExecDestroy(c->fexec);
    if (c->fgraph) cudaGraphDestroy(c->fgraph);
    c->fexec = nullptr;
    c->fgraph = nullptr;
    c->fg_max_iter = -1;
}

// Adds a conditional node (WHILE or IF) after dep and captures its body with fill().
template <typename Fill>
static cfust_status add_conditional(cfust_ctx* c, cudaGraph_t g, cudaGraphNode_t* dep,
                                    cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
                                    cudaGraphNode_t* node, long long* kernels, Fill fill)
{
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = type;
    cp.conditional.size = 1;
    CU(cudaGraphAddNode(node, g, dep, nullptr, dep ? 1 : 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    CU(cudaStreamBeginCaptureToGraph(c->gst, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    const cudaStream_t saved = c->st;
    c->st = c->gst;
    c->capturing = true;
    const long long n0 = c->launches;
    cfust_status s = fill();
    *kernels = c->launches - n0;
    c->launches = n0;
    c->capturing = false;
    c->st = saved;
    cudaGraph_t out = nullptr;
    const cudaError_t e = cudaStreamEndCapture(c->gst, &out);
    if (s != CFUST_OK) return s;
    if (e != cudaSuccess)
        return fail(c, CFUST_ECUDA, std::string("fit graph capture: ") + cudaGetErrorString(e));
    return CFUST_OK;
}

static cfust_status add_kernel_node(cfust_ctx* c, cudaGraph_t g, cudaGraphNode_t* dep, cudaGraphNode_t* node,
                                    void* func, void** args, int threads)
{
    cudaKernelNodeParams kp{};
    kp.func = func;
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(threads);
    kp.sharedMemBytes = 0;
    kp.kernelParams = args;
    kp.extra = nullptr;
    CU(cudaGraphAddKernelNode(node, g, dep, dep ? 1 : 0, &kp));
    return CFUST_OK;
}

static cfust_status build_fit_graph(cfust_ctx* c, int max_iter, double tol, int flags)
{
    if (c->fexec && c->fg_max_iter == max_iter && c->fg_tol == tol && c->fg_flags == flags)
        return CFUST_OK;
    drop_fit_graph(c);
    if (!c->gst) CU(cudaStreamCreateWithFlags(&c->gst, cudaStreamNonBlocking));
    if (!c->fstate) CU(cudaMalloc((void**)&c->fstate, sizeof(FitState)));
    if (!c->h_fstate) CU(cudaMallocHost((void**)&c->h_fstate, sizeof(FitState)));
    if (c->fhist_cap < max_iter + 1) {
        if (c->fhist) cudaFree(c->fhist);
        if (c->h_fhist) cudaFreeHost(c->h_fhist);
        c->fhist = nullptr;
        c->h_fhist = nullptr;
        c->fhist_cap = 0;
        CU(cudaMalloc((void**)&c->fhist, sizeof(double) * (max_iter + 1)));
        CU(cudaMallocHost((void**)&c->h_fhist, sizeof(double) * (max_iter + 1)));
        c->fhist_cap = max_iter + 1;
    }
    cudaGraph_t g = nullptr;
    CU(cudaGraphCreate(&g, 0));
    c->fgraph = g;
    cudaGraphNode_t n_hist, n_init, n_loop, n_fgate, n_final;
    // hist := NaN (all-ones bytes), state := initial
    cudaMemsetParams mp{};
    mp.dst = c->fhist;
    mp.pitch = 0;
    mp.value = 0xFF;
    mp.elementSize = 1;
    mp.width = sizeof(double) * (max_iter + 1);
    mp.height = 1;
    CU(cudaGraphAddMemsetNode(&n_hist, g, nullptr, 0, &mp));
    FitState* st = c->fstate;
    int mi = max_iter;
    {
        void* args[] = {&st, &mi};
        cfust_status s = add_kernel_node(c, g, &n_hist, &n_init, (void*)fit_init_kernel, args, 1);
        if (s != CFUST_OK) return s;
    }
    // WHILE: one EM iteration per pass
    cudaGraphConditionalHandle hloop;
    CU(cudaGraphConditionalHandleCreate(&hloop, g, max_iter > 0 ? 1u : 0u, cudaGraphCondAssignDefault));
    const int width = c->g * stats_per_comp(c->p, c->q) + 1;
    cfust_status s = add_conditional(c, g, &n_init, hloop, cudaGraphCondTypeWhile, &n_loop,
                                     &c->fg_body_kernels, [&]() -> cfust_status {
        cfust_status r;
        if ((r = enqueue_estep(c)) != CFUST_OK) return r;
        fit_gate_kernel<<<1, 1, 0, c->st>>>(c->fstate, c->stats + (width - 1), c->flags, c->fhist, tol);
        LAUNCHED();
        if ((r = enqueue_mstep(c, (const int*)((char*)c->fstate + offsetof(FitState, done)))) != CFUST_OK)
            return r;
        fit_commit_kernel<<<1, 128, 0, c->st>>>(c->D, c->fstate, c->flags, c->comp_status, c->pi_n, c->mu_n,
                                                c->Sigma_n, c->Delta_n, c->nu_n, c->pi, c->mu, c->Sigma,
                                                c->Delta, c->nu, max_iter, hloop);
        LAUNCHED();
        return CFUST_OK;
    });
    if (s != CFUST_OK) return s;
    c->fg_final_kernels = 0;
    if (!(flags & CFUST_FIT_NO_FINAL)) {
        // every handle must belong to a conditional node: create this one only when used
        cudaGraphConditionalHandle hfinal;
        CU(cudaGraphConditionalHandleCreate(&hfinal, g, 0u, cudaGraphCondAssignDefault));
        {
            const FitState* cst = c->fstate;
            void* args[] = {(void*)&cst, &hfinal};
            if ((s = add_kernel_node(c, g, &n_loop, &n_fgate, (void*)fit_final_gate_kernel, args, 1)) != CFUST_OK)
                return s;
        }
        s = add_conditional(c, g, &n_fgate, hfinal, cudaGraphCondTypeIf, &n_final, &c->fg_final_kernels,
                            [&]() -> cfust_status {
            cfust_status r;
            if ((r = enqueue_loglik(c)) != CFUST_OK) return r;
            fit_final_kernel<<<1, 1, 0, c->st>>>(c->fstate, c->stats, c->flags, c->fhist, max_iter);
            LAUNCHED();
            return CFUST_OK;
        });
        if (s != CFUST_OK) return s;
    }
    CU(cudaGraphInstantiate(&c->fexec, g, 0));
    c->fg_max_iter = max_iter;
    c->fg_tol = tol;
    c->fg_flags = flags;
    return CFUST_OK;
}

static const char* status_name(int s)
{
    switch (s) {
    case CFUST_EEMPTY: return "has no weight (sum tau = 0)";
    case CFUST_ENOTPD: return "not positive definite";
    default: return "failed";
    }
}

extern "C" cfust_status cfust_fit_batch(int nfits, cfust_ctx* const* ctxs, int max_iter, double tol,
                                        int flags, int* iters_out, double* loglik_hist,
                                        cfust_status* status_out)
{
    if (nfits < 0 || (nfits > 0 && !ctxs))
        return fail(nullptr, CFUST_EINVAL, "cfust_fit_batch: bad nfits or ctxs");
    if (max_iter < 0) return fail(nullptr, CFUST_EINVAL, "cfust_fit_batch: max_iter < 0");
    if (flags & ~CFUST_FIT_NO_FINAL) return fail(nullptr, CFUST_EINVAL, "cfust_fit_batch: unknown flags");
    for (int i = 0; i < nfits; ++i) {
        cfust_ctx* c = ctxs[i];
        if (!c) return fail(nullptr, CFUST_EINVAL, "cfust_fit_batch: ctxs[" + std::to_string(i) + "] is NULL");
        if (!c->have_data || !c->have_params)
            return fail(c, CFUST_ESTATE, "cfust_fit_batch: set_data and set_params must come first");
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == c) return fail(nullptr, CFUST_EINVAL, "cfust_fit_batch: a context appears twice");
    }
    // build (or reuse) each fit's graph, then launch them all: each context's
    // graph runs on its own stream, ordered after the work already on c->st
    for (int i = 0; i < nfits; ++i) {
        cfust_ctx* c = ctxs[i];
        CU(cudaSetDevice(c->opts.device));
        cfust_status s = build_fit_graph(c, max_iter, tol, flags);
        if (s != CFUST_OK) {
            drop_fit_graph(c);
            g_create_err = "fit " + std::to_string(i) + ": " + c->err;
            return s;
        }
    }
    // a CUDA error here is not one fit's failure: report it for the batch
    auto cuda_fail = [&](int i, const char* what, cudaError_t e) {
        g_create_err = "cfust_fit_batch: fit " + std::to_string(i) + ": " + what + ": " +
                       cudaGetErrorString(e);
        ctxs[i]->err = g_create_err;
        return CFUST_ECUDA;
    };
    cudaError_t e;
    for (int i = 0; i < nfits; ++i) {
        cfust_ctx* c = ctxs[i];
        if ((e = cudaSetDevice(c->opts.device)) != cudaSuccess) return cuda_fail(i, "cudaSetDevice", e);
        if ((e = cudaStreamSynchronize(c->st)) != cudaSuccess) return cuda_fail(i, "stream sync", e);
        if ((e = cudaGraphLaunch(c->fexec, c->gst)) != cudaSuccess) return cuda_fail(i, "cudaGraphLaunch", e);
        if ((e = cudaMemcpyAsync(c->h_fstate, c->fstate, sizeof(FitState), cudaMemcpyDeviceToHost, c->gst)) ||
            (e = cudaMemcpyAsync(c->h_fhist, c->fhist, sizeof(double) * (max_iter + 1),
                                 cudaMemcpyDeviceToHost, c->gst)))
            return cuda_fail(i, "result copy", e);
    }
    cfust_status first = CFUST_OK;
    for (int i = 0; i < nfits; ++i) {
        cfust_ctx* c = ctxs[i];
        if ((e = cudaSetDevice(c->opts.device)) != cudaSuccess) return cuda_fail(i, "cudaSetDevice", e);
        if ((e = cudaStreamSynchronize(c->gst)) != cudaSuccess) return cuda_fail(i, "fit graph", e);
        const FitState& fs = *c->h_fstate;
        const int body_runs = max_iter == 0 ? 0 : (fs.final_pass ? max_iter : fs.it + 1);
        c->launches += 1 + c->fg_body_kernels * body_runs + (fs.final_pass ? 1 + c->fg_final_kernels : 0);
        c->have_stats = false;
        const int it = fs.it;
        if (iters_out) iters_out[i] = it;
        if (loglik_hist) std::memcpy(loglik_hist + (size_t)i * (max_iter + 1), c->h_fhist,
                                     sizeof(double) * (max_iter + 1));
        cfust_status s = (cfust_status)fs.status;
        if (s != CFUST_OK) {
            if (fs.comp >= 0)
                fail(c, s, "cfust_fit_batch: iteration " + std::to_string(it) + ": component " +
                               std::to_string(fs.comp) + " " + status_name(s));
            else
                fail(c, s, "cfust_fit_batch: iteration " + std::to_string(it) +
                               (s == CFUST_ENAN ? ": non-finite density or log-likelihood"
                                                : ": Sigma, Omega or Lambda not positive definite"));
            if (first == CFUST_OK) first = s;
        }
        if (status_out) status_out[i] = s;
    }
    return first;
}

// ---------------------------------------------------------------------------
// Initialisation (Sec. 3.3, Algorithm 1 with the moment starts of eq 23).
// ---------------------------------------------------------------------------
// k-means partitions for Algorithm 1 (Sec. 3.3): Lloyd's iteration on the device from
// seeded starting centres; the assignment and the fixed-order cluster sums run as kernels,
// the g x p centre update (a division per entry) on the host.
extern "C" cfust_status cfust_kmeans(cfust_ctx* c, int nstarts, uint64_t seed, int max_iter, int32_t* labels_out,
                                     int* iters_out, double* centres_out)
{
    if (!c) return fail(nullptr, CFUST_EINVAL, "cfust_kmeans: ctx is NULL");
    if (!c->have_data) return fail(c, CFUST_ESTATE, "cfust_kmeans: set_data must come first");
    if (nstarts < 1 || max_iter < 1 || !labels_out)
        return fail(c, CFUST_EINVAL, "cfust_kmeans: need nstarts >= 1, max_iter >= 1 and labels_out");
    const int p = c->p, g = c->g;
    const long long n = c->n;
    if (n < g) return fail(c, CFUST_EINVAL, "cfust_kmeans: fewer observations than clusters");
    CU(cudaSetDevice(c->opts.device));
    const int chunk = 64;
    const long long nchunks = (n + chunk - 1) / chunk;
    const int blocks = (int)std::min<long long>(nchunks, 4LL * c->nsm);
    const int W0 = 1 + p;
    int *dlab = nullptr, *dchg = nullptr;
    double *partial = nullptr, *sums = nullptr, *dcen = nullptr;
    cudaError_t e;
    auto cleanup = [&]() { cudaFree(dlab); cudaFree(dchg); cudaFree(partial); cudaFree(sums); cudaFree(dcen); };
    if ((e = dalloc(&dlab, (size_t)n)) != cudaSuccess || (e = dalloc(&dchg, 1)) != cudaSuccess ||
        (e = dalloc(&partial, (size_t)blocks * g * W0)) != cudaSuccess ||
        (e = dalloc(&sums, (size_t)g * W0)) != cudaSuccess || (e = dalloc(&dcen, (size_t)g * p)) != cudaSuccess) {
        cleanup();
        return fail(c, CFUST_ENOMEM, std::string("cfust_kmeans: ") + cudaGetErrorString(e));
    }
    std::vector<double> cen((size_t)g * p), s0((size_t)g * W0);
    std::vector<long long> idx(g);
    cfust_status s = CFUST_OK;
    for (int st = 0; st < nstarts && s == CFUST_OK; ++st) {
        // starting centres: g distinct observations, index floor(u n) with u the SplitMix64
        // output for key seed ^ ((st+1) << 40) ^ (1 << 36) ^ (h + 1 + g a), a = 0, 1, ...
        for (int h = 0; h < g; ++h)
            for (uint64_t a = 0;; ++a) {
                const uint64_t key = seed ^ ((uint64_t)(st + 1) << 40) ^ ((uint64_t)1 << 36) ^
                                     (uint64_t)(h + 1 + (uint64_t)g * a);
                long long j = (long long)(splitmix_u01(key) * (double)n);
                if (j > n - 1) j = n - 1;
                bool dup = false;
                for (int l = 0; l < h; ++l) dup |= idx[l] == j;
                if (!dup) { idx[h] = j; break; }
            }
        e = cudaSuccess;
        for (int h = 0; h < g && e == cudaSuccess; ++h)
            e = cudaMemcpyAsync(dcen + (size_t)h * p, c->y + (size_t)idx[h] * p, sizeof(double) * p,
                                cudaMemcpyDeviceToDevice, c->st);
        if (e == cudaSuccess) e = cudaMemsetAsync(dlab, 0xff, sizeof(int) * n, c->st);  // -1: no label yet
        int it = 0;
        while (e == cudaSuccess) {
            int chg = 0;
            e = cudaMemsetAsync(dchg, 0, sizeof(int), c->st);
            if (e == cudaSuccess) e = launch_kmeans_assign(c->D, c->y, dcen, dlab, dchg, c->nsm, c->st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(&chg, dchg, sizeof(int), cudaMemcpyDeviceToHost, c->st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
            if (e != cudaSuccess) break;
            ++c->launches;
            ++it;
            if (chg == 0 || it == max_iter) break;
            // update: the cluster means (an empty cluster keeps its centre)
            e = launch_cluster_moments(0, c->D, c->y, dlab, nullptr, chunk, blocks, partial, c->st);
            if (e == cudaSuccess) {
                reduce_partials_kernel<<<(g * W0 + 127) / 128, 128, 0, c->st>>>(partial, blocks, g * W0, sums, c->flags);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess) e = cudaMemcpyAsync(s0.data(), sums, sizeof(double) * g * W0, cudaMemcpyDeviceToHost, c->st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(cen.data(), dcen, sizeof(double) * g * p, cudaMemcpyDeviceToHost, c->st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
            if (e != cudaSuccess) break;
            c->launches += 2;
            for (int h = 0; h < g; ++h) {
                const double cnt = s0[(size_t)h * W0];
                if (cnt > 0.0)
                    for (int d = 0; d < p; ++d) cen[(size_t)h * p + d] = s0[(size_t)h * W0 + 1 + d] / cnt;
            }
            e = cudaMemcpyAsync(dcen, cen.data(), sizeof(double) * g * p, cudaMemcpyHostToDevice, c->st);
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(labels_out + (size_t)st * n, dlab, sizeof(int) * n, cudaMemcpyDeviceToHost, c->st);
        if (e == cudaSuccess && centres_out)
            e = cudaMemcpyAsync(centres_out + (size_t)st * g * p, dcen, sizeof(double) * g * p, cudaMemcpyDeviceToHost, c->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
        if (e != cudaSuccess) s = fail(c, CFUST_ECUDA, std::string("cfust_kmeans: ") + cudaGetErrorString(e));
        if (iters_out) iters_out[st] = it;
    }
    cleanup();
    return s;
}

extern "C" cfust_status cfust_init(cfust_ctx* c, int nstarts, const int32_t* labels, uint64_t seed,
                                   int nalpha, const double* alphas, double nu0, double* loglik_out,
                                   int* best_out)
{
    if (!c) return fail(nullptr, CFUST_EINVAL, "cfust_init: ctx is NULL");
    if (!c->have_data) return fail(c, CFUST_ESTATE, "cfust_init: set_data must come first");
    static const double grid[9] = {0.1, 0.2, 0.3, 0.4, 0.5, 0.6, 0.7, 0.8, 0.9};
    if (!alphas) {
        if (nalpha != 0 && nalpha != 9)
            return fail(c, CFUST_EINVAL, "cfust_init: with alphas NULL, nalpha must be 0 or 9");
        alphas = grid;
        nalpha = 9;
    }
    if (nstarts < 1 || nalpha < 1) return fail(c, CFUST_EINVAL, "cfust_init: need nstarts >= 1, nalpha >= 1");
    for (int a = 0; a < nalpha; ++a)
        if (!(alphas[a] > 0.0 && alphas[a] < 1.0))
            return fail(c, CFUST_EINVAL, "cfust_init: alpha must lie in (0, 1)");
    if (!(nu0 > 0.0)) return fail(c, CFUST_EINVAL, "cfust_init: nu0 must be positive");
    const int p = c->p, q = c->q, g = c->g;
    const long long n = c->n;
    if (labels)
        for (long long t = 0; t < (long long)nstarts * n; ++t)
            if (labels[t] < 0 || labels[t] >= g)
                return fail(c, CFUST_EINVAL, "cfust_init: labels must lie in [0, g)");
    CU(cudaSetDevice(c->opts.device));
    const int chunk = 64;
    const long long nchunks = (n + chunk - 1) / chunk;
    const int blocks = (int)std::min<long long>(nchunks, 4LL * c->nsm);
    const int W0 = 1 + p, W1 = p * (p + 1) / 2 + p;
    int* dlab = nullptr;
    double *partial = nullptr, *sums = nullptr, *dmean = nullptr;
    cudaError_t e;
    auto cleanup = [&]() { cudaFree(dlab); cudaFree(partial); cudaFree(sums); cudaFree(dmean); };
    if ((e = dalloc(&dlab, (size_t)n)) != cudaSuccess || (e = dalloc(&partial, (size_t)blocks * g * W1)) != cudaSuccess ||
        (e = dalloc(&sums, (size_t)g * W1)) != cudaSuccess || (e = dalloc(&dmean, (size_t)g * p)) != cudaSuccess) {
        cleanup();
        return fail(c, CFUST_ENOMEM, std::string("cfust_init: ") + cudaGetErrorString(e));
    }
    const double PI = 3.14159265358979323846;
    std::vector<double> s0((size_t)g * W0), s1((size_t)g * W1), mean((size_t)g * p);
    std::vector<double> cp(g), cm((size_t)g * p), cS((size_t)g * p * p), cD((size_t)g * p * q), cn(g);
    std::vector<double> bp, bm, bS, bD, bn;
    double lbest = -INFINITY;  // the best log-likelihood so far
    int ibest = -1;            // no candidate kept yet
    cfust_status s = CFUST_OK;
    for (int st = 0; st < nstarts && s == CFUST_OK; ++st) {  // each start
        // its partition: given labels or a random one
        if (labels) e = cudaMemcpyAsync(dlab, labels + (size_t)st * n, sizeof(int) * n, cudaMemcpyHostToDevice, c->st);
        else e = launch_random_partition(n, g, seed, st, dlab, c->st);
        if (e == cudaSuccess) e = launch_cluster_moments(0, c->D, c->y, dlab, nullptr, chunk, blocks, partial, c->st);
        if (e == cudaSuccess) {
            reduce_partials_kernel<<<(g * W0 + 127) / 128, 128, 0, c->st>>>(partial, blocks, g * W0, sums, c->flags);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(s0.data(), sums, sizeof(double) * g * W0, cudaMemcpyDeviceToHost, c->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
        if (e != cudaSuccess) { s = fail(c, CFUST_ECUDA, std::string("cfust_init: ") + cudaGetErrorString(e)); break; }
        c->launches += (labels ? 0 : 1) + 2;
        // cluster means, then the centred second and third moments
        std::vector<long long> nh(g);
        for (int h = 0; h < g; ++h) {
            nh[h] = (long long)s0[(size_t)h * W0];
            for (int i = 0; i < p; ++i) mean[(size_t)h * p + i] = nh[h] > 0 ? s0[(size_t)h * W0 + 1 + i] / nh[h] : 0.0;
        }
        e = cudaMemcpyAsync(dmean, mean.data(), sizeof(double) * g * p, cudaMemcpyHostToDevice, c->st);
        if (e == cudaSuccess) e = launch_cluster_moments(1, c->D, c->y, dlab, dmean, chunk, blocks, partial, c->st);
        if (e == cudaSuccess) {
            reduce_partials_kernel<<<(g * W1 + 127) / 128, 128, 0, c->st>>>(partial, blocks, g * W1, sums, c->flags);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(s1.data(), sums, sizeof(double) * g * W1, cudaMemcpyDeviceToHost, c->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
        if (e != cudaSuccess) { s = fail(c, CFUST_ECUDA, std::string("cfust_init: ") + cudaGetErrorString(e)); break; }
        c->launches += 2;
        for (int a = 0; a < nalpha; ++a) {  // each alpha of the grid
            const double alpha = alphas[a];
            bool valid = true;
            for (int h = 0; h < g && valid; ++h) {  // each cluster
                if (nh[h] < 2) { valid = false; break; }
                const double* Sr = s1.data() + (size_t)h * W1;  // packed lower sum r r^T, then sum r^3
                auto Sab = [&](int x, int y2) {
                    const int hi = x > y2 ? x : y2, lo = x > y2 ? y2 : x;
                    return Sr[hi * (hi + 1) / 2 + lo] / (double)(nh[h] - 1);
                };
                cp[h] = (double)nh[h] / (double)n;  // pi from the cluster sizes
                double* Dh = cD.data() + (size_t)h * p * q;
                double* Sh = cS.data() + (size_t)h * p * p;
                for (int t = 0; t < p * q; ++t) Dh[t] = 0.0;
                // eq (23): delta = sign(m3) sqrt(pi (1 - alpha) s* / (pi - 2)) element-wise,
                // Sigma = S - (1 - alpha) diag(s*), mu = ybar - sqrt(2/pi) delta, nu = nu0; Delta is
                // diag(delta) (q = p), the column delta (q = 1), else delta on the leading diagonal
                for (int x = 0; x < p; ++x) {
                    const bool skewed = q == 1 || q >= p || x < q;
                    const double sa = Sab(x, x);
                    const double m3 = Sr[p * (p + 1) / 2 + x];
                    const double d = skewed ? (m3 >= 0.0 ? 1.0 : -1.0) * std::sqrt(PI * (1.0 - alpha) * sa / (PI - 2.0)) : 0.0;
                    if (q == 1) Dh[x * q] = d;
                    else if (x < q) Dh[x * q + x] = d;
                    cm[(size_t)h * p + x] = mean[(size_t)h * p + x] - std::sqrt(2.0 / PI) * d;
                    for (int y2 = 0; y2 < p; ++y2)
                        Sh[x * p + y2] = Sab(x, y2) - (x == y2 && skewed ? (1.0 - alpha) * sa : 0.0);
                }
                cn[h] = nu0;
                // Sigma^(0) must be positive definite
                std::vector<double> L((size_t)p * p, 0.0);
                for (int j = 0; j < p && valid; ++j) {
                    double sum = Sh[j * p + j];
                    for (int k = 0; k < j; ++k) sum -= L[j * p + k] * L[j * p + k];
                    if (!(sum > 0.0)) { valid = false; break; }
                    L[j * p + j] = std::sqrt(sum);
                    for (int i2 = j + 1; i2 < p; ++i2) {
                        double t = Sh[i2 * p + j];
                        for (int k = 0; k < j; ++k) t -= L[i2 * p + k] * L[j * p + k];
                        L[i2 * p + j] = t / L[j * p + j];
                    }
                }
            }
            double L = -INFINITY;
            if (valid) {
                cfust_params P{cp.data(), cm.data(), cS.data(), cD.data(), cn.data()};
                cfust_status r = cfust_set_params(c, &P);
                if (r == CFUST_OK) r = cfust_loglik(c, &L);  // the candidate's log-likelihood
                if (r == CFUST_ECUDA || r == CFUST_ENOMEM) { s = r; break; }
                if (r != CFUST_OK || !std::isfinite(L)) L = -INFINITY;
            }
            if (loglik_out) loglik_out[(size_t)st * nalpha + a] = L;
            if (L > lbest) {  // keep the best candidate (first maximum)
                lbest = L;
                ibest = st * nalpha + a;
                bp = cp; bm = cm; bS = cS; bD = cD; bn = cn;
            }
        }
    }
    cleanup();
    if (s != CFUST_OK) return s;
    if (best_out) *best_out = ibest;
    if (ibest < 0) {
        c->have_params = false;
        return fail(c, CFUST_ENOTPD, "cfust_init: no candidate start has a positive definite Sigma^(0)");
    }
    cfust_params P{bp.data(), bm.data(), bS.data(), bD.data(), bn.data()};
    return cfust_set_params(c, &P);
}

extern "C" cfust_status cfust_tk_eval(cfust_ctx* c, int k, int count, const double* b,
                                      const double* V, const double* nu, double* out, double* se)
{
    if (!c) return fail(nullptr, CFUST_EINVAL, "cfust_tk_eval: ctx is NULL");
    if (k < 0 || k > CF_MAXDIM || count < 1 || !b || !V || !nu || !out)
        return fail(c, CFUST_EINVAL, "cfust_tk_eval: bad arguments (0 <= k <= 8, count >= 1)");
    for (int i = 0; i < count; ++i)
        if (!(nu[i] > 0.0)) return fail(c, CFUST_EINVAL, "cfust_tk_eval: nu must be positive");
    if (k == 0) {
        for (int i = 0; i < count; ++i) {
            out[i] = 1.0;
            if (se) se[i] = 0.0;
        }
        return CFUST_OK;
    }
    // standardise on the host: limits b_i / sqrt(V_ii), Cholesky factor of corr(V)
    std::vector<double> bt((size_t)count * k), fac((size_t)count * k * k, 0.0), dofv(nu, nu + count);
    std::vector<int> foff(count), tab(count);
    for (int i = 0; i < count; ++i) {
        const double* Vi = V + (size_t)i * k * k;
        double* L = fac.data() + (size_t)i * k * k;
        std::vector<double> ds(k);
        for (int a = 0; a < k; ++a) {
            if (!(Vi[a * k + a] > 0.0)) return fail(c, CFUST_EINVAL, "cfust_tk_eval: V not positive definite");
            ds[a] = 1.0 / std::sqrt(Vi[a * k + a]);
            bt[(size_t)i * k + a] = b[(size_t)i * k + a] * ds[a];
        }
        for (int jj = 0; jj < k; ++jj) {
            double sum = 1.0;
            for (int l = 0; l < jj; ++l) sum -= L[jj * k + l] * L[jj * k + l];
            if (!(sum > 0.0)) return fail(c, CFUST_EINVAL, "cfust_tk_eval: V not positive definite");
            L[jj * k + jj] = std::sqrt(sum);
            for (int ii = jj + 1; ii < k; ++ii) {
                double t = Vi[ii * k + jj] * ds[ii] * ds[jj];
                for (int l = 0; l < jj; ++l) t -= L[ii * k + l] * L[jj * k + l];
                L[ii * k + jj] = t / L[jj * k + jj];
            }
        }
        foff[i] = i * k * k;
        tab[i] = i;
    }
    CU(cudaSetDevice(c->opts.device));
    const size_t NM = (size_t)c->lat.N * c->lat.M;
    const bool lattice = k >= 3;
    RecSet r{};
    r.k = k;
    r.nrec = count;
    double *dF = nullptr, *t64 = nullptr, *k64 = nullptr;
    float *t32 = nullptr, *k32 = nullptr;
    float2* t1t = nullptr;
    // FP32 T_2 reads per-case T_1 tables (32 KB each) when the cases are few
    const bool use_t1tab = k == 2 && c->opts.precision != CFUST_PREC_FP64 && count <= 4096;
    cudaError_t e = cudaSuccess;
    auto cleanup = [&]() {
        cudaFree(r.bt); cudaFree(r.fac); cudaFree(r.tab); cudaFree(r.dof); cudaFree(r.res);
        cudaFree(r.se); cudaFree(dF); cudaFree(t64); cudaFree(t32); cudaFree(k64); cudaFree(k32);
        cudaFree(t1t); cudaFree(r.t2f);
    };
    if ((e = dalloc(&r.bt, bt.size())) != cudaSuccess || (e = dalloc(&r.fac, count)) != cudaSuccess ||
        (e = dalloc(&r.tab, count)) != cudaSuccess || (e = dalloc(&r.dof, count)) != cudaSuccess ||
        (e = dalloc(&r.res, count)) != cudaSuccess || (e = dalloc(&r.se, count)) != cudaSuccess ||
        (e = dalloc(&dF, fac.size())) != cudaSuccess ||
        (e = dalloc(&k64, (size_t)count * CST_STRIDE)) != cudaSuccess ||
        (e = dalloc(&k32, (size_t)count * CST_STRIDE)) != cudaSuccess ||
        (e = dalloc(&t64, lattice ? NM * count : 1)) != cudaSuccess ||
        (e = dalloc(&t32, lattice ? NM * count : 1)) != cudaSuccess ||
        (e = dalloc(&t1t, use_t1tab ? (size_t)count * T1TAB_N : 1)) != cudaSuccess ||
        (k == 2 && c->opts.precision != CFUST_PREC_FP64 && (e = dalloc(&r.t2f, (size_t)2 * count)) != cudaSuccess)) {
        cleanup();
        return fail(c, CFUST_ENOMEM, std::string("cfust_tk_eval: ") + cudaGetErrorString(e));
    }
    do {
        if ((e = cudaMemcpyAsync(r.bt, bt.data(), sizeof(double) * bt.size(), cudaMemcpyHostToDevice, c->st))) break;
        if ((e = cudaMemcpyAsync(r.fac, foff.data(), sizeof(int) * count, cudaMemcpyHostToDevice, c->st))) break;
        if ((e = cudaMemcpyAsync(r.tab, tab.data(), sizeof(int) * count, cudaMemcpyHostToDevice, c->st))) break;
        if ((e = cudaMemcpyAsync(r.dof, dofv.data(), sizeof(double) * count, cudaMemcpyHostToDevice, c->st))) break;
        if ((e = cudaMemcpyAsync(dF, fac.data(), sizeof(double) * fac.size(), cudaMemcpyHostToDevice, c->st))) break;
        std::vector<float4> t2f;
        if (r.t2f) {
            t2f.resize((size_t)2 * count);
            for (int i = 0; i < count; ++i)
                t2_record_f32(bt[2 * i], bt[2 * i + 1], fac[(size_t)i * 4 + 2], dofv[i], &t2f[2 * i]);
            if ((e = cudaMemcpyAsync(r.t2f, t2f.data(), sizeof(float4) * t2f.size(), cudaMemcpyHostToDevice, c->st))) break;
        }
        dof_consts_kernel<<<(count + 127) / 128, 128, 0, c->st>>>(c->D, c->Ly, nullptr, count, r.dof, k64, k32);
        c->launches++;
        if ((e = cudaGetLastError())) break;
        if (lattice) {
            const long long total = (long long)count * NM;
            const int blocks = (int)std::min<long long>((total + 127) / 128, 64LL * c->nsm);
            chi_table_kernel<<<blocks, 128, 0, c->st>>>(count, 1, r.dof, k64, c->lat, c->shf64,
                                                         c->opts.precision == CFUST_PREC_FP64 ? 1e-15 : 1e-9,
                                                         t64, t32, nullptr, nullptr);
            c->launches++;
            if ((e = cudaGetLastError())) break;
        }
        if (use_t1tab) {
            const int total = count * T1TAB_N;
            t1_table_kernel<<<(total + 255) / 256, 256, 0, c->st>>>(count, r.dof, k64, t1t, 7);
            c->launches++;
            if ((e = cudaGetLastError())) break;
        }
        IntegArgs ia = integ_args(c);
        ia.t1tab = use_t1tab ? t1t : nullptr;
        ia.cst64 = k64;
        ia.cst32 = k32;
        ia.F = dF;
        ia.chi64 = t64;
        ia.chi32 = t32;
        if ((e = launch_integrals(r, ia, c->opts.precision != CFUST_PREC_FP64, c->nsm, c->st, &c->launches))) break;
        if ((e = cudaMemcpyAsync(out, r.res, sizeof(double) * count, cudaMemcpyDeviceToHost, c->st))) break;
        if (se && (e = cudaMemcpyAsync(se, r.se, sizeof(double) * count, cudaMemcpyDeviceToHost, c->st))) break;
        e = cudaStreamSynchronize(c->st);
    } while (0);
    cfust_status s = CFUST_OK;
    if (e != cudaSuccess) s = fail(c, CFUST_ECUDA, std::string("cfust_tk_eval: ") + cudaGetErrorString(e));
    cleanup();
    return s;
}

// ---------------------------------------------------------------------------
// Learned surrogate (not part of the paper)
// ---------------------------------------------------------------------------
extern "C" cfust_surrogate_opts cfust_surrogate_default_opts(void)
{
    cfust_surrogate_opts o;
    o.epochs = 48;
    o.batch = 8192;
    o.samples_per_epoch = 1 << 20;
    o.lr = 3e-3f;
    o.margin = 0.5f;
    o.seed = 1;
    return o;
}

extern "C" cfust_status cfust_surrogate_train(cfust_ctx* c, const cfust_surrogate_opts* opts, double* loglik_out,
                                              double* losses)
{
    if (!c) return fail(nullptr, CFUST_EINVAL, "cfust_surrogate_train: ctx is NULL");
    if (!opts) return fail(c, CFUST_EINVAL, "cfust_surrogate_train: opts is NULL");
    if (!c->single_pass)
        return fail(c, CFUST_EINVAL, "cfust_surrogate_train: needs single-pass moments (moments = 1, q >= 3)");
    if (c->opts.elogw == CFUST_ELOGW_EXACT)
        return fail(c, CFUST_EINVAL, "cfust_surrogate_train: the network predicts no E[log W]; use elogw = OSL");
    if (opts->epochs < 0 || opts->batch < 64 || opts->batch > (1 << 20) || opts->batch % 64 ||
        !(opts->lr > 0.f) || !(opts->margin >= 0.f))
        return fail(c, CFUST_EINVAL, "cfust_surrogate_train: epochs >= 0, batch a multiple of 64 in [64, 2^20], "
                                     "lr > 0, margin >= 0");
    CU(cudaSetDevice(c->opts.device));
    const bool was = c->sur.on;
    c->sur.on = false;
    cfust_status s = cfust_estep(c, loglik_out);  // the lattice E-step whose records are the samples
    if (s != CFUST_OK) {
        c->sur.on = was;
        return s;
    }
    const long long nr = c->n * c->g;
    cudaError_t e = sur_reserve(c->sur, c->q, nr, c->st);
    RecSet L0 = c->rec[0];
    L0.nrec = nr;
    if (!e) e = sur_collect(c->sur, L0, c->rec[3], c->F, c->st);
    if (e == cudaErrorInvalidValue)
        return fail(c, CFUST_ESTATE, "cfust_surrogate_train: fewer than 64 usable records");
    SurOpts so;
    so.epochs = opts->epochs; so.batch = opts->batch; so.samples_per_epoch = opts->samples_per_epoch;
    so.lr = opts->lr; so.margin = opts->margin; so.seed = opts->seed;
    if (!e) e = sur_train(c->sur, so, c->st, losses);
    if (e) return fail(c, CFUST_ECUDA, std::string("cfust_surrogate_train: ") + cudaGetErrorString(e));
    c->sur.on = true;
    return CFUST_OK;
}

extern "C" cfust_status cfust_surrogate_use(cfust_ctx* c, int on)
{
    if (!c) return fail(nullptr, CFUST_EINVAL, "cfust_surrogate_use: ctx is NULL");
    if (on && !c->sur.trained) return fail(c, CFUST_ESTATE, "cfust_surrogate_use: train the surrogate first");
    c->sur.on = on != 0;
    return CFUST_OK;
}

extern "C" cfust_status cfust_surrogate_info(cfust_ctx* c, int64_t* records, int64_t* fallbacks)
{
    if (!c) return fail(nullptr, CFUST_EINVAL, "cfust_surrogate_info: ctx is NULL");
    int nf[2] = {0, 0};
    if (c->sur.nfall) {
        CU(cudaSetDevice(c->opts.device));
        CU(cudaMemcpyAsync(nf, c->sur.nfall, sizeof(nf), cudaMemcpyDeviceToHost, c->st));
        CU(cudaStreamSynchronize(c->st));
    }
    if (records) *records = c->sur.last_records;
    // a pair in the moment list has both of its records (alpha_s, and alpha with the
    // moments) evaluated by the shared lattice pass
    if (fallbacks) *fallbacks = (int64_t)nf[0] + 2 * (int64_t)nf[1];
    return CFUST_OK;
}

extern "C" cfust_status cfust_surrogate_params(cfust_ctx* c, float* theta, float* stats)
{
    if (!c) return fail(nullptr, CFUST_EINVAL, "cfust_surrogate_params: ctx is NULL");
    if (!c->sur.trained) return fail(c, CFUST_ESTATE, "cfust_surrogate_params: not trained");
    CU(cudaSetDevice(c->opts.device));
    if (theta) CU(cudaMemcpyAsync(theta, c->sur.theta, sizeof(float) * MLP_NPARAM, cudaMemcpyDeviceToHost, c->st));
    if (stats) CU(cudaMemcpyAsync(stats, c->sur.stats, sizeof(float) * MLP_NSTAT, cudaMemcpyDeviceToHost, c->st));
    CU(cudaStreamSynchronize(c->st));
    return CFUST_OK;
}
