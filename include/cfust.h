/*
 * cfust.h -- C ABI of the GB300 (sm_103a) FM-CFUST EM library.
 *
 * The library runs the data-parallel hot path of the EM algorithm for finite
 * mixtures of canonical fundamental skew t (CFUST) distributions of
 * Lee, Leemaqz & McLachlan, "A simple multithreaded implementation of the EM
 * algorithm for mixture models" (arXiv:1606.02054), on one GPU:
 *
 *   E-step over every (observation j, component h) pair     Sec. 3.1, eqs (12)-(17)
 *     CFUST density                                         Sec. 2, eq (4)
 *     weighted sufficient statistics of the M-step          Sec. 3.2, eqs (18)-(22)
 *   M-step solve                                            Sec. 3.2, eqs (18)-(22)
 *   log-likelihood, fused into the E-step pass              Sec. 4.3, eq (27)
 *   Aitken stopping rule                                    Sec. 3.4, eqs (24)-(26)
 *
 * Conventions shared by every entry point:
 *   - Every call returns a cfust_status and never aborts.  On failure,
 *     cfust_last_error() gives a one-line reason (naming the component for
 *     CFUST_ENOTPD / CFUST_EEMPTY / CFUST_ENUROOT).
 *   - Parameters follow the paper's parameterisation exactly: pi (g),
 *     mu (g x p), Sigma (g x p x p), Delta (g x p x q), nu (g), all FP64,
 *     row-major, caller-owned.  They are copied in and out; the library keeps
 *     its own device copy.
 *   - A context is used from one host thread at a time.  All device work is
 *     issued on opts.cuda_stream (NULL = the legacy default stream).
 *   - There is no CPU fallback: without a usable CUDA device every call that
 *     needs one returns CFUST_ECUDA.
 */
#ifndef CFUST_H
#define CFUST_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cfust_ctx cfust_ctx; /* opaque; owned by the library */

typedef enum {
    CFUST_OK = 0,
    CFUST_EINVAL = 1,   /* bad argument (sizes, NULL pointer, option range) */
    CFUST_ENOTPD = 2,   /* Sigma, Omega = Sigma + Delta Delta^T, Lambda or sum tau e3 not positive definite */
    CFUST_EEMPTY = 3,   /* a component's sum of tau is not positive (eq 18) */
    CFUST_ENUROOT = 4,  /* eq (22) has no root in [nu_min, nu_max]; nu clamped to the bound */
    CFUST_ENAN = 5,     /* a non-finite log-likelihood or statistic */
    CFUST_ETIMEOUT = 6, /* a bounded device wait gave up */
    CFUST_ECUDA = 7,    /* CUDA runtime error (message in cfust_last_error) */
    CFUST_ENOMEM = 8,   /* device or host allocation failed */
    CFUST_ESTATE = 9    /* call out of order (e.g. estep before set_data/set_params) */
} cfust_status;

/* Arithmetic of the E-step.
 *   CFUST_PREC_FP64:  everything in FP64.
 *   CFUST_PREC_FP32:  the integrals (the T_q terms of eqs (4), (13) and the
 *                     truncated-t moments of eqs (16)-(17)) in FP32; whitening,
 *                     log t_p, the log-sum-exp of eq (12), the log-likelihood of
 *                     eq (27), the sufficient statistics and the M-step in FP64.
 *   CFUST_PREC_MIXED: as FP32, and also the whitening (from FP32 copies of y and
 *                     of the factors) and the tau-weighted statistics (FP32 sums
 *                     per block of observations with compensation, FP64 across
 *                     blocks) in FP32; FP64 stays for the Cholesky factorisations
 *                     and inverses, tau, the log-likelihood, the M-step and nu. */
enum { CFUST_PREC_FP64 = 0, CFUST_PREC_FP32 = 1, CFUST_PREC_MIXED = 2 };

/* Element type of the observation matrix passed to cfust_set_data. */
enum { CFUST_F32 = 0, CFUST_F64 = 1 };

typedef struct {
    int precision;       /* CFUST_PREC_FP64 (default), _FP32 or _MIXED */
    int qmc_points;      /* N: points of the rank-1 Korobov lattice for T_k, k >= 3 (default 1024) */
    int qmc_shifts;      /* M: random shifts of the lattice, 2..64 (default 8) */
    int qmc_korobov_a;   /* Korobov generator a: z_d = a^d mod N (default 119) */
    uint64_t seed;       /* key of the SplitMix64 shifts: shift(m,d) = u01(seed ^ (m+1)<<32 ^ (d+1)) */
    double nu_min;       /* bracket of the eq (22) root (default 1) */
    double nu_max;       /* (default 200) */
    int device;          /* CUDA device ordinal (default 0) */
    void* cuda_stream;   /* cudaStream_t to issue work on (default NULL) */
    int t2_nodes;        /* Gauss-Legendre nodes per piece of the T_2 quadrature, 8..64,
                            for every piece (0: 64 in FP64 mode; in the FP32 and mixed
                            modes 8 to 32 by the piece's length in units of the
                            integrand's widths where 4 <= dof <= 64 and |rho| < 0.9, 32
                            elsewhere; the T_1 inside each node is interpolated there from
                            a per-dof table built once per E-step) */
    int profile;         /* 1: time every kernel class with CUDA events on the context
                            stream (read with cfust_profile); 0 (default): off */
    int moments;         /* truncated-t moments of eqs (16)-(17) for q >= 3:
                            0 (default): exact recursion through T_{q-1} and T_{q-2};
                            1: ratio estimators E[X], E[X X^T] from the lattice pass of
                               alpha_s (eq 4), which also samples the last coordinate;
                               its points weighted by W/(nu+p) give alpha of eq (13)
                               and the moments at dof nu+p+2 (one integral per pair
                               instead of 2 + q + q(q-1)).
                            q <= 2 always uses the recursion. */
    int hold;            /* parameters the M-step keeps at their current values, a bitwise
                            OR of CFUST_HOLD_DELTA (eq 20 skipped; eq 21 then uses Delta^(k):
                            from Delta^(0) = 0 the fit is the EM of a mixture of multivariate
                            t, the Delta = 0 special case of Sec. 2) and CFUST_HOLD_NU (eq 22
                            skipped); 0 (default): none */
    int model;           /* CFUST_MODEL_CFUST (0, default): the CFUST mixture of eq (4);
                            CFUST_MODEL_CFUSN: its nu -> infinity limit, the CFUSN mixture
                            of eq (5) (density 2^q phi_p(y; mu, Omega) Phi_q(c; 0, Lambda),
                            u = 1, no nu step: nu is held and stored as +infinity) */
    int elogw;           /* E[log W | y] of the nu update (eq 22): CFUST_ELOGW_OSL (0,
                            default): the one-step-late form of eq (15);
                            CFUST_ELOGW_EXACT: the exact conditional expectation -- the
                            posterior of W given y is the Gamma((nu+p)/2, (nu+d)/2) law
                            tilted by Phi_q(sqrt(W) c; 0, Lambda), which the points of the
                            lattice pass of alpha_s sample with weight f, so E[log W | y] is
                            the f-weighted mean of log W over them (needs moments = 1,
                            q >= 3, the CFUST model; not with the learned surrogate) */
    int tensor_stats;    /* CFUST_PREC_MIXED: 1: the cross statistics Srr = sum tau u r r^T,
                            Sre = sum tau r e2^T and Sr = sum tau u r of eqs (18)-(21) as one
                            tcgen05 tensor-core contraction per block of observations (TF32
                            hi/lo split, FP32 accumulation per block, FP64 across blocks)
                            where g p <= 128 and g (p + q + 1) <= 256; 0 (default):
                            compensated FP32 sums on the CUDA cores.  Ignored by the other
                            precisions. */
} cfust_opts;

#define CFUST_ELOGW_OSL 0
#define CFUST_ELOGW_EXACT 1

#define CFUST_MODEL_CFUST 0
#define CFUST_MODEL_CFUSN 1

#define CFUST_HOLD_DELTA 1
#define CFUST_HOLD_NU 2

/* Kernel classes reported by cfust_profile. */
enum {
    CFUST_PROF_SETUP = 0,   /* per-component factors (defs under eq 4) */
    CFUST_PROF_CHI,         /* chi table of the lattice integrator */
    CFUST_PROF_PLAN,        /* whitening, log t_p, integral limits */
    CFUST_PROF_LEVEL0,      /* T_q of eqs (4) and (13) */
    CFUST_PROF_LEVEL1,      /* T_{q-1} of the truncated-t first moments */
    CFUST_PROF_LEVEL2,      /* T_{q-2} of the truncated-t second moments */
    CFUST_PROF_MOMENTS,     /* alpha with single-pass moments (opts.moments = 1) */
    CFUST_PROF_COMBINE,     /* eqs (4), (13), (15)-(17) from the integrals */
    CFUST_PROF_FIXUP,       /* FP64 re-evaluation of far-tail pairs (FP32 mode) */
    CFUST_PROF_REDUCE,      /* eqs (12), (27) and the tau-weighted statistics */
    CFUST_PROF_MSTEP,       /* eqs (18)-(22) */
    CFUST_PROF_SURROGATE,   /* the learned surrogate's inference (level-0 and moment records) */
    CFUST_NPROF
};

/* Caller-owned parameter buffers (host memory), sizes as above. */
typedef struct {
    double* pi;     /* g */
    double* mu;     /* g * p */
    double* Sigma;  /* g * p * p */
    double* Delta;  /* g * p * q */
    double* nu;     /* g */
} cfust_params;

/* Fill *opts with the defaults listed above. */
void cfust_default_opts(cfust_opts* opts);

/* Create a context for n observations of dimension p, q latent skewing
 * variables and g components (Sec. 2: p-variate CFUST with p x q Delta).
 * Limits: 1 <= p <= 32, 1 <= q <= 8, 1 <= g <= 16, 1 <= n < 2^31.
 * opts may be NULL (defaults).  Allocates every device buffer the E- and
 * M-steps need; *out receives the context or NULL on failure. */
cfust_status cfust_create(cfust_ctx** out, int p, int q, int g, int64_t n, const cfust_opts* opts);

/* Release a context and all its device memory.  NULL is accepted. */
cfust_status cfust_destroy(cfust_ctx* ctx);

/* Observations y_j (Sec. 2), row j at y + j*ld elements, p used per row.
 * dtype CFUST_F64 or CFUST_F32 (FP32 rows are widened to FP64 on the device).
 * on_device = 1: y is a device pointer on ctx's device (e.g. a torch
 * tensor's data_ptr), read on the context stream; 0: host memory, copied.
 * The data are copied; the caller keeps ownership of y. */
cfust_status cfust_set_data(cfust_ctx* ctx, const void* y, int dtype, int64_t ld, int on_device);

/* Copy Psi = (pi, mu, Sigma, Delta, nu) in (Sec. 2, eq (1)).  Returns
 * CFUST_EINVAL if a pi is not in (0, 1], a nu not in [nu_min, nu_max], or a
 * non-finite value is present (under CFUST_MODEL_CFUSN nu is not read and is
 * set to +inf). */
cfust_status cfust_set_params(cfust_ctx* ctx, const cfust_params* params);

/* Copy the current Psi out into caller buffers. */
cfust_status cfust_get_params(cfust_ctx* ctx, cfust_params* out);

/* One E-step at the current Psi^(k): eqs (4), (12)-(17) for every pair and
 * the tau-weighted sufficient statistics of eqs (18)-(22).  *loglik_out
 * (may be NULL) receives l(Psi^(k)) of eq (27), computed from the same
 * density pass (Sec. 4.3).  The statistics stay on the device for
 * cfust_mstep.  A pair whose T_q is 0 in the working precision is null:
 * log f = -inf, tau = 0, u = 1, E log w = 0, e2 = e3 = 0.  CFUST_ENAN when a
 * density or statistic is NaN or +inf, or l is not finite (an observation
 * whose every pair is null). */
cfust_status cfust_estep(cfust_ctx* ctx, double* loglik_out);

/* Copy the per-pair E-step arrays of the last cfust_estep to host buffers
 * (any pointer may be NULL).  Layout component-major, index h*n + j:
 * logf = log f_h(y_j) (eq 4); tau (eq 12); u (eq 13); elogu (eq 15);
 * eu (q per pair, eq 16); euu (q x q per pair, eq 17); se = standard error
 * of the lattice estimate of the T_q factor of eq (4) (0 when q <= 2). */
cfust_status cfust_get_pairs(cfust_ctx* ctx, double* logf, double* tau, double* u,
                             double* elogu, double* eu, double* euu, double* se);

/* Copy the reduced sufficient statistics of the last E-step, per component h
 * (stride 3 + p + q + p*q + q*q + p*p doubles): N = sum tau, U = sum tau u,
 * Snu = sum tau (elogu - u), Sr = sum tau u r (p), Se = sum tau eu (q),
 * Sre = sum tau r eu^T (p x q), See = sum tau euu (q x q),
 * Srr = sum tau u r r^T (p x p), with r = y_j - mu_h^(k). */
cfust_status cfust_get_stats(cfust_ctx* ctx, double* stats);

/* M-step (eqs 18-22, in the order pi, mu, Delta, Sigma, nu) from the
 * statistics of the last E-step; Psi^(k+1) replaces Psi^(k) on the device.
 * On CFUST_EEMPTY / CFUST_ENOTPD the parameters are left unchanged.
 * CFUST_ENUROOT is reported after the update, with nu clamped. */
cfust_status cfust_mstep(cfust_ctx* ctx);

/* Log-likelihood (eq 27) at the current Psi: a density-only pass (one T_q
 * per pair, no moments). */
cfust_status cfust_loglik(cfust_ctx* ctx, double* out);

/* EM fit from the current Psi (Sec. 3): iteration k runs the E-step at
 * Psi^(k) (giving l(Psi^(k)), Sec. 4.3) then the M-step.  With tol > 0 the
 * Aitken rule (eqs 24-26) stops after the E-step whose l satisfies it;
 * otherwise exactly max_iter M-steps run and one density pass gives
 * l(Psi^(max_iter)).  loglik_hist (may be NULL) receives iters+1 values
 * l(Psi^(0..iters)); *iters_out the number of M-steps run. */
cfust_status cfust_fit(cfust_ctx* ctx, int max_iter, double tol, int* iters_out,
                       double* loglik_hist);

/* Diagnostic: evaluates, on `device`, the FP32 normal CDF Phi (fn = 0) or its
 * inverse (fn = 1) exactly as the FP32 lattice integrators of T_k (k >= 3)
 * compute them, or the CUDA math library's normcdff (fn = 2) / normcdfinvf
 * (fn = 3) for comparison.  x and y are host arrays of count floats.  The
 * paper needs Phi and Phi^-1 only inside T_q (Sec. 3.1); it fixes no method. */
cfust_status cfust_special_f32(int fn, int64_t count, const float* x, float* y, int device);

/* Initial values by Algorithm 1 (Sec. 3.3): for each of nstarts partitions of the
 * observations and each alpha of the grid, the moment-based start of eq (23) per cluster
 * (cluster mean, covariance S with divisor n_h - 1 and its diagonal s*, the sign of the
 * third moment about the mean; delta = sign sqrt(pi (1 - alpha) s* / (pi - 2)) element-wise,
 * Sigma = S - (1 - alpha) diag(s*), mu = mean - sqrt(2/pi) delta, nu = nu0, pi_h = n_h/n;
 * Delta is diag(delta) for q = p, the column delta for q = 1, otherwise delta on its leading
 * diagonal) and its log-likelihood (eq 27, the density pass of cfust_loglik).  The first
 * candidate with the highest log-likelihood becomes the context's Psi.
 *   labels: host array nstarts x n of cluster labels in [0, g), or NULL for random
 *           partitions drawn on the device (label_j = floor(u g), u the SplitMix64 output
 *           for key seed ^ ((start + 1) << 40) ^ (j + 1));
 *   alphas: nalpha values in (0, 1), or NULL for 0.1, 0.2, ..., 0.9 (nalpha 0 or 9);
 *   loglik_out (nstarts x nalpha, may be NULL): each candidate's log-likelihood, -inf when
 *           a cluster has fewer than 2 points or Sigma^(0) is not positive definite;
 *   best_out (may be NULL): start * nalpha + alpha index of the chosen candidate.
 * Returns CFUST_ENOTPD (Psi unset) when no candidate is valid.  Needs cfust_set_data. */
cfust_status cfust_init(cfust_ctx* ctx, int nstarts, const int32_t* labels, uint64_t seed,
                        int nalpha, const double* alphas, double nu0, double* loglik_out,
                        int* best_out);

/* k-means partitions for Algorithm 1 (Sec. 3.3: the initial clusterings are typically
 * k-means or random), on the device, for cfust_init's labels.  For each of nstarts starts,
 * Lloyd's iteration from g distinct observations: centre h is observation floor(u n), u the
 * SplitMix64 output for key seed ^ ((start + 1) << 40) ^ (1 << 36) ^ (h + 1 + g a), with
 * a = 0, 1, ... until the index differs from those of centres 0..h-1.  Each iteration assigns
 * every observation to the nearest centre (squared Euclidean distance in FP64, products and
 * sums rounded one at a time, the first centre on ties) and stops when no label changes or
 * after max_iter assignments; otherwise each centre becomes its cluster's mean (an empty
 * cluster keeps its centre).  labels_out: host, nstarts x n; iters_out (nstarts, may be
 * NULL): assignments run; centres_out (nstarts x g x p, may be NULL): the centres of the
 * last assignment.  Needs cfust_set_data and n >= g. */
cfust_status cfust_kmeans(cfust_ctx* ctx, int nstarts, uint64_t seed, int max_iter, int32_t* labels_out,
                          int* iters_out, double* centres_out);

/* Autotuner of the integrators' launch shapes (not part of the paper).  Runs one
 * E-step at the current Psi, then times (CUDA events, best of reps runs after one
 * warm-up) each candidate shape of the context's integral records:
 *   - FP32 T_2 records of finite dof: 2, 4, 8 or 16 lanes per quadrature piece (a
 *     warp's pieces dealt to groups of that many lanes) or 32 (a warp per record)
 *     (ms[0..4]; -1 where the context has no such records);
 *   - the FP32 single-pass moment pass at q <= 4: 1 or 2 lattice points in flight
 *     per lane (ms[5..6]; -1 where not applicable);
 * and keeps the fastest (choices[0]: lanes per T_2 piece, choices[1]: points per
 * lane; 0 where not applicable).  The choice holds for this context and, for the rest
 * of the process, for every context (one not tuned itself) with records of the same
 * (kernel, dimension, precision), from its next E-step on (a fit graph of
 * cfust_fit_batch keeps the shapes it was captured with).  The lanes per T_2 piece
 * decide the order in which a record's nodes are added, so the choice is one per shape,
 * not per problem size: the shards of one problem stay bitwise equal to it.  Leaves no E-step
 * results (run cfust_estep before cfust_mstep).  Without tuning the shapes are 2 lanes
 * per T_2 piece and 2 points per lane.  choices (2) and ms (7) may be NULL. */
cfust_status cfust_autotune(cfust_ctx* ctx, int reps, int* choices, double* ms);

/* Flags of cfust_fit_batch. *//* Flags of cfust_fit_batch. *//* Flags of cfust_fit_batch. */
#define CFUST_FIT_NO_FINAL 1 /* skip the density pass that gives l(Psi^(max_iter)) */

/* Batched form of cfust_fit: nfits independent fits (different contexts,
 * any sizes) run concurrently on the device.  Each context's whole fit --
 * the loop of cfust_fit (Sec. 3; Aitken rule eqs 24-26; l from the E-step's
 * density pass, Sec. 4.3) -- is one CUDA graph whose loop control runs on
 * the device, so no host synchronisation happens between iterations; the
 * graph is built on first use and reused while (max_iter, tol, flags) stay
 * the same.  Results equal those of cfust_fit on the same context bit for
 * bit.  Outputs (each may be NULL): iters_out[i] = M-steps run by fit i;
 * loglik_hist[i*(max_iter+1) + k] = l(Psi^(k)) of fit i, NaN where not
 * reached; status_out[i] = the status cfust_fit would return (a failing fit
 * keeps its last good Psi and its message is in cfust_last_error(ctxs[i])).
 * Returns the first failing fit's status, or CFUST_OK.  Contexts must be
 * distinct, and no other call may use them until this one returns. */
cfust_status cfust_fit_batch(int nfits, cfust_ctx* const* ctxs, int max_iter, double tol,
                             int flags, int* iters_out, double* loglik_hist,
                             cfust_status* status_out);

/* ------------------------------------------------------------------------
 * Row-sharded E-step over several processes (one GPU each).  The paper's
 * parallel EM (Sec. 4) computes per-component partial results in threads and
 * collects them once per iteration (Sec. 4.3); here the observations are split
 * by rows instead, each process computes the sufficient statistics of its rows,
 * and one exchange per iteration gives every process the same sums, after which
 * each runs the identical M-step (eqs 18-22).
 *
 * The statistics are reduced in two fixed-order levels: sums over blocks of
 * observations, then sums of consecutive segments of SEG blocks, then the
 * segments in order.  A shard whose first row is a multiple of
 * cfust_rows_per_segment has exactly the segments the whole problem has over
 * those rows, so gathering every shard's segments in rank order and reducing
 * them reproduces the single-process statistics bit for bit.
 * ------------------------------------------------------------------------ */

/* Rows per segment for a problem of these sizes and precision (it does not
 * depend on n): shard boundaries must be multiples of it. */
cfust_status cfust_rows_per_segment(int p, int q, int g, int precision, int64_t* rows);

/* Segments of this context's rows (*nseg, may be NULL) and doubles per segment
 * (*width = g*(3+p+q+pq+q^2+p^2) + 1: the statistics of cfust_get_stats, then
 * the log-likelihood sum, may be NULL). */
cfust_status cfust_segment_count(cfust_ctx* ctx, int64_t* nseg, int* width);

/* Enqueue the E-step at the current Psi (eqs 4, 12-17) and the segment sums of
 * its statistics into seg: a device buffer of nseg_out x width doubles,
 * nseg_out >= the context's segment count; rows past that count are written
 * as 0 (padding to a common count per process).  Asynchronous on the context
 * stream: kernel errors surface in cfust_reduce_segments. */
cfust_status cfust_estep_segments(cfust_ctx* ctx, double* seg, int64_t nseg_out);

/* Reduce nseg segment rows (device, nseg x width; the gathered segments of all
 * processes in rank order, zero padding allowed) into the context's statistics
 * and log-likelihood, in order; *loglik_out (may be NULL) receives the total
 * l(Psi) of eq (27).  n_total: the observations of all shards together, the n
 * of eq (18) that the following cfust_mstep divides by (>= this context's n).
 * Synchronises; then cfust_mstep may follow.  CFUST_ENAN for a non-finite sum;
 * the per-component set-up checks as in cfust_estep. */
cfust_status cfust_reduce_segments(cfust_ctx* ctx, const double* seg, int64_t nseg, int64_t n_total,
                                   double* loglik_out);

/* Aitken's stopping rule (Sec. 3.4, eqs 24-26) on three consecutive
 * log-likelihoods: 1 when |l_inf^(k+1) - l^(k+1)| < tol (or l^k = l^(k-1)),
 * else 0.  The rule cfust_fit applies, for drivers that run the loop
 * themselves (the sharded fit). */
int cfust_aitken_converged(double l_km1, double l_k, double l_kp1, double tol);

/* Evaluate T_k(b; 0, V, nu) for `count` independent cases with the
 * library's device integrators (k <= 2 deterministic, k >= 3 lattice), host
 * buffers: b (count x k), V (count x k x k scale matrices), nu (count);
 * out (count), se (count, may be NULL).  Uses opts of ctx (precision,
 * lattice, seed); ctx may be created with any n >= 1. */
cfust_status cfust_tk_eval(cfust_ctx* ctx, int k, int count, const double* b, const double* V,
                           const double* nu, double* out, double* se);

/* Posterior weights, log-likelihood and tau-weighted sufficient statistics
 * (the reduction half of cfust_estep) from per-pair E-step arrays that the
 * caller already holds on the device, allocating nothing.  The paper has no
 * counterpart: it is an entry point for callers that cannot call cudaMalloc
 * -- code that owns all device memory through its own pool, or that must not
 * incur the device-wide synchronisation of cudaMalloc/cudaFree inside a
 * latency-critical loop.
 *
 * Every pointer is a device pointer on the current device; layouts as in
 * cfust_get_pairs (component-major h*n + j) and cfust_get_stats:
 *   y (n x p), pi (g), mu (g x p) at which r = y - mu is centred, logf, u,
 *   elogu (g*n), eu (g*n*q), euu (g*n*q*q) in;  tau (g*n, may be NULL) and
 *   stats (g*(3+p+q+pq+q^2+p^2) + 1 doubles: the per-component statistics,
 *   then the log-likelihood sum over observations) out.
 * Work is issued on cuda_stream (NULL = legacy default stream) and the call
 * returns after it completes.  Its only scratch, the per-block partial sums
 * and an error flag, lives in a fixed device array of 2^19 doubles (4 MiB)
 * that every GPU loading the library holds until exit: sizes needing more
 * than ceil(n/chunk) x (g*(3+p+q+pq+q^2+p^2)+1) <= 2^19 partial sums (chunk
 * <= 256 observations per block, fewer when p, q or g are large) are
 * rejected with CFUST_EINVAL.  Every call looks up the scratch's device
 * address in the current context (the address belongs to the context, so a
 * context created after cudaDeviceReset gets its own); the first call in a
 * context also loads the library's device code there, so make the first
 * call on each device before any stream capture.  The block size is chosen
 * without raising the default shared-memory limit, so the statistics equal
 * those of cfust_estep to rounding, not bit for bit.  All calls share the scratch and it
 * keeps the last call's contents: calls that overlap on the GPU (other
 * streams, other host threads) race and must be serialised by the caller.
 * Errors are reported through cfust_last_error(NULL). */
cfust_status cfust_reduce_stats_noalloc(int p, int q, int g, int64_t n, const double* y,
                                        const double* pi, const double* mu, const double* logf,
                                        const double* u, const double* elogu, const double* eu,
                                        const double* euu, double* tau, double* stats,
                                        void* cuda_stream);

/* ------------------------------------------------------------------------
 * Pipe rates (not part of the paper): the denominators of the E-step's
 * roofline.  The lattice integrators of T_k are bound by per-point arithmetic
 * (normal CDF and inverse on the MUFU and FMA pipes, FP32 FMAs), for which no
 * data-sheet figure states an achievable rate, so the library measures them
 * on the device it runs on.  All rates are whole-GPU operations per second.
 * ------------------------------------------------------------------------ */
typedef struct {
    double sm_mhz;        /* SM clock during the measurement: clock64() cycles / event time */
    double fp32_fma;      /* FP32 FMA per second (8 independent chains per thread) */
    double fp64_fma;      /* FP64 FMA per second */
    double mufu_ex2;      /* ex2.approx.ftz.f32 per second */
    double mufu_lg2;      /* lg2.approx.ftz.f32 per second */
    double mufu_rcp;      /* rcp.approx.ftz.f32 per second */
    double mix_points[9]; /* [K], K = 3..8: lattice points per second of the single-pass
                             integrand of dimension K alone -- K normal CDFs, K inverse
                             normal CDFs (the FP32 forms of the integrators), the
                             K(K-1)/2 + 3K FMAs of the chain and the 2 + K + K(K+1)/2
                             FMAs of the weighted moment sums per point, no memory
                             traffic; the best of 1, 2 and 4 independent points per
                             thread; [0..2] unused (0) */
    double t2_nodes;      /* nodes per second of the FP32 T_2 quadrature alone -- per node
                             two sines, the sin^(nu-1) weight (lg2, ex2) and the inner T_1
                             from its per-dof table -- the best of 1, 2 and 4 independent
                             nodes per thread */
} cfust_rates;

/* Run the microbenchmarks on `device` for about `seconds` (0 < seconds <= 5) in
 * all, on the legacy default stream, and fill *out.  Allocates one scratch
 * buffer (8 x SMs x 256 doubles and a 32 KB table) for the duration of the call.  Changes no
 * device setting (clocks are read, never set). */
cfust_status cfust_measure_rates(int device, double seconds, cfust_rates* out);

/* Last error message of ctx (or of the last failed cfust_create when ctx is
 * NULL).  Valid until the next call on the same context. */
const char* cfust_last_error(const cfust_ctx* ctx);

/* Number of kernels the library has launched on ctx since creation (for
 * launch accounting in benchmarks). */
int64_t cfust_launch_count(const cfust_ctx* ctx);

/* Diagnostic read-back of internal device buffers into host memory (at most
 * `bytes` bytes; *written receives the byte count copied).  what:
 *   0 per-component factor blocks (g x stride doubles, stride = *written/8/g),
 *   1 per-pair (d, log t_p), 2 per-pair c (q doubles),
 *   3-5 standardised limits of the level 0/1/2 integral records,
 *   6-8 values of the level 0/1/2 integral records,
 *   9 the kernel error flags (one int).
 * For tests that localise a mismatch to one pipeline stage. */
cfust_status cfust_debug_read(cfust_ctx* ctx, int what, void* dst, int64_t bytes, int64_t* written);

/* Accumulated device time (ms, CUDA events) and launch count of each kernel
 * class since creation or the last reset; arrays of CFUST_NPROF entries (either
 * may be NULL).  Requires opts.profile = 1 (else CFUST_ESTATE).  reset = 1
 * zeroes the totals after reading. */
cfust_status cfust_profile(cfust_ctx* ctx, double* ms, int64_t* launches, int reset);

/* Algorithmic work done by each kernel class since creation or the last
 * cfust_profile reset (units: CFUST_NPROF entries): lattice points (records x
 * N x M) for the lattice T_k classes (k >= 3: level 0-2 and the single-pass
 * moments), quadrature nodes for T_2 records (counted on the device), records
 * for T_1; 0 for the other classes and for records a surrogate selection list
 * sends to the lattice.  Requires opts.profile = 1 (else CFUST_ESTATE).  The
 * numerator of the integrators' roofline (see cfust_measure_rates). */
cfust_status cfust_profile_work(cfust_ctx* ctx, double* units);

/* ------------------------------------------------------------------------
 * Learned surrogate (not part of the paper).  A 3 x 256 tanh MLP with BF16
 * operands and FP32 accumulation maps one integral record of the
 * single-pass E-step -- features (b_1..b_q standardised limits, the
 * correlations R_ij, i > j, of Lambda in row-major order, 1/dof) -- to
 * log T_q (eq 4 at dof nu+p, eq 13 at nu+p+2) and the standardised
 * truncated moments of eqs (16)-(17) (E[X], then the lower triangle of
 * E[X X^T] row-major).  Features are standardised by training-set means
 * and deviations (stats: fmean, fstd, zlo, zhi [48 each], tmean, tstd
 * [48 each]); a record whose standardised feature leaves the training
 * range [zlo, zhi] widened by margin (in standard deviations) is left to
 * the lattice.
 * Parameter vector (CFUST_MLP_NPARAM floats): W1 [48 x 256], b1, W2
 * [256 x 256], b2, W3 [256 x 256], b3, W4 [256 x 48], b4, matrices
 * row-major with the input index first; inputs and outputs zero-padded to
 * 48.
 * ------------------------------------------------------------------------ */
#define CFUST_MLP_IN 48
#define CFUST_MLP_H 256
#define CFUST_MLP_OUT 48
#define CFUST_MLP_NPARAM 156464
#define CFUST_MLP_NSTAT 288

/* Device initialisation of a parameter vector: W ~ U(-1/sqrt(fan_in),
 * 1/sqrt(fan_in)) on the used rows of W1 (nin) and columns of W4 (nout),
 * element e drawn by SplitMix64 at key seed ^ (e + 1); padding and biases 0.
 * theta_out: host, CFUST_MLP_NPARAM floats. */
cfust_status cfust_mlp_init(uint64_t seed, int nin, int nout, float* theta_out, int device);

/* Forward and backward pass over rows x 48 standardised features f (host,
 * FP32; rounded to BF16 as the network's input), targets t and masks m (rows
 * x 48): loss = sum m (y - t)^2 / (2 rows nout).  grad_out (NPARAM), y_out
 * (rows x 48) and loss_out may be NULL.  rows <= 2^22.  Host buffers. */
cfust_status cfust_mlp_grad(const float* theta, int64_t rows, int nout, const float* f, const float* t,
                            const float* m, float* grad_out, float* y_out, double* loss_out, int device);

/* One Adam step (Kingma & Ba; beta1 0.9, beta2 0.999, eps 1e-8, step >= 1
 * counts this step) on host vectors theta, m, v (updated in place). */
cfust_status cfust_mlp_adam(float* theta, const float* grad, float* m, float* v, int64_t step, float lr,
                            int device);

/* The fused inference kernel on records given on the host: bt (rows x q),
 * Lc (rows x q x q, lower Cholesky factors of correlation matrices,
 * row-major), dof (rows).  logT (rows) and mom (rows x (q + q(q+1)/2), may be
 * NULL) receive the network's outputs for in-range records; inbox[i] = 0 (and
 * logT NaN) for a record outside the training range.  3 <= q <= 8. */
cfust_status cfust_mlp_records(const float* theta, const float* stats, float margin, int q, int64_t rows,
                               const double* bt, const double* Lc, const double* dof, double* logT,
                               double* mom, int* inbox, int device);

typedef struct {
    int epochs;                /* passes over samples_per_epoch samples (default 48) */
    int batch;                 /* minibatch rows (default 8192) */
    int64_t samples_per_epoch; /* at most (default 2^20); <= 0: every collected sample */
    float lr;                  /* Adam step size (default 3e-3) */
    float margin;              /* training-range margin in standard deviations (default 0.5) */
    uint64_t seed;             /* initial weights and shuffles */
} cfust_surrogate_opts;

cfust_surrogate_opts cfust_surrogate_default_opts(void);

/* Train the surrogate on the records of one lattice E-step at the current
 * Psi: runs cfust_estep with the lattice (its statistics and *loglik_out
 * stand, so cfust_mstep may follow), collects every record with T > 1e-300
 * (level 0 at dof nu+p: log T only; moment records at nu+p+2: log T and
 * moments), standardises, and trains.  The first call initialises the
 * weights and fixes the standardisation; later calls (at later iterates of a
 * fit) continue from the current weights and only widen the training range.  Then switches the surrogate on.  Requires
 * single-pass moments (moments = 1, q >= 3).  losses (opts.epochs entries,
 * may be NULL) receive each epoch's last minibatch loss. */
cfust_status cfust_surrogate_train(cfust_ctx* ctx, const cfust_surrogate_opts* opts, double* loglik_out,
                                   double* losses);

/* on = 1: E-steps and cfust_loglik take level-0 and moment records from the
 * network (out-of-range records from the lattice); 0: the lattice only. */
cfust_status cfust_surrogate_use(cfust_ctx* ctx, int on);

/* Records evaluated and records left to the lattice by the last E-step's
 * surrogate pass (both sets; in a full E-step a pair whose level-0 or moment
 * record leaves the training range has both records taken by the shared
 * lattice pass). */
cfust_status cfust_surrogate_info(cfust_ctx* ctx, int64_t* records, int64_t* fallbacks);

/* Copy the trained parameters (NPARAM floats) and statistics (NSTAT floats)
 * out (either may be NULL). */
cfust_status cfust_surrogate_params(cfust_ctx* ctx, float* theta, float* stats);

#ifdef __cplusplus
}
#endif
#endif
