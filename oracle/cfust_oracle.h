/*
 * cfust_oracle.h -- plain FP64 CPU oracle for the FM-CFUST EM algorithm.
 *
 * TEST INFRASTRUCTURE ONLY.  This oracle exists to check the CUDA library.
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * load it.  It shares no code, header, table or constant with the CUDA path:
 * the only things both sides see are the seeded synthetic inputs and the
 * published definitions (SplitMix64, rank-1 Korobov lattices) that each
 * side implements on its own.
 *
 * Paper: Lee, Leemaqz & McLachlan, "A simple multithreaded implementation
 * of the EM algorithm for mixture models" (arXiv:1606.02054).
 *   Sec. 2, eqs (1)-(4): mixture and CFUST component density.
 *   Sec. 3.1, eqs (12)-(17): E-step conditional expectations.
 *   Sec. 3.2, eqs (18)-(22): M-step updates.
 *   Sec. 3.3, eq (23), Algorithm 1: initialisation.
 *   Sec. 3.4, eqs (24)-(26): Aitken stopping rule.
 *   Sec. 4.3, eq (27): log-likelihood.
 *
 * Layouts (all row-major, FP64):
 *   y      n x p            observations
 *   pi     g                mixing proportions
 *   mu     g x p            locations
 *   Sigma  g x p x p        scale matrices
 *   Delta  g x p x q        skewness matrices
 *   nu     g                degrees of freedom
 *   per-pair outputs are component-major: X[h*n + j] (eu: [h][j][q],
 *   euu: [h][j][q][q]).
 */
#ifndef CFUST_ORACLE_H
#define CFUST_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Randomised rank-1 lattice rule used for every T_k with k >= 3.
 * Points: x_{i,m,d} = frac(((i * z_d) mod N)/N + shift_{m,d}), z_d = a^d mod N,
 * then the baker's (tent) transform w = 1 - |2x - 1|. */
typedef struct {
    int npoints;        /* N (power of two not required) */
    int nshifts;        /* M */
    int korobov_a;      /* Korobov generator a */
    uint64_t seed;      /* SplitMix64 key for the random shifts */
    int moments;        /* 0: truncated-t moments by the T_{q-1}/T_{q-2} recursion;
                           1 (q >= 3): ratio estimators from the lattice pass of alpha */
    int elogw;          /* E[log W | y] of the nu update: 0: the one-step-late form of eq (15);
                           1 (moments = 1, q >= 3): exact, the ratio estimator of log W over the
                           points of the pass of alpha_s (the posterior of W given y is the
                           Gamma((nu+p)/2, (nu+d)/2) law tilted by Phi_q(sqrt(W) c; 0, Lambda)) */
} ora_qmc;

/* ---- special functions (exposed for the pin tests) ---- */
double ora_digamma(double x);
double ora_phi(double x);                 /* standard normal CDF */
double ora_phi_inv(double p);             /* its inverse */
double ora_incbeta(double a, double b, double x);   /* regularised I_x(a,b) */
double ora_incgamma_p(double a, double x);          /* regularised P(a,x) */
double ora_chi2_quantile(double w, double wc, double nu);  /* P(nu/2,x/2)=w; wc = 1-w */
double ora_t1pdf(double x, double nu);    /* univariate standard t density */
double ora_t1cdf(double x, double nu);    /* T_1(x; nu) */
double ora_t2cdf(double h, double k, double rho, double nu);  /* standard bivariate T_2 */
double ora_phi2(double h, double k, double rho);              /* standard bivariate normal CDF */
/* nu = +infinity anywhere (T_1, T_2, T_k, the density and the E-step) selects the normal limit:
 * the CFUSN model of eq (5) for the E-step; fit it with ORA_HOLD_NU. */
double ora_splitmix64_u01(uint64_t key);  /* one SplitMix64 output as a double in [0,1) */
double ora_qmc_shift(const ora_qmc* qmc, int m, int d);
/* T_k(b; 0, V, nu) for any k (k<=2 deterministic, k>=3 lattice QMC).
 * V is k x k row-major.  *se receives the QMC standard error (0 for k<=2). */
double ora_tkcdf(int k, const double* b, const double* V, double nu,
                 const ora_qmc* qmc, double* se);

/* Truncated moments of X ~ t_k(0, V, nu) given X <= b by ratio estimators
 * on the lattice (dimension k + 1: the last coordinate is sampled too):
 * alpha = T_k(b; 0, V, nu), m1 = E[X | X <= b] (k), m2 = E[X X^T | X <= b]
 * (k x k).  Returns alpha. */
/* The single-pass pass of alpha_s (dof k1 = nu + p, limits c sqrt(k1/nud), nud = nu + d) with
 * points weighted by W/k1: returns alpha = T_k at dof k1 + 2 of c sqrt((k1+2)/nud), and the
 * moments of X ~ t_k(0, (nud/(k1+2)) Lam, k1 + 2) truncated to X <= c. */
double ora_tk_joint(int k, const double* c, const double* Lam, double nud, double k1, const ora_qmc* qmc,
                    double* m1, double* m2);
double ora_tk_moments(int k, const double* b, const double* V, double nu, const ora_qmc* qmc,
                      double* m1, double* m2);

/* ---- E-step for one (observation, component) pair ----
 * Inputs are one component's parameters.  Outputs: log f_h(y) (eq 4),
 * u (eq 13), elogu (eq 15), eu (eq 16, q), euu (eq 17, q x q),
 * se_alpha_s = QMC standard error of the T_q factor of eq 4. */
int ora_pair(int p, int q, const double* y, const double* mu,
             const double* Sigma, const double* Delta, double nu,
             const ora_qmc* qmc, double* logf, double* u, double* elogu,
             double* eu, double* euu, double* se_alpha_s);

/* ---- full E-step over all pairs (eqs 12-17, 27) ----
 * Any of the per-pair output pointers may be NULL.  Returns 0 on success. */
int ora_estep(int n, int p, int q, int g, const double* y,
              const double* pi, const double* mu, const double* Sigma,
              const double* Delta, const double* nu, const ora_qmc* qmc,
              int nthreads, double* logf, double* tau, double* u,
              double* elogu, double* eu, double* euu, double* se,
              double* loglik);

/* Density-only pass: log-likelihood (eq 27) at the given parameters. */
int ora_loglik(int n, int p, int q, int g, const double* y,
               const double* pi, const double* mu, const double* Sigma,
               const double* Delta, const double* nu, const ora_qmc* qmc,
               int nthreads, double* loglik);

/* ---- M-step (eqs 18-22) from per-pair E-step arrays ----
 * Parameters are updated in place.  nu is found in [nu_min, nu_max];
 * nu_flag[h] = -1/+1 if clamped at the lower/upper bound, else 0.
 * Returns 0, or 1 + h for the first component whose update failed. */
int ora_mstep(int n, int p, int q, int g, const double* y,
              const double* tau, const double* u, const double* elogu,
              const double* eu, const double* euu, double nu_min,
              double nu_max, double* pi, double* mu, double* Sigma,
              double* Delta, double* nu, int* nu_flag);

/* The same M-step with parameters held at their current values: hold is a
 * bitwise OR of ORA_HOLD_DELTA (eq 20 skipped, eq 21 uses Delta^(k); from
 * Delta^(0) = 0 this is the EM of a t mixture) and ORA_HOLD_NU (eq 22 skipped). */
#define ORA_HOLD_DELTA 1
#define ORA_HOLD_NU 2
int ora_mstep_hold(int n, int p, int q, int g, const double* y, const double* tau,
                   const double* u, const double* elogu, const double* eu, const double* euu,
                   double nu_min, double nu_max, double* pi, double* mu, double* Sigma,
                   double* Delta, double* nu, int* nu_flag, int hold);

/* Root of eq (22) (sign read as + and sum over j) for one component:
 * n_h [log(nu/2) - psi(nu/2) + 1] + s_h = 0 on [nu_min, nu_max]. */
double ora_nu_root(double n_h, double s_h, double nu_min, double nu_max,
                   int* flag);

/* ---- EM fit: iters iterations (tol > 0 enables the Aitken rule) ----
 * loglik_hist[k] = l(Psi^(k)) for k = 0..iters_done (iters_done+1 values).
 * Returns 0 on success. */
int ora_fit(int n, int p, int q, int g, const double* y, double* pi,
            double* mu, double* Sigma, double* Delta, double* nu,
            const ora_qmc* qmc, int max_iter, double tol, double nu_min,
            double nu_max, int nthreads, int* iters_done,
            double* loglik_hist);

/* ---- Initialisation (Sec. 3.3, Algorithm 1, eq 23) ----
 * Random partition of start s: label_j = floor(u g), u = SplitMix64 output for the key
 * seed ^ ((s+1) << 40) ^ (j+1). */
void ora_random_partition(int n, int g, uint64_t seed, int start, int* labels);
/* k-means partitions for Algorithm 1 (Sec. 3.3: the initial clusterings are typically
 * k-means or random).  Lloyd's iteration from g distinct observations chosen by SplitMix64:
 * centre h of start s is observation floor(u n), u = u01(seed ^ ((s+1) << 40) ^ (1 << 36) ^
 * (h + 1 + g a)), a = 0, 1, ... until the index differs from those of centres 0..h-1.  Each
 * iteration assigns every observation to the nearest centre (squared Euclidean distance,
 * the first centre on ties); it stops when an assignment changes no label or after max_iter
 * assignments, otherwise the centres become the cluster means (an empty cluster keeps its
 * centre).  labels (nstarts x n), iters (nstarts, assignments run) and centres (nstarts x
 * g x p, those of the last assignment; may be NULL).  Returns 0, or 1 if n < g. */
int ora_kmeans(int n, int p, int g, const double* y, int nstarts, uint64_t seed, int max_iter,
               int* labels, int* iters, double* centres);
/* Eq (23) per cluster of a partition (sample covariance with divisor n_h - 1, third moment
 * about the mean for the sign of delta, nu = nu0, pi = n_h/n).  Returns 0, or 1 + h for the
 * first cluster with fewer than 2 points or a non-PD Sigma^(0). */
int ora_moment_start(int n, int p, int q, int g, const double* y, const int* labels,
                     double alpha, double nu0, double* pi, double* mu, double* Sigma,
                     double* Delta, double* nu);
/* Algorithm 1: for each start (labels: nstarts x n, or NULL for random partitions from seed)
 * and each alpha, the moment start and its log-likelihood (eq 27); the first candidate with
 * the highest l is returned (l is updated as candidates improve).  loglik_out (nstarts x
 * nalpha, may be NULL) gets -inf for invalid candidates; *best = s*nalpha + a or -1.
 * Returns 0, or 1 when no candidate is valid. */
int ora_init(int n, int p, int q, int g, const double* y, int nstarts, const int* labels,
             uint64_t seed, int nalpha, const double* alphas, double nu0, const ora_qmc* qmc,
             int nthreads, double* loglik_out, int* best, double* pi, double* mu,
             double* Sigma, double* Delta, double* nu);

/* ora_fit with the M-step's held parameters (see ora_mstep_hold). */
int ora_fit_hold(int n, int p, int q, int g, const double* y, double* pi,
                 double* mu, double* Sigma, double* Delta, double* nu,
                 const ora_qmc* qmc, int max_iter, double tol, double nu_min,
                 double nu_max, int nthreads, int* iters_done,
                 double* loglik_hist, int hold);

/* Aitken rule (eqs 24-26) on three consecutive log-likelihoods. */
int ora_aitken_converged(double l_km1, double l_k, double l_kp1, double eps,
                         double* l_inf);

#ifdef __cplusplus
}
#endif
#endif
