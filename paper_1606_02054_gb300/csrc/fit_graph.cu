// fit_graph.cu -- device-side control of a whole EM fit captured in one CUDA graph.
//
// The graph (built in api.cu) is
//   init -> WHILE(cond) { E-step kernels -> fit_gate -> M-step (gated) -> fit_commit }
//        -> final_gate -> IF(final) { density-only pass -> fit_final }
// and reproduces the host loop of cfust_fit exactly: iteration k runs the
// E-step at Psi^(k) (giving l(Psi^(k)), Sec. 4.3), applies the Aitken rule of
// eqs (24)-(26) from iteration 2 on, and otherwise commits the M-step of
// eqs (18)-(22) unless a component failed.  After max_iter iterations one
// density pass gives l(Psi^(max_iter)).  The loop condition is set only by
// fit_commit_kernel, which clears it at max_iter at the latest, so the WHILE
// node always ends.
#include "internal.cuh"
#include "cfust.h"

__global__ void fit_init_kernel(FitState* s, int max_iter)
{
    if (threadIdx.x || blockIdx.x) return;
    s->it = 0;
    s->done = max_iter <= 0;
    s->converged = 0;
    s->status = CFUST_OK;
    s->comp = -1;
    s->nuroot = 0;
    s->final_pass = max_iter <= 0;
    s->pad = 0;
}

static __device__ int flag_status(int f, double L)
{
    if (f & (KF_NOTPD_OMEGA | KF_NOTPD_LAMBDA)) return CFUST_ENOTPD;
    if (f & KF_NAN) return CFUST_ENAN;
    if (!isfinite(L)) return CFUST_ENAN;
    return CFUST_OK;
}

// After the E-step of iteration s->it: record l(Psi^(it)) and apply the
// Aitken rule (eqs 24-26; equal consecutive values count as converged).
__global__ void fit_gate_kernel(FitState* s, const double* ll, const int* flags, double* hist,
                                double tol)
{
    if (threadIdx.x || blockIdx.x) return;
    if (s->done) return;
    const double L = *ll;
    const int st = flag_status(*flags, L);
    if (st != CFUST_OK) {
        s->status = st;
        s->done = 1;
        return;
    }
    const int it = s->it;
    hist[it] = L;
    if (tol > 0.0 && it >= 2) {
        const double den = hist[it - 1] - hist[it - 2];
        if (den == 0.0) {
            s->converged = 1;
            s->done = 1;
            return;
        }
        const double acc = (L - hist[it - 1]) / den;
        const double linf = hist[it - 1] + (L - hist[it - 1]) / (1.0 - acc);
        if (fabs(linf - L) < tol) {
            s->converged = 1;
            s->done = 1;
        }
    }
}

// After the M-step: commit Psi^(k+1) when no component failed (an empty
// component or a non-PD See / Sigma leaves Psi^(k) in place and stops the
// fit), count the iteration, and set the loop condition.
__global__ void fit_commit_kernel(Dims D, FitState* s, const int* flags, const int* comp,
                                  const double* pi_n, const double* mu_n, const double* Sigma_n,
                                  const double* Delta_n, const double* nu_n, double* pi, double* mu,
                                  double* Sigma, double* Delta, double* nu, int max_iter,
                                  cudaGraphConditionalHandle cond)
{
    __shared__ int ok;
    if (threadIdx.x == 0) {
        ok = 0;
        if (!s->done) {
            const int f = *flags;
            int st = CFUST_OK, bit = 0;
            if (f & KF_EMPTY) { st = CFUST_EEMPTY; bit = KF_EMPTY; }
            else if (f & KF_NOTPD_SEE) { st = CFUST_ENOTPD; bit = KF_NOTPD_SEE; }
            else if (f & KF_NOTPD_SIGMA) { st = CFUST_ENOTPD; bit = KF_NOTPD_SIGMA; }
            if (st != CFUST_OK) {
                int first = -1;
                for (int h = D.g - 1; h >= 0; --h)
                    if (comp[h] & bit) first = h;
                s->status = st;
                s->comp = first;
                s->done = 1;
            } else {
                ok = 1;
                if (f & KF_NUROOT) s->nuroot++;
            }
        }
    }
    __syncthreads();
    if (ok) {
        const int p = D.p, q = D.q, g = D.g;
        for (int t = threadIdx.x; t < g; t += blockDim.x) { pi[t] = pi_n[t]; nu[t] = nu_n[t]; }
        for (int t = threadIdx.x; t < g * p; t += blockDim.x) mu[t] = mu_n[t];
        for (int t = threadIdx.x; t < g * p * p; t += blockDim.x) Sigma[t] = Sigma_n[t];
        for (int t = threadIdx.x; t < g * p * q; t += blockDim.x) Delta[t] = Delta_n[t];
    }
    if (threadIdx.x == 0) {
        if (ok) {
            s->it += 1;
            if (s->it >= max_iter) {
                s->done = 1;
                s->final_pass = 1;
            }
        }
        cudaGraphSetConditional(cond, s->done ? 0u : 1u);
    }
}

__global__ void fit_final_gate_kernel(const FitState* s, cudaGraphConditionalHandle cond)
{
    if (threadIdx.x || blockIdx.x) return;
    cudaGraphSetConditional(cond, s->final_pass ? 1u : 0u);
}

// After the density-only pass: l(Psi^(max_iter)) into hist[max_iter].
__global__ void fit_final_kernel(FitState* s, const double* ll, const int* flags, double* hist,
                                 int max_iter)
{
    if (threadIdx.x || blockIdx.x) return;
    const double L = *ll;
    const int st = flag_status(*flags, L);
    if (st != CFUST_OK) s->status = st;
    else hist[max_iter] = L;
    s->it = max_iter;
}
