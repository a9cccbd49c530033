// mstep.cu -- M-step solve (S11), one warp per component, FP64.
//
// From the statistics of estep_reduce (centred at mu^(k), r = y - mu^(k)):
//   eq (18)  pi = N / n
//   eq (19)  mu^(k+1) = mu^(k) + delta,  delta = (Sr - Delta^(k) Se) / U
//   eq (20)  Delta^(k+1) = A See^{-1},  A = sum tau (y - mu^(k+1)) e2^T = Sre - delta Se^T
//   eq (21)  Sigma^(k+1) = [Srr - Sr delta^T - delta Sr^T + U delta delta^T
//                            - Delta A^T - A Delta^T + Delta See Delta^T] / N
//            (with Delta = Delta^(k+1); sum tau e2 (y - mu)^T = A^T)
//   eq (22)  nu: root of N [log(nu/2) - psi(nu/2) + 1] + Snu = 0 (sum over j,
//            second term with +), safeguarded Newton on [nu_min, nu_max].
// Results go to separate output arrays; the host commits them only when no
// component failed (empty component, non-PD See or Sigma), so a failed
// M-step leaves Psi^(k) untouched.
#include "cfust.h"
#include "internal.cuh"
#include "special.cuh"

namespace {
__device__ bool chol_small(int n, const double* A, double* L)
{
    for (int j = 0; j < n; ++j) {
        double s = A[j * n + j];
        for (int k = 0; k < j; ++k) s -= L[j * n + k] * L[j * n + k];
        if (!(s > 0.0)) return false;
        L[j * n + j] = sqrt(s);
        for (int i = j + 1; i < n; ++i) {
            double t = A[i * n + j];
            for (int k = 0; k < j; ++k) t -= L[i * n + k] * L[j * n + k];
            L[i * n + j] = t / L[j * n + j];
        }
    }
    return true;
}

// digamma and trigamma at x > 0 together, by all 32 lanes of a warp: the recurrence terms
// 1/(x + i), i < k (k the steps that bring x + k to at least 12), one per lane and added by a
// butterfly (every lane ends with the same bits), then the asymptotic series at x + k (the
// expansions of cf_digamma and cf_trigamma)
__device__ void psi_pair_warp(double x, int lane, double& psi, double& tri)
{
    const int k = x < 12.0 ? (int)ceil(12.0 - x) : 0;
    double a = 0.0, b = 0.0;
    if (lane < k) {
        const double r = 1.0 / (x + lane);
        a = r;
        b = r * r;
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    const double y = x + k, r = 1.0 / y, r2 = r * r;
    psi = -a + log(y) - 0.5 * r - r2 * (1.0 / 12 + r2 * (-1.0 / 120 + r2 * (1.0 / 252 + r2 * (-1.0 / 240
                 + r2 * (1.0 / 132 + r2 * (-691.0 / 32760))))));
    tri = b + r * (1.0 + r * (0.5 + r * (1.0 / 6 + r2 * (-1.0 / 30 + r2 * (1.0 / 42
                 + r2 * (-1.0 / 30 + r2 * (5.0 / 66)))))));
}

// eq (22) at v and its derivative in v, by all lanes
__device__ double nu_eq_warp(double v, double N, double Snu, int lane, double* fp)
{
    double psi, tri;
    psi_pair_warp(0.5 * v, lane, psi, tri);
    if (fp) *fp = N * (1.0 / v - 0.5 * tri);
    return N * (log(0.5 * v) - psi + 1.0) + Snu;
}
}  // namespace

__global__ void __launch_bounds__(32) mstep_kernel(Dims D, const double* __restrict__ stats, double nu_min,
                                                   double nu_max, const double* __restrict__ mu,
                                                   const double* __restrict__ Delta, const double* __restrict__ nu,
                                                   double* pi_o, double* mu_o, double* Sigma_o, double* Delta_o,
                                                   double* nu_o, int* flags, int* comp_status, const int* gate,
                                                   int hold)
{
    // one warp per component (blockIdx.x); rows and matrix entries over the lanes, each
    // entry summed in the order of the serial definition
    __shared__ double delta[CF_MAXP], A[CF_MAXP * CF_MAXQ], Dn[CF_MAXP * CF_MAXQ];
    __shared__ double Bs[CF_MAXQ * CF_MAXQ], LB[CF_MAXQ * CF_MAXQ];
    __shared__ double Sn[CF_MAXP * CF_MAXP];
    __shared__ int fail;
    const int h = blockIdx.x, lane = threadIdx.x;
    if (h >= D.g) return;
    if (gate && *gate) return;  // a fit captured in a graph has already stopped
    const int p = D.p, q = D.q;
    const int S = stats_per_comp(p, q);
    const double* st = stats + (size_t)h * S;
    const double N = st[0], U = st[1], Snu = st[2];
    const double* Sr = st + 3;
    const double* Se = Sr + p;
    const double* Sre = Se + q;
    const double* See = Sre + p * q;
    const double* Srr = See + q * q;
    const double* muh = mu + (size_t)h * p;
    const double* Dh = Delta + (size_t)h * p * q;
    if (lane == 0) comp_status[h] = 0;
    if (!(N > 1e-12 * (double)D.n) || !(U > 0.0)) {
        if (lane == 0) {
            atomicOr(flags, KF_EMPTY);
            comp_status[h] = KF_EMPTY;
        }
        return;
    }
    for (int i = lane; i < p; i += 32) {
        double s = Sr[i];
        for (int k = 0; k < q; ++k) s -= Dh[i * q + k] * Se[k];
        delta[i] = s / U;
    }
    __syncwarp();
    for (int e = lane; e < p * q; e += 32) A[e] = Sre[e] - delta[e / q] * Se[e % q];
    for (int e = lane; e < q * q; e += 32) {
        const int a = e / q, b = e % q;
        Bs[e] = 0.5 * (See[a * q + b] + See[b * q + a]);
    }
    __syncwarp();
    const bool hold_delta = hold & CFUST_HOLD_DELTA;
    if (lane == 0) fail = (!hold_delta && !chol_small(q, Bs, LB)) ? 1 : 0;
    __syncwarp();
    if (fail) {
        if (lane == 0) {
            atomicOr(flags, KF_NOTPD_SEE);
            comp_status[h] = KF_NOTPD_SEE;
        }
        return;
    }
    // Delta = A See^{-1}: row i (lane i) solves See x = A_i^T; held: Delta^(k), which
    // eq (21) below then uses in place of Delta^(k+1)
    for (int i = lane; i < p; i += 32) {
        if (hold_delta) {
            for (int k = 0; k < q; ++k) Dn[i * q + k] = Dh[i * q + k];
            continue;
        }
        double zz[CF_MAXQ];
        for (int k = 0; k < q; ++k) {
            double s = A[i * q + k];
            for (int l = 0; l < k; ++l) s -= LB[k * q + l] * zz[l];
            zz[k] = s / LB[k * q + k];
        }
        for (int k = q - 1; k >= 0; --k) {
            double s = zz[k];
            for (int l = k + 1; l < q; ++l) s -= LB[l * q + k] * Dn[i * q + l];
            Dn[i * q + k] = s / LB[k * q + k];
        }
    }
    __syncwarp();
    // Sigma (eq 21), lower-triangle entries over the lanes
    for (int e = lane; e < p * p; e += 32) {
        const int i = e / p, l = e % p;
        if (l > i) continue;
        double s = Srr[i * p + l] - Sr[i] * delta[l] - delta[i] * Sr[l] + U * delta[i] * delta[l];
        for (int k = 0; k < q; ++k) s -= Dn[i * q + k] * A[l * q + k] + A[i * q + k] * Dn[l * q + k];
        for (int a = 0; a < q; ++a) {
            double t = 0.0;
            for (int b = 0; b < q; ++b) t += Bs[a * q + b] * Dn[l * q + b];
            s += Dn[i * q + a] * t;
        }
        Sn[i * p + l] = s / N;
        Sn[l * p + i] = s / N;
    }
    __syncwarp();
    // positive definiteness of Sigma: Cholesky, column j at step j, lane i >= j on row i
    // (the factor itself is not kept: L overwrites a copy in registers' place, W below)
    __shared__ double W[CF_MAXP * CF_MAXP];
    for (int e = lane; e < p * p; e += 32) W[e] = Sn[e];
    __syncwarp();
    for (int j = 0; j < p; ++j) {
        double t = 0.0;
        if (lane >= j && lane < p) {
            t = W[lane * p + j];
            for (int k = 0; k < j; ++k) t -= W[lane * p + k] * W[j * p + k];
        }
        const double sjj = __shfl_sync(0xffffffffu, t, j);
        if (!(sjj > 0.0)) {
            if (lane == 0) {
                atomicOr(flags, KF_NOTPD_SIGMA);
                comp_status[h] = KF_NOTPD_SIGMA;
            }
            return;
        }
        const double dj = sqrt(sjj);
        __syncwarp();
        if (lane == j) W[j * p + j] = dj;
        else if (lane > j && lane < p) W[lane * p + j] = t / dj;
        __syncwarp();
    }
    // nu (eq 22): F decreasing in nu; every lane runs the same safeguarded Newton (the values,
    // hence the branches, are the same in all lanes), lane 0 writes
    {
        double vnew;
        int st = 0;
        if (hold & CFUST_HOLD_NU) {
            vnew = nu[h];
        } else {
            const double flo = nu_eq_warp(nu_min, N, Snu, lane, nullptr);
            const double fhi = nu_eq_warp(nu_max, N, Snu, lane, nullptr);
            if (!(flo > 0.0)) { vnew = nu_min; st = KF_NUROOT; }
            else if (!(fhi < 0.0)) { vnew = nu_max; st = KF_NUROOT; }
            else {
                double lo = nu_min, hi = nu_max;
                double v = nu[h] > lo && nu[h] < hi ? nu[h] : 0.5 * (lo + hi);
                for (int it = 0; it < 200; ++it) {
                    double fp;
                    const double f = nu_eq_warp(v, N, Snu, lane, &fp);
                    if (f > 0.0) lo = v; else hi = v;
                    double vn = v - f / fp;
                    if (!(vn > lo && vn < hi)) vn = 0.5 * (lo + hi);
                    const bool done = fabs(vn - v) <= 1e-14 * v || hi - lo <= 1e-14 * hi;
                    v = vn;
                    if (done) break;
                }
                vnew = v;
            }
        }
        if (lane == 0) {
            if (st) { atomicOr(flags, st); comp_status[h] = st; }
            pi_o[h] = N / (double)D.n;
            nu_o[h] = vnew;
        }
    }
    for (int i = lane; i < p; i += 32) mu_o[(size_t)h * p + i] = muh[i] + delta[i];
    for (int i = lane; i < p * q; i += 32) Delta_o[(size_t)h * p * q + i] = Dn[i];
    for (int i = lane; i < p * p; i += 32) Sigma_o[(size_t)h * p * p + i] = Sn[i];
}
