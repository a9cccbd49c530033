// reduce.cu -- posterior weights, log-likelihood and the tau-weighted
// sufficient statistics of the M-step, FP64, deterministic (no atomics).
//
// S8: tau_hj = pi_h f_h(y_j) / sum_h' pi_h' f_h'(y_j)   (eq 12, log-sum-exp)
//     l_j = log sum_h pi_h f_h(y_j)                     (eq 27; Sec. 4.3: the
//     same density pass gives l(Psi^(k)) and tau^(k))
// S9: per block of observations, per component h, with r = y_j - mu_h^(k):
//     N = sum tau, U = sum tau u, Snu = sum tau (elogu - u),
//     Sr = sum tau u r, Se = sum tau eu, Sre = sum tau r eu^T,
//     See = sum tau euu, Srr = sum tau u r r^T
//     (eqs 18-22 written as sums; centring at mu_h^(k) avoids cancellation).
// S10: fixed-order sum of the block partials.
#include "internal.cuh"



// Staged FP64 row of one observation for component h:
//   [0] tau, [1] tau*u, [2] elogu - u, [3] 1, [4..4+p) r, then eu (q), euu (q*q).
// Each statistic is the sum over the chunk of row[ia]*row[ib]*row[ic] (the FP32 rows:
// stat_operands_w below).  The
// symmetric See and Srr are computed for their lower triangles only
// (stats_reduced(p, q) statistics) and written to both positions o1, o2 of the
// full layout (o2 = -1 when there is one).
__device__ inline int stats_reduced(int p, int q)
{
    return 3 + p + q + p * q + q * (q + 1) / 2 + p * (p + 1) / 2;
}

__device__ inline void stat_operands(int e, int p, int q, int& ia, int& ib, int& ic, int& o1, int& o2)
{
    const int R0 = 4, E0 = 4 + p, EE0 = 4 + p + q;
    const int fSee = 3 + p + q + p * q, fSrr = fSee + q * q;
    o2 = -1;
    if (e == 0) { ia = 0; ib = 3; ic = 3; o1 = 0; return; }                   // N
    if (e == 1) { ia = 1; ib = 3; ic = 3; o1 = 1; return; }                   // U
    if (e == 2) { ia = 0; ib = 2; ic = 3; o1 = 2; return; }                   // Snu
    o1 = e;
    e -= 3;
    if (e < p) { ia = 1; ib = R0 + e; ic = 3; return; }                       // Sr
    e -= p;
    if (e < q) { ia = 0; ib = E0 + e; ic = 3; return; }                       // Se
    e -= q;
    if (e < p * q) { ia = 0; ib = R0 + e / q; ic = E0 + e % q; return; }      // Sre
    e -= p * q;
    int a = 0;
    if (e < q * (q + 1) / 2) {                                                // See (lower)
        while ((a + 1) * (a + 2) / 2 <= e) ++a;
        const int b = e - a * (a + 1) / 2;
        ia = 0; ib = EE0 + a * q + b; ic = 3;
        o1 = fSee + a * q + b;
        if (a != b) o2 = fSee + b * q + a;
        return;
    }
    e -= q * (q + 1) / 2;
    while ((a + 1) * (a + 2) / 2 <= e) ++a;                                   // Srr (lower)
    const int b = e - a * (a + 1) / 2;
    ia = 1; ib = R0 + a; ic = R0 + b;
    o1 = fSrr + a * p + b;
    if (a != b) o2 = fSrr + b * p + a;
}

// The FP32 rows hold the weighted vectors too: [0] tau, [1] tau u, [2] tau (elogu - u),
// [3] 1, then r (p), tau u r (p), tau eu (q), tau euu (q*q), so that every statistic is the
// sum over the chunk of row[ia] * row[ib] (two operands instead of three).
__device__ inline void stat_operands_w(int e, int p, int q, int& ia, int& ib, int& o1, int& o2)
{
    const int R0 = 4, WR0 = 4 + p, E0 = 4 + 2 * p, EE0 = 4 + 2 * p + q;
    const int fSee = 3 + p + q + p * q, fSrr = fSee + q * q;
    o2 = -1;
    ib = 3;
    if (e < 3) { ia = e; o1 = e; return; }                                       // N, U, Snu
    o1 = e;
    e -= 3;
    if (e < p) { ia = WR0 + e; return; }                                         // Sr
    e -= p;
    if (e < q) { ia = E0 + e; return; }                                          // Se
    e -= q;
    if (e < p * q) { ia = R0 + e / q; ib = E0 + e % q; return; }                 // Sre
    e -= p * q;
    int a = 0;
    if (e < q * (q + 1) / 2) {                                                   // See (lower)
        while ((a + 1) * (a + 2) / 2 <= e) ++a;
        const int b = e - a * (a + 1) / 2;
        ia = EE0 + a * q + b;
        o1 = fSee + a * q + b;
        if (a != b) o2 = fSee + b * q + a;
        return;
    }
    e -= q * (q + 1) / 2;
    while ((a + 1) * (a + 2) / 2 <= e) ++a;                                      // Srr (lower)
    const int b = e - a * (a + 1) / 2;
    ia = WR0 + a; ib = R0 + b;
    o1 = fSrr + a * p + b;
    if (a != b) o2 = fSrr + b * p + a;
}

// T = double: FP64 rows and sums.  T = float (mixed precision): FP32 rows
// (centred observations from the FP32 copy of y), compensated FP32 sums per
// block, FP32 exponentials of the log-sum-exp; the log-sum-exp's terms, l_j and
// the block partials stay FP64.
// PF (mixed form, p = P a multiple of 4 and q = Q = 2 known at compile time, pair rows
// present, full statistics): the observation's FP32 row is read once into registers for all
// components, and the next component's pair row is loaded while the current one's sums run.
// The staged values are the same operations in the same order either way.
template <typename T, int P = 0, int Q = 0>
__device__ void estep_reduce_body(const ReduceArgs& a, T* rows)
{
    constexpr bool PF = sizeof(T) == sizeof(float) && P > 0 && P % 4 == 0 && Q == 2;
    constexpr int PW = 2 + Q + Q * Q;  // FP32 pair-row width at q = Q
    const int p = P > 0 ? P : a.D.p, q = Q > 0 ? Q : a.D.q, g = a.D.g;
    const long long n = a.D.n;
    const int S = stats_per_comp(p, q);
    const long long j0 = (long long)blockIdx.x * a.chunk;
    const int cnt = (int)((n - j0) < a.chunk ? (n - j0) : a.chunk);
    // chunk is a multiple of 32, so the FP32 rows end on an 8-byte boundary
    T* taus = rows + (size_t)a.chunk * a.row;  // in the row type: the rows hold tau as T anyway
    double* lj = (double*)(taus + (size_t)g * a.chunk);
    double* lpi = lj + a.chunk;  // log pi_h (CF_MAXG slots)
    double* out = a.partial + (size_t)blockIdx.x * (g * S + 1);
    const int t = threadIdx.x;

    // FP32 rows: mu^(k) converted once per block, not once per staged row
    __shared__ float mu32[sizeof(T) == sizeof(float) ? CF_MAXG * CF_MAXP : 1];
    if (sizeof(T) == sizeof(float))
        for (int e = t; e < g * p; e += blockDim.x) mu32[e] = (float)a.mu[e];

    // S8: tau and l_j for this chunk (log-sum-exp about the largest term, one exp per component)
    if (t < g) lpi[t] = log(a.pi[t]);
    __syncthreads();
    if (t < cnt) {
        const long long j = j0 + t;
        double v[CF_MAXG];
        double mx = -INFINITY;
#pragma unroll
        for (int h = 0; h < CF_MAXG; ++h) {
            if (h < g) {
                v[h] = lpi[h] + a.logf[(size_t)h * n + j];
                mx = v[h] > mx ? v[h] : mx;
            }
        }
        if (sizeof(T) == sizeof(float)) {
            // FP32 rows: each term's distance from the largest one is formed in FP64 and
            // rounded once, the exponentials, their sum (between 1 and g), its logarithm and
            // the quotients are FP32: tau to a few ulp of FP32, l_j = max + log s to ~1e-7
            // absolute, the largest term itself exact
            float e[CF_MAXG];
            float s = 0.0f;
#pragma unroll
            for (int h = 0; h < CF_MAXG; ++h) {
                if (h < g) {
                    e[h] = expf((float)(v[h] - mx));
                    s += e[h];
                }
            }
            lj[t] = mx + (double)logf(s);
            const float rs = 1.0f / s;
#pragma unroll
            for (int h = 0; h < CF_MAXG; ++h) {
                if (h < g) {
                    const float tv = e[h] * rs;
                    taus[h * a.chunk + t] = (T)tv;
                    if (a.tau) a.tau[(size_t)h * n + j] = (double)tv;
                }
            }
        } else {
            double s = 0.0;
#pragma unroll
            for (int h = 0; h < CF_MAXG; ++h) {
                if (h < g) {
                    v[h] = exp(v[h] - mx);
                    s += v[h];
                }
            }
            lj[t] = mx + log(s);
            const double rs = 1.0 / s;
#pragma unroll
            for (int h = 0; h < CF_MAXG; ++h) {
                if (h < g) {
                    const double tv = v[h] * rs;
                    taus[h * a.chunk + t] = (T)tv;
                    if (a.tau) a.tau[(size_t)h * n + j] = tv;
                }
            }
        }
    } else if (t < a.chunk) {
        lj[t] = 0.0;
    }
    __syncthreads();
    // partial log-likelihood: fixed-order tree over the chunk
    for (int w = 1; w < a.chunk; w <<= 1) {
        if ((t % (2 * w)) == 0 && t + w < a.chunk) lj[t] += lj[t + w];
        __syncthreads();
    }
    if (t == 0) out[g * S] = lj[0];
    __syncthreads();

    float yr[PF ? P : 1], pc[PF ? PW : 1];
    if constexpr (PF) {
        if (t < cnt) {
#pragma unroll
            for (int i = 0; i < P; i += 4) {
                const float4 v = *reinterpret_cast<const float4*>(a.y32 + (size_t)(j0 + t) * P + i);
                yr[i] = v.x; yr[i + 1] = v.y; yr[i + 2] = v.z; yr[i + 3] = v.w;
            }
            const float4* src = reinterpret_cast<const float4*>(a.pr32 + (size_t)(j0 + t) * PW);
#pragma unroll
            for (int k = 0; k < PW / 4; ++k) {
                const float4 v = src[k];
                pc[4 * k] = v.x; pc[4 * k + 1] = v.y; pc[4 * k + 2] = v.z; pc[4 * k + 3] = v.w;
            }
        }
    }

    // S9: statistics, one component at a time
    for (int h = 0; h < g; ++h) {
        if (t < a.chunk) {
            T* rw = rows + (size_t)t * a.row;
            if (PF && t < cnt) {
                const T tv = taus[h * a.chunk + t];
                rw[0] = tv;
                rw[1] = tv * pc[0];
                rw[2] = tv * (pc[1] - pc[0]);
                rw[3] = T(1);
#pragma unroll
                for (int i = 0; i < (PF ? P : 1); ++i) {
                    const T ri = yr[i] - mu32[h * p + i];
                    rw[4 + i] = ri;
                    rw[4 + p + i] = rw[1] * ri;
                }
#pragma unroll
                for (int k = 0; k < (PF ? Q + Q * Q : 1); ++k) rw[4 + 2 * p + k] = rw[0] * pc[2 + k];
            } else if (t < cnt) {
                const size_t pid = (size_t)h * n + j0 + t;
                const float* pr = a.pr32 ? a.pr32 + pid * pr32_width(q) : nullptr;
                if (pr) {  // mixed form: the FP32 pair row, no conversions
                    const T tv = taus[h * a.chunk + t];
                    rw[0] = tv;
                    rw[1] = tv * (T)pr[0];
                    rw[2] = tv * ((T)pr[1] - (T)pr[0]);
                } else {
                    const double tv = (double)taus[h * a.chunk + t];
                    const double uv = a.u[pid];
                    rw[0] = (T)tv;
                    rw[1] = (T)(tv * uv);
                    rw[2] = (T)(a.elogu[pid] - uv);
                }
                rw[3] = T(1);
                if (a.small_only) {
                    // r is not read
                } else if (sizeof(T) == sizeof(float)) {
                    const float* yj = a.y32 + (size_t)(j0 + t) * p;
                    for (int i = 0; i < p; ++i) {
                        const T ri = (T)(yj[i] - mu32[h * p + i]);
                        rw[4 + i] = ri;
                        rw[4 + p + i] = rw[1] * ri;
                    }
                } else {
                    const double* yj = a.y + (size_t)(j0 + t) * p;
                    for (int i = 0; i < p; ++i) rw[4 + i] = (T)(yj[i] - a.mu[(size_t)h * p + i]);
                }
                if (pr) {
                    for (int k = 0; k < q + q * q; ++k) rw[4 + 2 * p + k] = rw[0] * (T)pr[2 + k];
                } else {
                    for (int k = 0; k < q; ++k) rw[4 + p + k] = (T)a.eu[pid * q + k];
                    for (int k = 0; k < q * q; ++k) rw[4 + p + q + k] = (T)a.euu[pid * q * q + k];
                }
            } else {
                for (int i = 0; i < a.row; ++i) rw[i] = T(0);
            }
        }
        __syncthreads();
        if constexpr (PF) {  // the next component's pair row, consumed at its staging
            if (h + 1 < g && t < cnt) {
                const float4* src = reinterpret_cast<const float4*>(a.pr32 + ((size_t)(h + 1) * n + j0 + t) * PW);
#pragma unroll
                for (int k = 0; k < PW / 4; ++k) {
                    const float4 v = src[k];
                    pc[4 * k] = v.x; pc[4 * k + 1] = v.y; pc[4 * k + 2] = v.z; pc[4 * k + 3] = v.w;
                }
            }
        }
        // small_only: N, U, Snu, Se and See (the tensor-core kernel writes Sr, Sre, Srr)
        const int Sred = a.small_only ? 3 + q + q * (q + 1) / 2 : stats_reduced(p, q);
        for (int es = t; es < Sred; es += blockDim.x) {
            const int e = !a.small_only || es < 3 ? es : es < 3 + q ? 3 + p + (es - 3) : 3 + p + q + p * q + (es - 3 - q);
            int ia, ib, ic, o1, o2;
            T acc = T(0), comp = T(0);
            if (sizeof(T) == sizeof(float)) {
                stat_operands_w(e, p, q, ia, ib, o1, o2);
                // two compensated sums, even and odd rows (independent chains), added at the end
                T acc1 = T(0), comp1 = T(0);
                const T* ra = rows + ia;
                const T* rb = rows + ib;
                int jj = 0;
                for (; jj + 1 < cnt; jj += 2) {
                    const T x0 = ra[(size_t)jj * a.row], y0 = rb[(size_t)jj * a.row];
                    const T x1 = ra[(size_t)(jj + 1) * a.row], y1 = rb[(size_t)(jj + 1) * a.row];
                    const T v0 = fmaf(x0, y0, -comp);
                    const T v1 = fmaf(x1, y1, -comp1);
                    const T t0 = acc + v0, t1 = acc1 + v1;
                    comp = (t0 - acc) - v0;
                    comp1 = (t1 - acc1) - v1;
                    acc = t0;
                    acc1 = t1;
                }
                if (jj < cnt) {
                    const T v0 = fmaf(ra[(size_t)jj * a.row], rb[(size_t)jj * a.row], -comp);
                    const T t0 = acc + v0;
                    comp = (t0 - acc) - v0;
                    acc = t0;
                }
                {   // the odd rows' sum into the even rows' one
                    const T v = acc1 - comp1 - comp;
                    const T tt = acc + v;
                    acc = tt;
                }
            } else {
                stat_operands(e, p, q, ia, ib, ic, o1, o2);
                for (int jj = 0; jj < cnt; ++jj) {
                    const T* rw = rows + (size_t)jj * a.row;
                    acc += rw[ia] * rw[ib] * rw[ic];
                }
            }
            out[h * S + o1] = (double)acc;
            if (o2 >= 0) out[h * S + o2] = (double)acc;
        }
        __syncthreads();
    }
}

__global__ void estep_reduce_kernel(ReduceArgs a)
{
    extern __shared__ double sm[];
    estep_reduce_body<double>(a, sm);
}

__global__ void estep_reduce_kernel_f32(ReduceArgs a)
{
    extern __shared__ double sm[];
    estep_reduce_body<float>(a, (float*)sm);
}

template <int P>
__global__ void __launch_bounds__(256, 4) estep_reduce_kernel_f32_pq(ReduceArgs a)
{
    extern __shared__ double sm[];
    estep_reduce_body<float, P, 2>(a, (float*)sm);
}

// The mixed form's statistics kernel: compile-time p and q = 2 where they apply (pair rows
// present, all statistics on the CUDA cores), else the general one.
cudaError_t launch_reduce_f32(const ReduceArgs& a, int nblocks, size_t smem, cudaStream_t st)
{
    const bool pf = a.pr32 != nullptr && !a.small_only && a.D.q == 2;
    if (pf && a.D.p == 16) estep_reduce_kernel_f32_pq<16><<<nblocks, 256, smem, st>>>(a);
    else if (pf && a.D.p == 8) estep_reduce_kernel_f32_pq<8><<<nblocks, 256, smem, st>>>(a);
    else if (pf && a.D.p == 4) estep_reduce_kernel_f32_pq<4><<<nblocks, 256, smem, st>>>(a);
    else if (pf && a.D.p == 32) estep_reduce_kernel_f32_pq<32><<<nblocks, 256, smem, st>>>(a);
    else estep_reduce_kernel_f32<<<nblocks, 256, smem, st>>>(a);
    return cudaGetLastError();
}

// dynamic shared memory above the default 48 KB for every statistics kernel (set once per
// context, before any launch or capture)
void reduce_set_smem_limits(int bytes)
{
    cudaFuncSetAttribute(estep_reduce_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    cudaFuncSetAttribute(estep_reduce_kernel_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    cudaFuncSetAttribute(estep_reduce_kernel_f32_pq<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    cudaFuncSetAttribute(estep_reduce_kernel_f32_pq<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    cudaFuncSetAttribute(estep_reduce_kernel_f32_pq<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    cudaFuncSetAttribute(estep_reduce_kernel_f32_pq<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

// S10, first level: seg[s][e] = sum of partial[b][e] over the blocks b of segment s
// (blocks s*per .. s*per + per - 1, the last segment possibly shorter), b in increasing
// order; segments at or beyond ceil(nblocks/per) (padding up to nseg) are 0.  A shard of
// the observations that starts on a segment boundary has the same segments as the whole
// problem, so the second level (reduce_partials_kernel over the segments of every shard
// in order) gives the same sums bit for bit.
__global__ void segment_partials_kernel(const double* __restrict__ partial, int nblocks, int per, int width,
                                        double* __restrict__ seg, long long nseg)
{
    const long long total = nseg * width;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long s = t / width;
        const int e = (int)(t - s * width);
        const long long b0 = s * per;
        const long long b1 = b0 + per < nblocks ? b0 + per : nblocks;
        double v = 0.0;
#pragma unroll 8  // loads in flight; the sum's order is unchanged
        for (long long b = b0; b < b1; ++b) v += partial[b * width + e];
        seg[t] = v;
    }
}

// S10: stats[e] = sum_b partial[b][e], b in increasing order.
__global__ void reduce_partials_kernel(const double* __restrict__ partial, int nblocks, int width,
                                       double* __restrict__ stats, int* flags)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < width; e += gridDim.x * blockDim.x) {
        double s = 0.0;
#pragma unroll 8  // loads in flight; the sum's order is unchanged
        for (int b = 0; b < nblocks; ++b) s += partial[(size_t)b * width + e];
        stats[e] = s;
        if (!isfinite(s)) atomicOr(flags, KF_NAN);
    }
}

// Density-only pass: l = sum_j log sum_h pi_h f_h(y_j), per-block partials.
__global__ void loglik_partial_kernel(Dims D, const double* __restrict__ pi,
                                      const double* __restrict__ logf, double* __restrict__ partial)
{
    __shared__ double sh[256];
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double v = 0.0;
    if (j < D.n) {
        double mx = -INFINITY;
        for (int h = 0; h < D.g; ++h) {
            const double t = log(pi[h]) + logf[(size_t)h * D.n + j];
            mx = t > mx ? t : mx;
        }
        double s = 0.0;
        for (int h = 0; h < D.g; ++h) s += exp(log(pi[h]) + logf[(size_t)h * D.n + j] - mx);
        v = mx + log(s);
    }
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int w = 1; w < blockDim.x; w <<= 1) {
        if ((threadIdx.x % (2 * w)) == 0 && threadIdx.x + w < blockDim.x)
            sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}
