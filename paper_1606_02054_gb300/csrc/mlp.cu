// mlp.cu -- the learned surrogate's network (not part of the paper).
//
// Training: BF16 tensor-core GEMMs (mma.sync m16n8k16, FP32 accumulation) for
// the forward and backward passes of a 3 x 256 tanh MLP, split-K partials for
// the weight gradients (fixed-order reduction), Adam in FP32.
// Inference over E-step records: one fused kernel; a warp evaluates 16 records
// with every activation kept in registers (the m16n8 accumulator fragments of
// one layer are the A fragments of the next), weights staged per layer in
// shared memory in fragment order.
#include "internal.cuh"
#include "cfust.h"
#include "tc_ptx.cuh"

#include <cuda_bf16.h>

#include <cmath>
#include <vector>

namespace {

typedef unsigned short bf16_t;  // raw bfloat16 bits

__device__ __forceinline__ void mma_bf16(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};\n"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// two floats -> packed bf16x2, round to nearest even; lo in the low half
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}
__device__ __forceinline__ bf16_t to_bf16(float x)
{
    __nv_bfloat16 v = __float2bfloat16_rn(x);
    return *reinterpret_cast<bf16_t*>(&v);
}
__device__ __forceinline__ float from_bf16(bf16_t b) { return __uint_as_float((uint32_t)b << 16); }

// ---------------------------------------------------------------------------
// Generic GEMM for training: C(m, n) = sum_k A(m, k) B(k, n), A and B BF16 with
// arbitrary element strides (transposes are strides), FP32 accumulation.
// 64 x 64 x 32 tiles, 4 warps of 32 x 32; split-K over gridDim.z.
// ---------------------------------------------------------------------------
enum { GEMM_TANH = 0, GEMM_BIAS = 1, GEMM_DTANH = 2, GEMM_PARTIAL = 3 };

struct GemmArgs {
    int M, N, K;
    const bf16_t* A;
    long long sam, sak;  // A(m, k) = A[m * sam + k * sak]
    const bf16_t* B;
    long long sbk, sbn;  // B(k, n) = B[k * sbk + n * sbn]
    int epi;
    const float* bias;   // TANH, BIAS: [N]
    const bf16_t* h;     // DTANH: h(m, n) = h[m * ldh + n] (the forward tanh output)
    long long ldh;
    void* out;           // out(m, n) = out[m * ldo + n]; PARTIAL: plus z * M * ldo
    long long ldo;
    int kchunk;          // split-K chunk, a multiple of 32
};

constexpr int GBM = 64, GBN = 64, GBK = 32, GPAD = 8;

__global__ void __launch_bounds__(128) gemm_bf16_kernel(GemmArgs g)
{
    __shared__ __align__(16) bf16_t As[GBM][GBK + GPAD];  // [m][k]
    __shared__ __align__(16) bf16_t Bs[GBN][GBK + GPAD];  // [n][k]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int wm = warp >> 1, wn = warp & 1;
    const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
    const int kbeg = blockIdx.z * g.kchunk;
    const int kend = min(g.K, kbeg + g.kchunk);
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;
    const bool a_mfast = g.sam == 1 && g.sak != 1;  // walk the contiguous index fastest
    const bool b_nfast = g.sbn == 1;
    const int r = lane >> 2, cq = (lane & 3) * 2;
    for (int k0 = kbeg; k0 < kend; k0 += GBK) {
        for (int e = tid; e < GBM * GBK; e += 128) {
            const int mm = a_mfast ? e % GBM : e / GBK, kk = a_mfast ? e / GBM : e % GBK;
            const int m = m0 + mm, k = k0 + kk;
            As[mm][kk] = (m < g.M && k < kend) ? g.A[m * g.sam + k * g.sak] : (bf16_t)0;
        }
        for (int e = tid; e < GBN * GBK; e += 128) {
            const int nn = b_nfast ? e % GBN : e / GBK, kk = b_nfast ? e / GBN : e % GBK;
            const int n = n0 + nn, k = k0 + kk;
            Bs[nn][kk] = (n < g.N && k < kend) ? g.B[k * g.sbk + n * g.sbn] : (bf16_t)0;
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < GBK; ks += 16) {
            uint32_t af[2][4], bfr[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int mr = wm * 32 + i * 16 + r;
                af[i][0] = *reinterpret_cast<const uint32_t*>(&As[mr][ks + cq]);
                af[i][1] = *reinterpret_cast<const uint32_t*>(&As[mr + 8][ks + cq]);
                af[i][2] = *reinterpret_cast<const uint32_t*>(&As[mr][ks + cq + 8]);
                af[i][3] = *reinterpret_cast<const uint32_t*>(&As[mr + 8][ks + cq + 8]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int nc = wn * 32 + j * 8 + r;
                bfr[j][0] = *reinterpret_cast<const uint32_t*>(&Bs[nc][ks + cq]);
                bfr[j][1] = *reinterpret_cast<const uint32_t*>(&Bs[nc][ks + cq + 8]);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    mma_bf16(acc[i][j], af[i][0], af[i][1], af[i][2], af[i][3], bfr[j][0], bfr[j][1]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int m = m0 + wm * 32 + i * 16 + r + (e >= 2 ? 8 : 0);
                const int n = n0 + wn * 32 + j * 8 + cq + (e & 1);
                if (m >= g.M || n >= g.N) continue;
                const float v = acc[i][j][e];
                const long long o = (long long)m * g.ldo + n;
                switch (g.epi) {
                case GEMM_TANH: ((bf16_t*)g.out)[o] = to_bf16(tanhf(v + g.bias[n])); break;
                case GEMM_BIAS: ((float*)g.out)[o] = v + g.bias[n]; break;
                case GEMM_DTANH: {
                    const float hv = from_bf16(g.h[(long long)m * g.ldh + n]);
                    ((bf16_t*)g.out)[o] = to_bf16(v * (1.f - hv * hv));
                    break;
                }
                default: ((float*)g.out)[(long long)blockIdx.z * g.M * g.ldo + o] = v; break;
                }
            }
}

// launches the GEMM; *zout (if set) receives the number of split-K partials
cudaError_t gemm(const GemmArgs& g0, int splits, cudaStream_t st, int* zout = nullptr)
{
    GemmArgs g = g0;
    if (splits < 1) splits = 1;
    g.kchunk = ((g.K + splits - 1) / splits + GBK - 1) / GBK * GBK;
    const int z = (g.K + g.kchunk - 1) / g.kchunk;
    if (zout) *zout = z;
    dim3 grid((g.N + GBN - 1) / GBN, (g.M + GBM - 1) / GBM, z);
    gemm_bf16_kernel<<<grid, 128, 0, st>>>(g);
    return cudaGetLastError();
}

// out[e] = sum_z part[z][e], z in increasing order
__global__ void sum_partials_kernel(const float* __restrict__ part, int z, long long count, float* __restrict__ out)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
         e += (long long)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int k = 0; k < z; ++k) s += part[(long long)k * count + e];
        out[e] = s;
    }
}

// ---------------------------------------------------------------------------
// Parameters: initialisation, BF16 copies, Adam
// ---------------------------------------------------------------------------
__device__ __forceinline__ double splitmix_u01_dev(unsigned long long key)
{
    unsigned long long z = key + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z = z ^ (z >> 31);
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

// W ~ U(-1/sqrt(fan_in), 1/sqrt(fan_in)) on the used rows / columns (element e of the
// flat vector draws SplitMix64 at key seed ^ (e + 1)); padding and biases 0
__global__ void mlp_init_kernel(float* theta, unsigned long long seed, int nin, int nout)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < MLP_NPARAM;
         e += (long long)gridDim.x * blockDim.x) {
        double v = 0.0;
        long long o = -1, cols = 0;
        int fan = MLP_H;
        bool live = true;
        if (e < MLP_B1) { o = MLP_W1; cols = MLP_H; fan = nin; live = (e - o) / cols < nin; }
        else if (e >= MLP_W2 && e < MLP_B2) { o = MLP_W2; cols = MLP_H; }
        else if (e >= MLP_W3 && e < MLP_B3) { o = MLP_W3; cols = MLP_H; }
        else if (e >= MLP_W4 && e < MLP_B4) { o = MLP_W4; cols = MLP_OUT; live = (e - o) % cols < nout; }
        if (o >= 0 && live) {
            const double u = splitmix_u01_dev(seed ^ (unsigned long long)(e + 1));
            v = (2.0 * u - 1.0) / sqrt((double)fan);
        }
        theta[e] = (float)v;
    }
}

// BF16 row-major copy of every parameter, and the four weight matrices in
// mma B-fragment order: for layer (K x N), n-tile nt, k-tile kt and lane,
// uint2 at ((nt * K/16 + kt) * 32 + lane) holds
// (W[k0][n], W[k0+1][n]), (W[k0+8][n], W[k0+9][n]), k0 = 16 kt + 2 (lane % 4), n = 8 nt + lane / 4.
__global__ void mlp_convert_kernel(const float* __restrict__ theta, bf16_t* __restrict__ wb, uint2* __restrict__ wf)
{
    const long long tot = MLP_NPARAM;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x)
        wb[e] = to_bf16(theta[e]);
    const long long sizes[4] = {MLP_IN * MLP_H / 4, MLP_H * MLP_H / 4, MLP_H * MLP_H / 4, MLP_H * MLP_OUT / 4};
    const long long offs[4] = {MLP_W1, MLP_W2, MLP_W3, MLP_W4};
    const int Ks[4] = {MLP_IN, MLP_H, MLP_H, MLP_H}, Ns[4] = {MLP_H, MLP_H, MLP_H, MLP_OUT};
    long long base = 0;
    for (int l = 0; l < 4; ++l) {
        const int K = Ks[l], N = Ns[l], KT = K / 16;
        const float* W = theta + offs[l];
        for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < sizes[l];
             e += (long long)gridDim.x * blockDim.x) {
            const int lane = (int)(e % 32);
            const long long tile = e / 32;
            const int kt = (int)(tile % KT), nt = (int)(tile / KT);
            const int k0 = 16 * kt + 2 * (lane % 4), n = 8 * nt + lane / 4;
            uint2 v;
            v.x = pack_bf16(W[(long long)k0 * N + n], W[(long long)(k0 + 1) * N + n]);
            v.y = pack_bf16(W[(long long)(k0 + 8) * N + n], W[(long long)(k0 + 9) * N + n]);
            wf[base + e] = v;
        }
        base += sizes[l];
    }
}

__global__ void adam_kernel(float* __restrict__ theta, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, long long count, float lr, float b1, float b2, float eps,
                            float c1, float c2)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
         e += (long long)gridDim.x * blockDim.x) {
        const float ge = g[e];
        const float me = b1 * m[e] + (1.f - b1) * ge;
        const float ve = b2 * v[e] + (1.f - b2) * ge * ge;
        m[e] = me;
        v[e] = ve;
        theta[e] -= lr * (me * c1) / (sqrtf(ve * c2) + eps);
    }
}

// dy = m (y - t) / (B nout) rounded to BF16; per-block partial sums of m (y - t)^2
__global__ void mlp_dy_kernel(int B, const float* __restrict__ y, const float* __restrict__ t,
                              const float* __restrict__ m, float inv_norm, bf16_t* __restrict__ dy,
                              double* __restrict__ lpart)
{
    __shared__ double red[256];
    double s = 0.0;
    const long long tot = (long long)B * MLP_OUT;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        const float d = y[e] - t[e];
        const float w = m[e];
        dy[e] = to_bf16(w * d * inv_norm);
        s += (double)w * d * d;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) lpart[blockIdx.x] = red[0];
}

// f32 rows -> bf16 rows (the network's input rounding)
__global__ void to_bf16_kernel(const float* __restrict__ x, long long count, bf16_t* __restrict__ out)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
         e += (long long)gridDim.x * blockDim.x)
        out[e] = to_bf16(x[e]);
}

constexpr int DY_BLOCKS = 256;

// ---------------------------------------------------------------------------
// Features of one record: standardised limits b (q), correlations R_ij = (L L^T)_ij
// for i > j in row-major order, and 1/dof (0 at dof = inf, the normal limit).
// ---------------------------------------------------------------------------
__device__ int sur_features(int q, const double* bt, const double* Lc, double dof, float* f)
{
    int o = 0;
    for (int i = 0; i < q; ++i) f[o++] = (float)bt[i];
    for (int i = 1; i < q; ++i)
        for (int j = 0; j < i; ++j) {
            double s = 0.0;
            for (int l = 0; l <= j; ++l) s += Lc[i * q + l] * Lc[j * q + l];
            f[o++] = (float)s;
        }
    f[o++] = (float)(1.0 / dof);
    return o;
}

// ---------------------------------------------------------------------------
// Training-set collection from a finished lattice E-step (records of level 0 at
// dof nu + p and the moment records at nu + p + 2).
// ---------------------------------------------------------------------------
// Sample base + i is record i of the set (fixed positions: the training order does
// not depend on thread scheduling); unusable records get type 2 (no loss, no statistics).
__global__ void sur_collect_kernel(RecSet r, const double* __restrict__ F, int q, int type, long long base,
                                   float* __restrict__ X, float* __restrict__ T, unsigned char* __restrict__ ty,
                                   unsigned long long* __restrict__ count)
{
    const int W = q + q * (q + 1) / 2;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < r.nrec;
         i += (long long)gridDim.x * blockDim.x) {
        const long long slot = base + i;
        const double v = r.res[i];
        if (!(v > 1e-300) || !isfinite(v)) {  // null or far-tail records stay with the lattice
            ty[slot] = 2;
            continue;
        }
        // moment targets: m1 and the Cholesky factor of Cov = E[X X^T] - m1 m1^T with log
        // diagonal; a record whose lattice covariance is not positive definite keeps
        // only its log T target
        int tt = type;
        double tg[MLP_OUT - 1];
        for (int k = 0; k < MLP_OUT - 1; ++k) tg[k] = 0.0;
        if (tt == 1) {
            const double* m = r.mom + i * W;
            double L[CF_MAXQ][CF_MAXQ];
            for (int a = 0; a < q && tt; ++a)
                for (int b = 0; b <= a && tt; ++b) {
                    double sum = m[q + a * (a + 1) / 2 + b] - m[a] * m[b];
                    for (int l = 0; l < b; ++l) sum -= L[a][l] * L[b][l];
                    if (a == b) {
                        if (!(sum > 0.0) || !isfinite(sum)) tt = 0;
                        else L[a][a] = sqrt(sum);
                    } else {
                        L[a][b] = sum / L[b][b];
                    }
                }
            if (tt) {
                for (int a = 0; a < q; ++a) tg[a] = m[a];
                for (int a = 0; a < q; ++a)
                    for (int b = 0; b <= a; ++b) tg[q + a * (a + 1) / 2 + b] = a == b ? log(L[a][a]) : L[a][b];
            }
        }
        atomicAdd(count, 1ULL);  // usable records (a count only)
        float f[MLP_IN];
        const int nin = sur_features(q, r.bt + i * q, F + r.fac[i], r.dof[i], f);
        float* x = X + slot * MLP_IN;
        for (int k = 0; k < MLP_IN; ++k) x[k] = k < nin ? f[k] : 0.f;
        float* t = T + slot * MLP_OUT;
        t[0] = (float)log(v);
        for (int k = 0; k < MLP_OUT - 1; ++k) t[1 + k] = (tt == 1 && k < W) ? (float)tg[k] : 0.f;
        ty[slot] = (unsigned char)tt;
    }
}

// Per-column sums (mask-aware for targets), sums of squares, min and max over
// row chunks: part[block][col][4] in double.
__global__ void col_stats_kernel(const float* __restrict__ Z, const unsigned char* __restrict__ ty, long long rows,
                                 int cols, int target, double* __restrict__ part)
{
    const int c = threadIdx.x;
    if (c >= cols) return;
    const long long chunk = (rows + gridDim.x - 1) / gridDim.x;
    const long long r0 = blockIdx.x * chunk, r1 = min(rows, r0 + chunk);
    double s = 0.0, s2 = 0.0, n = 0.0, lo = INFINITY, hi = -INFINITY;
    for (long long r = r0; r < r1; ++r) {
        if (ty[r] == 2 || (target && c > 0 && ty[r] == 0)) continue;
        const double v = Z[r * cols + c];
        s += v; s2 += v * v; n += 1.0;
        lo = v < lo ? v : lo; hi = v > hi ? v : hi;
    }
    double* o = part + ((long long)blockIdx.x * cols + c) * 5;
    o[0] = s; o[1] = s2; o[2] = n; o[3] = lo; o[4] = hi;
}

// Z[r][c] = (Z[r][c] - mean[c]) / std[c]
__global__ void standardise_kernel(float* __restrict__ Z, long long rows, int cols, const float* __restrict__ mean,
                                   const float* __restrict__ sd)
{
    const long long tot = rows * cols;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e % cols);
        Z[e] = (Z[e] - mean[c]) / sd[c];
    }
}

// Minibatch: rows idx(b) = (a * (b0 + b) + c) mod ns of the shuffled epoch
__global__ void gather_kernel(const float* __restrict__ X, const float* __restrict__ T,
                              const unsigned char* __restrict__ ty, long long ns, long long b0, int B,
                              unsigned long long a, unsigned long long c, int nout, bf16_t* __restrict__ xb,
                              float* __restrict__ tb, float* __restrict__ mb)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)B * MLP_OUT;
         e += (long long)gridDim.x * blockDim.x) {
        const long long b = e / MLP_OUT;
        const int k = (int)(e % MLP_OUT);
        // a, c < ns < 2^32: the product stays below 2^64
        const unsigned long long row = (a * ((unsigned long long)(b0 + b) % (unsigned long long)ns) + c) %
                                       (unsigned long long)ns;
        if (k < MLP_IN) xb[b * MLP_IN + k] = to_bf16(X[row * MLP_IN + k]);
        tb[e] = T[row * MLP_OUT + k];
        mb[e] = ty[row] != 2 && k < nout && (k == 0 || ty[row] == 1) ? 1.f : 0.f;
    }
}

// ---------------------------------------------------------------------------
// Fused inference over a record set
// ---------------------------------------------------------------------------
struct InferArgs {
    const uint2* wf;      // fragment-ordered W1, W2, W3, W4 (concatenated)
    const float* theta;   // biases read from here
    const float* stats;   // MLP_NSTAT
    float margin;
    int q, nin, nout, moments;
    RecSet r;
    const double* F;
    int* fall;
    int* nfall;
    unsigned char* mark;  // moment records: mark[i] = 1 when record i went to the fallback list;
                          // level-0 records with mark set: skip pairs already in that list
};

constexpr int INF_WARPS = 8, INF_ROWS = 16;
constexpr int TILE_LD = MLP_IN + 1;
constexpr size_t SM_W1 = (size_t)MLP_IN * MLP_H * 2, SM_W4 = (size_t)MLP_H * MLP_OUT * 2,
                 SM_W23 = (size_t)MLP_H * MLP_H * 2;
constexpr size_t SM_BIAS = sizeof(float) * (3 * MLP_H + MLP_OUT);
constexpr size_t SM_STAT = sizeof(float) * MLP_NSTAT;
constexpr size_t SM_TILE = sizeof(float) * INF_WARPS * INF_ROWS * TILE_LD;
constexpr size_t SM_OK = sizeof(int) * INF_WARPS * INF_ROWS;
constexpr size_t INFER_SMEM = SM_W1 + SM_W4 + SM_W23 + SM_BIAS + SM_STAT + SM_TILE + SM_OK;

// one hidden layer: in (KT k-tiles of A fragments) -> out (NT/2 k-tiles of the next
// layer's A fragments), tanh, four n-tiles at a time
template <int KT, int NT>
__device__ __forceinline__ void layer_tanh(const uint32_t (&in)[16][4], uint32_t (&out)[16][4],
                                           const uint2* __restrict__ w, const float* __restrict__ bias, int lane)
{
    const int cq = (lane & 3) * 2;
#pragma unroll
    for (int j = 0; j < NT / 2; j += 2) {
        float c[4][4];
#pragma unroll
        for (int t = 0; t < 4; ++t) { c[t][0] = 0.f; c[t][1] = 0.f; c[t][2] = 0.f; c[t][3] = 0.f; }
#pragma unroll
        for (int kt = 0; kt < KT; ++kt) {
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const uint2 b = w[((2 * j + t) * KT + kt) * 32 + lane];
                mma_bf16(c[t], in[kt][0], in[kt][1], in[kt][2], in[kt][3], b.x, b.y);
            }
        }
#pragma unroll
        for (int t = 0; t < 4; t += 2) {
            const int na = (2 * j + t) * 8 + cq, nb = (2 * j + t + 1) * 8 + cq;
            const float ba0 = bias[na], ba1 = bias[na + 1], bb0 = bias[nb], bb1 = bias[nb + 1];
            uint32_t* o = out[j + t / 2];
            o[0] = pack_bf16(tanhf(c[t][0] + ba0), tanhf(c[t][1] + ba1));
            o[1] = pack_bf16(tanhf(c[t][2] + ba0), tanhf(c[t][3] + ba1));
            o[2] = pack_bf16(tanhf(c[t + 1][0] + bb0), tanhf(c[t + 1][1] + bb1));
            o[3] = pack_bf16(tanhf(c[t + 1][2] + bb0), tanhf(c[t + 1][3] + bb1));
        }
    }
}

// output layer (K = 256, N = MLP_OUT): results into the warp's row tile
__device__ __forceinline__ void layer_out(const uint32_t (&in)[16][4], const uint2* __restrict__ w,
                                          const float* __restrict__ bias, int lane, float* tile)
{
    constexpr int KT = MLP_H / 16, NT = MLP_OUT / 8;
    const int cq = (lane & 3) * 2, r = lane >> 2;
    float c[NT][4];
#pragma unroll
    for (int t = 0; t < NT; ++t) { c[t][0] = 0.f; c[t][1] = 0.f; c[t][2] = 0.f; c[t][3] = 0.f; }
#pragma unroll
    for (int kt = 0; kt < KT; ++kt)
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const uint2 b = w[(t * KT + kt) * 32 + lane];
            mma_bf16(c[t], in[kt][0], in[kt][1], in[kt][2], in[kt][3], b.x, b.y);
        }
#pragma unroll
    for (int t = 0; t < NT; ++t) {
        const int n = t * 8 + cq;
        tile[r * TILE_LD + n] = c[t][0] + bias[n];
        tile[r * TILE_LD + n + 1] = c[t][1] + bias[n + 1];
        tile[(r + 8) * TILE_LD + n] = c[t][2] + bias[n];
        tile[(r + 8) * TILE_LD + n + 1] = c[t][3] + bias[n + 1];
    }
}

__device__ __forceinline__ void copy_smem(void* dst, const void* src, size_t bytes)
{
    const uint4* s = reinterpret_cast<const uint4*>(src);
    uint4* d = reinterpret_cast<uint4*>(dst);
    for (size_t e = threadIdx.x; e < bytes / 16; e += blockDim.x) d[e] = s[e];
}

__global__ void __launch_bounds__(INF_WARPS * 32, 1) mlp_infer_kernel(InferArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    uint2* s_w1 = reinterpret_cast<uint2*>(smem);
    uint2* s_w4 = reinterpret_cast<uint2*>(smem + SM_W1);
    uint2* s_w23 = reinterpret_cast<uint2*>(smem + SM_W1 + SM_W4);
    float* s_bias = reinterpret_cast<float*>(smem + SM_W1 + SM_W4 + SM_W23);
    float* s_stat = s_bias + 3 * MLP_H + MLP_OUT;
    float* s_tile = s_stat + MLP_NSTAT;
    int* s_ok = reinterpret_cast<int*>(s_tile + INF_WARPS * INF_ROWS * TILE_LD);
    const uint2* g_w1 = a.wf;
    const uint2* g_w2 = g_w1 + MLP_IN * MLP_H / 4;
    const uint2* g_w3 = g_w2 + MLP_H * MLP_H / 4;
    const uint2* g_w4 = g_w3 + MLP_H * MLP_H / 4;
    copy_smem(s_w1, g_w1, SM_W1);
    copy_smem(s_w4, g_w4, SM_W4);
    for (int e = threadIdx.x; e < MLP_H; e += blockDim.x) {
        s_bias[e] = a.theta[MLP_B1 + e];
        s_bias[MLP_H + e] = a.theta[MLP_B2 + e];
        s_bias[2 * MLP_H + e] = a.theta[MLP_B3 + e];
    }
    for (int e = threadIdx.x; e < MLP_OUT; e += blockDim.x) s_bias[3 * MLP_H + e] = a.theta[MLP_B4 + e];
    for (int e = threadIdx.x; e < MLP_NSTAT; e += blockDim.x) s_stat[e] = a.stats[e];
    const float* fmean = s_stat;
    const float* fstd = s_stat + MLP_IN;
    const float* zlo = s_stat + 2 * MLP_IN;
    const float* zhi = s_stat + 3 * MLP_IN;
    const float* tmean = s_stat + 4 * MLP_IN;
    const float* tstd = tmean + MLP_OUT;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* tile = s_tile + warp * INF_ROWS * TILE_LD;
    int* ok = s_ok + warp * INF_ROWS;
    const int q = a.q, W = q + q * (q + 1) / 2;
    const long long nrec = a.r.nrec;
    for (long long base = (long long)blockIdx.x * INF_WARPS * INF_ROWS; base < nrec;
         base += (long long)gridDim.x * INF_WARPS * INF_ROWS) {
        __syncthreads();  // the previous group is done with s_w23
        copy_smem(s_w23, g_w2, SM_W23);
        const long long i = base + warp * INF_ROWS + lane;
        if (lane < INF_ROWS) {
            float* row = tile + lane * TILE_LD;
            int inbox = 0;
            if (i < nrec) {
                float f[MLP_IN];
                const int nin = sur_features(q, a.r.bt + i * q, a.F + a.r.fac[i], a.r.dof[i], f);
                inbox = 1;
                for (int k = 0; k < MLP_IN; ++k) {
                    float z = 0.f;
                    if (k < nin) {
                        z = (f[k] - fmean[k]) / fstd[k];
                        // in range: the training range widened by margin standard deviations
                        if (!(z >= zlo[k] - a.margin && z <= zhi[k] + a.margin)) inbox = 0;
                    }
                    row[k] = z;
                }
            } else {
                for (int k = 0; k < MLP_IN; ++k) row[k] = 0.f;
            }
            ok[lane] = inbox;
        }
        __syncwarp();
        uint32_t xa[16][4], ya[16][4];
        {
            const int r = lane >> 2, cq = (lane & 3) * 2;
#pragma unroll
            for (int kt = 0; kt < MLP_IN / 16; ++kt) {
                const int k = kt * 16 + cq;
                xa[kt][0] = pack_bf16(tile[r * TILE_LD + k], tile[r * TILE_LD + k + 1]);
                xa[kt][1] = pack_bf16(tile[(r + 8) * TILE_LD + k], tile[(r + 8) * TILE_LD + k + 1]);
                xa[kt][2] = pack_bf16(tile[r * TILE_LD + k + 8], tile[r * TILE_LD + k + 9]);
                xa[kt][3] = pack_bf16(tile[(r + 8) * TILE_LD + k + 8], tile[(r + 8) * TILE_LD + k + 9]);
            }
        }
        __syncthreads();  // W2 staged (and W1, W4, biases on the first pass)
        layer_tanh<MLP_IN / 16, MLP_H / 8>(xa, ya, s_w1, s_bias, lane);
        layer_tanh<MLP_H / 16, MLP_H / 8>(ya, xa, s_w23, s_bias + MLP_H, lane);
        __syncthreads();
        copy_smem(s_w23, g_w3, SM_W23);
        __syncthreads();
        layer_tanh<MLP_H / 16, MLP_H / 8>(xa, ya, s_w23, s_bias + 2 * MLP_H, lane);
        __syncwarp();
        layer_out(ya, s_w4, s_bias + 3 * MLP_H, lane, tile);
        __syncwarp();
        if (lane < INF_ROWS && i < nrec) {
            const float* row = tile + lane * TILE_LD;
            if (a.mark && a.moments) a.mark[i] = ok[lane] ? 0 : 1;
            if (ok[lane]) {
                const double logT = (double)(row[0] * tstd[0] + tmean[0]);
                a.r.res[i] = exp(logT);
                if (a.r.se) a.r.se[i] = 0.0;
                if (a.moments) {
                    // m1 and E[X X^T] = L L^T + m1 m1^T, L with exp of its predicted log diagonal
                    double m1[CF_MAXQ], L[CF_MAXQ][CF_MAXQ];
                    for (int k = 0; k < q; ++k) m1[k] = (double)(row[1 + k] * tstd[1 + k] + tmean[1 + k]);
                    for (int r2 = 0; r2 < q; ++r2)
                        for (int c2 = 0; c2 <= r2; ++c2) {
                            const int k = 1 + q + r2 * (r2 + 1) / 2 + c2;
                            const double v = (double)(row[k] * tstd[k] + tmean[k]);
                            L[r2][c2] = r2 == c2 ? exp(v) : v;
                        }
                    double* out = a.r.mom + i * W;
                    for (int k = 0; k < q; ++k) out[k] = m1[k];
                    for (int r2 = 0; r2 < q; ++r2)
                        for (int c2 = 0; c2 <= r2; ++c2) {
                            double sm = m1[r2] * m1[c2];
                            for (int l = 0; l <= c2; ++l) sm += L[r2][l] * L[c2][l];
                            out[q + r2 * (r2 + 1) / 2 + c2] = sm;
                        }
                }
            } else if (!(a.mark && !a.moments && a.mark[i])) {
                a.fall[atomicAdd(a.nfall, 1)] = (int)i;
            }
        }
        __syncwarp();
    }
}

#include "mlp_tc.cuh"

int grid_of(long long work, int threads, int cap)
{
    long long b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    return (int)(b < cap ? b : cap);
}

template <typename T>
cudaError_t dalloc(T** p, size_t count)
{
    return cudaMalloc((void**)p, sizeof(T) * (count ? count : 1));
}

int sm_count()
{
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

// forward + backward of one minibatch already in s.xb / s.tb / s.mb; gradient into s.grad
cudaError_t mlp_fwd_bwd(Surrogate& s, int B, int nout, double* loss, cudaStream_t st)
{
    const bf16_t* wb = (const bf16_t*)s.wb;
    const bf16_t* xb = (const bf16_t*)s.xb;
    bf16_t *h1 = (bf16_t*)s.h1, *h2 = (bf16_t*)s.h2, *h3 = (bf16_t*)s.h3;
    bf16_t *dz = (bf16_t*)s.dz, *dz2 = (bf16_t*)s.dz2;
    cudaError_t e;
    auto fwd = [&](const bf16_t* in, int K, long long woff, long long boff, int N, int epi, void* out) {
        GemmArgs g{};
        g.M = B; g.N = N; g.K = K;
        g.A = in; g.sam = K; g.sak = 1;
        g.B = wb + woff; g.sbk = N; g.sbn = 1;
        g.epi = epi; g.bias = s.theta + boff; g.out = out; g.ldo = N;
        return gemm(g, 1, st);
    };
    if ((e = fwd(xb, MLP_IN, MLP_W1, MLP_B1, MLP_H, GEMM_TANH, h1))) return e;
    if ((e = fwd(h1, MLP_H, MLP_W2, MLP_B2, MLP_H, GEMM_TANH, h2))) return e;
    if ((e = fwd(h2, MLP_H, MLP_W3, MLP_B3, MLP_H, GEMM_TANH, h3))) return e;
    if ((e = fwd(h3, MLP_H, MLP_W4, MLP_B4, MLP_OUT, GEMM_BIAS, s.y))) return e;
    const float inv_norm = (float)(1.0 / ((double)B * nout));
    mlp_dy_kernel<<<DY_BLOCKS, 256, 0, st>>>(B, s.y, s.tb, s.mb, inv_norm, dz, s.lpart);
    if ((e = cudaGetLastError())) return e;
    const int splits = B >= 2048 ? B / 512 : 1;
    // layer l: dW = h_{l-1}^T dz (split-K partials), db = 1^T dz, dh_{l-1} = dz W^T (* tanh')
    const bf16_t* hin[4] = {xb, h1, h2, h3};
    const int Ks[4] = {MLP_IN, MLP_H, MLP_H, MLP_H}, Ns[4] = {MLP_H, MLP_H, MLP_H, MLP_OUT};
    const long long Wo[4] = {MLP_W1, MLP_W2, MLP_W3, MLP_W4}, Bo[4] = {MLP_B1, MLP_B2, MLP_B3, MLP_B4};
    bf16_t* cur = dz;
    bf16_t* nxt = dz2;
    for (int l = 3; l >= 0; --l) {
        const int K = Ks[l], N = Ns[l];
        GemmArgs g{};
        g.M = K; g.N = N; g.K = B;
        g.A = hin[l]; g.sam = 1; g.sak = K;   // A(m = input unit, k = row) = h[row][m]
        g.B = cur; g.sbk = N; g.sbn = 1;      // B(k = row, n) = dz[row][n]
        g.epi = GEMM_PARTIAL; g.out = s.part; g.ldo = N;
        int z = 1;
        if ((e = gemm(g, splits, st, &z))) return e;
        sum_partials_kernel<<<grid_of((long long)K * N, 256, 1024), 256, 0, st>>>(s.part, z, (long long)K * N,
                                                                                  s.grad + Wo[l]);
        if ((e = cudaGetLastError())) return e;
        GemmArgs gb{};
        gb.M = 1; gb.N = N; gb.K = B;
        gb.A = (const bf16_t*)s.one; gb.sam = 0; gb.sak = 0;
        gb.B = cur; gb.sbk = N; gb.sbn = 1;
        gb.epi = GEMM_PARTIAL; gb.out = s.part; gb.ldo = N;
        if ((e = gemm(gb, splits, st))) return e;
        sum_partials_kernel<<<grid_of(N, 256, 16), 256, 0, st>>>(s.part, z, (long long)N, s.grad + Bo[l]);
        if ((e = cudaGetLastError())) return e;
        if (l > 0) {
            GemmArgs gd{};
            gd.M = B; gd.N = K; gd.K = N;
            gd.A = cur; gd.sam = N; gd.sak = 1;
            gd.B = wb + Wo[l]; gd.sbk = 1; gd.sbn = N;  // B(k = out unit, n = in unit) = W[n][k]
            gd.epi = GEMM_DTANH; gd.h = hin[l]; gd.ldh = K; gd.out = nxt; gd.ldo = K;
            if ((e = gemm(gd, 1, st))) return e;
            bf16_t* tmp = cur; cur = nxt; nxt = tmp;
        }
    }
    if (loss) {
        if ((e = cudaMemcpyAsync(s.host_part, s.lpart, sizeof(double) * DY_BLOCKS, cudaMemcpyDeviceToHost, st)))
            return e;
        if ((e = cudaStreamSynchronize(st))) return e;
        double t = 0.0;
        for (int b = 0; b < DY_BLOCKS; ++b) t += s.host_part[b];
        *loss = 0.5 * t / ((double)B * nout);
    }
    return cudaSuccess;
}

cudaError_t convert(Surrogate& s, cudaStream_t st)
{
    mlp_convert_kernel<<<grid_of(MLP_NPARAM, 256, 1024), 256, 0, st>>>(s.theta, (bf16_t*)s.wb, (uint2*)s.wf);
    mlp_tc_pack_kernel<<<grid_of((long long)(TCI_WTC / 2), 256, 1024), 256, 0, st>>>(s.theta, (bf16_t*)s.wtc);
    return cudaGetLastError();
}

cudaError_t adam_step(Surrogate& s, float lr, cudaStream_t st)
{
    s.step += 1;
    const double b1 = 0.9, b2 = 0.999;
    const float c1 = (float)(1.0 / (1.0 - pow(b1, (double)s.step)));
    const float c2 = (float)(1.0 / (1.0 - pow(b2, (double)s.step)));
    adam_kernel<<<grid_of(MLP_NPARAM, 256, 1024), 256, 0, st>>>(s.theta, s.grad, s.am, s.av, MLP_NPARAM, lr,
                                                               (float)b1, (float)b2, 1e-8f, c1, c2);
    cudaError_t e = cudaGetLastError();
    if (e) return e;
    return convert(s, st);
}

cudaError_t alloc_params(Surrogate& s)
{
    cudaError_t e;
    if (s.theta) return cudaSuccess;
    if ((e = dalloc(&s.theta, MLP_NPARAM)) || (e = dalloc(&s.grad, MLP_NPARAM)) || (e = dalloc(&s.am, MLP_NPARAM)) ||
        (e = dalloc(&s.av, MLP_NPARAM)) || (e = dalloc(&s.stats, MLP_NSTAT)) ||
        (e = dalloc((bf16_t**)&s.wb, MLP_NPARAM)) || (e = dalloc((bf16_t**)&s.wf, MLP_NPARAM)) ||
        (e = dalloc((bf16_t**)&s.wtc, TCI_WTC / 2)) ||
        (e = dalloc(&s.nfall, 2)) || (e = dalloc(&s.count, 1)))
        return e;
    return cudaSuccess;
}

cudaError_t alloc_batch(Surrogate& s, int B)
{
    if (s.bcap >= B) return cudaSuccess;
    cudaFree(s.xb); cudaFree(s.h1); cudaFree(s.h2); cudaFree(s.h3); cudaFree(s.dz); cudaFree(s.dz2);
    cudaFree(s.one); cudaFree(s.y); cudaFree(s.tb); cudaFree(s.mb); cudaFree(s.part); cudaFree(s.lpart);
    cudaFreeHost(s.host_part);
    s.bcap = 0;
    cudaError_t e;
    const int splits = B >= 2048 ? B / 512 : 1;
    if ((e = dalloc((bf16_t**)&s.xb, (size_t)B * MLP_IN)) || (e = dalloc((bf16_t**)&s.h1, (size_t)B * MLP_H)) ||
        (e = dalloc((bf16_t**)&s.h2, (size_t)B * MLP_H)) || (e = dalloc((bf16_t**)&s.h3, (size_t)B * MLP_H)) ||
        (e = dalloc((bf16_t**)&s.dz, (size_t)B * MLP_H)) || (e = dalloc((bf16_t**)&s.dz2, (size_t)B * MLP_H)) ||
        (e = dalloc((bf16_t**)&s.one, 8)) || (e = dalloc(&s.y, (size_t)B * MLP_OUT)) ||
        (e = dalloc(&s.tb, (size_t)B * MLP_OUT)) || (e = dalloc(&s.mb, (size_t)B * MLP_OUT)) ||
        (e = dalloc(&s.part, (size_t)(splits + 1) * MLP_H * MLP_H)) || (e = dalloc(&s.lpart, DY_BLOCKS)) ||
        (e = cudaMallocHost((void**)&s.host_part, sizeof(double) * DY_BLOCKS)))
        return e;
    const bf16_t one[8] = {0x3F80, 0x3F80, 0x3F80, 0x3F80, 0x3F80, 0x3F80, 0x3F80, 0x3F80};  // 1.0
    if ((e = cudaMemcpy(s.one, one, sizeof(one), cudaMemcpyHostToDevice))) return e;
    s.bcap = B;
    return cudaSuccess;
}

}  // namespace

// ---------------------------------------------------------------------------
// Surrogate state used by the E-step (api.cu)
// ---------------------------------------------------------------------------
cudaError_t sur_reserve(Surrogate& s, int q, long long records, cudaStream_t)
{
    cudaError_t e;
    if ((e = alloc_params(s))) return e;
    // the inference kernel's shared memory (set here, outside any stream capture)
    if ((e = cudaFuncSetAttribute(mlp_infer_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)INFER_SMEM)) ||
        (e = cudaFuncSetAttribute(mlp_infer_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TCI_SMEM)))
        return e;
    s.q = q;
    s.nin = q + q * (q - 1) / 2 + 1;
    s.nout = 1 + q + q * (q + 1) / 2;
    if (s.cap < records) {
        cudaFree(s.fall0); cudaFree(s.fallM); cudaFree(s.mark);
        s.fall0 = s.fallM = nullptr;
        s.mark = nullptr;
        s.cap = 0;
        if ((e = dalloc(&s.fall0, records)) || (e = dalloc(&s.fallM, records)) || (e = dalloc(&s.mark, records)))
            return e;
        s.cap = records;
    }
    return cudaSuccess;
}

void sur_free(Surrogate& s)
{
    void* ps[] = {s.theta, s.grad, s.am, s.av, s.stats, s.wb, s.wf, s.wtc, s.X, s.T, s.type, s.count, s.xb, s.h1,
                  s.h2, s.h3, s.dz, s.dz2, s.one, s.y, s.tb, s.mb, s.part, s.lpart, s.fall0, s.fallM, s.nfall,
                  s.mark};
    for (void* p : ps) cudaFree(p);
    cudaFreeHost(s.host_part);
    s = Surrogate{};
}

cudaError_t sur_collect(Surrogate& s, const RecSet& L0, const RecSet& LM, const double* F, cudaStream_t st)
{
    cudaError_t e;
    const long long need = L0.nrec + LM.nrec;
    if (s.ns_cap < need) {
        cudaFree(s.X); cudaFree(s.T); cudaFree(s.type);
        s.X = s.T = nullptr; s.type = nullptr; s.ns_cap = 0;
        if ((e = dalloc(&s.X, (size_t)need * MLP_IN)) || (e = dalloc(&s.T, (size_t)need * MLP_OUT)) ||
            (e = dalloc(&s.type, (size_t)need)))
            return e;
        s.ns_cap = need;
    }
    if ((e = cudaMemsetAsync(s.count, 0, sizeof(unsigned long long), st))) return e;
    const int nsm = sm_count();
    sur_collect_kernel<<<grid_of(L0.nrec, 256, nsm * 8), 256, 0, st>>>(L0, F, s.q, 0, 0, s.X, s.T, s.type,
                                                                       s.count);
    if ((e = cudaGetLastError())) return e;
    sur_collect_kernel<<<grid_of(LM.nrec, 256, nsm * 8), 256, 0, st>>>(LM, F, s.q, 1, L0.nrec, s.X, s.T, s.type,
                                                                       s.count);
    if ((e = cudaGetLastError())) return e;
    unsigned long long n = 0;
    if ((e = cudaMemcpyAsync(&n, s.count, sizeof(n), cudaMemcpyDeviceToHost, st))) return e;
    if ((e = cudaStreamSynchronize(st))) return e;
    if (n < 64) return cudaErrorInvalidValue;
    s.ns = need;
    // feature and target statistics (double partials, summed on the host)
    const int nb = 1024;
    double* part = nullptr;
    if ((e = dalloc(&part, (size_t)nb * MLP_OUT * 5))) return e;
    std::vector<double> hp((size_t)nb * MLP_OUT * 5);
    // the first training fixes the standardisation; later ones only widen the range
    const bool keep = s.trained;
    std::vector<float> stats(s.hstats, s.hstats + MLP_NSTAT);
    for (int target = 0; target < 2; ++target) {
        const int cols = target ? MLP_OUT : MLP_IN;
        col_stats_kernel<<<nb, 64, 0, st>>>(target ? s.T : s.X, s.type, s.ns, cols, target, part);
        if ((e = cudaGetLastError())) break;
        if ((e = cudaMemcpyAsync(hp.data(), part, sizeof(double) * nb * cols * 5, cudaMemcpyDeviceToHost, st))) break;
        if ((e = cudaStreamSynchronize(st))) break;
        for (int c = 0; c < cols; ++c) {
            double sm = 0, s2 = 0, n2 = 0, lo = INFINITY, hi = -INFINITY;
            for (int b = 0; b < nb; ++b) {
                const double* o = &hp[((size_t)b * cols + c) * 5];
                sm += o[0]; s2 += o[1]; n2 += o[2];
                lo = o[3] < lo ? o[3] : lo; hi = o[4] > hi ? o[4] : hi;
            }
            if (keep) {
                if (!target && n2 > 0) {
                    const double mean = stats[c], sd = stats[MLP_IN + c];
                    stats[2 * MLP_IN + c] = std::min(stats[2 * MLP_IN + c], (float)((lo - mean) / sd));
                    stats[3 * MLP_IN + c] = std::max(stats[3 * MLP_IN + c], (float)((hi - mean) / sd));
                }
                continue;
            }
            const double mean = n2 > 0 ? sm / n2 : 0.0;
            double var = n2 > 0 ? s2 / n2 - mean * mean : 0.0;
            double sd = var > 0 ? std::sqrt(var) : 0.0;
            if (!(sd > 1e-6 * (std::fabs(mean) + 1e-30)) || !(sd > 1e-12)) sd = 1.0;  // constant column
            if (target) {
                stats[4 * MLP_IN + c] = (float)mean;
                stats[4 * MLP_IN + MLP_OUT + c] = (float)sd;
            } else {
                stats[c] = (float)mean;
                stats[MLP_IN + c] = (float)sd;
                stats[2 * MLP_IN + c] = n2 > 0 ? (float)((lo - mean) / sd) : 0.f;
                stats[3 * MLP_IN + c] = n2 > 0 ? (float)((hi - mean) / sd) : 0.f;
            }
        }
    }
    cudaFree(part);
    if (e) return e;
    for (int k = 0; k < MLP_NSTAT; ++k) s.hstats[k] = stats[k];
    if ((e = cudaMemcpyAsync(s.stats, s.hstats, sizeof(float) * MLP_NSTAT, cudaMemcpyHostToDevice, st))) return e;
    standardise_kernel<<<grid_of(s.ns * MLP_IN, 256, nsm * 8), 256, 0, st>>>(s.X, s.ns, MLP_IN, s.stats,
                                                                            s.stats + MLP_IN);
    if ((e = cudaGetLastError())) return e;
    standardise_kernel<<<grid_of(s.ns * MLP_OUT, 256, nsm * 8), 256, 0, st>>>(
        s.T, s.ns, MLP_OUT, s.stats + 4 * MLP_IN, s.stats + 4 * MLP_IN + MLP_OUT);
    if ((e = cudaGetLastError())) return e;
    return cudaStreamSynchronize(st);
}

cudaError_t sur_train(Surrogate& s, const SurOpts& o, cudaStream_t st, double* losses)
{
    cudaError_t e;
    if ((e = alloc_batch(s, o.batch))) return e;
    if (!s.trained) {
        mlp_init_kernel<<<grid_of(MLP_NPARAM, 256, 1024), 256, 0, st>>>(s.theta, o.seed, s.nin, s.nout);
        if ((e = cudaGetLastError())) return e;
        if ((e = cudaMemsetAsync(s.am, 0, sizeof(float) * MLP_NPARAM, st))) return e;
        if ((e = cudaMemsetAsync(s.av, 0, sizeof(float) * MLP_NPARAM, st))) return e;
        s.step = 0;
        if ((e = convert(s, st))) return e;
    }
    s.margin = o.margin;
    const long long per_epoch = o.samples_per_epoch > 0 && o.samples_per_epoch < s.ns ? o.samples_per_epoch : s.ns;
    const int nb = (int)((per_epoch + o.batch - 1) / o.batch);
    for (int ep = 0; ep < o.epochs; ++ep) {
        // shuffle: row(b) = (a b + c) mod ns with a coprime to ns
        unsigned long long key = o.seed ^ ((unsigned long long)(ep + 1) << 32) ^ (unsigned long long)s.step;
        auto next = [&]() {
            key += 0x9E3779B97F4A7C15ULL;
            unsigned long long z = key;
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
            z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
            return z ^ (z >> 31);
        };
        const unsigned long long ns = (unsigned long long)s.ns;
        unsigned long long a = next() % ns;
        auto gcd = [](unsigned long long x, unsigned long long y) {
            while (y) { unsigned long long t = x % y; x = y; y = t; }
            return x;
        };
        if (a == 0) a = 1;
        while (gcd(a, ns) != 1) a = a % ns + 1;
        const unsigned long long c = next() % ns;
        double tot = 0.0;
        for (int b = 0; b < nb; ++b) {
            gather_kernel<<<grid_of((long long)o.batch * MLP_OUT, 256, 2048), 256, 0, st>>>(
                s.X, s.T, s.type, s.ns, (long long)b * o.batch, o.batch, a, c, s.nout, (bf16_t*)s.xb, s.tb, s.mb);
            if ((e = cudaGetLastError())) return e;
            double l = 0.0;
            const bool want = losses && (b == nb - 1 || nb <= 8);
            if ((e = mlp_fwd_bwd(s, o.batch, s.nout, want ? &l : nullptr, st))) return e;
            if ((e = adam_step(s, o.lr, st))) return e;
            if (want) tot = l;
        }
        if (losses) losses[ep] = tot;
    }
    s.trained = true;
    return cudaStreamSynchronize(st);
}

cudaError_t sur_infer(const Surrogate& s, const RecSet& r, const double* F, int moments, int* fall, int* nfall,
                      int* err, cudaStream_t st, unsigned char* mark)
{
    if (r.nrec == 0) return cudaSuccess;
    InferArgs a;
    a.wf = (const uint2*)s.wf; a.theta = s.theta; a.stats = s.stats; a.margin = s.margin;
    a.q = s.q; a.nin = s.nin; a.nout = s.nout; a.moments = moments;
    a.r = r; a.F = F; a.fall = fall; a.nfall = nfall; a.mark = mark;
    // the tensor-core kernel: one CTA per SM at most, tiles of 128 records
    const long long tiles = (r.nrec + TCI_M - 1) / TCI_M;
    const int nsm = sm_count();
    const int blocks = (int)(tiles < nsm ? tiles : nsm);
    mlp_infer_tc_kernel<<<blocks, TCI_THREADS, TCI_SMEM, st>>>(a, (const bf16_t*)s.wtc, err);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Stateless entry points (host buffers), used to check the kernels against the
// oracle's network
// ---------------------------------------------------------------------------
namespace {
cfust_status mlp_fail(cudaError_t e)
{
    return e == cudaSuccess ? CFUST_OK : (e == cudaErrorInvalidValue ? CFUST_EINVAL : CFUST_ECUDA);
}
}  // namespace

extern "C" cfust_status cfust_mlp_init(uint64_t seed, int nin, int nout, float* theta_out, int device)
{
    if (!theta_out || nin < 1 || nin > MLP_IN || nout < 1 || nout > MLP_OUT) return CFUST_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return CFUST_ECUDA;
    float* d = nullptr;
    cudaError_t e = dalloc(&d, MLP_NPARAM);
    if (!e) {
        mlp_init_kernel<<<grid_of(MLP_NPARAM, 256, 1024), 256>>>(d, seed, nin, nout);
        e = cudaGetLastError();
    }
    if (!e) e = cudaMemcpy(theta_out, d, sizeof(float) * MLP_NPARAM, cudaMemcpyDeviceToHost);
    cudaFree(d);
    return mlp_fail(e);
}

extern "C" cfust_status cfust_mlp_grad(const float* theta, int64_t rows, int nout, const float* f, const float* t,
                                       const float* m, float* grad_out, float* y_out, double* loss_out, int device)
{
    if (!theta || !f || !t || !m || rows < 1 || nout < 1 || nout > MLP_OUT || rows > (1 << 22)) return CFUST_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return CFUST_ECUDA;
    Surrogate s;
    cudaStream_t st = nullptr;
    float* fx = nullptr;
    cudaError_t e = cudaStreamCreate(&st);
    const int B = (int)rows;
    if (!e) e = alloc_params(s);
    if (!e) e = alloc_batch(s, B);
    if (!e) e = dalloc(&fx, (size_t)B * MLP_IN);
    if (!e) e = cudaMemcpyAsync(s.theta, theta, sizeof(float) * MLP_NPARAM, cudaMemcpyHostToDevice, st);
    if (!e) e = cudaMemcpyAsync(fx, f, sizeof(float) * B * MLP_IN, cudaMemcpyHostToDevice, st);
    if (!e) e = cudaMemcpyAsync(s.tb, t, sizeof(float) * B * MLP_OUT, cudaMemcpyHostToDevice, st);
    if (!e) e = cudaMemcpyAsync(s.mb, m, sizeof(float) * B * MLP_OUT, cudaMemcpyHostToDevice, st);
    if (!e) {
        to_bf16_kernel<<<grid_of((long long)B * MLP_IN, 256, 1024), 256, 0, st>>>(fx, (long long)B * MLP_IN,
                                                                                 (bf16_t*)s.xb);
        e = cudaGetLastError();
    }
    if (!e) e = convert(s, st);
    double l = 0.0;
    if (!e) e = mlp_fwd_bwd(s, B, nout, &l, st);
    if (!e && grad_out) e = cudaMemcpyAsync(grad_out, s.grad, sizeof(float) * MLP_NPARAM, cudaMemcpyDeviceToHost, st);
    if (!e && y_out) e = cudaMemcpyAsync(y_out, s.y, sizeof(float) * B * MLP_OUT, cudaMemcpyDeviceToHost, st);
    if (!e) e = cudaStreamSynchronize(st);
    if (!e && loss_out) *loss_out = l;
    cudaFree(fx);
    sur_free(s);
    if (st) cudaStreamDestroy(st);
    return mlp_fail(e);
}

extern "C" cfust_status cfust_mlp_adam(float* theta, const float* grad, float* m, float* v, int64_t step, float lr,
                                       int device)
{
    if (!theta || !grad || !m || !v || step < 1) return CFUST_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return CFUST_ECUDA;
    Surrogate s;
    cudaError_t e = alloc_params(s);
    const size_t nb = sizeof(float) * MLP_NPARAM;
    if (!e) e = cudaMemcpy(s.theta, theta, nb, cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(s.grad, grad, nb, cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(s.am, m, nb, cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(s.av, v, nb, cudaMemcpyHostToDevice);
    s.step = step - 1;
    if (!e) e = adam_step(s, lr, nullptr);
    if (!e) e = cudaDeviceSynchronize();
    if (!e) e = cudaMemcpy(theta, s.theta, nb, cudaMemcpyDeviceToHost);
    if (!e) e = cudaMemcpy(m, s.am, nb, cudaMemcpyDeviceToHost);
    if (!e) e = cudaMemcpy(v, s.av, nb, cudaMemcpyDeviceToHost);
    sur_free(s);
    return mlp_fail(e);
}

extern "C" cfust_status cfust_mlp_records(const float* theta, const float* stats, float margin, int q, int64_t rows,
                                          const double* bt, const double* Lc, const double* dof, double* logT,
                                          double* mom, int* inbox, int device)
{
    if (!theta || !stats || !bt || !Lc || !dof || !logT || !inbox || q < 3 || q > CF_MAXQ || rows < 1 ||
        rows > (1 << 24))
        return CFUST_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return CFUST_ECUDA;
    Surrogate s;
    cudaStream_t st = nullptr;
    const int W = q + q * (q + 1) / 2;
    double *dbt = nullptr, *dF = nullptr, *ddof = nullptr, *dres = nullptr, *dmom = nullptr;
    int *dfac = nullptr, *dfall = nullptr, *derr = nullptr;
    cudaError_t e = cudaStreamCreate(&st);
    if (!e) e = alloc_params(s);
    if (!e) e = sur_reserve(s, q, rows, st);
    if (!e) e = dalloc(&dbt, (size_t)rows * q);
    if (!e) e = dalloc(&dF, (size_t)rows * q * q);
    if (!e) e = dalloc(&ddof, (size_t)rows);
    if (!e) e = dalloc(&dres, (size_t)rows);
    if (!e) e = dalloc(&dmom, (size_t)rows * W);
    if (!e) e = dalloc(&dfac, (size_t)rows);
    if (!e) e = dalloc(&dfall, (size_t)rows);
    if (!e) e = dalloc(&derr, 1);
    if (!e) e = cudaMemsetAsync(derr, 0, sizeof(int), st);
    std::vector<int> fac((size_t)rows);
    for (int64_t i = 0; i < rows; ++i) fac[i] = (int)(i * q * q);
    if (!e) e = cudaMemcpyAsync(s.theta, theta, sizeof(float) * MLP_NPARAM, cudaMemcpyHostToDevice, st);
    if (!e) e = cudaMemcpyAsync(s.stats, stats, sizeof(float) * MLP_NSTAT, cudaMemcpyHostToDevice, st);
    if (!e) e = cudaMemcpyAsync(dbt, bt, sizeof(double) * rows * q, cudaMemcpyHostToDevice, st);
    if (!e) e = cudaMemcpyAsync(dF, Lc, sizeof(double) * rows * q * q, cudaMemcpyHostToDevice, st);
    if (!e) e = cudaMemcpyAsync(ddof, dof, sizeof(double) * rows, cudaMemcpyHostToDevice, st);
    if (!e) e = cudaMemcpyAsync(dfac, fac.data(), sizeof(int) * rows, cudaMemcpyHostToDevice, st);
    if (!e) e = cudaMemsetAsync(s.nfall, 0, sizeof(int), st);
    if (!e) e = cudaMemsetAsync(dres, 0, sizeof(double) * rows, st);
    if (!e) e = convert(s, st);
    s.margin = margin;
    RecSet r{};
    r.k = q; r.nrec = rows; r.bt = dbt; r.fac = dfac; r.dof = ddof; r.res = dres; r.mom = dmom;
    if (!e) e = sur_infer(s, r, dF, 1, dfall, s.nfall, derr, st);
    std::vector<double> res((size_t)rows);
    int nf = 0, herr = 0;
    if (!e) e = cudaMemcpyAsync(res.data(), dres, sizeof(double) * rows, cudaMemcpyDeviceToHost, st);
    if (!e && mom) e = cudaMemcpyAsync(mom, dmom, sizeof(double) * rows * W, cudaMemcpyDeviceToHost, st);
    if (!e) e = cudaMemcpyAsync(&nf, s.nfall, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (!e) e = cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (!e) e = cudaStreamSynchronize(st);
    if (!e && herr) {
        cudaFree(dbt); cudaFree(dF); cudaFree(ddof); cudaFree(dres); cudaFree(dmom); cudaFree(dfac); cudaFree(dfall);
        cudaFree(derr);
        sur_free(s);
        if (st) cudaStreamDestroy(st);
        return CFUST_ETIMEOUT;
    }
    std::vector<int> fl;
    if (!e && nf > 0) {
        fl.resize((size_t)nf);
        e = cudaMemcpy(fl.data(), dfall, sizeof(int) * nf, cudaMemcpyDeviceToHost);
    }
    if (!e) {
        for (int64_t i = 0; i < rows; ++i) {
            inbox[i] = 1;
            logT[i] = std::log(res[i]);
        }
        for (int v : fl) {
            inbox[v] = 0;
            logT[v] = NAN;
        }
    }
    cudaFree(dbt); cudaFree(dF); cudaFree(ddof); cudaFree(dres); cudaFree(dmom); cudaFree(dfac); cudaFree(dfall);
    cudaFree(derr);
    sur_free(s);
    if (st) cudaStreamDestroy(st);
    return mlp_fail(e);
}
