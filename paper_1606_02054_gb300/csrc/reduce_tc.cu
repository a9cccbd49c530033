// reduce_tc.cu -- the mixed form's cross statistics of eqs (18)-(21) on the tensor cores.
//
// Per block of observations and component h, with r = y_j - mu_h^(k), w = tau u:
//   Srr_h = sum_j w r r^T (p x p),  Sre_h = sum_j tau r eu^T (p x q),  Sr_h = sum_j w r (p).
// They are one contraction over the observations: with A[(h,a)][j] = r_hj,a (rows
// (h, a), a < p) and B[(h,b)][j] = [w r_hj,b | tau eu_hj,b' | w] (rows (h, b), p + q + 1
// per component), D = A B^T holds [Srr_h | Sre_h | Sr_h] in its (h, h) blocks (the other
// blocks are not needed; at g p <= 128 rows all components fit one 128-row tile).
//
// tcgen05.mma kind::tf32 (M = 128, N = the B rows padded to a multiple of 16), the
// operands in shared memory in the K-major canonical layout without swizzle, the
// accumulator in tensor memory.  Every FP32 operand x is split as x = hi + lo with hi
// its TF32 rounding, and A B^T = Ahi Bhi^T + Ahi Blo^T + Alo Bhi^T (lo lo dropped:
// products to ~2^-21 relative).  The tensor core accumulates in FP32 over one block of
// the reduction (a.chunk <= 256 observations, the CUDA-core kernel's blocks); the
// block's D is written to the FP64 block partials, which the
// fixed-order reduction sums as for the CUDA-core statistics.  The other statistics
// (N, U, Snu, Se, See) stay in the CUDA-core kernel, which also writes tau.
//
// Each CTA (256 threads) loops over blocks; a block is chunk/16 sub-chunks of 16
// observations, double-buffered in shared memory: while the tensor core multiplies one
// buffer, the threads fill the other.  Waits on the MMA completion barriers are bounded
// (an error flag is set and the kernel leaves after freeing its tensor memory).
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.cuh"

namespace {

constexpr int TC_THREADS = 256;
constexpr int TC_SUB = 16;     // observations per sub-chunk (two K-slices of 8 TF32)
constexpr int TC_M = 128;
constexpr long long TC_SPIN = 1LL << 24;  // iteration limit of a barrier wait

// element offset (4-byte units) of (row r, k) in an operand of R rows, k < 16:
// [K-slice][8-row group][16-byte column group][row in group][4 values]; a core matrix
// (8 rows x 16 bytes) is 128 contiguous bytes, the next along K 128 bytes on (LBO), the
// next 8-row group 256 bytes on (SBO); one K-slice of R rows spans R x 32 bytes.
__device__ __forceinline__ int tc_off(int r, int k, int R)
{
    const int ks = k >> 3, kin = k & 7;
    return ks * (R * 8) + (r >> 3) * 64 + (kin >> 2) * 32 + (r & 7) * 4 + (kin & 3);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start address, leading (K) and stride (8-row group)
// byte offsets, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

__device__ __forceinline__ float tf32_rn(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    for (long long it = 0; it < TC_SPIN; ++it) {
        uint32_t done;
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done)
                     : "r"(bar), "r"(parity));
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v)
{
    uint32_t r[32];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
                   "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
                   "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

}  // namespace

// Shared memory: two buffers of {Ahi, Alo} (128 x 16) and {Bhi, Blo} (NP x 16) floats,
// then the sub-chunk's inputs (y: 16 x p, tau, u: g x 16, eu: g x 16 x q floats), the
// means (g x p floats), the completion barriers and the tensor-memory address.
size_t reduce_tc_smem(int p, int q, int g)
{
    const int NP = (g * (p + q + 1) + 15) / 16 * 16;
    const size_t buf = (size_t)2 * (TC_M + NP) * TC_SUB;
    const size_t in = (size_t)TC_SUB * p + (size_t)g * TC_SUB * (2 + q) + (size_t)g * p + TC_M + NP;
    return sizeof(float) * (2 * buf + in) + 64;
}

bool reduce_tc_fits(int p, int q, int g)
{
    return g * p <= TC_M && g * (p + q + 1) <= 256 && reduce_tc_smem(p, q, g) <= 110 * 1024;
}

__global__ void __launch_bounds__(TC_THREADS) estep_reduce_tc_kernel(ReduceArgs a, int* err)
{
    extern __shared__ __align__(1024) float sm[];
    const int p = a.D.p, q = a.D.q, g = a.D.g;
    const long long n = a.D.n;
    const int S = stats_per_comp(p, q);
    const int W = p + q + 1;             // B rows per component
    const int NP = (g * W + 15) / 16 * 16;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    float* buf[2][4];
    {
        float* o = sm;
        for (int b = 0; b < 2; ++b) {
            buf[b][0] = o; o += TC_M * TC_SUB;   // Ahi
            buf[b][1] = o; o += TC_M * TC_SUB;   // Alo
            buf[b][2] = o; o += NP * TC_SUB;     // Bhi
            buf[b][3] = o; o += NP * TC_SUB;     // Blo
        }
    }
    float* sy = sm + 2 * (2 * TC_M + 2 * NP) * TC_SUB;  // 16 x p
    float* stau = sy + TC_SUB * p;                       // g x 16
    float* su = stau + g * TC_SUB;                       // g x 16
    float* seu = su + g * TC_SUB;                        // g x 16 x q
    float* smu = seu + g * TC_SUB * q;                   // g x p (FP32 means)
    int* arow = (int*)(smu + g * p);                     // A row r: (h << 8 | a), or -1
    int* brow = arow + TC_M;                             // B row r: (h << 16 | c << 8 | kind), or -1
    uint64_t* mbar = (uint64_t*)(((uintptr_t)(brow + NP) + 15) & ~(uintptr_t)15);
    uint32_t* tmem_slot = (uint32_t*)(mbar + 2);
    const int ncols = NP <= 32 ? 32 : NP <= 64 ? 64 : NP <= 128 ? 128 : 256;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    for (int i = t; i < g * p; i += TC_THREADS) smu[i] = (float)a.mu[i];
    // row tables (kind 0: w r_c, 1: tau eu_c, 2: w); the mean index h p + c is packed in A
    for (int r = t; r < TC_M; r += TC_THREADS) arow[r] = r < g * p ? ((r / p) * p + r % p) << 8 | (r % p) : -1;
    for (int r = t; r < NP; r += TC_THREADS) {
        if (r >= g * W) { brow[r] = -1; continue; }
        const int h = r / W, c = r % W;
        brow[r] = c < p ? (h << 16 | c << 8 | 0) : c < p + q ? (h << 16 | (c - p) << 8 | 1) : (h << 16 | 2);
    }
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_slot;
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(NP >> 3) << 17) |
                           ((uint32_t)(TC_M >> 4) << 24);
    uint32_t uses[2] = {0, 0};  // completed commits expected per buffer
    bool ok = true;
    const int chunk = a.chunk;  // a multiple of 32
    const long long nblk = (n + chunk - 1) / chunk;
    // the sub-chunk inputs this thread stages: y (16 p <= 512: 2 per thread), tau and u
    // (16 g <= 256: 1), eu (16 g q <= 2048: 8); loaded one sub-chunk ahead into registers
    float pf_y[2], pf_tau = 0.f, pf_u = 0.f, pf_eu[8];
    auto prefetch = [&](long long js, long long jend) {
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int i = t + u * TC_THREADS;
            const long long j = js + i / p;
            pf_y[u] = (i < TC_SUB * p && j < jend) ? a.y32[(size_t)j * p + i % p] : 0.0f;
        }
        {
            const int h = t / TC_SUB;
            const long long j = js + (t % TC_SUB);
            const bool live = t < g * TC_SUB && j < jend;
            pf_tau = live ? (float)a.tau[(size_t)h * n + j] : 0.0f;
            pf_u = !live ? 0.0f : a.pr32 ? a.pr32[((size_t)h * n + j) * pr32_width(q)] : (float)a.u[(size_t)h * n + j];
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int i = t + u * TC_THREADS;  // (h, jj, k) with k fastest
            const int h = i / (TC_SUB * q), jj = (i / q) % TC_SUB, k = i % q;
            const long long j = js + jj;
            pf_eu[u] = !(i < g * TC_SUB * q && j < jend) ? 0.0f
                     : a.pr32 ? a.pr32[((size_t)h * n + j) * pr32_width(q) + 2 + k]
                              : (float)a.eu[((size_t)h * n + j) * q + k];
        }
    };
    auto stage = [&]() {
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int i = t + u * TC_THREADS;
            if (i < TC_SUB * p) sy[i] = pf_y[u];
        }
        if (t < g * TC_SUB) {
            stau[t] = pf_tau;
            su[t] = pf_u;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int i = t + u * TC_THREADS;
            if (i < g * TC_SUB * q) seu[i] = pf_eu[u];
        }
    };
    long long sub = 0;  // sub-chunks issued by this CTA
    {
        const long long j0 = (long long)blockIdx.x * chunk;
        if (j0 < n) prefetch(j0, j0 + chunk < n ? j0 + chunk : n);
    }
    for (long long blk = blockIdx.x; blk < nblk && ok; blk += gridDim.x) {
        const long long j0 = blk * chunk;
        const long long jend = j0 + chunk < n ? j0 + chunk : n;  // this block's observations
        const int nsub = chunk / TC_SUB;
        for (int sc = 0; sc < nsub && ok; ++sc, ++sub) {
            const int b = (int)(sub & 1);
            const long long js = j0 + sc * TC_SUB;
            const int kvalid = (int)(jend - js < TC_SUB ? jend - js : TC_SUB);  // observations here
            // this sub-chunk's inputs into shared memory (the previous build has finished
            // reading them: it ended in a barrier), then wait until the tensor core has
            // finished with buffer b; the vote keeps a wait that ran out on some threads from
            // splitting the block
            stage();
            const bool w = uses[b] == 0 || mbar_wait(smem_u32(&mbar[b]), (uses[b] - 1) & 1);
            if (!__syncthreads_and(w)) { ok = false; break; }
            // the next sub-chunk's loads fly while this one is built
            {
                long long nj0 = j0, njs = js + TC_SUB, nend = jend;
                if (sc + 1 == nsub) {  // the CTA's next block
                    nj0 = (blk + gridDim.x) * chunk;
                    njs = nj0;
                    nend = nj0 + chunk < n ? nj0 + chunk : n;
                }
                if (njs < n) prefetch(njs, nend);
            }
            // A: r_hj,a = y_ja - mu_ha (rows h*p + a); B: w r | tau eu | w (rows h*W + b)
            float* Ahi = buf[b][0];
            float* Alo = buf[b][1];
            float* Bhi = buf[b][2];
            float* Blo = buf[b][3];
#pragma unroll 4
            for (int i = t; i < TC_M * TC_SUB; i += TC_THREADS) {
                const int r = i >> 4, k = i & (TC_SUB - 1);
                const int info = arow[r];
                float x = 0.0f;
                if (info >= 0 && k < kvalid) x = sy[k * p + (info & 255)] - smu[info >> 8];
                const float hi = tf32_rn(x);
                const int o = tc_off(r, k, TC_M);
                Ahi[o] = hi;
                Alo[o] = x - hi;
            }
#pragma unroll 4
            for (int i = t; i < NP * TC_SUB; i += TC_THREADS) {
                const int r = i >> 4, k = i & (TC_SUB - 1);
                const int info = brow[r];
                float x = 0.0f;
                if (info >= 0 && k < kvalid) {
                    const int h = info >> 16, c = (info >> 8) & 255, kind = info & 3;
                    const float tv = stau[h * TC_SUB + k], wv = tv * su[h * TC_SUB + k];
                    if (kind == 0) x = wv * (sy[k * p + c] - smu[h * p + c]);
                    else if (kind == 1) x = tv * seu[(h * TC_SUB + k) * q + c];
                    else x = wv;
                }
                const float hi = tf32_rn(x);
                const int o = tc_off(r, k, NP);
                Bhi[o] = hi;
                Blo[o] = x - hi;
            }
            asm volatile("fence.proxy.async.shared::cta;");  // the generic-proxy writes, to the tensor core
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncthreads();
            if (t == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;");
                for (int ks = 0; ks < 2; ++ks) {
                    const uint64_t ah = smem_desc(smem_u32(Ahi + ks * TC_M * 8), 128, 256);
                    const uint64_t al = smem_desc(smem_u32(Alo + ks * TC_M * 8), 128, 256);
                    const uint64_t bh = smem_desc(smem_u32(Bhi + ks * NP * 8), 128, 256);
                    const uint64_t bl = smem_desc(smem_u32(Blo + ks * NP * 8), 128, 256);
                    const uint32_t first = (sc == 0 && ks == 0) ? 0u : 1u;  // a new block starts from 0
                    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
                                 "l"(ah), "l"(bh), "r"(idesc), "r"(first));
                    asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, 1;" ::"r"(tmem), "l"(ah),
                                 "l"(bl), "r"(idesc));
                    asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, 1;" ::"r"(tmem), "l"(al),
                                 "l"(bh), "r"(idesc));
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_u32(&mbar[b])));
            }
            ++uses[b];
        }
        if (!ok) break;
        // the block's accumulator: wait for its last commit, then rows (h, a) of D
        {
            const int b = (int)((sub - 1) & 1);
            const bool w = mbar_wait(smem_u32(&mbar[b]), (uses[b] - 1) & 1);
            if (!__syncthreads_and(w)) { ok = false; break; }
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (warp < 4) {
            const int row = warp * 32 + lane;
            const bool live = row < g * p;
            const int h = live ? row / p : 0, ra = live ? row % p : 0;
            double* out = a.partial + (size_t)blk * (g * S + 1) + (size_t)h * S;
            const int fSr = 3, fSre = 3 + p + q, fSrr = 3 + p + q + p * q + q * q;
            const int c0 = h * W;  // this row's block of columns
            for (int cb = 0; cb < NP; cb += 32) {
                float v[32];
                tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cb, v);
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const int c = cb + i - c0;
                    if (!live || c < 0 || c >= W) continue;
                    const double d = (double)v[i];
                    if (c < p) {
                        if (c <= ra) {  // lower triangle, mirrored: Srr exactly symmetric
                            out[fSrr + ra * p + c] = d;
                            out[fSrr + c * p + ra] = d;
                        }
                    } else if (c < p + q) {
                        out[fSre + ra * q + (c - p)] = d;
                    } else {
                        out[fSr + ra] = d;
                    }
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();  // the readout is complete before the next block's first MMA
    }
    if (!ok && lane == 0) atomicOr(err, KF_TIMEOUT);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
}

cudaError_t launch_reduce_tc(const ReduceArgs& a, int* flags, int nsm, cudaStream_t st)
{
    const size_t smem = reduce_tc_smem(a.D.p, a.D.q, a.D.g);
    cudaError_t e = cudaFuncSetAttribute(estep_reduce_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long long nblk = (a.D.n + a.chunk - 1) / a.chunk;
    const int grid = (int)(nblk < 2LL * nsm ? nblk : 2LL * nsm);
    estep_reduce_tc_kernel<<<grid, TC_THREADS, smem, st>>>(a, flags);
    return cudaGetLastError();
}
