// mlp_tc.cuh -- the surrogate's inference over a record set on the tensor cores
// (tcgen05.mma kind::f16, BF16 operands, FP32 accumulators in tensor memory).
// Included by mlp.cu (it uses InferArgs and sur_features there).
//
// A CTA takes tiles of 128 records (one per tensor-memory lane).  Per tile:
//   features -> A (128 x 48, BF16, shared) -> D = A W1 (128 x 256 FP32, tensor memory)
//   -> tanh(D + b1) as BF16 into A (128 x 256) -> D = A W2 -> ... W3 -> D = A W4 (128 x 48)
//   -> outputs (log T_q, the moments) per record.
// W1 and W4 stay in shared memory; W2 and W3 stream through a ring of four 16 KB slots
// (32 K-columns of all 256 outputs each) by bulk copies, the weights having been packed
// in global memory in that very layout (mlp_tc_pack_kernel).  Thread 0 issues the copies
// and the MMAs; it refills a slot as soon as the MMAs that read it have completed (its
// commit barrier), after queueing the next slot's MMAs, so the tensor core is not left
// idle by the refill.  The 8 warps run the epilogues: warp w reads tensor-memory lanes
// 32 (w mod 4) .. + 31 (its rows) and columns 128 (w / 4) .. + 127.
// Every barrier wait is bounded; a CTA whose wait runs out sets KF_TIMEOUT, drains its
// copies and MMAs, frees its tensor memory and leaves.
#include "tc_ptx.cuh"

constexpr int TCI_THREADS = 256;
constexpr int TCI_M = 128;                                 // records per tile
constexpr int TCI_CK = 32;                                 // K-columns of W2 / W3 per chunk
constexpr int TCI_CHUNKS = 2 * MLP_H / TCI_CK;             // chunks per tile: W2, then W3
constexpr int TCI_SLOTS = 4;
constexpr int TCI_TMEM_COLS = 256;
constexpr size_t TCI_ACT = (size_t)TCI_M * MLP_H * 2;       // activations, BF16
constexpr size_t TCI_W1 = (size_t)MLP_H * MLP_IN * 2;       // W1^T (256 x 48)
constexpr size_t TCI_W4 = (size_t)MLP_OUT * MLP_H * 2;      // W4^T (48 x 256)
constexpr size_t TCI_CH = (size_t)MLP_H * TCI_CK * 2;       // one chunk (256 x 32)
constexpr size_t TCI_WTC = TCI_W1 + TCI_W4 + (size_t)TCI_CHUNKS * TCI_CH;  // packed weights
constexpr size_t TCI_FLOATS = 3 * MLP_H + MLP_OUT + MLP_NSTAT;
constexpr int TCI_NBAR = 2 * TCI_SLOTS + 3;                 // full, empty, acc, static weights, final
constexpr size_t TCI_SMEM = TCI_ACT + TCI_W1 + TCI_W4 + TCI_SLOTS * TCI_CH + sizeof(float) * TCI_FLOATS +
                            8 * TCI_NBAR + 16 + 1024;      // + the 1 KB alignment of the base
static_assert(MLP_IN % 16 == 0 && MLP_H % TCI_CK == 0 && MLP_OUT % 16 == 0, "tile shapes");

// W^T of each layer (rows = outputs n, columns = inputs k: the K-major B operand) in the
// canonical layout: [W1 (256 x 48)][W4 (48 x 256)][W2 chunks 0..7][W3 chunks 0..7], chunk
// c holding inputs 32 c .. 32 c + 31 of all 256 outputs.
__global__ void mlp_tc_pack_kernel(const float* __restrict__ theta, bf16_t* __restrict__ wtc)
{
    const long long n1 = (long long)MLP_H * MLP_IN, n4 = (long long)MLP_OUT * MLP_H, n2 = (long long)MLP_H * MLP_H;
    const long long tot = n1 + n4 + 2 * n2;
    const long long o4 = TCI_W1 / 2, o2 = (TCI_W1 + TCI_W4) / 2, och = TCI_CH / 2;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        long long dst;
        float v;
        if (e < n1) {
            const int n = (int)(e / MLP_IN), k = (int)(e % MLP_IN);
            v = theta[MLP_W1 + (long long)k * MLP_H + n];
            dst = tcx::bf16_canon(n, k, MLP_H);
        } else if (e < n1 + n4) {
            const long long x = e - n1;
            const int n = (int)(x / MLP_H), k = (int)(x % MLP_H);
            v = theta[MLP_W4 + (long long)k * MLP_OUT + n];
            dst = o4 + tcx::bf16_canon(n, k, MLP_OUT);
        } else {
            const long long x = e - n1 - n4;
            const int l = (int)(x / n2);  // 0: W2, 1: W3
            const long long y = x % n2;
            const int n = (int)(y / MLP_H), k = (int)(y % MLP_H);
            v = theta[(l ? MLP_W3 : MLP_W2) + (long long)k * MLP_H + n];
            dst = o2 + (long long)(l * (MLP_H / TCI_CK) + k / TCI_CK) * och + tcx::bf16_canon(n, k % TCI_CK, MLP_H);
        }
        wtc[dst] = to_bf16(v);
    }
}

__global__ void __launch_bounds__(TCI_THREADS, 1) mlp_infer_tc_kernel(InferArgs a, const bf16_t* __restrict__ wtc,
                                                                     int* err)
{
    using namespace tcx;
    extern __shared__ unsigned char tsm_raw[];
    unsigned char* tsm = (unsigned char*)(((uintptr_t)tsm_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* act = tsm;
    unsigned char* w1s = act + TCI_ACT;
    unsigned char* w4s = w1s + TCI_W1;
    unsigned char* ring = w4s + TCI_W4;
    float* s_bias = (float*)(ring + TCI_SLOTS * TCI_CH);
    float* s_stat = s_bias + 3 * MLP_H + MLP_OUT;
    uint64_t* bars = (uint64_t*)(s_stat + MLP_NSTAT);
    uint32_t* tslot = (uint32_t*)(bars + TCI_NBAR);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + TCI_SLOTS);
    const uint32_t accb = smem_u32(bars + 2 * TCI_SLOTS), wbar = accb + 8, finb = accb + 16;
    const uint32_t act_u = smem_u32(act), w1_u = smem_u32(w1s), w4_u = smem_u32(w4s), ring_u = smem_u32(ring);
    const long long nrec = a.r.nrec;
    const long long ntiles = (nrec + TCI_M - 1) / TCI_M;
    const long long my_tiles = (long long)blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const long long total_chunks = my_tiles * TCI_CHUNKS;
    const char* wsrc = (const char*)wtc;

    for (int e = t; e < MLP_H; e += TCI_THREADS) {
        s_bias[e] = a.theta[MLP_B1 + e];
        s_bias[MLP_H + e] = a.theta[MLP_B2 + e];
        s_bias[2 * MLP_H + e] = a.theta[MLP_B3 + e];
    }
    for (int e = t; e < MLP_OUT; e += TCI_THREADS) s_bias[3 * MLP_H + e] = a.theta[MLP_B4 + e];
    for (int e = t; e < MLP_NSTAT; e += TCI_THREADS) s_stat[e] = a.stats[e];
    if (warp == 0) tmem_alloc(smem_u32(tslot), TCI_TMEM_COLS);
    if (t == 0) {
        for (int s = 0; s < TCI_SLOTS; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        mbar_init(accb, 1);
        mbar_init(wbar, 1);
        mbar_init(finb, 1);
        mbar_init_fence();
    }
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = *tslot;

    bool ok = true;
    long long issued = 0, consumed = 0;  // weight chunks (thread 0)
    if (t == 0 && my_tiles > 0) {
        mbar_arrive_expect_tx(wbar, (uint32_t)(TCI_W1 + TCI_W4));
        bulk_g2s(w1_u, wsrc, (uint32_t)TCI_W1, wbar);
        bulk_g2s(w4_u, wsrc + TCI_W1, (uint32_t)TCI_W4, wbar);
        for (; issued < TCI_SLOTS && issued < total_chunks; ++issued) {
            const int s = (int)issued;
            mbar_arrive_expect_tx(full0 + 8 * s, (uint32_t)TCI_CH);
            bulk_g2s(ring_u + s * (uint32_t)TCI_CH, wsrc + TCI_W1 + TCI_W4 + (issued % TCI_CHUNKS) * TCI_CH,
                     (uint32_t)TCI_CH, full0 + 8 * s);
        }
    }
    const float* fmean = s_stat;
    const float* fstd = s_stat + MLP_IN;
    const float* zlo = s_stat + 2 * MLP_IN;
    const float* zhi = s_stat + 3 * MLP_IN;
    const float* tmean = s_stat + 4 * MLP_IN;
    const float* tstd = tmean + MLP_OUT;
    const uint32_t id_h = idesc_bf16(TCI_M, MLP_H), id_o = idesc_bf16(TCI_M, MLP_OUT);
    const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
    const int q = a.q, W = q + q * (q + 1) / 2;
    uint32_t acc_phase = 0;
    bool wready = false;

    for (long long kt = 0; kt < my_tiles; ++kt) {
        const long long base = ((long long)blockIdx.x + kt * gridDim.x) * TCI_M;
        // features of row t (warps 0-3), standardised, BF16 into A (K = 48)
        int inbox = 0;
        if (t < TCI_M) {
            const long long i = base + t;
            float z[MLP_IN];
#pragma unroll
            for (int k = 0; k < MLP_IN; ++k) z[k] = 0.0f;
            if (i < nrec) {
                float f[MLP_IN];
                const int nin = sur_features(q, a.r.bt + i * q, a.F + a.r.fac[i], a.r.dof[i], f);
                inbox = 1;
                for (int k = 0; k < nin; ++k) {
                    z[k] = (f[k] - fmean[k]) / fstd[k];
                    // in range: the training range widened by margin standard deviations
                    if (!(z[k] >= zlo[k] - a.margin && z[k] <= zhi[k] + a.margin)) inbox = 0;
                }
            }
#pragma unroll
            for (int c8 = 0; c8 < MLP_IN / 8; ++c8) {
                const uint4 v = make_uint4(pack_bf16(z[8 * c8], z[8 * c8 + 1]), pack_bf16(z[8 * c8 + 2], z[8 * c8 + 3]),
                                           pack_bf16(z[8 * c8 + 4], z[8 * c8 + 5]), pack_bf16(z[8 * c8 + 6], z[8 * c8 + 7]));
                *(uint4*)(act + 2 * bf16_canon(t, 8 * c8, TCI_M)) = v;
            }
        }
        fence_async_smem();
        tc_before_sync();
        __syncthreads();
        if (t == 0) {  // layer 1: K = 48, three K-slices
            tc_after_sync();
            if (!wready) {
                ok = mbar_wait(wbar, 0) && ok;
                wready = true;
            }
#pragma unroll
            for (int ks = 0; ks < MLP_IN / 16; ++ks)
                umma_bf16(tmem, smem_desc(act_u + ks * (TCI_M * 32), 128, 256),
                         smem_desc(w1_u + ks * (MLP_H * 32), 128, 256), id_h, ks > 0);
            mma_commit(accb);
        }
        for (int layer = 0; layer < 3; ++layer) {
            // epilogue of hidden layer `layer` (D + b, tanh, BF16 into A), then the next layer's MMAs
            ok = mbar_wait(accb, acc_phase) && ok;
            acc_phase ^= 1;
            tc_after_sync();
            {
                const int row = 32 * (warp & 3) + lane, cb = 128 * (warp >> 2);
                const float* bias = s_bias + layer * MLP_H;
#pragma unroll 1
                for (int cc = 0; cc < 128; cc += 32) {
                    float v[32];
                    tmem_ld32(tmem + lane_base + (uint32_t)(cb + cc), v);
                    uint32_t pk[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        pk[j] = pack_bf16(tanhf(v[2 * j] + bias[cb + cc + 2 * j]),
                                          tanhf(v[2 * j + 1] + bias[cb + cc + 2 * j + 1]));
#pragma unroll
                    for (int g8 = 0; g8 < 4; ++g8)
                        *(uint4*)(act + 2 * bf16_canon(row, cb + cc + 8 * g8, TCI_M)) =
                            make_uint4(pk[4 * g8], pk[4 * g8 + 1], pk[4 * g8 + 2], pk[4 * g8 + 3]);
                }
            }
            fence_async_smem();
            tc_before_sync();
            __syncthreads();
            if (t == 0) {
                tc_after_sync();
                if (layer < 2) {
                    // layer 2 or 3: eight streamed chunks of two K-slices
                    for (int c = 0; c < MLP_H / TCI_CK; ++c) {
                        const int s = (int)(consumed % TCI_SLOTS);
                        ok = mbar_wait(full0 + 8 * s, (uint32_t)((consumed / TCI_SLOTS) & 1)) && ok;
                        tc_after_sync();
#pragma unroll
                        for (int kk = 0; kk < TCI_CK / 16; ++kk) {
                            const int ks = c * (TCI_CK / 16) + kk;
                            umma_bf16(tmem, smem_desc(act_u + ks * (TCI_M * 32), 128, 256),
                                     smem_desc(ring_u + s * (uint32_t)TCI_CH + kk * (MLP_H * 32), 128, 256), id_h, ks > 0);
                        }
                        mma_commit(empty0 + 8 * s);
                        ++consumed;
                        // the previous chunk's slot, once its MMAs are done, takes chunk `issued`
                        if (consumed >= 2 && issued < total_chunks) {
                            const long long prev = consumed - 2;
                            const int sp = (int)(prev % TCI_SLOTS);
                            ok = mbar_wait(empty0 + 8 * sp, (uint32_t)((prev / TCI_SLOTS) & 1)) && ok;
                            mbar_arrive_expect_tx(full0 + 8 * sp, (uint32_t)TCI_CH);
                            bulk_g2s(ring_u + sp * (uint32_t)TCI_CH,
                                     wsrc + TCI_W1 + TCI_W4 + (issued % TCI_CHUNKS) * TCI_CH, (uint32_t)TCI_CH,
                                     full0 + 8 * sp);
                            ++issued;
                        }
                    }
                } else {
                    // output layer: N = 48 from the resident W4, sixteen K-slices
#pragma unroll 4
                    for (int ks = 0; ks < MLP_H / 16; ++ks)
                        umma_bf16(tmem, smem_desc(act_u + ks * (TCI_M * 32), 128, 256),
                                 smem_desc(w4_u + ks * (MLP_OUT * 32), 128, 256), id_o, ks > 0);
                }
                mma_commit(accb);
            }
        }
        // outputs of row t (warps 0-3)
        ok = mbar_wait(accb, acc_phase) && ok;
        acc_phase ^= 1;
        tc_after_sync();
        if (warp < 4) {
            float o[MLP_OUT];
            tmem_ld32(tmem + lane_base, o);
            tmem_ld16(tmem + lane_base + 32, o + 32);
            const long long i = base + t;
            if (i < nrec) {
                if (a.mark && a.moments) a.mark[i] = inbox ? 0 : 1;
                if (inbox) {
#pragma unroll
                    for (int k = 0; k < MLP_OUT; ++k) o[k] = (o[k] + s_bias[3 * MLP_H + k]) * tstd[k] + tmean[k];
                    a.r.res[i] = exp((double)o[0]);
                    if (a.r.se) a.r.se[i] = 0.0;
                    if (a.moments) {
                        // m1 and E[X X^T] = L L^T + m1 m1^T, L with exp of its predicted log diagonal
                        float L[CF_MAXQ * (CF_MAXQ + 1) / 2];
                        for (int r2 = 0, k = 1 + q; r2 < q; ++r2)
                            for (int c2 = 0; c2 <= r2; ++c2, ++k) L[r2 * (r2 + 1) / 2 + c2] = r2 == c2 ? expf(o[k]) : o[k];
                        double* out = a.r.mom + i * W;
                        for (int k = 0; k < q; ++k) out[k] = (double)o[1 + k];
                        for (int r2 = 0; r2 < q; ++r2)
                            for (int c2 = 0; c2 <= r2; ++c2) {
                                float sm = o[1 + r2] * o[1 + c2];
                                for (int l = 0; l <= c2; ++l) sm += L[r2 * (r2 + 1) / 2 + l] * L[c2 * (c2 + 1) / 2 + l];
                                out[q + r2 * (r2 + 1) / 2 + c2] = (double)sm;
                            }
                    }
                } else if (!(a.mark && !a.moments && a.mark[i])) {
                    a.fall[atomicAdd(a.nfall, 1)] = (int)i;
                }
            }
        }
        tc_before_sync();
        if (__syncthreads_or(!ok)) {  // a wait ran out: leave (the host reports the error)
            if (t == 0) atomicOr(err, KF_TIMEOUT);
            break;
        }
    }
    // drain: copies issued but not consumed, and every MMA issued, before the memory goes
    if (t == 0) {
        for (long long c = consumed; c < issued; ++c)
            mbar_wait(full0 + 8 * (int)(c % TCI_SLOTS), (uint32_t)((c / TCI_SLOTS) & 1));
        if (my_tiles > 0 && !wready) mbar_wait(wbar, 0);
        mma_commit(finb);
        mbar_wait(finb, 0);
    }
    tc_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, TCI_TMEM_COLS);
}
