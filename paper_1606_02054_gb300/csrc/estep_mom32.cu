// estep_mom32.cu -- lattice T_k with truncated moments (single-pass ratio
// estimators), k = 3..8, in float: warp per record, lattice points over lanes
// (see tk_lattice_mom_warp in special.cuh).
#include "internal.cuh"
#include "special.cuh"

// Blocks of 4 warps.  K = 7, 8 need 147-168 registers: 3 such blocks (12 warps) share an
// SM where one block of 8 would leave it at 8.
template <int K>
__host__ __device__ constexpr int mom32_block() { return K >= 7 || K <= 4 ? 128 : 256; }
// Minimum resident blocks (an explicit 1 would let ptxas take up to 255 registers: K = 6
// went from 128 to 154, halving its resident warps).  K <= 4 with P lattice points in flight
// per lane: P = 1: 7 blocks (72 registers), P = 2: 5 (92); K = 5, 6: 2 (128); K = 7, 8: 3
// (170).  Measured at flow_p4 (K = 4, 8e5 records): P = 1 40.4 ms, P = 2 39.1 ms.
template <int K, int P>
__host__ __device__ constexpr int mom32_minb() { return K <= 4 ? (P == 1 ? 7 : 5) : (K <= 6 ? 2 : 3); }

template <int K, bool SEL, bool LW, int P>
__global__ void __launch_bounds__(mom32_block<K>(), mom32_minb<K, P>()) lattice_mom_kernel_32(RecSet r, IntegArgs a)
{
    constexpr int W = K + K * (K + 1) / 2;
    const int lane = threadIdx.x & (CF_WARP - 1);
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const size_t NM = (size_t)a.lat.N * a.lat.M;
    __shared__ double slot[mom32_block<K>() / CF_WARP][W + 3 + CF_MAXSHIFT];
    double* acc = slot[threadIdx.x >> 5];
    const long long nr = rec_count<SEL>(r);
    for (long long t = warp; t < nr; t += nwarps) {
        const long long i = rec_index<SEL>(r, t);
        double bt[K];
#pragma unroll
        for (int k = 0; k < K; ++k) bt[k] = r.bt[i * K + k];
        // the pass of alpha_s (chi table at dof k1 = dof - 2) weighted to dof k2 = r.dof
        const float k2 = (float)r.dof[i];
        const float rk = isinf(k2) ? 1.0f : sqrtf(k2 / (k2 - 2.0f));
        double as = 0.0, se = 0.0, lw = 0.0;
        const float* lchi = LW ? a.lchi32 + (size_t)r.tab[i] * NM : nullptr;
        // the coordinate table only at K <= 4 (one float4 per point); at K = 6 it measured
        // 1.6x slower than advancing the coordinates
        double v;
        if constexpr (K <= 4)
            v = tk_lattice_mom_f32<K, true, P, LW>(bt, a.F + r.fac[i], a.chi32 + (size_t)r.tab[i] * NM,
                                                          a.shf32, a.lat, lane, acc, rk, &as, &se, a.wtab, lchi, &lw);
        else
            v = tk_lattice_mom_f32<K, false, 1, LW>(bt, a.F + r.fac[i], a.chi32 + (size_t)r.tab[i] * NM, a.shf32,
                                                    a.lat, lane, acc, rk, &as, &se, nullptr, lchi, &lw);
        if (lane == 0) {
            r.res[i] = v;
            if (r.res0) r.res0[i] = as;
            if (r.se0) r.se0[i] = se;
            if (LW) r.lw[i] = lw;
        }
        for (int k = lane; k < W; k += CF_WARP) r.mom[i * W + k] = acc[1 + k];
        __syncwarp();  // the slot is reset by the next record
    }
}

// the selection-list instantiation only where a list is given
template <int K, int P>
static void go_p(const RecSet& r, const IntegArgs& a, int blocks, int threads, cudaStream_t st)
{
    // exact E[log W] (r.lw) only without a selection list (the surrogate excludes it)
    if (r.sel) lattice_mom_kernel_32<K, true, false, P><<<blocks, threads, 0, st>>>(r, a);
    else if (r.lw) lattice_mom_kernel_32<K, false, true, P><<<blocks, threads, 0, st>>>(r, a);
    else lattice_mom_kernel_32<K, false, false, P><<<blocks, threads, 0, st>>>(r, a);
}

// points in flight per lane: a.mom_p (1 or 2) with the coordinate table (K <= 4), else 1
template <int K>
static void go(const RecSet& r, const IntegArgs& a, int blocks, int threads, cudaStream_t st)
{
    if constexpr (K <= 4) {
        if (a.mom_p == 1) go_p<K, 1>(r, a, blocks, threads, st);
        else go_p<K, 2>(r, a, blocks, threads, st);
    } else {
        go_p<K, 1>(r, a, blocks, threads, st);
    }
}

cudaError_t launch_mom32(int k, const RecSet& r, const IntegArgs& a, int blocks, cudaStream_t st)
{
    switch (k) {
    case 3: go<3>(r, a, 2 * blocks, 128, st); break;  // same warps
    case 4: go<4>(r, a, 2 * blocks, 128, st); break;
    case 5: go<5>(r, a, blocks, 256, st); break;
    case 6: go<6>(r, a, blocks, 256, st); break;
    case 7: go<7>(r, a, 2 * blocks, 128, st); break;  // same warps
    case 8: go<8>(r, a, 2 * blocks, 128, st); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}
