// estep_mom64.cu -- lattice T_k with truncated moments (single-pass ratio
// estimators), k = 3..8, in double: warp per record, lattice points over lanes
// (see tk_lattice_mom_warp in special.cuh).
#include "internal.cuh"
#include "special.cuh"

template <int K, bool SEL>
__global__ void __launch_bounds__(256) lattice_mom_kernel_64(RecSet r, IntegArgs a)
{
    constexpr int W = K + K * (K + 1) / 2;
    const int lane = threadIdx.x & (CF_WARP - 1);
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const size_t NM = (size_t)a.lat.N * a.lat.M;
    __shared__ double slot[8][W + 3 + CF_MAXSHIFT];
    double* acc = slot[threadIdx.x >> 5];
    const long long nr = rec_count<SEL>(r);
    for (long long t = warp; t < nr; t += nwarps) {
        const long long i = rec_index<SEL>(r, t);
        double bt[K];
#pragma unroll
        for (int k = 0; k < K; ++k) bt[k] = r.bt[i * K + k];
        // the pass of alpha_s (chi table at dof k1 = dof - 2) weighted to dof k2 = r.dof
        const double k2 = r.dof[i];
        const double rk = isinf(k2) ? double(1) : (double)sqrt(k2 / (k2 - 2.0));
        double as = 0.0, se = 0.0, lw = 0.0;
        const double* lchi = r.lw ? a.lchi64 + (size_t)r.tab[i] * NM : nullptr;
        const double v = tk_lattice_mom_warp<double, K>(bt, a.F + r.fac[i], a.chi64 + (size_t)r.tab[i] * NM,
                                                      a.shf64, a.lat, lane, acc, rk, &as, &se, lchi,
                                                      r.lw ? &lw : nullptr);
        if (lane == 0) {
            r.res[i] = v;
            if (r.res0) r.res0[i] = as;
            if (r.se0) r.se0[i] = se;
            if (r.lw) r.lw[i] = lw;
        }
        for (int k = lane; k < W; k += CF_WARP) r.mom[i * W + k] = acc[1 + k];
        __syncwarp();  // the slot is reset by the next record
    }
}

// the selection-list instantiation only where a list is given
template <int K>
static void go(const RecSet& r, const IntegArgs& a, int blocks, int threads, cudaStream_t st)
{
    if (r.sel) lattice_mom_kernel_64<K, true><<<blocks, threads, 0, st>>>(r, a);
    else lattice_mom_kernel_64<K, false><<<blocks, threads, 0, st>>>(r, a);
}

cudaError_t launch_mom64(int k, const RecSet& r, const IntegArgs& a, int blocks, cudaStream_t st)
{
    switch (k) {
    case 3: go<3>(r, a, blocks, 256, st); break;
    case 4: go<4>(r, a, blocks, 256, st); break;
    case 5: go<5>(r, a, blocks, 256, st); break;
    case 6: go<6>(r, a, blocks, 256, st); break;
    case 7: go<7>(r, a, blocks, 256, st); break;
    case 8: go<8>(r, a, blocks, 256, st); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}
