// estep_t2.cu -- T_2 records (warp per record, quadrature nodes over lanes).
#include "internal.cuh"
#include "special.cuh"

template <typename R>
__global__ void __launch_bounds__(256) t2_records_kernel(RecSet r, IntegArgs a)
{
    const int lane = threadIdx.x & (CF_WARP - 1);
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const bool f32 = sizeof(R) == sizeof(float);
    const R* glx = f32 ? (const R*)a.glx32 : (const R*)a.glx64;
    const R* glw = f32 ? (const R*)a.glw32 : (const R*)a.glw64;
    const R* cst = f32 ? (const R*)a.cst32 : (const R*)a.cst64;
    unsigned long long nodes = 0;  // this warp's quadrature nodes (profiler count)
    for (long long i = warp; i < r.nrec; i += nwarps) {
        const R* c = cst + r.tab[i] * CST_STRIDE;
        R h, k, rho, nu, omr2, cr;
        if (f32 && r.t2f) {
            // FP32 record fields written by the plan: no FP64 instruction here
            const float4 u0 = r.t2f[2 * i], u1 = r.t2f[2 * i + 1];
            h = u0.x; k = u0.y; rho = u0.z; nu = u0.w; omr2 = u1.x; cr = u1.y;
        } else {
            const double h64 = r.bt[2 * i], k64 = r.bt[2 * i + 1];
            const double rho64 = a.F[r.fac[i] + 2];  // L[1][0] of the 2 x 2 correlation factor
            h = (R)h64; k = (R)k64; rho = (R)rho64; nu = (R)r.dof[i];
            omr2 = (R)((1.0 - rho64) * (1.0 + rho64));
            cr = (R)(h64 * (rho64 > 0.0 ? rho64 : -rho64) - (rho64 > 0.0 ? k64 : -k64));
        }
        const float2* tab = f32 && a.t1tab ? a.t1tab + (size_t)r.tab[i] * T1TAB_N : nullptr;
        int nn = 2 * a.t2n;
        const double v = isinf(nu) ? phi2_warp<R>(h, k, rho, a.t2n, glx, glw, lane)
                                   : t2cdf_warp<R>(h, k, rho, nu, omr2, cr, c[CST_LGB], c[CST_LGB1], c[CST_C2], a.t2n,
                                       glx, glw, f32 ? T2_NH : a.t2n,
                                       f32 ? (const R*)a.glx32h : glx, f32 ? (const R*)a.glw32h : glw,
                                       lane, tab, &nn, f32 ? a.t2n_lo : 0, f32 ? (const R*)a.glx32l : nullptr,
                                       f32 ? (const R*)a.glw32l : nullptr);
        nodes += (unsigned long long)nn;
        if (lane == 0) {
            r.res[i] = v;
            if (r.se) r.se[i] = 0.0;
        }
    }
    if (a.nodes && lane == 0 && nodes) atomicAdd(a.nodes, nodes);
}

// FP32 T_2 records (finite dof) on groups of L lanes: 32/L records per warp at a time.
// The record loop is uniform over the warp (a group past the last record evaluates the
// last record again and writes nothing), so the group reductions see all 32 lanes.
template <int L>
__global__ void __launch_bounds__(256) t2_records_group_kernel(RecSet r, IntegArgs a)
{
    constexpr int G = CF_WARP / L;
    const int lane = threadIdx.x & (CF_WARP - 1);
    const int sub = lane & (L - 1), grp = lane / L;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    unsigned long long nodes = 0;  // this group's quadrature nodes (profiler count)
    for (long long base = warp * G; base < r.nrec; base += nwarps * G) {
        const long long want = base + grp;
        const bool own = want < r.nrec;
        const long long i = own ? want : r.nrec - 1;
        const float* c = a.cst32 + r.tab[i] * CST_STRIDE;
        float h, k, rho, nu, omr2, cr;
        if (r.t2f) {
            const float4 u0 = r.t2f[2 * i], u1 = r.t2f[2 * i + 1];
            h = u0.x; k = u0.y; rho = u0.z; nu = u0.w; omr2 = u1.x; cr = u1.y;
        } else {
            const double h64 = r.bt[2 * i], k64 = r.bt[2 * i + 1];
            const double rho64 = a.F[r.fac[i] + 2];  // L[1][0] of the 2 x 2 correlation factor
            h = (float)h64; k = (float)k64; rho = (float)rho64; nu = (float)r.dof[i];
            omr2 = (float)((1.0 - rho64) * (1.0 + rho64));
            cr = (float)(h64 * (rho64 > 0.0 ? rho64 : -rho64) - (rho64 > 0.0 ? k64 : -k64));
        }
        const float2* tab = a.t1tab ? a.t1tab + (size_t)r.tab[i] * T1TAB_N : nullptr;
        int nn = 0;
        const double v = t2cdf_group_f32<L>(h, k, rho, nu, omr2, cr, c[CST_LGB], c[CST_LGB1], c[CST_C2], a.t2n,
                                            a.glx32, a.glw32, T2_NH, a.glx32h, a.glw32h, sub, tab, &nn,
                                            a.t2n_lo, a.glx32l, a.glw32l);
        if (own) {
            nodes += (unsigned long long)nn;
            if (sub == 0) {
                r.res[i] = v;
                if (r.se) r.se[i] = 0.0;
            }
        }
    }
    if (a.nodes && sub == 0 && nodes) atomicAdd(a.nodes, nodes);
}

// Lanes per FP32 T_2 record (finite dof), a.t2_group in {2, 4, 8, 16}; 32 (or 0: the CFUSN
// model's records) = the warp-per-record kernel.  Measured at p = 16, q = 2, g = 8,
// n = 2e6 (3.2e7 records, ~45 nodes each): 14.3 ms with 32 lanes, 9.6 with 16, 7.9 with 8,
// 7.1 with 4, 6.8 with 2.
template <int L>
static void go_group(const RecSet& r, const IntegArgs& a, int blocks, cudaStream_t st)
{
    // the same warps, each on 32/L records at a time
    const long long need = (r.nrec + 8LL * (CF_WARP / L) - 1) / (8LL * (CF_WARP / L));
    const int gb = (int)(need < blocks ? need : blocks);
    t2_records_group_kernel<L><<<gb > 0 ? gb : 1, 256, 0, st>>>(r, a);
}

cudaError_t launch_t2(const RecSet& r, const IntegArgs& a, int fp32, int blocks, cudaStream_t st)
{
    const int L = a.t2_group;
    if (fp32 && L == 2) go_group<2>(r, a, blocks, st);
    else if (fp32 && L == 4) go_group<4>(r, a, blocks, st);
    else if (fp32 && L == 8) go_group<8>(r, a, blocks, st);
    else if (fp32 && L == 16) go_group<16>(r, a, blocks, st);
    else if (fp32) {
        t2_records_kernel<float><<<blocks, 256, 0, st>>>(r, a);
    } else {
        t2_records_kernel<double><<<blocks, 256, 0, st>>>(r, a);
    }
    return cudaGetLastError();
}
