// estep_t2.cu -- T_2 records: a warp per record (quadrature nodes over lanes), or in FP32
// the records' quadrature pieces dealt to groups of lanes.
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
            if (r.res32) r.res32[i] = (float)v;
            else r.res[i] = v;
            if (r.se) r.se[i] = 0.0;
        }
    }
    if (a.nodes && lane == 0 && nodes) atomicAdd(a.nodes, nodes);
}

// FP32 T_2 records (finite dof), scheduled by quadrature piece.  A warp takes a chunk of
// 64 records; lane l sets up records l and l + 32 (the angles of the split and the pieces'
// lengths, once per record), the chunk's pieces (one or two per record, 24, 32 or 64
// nodes each) are ordered by node count and dealt to the warp's 32/L groups of L lanes,
// a group sums its piece's nodes (lane sub takes nodes sub, sub + L, ...), and the record's
// value is C_nu (piece 0 + piece 1).  Dealing pieces rather than records keeps the groups
// of a round on equal node counts: a record with one piece no longer idles its lanes
// while a neighbour's second piece runs.  The same L gives the same bits.
namespace {
constexpr int T2P_WARPS = 8;
constexpr int T2P_CH = 2 * CF_WARP;  // records per warp chunk
// a record's set-up fields, one array per field (consecutive records in distinct banks)
enum { T2F_ANC0, T2F_PHIS, T2F_L0, T2F_L1, T2F_D0, T2F_ZS, T2F_NU, T2F_LGB1, T2F_N };
constexpr int T2P_NMAX = 64;  // nodes per piece at most (t2_nodes <= 64, T2_NH = 64)
}  // namespace

// TAB: the inner T_1 from the per-dof tables (a.t1tab), else by its continued fraction
template <int L, bool TAB>
__global__ void __launch_bounds__(T2P_WARPS * CF_WARP, 4) t2_pieces_kernel(RecSet r, IntegArgs a)
{
    constexpr int G = CF_WARP / L;
    __shared__ float srf[T2P_WARPS][T2F_N][T2P_CH];
    __shared__ int srt[T2P_WARPS][T2P_CH], srk[T2P_WARPS][T2P_CH];  // table index, kind (0: t2n_lo
                                                                    // nodes, 1: t2n, 2: graded)
    __shared__ float sgx[3][T2P_NMAX], sgw[3][T2P_NMAX];            // the node sets by kind
    __shared__ float spsum[T2P_WARPS][T2P_CH][2];
    __shared__ unsigned char sitem[T2P_WARPS][2 * T2P_CH];  // (record << 1) | piece
    const int lane = threadIdx.x & (CF_WARP - 1), wib = threadIdx.x >> 5;
    const int sub = lane & (L - 1), grp = lane / L;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    float (*Rf)[T2P_CH] = srf[wib];
    int* Rt = srt[wib];
    int* Rk = srk[wib];
    float (*P)[2] = spsum[wib];
    unsigned char* items = sitem[wib];
    const int nlo = a.t2n_lo > 0 ? a.t2n_lo : a.t2n;
    for (int e = threadIdx.x; e < T2P_NMAX; e += blockDim.x) {
        sgx[0][e] = e < nlo && a.t2n_lo > 0 ? a.glx32l[e] : 0.0f;
        sgw[0][e] = e < nlo && a.t2n_lo > 0 ? a.glw32l[e] : 0.0f;
        sgx[1][e] = e < a.t2n ? a.glx32[e] : 0.0f;
        sgw[1][e] = e < a.t2n ? a.glw32[e] : 0.0f;
        sgx[2][e] = e < T2_NH ? a.glx32h[e] : 0.0f;
        sgw[2][e] = e < T2_NH ? a.glw32h[e] : 0.0f;
    }
    __syncthreads();
    unsigned long long nodes = 0;  // this lane's records' quadrature nodes (profiler count)
    for (long long base = warp * T2P_CH; base < r.nrec; base += nwarps * T2P_CH) {
        // phase 1: set-up of records lane and lane + 32
        int np[2], kind[2];
        float C2[2], lim[2];
        bool limit[2];
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            const int rr = lane + m * CF_WARP;
            const long long i = base + rr;
            np[m] = 0; kind[m] = 1; C2[m] = 0.0f; lim[m] = 0.0f; limit[m] = false;
            if (i >= r.nrec) continue;
            const float* c = a.cst32 + r.tab[i] * CST_STRIDE;
            float h, k, rho, nu, omr2, cr;
            if (r.t2f) {  // FP32 record fields written by the plan
                const float4 u0 = r.t2f[2 * i], u1 = r.t2f[2 * i + 1];
                h = u0.x; k = u0.y; rho = u0.z; nu = u0.w; omr2 = u1.x; cr = u1.y;
            } else {
                const double h64 = r.bt[2 * i], k64 = r.bt[2 * i + 1];
                const double rho64 = a.F[r.fac[i] + 2];  // L[1][0] of the 2 x 2 correlation factor
                h = (float)h64; k = (float)k64; rho = (float)rho64; nu = (float)r.dof[i];
                omr2 = (float)((1.0 - rho64) * (1.0 + rho64));
                cr = (float)(h64 * (rho64 > 0.0 ? rho64 : -rho64) - (rho64 > 0.0 ? k64 : -k64));
            }
            C2[m] = c[CST_C2];
            if (rho >= 1.0f || rho <= -1.0f) {  // the |rho| = 1 limits: no pieces
                limit[m] = true;
                if (rho >= 1.0f) {
                    lim[m] = t1cdf_dev<float>(h < k ? h : k, nu, c[CST_LGB]);
                } else {
                    const float v = t1cdf_dev<float>(h, nu, c[CST_LGB]) + t1cdf_dev<float>(k, nu, c[CST_LGB]) - 1.0f;
                    lim[m] = v > 0.0f ? v : 0.0f;
                }
                continue;
            }
            const bool graded = fabsf(rho) > 0.99f;
            // fewer nodes where the integrand is smooth enough (the rule of T2_LO)
            const bool lo = a.t2n_lo > 0 && !graded && fabsf(rho) < T2_LO_RHO && nu >= T2_LO_DOF_MIN &&
                            nu <= T2_LO_DOF_MAX;
            const T2Setup<float> S = t2_setup<float>(h, k, rho, nu, omr2, cr);
            kind[m] = graded ? 2 : lo ? 0 : 1;
            np[m] = S.split ? 2 : 1;
            nodes += (unsigned long long)(np[m] * (kind[m] == 0 ? nlo : kind[m] == 1 ? a.t2n : T2_NH));
            Rf[T2F_ANC0][rr] = S.anc0; Rf[T2F_PHIS][rr] = S.phis;
            Rf[T2F_L0][rr] = S.L0; Rf[T2F_L1][rr] = S.L1;
            Rf[T2F_D0][rr] = S.d0; Rf[T2F_ZS][rr] = S.zs;
            Rf[T2F_NU][rr] = nu; Rf[T2F_LGB1][rr] = c[CST_LGB1];
            Rt[rr] = r.tab[i]; Rk[rr] = kind[m];
        }
        // the chunk's pieces, grouped by node count (kind 0, then 1, then 2)
        int M = 0;
#pragma unroll
        for (int kd = 0; kd < 3; ++kd) {
            const int cnt = (kind[0] == kd ? np[0] : 0) + (kind[1] == kd ? np[1] : 0);
            int incl = cnt;
#pragma unroll
            for (int o = 1; o < CF_WARP; o <<= 1) {
                const int v = __shfl_up_sync(CF_FULL, incl, o);
                if (lane >= o) incl += v;
            }
            int pos = M + incl - cnt;
#pragma unroll
            for (int m = 0; m < 2; ++m)
                if (kind[m] == kd)
                    for (int pc = 0; pc < np[m]; ++pc) items[pos++] = (unsigned char)(((lane + m * CF_WARP) << 1) | pc);
            M += __shfl_sync(CF_FULL, incl, CF_WARP - 1);
        }
        __syncwarp();
        // phase 2: rounds of G pieces, one per group
        for (int it0 = 0; it0 < M; it0 += G) {
            const int it = it0 + grp;
            float acc = 0.0f;
            int rr = 0, pc = 0;
            if (it < M) {
                rr = items[it] >> 1;
                pc = items[it] & 1;
                const int kd = Rk[rr];
                const int nn = kd == 0 ? nlo : kd == 1 ? a.t2n : T2_NH;
                const float* gx = sgx[kd];
                const float* gw = sgw[kd];
                const bool graded = kd == 2;
                const float anc = pc ? Rf[T2F_PHIS][rr] : Rf[T2F_ANC0][rr];
                const float Lp = pc ? Rf[T2F_L1][rr] : Rf[T2F_L0][rr];
                const float d0 = pc ? 0.0f : Rf[T2F_D0][rr];
                const float zs = Rf[T2F_ZS][rr], nu = Rf[T2F_NU][rr], lgb1 = Rf[T2F_LGB1][rr];
                const float num1 = nu - 1.0f, nu1 = nu + 1.0f;
                const float2* tab = TAB ? a.t1tab + (size_t)Rt[rr] * T1TAB_N : nullptr;
                // the node's integrand; the piece's sum is scaled by |L| once, below
                auto node = [&](float off) {
                    const float sp = cf_sin_pi(anc + off);  // both arguments lie in [-pi, pi]
                    const float sd = cf_sin_pi(d0 + off);
                    const float z = zs * sd;
                    float t1;
                    if constexpr (TAB) t1 = t1cdf_table(z, tab);
                    else t1 = t1cdf_dev<float>(z, nu1, lgb1);
                    return ptx_ex2_approx(num1 * ptx_lg2_approx(sp)) * t1;
                };
                if (graded) {  // nodes anchor + L u^3, weights 3 u^2
                    for (int t = sub; t < nn; t += L) {
                        const float u = gx[t];
                        acc = fmaf(gw[t] * (3.0f * u * u), node(Lp * (u * u * u)), acc);
                    }
                } else {
                    for (int t = sub; t < nn; t += L) acc = fmaf(gw[t], node(Lp * gx[t]), acc);
                }
                acc *= fabsf(Lp);
            }
            acc = group_sum<L>(acc);
            if (it < M && sub == 0) P[rr][pc] = acc;
        }
        __syncwarp();
        // phase 3: records lane and lane + 32
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            const int rr = lane + m * CF_WARP;
            const long long i = base + rr;
            if (i >= r.nrec) continue;
            float v;
            if (limit[m]) v = lim[m];
            else v = C2[m] * (np[m] == 2 ? P[rr][0] + P[rr][1] : P[rr][0]);
            if (r.res32) r.res32[i] = v;
            else r.res[i] = (double)v;
            if (r.se) r.se[i] = 0.0;
        }
        __syncwarp();
    }
    if (a.nodes) {
#pragma unroll
        for (int o = CF_WARP / 2; o > 0; o >>= 1) nodes += __shfl_xor_sync(CF_FULL, nodes, o);
        if (lane == 0 && nodes) atomicAdd(a.nodes, nodes);
    }
}

// Lanes per FP32 T_2 piece (finite dof), a.t2_group in {2, 4, 8, 16}; 32 (or 0: the CFUSN
// model's records) = the warp-per-record kernel.
template <int L>
static void go_group(const RecSet& r, const IntegArgs& a, int blocks, cudaStream_t st)
{
    const long long per_block = (long long)T2P_WARPS * T2P_CH;
    const long long need = (r.nrec + per_block - 1) / per_block;
    const int gb = (int)(need < blocks ? need : blocks);
    if (a.t1tab) t2_pieces_kernel<L, true><<<gb > 0 ? gb : 1, T2P_WARPS * CF_WARP, 0, st>>>(r, a);
    else t2_pieces_kernel<L, false><<<gb > 0 ? gb : 1, T2P_WARPS * CF_WARP, 0, st>>>(r, a);
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
