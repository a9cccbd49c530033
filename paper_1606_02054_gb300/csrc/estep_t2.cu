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
// 64 records; lane l sets up records l and l + 32 (the angles of the split, the pieces'
// lengths and node counts, once per record), the chunk's pieces (one or two per record,
// 8 to 64 nodes each) are ordered by node set and dealt to the warp's 32/L groups of L
// lanes, a group sums its piece's nodes (lane sub takes nodes sub, sub + L, ...), and the
// record's value is C_nu (piece 0 + piece 1).  Dealing pieces rather than records keeps
// the groups of a round on equal node counts: a record with one piece no longer idles its
// lanes while a neighbour's second piece runs.  The same L gives the same bits.
namespace {
constexpr int T2P_WARPS = 8;
constexpr int T2P_CH = 2 * CF_WARP;  // records per warp chunk
// a record's set-up fields, one array per field (consecutive records in distinct banks)
enum { T2F_ANC0, T2F_PHIS, T2F_L0, T2F_L1, T2F_D0, T2F_ZS, T2F_NU, T2F_LGB1, T2F_N };
constexpr int T2P_NMAX = 64;  // nodes per piece at most (t2_nodes <= 64, T2_NH = 64)
// node sets: the classes 0-4 of t2_lo_class, then t2n nodes, then the graded pieces' T2_NH
constexpr int T2P_NK = T2_LO_NCLS + 2, T2P_KN = T2_LO_NCLS, T2P_KG = T2_LO_NCLS + 1;
}  // namespace

// TAB: the inner T_1 from the per-dof tables (a.t1tab), else by its continued fraction
template <int L, bool TAB>
__global__ void __launch_bounds__(T2P_WARPS * CF_WARP, 4) t2_pieces_kernel(RecSet r, IntegArgs a)
{
    constexpr int G = CF_WARP / L;
    __shared__ float srf[T2P_WARPS][T2F_N][T2P_CH];
    __shared__ int srt[T2P_WARPS][T2P_CH];                     // table index
    __shared__ unsigned char srk[T2P_WARPS][2 * T2P_CH];       // node set of piece (record << 1) | pc
    __shared__ float sgx[T2P_NK][T2P_NMAX], sgw[T2P_NK][T2P_NMAX];  // the node sets
    __shared__ float spsum[T2P_WARPS][T2P_CH][2];
    __shared__ unsigned char sitem[T2P_WARPS][2 * T2P_CH];  // (record << 1) | piece
    const int lane = threadIdx.x & (CF_WARP - 1), wib = threadIdx.x >> 5;
    const int sub = lane & (L - 1), grp = lane / L;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    float (*Rf)[T2P_CH] = srf[wib];
    int* Rt = srt[wib];
    unsigned char* Rk = srk[wib];
    float (*P)[2] = spsum[wib];
    unsigned char* items = sitem[wib];
    auto count = [&](int kd) { return kd < T2P_KN ? t2_lo_nodes(kd) : kd == T2P_KN ? a.t2n : T2_NH; };
    for (int e = threadIdx.x; e < T2P_NK * T2P_NMAX; e += blockDim.x) {
        const int kd = e / T2P_NMAX, i = e % T2P_NMAX;
        float x = 0.0f, w = 0.0f;
        if (kd < T2P_KN) {
            if (a.t2n_lo > 0 && i < t2_lo_nodes(kd)) { x = a.glx32l[t2_lo_off(kd) + i]; w = a.glw32l[t2_lo_off(kd) + i]; }
        } else if (kd == T2P_KN) {
            if (i < a.t2n) { x = a.glx32[i]; w = a.glw32[i]; }
        } else if (i < T2_NH) {
            x = a.glx32h[i]; w = a.glw32h[i];
        }
        sgx[kd][i] = x;
        sgw[kd][i] = w;
    }
    __syncthreads();
    unsigned long long nodes = 0;  // this lane's records' quadrature nodes (profiler count)
    for (long long base = warp * T2P_CH; base < r.nrec; base += nwarps * T2P_CH) {
        // phase 1: set-up of records lane and lane + 32
        int np[2], kind[2][2];
        float C2[2], lim[2];
        bool limit[2];
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            const int rr = lane + m * CF_WARP;
            const long long i = base + rr;
            np[m] = 0; kind[m][0] = kind[m][1] = T2P_KN; C2[m] = 0.0f; lim[m] = 0.0f; limit[m] = false;
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
            // fewer nodes where the integrand is smooth enough (t2_lo_class, per piece)
            const bool lo = a.t2n_lo > 0 && !graded && fabsf(rho) < T2_LO_RHO && nu >= T2_LO_DOF_MIN &&
                            nu <= T2_LO_DOF_MAX;
            const T2Setup<float> S = t2_setup<float>(h, k, rho, nu, omr2, cr);
            np[m] = S.split ? 2 : 1;
            kind[m][0] = graded ? T2P_KG : lo ? t2_lo_class(S.L0, nu, S.zs) : T2P_KN;
            kind[m][1] = graded ? T2P_KG : lo ? t2_lo_class(S.L1, nu, S.zs) : T2P_KN;
            nodes += (unsigned long long)(count(kind[m][0]) + (S.split ? count(kind[m][1]) : 0));
            Rf[T2F_ANC0][rr] = S.anc0; Rf[T2F_PHIS][rr] = S.phis;
            Rf[T2F_L0][rr] = S.L0; Rf[T2F_L1][rr] = S.L1;
            Rf[T2F_D0][rr] = S.d0; Rf[T2F_ZS][rr] = S.zs;
            Rf[T2F_NU][rr] = nu; Rf[T2F_LGB1][rr] = c[CST_LGB1];
            Rt[rr] = r.tab[i];
            Rk[2 * rr] = (unsigned char)kind[m][0];
            Rk[2 * rr + 1] = (unsigned char)kind[m][1];
        }
        // the chunk's pieces, grouped by node set (the sets present in the chunk, in order)
        int M = 0;
        unsigned present = 0;
#pragma unroll
        for (int m = 0; m < 2; ++m)
#pragma unroll
            for (int pc = 0; pc < 2; ++pc)
                if (pc < np[m]) present |= 1u << kind[m][pc];
        present = __reduce_or_sync(CF_FULL, present);
        while (present) {
            const int kd = __ffs(present) - 1;
            present &= present - 1;
            int cnt = 0;
#pragma unroll
            for (int m = 0; m < 2; ++m)
#pragma unroll
                for (int pc = 0; pc < 2; ++pc) cnt += pc < np[m] && kind[m][pc] == kd;
            int incl = cnt;
#pragma unroll
            for (int o = 1; o < CF_WARP; o <<= 1) {
                const int v = __shfl_up_sync(CF_FULL, incl, o);
                if (lane >= o) incl += v;
            }
            int pos = M + incl - cnt;
#pragma unroll
            for (int m = 0; m < 2; ++m)
#pragma unroll
                for (int pc = 0; pc < 2; ++pc)
                    if (pc < np[m] && kind[m][pc] == kd) items[pos++] = (unsigned char)(((lane + m * CF_WARP) << 1) | pc);
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
                const int kd = Rk[items[it]];
                const int nn = count(kd);
                const float* gx = sgx[kd];
                const float* gw = sgw[kd];
                const bool graded = kd == T2P_KG;
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
