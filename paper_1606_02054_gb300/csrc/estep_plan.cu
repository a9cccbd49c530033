// estep_plan.cu -- E-step plan and combine kernels (one thread per pair, FP64)
// and the T_1 record evaluator.
//
// Plan: whitening and log t_p of every (observation, component) pair, and the
// standardised limits of every T_k the pair needs (levels 0-2, see
// internal.cuh).  Combine: eqs (4), (13), (15)-(17) from the evaluated T_k.
// Pairs are component-major (pid = h*n + j).
#include "estep_common.cuh"

// FP32 modes: the T_2 record's FP32 inputs (RecSet::t2f); F is the component's
// factor block, fac the record's 2 x 2 correlation factor within it.
__device__ __forceinline__ void put_t2f(const RecSet& L, long long rec, const double* bt,
                                        const double* F, int fac, double dof)
{
    if (L.t2f) t2_record_f32(bt[0], bt[1], F[fac + 2], dof, L.t2f + 2 * rec);
}

// Mixed form: the same record inputs from FP32 limits and the FP32 copy of the
// factor (Fc: the record's 2 x 2 correlation factor [1, 0; rho, sqrt(1 - rho^2)]),
// so 1 - rho^2 is the square of its last entry and h|rho| - sign(rho) k one FMA.
__device__ __forceinline__ void put_t2f32(const RecSet& L, long long rec, const float* bt, const float* Fc,
                                          float dof)
{
    const float rho = Fc[2], l11 = Fc[3];
    L.t2f[2 * rec] = make_float4(bt[0], bt[1], rho, dof);
    L.t2f[2 * rec + 1] = make_float4(l11 * l11, fmaf(bt[0], fabsf(rho), rho > 0.0f ? -bt[1] : bt[1]), 0.0f, 0.0f);
}

// Mixed form: one pair in FP32 (whitening, log t_p, limits, FP32 T_2 inputs);
// T_2 records of the FP32 modes need no FP64 fields, the others get them.
// F: the component's FP32 factor block (staged in shared memory by the kernel)
template <int P, int Q>
__device__ void plan_pair_f32(const PlanArgs& a, long long pid, int h, const float* yj, const float* F)
{
    const int p = a.D.p, q = Q > 0 ? Q : a.D.q;
    const int m0 = (a.density_only || a.single_pass) ? 1 : 2;
    const int foff = h * a.Ly.stride;
    // dof nu + p in FP64 for the records with FP64 fields (read only where used)
    auto nu1d = [&]() { return a.F[(size_t)h * a.Ly.stride + a.Ly.scal + SC_NU] + p; };
    const float nu1 = F[a.Ly.scal + SC_NU] + p;
    float c[CF_MAXQ], d, logtp, bt[CF_MAXQ];
    pair_whiten_f32<P>(F, a.Ly, p, q, yj, &d, c, &logtp);
    reinterpret_cast<float2*>(a.pd32)[pid] = make_float2(d, logtp);
    if (Q == 2) reinterpret_cast<float2*>(a.pc32)[pid] = make_float2(c[0], c[1]);
    else for (int k = 0; k < q; ++k) a.pc32[pid * q + k] = c[k];
    // a record gets the fields its integrator reads: FP32 T_2 records their FP32 fields and
    // table index, T_1 records no factor.  With the level-1 T_1s fused into combine (q = 2),
    // the level-0 records are stored record-major (alpha_s of every pair, then alpha), so the
    // threads of a warp write consecutive records.
    const long long np = a.D.n * a.D.g;
    for (int w = 0; w < m0; ++w) {
        const long long rec = (Q == 2 && a.fuse_l1) ? w * np + pid : pid * m0 + w;
        limits_l0<float>(F, a.Ly, p, q, c, d, w, bt);
        a.L0.tab[rec] = 3 * h + 2 * w;
        if (q == 2 && a.L0.t2f) {
            put_t2f32(a.L0, rec, bt, F + fac_l0(a.Ly), nu1 + 2.0f * w);
        } else {
            a.L0.fac[rec] = foff + fac_l0(a.Ly);
            for (int k = 0; k < q; ++k) a.L0.bt[rec * q + k] = bt[k];
            a.L0.dof[rec] = nu1d() + 2.0 * w;
        }
    }
    if (a.density_only) return;
    if (a.single_pass) {
        // alpha and the moments at dof nu+p+2 from the pass of alpha_s: its limits and chi table
        limits_l0<float>(F, a.Ly, p, q, c, d, 0, bt);
        for (int k = 0; k < q; ++k) a.LM.bt[pid * q + k] = bt[k];
        a.LM.fac[pid] = foff + fac_l0(a.Ly);
        a.LM.tab[pid] = 3 * h;
        a.LM.dof[pid] = nu1d() + 2.0;
        return;
    }
    if (Q == 2 && a.fuse_l1) return;  // combine evaluates the level-1 T_1s itself
    const int q1 = q - 1, q2 = q - 2;
    for (int r = 0; r < q && q1 > 0; ++r) {
        const long long rec = pid * q + r;
        limits_l1<float>(F, a.Ly, p, q, c, d, r, bt);
        a.L1.tab[rec] = 3 * h + 1;
        if (q1 == 2 && a.L1.t2f) {
            put_t2f32(a.L1, rec, bt, F + fac_l1(a.Ly, q, r), nu1 + 1.0f);
        } else {
            if (q1 >= 2) a.L1.fac[rec] = foff + fac_l1(a.Ly, q, r);
            for (int k = 0; k < q1; ++k) a.L1.bt[rec * q1 + k] = bt[k];
            a.L1.dof[rec] = nu1d() + 1.0;
        }
        for (int s = 0; s < q1 && q2 > 0; ++s) {
            const long long r2 = pid * q * q1 + r * q1 + s;
            limits_l2<float>(F, a.Ly, p, q, c, d, r, s, bt);
            a.L2.tab[r2] = 3 * h;
            if (q2 == 2 && a.L2.t2f) {
                put_t2f32(a.L2, r2, bt, F + fac_l2(a.Ly, q, r, s), nu1);
            } else {
                if (q2 >= 2) a.L2.fac[r2] = foff + fac_l2(a.Ly, q, r, s);
                for (int k = 0; k < q2; ++k) a.L2.bt[r2 * q2 + k] = bt[k];
                a.L2.dof[r2] = nu1d();
            }
        }
    }
}

// Mixed form: FP32 pairs in a kernel of their own, so the FP64 path's registers do not
// limit its occupancy (one kernel for both took 118 registers, 24 % warps active).
// P, Q: the dimensions p and q at compile time for common sizes (whitening and limits in
// registers), 0 for any
// The pairs in tiles of 128 observations of one component (pid = h n + j as before): a
// block stages its component's FP32 factor block in shared memory (when the component
// changes), so the whitening reads it there, four values per load, rather than as
// warp-uniform global loads that filled the load/store queue.
template <int P, int Q>
__global__ void __launch_bounds__(128) plan_kernel_f32(PlanArgs a)
{
    extern __shared__ float4 plan_sF4[];
    float* sF = reinterpret_cast<float*>(plan_sF4);
    const int p = a.D.p;
    const long long n = a.D.n;
    const long long tpc = (n + 127) / 128;  // tiles per component
    const long long ntiles = tpc * a.D.g;
    int hs = -1;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int h = (int)(tile / tpc);
        if (h != hs) {  // the same for the whole block
            __syncthreads();
            for (int e = threadIdx.x; e < a.Ly.stride; e += blockDim.x) sF[e] = a.F32[(size_t)h * a.Ly.stride + e];
            __syncthreads();
            hs = h;
        }
        const long long j = (tile - (long long)h * tpc) * 128 + threadIdx.x;
        if (j < n) plan_pair_f32<P, Q>(a, (long long)h * n + j, h, a.y32 + (size_t)j * p, sF);
    }
}

template <int P>
static void launch_plan_f32(const PlanArgs& a, int gb, cudaStream_t st)
{
    const size_t sh = sizeof(float) * (size_t)a.Ly.stride;
    if (a.D.q == 2) plan_kernel_f32<P, 2><<<gb, 128, sh, st>>>(a);
    else plan_kernel_f32<P, 0><<<gb, 128, sh, st>>>(a);
}

__global__ void __launch_bounds__(128) plan_kernel(PlanArgs a)
{
    const int p = a.D.p, q = a.D.q;
    const long long np = a.D.n * a.D.g;
    const int m0 = (a.density_only || a.single_pass) ? 1 : 2;
    for (long long pid = blockIdx.x * (long long)blockDim.x + threadIdx.x; pid < np;
         pid += (long long)gridDim.x * blockDim.x) {
        const int h = (int)(pid / a.D.n);
        const long long j = pid - (long long)h * a.D.n;
        const double* F = a.F + (size_t)h * a.Ly.stride;
        const int foff = h * a.Ly.stride;
        const double nu1 = F[a.Ly.scal + SC_NU] + p;
        double c[CF_MAXQ], d, logtp;
        pair_whiten(F, a.Ly, p, q, a.y + (size_t)j * p, &d, c, &logtp);
        a.pd[2 * pid] = d;
        a.pd[2 * pid + 1] = logtp;
        for (int k = 0; k < q; ++k) a.pc[pid * q + k] = c[k];
        double bt[CF_MAXQ];
        for (int w = 0; w < m0; ++w) {
            const long long rec = pid * m0 + w;
            limits_l0(F, a.Ly, p, q, c, d, w, bt);
            for (int k = 0; k < q; ++k) a.L0.bt[rec * q + k] = bt[k];
            a.L0.fac[rec] = foff + fac_l0(a.Ly);
            a.L0.tab[rec] = 3 * h + 2 * w;
            a.L0.dof[rec] = nu1 + 2.0 * w;
            if (q == 2) put_t2f(a.L0, rec, bt, F, fac_l0(a.Ly), nu1 + 2.0 * w);
        }
        if (a.density_only) continue;
        if (a.single_pass) {
            // alpha and the moments at dof nu+p+2 (eqs 13, 16, 17) from the pass of
            // alpha_s: its limits and chi table, points weighted by W/(nu+p)
            limits_l0(F, a.Ly, p, q, c, d, 0, bt);
            for (int k = 0; k < q; ++k) a.LM.bt[pid * q + k] = bt[k];
            a.LM.fac[pid] = foff + fac_l0(a.Ly);
            a.LM.tab[pid] = 3 * h;
            a.LM.dof[pid] = nu1 + 2.0;
            continue;
        }
        const int q1 = q - 1, q2 = q - 2;
        for (int r = 0; r < q && q1 > 0; ++r) {
            const long long rec = pid * q + r;
            limits_l1(F, a.Ly, p, q, c, d, r, bt);
            for (int k = 0; k < q1; ++k) a.L1.bt[rec * q1 + k] = bt[k];
            a.L1.fac[rec] = foff + fac_l1(a.Ly, q, r);
            a.L1.tab[rec] = 3 * h + 1;
            a.L1.dof[rec] = nu1 + 1.0;
            if (q1 == 2) put_t2f(a.L1, rec, bt, F, fac_l1(a.Ly, q, r), nu1 + 1.0);
            for (int s = 0; s < q1 && q2 > 0; ++s) {
                const long long r2 = pid * q * q1 + r * q1 + s;
                limits_l2(F, a.Ly, p, q, c, d, r, s, bt);
                for (int k = 0; k < q2; ++k) a.L2.bt[r2 * q2 + k] = bt[k];
                a.L2.fac[r2] = foff + fac_l2(a.Ly, q, r, s);
                a.L2.tab[r2] = 3 * h;
                a.L2.dof[r2] = nu1;
                if (q2 == 2) put_t2f(a.L2, r2, bt, F, fac_l2(a.Ly, q, r, s), nu1);
            }
        }
    }
}

// The mixed form's recursion-moment pairs (and its density passes): FP32 assembly into the
// FP32 pair rows, in a kernel of its own (its code and registers only; Q = q at compile time
// for q = 2, where the moment arrays stay in registers, 0 for any q).
template <int Q>
__global__ void __launch_bounds__(128) combine_mixed_kernel(CombineArgs a)
{
    const int p = a.D.p, q = Q > 0 ? Q : a.D.q;
    const long long np = a.D.n * a.D.g;
    const int m0 = a.density_only ? 1 : 2;
    const int q1 = q - 1;
    for (long long pid = blockIdx.x * (long long)blockDim.x + threadIdx.x; pid < np;
         pid += (long long)gridDim.x * blockDim.x) {
        const int h = (int)(pid / a.D.n);
        const float2 dl = reinterpret_cast<const float2*>(a.pd32)[pid];
        const float d = dl.x, logtp = dl.y;
        float c[CF_MAXQ];
        if (Q == 2) {
            const float2 c2 = reinterpret_cast<const float2*>(a.pc32)[pid];
            c[0] = c2.x;
            c[1] = c2.y;
        } else {
            for (int k = 0; k < q; ++k) c[k] = a.pc32[pid * q + k];
        }
        // level-0 records: record-major with the fused level 1 (see plan_pair_f32)
        const bool rmaj = Q == 2 && a.fuse_l1;
        const long long r0 = rmaj ? pid : pid * m0;
        // FP32 results where the T_2 kernel wrote them (res32), else the FP64 ones
        const float alpha_s = a.L0.res32 ? a.L0.res32[r0] : (float)a.L0.res[r0];
        const double se = a.L0.se ? a.L0.se[r0] : 0.0;
        if (!(alpha_s >= 1e-35f)) {
            // outside the FP32 range of the lattice products: redo in FP64
            const int slot = atomicAdd(a.fix_count, 1);
            a.fix_list[slot] = (int)pid;
            continue;
        }
        const long long r1 = rmaj ? np + pid : pid * m0 + 1;
        const float alpha = a.density_only ? 0.0f : a.L0.res32 ? a.L0.res32[r1] : (float)a.L0.res[r1];
        const float* F32 = a.F32 + (size_t)h * a.Ly.stride;
        float tq1[CF_MAXQ], tq2[Q == 2 ? 1 : CF_MAXQ * CF_MAXQ];
        if (!a.density_only) {
            if (Q == 2 && a.fuse_l1) {
                // the level-1 T_1 at dof nu+p+1 (table 3h holds T_1 at that dof; the normal
                // limit takes Phi), from the same FP32 limits the records would carry
                const bool nrm = isinf(F32[a.Ly.scal + SC_NU]);
                for (int r = 0; r < 2; ++r) {
                    float bt1[CF_MAXQ];
                    limits_l1<float>(F32, a.Ly, p, 2, c, d, r, bt1);
                    tq1[r] = nrm ? m_ncdf(bt1[0]) : t1cdf_table(bt1[0], a.t1tab + (size_t)(3 * h) * T1TAB_N);
                }
            } else {
                for (int r = 0; r < q && q1 > 0; ++r) tq1[r] = (float)a.L1.res[pid * q + r];
            }
            if (Q != 2 && q1 > 1)
                for (int i = 0; i < q * q1; ++i) tq2[i] = (float)a.L2.res[pid * q * q1 + i];
        }
        PairOutF of;
        pair_assemble_f32(F32, a.Ly, p, q, c, d, logtp, alpha_s, alpha, tq1, tq2,
                          a.density_only, a.cst32 + (size_t)(3 * h) * CST_STRIDE, of);
        a.logf[pid] = of.logf;
        if (a.se) a.se[pid] = se;
        if (!(of.logf < INFINITY)) atomicOr(a.flags, KF_NAN);  // NaN or +inf; -inf is a null pair
        if (!a.density_only) store_pr32(a.pr32 + pid * pr32_width(q), q, of);
    }
}

// MIXED: the mixed form's single-pass pairs (FP64 assembly, FP32 rows)
template <bool MIXED>
__global__ void __launch_bounds__(128) combine_kernel(CombineArgs a)
{
    const int p = a.D.p, q = a.D.q;
    const long long np = a.D.n * a.D.g;
    const int m0 = (a.density_only || a.single_pass) ? 1 : 2;
    const int q1 = q - 1;
    const int W = q + q * (q + 1) / 2;
    for (long long pid = blockIdx.x * (long long)blockDim.x + threadIdx.x; pid < np;
         pid += (long long)gridDim.x * blockDim.x) {
        const int h = (int)(pid / a.D.n);
        const double* F = a.F + (size_t)h * a.Ly.stride;
        double d, logtp, c[CF_MAXQ];
        if (MIXED) {
            d = a.pd32[2 * pid];
            logtp = a.pd32[2 * pid + 1];
            for (int k = 0; k < q; ++k) c[k] = a.pc32[pid * q + k];
        } else {
            d = a.pd[2 * pid];
            logtp = a.pd[2 * pid + 1];
            for (int k = 0; k < q; ++k) c[k] = a.pc[pid * q + k];
        }
        const double alpha_s = a.L0.res[pid * m0];
        const double se = a.L0.se ? a.L0.se[pid * m0] : 0.0;
        if (a.fp32 && !(alpha_s >= 1e-35)) {
            // outside the FP32 range of the lattice products: redo in FP64
            const int slot = atomicAdd(a.fix_count, 1);
            a.fix_list[slot] = (int)pid;
            continue;
        }
        PairOut o;
        if (a.single_pass && !a.density_only) {
            pair_assemble_sp(F, a.Ly, p, q, c, d, logtp, alpha_s, a.LM.res[pid], a.LM.mom + pid * W, o,
                             a.LM.lw ? a.LM.lw[pid] : NAN);
        } else {
            const double alpha = a.density_only ? 0.0 : a.L0.res[pid * m0 + 1];
            double tq1[CF_MAXQ], tq2[CF_MAXQ * CF_MAXQ];
            if (!a.density_only) {
                for (int r = 0; r < q && q1 > 0; ++r) tq1[r] = a.L1.res[pid * q + r];
                if (q1 > 1)
                    for (int i = 0; i < q * q1; ++i) tq2[i] = a.L2.res[pid * q * q1 + i];
            }
            pair_assemble(F, a.Ly, p, q, c, d, logtp, alpha_s, alpha, tq1, tq2, a.density_only,
                          a.cst64 + (size_t)(3 * h) * CST_STRIDE, o);
        }
        a.logf[pid] = o.logf;
        if (a.se) a.se[pid] = se;
        if (!(o.logf < INFINITY)) atomicOr(a.flags, KF_NAN);  // NaN or +inf; -inf is a null pair
        if (a.density_only) continue;
        if (a.pr32) {  // mixed form, single pass: FP64 assembly, FP32 row
            store_pr32(a.pr32 + pid * pr32_width(q), q, o);
            continue;
        }
        a.u[pid] = o.u;
        a.elogu[pid] = o.elogu;
        for (int k = 0; k < q; ++k) a.eu[pid * q + k] = o.eu[k];
        for (int k = 0; k < q * q; ++k) a.euu[pid * q * q + k] = o.euu[k];
    }
}

// FP32 with the T_1 tables (a.t1tab) and a record of table index 3h + 1 (dof nu + p + 1,
// the q = 2 moments' level 1): T_1 by interpolation in the table 3h, which holds T_1 at
// that dof (see t1cdf_table), instead of the continued fraction.
template <typename R>
__global__ void __launch_bounds__(128) t1_records_kernel(RecSet r, IntegArgs a)
{
    const R* cst = sizeof(R) == sizeof(float) ? (const R*)a.cst32 : (const R*)a.cst64;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < r.nrec;
         i += (long long)gridDim.x * blockDim.x) {
        const R dof = (R)r.dof[i];  // infinite: the normal limit, Phi
        const int tab = r.tab[i];
        if (sizeof(R) == sizeof(float) && a.t1tab && tab % 3 == 1 && !isinf(dof))
            r.res[i] = (double)t1cdf_table((float)r.bt[i], a.t1tab + (size_t)(tab - 1) * T1TAB_N);
        else
            r.res[i] = isinf(dof) ? (double)m_ncdf((R)r.bt[i])
                                  : (double)t1cdf_dev<R>((R)r.bt[i], dof, cst[tab * CST_STRIDE + CST_LGB]);
        if (r.se) r.se[i] = 0.0;
    }
}

static int grid_for(long long work, int threads, int cap)
{
    long long b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    return (int)(b < cap ? b : cap);
}

cudaError_t launch_plan(const PlanArgs& a, cudaStream_t st, long long* launches)
{
    const long long np = a.D.n * a.D.g;
    const int gb = grid_for(np, 128, 1 << 20);
    if (a.F32) {
        const long long ntiles = (a.D.n + 127) / 128 * a.D.g;
        const int gf = a.blocks > 0 && a.blocks < ntiles ? a.blocks : (int)(ntiles < (1 << 20) ? ntiles : (1 << 20));
        switch (a.D.p) {
        case 4: launch_plan_f32<4>(a, gf, st); break;
        case 6: launch_plan_f32<6>(a, gf, st); break;
        case 8: launch_plan_f32<8>(a, gf, st); break;
        case 16: launch_plan_f32<16>(a, gf, st); break;
        case 32: launch_plan_f32<32>(a, gf, st); break;
        default: launch_plan_f32<0>(a, gf, st); break;
        }
    }
    else plan_kernel<<<gb, 128, 0, st>>>(a);
    ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_combine(const CombineArgs& a, cudaStream_t st, long long* launches)
{
    const long long np = a.D.n * a.D.g;
    const int gb = grid_for(np, 128, 1 << 20);
    if (a.mixed && !(a.single_pass && !a.density_only)) {
        if (a.D.q == 2) combine_mixed_kernel<2><<<gb, 128, 0, st>>>(a);
        else combine_mixed_kernel<0><<<gb, 128, 0, st>>>(a);
    } else if (a.mixed) {
        combine_kernel<true><<<gb, 128, 0, st>>>(a);
    } else {
        combine_kernel<false><<<gb, 128, 0, st>>>(a);
    }
    ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_moments(const RecSet& r, const IntegArgs& a, int fp32, int nsm, cudaStream_t st,
                           long long* launches)
{
    if (r.k < 3 || r.nrec == 0) return cudaSuccess;
    const long long blocks_needed = (r.nrec + 7) / 8;
    const int cap = nsm * 16;
    const int blocks = (int)(blocks_needed < cap ? blocks_needed : cap);
    cudaError_t e = fp32 ? launch_mom32(r.k, r, a, blocks, st) : launch_mom64(r.k, r, a, blocks, st);
    ++*launches;
    return e;
}

cudaError_t launch_integrals(const RecSet& r, const IntegArgs& a, int fp32, int nsm,
                             cudaStream_t st, long long* launches)
{
    if (r.k == 0 || r.nrec == 0) return cudaSuccess;
    cudaError_t e;
    if (r.k == 1) {
        if (fp32) t1_records_kernel<float><<<grid_for(r.nrec, 128, 1 << 20), 128, 0, st>>>(r, a);
        else t1_records_kernel<double><<<grid_for(r.nrec, 128, 1 << 20), 128, 0, st>>>(r, a);
        e = cudaGetLastError();
    } else {
        // one warp per record, 8 warps per block, enough blocks to fill every SM
        const long long blocks_needed = (r.nrec + 7) / 8;
        const int cap = nsm * 16;
        const int blocks = (int)(blocks_needed < cap ? blocks_needed : cap);
        if (r.k == 2) e = launch_t2(r, a, fp32, blocks, st);
        else if (fp32) e = launch_lattice32(r.k, r, a, blocks, st);
        else e = launch_lattice64(r.k, r, a, blocks, st);
    }
    ++*launches;
    return e;
}

// The mixed form's FP32 pair rows widened into the FP64 pair buffers (read-back only).
__global__ void widen_pairs_kernel(const float* __restrict__ pr32, long long ng, int q, double* __restrict__ u,
                                   double* __restrict__ elogu, double* __restrict__ eu, double* __restrict__ euu)
{
    const int w = pr32_width(q);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ng;
         i += (long long)gridDim.x * blockDim.x) {
        const float* r = pr32 + i * w;
        u[i] = r[0];
        elogu[i] = r[1];
        for (int k = 0; k < q; ++k) eu[i * q + k] = r[2 + k];
        for (int k = 0; k < q * q; ++k) euu[i * q * q + k] = r[2 + q + k];
    }
}

// FP32 copies of the factor blocks (mixed precision)
__global__ void factors_to_f32_kernel(const double* __restrict__ F, float* __restrict__ F32, long long count)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < count;
         t += (long long)gridDim.x * blockDim.x)
        F32[t] = (float)F[t];
}

cudaError_t launch_factors_f32(const double* F, float* F32, long long count, cudaStream_t st,
                               long long* launches)
{
    factors_to_f32_kernel<<<grid_for(count, 256, 1024), 256, 0, st>>>(F, F32, count);
    ++*launches;
    return cudaGetLastError();
}
