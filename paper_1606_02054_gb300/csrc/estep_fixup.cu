// estep_fixup.cu -- FP64 re-evaluation of listed pairs, one warp per pair.
//
// In FP32 mode the lattice products of a pair whose alpha_s (eq 4) is below
// 1e-35 leave the FP32 range; the combine kernel lists such pairs and this
// kernel recomputes every integral of those pairs in FP64, then the same
// assembly as the combine kernel.
#include "estep_common.cuh"

// T_k(bt; 0, corr(Lc Lc^T), nu) in FP64, warp-cooperative; chi = table of this dof.
__device__ double tk_fp64(int k, const double* bt, const double* Lc, double nu, const double* chi,
                          const EstepArgs& a, int lane, double* se)
{
    if (se) *se = 0.0;
    switch (k) {
    case 0: return 1.0;
    case 1: return isinf(nu) ? normcdf(bt[0]) : t1cdf_dev<double>(bt[0], nu, t1_lgb(nu));
    case 2: {
        const double rho = Lc[2];
        if (isinf(nu))
            return phi2_warp<double>(bt[0], bt[1], rho, a.t2n, a.glx64, a.glw64, lane);
        return t2cdf_warp<double>(bt[0], bt[1], rho, nu, (1.0 - rho) * (1.0 + rho),
                                  bt[0] * (rho > 0.0 ? rho : -rho) - (rho > 0.0 ? bt[1] : -bt[1]),
                                  t1_lgb(nu), t1_lgb(nu + 1.0),
                                  exp(lgamma(0.5 * (nu + 1.0)) - lgamma(0.5 * nu)) / sqrt(CF_PI),
                                  a.t2n, a.glx64, a.glw64, a.t2n, a.glx64, a.glw64, lane);
    }
    case 3: return tk_lattice_warp<double, 3>(bt, Lc, chi, a.shf64, a.lat, lane, se);
    case 4: return tk_lattice_warp<double, 4>(bt, Lc, chi, a.shf64, a.lat, lane, se);
    case 5: return tk_lattice_warp<double, 5>(bt, Lc, chi, a.shf64, a.lat, lane, se);
    case 6: return tk_lattice_warp<double, 6>(bt, Lc, chi, a.shf64, a.lat, lane, se);
    case 7: return tk_lattice_warp<double, 7>(bt, Lc, chi, a.shf64, a.lat, lane, se);
    default: return tk_lattice_warp<double, 8>(bt, Lc, chi, a.shf64, a.lat, lane, se);
    }
}

__global__ void __launch_bounds__(128) fixup_kernel(EstepArgs a, const int* count, const int* list)
{
    const int lane = threadIdx.x & (CF_WARP - 1);
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int p = a.D.p, q = a.D.q, q1 = q - 1, q2 = q - 2;
    const int cnt = *count;
    const size_t NM = (size_t)a.lat.N * a.lat.M;
    __shared__ double slot[4][CF_MAXQ + CF_MAXQ * (CF_MAXQ + 1) / 2 + 3 + CF_MAXSHIFT];
    double* acc = slot[threadIdx.x >> 5];
    for (int i = warp; i < cnt; i += nwarps) {
        const long long pid = list[i];
        const int h = (int)(pid / a.D.n);
        const long long j = pid - (long long)h * a.D.n;
        const double* F = a.F + (size_t)h * a.Ly.stride;
        const double* chi = a.chi64 + (size_t)(3 * h) * NM;
        const double nu1 = F[a.Ly.scal + SC_NU] + p;
        double c[CF_MAXQ], d, logtp, bt[CF_MAXQ], se = 0.0;
        pair_whiten(F, a.Ly, p, q, a.y + (size_t)j * p, &d, c, &logtp);
        limits_l0(F, a.Ly, p, q, c, d, 0, bt);
        const double alpha_s = tk_fp64(q, bt, F + fac_l0(a.Ly), nu1, chi, a, lane, &se);
        double alpha = 0.0, tq1[CF_MAXQ], tq2[CF_MAXQ * CF_MAXQ];
        if (a.single_pass && !a.density_only) {
            double m[CF_MAXQ + CF_MAXQ * (CF_MAXQ + 1) / 2];
            // the pass of alpha_s (bt still holds its limits) weighted to dof nu+p+2
            const double* Lq = F + fac_l0(a.Ly);
            const double rk = isinf(nu1) ? 1.0 : sqrt((nu1 + 2.0) / nu1);
            double as = 0.0, sej = 0.0, lw = NAN;
            const double* lchi = a.lchi64 ? a.lchi64 + (size_t)(3 * h) * NM : nullptr;
            double* lwp = lchi ? &lw : nullptr;
            switch (q) {
            case 3: alpha = tk_lattice_mom_warp<double, 3>(bt, Lq, chi, a.shf64, a.lat, lane, acc, rk, &as, &sej, lchi, lwp); break;
            case 4: alpha = tk_lattice_mom_warp<double, 4>(bt, Lq, chi, a.shf64, a.lat, lane, acc, rk, &as, &sej, lchi, lwp); break;
            case 5: alpha = tk_lattice_mom_warp<double, 5>(bt, Lq, chi, a.shf64, a.lat, lane, acc, rk, &as, &sej, lchi, lwp); break;
            case 6: alpha = tk_lattice_mom_warp<double, 6>(bt, Lq, chi, a.shf64, a.lat, lane, acc, rk, &as, &sej, lchi, lwp); break;
            case 7: alpha = tk_lattice_mom_warp<double, 7>(bt, Lq, chi, a.shf64, a.lat, lane, acc, rk, &as, &sej, lchi, lwp); break;
            default: alpha = tk_lattice_mom_warp<double, 8>(bt, Lq, chi, a.shf64, a.lat, lane, acc, rk, &as, &sej, lchi, lwp); break;
            }
            for (int k = 0; k < q + q * (q + 1) / 2; ++k) m[k] = acc[1 + k];
            __syncwarp();
            PairOut o;
            pair_assemble_sp(F, a.Ly, p, q, c, d, logtp, alpha_s, alpha, m, o, lw);
            if (lane == 0) {
                a.logf[pid] = o.logf;
                if (a.se) a.se[pid] = se;
                if (!(o.logf < INFINITY)) atomicOr(a.flags, KF_NAN);  // NaN or +inf; -inf is a null pair
                if (a.pr32) {
                    store_pr32(a.pr32 + pid * pr32_width(q), q, o);
                } else {
                    a.u[pid] = o.u;
                    a.elogu[pid] = o.elogu;
                    for (int k = 0; k < q; ++k) a.eu[pid * q + k] = o.eu[k];
                    for (int k = 0; k < q * q; ++k) a.euu[pid * q * q + k] = o.euu[k];
                }
            }
            continue;
        }
        if (!a.density_only) {
            limits_l0(F, a.Ly, p, q, c, d, 1, bt);
            alpha = tk_fp64(q, bt, F + fac_l0(a.Ly), nu1 + 2.0, chi + 2 * NM, a, lane, nullptr);
            for (int r = 0; r < q && q1 > 0; ++r) {
                limits_l1(F, a.Ly, p, q, c, d, r, bt);
                tq1[r] = tk_fp64(q1, bt, F + fac_l1(a.Ly, q, r), nu1 + 1.0, chi + NM, a, lane, nullptr);
                for (int s = 0; s < q1 && q2 > 0; ++s) {
                    limits_l2(F, a.Ly, p, q, c, d, r, s, bt);
                    tq2[r * q1 + s] = tk_fp64(q2, bt, F + fac_l2(a.Ly, q, r, s), nu1, chi, a, lane, nullptr);
                }
            }
        }
        PairOut o;
        pair_assemble(F, a.Ly, p, q, c, d, logtp, alpha_s, alpha, tq1, tq2, a.density_only,
                      a.cst64 + (size_t)(3 * h) * CST_STRIDE, o);
        if (lane == 0) {
            a.logf[pid] = o.logf;
            if (a.se) a.se[pid] = se;
            if (!(o.logf < INFINITY)) atomicOr(a.flags, KF_NAN);  // NaN or +inf; -inf is a null pair
            if (!a.density_only && a.pr32) {
                store_pr32(a.pr32 + pid * pr32_width(q), q, o);
            } else if (!a.density_only) {
                a.u[pid] = o.u;
                a.elogu[pid] = o.elogu;
                for (int k = 0; k < q; ++k) a.eu[pid * q + k] = o.eu[k];
                for (int k = 0; k < q * q; ++k) a.euu[pid * q * q + k] = o.euu[k];
            }
        }
    }
}

cudaError_t launch_fixup(const EstepArgs& a, const int* count, const int* list, int nsm,
                         cudaStream_t st, long long* launches)
{
    fixup_kernel<<<2 * nsm, 128, 0, st>>>(a, count, list);
    ++*launches;
    return cudaGetLastError();
}
