// noalloc.cu -- cfust_reduce_stats_noalloc: the posterior-weight and
// sufficient-statistic reduction of the E-step for callers that cannot
// allocate device memory.
//
// Such callers include code that owns all device memory through its own
// pool, code that must not trigger the implicit device synchronisation of
// cudaMalloc/cudaFree inside a latency-critical loop, and code running while
// allocation is forbidden.  The entry point takes every input and output as a
// caller-provided device pointer and keeps its only scratch -- the per-block
// partial sums and an error flag -- in the file-scope device arrays below,
// which every GPU that loads the library holds until the process exits.
#include <cuda_runtime.h>

#include <string>

#include "cfust.h"
#include "internal.cuh"

__global__ void estep_reduce_kernel(ReduceArgs);
__global__ void reduce_partials_kernel(const double*, int, int, double*, int*);

// Block partials: nblocks x (g * S + 1) doubles must fit (4 MiB).
#define CF_NOALLOC_PARTIAL_DOUBLES (1 << 19)
static __device__ __align__(256) double g_noalloc_partial[CF_NOALLOC_PARTIAL_DOUBLES];
static __device__ __align__(256) int g_noalloc_flag[64];

namespace {
// failures are reported through cfust_last_error(NULL)
cfust_status nerr(cfust_status s, const std::string& m)
{
    cf_set_global_error(m);
    return s;
}
}  // namespace

extern "C" cfust_status cfust_reduce_stats_noalloc(int p, int q, int g, int64_t n, const double* y,
                                                   const double* pi, const double* mu,
                                                   const double* logf, const double* u,
                                                   const double* elogu, const double* eu,
                                                   const double* euu, double* tau, double* stats,
                                                   void* cuda_stream)
{
    if (p < 1 || p > CF_MAXP || q < 1 || q > CF_MAXQ || g < 1 || g > CF_MAXG || n < 1 ||
        n >= (int64_t(1) << 31))
        return nerr(CFUST_EINVAL, "cfust_reduce_stats_noalloc: sizes out of range");
    if (!y || !pi || !mu || !logf || !u || !elogu || !eu || !euu || !stats)
        return nerr(CFUST_EINVAL, "cfust_reduce_stats_noalloc: NULL device pointer");
    // rows of 4 + p + q + q^2 doubles, chunk <= 256 observations, at most 48 KB of
    // shared memory per block (the default limit: no attribute is set here).  The
    // allocating path raises its limit to 64 KB and may stage more observations per
    // block, so the two agree to rounding, not bit for bit.
    const int row = 4 + p + q + q * q;
    int chunk = 256;
    while (chunk > 32 && ((size_t)chunk * (row + g + 1) + CF_MAXG) * sizeof(double) > 48 * 1024) chunk -= 32;
    const int nblocks = (int)((n + chunk - 1) / chunk);
    const int width = g * stats_per_comp(p, q) + 1;
    if ((long long)nblocks * width > CF_NOALLOC_PARTIAL_DOUBLES)
        return nerr(CFUST_EINVAL,
                    "cfust_reduce_stats_noalloc: ceil(n/" + std::to_string(chunk) + ") x (g*(3+p+q+pq+q^2+p^2)+1) = " +
                        std::to_string((long long)nblocks * width) + " partial sums exceed the fixed scratch of " +
                        std::to_string(CF_NOALLOC_PARTIAL_DOUBLES) + " doubles");
    // device addresses of the file-scope scratch in the current context (host code
    // cannot use the symbols directly).  Looked up on every call rather than cached:
    // the address belongs to the context, and a context created after
    // cudaDeviceReset, or another context on the same device, has its own copy.
    // The first lookup in a context also loads the library's device code there.
    cudaError_t e;
    void* a = nullptr;
    if ((e = cudaGetSymbolAddress(&a, g_noalloc_partial)) != cudaSuccess)
        return nerr(CFUST_ECUDA, std::string("cfust_reduce_stats_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    void* b = nullptr;
    if ((e = cudaGetSymbolAddress(&b, g_noalloc_flag)) != cudaSuccess)
        return nerr(CFUST_ECUDA, std::string("cfust_reduce_stats_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    double* partial = (double*)a;
    int* flag = (int*)b;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if ((e = cudaMemsetAsync(flag, 0, sizeof(int), st)) != cudaSuccess)
        return nerr(CFUST_ECUDA, std::string("cfust_reduce_stats_noalloc: ") + cudaGetErrorString(e));
    ReduceArgs r;
    r.D = Dims{p, q, g, (long long)n};
    r.y = y; r.pi = pi; r.mu = mu; r.logf = logf; r.u = u; r.elogu = elogu; r.eu = eu; r.euu = euu;
    r.tau = tau;
    r.partial = partial;
    r.chunk = chunk;
    r.row = row;
    r.y32 = nullptr;
    r.pr32 = nullptr;
    r.small_only = 0;
    const size_t smem = sizeof(double) * ((size_t)chunk * row + (size_t)g * chunk + chunk + CF_MAXG);
    estep_reduce_kernel<<<nblocks, 256, smem, st>>>(r);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return nerr(CFUST_ECUDA, std::string("cfust_reduce_stats_noalloc: ") + cudaGetErrorString(e));
    reduce_partials_kernel<<<(width + 127) / 128, 128, 0, st>>>(partial, nblocks, width, stats, flag);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return nerr(CFUST_ECUDA, std::string("cfust_reduce_stats_noalloc: ") + cudaGetErrorString(e));
    // complete before returning so a non-finite statistic can be reported
    int hflag = 0;
    if ((e = cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return nerr(CFUST_ECUDA, std::string("cfust_reduce_stats_noalloc: ") + cudaGetErrorString(e));
    if (hflag & KF_NAN) return nerr(CFUST_ENAN, "cfust_reduce_stats_noalloc: non-finite statistic");
    return CFUST_OK;
}
