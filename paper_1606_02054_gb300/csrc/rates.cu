// rates.cu -- cfust_measure_rates: throughput microbenchmarks of the pipes the
// E-step integrators are bound by, measured on the device the library runs on.
//
// The lattice integrators of T_k (k >= 3) spend their time in per-point
// arithmetic: the normal CDF and its inverse (MUFU rcp/ex2/lg2 plus FP32
// polynomials) and the FP32 FMAs of the separation of variables and of the
// moment sums.  No data-sheet number states how fast that mix can run, so it is
// measured here:
//   - FP32 FMA, FP64 FMA: 8 independent FMA chains per thread;
//   - MUFU ex2, lg2, rcp (the approximate PTX forms the FP32 integrators use):
//     8 independent chains per thread;
//   - the single-pass integrand mix of dimension K: per lattice point K normal
//     CDFs, K inverse normal CDFs (this library's FP32 forms, cf_ncdf_f32 and
//     cf_ncdfinv_f32), the K(K-1)/2 + 3K FMAs of the chain and the
//     2 + K + K(K+1)/2 FMAs of the weighted moment sums, with 1, 2 or 4
//     independent points in flight per thread (the best of the three) and no
//     memory traffic: the rate an implementation of the same algorithm could
//     reach if it did nothing else;
//   - one node of the FP32 T_2 quadrature (two sines, the sin^(nu-1) weight, the
//     inner T_1 from its table), 1, 2 or 4 independent nodes per thread (the best).
// Every kernel runs a full grid (8 blocks of 256 threads per SM) for a fixed
// number of iterations; rates are operations (or points) per second of
// CUDA-event time after one warm-up launch, and the SM clock is read with
// clock64() against the same events.
#include <cuda_runtime.h>

#include <string>

#include "cfust.h"
#include "internal.cuh"
#include "special.cuh"

void cf_set_global_error(const std::string& msg);

namespace {

constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) fma32_rate_kernel(float* out, int iters, float m, float c)
{
    float a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = threadIdx.x * 1e-7f + k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int k = 0; k < 8; ++k) a[k] = fmaf(a[k], m, c);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) fma64_rate_kernel(double* out, int iters, double m, double c)
{
    double a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = threadIdx.x * 1e-7 + k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int k = 0; k < 8; ++k) a[k] = fma(a[k], m, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// fn 0: x = ex2(-x) (stays in [0.5, 1]); 1: x = lg2(x) + 1.5 (stays in [0.5, 3]);
// 2: x = rcp(x) + 0.5 (stays near 1.28; the added constant keeps the compiler from
// cancelling two reciprocals)
template <int FN>
__global__ void __launch_bounds__(kThreads) mufu_rate_kernel(float* out, int iters)
{
    float a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = 0.6f + threadIdx.x * 1e-6f + 0.01f * k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                if constexpr (FN == 0) a[k] = ptx_ex2_approx(-a[k]);
                else if constexpr (FN == 1) a[k] = ptx_lg2_approx(a[k]) + 1.5f;
                else a[k] = ptx_rcp_approx(a[k]) + 0.5f;
            }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// The single-pass integrand of dimension K for two independent points per thread.
// Coordinates w advance by a fixed irrational-like step (one add and one select per
// coordinate, kept in [0, 1)); the chi variate s is taken from the first coordinate.
template <int K, int P>
__global__ void __launch_bounds__(kThreads) mix_rate_kernel(float* out, int iters)
{
    constexpr int K2 = K * (K + 1) / 2;
    const float t0 = threadIdx.x * (1.0f / 4096.0f);
    float b[K], invd[K], L[K][K];
#pragma unroll
    for (int r = 0; r < K; ++r) {
        b[r] = 0.3f + 0.1f * r + t0;
        invd[r] = 1.0f / (1.0f + 0.05f * r);
#pragma unroll
        for (int l = 0; l < K; ++l) L[r][l] = l < r ? 0.2f / (1 + r + l) : 0.f;
    }
    float w[P][K + 1], dw[K + 1];
#pragma unroll
    for (int d = 0; d <= K; ++d) {
        dw[d] = 0.6180339f * (d + 1) - (int)(0.6180339f * (d + 1));
#pragma unroll
        for (int p = 0; p < P; ++p) w[p][d] = 0.5f * dw[d] + 0.125f * p + t0 * 0.1f;
    }
    float af[P], aw[P], a1[P][K], a2[P][K2];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        af[p] = aw[p] = 0.f;
#pragma unroll
        for (int r = 0; r < K; ++r) a1[p][r] = 0.f;
#pragma unroll
        for (int r = 0; r < K2; ++r) a2[p][r] = 0.f;
    }
    const float rk = 1.1f, rk2 = rk * rk;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const float s = 0.5f + w[p][0];
            float y[K], f = 1.f;
#pragma unroll
            for (int r = 0; r < K; ++r) {
                float a = b[r] * s;
#pragma unroll
                for (int l = 0; l < r; ++l) a = fmaf(-L[r][l], y[l], a);
                const float e = cf_ncdf_f32(a * invd[r]);
                f *= e;
                y[r] = cf_ncdfinv_f32(w[p][r + 1] * e);
            }
            const float fs = f * s, w1 = fs * rk, w2 = f * rk2;
            af[p] += f;
            aw[p] = fmaf(fs, s, aw[p]);
#pragma unroll
            for (int r = 0; r < K; ++r) {
                a1[p][r] = fmaf(w1, y[r], a1[p][r]);
                const float t = w2 * y[r];
#pragma unroll
                for (int c = 0; c <= r; ++c) a2[p][r * (r + 1) / 2 + c] = fmaf(t, y[c], a2[p][r * (r + 1) / 2 + c]);
            }
#pragma unroll
            for (int d = 0; d <= K; ++d) {
                const float t = w[p][d] + dw[d];
                w[p][d] = t >= 1.f ? t - 1.f : t;
            }
        }
    }
    float s = 0.f;
#pragma unroll
    for (int p = 0; p < P; ++p) {
        s += af[p] + aw[p];
#pragma unroll
        for (int r = 0; r < K; ++r) s += a1[p][r];
#pragma unroll
        for (int r = 0; r < K2; ++r) s += a2[p][r];
    }
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// One node of the FP32 T_2 quadrature, per node: the two sines of the angle
// (cf_sin_pi), the weight sin^(nu-1) (lg2, ex2), the inner T_1 from a per-dof table
// (t1cdf_table: log2(1 + |z|) by lg2, cubic Hermite, ex2) and the weighted sum; two
// independent nodes per thread, angles advancing by a fixed step, the table L1-resident.
template <int P>
__global__ void __launch_bounds__(kThreads) t2node_rate_kernel(float* out, const float2* __restrict__ tab, int iters)
{
    const float t0 = threadIdx.x * (1.0f / 8192.0f);
    float th[P], acc[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        th[p] = 0.1f + 0.7f * (p & 3) + 0.05f * (p >> 2) + t0;
        acc[p] = 0.f;
    }
    const float dth = 0.00613f, zs = -2.3f, d0 = 0.4f, num1 = 7.5f, wgt = 0.01f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const float sp = cf_sin_pi(th[p]);
            const float sd = cf_sin_pi(d0 - th[p]);
            const float f = ptx_ex2_approx(num1 * ptx_lg2_approx(sp)) * t1cdf_table(zs * sd, tab);
            acc[p] = fmaf(wgt, f, acc[p]);
            const float t = th[p] + dth;
            th[p] = t >= 3.0f ? t - 2.9f : t;
        }
    }
    float sum = 0.f;
#pragma unroll
    for (int p = 0; p < P; ++p) sum += acc[p];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = sum;
}

__global__ void fill_t1tab_kernel(float2* tab)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < T1TAB_N) tab[i] = make_float2(-1.0f - 3.0f * i * (T1TAB_V / (T1TAB_N - 1)), -3.0f);
}

__global__ void clock_kernel(long long* out, long long spin)
{
    const long long c0 = clock64();
    while (clock64() - c0 < spin) {
    }
    if (threadIdx.x == 0) out[blockIdx.x] = clock64() - c0;
}

struct Timer {
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t init()
    {
        cudaError_t e = cudaEventCreate(&a);
        return e == cudaSuccess ? cudaEventCreate(&b) : e;
    }
    ~Timer()
    {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

// Launch `launch` once untimed, then once timed; returns seconds.
template <class F>
cudaError_t timed(Timer& t, F launch, double* secs)
{
    launch();
    cudaError_t e = cudaEventRecord(t.a);
    if (e != cudaSuccess) return e;
    launch();
    if ((e = cudaEventRecord(t.b)) != cudaSuccess) return e;
    if ((e = cudaEventSynchronize(t.b)) != cudaSuccess) return e;
    float ms = 0.f;
    if ((e = cudaEventElapsedTime(&ms, t.a, t.b)) != cudaSuccess) return e;
    *secs = ms * 1e-3;
    return cudaGetLastError();
}

// iterations so that one launch takes about `target` seconds, from a first launch of
// `probe` iterations
template <class F>
cudaError_t calibrate(Timer& t, F launch_iters, int probe, double target, int* iters, double* secs)
{
    double s = 0.0;
    cudaError_t e = timed(t, [&] { launch_iters(probe); }, &s);
    if (e != cudaSuccess) return e;
    double scale = s > 0.0 ? target / s : 1.0;
    if (scale > 1e4) scale = 1e4;
    *iters = (int)(probe * scale) > probe ? (int)(probe * scale) : probe;
    return timed(t, [&] { launch_iters(*iters); }, secs);
}

// the best of 1, 2 and 4 independent points per thread (the rate of the arithmetic alone)
template <int K, int P>
cudaError_t mix_rate_p(Timer& t, float* out, int blocks, double target, double* rate)
{
    int it = 0;
    double s = 0.0;
    cudaError_t e = calibrate(t, [&](int n) { mix_rate_kernel<K, P><<<blocks, kThreads>>>(out, n); }, 64, target, &it, &s);
    if (e == cudaSuccess) {
        const double r = (double)P * blocks * kThreads * it / s;
        if (r > *rate) *rate = r;
    }
    return e;
}

template <int K>
cudaError_t mix_rate(Timer& t, float* out, int blocks, double target, double* rate)
{
    cudaError_t e = mix_rate_p<K, 1>(t, out, blocks, target / 3, rate);
    if (e == cudaSuccess) e = mix_rate_p<K, 2>(t, out, blocks, target / 3, rate);
    if (e == cudaSuccess) e = mix_rate_p<K, 4>(t, out, blocks, target / 3, rate);
    return e;
}

template <int P>
cudaError_t t2node_rate(Timer& t, float* out, const float2* tab, int blocks, double target, double* rate)
{
    int it = 0;
    double s = 0.0;
    cudaError_t e = calibrate(t, [&](int n) { t2node_rate_kernel<P><<<blocks, kThreads>>>(out, tab, n); }, 64, target, &it, &s);
    if (e == cudaSuccess) {
        const double r = (double)P * blocks * kThreads * it / s;
        if (r > *rate) *rate = r;
    }
    return e;
}

}  // namespace

extern "C" cfust_status cfust_measure_rates(int device, double seconds, cfust_rates* out)
{
    if (!out || !(seconds > 0.0) || seconds > 5.0) {
        cf_set_global_error("cfust_measure_rates: out is NULL or seconds not in (0, 5]");
        return CFUST_EINVAL;
    }
    *out = cfust_rates{};
    int nsm = 0;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) {
        cf_set_global_error(std::string("cfust_measure_rates: ") + cudaGetErrorString(e));
        return CFUST_ECUDA;
    }
    const int blocks = 8 * nsm;
    const size_t nthr = (size_t)blocks * kThreads;
    void* buf = nullptr;
    if ((e = cudaMalloc(&buf, nthr * sizeof(double) + (size_t)nsm * sizeof(long long) +
                                  T1TAB_N * sizeof(float2))) != cudaSuccess) {
        cf_set_global_error(std::string("cfust_measure_rates: ") + cudaGetErrorString(e));
        return CFUST_ENOMEM;
    }
    float* f32 = (float*)buf;
    double* f64 = (double*)buf;
    long long* clk = (long long*)((char*)buf + nthr * sizeof(double));
    float2* t1tab = (float2*)((char*)buf + nthr * sizeof(double) + (size_t)nsm * sizeof(long long));
    Timer t;
    const double tgt = seconds / 13.0;  // 13 measurements share the budget
    int it = 0;
    double s = 0.0;
    do {
        if ((e = t.init()) != cudaSuccess) break;
        // SM clock: cycles counted by clock64() over an event-timed spin of ~tgt
        {
            const long long spin = (long long)(tgt * 1.5e9);
            if ((e = timed(t, [&] { clock_kernel<<<nsm, 32>>>(clk, spin); }, &s)) != cudaSuccess) break;
            long long c = 0;
            if ((e = cudaMemcpy(&c, clk, sizeof(c), cudaMemcpyDeviceToHost)) != cudaSuccess) break;
            out->sm_mhz = (double)c / s / 1e6;
        }
        e = calibrate(t, [&](int n) { fma32_rate_kernel<<<blocks, kThreads>>>(f32, n, 0.9999f, 1e-6f); }, 256, tgt, &it, &s);
        if (e != cudaSuccess) break;
        out->fp32_fma = 128.0 * nthr * it / s;
        e = calibrate(t, [&](int n) { fma64_rate_kernel<<<blocks, kThreads>>>(f64, n, 0.9999, 1e-6); }, 4, tgt, &it, &s);
        if (e != cudaSuccess) break;
        out->fp64_fma = 128.0 * nthr * it / s;
        e = calibrate(t, [&](int n) { mufu_rate_kernel<0><<<blocks, kThreads>>>(f32, n); }, 32, tgt, &it, &s);
        if (e != cudaSuccess) break;
        out->mufu_ex2 = 128.0 * nthr * it / s;
        e = calibrate(t, [&](int n) { mufu_rate_kernel<1><<<blocks, kThreads>>>(f32, n); }, 32, tgt, &it, &s);
        if (e != cudaSuccess) break;
        out->mufu_lg2 = 128.0 * nthr * it / s;
        e = calibrate(t, [&](int n) { mufu_rate_kernel<2><<<blocks, kThreads>>>(f32, n); }, 32, tgt, &it, &s);
        if (e != cudaSuccess) break;
        out->mufu_rcp = 128.0 * nthr * it / s;
        if ((e = mix_rate<3>(t, f32, blocks, tgt, &out->mix_points[3])) != cudaSuccess) break;
        if ((e = mix_rate<4>(t, f32, blocks, tgt, &out->mix_points[4])) != cudaSuccess) break;
        if ((e = mix_rate<5>(t, f32, blocks, tgt, &out->mix_points[5])) != cudaSuccess) break;
        if ((e = mix_rate<6>(t, f32, blocks, tgt, &out->mix_points[6])) != cudaSuccess) break;
        if ((e = mix_rate<7>(t, f32, blocks, tgt, &out->mix_points[7])) != cudaSuccess) break;
        if ((e = mix_rate<8>(t, f32, blocks, tgt, &out->mix_points[8])) != cudaSuccess) break;
        fill_t1tab_kernel<<<(T1TAB_N + 255) / 256, 256>>>(t1tab);
        if ((e = t2node_rate<1>(t, f32, t1tab, blocks, tgt / 3, &out->t2_nodes)) != cudaSuccess) break;
        if ((e = t2node_rate<2>(t, f32, t1tab, blocks, tgt / 3, &out->t2_nodes)) != cudaSuccess) break;
        if ((e = t2node_rate<4>(t, f32, t1tab, blocks, tgt / 3, &out->t2_nodes)) != cudaSuccess) break;
    } while (0);
    cudaFree(buf);
    if (e != cudaSuccess) {
        cf_set_global_error(std::string("cfust_measure_rates: ") + cudaGetErrorString(e));
        return CFUST_ECUDA;
    }
    return CFUST_OK;
}
