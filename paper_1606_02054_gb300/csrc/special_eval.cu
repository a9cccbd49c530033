// special_eval.cu -- cfust_special_f32: evaluates the FP32 normal CDF and its
// inverse exactly as the lattice integrators do (and, for comparison, the CUDA
// math library's normcdff / normcdfinvf), so tests can bound their error.
#include <cuda_runtime.h>

#include <string>

#include "cfust.h"
#include "internal.cuh"
#include "special.cuh"

__global__ void special_f32_kernel(int fn, long long count, const float* __restrict__ x,
                                   float* __restrict__ y)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        const float v = x[i];
        float r;
        switch (fn) {
        case 0: r = m_ncdf(v); break;
        case 1: r = m_ncdfinv(v); break;
        case 2: r = normcdff(v); break;
        default: r = normcdfinvf(v); break;
        }
        y[i] = r;
    }
}

extern "C" cfust_status cfust_special_f32(int fn, int64_t count, const float* x, float* y, int device)
{
    if (fn < 0 || fn > 3 || count < 0 || (count > 0 && (!x || !y))) {
        cf_set_global_error("cfust_special_f32: bad arguments");
        return CFUST_EINVAL;
    }
    if (count == 0) return CFUST_OK;
    cudaError_t e = cudaSetDevice(device);
    float *dx = nullptr, *dy = nullptr;
    if (e == cudaSuccess) e = cudaMalloc((void**)&dx, sizeof(float) * count);
    if (e == cudaSuccess) e = cudaMalloc((void**)&dy, sizeof(float) * count);
    if (e == cudaSuccess) e = cudaMemcpy(dx, x, sizeof(float) * count, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        const long long blocks = (count + 255) / 256;
        special_f32_kernel<<<(int)(blocks < 4096 ? blocks : 4096), 256>>>(fn, count, dx, dy);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(y, dy, sizeof(float) * count, cudaMemcpyDeviceToHost);
    if (dx) cudaFree(dx);
    if (dy) cudaFree(dy);
    if (e != cudaSuccess) {
        cf_set_global_error(std::string("cfust_special_f32: ") + cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? CFUST_ENOMEM : CFUST_ECUDA;
    }
    return CFUST_OK;
}
