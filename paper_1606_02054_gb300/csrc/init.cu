// init.cu -- device parts of the initialisation of Sec. 3.3 (Algorithm 1):
// random partitions of the observations and the cluster moments that eq (23)
// needs (sample mean, covariance and third moment of every cluster).
// The per-cluster arithmetic of eq (23) is O(g p^2) and runs on the host in
// FP64; each candidate's log-likelihood is the library's density pass.
#include "internal.cuh"

// label_j = floor(u g), u = SplitMix64 output for key seed ^ ((start+1) << 40) ^ (j+1)
__global__ void random_partition_kernel(long long n, int g, uint64_t seed, int start, int* labels)
{
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n;
         j += (long long)gridDim.x * blockDim.x) {
        uint64_t z = (seed ^ ((uint64_t)(start + 1) << 40) ^ (uint64_t)(j + 1)) + 0x9E3779B97F4A7C15ULL;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        z ^= z >> 31;
        const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
        const int h = (int)(u * g);
        labels[j] = h < g ? h : g - 1;
    }
}

// k-means assignment (Lloyd): label_j = argmin_h ||y_j - c_h||^2, the first centre on ties;
// every product and sum rounded on its own (no fused multiply-add), in coordinate order.
// *changes counts the labels that changed (one atomic per warp).
__global__ void kmeans_assign_kernel(Dims D, const double* __restrict__ y, const double* __restrict__ centres,
                                     int* __restrict__ labels, int* __restrict__ changes)
{
    extern __shared__ double cs[];  // g x p centres
    const int p = D.p, g = D.g;
    for (int t = threadIdx.x; t < g * p; t += blockDim.x) cs[t] = centres[t];
    __syncthreads();
    const long long stride = (long long)gridDim.x * blockDim.x;
    // the loop runs the same number of times on every lane of a warp (j past n does no work)
    const long long n_pad = (D.n + 31) / 32 * 32;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n_pad; j += stride) {
        bool changed = false;
        if (j < D.n) {
            double best = INFINITY;
            int hb = 0;
            for (int h = 0; h < g; ++h) {
                double dist = 0.0;
                for (int d = 0; d < p; ++d) {
                    const double t = __dsub_rn(y[(size_t)j * p + d], cs[h * p + d]);
                    dist = __dadd_rn(dist, __dmul_rn(t, t));
                }
                if (dist < best) {
                    best = dist;
                    hb = h;
                }
            }
            changed = labels[j] != hb;
            labels[j] = hb;
        }
        const unsigned m = __ballot_sync(0xffffffffu, changed);
        if ((threadIdx.x & 31) == 0 && m) atomicAdd(changes, __popc(m));
    }
}

cudaError_t launch_kmeans_assign(const Dims& D, const double* y, const double* centres, int* labels,
                                 int* changes, int nsm, cudaStream_t st)
{
    const long long blocks = (D.n + 255) / 256;
    const int b = (int)(blocks < 8LL * nsm ? blocks : 8LL * nsm);
    kmeans_assign_kernel<<<b, 256, sizeof(double) * D.g * D.p, st>>>(D, y, centres, labels, changes);
    return cudaGetLastError();
}

// Per-cluster sums, one block partial per block (FP64, fixed order).
//   pass 0: [count, sum y (p)]                      W = 1 + p
//   pass 1: [sum r r^T (lower, packed), sum r^3 (p)] W = p(p+1)/2 + p, r = y - mean_h
// A thread owns statistics w = threadIdx.x (+ blockDim.x ...) of every cluster, so
// no two threads update one accumulator; observations are staged per chunk.
__global__ void cluster_moments_kernel(int pass, Dims D, const double* __restrict__ y,
                                       const int* __restrict__ labels, const double* __restrict__ mean,
                                       int chunk, double* __restrict__ partial)
{
    extern __shared__ double sm[];
    const int p = D.p, g = D.g;
    const int P2 = p * (p + 1) / 2;
    const int W = pass == 0 ? 1 + p : P2 + p;
    double* acc = sm;                   // g x W
    double* yc = acc + (size_t)g * W;   // chunk x p
    int* lc = (int*)(yc + (size_t)chunk * p);
    for (int t = threadIdx.x; t < g * W; t += blockDim.x) acc[t] = 0.0;
    for (long long base = (long long)blockIdx.x * chunk; base < D.n; base += (long long)gridDim.x * chunk) {
        const int m = (int)(D.n - base < chunk ? D.n - base : chunk);
        __syncthreads();
        for (int t = threadIdx.x; t < m; t += blockDim.x) lc[t] = labels[base + t];
        __syncthreads();
        for (int t = threadIdx.x; t < m * p; t += blockDim.x) {
            double v = y[(size_t)base * p + t];
            if (pass == 1) v -= mean[(size_t)lc[t / p] * p + t % p];
            yc[t] = v;
        }
        __syncthreads();
        for (int w = threadIdx.x; w < W; w += blockDim.x) {
            int a = 0, b = 0, kind;   // 0: count, 1: y_a, 2: r_a r_b, 3: r_a^3
            if (pass == 0) {
                kind = w == 0 ? 0 : 1;
                a = w - 1;
            } else if (w < P2) {
                kind = 2;
                while ((a + 1) * (a + 2) / 2 <= w) ++a;
                b = w - a * (a + 1) / 2;
            } else {
                kind = 3;
                a = w - P2;
            }
            for (int j = 0; j < m; ++j) {
                const double* r = yc + (size_t)j * p;
                const double t = kind == 0 ? 1.0 : kind == 1 ? r[a] : kind == 2 ? r[a] * r[b] : r[a] * r[a] * r[a];
                acc[(size_t)lc[j] * W + w] += t;
            }
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < g * W; t += blockDim.x) partial[(size_t)blockIdx.x * g * W + t] = acc[t];
}

size_t cluster_moments_smem(int pass, int p, int g, int chunk)
{
    const int W = pass == 0 ? 1 + p : p * (p + 1) / 2 + p;
    return sizeof(double) * ((size_t)g * W + (size_t)chunk * p) + sizeof(int) * (size_t)chunk;
}

cudaError_t launch_random_partition(long long n, int g, uint64_t seed, int start, int* labels,
                                    cudaStream_t st)
{
    const long long blocks = (n + 255) / 256;
    random_partition_kernel<<<(int)(blocks < 4096 ? blocks : 4096), 256, 0, st>>>(n, g, seed, start, labels);
    return cudaGetLastError();
}

cudaError_t launch_cluster_moments(int pass, const Dims& D, const double* y, const int* labels,
                                   const double* mean, int chunk, int blocks, double* partial,
                                   cudaStream_t st)
{
    const size_t smem = cluster_moments_smem(pass, D.p, D.g, chunk);
    cudaError_t e = cudaFuncSetAttribute(cluster_moments_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    cluster_moments_kernel<<<blocks, 256, smem, st>>>(pass, D, y, labels, mean, chunk, partial);
    return cudaGetLastError();
}
