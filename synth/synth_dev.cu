/* Device build of the seeded input generator (see philox.h): fills device
 * buffers with the same values as the host build, so large inputs never
 * cross the host link.  Values agree with the host build to a few ulps
 * (the libm and CUDA log/sin/cos may round differently). */
#include <cstdint>
#include <cuda_runtime.h>
#include "philox.h"

#define SYNTH_API extern "C" __attribute__((visibility("default")))

static __global__ void k_normal(uint64_t seed, uint32_t tid, uint64_t start, int64_t n,
                                double* o64, float* o32)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double v = synth_normal(seed, tid, start + (uint64_t)i);
        if (o64) o64[i] = v; else o32[i] = (float)v;
    }
}

static __global__ void k_uniform(uint64_t seed, uint32_t tid, uint64_t start, int64_t n,
                                 double lo, double hi, double* o64, float* o32)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double v = lo + (hi - lo) * synth_uniform(seed, tid, start + (uint64_t)i);
        if (o64) o64[i] = v; else o32[i] = (float)v;
    }
}

static __global__ void k_blocks(uint64_t seed, int64_t N_d, int64_t N_m, double tau,
                                const double* env_d, const double* env_m,
                                int64_t k0, int64_t n, double* out)
{
    int64_t per = N_d * N_m;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t k = k0 + i / per;
        int64_t r = i % per;
        out[i] = synth_block_entry(seed, N_d, N_m, tau, env_d, env_m, k, r / N_m, r % N_m);
    }
}

static int grid_for(int64_t n)
{
    int64_t g = (n + 255) / 256;
    if (g > 152 * 32) g = 152 * 32;
    if (g < 1) g = 1;
    return (int)g;
}

/* Each call returns the cudaError_t of its launch (0 = success). */
SYNTH_API int synth_dev_normal(uint64_t seed, uint32_t tensor_id, uint64_t start, int64_t n,
                               double* out64, float* out32, void* stream)
{
    if (n <= 0) return 0;
    k_normal<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(seed, tensor_id, start, n, out64, out32);
    return (int)cudaGetLastError();
}

SYNTH_API int synth_dev_uniform(uint64_t seed, uint32_t tensor_id, uint64_t start, int64_t n,
                                double lo, double hi, double* out64, float* out32, void* stream)
{
    if (n <= 0) return 0;
    k_uniform<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(seed, tensor_id, start, n, lo, hi,
                                                             out64, out32);
    return (int)cudaGetLastError();
}

/* env_d / env_m are device pointers or NULL. */
SYNTH_API int synth_dev_blocks(uint64_t seed, int64_t N_d, int64_t N_m, double tau,
                               const double* env_d, const double* env_m, int64_t k0, int64_t k1,
                               double* out, void* stream)
{
    int64_t n = (k1 - k0) * N_d * N_m;
    if (n <= 0) return 0;
    k_blocks<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(seed, N_d, N_m, tau, env_d, env_m, k0,
                                                            n, out);
    return (int)cudaGetLastError();
}
