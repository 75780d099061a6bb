/* Host build of the seeded input generator (see philox.h).  Plain C with
 * optional OpenMP; every entry point fills a caller-owned buffer. */
#include <stdint.h>
#include <stddef.h>
#include "philox.h"

#define SYNTH_API __attribute__((visibility("default")))

SYNTH_API void synth_host_philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                 uint32_t k0, uint32_t k1, uint32_t* out)
{
    synth_u32x4 r = synth_philox4x32_10(c0, c1, c2, c3, k0, k1);
    for (int i = 0; i < 4; ++i) out[i] = r.w[i];
}

/* out[i] = normal(seed, tensor_id, start + i) */
SYNTH_API void synth_host_normal(uint64_t seed, uint32_t tensor_id, uint64_t start,
                                 int64_t count, double* out)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < count; ++i) out[i] = synth_normal(seed, tensor_id, start + (uint64_t)i);
}

/* out[i] = lo + (hi - lo) * uniform(seed, tensor_id, start + i) */
SYNTH_API void synth_host_uniform(uint64_t seed, uint32_t tensor_id, uint64_t start,
                                  int64_t count, double lo, double hi, double* out)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < count; ++i)
        out[i] = lo + (hi - lo) * synth_uniform(seed, tensor_id, start + (uint64_t)i);
}

/* Blocks F_k for k in [k0, k1), written as out[(k-k0)][s][l] (row-major). */
SYNTH_API void synth_host_blocks(uint64_t seed, int64_t N_d, int64_t N_m, double tau,
                                 const double* env_d, const double* env_m,
                                 int64_t k0, int64_t k1, double* out)
{
    int64_t per = N_d * N_m;
    int64_t total = (k1 - k0) * per;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < total; ++i) {
        int64_t k = k0 + i / per;
        int64_t r = i % per;
        out[i] = synth_block_entry(seed, N_d, N_m, tau, env_d, env_m, k, r / N_m, r % N_m);
    }
}

/* Scattered entries out[i] = F_{k[i]}[s[i]][l[i]]. */
SYNTH_API void synth_host_block_entries(uint64_t seed, int64_t N_d, int64_t N_m, double tau,
                                        const double* env_d, const double* env_m, int64_t n,
                                        const int64_t* k, const int64_t* s, const int64_t* l,
                                        double* out)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i)
        out[i] = synth_block_entry(seed, N_d, N_m, tau, env_d, env_m, k[i], s[i], l[i]);
}
