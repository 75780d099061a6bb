/* Seeded synthetic-input generator shared by the host (C) and device (CUDA)
 * builds of the input module.  It holds no arithmetic of the method itself.
 *
 * Counter-based generator: Philox4x32-10 as published by Salmon, Moraes,
 * Dror and Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11):
 * ten rounds of two 32x32->64 multiplies with constants 0xD2511F53 and
 * 0xCD9E8D57, key bumped by the Weyl constants 0x9E3779B9 and 0xBB67AE85.
 *
 * Element e of stream (seed, tensor_id) uses counter (j, j>>32, tensor_id, 0)
 * with j = e>>1 and key (seed, seed>>32).  The four output words give two
 * 53-bit uniforms u1, u2 in (0,1); Box-Muller gives two normals:
 * element 2j is r*cos(2*pi*u2), element 2j+1 is r*sin(2*pi*u2),
 * r = sqrt(-2 ln u1).  A uniform element uses words (0,1) if e is even and
 * words (2,3) if e is odd.
 */
#ifndef SYNTH_PHILOX_H
#define SYNTH_PHILOX_H

#include <stdint.h>
#include <math.h>

#if defined(__CUDACC__)
#define SYNTH_FN static __host__ __device__ __forceinline__
#else
#define SYNTH_FN static inline
#endif

typedef struct { uint32_t w[4]; } synth_u32x4;

SYNTH_FN synth_u32x4 synth_philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                         uint32_t k0, uint32_t k1)
{
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    synth_u32x4 out;
    out.w[0] = c0; out.w[1] = c1; out.w[2] = c2; out.w[3] = c3;
    return out;
}

/* 53-bit uniform in the open interval (0,1) from two 32-bit words. */
SYNTH_FN double synth_u53(uint32_t a, uint32_t b)
{
    uint64_t m = ((uint64_t)a << 21) | (uint64_t)(b >> 11);
    return ((double)m + 0.5) * (1.0 / 9007199254740992.0);
}

SYNTH_FN synth_u32x4 synth_draw(uint64_t seed, uint32_t tensor_id, uint64_t e)
{
    uint64_t j = e >> 1;
    return synth_philox4x32_10((uint32_t)j, (uint32_t)(j >> 32), tensor_id, 0u,
                               (uint32_t)seed, (uint32_t)(seed >> 32));
}

SYNTH_FN double synth_normal(uint64_t seed, uint32_t tensor_id, uint64_t e)
{
    synth_u32x4 r = synth_draw(seed, tensor_id, e);
    double u1 = synth_u53(r.w[0], r.w[1]);
    double u2 = synth_u53(r.w[2], r.w[3]);
    double rad = sqrt(-2.0 * log(u1));
    double ang = 6.283185307179586476925286766559 * u2;
    return (e & 1u) ? rad * sin(ang) : rad * cos(ang);
}

SYNTH_FN double synth_uniform(uint64_t seed, uint32_t tensor_id, uint64_t e)
{
    synth_u32x4 r = synth_draw(seed, tensor_id, e);
    return (e & 1u) ? synth_u53(r.w[2], r.w[3]) : synth_u53(r.w[0], r.w[1]);
}

/* Entry F_k[s][l] of the synthetic first block column:
 *   normal(seed, 0, (k*N_d + s)*N_m + l) * exp(-k/tau) * env_d[s] * env_m[l]
 * tau <= 0 means no decay; a NULL envelope means 1. */
SYNTH_FN double synth_block_entry(uint64_t seed, int64_t N_d, int64_t N_m, double tau,
                                  const double* env_d, const double* env_m,
                                  int64_t k, int64_t s, int64_t l)
{
    double v = synth_normal(seed, 0u, (uint64_t)((k * N_d + s) * N_m + l));
    if (tau > 0.0) v *= exp(-(double)k / tau);
    if (env_d) v *= env_d[s];
    if (env_m) v *= env_m[l];
    return v;
}

#endif /* SYNTH_PHILOX_H */
