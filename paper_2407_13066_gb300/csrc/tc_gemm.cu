// Multi-right-hand-side per-frequency products on the 5th-generation tensor
// cores (tcgen05 + TMEM + TMA), for BF16 Fhat.
//
// With B right-hand sides the per-frequency products of Alg. 2 become
// complex GEMMs, dhat(w) [N_d x B] = Fhat(w) [N_d x N_m] mhat(w) [N_m x B],
// which stay bound by the Fhat stream only if the multiply-adds run on the
// tensor cores.  Complex arithmetic is mapped to one real GEMM per frequency
// with the 4 real products per complex multiply-add ("4M"):
//
//   Fhat(w) stored interleaved [s][2l + p] (p = 0 real, 1 imaginary) is the
//   B operand as it sits in HBM (N = s rows, K = 2 ldm, K-major).
//   The A operand stacks, per 64 right-hand sides, 64 rows conj(mhat_b)
//   = [Re, -Im] interleaved and 64 rows swap(mhat_b) = [Im, Re]: row b of
//   A B^T is then sum_l Re(Fhat mhat_b) and row 64 + b is its imaginary part.
//   Only the conj rows are stored; two warps derive the swap rows from them
//   in shared memory (a per-word rotate and sign flip, unaffected by the
//   128-byte swizzle), so the spectra are read from HBM once.
//
// One CTA computes a 128 x N tile (N <= 256 rows of Fhat) over a slice of K
// (split-K); partial sums go to a buffer and a small kernel adds the splits
// and writes dhat in the layout the inverse FFT reads.  Warp 0 issues TMA
// loads into a ring of shared-memory stages, one thread of warp 1 issues
// tcgen05.mma into TMEM, and all four warps read the accumulator back with
// tcgen05.ld.  Every wait on an mbarrier is bounded in time; on timeout the
// kernel records an error code, waits (bounded) for its own copies, frees
// TMEM and returns.
#include <cmath>
#include <cuda.h>

#include "kernels.h"

namespace btt {
namespace tc {

constexpr int kTileM = 128;          // stacked rows per M tile (64 right-hand sides)
constexpr int kTileK = 64;           // BF16 elements per K tile: one 128-byte swizzle row
constexpr uint64_t kWaitNs = 2000000000ull;   // bounded waits: 2 s

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t globaltimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for the phase of `bar` with parity `parity`; false after limit_ns.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns = kWaitNs)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    while (!mbar_try_wait(bar, parity)) {
        if (globaltimer() - t0 > limit_ns) return false;
    }
    return true;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* tm, int x, int y, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"(tm), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* tm, int x, int y, int z, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"(tm), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major operand tile written by TMA
// with 128-byte swizzling: rows of 128 bytes, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t desc_kmajor_sw128(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);     // start address / 16
    d |= (uint64_t)(16 >> 4) << 16;               // leading byte offset (unused when swizzled)
    d |= (uint64_t)(1024 >> 4) << 32;             // stride byte offset: next 8-row group
    d |= (uint64_t)1 << 46;                       // descriptor version
    d |= (uint64_t)2 << 61;                       // 128-byte swizzle
    return d;
}

// Instruction descriptor: BF16 x BF16 -> FP32, both operands K-major.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N)
{
    return (1u << 4)                        // accumulator FP32
         | (1u << 7)                        // A BF16
         | (1u << 10)                       // B BF16
         | ((uint32_t)(N >> 3) << 17)       // N / 8
         | ((uint32_t)(M >> 4) << 24);      // M / 16
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// ------------------------------------------------------------ forward GEMM
// grid = (frequency w, N tile, K split); 128 threads: warp 0 TMA, warp 1
// MMA, warps 2-3 derive the swap rows, all four read the accumulator.
// part[((split * n_freq + w) * n_ntiles + nt) * NM * 128 + row][col], row in
// [0, 128 NM), col in [0, ntile_rows): partial sums of this CTA.
template <int NM, int STAGES>
__global__ void __launch_bounds__(128, 1)
k_tc_fwd(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int n_freq,
         int ntile_rows, int ktiles, int kt_per_split, int mt_stride, int mt0, float* __restrict__ part,
         int* __restrict__ err)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    constexpr int A_BYTES = kTileM * kTileK * 2;
    constexpr int NAT = NM;                  // A tiles per stage
    const int b_bytes = ntile_rows * kTileK * 2;
    const int stage_bytes = NAT * A_BYTES + b_bytes;
    constexpr uint32_t NCOLS = NM == 1 ? 256 : 512;

    __shared__ uint64_t full[STAGES], empty[STAGES], xready[STAGES], accum;
    __shared__ uint32_t tmem_base;
    __shared__ volatile int abort_flag;
    constexpr int HALF = A_BYTES / 2;   // 64 conj rows as loaded; the swap rows follow

    const int w = blockIdx.x, nt = blockIdx.y, sp = blockIdx.z;
    const int n_ntiles = gridDim.y;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int kt0 = sp * kt_per_split;
    const int nk = min(ktiles, kt0 + kt_per_split) - kt0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
            mbar_init(&xready[s], 64);
        }
        mbar_init(&accum, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(&tmem_base)), "r"(NCOLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = tmem_base;

    if (warp >= 2) {
        // ---- swap rows: (Re, -Im) -> (Im, Re) per 32-bit word of BF16 pairs
        const int t = threadIdx.x - 64;
        for (int i = 0; i < nk; ++i) {
            const int s = i % STAGES;
            const bool ok = mbar_wait(&full[s], (uint32_t)(i / STAGES) & 1u);
            if (!ok || abort_flag) {
                if (!ok) atomicExch(err, 9);
                abort_flag = 1;
                break;
            }
            unsigned char* st = smem + s * stage_bytes;
#pragma unroll
            for (int mt = 0; mt < NAT; ++mt) {
                const uint4* src = reinterpret_cast<const uint4*>(st + mt * A_BYTES);
                uint4* dst = reinterpret_cast<uint4*>(st + mt * A_BYTES + HALF);
#pragma unroll
                for (int q = 0; q < HALF / 16 / 64; ++q) {
                    uint4 v = src[t + 64 * q];
                    v.x = (v.x << 16) | ((v.x >> 16) ^ 0x8000u);
                    v.y = (v.y << 16) | ((v.y >> 16) ^ 0x8000u);
                    v.z = (v.z << 16) | ((v.z >> 16) ^ 0x8000u);
                    v.w = (v.w << 16) | ((v.w >> 16) ^ 0x8000u);
                    dst[t + 64 * q] = v;
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(&xready[s]);
        }
    } else if (warp == 0 && lane == 0) {
        // ---- TMA producer
        int issued = 0;
        for (int i = 0; i < nk; ++i) {
            const int s = i % STAGES;
            const uint32_t ph = (uint32_t)(i / STAGES) & 1u;
            if (!mbar_wait(&empty[s], ph ^ 1u) || abort_flag) {
                atomicExch(err, 1);
                abort_flag = 1;
                break;
            }
            unsigned char* st = smem + s * stage_bytes;
            mbar_expect_tx(&full[s], (uint32_t)(stage_bytes - NAT * HALF));
            const int kx = (kt0 + i) * kTileK;
#pragma unroll
            for (int mt = 0; mt < NM; ++mt)
                tma_load_2d(st + mt * A_BYTES, &tmA, kx, (w * mt_stride + mt0 + mt) * 64, &full[s]);
            tma_load_3d(st + NM * A_BYTES, &tmB, kx, nt * ntile_rows, w, &full[s]);
            ++issued;
        }
        // copies still in flight complete on their full barriers
        for (int j = issued > STAGES ? issued - STAGES : 0; j < issued; ++j)
            if (!mbar_wait(&full[j % STAGES], (uint32_t)(j / STAGES) & 1u)) atomicExch(err, 2);
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer
        const uint32_t idesc = idesc_bf16_f32(kTileM, ntile_rows);
        for (int i = 0; i < nk; ++i) {
            const int s = i % STAGES;
            const uint32_t ph = (uint32_t)(i / STAGES) & 1u;
            if (!mbar_wait(&xready[s], ph) || abort_flag) {
                atomicExch(err, 3);
                abort_flag = 1;
                break;
            }
            tc_fence_after();
            const uint32_t sa = smem_u32(smem + s * stage_bytes);
            const uint32_t sb = sa + NM * A_BYTES;
#pragma unroll
            for (int mt = 0; mt < NM; ++mt)
#pragma unroll
                for (int kk = 0; kk < kTileK / 16; ++kk)
                    mma_bf16(tbase + mt * 256, desc_kmajor_sw128(sa + mt * A_BYTES + kk * 32),
                             desc_kmajor_sw128(sb + kk * 32), idesc, (i > 0 || kk > 0) ? 1u : 0u);
            mma_commit(&empty[s]);
        }
        mma_commit(&accum);
    }
    __syncwarp();

    // ---- epilogue: TMEM -> registers -> partial sums
    const bool waited = mbar_wait(&accum, 0);
    tc_fence_after();
    if (!waited) atomicExch(err, 4);
    // tcgen05.ld is warp-collective: decide per warp
    if (__all_sync(0xffffffffu, waited && !abort_flag)) {
        const int row = warp * 32 + lane;
        const size_t tile = ((size_t)sp * n_freq + w) * n_ntiles + nt;
#pragma unroll
        for (int mt = 0; mt < NM; ++mt) {
            float* dst = part + (tile * NM * kTileM + (size_t)mt * kTileM + row) * ntile_rows;
            for (int c = 0; c < ntile_rows; c += 16) {
                float v[16];
                tmem_ld16(tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)(mt * 256 + c), v);
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    reinterpret_cast<float4*>(dst + c)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(NCOLS) : "memory");
    }
}

// ------------------------------------------------- split-pair forward GEMM
// The forward GEMM for BF16 hi+lo pairs (64 right-hand sides): each K step
// issues A_hi B_hi into the main accumulator (TMEM columns [0, 256)) and
// A_hi B_lo + A_lo B_hi into the cross accumulator ([256, 512)); the
// A_lo B_lo term is below the pair's own rounding.
//
// The tensor cores' FP32 accumulation error grows with the length of the
// chain one accumulator sums (measured ~3e-9 relative per BF16 product),
// and the pair must stay near 1e-5.  So the main accumulator restarts every
// `chain` K tiles, and eight drain warps add each finished chain into FP32
// registers (CUDA-core adds, round to nearest) while the next chain waits
// for them; the cross terms, 2^-8 of the main products, run the CTA's whole
// K range.  A CTA therefore covers a long K slice with one partial tile.
//
// grid = (frequency w, N tile, K split); warps: 0 TMA, 1 MMA, 2-3 swap
// rows (as in k_tc_fwd), 4-11 drain: warp 4 + e reads TMEM lanes
// 32 (e % 4) .. +31 and columns [128 (e / 4), +128) of the tile.
constexpr int kDrainWarps = 8;
constexpr int kFwdSplitThreads = 128 + 32 * kDrainWarps;
constexpr int kFwdSplitStages = 2;

__global__ void __launch_bounds__(kFwdSplitThreads, 1)
k_tc_fwd_split(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               const __grid_constant__ CUtensorMap tmA_lo, const __grid_constant__ CUtensorMap tmB_lo, int n_freq,
               int ntile_rows, int ktiles, int kt_per_split, int chain, int mt_stride, int mt0,
               float* __restrict__ part, int* __restrict__ err)
{
    constexpr int STAGES = kFwdSplitStages;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    constexpr int A_BYTES = kTileM * kTileK * 2;
    const int b_bytes = ntile_rows * kTileK * 2;
    const int stage_bytes = 2 * A_BYTES + 2 * b_bytes;   // A_hi, A_lo, B_hi, B_lo
    constexpr uint32_t NCOLS = 512;
    constexpr int HALF = A_BYTES / 2;   // 64 conj rows as loaded; the swap rows follow

    __shared__ uint64_t full[STAGES], empty[STAGES], xready[STAGES], chain_full, chain_free;
    __shared__ uint32_t tmem_base;
    __shared__ volatile int abort_flag;

    const int w = blockIdx.x, nt = blockIdx.y, sp = blockIdx.z;
    const int n_ntiles = gridDim.y;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int kt0 = sp * kt_per_split;
    const int nk = min(ktiles, kt0 + kt_per_split) - kt0;
    const int nchains = (nk + chain - 1) / chain;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
            mbar_init(&xready[s], 64);
        }
        mbar_init(&chain_full, 1);
        mbar_init(&chain_free, 32 * kDrainWarps);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(&tmem_base)), "r"(NCOLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = tmem_base;

    if (warp == 2 || warp == 3) {
        // ---- swap rows: (Re, -Im) -> (Im, Re) per 32-bit word of BF16 pairs
        const int t = threadIdx.x - 64;
        for (int i = 0; i < nk; ++i) {
            const int s = i % STAGES;
            const bool ok = mbar_wait(&full[s], (uint32_t)(i / STAGES) & 1u);
            if (!ok || abort_flag) {
                if (!ok) atomicExch(err, 9);
                abort_flag = 1;
                break;
            }
            unsigned char* st = smem + s * stage_bytes;
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                const uint4* src = reinterpret_cast<const uint4*>(st + a * A_BYTES);
                uint4* dst = reinterpret_cast<uint4*>(st + a * A_BYTES + HALF);
#pragma unroll
                for (int q = 0; q < HALF / 16 / 64; ++q) {
                    uint4 v = src[t + 64 * q];
                    v.x = (v.x << 16) | ((v.x >> 16) ^ 0x8000u);
                    v.y = (v.y << 16) | ((v.y >> 16) ^ 0x8000u);
                    v.z = (v.z << 16) | ((v.z >> 16) ^ 0x8000u);
                    v.w = (v.w << 16) | ((v.w >> 16) ^ 0x8000u);
                    dst[t + 64 * q] = v;
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(&xready[s]);
        }
    } else if (warp == 0) {
        if (lane == 0) {
            // ---- TMA producer
            int issued = 0;
            for (int i = 0; i < nk; ++i) {
                const int s = i % STAGES;
                const uint32_t ph = (uint32_t)(i / STAGES) & 1u;
                if (!mbar_wait(&empty[s], ph ^ 1u) || abort_flag) {
                    atomicExch(err, 1);
                    abort_flag = 1;
                    break;
                }
                unsigned char* st = smem + s * stage_bytes;
                mbar_expect_tx(&full[s], (uint32_t)(stage_bytes - 2 * HALF));
                const int kx = (kt0 + i) * kTileK;
                tma_load_2d(st, &tmA, kx, (w * mt_stride + mt0) * 64, &full[s]);
                tma_load_2d(st + A_BYTES, &tmA_lo, kx, (w * mt_stride + mt0) * 64, &full[s]);
                tma_load_3d(st + 2 * A_BYTES, &tmB, kx, nt * ntile_rows, w, &full[s]);
                tma_load_3d(st + 2 * A_BYTES + b_bytes, &tmB_lo, kx, nt * ntile_rows, w, &full[s]);
                ++issued;
            }
            // copies still in flight complete on their full barriers
            for (int j = issued > STAGES ? issued - STAGES : 0; j < issued; ++j)
                if (!mbar_wait(&full[j % STAGES], (uint32_t)(j / STAGES) & 1u)) atomicExch(err, 2);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer
            const uint32_t idesc = idesc_bf16_f32(kTileM, ntile_rows);
            for (int i = 0; i < nk; ++i) {
                const int c = i / chain, ic = i - c * chain;
                if (ic == 0 && c > 0 && !mbar_wait(&chain_free, (uint32_t)(c - 1) & 1u)) {
                    // the drain of the previous chain never finished
                    atomicExch(err, 11);
                    abort_flag = 1;
                    break;
                }
                const int s = i % STAGES;
                const uint32_t ph = (uint32_t)(i / STAGES) & 1u;
                if (!mbar_wait(&xready[s], ph) || abort_flag) {
                    atomicExch(err, 3);
                    abort_flag = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t sa = smem_u32(smem + s * stage_bytes);
                const uint32_t sb = sa + 2 * A_BYTES, sbl = sb + (uint32_t)b_bytes;
#pragma unroll
                for (int kk = 0; kk < kTileK / 16; ++kk) {
                    const uint64_t ah = desc_kmajor_sw128(sa + kk * 32), al = desc_kmajor_sw128(sa + A_BYTES + kk * 32);
                    const uint64_t bh = desc_kmajor_sw128(sb + kk * 32), bl = desc_kmajor_sw128(sbl + kk * 32);
                    mma_bf16(tbase, ah, bh, idesc, (ic > 0 || kk > 0) ? 1u : 0u);
                    mma_bf16(tbase + 256, ah, bl, idesc, (i > 0 || kk > 0) ? 1u : 0u);
                    mma_bf16(tbase + 256, al, bh, idesc, 1u);
                }
                mma_commit(&empty[s]);
                if (ic == chain - 1 || i == nk - 1) mma_commit(&chain_full);
            }
        }
    } else {
        // ---- drain warps: running FP32 sums of this thread's row and columns
        const int e = warp - 4, grp = warp & 3, h = e >> 2;
        const int row = grp * 32 + lane;
        const uint32_t lanes = (uint32_t)(grp * 32) << 16;
        float acc[128];
#pragma unroll
        for (int q = 0; q < 128; ++q) acc[q] = 0.f;
        bool ok = true;
        for (int c = 0; c < nchains; ++c) {
            const bool got = mbar_wait(&chain_full, (uint32_t)c & 1u);
            // tcgen05.ld is warp-collective: decide per warp
            ok = __all_sync(0xffffffffu, got) && !abort_flag;
            if (!ok) {
                if (lane == 0 && !got) atomicExch(err, 4);
                abort_flag = 1;
                break;
            }
            tc_fence_after();
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int col = h * 128 + 16 * q;
                if (col < ntile_rows) {
                    float v[16];
                    tmem_ld16(tbase + lanes + (uint32_t)col, v);
#pragma unroll
                    for (int i = 0; i < 16; ++i) acc[16 * q + i] += v[i];
                }
            }
            tc_fence_before();
            mbar_arrive(&chain_free);
        }
        if (ok && nchains > 0) {
            // the last chain's commit also covers every cross-term product
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int col = h * 128 + 16 * q;
                if (col < ntile_rows) {
                    float v[16];
                    tmem_ld16(tbase + lanes + (uint32_t)(256 + col), v);
#pragma unroll
                    for (int i = 0; i < 16; ++i) acc[16 * q + i] += v[i];
                }
            }
            const size_t tile = ((size_t)sp * n_freq + w) * n_ntiles + nt;
            float* dst = part + (tile * kTileM + row) * ntile_rows;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int col = h * 128 + 16 * q;
                if (col < ntile_rows) {
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        reinterpret_cast<float4*>(dst + col)[u] =
                            make_float4(acc[16 * q + 4 * u], acc[16 * q + 4 * u + 1], acc[16 * q + 4 * u + 2],
                                        acc[16 * q + 4 * u + 3]);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(NCOLS) : "memory");
    }
}

// dhat[b][w][s] = sum over splits of (row j, row 64 + j) of the partial tile,
// b = 64 mt + j (b counted within this launch).
__global__ void k_tc_reduce(const float* __restrict__ part, int nsplit, int n_freq, int n_ntiles, int NM,
                            int ntile_rows, int N_d, int nb, float2* __restrict__ dh, int64_t dbs)
{
    const int64_t total = (int64_t)nb * n_freq * N_d;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int s = (int)(i % N_d);
        const int w = (int)((i / N_d) % n_freq);
        const int b = (int)(i / ((int64_t)N_d * n_freq));
        const int nt = s / ntile_rows, col = s - nt * ntile_rows;
        const int mt = b >> 6, j = b & 63;
        float re = 0.f, im = 0.f;
        for (int sp = 0; sp < nsplit; ++sp) {
            const size_t tile = ((size_t)sp * n_freq + w) * n_ntiles + nt;
            const float* t = part + (tile * NM * kTileM + (size_t)mt * kTileM) * ntile_rows;
            re += t[(size_t)j * ntile_rows + col];
            im += t[(size_t)(64 + j) * ntile_rows + col];
        }
        dh[(int64_t)b * dbs + (int64_t)w * N_d + s] = make_float2(re, im);
    }
}

// Shared-memory descriptor of an MN-major operand tile written by TMA with
// 128-byte swizzling as blocks of 64 MN-elements (128 B) x K rows: K rows 128
// bytes apart in 8-row groups of 1024 bytes (SBO), MN blocks `lbo` apart.
__device__ __forceinline__ uint64_t desc_mnmajor_sw128(uint32_t saddr, uint32_t lbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;  // next 64-element block along N
    d |= (uint64_t)(1024 >> 4) << 32;             // next 8-row group along K
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// ------------------------------------------------------------ adjoint GEMM
// mhat_b[l] = sum_s conj(Fhat[s][l]) dhat_b[s] (Alg. 3) for 64 vectors.
// B operand: Fhat(w) as stored, read MN-major: N = 256 interleaved reals
// 2l + p of 128 columns l, K = s.  A operand: rows 2j = Re(dhat_j), rows
// 2j + 1 = Im(dhat_j), K = s (K-major).  With D = A B^T:
//   Re mhat_j[l] = D[2j][2l] + D[2j+1][2l+1],  Im mhat_j[l] = D[2j+1][2l] - D[2j][2l+1].
// Row i of D sits in TMEM lane i, so the two rows of vector j are
// neighbouring lanes of one warp: the epilogue pairs them with a warp
// shuffle and stores straight from registers.
//
// Persistent, one CTA per SM, 320 threads: warp 0 streams tiles (frequency,
// 128 columns) through a ring of shared-memory stages with TMA, warp 1
// allocates TMEM and issues the MMAs into one of two accumulators, warps
// 2-9 drain the other accumulator (tcgen05.ld -> shuffle -> combined
// complex columns -> global stores; two warps per TMEM lane quarter, each
// half the columns), so the epilogue of one tile overlaps the loads and
// MMAs of the next.
// SPLIT (BF16 hi+lo pairs): stages hold A_hi, A_lo, B_hi, B_lo; each K step
// issues A_hi B_hi + A_hi B_lo + A_lo B_hi.
constexpr int kAdjN = 256;
constexpr int kAdjThreads = 320;
constexpr int kAdjEpiWarps = kAdjThreads / 32 - 2;     // two per TMEM lane quarter
constexpr int kAdjA = kTileM * kTileK * 2;             // 16 KB
constexpr int kAdjBlk = kTileK * kTileK * 2;           // 64 reals x 64 rows: 8 KB
constexpr int kAdjXPitch = 36;                         // floats per row of an epilogue transpose
template <bool SPLIT> struct AdjCfg {
    static constexpr int kParts = SPLIT ? 2 : 1;
    static constexpr int kStages = SPLIT ? 2 : 4;
    static constexpr int kStage = kParts * (kAdjA + (kAdjN / 64) * kAdjBlk);
    static constexpr int kSmem = kStages * kStage + kAdjEpiWarps * 16 * kAdjXPitch * 4 + 1024;
};
static_assert(AdjCfg<true>::kSmem <= 227 * 1024 - 1024, "split adjoint stages exceed shared memory");

// OUT16: mhat is written as BF16 pairs (for the inverse transform's BF16
// input form; half the output bytes), else as complex64.
template <bool SPLIT, bool OUT16>
__global__ void __launch_bounds__(kAdjThreads, 1)
k_tc_adj(const __grid_constant__ CUtensorMap tmD, const __grid_constant__ CUtensorMap tmF,
         const __grid_constant__ CUtensorMap tmD_lo, const __grid_constant__ CUtensorMap tmF_lo, int n_freq,
         int N_d, int N_m, int ldm, int kd_tiles, int n_ntiles, int mt_stride, int mt0, int nb,
         void* __restrict__ mh_out, int64_t mbs, int* __restrict__ err)
{
    static_assert(!(SPLIT && OUT16), "split pairs keep complex64 mhat");
    using C = AdjCfg<SPLIT>;
    constexpr int kAdjStages = C::kStages;
    constexpr int kAdjStage = C::kStage;
    constexpr int kHalf = kAdjA + (kAdjN / 64) * kAdjBlk;   // one part: A tile + B blocks
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    constexpr uint32_t NCOLS = 512;
    float* xbuf = reinterpret_cast<float*>(smem + kAdjStages * kAdjStage);   // epilogue transposes

    __shared__ uint64_t full[kAdjStages], empty[kAdjStages], tfull[2], tempty[2];
    __shared__ uint32_t tmem_base;
    __shared__ volatile int abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ntiles = n_freq * n_ntiles;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kAdjStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&tfull[a], 1);
            mbar_init(&tempty[a], 32 * kAdjEpiWarps);
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(&tmem_base)), "r"(NCOLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = tmem_base;

    if (warp == 0) {
        if (lane == 0) {
            // ---- TMA producer
            int it = 0;
            for (int tile = blockIdx.x; tile < ntiles && !abort_flag; tile += gridDim.x) {
                const int w = tile / n_ntiles, n0 = (tile - w * n_ntiles) * kAdjN;
                for (int kt = 0; kt < kd_tiles; ++kt, ++it) {
                    const int s = it % kAdjStages;
                    if (!mbar_wait(&empty[s], ((uint32_t)(it / kAdjStages) & 1u) ^ 1u) || abort_flag) {
                        atomicExch(err, 5);
                        abort_flag = 1;
                        break;
                    }
                    unsigned char* st = smem + s * kAdjStage;
                    mbar_expect_tx(&full[s], (uint32_t)kAdjStage);
                    tma_load_2d(st, &tmD, kt * kTileK, (w * mt_stride + mt0) * kTileM, &full[s]);
#pragma unroll
                    for (int a = 0; a < kAdjN / 64; ++a)
                        tma_load_3d(st + kAdjA + a * kAdjBlk, &tmF, n0 + 64 * a, kt * kTileK, w, &full[s]);
                    if constexpr (SPLIT) {
                        tma_load_2d(st + kHalf, &tmD_lo, kt * kTileK, (w * mt_stride + mt0) * kTileM, &full[s]);
#pragma unroll
                        for (int a = 0; a < kAdjN / 64; ++a)
                            tma_load_3d(st + kHalf + kAdjA + a * kAdjBlk, &tmF_lo, n0 + 64 * a, kt * kTileK, w,
                                        &full[s]);
                    }
                }
            }
            // copies still in flight complete on their full barriers
            for (int j = it > kAdjStages ? it - kAdjStages : 0; j < it; ++j)
                if (!mbar_wait(&full[j % kAdjStages], (uint32_t)(j / kAdjStages) & 1u)) atomicExch(err, 6);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer: A K-major, B MN-major (bit 16), M = 128, N = 256
            const uint32_t idesc = idesc_bf16_f32(kTileM, kAdjN) | (1u << 16);
            int it = 0, ti = 0;
            for (int tile = blockIdx.x; tile < ntiles && !abort_flag; tile += gridDim.x, ++ti) {
                const int acc = ti & 1;
                if (!mbar_wait(&tempty[acc], ((uint32_t)(ti >> 1) & 1u) ^ 1u)) {
                    atomicExch(err, 7);
                    abort_flag = 1;
                    break;
                }
                tc_fence_after();
                for (int kt = 0; kt < kd_tiles; ++kt, ++it) {
                    const int s = it % kAdjStages;
                    if (!mbar_wait(&full[s], (uint32_t)(it / kAdjStages) & 1u) || abort_flag) {
                        atomicExch(err, 7);
                        abort_flag = 1;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sa = smem_u32(smem + s * kAdjStage);
                    const uint32_t sb = sa + kAdjA;
                    // K steps past N_d would multiply the copies' zero fill
                    const int nkk = min(kTileK / 16, (N_d - kt * kTileK + 15) / 16);
#pragma unroll
                    for (int kk = 0; kk < kTileK / 16; ++kk) {
                        if (kk >= nkk) break;
                        const uint64_t ah = desc_kmajor_sw128(sa + kk * 32);
                        const uint64_t bh = desc_mnmajor_sw128(sb + kk * 2048, kAdjBlk);
                        mma_bf16(tbase + acc * 256, ah, bh, idesc, (kt > 0 || kk > 0) ? 1u : 0u);
                        if constexpr (SPLIT) {
                            const uint64_t al = desc_kmajor_sw128(sa + kHalf + kk * 32);
                            const uint64_t bl = desc_mnmajor_sw128(sb + kHalf + kk * 2048, kAdjBlk);
                            mma_bf16(tbase + acc * 256, ah, bl, idesc, 1u);
                            mma_bf16(tbase + acc * 256, al, bh, idesc, 1u);
                        }
                    }
                    mma_commit(&empty[s]);
                }
                mma_commit(&tfull[acc]);
            }
        }
    } else {
        // ---- epilogue warps 2..9: TMEM lane group grp = warp % 4 holds
        // rows 32 grp .. +31, i.e. vectors j = 16 grp .. +15 (lane 2j' the
        // Re row, lane 2j' + 1 the Im row of vector 16 grp + j'); two warps
        // per group, each draining half of the 256 accumulator columns (the
        // drain is a chain of TMEM load, shuffle, transpose and stores, so
        // halving it per warp halves the epilogue's time per tile)
        const int grp = warp & 3;
        const int cbeg = ((warp - 2) >> 2) * (kAdjN / 2);
        const int odd = lane & 1;
        const uint32_t lanes = (uint32_t)(grp * 32) << 16;
        float* xw = xbuf + (warp - 2) * 16 * kAdjXPitch;
        int ti = 0;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++ti) {
            const int acc = ti & 1;
            const bool ok = mbar_wait(&tfull[acc], (uint32_t)(ti >> 1) & 1u);
            // tcgen05.ld is warp-collective: decide per warp
            if (!__all_sync(0xffffffffu, ok) || abort_flag) {
                if (lane == 0) atomicExch(err, 8);
                abort_flag = 1;
                break;
            }
            tc_fence_after();
            const int w = tile / n_ntiles, n0 = (tile - w * n_ntiles) * kAdjN;
            // a warp whose 16 vectors all lie beyond the batch has nothing to
            // store: it skips the drain (warp-uniform) and only hands the
            // accumulator back
            const bool live = mt0 * 64 + 16 * grp < nb;
#pragma unroll 1
            for (int c0 = cbeg; live && c0 < cbeg + kAdjN / 2; c0 += 32) {
                // v[2q + p] = D[row][c0 + 2q + p]: column l = (n0 + c0) / 2 + q
                float v[32];
                tmem_ld32(tbase + lanes + (uint32_t)(acc * 256 + c0), v);
                // the even lane finishes columns q < 8, the odd lane q >= 8;
                // each takes the partner row's values for its own columns
                float u[16];
#pragma unroll
                for (int k = 0; k < 16; ++k) u[k] = __shfl_xor_sync(0xffffffffu, odd ? v[k] : v[16 + k], 1);
                float o[16];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const float r0 = odd ? u[2 * q] : v[2 * q], r1 = odd ? u[2 * q + 1] : v[2 * q + 1];
                    const float m0 = odd ? v[16 + 2 * q] : u[2 * q], m1 = odd ? v[17 + 2 * q] : u[2 * q + 1];
                    o[2 * q] = r0 + m1;
                    o[2 * q + 1] = m0 - r1;
                }
                // transpose through this warp's slice: [vector j'][16 columns],
                // rows 144 bytes apart (16-byte accesses of a warp then fall in
                // distinct bank groups), so that 8 lanes store one vector's
                // 128-byte line
#pragma unroll
                for (int u4 = 0; u4 < 4; ++u4)
                    *reinterpret_cast<float4*>(xw + (lane >> 1) * kAdjXPitch + 16 * odd + 4 * u4) =
                        make_float4(o[4 * u4], o[4 * u4 + 1], o[4 * u4 + 2], o[4 * u4 + 3]);
                __syncwarp();
                const int lc = (n0 + c0) / 2 + 2 * (lane & 7);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int jv = 4 * i + (lane >> 3);
                    const float4 q4 = *reinterpret_cast<const float4*>(xw + jv * kAdjXPitch + 4 * (lane & 7));
                    const int bv = mt0 * 64 + 16 * grp + jv;
                    if (bv < nb) {
                        const int64_t o = (int64_t)bv * mbs + (int64_t)w * ldm + lc;
                        if constexpr (OUT16) {
                            __nv_bfloat162* d = static_cast<__nv_bfloat162*>(mh_out) + o;
                            const __nv_bfloat162 h0 = __floats2bfloat162_rn(q4.x, q4.y);
                            const __nv_bfloat162 h1 = __floats2bfloat162_rn(q4.z, q4.w);
                            if (lc + 2 <= N_m) {
                                // 8-byte aligned: ldm % 4 == 0, lc even
                                __nv_bfloat162 two[2] = {h0, h1};
                                *reinterpret_cast<uint2*>(d) = *reinterpret_cast<const uint2*>(two);
                            } else if (lc < N_m) {
                                d[0] = h0;
                            }
                        } else {
                            float2* d = static_cast<float2*>(mh_out) + o;
                            if (lc + 2 <= N_m) {
                                *reinterpret_cast<float4*>(d) = q4;   // 16-byte aligned: ldm % 4 == 0, lc even
                            } else if (lc < N_m) {
                                d[0] = make_float2(q4.x, q4.y);
                            }
                        }
                    }
                }
                __syncwarp();
            }
            // accumulator fully read: hand it back to the MMA warp
            tc_fence_before();
            mbar_arrive(&tempty[acc]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(NCOLS) : "memory");
    }
}

// dhat[b][w][s] (complex64) -> stacked BF16 rows of the adjoint's A
// operand: row (w*mt_stride + b/64)*128 + 2 (b%64) = Re, the next row = Im,
// length kd.  With lo_off != 0 the BF16 remainders v - bf16(v) go to
// DA + lo_off.
__global__ void k_stack_planar(const float2* __restrict__ dh, int64_t dbs, int n_freq, int N_d, int nb,
                               int mt_stride, int kd, __nv_bfloat16* __restrict__ DA, int64_t lo_off)
{
    const int64_t total = (int64_t)nb * n_freq * N_d;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int s = (int)(i % N_d);
        const int w = (int)((i / N_d) % n_freq);
        const int b = (int)(i / ((int64_t)N_d * n_freq));
        const float2 v = dh[(int64_t)b * dbs + (int64_t)w * N_d + s];
        const int64_t row = ((int64_t)w * mt_stride + (b >> 6)) * kTileM + 2 * (b & 63);
        const __nv_bfloat16 re = __float2bfloat16_rn(v.x), im = __float2bfloat16_rn(v.y);
        DA[row * kd + s] = re;
        DA[(row + 1) * kd + s] = im;
        if (lo_off) {
            DA[lo_off + row * kd + s] = __float2bfloat16_rn(v.x - __bfloat162float(re));
            DA[lo_off + (row + 1) * kd + s] = __float2bfloat16_rn(v.y - __bfloat162float(im));
        }
    }
}

// Self test of the bounded waits: thread 0 waits on an mbarrier that nothing
// arrives at; the wait gives up after limit_ns and the kernel records code 10.
__global__ void k_wait_selftest(int* __restrict__ err, uint64_t limit_ns)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0 && !mbar_wait(&bar, 0, limit_ns)) atomicExch(err, 10);
}

}  // namespace tc

// ---------------------------------------------------------------- host side
namespace {

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn()
{
    static EncodeTiled fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
    }
    return fn;
}

template <int NM, int STAGES> size_t fwd_smem(int ntile_rows)
{
    return (size_t)STAGES * (NM * tc::kTileM * tc::kTileK * 2 + ntile_rows * tc::kTileK * 2) + 1024;
}

// split pairs: stages of A_hi, A_lo, B_hi, B_lo
size_t fwd_split_smem(int ntile_rows)
{
    return (size_t)tc::kFwdSplitStages * (2 * tc::kTileM * tc::kTileK * 2 + 2 * ntile_rows * tc::kTileK * 2) + 1024;
}

}  // namespace

// longest accumulation chain (K tiles of 64) per accumulator for split pairs
constexpr int kSplitChainTiles = 24;

TcPlan tc_plan(int n_freq, int N_d, int ldm, int max_nrhs, bool split)
{
    TcPlan p{};
    p.split = split;
    p.K2 = 2 * ldm;
    p.ktiles = (p.K2 + tc::kTileK - 1) / tc::kTileK;
    p.n_ntiles = (N_d + 255) / 256;
    const int per = (N_d + p.n_ntiles - 1) / p.n_ntiles;
    p.ntile_rows = (per + 15) / 16 * 16;
    p.mt_alloc = (max_nrhs + 63) / 64;
    int dev = 0, nsm = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    // K splits: about 4 CTAs per SM over the frequencies and N tiles, at
    // least 8 K tiles per split.  (Split pairs bound the tensor-core
    // accumulation chain inside the kernel, k_tc_fwd_split, so their splits
    // only balance the load.)
    const int tiles = n_freq * p.n_ntiles;
    int want = (4 * nsm + tiles - 1) / tiles;
    int maxs = p.ktiles / 8 > 0 ? p.ktiles / 8 : 1;
    int S = want < 1 ? 1 : (want > maxs ? maxs : want);
    {
        // one CTA per SM (shared memory): among want .. 4 want splits take
        // the one whose CTAs fill whole waves of nsm best, charging each
        // split its partial tile (written, then read by the reduction)
        // against the operand bytes of a tile
        const double ops = (double)(split ? 2 : 1) * (p.ntile_rows + 64) * p.K2 * 2;
        const double ptile = 2.0 * tc::kTileM * p.ntile_rows * 4;
        double best = 1e30;
        const int s0 = S, s1 = 4 * S < maxs ? 4 * S : maxs;
        for (int c = s0; c <= s1; ++c) {
            const int kps = (p.ktiles + c - 1) / c;
            const int ns = (p.ktiles + kps - 1) / kps;
            const double ctas = (double)tiles * ns;
            const double cost = std::ceil(ctas / nsm) * nsm / ctas * (1.0 + ns * ptile / ops);
            if (cost < best - 1e-9) {
                best = cost;
                S = c;
            }
        }
    }
    p.kt_per_split = (p.ktiles + S - 1) / S;
    p.nsplit = (p.ktiles + p.kt_per_split - 1) / p.kt_per_split;
    p.part_floats = (size_t)p.nsplit * n_freq * p.n_ntiles * 2 * tc::kTileM * p.ntile_rows;
    p.kd = (N_d + 7) / 8 * 8;
    const size_t dplane = (size_t)n_freq * p.mt_alloc * tc::kTileM * p.kd;   // BF16 elements
    p.dstack_bytes = dplane * 2 * (split ? 2 : 1);
    p.ds_lo = split ? (int64_t)dplane : 0;
    p.xs_lo = split ? (int64_t)n_freq * p.mt_alloc * 64 * ldm : 0;
    return p;
}

namespace {

// The four operand maps over one set of planes (hi, or lo of a split pair).
cudaError_t encode_maps(EncodeTiled enc, const TcPlan& p, void* xstack, const void* fhat, void* dstack,
                        int n_freq, int N_d, CUtensorMap* tmA, CUtensorMap* tmB, CUtensorMap* tmD,
                        CUtensorMap* tmF)
{
    {
        // A: conj spectra [w][mt][64][K2] BF16 as 2-D (K2, rows)
        cuuint64_t dims[2] = {(cuuint64_t)p.K2, (cuuint64_t)n_freq * p.mt_alloc * 64};
        cuuint64_t strides[1] = {(cuuint64_t)p.K2 * 2};
        cuuint32_t box[2] = {(cuuint32_t)tc::kTileK, 64};
        cuuint32_t es[2] = {1, 1};
        if (enc(tmA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, xstack, dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    {
        // B: Fhat [w][s][K2] BF16 as 3-D (K2, N_d, w); rows >= N_d read as zero
        cuuint64_t dims[3] = {(cuuint64_t)p.K2, (cuuint64_t)N_d, (cuuint64_t)n_freq};
        cuuint64_t strides[2] = {(cuuint64_t)p.K2 * 2, (cuuint64_t)p.K2 * 2 * N_d};
        cuuint32_t box[3] = {(cuuint32_t)tc::kTileK, (cuuint32_t)p.ntile_rows, 1};
        cuuint32_t es[3] = {1, 1, 1};
        if (enc(tmB, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(fhat), dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    {
        // adjoint A: stacked planar dhat [w][mt][128][kd] BF16 as 2-D (N_d, rows);
        // columns >= N_d read as zero
        cuuint64_t dims[2] = {(cuuint64_t)N_d, (cuuint64_t)n_freq * p.mt_alloc * tc::kTileM};
        cuuint64_t strides[1] = {(cuuint64_t)p.kd * 2};
        cuuint32_t box[2] = {(cuuint32_t)tc::kTileK, (cuuint32_t)tc::kTileM};
        cuuint32_t es[2] = {1, 1};
        if (enc(tmD, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, dstack, dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    {
        // adjoint B: Fhat [w][s][K2] BF16 as 3-D (K2, N_d, w), boxes of 64 reals x 64 rows
        cuuint64_t dims[3] = {(cuuint64_t)p.K2, (cuuint64_t)N_d, (cuuint64_t)n_freq};
        cuuint64_t strides[2] = {(cuuint64_t)p.K2 * 2, (cuuint64_t)p.K2 * 2 * N_d};
        cuuint32_t box[3] = {(cuuint32_t)tc::kTileK, (cuuint32_t)tc::kTileK, 1};
        cuuint32_t es[3] = {1, 1, 1};
        if (enc(tmF, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(fhat), dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    return cudaSuccess;
}

}  // namespace

cudaError_t tc_prepare(TcPlan* p, void* xstack, const void* fhat_bf16, int n_freq, int N_d)
{
    // p->dstack must be set by the caller (stacked planar dhat buffer)
    EncodeTiled enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    cudaError_t e = encode_maps(enc, *p, xstack, fhat_bf16, p->dstack, n_freq, N_d, &p->tmA, &p->tmB, &p->tmD,
                                &p->tmF);
    if (e != cudaSuccess) return e;
    if (p->split) {
        // lo planes: spectra and data spectra remainders, and the lo plane of Fhat
        const size_t fplane = (size_t)n_freq * N_d * p->K2 * 2;   // bytes of one Fhat plane
        e = encode_maps(enc, *p, static_cast<char*>(xstack) + p->xs_lo * 4,
                        static_cast<const char*>(fhat_bf16) + fplane, static_cast<char*>(p->dstack) + p->ds_lo * 2,
                        n_freq, N_d, &p->tmA_lo, &p->tmB_lo, &p->tmD_lo, &p->tmF_lo);
        if (e != cudaSuccess) return e;
    } else {
        p->tmA_lo = p->tmA;
        p->tmB_lo = p->tmB;
        p->tmD_lo = p->tmD;
        p->tmF_lo = p->tmF;
    }
    e = cudaFuncSetAttribute(tc::k_tc_fwd<1, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)fwd_smem<1, 4>(256));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(tc::k_tc_fwd<2, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)fwd_smem<2, 3>(256));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(tc::k_tc_fwd_split, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)fwd_split_smem(256));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(tc::k_tc_adj<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 tc::AdjCfg<false>::kSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(tc::k_tc_adj<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 tc::AdjCfg<false>::kSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(tc::k_tc_adj<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 tc::AdjCfg<true>::kSmem);
    p->ready = e == cudaSuccess;
    return e;
}

cudaError_t launch_tc_adj(const TcPlan& p, int n_freq, int N_d, int N_m, int ldm, int nrhs, const float2* dh,
                          int64_t dbs, int* err, void* mh, int64_t mbs, cudaStream_t st, bool out_bf16)
{
    if (out_bf16 && p.split) return cudaErrorInvalidValue;
    if (!p.ready) return cudaErrorNotReady;
    {
        const int64_t total = (int64_t)nrhs * n_freq * N_d;
        const int blocks = (int)((total + 255) / 256 < 152 * 16 ? (total + 255) / 256 : 152 * 16);
        tc::k_stack_planar<<<blocks, 256, 0, st>>>(dh, dbs, n_freq, N_d, nrhs, p.mt_alloc, p.kd,
                                                   static_cast<__nv_bfloat16*>(p.dstack), p.ds_lo);
        count_launch();
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const int kd_tiles = (N_d + tc::kTileK - 1) / tc::kTileK;
    const int n_ntiles = (2 * ldm + tc::kAdjN - 1) / tc::kAdjN;
    int dev = 0, nsm = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int ntiles = n_freq * n_ntiles;
    const int grid = ntiles < nsm ? ntiles : nsm;
    for (int b0 = 0; b0 < nrhs; b0 += 64) {
        if (p.split)
            tc::k_tc_adj<true, false><<<grid, tc::kAdjThreads, tc::AdjCfg<true>::kSmem, st>>>(
                p.tmD, p.tmF, p.tmD_lo, p.tmF_lo, n_freq, N_d, N_m, ldm, kd_tiles, n_ntiles, p.mt_alloc, b0 / 64, nrhs,
                mh, mbs, err);
        else if (out_bf16)
            tc::k_tc_adj<false, true><<<grid, tc::kAdjThreads, tc::AdjCfg<false>::kSmem, st>>>(
                p.tmD, p.tmF, p.tmD_lo, p.tmF_lo, n_freq, N_d, N_m, ldm, kd_tiles, n_ntiles, p.mt_alloc, b0 / 64, nrhs,
                mh, mbs, err);
        else
            tc::k_tc_adj<false, false><<<grid, tc::kAdjThreads, tc::AdjCfg<false>::kSmem, st>>>(
                p.tmD, p.tmF, p.tmD_lo, p.tmF_lo, n_freq, N_d, N_m, ldm, kd_tiles, n_ntiles, p.mt_alloc, b0 / 64, nrhs,
                mh, mbs, err);
        count_launch();
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_wait_selftest(int* err, double seconds, cudaStream_t st)
{
    tc::k_wait_selftest<<<1, 32, 0, st>>>(err, (uint64_t)(seconds * 1e9));
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_tc_fwd(const TcPlan& p, int n_freq, int N_d, int nrhs, float* part, int* err, float2* dh,
                          int64_t dbs, cudaStream_t st)
{
    if (!p.ready) return cudaErrorNotReady;
    const int step = p.split ? 64 : 128;   // split pairs: one 64-vector tile per launch
    for (int b0 = 0; b0 < nrhs; b0 += step) {
        const int nb = nrhs - b0 < step ? nrhs - b0 : step;
        const int NM = (nb + 63) / 64;
        dim3 grid((unsigned)n_freq, (unsigned)p.n_ntiles, (unsigned)p.nsplit);
        if (p.split)
            tc::k_tc_fwd_split<<<grid, tc::kFwdSplitThreads, fwd_split_smem(p.ntile_rows), st>>>(
                p.tmA, p.tmB, p.tmA_lo, p.tmB_lo, n_freq, p.ntile_rows, p.ktiles, p.kt_per_split, kSplitChainTiles,
                p.mt_alloc, b0 / 64, part, err);
        else if (NM == 1)
            tc::k_tc_fwd<1, 4><<<grid, 128, fwd_smem<1, 4>(p.ntile_rows), st>>>(
                p.tmA, p.tmB, n_freq, p.ntile_rows, p.ktiles, p.kt_per_split, p.mt_alloc, b0 / 64, part, err);
        else
            tc::k_tc_fwd<2, 3><<<grid, 128, fwd_smem<2, 3>(p.ntile_rows), st>>>(
                p.tmA, p.tmB, n_freq, p.ntile_rows, p.ktiles, p.kt_per_split, p.mt_alloc, b0 / 64, part, err);
        count_launch();
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        const int64_t total = (int64_t)nb * n_freq * N_d;
        const int blocks = (int)((total + 255) / 256 < 152 * 16 ? (total + 255) / 256 : 152 * 16);
        tc::k_tc_reduce<<<blocks, 256, 0, st>>>(part, p.nsplit, n_freq, p.n_ntiles, NM, p.ntile_rows, N_d, nb,
                                                dh + (int64_t)b0 * dbs, dbs);
        count_launch();
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace btt
