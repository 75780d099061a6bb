// Time transforms of FP32 vectors with the radix plan fixed at compile time
// for the common lengths 2 N_t in {128, 256, 512, 1024, 2048, 4096, 2000,
// 4000, 8000}.
//
// Same transforms as the generic kernels in fft_kernels.cu (decimation in
// frequency forward, in time inverse, in place in shared memory, see
// fft.cuh), with two differences that matter for throughput:
//   * every index computation is a compile-time constant expression (the
//     divisions by pass strides become multiply-shifts), and
//   * the zero padding is never materialised: the first forward pass reads
//     the N_t real samples straight from memory (its other inputs are the
//     padding zeros), and the last inverse pass emits only the N_t samples
//     that are kept (the unpad of Alg. 2), straight to memory or, in the
//     Hessian's middle step, back into shared memory for the next forward
//     transform.
// Two kernel forms: pair kernels (one complex sequence of two real columns
// per butterfly, scalar FP32) and, at the lengths where they measured
// faster, quad kernels (two sequences per butterfly in paired FP32
// instructions, fftq.cuh), which issue a third fewer instructions per column
// pair; the quad kernels fuse the unpack of the real spectra into the last
// forward pass (and the Hermitian load into the first inverse pass), in
// 512-thread CTAs with one lane of a quad per thread in the fused pass, or
// in 256-thread CTAs with both.
// For the long plans (2 N_t >= 2000), whose 64 KB tiles are only a few
// columns wide, the transforms run on clusters of four CTAs (cluster
// kernels below) with four times wider rows, where that measured faster.
// The launchers return false for lengths without a fixed plan; the generic
// kernels take those.
#include <type_traits>

#include <cooperative_groups.h>

#include "fft.cuh"
#include "fftq.cuh"
#include "kernels.h"

namespace btt {
namespace {

constexpr int NT = kFftThreads;

// Shared-memory and table accesses of the transforms, index-checked in the
// bounds-check build (an access outside the extent is recorded and skipped).
template <typename V> __device__ __forceinline__ V sld(const V* a, int i, int n, int site = CK_FFT_SMEM)
{
    return BTT_IN(i, n, site) ? a[i] : V{};
}
template <typename V> __device__ __forceinline__ void sst(V* a, int i, int n, V v, int site = CK_FFT_SMEM)
{
    if (BTT_IN(i, n, site)) a[i] = v;
}
template <typename V> __device__ __forceinline__ V tld(const V* a, int i, int n)
{
    return BTT_IN(i, n, CK_FFT_TABLE) ? __ldg(a + i) : V{};
}

// CTAs per SM for the forward and inverse transforms: three 512-thread CTAs
// fit the 64 KB buffers when the kernel fits in 40 registers without
// spilling, which holds for these plans (checked with -Xptxas -v); the
// others (three radix-8 passes and more, and the Hessian's middle kernel)
// keep the register count they need.
template <int L, int WL> constexpr int min_blocks()
{
    return ((L << WL) * 8 <= 65536 && (L == 128 || L == 256 || L == 512 || L == 2000 || L == 4000 || L == 8000)) ? 3
                                                                                                              : 1;
}

template <typename V, int R, int L, int M, int WL, bool INV>
__device__ __forceinline__ void pass(V* buf, const V* __restrict__ tw)
{
    constexpr int Wc = 1 << WL, S = M / R, nb = (L / R) << WL, tstep = L / M;
    for (int b = threadIdx.x; b < nb; b += NT) {
        const int c = b & (Wc - 1), j = b >> WL;
        const int blk = j / S, n1 = j - blk * S;
        const int base = blk * M + n1;
        V v[R];
#pragma unroll
        for (int i = 0; i < R; ++i) v[i] = sld(buf, ((base + i * S) << WL) + c, L << WL);
        if (INV) {
            if (n1 != 0) {
#pragma unroll
                for (int k = 1; k < R; ++k) {
                    V w = sld(tw, n1 * k * tstep, L, CK_FFT_TABLE);
                    w.y = -w.y;
                    v[k] = cmul(v[k], w);
                }
            }
            dft<R>(v, -1);
        } else {
            dft<R>(v, +1);
            if (n1 != 0) {
#pragma unroll
                for (int k = 1; k < R; ++k) v[k] = cmul(v[k], sld(tw, n1 * k * tstep, L, CK_FFT_TABLE));
            }
        }
#pragma unroll
        for (int i = 0; i < R; ++i) sst(buf, ((base + i * S) << WL) + c, L << WL, v[i]);
    }
    __syncthreads();
}

// forward passes of radices R, Rest... starting at sub-block length M
template <typename V, int L, int M, int WL, int R, int... Rest>
__device__ __forceinline__ void forward_from(V* buf, const V* __restrict__ tw)
{
    pass<V, R, L, M, WL, false>(buf, tw);
    if constexpr (sizeof...(Rest) > 0) forward_from<V, L, M / R, WL, Rest...>(buf, tw);
}

// inverse passes of radices R, Rest... (the later passes run first)
template <typename V, int L, int M, int WL, int R, int... Rest>
__device__ __forceinline__ void inverse_from(V* buf, const V* __restrict__ tw)
{
    if constexpr (sizeof...(Rest) > 0) inverse_from<V, L, M / R, WL, Rest...>(buf, tw);
    pass<V, R, L, M, WL, true>(buf, tw);
}

// First forward pass (sub-block length L): inputs t = n1 + i L/R0; those with
// i >= R0/2 are the padding zeros.  load(t, c) gives sample t of pair c.
template <int R0, int L, int WL, typename Load>
__device__ __forceinline__ void first_forward(float2* buf, const float2* __restrict__ tw, Load load)
{
    constexpr int Wc = 1 << WL, S = L / R0, nb = S << WL;
    static_assert(R0 % 2 == 0, "the first radix of an even length is even");
    for (int b = threadIdx.x; b < nb; b += NT) {
        const int c = b & (Wc - 1), n1 = b >> WL;
        float2 v[R0];
#pragma unroll
        for (int i = 0; i < R0; ++i)
            v[i] = (i < R0 / 2 && BTT_IN(n1 + i * S, L / 2, CK_FFT_LOAD)) ? load(n1 + i * S, c) : make_float2(0.f, 0.f);
        dft_half<R0>(v, +1);
        if (n1 != 0) {
#pragma unroll
            for (int k = 1; k < R0; ++k) v[k] = cmul(v[k], sld(tw, n1 * k, L, CK_FFT_TABLE));
        }
#pragma unroll
        for (int i = 0; i < R0; ++i) sst(buf, ((n1 + i * S) << WL) + c, L << WL, v[i]);
    }
    __syncthreads();
}

// Last inverse pass (sub-block length L): outputs t = n1 + i L/R0; only
// i < R0/2 (t < N_t) are emitted, through emit(t, c, value).
template <int R0, int L, int WL, typename Emit>
__device__ __forceinline__ void last_inverse(float2* buf, const float2* __restrict__ tw, Emit emit)
{
    constexpr int Wc = 1 << WL, S = L / R0, nb = S << WL;
    for (int b = threadIdx.x; b < nb; b += NT) {
        const int c = b & (Wc - 1), n1 = b >> WL;
        float2 v[R0];
#pragma unroll
        for (int i = 0; i < R0; ++i) v[i] = sld(buf, ((n1 + i * S) << WL) + c, L << WL);
        if (n1 != 0) {
#pragma unroll
            for (int k = 1; k < R0; ++k) {
                float2 w = sld(tw, n1 * k, L, CK_FFT_TABLE);
                w.y = -w.y;
                v[k] = cmul(v[k], w);
            }
        }
        dft<R0>(v, -1);
#pragma unroll
        for (int i = 0; i < R0 / 2; ++i)
            if (BTT_IN(n1 + i * S, L / 2, CK_FFT_STORE)) emit(n1 + i * S, c, v[i]);
    }
}

// Sample t of real columns ca, ca + 1 (ca even) of a time-outer array: one
// 8-byte load when the pair is whole and the rows are 8-byte aligned (v2).
__device__ __forceinline__ float2 load_pair(const float* __restrict__ xb, int64_t ldx, int t, int ca, int ncols,
                                            bool v2)
{
    const float* p = xb + (int64_t)t * ldx + ca;
    if (v2 && ca + 1 < ncols) return __ldg(reinterpret_cast<const float2*>(p));
    return make_float2(ca < ncols ? __ldg(p) : 0.f, ca + 1 < ncols ? __ldg(p + 1) : 0.f);
}

__device__ __forceinline__ bool aligned8(const void* p, int64_t ld)
{
    return ((reinterpret_cast<uintptr_t>(p) & 7) == 0) && ((ld & 1) == 0);
}

// Calls f(w, p) for every frequency w <= N_t of column pair p, with p fixed
// per thread (NT is a multiple of the pair count): the column, its bounds
// test and its row pointers are set once and stepped by a constant.
template <int WL, typename F> __device__ __forceinline__ void for_pair_rows(int n_rows, F&& f)
{
    constexpr int Wc = 1 << WL, STEP = NT >> WL;
    static_assert(NT % Wc == 0, "pairs per CTA divide the thread count");
    const int p = threadIdx.x & (Wc - 1);
    for (int w = threadIdx.x >> WL; w < n_rows; w += STEP) f(w, p);
}

// Half spectra X[w][col] (w <= N_t) of the tile's column pairs into the
// paired length-L sequence at the digit-reversed positions (the static-plan
// form of load_hermitian_pairs: one 16-byte load per pair when aligned).
// Two neighbouring complex values (columns ca, ca + 1) of a spectrum row,
// as float2 pairs (complex64) or BF16 pairs; one 16- or 8-byte load when
// the pair is whole and aligned (v2).
__device__ __forceinline__ void load_two(const float2* src, int ca, int ncols, bool v2, float2& xa, float2& xb)
{
    if (v2 && ca + 1 < ncols) {
        const float4 q = *reinterpret_cast<const float4*>(src);   // plain load: the middle step rewrites X
        xa = make_float2(q.x, q.y);
        xb = make_float2(q.z, q.w);
    } else {
        if (ca < ncols) xa = src[0];
        if (ca + 1 < ncols) xb = src[1];
    }
}
__device__ __forceinline__ void load_two(const __nv_bfloat162* src, int ca, int ncols, bool v2, float2& xa,
                                         float2& xb)
{
    if (v2 && ca + 1 < ncols) {
        const uint2 q = __ldg(reinterpret_cast<const uint2*>(src));
        xa = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&q.x));
        xb = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&q.y));
    } else {
        if (ca < ncols) xa = __bfloat1622float2(src[0]);
        if (ca + 1 < ncols) xb = __bfloat1622float2(src[1]);
    }
}

// Rows are taken K at a time, their loads issued before the first is used.
template <int L, int WL, typename TX>
__device__ __forceinline__ void load_hermitian_ct(float2* buf, const int* __restrict__ pos,
                                                  const TX* __restrict__ X, int64_t ldx, int col0, int ncols)
{
    constexpr int N_t = L / 2, K = 2, STEP = NT >> WL;
    const bool v2 = ((reinterpret_cast<uintptr_t>(X) & (2 * sizeof(TX) - 1)) == 0) && ((ldx & 1) == 0);
    const int p = threadIdx.x & ((1 << WL) - 1);
    const int ca = col0 + 2 * p;
    for (int w0 = threadIdx.x >> WL; w0 <= N_t; w0 += K * STEP) {
        float2 xa[K], xb[K];
#pragma unroll
        for (int u = 0; u < K; ++u) {
            xa[u] = make_float2(0.f, 0.f);
            xb[u] = xa[u];
            const int w = w0 + u * STEP;
            if (w <= N_t) load_two(X + (int64_t)w * ldx + ca, ca, ncols, v2, xa[u], xb[u]);
        }
#pragma unroll
        for (int u = 0; u < K; ++u) {
            const int w = w0 + u * STEP;
            if (w <= N_t) {
                if (w == 0 || w == N_t) {
                    xa[u].y = 0.f;
                    xb[u].y = 0.f;
                }
                sst(buf, (tld(pos, w, L) << WL) + p, L << WL, make_float2(xa[u].x - xb[u].y, xa[u].y + xb[u].x));
                if (w > 0 && w < N_t)
                    sst(buf, (tld(pos, L - w, L) << WL) + p, L << WL, make_float2(xa[u].x + xb[u].y, xb[u].x - xa[u].y));
            }
        }
    }
}

// Both real spectra (columns 2p and 2p+1) of pair p at frequency w from one
// read of Z[w] and Z[L-w] (see unpack_pair in fft.cuh).
__device__ __forceinline__ void unpack_both(const float2* buf, const int* __restrict__ pos, int L, int w, int p,
                                            int wc_log2, float2& A, float2& B)
{
    const float2 z = sld(buf, (tld(pos, w, L) << wc_log2) + p, L << wc_log2);
    const float2 zc = sld(buf, (tld(pos, w == 0 ? 0 : L - w, L) << wc_log2) + p, L << wc_log2);
    A = make_float2(0.5f * (z.x + zc.x), 0.5f * (z.y - zc.y));
    B = make_float2(0.5f * (z.y + zc.y), 0.5f * (zc.x - z.x));
}

// ------------------------------------------------------------------ kernels
template <int L, int WL, int R0, int... Rs>
__global__ void __launch_bounds__(NT, min_blocks<L, WL>())
k_rfft_ct(const float* __restrict__ x, int64_t ldx, int64_t bsx, int ncols, float2* __restrict__ X, int64_t ldo,
          int64_t bso, const float2* __restrict__ tw, const int* __restrict__ pos,
          const float* const* __restrict__ xptr)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* buf = reinterpret_cast<float2*>(smem_raw);
    constexpr int W = 2 << WL, N_t = L / 2;
    const int col0 = blockIdx.x * W;
    const int64_t b = blockIdx.y;
    const float* xb = xptr ? xptr[b] : x + b * bsx;
    const bool v2 = aligned8(xb, ldx);
    first_forward<R0, L, WL>(buf, tw, [&](int t, int c) { return load_pair(xb, ldx, t, col0 + 2 * c, ncols, v2); });
    if constexpr (sizeof...(Rs) > 0) forward_from<float2, L, L / R0, WL, Rs...>(buf, tw);
    float2* Xb = X + b * bso;
    const bool o2 = ((reinterpret_cast<uintptr_t>(Xb) & 15) == 0) && ((ldo & 1) == 0);
    // one thread per column pair: both spectra from one read of Z[w], Z[L-w]
    for_pair_rows<WL>(N_t + 1, [&](int w, int p) {
        const int col = col0 + 2 * p;
        if (col < ncols) {
            float2 A, B;
            unpack_both(buf, pos, L, w, p, WL, A, B);
            float2* dst = Xb + (int64_t)w * ldo + col;
            if (o2 && col + 1 < ncols) {
                *reinterpret_cast<float4*>(dst) = make_float4(A.x, A.y, B.x, B.y);
            } else {
                dst[0] = A;
                if (col + 1 < ncols) dst[1] = B;
            }
        }
    });
}

template <int L, int WL, int R0, int... Rs>
__global__ void __launch_bounds__(NT, min_blocks<L, WL>())
k_rfft_stack_ct(const float* __restrict__ x, int64_t ldx, int64_t bsx, int ncols, __nv_bfloat162* __restrict__ XA,
                int ldm, int mt_stride, const float2* __restrict__ tw, const int* __restrict__ pos,
                const float* const* __restrict__ xptr, int64_t lo_off)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* buf = reinterpret_cast<float2*>(smem_raw);
    constexpr int W = 2 << WL, N_t = L / 2;
    const int col0 = blockIdx.x * W;
    const int b = blockIdx.y;
    const float* xb = xptr ? xptr[b] : x + (int64_t)b * bsx;
    const bool v2 = aligned8(xb, ldx);
    first_forward<R0, L, WL>(buf, tw, [&](int t, int c) { return load_pair(xb, ldx, t, col0 + 2 * c, ncols, v2); });
    if constexpr (sizeof...(Rs) > 0) forward_from<float2, L, L / R0, WL, Rs...>(buf, tw);
    const int mt = b >> 6, j = b & 63;
    __nv_bfloat162* const XAb = XA + ((int64_t)mt * 64 + j) * ldm;
    const int64_t wstride = (int64_t)mt_stride * 64 * ldm;
    for_pair_rows<WL>(N_t + 1, [&](int w, int p) {
        const int col = col0 + 2 * p;
        if (col < ncols) {
            float2 A, B;
            unpack_both(buf, pos, L, w, p, WL, A, B);
            __nv_bfloat162* dst = XAb + w * wstride + col;
            const __nv_bfloat162 ha = __floats2bfloat162_rn(A.x, -A.y), hb = __floats2bfloat162_rn(B.x, -B.y);
            if (col + 1 < ncols) {
                // two conj BF16 pairs in one 8-byte store (ldm and col are even)
                __nv_bfloat162 two[2] = {ha, hb};
                *reinterpret_cast<uint2*>(dst) = *reinterpret_cast<const uint2*>(two);
            } else {
                dst[0] = ha;
            }
            if (lo_off) {
                // split pairs: the remainders conj(X) - hi, lo_off pairs further
                const float2 fa = __bfloat1622float2(ha), fb = __bfloat1622float2(hb);
                const __nv_bfloat162 la = __floats2bfloat162_rn(A.x - fa.x, -A.y - fa.y);
                const __nv_bfloat162 lb = __floats2bfloat162_rn(B.x - fb.x, -B.y - fb.y);
                if (col + 1 < ncols) {
                    __nv_bfloat162 two[2] = {la, lb};
                    *reinterpret_cast<uint2*>(dst + lo_off) = *reinterpret_cast<const uint2*>(two);
                } else {
                    dst[lo_off] = la;
                }
            }
        }
    });
}

// CG: the output feeds the fused CG step (CgFuse) instead of y.
template <typename TX, bool CG, int L, int WL, int R0, int... Rs>
__global__ void __launch_bounds__(NT, min_blocks<L, WL>())
k_irfft_ct(const TX* __restrict__ X, int64_t ldx, int64_t bsx, int ncols, float* __restrict__ y, int64_t ldy,
           int64_t bsy, const float* __restrict__ g, const float2* __restrict__ tw, const int* __restrict__ pos,
           float* const* __restrict__ yptr, CgFuse cg)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* buf = reinterpret_cast<float2*>(smem_raw);
    constexpr int W = 2 << WL;
    const int col0 = blockIdx.x * W;
    const int64_t b = blockIdx.y;
    load_hermitian_ct<L, WL, TX>(buf, pos, X + b * bsx, ldx, col0, ncols);
    __syncthreads();
    if constexpr (sizeof...(Rs) > 0) inverse_from<float2, L, L / R0, WL, Rs...>(buf, tw);
    constexpr float inv = 1.0f / (float)L;
    if constexpr (CG) {
        // x += a p, r -= a (Hp + shift p) on this tile's columns; r.r partials
        const float aj = cg.cv[b].alpha, sh = cg.shift;
        const int64_t vb = b * cg.n;
        const bool v2 = aligned8(cg.p + vb, ncols) && aligned8(cg.x + vb, ncols) && aligned8(cg.r + vb, ncols);
        float q = 0.f;
        last_inverse<R0, L, WL>(buf, tw, [&](int t, int c, float2 v) {
            const int ca = col0 + 2 * c;
            const int64_t i = vb + (int64_t)t * ncols + ca;
            const float h0 = v.x * inv, h1 = v.y * inv;
            if (v2 && ca + 1 < ncols) {
                const float2 pp = *reinterpret_cast<const float2*>(cg.p + i);
                float2 xx = *reinterpret_cast<const float2*>(cg.x + i);
                float2 rr = *reinterpret_cast<const float2*>(cg.r + i);
                xx.x = fmaf(aj, pp.x, xx.x);
                xx.y = fmaf(aj, pp.y, xx.y);
                rr.x = fmaf(-aj, fmaf(sh, pp.x, h0), rr.x);
                rr.y = fmaf(-aj, fmaf(sh, pp.y, h1), rr.y);
                *reinterpret_cast<float2*>(cg.x + i) = xx;
                *reinterpret_cast<float2*>(cg.r + i) = rr;
                q = fmaf(rr.x, rr.x, fmaf(rr.y, rr.y, q));
                return;
            }
            if (ca < ncols) {
                const float pp = cg.p[i];
                cg.x[i] = fmaf(aj, pp, cg.x[i]);
                const float rv = fmaf(-aj, fmaf(sh, pp, h0), cg.r[i]);
                cg.r[i] = rv;
                q = fmaf(rv, rv, q);
            }
            if (ca + 1 < ncols) {
                const float pp = cg.p[i + 1];
                cg.x[i + 1] = fmaf(aj, pp, cg.x[i + 1]);
                const float rv = fmaf(-aj, fmaf(sh, pp, h1), cg.r[i + 1]);
                cg.r[i + 1] = rv;
                q = fmaf(rv, rv, q);
            }
        });
        block_sum_store<NT>((double)q, cg.part + b * gridDim.x + blockIdx.x);
        return;
    }
    float* yb = yptr ? yptr[b] : y + b * bsy;
    const bool y2 = aligned8(yb, ldy) && (g == nullptr || aligned8(g, ncols));
    last_inverse<R0, L, WL>(buf, tw, [&](int t, int c, float2 v) {
        const int ca = col0 + 2 * c;
        float a = v.x * inv, e = v.y * inv;
        if (y2 && ca + 1 < ncols) {
            if (g) {
                const float2 gg = *reinterpret_cast<const float2*>(g + (int64_t)t * ncols + ca);
                a *= gg.x;
                e *= gg.y;
            }
            *reinterpret_cast<float2*>(yb + (int64_t)t * ldy + ca) = make_float2(a, e);
            return;
        }
        if (ca < ncols) {
            if (g) a *= g[(int64_t)t * ncols + ca];
            yb[(int64_t)t * ldy + ca] = a;
        }
        if (ca + 1 < ncols) {
            if (g) e *= g[(int64_t)t * ncols + ca + 1];
            yb[(int64_t)t * ldy + ca + 1] = e;
        }
    });
}

template <int L, int WL, int R0, int... Rs>
__global__ void __launch_bounds__(NT)
k_hess_mid_ct(float2* X, int64_t ldx, int64_t bsx, int ncols, const float* __restrict__ g,
              const float2* __restrict__ tw, const int* __restrict__ pos, double* __restrict__ part)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* buf = reinterpret_cast<float2*>(smem_raw);
    constexpr int W = 2 << WL, N_t = L / 2;
    const int col0 = blockIdx.x * W;
    const int64_t b = blockIdx.y;
    float2* Xb = X + b * bsx;
    load_hermitian_ct<L, WL, float2>(buf, pos, Xb, ldx, col0, ncols);
    __syncthreads();
    if constexpr (sizeof...(Rs) > 0) inverse_from<float2, L, L / R0, WL, Rs...>(buf, tw);
    // time samples t < N_t, scaled by 1/L and the noise precision of each
    // real column, go back to their natural places; the padding is never read
    constexpr float inv = 1.0f / (float)L;
    float q = 0.f;   // this thread's share of sum g (F m)^2 (part != nullptr)
    last_inverse<R0, L, WL>(buf, tw, [&](int t, int c, float2 v) {
        const int ca = col0 + 2 * c;
        const float a0 = ca < ncols ? v.x * inv : 0.f, e0 = ca + 1 < ncols ? v.y * inv : 0.f;
        float a = a0, e = e0;
        if (g) {
            if (ca < ncols) a *= g[(int64_t)t * ncols + ca];
            if (ca + 1 < ncols) e *= g[(int64_t)t * ncols + ca + 1];
        }
        q = fmaf(a0, a, fmaf(e0, e, q));
        sst(buf, (t << WL) + c, L << WL, make_float2(a, e));
    });
    __syncthreads();
    if (part) block_sum_store<NT>((double)q, part + b * gridDim.x + blockIdx.x);
    first_forward<R0, L, WL>(buf, tw, [&](int t, int c) { return sld(buf, (t << WL) + c, L << WL); });
    if constexpr (sizeof...(Rs) > 0) forward_from<float2, L, L / R0, WL, Rs...>(buf, tw);
    const bool o2 = ((reinterpret_cast<uintptr_t>(Xb) & 15) == 0) && ((ldx & 1) == 0);
    for_pair_rows<WL>(N_t + 1, [&](int w, int p) {
        const int col = col0 + 2 * p;
        if (col < ncols) {
            float2 A, B;
            unpack_both(buf, pos, L, w, p, WL, A, B);
            float2* dst = Xb + (int64_t)w * ldx + col;
            if (o2 && col + 1 < ncols) {
                *reinterpret_cast<float4*>(dst) = make_float4(A.x, A.y, B.x, B.y);
            } else {
                dst[0] = A;
                if (col + 1 < ncols) dst[1] = B;
            }
        }
    });
}

// ------------------------------------------------------------ quad kernels
// The kernels above on quads of four adjacent real columns (fftq.cuh): for
// tiles of at least two column pairs (WL >= 1) every butterfly operation is
// one paired FP32 instruction for two complex sequences, and a quad's
// 16 bytes of a time-outer row load or store as one vector.  Shared layout:
// buf[n * Wq + q] = quad q's two complex values at position n, Wq = Wc / 2.
// Quad q covers columns c = col0 + 4 q .. c + 3; lane 0 is x[c] + i x[c+2],
// lane 1 is x[c+1] + i x[c+3].  The twiddle table holds, after the L
// complex64 entries tw[e], L quad entries (c, c, d, d) of the same values.
// Every plan starts with radix 8 (its first forward and last inverse pass).

// Lane-split layout of a quad element: the two complex values one after the
// other, (Re z0, Im z0, Re z1, Im z1), so that one lane's value is 8
// contiguous bytes (written by the one-lane merged inverse pass below).
__device__ __forceinline__ fq::cq from_split(ulonglong2 u)
{
    const fq::f2 a{u.x}, b{u.y};
    return {fq::pack(fq::lo(a), fq::lo(b)), fq::pack(fq::hi(a), fq::hi(b))};
}

// f(b) for b < NBT over the CTA's NTH threads; in the 256-thread kernels
// (NTH below NT) the iterations are unrolled, so that a thread's
// butterflies overlap.
template <int NBT, int NTH, typename F> __device__ __forceinline__ void for_blocks(F&& f)
{
    if constexpr (NTH != NT && NBT % NTH == 0) {
#pragma unroll
        for (int r = 0; r < NBT / NTH; ++r) f(threadIdx.x + r * NTH);
    } else {
        for (int b = threadIdx.x; b < NBT; b += NTH) f(b);
    }
}

// forward / inverse pass of radix R on sub-blocks of length M (as pass());
// IN_SPLIT: read the lane-split layout
template <int R, int L, int M, int WL, bool INV, bool IN_SPLIT = false, int NTH = NT>
__device__ __forceinline__ void pass_q(ulonglong2* buf, const ulonglong2* __restrict__ twq)
{
    constexpr int QW = WL - 1, Wq = 1 << QW, S = M / R, nb = (L / R) << QW, tstep = L / M;
    for_blocks<nb, NTH>([&](int b) {
        const int q = b & (Wq - 1), j = b >> QW;
        const int blk = j / S, n1 = j - blk * S;
        const int base = blk * M + n1;
        fq::cq v[R];
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const ulonglong2 u = sld(buf, ((base + i * S) << QW) + q, L << QW);
            v[i] = IN_SPLIT ? from_split(u) : fq::from_u2(u);
        }
        if (INV) {
            if (n1 != 0) {
#pragma unroll
                for (int k = 1; k < R; ++k) v[k] = fq::twiddle_conj(v[k], tld(twq, n1 * k * tstep, L));
            }
            fq::dft<R, -1>(v);
        } else {
            fq::dft<R, 1>(v);
            if (n1 != 0) {
#pragma unroll
                for (int k = 1; k < R; ++k) v[k] = fq::twiddle(v[k], tld(twq, n1 * k * tstep, L));
            }
        }
#pragma unroll
        for (int i = 0; i < R; ++i) sst(buf, ((base + i * S) << QW) + q, L << QW, fq::to_u2(v[i]));
    });
    __syncthreads();
}

// First forward pass (radix 8 over the whole length): inputs t = n1 + i L/8,
// i < 4 from load(t, q); i >= 4 are the padding zeros.
template <int L, int WL, int NTH = NT, typename Load>
__device__ __forceinline__ void first_forward_q(ulonglong2* buf, const ulonglong2* __restrict__ twq, Load load)
{
    constexpr int QW = WL - 1, Wq = 1 << QW, S = L / 8, nb = S << QW;
    for_blocks<nb, NTH>([&](int b) {
        const int q = b & (Wq - 1), n1 = b >> QW;
        fq::cq v[8];
#pragma unroll
        for (int i = 0; i < 4; ++i)
            v[i] = BTT_IN(n1 + i * S, L / 2, CK_FFT_LOAD) ? load(n1 + i * S, q) : fq::cq{fq::dup(0.f), fq::dup(0.f)};
        fq::dft8_half_fwd(v);
        if (n1 != 0) {
#pragma unroll
            for (int k = 1; k < 8; ++k) v[k] = fq::twiddle(v[k], tld(twq, n1 * k, L));
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) sst(buf, ((n1 + i * S) << QW) + q, L << QW, fq::to_u2(v[i]));
    });
    __syncthreads();
}

// Last inverse pass (radix 8 over the whole length): outputs t = n1 + i L/8,
// only i < 4 (t < N_t) emitted through emit(t, q, value).
template <int L, int WL, int NTH = NT, typename Emit>
__device__ __forceinline__ void last_inverse_q(ulonglong2* buf, const ulonglong2* __restrict__ twq, Emit emit)
{
    constexpr int QW = WL - 1, Wq = 1 << QW, S = L / 8, nb = S << QW;
    for_blocks<nb, NTH>([&](int b) {
        const int q = b & (Wq - 1), n1 = b >> QW;
        fq::cq v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = fq::from_u2(sld(buf, ((n1 + i * S) << QW) + q, L << QW));
        if (n1 != 0) {
#pragma unroll
            for (int k = 1; k < 8; ++k) v[k] = fq::twiddle_conj(v[k], tld(twq, n1 * k, L));
        }
        fq::dft8<-1>(v);
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (BTT_IN(n1 + i * S, L / 2, CK_FFT_STORE)) emit(n1 + i * S, q, v[i]);
    });
}

__device__ __forceinline__ bool aligned16(const void* p, int64_t ld_elems, int elem_bytes)
{
    return ((reinterpret_cast<uintptr_t>(p) & 15) == 0) && (((ld_elems * elem_bytes) & 15) == 0);
}

// Real columns c .. c+3 of row t as a quad (one 16-byte load when whole and aligned).
__device__ __forceinline__ fq::cq load_quad(const float* __restrict__ xb, int64_t ldx, int t, int c, int ncols,
                                            bool v4)
{
    const float* p = xb + (int64_t)t * ldx + c;
    if (v4 && c + 3 < ncols) return fq::from_u2(__ldg(reinterpret_cast<const ulonglong2*>(p)));
    const float x0 = c < ncols ? __ldg(p) : 0.f, x1 = c + 1 < ncols ? __ldg(p + 1) : 0.f;
    const float x2 = c + 2 < ncols ? __ldg(p + 2) : 0.f, x3 = c + 3 < ncols ? __ldg(p + 3) : 0.f;
    return {fq::pack(x0, x1), fq::pack(x2, x3)};
}

// BF16 pair halves (Re in the low half) as FP32
__device__ __forceinline__ float bf16_lo(uint32_t h) { return __uint_as_float(h << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t h) { return __uint_as_float(h & 0xFFFF0000u); }

// ---------------------------------------------- merged last forward pass
// The quad kernels above pass the data through shared memory once per
// radix-8 pass and once more for the unpack of the real spectra, which
// needs Z[k] and Z[L-k] together: at 2 N_t = 512 three passes and the
// unpack move six tile-sized volumes through shared memory per tile, and
// the shared-memory pipe bounds the kernels.  The last forward pass (radix
// RL over blocks of RL consecutive digit-reversed positions, no twiddles)
// holds the frequencies j + NB i (i < RL, NB = L / RL) of one j per
// butterfly, and the partner L - k of each of them lies in the butterfly of
// NB - j (output RL - 1 - i; for j = 0 and j = NB / 2 in the same
// butterfly).  So a thread that runs the butterflies of j and NB - j can
// unpack every frequency it computes from its registers: the last pass
// and the unpack share one read of shared memory.  The inverse mirrors
// this: the load of the half spectra and the first inverse pass are one
// step.  Two forms: one lane (one complex sequence) of a quad per thread,
// whose value the previous pass leaves in the lane-split layout, the two
// lanes of a quad exchanging a column by warp shuffle (the 512-thread
// kernels, below; the inverse only), and both lanes per thread (the
// 256-thread kernels further below).

// Digit-reversed position of frequency k after the forward passes with
// radices R, Rest... (the digit_reversal table as a function).
template <int L, int PROD> __device__ __forceinline__ int rev_pos(int) { return 0; }
template <int L, int PROD, int R, int... Rest> __device__ __forceinline__ int rev_pos(int k)
{
    return (k % R) * (L / (PROD * R)) + rev_pos<L, PROD * R, Rest...>(k / R);
}

template <int R, int... Rest> constexpr int last_radix()
{
    if constexpr (sizeof...(Rest) == 0) return R;
    else return last_radix<Rest...>();
}

// inverse passes of the radices before the last, later ones first (the
// first to run reads the lane-split layout)
template <int L, int M, int WL, int R, int... Rest>
__device__ __forceinline__ void inverse_mid_q(ulonglong2* buf, const ulonglong2* __restrict__ twq)
{
    if constexpr (sizeof...(Rest) > 0) {
        inverse_mid_q<L, M / R, WL, Rest...>(buf, twq);
        pass_q<R, L, M, WL, true, sizeof...(Rest) == 1>(buf, twq);
    }
}

// Threads of one task: the 2 Wq lanes of a quad row (q fastest, then lane).
template <int WL> struct MergedTask {
    static constexpr int QW = WL - 1, Wq = 1 << QW, G = 2 * Wq, STEP = NT / G;
    static_assert(G <= 32 && NT % G == 0, "a task's threads lie in one warp");
    __device__ __forceinline__ static int q() { return threadIdx.x & (Wq - 1); }
    __device__ __forceinline__ static int lane() { return (threadIdx.x >> QW) & 1; }
    __device__ __forceinline__ static int task() { return threadIdx.x / G; }
    // shuffle mask of the task's threads (all follow the same control flow)
    __device__ __forceinline__ static unsigned mask()
    {
        return (G == 32 ? 0xffffffffu : ((1u << G) - 1u)) << ((threadIdx.x & 31) & ~(G - 1));
    }
};

// Two neighbouring complex values (real columns c, c + 1) of a spectrum row
// as loaded, exchanged between the lanes of a quad, and decoded.
template <typename TX> struct RawTwo;
template <> struct RawTwo<float2> {
    float4 v;   // (Re, Im) of column c, then of column c + 1
    __device__ __forceinline__ static RawTwo load(const float2* src, int c, int ncols, bool v2)
    {
        RawTwo r;
        if (v2 && c + 1 < ncols) {
            r.v = *reinterpret_cast<const float4*>(src);   // plain load: the middle step rewrites X
        } else {
            const float2 z = make_float2(0.f, 0.f), a = c < ncols ? src[0] : z, b = c + 1 < ncols ? src[1] : z;
            r.v = make_float4(a.x, a.y, b.x, b.y);
        }
        return r;
    }
    // the first (second) column's value, and a value received in its place
    __device__ __forceinline__ float2 first() const { return make_float2(v.x, v.y); }
    __device__ __forceinline__ float2 second() const { return make_float2(v.z, v.w); }
    __device__ __forceinline__ static float2 swap(unsigned mk, float2 give, int lanes)
    {
        return make_float2(__shfl_xor_sync(mk, give.x, lanes), __shfl_xor_sync(mk, give.y, lanes));
    }
};
template <> struct RawTwo<__nv_bfloat162> {
    uint2 v;    // BF16 pairs (Re in the low half) of columns c, c + 1
    __device__ __forceinline__ static RawTwo load(const __nv_bfloat162* src, int c, int ncols, bool v2)
    {
        RawTwo r;
        const uint32_t* s = reinterpret_cast<const uint32_t*>(src);
        if (v2 && c + 1 < ncols) r.v = __ldg(reinterpret_cast<const uint2*>(src));
        else r.v = make_uint2(c < ncols ? __ldg(s) : 0u, c + 1 < ncols ? __ldg(s + 1) : 0u);
        return r;
    }
    __device__ __forceinline__ static float2 dec(uint32_t h) { return make_float2(bf16_lo(h), bf16_hi(h)); }
    __device__ __forceinline__ float2 first() const { return dec(v.x); }
    __device__ __forceinline__ float2 second() const { return dec(v.y); }
    // one 32-bit shuffle moves a BF16 pair
    __device__ __forceinline__ uint32_t first_raw() const { return v.x; }
    __device__ __forceinline__ uint32_t second_raw() const { return v.y; }
};

// The load of the half spectra X[w][col] (w <= N_t) fused with the first
// inverse pass (the inverse of the last forward pass); writes the
// lane-split layout.  All of a task's rows are loaded before the first is
// used (several loads in flight per thread).
template <int L, int WL, int R0, int... Rs, typename TX>
__device__ __forceinline__ void load_first_inverse_q(ulonglong2* buf, int col0, const TX* __restrict__ X,
                                                     int64_t ldx, int ncols)
{
    using T = MergedTask<WL>;
    using Raw = RawTwo<TX>;
    constexpr int RL = last_radix<R0, Rs...>(), NB = L / RL, N_t = L / 2, H = RL / 2, NR = 2 * H + 1;
    float2* b2 = reinterpret_cast<float2*>(buf);
    const int q = T::q(), ln = T::lane();
    const int cl = col0 + 4 * q + 2 * ln;   // this thread loads columns cl, cl + 1
    const unsigned mk = T::mask();
    const bool v2 = ((reinterpret_cast<uintptr_t>(X) & (2 * sizeof(TX) - 1)) == 0) && ((ldx & 1) == 0);
    for (int u = T::task(); u < NB / 2; u += T::STEP) {
        const int j0 = u, j1 = u == 0 ? NB / 2 : NB - u;
        // rows j0 + NB i and j1 + NB i (i < H), and N_t for task 0
        Raw raw[NR];
#pragma unroll
        for (int i = 0; i < NR; ++i) {
            const int w = i < H ? j0 + NB * i : (i < 2 * H ? j1 + NB * (i - H) : N_t);
            if ((i < 2 * H || u == 0) && BTT_IN(w, N_t + 1, CK_FFT_LOAD))
                raw[i] = Raw::load(X + (int64_t)w * ldx + cl, cl, ncols, v2);
        }
        // lane 0 keeps column c (its first) and takes c + 2; lane 1 keeps
        // c + 3 (its second) and takes c + 1 (the partner's first / second)
        float2 P[NR], Q[NR];
#pragma unroll
        for (int i = 0; i < NR; ++i) {
            if (i == 2 * H && u != 0) {   // row N_t belongs to task 0 (the same branch for the whole task)
                P[i] = make_float2(0.f, 0.f);
                Q[i] = P[i];
                continue;
            }
            float2 got;
            if constexpr (std::is_same_v<TX, __nv_bfloat162>)
                got = Raw::dec(__shfl_xor_sync(mk, ln ? raw[i].first_raw() : raw[i].second_raw(), T::Wq));
            else
                got = Raw::swap(mk, ln ? raw[i].first() : raw[i].second(), T::Wq);
            P[i] = ln ? got : raw[i].first();
            Q[i] = ln ? raw[i].second() : got;
            const int w = i < H ? j0 + NB * i : (i < 2 * H ? j1 + NB * (i - H) : N_t);
            if (w == 0 || w == N_t) {
                P[i].y = 0.f;
                Q[i].y = 0.f;
            }
        }
        // Z[w] = P + i Q and Z[L - w] = conj P + i conj Q
        auto zf = [&](int i) { return make_float2(P[i].x - Q[i].y, P[i].y + Q[i].x); };
        auto zb = [&](int i) { return make_float2(P[i].x + Q[i].y, Q[i].x - P[i].y); };
        float2 a[RL], e[RL];
#pragma unroll
        for (int i = 0; i < H; ++i) {
            a[i] = zf(i);
            e[i] = zf(H + i);
        }
#pragma unroll
        for (int i = H; i < RL; ++i) {
            // Z[j0 + NB i] and Z[j1 + NB i] for i >= H: from the partner rows
            a[i] = u == 0 ? (i == H ? zf(2 * H) : zb(RL - i)) : zb(H + RL - 1 - i);
            e[i] = u == 0 ? zb(H + RL - 1 - i) : zb(RL - 1 - i);
        }
        dft<RL>(a, -1);
        dft<RL>(e, -1);
        const int p0 = rev_pos<L, 1, R0, Rs...>(j0), p1 = rev_pos<L, 1, R0, Rs...>(j1);
#pragma unroll
        for (int i = 0; i < RL; ++i) {
            sst(b2, (((p0 + i) << T::QW) + q) * 2 + ln, 2 * (L << T::QW), a[i]);
            sst(b2, (((p1 + i) << T::QW) + q) * 2 + ln, 2 * (L << T::QW), e[i]);
        }
    }
    __syncthreads();
}

__device__ __forceinline__ uint32_t bf16_pair(float re, float im)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(re, im);
    return *reinterpret_cast<const uint32_t*>(&h);
}

// ------------------------------------ two-lane merged passes, 256 threads
// The merged passes above give each thread one lane of a quad, so the
// butterflies of the last forward (first inverse) pass run in scalar FP32
// and the lanes swap a column by shuffle.  The forms below give a thread
// both lanes of its quad for one task (j, NB - j): the two butterflies, the
// unpack and the decode are paired FP32 instructions, and a thread loads or
// stores four neighbouring columns (16 bytes of BF16 pairs) with no
// exchange.  A task then needs 2 Wq threads fewer, so these kernels run
// 256-thread CTAs, three per SM (64 KB tiles), and in the other passes a
// thread runs two butterflies.

// Threads per CTA of the two-lane kernels.
constexpr int NTW = 256;

// forward passes of the radices before the last, quad layout throughout
template <int NTH, int L, int M, int WL, int R, int... Rest>
__device__ __forceinline__ void forward_mid_w(ulonglong2* buf, const ulonglong2* __restrict__ twq)
{
    if constexpr (sizeof...(Rest) > 0) {
        pass_q<R, L, M, WL, false, false, NTH>(buf, twq);
        forward_mid_w<NTH, L, M / R, WL, Rest...>(buf, twq);
    }
}

// inverse passes of the radices before the last, later ones first
template <int NTH, int L, int M, int WL, int R, int... Rest>
__device__ __forceinline__ void inverse_mid_w(ulonglong2* buf, const ulonglong2* __restrict__ twq)
{
    if constexpr (sizeof...(Rest) > 0) {
        inverse_mid_w<NTH, L, M / R, WL, Rest...>(buf, twq);
        pass_q<R, L, M, WL, true, false, NTH>(buf, twq);
    }
}

// The last forward pass fused with the unpack, both lanes per thread.
// f(w, A, B) receives, for every frequency w <= N_t of the thread's task,
// the conjugate spectra of real columns c, c + 1 (A, one per lane) and
// c + 2, c + 3 (B), c = col0 + 4 q.
template <bool CONJ, int L, int NTH, int WL, int R0, int... Rs, typename F>
__device__ __forceinline__ void last_forward_unpack_w(const ulonglong2* buf, F&& f)
{
    constexpr int QW = WL - 1, Wq = 1 << QW;
    constexpr int RL = last_radix<R0, Rs...>(), NB = L / RL, N_t = L / 2, H = RL / 2;
    const int q = threadIdx.x & (Wq - 1);
    const fq::f2 half = fq::dup(0.5f);
    for (int u = threadIdx.x >> QW; u < NB / 2; u += NTH >> QW) {
        const int j0 = u, j1 = u == 0 ? NB / 2 : NB - u;
        const int p0 = rev_pos<L, 1, R0, Rs...>(j0), p1 = rev_pos<L, 1, R0, Rs...>(j1);   // RL * block
        fq::cq a[RL], e[RL];
#pragma unroll
        for (int i = 0; i < RL; ++i) {
            a[i] = fq::from_u2(sld(buf, ((p0 + i) << QW) + q, L << QW));
            e[i] = fq::from_u2(sld(buf, ((p1 + i) << QW) + q, L << QW));
        }
        fq::dft<RL, 1>(a);
        fq::dft<RL, 1>(e);
        // X_c = (Z[w] + conj Z[L - w]) / 2, X_{c+2} = (Z[w] - conj Z[L - w]) / 2i, conjugated
        auto emit = [&](int w, const fq::cq& z, const fq::cq& zc) {
            if (BTT_IN(w, N_t + 1, CK_FFT_STORE))
                f(w, fq::cq{fq::mul(half, fq::add(z.re, zc.re)), fq::mul(half, CONJ ? fq::sub(zc.im, z.im) : fq::sub(z.im, zc.im))},
                  fq::cq{fq::mul(half, fq::add(z.im, zc.im)), fq::mul(half, CONJ ? fq::sub(z.re, zc.re) : fq::sub(zc.re, z.re))});
        };
#pragma unroll
        for (int i = 0; i < H; ++i) {
            emit(j0 + NB * i, a[i], u == 0 ? a[(RL - i) % RL] : e[RL - 1 - i]);
            emit(j1 + NB * i, e[i], u == 0 ? e[RL - 1 - i] : a[RL - 1 - i]);
        }
        if (u == 0) emit(N_t, a[H], a[H]);
    }
}

// Four neighbouring complex values (real columns c .. c + 3) of a spectrum
// row, as loaded, and as the two lane pairs P = (c, c + 1), Q = (c + 2, c + 3).
template <typename TX> struct RawFour;
template <> struct RawFour<float2> {
    float4 v0, v1;
    __device__ __forceinline__ static RawFour load(const float2* src, int c, int ncols, bool v4)
    {
        RawFour r;
        if (v4 && c + 3 < ncols) {
            r.v0 = reinterpret_cast<const float4*>(src)[0];   // plain loads: the middle step rewrites X
            r.v1 = reinterpret_cast<const float4*>(src)[1];
        } else {
            const float2 z = make_float2(0.f, 0.f);
            const float2 a = c < ncols ? src[0] : z, b = c + 1 < ncols ? src[1] : z;
            const float2 d = c + 2 < ncols ? src[2] : z, e = c + 3 < ncols ? src[3] : z;
            r.v0 = make_float4(a.x, a.y, b.x, b.y);
            r.v1 = make_float4(d.x, d.y, e.x, e.y);
        }
        return r;
    }
    __device__ __forceinline__ static RawFour zero() { return {make_float4(0.f, 0.f, 0.f, 0.f), make_float4(0.f, 0.f, 0.f, 0.f)}; }
    __device__ __forceinline__ fq::cq P() const { return {fq::pack(v0.x, v0.z), fq::pack(v0.y, v0.w)}; }
    __device__ __forceinline__ fq::cq Q() const { return {fq::pack(v1.x, v1.z), fq::pack(v1.y, v1.w)}; }
};
template <> struct RawFour<__nv_bfloat162> {
    uint4 v;   // BF16 pairs (Re in the low half) of columns c .. c + 3
    __device__ __forceinline__ static RawFour load(const __nv_bfloat162* src, int c, int ncols, bool v4)
    {
        RawFour r;
        const uint32_t* s = reinterpret_cast<const uint32_t*>(src);
        if (v4 && c + 3 < ncols) r.v = __ldg(reinterpret_cast<const uint4*>(src));
        else
            r.v = make_uint4(c < ncols ? __ldg(s) : 0u, c + 1 < ncols ? __ldg(s + 1) : 0u,
                             c + 2 < ncols ? __ldg(s + 2) : 0u, c + 3 < ncols ? __ldg(s + 3) : 0u);
        return r;
    }
    __device__ __forceinline__ static RawFour zero() { return {make_uint4(0u, 0u, 0u, 0u)}; }
    __device__ __forceinline__ fq::cq P() const
    {
        return {fq::pack(bf16_lo(v.x), bf16_lo(v.y)), fq::pack(bf16_hi(v.x), bf16_hi(v.y))};
    }
    __device__ __forceinline__ fq::cq Q() const
    {
        return {fq::pack(bf16_lo(v.z), bf16_lo(v.w)), fq::pack(bf16_hi(v.z), bf16_hi(v.w))};
    }
};

// The load of the half spectra fused with the first inverse pass, both
// lanes per thread; writes the quad layout.
template <int L, int NTH, int WL, int R0, int... Rs, typename TX>
__device__ __forceinline__ void load_first_inverse_w(ulonglong2* buf, int col0, const TX* __restrict__ X,
                                                     int64_t ldx, int ncols)
{
    using Raw = RawFour<TX>;
    constexpr int QW = WL - 1, Wq = 1 << QW;
    constexpr int RL = last_radix<R0, Rs...>(), NB = L / RL, N_t = L / 2, H = RL / 2, NR = 2 * H + 1;
    const int q = threadIdx.x & (Wq - 1), c = col0 + 4 * q;
    const bool v4 = ((reinterpret_cast<uintptr_t>(X) & 15) == 0) && ((ldx * (int64_t)sizeof(TX)) % 16 == 0);
    for (int u = threadIdx.x >> QW; u < NB / 2; u += NTH >> QW) {
        const int j0 = u, j1 = u == 0 ? NB / 2 : NB - u;
        // rows j0 + NB i and j1 + NB i (i < H), and N_t for task 0
        Raw raw[NR];
#pragma unroll
        for (int i = 0; i < NR; ++i) {
            const int w = i < H ? j0 + NB * i : (i < 2 * H ? j1 + NB * (i - H) : N_t);
            raw[i] = (i < 2 * H || u == 0) && BTT_IN(w, N_t + 1, CK_FFT_LOAD)
                         ? Raw::load(X + (int64_t)w * ldx + c, c, ncols, v4)
                         : Raw::zero();
        }
        fq::cq P[NR], Q[NR];
#pragma unroll
        for (int i = 0; i < NR; ++i) {
            P[i] = raw[i].P();
            Q[i] = raw[i].Q();
            const int w = i < H ? j0 + NB * i : (i < 2 * H ? j1 + NB * (i - H) : N_t);
            if (w == 0 || w == N_t) {
                P[i].im = fq::dup(0.f);
                Q[i].im = P[i].im;
            }
        }
        // Z[w] = P + i Q and Z[L - w] = conj P + i conj Q, per lane
        auto zf = [&](int i) { return fq::cq{fq::sub(P[i].re, Q[i].im), fq::add(P[i].im, Q[i].re)}; };
        auto zb = [&](int i) { return fq::cq{fq::add(P[i].re, Q[i].im), fq::sub(Q[i].re, P[i].im)}; };
        fq::cq a[RL], e[RL];
#pragma unroll
        for (int i = 0; i < H; ++i) {
            a[i] = zf(i);
            e[i] = zf(H + i);
        }
#pragma unroll
        for (int i = H; i < RL; ++i) {
            a[i] = u == 0 ? (i == H ? zf(2 * H) : zb(RL - i)) : zb(H + RL - 1 - i);
            e[i] = u == 0 ? zb(H + RL - 1 - i) : zb(RL - 1 - i);
        }
        fq::dft<RL, -1>(a);
        fq::dft<RL, -1>(e);
        const int p0 = rev_pos<L, 1, R0, Rs...>(j0), p1 = rev_pos<L, 1, R0, Rs...>(j1);
#pragma unroll
        for (int i = 0; i < RL; ++i) {
            sst(buf, ((p0 + i) << QW) + q, L << QW, fq::to_u2(a[i]));
            sst(buf, ((p1 + i) << QW) + q, L << QW, fq::to_u2(e[i]));
        }
    }
    __syncthreads();
}

// The operand transform in 256-thread CTAs: first pass, middle passes,
// last pass fused with the unpack; conj spectra as BF16 pairs in
// [w][mt][64][ldm] (and with lo_off the remainder plane).
template <int L, int WL, int R0, int... Rs>
__global__ void __launch_bounds__(NTW, 3)
k_rfft_stack_w(const float* __restrict__ x, int64_t ldx, int64_t bsx, int ncols, __nv_bfloat162* __restrict__ XA,
               int ldm, int mt_stride, const float2* __restrict__ tw, const int* __restrict__ pos,
               const float* const* __restrict__ xptr, int64_t lo_off)
{
    static_assert(WL >= 1, "quads need at least two column pairs per tile");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ulonglong2* buf = reinterpret_cast<ulonglong2*>(smem_raw);
    const ulonglong2* twq = reinterpret_cast<const ulonglong2*>(tw + L);
    constexpr int W = 2 << WL;
    const int col0 = blockIdx.x * W;
    const int b = blockIdx.y;
    const float* xb = xptr ? xptr[b] : x + (int64_t)b * bsx;
    const bool v4 = aligned16(xb, ldx, 4);
    first_forward_q<L, WL, NTW>(buf, twq, [&](int t, int q) { return load_quad(xb, ldx, t, col0 + 4 * q, ncols, v4); });
    forward_mid_w<NTW, L, L / R0, WL, Rs...>(buf, twq);
    const int mt = b >> 6, j = b & 63;
    __nv_bfloat162* const XAb = XA + ((int64_t)mt * 64 + j) * ldm;
    const int64_t wstride = (int64_t)mt_stride * 64 * ldm;
    const bool o4 = ((reinterpret_cast<uintptr_t>(XA) & 15) == 0) && ((ldm & 3) == 0) && ((lo_off & 3) == 0);
    const int c = col0 + 4 * (threadIdx.x & ((1 << (WL - 1)) - 1));
    last_forward_unpack_w<true, L, NTW, WL, R0, Rs...>(buf, [&](int w, const fq::cq& A, const fq::cq& B) {
        const uint32_t h[4] = {bf16_pair(fq::lo(A.re), fq::lo(A.im)), bf16_pair(fq::hi(A.re), fq::hi(A.im)),
                               bf16_pair(fq::lo(B.re), fq::lo(B.im)), bf16_pair(fq::hi(B.re), fq::hi(B.im))};
        __nv_bfloat162* dst = XAb + w * wstride + c;
        if (o4 && c + 3 < ncols) {
            *reinterpret_cast<uint4*>(dst) = make_uint4(h[0], h[1], h[2], h[3]);
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (c + k < ncols) reinterpret_cast<uint32_t*>(dst)[k] = h[k];
        }
        if (lo_off) {
            // split pairs: the remainders conj(X) - hi, lo_off pairs further
            const float v[8] = {fq::lo(A.re), fq::lo(A.im), fq::hi(A.re), fq::hi(A.im),
                                fq::lo(B.re), fq::lo(B.im), fq::hi(B.re), fq::hi(B.im)};
            uint32_t l[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) l[k] = bf16_pair(v[2 * k] - bf16_lo(h[k]), v[2 * k + 1] - bf16_hi(h[k]));
            if (o4 && c + 3 < ncols) {
                *reinterpret_cast<uint4*>(dst + lo_off) = make_uint4(l[0], l[1], l[2], l[3]);
            } else {
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (c + k < ncols) reinterpret_cast<uint32_t*>(dst + lo_off)[k] = l[k];
            }
        }
    });
}

// The FP32 input transform in 256-thread CTAs (spectra as complex64,
// X[b][w][ldo]).
template <int L, int WL, int R0, int... Rs>
__global__ void __launch_bounds__(NTW, 3)
k_rfft_w(const float* __restrict__ x, int64_t ldx, int64_t bsx, int ncols, float2* __restrict__ X, int64_t ldo,
         int64_t bso, const float2* __restrict__ tw, const int* __restrict__ pos,
         const float* const* __restrict__ xptr)
{
    static_assert(WL >= 1, "quads need at least two column pairs per tile");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ulonglong2* buf = reinterpret_cast<ulonglong2*>(smem_raw);
    const ulonglong2* twq = reinterpret_cast<const ulonglong2*>(tw + L);
    constexpr int W = 2 << WL;
    const int col0 = blockIdx.x * W;
    const int64_t b = blockIdx.y;
    const float* xb = xptr ? xptr[b] : x + b * bsx;
    const bool v4 = aligned16(xb, ldx, 4);
    first_forward_q<L, WL, NTW>(buf, twq, [&](int t, int q) { return load_quad(xb, ldx, t, col0 + 4 * q, ncols, v4); });
    forward_mid_w<NTW, L, L / R0, WL, Rs...>(buf, twq);
    float2* Xb = X + b * bso;
    const bool o4 = ((reinterpret_cast<uintptr_t>(Xb) & 15) == 0) && ((ldo & 1) == 0);
    const int c = col0 + 4 * (threadIdx.x & ((1 << (WL - 1)) - 1));
    last_forward_unpack_w<false, L, NTW, WL, R0, Rs...>(buf, [&](int w, const fq::cq& A, const fq::cq& B) {
        float2* dst = Xb + (int64_t)w * ldo + c;
        const float4 u = make_float4(fq::lo(A.re), fq::lo(A.im), fq::hi(A.re), fq::hi(A.im));
        const float4 v = make_float4(fq::lo(B.re), fq::lo(B.im), fq::hi(B.re), fq::hi(B.im));
        if (o4 && c + 3 < ncols) {
            reinterpret_cast<float4*>(dst)[0] = u;
            reinterpret_cast<float4*>(dst)[1] = v;
        } else {
            if (c < ncols) dst[0] = make_float2(u.x, u.y);
            if (c + 1 < ncols) dst[1] = make_float2(u.z, u.w);
            if (c + 2 < ncols) dst[2] = make_float2(v.x, v.y);
            if (c + 3 < ncols) dst[3] = make_float2(v.z, v.w);
        }
    });
}

// CG: the output feeds the fused CG step (CgFuse) instead of y.
// WIDE: 256-thread CTAs with the two-lane first pass (above).
template <typename TX, bool CG, bool WIDE, int L, int WL, int R0, int... Rs>
__global__ void __launch_bounds__(WIDE ? NTW : NT, WIDE ? 3 : 2)
k_irfft_q(const TX* __restrict__ X, int64_t ldx, int64_t bsx, int ncols, float* __restrict__ y, int64_t ldy,
          int64_t bsy, const float* __restrict__ g, const float2* __restrict__ tw, const int* __restrict__ pos,
          float* const* __restrict__ yptr, CgFuse cg)
{
    static_assert(WL >= 1, "quads need at least two column pairs per tile");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ulonglong2* buf = reinterpret_cast<ulonglong2*>(smem_raw);
    const ulonglong2* twq = reinterpret_cast<const ulonglong2*>(tw + L);
    constexpr int W = 2 << WL;
    const int col0 = blockIdx.x * W;
    const int64_t b = blockIdx.y;
    constexpr int NTH = WIDE ? NTW : NT;
    if constexpr (WIDE) {
        load_first_inverse_w<L, NTH, WL, R0, Rs...>(buf, col0, X + b * bsx, ldx, ncols);
        inverse_mid_w<NTH, L, L / R0, WL, Rs...>(buf, twq);
    } else {
        load_first_inverse_q<L, WL, R0, Rs...>(buf, col0, X + b * bsx, ldx, ncols);
        inverse_mid_q<L, L / R0, WL, Rs...>(buf, twq);
    }
    const fq::f2 inv = fq::dup(1.0f / (float)L);
    if constexpr (CG) {
        // x += a p, r -= a (Hp + shift p) on this tile's columns; r.r partials
        const float aj = cg.cv[b].alpha;
        const fq::f2 a2 = fq::dup(aj), na2 = fq::dup(-aj), sh2 = fq::dup(cg.shift);
        const int64_t vb = b * cg.n;
        // x, r and p are distinct arrays
        const float* __restrict__ cp = cg.p + vb;
        float* __restrict__ cx = cg.x + vb;
        float* __restrict__ cr = cg.r + vb;
        const bool v4 = aligned16(cp, ncols, 4) && aligned16(cx, ncols, 4) && aligned16(cr, ncols, 4);
        fq::f2 acc{0ull};
        float qs = 0.f;
        last_inverse_q<L, WL, NTH>(buf, twq, [&](int t, int q, fq::cq v) {
            const int c = col0 + 4 * q;
            const int64_t i = (int64_t)t * ncols + c;
            const fq::f2 h0 = fq::mul(v.re, inv), h1 = fq::mul(v.im, inv);   // Hp at columns c, c+1 | c+2, c+3
            if (v4 && c + 3 < ncols) {
                const fq::cq pp = fq::from_u2(*reinterpret_cast<const ulonglong2*>(cp + i));
                fq::cq xx = fq::from_u2(*reinterpret_cast<const ulonglong2*>(cx + i));
                fq::cq rr = fq::from_u2(*reinterpret_cast<const ulonglong2*>(cr + i));
                xx.re = fq::fma(a2, pp.re, xx.re);
                xx.im = fq::fma(a2, pp.im, xx.im);
                rr.re = fq::fma(na2, fq::fma(sh2, pp.re, h0), rr.re);
                rr.im = fq::fma(na2, fq::fma(sh2, pp.im, h1), rr.im);
                *reinterpret_cast<ulonglong2*>(cx + i) = fq::to_u2(xx);
                *reinterpret_cast<ulonglong2*>(cr + i) = fq::to_u2(rr);
                acc = fq::fma(rr.re, rr.re, fq::fma(rr.im, rr.im, acc));
                return;
            }
            const float hv[4] = {fq::lo(h0), fq::hi(h0), fq::lo(h1), fq::hi(h1)};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (c + k < ncols) {
                    const float pp = cp[i + k];
                    cx[i + k] = fmaf(aj, pp, cx[i + k]);
                    const float rv = fmaf(-aj, fmaf(cg.shift, pp, hv[k]), cr[i + k]);
                    cr[i + k] = rv;
                    qs = fmaf(rv, rv, qs);
                }
            }
        });
        block_sum_store<NTH>((double)(fq::lo(acc) + fq::hi(acc) + qs), cg.part + b * gridDim.x + blockIdx.x);
        return;
    }
    float* yb = yptr ? yptr[b] : y + b * bsy;
    const bool y4 = aligned16(yb, ldy, 4) && (g == nullptr || aligned16(g, ncols, 4));
    last_inverse_q<L, WL, NTH>(buf, twq, [&](int t, int q, fq::cq v) {
        const int c = col0 + 4 * q;
        fq::f2 a = fq::mul(v.re, inv), e = fq::mul(v.im, inv);   // columns c, c+1 | c+2, c+3
        if (y4 && c + 3 < ncols) {
            if (g) {
                const ulonglong2 gg = __ldg(reinterpret_cast<const ulonglong2*>(g + (int64_t)t * ncols + c));
                a = fq::mul(a, fq::f2{gg.x});
                e = fq::mul(e, fq::f2{gg.y});
            }
            *reinterpret_cast<ulonglong2*>(yb + (int64_t)t * ldy + c) = make_ulonglong2(a.u, e.u);
            return;
        }
        const float yv[4] = {fq::lo(a), fq::hi(a), fq::lo(e), fq::hi(e)};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (c + k < ncols) {
                float val = yv[k];
                if (g) val *= g[(int64_t)t * ncols + c + k];
                yb[(int64_t)t * ldy + c + k] = val;
            }
        }
    });
}

// ---------------------------------------------------------- cluster kernels
// For the long fixed plans (2 N_t >= 2000) a CTA holds only a few column
// pairs (the 64 KB tile), so its row segments are 8-32 bytes and the
// transforms are bound by the L2 requests of those narrow rows.  The
// cluster kernels spread one transform over a cluster of four CTAs that
// together hold 4 Wc column pairs -- rows four times as wide -- while each
// CTA still holds 64 KB: after the first forward pass (radix 8 over the
// whole length, decimation in frequency) the eight sub-blocks of length
// L/8 are independent transforms, and CTA r keeps two of them, the pair
// {k0, 8 - k0} mod 8 of first digits (OWN below), so that every frequency
// it holds has its Hermitian partner L - k in the same CTA.  The first
// pass is split over the CTAs by butterfly and writes each output to the
// CTA that owns its sub-block through distributed shared memory; the
// inverse mirrors this (own frequencies in, own sub-blocks, then the last
// radix-8 pass reads the other CTAs' sub-blocks).
//
// Local layout: buf[((slot * S + n) << WLC) + c], slot 0/1 the CTA's two
// sub-blocks, n < S = L/8, c < 2^WLC = 4 Wc column pairs of the cluster tile.
namespace cl {
constexpr int C = 4;   // CTAs per cluster
// 32-bit shared::cluster address of this CTA's shared byte offset `a` in the CTA of rank q
__device__ __forceinline__ uint32_t map(uint32_t a, int q)
{
    uint32_t r;
    asm("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(q));
    return r;
}
__device__ __forceinline__ void st(uint32_t a, float2 v)
{
    asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(a), "f"(v.x), "f"(v.y) : "memory");
}
// Split cluster barrier.  Distributed shared memory of another CTA may be
// touched only after that CTA has started, so every CTA arrives (relaxed:
// it publishes no data yet) on entry and waits before its first remote store.
__device__ __forceinline__ void arrive_relaxed() { asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory"); }
__device__ __forceinline__ void wait() { asm volatile("barrier.cluster.wait.aligned;" ::: "memory"); }
__device__ __forceinline__ float2 ld(uint32_t a)
{
    float2 v;
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a) : "memory");
    return v;
}
// first digits (sub-blocks) owned by rank r: {OWN[r][0], OWN[r][1]}
__device__ __forceinline__ int own(int r, int s) { return s == 0 ? r : (r == 0 ? 4 : 8 - r); }
// owner rank and slot of sub-block i
__device__ __forceinline__ int owner(int i) { return i == 0 || i == 4 ? 0 : (i < 4 ? i : 8 - i); }
__device__ __forceinline__ int slot(int i) { return i >= 4 && i != 0 ? 1 : 0; }
}  // namespace cl

// forward / inverse pass of radix R on the CTA's LB = 2 L/8 local
// elements (sub-blocks of length M), twiddles of the length-L transform
template <int R, int LB, int L, int M, int WLC, bool INV>
__device__ __forceinline__ void pass_cl(float2* buf, const float2* __restrict__ tw)
{
    constexpr int Wc = 1 << WLC, S = M / R, nb = (LB / R) << WLC, tstep = L / M;
    for (int b = threadIdx.x; b < nb; b += NT) {
        const int c = b & (Wc - 1), j = b >> WLC;
        const int blk = j / S, n1 = j - blk * S;
        const int base = blk * M + n1;
        float2 v[R];
#pragma unroll
        for (int i = 0; i < R; ++i) v[i] = sld(buf, ((base + i * S) << WLC) + c, LB << WLC);
        if (INV) {
            if (n1 != 0) {
#pragma unroll
                for (int k = 1; k < R; ++k) {
                    float2 w = sld(tw, n1 * k * tstep, L, CK_FFT_TABLE);
                    w.y = -w.y;
                    v[k] = cmul(v[k], w);
                }
            }
            dft<R>(v, -1);
        } else {
            dft<R>(v, +1);
            if (n1 != 0) {
#pragma unroll
                for (int k = 1; k < R; ++k) v[k] = cmul(v[k], sld(tw, n1 * k * tstep, L, CK_FFT_TABLE));
            }
        }
#pragma unroll
        for (int i = 0; i < R; ++i) sst(buf, ((base + i * S) << WLC) + c, LB << WLC, v[i]);
    }
    __syncthreads();
}

template <int LB, int L, int M, int WLC, int R, int... Rest>
__device__ __forceinline__ void forward_from_cl(float2* buf, const float2* __restrict__ tw)
{
    pass_cl<R, LB, L, M, WLC, false>(buf, tw);
    if constexpr (sizeof...(Rest) > 0) forward_from_cl<LB, L, M / R, WLC, Rest...>(buf, tw);
}

template <int LB, int L, int M, int WLC, int R, int... Rest>
__device__ __forceinline__ void inverse_from_cl(float2* buf, const float2* __restrict__ tw)
{
    if constexpr (sizeof...(Rest) > 0) inverse_from_cl<LB, L, M / R, WLC, Rest...>(buf, tw);
    pass_cl<R, LB, L, M, WLC, true>(buf, tw);
}

// Local index of frequency k (its digit-reversed position pos[k] lies in
// sub-block k mod 8, which this CTA owns).
template <int L> __device__ __forceinline__ int local_pos(const int* __restrict__ pos, int k)
{
    constexpr int S = L / 8;
    const int k0 = k & 7;
    return tld(pos, k, L) + (cl::slot(k0) - k0) * S;
}

// Row j of the CTA's frequencies: w = 8 (j / 2) + (own first digit j % 2).
__device__ __forceinline__ int own_row(int r, int j) { return 8 * (j >> 1) + cl::own(r, j & 1); }

// The input transform of one cluster tile up to the unpack: the first pass
// split over the cluster (outputs to the sub-blocks' owners), a cluster
// barrier, then this CTA's two sub-blocks; returns with them complete.
template <int L, int WL, int... Rs>
__device__ __forceinline__ void forward_cl(float2* buf, const float* __restrict__ xb, int64_t ldx, int ncols, int col0,
                                           const float2* __restrict__ tw, int r)
{
    constexpr int WLC = WL + 2, Wc = 1 << WLC, S = L / 8;
    cl::arrive_relaxed();  // matched by the wait before the first remote store
    uint32_t dst[cl::C];   // the four CTAs' buffers in the cluster's shared window
#pragma unroll
    for (int q = 0; q < cl::C; ++q) dst[q] = cl::map((uint32_t)__cvta_generic_to_shared(buf), q);
    const bool v2 = aligned8(xb, ldx);
    cl::wait();            // every CTA of the cluster has started: its shared memory may be written
    // first pass, butterflies n1 in this CTA's quarter; output i goes to sub-block i
    const int n_lo = r * S / cl::C, n_hi = (r + 1) * S / cl::C;
    for (int bb = threadIdx.x; bb < ((n_hi - n_lo) << WLC); bb += NT) {
        const int c = bb & (Wc - 1), n1 = n_lo + (bb >> WLC);
        float2 v[8];
#pragma unroll
        for (int i = 0; i < 4; ++i)
            v[i] = BTT_IN(n1 + i * S, L / 2, CK_FFT_LOAD) ? load_pair(xb, ldx, n1 + i * S, col0 + 2 * c, ncols, v2)
                                                          : make_float2(0.f, 0.f);
#pragma unroll
        for (int i = 4; i < 8; ++i) v[i] = make_float2(0.f, 0.f);
        dft_half<8>(v, +1);
        if (n1 != 0) {
#pragma unroll
            for (int k = 1; k < 8; ++k) v[k] = cmul(v[k], sld(tw, n1 * k, L, CK_FFT_TABLE));
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int slot_idx = ((cl::slot(i) * S + n1) << WLC) + c;
            if (BTT_IN(slot_idx, (2 * S) << WLC, CK_FFT_REMOTE))
                cl::st(dst[cl::owner(i)] + (uint32_t)slot_idx * 8u, v[i]);
        }
    }
    cooperative_groups::this_cluster().sync();
    if constexpr (sizeof...(Rs) > 0) forward_from_cl<2 * S, L, S, WLC, Rs...>(buf, tw);
}

// Calls f(w, col, A, B) for this CTA's frequencies w <= N_t and column
// pairs col < ncols of the tile: both real spectra of the pair from Z[w]
// and Z[L-w].
template <int L, int WL, typename F>
__device__ __forceinline__ void for_own_spectra(const float2* buf, const int* __restrict__ pos, int r, int col0,
                                                int ncols, F&& f)
{
    constexpr int WLC = WL + 2, Wc = 1 << WLC, N_t = L / 2;
    const int nrows = 2 * (N_t / 8 + 1);
    for (int bb = threadIdx.x; bb < (nrows << WLC); bb += NT) {
        const int c = bb & (Wc - 1), w = own_row(r, bb >> WLC);
        const int col = col0 + 2 * c;
        if (w <= N_t && col < ncols) {
            const float2 z = sld(buf, (local_pos<L>(pos, w) << WLC) + c, (L / 4) << WLC);
            const float2 zc = sld(buf, (local_pos<L>(pos, w == 0 ? 0 : L - w) << WLC) + c, (L / 4) << WLC);
            f(w, col, make_float2(0.5f * (z.x + zc.x), 0.5f * (z.y - zc.y)),
              make_float2(0.5f * (z.y + zc.y), 0.5f * (zc.x - z.x)));
        }
    }
}

template <int L, int WL, int R0, int... Rs>
__global__ void __cluster_dims__(cl::C, 1, 1) __launch_bounds__(NT, min_blocks<L, WL>())
k_rfft_cl(const float* __restrict__ x, int64_t ldx, int64_t bsx, int ncols, float2* __restrict__ X, int64_t ldo,
          int64_t bso, const float2* __restrict__ tw, const int* __restrict__ pos,
          const float* const* __restrict__ xptr)
{
    static_assert(R0 == 8, "the cluster split follows the first radix-8 pass");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* buf = reinterpret_cast<float2*>(smem_raw);
    const int r = (int)cooperative_groups::this_cluster().block_rank();
    const int col0 = (blockIdx.x / cl::C) * (8 << WL);
    const int64_t b = blockIdx.y;
    forward_cl<L, WL, Rs...>(buf, xptr ? xptr[b] : x + b * bsx, ldx, ncols, col0, tw, r);
    float2* Xb = X + b * bso;
    const bool o2 = ((reinterpret_cast<uintptr_t>(Xb) & 15) == 0) && ((ldo & 1) == 0);
    for_own_spectra<L, WL>(buf, pos, r, col0, ncols, [&](int w, int col, float2 A, float2 B) {
        float2* d = Xb + (int64_t)w * ldo + col;
        if (o2 && col + 1 < ncols) {
            *reinterpret_cast<float4*>(d) = make_float4(A.x, A.y, B.x, B.y);
        } else {
            d[0] = A;
            if (col + 1 < ncols) d[1] = B;
        }
    });
}

// The BF16 tensor-core operand form (as k_rfft_stack_ct): conj spectra as
// BF16 pairs in [w][mt][64][ldm], and with lo_off the remainder plane.
template <int L, int WL, int R0, int... Rs>
__global__ void __cluster_dims__(cl::C, 1, 1) __launch_bounds__(NT, min_blocks<L, WL>())
k_rfft_stack_cl(const float* __restrict__ x, int64_t ldx, int64_t bsx, int ncols, __nv_bfloat162* __restrict__ XA,
                int ldm, int mt_stride, const float2* __restrict__ tw, const int* __restrict__ pos,
                const float* const* __restrict__ xptr, int64_t lo_off)
{
    static_assert(R0 == 8, "the cluster split follows the first radix-8 pass");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* buf = reinterpret_cast<float2*>(smem_raw);
    const int r = (int)cooperative_groups::this_cluster().block_rank();
    const int col0 = (blockIdx.x / cl::C) * (8 << WL);
    const int b = blockIdx.y;
    forward_cl<L, WL, Rs...>(buf, xptr ? xptr[b] : x + (int64_t)b * bsx, ldx, ncols, col0, tw, r);
    const int mt = b >> 6, j = b & 63;
    __nv_bfloat162* const XAb = XA + ((int64_t)mt * 64 + j) * ldm;
    const int64_t wstride = (int64_t)mt_stride * 64 * ldm;
    for_own_spectra<L, WL>(buf, pos, r, col0, ncols, [&](int w, int col, float2 A, float2 B) {
        __nv_bfloat162* d = XAb + w * wstride + col;
        const __nv_bfloat162 ha = __floats2bfloat162_rn(A.x, -A.y), hb = __floats2bfloat162_rn(B.x, -B.y);
        if (col + 1 < ncols) {
            __nv_bfloat162 two[2] = {ha, hb};
            *reinterpret_cast<uint2*>(d) = *reinterpret_cast<const uint2*>(two);
        } else {
            d[0] = ha;
        }
        if (lo_off) {
            const float2 fa = __bfloat1622float2(ha), fb = __bfloat1622float2(hb);
            const __nv_bfloat162 la = __floats2bfloat162_rn(A.x - fa.x, -A.y - fa.y);
            const __nv_bfloat162 lb = __floats2bfloat162_rn(B.x - fb.x, -B.y - fb.y);
            if (col + 1 < ncols) {
                __nv_bfloat162 two[2] = {la, lb};
                *reinterpret_cast<uint2*>(d + lo_off) = *reinterpret_cast<const uint2*>(two);
            } else {
                d[lo_off] = la;
            }
        }
    });
}

template <typename TX, int L, int WL, int R0, int... Rs>
__global__ void __cluster_dims__(cl::C, 1, 1) __launch_bounds__(NT, min_blocks<L, WL>())
k_irfft_cl(const TX* __restrict__ X, int64_t ldx, int64_t bsx, int ncols, float* __restrict__ y, int64_t ldy,
           int64_t bsy, const float* __restrict__ g, const float2* __restrict__ tw, const int* __restrict__ pos,
           float* const* __restrict__ yptr)
{
    static_assert(R0 == 8, "the cluster split follows the last radix-8 pass");
    namespace cgr = cooperative_groups;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* buf = reinterpret_cast<float2*>(smem_raw);
    constexpr int WLC = WL + 2, Wc = 1 << WLC, W = 2 << WLC, N_t = L / 2, S = L / 8;
    cgr::cluster_group cluster = cgr::this_cluster();
    const int r = (int)cluster.block_rank();
    const int col0 = (blockIdx.x / cl::C) * W;
    const int64_t b = blockIdx.y;
    // this CTA's frequencies into its sub-blocks (Hermitian pairs stay local)
    const TX* Xb = X + b * bsx;
    const bool v2 = ((reinterpret_cast<uintptr_t>(Xb) & (2 * sizeof(TX) - 1)) == 0) && ((ldx & 1) == 0);
    const int nrows = 2 * (N_t / 8 + 1);
    for (int bb = threadIdx.x; bb < (nrows << WLC); bb += NT) {
        const int c = bb & (Wc - 1), w = own_row(r, bb >> WLC);
        if (w <= N_t) {
            const int ca = col0 + 2 * c;
            float2 xa = make_float2(0.f, 0.f), xb = xa;
            load_two(Xb + (int64_t)w * ldx + ca, ca, ncols, v2, xa, xb);
            if (w == 0 || w == N_t) {
                xa.y = 0.f;
                xb.y = 0.f;
            }
            sst(buf, (local_pos<L>(pos, w) << WLC) + c, (L / 4) << WLC, make_float2(xa.x - xb.y, xa.y + xb.x));
            if (w > 0 && w < N_t)
                sst(buf, (local_pos<L>(pos, L - w) << WLC) + c, (L / 4) << WLC, make_float2(xa.x + xb.y, xb.x - xa.y));
        }
    }
    __syncthreads();
    if constexpr (sizeof...(Rs) > 0) inverse_from_cl<2 * S, L, S, WLC, Rs...>(buf, tw);
    cluster.sync();   // every CTA's sub-blocks are final
    uint32_t src[cl::C];
#pragma unroll
    for (int q = 0; q < cl::C; ++q) src[q] = cl::map((uint32_t)__cvta_generic_to_shared(buf), q);
    float* yb = yptr ? yptr[b] : y + b * bsy;
    const bool y2 = aligned8(yb, ldy) && (g == nullptr || aligned8(g, ncols));
    constexpr float inv = 1.0f / (float)L;
    // last pass, butterflies n1 in this CTA's quarter, inputs from all four
    const int n_lo = r * S / cl::C, n_hi = (r + 1) * S / cl::C;
    for (int bb = threadIdx.x; bb < ((n_hi - n_lo) << WLC); bb += NT) {
        const int c = bb & (Wc - 1), n1 = n_lo + (bb >> WLC);
        float2 v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int slot_idx = ((cl::slot(i) * S + n1) << WLC) + c;
            v[i] = BTT_IN(slot_idx, (2 * S) << WLC, CK_FFT_REMOTE) ? cl::ld(src[cl::owner(i)] + (uint32_t)slot_idx * 8u)
                                                                   : make_float2(0.f, 0.f);
        }
        if (n1 != 0) {
#pragma unroll
            for (int k = 1; k < 8; ++k) {
                float2 w = sld(tw, n1 * k, L, CK_FFT_TABLE);
                w.y = -w.y;
                v[k] = cmul(v[k], w);
            }
        }
        dft<8>(v, -1);
        const int ca = col0 + 2 * c;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int t = n1 + i * S;
            float a = v[i].x * inv, e = v[i].y * inv;
            if (y2 && ca + 1 < ncols) {
                if (g) {
                    const float2 gg = __ldg(reinterpret_cast<const float2*>(g + (int64_t)t * ncols + ca));
                    a *= gg.x;
                    e *= gg.y;
                }
                *reinterpret_cast<float2*>(yb + (int64_t)t * ldy + ca) = make_float2(a, e);
            } else {
                if (ca < ncols) yb[(int64_t)t * ldy + ca] = g ? a * g[(int64_t)t * ncols + ca] : a;
                if (ca + 1 < ncols) yb[(int64_t)t * ldy + ca + 1] = g ? e * g[(int64_t)t * ncols + ca + 1] : e;
            }
        }
    }
    cluster.sync();   // the other CTAs have finished reading this one's shared memory
}

// ------------------------------------------------------------- dispatch
// The fixed plans: the radices make_fft_geom chooses for these lengths.
template <int L, int WL, int... Rs> struct Plan {};

template <typename F> bool for_plan(const FftGeom& g, F&& f)
{
    auto is = [&](int L, int WL, std::initializer_list<int> rs) {
        if (g.L != L || g.wc_log2 != WL || g.plan.nstages != (int)rs.size()) return false;
        int i = 0;
        for (int r : rs)
            if (g.plan.radix[i++] != r) return false;
        return true;
    };
    if (is(128, 4, {8, 8, 2})) { f(Plan<128, 4, 8, 8, 2>{}); return true; }
    if (is(256, 4, {8, 8, 4})) { f(Plan<256, 4, 8, 8, 4>{}); return true; }
    if (is(512, 4, {8, 8, 8})) { f(Plan<512, 4, 8, 8, 8>{}); return true; }
    if (is(1024, 3, {8, 8, 8, 2})) { f(Plan<1024, 3, 8, 8, 8, 2>{}); return true; }
    if (is(2048, 2, {8, 8, 8, 4})) { f(Plan<2048, 2, 8, 8, 8, 4>{}); return true; }
    if (is(4096, 1, {8, 8, 8, 8})) { f(Plan<4096, 1, 8, 8, 8, 8>{}); return true; }
    if (is(2000, 2, {8, 2, 5, 5, 5})) { f(Plan<2000, 2, 8, 2, 5, 5, 5>{}); return true; }
    if (is(4000, 1, {8, 4, 5, 5, 5})) { f(Plan<4000, 1, 8, 4, 5, 5, 5>{}); return true; }
    if (is(8000, 0, {8, 8, 5, 5, 5})) { f(Plan<8000, 0, 8, 8, 5, 5, 5>{}); return true; }
    return false;
}

template <int L, int WL> size_t smem_of() { return (size_t)(L << WL) * sizeof(float2); }
template <int WL> dim3 grid_of(int ncols, int nb) { return dim3((unsigned)((ncols + (2 << WL) - 1) / (2 << WL)), (unsigned)nb, 1); }
// clusters of four CTAs, each cluster 4 x (2 << WL) columns
template <int WL> dim3 grid_cl(int ncols, int nb)
{
    constexpr int W = 8 << WL;
    return dim3((unsigned)((ncols + W - 1) / W * cl::C), (unsigned)nb, 1);
}

// Which fixed plans take the quad kernels: the lengths where they measured
// faster on a GB300 than the pair kernels (stage times over 8- and 64-vector
// batches; tiles of at least 8 quads at L <= 1024).  Elsewhere (short
// transforms with few butterflies per CTA, and the 2- and 4-quad tiles of
// L >= 2000, bound by the L2 requests of narrow rows, where the pair
// kernels' third CTA per SM keeps more loads in flight) the pair kernels run.
// Among the quad kernels, the two-lane 256-thread forms (three CTAs per SM)
// against the one-lane 512-thread forms (two per SM) and, at L = 256, the
// pair stack kernel, 64-vector BF16 batches: BF16 operand transform -24% at
// L = 256, -2 to -10% at 512 (by the number of columns), -5% at 1024; BF16
// inverse -26%, -11 to -20%, -19%; FP32 inverse (8-vector batches) -23% at
// 256, -18% at 1024, but +2% at 512, where its two-lane first pass spills.
// The CG forms (whose epilogue streams p, x and r: 20 iterations of btt_cg)
// follow, except the BF16 one at 512 (+2%).  At L = 2048 (2-quad tiles)
// the BF16 inverse -2%, the operand transform +10% against the cluster
// kernel.  The FP32 input transform with complex64 spectra (8-vector
// batches, against the pair kernel): -7% at 256, -15% at 1024, +1% at 512.
template <int L> constexpr bool wide_stack() { return L == 256 || L == 512 || L == 1024; }
template <int L> constexpr bool wide_fwd() { return L == 256 || L == 1024; }
template <int L, typename TX, bool CG> constexpr bool wide_inverse()
{
    return L == 256 || L == 1024 || ((L == 512 || L == 2048) && std::is_same_v<TX, __nv_bfloat162> && !CG);
}
// Fixed plans whose complex64 transforms run on clusters of four CTAs
// (measured against the pair kernels on a GB300, 8-vector FP32 batches:
// input transform -12% at 2 N_t = 2000, -17% at 2048, -41 to -54% at
// 4000-8000; inverse -8% at 2048, -29 to -52% at 4000-8000, but +3% at
// 2000, where its last pass's remote reads cost more than the wider rows
// save).
template <int L> constexpr bool cluster_fwd() { return L == 2000 || L == 2048 || L == 4000 || L == 4096 || L == 8000; }
template <int L> constexpr bool cluster_inv() { return L == 2048 || L == 4000 || L == 4096 || L == 8000; }
// The BF16 tensor-core forms (64-vector batches): stack input -8% at 2000,
// -24% at 2048, -41 to -56% at 4000-8000; BF16 inverse -27 to -51% at
// 4000-8000 (+11% at 2000 against pairs, +8% at 2048 against quads).
template <int L> constexpr bool cluster_stack() { return L == 2000 || L == 2048 || L == 4000 || L == 4096 || L == 8000; }
template <int L> constexpr bool cluster_inv_bf16() { return L == 4000 || L == 4096 || L == 8000; }
// one-lane quad inverse where the two-lane form is not taken
template <int L, typename TX> constexpr bool quad_inverse()
{
    return L == 512 || (L == 2048 && std::is_same_v<TX, __nv_bfloat162>);
}

}  // namespace

cudaError_t prepare_static_fft()
{
    cudaError_t e = cudaSuccess;
    const int mx = kFftCap * (int)sizeof(float2);
    auto set = [&](auto kern) {
        if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    };
    FftGeom g{};
    for (int N_t : {64, 128, 256, 512, 1024, 2048, 1000, 2000, 4000}) {
        if (!make_fft_geom(N_t, &g)) continue;
        for_plan(g, [&](auto p) {
            [&]<int L, int WL, int... Rs>(Plan<L, WL, Rs...>) {
                if constexpr (cluster_fwd<L>()) set(k_rfft_cl<L, WL, Rs...>);
                else if constexpr (wide_fwd<L>()) set(k_rfft_w<L, WL, Rs...>);
                else set(k_rfft_ct<L, WL, Rs...>);
                if constexpr (cluster_inv<L>()) set(k_irfft_cl<float2, L, WL, Rs...>);
                if constexpr (cluster_inv_bf16<L>()) set(k_irfft_cl<__nv_bfloat162, L, WL, Rs...>);
                if constexpr (cluster_stack<L>()) set(k_rfft_stack_cl<L, WL, Rs...>);
                set(k_hess_mid_ct<L, WL, Rs...>);
                if constexpr (wide_stack<L>()) set(k_rfft_stack_w<L, WL, Rs...>);
                else set(k_rfft_stack_ct<L, WL, Rs...>);
                auto set_inverse = [&]<typename TX, bool CG>(TX*, std::bool_constant<CG>) {
                    if constexpr (wide_inverse<L, TX, CG>()) set(k_irfft_q<TX, CG, true, L, WL, Rs...>);
                    else if constexpr (quad_inverse<L, TX>()) set(k_irfft_q<TX, CG, false, L, WL, Rs...>);
                    else set(k_irfft_ct<TX, CG, L, WL, Rs...>);
                };
                set_inverse((float2*)nullptr, std::false_type{});
                set_inverse((float2*)nullptr, std::true_type{});
                set_inverse((__nv_bfloat162*)nullptr, std::false_type{});
                set_inverse((__nv_bfloat162*)nullptr, std::true_type{});
            }(p);
        });
    }
    return e;
}

bool static_rfft(const float* x, int64_t ldx, int64_t bsx, int ncols, float2* X, int64_t ldo, int64_t bso, int nb,
                 const FftGeom& g, const float2* tw, cudaStream_t st, const float* const* xptr, cudaError_t* err)
{
    return for_plan(g, [&]<int L, int WL, int... Rs>(Plan<L, WL, Rs...>) {
        if constexpr (cluster_fwd<L>())
            k_rfft_cl<L, WL, Rs...><<<grid_cl<WL>(ncols, nb), NT, smem_of<L, WL>(), st>>>(x, ldx, bsx, ncols, X, ldo,
                                                                                        bso, tw, g.pos, xptr);
        else if constexpr (wide_fwd<L>())
            k_rfft_w<L, WL, Rs...><<<grid_of<WL>(ncols, nb), NTW, smem_of<L, WL>(), st>>>(x, ldx, bsx, ncols, X, ldo,
                                                                                        bso, tw, g.pos, xptr);
        else
            k_rfft_ct<L, WL, Rs...><<<grid_of<WL>(ncols, nb), NT, smem_of<L, WL>(), st>>>(x, ldx, bsx, ncols, X, ldo,
                                                                                        bso, tw, g.pos, xptr);
        count_launch();
        *err = cudaGetLastError();
    });
}

bool static_rfft_stack(const float* x, int64_t ldx, int64_t bsx, int ncols, void* xstack, int ldm, int mt_stride,
                       int nb, const FftGeom& g, const float2* tw, cudaStream_t st, int64_t lo_off,
                       const float* const* xptr, cudaError_t* err)
{
    return for_plan(g, [&]<int L, int WL, int... Rs>(Plan<L, WL, Rs...>) {
        auto* xs = static_cast<__nv_bfloat162*>(xstack);
        if constexpr (cluster_stack<L>())
            k_rfft_stack_cl<L, WL, Rs...><<<grid_cl<WL>(ncols, nb), NT, smem_of<L, WL>(), st>>>(
                x, ldx, bsx, ncols, xs, ldm, mt_stride, tw, g.pos, xptr, lo_off);
        else if constexpr (wide_stack<L>())
            k_rfft_stack_w<L, WL, Rs...><<<grid_of<WL>(ncols, nb), NTW, smem_of<L, WL>(), st>>>(
                x, ldx, bsx, ncols, xs, ldm, mt_stride, tw, g.pos, xptr, lo_off);
        else
            k_rfft_stack_ct<L, WL, Rs...><<<grid_of<WL>(ncols, nb), NT, smem_of<L, WL>(), st>>>(
                x, ldx, bsx, ncols, xs, ldm, mt_stride, tw, g.pos, xptr, lo_off);
        count_launch();
        *err = cudaGetLastError();
    });
}

namespace {

// the inverse transform of one plan: two-lane quad, one-lane quad or pair kernel
template <typename TX, bool CG, int L, int WL, int... Rs>
void launch_inverse(const TX* X, int64_t ldx, int64_t bsx, int ncols, float* y, int64_t ldy, int64_t bsy,
                    const float* gam, const float2* tw, const int* pos, float* const* yptr, const CgFuse& cg, int nb,
                    cudaStream_t st)
{
    if constexpr (wide_inverse<L, TX, CG>())
        k_irfft_q<TX, CG, true, L, WL, Rs...><<<grid_of<WL>(ncols, nb), NTW, smem_of<L, WL>(), st>>>(
            X, ldx, bsx, ncols, y, ldy, bsy, gam, tw, pos, yptr, cg);
    else if constexpr (quad_inverse<L, TX>())
        k_irfft_q<TX, CG, false, L, WL, Rs...><<<grid_of<WL>(ncols, nb), NT, smem_of<L, WL>(), st>>>(
            X, ldx, bsx, ncols, y, ldy, bsy, gam, tw, pos, yptr, cg);
    else
        k_irfft_ct<TX, CG, L, WL, Rs...><<<grid_of<WL>(ncols, nb), NT, smem_of<L, WL>(), st>>>(
            X, ldx, bsx, ncols, y, ldy, bsy, gam, tw, pos, yptr, cg);
    count_launch();
}

}  // namespace

bool static_irfft(const float2* X, int64_t ldx, int64_t bsx, int ncols, float* y, int64_t ldy, int64_t bsy,
                  const float* gam, int nb, const FftGeom& g, const float2* tw, cudaStream_t st, float* const* yptr,
                  cudaError_t* err)
{
    return for_plan(g, [&]<int L, int WL, int... Rs>(Plan<L, WL, Rs...>) {
        if constexpr (cluster_inv<L>()) {
            k_irfft_cl<float2, L, WL, Rs...><<<grid_cl<WL>(ncols, nb), NT, smem_of<L, WL>(), st>>>(
                X, ldx, bsx, ncols, y, ldy, bsy, gam, tw, g.pos, yptr);
            count_launch();
        } else {
            launch_inverse<float2, false, L, WL, Rs...>(X, ldx, bsx, ncols, y, ldy, bsy, gam, tw, g.pos, yptr,
                                                        CgFuse{}, nb, st);
        }
        *err = cudaGetLastError();
    });
}

bool static_irfft_bf16(const __nv_bfloat162* X, int64_t ldx, int64_t bsx, int ncols, float* y, int64_t ldy,
                       int64_t bsy, int nb, const FftGeom& g, const float2* tw, cudaStream_t st, float* const* yptr,
                       cudaError_t* err)
{
    return for_plan(g, [&]<int L, int WL, int... Rs>(Plan<L, WL, Rs...>) {
        if constexpr (cluster_inv_bf16<L>()) {
            k_irfft_cl<__nv_bfloat162, L, WL, Rs...><<<grid_cl<WL>(ncols, nb), NT, smem_of<L, WL>(), st>>>(
                X, ldx, bsx, ncols, y, ldy, bsy, nullptr, tw, g.pos, yptr);
            count_launch();
        } else {
            launch_inverse<__nv_bfloat162, false, L, WL, Rs...>(X, ldx, bsx, ncols, y, ldy, bsy, nullptr, tw, g.pos,
                                                                yptr, CgFuse{}, nb, st);
        }
        *err = cudaGetLastError();
    });
}

bool static_irfft_cg(const void* X, bool bf16, int64_t ldx, int64_t bsx, int ncols, int nb, const FftGeom& g,
                     const float2* tw, cudaStream_t st, const CgFuse& cg, cudaError_t* err)
{
    return for_plan(g, [&]<int L, int WL, int... Rs>(Plan<L, WL, Rs...>) {
        if (bf16)
            launch_inverse<__nv_bfloat162, true, L, WL, Rs...>(static_cast<const __nv_bfloat162*>(X), ldx, bsx, ncols,
                                                               nullptr, 0, 0, nullptr, tw, g.pos, nullptr, cg, nb, st);
        else
            launch_inverse<float2, true, L, WL, Rs...>(static_cast<const float2*>(X), ldx, bsx, ncols, nullptr, 0, 0,
                                                       nullptr, tw, g.pos, nullptr, cg, nb, st);
        *err = cudaGetLastError();
    });
}

bool static_plan(const FftGeom& g)
{
    return for_plan(g, [](auto) {});
}

bool static_hess_mid(float2* X, int64_t ldx, int64_t bsx, int ncols, const float* gam, int nb, const FftGeom& g,
                     const float2* tw, cudaStream_t st, double* part, cudaError_t* err)
{
    return for_plan(g, [&]<int L, int WL, int... Rs>(Plan<L, WL, Rs...>) {
        k_hess_mid_ct<L, WL, Rs...><<<grid_of<WL>(ncols, nb), NT, smem_of<L, WL>(), st>>>(X, ldx, bsx, ncols, gam, tw,
                                                                                        g.pos, part);
        count_launch();
        *err = cudaGetLastError();
    });
}

}  // namespace btt

#ifdef BTT_CHECK
namespace btt {
BTT_CHECK_TU(check_record_fft_static)
}  // namespace btt
#endif
