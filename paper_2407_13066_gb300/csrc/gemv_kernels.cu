// Per-frequency complex products with the stored Fhat (the apply_matrix step
// of Alg. 2 and Alg. 3).  After the time transform the operator is block
// diagonal over frequency (Sec. 3.2), so for every w
//     F :  dhat[w][s] = sum_l Fhat[w][s][l] xhat[w][l]
//     F*:  mhat[w][l] = sum_s conj(Fhat[w][s][l]) dhat[w][s]
// Both stream all of Fhat once per pass and are bound by HBM bandwidth
// (about 1 flop per byte at complex64).  Fhat is laid out [w][s][ldm] with
// l fastest, so both products read it in coalesced 16-byte row segments:
// F reduces along a row (threads stride l, then warp shuffles and a
// shared-memory combine), F* combines rows (each thread owns a few l and
// loops over s, with dhat[w][:] staged in shared memory).
#include "kernels.h"

namespace btt {

// ------------------------------------------------------ storage decoding
template <int PREC> struct Store;

template <> struct Store<P_F32> {
    using elem = float2;
    using acc = float;
    static constexpr int VPL = 2;  // complex values per 16-byte load
    static __device__ __forceinline__ void load(const elem* p, float2 (&f)[VPL], int64_t)
    {
        const float4 q = __ldcs(reinterpret_cast<const float4*>(p));
        f[0] = make_float2(q.x, q.y);
        f[1] = make_float2(q.z, q.w);
    }
};

template <> struct Store<P_F64> {
    using elem = double2;
    using acc = double;
    static constexpr int VPL = 1;
    static __device__ __forceinline__ void load(const elem* p, double2 (&f)[VPL], int64_t)
    {
        f[0] = __ldcs(p);
    }
};

template <> struct Store<P_F16S> {
    using elem = __half2;
    using acc = float;
    static constexpr int VPL = 4;
    static __device__ __forceinline__ void load(const elem* p, float2 (&f)[VPL], int64_t)
    {
        const uint4 q = __ldcs(reinterpret_cast<const uint4*>(p));
        const unsigned w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            __half2 h = *reinterpret_cast<const __half2*>(&w[i]);
            f[i] = __half22float2(h);
        }
    }
};

template <> struct Store<P_BF16> {
    using elem = __nv_bfloat162;
    using acc = float;
    static constexpr int VPL = 4;
    static __device__ __forceinline__ void load(const elem* p, float2 (&f)[VPL], int64_t)
    {
        const uint4 q = __ldcs(reinterpret_cast<const uint4*>(p));
        const unsigned w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162*>(&w[i]);
            f[i] = __bfloat1622float2(h);
        }
    }
};

// BF16 hi+lo split pair, stored as two planes of BF16 Fhat: hi at p, lo at
// p + lo (the same [w][s][ldm] layout each, so either plane is also a BF16
// operand of the tensor-core products).
template <> struct Store<P_BF16X2> {
    using elem = __nv_bfloat162;
    using acc = float;
    static constexpr int VPL = 4;
    static __device__ __forceinline__ void load(const elem* p, float2 (&f)[VPL], int64_t lo)
    {
        const uint4 qh = __ldcs(reinterpret_cast<const uint4*>(p));
        const uint4 ql = __ldcs(reinterpret_cast<const uint4*>(p + lo));
        const unsigned h[4] = {qh.x, qh.y, qh.z, qh.w};
        const unsigned l[4] = {ql.x, ql.y, ql.z, ql.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&h[i]));
            const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&l[i]));
            f[i] = make_float2(a.x + b.x, a.y + b.y);
        }
    }
};

template <> struct Store<P_FP8S> {
    using elem = __nv_fp8x2_storage_t;   // (Re, Im) E4M3 codes of Fhat / s_w
    using acc = float;
    static constexpr int VPL = 8;
    static __device__ __forceinline__ void load(const elem* p, float2 (&f)[VPL], int64_t)
    {
        const uint4 q = __ldcs(reinterpret_cast<const uint4*>(p));
        const unsigned w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const __half2 lo = __half2(__nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w[i] & 0xFFFFu), __NV_E4M3));
            const __half2 hi = __half2(__nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w[i] >> 16), __NV_E4M3));
            f[2 * i] = __half22float2(lo);
            f[2 * i + 1] = __half22float2(hi);
        }
    }
};

template <typename V> __device__ __forceinline__ void load_vec(const V* p, V (&x)[1]) { x[0] = __ldg(p); }
__device__ __forceinline__ void load_vec(const float2* p, float2 (&x)[2])
{
    const float4 q = __ldg(reinterpret_cast<const float4*>(p));
    x[0] = make_float2(q.x, q.y);
    x[1] = make_float2(q.z, q.w);
}
__device__ __forceinline__ void load_vec(const float2* p, float2 (&x)[8])
{
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float4 q = __ldg(reinterpret_cast<const float4*>(p) + i);
        x[2 * i] = make_float2(q.x, q.y);
        x[2 * i + 1] = make_float2(q.z, q.w);
    }
}
__device__ __forceinline__ void load_vec(const float2* p, float2 (&x)[4])
{
    const float4 q0 = __ldg(reinterpret_cast<const float4*>(p));
    const float4 q1 = __ldg(reinterpret_cast<const float4*>(p) + 1);
    x[0] = make_float2(q0.x, q0.y);
    x[1] = make_float2(q0.z, q0.w);
    x[2] = make_float2(q1.x, q1.y);
    x[3] = make_float2(q1.z, q1.w);
}

template <typename V> __device__ __forceinline__ void cfma(V& acc, V a, V b)
{
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}
// acc += conj(a) * b
template <typename V> __device__ __forceinline__ void cfma_conj(V& acc, V a, V b)
{
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(-a.y, b.x, acc.y);
}

// ------------------------------------------------------------ F (Alg. 2)
// CTA = (right-hand-side group of NB, row tile of R, frequency w).  The
// group index is the fastest grid dimension so that the CTAs sharing one
// Fhat tile run back to back and the repeats hit L2.
template <int PREC, int R, int NB, int NT>
__global__ void __launch_bounds__(NT)
k_gemv_fwd(const typename Store<PREC>::elem* __restrict__ fhat, const float* __restrict__ scales,
           int N_d, int ldm, const cplx_t<typename Store<PREC>::acc>* __restrict__ xh, int64_t xbs,
           cplx_t<typename Store<PREC>::acc>* __restrict__ dh, int64_t dbs, int nrhs, int64_t lo_off)
{
    using S = Store<PREC>;
    using A = typename S::acc;
    using V = cplx_t<A>;
    constexpr int VPL = S::VPL;
    const int b0 = blockIdx.x * NB;
    const int r0 = blockIdx.y * R;
    const int w = blockIdx.z;
    const typename S::elem* F0 = fhat + ((int64_t)w * N_d + r0) * ldm;
    const V* x0 = xh + (int64_t)b0 * xbs + (int64_t)w * ldm;

    V acc[R][NB];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int n = 0; n < NB; ++n) acc[r][n] = cmake<V>(0, 0);

    for (int k = threadIdx.x * VPL; k < ldm; k += NT * VPL) {
        V xv[NB][VPL];
#pragma unroll
        for (int n = 0; n < NB; ++n) {
            if (b0 + n < nrhs) load_vec(x0 + (int64_t)n * xbs + k, xv[n]);
            else
#pragma unroll
                for (int v = 0; v < VPL; ++v) xv[n][v] = cmake<V>(0, 0);
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (r0 + r < N_d) {
                V f[VPL];
                S::load(F0 + (int64_t)r * ldm + k, f, lo_off);
#pragma unroll
                for (int n = 0; n < NB; ++n)
#pragma unroll
                    for (int v = 0; v < VPL; ++v) cfma(acc[r][n], f[v], xv[n][v]);
            }
        }
    }

    // reduce over the CTA: warp shuffles, then one partial per warp in smem
    __shared__ V red[NT / 32][R * NB];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int n = 0; n < NB; ++n) {
            V a = acc[r][n];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                a.x += __shfl_xor_sync(0xffffffffu, a.x, o);
                a.y += __shfl_xor_sync(0xffffffffu, a.y, o);
            }
            if (lane == 0) red[wid][r * NB + n] = a;
        }
    __syncthreads();
    if (threadIdx.x < R * NB) {
        const int r = threadIdx.x / NB, n = threadIdx.x % NB;
        V a = red[0][threadIdx.x];
#pragma unroll
        for (int i = 1; i < NT / 32; ++i) a = cadd(a, red[i][threadIdx.x]);
        if (PREC == P_F16S || PREC == P_FP8S) a = cscale(a, (A)scales[w]);
        if (r0 + r < N_d && b0 + n < nrhs) dh[(int64_t)(b0 + n) * dbs + (int64_t)w * N_d + r0 + r] = a;
    }
}

// Single-vector F with mhat staged in shared memory: CTA = RW rows of one
// frequency, one warp per row streaming 16-byte loads of Fhat (UNR in
// flight per lane), mhat(w) copied into shared memory in chunks of CH
// values (cp.async, double buffered) and read there by all RW rows.  Every
// CTA of the 4-row kernel above re-reads mhat(w) through L2; here it is
// read once per RW rows, which takes a sixth of the L2 requests off the
// stream (measured at the bandwidth shape: 7.30 against 6.28-6.32 TB/s).
// (launch bounds ask for two 20-warp or four 8-warp CTAs per SM)
template <int PREC, int RW, int UNR, int CH>
__global__ void __launch_bounds__(RW * 32, RW >= 16 ? 2 : 4)
k_gemv_fwd_rows(const typename Store<PREC>::elem* __restrict__ fhat, const float* __restrict__ scales, int N_d,
                int ldm, const float2* __restrict__ xh, float2* __restrict__ dh, int64_t lo_off)
{
    using S = Store<PREC>;
    constexpr int VPL = S::VPL;
    static_assert(CH % (2 * VPL) == 0, "chunks hold whole 16-byte units");
    __shared__ __align__(16) float2 sx[2][CH];
    const int r0 = blockIdx.x * RW, w = blockIdx.y;
    const float2* xg = xh + (int64_t)w * ldm;
    const int nch = (ldm + CH - 1) / CH;
    const int lane = threadIdx.x & 31, row = r0 + (threadIdx.x >> 5);
    const bool live = row < N_d;
    const typename S::elem* Fr = fhat + ((int64_t)w * N_d + (live ? row : 0)) * ldm;
    // 16-byte copies of mhat[c*CH, min(ldm, (c+1)*CH)) into buffer `buf`
    auto stage = [&](int c, int buf) {
        const int base = c * CH, n = min(CH, ldm - base) / 2;
        for (int i = threadIdx.x; i < n; i += RW * 32) {
            const unsigned sa = (unsigned)__cvta_generic_to_shared(&sx[buf][2 * i]);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(xg + base + 2 * i) : "memory");
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    float2 acc0 = make_float2(0.f, 0.f), acc1 = make_float2(0.f, 0.f);
    stage(0, 0);
    for (int c = 0; c < nch; ++c) {
        if (c + 1 < nch) {
            stage(c + 1, (c + 1) & 1);
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        __syncthreads();
        const float2* sb = sx[c & 1];
        const int base = c * CH, end = min(CH, ldm - base);
        if (live) {
            int k = lane * VPL;
            for (; k + 32 * VPL * (UNR - 1) < end; k += 32 * VPL * UNR) {
                float2 f[UNR][VPL];
#pragma unroll
                for (int u = 0; u < UNR; ++u) S::load(Fr + base + k + 32 * VPL * u, f[u], lo_off);
#pragma unroll
                for (int u = 0; u < UNR; ++u)
#pragma unroll
                    for (int v = 0; v < VPL; ++v) {
                        if (v & 1) cfma(acc1, f[u][v], sb[k + 32 * VPL * u + v]);
                        else cfma(acc0, f[u][v], sb[k + 32 * VPL * u + v]);
                    }
            }
            for (; k < end; k += 32 * VPL) {
                float2 f[VPL];
                S::load(Fr + base + k, f, lo_off);
#pragma unroll
                for (int v = 0; v < VPL; ++v) {
                    if (v & 1) cfma(acc1, f[v], sb[k + v]);
                    else cfma(acc0, f[v], sb[k + v]);
                }
            }
        }
        __syncthreads();   // buffer c & 1 is staged again two chunks later
    }
    if (!live) return;
    float2 a = make_float2(acc0.x + acc1.x, acc0.y + acc1.y);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a.x += __shfl_xor_sync(0xffffffffu, a.x, o);
        a.y += __shfl_xor_sync(0xffffffffu, a.y, o);
    }
    if (PREC == P_F16S || PREC == P_FP8S) a = cscale(a, scales[w]);
    if (lane == 0) dh[(int64_t)w * N_d + row] = a;
}

// ----------------------------------------------------------- F* (Alg. 3)
// CTA = (right-hand-side group, column tile of NT*VPL, frequency w).
template <int PREC, int NB, int NT, int UNR>
__global__ void __launch_bounds__(NT)
k_gemv_adj(const typename Store<PREC>::elem* __restrict__ fhat, const float* __restrict__ scales,
           int N_d, int N_m, int ldm, const cplx_t<typename Store<PREC>::acc>* __restrict__ dh,
           int64_t dbs, cplx_t<typename Store<PREC>::acc>* __restrict__ mh, int64_t mbs, int nrhs, int64_t lo_off)
{
    using S = Store<PREC>;
    using A = typename S::acc;
    using V = cplx_t<A>;
    constexpr int VPL = S::VPL;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* sd = reinterpret_cast<V*>(smem_raw);  // [NB][N_d]
    const int b0 = blockIdx.x * NB;
    const int w = blockIdx.z;
    const int k = (blockIdx.y * NT + threadIdx.x) * VPL;
    const A sc = (PREC == P_F16S || PREC == P_FP8S) ? (A)scales[w] : (A)1;
    for (int i = threadIdx.x; i < NB * N_d; i += NT) {
        const int n = i / N_d, s = i - n * N_d;
        V v = cmake<V>(0, 0);
        if (b0 + n < nrhs) v = dh[(int64_t)(b0 + n) * dbs + (int64_t)w * N_d + s];
        sd[i] = cscale(v, sc);
    }
    __syncthreads();
    if (k >= ldm) return;

    V acc[VPL][NB];
#pragma unroll
    for (int v = 0; v < VPL; ++v)
#pragma unroll
        for (int n = 0; n < NB; ++n) acc[v][n] = cmake<V>(0, 0);

    const typename S::elem* p = fhat + (int64_t)w * N_d * ldm + k;
    int s = 0;
    for (; s + UNR <= N_d; s += UNR) {
        V f[UNR][VPL];
#pragma unroll
        for (int u = 0; u < UNR; ++u) S::load(p + (int64_t)(s + u) * ldm, f[u], lo_off);
#pragma unroll
        for (int u = 0; u < UNR; ++u)
#pragma unroll
            for (int n = 0; n < NB; ++n) {
                const V y = sd[n * N_d + s + u];
#pragma unroll
                for (int v = 0; v < VPL; ++v) cfma_conj(acc[v][n], f[u][v], y);
            }
    }
    for (; s < N_d; ++s) {
        V f[VPL];
        S::load(p + (int64_t)s * ldm, f, lo_off);
#pragma unroll
        for (int n = 0; n < NB; ++n) {
            const V y = sd[n * N_d + s];
#pragma unroll
            for (int v = 0; v < VPL; ++v) cfma_conj(acc[v][n], f[v], y);
        }
    }
#pragma unroll
    for (int n = 0; n < NB; ++n) {
        if (b0 + n >= nrhs) break;
        V* out = mh + (int64_t)(b0 + n) * mbs + (int64_t)w * ldm + k;
#pragma unroll
        for (int v = 0; v < VPL; ++v)
            if (k + v < N_m) out[v] = acc[v][n];
    }
}

// ---------------------------------------------------------------- launchers
constexpr int kGemvThreads = 256;

// element offset of the lo plane of a split-pair Fhat (0 for other formats)
static int64_t lo_plane(int prec, int n_freq, int N_d, int ldm)
{
    return prec == P_BF16X2 ? (int64_t)n_freq * N_d * ldm : 0;
}
constexpr int kAdjUnroll = 8;

template <int PREC, int R, int NB>
static cudaError_t fwd_launch(const void* fhat, const float* scales, int n_freq, int N_d, int ldm,
                              const void* xh, int64_t xbs, void* dh, int64_t dbs, int nrhs,
                              cudaStream_t st)
{
    using S = Store<PREC>;
    using V = cplx_t<typename S::acc>;
    dim3 grid((nrhs + NB - 1) / NB, (N_d + R - 1) / R, n_freq);
    k_gemv_fwd<PREC, R, NB, kGemvThreads><<<grid, kGemvThreads, 0, st>>>(
        static_cast<const typename S::elem*>(fhat), scales, N_d, ldm, static_cast<const V*>(xh), xbs,
        static_cast<V*>(dh), dbs, nrhs, lo_plane(PREC, n_freq, N_d, ldm));
    count_launch();
    return cudaGetLastError();
}

template <int PREC, int RW>
static cudaError_t rows_launch(const void* fhat, const float* scales, int n_freq, int N_d, int ldm, const void* xh,
                               void* dh, cudaStream_t st)
{
    using S = Store<PREC>;
    dim3 grid((N_d + RW - 1) / RW, n_freq);
    // 16-byte loads in flight per lane: as many as fit the register budget
    // of two CTAs per SM after the decode (FP32 8, the other formats 4)
    constexpr int UNR = PREC == P_F32 ? 8 : 4;
    k_gemv_fwd_rows<PREC, RW, UNR, 2048><<<grid, RW * 32, 0, st>>>(
        static_cast<const typename S::elem*>(fhat), scales, N_d, ldm, static_cast<const float2*>(xh),
        static_cast<float2*>(dh), lo_plane(PREC, n_freq, N_d, ldm));
    count_launch();
    return cudaGetLastError();
}

template <int PREC>
static cudaError_t fwd_dispatch(const void* fhat, const float* scales, int n_freq, int N_d, int ldm,
                                const void* xh, int64_t xbs, void* dh, int64_t dbs, int nrhs,
                                cudaStream_t st)
{
    if (nrhs == 1) {
        // one warp per row: 20 rows per CTA, or 8 when that idles fewer warps
        const int w20 = (N_d + 19) / 20 * 20 - N_d, w8 = (N_d + 7) / 8 * 8 - N_d;
        if (w20 * 10 <= N_d || w20 <= w8) return rows_launch<PREC, 20>(fhat, scales, n_freq, N_d, ldm, xh, dh, st);
        return rows_launch<PREC, 8>(fhat, scales, n_freq, N_d, ldm, xh, dh, st);
    }
    // 4 rows per CTA: measured faster than 8 (fewer concurrent row streams
    // per CTA, more CTAs resident) even though mhat is re-read twice as often
    if (nrhs == 1) return fwd_launch<PREC, 4, 1>(fhat, scales, n_freq, N_d, ldm, xh, xbs, dh, dbs, nrhs, st);
    if (nrhs == 2) return fwd_launch<PREC, 4, 2>(fhat, scales, n_freq, N_d, ldm, xh, xbs, dh, dbs, nrhs, st);
    return fwd_launch<PREC, 4, 4>(fhat, scales, n_freq, N_d, ldm, xh, xbs, dh, dbs, nrhs, st);
}

cudaError_t launch_gemv_fwd(int prec, const void* fhat, const float* scales, int n_freq, int N_d,
                            int ldm, const void* xh, int64_t xbs, void* dh, int64_t dbs, int nrhs,
                            cudaStream_t st)
{
    if (nrhs <= 0) return cudaSuccess;
    switch (prec) {
        case P_F32: return fwd_dispatch<P_F32>(fhat, scales, n_freq, N_d, ldm, xh, xbs, dh, dbs, nrhs, st);
        case P_F64: return fwd_launch<P_F64, 4, 1>(fhat, scales, n_freq, N_d, ldm, xh, xbs, dh, dbs, nrhs, st);
        case P_F16S: return fwd_dispatch<P_F16S>(fhat, scales, n_freq, N_d, ldm, xh, xbs, dh, dbs, nrhs, st);
        case P_BF16: return fwd_dispatch<P_BF16>(fhat, scales, n_freq, N_d, ldm, xh, xbs, dh, dbs, nrhs, st);
        case P_BF16X2: return fwd_dispatch<P_BF16X2>(fhat, scales, n_freq, N_d, ldm, xh, xbs, dh, dbs, nrhs, st);
        case P_FP8S: return fwd_dispatch<P_FP8S>(fhat, scales, n_freq, N_d, ldm, xh, xbs, dh, dbs, nrhs, st);
        default: return cudaErrorInvalidValue;
    }
}

template <int PREC, int NB>
static cudaError_t adj_launch(const void* fhat, const float* scales, int n_freq, int N_d, int N_m,
                              int ldm, const void* dh, int64_t dbs, void* mh, int64_t mbs, int nrhs,
                              cudaStream_t st)
{
    using S = Store<PREC>;
    using V = cplx_t<typename S::acc>;
    const int cols = kGemvThreads * S::VPL;
    dim3 grid((nrhs + NB - 1) / NB, (ldm + cols - 1) / cols, n_freq);
    const size_t sm = (size_t)NB * N_d * sizeof(V);
    auto kern = k_gemv_adj<PREC, NB, kGemvThreads, kAdjUnroll>;
    if (sm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    kern<<<grid, kGemvThreads, sm, st>>>(static_cast<const typename S::elem*>(fhat), scales, N_d, N_m,
                                         ldm, static_cast<const V*>(dh), dbs, static_cast<V*>(mh), mbs,
                                         nrhs, lo_plane(PREC, n_freq, N_d, ldm));
    count_launch();
    return cudaGetLastError();
}

template <int PREC>
static cudaError_t adj_dispatch(const void* fhat, const float* scales, int n_freq, int N_d, int N_m,
                                int ldm, const void* dh, int64_t dbs, void* mh, int64_t mbs, int nrhs,
                                cudaStream_t st)
{
    if (nrhs == 1) return adj_launch<PREC, 1>(fhat, scales, n_freq, N_d, N_m, ldm, dh, dbs, mh, mbs, nrhs, st);
    if (nrhs == 2) return adj_launch<PREC, 2>(fhat, scales, n_freq, N_d, N_m, ldm, dh, dbs, mh, mbs, nrhs, st);
    if (nrhs <= 4) return adj_launch<PREC, 4>(fhat, scales, n_freq, N_d, N_m, ldm, dh, dbs, mh, mbs, nrhs, st);
    return adj_launch<PREC, 8>(fhat, scales, n_freq, N_d, N_m, ldm, dh, dbs, mh, mbs, nrhs, st);
}

cudaError_t launch_gemv_adj(int prec, const void* fhat, const float* scales, int n_freq, int N_d,
                            int N_m, int ldm, const void* dh, int64_t dbs, void* mh, int64_t mbs,
                            int nrhs, cudaStream_t st)
{
    if (nrhs <= 0) return cudaSuccess;
    switch (prec) {
        case P_F32: return adj_dispatch<P_F32>(fhat, scales, n_freq, N_d, N_m, ldm, dh, dbs, mh, mbs, nrhs, st);
        case P_F64: return adj_launch<P_F64, 1>(fhat, scales, n_freq, N_d, N_m, ldm, dh, dbs, mh, mbs, nrhs, st);
        case P_F16S: return adj_dispatch<P_F16S>(fhat, scales, n_freq, N_d, N_m, ldm, dh, dbs, mh, mbs, nrhs, st);
        case P_BF16: return adj_dispatch<P_BF16>(fhat, scales, n_freq, N_d, N_m, ldm, dh, dbs, mh, mbs, nrhs, st);
        case P_BF16X2: return adj_dispatch<P_BF16X2>(fhat, scales, n_freq, N_d, N_m, ldm, dh, dbs, mh, mbs, nrhs, st);
        case P_FP8S: return adj_dispatch<P_FP8S>(fhat, scales, n_freq, N_d, N_m, ldm, dh, dbs, mh, mbs, nrhs, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace btt
