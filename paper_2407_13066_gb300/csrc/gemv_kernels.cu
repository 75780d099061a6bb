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
#include "fftq.cuh"
#include "kernels.h"

namespace btt {

// ------------------------------------------------------ storage decoding
// Store<PREC>: one 16-byte unit of a Fhat row (VPL complex values).
// load_raw fetches the unit (evict-first; the split pair also its lo-plane
// twin at p + lo), decode turns it into FP32 complex values, and load does
// both.  Kernels that keep many units in flight hold raw units and decode
// late.
template <int PREC> struct Store;

template <> struct Store<P_F32> {
    using elem = float2;
    using acc = float;
    using raw = float4;
    static constexpr int VPL = 2;  // complex values per 16-byte load
    static __device__ __forceinline__ raw load_raw(const elem* p, int64_t)
    {
        return __ldcs(reinterpret_cast<const float4*>(p));
    }
    static __device__ __forceinline__ void decode(const raw& q, float2 (&f)[VPL])
    {
        f[0] = make_float2(q.x, q.y);
        f[1] = make_float2(q.z, q.w);
    }
    static __device__ __forceinline__ void load(const elem* p, float2 (&f)[VPL], int64_t lo) { decode(load_raw(p, lo), f); }
};

template <> struct Store<P_F64> {
    using elem = double2;
    using acc = double;
    using raw = double2;
    static constexpr int VPL = 1;
    static __device__ __forceinline__ raw load_raw(const elem* p, int64_t) { return __ldcs(p); }
    static __device__ __forceinline__ void decode(const raw& q, double2 (&f)[VPL]) { f[0] = q; }
    static __device__ __forceinline__ void load(const elem* p, double2 (&f)[VPL], int64_t lo) { decode(load_raw(p, lo), f); }
};

template <> struct Store<P_F16S> {
    using elem = __half2;
    using acc = float;
    using raw = uint4;
    static constexpr int VPL = 4;
    static __device__ __forceinline__ raw load_raw(const elem* p, int64_t)
    {
        return __ldcs(reinterpret_cast<const uint4*>(p));
    }
    static __device__ __forceinline__ void decode(const raw& q, float2 (&f)[VPL])
    {
        const unsigned w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) f[i] = __half22float2(*reinterpret_cast<const __half2*>(&w[i]));
    }
    static __device__ __forceinline__ void load(const elem* p, float2 (&f)[VPL], int64_t lo) { decode(load_raw(p, lo), f); }
};

template <> struct Store<P_BF16> {
    using elem = __nv_bfloat162;
    using acc = float;
    using raw = uint4;
    static constexpr int VPL = 4;
    static __device__ __forceinline__ raw load_raw(const elem* p, int64_t)
    {
        return __ldcs(reinterpret_cast<const uint4*>(p));
    }
    static __device__ __forceinline__ void decode(const raw& q, float2 (&f)[VPL])
    {
        const unsigned w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) f[i] = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w[i]));
    }
    static __device__ __forceinline__ void load(const elem* p, float2 (&f)[VPL], int64_t lo) { decode(load_raw(p, lo), f); }
};

// BF16 hi+lo split pair, stored as two planes of BF16 Fhat: hi at p, lo at
// p + lo (the same [w][s][ldm] layout each, so either plane is also a BF16
// operand of the tensor-core products).
struct SplitRaw {
    uint4 h, l;
};
template <> struct Store<P_BF16X2> {
    using elem = __nv_bfloat162;
    using acc = float;
    using raw = SplitRaw;
    static constexpr int VPL = 4;
    static __device__ __forceinline__ raw load_raw(const elem* p, int64_t lo)
    {
        return SplitRaw{__ldcs(reinterpret_cast<const uint4*>(p)), __ldcs(reinterpret_cast<const uint4*>(p + lo))};
    }
    static __device__ __forceinline__ void decode(const raw& q, float2 (&f)[VPL])
    {
        const unsigned h[4] = {q.h.x, q.h.y, q.h.z, q.h.w};
        const unsigned l[4] = {q.l.x, q.l.y, q.l.z, q.l.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&h[i]));
            const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&l[i]));
            f[i] = make_float2(a.x + b.x, a.y + b.y);
        }
    }
    static __device__ __forceinline__ void load(const elem* p, float2 (&f)[VPL], int64_t lo) { decode(load_raw(p, lo), f); }
};

template <> struct Store<P_FP8S> {
    using elem = __nv_fp8x2_storage_t;   // (Re, Im) E4M3 codes of Fhat / s_w
    using acc = float;
    using raw = uint4;
    static constexpr int VPL = 8;
    static __device__ __forceinline__ raw load_raw(const elem* p, int64_t)
    {
        return __ldcs(reinterpret_cast<const uint4*>(p));
    }
    static __device__ __forceinline__ void decode(const raw& q, float2 (&f)[VPL])
    {
        const unsigned w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const __half2 lo = __half2(__nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w[i] & 0xFFFFu), __NV_E4M3));
            const __half2 hi = __half2(__nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w[i] >> 16), __NV_E4M3));
            f[2 * i] = __half22float2(lo);
            f[2 * i + 1] = __half22float2(hi);
        }
    }
    static __device__ __forceinline__ void load(const elem* p, float2 (&f)[VPL], int64_t lo) { decode(load_raw(p, lo), f); }
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

// F with the vectors staged in shared memory: CTA = RW warps x RPW rows of
// one frequency for NB right-hand sides.  Each warp streams its RPW rows
// with 16-byte loads (UNR units per row in flight per lane, held raw and
// decoded late); the NB vectors' mhat(w) are copied into shared memory in
// chunks of CH values (cp.async, double buffered) and each value read
// there serves RPW rows.  Every CTA of the 4-row kernel below re-reads
// mhat through L2 (a quarter more L2 requests than Fhat alone, NB times
// that for NB vectors); here mhat crosses L2 once per RW * RPW rows.
// Single vector, FP32, 20 rows: 7.30-7.42 TB/s in isolation against
// 6.28-6.39 TB/s for the 4-row kernel.
template <int PREC, int RW, int RPW, int NB, int UNR, int CH, int MINB>
__global__ void __launch_bounds__(RW * 32, MINB)
k_gemv_fwd_rows(const typename Store<PREC>::elem* __restrict__ fhat, const float* __restrict__ scales, int N_d,
                int ldm, const float2* __restrict__ xh, int64_t xbs, float2* __restrict__ dh, int64_t dbs, int nrhs,
                int64_t lo_off)
{
    using S = Store<PREC>;
    constexpr int VPL = S::VPL;
    static_assert(CH % (2 * VPL) == 0, "chunks hold whole 16-byte units");
    __shared__ __align__(16) float2 sx[2][NB][CH];
    const int r0 = blockIdx.x * RW * RPW, w = blockIdx.y, b0 = blockIdx.z * NB;
    const int nch = (ldm + CH - 1) / CH;
    const int lane = threadIdx.x & 31, wr = r0 + (threadIdx.x >> 5) * RPW;
    const typename S::elem* Fw = fhat + (int64_t)w * N_d * ldm;
    // 16-byte copies of mhat_b[c*CH, min(ldm, (c+1)*CH)) into buffer `buf`
    auto stage = [&](int c, int buf) {
        const int base = c * CH, n2 = min(CH, ldm - base) / 2;
#pragma unroll
        for (int n = 0; n < NB; ++n) {
            if (b0 + n >= nrhs) break;
            const float2* xg = xh + (int64_t)(b0 + n) * xbs + (int64_t)w * ldm + base;
            for (int i = threadIdx.x; i < n2; i += RW * 32) {
                if (!BTT_IN(2 * i + 1, CH, CK_GEMV_SMEM) || !BTT_IN(base + 2 * i + 1, ldm, CK_GEMV_VEC)) continue;
                const unsigned sa = (unsigned)__cvta_generic_to_shared(&sx[buf][n][2 * i]);
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(xg + 2 * i) : "memory");
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    float2 acc[RPW][NB];
#pragma unroll
    for (int r = 0; r < RPW; ++r)
#pragma unroll
        for (int n = 0; n < NB; ++n) acc[r][n] = make_float2(0.f, 0.f);
    stage(0, 0);
    for (int c = 0; c < nch; ++c) {
        if (c + 1 < nch) {
            stage(c + 1, (c + 1) & 1);
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        __syncthreads();
        const int base = c * CH, end = min(CH, ldm - base);
        if (wr < N_d) {
            int k = lane * VPL;
            for (; k + 32 * VPL * (UNR - 1) < end; k += 32 * VPL * UNR) {
                typename S::raw q[UNR][RPW];
#pragma unroll
                for (int u = 0; u < UNR; ++u)
#pragma unroll
                    for (int r = 0; r < RPW; ++r)
                        if (wr + r < N_d && BTT_IN(base + k + 32 * VPL * u + VPL - 1, ldm, CK_GEMV_FHAT))
                            q[u][r] = S::load_raw(Fw + (int64_t)(wr + r) * ldm + base + k + 32 * VPL * u, lo_off);
#pragma unroll
                for (int u = 0; u < UNR; ++u) {
                    const int kk = k + 32 * VPL * u;
#pragma unroll
                    for (int r = 0; r < RPW; ++r) {
                        if (wr + r >= N_d) continue;
                        float2 f[VPL];
                        S::decode(q[u][r], f);
#pragma unroll
                        for (int n = 0; n < NB; ++n)
#pragma unroll
                            for (int v = 0; v < VPL; ++v)
                                if (BTT_IN(kk + v, CH, CK_GEMV_SMEM)) cfma(acc[r][n], f[v], sx[c & 1][n][kk + v]);
                    }
                }
            }
            for (; k < end; k += 32 * VPL) {
#pragma unroll
                for (int r = 0; r < RPW; ++r) {
                    if (wr + r >= N_d) continue;
                    float2 f[VPL];
                    if (!BTT_IN(base + k + VPL - 1, ldm, CK_GEMV_FHAT)) continue;
                    S::load(Fw + (int64_t)(wr + r) * ldm + base + k, f, lo_off);
#pragma unroll
                    for (int n = 0; n < NB; ++n)
#pragma unroll
                        for (int v = 0; v < VPL; ++v)
                            if (BTT_IN(k + v, CH, CK_GEMV_SMEM)) cfma(acc[r][n], f[v], sx[c & 1][n][k + v]);
                }
            }
        }
        __syncthreads();   // buffer c & 1 is staged again two chunks later
    }
    if (wr >= N_d) return;
    const float sc = (PREC == P_F16S || PREC == P_FP8S) ? scales[w] : 1.f;
#pragma unroll
    for (int r = 0; r < RPW; ++r)
#pragma unroll
        for (int n = 0; n < NB; ++n) {
            float2 a = acc[r][n];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                a.x += __shfl_xor_sync(0xffffffffu, a.x, o);
                a.y += __shfl_xor_sync(0xffffffffu, a.y, o);
            }
            if (lane == 0 && wr + r < N_d && b0 + n < nrhs && BTT_IN((int64_t)w * N_d + wr + r, dbs, CK_GEMV_VEC))
                dh[(int64_t)(b0 + n) * dbs + (int64_t)w * N_d + wr + r] = cscale(a, sc);
        }
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

    if constexpr (std::is_same<A, float>::value && VPL >= 4) {
        // The formats that decode (4-8 values per 16-byte unit): FP32
        // accumulation on column pairs (v, v + 1) as paired f32x2
        // instructions -- the same fused multiply-adds, in the same order, as
        // cfma_conj per column (conj(f) y = (fr yr + fi yi, fr yi - fi yr)),
        // so results are bit-identical, with half the FMA instructions
        // (FP8 F* at the bandwidth shape 0.379 -> 0.315 ms per launch)
        const typename S::elem* p = fhat + (int64_t)w * N_d * ldm + k;
        const bool k_ok = BTT_IN(k + VPL - 1, ldm, CK_GEMV_FHAT);
        constexpr int VP = VPL / 2;
        fq::f2 are[VP][NB], aim[VP][NB];
#pragma unroll
        for (int v = 0; v < VP; ++v)
#pragma unroll
            for (int n = 0; n < NB; ++n) are[v][n] = aim[v][n] = fq::dup(0.f);
        auto step = [&](const V (&f)[VPL], int srow) {
#pragma unroll
            for (int n = 0; n < NB; ++n) {
                const V y = BTT_IN(n * N_d + srow, NB * N_d, CK_GEMV_SMEM) ? sd[n * N_d + srow] : cmake<V>(0, 0);
                const fq::f2 yr = fq::dup(y.x), yi = fq::dup(y.y), nyr = fq::dup(-y.x);
#pragma unroll
                for (int v = 0; v < VP; ++v) {
                    const fq::f2 fr = fq::pack(f[2 * v].x, f[2 * v + 1].x), fi = fq::pack(f[2 * v].y, f[2 * v + 1].y);
                    are[v][n] = fq::fma(fr, yr, are[v][n]);
                    are[v][n] = fq::fma(fi, yi, are[v][n]);
                    aim[v][n] = fq::fma(fr, yi, aim[v][n]);
                    aim[v][n] = fq::fma(fi, nyr, aim[v][n]);
                }
            }
        };
        int s = 0;
        for (; s + UNR <= N_d; s += UNR) {
            V f[UNR][VPL];
#pragma unroll
            for (int u = 0; u < UNR; ++u)
                if (k_ok && BTT_IN(s + u, N_d, CK_GEMV_FHAT)) S::load(p + (int64_t)(s + u) * ldm, f[u], lo_off);
#pragma unroll
            for (int u = 0; u < UNR; ++u) step(f[u], s + u);
        }
        for (; s < N_d; ++s) {
            V f[VPL];
            if (!k_ok) break;
            S::load(p + (int64_t)s * ldm, f, lo_off);
            step(f, s);
        }
#pragma unroll
        for (int n = 0; n < NB; ++n) {
            if (b0 + n >= nrhs) break;
            V* out = mh + (int64_t)(b0 + n) * mbs + (int64_t)w * ldm + k;
#pragma unroll
            for (int v = 0; v < VPL; ++v) {
                const fq::f2 r = are[v / 2][n], m = aim[v / 2][n];
                const V o = (v & 1) ? cmake<V>(fq::hi(r), fq::hi(m)) : cmake<V>(fq::lo(r), fq::lo(m));
                if (k + v < N_m && BTT_IN(k + v, ldm, CK_GEMV_VEC)) out[v] = o;
            }
        }
        return;
    } else {
    V acc[VPL][NB];
#pragma unroll
    for (int v = 0; v < VPL; ++v)
#pragma unroll
        for (int n = 0; n < NB; ++n) acc[v][n] = cmake<V>(0, 0);

    const typename S::elem* p = fhat + (int64_t)w * N_d * ldm + k;
    int s = 0;
    const bool k_ok = BTT_IN(k + VPL - 1, ldm, CK_GEMV_FHAT);
    for (; s + UNR <= N_d; s += UNR) {
        V f[UNR][VPL];
#pragma unroll
        for (int u = 0; u < UNR; ++u)
            if (k_ok && BTT_IN(s + u, N_d, CK_GEMV_FHAT)) S::load(p + (int64_t)(s + u) * ldm, f[u], lo_off);
#pragma unroll
        for (int u = 0; u < UNR; ++u)
#pragma unroll
            for (int n = 0; n < NB; ++n) {
                const V y = BTT_IN(n * N_d + s + u, NB * N_d, CK_GEMV_SMEM) ? sd[n * N_d + s + u] : cmake<V>(0, 0);
#pragma unroll
                for (int v = 0; v < VPL; ++v) cfma_conj(acc[v][n], f[u][v], y);
            }
    }
    for (; s < N_d; ++s) {
        V f[VPL];
        if (!k_ok) break;
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
            if (k + v < N_m && BTT_IN(k + v, ldm, CK_GEMV_VEC)) out[v] = acc[v][n];
    }
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

// Resident CTAs per SM the launch bounds ask for, from a register budget
// per thread: 48 for the 20-warp FP32 kernel (two CTAs per SM), 64 for the
// 8-warp one, 72 for the formats that decode (raw units of RPW rows in
// flight plus decoded values), 96 with four vectors.
template <int PREC, int RW, int NB> constexpr int rows_min_blocks()
{
    constexpr int regs = PREC == P_F32 ? (RW >= 16 ? 48 : 64) : (NB >= 4 ? 96 : 72);
    constexpr int b = 65536 / (RW * 32 * regs);
    return b < 1 ? 1 : b;
}

template <int PREC, int RW, int RPW, int NB, int UNR, int CH>
static cudaError_t rows_launch(const void* fhat, const float* scales, int n_freq, int N_d, int ldm, const void* xh,
                               int64_t xbs, void* dh, int64_t dbs, int nrhs, cudaStream_t st)
{
    using S = Store<PREC>;
    dim3 grid((N_d + RW * RPW - 1) / (RW * RPW), n_freq, (nrhs + NB - 1) / NB);
    k_gemv_fwd_rows<PREC, RW, RPW, NB, UNR, CH, rows_min_blocks<PREC, RW, NB>()><<<grid, RW * 32, 0, st>>>(
        static_cast<const typename S::elem*>(fhat), scales, N_d, ldm, static_cast<const float2*>(xh), xbs,
        static_cast<float2*>(dh), dbs, nrhs, lo_plane(PREC, n_freq, N_d, ldm));
    count_launch();
    return cudaGetLastError();
}

// Rows per CTA: 20, or 8 when that idles fewer warps.  Rows per warp: 1
// for FP32 (a 16-byte Fhat unit uses 16 bytes of mhat per vector), 2 for
// the 16-bit formats and the split pair, 4 for FP8 (32 and 64 bytes of mhat
// per unit: one shared-memory read serves that many rows).  Units in
// flight per lane and row: UNR.
template <int PREC, int NB, int UNR, int CH>
static cudaError_t rows_shape(const void* fhat, const float* scales, int n_freq, int N_d, int ldm, const void* xh,
                              int64_t xbs, void* dh, int64_t dbs, int nrhs, cudaStream_t st)
{
    constexpr int RPW = PREC == P_F32 ? 1 : ((PREC == P_FP8S && NB < 4) ? 4 : 2);
    const int w20 = (N_d + 19) / 20 * 20 - N_d, w8 = (N_d + 7) / 8 * 8 - N_d;
    if (w20 * 10 <= N_d || w20 <= w8)
        return rows_launch<PREC, 20 / RPW, RPW, NB, UNR, CH>(fhat, scales, n_freq, N_d, ldm, xh, xbs, dh, dbs, nrhs, st);
    return rows_launch<PREC, 8 / RPW, RPW, NB, UNR, CH>(fhat, scales, n_freq, N_d, ldm, xh, xbs, dh, dbs, nrhs, st);
}

template <int PREC>
static cudaError_t fwd_dispatch(const void* fhat, const float* scales, int n_freq, int N_d, int ldm,
                                const void* xh, int64_t xbs, void* dh, int64_t dbs, int nrhs,
                                cudaStream_t st)
{
    // UNR: 16-byte units in flight per lane and row (8 rows' worth for
    // FP32, ~8 per lane for the formats that decode); CH: mhat values per
    // chunk and vector (32 KB of shared memory at NB vectors)
    constexpr int U1 = PREC == P_F32 ? 8 : ((PREC == P_FP8S || PREC == P_BF16X2) ? 2 : 4);
    if (nrhs == 1) return rows_shape<PREC, 1, U1, 2048>(fhat, scales, n_freq, N_d, ldm, xh, xbs, dh, dbs, nrhs, st);
    constexpr int U2 = (U1 / 2 > 0) ? U1 / 2 : 1, U4 = (U1 / 4 > 0) ? U1 / 4 : 1;
    if (nrhs == 2) return rows_shape<PREC, 2, U2, 1024>(fhat, scales, n_freq, N_d, ldm, xh, xbs, dh, dbs, nrhs, st);
    return rows_shape<PREC, 4, U4, 512>(fhat, scales, n_freq, N_d, ldm, xh, xbs, dh, dbs, nrhs, st);
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

#ifdef BTT_CHECK
namespace btt {
BTT_CHECK_TU(check_record_gemv)
}  // namespace btt
#endif
