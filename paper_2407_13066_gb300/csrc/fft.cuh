// Shared-memory mixed-radix FFT along time for a tile of columns.
//
// The circulant embedding of Sec. 2.4 turns each time convolution into a
// length-L = 2 N_t cyclic one, diagonalised by the DFT (Eq. CirculantMatrix,
// Eq. FFTMatrixVectorProduct).  Every FFT in this library transforms
// columns of a time-outer array: the time index is the slow one in memory
// and consecutive columns are consecutive addresses, so a CTA loads a tile
// of W adjacent columns over all times with coalesced row segments, pairs
// two real columns into one complex sequence (a + i b), and runs the
// transform of the Wc = W/2 complex sequences in shared memory.
//
// Transform: in-place mixed radix (8, 4, 2, 3, 5, 7), decimation in
// frequency forward and in time inverse (details at fft_pass).  Spectra sit
// in shared memory in digit-reversed order; pos[k] (a per-length table)
// gives the position of frequency k.
//
// Shared layout: buf[n * Wc + c] for time/frequency n and complex column c.
#pragma once

#include "common.cuh"

namespace btt {

// -s*i times a (s = +1 forward kernel exp(-2 pi i/R), s = -1 inverse)
template <typename V> BTT_HD V mul_neg_si(V a, int s)
{
    return s > 0 ? cmake<V>(a.y, -a.x) : cmake<V>(-a.y, a.x);
}

template <typename V> BTT_HD void dft2(V* v, int)
{
    V a = v[0];
    v[0] = cadd(a, v[1]);
    v[1] = csub(a, v[1]);
}

template <typename V> BTT_HD void dft4(V* v, int s)
{
    V apc = cadd(v[0], v[2]), amc = csub(v[0], v[2]);
    V bpd = cadd(v[1], v[3]), t = mul_neg_si(csub(v[1], v[3]), s);
    v[0] = cadd(apc, bpd);
    v[2] = csub(apc, bpd);
    v[1] = cadd(amc, t);
    v[3] = csub(amc, t);
}

// 8-point DFT as two 4-point DFTs (even / odd inputs) and one radix-2 layer
// with the eighth roots of unity.
template <typename V> BTT_HD void dft8(V* v, int s)
{
    using T = decltype(V::x);
    const T h = (T)0.70710678118654752440084436210485;
    V e[4] = {v[0], v[2], v[4], v[6]};
    V o[4] = {v[1], v[3], v[5], v[7]};
    dft4(e, s);
    dft4(o, s);
    V o1 = cmake<V>(h * (o[1].x + s * o[1].y), h * (o[1].y - s * o[1].x));
    V o2 = mul_neg_si(o[2], s);
    V o3 = cmake<V>(h * (-o[3].x + s * o[3].y), h * (-s * o[3].x - o[3].y));
    v[0] = cadd(e[0], o[0]);
    v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], o1);
    v[5] = csub(e[1], o1);
    v[2] = cadd(e[2], o2);
    v[6] = csub(e[2], o2);
    v[3] = cadd(e[3], o3);
    v[7] = csub(e[3], o3);
}

// cos / sin of 2 pi e / R for the odd radices
template <int R> struct RootTable;
template <> struct RootTable<3> {
    static BTT_HD double c(int e) { return e == 0 ? 1.0 : -0.5; }
    static BTT_HD double s(int e)
    {
        return e == 0 ? 0.0 : (e == 1 ? 0.86602540378443864676372317075294 : -0.86602540378443864676372317075294);
    }
};
template <> struct RootTable<5> {
    static BTT_HD double c(int e)
    {
        return e == 0 ? 1.0
             : (e == 1 || e == 4) ? 0.30901699437494742410229341718282
                                  : -0.80901699437494742410229341718282;
    }
    static BTT_HD double s(int e)
    {
        return e == 0 ? 0.0
             : e == 1 ? 0.95105651629515357211643933337938
             : e == 2 ? 0.58778525229247312916870595463907
             : e == 3 ? -0.58778525229247312916870595463907
                      : -0.95105651629515357211643933337938;
    }
};
template <> struct RootTable<7> {
    static BTT_HD double c(int e)
    {
        return e == 0 ? 1.0
             : (e == 1 || e == 6) ? 0.62348980185873353052500488400424
             : (e == 2 || e == 5) ? -0.22252093395631440428890256449680
                                  : -0.90096886790241912623610231950745;
    }
    static BTT_HD double s(int e)
    {
        return e == 0 ? 0.0
             : e == 1 ? 0.78183148246802980870844452667406
             : e == 2 ? 0.97492791218182360701813168299393
             : e == 3 ? 0.43388373911755812047576833284836
             : e == 4 ? -0.43388373911755812047576833284836
             : e == 5 ? -0.97492791218182360701813168299393
                      : -0.78183148246802980870844452667406;
    }
};

// Odd R: pair inputs p and R-p, y_q = v_0 + sum_p (a_p cos - i s b_p sin)
// with a_p = v_p + v_{R-p}, b_p = v_p - v_{R-p}, angle 2 pi (p q mod R)/R.
template <int R, typename V> BTT_HD void dft_odd(V* v, int s)
{
    using T = decltype(V::x);
    constexpr int H = (R - 1) / 2;
    V a[H], b[H];
    V y0 = v[0];
#pragma unroll
    for (int p = 1; p <= H; ++p) {
        a[p - 1] = cadd(v[p], v[R - p]);
        b[p - 1] = csub(v[p], v[R - p]);
        y0 = cadd(y0, a[p - 1]);
    }
    V y[R];
    y[0] = y0;
#pragma unroll
    for (int q = 1; q < R; ++q) {
        T re = v[0].x, im = v[0].y;
#pragma unroll
        for (int p = 1; p <= H; ++p) {
            const int e = (p * q) % R;
            const T cs = (T)RootTable<R>::c(e);
            const T sn = (T)RootTable<R>::s(e) * (T)s;
            re += a[p - 1].x * cs + b[p - 1].y * sn;
            im += a[p - 1].y * cs - b[p - 1].x * sn;
        }
        y[q] = cmake<V>(re, im);
    }
#pragma unroll
    for (int q = 0; q < R; ++q) v[q] = y[q];
}

template <int R, typename V> BTT_HD void dft(V* v, int s)
{
    if constexpr (R == 2) dft2(v, s);
    else if constexpr (R == 4) dft4(v, s);
    else if constexpr (R == 8) dft8(v, s);
    else dft_odd<R>(v, s);
}

// R-point DFT of v[0 .. R/2-1] followed by R/2 zeros (the first forward
// pass over zero-padded data).  For R = 8 the even outputs are the 4-point
// DFT of the four inputs and the odd outputs the 4-point DFT of the inputs
// times the eighth roots of unity w^n (a radix-2 decimation in frequency
// whose second halves vanish), which skips the additions of zeros the full
// 8-point DFT would make.  Other radices take the full DFT.
template <typename V> BTT_HD void dft4_zero_half(V* v, int s)
{
    // inputs v[0], v[1]; v[2] = v[3] = 0
    const V a = v[0], b = v[1], t = mul_neg_si(b, s);
    v[0] = cadd(a, b);
    v[2] = csub(a, b);
    v[1] = cadd(a, t);
    v[3] = csub(a, t);
}

template <int R, typename V> BTT_HD void dft_half(V* v, int s)
{
    if constexpr (R == 8) {
        using T = decltype(V::x);
        const T h = (T)0.70710678118654752440084436210485;
        V e[4] = {v[0], v[1], v[2], v[3]};
        // o[n] = v[n] w_8^{n s}:  w_8^{s} = h (1 - s i), w_8^{2 s} = -s i, w_8^{3 s} = -h (1 + s i)
        V o[4] = {v[0],
                  cmake<V>(h * (v[1].x + s * v[1].y), h * (v[1].y - s * v[1].x)),
                  mul_neg_si(v[2], s),
                  cmake<V>(h * (-v[3].x + s * v[3].y), h * (-s * v[3].x - v[3].y))};
        dft4(e, s);
        dft4(o, s);
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            v[2 * m] = e[m];
            v[2 * m + 1] = o[m];
        }
    } else if constexpr (R == 4) {
        dft4_zero_half(v, s);
    } else if constexpr (R == 2) {
        v[1] = v[0];
    } else {
        dft<R>(v, s);
    }
}

// Sum of v over the NT threads of the block, written by thread 0 to *out.
// Called by every thread; uses its own shared scratch.
template <int NT> __device__ __forceinline__ void block_sum_store(double v, double* out)
{
    __shared__ double red[NT / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < NT / 32; ++i) s += red[i];
        *out = s;
    }
}

// In-place mixed-radix passes.  Forward transforms are decimation in
// frequency (natural order in, digit-reversed order out); inverse
// transforms are decimation in time (digit-reversed in, natural out), so a
// forward + inverse pair needs no reordering pass.  In a pass of radix R on
// sub-blocks of length M (M = L / product of the radices of earlier
// forward passes), butterfly (block, n1), n1 < M/R, owns the R elements
// block*M + n1 + i*M/R and writes its outputs back to the same places:
//   forward: v = DFT_R(v); v[k] *= w_M^{n1 k}
//   inverse: v[k] *= conj(w_M^{n1 k}); v = IDFT_R(v)
// with w_M^e = tw[e * L / M], tw[e] = exp(-2 pi i e / L).  Butterflies of one
// pass touch disjoint elements, so a pass needs only its R values in
// registers and one barrier at the end.
template <typename T, int R, int NT, bool INVERSE>
__device__ __forceinline__ void fft_pass(cplx_t<T>* buf, int L, int wc_log2, int M,
                                         const cplx_t<T>* __restrict__ tw)
{
    using V = cplx_t<T>;
    const int Wc = 1 << wc_log2;
    const int S = M / R;
    const int nb = (L / R) << wc_log2;
    const int tstep = L / M;
    for (int b = threadIdx.x; b < nb; b += NT) {
        const int c = b & (Wc - 1), j = b >> wc_log2;
        const int blk = j / S, n1 = j - blk * S;
        const int base = blk * M + n1;
        V v[R];
#pragma unroll
        for (int i = 0; i < R; ++i) v[i] = buf[((base + i * S) << wc_log2) + c];
        if (INVERSE) {
            if (n1 != 0) {
#pragma unroll
                for (int k = 1; k < R; ++k) {
                    V w = tw[n1 * k * tstep];
                    w.y = -w.y;
                    v[k] = cmul(v[k], w);
                }
            }
            dft<R>(v, -1);
        } else {
            dft<R>(v, +1);
            if (n1 != 0) {
#pragma unroll
                for (int k = 1; k < R; ++k) v[k] = cmul(v[k], tw[n1 * k * tstep]);
            }
        }
#pragma unroll
        for (int i = 0; i < R; ++i) buf[((base + i * S) << wc_log2) + c] = v[i];
    }
    __syncthreads();
}

template <typename T, int NT, bool INVERSE>
__device__ __forceinline__ void fft_radix_pass(int R, cplx_t<T>* buf, int L, int wc_log2, int M,
                                               const cplx_t<T>* __restrict__ tw)
{
    if (R == 8) fft_pass<T, 8, NT, INVERSE>(buf, L, wc_log2, M, tw);
    else if (R == 4) fft_pass<T, 4, NT, INVERSE>(buf, L, wc_log2, M, tw);
    else if (R == 2) fft_pass<T, 2, NT, INVERSE>(buf, L, wc_log2, M, tw);
    else if (R == 3) fft_pass<T, 3, NT, INVERSE>(buf, L, wc_log2, M, tw);
    else if (R == 5) fft_pass<T, 5, NT, INVERSE>(buf, L, wc_log2, M, tw);
    else fft_pass<T, 7, NT, INVERSE>(buf, L, wc_log2, M, tw);
}

// Forward DFT (kernel exp(-2 pi i n k / L)) of the Wc = 2^wc_log2 columns in
// buf: natural order in, X[k] ends at position pos[k] (digit reversed).
// The caller synchronises after filling buf.
template <typename T, int NT>
__device__ __forceinline__ void fft_forward(cplx_t<T>* buf, const FftPlan& plan, int wc_log2,
                                            const cplx_t<T>* __restrict__ tw)
{
    int M = plan.L;
    for (int p = 0; p < plan.nstages; ++p) {
        const int R = plan.radix[p];
        fft_radix_pass<T, NT, false>(R, buf, plan.L, wc_log2, M, tw);
        M /= R;
    }
}

// Inverse DFT without the 1/L factor: input X[k] at position pos[k],
// output x[n] at position n.
template <typename T, int NT>
__device__ __forceinline__ void fft_inverse(cplx_t<T>* buf, const FftPlan& plan, int wc_log2,
                                            const cplx_t<T>* __restrict__ tw)
{
    int M = 1;
    for (int p = plan.nstages - 1; p >= 0; --p) {
        const int R = plan.radix[p];
        M *= R;
        fft_radix_pass<T, NT, true>(R, buf, plan.L, wc_log2, M, tw);
    }
}

// Loads W = 2 Wc real columns col0 .. col0+W-1 of x[t][col] (t < N_t) as Wc
// complex sequences (column 2p -> real part, 2p+1 -> imaginary part of
// sequence p) and zero-pads times N_t .. L-1 (the padding of Sec. 2.4).
template <typename T, typename Tin, int NT>
__device__ __forceinline__ void load_real_pairs(cplx_t<T>* buf, const Tin* __restrict__ x,
                                                int64_t ldx, int N_t, int L, int col0, int ncols,
                                                int wc_log2)
{
    T* fb = reinterpret_cast<T*>(buf);
    const int wl = wc_log2 + 1;
    const int W = 1 << wl;
    const int n = N_t << wl;
    for (int idx = threadIdx.x; idx < n; idx += NT) {
        const int t = idx >> wl, c = idx & (W - 1);
        const int col = col0 + c;
        fb[idx] = col < ncols ? (T)x[(int64_t)t * ldx + col] : (T)0;
    }
    for (int idx = n + threadIdx.x; idx < (L << wl); idx += NT) fb[idx] = (T)0;
}

// Spectrum X_c[w] (w <= N_t) of real column c = 2p + h of the paired
// transform Z = A + i B (held at the digit-reversed positions pos[k]):  A[w] = (Z[w] + conj Z[L-w]) / 2,
//                          B[w] = (Z[w] - conj Z[L-w]) / (2 i).
template <typename V>
__device__ __forceinline__ V unpack_pair(const V* buf, const int* __restrict__ pos, int L, int w,
                                         int c, int wc_log2)
{
    const int p = c >> 1;
    const V z = buf[(__ldg(pos + w) << wc_log2) + p];
    const V zc = buf[(__ldg(pos + (w == 0 ? 0 : L - w)) << wc_log2) + p];
    using T = decltype(V::x);
    if ((c & 1) == 0) return cmake<V>((T)0.5 * (z.x + zc.x), (T)0.5 * (z.y - zc.y));
    return cmake<V>((T)0.5 * (z.y + zc.y), (T)0.5 * (zc.x - z.x));
}

// Loads the half spectra X[w][col] (w <= N_t) of W = 2 Wc real columns and
// forms, at the digit-reversed positions pos[k], the full length-L paired
// sequence Z = A + i B using Hermitian
// symmetry A[L-w] = conj A[w].  Bins 0 and N_t of a real series are real;
// their imaginary parts are dropped.
// One complex spectrum value as the transform's working type: complex64 /
// complex128 as stored, BF16 pairs widened to complex64.
__device__ __forceinline__ float2 cplx_in(const float2* p) { return *p; }
__device__ __forceinline__ double2 cplx_in(const double2* p) { return *p; }
__device__ __forceinline__ float2 cplx_in(const __nv_bfloat162* p) { return __bfloat1622float2(*p); }

template <typename V, int NT, typename TX = V>
__device__ __forceinline__ void load_hermitian_pairs(V* buf, const int* __restrict__ pos,
                                                     const TX* __restrict__ X, int64_t ldx,
                                                     int N_t, int L, int col0, int ncols,
                                                     int wc_log2)
{
    using T = decltype(V::x);
    const int Wc = 1 << wc_log2;
    const int n = (N_t + 1) << wc_log2;
    for (int idx = threadIdx.x; idx < n; idx += NT) {
        const int w = idx >> wc_log2, p = idx & (Wc - 1);
        const int ca = col0 + 2 * p, cb = ca + 1;
        V xa = cmake<V>(0, 0), xb = cmake<V>(0, 0);
        if (ca < ncols) xa = cplx_in(X + (int64_t)w * ldx + ca);
        if (cb < ncols) xb = cplx_in(X + (int64_t)w * ldx + cb);
        if (w == 0 || w == N_t) {
            xa.y = (T)0;
            xb.y = (T)0;
        }
        buf[(__ldg(pos + w) << wc_log2) + p] = cmake<V>(xa.x - xb.y, xa.y + xb.x);
        if (w > 0 && w < N_t)
            buf[(__ldg(pos + L - w) << wc_log2) + p] = cmake<V>(xa.x + xb.y, xb.x - xa.y);
    }
}

}  // namespace btt
