// Paired FP32 arithmetic for the fixed-plan time transforms.
//
// Blackwell executes two FP32 additions, multiplications or fused
// multiply-adds in one instruction (PTX add/sub/mul/fma.rn.f32x2 on a
// 64-bit register pair, each lane rounded exactly as the scalar operation
// would be).  The fixed-plan kernels give each thread a quad of four
// adjacent real columns: two complex sequences,
//     lane 0:  z0 = x[c] + i x[c+2],     lane 1:  z1 = x[c+1] + i x[c+3],
// held as one cq = {re = (Re z0, Re z1), im = (Im z0, Im z1)}.  Every
// butterfly operation is then one paired instruction for both sequences,
// and 16 bytes of a time-outer row (columns c .. c+3) are exactly {re, im}:
// one vector load or store moves a whole quad without reshuffling.
//
// The radix-2/4/8 DFTs below are the ones of fft.cuh (same definitions, same
// sign convention s = +1 forward, -1 inverse) written so that products with
// -s i never need a negation: the rotated operand's components enter the
// following additions with their signs swapped.
#pragma once

#include "fft.cuh"

namespace btt {
namespace fq {

struct f2 {
    unsigned long long u;
};

__device__ __forceinline__ f2 add(f2 a, f2 b)
{
    f2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.u) : "l"(a.u), "l"(b.u));
    return r;
}
__device__ __forceinline__ f2 sub(f2 a, f2 b)
{
    f2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.u) : "l"(a.u), "l"(b.u));
    return r;
}
__device__ __forceinline__ f2 mul(f2 a, f2 b)
{
    f2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.u) : "l"(a.u), "l"(b.u));
    return r;
}
// a * b + c, one rounding per lane
__device__ __forceinline__ f2 fma(f2 a, f2 b, f2 c)
{
    f2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.u) : "l"(a.u), "l"(b.u), "l"(c.u));
    return r;
}
__device__ __forceinline__ f2 pack(float lo, float hi)
{
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.u) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ f2 dup(float a) { return pack(a, a); }
__device__ __forceinline__ float lo(f2 a)
{
    float x;
    asm("{ .reg .f32 t; mov.b64 {%0, t}, %1; }" : "=f"(x) : "l"(a.u));
    return x;
}
__device__ __forceinline__ float hi(f2 a)
{
    float y;
    asm("{ .reg .f32 t; mov.b64 {t, %0}, %1; }" : "=f"(y) : "l"(a.u));
    return y;
}

// two complex values, one per lane
struct cq {
    f2 re, im;
};

__device__ __forceinline__ cq cadd(cq a, cq b) { return {add(a.re, b.re), add(a.im, b.im)}; }
__device__ __forceinline__ cq csub(cq a, cq b) { return {sub(a.re, b.re), sub(a.im, b.im)}; }

// 16 bytes <-> one quad
__device__ __forceinline__ cq from_u2(ulonglong2 u) { return {{u.x}, {u.y}}; }
__device__ __forceinline__ ulonglong2 to_u2(cq v) { return make_ulonglong2(v.re.u, v.im.u); }

// a + (-s i) b and a - (-s i) b
template <int S> __device__ __forceinline__ cq add_rot(cq a, cq b)
{
    return S > 0 ? cq{add(a.re, b.im), sub(a.im, b.re)} : cq{sub(a.re, b.im), add(a.im, b.re)};
}
template <int S> __device__ __forceinline__ cq sub_rot(cq a, cq b)
{
    return S > 0 ? cq{sub(a.re, b.im), add(a.im, b.re)} : cq{add(a.re, b.im), sub(a.im, b.re)};
}

// Twiddle factors: a quad table entry holds (c, c, d, d) for w = c + i d,
// the same factor for both lanes.  v * w and v * conj(w).
__device__ __forceinline__ cq twiddle(cq v, ulonglong2 w)
{
    const f2 c{w.x}, d{w.y};
    return {sub(mul(v.re, c), mul(v.im, d)), fma(v.re, d, mul(v.im, c))};
}
__device__ __forceinline__ cq twiddle_conj(cq v, ulonglong2 w)
{
    const f2 c{w.x}, d{w.y};
    return {fma(v.im, d, mul(v.re, c)), sub(mul(v.im, c), mul(v.re, d))};
}

template <int S> __device__ __forceinline__ void dft2(cq* v)
{
    const cq a = v[0];
    v[0] = cadd(a, v[1]);
    v[1] = csub(a, v[1]);
}

template <int S> __device__ __forceinline__ void dft4(cq* v)
{
    const cq apc = cadd(v[0], v[2]), amc = csub(v[0], v[2]);
    const cq bpd = cadd(v[1], v[3]), bmd = csub(v[1], v[3]);
    v[0] = cadd(apc, bpd);
    v[2] = csub(apc, bpd);
    v[1] = add_rot<S>(amc, bmd);
    v[3] = sub_rot<S>(amc, bmd);
}

// eighth roots of unity applied to o (o * w_8^{s}, o * w_8^{3 s}), h = 1/sqrt 2
template <int S> __device__ __forceinline__ cq root8_1(cq o)
{
    const f2 h = dup(0.70710678118654752440f);
    return S > 0 ? cq{mul(add(o.re, o.im), h), mul(sub(o.im, o.re), h)}
                 : cq{mul(sub(o.re, o.im), h), mul(add(o.im, o.re), h)};
}
template <int S> __device__ __forceinline__ cq root8_3(cq o)
{
    const f2 h = dup(0.70710678118654752440f), nh = dup(-0.70710678118654752440f);
    return S > 0 ? cq{mul(sub(o.im, o.re), h), mul(add(o.re, o.im), nh)}
                 : cq{mul(add(o.re, o.im), nh), mul(sub(o.re, o.im), h)};
}

template <int S> __device__ __forceinline__ void dft8(cq* v)
{
    cq e[4] = {v[0], v[2], v[4], v[6]};
    cq o[4] = {v[1], v[3], v[5], v[7]};
    dft4<S>(e);
    dft4<S>(o);
    const cq o1 = root8_1<S>(o[1]), o3 = root8_3<S>(o[3]);
    v[0] = cadd(e[0], o[0]);
    v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], o1);
    v[5] = csub(e[1], o1);
    v[2] = add_rot<S>(e[2], o[2]);   // o2 * w_8^{2s} = -s i o2
    v[6] = sub_rot<S>(e[2], o[2]);
    v[3] = cadd(e[3], o3);
    v[7] = csub(e[3], o3);
}

// Odd R: the pairing of dft_odd in fft.cuh (inputs p and R-p), constants as
// lane pairs.
template <int R, int S> __device__ __forceinline__ void dft_odd(cq* v)
{
    constexpr int H = (R - 1) / 2;
    cq a[H], b[H];
    cq y0 = v[0];
#pragma unroll
    for (int p = 1; p <= H; ++p) {
        a[p - 1] = cadd(v[p], v[R - p]);
        b[p - 1] = csub(v[p], v[R - p]);
        y0 = cadd(y0, a[p - 1]);
    }
    cq y[R];
    y[0] = y0;
#pragma unroll
    for (int q = 1; q < R; ++q) {
        f2 re = v[0].re, im = v[0].im;
#pragma unroll
        for (int p = 1; p <= H; ++p) {
            const int e = (p * q) % R;
            const float cs = (float)RootTable<R>::c(e);
            const float sn = (float)RootTable<R>::s(e) * (float)S;
            re = fma(a[p - 1].re, dup(cs), re);
            re = fma(b[p - 1].im, dup(sn), re);
            im = fma(a[p - 1].im, dup(cs), im);
            im = fma(b[p - 1].re, dup(-sn), im);
        }
        y[q] = {re, im};
    }
#pragma unroll
    for (int q = 0; q < R; ++q) v[q] = y[q];
}

template <int R, int S> __device__ __forceinline__ void dft(cq* v)
{
    if constexpr (R == 2) dft2<S>(v);
    else if constexpr (R == 4) dft4<S>(v);
    else if constexpr (R == 8) dft8<S>(v);
    else dft_odd<R, S>(v);
}

// 8-point forward DFT of v[0..3] followed by four zeros (the first pass over
// zero-padded data, as dft_half<8> in fft.cuh): even outputs are the 4-point
// DFT of the inputs, odd outputs the 4-point DFT of the inputs times w_8^{n}.
__device__ __forceinline__ void dft8_half_fwd(cq* v)
{
    cq e[4] = {v[0], v[1], v[2], v[3]};
    dft4<1>(e);
    // o = (v0, w v1, -i v2, w^3 v3); the -i v2 term enters the 4-point DFT
    // through add_rot / sub_rot
    const cq o0 = v[0], o1 = root8_1<1>(v[1]), o3 = root8_3<1>(v[3]);
    const cq apc = add_rot<1>(o0, v[2]), amc = sub_rot<1>(o0, v[2]);
    const cq bpd = cadd(o1, o3), bmd = csub(o1, o3);
    v[0] = e[0];
    v[2] = e[1];
    v[4] = e[2];
    v[6] = e[3];
    v[1] = cadd(apc, bpd);
    v[5] = csub(apc, bpd);
    v[3] = add_rot<1>(amc, bmd);
    v[7] = sub_rot<1>(amc, bmd);
}

}  // namespace fq
}  // namespace btt
