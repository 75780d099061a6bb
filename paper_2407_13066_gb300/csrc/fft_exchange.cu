// Time transforms of the lengths 2 N_t = 128, 256, 512, 1024 and 2048 with
// one exchange through shared memory (for_len below says which forms take
// them at each length).
//
// The fixed-plan kernels of fft_static.cu run a length-512 transform as
// three radix-8 passes, which moves the tile through shared memory twice
// (after the first pass and after the second).  Here the length splits as
// L = R1 x N2 with t = n2 + N2 n1 and k = k1 + R1 k2 (the four-step form of
// the DFT behind Alg. 2's FFT along time): R1 = L/16, N2 = 16 for L <= 512,
// R1 = 32, N2 = 16 E (E = 2, 4) for L = 1024, 2048:
//
//   stage 1:  y[k1][n2] = W_L^{n2 k1} sum_{n1 < R1} z[n2 + N2 n1] W_R1^{n1 k1}
//   stage 2:  Z[k1 + R1 k2] = sum_{n2 < N2} y[k1][n2] W_N2^{n2 k2}
//
// with W_n = exp(-2 pi i / n).  Stage 2 splits k2 = E j + e and starts with
// the length-E step sum_h W_E^{h e} y[k1][n + 16 h] times W_N2^{n e}, after
// which a 16-point DFT over n < 16 gives the outputs k1 + R1 (E j + e).
// Stage 1 reads its inputs straight from memory (the padding half, n1 >=
// R1/2, is zero and never read) and stage 2 writes the spectra straight to
// memory, so the tile is written to shared memory once (and read E times).
// Both stages run in paired FP32 instructions (fftq.cuh), each thread
// holding two complex sequences of one column pair (z = x[c] + i x[c+1]) as
// the two lanes:
//
//   * stage 1, task (n2, pair): lane 0 = z[n2 + N2 n1], lane 1 = the same
//     times W_R1^{n1}; one R1/2-point DFT of both lanes gives the even and
//     the odd k1 (y[2m] and y[2m+1]), twiddled by W_L^{n2 (2m)} and
//     W_L^{n2 (2m+1)} (a lane-pair table after the quad twiddles);
//   * stage 2, task (lanes, pair): lane 0 the outputs of (k1, e) = (u, e),
//     lane 1 those of (R1 - u, E - 1 - e) (task 0 of each pair: see
//     lanes_of); one 16-point DFT of both.  The Hermitian partner L - k of
//     every frequency k a thread computes lies in the same thread, so the
//     two real columns' spectra X_c = (Z[k] + conj Z[L-k]) / 2 and
//     X_{c+1} = (Z[k] - conj Z[L-k]) / 2i come from registers.
//
// The inverse mirrors this: stage 2' loads the half spectra of its
// frequencies and their partners (Z[k] = X_c + i X_{c+1}, Z[L-k] =
// conj X_c + i conj X_{c+1}) and runs the inverse 16-point DFTs; stage 1'
// combines the E halves, applies the conjugate twiddles and runs the
// inverse R1-point DFT, of which only the outputs n1 < R1/2 (t < N_t, the
// unpad of Alg. 2) are formed.
//
// Shared memory holds y as two planes (real and imaginary parts), P column
// pairs per CTA: element (k1, n2, c) at k1 (N2 P + P) + n2 P + c; the P
// floats between k1 blocks put the stage-2 reads of the 32 / P tasks of a
// warp at one n2 in distinct banks.  The lane-pair twiddles carry a factor
// 1/2 (exact in FP32): it is the 1/2 of the unpack in the forward
// transform, and the inverse scales by 2/L instead of 1/L.
#include <type_traits>
#include <utility>

#include "fft.cuh"
#include "fftq.cuh"
#include "kernels.h"

namespace btt {
namespace {

using fq::cq;
using fq::f2;

// cos(2 pi k / 32), k = 0..8 (cos(pi k / 16))
constexpr double kCos32[9] = {1.0,
                              0.98078528040323044912618223613424,
                              0.92387953251128675612818318939679,
                              0.83146961230254523707878837761791,
                              0.70710678118654752440084436210485,
                              0.55557023301960222474283081394853,
                              0.38268343236508977172845998403040,
                              0.19509032201612826784828486847702,
                              0.0};
constexpr double cos32(int k)
{
    k = ((k % 32) + 32) % 32;
    return k <= 8 ? kCos32[k] : k <= 16 ? -kCos32[16 - k] : k <= 24 ? -kCos32[k - 16] : kCos32[32 - k];
}
constexpr double sin32(int k) { return cos32(k - 8); }

// cos(2 pi k / 64), k = 0..16 (cos(pi k / 32))
constexpr double kCos64[17] = {1.0,
                               0.99518472667219688624483695310948,
                               0.98078528040323044912618223613424,
                               0.95694033573220886493579788698027,
                               0.92387953251128675612818318939679,
                               0.88192126434835502971275686366039,
                               0.83146961230254523707878837761791,
                               0.77301045336273696081090660975847,
                               0.70710678118654752440084436210485,
                               0.63439328416364549821517161322549,
                               0.55557023301960222474283081394853,
                               0.47139673682599764855638762590525,
                               0.38268343236508977172845998403040,
                               0.29028467725446236763619237581740,
                               0.19509032201612826784828486847702,
                               0.09801714032956060199419556388864,
                               0.0};
constexpr double cos64(int k)
{
    k = ((k % 64) + 64) % 64;
    return k <= 16 ? kCos64[k] : k <= 32 ? -kCos64[32 - k] : k <= 48 ? -kCos64[k - 32] : kCos64[64 - k];
}
constexpr double sin64(int k) { return cos64(k - 16); }

// f(integral_constant<int, i>) for i < N, every i a compile-time constant
template <int N, typename F> __device__ __forceinline__ void static_for(F&& f)
{
    [&]<int... I>(std::integer_sequence<int, I...>) { (f(std::integral_constant<int, I>{}), ...); }(
        std::make_integer_sequence<int, N>{});
}

__device__ __forceinline__ f2 swap_lanes(f2 a) { return fq::pack(fq::hi(a), fq::lo(a)); }

// v * exp(-S 2 pi i K / 32) on both lanes
template <int K, int S> __device__ __forceinline__ cq rot32(cq v)
{
    constexpr int k = ((K % 32) + 32) % 32;
    if constexpr (k == 0) {
        return v;
    } else if constexpr (k == 8 || k == 24) {
        // exp(-S i pi / 2) = -S i (k = 8); +S i (k = 24)
        constexpr int s = k == 8 ? S : -S;
        const f2 z = fq::dup(0.f);
        return s > 0 ? cq{v.im, fq::sub(z, v.re)} : cq{fq::sub(z, v.im), v.re};
    } else {
        const f2 c = fq::dup((float)cos32(k)), d = fq::dup((float)(-S * sin32(k)));
        return {fq::sub(fq::mul(v.re, c), fq::mul(v.im, d)), fq::fma(v.re, d, fq::mul(v.im, c))};
    }
}

// 16-point DFT of both lanes, natural order in and out: 4 x 4 with the
// twiddles W_16^{nb ka} between the two radix-4 layers.
template <int S> __device__ __forceinline__ void dft16(cq* v)
{
    cq a[4] = {v[0], v[4], v[8], v[12]};
    cq b[4] = {v[1], v[5], v[9], v[13]};
    cq c[4] = {v[2], v[6], v[10], v[14]};
    cq d[4] = {v[3], v[7], v[11], v[15]};
    fq::dft4<S>(a);
    fq::dft4<S>(b);
    fq::dft4<S>(c);
    fq::dft4<S>(d);
    b[1] = rot32<2, S>(b[1]);
    b[2] = rot32<4, S>(b[2]);
    b[3] = rot32<6, S>(b[3]);
    c[1] = rot32<4, S>(c[1]);
    c[2] = rot32<8, S>(c[2]);
    c[3] = rot32<12, S>(c[3]);
    d[1] = rot32<6, S>(d[1]);
    d[2] = rot32<12, S>(d[2]);
    d[3] = rot32<18, S>(d[3]);
#pragma unroll
    for (int ka = 0; ka < 4; ++ka) {
        cq t[4] = {a[ka], b[ka], c[ka], d[ka]};
        fq::dft4<S>(t);
#pragma unroll
        for (int kb = 0; kb < 4; ++kb) v[ka + 4 * kb] = t[kb];
    }
}

template <int N, int S> __device__ __forceinline__ void dft_lanes(cq* v)
{
    if constexpr (N == 16) dft16<S>(v);
    else if constexpr (N == 8) fq::dft8<S>(v);
    else fq::dft4<S>(v);
}

// Geometry: L = R1 N2, N2 = 16 E; stage 1 runs the R1-point DFTs (tasks n2
// < N2), stage 2 a length-E step and the 16-point DFTs (tasks: lane pairs).
template <int R1_, int E_, int PL_, int MINB_> struct XG {
    static constexpr int R1 = R1_, E = E_, N2 = 16 * E_, PL = PL_, P = 1 << PL, L = R1 * N2, N_t = L / 2, H = R1 / 2;
    static constexpr int MINB = MINB_;                  // CTAs per SM the registers are sized for
    static constexpr int NTX = N2 * P;                  // threads: one stage-1 task each
    static constexpr int KSTR = N2 * P + P;             // floats per k1 block (P floats of padding)
    static constexpr int PLANE = R1 * KSTR;             // floats per plane
    static constexpr size_t smem = 2 * (size_t)PLANE * sizeof(float);
    static_assert(E == 1 || ((E == 2 || E == 4) && R1 == 32), "lengths 16 R1, 1024 and 2048");
    __device__ __forceinline__ static int at(int k1, int n2, int c) { return k1 * KSTR + (n2 << PL) + c; }
};

// The two lanes of a stage-2 task: sequences (k1, e) -- the outputs
// k = k1 + R1 (E j + e), j < 16, e the residue of k2 = E j + e mod E -- with
// each output's Hermitian partner L - k in the same task: in general lane 0
// (u, e) and lane 1 (R1 - u, E - 1 - e), partners at j and 15 - j across
// the lanes; task 0 of each pair (u0) holds k1 = 0 (lane 0, partner of j
// at 16 - j) and a self-partnered lane 1 (partner at 15 - j): (0, 0) and
// (R1/2, 0) for E = 1, (0, 0) and (0, 1) for E = 2 (whose (R1/2, 0) and
// (R1/2, 1) pair in general form), (0, 0) and (0, 2) for E = 4.
struct Lanes {
    int ka, ea, kb, eb;
    bool u0;
};
template <class G> __device__ __forceinline__ Lanes lanes_of(int ti)
{
    constexpr int H = G::H;
    const int u = ti & (H - 1), ei = ti / H;
    if (u != 0) return {u, ei, G::R1 - u, G::E - 1 - ei, false};
    if constexpr (G::E == 1) return {0, 0, H, 0, true};
    else if constexpr (G::E == 2) return ei == 0 ? Lanes{0, 0, 0, 1, true} : Lanes{H, 0, H, 1, false};
    else {
        // E = 4: (0, 0) with (0, 2) self-partnered; (0, 1) with (0, 3), and
        // (R1/2, e) with (R1/2, 3 - e), in general form
        if (ei == 0) return {0, 0, 0, 2, true};
        if (ei == 1) return {0, 1, 0, 3, false};
        return {H, ei - 2, H, 5 - ei, false};
    }
}

__device__ __forceinline__ float sldx(const float* a, int i, int n)
{
    return BTT_IN(i, n, CK_FFT_SMEM) ? a[i] : 0.f;
}
__device__ __forceinline__ void sstx(float* a, int i, int n, float v)
{
    if (BTT_IN(i, n, CK_FFT_SMEM)) a[i] = v;
}

__device__ __forceinline__ bool al8(const void* p, int64_t ld)
{
    return ((reinterpret_cast<uintptr_t>(p) & 7) == 0) && ((ld & 1) == 0);
}

// A BF16 pair (re in the low half), round to nearest even, as 32 bits
__device__ __forceinline__ uint32_t bf16_bits(float re, float im)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(re, im);
    return *reinterpret_cast<const uint32_t*>(&h);
}

// Raw spectrum values of real columns cc, cc + 1 at one row: complex64
// (16 bytes) or BF16 pairs (8 bytes), decoded only after all of a task's
// rows are loaded (so that the loads are in flight together).
template <typename TX> struct Spec2;
template <> struct Spec2<float2> {
    using raw = float4;
    __device__ __forceinline__ static raw load(const float2* src) { return *reinterpret_cast<const float4*>(src); }
    __device__ __forceinline__ static raw load_part(const float2* src, int cc, int ncols)
    {
        const float2 z = make_float2(0.f, 0.f), a = cc < ncols ? src[0] : z, b = cc + 1 < ncols ? src[1] : z;
        return make_float4(a.x, a.y, b.x, b.y);
    }
    __device__ __forceinline__ static raw zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
    __device__ __forceinline__ static void dec(raw r, float2& a, float2& b)
    {
        a = make_float2(r.x, r.y);
        b = make_float2(r.z, r.w);
    }
};
template <> struct Spec2<__nv_bfloat162> {
    using raw = uint2;
    __device__ __forceinline__ static raw load(const __nv_bfloat162* src)
    {
        return __ldg(reinterpret_cast<const uint2*>(src));
    }
    __device__ __forceinline__ static raw load_part(const __nv_bfloat162* src, int cc, int ncols)
    {
        const uint32_t* s = reinterpret_cast<const uint32_t*>(src);
        return make_uint2(cc < ncols ? __ldg(s) : 0u, cc + 1 < ncols ? __ldg(s + 1) : 0u);
    }
    __device__ __forceinline__ static raw zero() { return make_uint2(0u, 0u); }
    __device__ __forceinline__ static void dec(raw r, float2& a, float2& b)
    {
        a = make_float2(__uint_as_float(r.x << 16), __uint_as_float(r.x & 0xFFFF0000u));
        b = make_float2(__uint_as_float(r.y << 16), __uint_as_float(r.y & 0xFFFF0000u));
    }
};

// Stage 1 of the forward transform for this thread's task (n2, c); leaves
// y in the planes.  FULL: the tile's columns are all inside the array and
// its rows 8-byte aligned (no per-column tests).
template <class G, bool FULL> __device__ __forceinline__ void stage1_fwd(float* re, float* im,
                                                                     const ulonglong2* __restrict__ twp,
                                                                     const float* __restrict__ xb, int64_t ldx,
                                                                     int col, int ncols)
{
    constexpr int H = G::H;
    const int c = threadIdx.x & (G::P - 1), n2 = threadIdx.x >> G::PL;
    float2 z[H];
    const float* p0 = xb + (int64_t)n2 * ldx + col;
    const int64_t step = G::N2 * ldx;
#pragma unroll
    for (int n1 = 0; n1 < H; ++n1) {
        const float* p = p0 + n1 * step;
        if (!BTT_IN(n2 + G::N2 * n1, G::N_t, CK_FFT_LOAD)) z[n1] = make_float2(0.f, 0.f);
        else if (FULL) z[n1] = __ldg(reinterpret_cast<const float2*>(p));
        else z[n1] = make_float2(col < ncols ? __ldg(p) : 0.f, col + 1 < ncols ? __ldg(p + 1) : 0.f);
    }
    cq v[H];
    static_for<H>([&](auto I) {
        constexpr int n1 = I;
        constexpr int k = n1 * (32 / G::R1);
        const float cw = (float)cos32(k), sw = (float)(-sin32(k));   // W_R1^{n1} = cw + i sw
        const float zr = z[n1].x, zi = z[n1].y;
        if constexpr (n1 == 0) v[n1] = {fq::dup(zr), fq::dup(zi)};
        else v[n1] = {fq::pack(zr, fmaf(zr, cw, -zi * sw)), fq::pack(zi, fmaf(zr, sw, zi * cw))};
    });
    dft_lanes<H, 1>(v);
#pragma unroll
    for (int m = 0; m < H; ++m) {
        v[m] = fq::twiddle(v[m], BTT_IN(n2 * H + m, G::L / 2, CK_FFT_TABLE) ? __ldg(twp + n2 * H + m) : ulonglong2{});
        sstx(re, G::at(2 * m, n2, c), G::PLANE, fq::lo(v[m].re));
        sstx(re, G::at(2 * m + 1, n2, c), G::PLANE, fq::hi(v[m].re));
        sstx(im, G::at(2 * m, n2, c), G::PLANE, fq::lo(v[m].im));
        sstx(im, G::at(2 * m + 1, n2, c), G::PLANE, fq::hi(v[m].im));
    }
}

// Stage 2 of the forward transform with the unpack: for every task (lanes
// of lanes_of, column pair c) of the tile, emit(w, c, A, B) receives the
// spectra of real columns
// col0 + 2c (A) and col0 + 2c + 1 (B) at every frequency w <= N_t of the
// task (conjugated when CONJ).
template <class G, bool CONJ, typename Emit> __device__ __forceinline__ void stage2_fwd(const float* re, const float* im,
                                                                                    Emit emit)
{
    constexpr int R1 = G::R1, H = G::H, E = G::E;
    for (int tk = threadIdx.x; tk < H * E * G::P; tk += G::NTX) {
        const int c = tk & (G::P - 1);
        const Lanes ln = lanes_of<G>(tk >> G::PL);
        const int ka = ln.ka, kb = ln.kb;
        cq v[16];
        if constexpr (E == 1) {
#pragma unroll
            for (int n2 = 0; n2 < 16; ++n2) {
                const int ia = G::at(ka, n2, c), ib = G::at(kb, n2, c);
                v[n2] = {fq::pack(sldx(re, ia, G::PLANE), sldx(re, ib, G::PLANE)),
                         fq::pack(sldx(im, ia, G::PLANE), sldx(im, ib, G::PLANE))};
            }
        } else if constexpr (E == 4) {
            // the length-4 step: sum_h W_4^{h e} y[k1][n + 16 h], times
            // W_64^{n e}, e chosen per lane through one-hot lane masks
            auto oh = [&](int k) { return fq::pack(ln.ea == k ? 1.f : 0.f, ln.eb == k ? 1.f : 0.f); };
            const f2 o0 = oh(0), o1 = oh(1), o2 = oh(2), o3 = oh(3);
            const f2 s2 = fq::sub(fq::add(o0, o2), fq::add(o1, o3));   // (-1)^e
            const f2 wr = fq::sub(o0, o2), wi = fq::sub(o3, o1);        // W_4^e = wr + i wi
            const f2 nwi = fq::sub(fq::dup(0.f), wi);
            static_for<16>([&](auto I) {
                constexpr int n = I;
                cq y[4];
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const int ia = G::at(ka, n + 16 * h, c), ib = G::at(kb, n + 16 * h, c);
                    y[h] = {fq::pack(sldx(re, ia, G::PLANE), sldx(re, ib, G::PLANE)),
                            fq::pack(sldx(im, ia, G::PLANE), sldx(im, ib, G::PLANE))};
                }
                const cq a = {fq::fma(s2, y[2].re, y[0].re), fq::fma(s2, y[2].im, y[0].im)};
                const cq b = {fq::fma(s2, y[3].re, y[1].re), fq::fma(s2, y[3].im, y[1].im)};
                const cq q = {fq::fma(wr, b.re, fq::fma(nwi, b.im, a.re)), fq::fma(wr, b.im, fq::fma(wi, b.re, a.im))};
                if constexpr (n == 0) {
                    v[n] = q;
                } else {
                    const f2 cw = fq::fma(o3, fq::dup((float)cos64(3 * n)),
                                          fq::fma(o2, fq::dup((float)cos64(2 * n)), fq::fma(o1, fq::dup((float)cos64(n)), o0)));
                    const f2 dw = fq::fma(o3, fq::dup((float)-sin64(3 * n)),
                                          fq::fma(o2, fq::dup((float)-sin64(2 * n)), fq::mul(o1, fq::dup((float)-sin64(n)))));
                    v[n] = {fq::sub(fq::mul(q.re, cw), fq::mul(q.im, dw)), fq::fma(q.re, dw, fq::mul(q.im, cw))};
                }
            });
        } else {
            // the length-2 step: y[k1][n] + (-1)^e y[k1][n + 16], times W_32^{n e}
            const f2 sg = fq::pack(ln.ea ? -1.f : 1.f, ln.eb ? -1.f : 1.f);
            const f2 ep = fq::pack((float)ln.ea, (float)ln.eb);
            static_for<16>([&](auto I) {
                constexpr int n = I;
                const int a0 = G::at(ka, n, c), a1 = G::at(ka, n + 16, c);
                const int b0 = G::at(kb, n, c), b1 = G::at(kb, n + 16, c);
                const cq p0 = {fq::pack(sldx(re, a0, G::PLANE), sldx(re, b0, G::PLANE)),
                               fq::pack(sldx(im, a0, G::PLANE), sldx(im, b0, G::PLANE))};
                const cq p1 = {fq::pack(sldx(re, a1, G::PLANE), sldx(re, b1, G::PLANE)),
                               fq::pack(sldx(im, a1, G::PLANE), sldx(im, b1, G::PLANE))};
                const cq q = {fq::fma(sg, p1.re, p0.re), fq::fma(sg, p1.im, p0.im)};
                if constexpr (n == 0) {
                    v[n] = q;
                } else {
                    const f2 cw = fq::fma(ep, fq::dup((float)(cos32(n) - 1.0)), fq::dup(1.f));
                    const f2 dw = fq::mul(ep, fq::dup((float)(-sin32(n))));
                    v[n] = {fq::sub(fq::mul(q.re, cw), fq::mul(q.im, dw)), fq::fma(q.re, dw, fq::mul(q.im, cw))};
                }
            });
        }
        dft16<1>(v);
        // Task 0 (lanes k1 = 0 and R1/2) pairs differently: lane 0's partner
        // of R1 k2 is lane 0 at (16 - k2) mod 16, lane 1's lane 1 at 15 - k2;
        // the other tasks pair lane 0 at k2 with lane 1 at 15 - k2 and back.
        // Per-lane selects take the partners, so every task runs one path.
        const bool u0 = ln.u0;
#pragma unroll
        for (int k2 = 0; k2 < 8; ++k2) {
            const cq zf = v[k2], x = v[15 - k2], y = v[(16 - k2) & 15];
            const cq zp = {fq::pack(u0 ? fq::lo(y.re) : fq::hi(x.re), u0 ? fq::hi(x.re) : fq::lo(x.re)),
                           fq::pack(u0 ? fq::lo(y.im) : fq::hi(x.im), u0 ? fq::hi(x.im) : fq::lo(x.im))};   // Z[L - k]
            // (the 1/2 of the unpack is in the twiddles)
            const f2 ar = fq::add(zf.re, zp.re);
            const f2 ai = CONJ ? fq::sub(zp.im, zf.im) : fq::sub(zf.im, zp.im);
            const f2 br = fq::add(zf.im, zp.im);
            const f2 bi = CONJ ? fq::sub(zf.re, zp.re) : fq::sub(zp.re, zf.re);
            const int wa = ka + R1 * (E * k2 + ln.ea), wb = kb + R1 * (E * k2 + ln.eb);
            if (BTT_IN(wa, G::N_t + 1, CK_FFT_STORE))
                emit(wa, c, make_float2(fq::lo(ar), fq::lo(ai)), make_float2(fq::lo(br), fq::lo(bi)));
            if (BTT_IN(wb, G::N_t + 1, CK_FFT_STORE))
                emit(wb, c, make_float2(fq::hi(ar), fq::hi(ai)), make_float2(fq::hi(br), fq::hi(bi)));
        }
        // N_t = R1 * 8 E (task 0, lane 0, its own partner): 2 Re Z and 2 Im Z
        if (u0) emit(G::N_t, c, make_float2(2.f * fq::lo(v[8].re), 0.f), make_float2(2.f * fq::lo(v[8].im), 0.f));
    }
}

// Stage 2' of the inverse transform: for every task (lanes (ka, ea), (kb,
// eb), column pair c) the half spectra of its frequencies and the Hermitian
// extension, then the inverse 16-point DFT; leaves G_e[k1][n] (the inverse
// DFT of the outputs of residue e) in the planes at (k1, n + 16 e).  Every
// task loads the rows ka + R1 (E j + ea) and kb + R1 (E j + eb) (j < 8),
// task 0 also row N_t; all loads of a task are issued before the first is
// decoded.  FULL: the tile's columns are all inside the array and its rows
// aligned.
template <class G, bool FULL, typename TX> __device__ __forceinline__ void stage2_inv(float* re, float* im,
                                                                                  const TX* __restrict__ Xb,
                                                                                  int64_t ldx, int col0, int ncols)
{
    using S = Spec2<TX>;
    constexpr int R1 = G::R1, H = G::H, E = G::E, N_t = G::N_t;
    for (int tk = threadIdx.x; tk < H * E * G::P; tk += G::NTX) {
        const int c = tk & (G::P - 1);
        const Lanes ln = lanes_of<G>(tk >> G::PL);
        const int ka = ln.ka, kb = ln.kb;
        const int cc = col0 + 2 * c;
        auto ld = [&](int w) {
            if (!BTT_IN(w, N_t + 1, CK_FFT_LOAD)) return S::zero();
            const TX* src = Xb + (int64_t)w * ldx + cc;
            return FULL ? S::load(src) : S::load_part(src, cc, ncols);
        };
        typename S::raw r[17];
#pragma unroll
        for (int k2 = 0; k2 < 8; ++k2) {
            r[k2] = ld(ka + R1 * (E * k2 + ln.ea));
            r[8 + k2] = ld(kb + R1 * (E * k2 + ln.eb));
        }
        r[16] = ln.u0 ? ld(N_t) : S::zero();
        float2 A[17], B[17];   // rows of lane 0 (j < 8), of lane 1, N_t
#pragma unroll
        for (int i = 0; i < 17; ++i) S::dec(r[i], A[i], B[i]);
        // Z[w] = X_c + i X_{c+1} and Z[L - w] = conj X_c + i conj X_{c+1} of
        // each row; task 0 (lanes k1 = 0 and R1/2) places its partners
        // differently (lane 0: Z[L - R1 k2] at 16 - k2, Z[N_t] at 8, rows 0
        // and N_t real; lane 1 as the others' lane 0 mirrored), by per-lane
        // selects, so every task runs one path
        const bool u0 = ln.u0;
        if (u0) A[0].y = B[0].y = 0.f;
        cq v[16], zb[8];
#pragma unroll
        for (int k2 = 0; k2 < 8; ++k2) {
            const cq p = {fq::pack(A[k2].x, A[8 + k2].x), fq::pack(A[k2].y, A[8 + k2].y)};
            const cq q = {fq::pack(B[k2].x, B[8 + k2].x), fq::pack(B[k2].y, B[8 + k2].y)};
            v[k2] = {fq::sub(p.re, q.im), fq::add(p.im, q.re)};
            zb[k2] = {fq::add(p.re, q.im), fq::sub(q.re, p.im)};
        }
        const float znr = A[16].x, zni = B[16].x;   // Z[N_t] (row N_t real; zero unless task 0)
#pragma unroll
        for (int p = 8; p < 16; ++p) {
            const cq x = zb[15 - p];
            const float lr = p == 8 ? znr : fq::lo(zb[(16 - p) & 7].re), li = p == 8 ? zni : fq::lo(zb[(16 - p) & 7].im);
            v[p] = {fq::pack(u0 ? lr : fq::hi(x.re), u0 ? fq::hi(x.re) : fq::lo(x.re)),
                    fq::pack(u0 ? li : fq::hi(x.im), u0 ? fq::hi(x.im) : fq::lo(x.im))};
        }
        dft16<-1>(v);
#pragma unroll
        for (int n2 = 0; n2 < 16; ++n2) {
            const int ia = G::at(ka, n2 + 16 * ln.ea, c), ib = G::at(kb, n2 + 16 * ln.eb, c);
            sstx(re, ia, G::PLANE, fq::lo(v[n2].re));
            sstx(re, ib, G::PLANE, fq::hi(v[n2].re));
            sstx(im, ia, G::PLANE, fq::lo(v[n2].im));
            sstx(im, ib, G::PLANE, fq::hi(v[n2].im));
        }
    }
}

// Stage 1' of the inverse transform for this thread's task (n2, c):
// y[k1][n2] = sum_e W_N2^{-n2 e} G_e[k1][n2 mod 16] (the twiddles from the
// complex table, conjugated), then the conjugate lane-pair twiddles and
// the inverse R1-point DFT; emit(t, c, value) for t = n2 + N2 n1 < N_t,
// value = the unscaled complex sample (columns col0 + 2c, + 1 as real and
// imaginary part).
template <class G, typename Emit> __device__ __forceinline__ void stage1_inv(const float* re, const float* im,
                                                                          const ulonglong2* __restrict__ twp,
                                                                          const float2* __restrict__ twc, Emit emit)
{
    constexpr int H = G::H;
    const int c = threadIdx.x & (G::P - 1), n2 = threadIdx.x >> G::PL;
    // W_N2^{-n2 e}, e = 1 .. E-1, from the complex table (conjugated)
    f2 wc[G::E], ws[G::E];
#pragma unroll
    for (int e = 1; e < G::E; ++e) {
        const int k = ((G::L / G::N2) * n2 * e) & (G::L - 1);
        const float2 w = BTT_IN(k, G::L, CK_FFT_TABLE) ? __ldg(twc + k) : make_float2(1.f, 0.f);
        wc[e] = fq::dup(w.x);
        ws[e] = fq::dup(-w.y);
    }
    cq v[H];
#pragma unroll
    for (int m = 0; m < H; ++m) {
        const int n = n2 & 15;
        const int ie = G::at(2 * m, n, c), io = G::at(2 * m + 1, n, c);
        v[m] = {fq::pack(sldx(re, ie, G::PLANE), sldx(re, io, G::PLANE)),
                fq::pack(sldx(im, ie, G::PLANE), sldx(im, io, G::PLANE))};
#pragma unroll
        for (int e = 1; e < G::E; ++e) {
            const int je = G::at(2 * m, n + 16 * e, c), jo = G::at(2 * m + 1, n + 16 * e, c);
            const cq g = {fq::pack(sldx(re, je, G::PLANE), sldx(re, jo, G::PLANE)),
                          fq::pack(sldx(im, je, G::PLANE), sldx(im, jo, G::PLANE))};
            v[m].re = fq::fma(g.re, wc[e], fq::fma(g.im, fq::sub(fq::dup(0.f), ws[e]), v[m].re));
            v[m].im = fq::fma(g.re, ws[e], fq::fma(g.im, wc[e], v[m].im));
        }
        v[m] = fq::twiddle_conj(v[m], BTT_IN(n2 * H + m, G::L / 2, CK_FFT_TABLE) ? __ldg(twp + n2 * H + m) : ulonglong2{});
    }
    dft_lanes<H, -1>(v);
    static_for<H>([&](auto I) {
        constexpr int n1 = I;
        constexpr int k = n1 * (32 / G::R1);
        const float cw = (float)cos32(k), sw = (float)sin32(k);   // W_R1^{-n1} = cw + i sw
        const float er = fq::lo(v[n1].re), ei = fq::lo(v[n1].im), orr = fq::hi(v[n1].re), oi = fq::hi(v[n1].im);
        float2 zz;
        if constexpr (n1 == 0) zz = make_float2(er + orr, ei + oi);
        else zz = make_float2(er + fmaf(orr, cw, -oi * sw), ei + fmaf(orr, sw, oi * cw));
        if (BTT_IN(n2 + G::N2 * n1, G::N_t, CK_FFT_STORE)) emit(n2 + G::N2 * n1, c, zz);
    });
}

// ------------------------------------------------------------------ kernels
// Operand transform for the tensor-core products: conj spectra as BF16
// pairs in [w][mt][64][ldm] (SPLIT: and the remainders conj X - hi as a
// second BF16 plane lo_off pairs further, the split pair's lo plane).
template <class G, bool FULL, bool SPLIT>
__device__ __forceinline__ void rfft_stack_body(float* re, float* im, const float* __restrict__ xb, int64_t ldx,
                                                int ncols, int col0, int b, __nv_bfloat162* __restrict__ XA, int ldm,
                                                int mt_stride, const ulonglong2* __restrict__ twp, int64_t lo_off)
{
    const int col = col0 + 2 * (threadIdx.x & (G::P - 1));
    stage1_fwd<G, FULL>(re, im, twp, xb, ldx, col, ncols);
    __syncthreads();
    const int mt = b >> 6, j = b & 63;
    __nv_bfloat162* const XAb = XA + ((int64_t)mt * 64 + j) * ldm + col0;
    const int64_t wstride = (int64_t)mt_stride * 64 * ldm;
    stage2_fwd<G, true>(re, im, [&](int w, int c, float2 A, float2 B) {
        const int cc = col0 + 2 * c;
        if (!FULL && cc >= ncols) return;
        __nv_bfloat162* dst = XAb + w * wstride + 2 * c;
        const uint32_t ha = bf16_bits(A.x, A.y), hb = bf16_bits(B.x, B.y);
        const bool two = FULL || cc + 1 < ncols;
        if (two) *reinterpret_cast<uint2*>(dst) = make_uint2(ha, hb);
        else *reinterpret_cast<uint32_t*>(dst) = ha;
        if constexpr (SPLIT) {
            const uint32_t la = bf16_bits(A.x - __uint_as_float(ha << 16), A.y - __uint_as_float(ha & 0xFFFF0000u));
            const uint32_t lb = bf16_bits(B.x - __uint_as_float(hb << 16), B.y - __uint_as_float(hb & 0xFFFF0000u));
            if (two) *reinterpret_cast<uint2*>(dst + lo_off) = make_uint2(la, lb);
            else *reinterpret_cast<uint32_t*>(dst + lo_off) = la;
        }
    });
}

template <class G, bool SPLIT>
__global__ void __launch_bounds__(G::NTX, G::MINB)
k_rfft_stack_x(const float* __restrict__ x, int64_t ldx, int64_t bsx, int ncols, __nv_bfloat162* __restrict__ XA,
               int ldm, int mt_stride, const ulonglong2* __restrict__ twp, const float* const* __restrict__ xptr,
               int64_t lo_off)
{
    extern __shared__ __align__(16) float smem_x[];
    float* re = smem_x;
    float* im = smem_x + G::PLANE;
    const int col0 = blockIdx.x * 2 * G::P;
    const int b = blockIdx.y;
    const float* xb = xptr ? xptr[b] : x + (int64_t)b * bsx;
    // 8-byte stores need an even ldm and lo_off (and the aligned base the allocator gives)
    if (al8(xb, ldx) && col0 + 2 * G::P <= ncols && (ldm & 1) == 0 && (lo_off & 1) == 0)
        rfft_stack_body<G, true, SPLIT>(re, im, xb, ldx, ncols, col0, b, XA, ldm, mt_stride, twp, lo_off);
    else
        rfft_stack_body<G, false, SPLIT>(re, im, xb, ldx, ncols, col0, b, XA, ldm, mt_stride, twp, lo_off);
}

// Input transform with complex64 spectra X[b][w][ldo].
template <class G, bool FULL>
__device__ __forceinline__ void rfft_body(float* re, float* im, const float* __restrict__ xb, int64_t ldx, int ncols,
                                          int col0, float2* __restrict__ Xb, int64_t ldo,
                                          const ulonglong2* __restrict__ twp)
{
    const int col = col0 + 2 * (threadIdx.x & (G::P - 1));
    stage1_fwd<G, FULL>(re, im, twp, xb, ldx, col, ncols);
    __syncthreads();
    stage2_fwd<G, false>(re, im, [&](int w, int c, float2 A, float2 B) {
        const int cc = col0 + 2 * c;
        if (!FULL && cc >= ncols) return;
        float2* dst = Xb + (int64_t)w * ldo + cc;
        if (FULL) {
            *reinterpret_cast<float4*>(dst) = make_float4(A.x, A.y, B.x, B.y);
        } else {
            dst[0] = A;
            if (cc + 1 < ncols) dst[1] = B;
        }
    });
}

template <class G>
__global__ void __launch_bounds__(G::NTX, G::MINB)
k_rfft_x(const float* __restrict__ x, int64_t ldx, int64_t bsx, int ncols, float2* __restrict__ X, int64_t ldo,
         int64_t bso, const ulonglong2* __restrict__ twp, const float* const* __restrict__ xptr)
{
    extern __shared__ __align__(16) float smem_x[];
    float* re = smem_x;
    float* im = smem_x + G::PLANE;
    const int col0 = blockIdx.x * 2 * G::P;
    const int64_t b = blockIdx.y;
    const float* xb = xptr ? xptr[b] : x + b * bsx;
    float2* Xb = X + b * bso;
    const bool o4 = ((reinterpret_cast<uintptr_t>(Xb) & 15) == 0) && ((ldo & 1) == 0);
    if (al8(xb, ldx) && o4 && col0 + 2 * G::P <= ncols)
        rfft_body<G, true>(re, im, xb, ldx, ncols, col0, Xb, ldo, twp);
    else
        rfft_body<G, false>(re, im, xb, ldx, ncols, col0, Xb, ldo, twp);
}

// Inverse transform from complex64 or BF16 half spectra X[b][w][ldx] to
// y[b][t][ldy] (t < N_t), scaled by 1/L and, with g, by g[t][col].
template <class G, bool FULL, typename TX>
__device__ __forceinline__ void irfft_body(float* re, float* im, const TX* __restrict__ Xb, int64_t ldx, int ncols,
                                           int col0, float* __restrict__ yb, int64_t ldy,
                                           const float* __restrict__ g, const ulonglong2* __restrict__ twp,
                                           const float2* __restrict__ twc)
{
    stage2_inv<G, FULL, TX>(re, im, Xb, ldx, col0, ncols);
    __syncthreads();
    constexpr float inv = 2.0f / (float)G::L;   // the twiddles' 1/2 undone
    stage1_inv<G>(re, im, twp, twc, [&](int t, int c, float2 v) {
        const int cc = col0 + 2 * c;
        float a = v.x * inv, e = v.y * inv;
        if (FULL) {
            if (g) {
                const float2 gg = __ldg(reinterpret_cast<const float2*>(g + (int64_t)t * ncols + cc));
                a *= gg.x;
                e *= gg.y;
            }
            *reinterpret_cast<float2*>(yb + (int64_t)t * ldy + cc) = make_float2(a, e);
            return;
        }
        if (cc < ncols) {
            if (g) a *= g[(int64_t)t * ncols + cc];
            yb[(int64_t)t * ldy + cc] = a;
        }
        if (cc + 1 < ncols) {
            if (g) e *= g[(int64_t)t * ncols + cc + 1];
            yb[(int64_t)t * ldy + cc + 1] = e;
        }
    });
}

template <class G, typename TX>
__global__ void __launch_bounds__(G::NTX, G::MINB)
k_irfft_x(const TX* __restrict__ X, int64_t ldx, int64_t bsx, int ncols, float* __restrict__ y, int64_t ldy,
          int64_t bsy, const float* __restrict__ g, const ulonglong2* __restrict__ twp, const float2* __restrict__ twc,
          float* const* __restrict__ yptr)
{
    extern __shared__ __align__(16) float smem_x[];
    float* re = smem_x;
    float* im = smem_x + G::PLANE;
    const int col0 = blockIdx.x * 2 * G::P;
    const int64_t b = blockIdx.y;
    const TX* Xb = X + b * bsx;
    float* yb = yptr ? yptr[b] : y + b * bsy;
    const bool in2 = ((reinterpret_cast<uintptr_t>(Xb) & (2 * sizeof(TX) - 1)) == 0) && ((ldx & 1) == 0);
    const bool out2 = al8(yb, ldy) && (g == nullptr || al8(g, ncols));
    if (in2 && out2 && col0 + 2 * G::P <= ncols)
        irfft_body<G, true, TX>(re, im, Xb, ldx, ncols, col0, yb, ldy, g, twp, twc);
    else
        irfft_body<G, false, TX>(re, im, Xb, ldx, ncols, col0, yb, ldy, g, twp, twc);
}

// ------------------------------------------------------------- dispatch
// Whether the environment switched these kernels off (BTT_FFT_EXCHANGE=0,
// read once: the fft_static.cu forms then run at every length, for
// comparisons).
bool enabled()
{
    static const bool on = [] {
        const char* s = getenv("BTT_FFT_EXCHANGE");
        return !(s && s[0] == '0');
    }();
    return on;
}

// The transforms these kernels replace, and where: the lengths and forms
// that measured faster on a GB300 than the fft_static.cu kernels (library
// stage timers, 20 calls; 64-vector BF16 batches on the tensor cores and
// 8-vector FP32 batches, N_t N_m = 6.4 M and 12.8 M):
//   2 N_t = 2048: FP32 input -32%, FP32 inverse -48%, BF16 operand
//                 transform -31%, BF16 inverse -46% (32-vector BF16 batches
//                 at N_m = 50 000: operand -37%, inverse -31%);
//   2 N_t = 1024: FP32 input -35%, FP32 inverse -28%, BF16 operand
//                 transform -28%, BF16 inverse -26%;
//   2 N_t = 512:  BF16 operand transform -17%, BF16 inverse -16%, FP32
//                 input transform -26%, FP32 inverse -23% (the split pair's
//                 complex64 inverse -21%);
//   2 N_t = 256:  FP32 input -4%, BF16 inverse -16% (BF16 operand transform
//                 +3.5%, FP32 inverse +3%: not taken);
//   2 N_t = 128:  FP32 input -4%, FP32 inverse -8%, BF16 operand transform
//                 -11%, BF16 inverse -22%.
// The split pair's operand transform (a second BF16 plane per spectrum)
// takes them too: -11% at 512 (64 vectors).  4-pair tiles for the inverses
// at 512 measured 16-18% slower.
// Tiles: 8 column pairs per CTA at 128-512 (128 threads, 34 KB of shared
// memory), registers for four CTAs per SM (96 registers for five measured
// 1-5% slower; 80 for six, with spills, 30-40% slower), except the operand
// transform at 512 (16 pairs, 256 threads, 68 KB, two CTAs per SM); at 1024
// 8 pairs (256 threads, 68 KB, two CTAs per SM) for the input transforms
// and 4 pairs (128 threads, 34 KB, four per SM) for the inverses; at 2048
// 4 pairs (256 threads, 66 KB, two per SM), the operand transform 8 pairs
// (512 threads, 130 KB, one per SM).
enum Form { F_INPUT, F_STACK, F_INV32, F_INV16 };

template <Form FORM, typename F> bool for_len(int L, F&& f)
{
    if (!enabled()) return false;
    if (L == 2048) {
        // the operand transform on 8-pair tiles (512 threads, 130 KB, one CTA
        // per SM): -6% (64 x 6 250 columns) to -26% (32 x 50 000) against 4
        // pairs; the other forms 13-23% slower so
        if constexpr (FORM == F_STACK) f(XG<32, 4, 3, 1>{});
        else f(XG<32, 4, 2, 2>{});
        return true;
    }
    if (L == 1024) {
        // the inverses on 4-pair tiles (34 KB, four CTAs per SM): FP32 -7%,
        // BF16 -6% against 8 pairs; the input transforms 2-28% slower so
        if constexpr (FORM == F_INV32 || FORM == F_INV16) f(XG<32, 2, 2, 4>{});
        else f(XG<32, 2, 3, 2>{});
        return true;
    }
    if (L == 512) {
        // the operand transform on 16-pair tiles (128-byte rows, two CTAs
        // per SM): -2.4% against 8 pairs; the other forms +11% to +25% (and
        // 4 pairs for the inverses +16-18%)
        if constexpr (FORM == F_STACK) f(XG<32, 1, 4, 2>{});
        else f(XG<32, 1, 3, 4>{});
        return true;
    }
    if constexpr (FORM == F_INPUT || FORM == F_INV16) {
        if (L == 256) {
            f(XG<16, 1, 3, 4>{});
            return true;
        }
    }
    if (L == 128) {
        f(XG<8, 1, 3, 4>{});
        return true;
    }
    return false;
}

template <class G> dim3 grid_x(int ncols, int nb) { return dim3((unsigned)((ncols + 2 * G::P - 1) / (2 * G::P)), (unsigned)nb, 1); }

const ulonglong2* pair_table(const float2* tw, int L) { return reinterpret_cast<const ulonglong2*>(tw + 3 * (size_t)L); }

}  // namespace

// Shared-memory limits of the kernels whose tiles exceed the 48 KB default.
cudaError_t prepare_exchange_fft()
{
    cudaError_t e = cudaSuccess;
    auto set = [&](auto kern, size_t bytes) {
        if (e == cudaSuccess && bytes > 48 * 1024)
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    };
    auto stack = [&](auto geo) {
        using G = decltype(geo);
        set(k_rfft_stack_x<G, false>, G::smem);
        set(k_rfft_stack_x<G, true>, G::smem);
    };
    stack(XG<32, 1, 4, 2>{});
    using G10 = XG<32, 2, 3, 2>;
    stack(G10{});
    set(k_rfft_x<G10>, G10::smem);
    auto all = [&](auto geo) {
        using G = decltype(geo);
        set(k_rfft_x<G>, G::smem);
        set(k_irfft_x<G, float2>, G::smem);
        set(k_irfft_x<G, __nv_bfloat162>, G::smem);
    };
    all(XG<32, 4, 2, 2>{});
    stack(XG<32, 4, 3, 1>{});

    return e;
}

bool exchange_rfft_stack(const float* x, int64_t ldx, int64_t bsx, int ncols, void* xstack, int ldm, int mt_stride,
                         int nb, const FftGeom& g, const float2* tw, cudaStream_t st, int64_t lo_off,
                         const float* const* xptr, cudaError_t* err)
{
    return for_len<F_STACK>(g.L, [&](auto geo) {
        using G = decltype(geo);
        auto* xs = static_cast<__nv_bfloat162*>(xstack);
        if (lo_off)
            k_rfft_stack_x<G, true><<<grid_x<G>(ncols, nb), G::NTX, G::smem, st>>>(x, ldx, bsx, ncols, xs, ldm,
                                                                                mt_stride, pair_table(tw, g.L), xptr,
                                                                                lo_off);
        else
            k_rfft_stack_x<G, false><<<grid_x<G>(ncols, nb), G::NTX, G::smem, st>>>(x, ldx, bsx, ncols, xs, ldm,
                                                                                 mt_stride, pair_table(tw, g.L), xptr,
                                                                                 0);
        count_launch();
        *err = cudaGetLastError();
    });
}

bool exchange_rfft(const float* x, int64_t ldx, int64_t bsx, int ncols, float2* X, int64_t ldo, int64_t bso, int nb,
                   const FftGeom& g, const float2* tw, cudaStream_t st, const float* const* xptr, cudaError_t* err)
{
    return for_len<F_INPUT>(g.L, [&](auto geo) {
        using G = decltype(geo);
        k_rfft_x<G><<<grid_x<G>(ncols, nb), G::NTX, G::smem, st>>>(x, ldx, bsx, ncols, X, ldo, bso,
                                                                    pair_table(tw, g.L), xptr);
        count_launch();
        *err = cudaGetLastError();
    });
}

bool exchange_irfft(const float2* X, int64_t ldx, int64_t bsx, int ncols, float* y, int64_t ldy, int64_t bsy,
                    const float* gam, int nb, const FftGeom& g, const float2* tw, cudaStream_t st, float* const* yptr,
                    cudaError_t* err)
{
    return for_len<F_INV32>(g.L, [&](auto geo) {
        using G = decltype(geo);
        k_irfft_x<G, float2><<<grid_x<G>(ncols, nb), G::NTX, G::smem, st>>>(X, ldx, bsx, ncols, y, ldy, bsy, gam,
                                                                           pair_table(tw, g.L), tw, yptr);
        count_launch();
        *err = cudaGetLastError();
    });
}

bool exchange_irfft_bf16(const __nv_bfloat162* X, int64_t ldx, int64_t bsx, int ncols, float* y, int64_t ldy,
                         int64_t bsy, int nb, const FftGeom& g, const float2* tw, cudaStream_t st, float* const* yptr,
                         cudaError_t* err)
{
    return for_len<F_INV16>(g.L, [&](auto geo) {
        using G = decltype(geo);
        k_irfft_x<G, __nv_bfloat162><<<grid_x<G>(ncols, nb), G::NTX, G::smem, st>>>(
            X, ldx, bsx, ncols, y, ldy, bsy, nullptr, pair_table(tw, g.L), tw, yptr);
        count_launch();
        *err = cudaGetLastError();
    });
}

}  // namespace btt

#ifdef BTT_CHECK
namespace btt {
BTT_CHECK_TU(check_record_fft_exchange)
}  // namespace btt
#endif
