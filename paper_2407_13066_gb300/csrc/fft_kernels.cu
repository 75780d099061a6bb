// Time-axis transforms: pad + real DFT of vectors, inverse DFT + unpad
// (+ noise-precision scaling), the fused middle step of the Hessian, and the
// FP64 setup transform of the blocks (Alg. 1).  See fft.cuh for the
// shared-memory transform they all use.
#include <type_traits>

#include "fft.cuh"
#include "kernels.h"

namespace btt {

bool make_fft_geom(int N_t, FftGeom* g)
{
    if (N_t < 1) return false;
    const int L = 2 * N_t;
    if (L > kFftMaxL) return false;
    FftPlan p{};
    p.L = L;
    int n = L, k = 0;
    while (n % 8 == 0 && k < kMaxStages) { p.radix[k++] = 8; n /= 8; }
    while (n % 4 == 0 && k < kMaxStages) { p.radix[k++] = 4; n /= 4; }
    while (n % 2 == 0 && k < kMaxStages) { p.radix[k++] = 2; n /= 2; }
    for (int r : {3, 5, 7})
        while (n % r == 0 && k < kMaxStages) { p.radix[k++] = r; n /= r; }
    if (n != 1) return false;
    p.nstages = k;
    int wc_log2 = 0;
    while (wc_log2 < 4 && (L << (wc_log2 + 1)) <= kFftCap) ++wc_log2;
    g->N_t = N_t;
    g->L = L;
    g->wc_log2 = wc_log2;
    g->plan = p;
    g->pos = nullptr;
    return true;
}

void digit_reversal(const FftGeom& g, int* pos)
{
    // forward pass p leaves output digit k_p (radix R_p, least significant
    // first) at offset k_p * L / (R_0 ... R_p)
    const int L = g.L;
    for (int k = 0; k < L; ++k) {
        int rem = k, prod = 1, at = 0;
        for (int p = 0; p < g.plan.nstages; ++p) {
            const int R = g.plan.radix[p];
            const int d = rem % R;
            rem /= R;
            prod *= R;
            at += d * (L / prod);
        }
        pos[k] = at;
    }
}

// ---------------------------------------------------------------- kernels
template <typename T>
__global__ void __launch_bounds__(kFftThreads)
k_rfft(const T* __restrict__ x, int64_t ldx, int64_t bsx, int ncols, cplx_t<T>* __restrict__ X,
       int64_t ldo, int64_t bso, int N_t, FftPlan plan, int wc_log2,
       const cplx_t<T>* __restrict__ tw, const int* __restrict__ pos, const T* const* __restrict__ xptr)
{
    using V = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* buf = reinterpret_cast<V*>(smem_raw);
    const int L = plan.L;
    const int W = 2 << wc_log2;
    const int col0 = blockIdx.x * W;
    const int64_t b = blockIdx.y;
    load_real_pairs<T, T, kFftThreads>(buf, xptr ? xptr[b] : x + b * bsx, ldx, N_t, L, col0, ncols, wc_log2);
    __syncthreads();
    fft_forward<T, kFftThreads>(buf, plan, wc_log2, tw);
    V* Xb = X + b * bso;
    const int wl = wc_log2 + 1;
    for (int idx = threadIdx.x; idx < ((N_t + 1) << wl); idx += kFftThreads) {
        const int w = idx >> wl, c = idx & (W - 1);
        const int col = col0 + c;
        if (col < ncols) Xb[(int64_t)w * ldo + col] = unpack_pair(buf, pos, L, w, c, wc_log2);
    }
}

template <typename T, typename TX = cplx_t<T>>
__global__ void __launch_bounds__(kFftThreads)
k_irfft(const TX* __restrict__ X, int64_t ldx, int64_t bsx, int ncols, T* __restrict__ y,
        int64_t ldy, int64_t bsy, const T* __restrict__ g, int N_t, FftPlan plan, int wc_log2,
        const cplx_t<T>* __restrict__ tw, const int* __restrict__ pos, T* const* __restrict__ yptr)
{
    using V = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* buf = reinterpret_cast<V*>(smem_raw);
    const int L = plan.L;
    const int W = 2 << wc_log2;
    const int col0 = blockIdx.x * W;
    const int64_t b = blockIdx.y;
    load_hermitian_pairs<V, kFftThreads, TX>(buf, pos, X + b * bsx, ldx, N_t, L, col0, ncols, wc_log2);
    __syncthreads();
    fft_inverse<T, kFftThreads>(buf, plan, wc_log2, tw);
    const T inv = (T)1 / (T)L;
    const T* fb = reinterpret_cast<const T*>(buf);
    T* yb = yptr ? yptr[b] : y + b * bsy;
    const int wl = wc_log2 + 1;
    for (int idx = threadIdx.x; idx < (N_t << wl); idx += kFftThreads) {
        const int t = idx >> wl, c = idx & (W - 1);
        const int col = col0 + c;
        if (col < ncols) {
            T v = fb[idx] * inv;
            if (g) v *= g[(int64_t)t * ncols + col];
            yb[(int64_t)t * ldy + col] = v;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kFftThreads)
k_hess_mid(cplx_t<T>* X, int64_t ldx, int64_t bsx, int ncols, const T* __restrict__ g, int N_t,
           FftPlan plan, int wc_log2, const cplx_t<T>* __restrict__ tw,
           const int* __restrict__ pos, double* __restrict__ part)
{
    using V = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* buf = reinterpret_cast<V*>(smem_raw);
    const int L = plan.L;
    const int W = 2 << wc_log2;
    const int col0 = blockIdx.x * W;
    const int64_t b = blockIdx.y;
    V* Xb = X + b * bsx;
    load_hermitian_pairs<V, kFftThreads>(buf, pos, Xb, ldx, N_t, L, col0, ncols, wc_log2);
    __syncthreads();
    fft_inverse<T, kFftThreads>(buf, plan, wc_log2, tw);
    // time domain: keep t < N_t (the unpad of Alg. 2), scale by 1/L and by the
    // noise precision of each real column, zero the padding (Alg. 3's pad)
    const T inv = (T)1 / (T)L;
    T* fb = reinterpret_cast<T*>(buf);
    const int wl = wc_log2 + 1;
    T q = (T)0;   // this thread's share of sum g (F m)^2 (part != nullptr)
    for (int idx = threadIdx.x; idx < (L << wl); idx += kFftThreads) {
        const int t = idx >> wl, c = idx & (W - 1);
        const int col = col0 + c;
        T v = (T)0;
        if (t < N_t && col < ncols) {
            const T u = fb[idx] * inv;
            v = u;
            if (g) v *= g[(int64_t)t * ncols + col];
            q += u * v;
        }
        fb[idx] = v;
    }
    __syncthreads();
    // FP32 only (the CG solver's operators): the FP64 form may claim all the
    // shared memory a CTA has for its buffer, leaving none for the reduction
    if constexpr (std::is_same<T, float>::value)
        if (part) block_sum_store<kFftThreads>((double)q, part + b * gridDim.x + blockIdx.x);
    fft_forward<T, kFftThreads>(buf, plan, wc_log2, tw);
    for (int idx = threadIdx.x; idx < ((N_t + 1) << wl); idx += kFftThreads) {
        const int w = idx >> wl, c = idx & (W - 1);
        const int col = col0 + c;
        if (col < ncols) Xb[(int64_t)w * ldx + col] = unpack_pair(buf, pos, L, w, c, wc_log2);
    }
}

// Real DFT of vectors written as the BF16 A operand of the tensor-core
// products (tc_gemm.cu): for vector b of the batch and frequency w, row
// (w*mt_stride + b/64)*64 + b%64 gets conj(X) = (Re, -Im) as ldm BF16 pairs
// (column l); the GEMM derives the (Im, Re) rows in shared memory.
__global__ void __launch_bounds__(kFftThreads)
k_rfft_stack(const float* __restrict__ x, int64_t ldx, int64_t bsx, int ncols,
             __nv_bfloat162* __restrict__ XA, int ldm, int mt_stride, int N_t, FftPlan plan, int wc_log2,
             const float2* __restrict__ tw, const int* __restrict__ pos, const float* const* __restrict__ xptr,
             int64_t lo_off)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* buf = reinterpret_cast<float2*>(smem_raw);
    const int L = plan.L;
    const int W = 2 << wc_log2;
    const int col0 = blockIdx.x * W;
    const int b = blockIdx.y;
    load_real_pairs<float, float, kFftThreads>(buf, xptr ? xptr[b] : x + (int64_t)b * bsx, ldx, N_t, L, col0,
                                               ncols, wc_log2);
    __syncthreads();
    fft_forward<float, kFftThreads>(buf, plan, wc_log2, tw);
    const int mt = b >> 6, j = b & 63;
    const int wl = wc_log2 + 1;
    for (int idx = threadIdx.x; idx < ((N_t + 1) << wl); idx += kFftThreads) {
        const int w = idx >> wl, c = idx & (W - 1);
        const int col = col0 + c;
        if (col < ncols) {
            const float2 X = unpack_pair(buf, pos, L, w, c, wc_log2);
            const int64_t row = ((int64_t)w * mt_stride + mt) * 64 + j;
            const __nv_bfloat162 hi = __floats2bfloat162_rn(X.x, -X.y);
            XA[row * ldm + col] = hi;
            if (lo_off) {
                const float2 h = __bfloat1622float2(hi);
                XA[lo_off + row * ldm + col] = __floats2bfloat162_rn(X.x - h.x, -X.y - h.y);
            }
        }
    }
}

// Setup transform (Alg. 1): FP64 FFT of block columns, stored frequency-major
// in the storage format.  Persistent over column tiles.
template <int PREC>
__global__ void __launch_bounds__(kFftThreads)
k_create(const double* __restrict__ blk, int64_t ldb, int ncols, int64_t col_base, int N_t,
         int N_d, int N_m, int ldm, FftPlan plan, int wc_log2, const double2* __restrict__ tw,
         const int* __restrict__ pos, void* __restrict__ fhat, const float* __restrict__ scales,
         unsigned long long* __restrict__ maxbits, int pass, double2* __restrict__ gscratch)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int L = plan.L;
    const int W = 2 << wc_log2;
    const int wl = wc_log2 + 1;
    // transform buffer in shared memory, or this CTA's slice of the global
    // scratch when it does not fit (the per-frequency maxima stay shared)
    double2* buf = gscratch ? gscratch + (size_t)blockIdx.x * (L << wc_log2) : reinterpret_cast<double2*>(smem_raw);
    unsigned long long* smax = gscratch ? reinterpret_cast<unsigned long long*>(smem_raw)
                                        : reinterpret_cast<unsigned long long*>(buf + (L << wc_log2));
    const bool find_max = (PREC == P_F16S || PREC == P_FP8S) && pass == 0;
    if (find_max)
        for (int i = threadIdx.x; i <= N_t; i += kFftThreads) smax[i] = 0ull;
    const int ntiles = (ncols + W - 1) / W;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        __syncthreads();
        load_real_pairs<double, double, kFftThreads>(buf, blk, ldb, N_t, L, tile * W, ncols, wc_log2);
        __syncthreads();
        fft_forward<double, kFftThreads>(buf, plan, wc_log2, tw);
        for (int idx = threadIdx.x; idx < ((N_t + 1) << wl); idx += kFftThreads) {
            const int w = idx >> wl, c = idx & (W - 1);
            const int col = tile * W + c;
            if (col >= ncols) continue;
            const double2 z = unpack_pair(buf, pos, L, w, c, wc_log2);
            const int64_t gcol = col_base + col;
            const int64_t s = gcol / N_m;
            const int64_t l = gcol - s * N_m;
            const int64_t o = ((int64_t)w * N_d + s) * ldm + l;
            if constexpr (PREC == P_F64) {
                reinterpret_cast<double2*>(fhat)[o] = z;
            } else if constexpr (PREC == P_F32) {
                reinterpret_cast<float2*>(fhat)[o] = make_float2((float)z.x, (float)z.y);
            } else if constexpr (PREC == P_BF16) {
                __nv_bfloat162 v;
                v.x = __float2bfloat16_rn((float)z.x);
                v.y = __float2bfloat16_rn((float)z.y);
                reinterpret_cast<__nv_bfloat162*>(fhat)[o] = v;
            } else if constexpr (PREC == P_BF16X2) {
                // two planes: hi = bf16(fp32(z)), lo = bf16(fp32(z - hi))
                __nv_bfloat162 hi, lo;
                hi.x = __float2bfloat16_rn((float)z.x);
                hi.y = __float2bfloat16_rn((float)z.y);
                lo.x = __float2bfloat16_rn((float)(z.x - (double)__bfloat162float(hi.x)));
                lo.y = __float2bfloat16_rn((float)(z.y - (double)__bfloat162float(hi.y)));
                __nv_bfloat162* f2 = reinterpret_cast<__nv_bfloat162*>(fhat);
                f2[o] = hi;
                f2[o + (int64_t)(N_t + 1) * N_d * ldm] = lo;
            } else if (find_max) {  // P_F16S / P_FP8S, pass 0
                const double a = fmax(fabs(z.x), fabs(z.y));
                atomicMax(&smax[w], (unsigned long long)__double_as_longlong(a));
            } else if constexpr (PREC == P_F16S) {
                const double s_w = (double)scales[w];
                __half2 v;
                v.x = __float2half_rn((float)(z.x / s_w));
                v.y = __float2half_rn((float)(z.y / s_w));
                reinterpret_cast<__half2*>(fhat)[o] = v;
            } else {  // P_FP8S: E4M3, round to nearest even, saturating
                const double s_w = (double)scales[w];
                const float2 q = make_float2((float)(z.x / s_w), (float)(z.y / s_w));
                reinterpret_cast<__nv_fp8x2_storage_t*>(fhat)[o] = __nv_cvt_float2_to_fp8x2(q, __NV_SATFINITE, __NV_E4M3);
            }
        }
    }
    if (find_max) {
        __syncthreads();
        for (int i = threadIdx.x; i <= N_t; i += kFftThreads)
            if (smax[i]) atomicMax(&maxbits[i], smax[i]);
    }
}

__global__ void k_make_scales(const unsigned long long* __restrict__ maxbits, float* scales, int n, double target)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const double mx = __longlong_as_double((long long)maxbits[i]);
        scales[i] = mx > 0.0 ? (float)(mx / target) : 1.0f;
    }
}

// ---------------------------------------------------------------- launchers
template <typename T> static size_t fft_smem(const FftGeom& g)
{
    return (size_t)(g.L << g.wc_log2) * sizeof(cplx_t<T>);
}

static size_t create_smem(const FftGeom& g)
{
    return fft_smem<double>(g) + (size_t)(g.N_t + 1) * sizeof(unsigned long long);
}

static int create_grid(int ntiles)
{
    int dev = 0, nsm = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    return ntiles < nsm * 2 ? ntiles : nsm * 2;
}

size_t create_scratch_bytes(const FftGeom& g)
{
    if (create_smem(g) <= (size_t)kFftSmemMax) return 0;
    return (size_t)create_grid(0x7fffffff) * (size_t)(g.L << g.wc_log2) * sizeof(double2);
}

bool runtime_fits(const FftGeom& g, bool fp64)
{
    return (fp64 ? fft_smem<double>(g) : fft_smem<float>(g)) <= (size_t)kFftSmemMax;
}

static dim3 col_grid(int ncols, int nb, const FftGeom& g)
{
    const int W = 2 << g.wc_log2;
    return dim3((unsigned)((ncols + W - 1) / W), (unsigned)nb, 1);
}

cudaError_t prepare_kernels()
{
    // limits clamped to what this device lets one CTA claim
    int dev = 0, optin = kFftSmemMax;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const int cap = optin < kFftSmemMax ? optin : kFftSmemMax;
    const int fmax_f = kFftMaxL * (int)sizeof(float2) < cap ? kFftMaxL * (int)sizeof(float2) : cap;
    const int fmax_d = cap;
    const int cmax = cap;
    cudaError_t e = cudaSuccess;
#define BTT_SET(k, b) \
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, b)
    BTT_SET(k_rfft<float>, fmax_f);
    BTT_SET(k_rfft<double>, fmax_d);
    BTT_SET(k_irfft<float>, fmax_f);
    BTT_SET((k_irfft<float, __nv_bfloat162>), fmax_f);
    BTT_SET(k_irfft<double>, fmax_d);
    BTT_SET(k_hess_mid<float>, fmax_f);
    BTT_SET(k_hess_mid<double>, fmax_d);
    BTT_SET(k_rfft_stack, fmax_f);
    BTT_SET(k_create<P_F32>, cmax);
    BTT_SET(k_create<P_F64>, cmax);
    BTT_SET(k_create<P_F16S>, cmax);
    BTT_SET(k_create<P_BF16>, cmax);
    BTT_SET(k_create<P_BF16X2>, cmax);
    BTT_SET(k_create<P_FP8S>, cmax);
#undef BTT_SET
    if (e == cudaSuccess) e = prepare_static_fft();
    if (e == cudaSuccess) e = prepare_exchange_fft();
    return e;
}

template <typename T>
cudaError_t launch_rfft(const T* x, int64_t ldx, int64_t bsx, int ncols, cplx_t<T>* X,
                        int64_t ldo, int64_t bso, int nb, const FftGeom& g, const cplx_t<T>* tw,
                        cudaStream_t st, const T* const* xptr)
{
    if (nb <= 0 || ncols <= 0) return cudaSuccess;
    if constexpr (std::is_same<T, float>::value) {
        cudaError_t e;
        if (exchange_rfft(x, ldx, bsx, ncols, X, ldo, bso, nb, g, tw, st, xptr, &e)) return e;
        if (static_rfft(x, ldx, bsx, ncols, X, ldo, bso, nb, g, tw, st, xptr, &e)) return e;
    }
    k_rfft<T><<<col_grid(ncols, nb, g), kFftThreads, fft_smem<T>(g), st>>>(
        x, ldx, bsx, ncols, X, ldo, bso, g.N_t, g.plan, g.wc_log2, tw, g.pos, xptr);
    count_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_irfft(const cplx_t<T>* X, int64_t ldx, int64_t bsx, int ncols, T* y,
                         int64_t ldy, int64_t bsy, const T* gam, int nb, const FftGeom& g,
                         const cplx_t<T>* tw, cudaStream_t st, T* const* yptr)
{
    if (nb <= 0 || ncols <= 0) return cudaSuccess;
    if constexpr (std::is_same<T, float>::value) {
        cudaError_t e;
        if (exchange_irfft(X, ldx, bsx, ncols, y, ldy, bsy, gam, nb, g, tw, st, yptr, &e)) return e;
        if (static_irfft(X, ldx, bsx, ncols, y, ldy, bsy, gam, nb, g, tw, st, yptr, &e)) return e;
    }
    k_irfft<T><<<col_grid(ncols, nb, g), kFftThreads, fft_smem<T>(g), st>>>(
        X, ldx, bsx, ncols, y, ldy, bsy, gam, g.N_t, g.plan, g.wc_log2, tw, g.pos, yptr);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_irfft_bf16(const __nv_bfloat162* X, int64_t ldx, int64_t bsx, int ncols, float* y,
                              int64_t ldy, int64_t bsy, int nb, const FftGeom& g, const float2* tw,
                              cudaStream_t st, float* const* yptr)
{
    if (nb <= 0 || ncols <= 0) return cudaSuccess;
    cudaError_t e;
    if (exchange_irfft_bf16(X, ldx, bsx, ncols, y, ldy, bsy, nb, g, tw, st, yptr, &e)) return e;
    if (static_irfft_bf16(X, ldx, bsx, ncols, y, ldy, bsy, nb, g, tw, st, yptr, &e)) return e;
    k_irfft<float, __nv_bfloat162><<<col_grid(ncols, nb, g), kFftThreads, fft_smem<float>(g), st>>>(
        X, ldx, bsx, ncols, y, ldy, bsy, nullptr, g.N_t, g.plan, g.wc_log2, tw, g.pos, yptr);
    count_launch();
    return cudaGetLastError();
}

int fft_col_blocks(int ncols, const FftGeom& g) { return (int)col_grid(ncols, 1, g).x; }

template <typename T>
cudaError_t launch_hess_mid(cplx_t<T>* X, int64_t ldx, int64_t bsx, int ncols, const T* gam,
                            int nb, const FftGeom& g, const cplx_t<T>* tw, cudaStream_t st, double* part)
{
    if (nb <= 0 || ncols <= 0) return cudaSuccess;
    if constexpr (std::is_same<T, float>::value) {
        cudaError_t e;
        if (static_hess_mid(X, ldx, bsx, ncols, gam, nb, g, tw, st, part, &e)) return e;
    }
    k_hess_mid<T><<<col_grid(ncols, nb, g), kFftThreads, fft_smem<T>(g), st>>>(
        X, ldx, bsx, ncols, gam, g.N_t, g.plan, g.wc_log2, tw, g.pos, part);
    count_launch();
    return cudaGetLastError();
}

template cudaError_t launch_rfft<float>(const float*, int64_t, int64_t, int, float2*, int64_t,
                                        int64_t, int, const FftGeom&, const float2*, cudaStream_t,
                                        const float* const*);
template cudaError_t launch_rfft<double>(const double*, int64_t, int64_t, int, double2*, int64_t,
                                         int64_t, int, const FftGeom&, const double2*, cudaStream_t,
                                         const double* const*);
template cudaError_t launch_irfft<float>(const float2*, int64_t, int64_t, int, float*, int64_t,
                                         int64_t, const float*, int, const FftGeom&, const float2*,
                                         cudaStream_t, float* const*);
template cudaError_t launch_irfft<double>(const double2*, int64_t, int64_t, int, double*, int64_t,
                                          int64_t, const double*, int, const FftGeom&,
                                          const double2*, cudaStream_t, double* const*);
template cudaError_t launch_hess_mid<float>(float2*, int64_t, int64_t, int, const float*, int,
                                            const FftGeom&, const float2*, cudaStream_t, double*);
template cudaError_t launch_hess_mid<double>(double2*, int64_t, int64_t, int, const double*, int,
                                             const FftGeom&, const double2*, cudaStream_t, double*);

cudaError_t launch_rfft_stack(const float* x, int64_t ldx, int64_t bsx, int ncols, void* xstack, int ldm,
                              int mt_stride, int nb, const FftGeom& g, const float2* tw, cudaStream_t st,
                              int64_t lo_off, const float* const* xptr)
{
    if (nb <= 0 || ncols <= 0) return cudaSuccess;
    {
        cudaError_t e;
        if (exchange_rfft_stack(x, ldx, bsx, ncols, xstack, ldm, mt_stride, nb, g, tw, st, lo_off, xptr, &e))
            return e;
        if (static_rfft_stack(x, ldx, bsx, ncols, xstack, ldm, mt_stride, nb, g, tw, st, lo_off, xptr, &e)) return e;
    }
    k_rfft_stack<<<col_grid(ncols, nb, g), kFftThreads, fft_smem<float>(g), st>>>(
        x, ldx, bsx, ncols, static_cast<__nv_bfloat162*>(xstack), ldm, mt_stride, g.N_t, g.plan, g.wc_log2, tw,
        g.pos, xptr, lo_off);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_create(const double* blk, int64_t ldb, int ncols, int64_t col_base, int N_d,
                          int N_m, int ldm, int prec, void* fhat, const float* scales,
                          unsigned long long* maxbits, int pass, const FftGeom& g,
                          const double2* tw, double2* scratch, cudaStream_t st)
{
    if (ncols <= 0) return cudaSuccess;
    const int W = 2 << g.wc_log2;
    const int ntiles = (ncols + W - 1) / W;
    const int grid = create_grid(ntiles);
    const bool global = create_smem(g) > (size_t)kFftSmemMax;
    if (global && !scratch) return cudaErrorInvalidValue;
    const size_t sm = global ? (size_t)(g.N_t + 1) * sizeof(unsigned long long) : create_smem(g);
    double2* gs = global ? scratch : nullptr;
#define BTT_CREATE(P)                                                                          \
    k_create<P><<<grid, kFftThreads, sm, st>>>(blk, ldb, ncols, col_base, g.N_t, N_d, N_m, ldm, \
                                               g.plan, g.wc_log2, tw, g.pos, fhat, scales, maxbits, pass, gs)
    switch (prec) {
        case P_F32: BTT_CREATE(P_F32); break;
        case P_F64: BTT_CREATE(P_F64); break;
        case P_F16S: BTT_CREATE(P_F16S); break;
        case P_BF16: BTT_CREATE(P_BF16); break;
        case P_BF16X2: BTT_CREATE(P_BF16X2); break;
        case P_FP8S: BTT_CREATE(P_FP8S); break;
        default: return cudaErrorInvalidValue;
    }
#undef BTT_CREATE
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_make_scales(const unsigned long long* maxbits, float* scales, int n, double target,
                               cudaStream_t st)
{
    k_make_scales<<<(n + 255) / 256, 256, 0, st>>>(maxbits, scales, n, target);
    count_launch();
    return cudaGetLastError();
}

}  // namespace btt
