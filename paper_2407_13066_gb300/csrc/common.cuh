// Shared device/host definitions of the GB300 block-Toeplitz library.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#define BTT_HD __host__ __device__ __forceinline__

namespace btt {

// ------------------------------------------------------------ complex math
template <typename T> struct cplx;
template <> struct cplx<float> { using type = float2; };
template <> struct cplx<double> { using type = double2; };
template <typename T> using cplx_t = typename cplx<T>::type;

template <typename V> BTT_HD V cmake(decltype(V::x) a, decltype(V::x) b) { V v; v.x = a; v.y = b; return v; }
template <typename V> BTT_HD V cadd(V a, V b) { return cmake<V>(a.x + b.x, a.y + b.y); }
template <typename V> BTT_HD V csub(V a, V b) { return cmake<V>(a.x - b.x, a.y - b.y); }
template <typename V> BTT_HD V cmul(V a, V b) { return cmake<V>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
template <typename V> BTT_HD V cscale(V a, decltype(V::x) s) { return cmake<V>(a.x * s, a.y * s); }

// ------------------------------------------------------------- FFT plan
// Mixed-radix Stockham plan for one transform length L (radices 8,4,2,3,5,7).
constexpr int kMaxStages = 24;
struct FftPlan {
    int L;
    int nstages;
    int radix[kMaxStages];
};

// FFT kernels batch columns into one CTA while the batch holds at most
// kFftCap complex values; longer transforms (up to kFftMaxL) run one column
// pair per CTA.  FP32 transforms always fit in shared memory (kFftMaxL * 8
// bytes); an FP64 buffer that exceeds kFftSmemMax (the 227 KB a CTA may
// claim) lives in a per-CTA global scratch slice instead (setup only).
constexpr int kFftCap = 8192;
constexpr int kFftMaxL = 24576;
constexpr int kFftSmemMax = 227 * 1024;
constexpr int kFftThreads = 512;

// ------------------------------------------------- bounds-check build
// Compiled with -DBTT_CHECK (build.build(check=True): libbtt_check.so), the
// kernels test the indices of their shared- and global-memory accesses
// against the extents they are derived from; an index outside its extent
// is recorded (the first one: site, index, extent) and the access is
// skipped, so nothing faults and the run continues.  btt_check_status
// reports and clears the record.  In the normal build BTT_IN(...) is the
// constant true and the checks compile away.
enum CheckSite {
    CK_SELFTEST = 1,
    CK_FFT_SMEM = 2,       // transform tile in shared memory
    CK_FFT_LOAD = 3,       // transform input row / column
    CK_FFT_STORE = 4,      // transform output row / column
    CK_FFT_TABLE = 5,      // twiddle / position table
    CK_FFT_REMOTE = 6,     // cluster transforms: another CTA's shared memory
    CK_GEMV_FHAT = 7,      // Fhat row / column of the per-frequency products
    CK_GEMV_VEC = 8,       // spectra read or written by the products
    CK_GEMV_SMEM = 9,      // spectra staged in shared memory
    CK_NSITES = 10
};

#ifdef BTT_CHECK
// one record per translation unit (device variables are per module)
static __device__ unsigned int g_chk_site;
static __device__ long long g_chk_index, g_chk_extent;
static __device__ __noinline__ void chk_fail(long long i, long long n, int site)
{
    if (atomicCAS(&g_chk_site, 0u, (unsigned)site) == 0u) {
        g_chk_index = i;
        g_chk_extent = n;
    }
}
__device__ __forceinline__ bool chk_in(long long i, long long n, int site)
{
    if ((unsigned long long)i < (unsigned long long)n) return true;
    chk_fail(i, n, site);
    return false;
}
#define BTT_IN(i, n, site) (::btt::chk_in((long long)(i), (long long)(n), (site)))
// Host side of a translation unit's record: reads (and with clear resets) it.
#define BTT_CHECK_TU(NAME)                                                                        \
    cudaError_t NAME(long long* rec, bool clear)                                                  \
    {                                                                                             \
        unsigned int s = 0;                                                                       \
        cudaError_t e = cudaMemcpyFromSymbol(&s, g_chk_site, sizeof s);                           \
        if (e == cudaSuccess) e = cudaMemcpyFromSymbol(&rec[1], g_chk_index, sizeof(long long));  \
        if (e == cudaSuccess) e = cudaMemcpyFromSymbol(&rec[2], g_chk_extent, sizeof(long long)); \
        rec[0] = s;                                                                               \
        if (e == cudaSuccess && clear && s) {                                                     \
            const unsigned int z = 0;                                                             \
            e = cudaMemcpyToSymbol(g_chk_site, &z, sizeof z);                                     \
        }                                                                                         \
        return e;                                                                                 \
    }
#else
#define BTT_IN(i, n, site) true
#endif

// ----------------------------------------------------- storage formats
enum Precision { P_F32 = 0, P_F16S = 1, P_BF16 = 2, P_BF16X2 = 3, P_F64 = 4, P_FP8S = 5 };

// scale targets: largest |Re|, |Im| of a frequency slice maps to this code value
constexpr double kF16ScaleTarget = 16384.0;   // FP16 max 65504
constexpr double kFp8ScaleTarget = 256.0;     // FP8 E4M3 max 448

}  // namespace btt
