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

// ----------------------------------------------------- storage formats
enum Precision { P_F32 = 0, P_F16S = 1, P_BF16 = 2, P_BF16X2 = 3, P_F64 = 4, P_FP8S = 5 };

// scale targets: largest |Re|, |Im| of a frequency slice maps to this code value
constexpr double kF16ScaleTarget = 16384.0;   // FP16 max 65504
constexpr double kFp8ScaleTarget = 256.0;     // FP8 E4M3 max 448

}  // namespace btt
