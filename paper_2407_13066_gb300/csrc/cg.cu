// Vector kernels of the conjugate-gradient solver on the regularised
// Gauss-Newton Hessian (Sec. 2.2: the Hessian action exists to be applied
// repeatedly inside CG).  Each right-hand side is an independent CG run;
// all of them advance together so that every iteration is one batched
// Hessian call.  The scalars of the method (step length, direction weight,
// relative residual, convergence) live on the device in one CgVec per
// right-hand side, computed by the finishing reductions, so iterations run
// without host synchronisation.  An iteration is: Hp = H p, whose middle
// step leaves the partials of p.Hp (the Gamma^-1-weighted squared norm of
// F p, in data space); alpha = r.r / (p.Hp + shift p.p); the step
// x += alpha p, r -= alpha (Hp + shift p) with the partials of r.r -- inside
// the Hessian's last inverse transform for fixed-plan lengths (Hp is never
// stored), else k_step; k_direction (p = r + beta p, p.p).
//
// Dot products: each thread sums groups of 32 consecutive terms of its
// stride in FP32 and adds the group sums into an FP64 accumulator; blocks
// then combine in FP64 in a fixed order (one partial per block, then one
// block per vector), so results are identical run to run.  FP64 arithmetic
// is far slower than FP32 on this GPU (two conversions and an FP64 FMA per
// term made these kernels compute bound); with one FP64 add per 32 terms
// they stream at memory speed.  A group's FP32 rounding error is at most
// about 32 units in the last place of its terms' magnitudes, far below
// what CG's recursively updated residual tolerates.
//
// Vectors are read as float4 when their length is a multiple of 4 and every
// array is 16-byte aligned, else one float at a time.
#include "kernels.h"

namespace btt {
namespace {

constexpr int kCgThreads = 256;
constexpr int kGroup = 8;          // float4 per FP32 group (32 terms)
constexpr int kCgTarget = 8 * 152; // resident blocks of 256 threads over 152 SMs

__device__ __forceinline__ double block_sum(double v)
{
    __shared__ double red[kCgThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < kCgThreads / 32; ++i) s += red[i];
    return s;   // valid in thread 0
}

__device__ __forceinline__ bool al16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

__device__ __forceinline__ float dot4(float4 a, float4 b)
{
    return fmaf(a.w, b.w, fmaf(a.z, b.z, fmaf(a.y, b.y, a.x * b.x)));
}

// Runs body over this thread's share of vector blockIdx.y (float4 units
// i when vec, else floats i) and returns the thread's FP64 sum of what body
// returns, grouped as described above.
template <typename Body4, typename Body1>
__device__ __forceinline__ double sweep(int64_t n, bool vec, Body4 body4, Body1 body1)
{
    const int64_t T = (int64_t)gridDim.x * kCgThreads;
    int64_t i = (int64_t)blockIdx.x * kCgThreads + threadIdx.x;
    double s = 0.0;
    if (vec) {
        const int64_t n4 = n >> 2;
        while (i < n4) {
            float g = 0.f;
#pragma unroll
            for (int k = 0; k < kGroup; ++k, i += T)
                if (i < n4) g += body4(i);
            s += (double)g;
        }
    } else {
        while (i < n) {
            float g = 0.f;
#pragma unroll
            for (int k = 0; k < 4 * kGroup; ++k, i += T)
                if (i < n) g += body1(i);
            s += (double)g;
        }
    }
    return s;
}

// part[j * nblk + blk] = partial sum over this block of a_j . b_j
__global__ void __launch_bounds__(kCgThreads)
k_dot(const float* __restrict__ a, const float* __restrict__ b, int64_t n, double* __restrict__ part)
{
    const int j = blockIdx.y, nblk = gridDim.x;
    const float* x = a + (int64_t)j * n;
    const float* y = b + (int64_t)j * n;
    const bool vec = (n & 3) == 0 && al16(a) && al16(b);
    const float4* x4 = reinterpret_cast<const float4*>(x);
    const float4* y4 = reinterpret_cast<const float4*>(y);
    double s = sweep(
        n, vec, [&](int64_t i) { return dot4(x4[i], y4[i]); }, [&](int64_t i) { return x[i] * y[i]; });
    s = block_sum(s);
    if (threadIdx.x == 0) part[(int64_t)j * nblk + blockIdx.x] = s;
}

// Ap_j += alpha p_j, and the partials of p_j . Ap_j
__global__ void __launch_bounds__(kCgThreads)
k_shift_dot(float* __restrict__ Ap, const float* __restrict__ p, float alpha, int64_t n, double* __restrict__ part)
{
    const int j = blockIdx.y, nblk = gridDim.x;
    float* q = Ap + (int64_t)j * n;
    const float* x = p + (int64_t)j * n;
    const bool vec = (n & 3) == 0 && al16(Ap) && al16(p);
    float4* q4 = reinterpret_cast<float4*>(q);
    const float4* x4 = reinterpret_cast<const float4*>(x);
    double s = sweep(
        n, vec,
        [&](int64_t i) {
            const float4 u = x4[i];
            float4 v = q4[i];
            v.x = fmaf(alpha, u.x, v.x);
            v.y = fmaf(alpha, u.y, v.y);
            v.z = fmaf(alpha, u.z, v.z);
            v.w = fmaf(alpha, u.w, v.w);
            q4[i] = v;
            return dot4(u, v);
        },
        [&](int64_t i) {
            const float v = fmaf(alpha, x[i], q[i]);
            q[i] = v;
            return x[i] * v;
        });
    s = block_sum(s);
    if (threadIdx.x == 0) part[(int64_t)j * nblk + blockIdx.x] = s;
}

// r_j = b_j - Ap_j (Ap_j already holds (H + alpha) x_j), p_j = r_j, partials of r_j . r_j
__global__ void __launch_bounds__(kCgThreads)
k_residual(const float* __restrict__ b, const float* __restrict__ Ap, float* __restrict__ r, float* __restrict__ p,
           int64_t n, double* __restrict__ part)
{
    const int j = blockIdx.y, nblk = gridDim.x;
    const int64_t o = (int64_t)j * n;
    const bool vec = (n & 3) == 0 && al16(b) && al16(Ap) && al16(r) && al16(p);
    const float4* b4 = reinterpret_cast<const float4*>(b + o);
    const float4* q4 = reinterpret_cast<const float4*>(Ap + o);
    float4* r4 = reinterpret_cast<float4*>(r + o);
    float4* p4 = reinterpret_cast<float4*>(p + o);
    double s = sweep(
        n, vec,
        [&](int64_t i) {
            const float4 u = b4[i], q = q4[i];
            const float4 v = make_float4(u.x - q.x, u.y - q.y, u.z - q.z, u.w - q.w);
            r4[i] = v;
            p4[i] = v;
            return dot4(v, v);
        },
        [&](int64_t i) {
            const float v = b[o + i] - Ap[o + i];
            r[o + i] = v;
            p[o + i] = v;
            return v * v;
        });
    s = block_sum(s);
    if (threadIdx.x == 0) part[(int64_t)j * nblk + blockIdx.x] = s;
}

// x_j += a_j p_j, r_j -= a_j (Hp_j + shift p_j) (Hp holds H p, without the
// shift), partials of r_j . r_j
__global__ void __launch_bounds__(kCgThreads)
k_step(float* __restrict__ x, float* __restrict__ r, const float* __restrict__ p, const float* __restrict__ Ap,
       const CgVec* __restrict__ cv, float shift, int64_t n, double* __restrict__ part)
{
    const int j = blockIdx.y, nblk = gridDim.x;
    const int64_t o = (int64_t)j * n;
    const float aj = cv[j].alpha;
    const bool vec = (n & 3) == 0 && al16(x) && al16(r) && al16(p) && al16(Ap);
    float4* x4 = reinterpret_cast<float4*>(x + o);
    float4* r4 = reinterpret_cast<float4*>(r + o);
    const float4* p4 = reinterpret_cast<const float4*>(p + o);
    const float4* q4 = reinterpret_cast<const float4*>(Ap + o);
    double s = sweep(
        n, vec,
        [&](int64_t i) {
            const float4 pp = p4[i], q = q4[i];
            float4 xx = x4[i], v = r4[i];
            xx.x = fmaf(aj, pp.x, xx.x);
            xx.y = fmaf(aj, pp.y, xx.y);
            xx.z = fmaf(aj, pp.z, xx.z);
            xx.w = fmaf(aj, pp.w, xx.w);
            v.x = fmaf(-aj, fmaf(shift, pp.x, q.x), v.x);
            v.y = fmaf(-aj, fmaf(shift, pp.y, q.y), v.y);
            v.z = fmaf(-aj, fmaf(shift, pp.z, q.z), v.z);
            v.w = fmaf(-aj, fmaf(shift, pp.w, q.w), v.w);
            x4[i] = xx;
            r4[i] = v;
            return dot4(v, v);
        },
        [&](int64_t i) {
            const float pp = p[o + i];
            x[o + i] = fmaf(aj, pp, x[o + i]);
            const float v = fmaf(-aj, fmaf(shift, pp, Ap[o + i]), r[o + i]);
            r[o + i] = v;
            return v * v;
        });
    s = block_sum(s);
    if (threadIdx.x == 0) part[(int64_t)j * nblk + blockIdx.x] = s;
}

// p_j = r_j + beta_j p_j, partials of p_j . p_j
__global__ void __launch_bounds__(kCgThreads)
k_direction(float* __restrict__ p, const float* __restrict__ r, const CgVec* __restrict__ cv, int64_t n,
            double* __restrict__ part)
{
    const int j = blockIdx.y, nblk = gridDim.x;
    const int64_t o = (int64_t)j * n;
    const float bj = cv[j].beta;
    const bool vec = (n & 3) == 0 && al16(p) && al16(r);
    float4* p4 = reinterpret_cast<float4*>(p + o);
    const float4* r4 = reinterpret_cast<const float4*>(r + o);
    double s = sweep(
        n, vec,
        [&](int64_t i) {
            const float4 u = r4[i];
            float4 v = p4[i];
            v.x = fmaf(bj, v.x, u.x);
            v.y = fmaf(bj, v.y, u.y);
            v.z = fmaf(bj, v.z, u.z);
            v.w = fmaf(bj, v.w, u.w);
            p4[i] = v;
            return dot4(v, v);
        },
        [&](int64_t i) {
            const float v = fmaf(bj, p[o + i], r[o + i]);
            p[o + i] = v;
            return v * v;
        });
    s = block_sum(s);
    if (threadIdx.x == 0) part[(int64_t)j * nblk + blockIdx.x] = s;
}

// Sums the nblk partials of vector j in order, then updates its scalars:
//   FIN_BB     bb = b.b
//   FIN_RS     rs = r.r of the initial residual (= p.p, as p = r); relative
//              residual; active
//   FIN_ALPHA  the sum is p.Hp: step length alpha = rs / (p.Hp + shift p.p)
//              (0 once converged)
//   FIN_BETA   new r.r: iteration count, relative residual, convergence,
//              direction weight beta = r.r / rs (0 once converged), rs = r.r
//   FIN_PP     pp = p.p of the new direction
__global__ void k_finish(const double* __restrict__ part, int nblk, int fin, int it, double tol, float shift,
                         CgVec* __restrict__ cv)
{
    const int j = blockIdx.x;
    double s = 0.0;
    for (int i = threadIdx.x; i < nblk; i += kCgThreads) s += part[(int64_t)j * nblk + i];
    s = block_sum(s);
    if (threadIdx.x != 0) return;
    CgVec v = cv[j];
    if (fin == FIN_BB) {
        v.bb = s;
    } else if (fin == FIN_RS) {
        v.rs = s;
        v.pp = s;
        v.rel = v.bb > 0.0 ? (float)sqrt(s / v.bb) : 0.f;
        v.active = v.rel > tol ? 1 : 0;
        v.iters = 0;
        v.alpha = 0.f;
        v.beta = 0.f;
    } else if (fin == FIN_ALPHA) {
        const double pap = s + (double)shift * v.pp;
        v.alpha = (v.active && pap > 0.0) ? (float)(v.rs / pap) : 0.f;
    } else if (fin == FIN_PP) {
        v.pp = s;
    } else if (fin == FIN_BETA) {
        if (v.active) {
            v.iters = it;
            v.rel = v.bb > 0.0 ? (float)sqrt(s / v.bb) : 0.f;
            v.beta = v.rs > 0.0 ? (float)(s / v.rs) : 0.f;
            v.rs = s;
            if (!(v.rel > tol)) {
                v.active = 0;
                v.beta = 0.f;
            }
        } else {
            v.beta = 0.f;
        }
    }
    cv[j] = v;
}

}  // namespace

int cg_blocks(int nrhs)
{
    // about kCgTarget blocks in all: enough resident warps to stream memory
    return nrhs >= kCgTarget ? 1 : (kCgTarget + nrhs - 1) / nrhs;
}

size_t cg_partials(int nrhs) { return (size_t)kCgTarget + (size_t)nrhs; }

cudaError_t launch_cg(int kind, int fin, int it, double tol, int nrhs, int64_t n, float* x, float* r, float* p,
                      float* Ap, const float* b, float alpha, double* part, CgVec* cv, cudaStream_t st)
{
    const int nblk = cg_blocks(nrhs);
    dim3 grid((unsigned)nblk, (unsigned)nrhs);
    switch (kind) {
        case CG_DOT_BB: k_dot<<<grid, kCgThreads, 0, st>>>(b, b, n, part); break;
        case CG_SHIFT_DOT: k_shift_dot<<<grid, kCgThreads, 0, st>>>(Ap, p, alpha, n, part); break;
        case CG_RESIDUAL: k_residual<<<grid, kCgThreads, 0, st>>>(b, Ap, r, p, n, part); break;
        case CG_STEP: k_step<<<grid, kCgThreads, 0, st>>>(x, r, p, Ap, cv, alpha, n, part); break;
        case CG_DIRECTION: k_direction<<<grid, kCgThreads, 0, st>>>(p, r, cv, n, part); break;
        default: return cudaErrorInvalidValue;
    }
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || fin == FIN_NONE) return e;
    k_finish<<<nrhs, kCgThreads, 0, st>>>(part, nblk, fin, it, tol, alpha, cv);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_cg_finish(const double* part, int nblk, int fin, int it, double tol, float shift, int nrhs,
                             CgVec* cv, cudaStream_t st)
{
    k_finish<<<nrhs, kCgThreads, 0, st>>>(part, nblk, fin, it, tol, shift, cv);
    count_launch();
    return cudaGetLastError();
}

}  // namespace btt
