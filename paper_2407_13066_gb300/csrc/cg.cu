// Vector kernels of the conjugate-gradient solver on the regularised
// Gauss-Newton Hessian (Sec. 2.2: the Hessian action exists to be applied
// repeatedly inside CG).  Each right-hand side is an independent CG run;
// all of them advance together so that every iteration is one batched
// Hessian call.  Dot products accumulate in FP64 in a fixed order (one
// partial per block, then one block per vector), so results are identical
// run to run.  The scalars of the method (step length, direction weight,
// relative residual, convergence) live on the device in one CgVec per
// right-hand side, computed by the finishing reductions, so iterations run
// without host synchronisation.
#include "kernels.h"

namespace btt {
namespace {

constexpr int kCgThreads = 256;

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

// part[j * nblk + blk] = partial sum over this block of a_j . b_j
__global__ void __launch_bounds__(kCgThreads)
k_dot(const float* __restrict__ a, const float* __restrict__ b, int64_t n, double* __restrict__ part)
{
    const int j = blockIdx.y, nblk = gridDim.x;
    const float* x = a + (int64_t)j * n;
    const float* y = b + (int64_t)j * n;
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)kCgThreads + threadIdx.x; i < n; i += (int64_t)nblk * kCgThreads)
        s += (double)x[i] * (double)y[i];
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
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)kCgThreads + threadIdx.x; i < n; i += (int64_t)nblk * kCgThreads) {
        const float v = q[i] + alpha * x[i];
        q[i] = v;
        s += (double)x[i] * (double)v;
    }
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
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)kCgThreads + threadIdx.x; i < n; i += (int64_t)nblk * kCgThreads) {
        const float v = b[o + i] - Ap[o + i];
        r[o + i] = v;
        p[o + i] = v;
        s += (double)v * (double)v;
    }
    s = block_sum(s);
    if (threadIdx.x == 0) part[(int64_t)j * nblk + blockIdx.x] = s;
}

// x_j += a_j p_j, r_j -= a_j Ap_j, partials of r_j . r_j
__global__ void __launch_bounds__(kCgThreads)
k_step(float* __restrict__ x, float* __restrict__ r, const float* __restrict__ p, const float* __restrict__ Ap,
       const CgVec* __restrict__ cv, int64_t n, double* __restrict__ part)
{
    const int j = blockIdx.y, nblk = gridDim.x;
    const int64_t o = (int64_t)j * n;
    const float aj = cv[j].alpha;
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)kCgThreads + threadIdx.x; i < n; i += (int64_t)nblk * kCgThreads) {
        x[o + i] += aj * p[o + i];
        const float v = r[o + i] - aj * Ap[o + i];
        r[o + i] = v;
        s += (double)v * (double)v;
    }
    s = block_sum(s);
    if (threadIdx.x == 0) part[(int64_t)j * nblk + blockIdx.x] = s;
}

// p_j = r_j + beta_j p_j
__global__ void __launch_bounds__(kCgThreads)
k_direction(float* __restrict__ p, const float* __restrict__ r, const CgVec* __restrict__ cv, int64_t n)
{
    const int j = blockIdx.y, nblk = gridDim.x;
    const int64_t o = (int64_t)j * n;
    const float bj = cv[j].beta;
    for (int64_t i = blockIdx.x * (int64_t)kCgThreads + threadIdx.x; i < n; i += (int64_t)nblk * kCgThreads)
        p[o + i] = r[o + i] + bj * p[o + i];
}

// Sums the nblk partials of vector j in order, then updates its scalars:
//   FIN_BB     bb = b.b
//   FIN_RS     rs = r.r of the initial residual; relative residual; active
//   FIN_ALPHA  step length alpha = rs / p.Ap (0 once converged)
//   FIN_BETA   new r.r: iteration count, relative residual, convergence,
//              direction weight beta = r.r / rs (0 once converged), rs = r.r
__global__ void k_finish(const double* __restrict__ part, int nblk, int fin, int it, double tol,
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
        v.rel = v.bb > 0.0 ? (float)sqrt(s / v.bb) : 0.f;
        v.active = v.rel > tol ? 1 : 0;
        v.iters = 0;
        v.alpha = 0.f;
        v.beta = 0.f;
    } else if (fin == FIN_ALPHA) {
        v.alpha = (v.active && s > 0.0) ? (float)(v.rs / s) : 0.f;
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

int cg_blocks() { return 2 * 152; }

cudaError_t launch_cg(int kind, int fin, int it, double tol, int nrhs, int64_t n, float* x, float* r, float* p,
                      float* Ap, const float* b, float alpha, double* part, CgVec* cv, cudaStream_t st)
{
    const int nblk = cg_blocks();
    dim3 grid((unsigned)nblk, (unsigned)nrhs);
    switch (kind) {
        case CG_DOT_BB: k_dot<<<grid, kCgThreads, 0, st>>>(b, b, n, part); break;
        case CG_SHIFT_DOT: k_shift_dot<<<grid, kCgThreads, 0, st>>>(Ap, p, alpha, n, part); break;
        case CG_RESIDUAL: k_residual<<<grid, kCgThreads, 0, st>>>(b, Ap, r, p, n, part); break;
        case CG_STEP: k_step<<<grid, kCgThreads, 0, st>>>(x, r, p, Ap, cv, n, part); break;
        case CG_DIRECTION:
            k_direction<<<grid, kCgThreads, 0, st>>>(p, r, cv, n);
            count_launch();
            return cudaGetLastError();
        default: return cudaErrorInvalidValue;
    }
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || fin == FIN_NONE) return e;
    k_finish<<<nrhs, kCgThreads, 0, st>>>(part, nblk, fin, it, tol, cv);
    count_launch();
    return cudaGetLastError();
}

}  // namespace btt
