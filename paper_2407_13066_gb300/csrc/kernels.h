// Host-side launchers of the library's kernels (internal interface).
#pragma once

#include <cuda.h>

#include "common.cuh"

namespace btt {

// Geometry of the time transforms of one operator.
struct FftGeom {
    int N_t;       // samples kept
    int L;         // padded transform length, 2 N_t
    int wc_log2;   // log2 of the complex columns per CTA
    FftPlan plan;
    const int* pos;  // device table: position of frequency k after a forward transform
};

// Builds the radix plan for L and the column tile for a shared-memory
// budget of kFftCap complex values.  False if L does not factor into
// 2, 3, 5, 7 or exceeds kFftMaxL.
bool make_fft_geom(int N_t, FftGeom* g);

// True if the matvec transforms of this geometry (FP64 when fp64) fit in
// one CTA's shared memory.
bool runtime_fits(const FftGeom& g, bool fp64);

// Bytes of global scratch the setup transform needs when its FP64 buffer
// does not fit in shared memory (0 when it does).
size_t create_scratch_bytes(const FftGeom& g);

// Host: pos[k] for k < L, the digit-reversed position of frequency k.
void digit_reversal(const FftGeom& g, int* pos);

// Counts kernel launches made by the library (read by btt_launch_count).
void count_launch(int n = 1);

// Sets the dynamic shared-memory limits of all kernels (once per device).
cudaError_t prepare_kernels();

#ifdef BTT_CHECK
// Bounds-check build: each translation unit's first recorded failure
// (rec[0] = site, 0 if none; rec[1] = index; rec[2] = extent), cleared
// with clear.
cudaError_t check_record_fft_static(long long* rec, bool clear);
cudaError_t check_record_gemv(long long* rec, bool clear);
cudaError_t check_record_api(long long* rec, bool clear);
cudaError_t check_record_fft_exchange(long long* rec, bool clear);
#endif

// ---- time transforms (fft_kernels.cu) ----
// X[b][w][col] = sum_{t<N_t} x[b][t][col] exp(-2 pi i w t / L), w <= N_t.
// With xptr (device table of nb pointers) vector b is read from xptr[b].
template <typename T>
cudaError_t launch_rfft(const T* x, int64_t ldx, int64_t bsx, int ncols, cplx_t<T>* X,
                        int64_t ldo, int64_t bso, int nb, const FftGeom& g, const cplx_t<T>* tw,
                        cudaStream_t st, const T* const* xptr = nullptr);

// y[b][t][col] = (1/L) sum_{k<L} Xext[b][k][col] exp(+2 pi i k t / L) * (g ? g[t][col] : 1),
// t < N_t, with Xext the Hermitian extension of the half spectrum.  With
// yptr (device table of nb pointers) vector b is written to yptr[b].
template <typename T>
cudaError_t launch_irfft(const cplx_t<T>* X, int64_t ldx, int64_t bsx, int ncols, T* y,
                         int64_t ldy, int64_t bsy, const T* g, int nb, const FftGeom& g_,
                         const cplx_t<T>* tw, cudaStream_t st, T* const* yptr = nullptr);

// In place: X <- rfft(pad(irfft(X)[:N_t] * g)) -- the step between the F and
// F* passes of the Hessian (g = NULL means 1).  With part != NULL, block
// (tile, b) also writes part[b * fft_col_blocks(ncols) + tile] = its share of
// sum_t sum_col g (F m)^2, the Gamma^-1-weighted squared norm of vector b's
// data (p.Hp for the CG solver).
template <typename T>
cudaError_t launch_hess_mid(cplx_t<T>* X, int64_t ldx, int64_t bsx, int ncols, const T* g,
                            int nb, const FftGeom& geom, const cplx_t<T>* tw, cudaStream_t st,
                            double* part = nullptr);
// Column tiles (blocks per vector) of the transforms of ncols columns.
int fft_col_blocks(int ncols, const FftGeom& geom);

// Setup (Alg. 1): FP64 transform of the columns [col_base, col_base+ncols)
// of the blocks (given as blk[t][col - col_base] with row stride ldb) and
// store into Fhat[w][s][ldm] in precision `prec`.  For P_F16S, pass 0
// accumulates per-frequency maxima into maxbits (double bit patterns) and
// pass 1 stores with scales[w].
cudaError_t launch_create(const double* blk, int64_t ldb, int ncols, int64_t col_base, int N_d,
                          int N_m, int ldm, int prec, void* fhat, const float* scales,
                          unsigned long long* maxbits, int pass, const FftGeom& g,
                          const double2* tw, double2* scratch, cudaStream_t st);

// scales[w] = fp32(max_w / target), or 1 for an all-zero slice.
cudaError_t launch_make_scales(const unsigned long long* maxbits, float* scales, int n, double target,
                               cudaStream_t st);

// ---- per-frequency products (gemv_kernels.cu) ----
// dh[b][w][s] = sum_l Fhat[w][s][l] xh[b][w][l]          (Alg. 2, apply_matrix)
cudaError_t launch_gemv_fwd(int prec, const void* fhat, const float* scales, int n_freq, int N_d,
                            int ldm, const void* xh, int64_t xbs, void* dh, int64_t dbs, int nrhs,
                            cudaStream_t st);
// mh[b][w][l] = sum_s conj(Fhat[w][s][l]) dh[b][w][s]    (Alg. 3, conjugate=TRUE)
cudaError_t launch_gemv_adj(int prec, const void* fhat, const float* scales, int n_freq, int N_d,
                            int N_m, int ldm, const void* dh, int64_t dbs, void* mh, int64_t mbs,
                            int nrhs, cudaStream_t st);

// ---- fixed-plan FP32 transforms (fft_static.cu); false if no plan for g.L ----
cudaError_t prepare_static_fft();
bool static_rfft(const float* x, int64_t ldx, int64_t bsx, int ncols, float2* X, int64_t ldo, int64_t bso, int nb,
                 const FftGeom& g, const float2* tw, cudaStream_t st, const float* const* xptr, cudaError_t* err);
bool static_rfft_stack(const float* x, int64_t ldx, int64_t bsx, int ncols, void* xstack, int ldm, int mt_stride,
                       int nb, const FftGeom& g, const float2* tw, cudaStream_t st, int64_t lo_off,
                       const float* const* xptr, cudaError_t* err);
bool static_irfft(const float2* X, int64_t ldx, int64_t bsx, int ncols, float* y, int64_t ldy, int64_t bsy,
                  const float* gam, int nb, const FftGeom& g, const float2* tw, cudaStream_t st, float* const* yptr,
                  cudaError_t* err);
// The inverse transform (no gamma) from BF16 pairs X[b][w][col], the
// tensor-core adjoint's BF16 output.
cudaError_t launch_irfft_bf16(const __nv_bfloat162* X, int64_t ldx, int64_t bsx, int ncols, float* y,
                              int64_t ldy, int64_t bsy, int nb, const FftGeom& g, const float2* tw,
                              cudaStream_t st, float* const* yptr);
struct CgFuse;
// The fixed-plan inverse transform with the CG step fused (see CgFuse), from
// complex64 or (bf16) BF16 pairs; false for lengths without a fixed plan.
bool static_irfft_cg(const void* X, bool bf16, int64_t ldx, int64_t bsx, int ncols, int nb, const FftGeom& g,
                     const float2* tw, cudaStream_t st, const CgFuse& cg, cudaError_t* err);
// ---- one-exchange FP32 transforms (fft_exchange.cu) at 2 N_t = 128 .. 2048
// (the forms that measured faster there); false elsewhere or when
// BTT_FFT_EXCHANGE=0.  Arguments as the static_* forms;
// tw must hold the lane-pair twiddles after the 3 L quad-table floats2. ----
cudaError_t prepare_exchange_fft();
bool exchange_rfft(const float* x, int64_t ldx, int64_t bsx, int ncols, float2* X, int64_t ldo, int64_t bso, int nb,
                   const FftGeom& g, const float2* tw, cudaStream_t st, const float* const* xptr, cudaError_t* err);
bool exchange_rfft_stack(const float* x, int64_t ldx, int64_t bsx, int ncols, void* xstack, int ldm, int mt_stride,
                         int nb, const FftGeom& g, const float2* tw, cudaStream_t st, int64_t lo_off,
                         const float* const* xptr, cudaError_t* err);
bool exchange_irfft(const float2* X, int64_t ldx, int64_t bsx, int ncols, float* y, int64_t ldy, int64_t bsy,
                    const float* gam, int nb, const FftGeom& g, const float2* tw, cudaStream_t st, float* const* yptr,
                    cudaError_t* err);
bool exchange_irfft_bf16(const __nv_bfloat162* X, int64_t ldx, int64_t bsx, int ncols, float* y, int64_t ldy,
                         int64_t bsy, int nb, const FftGeom& g, const float2* tw, cudaStream_t st, float* const* yptr,
                         cudaError_t* err);
// True when 2 N_t has a fixed radix plan.
bool static_plan(const FftGeom& g);
// Its fixed-plan form; false for lengths without a fixed plan.
bool static_irfft_bf16(const __nv_bfloat162* X, int64_t ldx, int64_t bsx, int ncols, float* y, int64_t ldy,
                       int64_t bsy, int nb, const FftGeom& g, const float2* tw, cudaStream_t st, float* const* yptr,
                       cudaError_t* err);
bool static_hess_mid(float2* X, int64_t ldx, int64_t bsx, int ncols, const float* gam, int nb, const FftGeom& g,
                     const float2* tw, cudaStream_t st, double* part, cudaError_t* err);

// ---- conjugate-gradient vector kernels (cg.cu) ----
enum CgKind { CG_DOT_BB = 0, CG_SHIFT_DOT = 1, CG_RESIDUAL = 2, CG_STEP = 3, CG_DIRECTION = 4 };
enum CgFinish { FIN_NONE = 0, FIN_BB = 1, FIN_RS = 2, FIN_ALPHA = 3, FIN_BETA = 4, FIN_PP = 5 };
// Scalars of one right-hand side's CG run, kept on the device.
struct CgVec {
    double bb, rs, pp;    // b.b, current r.r, current p.p
    float rel;            // ||r|| / ||b||
    float alpha, beta;    // step length, direction weight of this iteration
    int active;           // 1 while rel > tol
    int iters;            // iterations taken
    int pad;
};
// Blocks per vector of the CG vector kernels for nrhs vectors, and the FP64
// partials a workspace for up to nrhs vectors needs (at least
// cg_blocks(k) * k for every k <= nrhs).
int cg_blocks(int nrhs);
size_t cg_partials(int nrhs);
// One CG vector step over nrhs vectors of length n (the dot-product kinds
// leave cg_blocks(nrhs) FP64 partials per vector in part), then the finishing
// reduction `fin` updates the CgVec of each vector (iteration `it`, relative
// tolerance `tol`).  CG_STEP / CG_DIRECTION read alpha / beta from cv;
// `alpha` is the regularisation shift of H + alpha I.
cudaError_t launch_cg(int kind, int fin, int it, double tol, int nrhs, int64_t n, float* x, float* r, float* p,
                      float* Ap, const float* b, float alpha, double* part, CgVec* cv, cudaStream_t st);
// The finishing reduction `fin` alone, over nblk partials per vector in
// part (FIN_ALPHA: the p.Hp partials of the Hessian's middle step, with the
// stored p.p: alpha_j = rs / (p.Hp + shift p.p); FIN_BETA: r.r partials).
cudaError_t launch_cg_finish(const double* part, int nblk, int fin, int it, double tol, float shift, int nrhs,
                             CgVec* cv, cudaStream_t st);

// The CG step fused into the Hessian's last inverse transform: with Hp the
// transform's output for vector b (never stored), x_b += alpha_b p_b and
// r_b -= alpha_b (Hp + shift p_b), alpha_b = cv[b].alpha; block (tile, b)
// leaves its share of r_b.r_b in part[b * fft_col_blocks(ncols) + tile].
// x, r, p are [nb][N_t][ncols] with vector stride n.
struct CgFuse {
    const float* p;
    float* x;
    float* r;
    CgVec* cv;           // read by the transform (alpha); written by the finishing reductions
    double* part;
    int64_t n;
    float shift;
};

// ---- tensor-core multi-RHS products (tc_gemm.cu) ----
// Plan of the BF16 tcgen05 path for one operator.
struct TcPlan {
    CUtensorMap tmA;      // conj BF16 spectra [w][mt][64][K2]
    CUtensorMap tmB;      // Fhat BF16 [w][s][K2], boxes of 64 x N rows (F pass)
    CUtensorMap tmD;      // stacked planar BF16 dhat [w][mt][128][kd] (F* pass)
    CUtensorMap tmF;      // Fhat BF16 [w][s][K2], boxes of 64 x 64 rows (F* pass)
    // split pairs (BF16 hi+lo): the same four maps over the lo planes
    CUtensorMap tmA_lo, tmB_lo, tmD_lo, tmF_lo;
    bool split;
    int64_t xs_lo;        // lo plane of the spectra buffer, in BF16 pairs (0 unless split)
    int64_t ds_lo;        // lo plane of the dhat stack, in BF16 elements (0 unless split)
    void* dstack;         // stacked planar dhat buffer (dstack_bytes, owned by the operator)
    size_t dstack_bytes;
    int kd;               // row length of dstack: N_d rounded up to 8
    int K2;               // 2 ldm: interleaved real/imaginary K extent
    int ktiles;           // K tiles of 64
    int n_ntiles, ntile_rows;
    int mt_alloc;         // 64-vector tiles held by the spectra buffer
    int kt_per_split, nsplit;
    size_t part_floats;   // partial-sum buffer size
    bool ready;
};
// split: Fhat stored as BF16 hi+lo planes; operands get lo planes too and
// the GEMMs add the hi-lo cross products.
TcPlan tc_plan(int n_freq, int N_d, int ldm, int max_nrhs, bool split);
cudaError_t tc_prepare(TcPlan* p, void* xstack, const void* fhat_bf16, int n_freq, int N_d);
// dhat[b][w][s] (complex64, batch stride dbs) for b < nrhs from the stacked
// spectra and Fhat; err receives a non-zero code if a bounded wait ran out.
cudaError_t launch_tc_fwd(const TcPlan& p, int n_freq, int N_d, int nrhs, float* part, int* err, float2* dh,
                          int64_t dbs, cudaStream_t st);
// A wait that nothing completes, bounded by `seconds`: sets *err = 10.
cudaError_t launch_wait_selftest(int* err, double seconds, cudaStream_t st);
// mhat[b][w][l] (batch stride mbs, l < N_m) = sum_s conj(Fhat) dhat for
// b < nrhs, from dhat[b][w][s] (complex64, batch stride dbs); mhat is
// complex64, or BF16 pairs with out_bf16 (not for split pairs).
cudaError_t launch_tc_adj(const TcPlan& p, int n_freq, int N_d, int N_m, int ldm, int nrhs, const float2* dh,
                          int64_t dbs, int* err, void* mh, int64_t mbs, cudaStream_t st, bool out_bf16 = false);
// Real DFT of nb vectors x[b][t][col] into the BF16 operand:
// row (w*mt_stride + b/64)*64 + b%64 holds conj(X); with lo_off != 0 the
// BF16 remainders conj(X) - hi go to the same place lo_off pairs further.
cudaError_t launch_rfft_stack(const float* x, int64_t ldx, int64_t bsx, int ncols, void* xstack, int ldm,
                              int mt_stride, int nb, const FftGeom& g, const float2* tw, cudaStream_t st,
                              int64_t lo_off, const float* const* xptr = nullptr);

}  // namespace btt
