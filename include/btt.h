/*
 * btt.h -- C ABI of the GB300 library for block lower-triangular Toeplitz
 * operators (parameter-to-observable maps of linear time-invariant systems)
 * applied through FFTs.
 *
 * The operator F has N_t x N_t blocks of size N_d x N_m; block (i, j) is
 * F_{i-j} for i >= j and zero above the diagonal (Sec. 2.1,
 * Eq. ShiftInvariance).  Only the first block column F_0 .. F_{N_t-1} is
 * given.  The library applies
 *     d = F m                     (Alg. 2, Sec. 3.3)
 *     m = F* d                    (Alg. 3, Sec. 3.4, Eq. AdjointFFTMatvec)
 *     y = F* Gamma^-1 F m         (Gauss-Newton Hessian of the misfit of
 *                                  Eq. ObjectiveFunctional weighted by a
 *                                  diagonal noise precision, Sec. 2.2)
 * by embedding each block-Toeplitz time convolution in a circulant of
 * length 2 N_t (Sec. 2.4, Eq. CirculantMatrix), so that after a real DFT
 * along time the operator is block diagonal over the N_t + 1 non-negative
 * frequencies w:  dhat(w) = Fhat(w) mhat(w),  mhat(w) = Fhat(w)^H dhat(w).
 *
 * Conventions shared by every entry point
 *   Layout.   Vectors are time-outer and row-major: m[b][t][l] (N_m
 *             fastest), d[b][t][s] (N_d fastest); b indexes nrhs
 *             independent right-hand sides.  Blocks are F[k][s][l].
 *   Memory.   Vector pointers may be device memory or host memory (pinned
 *             or pageable); the library detects which.  Device pointers are
 *             used in place.  Host pointers are staged through library-owned
 *             device buffers: with pinned host memory the call stays
 *             asynchronous on `stream` (synchronise before reading the
 *             output); with pageable host memory the call returns after the
 *             output has been written.
 *   Streams.  `stream` is a cudaStream_t (NULL = legacy default stream).
 *             All work of a call is ordered on it; calls on one operator
 *             must not run concurrently on different streams (they share
 *             the operator's workspace).
 *   Ownership. The caller owns every buffer it passes.  The operator owns
 *             Fhat, its FFT tables and its workspace, from btt_create until
 *             btt_destroy.  btt_create copies what it needs from `blocks`.
 *   Errors.   Every entry point returns a btt_status; on failure nothing is
 *             aborted or trapped, btt_last_error() describes the failure
 *             (thread-local), and the operator stays usable for later calls
 *             unless the status is BTT_ERR_CUDA from a sticky device error.
 */
#ifndef BTT_H
#define BTT_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct btt_op btt_op;

typedef enum {
    BTT_OK = 0,
    BTT_ERR_ARG = 1,          /* invalid argument: null pointer, bad size, wrong precision */
    BTT_ERR_OOM = 2,          /* device or pinned allocation failed */
    BTT_ERR_CUDA = 3,         /* a CUDA call failed; see btt_last_error() */
    BTT_ERR_TIMEOUT = 4,      /* a bounded device-side wait ran out */
    BTT_ERR_UNSUPPORTED = 5   /* size or option this build does not handle */
} btt_status;

/* Storage format of Fhat.  Arithmetic is FP32 with FP32 accumulation for all
 * but BTT_F64 (FP64 throughout, double I/O through the *_f64 calls).  The
 * precompute FFT (Alg. 1) is FP64 for every format. */
typedef enum {
    BTT_F32 = 0,          /* complex64, 8 B per entry */
    BTT_F16_SCALED = 1,   /* FP16 pair of Fhat/s_w, s_w = max|Re,Im| of the slice / 2^14; 4 B */
    BTT_BF16 = 2,         /* BF16 pair, 4 B */
    BTT_BF16_SPLIT = 3,   /* BF16 hi pair + BF16 lo pair, value hi + lo; 8 B, stored as two
                             planes (all hi pairs, then all lo pairs) */
    BTT_F64 = 4,          /* complex128, 16 B */
    BTT_FP8_SCALED = 5    /* FP8 E4M3 pair of Fhat/s_w, FP32 scale s_w per frequency; 2 B */
} btt_precision;

/* Which units run the per-frequency products when several right-hand
 * sides are applied together. */
typedef enum {
    BTT_GEMM_AUTO = 0,     /* tensor cores for BTT_BF16 / BTT_BF16_SPLIT and nrhs >= 16, else SIMT */
    BTT_GEMM_SIMT = 1,     /* always the streaming SIMT kernels */
    BTT_GEMM_TENSOR = 2    /* tensor cores whenever the format allows (BTT_BF16, and
                              BTT_BF16_SPLIT as three BF16 products: hi hi + hi lo + lo hi) */
} btt_gemm_mode;

typedef struct {
    int precision;             /* btt_precision */
    int max_nrhs;              /* right-hand sides one internal pass holds (>= 1);
                                  larger nrhs are processed in chunks of this size */
    size_t workspace_limit;    /* bytes; 0 = no limit.  BTT_ERR_OOM if the
                                  workspace for max_nrhs would exceed it */
    void* stream;              /* stream for the work of btt_create (NULL = default) */
    int gemm;                  /* btt_gemm_mode */
    int host_staging;          /* vectors the host-pointer staging buffers hold; -1 (default)
                                  = max_nrhs, 0 = none (host pointers then fail with BTT_ERR_ARG) */
} btt_options;

/* Fills *opt with defaults: BTT_F32, max_nrhs 1, no limit, default stream,
 * BTT_GEMM_AUTO, host staging for max_nrhs vectors. */
void btt_default_options(btt_options* opt);

/*
 * btt_create -- setup phase (Alg. 1; Sec. 3.2).
 *   blocks  first block column, float64 [N_t][N_d][N_m] row-major, host or
 *           device memory; read only during the call.
 *   N_t, N_d, N_m >= 1.  The padded transform length 2 N_t must factor into
 *           2, 3, 5 and 7 and be at most 24576 (else BTT_ERR_UNSUPPORTED);
 *           BTT_F64 operators also need 2 N_t <= 14528 (their transforms run
 *           in one CTA's shared memory).
 *   For every (s, l) the series F_k[s][l], k < N_t, is padded with N_t
 *   zeros at the end and transformed by an unnormalised FP64 real DFT of
 *   length 2 N_t; the N_t + 1 non-negative frequencies are stored
 *   frequency-major, Fhat[w][s][l], in the requested format.  Synchronises
 *   `opt->stream` before returning.  *out is set only on success.
 */
btt_status btt_create(btt_op** out, const double* blocks, int N_t, int N_d, int N_m,
                      const btt_options* opt);

/* Frees everything the operator owns (synchronises its device work first).
 * NULL is accepted. */
btt_status btt_destroy(btt_op* op);

/*
 * btt_matvec -- d = F m for nrhs vectors (Alg. 2; Sec. 3.3).
 *   m  float32 [nrhs][N_t][N_m];  d  float32 [nrhs][N_t][N_d] (overwritten).
 *   Steps: pad + real DFT of m along time -> mhat[w][l];
 *          dhat[w] = Fhat[w] mhat[w] for every frequency;
 *          inverse real DFT (1/(2 N_t)) and keep the first N_t samples.
 *   nrhs >= 0 (0 is a no-op).  BTT_ERR_ARG on an FP64 operator.
 */
btt_status btt_matvec(btt_op* op, const float* m, float* d, int nrhs, void* stream);

/*
 * btt_adjoint -- m = F* d for nrhs vectors (Alg. 3; Sec. 3.4).
 *   d  float32 [nrhs][N_t][N_d];  m  float32 [nrhs][N_t][N_m] (overwritten).
 *   Same steps as btt_matvec with mhat[w] = Fhat[w]^H dhat[w]
 *   (Eq. AdjointFFTMatvec): the stored Fhat is read, conjugate-transposed
 *   on the fly; nothing else is stored for F*.
 */
btt_status btt_adjoint(btt_op* op, const float* d, float* m, int nrhs, void* stream);

/*
 * btt_adjoint_weighted -- m = F* (Gamma^-1 d): the adjoint (Alg. 3,
 * Sec. 3.4) applied to data weighted by the diagonal noise precision, i.e.
 * the second pass of a Hessian action whose first pass ran elsewhere.
 *   d          float32 [nrhs][N_t][N_d]
 *   gamma_inv  float32 [N_t][N_d] (host or device); NULL makes this btt_adjoint.
 *   m          float32 [nrhs][N_t][N_m] (overwritten).
 * It serves the 1 x p parameter split of Sec. 3.2 (each GPU holds the
 * columns Fhat[:, :, a:b] of the operator and the slice m[:, :, a:b]):
 * F m = sum_q F_q m_q needs one sum-reduction of the N_t x N_d data vector
 * across the GPUs (the reduce of Alg. 2, Sec. 3.5), F* none, so a Hessian
 * action is, on GPU q,
 *     d_q = btt_matvec(op_q, m_q);   d = all-reduce-sum(d_q)   (the caller's
 *     collective, e.g. NCCL: one exchange of 4 N_t N_d bytes per vector);
 *     y_q = btt_adjoint_weighted(op_q, d, gamma_inv).
 * With one GPU (p = 1) the two calls give btt_hessian's result (btt_hessian
 * fuses the hand-off into one kernel instead).  The weighting is one pass
 * over the N_d-sized data into an operator buffer of max_nrhs vectors
 * before the adjoint's input transform.  FP32 operators only.
 */
btt_status btt_adjoint_weighted(btt_op* op, const float* d, const float* gamma_inv, float* m, int nrhs,
                                void* stream);

/*
 * btt_hessian -- y = F* Gamma^-1 F m (Sec. 2.2, Eq. LinearInverseProblem,
 * data-misfit term weighted by a diagonal noise precision).
 *   m          float32 [nrhs][N_t][N_m]
 *   gamma_inv  float32 [N_t][N_d], one precision per data entry, shared by
 *              all right-hand sides; NULL means the identity.
 *   y          float32 [nrhs][N_t][N_m] (overwritten; may not alias m).
 *   Between the two passes the data is brought back to the time domain,
 *   truncated to N_t samples, scaled, re-padded and re-transformed (one
 *   fused kernel), so Fhat is streamed twice per Hessian action.
 */
btt_status btt_hessian(btt_op* op, const float* m, const float* gamma_inv, float* y,
                       int nrhs, void* stream);

/*
 * Multi-right-hand-side products on the tensor cores (BTT_BF16 operators).
 * With nrhs vectors the per-frequency products become complex GEMMs; they
 * run as BF16 x BF16 -> FP32 tcgen05 MMAs: the spectra of the right-hand
 * sides are rounded to BF16 (on top of the BF16 Fhat), so results carry the
 * BF16 error level (relative l2 ~ 1e-3, within the 1e-2 stated for BF16).
 * The F pass of btt_matvec and btt_hessian uses them as btt_options.gemm
 * selects.  Device-side waits inside these kernels are bounded (2 s); a
 * wait that runs out leaves an error code that btt_device_status reports.
 *
 * btt_device_status(op, stream): synchronises `stream`, returns
 * BTT_ERR_TIMEOUT (and clears the code) if a bounded wait of the operator's
 * kernels ran out since the last check, else BTT_OK.
 */
btt_status btt_device_status(btt_op* op, void* stream);   /* (see also the bounds-check build below) */

/*
 * Bounds-check build.  Compiled with -DBTT_CHECK (libbtt_check.so, built
 * by paper_2407_13066_gb300.build.build(check=True) and loaded when the
 * environment sets BTT_CHECK=1), the transform and product kernels test the
 * indices of their shared- and global-memory accesses (tile positions,
 * twiddle and position tables, input and output rows, Fhat rows and
 * columns against the padded row length, staged spectra, the remote
 * shared memory of the cluster transforms) against the extents they derive
 * from; an index outside its extent is recorded (the first one: which
 * access, the index, the extent) and the access is skipped -- nothing
 * traps or faults.  This stands in for a memory checker.
 *   btt_check_build()     1 in the check build, 0 otherwise.
 *   btt_check_status(s)   synchronises stream s; BTT_ERR_CUDA with the
 *                         record in btt_last_error() (and clears it) if a
 *                         check failed since the last call, else BTT_OK
 *                         (always BTT_OK in the normal build).
 *                         btt_device_status reports the same record.
 *   btt_check_selftest(s) check build: launches a kernel that tests one
 *                         index beyond its extent and skips the access, so
 *                         the next btt_check_status reports it (a check of
 *                         the mechanism); BTT_ERR_UNSUPPORTED otherwise.
 */
int btt_check_build(void);
btt_status btt_check_status(void* stream);
btt_status btt_check_selftest(void* stream);

/* Self test of the bounded device waits: launches a kernel whose single
 * wait on an mbarrier is never satisfied; it gives up after `seconds`
 * (0 < seconds <= 10) and records the timeout, so this call returns
 * BTT_ERR_TIMEOUT (through btt_device_status) and the context stays usable.
 * No fault, trap or hang is involved. */
btt_status btt_selftest_wait(btt_op* op, double seconds, void* stream);

/*
 * btt_hessian_batched -- btt_hessian on nrhs vectors held at separate device
 * addresses: m[b] and y[b] are device pointers to float32 [N_t][N_m]
 * (host arrays of nrhs pointers; y[b] may not alias m[b]).  Lets a
 * scheduler batch vectors that live in different buffers without gathering
 * them.  BTT_ERR_ARG if any pointer is not device memory.  The pointer arrays
 * are read during the call only.
 */
btt_status btt_hessian_batched(btt_op* op, const float* const* m, const float* gamma_inv,
                               float* const* y, int nrhs, void* stream);

/*
 * btt_cg -- solves (F* Gamma^-1 F + alpha I) x = b by conjugate gradients:
 * the regularised normal equations of Eq. LinearInverseProblem with R = I
 * and the data misfit weighted by Gamma^-1 (Sec. 2.2), each of the nrhs
 * right-hand sides independently, all advanced together so that every
 * iteration is one batched btt_hessian call.
 *   b          float32 [nrhs][N_t][N_m], device.
 *   gamma_inv  as for btt_hessian (device or host, NULL = identity).
 *   alpha      >= 0; with alpha = 0 the Hessian must be positive definite.
 *   x          float32 [nrhs][N_t][N_m], device: initial guess in, solution out.
 *   Stops a vector when ||b - (H + alpha) x|| <= tol ||b|| (recursive
 *   residual), or after max_iter iterations.  iterations[nrhs] and
 *   relres[nrhs] (host arrays, may be NULL) receive the count and final
 *   relative residual per vector.  Dot products sum groups of 32 terms in
 *   FP32 and the group sums in FP64, in a fixed order (identical results
 *   run to run); the step lengths,
 *   direction weights and convergence flags are computed on the device, so
 *   iterations run without host synchronisation: the call looks at
 *   convergence every 8 iterations (a converged vector stays frozen while
 *   the others finish) and synchronises `stream` before returning when
 *   iterations or relres is given.  The first call (or one with more vectors
 *   than before) allocates 3 nrhs N_t N_m floats of CG workspace, kept by
 *   the operator.  FP32 operators only (any storage).
 */
btt_status btt_cg(btt_op* op, const float* b, const float* gamma_inv, float alpha, float* x, int nrhs,
                  int max_iter, float tol, int* iterations, float* relres, void* stream);

/* FP64 forms of the three actions for a BTT_F64 operator (BTT_ERR_ARG on
 * any other).  Same layouts and semantics with double elements. */
btt_status btt_matvec_f64(btt_op* op, const double* m, double* d, int nrhs, void* stream);
btt_status btt_adjoint_f64(btt_op* op, const double* d, double* m, int nrhs, void* stream);
btt_status btt_hessian_f64(btt_op* op, const double* m, const double* gamma_inv, double* y,
                           int nrhs, void* stream);

/* Sizes and introspection. */
int    btt_precision_of(const btt_op* op);
btt_status btt_operator_shape(const btt_op* op, int* N_t, int* N_d, int* N_m);  /* NULL outputs skipped */
size_t btt_operator_bytes(const btt_op* op);   /* bytes of Fhat (+ scales) in HBM */
/* Bytes of device workspace (spectra, staging, weighting and tensor-core
 * operand buffers; not Fhat, tables or a later btt_cg's vectors).  nrhs <= 0:
 * what this operator holds; nrhs > 0: what an operator of the same shape,
 * format and options would hold with max_nrhs = nrhs (host staging capped
 * as configured), so a caller can size a larger batch before creating it. */
size_t btt_workspace_bytes(const btt_op* op, int nrhs);
/* Bytes one Fhat entry occupies in `precision` (8, 4, 4, 8, 16, 2), 0 if invalid. */
size_t btt_entry_bytes(int precision);

/*
 * btt_copy_fhat -- copies the stored Fhat (storage format, layout
 * [w][s][ldm] with ldm = N_m rounded up to a multiple of 4 (8 for
 * BTT_FP8_SCALED), padding zero; BTT_BF16_SPLIT as two such planes,
 * [2][w][s][ldm] BF16 pairs, hi then lo)
 * into `dst` (host or device, at least btt_operator_bytes - scale bytes),
 * and the FP16 scales into `scales` (float32 [N_t+1], may be NULL).
 * Synchronous.  For inspection and tests.
 */
btt_status btt_copy_fhat(const btt_op* op, void* dst, float* scales);
int btt_fhat_ld(const btt_op* op);

/*
 * btt_save / btt_load -- operator files (the paper stores Fhat after setup
 * for later use, Sec. 3.2, Alg. 1).  btt_save writes an 80-byte header
 * (magic "BTTFHAT1", int32 version 1, precision, N_t, N_d, N_m, ldm,
 * uint64 Fhat and scale byte counts, 32 reserved bytes),
 * the stored Fhat in btt_copy_fhat's layout, then the per-frequency scales
 * of the scaled formats.  Synchronous; host byte order.
 * btt_load creates an operator from such a file without the setup
 * transform: the storage format is the file's (opt->precision is ignored),
 * the other options apply as in btt_create.  A missing, foreign, truncated
 * or inconsistent file returns BTT_ERR_ARG with no operator; allocation
 * failures return BTT_ERR_OOM.
 */
btt_status btt_save(const btt_op* op, const char* path);
btt_status btt_load(btt_op** out, const char* path, const btt_options* opt);

/*
 * btt_inject_fault -- host-side fault injection for failure tests (no GPU
 * fault is ever made): the next `count` device allocations
 * (BTT_FAULT_ALLOC: btt_create / btt_load / btt_cg workspace growth return
 * BTT_ERR_OOM) or the next `count` actions (BTT_FAULT_LAUNCH: btt_matvec,
 * btt_adjoint, btt_hessian and friends return BTT_ERR_CUDA before launching
 * anything) fail; BTT_FAULT_NONE clears both.  The environment variable
 * BTT_FAULT=alloc:N or BTT_FAULT=launch:N sets the same when the library
 * loads.  Operators stay usable after an injected failure.
 */
typedef enum { BTT_FAULT_NONE = 0, BTT_FAULT_ALLOC = 1, BTT_FAULT_LAUNCH = 2 } btt_fault;
btt_status btt_inject_fault(int kind, int count);

/*
 * Stage timers (the per-step breakdown of Sec. 4.1, measured with CUDA
 * events).  While enabled, every action records an event pair around each
 * of its kernel launches on the caller's stream (at most 4096 launches
 * between reads; later ones are counted as dropped).
 *   btt_profile_enable(op, on): on != 0 enables (creating the events once)
 *       and resets; 0 disables.  Host-side, no synchronisation.
 *   btt_profile_read(op, ms, launches): waits for the recorded events and
 *       returns, per stage, the summed milliseconds and launch counts since
 *       the last reset, then resets.  ms and launches hold BTT_NSTAGES
 *       entries.  BTT_ERR_ARG if launches were dropped (sums still filled).
 */
typedef enum {
    BTT_STAGE_RFFT = 0,      /* pad + real DFT of the input (+ reorder) */
    BTT_STAGE_GEMV_F = 1,    /* per-frequency Fhat products, F */
    BTT_STAGE_MID = 2,       /* Hessian: inverse DFT, unpad, Gamma^-1, pad, DFT */
    BTT_STAGE_GEMV_ADJ = 3,  /* per-frequency Fhat^H products, F* */
    BTT_STAGE_IRFFT = 4,     /* inverse real DFT + unpad */
    BTT_NSTAGES = 5
} btt_stage;

btt_status btt_profile_enable(btt_op* op, int on);
btt_status btt_profile_read(btt_op* op, double* ms, long long* launches);

/*
 * btt_matvec_noalloc -- d = F m for callers that cannot allocate device
 * memory.  The paper has no counterpart; this is an additional way to call
 * the F action.
 *
 * Code running inside another framework's execution step (a custom call
 * of XLA or a similar runtime that owns all device memory and hands over
 * every buffer), an inference-server plugin confined to a preallocated
 * arena, or a real-time loop that forbids allocation after start-up may not
 * call cudaMalloc when it applies the operator: an allocation can
 * synchronise the device, fail under the framework's memory cap, or break
 * a captured graph.  This entry point takes no operator handle and
 * allocates nothing; the caller passes Fhat, m and d, all in device memory.
 *   fhat  complex64 [N_t+1][N_d][ldm], ldm = N_m rounded up to a multiple of
 *         4, padding columns zero, 16-byte aligned -- the layout
 *         btt_copy_fhat writes for a BTT_F32 operator.
 *   m     float32 [nrhs][N_t][N_m];  d  float32 [nrhs][N_t][N_d] (overwritten).
 * The spectra and FFT tables live in one fixed device array of
 * BTT_NOALLOC_SCRATCH_BYTES (32 MiB), held by every GPU that loads the
 * library until the process exits.  BTT_ERR_UNSUPPORTED, with the byte
 * count in btt_last_error(), if 8 (9 N_t + (N_t+1)(nrhs (ldm + N_d)))
 * bytes (twiddle and position tables, then the spectra; plus alignment)
 * exceed it, and if nrhs > 65535 or N_d N_m > 2^31 - 1; these checks come
 * before anything is enqueued.
 * The first call on a device looks up the array's device address (and
 * sets kernel attributes) with that device current; make that first call
 * before any stream capture.  All calls share the array and it keeps the
 * previous call's contents (each call rewrites what it reads): calls that
 * overlap on the GPU -- on different streams or different host threads --
 * race, so order them on one stream.  Asynchronous on `stream`.
 */
#define BTT_NOALLOC_SCRATCH_BYTES ((size_t)32 << 20)
btt_status btt_matvec_noalloc(const void* fhat, int N_t, int N_d, int N_m, const float* m,
                              float* d, int nrhs, void* stream);

/*
 * Serving: Hessian actions F* Gamma^-1 F for a stream of requests against
 * several resident operators (the Hessian matvec of Sec. 2.2 as a service).
 *
 * A server runs one scheduler thread and one CUDA stream per operator.
 * Requests carry 1..max_batch vectors ([nvec][N_t][N_m] float32, input m and
 * output y, each in host or device memory).  Requests are admitted in
 * arrival order; one whose vectors are in host memory needs device slots
 * for its input and output, carved from a pool of pool_bytes allocated at
 * creation: it waits until the pool has room (later requests do not
 * overtake it), then its input is uploaded at once.  Whenever an operator
 * has finished its previous batch, all its admitted requests (arrival
 * order, whole requests, at most max_batch vectors) form its next batch --
 * one btt_hessian_batched call over their vectors -- so requests that
 * arrive while a batch runs join the next one (continuous batching), and
 * the operators' batches overlap on the device.  Results of host requests
 * are downloaded on a separate stream.  Use pinned host memory: with
 * pageable memory the copies block the scheduler thread.
 *
 *   btt_server_create   ops[n_ops] (not owned; they must outlive the server
 *                       and not be used by others meanwhile), gamma_inv[n_ops]
 *                       (device [N_t][N_d] float32 or NULL; the array may be
 *                       NULL).  BTT_ERR_OOM if the pool cannot be allocated.
 *   btt_server_submit   returns a ticket at once; BTT_ERR_ARG if nvec >
 *                       max_batch, BTT_ERR_OOM if the request could never fit
 *                       the pool.  The caller keeps m and y valid until the
 *                       request completes.
 *   btt_server_wait     blocks until the request is done (its status) or
 *                       timeout_s passes (BTT_ERR_TIMEOUT; < 0 waits forever);
 *                       a finished ticket is released by its wait.
 *   btt_server_poll     state: 0 waiting, 1 admitted, 2 running, 3 done, 4 failed.
 *   btt_server_stats    counters and latency percentiles (submit to result
 *                       on the host, completed requests) since the last reset.
 *   btt_server_inject   host-side fault injection for tests: 1 fails the next
 *                       batch as if its launch failed, 2 fails the next
 *                       admission as if memory ran out.  No GPU fault.
 *   btt_server_destroy  stops the scheduler, waits for the device work in
 *                       flight, fails unfinished requests, frees the pool.
 */
typedef struct btt_server btt_server;
typedef struct {
    long long submitted, completed, failed, vectors_completed, batches;
    double mean_batch_vectors;
    double latency_p50_ms, latency_p99_ms, latency_mean_ms;
    double span_s;                     /* first submit to last completion */
    size_t pool_bytes, pool_in_use, pool_high_water;
    long long waiting, admitted, running;
} btt_serving_stats;

btt_status btt_server_create(btt_server** out, btt_op* const* ops, const float* const* gamma_inv, int n_ops,
                             size_t pool_bytes, int max_batch);
btt_status btt_server_submit(btt_server* s, int op, const float* m, float* y, int nvec, long long* ticket);
btt_status btt_server_wait(btt_server* s, long long ticket, double timeout_s);
btt_status btt_server_poll(btt_server* s, long long ticket, int* state);
btt_status btt_server_stats(btt_server* s, btt_serving_stats* out, int reset);
btt_status btt_server_inject(btt_server* s, int fault);
btt_status btt_server_destroy(btt_server* s);

/* Number of kernels the library has launched in this process (all
 * operators and threads); differences around a region count its launches. */
long long btt_launch_count(void);

/* Thread-local description of the last failure on this thread ("" if none). */
const char* btt_last_error(void);

/* Library version string. */
const char* btt_version(void);

#ifdef __cplusplus
}
#endif

#endif /* BTT_H */
