// C ABI of the library (declared in include/btt.h): operator setup, the
// F / F* / Hessian actions, and introspection.  Host code only; the device
// work is in fft_kernels.cu and gemv_kernels.cu.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/btt.h"
#include "kernels.h"

#define BTT_API extern "C" __attribute__((visibility("default")))

using namespace btt;

namespace {

thread_local std::string g_err;

btt_status fail(btt_status s, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

btt_status cuda_fail(cudaError_t e, const char* where)
{
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(BTT_ERR_OOM, "%s: %s", where, cudaGetErrorString(e));
    }
    return fail(BTT_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define CK(call)                                              \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);   \
    } while (0)

// true if p can be read by kernels in place (device or managed memory)
bool on_device(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

size_t entry_bytes(int prec)
{
    switch (prec) {
        case P_F32: return 8;
        case P_F16S: return 4;
        case P_BF16: return 4;
        case P_BF16X2: return 8;
        case P_F64: return 16;
        case P_FP8S: return 2;
        default: return 0;
    }
}

}  // namespace

namespace btt {
void set_last_error(const char* msg) { g_err = msg; }
static std::atomic<long long> g_launches{0};
void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
}  // namespace btt

struct btt_op {
    int N_t = 0, N_d = 0, N_m = 0, ldm = 0, n_freq = 0;
    int prec = 0;
    int max_nrhs = 1;
    int staging_nrhs = 1;             // vectors the host staging buffers hold
    int device = 0;
    FftGeom geom{};
    void* fhat = nullptr;
    size_t fhat_bytes = 0;
    float* scales = nullptr;          // per-frequency scales (F16S only)
    float2* tw32 = nullptr;           // exp(-2 pi i e / L), e < L; then (c, c, d, d) quads of the same;
                                      // then the lane-pair twiddles of the one-exchange transforms
    double2* tw64 = nullptr;
    int* pos = nullptr;               // digit-reversed position of each frequency
    void* xhat = nullptr;             // [max_nrhs][n_freq][ldm] complex
    void* dhat = nullptr;             // [max_nrhs][n_freq][N_d] complex
    void* stage_in = nullptr;         // [max_nrhs][N_t][max(N_m,N_d)] real
    void* stage_out = nullptr;
    void* gamma = nullptr;            // [N_t][N_d] real
    float* dw = nullptr;              // [max_nrhs][N_t][N_d]: Gamma^-1 d for btt_adjoint_weighted
    void** ptab = nullptr;            // device tables of vector pointers: [2][max_nrhs]
    // conjugate-gradient workspace, allocated by the first btt_cg call
    float* cg_vec = nullptr;          // r, p, Ap: [3][cg_cap][N_t][N_m]
    double* cg_part = nullptr;        // dot-product partials and results
    CgVec* cg_state = nullptr;        // per-vector scalars of the method
    int cg_cap = 0;
    size_t ws_bytes = 0;
    // tensor-core path (BTT_BF16)
    int gemm = 0;
    bool tc = false;
    TcPlan tcp{};
    void* xstack = nullptr;           // conj BF16 spectra [w][mt][64][2 ldm]
    void* dstack = nullptr;           // stacked planar BF16 data spectra [w][mt][128][kd]
    float* tc_part = nullptr;         // split-K partial sums
    int* dev_err = nullptr;           // bounded-wait error code
    // stage timers (btt_profile_*): event pairs around each kernel launch
    bool prof = false;
    std::vector<cudaEvent_t> ev;      // 2 per record
    std::vector<int> ev_stage;
    size_t ev_used = 0;
    long long ev_dropped = 0;

    bool is64() const { return prec == P_F64; }
    size_t vbytes() const { return is64() ? 16 : 8; }   // complex workspace element
    size_t rbytes() const { return is64() ? 8 : 4; }    // real vector element
};

namespace {

void free_op(btt_op* op)
{
    if (!op) return;
    for (cudaEvent_t e : op->ev) cudaEventDestroy(e);
    void* ptrs[] = {op->fhat, op->scales, op->tw32, op->tw64, op->pos, op->xhat, op->dhat,
                    op->stage_in, op->stage_out, op->gamma, op->dw, op->xstack, op->dstack, op->tc_part,
                    op->dev_err, op->ptab, op->cg_vec, op->cg_part, op->cg_state};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete op;
}

// Host-side fault injection (btt_inject_fault, or BTT_FAULT=alloc:N /
// launch:N in the environment): the next N device allocations, or the next
// N actions, fail as if CUDA had refused them.  Nothing reaches the GPU.
std::atomic<int> g_fault_alloc{0}, g_fault_launch{0};

bool take_fault(std::atomic<int>& f)
{
    int v = f.load();
    while (v > 0)
        if (f.compare_exchange_weak(v, v - 1)) return true;
    return false;
}

const int g_fault_env = [] {
    const char* e = getenv("BTT_FAULT");
    if (!e) return 0;
    int n = 0;
    if (sscanf(e, "alloc:%d", &n) == 1) g_fault_alloc = n;
    else if (sscanf(e, "launch:%d", &n) == 1) g_fault_launch = n;
    return 1;
}();

btt_status alloc(void** p, size_t bytes, const char* what)
{
    if (take_fault(g_fault_alloc)) {
        *p = nullptr;
        return fail(BTT_ERR_OOM, "allocating %s: injected allocation failure", what);
    }
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(BTT_ERR_OOM, "allocating %s (%zu bytes): %s", what, bytes, cudaGetErrorString(e));
    }
    return BTT_OK;
}

// Runs the setup transform over all block columns; blocks in host memory are
// staged through a device buffer in column chunks.
btt_status run_create(btt_op* op, const double* blocks, bool dev_blocks, unsigned long long* maxbits,
                      int pass, double* chunk_buf, int64_t chunk_cols, double2* scratch, cudaStream_t st)
{
    const int64_t ncol = (int64_t)op->N_d * op->N_m;
    if (dev_blocks) {
        CK(launch_create(blocks, ncol, (int)ncol, 0, op->N_d, op->N_m, op->ldm, op->prec, op->fhat,
                         op->scales, maxbits, pass, op->geom, op->tw64, scratch, st));
        return BTT_OK;
    }
    for (int64_t c0 = 0; c0 < ncol; c0 += chunk_cols) {
        const int64_t nc = ncol - c0 < chunk_cols ? ncol - c0 : chunk_cols;
        CK(cudaMemcpy2DAsync(chunk_buf, nc * sizeof(double), blocks + c0, ncol * sizeof(double),
                             nc * sizeof(double), op->N_t, cudaMemcpyHostToDevice, st));
        CK(launch_create(chunk_buf, nc, (int)nc, c0, op->N_d, op->N_m, op->ldm, op->prec, op->fhat,
                         op->scales, maxbits, pass, op->geom, op->tw64, scratch, st));
    }
    return BTT_OK;
}

btt_status check_op(const btt_op* op, bool want64)
{
    if (!op) return fail(BTT_ERR_ARG, "null operator");
    if (op->is64() != want64)
        return fail(BTT_ERR_ARG, want64 ? "FP64 entry point on a non-FP64 operator"
                                        : "FP32 entry point on an FP64 operator (use the *_f64 calls)");
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != op->device) return fail(BTT_ERR_ARG, "operator lives on device %d, current is %d", op->device, dev);
    return BTT_OK;
}

enum Action { A_FWD, A_ADJ, A_HESS };

bool use_tc(const btt_op* op, int nb)
{
    if (!op->tc) return false;
    if (op->gemm == BTT_GEMM_TENSOR) return true;
    return op->gemm == BTT_GEMM_AUTO && nb >= 16;
}

constexpr size_t kProfRecords = 4096;

// Launches one stage; with profiling on, brackets it with events on `st`.
template <typename F>
btt_status stage(btt_op* op, int which, cudaStream_t st, const char* what, F&& launch)
{
    const bool rec = op->prof && op->ev_used < op->ev_stage.size();
    if (op->prof && !rec) ++op->ev_dropped;
    if (rec) CK(cudaEventRecord(op->ev[2 * op->ev_used], st));
    cudaError_t e = launch();
    if (e != cudaSuccess) return cuda_fail(e, what);
    if (rec) {
        CK(cudaEventRecord(op->ev[2 * op->ev_used + 1], st));
        op->ev_stage[op->ev_used++] = which;
    }
    return BTT_OK;
}

#define STAGE(which, call)                                                            \
    do {                                                                              \
        btt_status s_ = stage(op, which, st, #call, [&]() { return (call); });        \
        if (s_ != BTT_OK) return s_;                                                  \
    } while (0)

// One action on nrhs vectors of element type T (float or double).
// With in_tab / out_tab (host arrays of nrhs device pointers) vector b is
// read from in_tab[b] and written to out_tab[b]; `in` / `out` are unused.
template <typename T>
btt_status run_action(btt_op* op, Action act, const T* in, const T* gamma, T* out, int nrhs,
                      cudaStream_t st, const T* const* in_tab = nullptr, T* const* out_tab = nullptr,
                      double* mid_part = nullptr, const CgFuse* cgf = nullptr)
{
    using V = cplx_t<T>;
    if (nrhs < 0) return fail(BTT_ERR_ARG, "nrhs = %d < 0", nrhs);
    if (nrhs == 0) return BTT_OK;
    if (take_fault(g_fault_launch)) return fail(BTT_ERR_CUDA, "injected launch failure (nothing was launched)");
    const bool tab = in_tab != nullptr;
    if (tab) {
        if (!out_tab) return fail(BTT_ERR_ARG, "null pointer table");
        for (int b = 0; b < nrhs; ++b)
            if (!in_tab[b] || !out_tab[b] || !on_device(in_tab[b]) || !on_device(out_tab[b]))
                return fail(BTT_ERR_ARG, "batched call: vector %d is not a device pointer", b);
        in = in_tab[0];
        out = out_tab[0];
    }
    if (!in || !out) return fail(BTT_ERR_ARG, "null vector pointer");
    const int N_t = op->N_t, N_d = op->N_d, N_m = op->N_m, ldm = op->ldm, nf = op->n_freq;
    const int n_in = act == A_ADJ ? N_d : N_m;
    const int n_out = act == A_FWD ? N_d : N_m;
    const bool in_dev = tab || on_device(in), out_dev = tab || on_device(out);
    if (act == A_HESS && (const void*)in == (const void*)out)
        return fail(BTT_ERR_ARG, "btt_hessian: output aliases input");
    const T* g = nullptr;
    if (act == A_HESS && gamma) {
        if (on_device(gamma)) {
            g = gamma;
        } else {
            CK(cudaMemcpyAsync(op->gamma, gamma, (size_t)N_t * N_d * sizeof(T), cudaMemcpyHostToDevice, st));
            g = static_cast<const T*>(op->gamma);
        }
    }
    V* xh = static_cast<V*>(op->xhat);
    V* dh = static_cast<V*>(op->dhat);
    const FftGeom& geo = op->geom;
    const V* tw = reinterpret_cast<const V*>(op->is64() ? (void*)op->tw64 : (void*)op->tw32);
    const int64_t xbs = (int64_t)nf * ldm, dbs = (int64_t)nf * N_d;
    // host vectors go through the staging buffers, which may hold fewer
    int chunk = op->max_nrhs;
    if (!in_dev || !out_dev) {
        if (op->staging_nrhs == 0)
            return fail(BTT_ERR_ARG, "host vectors on an operator created without host staging");
        if (op->staging_nrhs < chunk) chunk = op->staging_nrhs;
    }
    for (int c0 = 0; c0 < nrhs; c0 += chunk) {
        const int nb = nrhs - c0 < chunk ? nrhs - c0 : chunk;
        const T* vin = in + (size_t)c0 * N_t * n_in;
        T* vout = out + (size_t)c0 * N_t * n_out;
        const T* const* xptr = nullptr;
        T* const* yptr = nullptr;
        if (tab) {
            // this chunk's pointers, copied in stream order into the device tables
            CK(cudaMemcpyAsync(op->ptab, in_tab + c0, nb * sizeof(void*), cudaMemcpyHostToDevice, st));
            CK(cudaMemcpyAsync(op->ptab + op->max_nrhs, out_tab + c0, nb * sizeof(void*), cudaMemcpyHostToDevice, st));
            xptr = reinterpret_cast<const T* const*>(op->ptab);
            yptr = reinterpret_cast<T* const*>(op->ptab + op->max_nrhs);
        }
        if (!in_dev) {
            CK(cudaMemcpyAsync(op->stage_in, vin, (size_t)nb * N_t * n_in * sizeof(T),
                               cudaMemcpyHostToDevice, st));
            vin = static_cast<const T*>(op->stage_in);
        }
        T* work = out_dev ? vout : static_cast<T*>(op->stage_out);
        const bool tc = use_tc(op, nb);
        // BF16 products on the tensor cores hand mhat to the inverse transform
        // as BF16 pairs (half the bytes; one more rounding, ~1e-3 against the
        // products' own ~3e-3); the split pair keeps complex64
        const bool mhat16 = std::is_same<T, float>::value && tc && !op->tcp.split;
        auto adj_irfft = [&]() -> cudaError_t {
            if constexpr (std::is_same<T, float>::value) {
                if (mhat16)
                    return launch_irfft_bf16(reinterpret_cast<const __nv_bfloat162*>(xh), ldm, xbs, N_m, work, N_m,
                                             (int64_t)N_t * N_m, nb, geo, op->tw32, st, yptr);
            }
            return launch_irfft<T>(xh, ldm, xbs, N_m, work, N_m, (int64_t)N_t * N_m, nullptr, nb, geo, tw, st, yptr);
        };
        if (tc && act != A_ADJ) {
            // tensor-core F pass: stacked BF16 spectra, tcgen05 GEMM, split-K reduction into dhat
            if constexpr (std::is_same<T, float>::value) {
                STAGE(BTT_STAGE_RFFT, launch_rfft_stack(vin, N_m, (int64_t)N_t * N_m, N_m, op->xstack, ldm,
                                                        op->tcp.mt_alloc, nb, geo, op->tw32, st, op->tcp.xs_lo, xptr));
                STAGE(BTT_STAGE_GEMV_F, launch_tc_fwd(op->tcp, nf, N_d, nb, op->tc_part, op->dev_err,
                                                      reinterpret_cast<float2*>(dh), dbs, st));
            }
        }
        if (act == A_FWD) {
            if (!tc) {
                STAGE(BTT_STAGE_RFFT, launch_rfft<T>(vin, N_m, (int64_t)N_t * N_m, N_m, xh, ldm, xbs, nb, geo, tw, st, xptr));
                STAGE(BTT_STAGE_GEMV_F, launch_gemv_fwd(op->prec, op->fhat, op->scales, nf, N_d, ldm, xh, xbs, dh, dbs, nb, st));
            }
            STAGE(BTT_STAGE_IRFFT, launch_irfft<T>(dh, N_d, dbs, N_d, work, N_d, (int64_t)N_t * N_d, nullptr, nb, geo, tw, st, yptr));
        } else if (act == A_ADJ) {
            STAGE(BTT_STAGE_RFFT, launch_rfft<T>(vin, N_d, (int64_t)N_t * N_d, N_d, dh, N_d, dbs, nb, geo, tw, st, xptr));
            if (tc) {
                if constexpr (std::is_same<T, float>::value)
                    STAGE(BTT_STAGE_GEMV_ADJ, launch_tc_adj(op->tcp, nf, N_d, N_m, ldm, nb, dh, dbs, op->dev_err, xh, xbs, st,
                                                            mhat16));
            } else {
                STAGE(BTT_STAGE_GEMV_ADJ, launch_gemv_adj(op->prec, op->fhat, op->scales, nf, N_d, N_m, ldm, dh, dbs, xh, xbs, nb, st));
            }
            STAGE(BTT_STAGE_IRFFT, adj_irfft());
        } else {
            if (!tc) {
                STAGE(BTT_STAGE_RFFT, launch_rfft<T>(vin, N_m, (int64_t)N_t * N_m, N_m, xh, ldm, xbs, nb, geo, tw, st, xptr));
                STAGE(BTT_STAGE_GEMV_F, launch_gemv_fwd(op->prec, op->fhat, op->scales, nf, N_d, ldm, xh, xbs, dh, dbs, nb, st));
            }
            // CG: the middle step also leaves the partials of p.Hp = ||F p||^2 (Gamma^-1)
            const int mid_nblk = fft_col_blocks(N_d, geo);
            double* mp = mid_part ? mid_part + (size_t)c0 * mid_nblk : nullptr;
            STAGE(BTT_STAGE_MID, launch_hess_mid<T>(dh, N_d, dbs, N_d, g, nb, geo, tw, st, mp));
            // fused CG step: the step lengths are known once p.Hp is
            if (cgf) CK(launch_cg_finish(mp, mid_nblk, FIN_ALPHA, 0, 0.0, cgf->shift, nb, cgf->cv + c0, st));
            if (tc) {
                if constexpr (std::is_same<T, float>::value)
                    STAGE(BTT_STAGE_GEMV_ADJ, launch_tc_adj(op->tcp, nf, N_d, N_m, ldm, nb, dh, dbs, op->dev_err, xh, xbs, st,
                                                            mhat16));
            } else {
                STAGE(BTT_STAGE_GEMV_ADJ, launch_gemv_adj(op->prec, op->fhat, op->scales, nf, N_d, N_m, ldm, dh, dbs, xh, xbs, nb, st));
            }
            if (cgf) {
                if constexpr (std::is_same<T, float>::value) {
                    CgFuse c = *cgf;
                    c.p += (size_t)c0 * c.n;
                    c.x += (size_t)c0 * c.n;
                    c.r += (size_t)c0 * c.n;
                    c.cv += c0;
                    c.part += (size_t)c0 * fft_col_blocks(N_m, geo);
                    STAGE(BTT_STAGE_IRFFT, [&]() {
                        cudaError_t e = cudaErrorInvalidValue;
                        static_irfft_cg(xh, mhat16, ldm, xbs, N_m, nb, geo, op->tw32, st, c, &e);
                        return e;
                    }());
                }
            } else {
                STAGE(BTT_STAGE_IRFFT, adj_irfft());
            }
        }
        if (!out_dev) {
            CK(cudaMemcpyAsync(vout, work, (size_t)nb * N_t * n_out * sizeof(T), cudaMemcpyDeviceToHost, st));
        }
    }
    return BTT_OK;
}

}  // namespace

BTT_API void btt_default_options(btt_options* opt)
{
    if (!opt) return;
    opt->precision = BTT_F32;
    opt->max_nrhs = 1;
    opt->workspace_limit = 0;
    opt->stream = nullptr;
    opt->gemm = BTT_GEMM_AUTO;
    opt->host_staging = -1;
}

namespace {

// Workspace of an operator (everything it allocates besides Fhat, its
// scales, the FFT tables and the CG workspace of a later btt_cg).
struct WsSizes {
    size_t xh = 0, dh = 0, st = 0, g = 0, dw = 0;   // spectra, staging (x2), gamma, weighted data
    size_t xs = 0, part = 0, dstack = 0;            // tensor-core operands
    bool tc = false;
    size_t total() const { return xh + dh + 2 * st + g + dw + xs + part + dstack; }
};

WsSizes ws_sizes(int N_t, int N_d, int N_m, int ldm, int prec, int max_nrhs, int staging_nrhs, int gemm,
                 TcPlan* tcp_out = nullptr)
{
    WsSizes w;
    const size_t vb = prec == P_F64 ? 16 : 8, rb = prec == P_F64 ? 8 : 4;
    const int nf = N_t + 1;
    w.xh = (size_t)max_nrhs * nf * ldm * vb;
    w.dh = (size_t)max_nrhs * nf * N_d * vb;
    w.st = (size_t)staging_nrhs * N_t * (N_m > N_d ? N_m : N_d) * rb;
    w.g = (size_t)N_t * N_d * rb;
    w.dw = prec == P_F64 ? 0 : (size_t)max_nrhs * N_t * N_d * sizeof(float);
    // tensor-core operands only where they can be used: BF16 formats, and
    // batches large enough for the AUTO rule (or TENSOR forced)
    if ((prec == P_BF16 || prec == P_BF16X2) &&
        (gemm == BTT_GEMM_TENSOR || (gemm == BTT_GEMM_AUTO && max_nrhs >= 16))) {
        const bool split = prec == P_BF16X2;
        TcPlan tcp = tc_plan(nf, N_d, ldm, max_nrhs, split);
        w.tc = true;
        w.xs = (size_t)nf * tcp.mt_alloc * 64 * tcp.K2 * 2 * (split ? 2 : 1);
        w.part = tcp.part_floats * sizeof(float);
        w.dstack = tcp.dstack_bytes;
        if (tcp_out) *tcp_out = tcp;
    }
    return w;
}

int staging_of(const btt_options& opt)
{
    return opt.host_staging < 0 ? opt.max_nrhs : (opt.host_staging < opt.max_nrhs ? opt.host_staging : opt.max_nrhs);
}

// Validates the sizes and options, allocates Fhat (zeroed), the FFT tables,
// the workspaces and the tensor-core operands; Fhat is filled by the caller
// (the setup transform in btt_create, the file in btt_load).
btt_status op_setup(btt_op** out, int N_t, int N_d, int N_m, const btt_options* opt_in)
{
    *out = nullptr;
    if (N_t < 1 || N_d < 1 || N_m < 1)
        return fail(BTT_ERR_ARG, "operator: sizes must be >= 1 (N_t=%d N_d=%d N_m=%d)", N_t, N_d, N_m);
    if ((int64_t)N_d * N_m > 0x7fffffffLL)
        return fail(BTT_ERR_UNSUPPORTED, "operator: N_d*N_m exceeds 2^31-1");
    btt_options opt;
    btt_default_options(&opt);
    if (opt_in) opt = *opt_in;
    if (entry_bytes(opt.precision) == 0) return fail(BTT_ERR_ARG, "operator: unknown precision %d", opt.precision);
    if (opt.max_nrhs < 1) return fail(BTT_ERR_ARG, "operator: max_nrhs must be >= 1");
    if (opt.gemm < BTT_GEMM_AUTO || opt.gemm > BTT_GEMM_TENSOR) return fail(BTT_ERR_ARG, "operator: unknown gemm mode %d", opt.gemm);
    FftGeom geom;
    if (!make_fft_geom(N_t, &geom))
        return fail(BTT_ERR_UNSUPPORTED,
                    "operator: transform length 2*N_t = %d must factor into 2,3,5,7 and be <= %d",
                    2 * N_t, kFftMaxL);
    if (!runtime_fits(geom, opt.precision == P_F64))
        return fail(BTT_ERR_UNSUPPORTED,
                    "operator: FP64 storage needs the length-%d transform in shared memory (2*N_t <= %d)",
                    2 * N_t, kFftSmemMax / (int)sizeof(double2));
    cudaStream_t st = static_cast<cudaStream_t>(opt.stream);

    btt_op* op = new btt_op;
    op->N_t = N_t;
    op->N_d = N_d;
    op->N_m = N_m;
    // rows of Fhat start on 16-byte boundaries in every format
    op->ldm = opt.precision == P_FP8S ? (N_m + 7) / 8 * 8 : (N_m + 3) / 4 * 4;
    op->n_freq = N_t + 1;
    op->prec = opt.precision;
    op->max_nrhs = opt.max_nrhs;
    op->staging_nrhs = staging_of(opt);
    op->gemm = opt.gemm;
    op->geom = geom;
    cudaGetDevice(&op->device);

    const size_t nfhat = (size_t)op->n_freq * N_d * op->ldm;
    op->fhat_bytes = nfhat * entry_bytes(op->prec);
    TcPlan tcp{};
    const WsSizes ws = ws_sizes(N_t, N_d, N_m, op->ldm, op->prec, op->max_nrhs, op->staging_nrhs, op->gemm, &tcp);
    const size_t xh_b = ws.xh, dh_b = ws.dh, st_b = ws.st, g_b = ws.g;
    op->ws_bytes = ws.total();
    if (opt.workspace_limit && op->ws_bytes > opt.workspace_limit) {
        size_t need = op->ws_bytes;
        free_op(op);
        return fail(BTT_ERR_OOM, "operator: workspace %zu bytes exceeds the limit %zu", need,
                    opt.workspace_limit);
    }

    btt_status s = BTT_OK;
    const int L = geom.L;
#define STEP(x)                 \
    do {                        \
        s = (x);                \
        if (s != BTT_OK) {      \
            free_op(op);        \
            return s;           \
        }                       \
    } while (0)
#define CKF(call)                                              \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) STEP(cuda_fail(e_, #call));     \
    } while (0)
    CKF(prepare_kernels());
    STEP(alloc(&op->fhat, op->fhat_bytes, "Fhat"));
    STEP(alloc((void**)&op->tw32, L * 2 * sizeof(float4), "twiddles"));
    STEP(alloc((void**)&op->tw64, L * sizeof(double2), "twiddles"));
    STEP(alloc((void**)&op->pos, L * sizeof(int), "digit-reversal table"));
    STEP(alloc(&op->xhat, xh_b, "mhat workspace"));
    STEP(alloc(&op->dhat, dh_b, "dhat workspace"));
    STEP(alloc(&op->stage_in, st_b, "staging"));
    STEP(alloc(&op->stage_out, st_b, "staging"));
    STEP(alloc(&op->gamma, g_b, "noise precision"));
    if (ws.dw) STEP(alloc((void**)&op->dw, ws.dw, "weighted data"));
    if (op->prec == P_F16S || op->prec == P_FP8S)
        STEP(alloc((void**)&op->scales, op->n_freq * sizeof(float), "scales"));
    STEP(alloc((void**)&op->dev_err, sizeof(int), "error flag"));
    STEP(alloc((void**)&op->ptab, 2 * (size_t)op->max_nrhs * sizeof(void*), "pointer tables"));
    CKF(cudaMemsetAsync(op->dev_err, 0, sizeof(int), st));
    // tensor-core operands (ws_sizes decides where they can be used)
    if (ws.tc) {
        op->tcp = tcp;
        STEP(alloc(&op->xstack, ws.xs, "stacked BF16 spectra"));
        STEP(alloc((void**)&op->tc_part, ws.part, "split-K partial sums"));
        STEP(alloc(&op->dstack, ws.dstack, "stacked BF16 data spectra"));
        op->tcp.dstack = op->dstack;
        CKF(cudaMemsetAsync(op->xstack, 0, ws.xs, st));
        CKF(cudaMemsetAsync(op->dstack, 0, ws.dstack, st));
        CKF(tc_prepare(&op->tcp, op->xstack, op->fhat, op->n_freq, N_d));
        op->tc = true;
    }

    // twiddles exp(-2 pi i e / L) in extended precision, rounded once
    std::vector<double2> t64(L);
    // (FP32: L complex64 entries, then the same L values as quad entries
    // (c, c, d, d) for the paired-lane fixed-plan transforms, then L/2
    // lane-pair entries (c_a, c_b, d_a, d_b) / 2 of e_a = 2 m n2 and e_b =
    // (2 m + 1) n2, entry n2 R1/2 + m, for the one-exchange transforms
    // (L = R1 N2, R1 = min(32, L/16), n2 < N2, m < R1/2; the 1/2 is exact))
    std::vector<float2> t32(4 * (size_t)L);
    for (int e = 0; e < L; ++e) {
        const long double a = 2.0L * 3.14159265358979323846264338327950288L * (long double)e / (long double)L;
        t64[e] = make_double2((double)cosl(a), (double)-sinl(a));
        const float c = (float)cosl(a), d = (float)-sinl(a);
        t32[e] = make_float2(c, d);
        t32[L + 2 * (size_t)e] = make_float2(c, c);
        t32[L + 2 * (size_t)e + 1] = make_float2(d, d);
    }
    if (L % 32 == 0) {
        const int H = L >= 512 ? 16 : L / 32;   // R1 / 2, R1 = min(32, L / 16)
        for (int i = 0; i < L / 2; ++i) {
            const int n2 = i / H, m = i % H;
            const float2 wa = t32[2 * m * n2], wb = t32[(2 * m + 1) * n2];
            t32[3 * (size_t)L + 2 * (size_t)i] = make_float2(0.5f * wa.x, 0.5f * wb.x);
            t32[3 * (size_t)L + 2 * (size_t)i + 1] = make_float2(0.5f * wa.y, 0.5f * wb.y);
        }
    }
    CKF(cudaMemcpyAsync(op->tw64, t64.data(), L * sizeof(double2), cudaMemcpyHostToDevice, st));
    CKF(cudaMemcpyAsync(op->tw32, t32.data(), t32.size() * sizeof(float2), cudaMemcpyHostToDevice, st));
    std::vector<int> pos(L);
    digit_reversal(op->geom, pos.data());
    CKF(cudaMemcpyAsync(op->pos, pos.data(), L * sizeof(int), cudaMemcpyHostToDevice, st));
    op->geom.pos = op->pos;
    // zero Fhat (row padding l >= N_m stays zero) and the workspace padding
    CKF(cudaMemsetAsync(op->fhat, 0, op->fhat_bytes, st));
    CKF(cudaMemsetAsync(op->xhat, 0, xh_b, st));
#undef CKF
#undef STEP
    *out = op;
    return BTT_OK;
}

}  // namespace

BTT_API btt_status btt_create(btt_op** out, const double* blocks, int N_t, int N_d, int N_m,
                              const btt_options* opt_in)
{
    g_err.clear();
    if (!out) return fail(BTT_ERR_ARG, "btt_create: null output handle");
    *out = nullptr;
    if (!blocks) return fail(BTT_ERR_ARG, "btt_create: null blocks");
    btt_op* op = nullptr;
    btt_status s = op_setup(&op, N_t, N_d, N_m, opt_in);
    if (s != BTT_OK) return s;
    btt_options opt;
    btt_default_options(&opt);
    if (opt_in) opt = *opt_in;
    cudaStream_t st = static_cast<cudaStream_t>(opt.stream);
    const FftGeom& geom = op->geom;
#define STEP(x)                 \
    do {                        \
        s = (x);                \
        if (s != BTT_OK) {      \
            free_op(op);        \
            return s;           \
        }                       \
    } while (0)
    const bool dev_blocks = on_device(blocks);
    double* chunk = nullptr;
    int64_t chunk_cols = 0;
    if (!dev_blocks) {
        const int W = 2 << geom.wc_log2;
        const int64_t ncol = (int64_t)N_d * N_m;
        chunk_cols = ((int64_t)(256u << 20) / ((int64_t)N_t * 8)) / W * W;
        if (chunk_cols < W) chunk_cols = W;
        if (chunk_cols > ncol) chunk_cols = ncol;
        cudaError_t e = cudaMalloc((void**)&chunk, (size_t)chunk_cols * N_t * sizeof(double));
        if (e != cudaSuccess) {
            cudaGetLastError();
            STEP(fail(BTT_ERR_OOM, "btt_create: staging for host blocks: %s", cudaGetErrorString(e)));
        }
    }
    double2* cscratch = nullptr;
    if (const size_t csb = create_scratch_bytes(geom)) {
        cudaError_t e = cudaMalloc((void**)&cscratch, csb);
        if (e != cudaSuccess) {
            cudaGetLastError();
            if (chunk) cudaFree(chunk);
            STEP(fail(BTT_ERR_OOM, "btt_create: transform scratch: %s", cudaGetErrorString(e)));
        }
    }
    unsigned long long* maxbits = nullptr;
    if (op->prec == P_F16S || op->prec == P_FP8S) {
        cudaError_t e = cudaMalloc((void**)&maxbits, op->n_freq * sizeof(unsigned long long));
        if (e == cudaSuccess) e = cudaMemsetAsync(maxbits, 0, op->n_freq * sizeof(unsigned long long), st);
        if (e == cudaSuccess)
            s = run_create(op, blocks, dev_blocks, maxbits, 0, chunk, chunk_cols, cscratch, st);
        if (e == cudaSuccess && s == BTT_OK) e = launch_make_scales(maxbits, op->scales, op->n_freq,
                                                                      op->prec == P_FP8S ? kFp8ScaleTarget : kF16ScaleTarget, st);
        if (e != cudaSuccess) s = cuda_fail(e, "btt_create: FP16 scales");
    }
    if (s == BTT_OK) s = run_create(op, blocks, dev_blocks, nullptr, 1, chunk, chunk_cols, cscratch, st);
    cudaError_t es = cudaStreamSynchronize(st);
    if (chunk) cudaFree(chunk);
    if (cscratch) cudaFree(cscratch);
    if (maxbits) cudaFree(maxbits);
    if (s != BTT_OK) STEP(s);
    if (es != cudaSuccess) STEP(cuda_fail(es, "btt_create: synchronize"));
#undef CKF
#undef STEP
    *out = op;
    return BTT_OK;
}

BTT_API btt_status btt_destroy(btt_op* op)
{
    if (!op) return BTT_OK;
    cudaDeviceSynchronize();
    free_op(op);
    return BTT_OK;
}

namespace {

// Operator file: this header, then the stored Fhat as btt_copy_fhat lays it
// out, then the per-frequency scales (FP16 / FP8 formats).
struct FileHeader {
    char magic[8];
    int32_t version;
    int32_t precision;
    int32_t N_t, N_d, N_m, ldm;
    uint64_t fhat_bytes;
    uint64_t scale_bytes;
    uint64_t reserved[4];
};
static_assert(sizeof(FileHeader) == 80, "operator file header is 80 bytes");
const char kMagic[8] = {'B', 'T', 'T', 'F', 'H', 'A', 'T', '1'};
constexpr size_t kFileChunk = 64u << 20;

}  // namespace

BTT_API btt_status btt_inject_fault(int kind, int count)
{
    g_err.clear();
    if (count < 0) return fail(BTT_ERR_ARG, "btt_inject_fault: count %d < 0", count);
    switch (kind) {
        case BTT_FAULT_NONE: g_fault_alloc = 0; g_fault_launch = 0; return BTT_OK;
        case BTT_FAULT_ALLOC: g_fault_alloc = count; return BTT_OK;
        case BTT_FAULT_LAUNCH: g_fault_launch = count; return BTT_OK;
        default: return fail(BTT_ERR_ARG, "btt_inject_fault: unknown kind %d", kind);
    }
}

BTT_API btt_status btt_save(const btt_op* op, const char* path)
{
    g_err.clear();
    if (!op || !path) return fail(BTT_ERR_ARG, "btt_save: null operator or path");
    FILE* f = fopen(path, "wb");
    if (!f) return fail(BTT_ERR_ARG, "btt_save: cannot open %s for writing", path);
    FileHeader h{};
    memcpy(h.magic, kMagic, 8);
    h.version = 1;
    h.precision = op->prec;
    h.N_t = op->N_t;
    h.N_d = op->N_d;
    h.N_m = op->N_m;
    h.ldm = op->ldm;
    h.fhat_bytes = op->fhat_bytes;
    h.scale_bytes = op->scales ? (uint64_t)op->n_freq * sizeof(float) : 0;
    btt_status s = BTT_OK;
    if (fwrite(&h, sizeof h, 1, f) != 1) s = fail(BTT_ERR_ARG, "btt_save: write failed on %s", path);
    std::vector<char> buf;
    const char* src = static_cast<const char*>(op->fhat);
    for (uint64_t off = 0; s == BTT_OK && off < h.fhat_bytes; off += kFileChunk) {
        const size_t n = (size_t)std::min<uint64_t>(kFileChunk, h.fhat_bytes - off);
        buf.resize(n);
        cudaError_t e = cudaMemcpy(buf.data(), src + off, n, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) s = cuda_fail(e, "btt_save: copy of Fhat");
        else if (fwrite(buf.data(), 1, n, f) != n) s = fail(BTT_ERR_ARG, "btt_save: write failed on %s", path);
    }
    if (s == BTT_OK && h.scale_bytes) {
        buf.resize(h.scale_bytes);
        cudaError_t e = cudaMemcpy(buf.data(), op->scales, h.scale_bytes, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) s = cuda_fail(e, "btt_save: copy of the scales");
        else if (fwrite(buf.data(), 1, h.scale_bytes, f) != h.scale_bytes)
            s = fail(BTT_ERR_ARG, "btt_save: write failed on %s", path);
    }
    if (fclose(f) != 0 && s == BTT_OK) s = fail(BTT_ERR_ARG, "btt_save: close failed on %s", path);
    return s;
}

BTT_API btt_status btt_load(btt_op** out, const char* path, const btt_options* opt_in)
{
    g_err.clear();
    if (!out) return fail(BTT_ERR_ARG, "btt_load: null output handle");
    *out = nullptr;
    if (!path) return fail(BTT_ERR_ARG, "btt_load: null path");
    FILE* f = fopen(path, "rb");
    if (!f) return fail(BTT_ERR_ARG, "btt_load: cannot open %s", path);
    FileHeader h{};
    if (fread(&h, sizeof h, 1, f) != 1 || memcmp(h.magic, kMagic, 8) != 0 || h.version != 1) {
        fclose(f);
        return fail(BTT_ERR_ARG, "btt_load: %s is not an operator file", path);
    }
    const size_t eb = entry_bytes(h.precision);
    const int ldm_want = h.precision == P_FP8S ? (h.N_m + 7) / 8 * 8 : (h.N_m + 3) / 4 * 4;
    const bool scaled = h.precision == P_F16S || h.precision == P_FP8S;
    if (eb == 0 || h.N_t < 1 || h.N_d < 1 || h.N_m < 1 || h.ldm != ldm_want ||
        h.fhat_bytes != (uint64_t)(h.N_t + 1) * h.N_d * h.ldm * eb ||
        h.scale_bytes != (scaled ? (uint64_t)(h.N_t + 1) * sizeof(float) : 0)) {
        fclose(f);
        return fail(BTT_ERR_ARG, "btt_load: inconsistent header in %s", path);
    }
    btt_options opt;
    btt_default_options(&opt);
    if (opt_in) opt = *opt_in;
    opt.precision = (btt_precision)h.precision;   // the file decides the format
    btt_op* op = nullptr;
    btt_status s = op_setup(&op, h.N_t, h.N_d, h.N_m, &opt);
    if (s != BTT_OK) {
        fclose(f);
        return s;
    }
    {
        // the setup's zeroing runs on opt.stream; the copies below do not
        cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(opt.stream));
        if (e != cudaSuccess) s = cuda_fail(e, "btt_load: synchronize");
    }
    std::vector<char> buf;
    char* dst = static_cast<char*>(op->fhat);
    for (uint64_t off = 0; s == BTT_OK && off < h.fhat_bytes; off += kFileChunk) {
        const size_t n = (size_t)std::min<uint64_t>(kFileChunk, h.fhat_bytes - off);
        buf.resize(n);
        if (fread(buf.data(), 1, n, f) != n) s = fail(BTT_ERR_ARG, "btt_load: %s is truncated", path);
        else {
            cudaError_t e = cudaMemcpy(dst + off, buf.data(), n, cudaMemcpyHostToDevice);
            if (e != cudaSuccess) s = cuda_fail(e, "btt_load: copy of Fhat");
        }
    }
    if (s == BTT_OK && h.scale_bytes) {
        buf.resize(h.scale_bytes);
        if (fread(buf.data(), 1, h.scale_bytes, f) != h.scale_bytes)
            s = fail(BTT_ERR_ARG, "btt_load: %s is truncated", path);
        else {
            cudaError_t e = cudaMemcpy(op->scales, buf.data(), h.scale_bytes, cudaMemcpyHostToDevice);
            if (e != cudaSuccess) s = cuda_fail(e, "btt_load: copy of the scales");
        }
    }
    fclose(f);
    if (s == BTT_OK) {
        cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(opt.stream));
        if (e != cudaSuccess) s = cuda_fail(e, "btt_load: synchronize");
    }
    if (s != BTT_OK) {
        free_op(op);
        return s;
    }
    *out = op;
    return BTT_OK;
}

BTT_API btt_status btt_matvec(btt_op* op, const float* m, float* d, int nrhs, void* stream)
{
    g_err.clear();
    btt_status s = check_op(op, false);
    if (s != BTT_OK) return s;
    return run_action<float>(op, A_FWD, m, nullptr, d, nrhs, static_cast<cudaStream_t>(stream));
}

BTT_API btt_status btt_adjoint(btt_op* op, const float* d, float* m, int nrhs, void* stream)
{
    g_err.clear();
    btt_status s = check_op(op, false);
    if (s != BTT_OK) return s;
    return run_action<float>(op, A_ADJ, d, nullptr, m, nrhs, static_cast<cudaStream_t>(stream));
}

namespace {
// y[b][i] = d[b][i] g[i] for nb vectors of n values (Gamma^-1 on data vectors)
__global__ void k_weight(const float* d, const float* __restrict__ g, float* y, int64_t n,
                         bool vec)
{
    const int64_t b = blockIdx.y, T = (int64_t)gridDim.x * blockDim.x;
    const float* db = d + b * n;
    float* yb = y + b * n;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (vec) {
        for (; i < n / 4; i += T) {
            const float4 a = reinterpret_cast<const float4*>(db)[i], w = reinterpret_cast<const float4*>(g)[i];
            reinterpret_cast<float4*>(yb)[i] = make_float4(a.x * w.x, a.y * w.y, a.z * w.z, a.w * w.w);
        }
    } else {
        for (; i < n; i += T) yb[i] = db[i] * g[i];
    }
}
}  // namespace

BTT_API btt_status btt_adjoint_weighted(btt_op* op, const float* d, const float* gamma_inv, float* m, int nrhs,
                                        void* stream)
{
    g_err.clear();
    btt_status s = check_op(op, false);
    if (s != BTT_OK) return s;
    if (!gamma_inv) return run_action<float>(op, A_ADJ, d, nullptr, m, nrhs, static_cast<cudaStream_t>(stream));
    if (nrhs < 0) return fail(BTT_ERR_ARG, "nrhs = %d < 0", nrhs);
    if (nrhs == 0) return BTT_OK;
    if (!d || !m) return fail(BTT_ERR_ARG, "null vector pointer");
    if (take_fault(g_fault_launch)) return fail(BTT_ERR_CUDA, "injected launch failure (nothing was launched)");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int N_t = op->N_t, N_d = op->N_d, N_m = op->N_m;
    const int64_t n = (int64_t)N_t * N_d;
    const float* g = gamma_inv;
    if (!on_device(g)) {
        CK(cudaMemcpyAsync(op->gamma, g, (size_t)n * sizeof(float), cudaMemcpyHostToDevice, st));
        g = static_cast<const float*>(op->gamma);
    }
    const bool d_dev = on_device(d);
    for (int c0 = 0; c0 < nrhs; c0 += op->max_nrhs) {
        const int nb = nrhs - c0 < op->max_nrhs ? nrhs - c0 : op->max_nrhs;
        const float* src = d + (size_t)c0 * n;
        if (!d_dev) {   // host data: copy into the weighting buffer, weight in place
            CK(cudaMemcpyAsync(op->dw, src, (size_t)nb * n * sizeof(float), cudaMemcpyHostToDevice, st));
            src = op->dw;
        }
        const bool vec = (n % 4 == 0) && ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(g)) & 15) == 0;
        const int64_t units = vec ? n / 4 : n;
        const int blocks = (int)std::min<int64_t>((units + 255) / 256, 4 * 152);
        k_weight<<<dim3(blocks, nb), 256, 0, st>>>(src, g, op->dw, n, vec);
        count_launch();
        CK(cudaGetLastError());
        s = run_action<float>(op, A_ADJ, op->dw, nullptr, m + (size_t)c0 * N_t * N_m, nb, st);
        if (s != BTT_OK) return s;
    }
    return BTT_OK;
}

BTT_API btt_status btt_hessian(btt_op* op, const float* m, const float* gamma_inv, float* y, int nrhs,
                               void* stream)
{
    g_err.clear();
    btt_status s = check_op(op, false);
    if (s != BTT_OK) return s;
    return run_action<float>(op, A_HESS, m, gamma_inv, y, nrhs, static_cast<cudaStream_t>(stream));
}

BTT_API btt_status btt_hessian_batched(btt_op* op, const float* const* m, const float* gamma_inv,
                                       float* const* y, int nrhs, void* stream)
{
    g_err.clear();
    btt_status s = check_op(op, false);
    if (s != BTT_OK) return s;
    if (nrhs > 0 && (!m || !y)) return fail(BTT_ERR_ARG, "btt_hessian_batched: null pointer array");
    return run_action<float>(op, A_HESS, nullptr, gamma_inv, nullptr, nrhs, static_cast<cudaStream_t>(stream), m, y);
}

BTT_API btt_status btt_cg(btt_op* op, const float* b, const float* gamma_inv, float alpha, float* x, int nrhs,
                          int max_iter, float tol, int* iterations, float* relres, void* stream)
{
    g_err.clear();
    btt_status s = check_op(op, false);
    if (s != BTT_OK) return s;
    if (nrhs < 0 || max_iter < 0 || !(tol >= 0.f) || !(alpha >= 0.f)) return fail(BTT_ERR_ARG, "btt_cg: bad arguments");
    if (nrhs == 0) return BTT_OK;
    if (!b || !x || !on_device(b) || !on_device(x)) return fail(BTT_ERR_ARG, "btt_cg: b and x must be device pointers");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t n = (int64_t)op->N_t * op->N_m;
    if (op->cg_cap < nrhs) {
        // workspace grows on demand (the only allocation outside btt_create)
        CK(cudaStreamSynchronize(st));
        if (op->cg_vec) cudaFree(op->cg_vec);
        if (op->cg_part) cudaFree(op->cg_part);
        if (op->cg_state) cudaFree(op->cg_state);
        op->cg_vec = nullptr;
        op->cg_part = nullptr;
        op->cg_state = nullptr;
        op->cg_cap = 0;
        btt_status a = alloc((void**)&op->cg_vec, 3 * (size_t)nrhs * n * sizeof(float), "CG vectors");
        const size_t np = cg_partials(nrhs) + (size_t)nrhs * fft_col_blocks(op->N_d, op->geom) +
                          (size_t)nrhs * fft_col_blocks(op->N_m, op->geom);
        if (a == BTT_OK) a = alloc((void**)&op->cg_part, np * sizeof(double), "CG partials");
        if (a == BTT_OK) a = alloc((void**)&op->cg_state, (size_t)nrhs * sizeof(CgVec), "CG scalars");
        if (a != BTT_OK) return a;
        op->cg_cap = nrhs;
    }
    float* r = op->cg_vec;
    float* p = r + (size_t)nrhs * n;
    float* Ap = p + (size_t)nrhs * n;
    double* part = op->cg_part;
    double* mid_part = part + cg_partials(nrhs);   // p.Hp partials of the Hessian's middle step
    const int mid_nblk = fft_col_blocks(op->N_d, op->geom);
    // with a fixed-plan transform length the step runs inside the Hessian's
    // last inverse transform (Hp is never stored); its r.r partials:
    double* step_part = mid_part + (size_t)nrhs * mid_nblk;
    const int step_nblk = fft_col_blocks(op->N_m, op->geom);
    const bool fused = static_plan(op->geom);
    CgVec* cv = op->cg_state;
    std::vector<CgVec> host(nrhs);
    // the host looks at convergence every kCheck iterations (one small copy
    // and a synchronisation); in between, iterations run back to back
    constexpr int kCheck = 8;
    auto any_active = [&](bool* any) -> btt_status {
        CK(cudaMemcpyAsync(host.data(), cv, nrhs * sizeof(CgVec), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        *any = false;
        for (const CgVec& v : host) *any = *any || v.active;
        return BTT_OK;
    };
#define CG(kind, fin, it, xx, pp) CK(launch_cg(kind, fin, it, tol, nrhs, n, x, r, pp, Ap, b, alpha, part, cv, st))
    // r = b - (H + alpha) x, p = r
    CG(CG_DOT_BB, FIN_BB, 0, x, p);
    if ((s = run_action<float>(op, A_HESS, x, gamma_inv, Ap, nrhs, st)) != BTT_OK) return s;
    CG(CG_SHIFT_DOT, FIN_NONE, 0, x, x);
    CG(CG_RESIDUAL, FIN_RS, 0, x, p);
    bool live = false;
    if ((s = any_active(&live)) != BTT_OK) return s;
    for (int it = 1; it <= max_iter && live; ++it) {
        // Ap = H p (its middle step leaves the partials of p.Hp);
        // alpha_j = r_j.r_j / (p_j.Hp_j + alpha p_j.p_j); x += alpha_j p;
        // r -= alpha_j (Hp + alpha p); beta_j = r.r (new) / r.r (old);
        // p = r + beta_j p, with the partials of p.p for the next step
        if (fused) {
            const CgFuse cgf{p, x, r, cv, step_part, n, alpha};
            if ((s = run_action<float>(op, A_HESS, p, gamma_inv, Ap, nrhs, st, nullptr, nullptr, mid_part, &cgf)) !=
                BTT_OK)
                return s;
            CK(launch_cg_finish(step_part, step_nblk, FIN_BETA, it, tol, alpha, nrhs, cv, st));
        } else {
            if ((s = run_action<float>(op, A_HESS, p, gamma_inv, Ap, nrhs, st, nullptr, nullptr, mid_part)) !=
                BTT_OK)
                return s;
            CK(launch_cg_finish(mid_part, mid_nblk, FIN_ALPHA, it, tol, alpha, nrhs, cv, st));
            CG(CG_STEP, FIN_BETA, it, x, p);
        }
        CG(CG_DIRECTION, FIN_PP, it, x, p);
        if (it % kCheck == 0 || it == max_iter)
            if ((s = any_active(&live)) != BTT_OK) return s;
    }
#undef CG
    if (!iterations && !relres) return BTT_OK;
    bool dummy;
    if ((s = any_active(&dummy)) != BTT_OK) return s;
    for (int j = 0; j < nrhs; ++j) {
        if (iterations) iterations[j] = host[j].iters;
        if (relres) relres[j] = host[j].rel;
    }
    return BTT_OK;
}

BTT_API btt_status btt_matvec_f64(btt_op* op, const double* m, double* d, int nrhs, void* stream)
{
    g_err.clear();
    btt_status s = check_op(op, true);
    if (s != BTT_OK) return s;
    return run_action<double>(op, A_FWD, m, nullptr, d, nrhs, static_cast<cudaStream_t>(stream));
}

BTT_API btt_status btt_adjoint_f64(btt_op* op, const double* d, double* m, int nrhs, void* stream)
{
    g_err.clear();
    btt_status s = check_op(op, true);
    if (s != BTT_OK) return s;
    return run_action<double>(op, A_ADJ, d, nullptr, m, nrhs, static_cast<cudaStream_t>(stream));
}

BTT_API btt_status btt_hessian_f64(btt_op* op, const double* m, const double* gamma_inv, double* y,
                                   int nrhs, void* stream)
{
    g_err.clear();
    btt_status s = check_op(op, true);
    if (s != BTT_OK) return s;
    return run_action<double>(op, A_HESS, m, gamma_inv, y, nrhs, static_cast<cudaStream_t>(stream));
}

namespace {
#ifdef BTT_CHECK
// A kernel that tests one index beyond its extent (the access is skipped):
// the record it leaves shows that the checks and their reporting work.
__global__ void k_check_selftest(int* sink, int n)
{
    if (BTT_IN(n, n, CK_SELFTEST)) sink[n] = 1;
}
#endif

const char* site_name(long long s)
{
    static const char* names[CK_NSITES] = {"none", "selftest", "transform shared tile", "transform input row",
                                          "transform output row", "twiddle or position table",
                                          "cluster remote shared memory", "Fhat row or column",
                                          "product spectra", "staged spectra"};
    return s >= 0 && s < CK_NSITES ? names[s] : "unknown";
}

// Collects and clears the first recorded bounds-check failure of every
// translation unit; BTT_OK if none (and always in the normal build).
btt_status check_records()
{
#ifdef BTT_CHECK
    cudaError_t (*units[])(long long*, bool) = {check_record_fft_static, check_record_gemv, check_record_api,
                                                check_record_fft_exchange};
    for (auto u : units) {
        long long rec[3] = {0, 0, 0};
        cudaError_t e = u(rec, true);
        if (e != cudaSuccess) return cuda_fail(e, "reading the bounds-check record");
        if (rec[0] != 0)
            return fail(BTT_ERR_CUDA, "bounds check: %s index %lld outside [0, %lld)", site_name(rec[0]), rec[1],
                        rec[2]);
    }
#endif
    return BTT_OK;
}
}  // namespace

#ifdef BTT_CHECK
namespace btt {
BTT_CHECK_TU(check_record_api)
}  // namespace btt
#endif

BTT_API int btt_check_build(void)
{
#ifdef BTT_CHECK
    return 1;
#else
    return 0;
#endif
}

BTT_API btt_status btt_check_status(void* stream)
{
    g_err.clear();
    CK(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    return check_records();
}

BTT_API btt_status btt_check_selftest(void* stream)
{
    g_err.clear();
#ifdef BTT_CHECK
    k_check_selftest<<<1, 1, 0, static_cast<cudaStream_t>(stream)>>>(nullptr, 7);
    count_launch();
    CK(cudaGetLastError());
    return BTT_OK;
#else
    (void)stream;
    return fail(BTT_ERR_UNSUPPORTED, "btt_check_selftest: this library was built without bounds checks");
#endif
}

BTT_API btt_status btt_device_status(btt_op* op, void* stream)
{
    g_err.clear();
    if (!op) return fail(BTT_ERR_ARG, "btt_device_status: null operator");
    CK(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    int code = 0;
    CK(cudaMemcpy(&code, op->dev_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (code != 0) {
        CK(cudaMemset(op->dev_err, 0, sizeof(int)));
        return fail(BTT_ERR_TIMEOUT, "a bounded device wait ran out (code %d)", code);
    }
    return check_records();
}

BTT_API btt_status btt_selftest_wait(btt_op* op, double seconds, void* stream)
{
    g_err.clear();
    if (!op || seconds <= 0 || seconds > 10) return fail(BTT_ERR_ARG, "btt_selftest_wait: bad arguments");
    CK(launch_wait_selftest(op->dev_err, seconds, static_cast<cudaStream_t>(stream)));
    return btt_device_status(op, stream);
}

BTT_API int btt_precision_of(const btt_op* op) { return op ? op->prec : -1; }

BTT_API btt_status btt_operator_shape(const btt_op* op, int* N_t, int* N_d, int* N_m)
{
    if (!op) return fail(BTT_ERR_ARG, "btt_operator_shape: null operator");
    if (N_t) *N_t = op->N_t;
    if (N_d) *N_d = op->N_d;
    if (N_m) *N_m = op->N_m;
    return BTT_OK;
}

BTT_API size_t btt_operator_bytes(const btt_op* op)
{
    if (!op) return 0;
    return op->fhat_bytes + (op->scales ? op->n_freq * sizeof(float) : 0);
}

BTT_API size_t btt_workspace_bytes(const btt_op* op, int nrhs)
{
    if (!op) return 0;
    if (nrhs <= 0) return op->ws_bytes;
    const int staging = op->staging_nrhs == op->max_nrhs ? nrhs : (op->staging_nrhs < nrhs ? op->staging_nrhs : nrhs);
    return ws_sizes(op->N_t, op->N_d, op->N_m, op->ldm, op->prec, nrhs, staging, op->gemm).total();
}

BTT_API size_t btt_entry_bytes(int precision) { return entry_bytes(precision); }

BTT_API int btt_fhat_ld(const btt_op* op) { return op ? op->ldm : 0; }

BTT_API btt_status btt_copy_fhat(const btt_op* op, void* dst, float* scales)
{
    g_err.clear();
    if (!op || !dst) return fail(BTT_ERR_ARG, "btt_copy_fhat: null argument");
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(dst, op->fhat, op->fhat_bytes, cudaMemcpyDefault));
    if (scales) {
        if (op->scales) {
            CK(cudaMemcpy(scales, op->scales, op->n_freq * sizeof(float), cudaMemcpyDefault));
        } else {
            std::vector<float> one(op->n_freq, 1.0f);
            CK(cudaMemcpy(scales, one.data(), op->n_freq * sizeof(float), cudaMemcpyDefault));
        }
    }
    return BTT_OK;
}

BTT_API btt_status btt_profile_enable(btt_op* op, int on)
{
    g_err.clear();
    if (!op) return fail(BTT_ERR_ARG, "btt_profile_enable: null operator");
    if (on && op->ev.empty()) {
        op->ev.resize(2 * kProfRecords, nullptr);
        for (auto& e : op->ev) CK(cudaEventCreate(&e));
        op->ev_stage.assign(kProfRecords, 0);
    }
    op->prof = on != 0;
    op->ev_used = 0;
    op->ev_dropped = 0;
    return BTT_OK;
}

BTT_API btt_status btt_profile_read(btt_op* op, double* ms, long long* launches)
{
    g_err.clear();
    if (!op || !ms || !launches) return fail(BTT_ERR_ARG, "btt_profile_read: null argument");
    for (int i = 0; i < BTT_NSTAGES; ++i) {
        ms[i] = 0.0;
        launches[i] = 0;
    }
    for (size_t r = 0; r < op->ev_used; ++r) {
        CK(cudaEventSynchronize(op->ev[2 * r + 1]));
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, op->ev[2 * r], op->ev[2 * r + 1]));
        ms[op->ev_stage[r]] += t;
        launches[op->ev_stage[r]] += 1;
    }
    if (op->ev_dropped) return fail(BTT_ERR_ARG, "btt_profile_read: %lld launches were not recorded (more than %zu since the reset)",
                                    op->ev_dropped, kProfRecords);
    op->ev_used = 0;
    return BTT_OK;
}

BTT_API long long btt_launch_count(void) { return btt::g_launches.load(); }

BTT_API const char* btt_last_error(void) { return g_err.c_str(); }

BTT_API const char* btt_version(void) { return "btt 0.1 (sm_103a)"; }
