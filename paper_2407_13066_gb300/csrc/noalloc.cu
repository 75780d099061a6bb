// btt_matvec_noalloc: the F action (pad + DFT, per-frequency product,
// inverse DFT + unpad) for callers that cannot allocate device memory.
//
// Some callers may not call cudaMalloc at the point where they apply the
// operator: a custom call inside another framework's compiled step (XLA or
// a similar runtime hands it every buffer and owns all device memory), an
// inference-server plugin confined to a preallocated arena, or a real-time
// loop that forbids allocation after start-up because an allocation can
// synchronise the device or fail under a memory cap.  Such a caller keeps
// Fhat in a buffer it owns (for example filled once by btt_copy_fhat) and
// passes it in with m and d.  The spectra mhat and dhat and the FFT tables
// that the action needs as scratch come from one file-scope device array of
// fixed size instead of a workspace.
#include <cstdint>
#include <cstdio>
#include <mutex>

#include "../../include/btt.h"
#include "kernels.h"

#define BTT_API extern "C" __attribute__((visibility("default")))

namespace btt {
void set_last_error(const char* msg);  // api.cu: the text btt_last_error() returns
}

// Fixed scratch for btt_matvec_noalloc (BTT_NOALLOC_SCRATCH_BYTES = 32 MiB).
// Every GPU that loads this part of the library holds it until the process
// exits.  In host code the name is only a host-side stand-in: the device
// address is looked up with cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[BTT_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr size_t kNoAllocScratchBytes = BTT_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

// Device address of g_noalloc_scratch per device, looked up once per device
// (with that device current) by the first call on it.
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

__global__ void k_noalloc_tables(float2* tw, int* pos, btt::FftPlan plan)
{
    const int L = plan.L;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < L; e += gridDim.x * blockDim.x) {
        double s, c;
        sincospi(2.0 * (double)e / (double)L, &s, &c);
        tw[e] = make_float2((float)c, (float)-s);
        // the quad copy (c, c, d, d) the fixed-plan transforms read after the L entries
        tw[L + 2 * e] = make_float2((float)c, (float)c);
        tw[L + 2 * e + 1] = make_float2((float)-s, (float)-s);
        // the lane-pair entries of the one-exchange transforms (L = R1 N2,
        // R1 = min(32, L / 16), entry n2 R1/2 + m)
        if (L % 32 == 0 && e < L / 2) {
            const int H = L >= 512 ? 16 : L / 32, n2 = e / H, m = e % H;
            double sa, ca, sb, cb;
            sincospi(2.0 * (double)(2 * m * n2) / (double)L, &sa, &ca);
            sincospi(2.0 * (double)((2 * m + 1) * n2) / (double)L, &sb, &cb);
            tw[3 * L + 2 * e] = make_float2(0.5f * (float)ca, 0.5f * (float)cb);   // halved (exact)
            tw[3 * L + 2 * e + 1] = make_float2(-0.5f * (float)sa, -0.5f * (float)sb);
        }
        int rem = e, prod = 1, at = 0;
        for (int p = 0; p < plan.nstages; ++p) {
            const int R = plan.radix[p];
            const int dgt = rem % R;
            rem /= R;
            prod *= R;
            at += dgt * (L / prod);
        }
        pos[e] = at;
    }
}

btt_status fail(btt_status s, const char* msg)
{
    char buf[320];
    snprintf(buf, sizeof buf, "btt_matvec_noalloc: %s", msg);
    btt::set_last_error(buf);
    return s;
}

}  // namespace

BTT_API btt_status btt_matvec_noalloc(const void* fhat, int N_t, int N_d, int N_m, const float* m,
                                      float* d, int nrhs, void* stream)
{
    btt::set_last_error("");
    if (!fhat || !m || !d) return fail(BTT_ERR_ARG, "null pointer");
    if (reinterpret_cast<uintptr_t>(fhat) % 16 != 0) return fail(BTT_ERR_ARG, "fhat must be 16-byte aligned");
    if (N_t < 1 || N_d < 1 || N_m < 1 || nrhs < 0) return fail(BTT_ERR_ARG, "sizes must be >= 1, nrhs >= 0");
    if (nrhs == 0) return BTT_OK;
    // limits of the launches below, checked before anything is enqueued:
    // the vectors index grid.y of the transforms, and N_d N_m elements of one
    // frequency slice are addressed with 32-bit offsets (as btt_create requires)
    if (nrhs > 65535) return fail(BTT_ERR_UNSUPPORTED, "nrhs must be <= 65535 (one transform grid row per vector)");
    if ((int64_t)N_d * N_m > 2147483647LL) return fail(BTT_ERR_UNSUPPORTED, "N_d * N_m must be <= 2^31 - 1");
    btt::FftGeom geom;
    if (!btt::make_fft_geom(N_t, &geom))
        return fail(BTT_ERR_UNSUPPORTED, "2*N_t must factor into 2,3,5,7 and be <= 24576");

    // scratch layout: twiddles [L] float2 + [L] quads + [L/2] lane pairs | pos [L] int | mhat | dhat
    const int ldm = (N_m + 3) / 4 * 4;
    const int nf = N_t + 1;
    const size_t tw_b = (size_t)geom.L * 2 * sizeof(float4);
    const size_t pos_b = ((size_t)geom.L * sizeof(int) + 255) / 256 * 256;
    const size_t xh_b = ((size_t)nrhs * nf * ldm * sizeof(float2) + 255) / 256 * 256;
    const size_t dh_b = (size_t)nrhs * nf * N_d * sizeof(float2);
    const size_t need = tw_b + pos_b + xh_b + dh_b;
    if (need > kNoAllocScratchBytes) {
        char buf[256];
        snprintf(buf, sizeof buf,
                 "needs %zu bytes of scratch for N_t=%d N_d=%d N_m=%d nrhs=%d, more than its fixed "
                 "%zu; use btt_matvec with an operator",
                 need, N_t, N_d, N_m, nrhs, kNoAllocScratchBytes);
        return fail(BTT_ERR_UNSUPPORTED, buf);
    }

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(BTT_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(BTT_ERR_UNSUPPORTED, "device index beyond 63");
    unsigned char* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_scratch_ptr[dev]) {
            // first call on this device: resolve the array's device address
            // and set the kernels' shared-memory limits
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) return fail(BTT_ERR_CUDA, cudaGetErrorString(e));
            e = btt::prepare_kernels();
            if (e != cudaSuccess) return fail(BTT_ERR_CUDA, cudaGetErrorString(e));
            g_scratch_ptr[dev] = p;
        }
        base = static_cast<unsigned char*>(g_scratch_ptr[dev]);
    }
    float2* tw = reinterpret_cast<float2*>(base);
    int* pos = reinterpret_cast<int*>(base + tw_b);
    float2* xh = reinterpret_cast<float2*>(base + tw_b + pos_b);
    float2* dh = reinterpret_cast<float2*>(base + tw_b + pos_b + xh_b);
    geom.pos = pos;
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    // the array keeps the previous call's contents: rebuild the tables and
    // zero mhat (its padding columns l >= N_m are read as zeros)
    k_noalloc_tables<<<(geom.L + 255) / 256, 256, 0, st>>>(tw, pos, geom.plan);
    btt::count_launch();
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemsetAsync(xh, 0, xh_b, st);
    const int64_t xbs = (int64_t)nf * ldm, dbs = (int64_t)nf * N_d;
    if (e == cudaSuccess)
        e = btt::launch_rfft<float>(m, N_m, (int64_t)N_t * N_m, N_m, xh, ldm, xbs, nrhs, geom, tw, st);
    if (e == cudaSuccess)
        e = btt::launch_gemv_fwd(btt::P_F32, fhat, nullptr, nf, N_d, ldm, xh, xbs, dh, dbs, nrhs, st);
    if (e == cudaSuccess)
        e = btt::launch_irfft<float>(dh, N_d, dbs, N_d, d, N_d, (int64_t)N_t * N_d, nullptr, nrhs, geom, tw, st);
    if (e != cudaSuccess) return fail(BTT_ERR_CUDA, cudaGetErrorString(e));
    return BTT_OK;
}
