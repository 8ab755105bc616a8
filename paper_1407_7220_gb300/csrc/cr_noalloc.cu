// cr_noalloc.cu -- KKT residual that allocates no memory of its own.
//
// Some callers cannot allocate device memory at the moment they need this
// check: serving processes that reserve their whole device-memory budget at
// start-up and forbid allocation afterwards, and hot loops that must not call
// cudaMalloc/cudaFree because those calls can synchronize the device.  For them
// cr_kkt_residual_noalloc computes the same metrics as cr_kkt_residual from
// caller-owned device buffers, with its scratch space in a fixed file-scope
// device array instead of an allocation.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "crgpu.h"

namespace {

constexpr long long kMaxRows = 1ll << 16;   // largest N accepted (scratch rows)
constexpr int kTerms = 4;                   // per-row partials: max viol, max comp, sum viol^2, sum theta*g

// Per-row partial sums of the KKT terms.  Every GPU that loads this library holds
// these 2 MiB until the process exits.  All calls share the array: each call
// rewrites rows 0..N-1 before reading them, and calls that overlap on the GPU race.
static __device__ __align__(256) double g_kkt_rows[kMaxRows * kTerms];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
// Device address of g_kkt_rows per device, with the context it was looked up in.  A host
// application that resets the device (cudaDeviceReset) destroys that context and the module
// with it; the next call then runs in a new context and looks the address up again.
struct RowsAddr {
    CUcontext ctx;
    double *ptr;
};
RowsAddr g_rows[kMaxDevices] = {};

// cuCtxGetCurrent through the runtime's driver entry point (no link-time libcuda).
typedef CUresult (*PFN_ctx_get_current)(CUcontext *);
PFN_ctx_get_current ctx_get_current()
{
    static PFN_ctx_get_current fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_ctx_get_current)p;
    }
    return fn;
}

}  // namespace

namespace crk {
void set_thread_error(const std::string &m);   // cr_last_error(NULL) reports it (crgpu.cu)
}

namespace {

cr_status err(cr_status s, const std::string &m)
{
    crk::set_thread_error(m);
    return s;
}

// One warp per row l1: (C eta)_p over l2 != l1 in FP64, plus the y >= 0 row of l1.
__global__ void k_rows(long long N, int n, const float *__restrict__ theta, long long ld, const double *__restrict__ X,
                       const double *__restrict__ y, const double *__restrict__ xi, const double *__restrict__ mu,
                       double *__restrict__ rows)
{
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long l1 = warp; l1 < N; l1 += nwarps) {
        double mv = 0.0, mc = 0.0, s2 = 0.0, tg = 0.0;
        for (long long l2 = lane; l2 < N; l2 += 32) {
            if (l2 == l1) continue;
            double g = y[l1] - y[l2];
            for (int k = 0; k < n; ++k) g -= xi[l2 * n + k] * (X[l1 * n + k] - X[l2 * n + k]);
            const double th = (double)theta[l1 * ld + l2];
            mv = fmax(mv, -g);
            mc = fmax(mc, th * fabs(g));
            if (g < 0.0) s2 += g * g;
            tg += th * g;
        }
        for (int o = 16; o > 0; o >>= 1) {
            mv = fmax(mv, __shfl_xor_sync(0xffffffffu, mv, o));
            mc = fmax(mc, __shfl_xor_sync(0xffffffffu, mc, o));
            s2 += __shfl_xor_sync(0xffffffffu, s2, o);
            tg += __shfl_xor_sync(0xffffffffu, tg, o);
        }
        if (lane == 0) {
            const double yl = y[l1], ml = mu ? mu[l1] : 0.0;
            mv = fmax(mv, -yl);
            mc = fmax(mc, ml * fabs(yl));
            if (yl < 0.0) s2 += yl * yl;
            tg += ml * yl;
            rows[l1 * kTerms + 0] = mv;
            rows[l1 * kTerms + 1] = mc;
            rows[l1 * kTerms + 2] = s2;
            rows[l1 * kTerms + 3] = tg;
        }
    }
}

// One CTA: rows 0..N-1 combined in a fixed order (deterministic), then the metrics.
__global__ void k_final(long long N, const double *__restrict__ rows, double sigma, double *__restrict__ out)
{
    __shared__ double red[32][kTerms];
    double mv = 0.0, mc = 0.0, s2 = 0.0, tg = 0.0;
    for (long long l = threadIdx.x; l < N; l += blockDim.x) {
        mv = fmax(mv, rows[l * kTerms + 0]);
        mc = fmax(mc, rows[l * kTerms + 1]);
        s2 += rows[l * kTerms + 2];
        tg += rows[l * kTerms + 3];
    }
    for (int o = 16; o > 0; o >>= 1) {
        mv = fmax(mv, __shfl_xor_sync(0xffffffffu, mv, o));
        mc = fmax(mc, __shfl_xor_sync(0xffffffffu, mc, o));
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        tg += __shfl_xor_sync(0xffffffffu, tg, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        red[w][0] = mv;
        red[w][1] = mc;
        red[w][2] = s2;
        red[w][3] = tg;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < (int)(blockDim.x >> 5); ++i) {
            mv = fmax(mv, red[i][0]);
            mc = fmax(mc, red[i][1]);
            s2 += red[i][2];
            tg += red[i][3];
        }
        const double np = (double)N * (double)(N - 1);
        const double pri = mv / sigma, comp = mc / (sigma * sigma);
        out[0] = fmax(pri, comp);
        out[1] = pri;
        out[2] = comp;
        out[3] = sqrt(s2) / sqrt(np);
        out[4] = tg / np;
    }
}

}  // namespace

extern "C" cr_status cr_kkt_residual_noalloc(int64_t N, int32_t n, const float *dtheta, int64_t ld, const double *dX,
                                             const double *dy, const double *dxi, const double *dmu, double sigma,
                                             void *stream, double *dout)
{
    if (N < 2 || n < 1 || !dtheta || !dX || !dy || !dxi || !dout || ld < N || !(sigma > 0.0))
        return err(CR_EINVAL, "cr_kkt_residual_noalloc: need N >= 2, n >= 1, ld >= N, sigma > 0 and non-NULL buffers");
    if (N > kMaxRows)
        return err(CR_EINVAL, "cr_kkt_residual_noalloc: N = " + std::to_string((long long)N) +
                                  " exceeds the fixed scratch of " + std::to_string(kMaxRows) + " rows");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return err(CR_ECUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return err(CR_EINVAL, "cr_kkt_residual_noalloc: device index out of range");
    double *rows = nullptr;
    {
        // set-up, once per device (and again if the device's context was replaced): look up the
        // device address of the scratch array with this device current.  With lazy module
        // loading this first lookup also loads the library's module and its 2 MiB array.
        // Calls from several threads are serialized by the lock.
        std::lock_guard<std::mutex> lk(g_mu);
        PFN_ctx_get_current get = ctx_get_current();
        if (!get) return err(CR_ECUDA, "cr_kkt_residual_noalloc: cuCtxGetCurrent is not available from the driver");
        CUcontext ctx = nullptr;
        if (get(&ctx) != CUDA_SUCCESS) ctx = nullptr;
        if (!ctx || !g_rows[dev].ptr || g_rows[dev].ctx != ctx) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_kkt_rows);   // also makes the device's context current
            if (e != cudaSuccess) return err(CR_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            if (get(&ctx) != CUDA_SUCCESS || !ctx)
                return err(CR_ECUDA, "cr_kkt_residual_noalloc: no current CUDA context");
            g_rows[dev].ptr = (double *)p;
            g_rows[dev].ctx = ctx;
        }
        rows = g_rows[dev].ptr;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return err(CR_ECUDA, cudaGetErrorString(e));
    const long long warps = N < (long long)sms * 64 ? N : (long long)sms * 64;
    const int threads = 256;
    const int blocks = (int)((warps * 32 + threads - 1) / threads);
    k_rows<<<blocks, threads, 0, s>>>(N, n, dtheta, ld, dX, dy, dxi, dmu, rows);
    k_final<<<1, 1024, 0, s>>>(N, rows, sigma, dout);
    e = cudaGetLastError();
    if (e != cudaSuccess) return err(CR_ECUDA, cudaGetErrorString(e));
    crk::set_thread_error("");
    return CR_OK;
}
