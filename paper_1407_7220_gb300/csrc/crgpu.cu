// crgpu.cu -- host side of the C ABI declared in include/crgpu.h.
//
// Owns the device buffers of one instance, computes the problem constants
// (shift s, step constant L_g of Eq. (eq:lischitz)) in FP64 on the host, and
// drives the iteration either as one cooperative persistent launch per call or
// as one launch per phase.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <limits>
#include <new>
#include <string>
#include <vector>

#include "cr_alcc.cuh"
#include "cr_launch.cuh"
#include "crgpu.h"

namespace crk {
// Widening copy of a stored multiplier array to FP32 (exact: every BF16 value and every FP16
// value times its power-of-two scale is an FP32 number).
__global__ void k_widen_bf16(const __nv_bfloat16 *in, float *out, size_t count)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
        out[i] = __bfloat162float(in[i]);
}
__global__ void k_widen_f16(const __half *in, float *out, size_t count, float inv_scale)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
        out[i] = __half2float(in[i]) * inv_scale;
}

__global__ void k_bwd_finish(long long N, int n, const float *ubar, const double *ybar_acc, const double *X_acc,
                             float *dybar, float *dX)
{
    for (long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x; l < N; l += (long long)gridDim.x * blockDim.x) {
        dybar[l] = (float)((double)ubar[l] + ybar_acc[l]);   // yhat = ybar + A_1^T theta + mu
        for (int k = 0; k < n; ++k) dX[l * n + k] = (float)X_acc[l * n + k];
    }
}
}  // namespace crk

using crk::DevState;
using crk::KernelSet;
using crk::Params;

struct cr_ctx {
    cr_options opt;
    int device = 0;
    int num_sms = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    long long N = 0;
    int n = 0;
    int NP = 0;
    long long ld = 0;
    double sigma = 1.0;
    long long iters = 0;     // iterations completed (host view)
    bool persistent_ok = false;
    bool prepared = false;   // foldB of iteration iters + 1 already performed (fused into foldA)
    KernelSet ks{};
    Params P{};
    std::vector<void *> allocs;
    std::string err;
    bool broken = false;     // a device-side wait timed out; only reset/destroy are valid
    // profiling (cr_options.profile): events around launches, summed per kind on cr_profile
    struct Ev {
        int kind;
        cudaEvent_t a, b;
    };
    std::vector<Ev> evs;
    std::vector<cudaEvent_t> pool;
    double prof_ms[4] = {0, 0, 0, 0};
    long long prof_n[4] = {0, 0, 0, 0};
    // differentiation: checkpoints every record_every iterations (cr_options.reserved[0])
    struct Checkpoint {
        long long iter = -1;
        void *th[2] = {nullptr, nullptr};
        double *v[2] = {nullptr, nullptr}, *w[2] = {nullptr, nullptr}, *mu[2] = {nullptr, nullptr};
        double *dd[2] = {nullptr, nullptr};
        DevState st;
        // full snapshots also keep the minimizer at theta^(1) and the fold partials
        bool full = false;
        double *y1 = nullptr, *xi1_64 = nullptr, *foldpart = nullptr;
        float *yrow1 = nullptr, *ccol1 = nullptr, *xi1 = nullptr;
    };
    int record_every = 0;
    std::vector<Checkpoint> ckpt;       // at iterations 0, k, 2k, ...
    std::vector<void *> ckpt_allocs;
    std::vector<void *> bwd_allocs;     // reverse-mode workspace (lazily allocated)
    // ALCC handles (cr_alcc_create): kernel, constants and the schedule of Fig. `fig:alcc`
    bool alcc = false;
    cr_alcc_options aopt{};
    crk::AlccKernel ak{};
    double a_s2a1 = 0.0, a_s2a2 = 0.0, a_By = 0.0, a_Bxi = 0.0;
    double a_mu = 0.0, a_tau = 0.0, a_alpha_y = 0.0, a_alpha_xi = 0.0;
    long long a_inner_total = 0;
    bool a_have_metrics = false;
    double a_metrics[4] = {0, 0, 0, 0};
    std::vector<float> a_rec0, a_ccol0;   // column data of (y_0, xi_0) = (ybar, 0)
    std::vector<double> a_ccol64;         // the same column values xi.x - y in FP64 (of the point ay2 holds)
    // P-APG with K blocks (cr_blocks_*): this handle holds the outer dual (pairs between blocks,
    // y >= 0 rows); `inner` the pairs inside the blocks (Step 1 by inner P-APG)
    bool blocks = false;
    cr_ctx *inner = nullptr;
    int inner_iters = 0;
    int K = 0;
    double *b_a = nullptr, *b_b = nullptr, *b_mu2 = nullptr;   // a, b of Step 1's block problems; mu^(2)
    std::vector<long long> perm;      // handle order q holds the caller's point perm[q] (sorted by block)
};

namespace {

const char *cr_status_str_impl(cr_status s)
{
    switch (s) {
    case CR_OK: return "ok";
    case CR_NOT_CONVERGED: return "not converged (max_iter reached)";
    case CR_EINVAL: return "invalid argument";
    case CR_ENOMEM: return "out of memory";
    case CR_ECUDA: return "CUDA error";
    case CR_ETIMEOUT: return "bounded device wait timed out";
    case CR_ENUMERIC: return "non-finite value in the iteration";
    case CR_ESTATE: return "invalid handle state";
    }
    return "unknown status";
}

cr_status fail(cr_ctx *h, cr_status s, const char *fmt, ...)
{
    if (h) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        h->err = buf;
    }
    return s;
}

#define CR_CUDA(h, call)                                                                     \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess) {                                                             \
            if (e_ == cudaErrorMemoryAllocation) return fail(h, CR_ENOMEM, "%s: %s", #call, cudaGetErrorString(e_)); \
            return fail(h, CR_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));                \
        }                                                                                    \
    } while (0)

int padded_n(int n)
{
    static const int list[] = {2, 4, 5, 8, 10, 16, 20, 32};
    for (int v : list)
        if (n <= v) return v;
    return 0;
}

KernelSet kernels_for(int dtype, int NP)
{
    switch (dtype) {
    case CR_THETA_F32: return crk::kernels_f32(NP);
    case CR_THETA_BF16: return crk::kernels_bf16(NP);
    case CR_THETA_F16: return crk::kernels_f16(NP);
    case CR_THETA_F64: return crk::kernels_f64(NP);
    default: return KernelSet{};
    }
}

size_t theta_elem_size(int dtype) { return dtype == CR_THETA_F64 ? 8 : dtype == CR_THETA_F32 ? 4 : 2; }

int rec_floats(int NP) { return ((NP + 1 + 3) / 4) * 4; }

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link-time libcuda).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// ---- problem constants (host, FP64) ----------------------------------------

// Observation shift (the paragraph after Eq. (omega_primal) asks only for "a
// sufficiently large quantity"): s = max(0, -min ybar) + (max ybar - min ybar).
double default_shift(const std::vector<double> &yb)
{
    double lo = yb[0], hi = yb[0];
    for (double v : yb) {
        lo = std::min(lo, v);
        hi = std::max(hi, v);
    }
    return std::max(0.0, -lo) + (hi - lo);
}

// Eigen-decomposition of a symmetric n x n matrix by cyclic Jacobi rotations with
// accumulated eigenvectors (columns of V).  a is overwritten; eigenvalues on its diagonal.
void sym_eig(std::vector<double> &a, std::vector<double> &V, int n)
{
    V.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
    for (int sweep = 0; sweep < 64; ++sweep) {
        double off = 0.0, diag = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) (i == j ? diag : off) += a[(size_t)i * n + j] * a[(size_t)i * n + j];
        if (off <= 1e-32 * std::max(diag, 1e-300)) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = a[(size_t)p * n + q];
                if (apq == 0.0) continue;
                const double theta = (a[(size_t)q * n + q] - a[(size_t)p * n + p]) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {  // columns p, q
                    const double kp = a[(size_t)k * n + p], kq = a[(size_t)k * n + q];
                    a[(size_t)k * n + p] = c * kp - s * kq;
                    a[(size_t)k * n + q] = s * kp + c * kq;
                }
                for (int k = 0; k < n; ++k) {  // rows p, q
                    const double pk = a[(size_t)p * n + k], qk = a[(size_t)q * n + k];
                    a[(size_t)p * n + k] = c * pk - s * qk;
                    a[(size_t)q * n + k] = s * pk + c * qk;
                }
                for (int k = 0; k < n; ++k) {
                    const double kp = V[(size_t)k * n + p], kq = V[(size_t)k * n + q];
                    V[(size_t)k * n + p] = c * kp - s * kq;
                    V[(size_t)k * n + q] = s * kp + c * kq;
                }
            }
    }
}

// ||A_2||^2 = max_l lambda_max(M_l), M_l = sum_m (x_m - x_l)(x_m - x_l)^T (A_2^T A_2 is block
// diagonal with blocks M_l).  M_l = N (Sigma + v v^T) with Sigma the population covariance
// and v = xbar - x_l, so with Sigma = Q diag(lam) Q^T the largest eigenvalue is the largest
// root of the secular equation 1 = sum_i z_i^2 / (mu - lam_i), z = Q^T v, which lies in
// [max lam, max lam + ||z||^2]; it is found by bisection.
double max_block_eig(const std::vector<double> &X, long long N, int n)
{
    std::vector<double> mean(n, 0.0), cov((size_t)n * n, 0.0), V;
    for (long long l = 0; l < N; ++l)
        for (int k = 0; k < n; ++k) mean[k] += X[(size_t)l * n + k];
    for (int k = 0; k < n; ++k) mean[k] /= (double)N;
    for (long long l = 0; l < N; ++l)
        for (int i = 0; i < n; ++i) {
            const double di = X[(size_t)l * n + i] - mean[i];
            for (int j = i; j < n; ++j) cov[(size_t)i * n + j] += di * (X[(size_t)l * n + j] - mean[j]);
        }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < i; ++j) cov[(size_t)i * n + j] = cov[(size_t)j * n + i];   // the same sums
    for (double &c : cov) c /= (double)N;
    sym_eig(cov, V, n);
    std::vector<double> lam(n), z(n);
    double lmax = -std::numeric_limits<double>::infinity();
    for (int i = 0; i < n; ++i) {
        lam[i] = cov[(size_t)i * n + i];
        lmax = std::max(lmax, lam[i]);
    }
    // The bisection only shrinks the bracket, so N (lmax + ||z||^2) bounds a point's result from
    // above; ||z|| = ||xbar - x_l|| (Q is orthogonal), taken directly and enlarged by 1e-12 to
    // cover its rounding.  The point with the largest bound is solved first, then every point
    // whose bound reaches the largest root found so far: the maximum is the same, bit for bit,
    // as over every point.
    auto zvec = [&](long long l) {
        double zz = 0.0;
        for (int i = 0; i < n; ++i) {
            double s = 0.0;
            for (int k = 0; k < n; ++k) s += V[(size_t)k * n + i] * (mean[k] - X[(size_t)l * n + k]);
            z[i] = s;
            zz += s * s;
        }
        return zz;
    };
    std::vector<double> zzs((size_t)N);
    long long l0 = 0;
    for (long long l = 0; l < N; ++l) {
        double dd = 0.0;
        for (int k = 0; k < n; ++k) {
            const double d = mean[k] - X[(size_t)l * n + k];
            dd += d * d;
        }
        zzs[(size_t)l] = dd * (1.0 + 1e-12);
        if (zzs[(size_t)l] > zzs[(size_t)l0]) l0 = l;
    }
    double best = 0.0;
    for (long long j = -1; j < N; ++j) {
        const long long l = j < 0 ? l0 : j;
        if ((j >= 0 && l == l0) || (double)N * (lmax + zzs[(size_t)l]) < best) continue;
        const double zz = zvec(l);
        double lo = lmax, hi = lmax + zz;
        for (int it = 0; it < 200 && hi > lo; ++it) {
            const double mid = 0.5 * (lo + hi);
            if (mid <= lo || mid >= hi) break;
            double f = 1.0;
            for (int i = 0; i < n; ++i) f -= z[i] * z[i] / (mid - lam[i]);
            (f < 0.0 ? lo : hi) = mid;
        }
        best = std::max(best, (double)N * hi);
    }
    return best;
}

bool all_finite(const double *a, size_t k)
{
    for (size_t i = 0; i < k; ++i)
        if (!std::isfinite(a[i])) return false;
    return true;
}

template <typename T> cr_status dev_alloc(cr_ctx *h, T **p, size_t count)
{
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(h, CR_ENOMEM, "cudaMalloc(%zu bytes): %s", count * sizeof(T), cudaGetErrorString(e));
    }
    h->allocs.push_back(q);
    *p = (T *)q;
    return CR_OK;
}

#define CR_TRY(x)                          \
    do {                                   \
        cr_status s_ = (x);                \
        if (s_ != CR_OK) return s_;        \
    } while (0)

// First unit of CTA c (the device's unit_begin): an even split, rounded down to an 8-row
// boundary inside the stripe.
long long unit_begin_host(long long c, long long total, long long N, int G)
{
    const long long u = (long long)(((unsigned long long)c * total) / G);
    const long long s = u / N;
    return s * N + ((u - s * N) & ~7ll);
}

// Entries of the partition table for a grid of up to G CTAs over S stripes.
size_t partition_entries(long long G, long long S) { return (size_t)(2 * G + 1 + 2 * S); }

// The device's partition table (capacity partition_entries(G at creation, S)):
//   ubeg[c], c = 0..G: first unit of CTA c;
//   cfs[c], c < G: first stripe of CTA c, or -1 for a CTA without units;
//   sc0[s], sc1[s], s < S: the CTAs [sc0, sc1) whose unit ranges meet stripe s (the folds add
//   their column partials in this ascending order).
cr_status upload_partition(cr_ctx *h, long long *dtab, const std::vector<long long> *ubeg = nullptr)
{
    Params &P = h->P;
    const long long G = P.G, N = P.N, S = P.S;
    std::vector<long long> t(partition_entries(G, S), 0);
    long long *ub = t.data(), *cfs = ub + G + 1, *sc0 = cfs + G, *sc1 = sc0 + S;
    for (long long c = 0; c <= G; ++c) ub[c] = ubeg ? (*ubeg)[c] : unit_begin_host(c, P.total, N, (int)G);
    for (long long s = 0; s < S; ++s) {
        sc0[s] = G;
        sc1[s] = 0;
    }
    for (long long c = 0; c < G; ++c) {
        if (ub[c + 1] <= ub[c]) {
            cfs[c] = -1;
            continue;
        }
        cfs[c] = ub[c] / N;
        const long long sl = (ub[c + 1] - 1) / N;
        for (long long s = cfs[c]; s <= sl; ++s) {
            sc0[s] = std::min(sc0[s], c);
            sc1[s] = std::max(sc1[s], c + 1);
        }
    }
    CR_CUDA(h, cudaMemcpy(dtab, t.data(), sizeof(long long) * t.size(), cudaMemcpyHostToDevice));
    P.ubeg = dtab;
    P.cfs = dtab + G + 1;
    P.sc0 = P.cfs + G;
    P.sc1 = P.sc0 + S;
    return CR_OK;
}

// Work partition of the pair pass: the number of column-partial slots per CTA.
int max_slots(long long total, long long N, int G)
{
    int best = 1;
    for (long long c = 0; c < G; ++c) {
        long long u0 = unit_begin_host(c, total, N, G);
        long long u1 = unit_begin_host(c + 1, total, N, G);
        if (u1 <= u0) continue;
        best = std::max(best, (int)((u1 - 1) / N - u0 / N + 1));
    }
    return best;
}

cudaEvent_t take_event(cr_ctx *h)
{
    if (!h->pool.empty()) {
        cudaEvent_t e = h->pool.back();
        h->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Events bracketing one launch of the given kind (profile option only).
struct ProfScope {
    cr_ctx *h;
    int kind;
    cudaEvent_t a = nullptr, b = nullptr;
    ProfScope(cr_ctx *h_, int kind_) : h(h_), kind(kind_)
    {
        if (!h->opt.profile) return;
        a = take_event(h);
        b = take_event(h);
        if (a) cudaEventRecord(a, h->stream);
    }
    ~ProfScope()
    {
        if (!a || !b) return;
        cudaEventRecord(b, h->stream);
        h->evs.push_back({kind, a, b});
    }
};

int phase_kind(int phase)
{
    if (phase == crk::PH_PAIR || phase == crk::PH_BALL_NORM || phase == crk::PH_BALL_SCALE) return 0;
    if (phase == crk::PH_FOLDA || phase == crk::PH_FOLDB) return 1;
    return 2;
}

cr_status launch_phase(cr_ctx *h, int phase, long long ell, double tol, int grid = -1, int fold_stats = 1)
{
    Params P = h->P;
    P.fold_stats = fold_stats;
    void *args[] = {&P, &phase, &ell, &tol, &h->sigma};
    const int g = grid > 0 ? grid : h->P.G;
    ProfScope ps(h, phase_kind(phase));
    if (phase == crk::PH_PAIR && h->P.tc) {
        void *targs[] = {&P, &ell};
        CR_CUDA(h, cudaLaunchKernel(h->ks.pair_tc, dim3(g), dim3(crk::kTcThreads), targs, h->ks.smem, h->stream));
        return CR_OK;
    }
    // programmatic dependent launch: k_phase waits (griddepcontrol.wait) for the previous grid
    // before it reads anything, so its launch may overlap the previous kernel's drain
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(g);
    cfg.blockDim = dim3(crk::kThreads);
    cfg.dynamicSmemBytes = h->ks.smem;
    cfg.stream = h->stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    CR_CUDA(h, cudaLaunchKernelExC(&cfg, h->ks.phase, args));
    if (phase == crk::PH_FOLDA) h->prepared = h->P.fuse != 0;
    else if (phase == crk::PH_FOLDB) h->prepared = false;
    return CR_OK;
}

cr_status launch_persistent(cr_ctx *h, long long ell0, long long ell1, int check_every, double tol)
{
    CR_CUDA(h, cudaMemsetAsync(&h->P.st->bar_count, 0, sizeof(unsigned long long), h->stream));
    Params P = h->P;
    int first_foldB = h->prepared ? 0 : 1;
    void *args[] = {&P, &ell0, &ell1, &check_every, &tol, &h->sigma, &first_foldB};
    ProfScope ps(h, 3);
    CR_CUDA(h, cudaLaunchCooperativeKernel(h->ks.persistent, dim3(h->P.G), dim3(crk::kThreads), args, h->ks.smem,
                                           h->stream));
    h->prepared = h->P.fuse != 0;   // its last foldA performed the next foldB
    return CR_OK;
}

// Iterations ell0..ell1 through the per-phase kernels; checks as in the persistent driver.
cr_status run_phases(cr_ctx *h, long long ell0, long long ell1, int check_every, double tol)
{
    for (long long ell = ell0; ell <= ell1; ++ell) {
        const bool check = check_every > 0 && ((ell % check_every) == 0 || ell == ell1);
        // the objective and y >= 0 partial sums: every iteration without P.fuse (the restart test
        // of foldB reads them), else where a check or the caller (cr_objective) reads them
        const int stats = (!h->P.fuse || check || ell == ell1) ? 1 : 0;
        if (!h->prepared) CR_TRY(launch_phase(h, crk::PH_FOLDB, ell, tol));
        CR_TRY(launch_phase(h, crk::PH_PAIR, ell, tol));
        if (h->P.ball) CR_TRY(launch_phase(h, crk::PH_BALL_NORM, ell, tol));
        CR_TRY(launch_phase(h, crk::PH_FOLDA, ell, tol, -1, stats));   // with P.fuse also foldB(ell + 1)
        if (h->P.ball) CR_TRY(launch_phase(h, crk::PH_BALL_SCALE, ell, tol));
        if (check) {
            CR_TRY(launch_phase(h, crk::PH_KKT32, ell, tol));
            CR_TRY(launch_phase(h, crk::PH_DECIDE32, ell, tol, 1));
            Params P = h->P;
            void *args[] = {&P, &ell};
            ProfScope ps(h, 2);
            CR_CUDA(h, cudaLaunchKernel(h->ks.kkt64_if, dim3(h->P.G), dim3(crk::kThreads), args, 0, h->stream));
            CR_TRY(launch_phase(h, crk::PH_DECIDE64, ell, tol, 1));
        }
    }
    return CR_OK;
}

cr_status read_state(cr_ctx *h, DevState *st)
{
    CR_CUDA(h, cudaMemcpyAsync(st, h->P.st, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream));
    CR_CUDA(h, cudaStreamSynchronize(h->stream));
    if (st->error == crk::ERR_BARRIER) {
        h->broken = true;
        return fail(h, CR_ETIMEOUT, "a grid barrier wait exceeded its bound");
    }
    if (st->error == crk::ERR_NUMERIC) return fail(h, CR_ENUMERIC, "non-finite value in the iteration");
    return CR_OK;
}

// Tensor-core operands that do not change: X rows (B of the residual product) and [X | 1]
// transposed (B of the adjoint product), TF32 hi/lo, in 8-row blocks of the canonical K-major
// layout (see cr_pair_tc.cuh); one group of zero padding past the last row.  The Xi array is
// zeroed here and written by every foldB.
float tf32_round_host(float x)
{
    // round to nearest, ties away from zero, to 10 explicit mantissa bits (finite inputs)
    uint32_t b;
    std::memcpy(&b, &x, 4);
    b = (b + 0x1000u) & 0xFFFFE000u;
    float r;
    std::memcpy(&r, &b, 4);
    return r;
}

cr_status setup_tc_operands(cr_ctx *h, const std::vector<double> &X)
{
    Params &P = h->P;
    const long long N = h->N;
    const int n = h->n, NP = h->NP;
    const int KP = crk::tc_kp(NP), N2 = crk::tc_n2(NP);
    const long long NB = (N + 7) / 8 + crk::kGR / 8;   // padding: a group load reads kGR/8 blocks
    std::vector<float> xr((size_t)NB * crk::tc_xr_floats(NP), 0.0f), xt((size_t)NB * crk::tc_xt_floats(NP), 0.0f);
    for (long long r = 0; r < N; ++r) {
        const long long blk = r >> 3;
        const int r8 = (int)(r & 7);
        for (int j = 0; j <= n; ++j) {
            const float v = j < n ? (float)X[(size_t)r * n + j] : 1.0f;
            const float hi = tf32_round_host(v), lo = tf32_round_host(v - hi);
            if (j < n) {
                const size_t o = (size_t)blk * crk::tc_xr_floats(NP) + (size_t)(j >> 2) * 32 + r8 * 4 + (j & 3);
                xr[o] = hi;
                xr[o + (size_t)KP * 8] = lo;
            }
            const size_t o = (size_t)blk * crk::tc_xt_floats(NP) + ((size_t)(j >> 3) * 2 + (r8 >> 2)) * 32 +
                             (j & 7) * 4 + (r8 & 3);
            xt[o] = hi;
            xt[o + (size_t)N2 * 8] = lo;
        }
    }
    CR_TRY(dev_alloc(h, &P.xr_tc, xr.size()));
    CR_TRY(dev_alloc(h, &P.xt_tc, xt.size()));
    CR_TRY(dev_alloc(h, &P.xi_tc, (size_t)P.S * crk::tc_xi_floats(NP)));
    CR_CUDA(h, cudaMemcpyAsync(P.xr_tc, xr.data(), sizeof(float) * xr.size(), cudaMemcpyHostToDevice, h->stream));
    CR_CUDA(h, cudaMemcpyAsync(P.xt_tc, xt.data(), sizeof(float) * xt.size(), cudaMemcpyHostToDevice, h->stream));
    CR_CUDA(h, cudaMemsetAsync(P.xi_tc, 0, sizeof(float) * (size_t)P.S * crk::tc_xi_floats(NP), h->stream));
    // the host vectors are released at return: finish the copies first
    CR_CUDA(h, cudaStreamSynchronize(h->stream));
    return CR_OK;
}

cr_status init_state(cr_ctx *h)
{
    const Params &P = h->P;
    const size_t th = (size_t)h->N * h->ld * theta_elem_size(h->opt.theta_dtype);
    for (int b = 0; b < 2; ++b) {
        CR_CUDA(h, cudaMemsetAsync(P.theta[b], 0, th, h->stream));
        CR_CUDA(h, cudaMemsetAsync(P.v[b], 0, sizeof(double) * h->N, h->stream));
        CR_CUDA(h, cudaMemsetAsync(P.w[b], 0, sizeof(double) * h->N * h->n, h->stream));
        CR_CUDA(h, cudaMemsetAsync(P.mu[b], 0, sizeof(double) * h->N, h->stream));
        CR_CUDA(h, cudaMemsetAsync(P.dd[b], 0, sizeof(double) * h->N, h->stream));
    }
    CR_CUDA(h, cudaMemsetAsync(P.rowpart, 0, sizeof(float) * (size_t)P.Q * h->N, h->stream));
    CR_CUDA(h, cudaMemsetAsync(P.colpart, 0, sizeof(float) * (size_t)P.G * P.slots * P.cgroups * (h->NP + 1) * crk::kW, h->stream));
    if (P.ball) CR_CUDA(h, cudaMemsetAsync(P.ballpart, 0, sizeof(double) * (size_t)P.G, h->stream));
    if (P.f64) {
        CR_CUDA(h, cudaMemsetAsync(P.rowpart64, 0, sizeof(double) * (size_t)P.Q * h->N, h->stream));
        CR_CUDA(h, cudaMemsetAsync(P.colpart64, 0,
                                   sizeof(double) * (size_t)P.G * P.slots * (h->NP + 1) * crk::kW,
                                   h->stream));
    }
    DevState st;
    std::memset(&st, 0, sizeof st);
    st.scal[0].t = 1.0;   // t_1 = 1 (Iteration 0 of Fig. 2)
    st.scal[0].dual = -std::numeric_limits<double>::infinity();
    st.scal[0].ball_c = 1.0;
    st.scal[1] = st.scal[0];
    CR_CUDA(h, cudaMemcpyAsync(P.st, &st, sizeof st, cudaMemcpyHostToDevice, h->stream));
    // eta(theta^(1)_0 = 0): y = h, xi = 0 (foldA of iteration 0 over zero partials)
    CR_TRY(launch_phase(h, crk::PH_FOLDA, 0, -1.0));
    CR_CUDA(h, cudaStreamSynchronize(h->stream));
    h->iters = 0;
    h->broken = false;
    return CR_OK;
}

// ---- checkpoints of the iteration state (differentiation) ------------------
cr_status ckpt_save(cr_ctx *h, cr_ctx::Checkpoint &c)
{
    const size_t th = (size_t)h->N * h->ld * theta_elem_size(h->opt.theta_dtype);
    const long long N = h->N;
    auto al = [&](void **p, size_t bytes) {
        if (cudaMalloc(p, bytes) != cudaSuccess) return false;
        h->ckpt_allocs.push_back(*p);
        return true;
    };
    if (!c.th[0]) {
        for (int b = 0; b < 2; ++b)
            if (!al(&c.th[b], th) || !al((void **)&c.v[b], sizeof(double) * h->N) ||
                !al((void **)&c.w[b], sizeof(double) * h->N * h->n) || !al((void **)&c.mu[b], sizeof(double) * h->N) ||
                !al((void **)&c.dd[b], sizeof(double) * h->N)) {
                (void)cudaGetLastError();
                return fail(h, CR_ENOMEM, "checkpoint allocation failed");
            }
    }
    if (c.full && !c.y1) {
        if (!al((void **)&c.y1, sizeof(double) * N) || !al((void **)&c.xi1_64, sizeof(double) * N * h->n) ||
            !al((void **)&c.foldpart, sizeof(double) * h->P.G * 8) || !al((void **)&c.yrow1, sizeof(float) * N) ||
            !al((void **)&c.ccol1, sizeof(float) * N) || !al((void **)&c.xi1, sizeof(float) * N * h->NP)) {
            (void)cudaGetLastError();
            return fail(h, CR_ENOMEM, "checkpoint allocation failed");
        }
    }
    if (c.full) {
        CR_CUDA(h, cudaMemcpyAsync(c.y1, h->P.y1, sizeof(double) * N, cudaMemcpyDeviceToDevice, h->stream));
        CR_CUDA(h, cudaMemcpyAsync(c.xi1_64, h->P.xi1_64, sizeof(double) * N * h->n, cudaMemcpyDeviceToDevice, h->stream));
        CR_CUDA(h, cudaMemcpyAsync(c.foldpart, h->P.foldpart, sizeof(double) * h->P.G * 8, cudaMemcpyDeviceToDevice, h->stream));
        CR_CUDA(h, cudaMemcpyAsync(c.yrow1, h->P.yrow1, sizeof(float) * N, cudaMemcpyDeviceToDevice, h->stream));
        CR_CUDA(h, cudaMemcpyAsync(c.ccol1, h->P.ccol1, sizeof(float) * N, cudaMemcpyDeviceToDevice, h->stream));
        CR_CUDA(h, cudaMemcpyAsync(c.xi1, h->P.xi1, sizeof(float) * N * h->NP, cudaMemcpyDeviceToDevice, h->stream));
    }
    for (int b = 0; b < 2; ++b) {
        CR_CUDA(h, cudaMemcpyAsync(c.th[b], h->P.theta[b], th, cudaMemcpyDeviceToDevice, h->stream));
        CR_CUDA(h, cudaMemcpyAsync(c.v[b], h->P.v[b], sizeof(double) * h->N, cudaMemcpyDeviceToDevice, h->stream));
        CR_CUDA(h, cudaMemcpyAsync(c.w[b], h->P.w[b], sizeof(double) * h->N * h->n, cudaMemcpyDeviceToDevice, h->stream));
        CR_CUDA(h, cudaMemcpyAsync(c.mu[b], h->P.mu[b], sizeof(double) * h->N, cudaMemcpyDeviceToDevice, h->stream));
        CR_CUDA(h, cudaMemcpyAsync(c.dd[b], h->P.dd[b], sizeof(double) * h->N, cudaMemcpyDeviceToDevice, h->stream));
    }
    CR_CUDA(h, cudaMemcpyAsync(&c.st, h->P.st, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream));
    CR_CUDA(h, cudaStreamSynchronize(h->stream));
    c.iter = h->iters;
    return CR_OK;
}

cr_status ckpt_restore(cr_ctx *h, const cr_ctx::Checkpoint &c)
{
    const size_t th = (size_t)h->N * h->ld * theta_elem_size(h->opt.theta_dtype);
    for (int b = 0; b < 2; ++b) {
        CR_CUDA(h, cudaMemcpyAsync(h->P.theta[b], c.th[b], th, cudaMemcpyDeviceToDevice, h->stream));
        CR_CUDA(h, cudaMemcpyAsync(h->P.v[b], c.v[b], sizeof(double) * h->N, cudaMemcpyDeviceToDevice, h->stream));
        CR_CUDA(h, cudaMemcpyAsync(h->P.w[b], c.w[b], sizeof(double) * h->N * h->n, cudaMemcpyDeviceToDevice, h->stream));
        CR_CUDA(h, cudaMemcpyAsync(h->P.mu[b], c.mu[b], sizeof(double) * h->N, cudaMemcpyDeviceToDevice, h->stream));
        CR_CUDA(h, cudaMemcpyAsync(h->P.dd[b], c.dd[b], sizeof(double) * h->N, cudaMemcpyDeviceToDevice, h->stream));
    }
    if (c.full) {
        const long long N = h->N;
        CR_CUDA(h, cudaMemcpyAsync(h->P.y1, c.y1, sizeof(double) * N, cudaMemcpyDeviceToDevice, h->stream));
        CR_CUDA(h, cudaMemcpyAsync(h->P.xi1_64, c.xi1_64, sizeof(double) * N * h->n, cudaMemcpyDeviceToDevice, h->stream));
        CR_CUDA(h, cudaMemcpyAsync(h->P.foldpart, c.foldpart, sizeof(double) * h->P.G * 8, cudaMemcpyDeviceToDevice, h->stream));
        CR_CUDA(h, cudaMemcpyAsync(h->P.yrow1, c.yrow1, sizeof(float) * N, cudaMemcpyDeviceToDevice, h->stream));
        CR_CUDA(h, cudaMemcpyAsync(h->P.ccol1, c.ccol1, sizeof(float) * N, cudaMemcpyDeviceToDevice, h->stream));
        CR_CUDA(h, cudaMemcpyAsync(h->P.xi1, c.xi1, sizeof(float) * N * h->NP, cudaMemcpyDeviceToDevice, h->stream));
    }
    DevState st = c.st;
    st.bar_count = 0;
    st.converged = 0;
    st.error = 0;
    CR_CUDA(h, cudaMemcpyAsync(h->P.st, &st, sizeof(DevState), cudaMemcpyHostToDevice, h->stream));
    h->iters = c.iter;
    return CR_OK;
}

void ckpt_clear(cr_ctx *h)
{
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (void *p : h->ckpt_allocs) cudaFree(p);
    h->ckpt_allocs.clear();
    h->ckpt.clear();
}

cr_status alcc_init(cr_ctx *h);

cr_status create_impl(std::vector<double> &X, std::vector<double> &yb, long long N, int n, const cr_options *opt,
                      cr_handle *out, int np_override = 0, const cr_alcc_options *aopt = nullptr)
{
    cr_ctx *h = new (std::nothrow) cr_ctx();
    if (!h) return CR_ENOMEM;
    *out = h;
    if (opt) h->opt = *opt;
    else cr_options_default(&h->opt);
    cr_options &o = h->opt;
    if (!(o.gamma > 0.0) || !std::isfinite(o.gamma)) return fail(h, CR_EINVAL, "gamma must be > 0");
    if (o.theta_dtype < 0 || o.theta_dtype > 3) return fail(h, CR_EINVAL, "unknown theta_dtype %d", o.theta_dtype);
    const bool f64 = o.theta_dtype == CR_THETA_F64;
    if (f64 && n > crk::kMaxNF64)
        return fail(h, CR_EINVAL, "FP64 multipliers are compiled for n <= %d (n = %d)", crk::kMaxNF64, n);
    if (f64 && (o.pair_engine == CR_PAIR_TENSOR_CORES || np_override > 0))
        return fail(h, CR_EINVAL, "FP64 multipliers: CUDA-core pass only, not in a batch");
    const bool ball = o.B_theta > 0.0 && std::isfinite(o.B_theta);
    if (ball && (o.theta_dtype == CR_THETA_BF16 || o.theta_dtype == CR_THETA_F16 || o.pair_engine == CR_PAIR_TENSOR_CORES ||
                 o.driver == CR_DRIVER_PERSISTENT || o.record_every > 0 || np_override > 0 || aopt))
        return fail(h, CR_EINVAL, "finite B_theta: FP32 or FP64 multipliers, CUDA-core pass, phase driver, single "
                                  "P-APG instances, no record_every");
    if (o.kkt_every < 1) return fail(h, CR_EINVAL, "kkt_every must be >= 1");
    h->N = N;
    h->n = n;
    h->NP = np_override > 0 ? np_override : padded_n(n);
    h->ks = kernels_for(o.theta_dtype, h->NP);
    if (!h->ks.phase) return fail(h, CR_EINVAL, "no kernel for n = %d", n);
    h->alcc = aopt != nullptr;
    if (h->alcc) {
        h->aopt = *aopt;
        if (o.theta_dtype != CR_THETA_F32) return fail(h, CR_EINVAL, "ALCC keeps theta in FP32");
        if (o.pair_engine == CR_PAIR_TENSOR_CORES) return fail(h, CR_EINVAL, "ALCC runs the CUDA-core pair pass");
        if (!(aopt->c > 1.0) || !(aopt->kappa > 0.0) || !(aopt->mu1_scale > 0.0) || !(aopt->tau1_rel > 0.0) ||
            !(aopt->alpha1_rel > 0.0) || aopt->lmax_cap < 0 || aopt->fixed_inner < 0 || aopt->launch_iters < 0 ||
            !(aopt->mu_max_scale >= 0.0))
            return fail(h, CR_EINVAL, "ALCC options: need c > 1, kappa > 0, positive scales, counts >= 0");
        o.record_every = 0;
        o.pair_engine = CR_PAIR_CUDA_CORES;
        o.shift = 0.0;
        h->ak = crk::alcc_kernel(h->NP);
        if (!h->ak.fn) return fail(h, CR_EINVAL, "no ALCC kernel for n = %d", n);
    }

    CR_CUDA(h, cudaGetDevice(&h->device));
    cudaDeviceProp prop;
    CR_CUDA(h, cudaGetDeviceProperties(&prop, h->device));
    if (prop.major * 10 + prop.minor < 100)
        return fail(h, CR_ECUDA, "device %s (sm_%d%d) is not a Blackwell part", prop.name, prop.major, prop.minor);
    h->num_sms = prop.multiProcessorCount;
    if (o.stream) {
        h->stream = (cudaStream_t)o.stream;
    } else {
        CR_CUDA(h, cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
        h->own_stream = true;
    }
    CR_CUDA(h, cudaFuncSetAttribute(h->ks.persistent, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)h->ks.smem));
    CR_CUDA(h, cudaFuncSetAttribute(h->ks.phase, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)h->ks.smem));
    if (h->ks.pair_tc)
        CR_CUDA(h, cudaFuncSetAttribute(h->ks.pair_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)h->ks.smem));
    if (h->alcc)
        CR_CUDA(h, cudaFuncSetAttribute(h->ak.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)h->ak.smem));
    int per_sm = 0;
    CR_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, h->alcc ? h->ak.fn : h->ks.persistent,
                                                             crk::kThreads, h->alcc ? h->ak.smem : h->ks.smem));
    int coop = 0;
    CR_CUDA(h, cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, h->device));
    const int max_coresident = per_sm * h->num_sms;

    // grid: one CTA per (SM x resident slot) by default; small problems use fewer
    long long S = (N + crk::kW - 1) / crk::kW;
    long long total = S * N;
    int G = o.grid > 0 ? o.grid : std::max(1, max_coresident);
    // keep at least 40 (stripe,row) units per CTA (N = 500: 25 CTAs, measured best); the FP64 pass
    // is bound by GB300's narrow FP64 pipe and spreads over more SMs
    const long long min_units = f64 ? 4 : 40;
    if (o.grid <= 0) G = (int)std::max<long long>(1, std::min<long long>(G, total / min_units));
    h->persistent_ok = coop && per_sm > 0 && G <= max_coresident && !ball;
    if (np_override > 0) h->persistent_ok = false;   // batch member: driven by the batch kernel only
    if (o.driver == CR_DRIVER_PERSISTENT && !h->persistent_ok)
        return fail(h, CR_EINVAL, "persistent driver: grid %d exceeds %d co-resident CTAs", G, max_coresident);
    if (h->alcc && !h->persistent_ok)
        return fail(h, CR_ECUDA, "ALCC: grid %d exceeds %d co-resident CTAs (or no cooperative launch)", G,
                    max_coresident);

    // host constants
    double s = o.shift >= 0.0 ? o.shift : default_shift(yb);
    double lo = yb[0], hi = yb[0];
    for (double v : yb) {
        lo = std::min(lo, v);
        hi = std::max(hi, v);
    }
    h->sigma = std::max(1.0, hi - lo);
    const double s2a2 = max_block_eig(X, N, n);   // sigma_max^2(A_2)
    double L = o.L > 0.0 ? o.L : (1.0 + 2.0 * (double)N + s2a2) / o.gamma;
    o.shift = s;
    o.L = L;

    Params &P = h->P;
    P.N = N;
    P.n = n;
    P.NP = h->NP;
    // rows of the multiplier arrays start on 256-byte boundaries (multiples of 128 elements): the
    // tile loads' L2 promotion fetches 256-byte lines, and a row start inside a line made every
    // tile row fetch one line more (N = 12,000: DRAM reads of the pass 1.07x -> 1.01x (FP32),
    // 1.28x -> 1.03x (BF16) of the two arrays)
    h->ld = ((N + 127) / 128) * 128;
    P.ld = h->ld;
    P.S = (int)S;
    // pair-pass engine: tensor cores for the two products when n is not tiny, unless the
    // iterations are recorded for cr_backward (which re-evaluates the CUDA-core arithmetic)
    const bool batch_member = np_override > 0;
    if (o.pair_engine < CR_PAIR_AUTO || o.pair_engine > CR_PAIR_TENSOR_CORES)
        return fail(h, CR_EINVAL, "unknown pair_engine %d", o.pair_engine);
    if (o.pair_engine == CR_PAIR_TENSOR_CORES &&
        (o.record_every > 0 || batch_member || o.driver == CR_DRIVER_PERSISTENT))
        return fail(h, CR_EINVAL, "pair_engine tensor cores: not with record_every > 0, the persistent driver or a batch");
    // auto: where the tensor-core pass measured faster on a GB300 (16-bit theta from n = 8,
    // FP32 theta from n = 16; at FP32, n = 10 both run at the same ~70% of HBM)
    const int tc_from = o.theta_dtype == CR_THETA_F32 ? 16 : 8;
    P.tc = (o.pair_engine == CR_PAIR_TENSOR_CORES ||
            (o.pair_engine == CR_PAIR_AUTO && h->NP >= tc_from && o.record_every <= 0 && !batch_member &&
             o.driver != CR_DRIVER_PERSISTENT && !f64 && !ball))
               ? 1
               : 0;
    if (P.tc) h->persistent_ok = false;   // the tensor-core pass runs in its own launch (phase driver)
    P.Q = (int)(((P.tc ? 1 : 2) * S + 3) / 4 * 4);   // row partials per row: one per warp column slab (CUDA
                                                               // cores) or per stripe (tensor cores)
    P.cgroups = P.tc ? 1 : crk::kWR;
    P.G = G;
    P.total = total;
    P.slots = max_slots(total, N, G);
    P.gamma = o.gamma;
    P.inv_gamma = 1.0 / o.gamma;
    P.L = L;
    P.invL_d = 1.0 / L;
    P.invL = (float)(1.0 / L);
    P.shift = s;
    P.sigma = h->sigma;
    P.st_scale = 1.0f;
    P.st_inv_scale = 1.0f;
    {
        double xm = 0.0;
        for (double v : X) xm = std::max(xm, std::fabs(v));
        P.xmax = (float)(xm * (1.0 + 1e-6));   // rounded up
        P.alcc_delta = (float)((n + 4) * std::ldexp(1.0, -23));
    }
    if (o.theta_dtype == CR_THETA_F16) {
        P.st_scale = std::ldexp(1.0f, o.fp16_exponent);
        P.st_inv_scale = std::ldexp(1.0f, -o.fp16_exponent);
    }
    P.momentum = o.momentum;
    P.restart = o.restart;
    // foldB(l+1) fused into foldA(l): plain P-APG (beta from the t-sequence alone), no recording
    // (cr_backward restores checkpoints and re-runs foldB), not in a batch
    P.fuse = (o.restart == 0 && o.record_every <= 0 && np_override <= 0 && !h->alcc) ? 1 : 0;
    P.fold_stats = 1;
    P.restart_tol = o.restart_tol > 0.0 ? o.restart_tol : 0.0;
    P.sr = o.stochastic_round;
    P.seed = (unsigned)(o.seed ^ (o.seed >> 32));
    P.bar_timeout_ns = (unsigned long long)(o.barrier_timeout_ms > 0 ? o.barrier_timeout_ms : 4000) * 1000000ull;
    P.bar_extra = o.test_barrier_extra > 0 ? o.test_barrier_extra : 0;
    h->record_every = o.record_every > 0 ? o.record_every : 0;
    if (h->record_every > 0 && ((o.theta_dtype != CR_THETA_F32 && o.theta_dtype != CR_THETA_F64) || !h->ks.bwd.pass1))
        return fail(h, CR_EINVAL, "record_every needs FP32 or FP64 theta and n <= 10");

    const size_t es = theta_elem_size(o.theta_dtype);
    for (int b = 0; b < (h->alcc ? 1 : 2); ++b) {   // ALCC keeps one multiplier array
        void *t = nullptr;
        CR_TRY(dev_alloc(h, (char **)&t, (size_t)N * h->ld * es));
        P.theta[b] = t;
    }
    if (h->alcc) P.theta[1] = P.theta[0];
    // TMA descriptors of the two multiplier arrays: N x N elements, row pitch ld, box kRS x kW;
    // out-of-range rows/columns read as zero
    auto encode = tensor_map_encoder();
    if (!encode) return fail(h, CR_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
    const CUtensorMapDataType tdt = o.theta_dtype == CR_THETA_F32    ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                    : o.theta_dtype == CR_THETA_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                                     : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    for (int b = 0; b < 2 && !f64; ++b) {   // the FP64 pass reads its tiles without TMA
        cuuint64_t gdim[2] = {(cuuint64_t)N, (cuuint64_t)N};
        cuuint64_t gstride[1] = {(cuuint64_t)h->ld * es};
        cuuint32_t box[2] = {(cuuint32_t)crk::kW, (cuuint32_t)crk::kRS};
        cuuint32_t estr[2] = {1, 1};
        CUresult r = encode(&P.tmap[b], tdt, 2, P.theta[b], gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(h, CR_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
        // 32-row boxes for the tensor-core pass (its stages are 32 rows)
        cuuint32_t box32[2] = {(cuuint32_t)crk::kW, 32u};
        r = encode(&P.tmap32[b], tdt, 2, P.theta[b], gdim, gstride, box32, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(h, CR_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
        // 8-row boxes for the 8-row stages of the batched launch
        cuuint32_t box8[2] = {(cuuint32_t)crk::kW, 8u};
        r = encode(&P.tmap8[b], tdt, 2, P.theta[b], gdim, gstride, box8, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(h, CR_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    }
    const int REC = rec_floats(h->NP);
    double *X64, *hh;
    CR_TRY(dev_alloc(h, &X64, (size_t)N * n));
    CR_TRY(dev_alloc(h, &P.rowrec, (size_t)N * REC));
    CR_TRY(dev_alloc(h, &hh, (size_t)N));
    P.X64 = X64;
    P.h = hh;
    CR_TRY(dev_alloc(h, &P.ccol2, N));
    CR_TRY(dev_alloc(h, &P.xi2, (size_t)N * h->NP));
    CR_TRY(dev_alloc(h, &P.yrow1, N));
    CR_TRY(dev_alloc(h, &P.ccol1, N));
    CR_TRY(dev_alloc(h, &P.xi1, (size_t)N * h->NP));
    CR_TRY(dev_alloc(h, &P.y1, N));
    CR_TRY(dev_alloc(h, &P.xi1_64, (size_t)N * n));
    for (int b = 0; b < 2; ++b) {
        CR_TRY(dev_alloc(h, &P.v[b], N));
        CR_TRY(dev_alloc(h, &P.w[b], (size_t)N * n));
        CR_TRY(dev_alloc(h, &P.mu[b], N));
        CR_TRY(dev_alloc(h, &P.dd[b], N));
    }
    CR_TRY(dev_alloc(h, &P.rowpart, (size_t)P.Q * N));
    CR_TRY(dev_alloc(h, &P.colpart, (size_t)G * P.slots * P.cgroups * (h->NP + 1) * crk::kW));
    {
        long long *tab = nullptr;
        CR_TRY(dev_alloc(h, &tab, partition_entries(G, S)));
        CR_TRY(upload_partition(h, tab));
    }
    CR_TRY(dev_alloc(h, &P.foldpart, (size_t)G * 8));
    CR_TRY(dev_alloc(h, &P.kktpart, (size_t)G * 8));
    CR_TRY(dev_alloc(h, &P.st, 1));
    P.f64 = f64 ? 1 : 0;
    P.ball = ball ? 1 : 0;
    P.B_theta = ball ? o.B_theta : 0.0;
    if (ball) CR_TRY(dev_alloc(h, &P.ballpart, (size_t)G));
    if (f64) {
        CR_TRY(dev_alloc(h, &P.rec64, (size_t)N * REC));
        CR_TRY(dev_alloc(h, &P.ccol2_64, (size_t)N));
        CR_TRY(dev_alloc(h, &P.xi2_64, (size_t)N * h->NP));
        CR_TRY(dev_alloc(h, &P.rowpart64, (size_t)P.Q * N));
        CR_TRY(dev_alloc(h, &P.colpart64, (size_t)G * P.slots * (h->NP + 1) * crk::kW));
    }
    if (h->alcc) {
        for (int b = 0; b < 2; ++b) {
            CR_TRY(dev_alloc(h, &P.ay[b], N));
            CR_TRY(dev_alloc(h, &P.axi[b], (size_t)N * n));
        }
        CR_TRY(dev_alloc(h, &P.ay2, N));
        CR_TRY(dev_alloc(h, &P.axi2, (size_t)N * n));
        if (!P.ccol2_64) CR_TRY(dev_alloc(h, &P.ccol2_64, N));   // xi.x - y of (y, xi)^(2), FP64
        // sigma_max^2(A_1) = 2N (A_1^T A_1 = 2(N I - 1 1^T)); radii from the feasible point
        // (mean(ybar) 1, 0): Bbar = ||ybar - mean||, Bbar_y = Bbar, Bbar_xi = Bbar / sqrt(gamma)
        double mean = 0.0;
        for (double v : yb) mean += v;
        mean /= (double)N;
        double B2 = 0.0;
        for (double v : yb) B2 += (v - mean) * (v - mean);
        h->a_s2a1 = 2.0 * (double)N;
        h->a_s2a2 = s2a2;
        h->a_By = std::sqrt(B2);
        h->a_Bxi = h->a_By / std::sqrt(o.gamma);
    }

    // row records {y - s (set by every fold), x_1..x_n, 0 ...}
    std::vector<float> rec((size_t)N * REC, 0.0f);
    std::vector<double> hv(N);
    for (long long l = 0; l < N; ++l) {
        for (int k = 0; k < n; ++k) rec[(size_t)l * REC + 1 + k] = (float)X[(size_t)l * n + k];
        hv[l] = yb[l] + s;
    }
    CR_CUDA(h, cudaMemcpyAsync(X64, X.data(), sizeof(double) * N * n, cudaMemcpyHostToDevice, h->stream));
    CR_CUDA(h, cudaMemcpyAsync(P.rowrec, rec.data(), sizeof(float) * rec.size(), cudaMemcpyHostToDevice, h->stream));
    CR_CUDA(h, cudaMemcpyAsync(hh, hv.data(), sizeof(double) * N, cudaMemcpyHostToDevice, h->stream));
    std::vector<double> rec64;
    if (f64) {
        // FP64 row records {y - s (set by every fold), x_1..x_n, 0 ...}
        rec64.assign((size_t)N * REC, 0.0);
        for (long long l = 0; l < N; ++l)
            for (int k = 0; k < n; ++k) rec64[(size_t)l * REC + 1 + k] = X[(size_t)l * n + k];
        CR_CUDA(h, cudaMemcpyAsync(P.rec64, rec64.data(), sizeof(double) * rec64.size(), cudaMemcpyHostToDevice,
                                   h->stream));
        CR_CUDA(h, cudaMemsetAsync(P.xi2_64, 0, sizeof(double) * (size_t)N * h->NP, h->stream));
    }
    if (P.tc) CR_TRY(setup_tc_operands(h, X));
    if (h->alcc) {
        // column data of (y_0, xi_0) = (ybar, 0): row records y = ybar, xi^T x - y = -ybar
        h->a_rec0 = rec;
        h->a_ccol0.resize(N);
        h->a_ccol64.resize(N);
        for (long long l = 0; l < N; ++l) {
            h->a_rec0[(size_t)l * REC] = (float)yb[l];
            h->a_ccol0[l] = (float)(-yb[l]);
            h->a_ccol64[l] = -hv[l];   // ay2 starts as h
        }
        return alcc_init(h);
    }
    return init_state(h);
}

// ---- ALCC (Sec. II-D) ----------------------------------------------------------

// Iteration 0 of Fig. `fig:alcc`: theta_1 = 0, (y_0, xi_0) = (ybar, 0), mu_1, tau_1, alpha_1.
cr_status alcc_init(cr_ctx *h)
{
    const Params &P = h->P;
    const long long N = h->N;
    const int n = h->n;
    CR_CUDA(h, cudaMemsetAsync(P.theta[0], 0, (size_t)N * h->ld * sizeof(float), h->stream));
    for (int b = 0; b < 2; ++b) {
        CR_CUDA(h, cudaMemcpyAsync(P.ay[b], P.h, sizeof(double) * N, cudaMemcpyDeviceToDevice, h->stream));
        CR_CUDA(h, cudaMemsetAsync(P.axi[b], 0, sizeof(double) * N * n, h->stream));
    }
    CR_CUDA(h, cudaMemcpyAsync(P.ay2, P.h, sizeof(double) * N, cudaMemcpyDeviceToDevice, h->stream));
    CR_CUDA(h, cudaMemcpyAsync(P.y1, P.h, sizeof(double) * N, cudaMemcpyDeviceToDevice, h->stream));
    CR_CUDA(h, cudaMemsetAsync(P.axi2, 0, sizeof(double) * N * n, h->stream));
    CR_CUDA(h, cudaMemsetAsync(P.xi1_64, 0, sizeof(double) * N * n, h->stream));
    CR_CUDA(h, cudaMemsetAsync(P.xi2, 0, sizeof(float) * N * h->NP, h->stream));
    CR_CUDA(h, cudaMemcpyAsync(P.rowrec, h->a_rec0.data(), sizeof(float) * h->a_rec0.size(), cudaMemcpyHostToDevice,
                               h->stream));
    CR_CUDA(h, cudaMemcpyAsync(P.ccol2, h->a_ccol0.data(), sizeof(float) * N, cudaMemcpyHostToDevice, h->stream));
    CR_CUDA(h, cudaMemcpyAsync(P.ccol2_64, h->a_ccol64.data(), sizeof(double) * N, cudaMemcpyHostToDevice, h->stream));
    CR_CUDA(h, cudaMemsetAsync(P.rowpart, 0, sizeof(float) * (size_t)P.Q * N, h->stream));
    CR_CUDA(h, cudaMemsetAsync(P.colpart, 0, sizeof(float) * (size_t)P.G * P.slots * P.cgroups * (h->NP + 1) * crk::kW,
                               h->stream));
    DevState st;
    std::memset(&st, 0, sizeof st);
    CR_CUDA(h, cudaMemcpyAsync(P.st, &st, sizeof st, cudaMemcpyHostToDevice, h->stream));
    CR_CUDA(h, cudaStreamSynchronize(h->stream));
    const cr_alcc_options &A = h->aopt;
    h->a_mu = A.mu1_scale / h->a_s2a1;
    h->a_tau = A.tau1_rel * h->a_By * h->a_By / h->a_mu;
    h->a_alpha_y = A.alpha1_rel * h->a_By;
    h->a_alpha_xi = A.alpha1_rel * h->a_Bxi;
    h->a_inner_total = 0;
    h->a_have_metrics = false;
    h->iters = 0;
    h->broken = false;
    return CR_OK;
}

// ell^max_k of Fig. `fig:alcc` step 2 at the current schedule (at least 1, at most lmax_cap).
long long alcc_lmax(const cr_ctx *h)
{
    if (h->aopt.fixed_inner > 0) return h->aopt.fixed_inner;
    const double Ly = 1.0 / h->a_mu + h->a_s2a1, Lxi = h->opt.gamma / h->a_mu + h->a_s2a2;
    double v = 4.0 * std::sqrt((Ly * h->a_By * h->a_By + Lxi * h->a_Bxi * h->a_Bxi) / h->a_tau);
    v = std::max(1.0, std::ceil(v));
    if (h->aopt.lmax_cap > 0) v = std::min(v, (double)h->aopt.lmax_cap);
    return v >= 4.0e18 ? (long long)4e18 : (long long)v;
}

// One outer iteration (steps 1-6).  MAPG runs in launches of at most launch_iters iterations;
// the kernel of the launch in which MAPG returns also takes the outer step and the KKT terms.
cr_status alcc_outer(cr_ctx *h, long long *inner)
{
    const cr_alcc_options &A = h->aopt;
    const double gamma = h->opt.gamma;
    const double Ly = 1.0 / h->a_mu + h->a_s2a1;        // step 1
    const double Lxi = gamma / h->a_mu + h->a_s2a2;
    const long long lmax = alcc_lmax(h);                // step 2
    double mu_next = A.c * h->a_mu;                     // step 5
    if (A.mu_max_scale > 0.0) mu_next = std::min(mu_next, std::max(h->a_mu, A.mu_max_scale / h->a_s2a1));
    crk::AlccStep S{};
    S.inv_mu = 1.0 / h->a_mu;
    S.gamma_inv_mu = gamma / h->a_mu;
    S.mu_next = mu_next;
    S.inv_Ly = 1.0 / Ly;
    S.inv_Lxi = 1.0 / Lxi;
    S.By = h->a_By;
    S.Bxi = h->a_Bxi;
    S.alpha_y = A.fixed_inner > 0 ? 0.0 : h->a_alpha_y;
    S.alpha_xi = A.fixed_inner > 0 ? 0.0 : h->a_alpha_xi;
    // steps far below the FP64 resolution of (y, xi) cannot change the FP64 margins of the active pairs
    S.res_rel = A.fixed_inner > 0 ? 0.0 : std::ldexp(1.0, -40);
    S.lmax = lmax;
    S.a = (float)(h->a_mu / mu_next);
    const double pairs = (double)h->N * (double)h->N;
    const long long chunk = A.launch_iters > 0 ? A.launch_iters
                                               : (long long)std::min(20000.0, std::max(16.0, 2e11 / pairs));
    long long ell0 = 1;
    double t0 = 1.0;
    DevState st;
    for (;;) {
        S.ell0 = ell0;
        S.ell1 = std::min(lmax, ell0 + chunk - 1);
        S.t0 = t0;
        CR_CUDA(h, cudaMemsetAsync(&h->P.st->bar_count, 0, sizeof(unsigned long long), h->stream));
        Params P = h->P;
        void *args[] = {&P, &S};
        {
            ProfScope ps(h, 3);
            CR_CUDA(h, cudaLaunchCooperativeKernel(h->ak.fn, dim3(h->P.G), dim3(crk::kThreads), args, h->ak.smem,
                                                   h->stream));
        }
        CR_TRY(read_state(h, &st));
        if (st.alcc_done) break;
        ell0 = S.ell1 + 1;
        t0 = st.alcc_t;
    }
    if (inner) *inner = st.alcc_ell;
    h->a_inner_total += st.alcc_ell;
    for (int i = 0; i < 4; ++i) h->a_metrics[i] = st.kkt[i];
    h->a_have_metrics = true;
    const double k = (double)(h->iters + 1);
    const double shrink = std::pow(A.c * std::pow(k, 1.0 + A.kappa), 2.0);   // steps 5-6
    h->a_tau /= shrink;
    h->a_alpha_y /= shrink;
    h->a_alpha_xi /= shrink;
    h->a_mu = mu_next;
    h->iters += 1;
    return CR_OK;
}

cr_status check_inputs(const double *X, const double *ybar, long long N, int n)
{
    if (!X || !ybar || n < 1 || n > crk::kMaxN || N < (long long)n + 1 || N > (1ll << 31)) return CR_EINVAL;
    if (!all_finite(X, (size_t)N * n) || !all_finite(ybar, (size_t)N)) return CR_EINVAL;
    return CR_OK;
}

// Creation errors have no handle to live on: they are kept per host thread and
// returned by cr_last_error(NULL).
thread_local std::string g_create_err;

cr_status create_error(cr_status s, const char *msg)
{
    g_create_err = msg;
    return s;
}

cr_status finish_create(cr_status s, cr_handle *out)
{
    if (s == CR_OK) {
        g_create_err.clear();
        return s;
    }
    g_create_err = *out ? (*out)->err : std::string(cr_status_str_impl(s));
    cr_destroy(*out);
    *out = nullptr;
    return s;
}

cr_status usable(cr_ctx *h)
{
    if (!h) return CR_EINVAL;
    if (h->broken) return fail(h, CR_ESTATE, "handle failed a bounded wait; call cr_reset");
    return CR_OK;
}

cr_status alcc_only(cr_ctx *h)
{
    CR_TRY(usable(h));
    if (!h->alcc) return fail(h, CR_ESTATE, "not an ALCC handle (cr_alcc_create)");
    return CR_OK;
}

cr_status papg_only(cr_ctx *h)
{
    CR_TRY(usable(h));
    if (h->alcc) return fail(h, CR_ESTATE, "an ALCC handle: use the cr_alcc_* calls");
    if (h->blocks) return fail(h, CR_ESTATE, "a K-block handle: use the cr_blocks_* calls");
    return CR_OK;
}

// Step 1 of the K-block P-APG at the outer iterate ell: a, b from the outer aggregates (at
// theta^(2)_ell, or at theta^(1)_ell itself), then inner_iters iterations of the inner P-APG.
cr_status blocks_step1(cr_ctx *h, long long ell, int at_theta1)
{
    cr_ctx *in = h->inner;
    const int grid = 4 * h->num_sms;
    {
        Params P = h->P;
        double *a = h->b_a, *b = h->b_b, *m2 = h->b_mu2;
        void *args[] = {&P, &a, &b, &m2, &ell, &at_theta1};
        CR_CUDA(h, cudaLaunchKernel(h->ks.blocks_prepare, dim3(grid), dim3(256), args, 0, h->stream));
    }
    // The inner handle runs on the same stream.  Every call restarts the inner P-APG as from its
    // Iteration 0 (t_1 = 1: no momentum in its first two iterations) at its current multipliers:
    // its iterations are numbered 1..M again, and with M even the last multipliers and their
    // aggregates sit in buffer 0, where iteration 1 reads its starting point.
    const double one = 1.0;
    CR_CUDA(h, cudaMemcpyAsync(&in->P.st->scal[0].t, &one, sizeof(double), cudaMemcpyHostToDevice, h->stream));
    cr_status s = run_phases(in, 1, h->inner_iters, 0, -1.0);
    if (s != CR_OK) return fail(h, s, "inner iterations: %s", in->err.c_str());
    in->iters = h->inner_iters;
    return CR_OK;
}

}  // namespace

namespace crk {
void set_thread_error(const std::string &m) { g_create_err = m; }
}  // namespace crk

extern "C" {

void cr_options_default(cr_options *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->gamma = 1e-2;
    o->L = 0.0;
    o->shift = -1.0;
    o->theta_dtype = CR_THETA_F32;
    o->stochastic_round = 1;
    o->kkt_every = 10;
    o->momentum = 1;
    o->restart = 0;
    o->driver = CR_DRIVER_AUTO;
    o->grid = 0;
    o->fp16_exponent = 8;
    o->seed = 0x5eedULL;
    o->stream = nullptr;
    o->restart_tol = 1e-7;
    o->pair_engine = CR_PAIR_AUTO;
}

cr_status cr_create(const double *X, const double *ybar, int64_t N, int32_t n, const cr_options *opt, cr_handle *out)
{
    if (!out) return create_error(CR_EINVAL, "out is NULL");
    *out = nullptr;
    if (check_inputs(X, ybar, N, n) != CR_OK)
        return create_error(CR_EINVAL, "need X, ybar finite, 1 <= n <= 32 and N >= n + 1");
    std::vector<double> Xv(X, X + (size_t)N * n), yv(ybar, ybar + N);
    return finish_create(create_impl(Xv, yv, N, n, opt, out), out);
}

cr_status cr_create_device(const float *dX, const float *dybar, int64_t N, int32_t n, const cr_options *opt,
                           cr_handle *out)
{
    if (!out) return create_error(CR_EINVAL, "out is NULL");
    *out = nullptr;
    if (!dX || !dybar || n < 1 || n > crk::kMaxN || N < (int64_t)n + 1)
        return create_error(CR_EINVAL, "need device X, ybar, 1 <= n <= 32 and N >= n + 1");
    std::vector<float> xf((size_t)N * n), yf(N);
    cudaError_t e = cudaMemcpy(xf.data(), dX, sizeof(float) * xf.size(), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(yf.data(), dybar, sizeof(float) * yf.size(), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return create_error(CR_ECUDA, cudaGetErrorString(e));
    }
    std::vector<double> Xv(xf.begin(), xf.end()), yv(yf.begin(), yf.end());
    if (check_inputs(Xv.data(), yv.data(), N, n) != CR_OK) return create_error(CR_EINVAL, "non-finite input");
    return finish_create(create_impl(Xv, yv, N, n, opt, out), out);
}

cr_status cr_promote(cr_handle h, int32_t theta_dtype)
{
    CR_TRY(papg_only(h));
    const int from = h->opt.theta_dtype;
    if (theta_dtype != CR_THETA_F32 || (from != CR_THETA_BF16 && from != CR_THETA_F16))
        return fail(h, CR_EINVAL, "cr_promote: from BF16 or FP16 multipliers to FP32 only (dtype %d -> %d)", from,
                    theta_dtype);
    Params &P = h->P;
    const long long N = h->N;
    const size_t count = (size_t)N * h->ld;
    KernelSet ks = kernels_for(CR_THETA_F32, h->NP);
    if (!ks.phase) return fail(h, CR_EINVAL, "cr_promote: no FP32 kernel for n = %d", h->n);
    // the engine: the tensor-core pass stays if the options allow it at FP32, else the CUDA cores
    // (a CUDA-core handle never moves to the tensor cores: their operands are written by foldB)
    const int newtc = (P.tc && (h->opt.pair_engine == CR_PAIR_TENSOR_CORES || h->NP >= 16)) ? 1 : 0;
    void *nt[2] = {nullptr, nullptr};
    for (int b = 0; b < 2; ++b) {
        CR_TRY(dev_alloc(h, (float **)&nt[b], count));
        const int grid = 4 * h->num_sms;
        if (from == CR_THETA_BF16)
            crk::k_widen_bf16<<<grid, 256, 0, h->stream>>>((const __nv_bfloat16 *)P.theta[b], (float *)nt[b], count);
        else
            crk::k_widen_f16<<<grid, 256, 0, h->stream>>>((const __half *)P.theta[b], (float *)nt[b], count,
                                                           P.st_inv_scale);
        CR_CUDA(h, cudaGetLastError());
    }
    CR_CUDA(h, cudaStreamSynchronize(h->stream));
    for (int b = 0; b < 2; ++b) {
        auto it = std::find(h->allocs.begin(), h->allocs.end(), P.theta[b]);
        if (it != h->allocs.end()) h->allocs.erase(it);
        cudaFree(P.theta[b]);
        P.theta[b] = nt[b];
    }
    auto encode = tensor_map_encoder();
    if (!encode) return fail(h, CR_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
    for (int b = 0; b < 2; ++b) {
        cuuint64_t gdim[2] = {(cuuint64_t)N, (cuuint64_t)N};
        cuuint64_t gstride[1] = {(cuuint64_t)h->ld * 4};
        cuuint32_t box[2] = {(cuuint32_t)crk::kW, (cuuint32_t)crk::kRS}, box32[2] = {(cuuint32_t)crk::kW, 32u};
        cuuint32_t box8[2] = {(cuuint32_t)crk::kW, 8u};
        cuuint32_t estr[2] = {1, 1};
        CUresult r = encode(&P.tmap[b], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, P.theta[b], gdim, gstride, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r == CUDA_SUCCESS)
            r = encode(&P.tmap32[b], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, P.theta[b], gdim, gstride, box32, estr,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r == CUDA_SUCCESS)
            r = encode(&P.tmap8[b], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, P.theta[b], gdim, gstride, box8, estr,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(h, CR_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    }
    if (newtc != P.tc) {
        // the partial-sum layouts of the two engines differ: rowpart is S (tensor cores) or 2S wide,
        // colpart has 1 or kWR row groups; the next pair pass writes them before the fold reads them
        const long long S = P.S;
        P.tc = newtc;
        P.Q = (int)(((P.tc ? 1 : 2) * S + 3) / 4 * 4);
        P.cgroups = P.tc ? 1 : crk::kWR;
        CR_TRY(dev_alloc(h, &P.rowpart, (size_t)P.Q * N));
        CR_TRY(dev_alloc(h, &P.colpart, (size_t)P.G * P.slots * P.cgroups * (h->NP + 1) * crk::kW));
        CR_CUDA(h, cudaMemsetAsync(P.rowpart, 0, sizeof(float) * (size_t)P.Q * N, h->stream));
    }
    h->ks = ks;
    CR_CUDA(h, cudaFuncSetAttribute(ks.persistent, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ks.smem));
    CR_CUDA(h, cudaFuncSetAttribute(ks.phase, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ks.smem));
    CR_CUDA(h, cudaFuncSetAttribute(ks.pair_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ks.smem));
    int per_sm = 0, coop = 0;
    CR_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ks.persistent, crk::kThreads, ks.smem));
    CR_CUDA(h, cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, h->device));
    h->persistent_ok = coop && per_sm > 0 && P.G <= per_sm * h->num_sms && !P.tc && !P.ball;
    P.st_scale = 1.0f;
    P.st_inv_scale = 1.0f;
    h->opt.theta_dtype = CR_THETA_F32;
    CR_CUDA(h, cudaStreamSynchronize(h->stream));
    return CR_OK;
}

cr_status cr_reset(cr_handle h)
{
    if (!h) return CR_EINVAL;
    if (h->blocks) return fail(h, CR_ESTATE, "a K-block handle is not reset: create it anew");
    if (h->alcc) return alcc_init(h);
    ckpt_clear(h);
    return init_state(h);
}

static cr_status run_iters(cr_handle h, long long k)
{
    CR_CUDA(h, cudaMemsetAsync(&h->P.st->converged, 0, sizeof(int), h->stream));
    const long long ell0 = h->iters + 1, ell1 = h->iters + k;
    const bool pers = h->opt.driver != CR_DRIVER_PHASES && h->persistent_ok;
    if (pers) CR_TRY(launch_persistent(h, ell0, ell1, 0, -1.0));
    else CR_TRY(run_phases(h, ell0, ell1, 0, -1.0));
    h->iters = ell1;
    return CR_OK;
}

cr_status cr_iterate(cr_handle h, int64_t k)
{
    CR_TRY(papg_only(h));
    if (k < 0) return fail(h, CR_EINVAL, "k < 0");
    if (k == 0) return CR_OK;
    if (h->record_every <= 0) return run_iters(h, k);
    // differentiation: a checkpoint at iteration 0 and after every record_every iterations
    if (h->ckpt.empty()) {
        if (h->iters != 0) return fail(h, CR_ESTATE, "recording must start at iteration 0 (cr_reset)");
        h->ckpt.emplace_back();
        CR_TRY(ckpt_save(h, h->ckpt.back()));
    }
    long long left = k;
    const long long re = h->record_every;
    while (left > 0) {
        const long long nb = (h->iters / re + 1) * re;
        const long long step = std::min(left, nb - h->iters);
        CR_TRY(run_iters(h, step));
        left -= step;
        if (h->iters % re == 0) {
            h->ckpt.emplace_back();
            CR_TRY(ckpt_save(h, h->ckpt.back()));
        }
    }
    return CR_OK;
}

static cr_status cr_solve_impl(cr_handle h, double tol, int64_t max_iter, int64_t *iters_done);

cr_status cr_solve(cr_handle h, double tol, int64_t max_iter, int64_t *iters_done)
{
    CR_TRY(papg_only(h));
    if (iters_done) *iters_done = 0;
    if (max_iter < 0 || !(tol >= 0.0)) return fail(h, CR_EINVAL, "bad tol/max_iter");
    // precision schedule: the 16-bit format down to promote_at, then FP32
    const int dt = h->opt.theta_dtype;
    if ((dt == CR_THETA_BF16 || dt == CR_THETA_F16) && h->opt.promote_at > tol) {
        int64_t d1 = 0;
        const cr_status s1 = cr_solve_impl(h, h->opt.promote_at, max_iter, &d1);
        if (s1 != CR_OK && s1 != CR_NOT_CONVERGED) return s1;
        if (s1 == CR_NOT_CONVERGED) {   // the cap came first
            if (iters_done) *iters_done = d1;
            return s1;
        }
        CR_TRY(cr_promote(h, CR_THETA_F32));
        int64_t d2 = 0;
        const cr_status s2 = cr_solve_impl(h, tol, max_iter - d1, &d2);
        if (iters_done) *iters_done = d1 + d2;
        return s2;
    }
    return cr_solve_impl(h, tol, max_iter, iters_done);
}

// cr_solve in the current storage format
static cr_status cr_solve_impl(cr_handle h, double tol, int64_t max_iter, int64_t *iters_done)
{
    if (iters_done) *iters_done = 0;
    CR_CUDA(h, cudaMemsetAsync(&h->P.st->converged, 0, sizeof(int), h->stream));
    const long long start = h->iters;
    const bool pers = h->opt.driver != CR_DRIVER_PHASES && h->persistent_ok;
    long long done = 0;
    const long long chunk = pers ? 20000 : 200;
    DevState st;
    while (done < max_iter) {
        const long long k = std::min<long long>(chunk, max_iter - done);
        const long long ell0 = h->iters + 1, ell1 = h->iters + k;
        if (pers) CR_TRY(launch_persistent(h, ell0, ell1, h->opt.kkt_every, tol));
        else CR_TRY(run_phases(h, ell0, ell1, h->opt.kkt_every, tol));
        CR_TRY(read_state(h, &st));
        if (st.converged) {
            h->iters = st.iters_done;
            done = h->iters - start;
            if (iters_done) *iters_done = done;
            return CR_OK;
        }
        h->iters = ell1;
        done += k;
    }
    if (iters_done) *iters_done = done;
    return CR_NOT_CONVERGED;
}

cr_status cr_kkt_residual(cr_handle h, double *kkt, double *infeas_norm, double *gap_norm)
{
    CR_TRY(papg_only(h));
    CR_CUDA(h, cudaMemsetAsync(&h->P.st->converged, 0, sizeof(int), h->stream));
    CR_TRY(launch_phase(h, crk::PH_KKT64, h->iters, -1.0));
    CR_TRY(launch_phase(h, crk::PH_DECIDE64, h->iters, -1.0, 1));
    DevState st;
    CR_TRY(read_state(h, &st));
    if (kkt) *kkt = st.kkt[0];
    if (infeas_norm) *infeas_norm = st.kkt[3];
    if (gap_norm) *gap_norm = st.kkt[4];
    return CR_OK;
}

cr_status cr_objective(cr_handle h, double *primal, double *dual, double *gap)
{
    CR_TRY(papg_only(h));
    std::vector<double> fp((size_t)h->P.G * 8);
    CR_CUDA(h, cudaMemcpyAsync(fp.data(), h->P.foldpart, sizeof(double) * fp.size(), cudaMemcpyDeviceToHost,
                               h->stream));
    CR_CUDA(h, cudaStreamSynchronize(h->stream));
    double a = 0.0, b = 0.0, c = 0.0;
    for (int i = 0; i < h->P.G; ++i) {
        a += fp[(size_t)i * 8 + 0];
        b += fp[(size_t)i * 8 + 1];
        c += fp[(size_t)i * 8 + 2];
    }
    // u = y - h:  primal = 1/2||u||^2 + gamma/2||xi||^2,  theta^T C eta = u^T y + gamma ||xi||^2
    const double pr = 0.5 * a + 0.5 * h->opt.gamma * b;
    const double gp = c + h->opt.gamma * b;
    if (primal) *primal = pr;
    if (gap) *gap = gp;
    if (dual) *dual = pr - gp;
    return CR_OK;
}

cr_status cr_get_solution(cr_handle h, double *yhat, double *xi)
{
    CR_TRY(usable(h));
    if (h->blocks) return fail(h, CR_ESTATE, "K-block handle: the primal point comes from cr_blocks_solution");
    if (yhat) {
        CR_CUDA(h, cudaMemcpyAsync(yhat, h->P.y1, sizeof(double) * h->N, cudaMemcpyDeviceToHost, h->stream));
    }
    if (xi) {
        CR_CUDA(h, cudaMemcpyAsync(xi, h->P.xi1_64, sizeof(double) * h->N * h->n, cudaMemcpyDeviceToHost,
                                   h->stream));
    }
    CR_CUDA(h, cudaStreamSynchronize(h->stream));
    if (yhat)
        for (long long l = 0; l < h->N; ++l) yhat[l] -= h->P.shift;
    return CR_OK;
}

// yhat = y1 - s and xi = xi1 into caller device buffers (one thread per value, grid-stride).
__global__ void k_solution_device(const double *__restrict__ y1, const double *__restrict__ xi1, double shift,
                                  long long N, long long Nn, double *yhat, double *xi)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N + Nn;
         i += (long long)gridDim.x * blockDim.x) {
        if (i < N) {
            if (yhat) yhat[i] = y1[i] - shift;
        } else if (xi) {
            xi[i - N] = xi1[i - N];
        }
    }
}

cr_status cr_get_solution_device(cr_handle h, double *yhat, double *xi)
{
    CR_TRY(usable(h));
    if (h->blocks) return fail(h, CR_ESTATE, "K-block handle: the primal point comes from cr_blocks_solution");
    if (yhat || xi) {
        const long long tot = h->N + h->N * (long long)h->n;
        const int grid = (int)std::min<long long>((tot + 255) / 256, (long long)h->num_sms * 4);
        k_solution_device<<<grid, 256, 0, h->stream>>>(h->P.y1, h->P.xi1_64, h->P.shift, h->N,
                                                       h->N * (long long)h->n, yhat, xi);
        CR_CUDA(h, cudaGetLastError());
    }
    CR_CUDA(h, cudaStreamSynchronize(h->stream));
    return CR_OK;
}

cr_status cr_get_info(cr_handle h, int64_t *iters, int64_t *restarts, double *L, double *shift)
{
    if (!h) return CR_EINVAL;
    if (iters) *iters = h->iters;
    if (L) *L = h->P.L;
    if (shift) *shift = h->P.shift;
    if (restarts) {
        DevState st;
        CR_TRY(read_state(h, &st));
        *restarts = st.scal[h->iters & 1].restarts;
    }
    return CR_OK;
}

cr_status cr_problem_constants(const double *X, const double *ybar, int64_t N, int32_t n, double gamma, double *L,
                               double *shift, double *sigma2_A1, double *sigma2_A2)
{
    if (check_inputs(X, ybar, N, n) != CR_OK || !(gamma > 0.0) || !std::isfinite(gamma))
        return create_error(CR_EINVAL, "need X, ybar finite, 1 <= n <= 32, N >= n + 1 and gamma > 0");
    std::vector<double> Xv(X, X + (size_t)N * n), yv(ybar, ybar + N);
    const double s2a2 = max_block_eig(Xv, N, n);
    if (L) *L = (1.0 + 2.0 * (double)N + s2a2) / gamma;
    if (shift) *shift = default_shift(yv);
    if (sigma2_A1) *sigma2_A1 = 2.0 * (double)N;
    if (sigma2_A2) *sigma2_A2 = s2a2;
    return CR_OK;
}

cr_status cr_get_engine(cr_handle h, int32_t *engine)
{
    if (!h || !engine) return CR_EINVAL;
    *engine = h->P.tc ? CR_PAIR_TENSOR_CORES : CR_PAIR_CUDA_CORES;
    return CR_OK;
}

cr_status cr_profile(cr_handle h, int32_t kind, double *ms, int64_t *launches)
{
    if (!h || kind < 0 || kind > 3) return CR_EINVAL;
    CR_CUDA(h, cudaStreamSynchronize(h->stream));
    for (auto &e : h->evs) {
        float t = 0.0f;
        if (cudaEventElapsedTime(&t, e.a, e.b) == cudaSuccess) {
            h->prof_ms[e.kind] += t;
            h->prof_n[e.kind] += 1;
        }
        h->pool.push_back(e.a);
        h->pool.push_back(e.b);
    }
    h->evs.clear();
    if (ms) *ms = h->prof_ms[kind];
    if (launches) *launches = h->prof_n[kind];
    h->prof_ms[kind] = 0.0;
    h->prof_n[kind] = 0;
    return CR_OK;
}

}  // extern "C"

// The FP32 multiplier arrays' tensor map (the same box and options as at creation) for another
// array of the same shape, used by the reverse mode's segment recompute.
static cr_status encode_theta_map(cr_ctx *h, CUtensorMap *m, const void *base)
{
    auto encode = tensor_map_encoder();
    if (!encode) return fail(h, CR_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
    cuuint64_t gdim[2] = {(cuuint64_t)h->N, (cuuint64_t)h->N};
    cuuint64_t gstride[1] = {(cuuint64_t)h->ld * sizeof(float)};
    cuuint32_t box[2] = {(cuuint32_t)crk::kW, (cuuint32_t)crk::kRS};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(base), gdim, gstride, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(h, CR_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return CR_OK;
}

// Puts back the multiplier pointers, their tensor maps and the row / column record pointers of a
// handle when the recompute ends, on the error paths too.
struct ThetaViewGuard {
    cr_ctx *h;
    void *saved_theta[2];
    CUtensorMap saved_map[2];
    float *saved_rowrec, *saved_ccol2, *saved_xi2;
    bool active = true;
    explicit ThetaViewGuard(cr_ctx *hh) : h(hh)
    {
        for (int b = 0; b < 2; ++b) {
            saved_theta[b] = h->P.theta[b];
            saved_map[b] = h->P.tmap[b];
        }
        saved_rowrec = h->P.rowrec;
        saved_ccol2 = h->P.ccol2;
        saved_xi2 = h->P.xi2;
    }
    void restore()
    {
        if (!active) return;
        for (int b = 0; b < 2; ++b) {
            h->P.theta[b] = saved_theta[b];
            h->P.tmap[b] = saved_map[b];
        }
        h->P.rowrec = saved_rowrec;
        h->P.ccol2 = saved_ccol2;
        h->P.xi2 = saved_xi2;
        active = false;
    }
    ~ThetaViewGuard() { restore(); }
};

// Reverse mode over FP32 (T = float) or FP64 (T = double) multipliers: the saved forward data of
// every recomputed iteration (multipliers, row records, column data) have the storage type.
template <typename T>
static cr_status backward_impl(cr_handle h, const float *dL_dyhat, float *dL_dybar, float *dL_dX)
{
    constexpr bool F64 = std::is_same<T, double>::value;
    const long long K = h->iters, k = h->record_every, N = h->N, ld = h->ld;
    const int n = h->n, NP = h->NP, K1 = NP + 1, REC = rec_floats(NP);
    if ((long long)h->ckpt.size() < (K + k - 1) / k) return fail(h, CR_ESTATE, "missing checkpoints");
    const size_t thb = (size_t)N * ld * sizeof(T);
    // workspace
    auto al = [&](void **p, size_t bytes) {
        if (cudaMalloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess) return false;
        h->bwd_allocs.push_back(*p);
        return true;
    };
    for (void *p : h->bwd_allocs) cudaFree(p);
    h->bwd_allocs.clear();
    std::vector<T *> segTh(k + 1), segRec(k), segCcol(k), segXi(k);
    std::vector<double *> segV(k + 2), segMu(k + 2);
    T *bb[2], *yb2, *ccolb, *xib;
    double *mub[2], *acc_row, *acc_col, *ybar_acc, *X_acc, *segBeta;
    bool ok = al((void **)&segBeta, sizeof(double) * k);
    for (long long i = 0; i <= k && ok; ++i) ok = al((void **)&segTh[i], thb);
    for (long long i = 0; i < k && ok; ++i)
        ok = al((void **)&segRec[i], sizeof(T) * N * REC) && al((void **)&segCcol[i], sizeof(T) * N) &&
             al((void **)&segXi[i], sizeof(T) * N * NP);
    for (long long i = 0; i < k + 2 && ok; ++i)
        ok = al((void **)&segV[i], sizeof(double) * N) && al((void **)&segMu[i], sizeof(double) * N);
    ok = ok && al((void **)&bb[0], thb) && al((void **)&bb[1], thb) && al((void **)&mub[0], sizeof(double) * N) &&
         al((void **)&mub[1], sizeof(double) * N) && al((void **)&acc_row, sizeof(double) * N * K1) &&
         al((void **)&acc_col, sizeof(double) * N * K1) && al((void **)&ybar_acc, sizeof(double) * N) &&
         al((void **)&X_acc, sizeof(double) * N * n) && al((void **)&yb2, sizeof(T) * N) &&
         al((void **)&ccolb, sizeof(T) * N) && al((void **)&xib, sizeof(T) * N * NP);
    if (!ok) {
        (void)cudaGetLastError();
        return fail(h, CR_ENOMEM, "reverse-mode workspace allocation failed");
    }
    if constexpr (!F64)   // the constant X columns of the row records the recompute writes into
        for (long long i = 0; i < k; ++i)
            CR_CUDA(h, cudaMemcpyAsync(segRec[i], h->P.rowrec, sizeof(T) * N * REC, cudaMemcpyDeviceToDevice, h->stream));
    CR_CUDA(h, cudaMemsetAsync(acc_row, 0, sizeof(double) * N * K1, h->stream));
    CR_CUDA(h, cudaMemsetAsync(acc_col, 0, sizeof(double) * N * K1, h->stream));
    CR_CUDA(h, cudaMemsetAsync(ybar_acc, 0, sizeof(double) * N, h->stream));
    CR_CUDA(h, cudaMemsetAsync(X_acc, 0, sizeof(double) * N * n, h->stream));
    for (int b = 0; b < 2; ++b) {
        CR_CUDA(h, cudaMemsetAsync(bb[b], 0, thb, h->stream));
        CR_CUDA(h, cudaMemsetAsync(mub[b], 0, sizeof(double) * N, h->stream));
    }
    // the final forward state, restored at the end
    cr_ctx::Checkpoint fin;
    fin.full = true;
    CR_TRY(ckpt_save(h, fin));
    std::vector<double> beta(K + 3, 0.0);
    const long long S128 = (N + crk::kBCols - 1) / crk::kBCols;
    const long long ntask = S128 * ((N + crk::kBRows - 1) / crk::kBRows);
    const int gpass = (int)std::min<long long>(ntask, (long long)h->num_sms * 8);
    const size_t bsm = h->ks.bwd.smem;
    if (bsm > 0) {
        CR_CUDA(h, cudaFuncSetAttribute(h->ks.bwd.pass1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bsm));
        CR_CUDA(h, cudaFuncSetAttribute(h->ks.bwd.pass2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bsm));
    }
    const int gfold = (int)std::max<long long>(1, std::min<long long>((N + 255) / 256, (long long)h->num_sms * 8));
    const long long nseg = (K + k - 1) / k;
    cr_status status = CR_OK;
    for (long long j = nseg - 1; j >= 0 && status == CR_OK; --j) {
        const long long c = j * k, e = std::min(c + k, K);
        CR_TRY(ckpt_restore(h, h->ckpt[j]));
        // segment entry i holds theta1_{c-1+i} (entries 0, 1 from the checkpoint)
        CR_CUDA(h, cudaMemcpyAsync(segTh[0], h->P.theta[(c + 1) & 1], thb, cudaMemcpyDeviceToDevice, h->stream));
        CR_CUDA(h, cudaMemcpyAsync(segTh[1], h->P.theta[c & 1], thb, cudaMemcpyDeviceToDevice, h->stream));
        CR_CUDA(h, cudaMemcpyAsync(segV[0], h->P.v[(c + 1) & 1], sizeof(double) * N, cudaMemcpyDeviceToDevice, h->stream));
        CR_CUDA(h, cudaMemcpyAsync(segMu[0], h->P.mu[(c + 1) & 1], sizeof(double) * N, cudaMemcpyDeviceToDevice, h->stream));
        CR_CUDA(h, cudaMemcpyAsync(segV[1], h->P.v[c & 1], sizeof(double) * N, cudaMemcpyDeviceToDevice, h->stream));
        CR_CUDA(h, cudaMemcpyAsync(segMu[1], h->P.mu[c & 1], sizeof(double) * N, cudaMemcpyDeviceToDevice, h->stream));
        // recompute the segment (bit for bit: same kernels, same partition, same rounding seeds).
        // FP32: the pass loads theta1_{l-1} and theta1_{l-2} through the tensor maps of
        // P.theta[(l + 1) & 1] and P.theta[l & 1] and stores theta1_l through the pointer
        // P.theta[l & 1], so the maps are pointed at the segment's entries q and q - 1 and the
        // pointer at entry q + 1: the iteration writes its result where the reverse steps read it
        // (the FP64 pass reads and writes its arrays in place and copies instead)
        ThetaViewGuard guard(h);
        for (long long ell = c + 1; ell <= e; ++ell) {
            const long long q = ell - c;
            if constexpr (!F64) {
                const int p = (int)(ell & 1), cc = 1 - p;
                CR_TRY(encode_theta_map(h, &h->P.tmap[cc], segTh[q]));
                CR_TRY(encode_theta_map(h, &h->P.tmap[p], segTh[q - 1]));
                h->P.theta[cc] = segTh[q];
                h->P.theta[p] = ell < e ? (void *)segTh[q + 1] : guard.saved_theta[p];
                // foldB writes the row and column data the pair pass reads straight into the
                // segment's entry (the X columns of its row records were filled once)
                h->P.rowrec = segRec[q - 1];
                h->P.ccol2 = segCcol[q - 1];
                h->P.xi2 = segXi[q - 1];
            }
            CR_TRY(run_iters(h, 1));
            if constexpr (F64) {
                if (ell < e)
                    CR_CUDA(h, cudaMemcpyAsync(segTh[q + 1], h->P.theta[ell & 1], thb, cudaMemcpyDeviceToDevice, h->stream));
                // the row and column data this iteration's pair pass read (the FP64 copies)
                CR_CUDA(h, cudaMemcpyAsync(segRec[q - 1], h->P.rec64, sizeof(T) * N * REC, cudaMemcpyDeviceToDevice, h->stream));
                CR_CUDA(h, cudaMemcpyAsync(segCcol[q - 1], h->P.ccol2_64, sizeof(T) * N, cudaMemcpyDeviceToDevice, h->stream));
                CR_CUDA(h, cudaMemcpyAsync(segXi[q - 1], h->P.xi2_64, sizeof(T) * N * NP, cudaMemcpyDeviceToDevice, h->stream));
            }
            CR_CUDA(h, cudaMemcpyAsync(segV[q + 1], h->P.v[ell & 1], sizeof(double) * N, cudaMemcpyDeviceToDevice, h->stream));
            CR_CUDA(h, cudaMemcpyAsync(segMu[q + 1], h->P.mu[ell & 1], sizeof(double) * N, cudaMemcpyDeviceToDevice, h->stream));
            // the momentum weight of this iteration, read back once per segment
            CR_CUDA(h, cudaMemcpyAsync(segBeta + (q - 1), &h->P.st->scal[ell & 1].beta, sizeof(double),
                                       cudaMemcpyDeviceToDevice, h->stream));
        }
        guard.restore();
        {
            std::vector<double> hb((size_t)(e - c));
            CR_CUDA(h, cudaMemcpyAsync(hb.data(), segBeta, sizeof(double) * (e - c), cudaMemcpyDeviceToHost, h->stream));
            DevState st;
            CR_TRY(read_state(h, &st));   // synchronizes the stream and checks the recompute's error flag
            for (long long ell = c + 1; ell <= e; ++ell) beta[ell] = hb[(size_t)(ell - c - 1)];
        }
        // reverse the segment
        for (long long ell = e; ell > c; --ell) {
            const long long q = ell - c;
            crk::BwdParamsT<T> B{};
            B.N = N;
            B.ld = ld;
            B.n = n;
            B.S128 = (int)S128;
            B.REC = REC;
            B.invL = F64 ? (T)h->P.invL_d : (T)h->P.invL;
            B.invL_d = h->P.invL_d;
            B.inv_gamma = h->P.inv_gamma;
            B.shift = h->P.shift;
            B.beta = (T)beta[ell];
            B.beta_d = beta[ell];
            B.c1_d = ell + 1 <= K ? 1.0 + beta[ell + 1] : 0.0;
            B.c2_d = ell + 2 <= K ? -beta[ell + 2] : 0.0;
            B.c1 = (T)B.c1_d;
            B.c2 = (T)B.c2_d;
            B.thc = segTh[q];
            B.thp = segTh[q - 1];
            B.rowrec = segRec[q - 1];
            B.ccol2 = segCcol[q - 1];
            B.xi2 = segXi[q - 1];
            B.b1 = ell + 1 <= K ? bb[(ell + 1) & 1] : nullptr;
            B.b2 = ell + 2 <= K ? bb[ell & 1] : nullptr;
            B.outb = bb[ell & 1];
            B.mub1 = ell + 1 <= K ? mub[(ell + 1) & 1] : nullptr;
            B.mub2 = ell + 2 <= K ? mub[ell & 1] : nullptr;
            B.mub_out = mub[ell & 1];
            B.ubar = ell == K ? dL_dyhat : nullptr;
            B.v1 = segV[q];
            B.v2 = segV[q - 1];
            B.mu1 = segMu[q];
            B.mu2 = segMu[q - 1];
            B.X64 = h->P.X64;
            B.h = h->P.h;
            B.acc_row = acc_row;
            B.acc_col = acc_col;
            B.ybar_acc = ybar_acc;
            B.X_acc = X_acc;
            B.yb2 = yb2;
            B.ccolb = ccolb;
            B.xib = xib;
            B.yb2_out = yb2;
            B.ccolb_out = ccolb;
            B.xib_out = xib;
            void *args[] = {&B};
            CR_CUDA(h, cudaLaunchKernel(h->ks.bwd.pass1, dim3(gpass), dim3(256), args, bsm, h->stream));
            CR_CUDA(h, cudaLaunchKernel(h->ks.bwd.fold1, dim3(gfold), dim3(256), args, 0, h->stream));
            CR_CUDA(h, cudaLaunchKernel(h->ks.bwd.pass2, dim3(gpass), dim3(256), args, bsm, h->stream));
            CR_CUDA(h, cudaLaunchKernel(h->ks.bwd.fold2, dim3(gfold), dim3(256), args, 0, h->stream));
        }
    }
    {
        long long NN = N;
        int nn = n;
        void *args[] = {&NN, &nn, (void *)&dL_dyhat, &ybar_acc, &X_acc, &dL_dybar, &dL_dX};
        CR_CUDA(h, cudaLaunchKernel((const void *)crk::k_bwd_finish, dim3(gfold), dim3(256), args, 0, h->stream));
    }
    CR_TRY(ckpt_restore(h, fin));
    CR_CUDA(h, cudaStreamSynchronize(h->stream));
    return status;
}

extern "C" {

cr_status cr_backward(cr_handle h, const float *dL_dyhat, float *dL_dybar, float *dL_dX)
{
    CR_TRY(papg_only(h));
    if (!dL_dyhat || !dL_dybar || !dL_dX) return fail(h, CR_EINVAL, "NULL buffer");
    const int dt = h->opt.theta_dtype;
    if (h->record_every <= 0 || h->ckpt.empty() || (dt != CR_THETA_F32 && dt != CR_THETA_F64))
        return fail(h, CR_ESTATE, "cr_backward needs iterations run with record_every > 0 (FP32 or FP64 theta)");
    return dt == CR_THETA_F64 ? backward_impl<double>(h, dL_dyhat, dL_dybar, dL_dX)
                              : backward_impl<float>(h, dL_dyhat, dL_dybar, dL_dX);
}

cr_status cr_get_device_state(cr_handle h, const void **dtheta, int64_t *ld, const double **dX, const double **dy,
                              const double **dxi, const double **dmu, double *sigma)
{
    if (!h) return CR_EINVAL;
    const int b = (int)(h->iters & 1);   // theta^(1)_l lives in buffer l & 1
    if (dtheta) *dtheta = h->P.theta[b];
    if (ld) *ld = h->ld;
    if (dX) *dX = h->P.X64;
    if (dy) *dy = h->P.y1;
    if (dxi) *dxi = h->P.xi1_64;
    if (dmu) *dmu = h->P.mu[b];
    if (sigma) *sigma = h->sigma;
    return CR_OK;
}

void cr_alcc_options_default(cr_alcc_options *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->mu1_scale = 1e3;
    o->tau1_rel = 1e-2;
    o->alpha1_rel = 1e-2;
    o->c = 2.0;
    o->kappa = 0.1;
}

cr_status cr_alcc_create(const double *X, const double *ybar, int64_t N, int32_t n, const cr_options *opt,
                         const cr_alcc_options *aopt, cr_handle *out)
{
    if (!out) return create_error(CR_EINVAL, "out is NULL");
    *out = nullptr;
    if (check_inputs(X, ybar, N, n) != CR_OK)
        return create_error(CR_EINVAL, "need X, ybar finite, 1 <= n <= 32 and N >= n + 1");
    cr_alcc_options a;
    if (aopt) a = *aopt;
    else cr_alcc_options_default(&a);
    std::vector<double> Xv(X, X + (size_t)N * n), yv(ybar, ybar + N);
    return finish_create(create_impl(Xv, yv, N, n, opt, out, 0, &a), out);
}

cr_status cr_alcc_iterate(cr_handle h, int64_t k, int64_t *inner)
{
    CR_TRY(alcc_only(h));
    if (k < 0) return fail(h, CR_EINVAL, "k < 0");
    for (int64_t i = 0; i < k; ++i) {
        long long it = 0;
        CR_TRY(alcc_outer(h, &it));
        if (inner) inner[i] = it;
    }
    return CR_OK;
}

cr_status cr_alcc_solve(cr_handle h, double tol, int64_t max_outer, int64_t *outer_done)
{
    CR_TRY(alcc_only(h));
    if (outer_done) *outer_done = 0;
    if (max_outer < 0 || !(tol >= 0.0)) return fail(h, CR_EINVAL, "bad tol/max_outer");
    for (int64_t i = 0; i < max_outer; ++i) {
        CR_TRY(alcc_outer(h, nullptr));
        if (outer_done) *outer_done = i + 1;
        if (h->a_metrics[0] <= tol) return CR_OK;
    }
    return CR_NOT_CONVERGED;
}

cr_status cr_alcc_metrics(cr_handle h, double *kkt, double *stat, double *pri, double *comp)
{
    CR_TRY(alcc_only(h));
    if (!h->a_have_metrics) return fail(h, CR_ESTATE, "no outer iteration has run");
    if (kkt) *kkt = h->a_metrics[0];
    if (stat) *stat = h->a_metrics[1];
    if (pri) *pri = h->a_metrics[2];
    if (comp) *comp = h->a_metrics[3];
    return CR_OK;
}

cr_status cr_alcc_info(cr_handle h, int64_t *outer, int64_t *inner_total, double *mu, int64_t *lmax_next)
{
    CR_TRY(alcc_only(h));
    if (outer) *outer = h->iters;
    if (inner_total) *inner_total = h->a_inner_total;
    if (mu) *mu = h->a_mu;
    if (lmax_next) *lmax_next = alcc_lmax(h);
    return CR_OK;
}

void cr_destroy(cr_handle h)
{
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->inner) cr_destroy(h->inner);
    ckpt_clear(h);
    for (void *p : h->bwd_allocs) cudaFree(p);
    for (auto &e : h->evs) {
        cudaEventDestroy(e.a);
        cudaEventDestroy(e.b);
    }
    for (cudaEvent_t e : h->pool) cudaEventDestroy(e);
    for (void *p : h->allocs) cudaFree(p);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

// ---- P-APG with K blocks (Sec. II-A) -------------------------------------------------------

cr_status cr_blocks_create(const double *X, const double *ybar, int64_t N, int32_t n, const int32_t *block_of,
                           const cr_options *opt, int32_t inner_iters, cr_handle *out)
{
    if (!out) return create_error(CR_EINVAL, "out is NULL");
    *out = nullptr;
    if (check_inputs(X, ybar, N, n) != CR_OK)
        return create_error(CR_EINVAL, "need X, ybar finite, 1 <= n <= 32 and N >= n + 1");
    if (!block_of || inner_iters < 2 || (inner_iters & 1))
        return create_error(CR_EINVAL, "need block_of (N entries) and an even inner_iters >= 2");
    if (n > crk::kMaxNF64) return create_error(CR_EINVAL, "K-block P-APG runs with FP64 multipliers: n <= 10");
    std::vector<int> used((size_t)N, 0);
    for (long long l = 0; l < N; ++l) {
        if (block_of[l] < 0 || block_of[l] >= N) return create_error(CR_EINVAL, "block ids must lie in [0, N)");
        used[block_of[l]] = 1;
    }
    int K = 0;
    for (int u : used) K += u;
    cr_options o;
    if (opt) o = *opt;
    else cr_options_default(&o);
    o.theta_dtype = CR_THETA_F64;
    o.driver = CR_DRIVER_PHASES;
    o.pair_engine = CR_PAIR_CUDA_CORES;
    o.record_every = 0;
    o.restart = 0;
    o.momentum = 1;
    o.B_theta = 0.0;
    // the handles hold the points sorted by block (stable), so that the pairs inside the blocks
    // are K diagonal squares of the multiplier arrays; cr_blocks_solution restores the caller's order
    std::vector<long long> perm((size_t)N);
    for (long long l = 0; l < N; ++l) perm[l] = l;
    std::stable_sort(perm.begin(), perm.end(), [&](long long a, long long b) { return block_of[a] < block_of[b]; });
    std::vector<double> Xv((size_t)N * n), yv((size_t)N);
    std::vector<int> bv((size_t)N);
    for (long long q = 0; q < N; ++q) {
        const long long l = perm[q];
        for (int k = 0; k < n; ++k) Xv[(size_t)q * n + k] = X[(size_t)l * n + k];
        yv[q] = ybar[l];
        bv[q] = block_of[l];
    }
    cr_handle h = nullptr, in = nullptr;
    cr_status s = create_impl(Xv, yv, N, n, &o, &h);
    if (s != CR_OK) return finish_create(s, &h);
    o.stream = h->stream;   // one stream for both duals
    std::vector<double> Xi(Xv), yi(yv);
    s = create_impl(Xi, yi, N, n, &o, &in);
    if (s != CR_OK) {
        std::string m = in ? in->err : std::string("inner handle");
        if (in) cr_destroy(in);
        cr_destroy(h);
        return create_error(s, m.c_str());
    }
    h->inner = in;
    h->blocks = true;
    h->K = K;
    h->inner_iters = inner_iters;
    h->perm = perm;
    int *blk = nullptr;
    CR_TRY(dev_alloc(h, &blk, (size_t)N));
    CR_CUDA(h, cudaMemcpyAsync(blk, bv.data(), sizeof(int) * N, cudaMemcpyHostToDevice, h->stream));
    // the inner pass visits, in stripe s, only the rows of the blocks that its columns belong to,
    // and its CTAs share those (stripe, row) units evenly
    {
        Params &Q = in->P;
        const long long S = Q.S, G = Q.G;
        std::vector<long long> bstart((size_t)N), bend((size_t)N), band((size_t)(2 * S)), cum((size_t)S + 1, 0);
        for (long long q = 0; q < N;) {
            long long e = q;
            while (e < N && bv[e] == bv[q]) ++e;
            for (long long t = q; t < e; ++t) {
                bstart[t] = q;
                bend[t] = e;
            }
            q = e;
        }
        for (long long st = 0; st < S; ++st) {
            const long long c0 = st * crk::kW, c1 = std::min<long long>(N, c0 + crk::kW) - 1;
            band[2 * st] = bstart[c0];
            band[2 * st + 1] = bend[c1];
            cum[st + 1] = cum[st] + (band[2 * st + 1] - band[2 * st]);
        }
        const long long T = cum[S];
        std::vector<long long> ub((size_t)G + 1);
        for (long long c = 0; c <= G; ++c) {
            if (c == G) {
                ub[c] = S * N;
                continue;
            }
            const long long k = (long long)(((unsigned long long)c * (unsigned long long)T) / (unsigned long long)G);
            long long st = 0;
            while (st + 1 < S && cum[st + 1] <= k) ++st;
            ub[c] = st * N + band[2 * st] + (k - cum[st]);
        }
        int slots = 1;
        for (long long c = 0; c < G; ++c)
            if (ub[c + 1] > ub[c]) slots = std::max(slots, (int)((ub[c + 1] - 1) / N - ub[c] / N + 1));
        if (slots > Q.slots) {   // both column-partial buffers are sized by the slots per CTA
            double *cp = nullptr;
            float *cp32 = nullptr;
            CR_TRY(dev_alloc(in, &cp, (size_t)G * slots * (in->NP + 1) * crk::kW));
            CR_TRY(dev_alloc(in, &cp32, (size_t)G * slots * Q.cgroups * (in->NP + 1) * crk::kW));
            Q.colpart64 = cp;
            Q.colpart = cp32;
            Q.slots = slots;
        }
        CR_TRY(upload_partition(in, const_cast<long long *>(Q.ubeg), &ub));
        long long *db = nullptr;
        CR_TRY(dev_alloc(h, &db, (size_t)(2 * S)));
        CR_CUDA(h, cudaMemcpyAsync(db, band.data(), sizeof(long long) * 2 * S, cudaMemcpyHostToDevice, h->stream));
        Q.band = db;
    }
    CR_TRY(dev_alloc(h, &h->b_a, (size_t)N));
    CR_TRY(dev_alloc(h, &h->b_b, (size_t)N * n));
    CR_TRY(dev_alloc(h, &h->b_mu2, (size_t)N));
    // outer: the pairs between blocks; its foldB is replaced by the block Step 1 (no fusion)
    h->P.blk = blk;
    h->P.blkmode = 1;
    h->P.fuse = 0;
    // inner: the pairs inside the blocks, Step 1 of the block problems (linear term a, subgradient
    // offset b, no y >= 0 rows), plain P-APG iterations without fusion (a and b change between calls)
    in->P.blk = blk;
    in->P.blkmode = 2;
    in->P.fuse = 0;
    in->P.no_mu = 1;
    in->P.h = h->b_a;
    in->P.xi_off = h->b_b;
    in->prepared = false;
    CR_CUDA(h, cudaMemcpyAsync(h->b_a, h->P.h, sizeof(double) * N, cudaMemcpyDeviceToDevice, h->stream));
    CR_CUDA(h, cudaMemsetAsync(h->b_b, 0, sizeof(double) * N * n, h->stream));
    CR_CUDA(h, cudaStreamSynchronize(h->stream));
    // Iteration 0 (theta = 0, mu = 0): the inner handle's state too
    s = init_state(in);
    if (s != CR_OK) {
        cr_destroy(h);
        return create_error(s, "inner reset failed");
    }
    *out = h;
    return CR_OK;
}

cr_status cr_blocks_iterate(cr_handle h, int64_t k)
{
    CR_TRY(usable(h));
    if (!h->blocks) return fail(h, CR_ESTATE, "not a K-block handle");
    if (k < 0) return fail(h, CR_EINVAL, "k < 0");
    const int grid = 4 * h->num_sms;
    for (long long i = 0; i < k; ++i) {
        const long long ell = h->iters + 1;
        CR_TRY(blocks_step1(h, ell, 0));   // eta_ell at theta^(2)_ell
        {
            Params P = h->P;
            const double *y = h->inner->P.y1, *xi = h->inner->P.xi1_64, *m2 = h->b_mu2;
            long long e = ell;
            void *args[] = {&P, &y, &xi, &m2, &e};
            CR_CUDA(h, cudaLaunchKernel(h->ks.blocks_records, dim3(grid), dim3(256), args, 0, h->stream));
        }
        CR_TRY(launch_phase(h, crk::PH_PAIR, ell, -1.0));
        CR_TRY(launch_phase(h, crk::PH_FOLDA, ell, -1.0));
        h->prepared = false;
        h->iters = ell;
    }
    // the primal point at the dual iterate theta^(1)_l (Theorem 1), Step 1 solved again
    if (k > 0) CR_TRY(blocks_step1(h, h->iters, 1));
    DevState st;
    return read_state(h, &st);
}

cr_status cr_blocks_solution(cr_handle h, double *yhat, double *xi)
{
    CR_TRY(usable(h));
    if (!h->blocks) return fail(h, CR_ESTATE, "not a K-block handle");
    if (h->iters == 0) CR_TRY(blocks_step1(h, 0, 1));   // Iteration 0: the block problems at (h, 0)
    cr_ctx *in = h->inner;
    const long long N = h->N;
    const int n = h->n;
    std::vector<double> yv((size_t)N), xv((size_t)N * n);
    CR_CUDA(h, cudaMemcpyAsync(yv.data(), in->P.y1, sizeof(double) * N, cudaMemcpyDeviceToHost, h->stream));
    CR_CUDA(h, cudaMemcpyAsync(xv.data(), in->P.xi1_64, sizeof(double) * N * n, cudaMemcpyDeviceToHost, h->stream));
    CR_CUDA(h, cudaStreamSynchronize(h->stream));
    for (long long q = 0; q < N; ++q) {   // back to the caller's order
        const long long l = h->perm[q];
        if (yhat) yhat[l] = yv[q] - h->P.shift;
        if (xi)
            for (int k = 0; k < n; ++k) xi[(size_t)l * n + k] = xv[(size_t)q * n + k];
    }
    return CR_OK;
}

const char *cr_status_str(cr_status s) { return cr_status_str_impl(s); }

const char *cr_last_error(cr_handle h) { return h ? h->err.c_str() : g_create_err.c_str(); }

}  // extern "C"

// ===========================================================================
// Batched solves: many independent instances in one persistent launch
// ===========================================================================
struct cr_batch_ctx {
    std::vector<cr_handle> inst;
    std::vector<long long> Gfine;     // finest virtual-CTA count per instance
    int B = 0, NP = 0;
    KernelSet ks{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int Gphys = 0;
    Params *dP = nullptr;
    int *d_item_inst = nullptr, *d_item_vc = nullptr, *d_off = nullptr, *d_active = nullptr, *d_err = nullptr;
    long long *d_ell = nullptr;
    unsigned long long *d_bar = nullptr;
    std::vector<void *> allocs;
    cudaGraphExec_t gexec = nullptr;
    long long gchunk = 0;
    int gcheck = 0;
    double gtol = -1.0;
    bool graph_ok = true;
    long long graph_launches = 0;     // launches replayed from the captured CUDA graph
    long long direct_launches = 0;    // launches made directly (capture not available)
    int factor = 1;                   // work granularity chosen by the autotuner
    int stage_rows = crk::kRS;        // rows per pipeline stage of the pair pass (16 or 8): tile shape
    long long iters = 0;
    std::string err;
    std::vector<double> tune_ms;      // autotuner measurements (ms per iteration) per candidate
    std::vector<int> tune_factor;
    std::vector<int> tune_rows;
    const void *kernel() const { return stage_rows == 8 ? ks.batch8 : ks.batch; }
    size_t smem() const { return stage_rows == 8 ? ks.smem_batch8 : ks.smem; }
};

namespace {

const int kTuneFactors[] = {1, 2, 4, 8, 16};
constexpr long long kPairsPerItemFine = 1ll << 17;   // finest work item: ~131k pairs

cr_status bfail(cr_batch_ctx *b, cr_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (b) b->err = buf;
    g_create_err = buf;
    return s;
}

#define CR_BCUDA(b, call)                                                             \
    do {                                                                              \
        cudaError_t e_ = (call);                                                      \
        if (e_ != cudaSuccess) return bfail(b, CR_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

// Sets every instance's virtual-CTA count for granularity factor f, assigns the work
// items to the physical CTAs (longest-processing-time first by pair count) and
// uploads the instance parameters and the item lists.
cr_status batch_plan(cr_batch_ctx *b, int f)
{
    struct Item {
        int i;
        int vc;
        double cost;
    };
    std::vector<Item> items;
    std::vector<Params> hp(b->B);
    for (int i = 0; i < b->B; ++i) {
        cr_ctx *h = b->inst[i];
        const long long G = std::max<long long>(1, b->Gfine[i] / f);
        h->P.G = (int)G;
        h->P.slots = max_slots(h->P.total, h->N, (int)G);
        CR_TRY(upload_partition(h, const_cast<long long *>(h->P.ubeg)));   // capacity: the finest grid
        hp[i] = h->P;
        const double pairs = (double)h->N * (double)(h->N - 1);
        for (long long v = 0; v < G; ++v) items.push_back({i, (int)v, pairs / (double)G + 2.0e4});
    }
    std::vector<int> order(items.size());
    for (size_t k = 0; k < order.size(); ++k) order[k] = (int)k;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return items[x].cost > items[y].cost; });
    std::vector<double> load(b->Gphys, 0.0);
    std::vector<std::vector<int>> per(b->Gphys);
    for (int k : order) {
        int best = 0;
        for (int c = 1; c < b->Gphys; ++c)
            if (load[c] < load[best]) best = c;
        load[best] += items[k].cost;
        per[best].push_back(k);
    }
    std::vector<int> ii, vv, off(b->Gphys + 1, 0);
    for (int c = 0; c < b->Gphys; ++c) {
        std::sort(per[c].begin(), per[c].end(), [&](int x, int y) {
            return items[x].i != items[y].i ? items[x].i < items[y].i : items[x].vc < items[y].vc;
        });
        for (int k : per[c]) {
            ii.push_back(items[k].i);
            vv.push_back(items[k].vc);
        }
        off[c + 1] = (int)ii.size();
    }
    // item arrays are sized for the finest plan (most items)
    CR_BCUDA(b, cudaMemcpyAsync(b->dP, hp.data(), sizeof(Params) * b->B, cudaMemcpyHostToDevice, b->stream));
    CR_BCUDA(b, cudaMemcpyAsync(b->d_item_inst, ii.data(), sizeof(int) * ii.size(), cudaMemcpyHostToDevice, b->stream));
    CR_BCUDA(b, cudaMemcpyAsync(b->d_item_vc, vv.data(), sizeof(int) * vv.size(), cudaMemcpyHostToDevice, b->stream));
    CR_BCUDA(b, cudaMemcpyAsync(b->d_off, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice, b->stream));
    CR_BCUDA(b, cudaStreamSynchronize(b->stream));
    b->factor = f;
    if (b->gexec) {
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
    }
    return CR_OK;
}

cr_status batch_reset(cr_batch_ctx *b)
{
    for (int i = 0; i < b->B; ++i) {
        cr_status s = init_state(b->inst[i]);
        if (s != CR_OK) return bfail(b, s, "instance %d: %s", i, b->inst[i]->err.c_str());
    }
    std::vector<int> ones(b->B, 1);
    CR_BCUDA(b, cudaMemcpyAsync(b->d_active, ones.data(), sizeof(int) * b->B, cudaMemcpyHostToDevice, b->stream));
    CR_BCUDA(b, cudaMemsetAsync(b->d_ell, 0, sizeof(long long), b->stream));
    CR_BCUDA(b, cudaMemsetAsync(b->d_err, 0, sizeof(int), b->stream));
    CR_BCUDA(b, cudaStreamSynchronize(b->stream));
    b->iters = 0;
    return CR_OK;
}

// One launch of `chunk` iterations (a graph replay when the launch could be captured).
cr_status batch_launch(cr_batch_ctx *b, long long chunk, int check_every, double tol)
{
    crk::BatchArgs A;
    A.inst = b->dP;
    A.item_inst = b->d_item_inst;
    A.item_vc = b->d_item_vc;
    A.off = b->d_off;
    A.active = b->d_active;
    A.ell_base = b->d_ell;
    A.bar_count = b->d_bar;
    A.error = b->d_err;
    A.bar_timeout_ns = b->inst[0]->P.bar_timeout_ns;
    A.Gphys = b->Gphys;
    A.B = b->B;
    void *args[] = {&A, &chunk, &check_every, &tol};
    const bool same = b->gexec && b->gchunk == chunk && b->gcheck == check_every && b->gtol == tol;
    if (!same && b->graph_ok) {
        if (b->gexec) {
            cudaGraphExecDestroy(b->gexec);
            b->gexec = nullptr;
        }
        cudaGraph_t g = nullptr;
        bool ok = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
            cudaMemsetAsync(b->d_bar, 0, sizeof(unsigned long long), b->stream);
            cudaLaunchCooperativeKernel(b->kernel(), dim3(b->Gphys), dim3(crk::kThreads), args, b->smem(), b->stream);
            ok = cudaStreamEndCapture(b->stream, &g) == cudaSuccess && g;
        }
        if (ok) ok = cudaGraphInstantiate(&b->gexec, g, 0) == cudaSuccess;
        if (g) cudaGraphDestroy(g);
        if (!ok) {
            (void)cudaGetLastError();
            b->gexec = nullptr;
            b->graph_ok = false;   // cooperative launches not capturable here: launch directly
        } else {
            b->gchunk = chunk;
            b->gcheck = check_every;
            b->gtol = tol;
        }
    }
    if (b->gexec) {
        CR_BCUDA(b, cudaGraphLaunch(b->gexec, b->stream));
        ++b->graph_launches;
    } else {
        ++b->direct_launches;
        CR_BCUDA(b, cudaMemsetAsync(b->d_bar, 0, sizeof(unsigned long long), b->stream));
        CR_BCUDA(b, cudaLaunchCooperativeKernel(b->kernel(), dim3(b->Gphys), dim3(crk::kThreads), args, b->smem(),
                                                b->stream));
    }
    return CR_OK;
}

cr_status batch_sync_error(cr_batch_ctx *b)
{
    int e = 0;
    CR_BCUDA(b, cudaMemcpyAsync(&e, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    CR_BCUDA(b, cudaStreamSynchronize(b->stream));
    if (e == crk::ERR_BARRIER || e == crk::ERR_PIPE) return bfail(b, CR_ETIMEOUT, "a bounded device wait gave up");
    if (e != 0) return bfail(b, CR_ENUMERIC, "device error %d", e);
    return CR_OK;
}

// Autotuner: times `probe` iterations for every tile shape (rows per pipeline stage: 16, or 8,
// which wastes fewer rows at the ragged end of a small instance's segments) and work granularity,
// and keeps the fastest pair.
cr_status batch_autotune(cr_batch_ctx *b, int probe, int fixed_rows)
{
    cudaEvent_t e0, e1;
    CR_BCUDA(b, cudaEventCreate(&e0));
    CR_BCUDA(b, cudaEventCreate(&e1));
    double best = 1e300;
    int bestf = 1, bestr = crk::kRS;
    b->tune_ms.clear();
    b->tune_factor.clear();
    b->tune_rows.clear();
    for (int rows : {crk::kRS, 8}) {
        if (fixed_rows != 0 && rows != fixed_rows) continue;
        b->stage_rows = rows;
        for (int f : kTuneFactors) {
            CR_TRY(batch_plan(b, f));
            CR_TRY(batch_reset(b));
            CR_TRY(batch_launch(b, 2, 0, -1.0));   // warm-up
            CR_BCUDA(b, cudaEventRecord(e0, b->stream));
            CR_TRY(batch_launch(b, probe, 0, -1.0));
            CR_BCUDA(b, cudaEventRecord(e1, b->stream));
            CR_TRY(batch_sync_error(b));
            float ms = 0.0f;
            CR_BCUDA(b, cudaEventElapsedTime(&ms, e0, e1));
            b->tune_ms.push_back(ms / probe);
            b->tune_factor.push_back(f);
            b->tune_rows.push_back(rows);
            if (ms < best) {
                best = ms;
                bestf = f;
                bestr = rows;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->stage_rows = bestr;
    CR_TRY(batch_plan(b, bestf));
    return batch_reset(b);
}

}  // namespace

extern "C" {

cr_status cr_batch_create(int32_t B, const int64_t *N, const int32_t *n, const double *const *X,
                          const double *const *ybar, const cr_options *opt, cr_batch_handle *out)
{
    if (!out) return create_error(CR_EINVAL, "out is NULL");
    *out = nullptr;
    if (B < 1 || !N || !n || !X || !ybar) return create_error(CR_EINVAL, "need B >= 1 and non-NULL arrays");
    cr_options o;
    if (opt) o = *opt;
    else cr_options_default(&o);
    int nmax = 0;
    for (int i = 0; i < B; ++i) {
        if (check_inputs(X[i], ybar[i], N[i], n[i]) != CR_OK)
            return create_error(CR_EINVAL, ("instance " + std::to_string(i) + ": invalid sizes or values").c_str());
        nmax = std::max(nmax, (int)n[i]);
    }
    cr_batch_ctx *b = new (std::nothrow) cr_batch_ctx();
    if (!b) return create_error(CR_ENOMEM, "out of host memory");
    b->B = B;
    b->NP = padded_n(nmax);
    b->ks = kernels_for(o.theta_dtype, b->NP);
    auto cleanup = [&](cr_status s) {
        cr_batch_destroy(b);
        return s;
    };
    if (!b->ks.batch || !b->ks.batch8) return cleanup(create_error(CR_EINVAL, "no kernel for this dtype / n"));
    if (o.stream) {
        b->stream = (cudaStream_t)o.stream;
    } else if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
        return cleanup(create_error(CR_ECUDA, "cannot create a stream"));
    } else {
        b->own_stream = true;
    }
    // instances: finest work items, shared stream, the batch's padded n
    for (int i = 0; i < B; ++i) {
        cr_options oi = o;
        oi.stream = b->stream;
        const double pairs = (double)N[i] * (double)(N[i] - 1);
        const long long Gf = std::max<long long>(1, (long long)std::ceil(pairs / (double)kPairsPerItemFine));
        oi.grid = (int)Gf;
        oi.driver = CR_DRIVER_PHASES;
        std::vector<double> Xv(X[i], X[i] + (size_t)N[i] * n[i]), yv(ybar[i], ybar[i] + N[i]);
        cr_handle h = nullptr;
        cr_status s = create_impl(Xv, yv, N[i], n[i], &oi, &h, b->NP);
        if (s != CR_OK) {
            std::string m = h ? h->err : "";
            cr_destroy(h);
            return cleanup(create_error(s, ("instance " + std::to_string(i) + ": " + m).c_str()));
        }
        b->inst.push_back(h);
        b->Gfine.push_back(Gf);
        // column partials sized for every granularity the autotuner may pick
        long long need = 0;
        for (int f : kTuneFactors) {
            const long long G = std::max<long long>(1, Gf / f);
            need = std::max<long long>(need, G * max_slots(h->P.total, h->N, (int)G));
        }
        if (need > (long long)h->P.G * h->P.slots) {
            float *cp = nullptr;
            if (dev_alloc(h, &cp, (size_t)need * crk::kWR * (b->NP + 1) * crk::kW) != CR_OK)
                return cleanup(create_error(CR_ENOMEM, "column partials"));
            cudaMemsetAsync(cp, 0, sizeof(float) * (size_t)need * crk::kWR * (b->NP + 1) * crk::kW, b->stream);
            h->P.colpart = cp;
        }
    }
    // physical grid: every co-resident CTA of the batch kernel
    // (both tile shapes: the smaller co-resident count of the two)
    int dev = 0, sms = 0, per_sm = 0, per_sm8 = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaFuncSetAttribute(b->ks.batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->ks.smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, b->ks.batch, crk::kThreads, b->ks.smem) != cudaSuccess ||
        cudaFuncSetAttribute(b->ks.batch8, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->ks.smem_batch8) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm8, b->ks.batch8, crk::kThreads, b->ks.smem_batch8) != cudaSuccess ||
        std::min(per_sm, per_sm8) < 1)
        return cleanup(create_error(CR_ECUDA, "batch kernel does not fit on this device"));
    b->Gphys = sms * std::min(per_sm, per_sm8);
    long long nitems = 0;
    for (long long g : b->Gfine) nitems += g;
    auto balloc = [&](void **p, size_t bytes) {
        if (cudaMalloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess) return false;
        b->allocs.push_back(*p);
        return true;
    };
    if (!balloc((void **)&b->dP, sizeof(Params) * B) || !balloc((void **)&b->d_item_inst, sizeof(int) * nitems) ||
        !balloc((void **)&b->d_item_vc, sizeof(int) * nitems) || !balloc((void **)&b->d_off, sizeof(int) * (b->Gphys + 1)) ||
        !balloc((void **)&b->d_active, sizeof(int) * B) || !balloc((void **)&b->d_ell, sizeof(long long)) ||
        !balloc((void **)&b->d_bar, sizeof(unsigned long long)) || !balloc((void **)&b->d_err, sizeof(int)))
        return cleanup(create_error(CR_ENOMEM, "batch descriptors"));
    if (o.batch_stage_rows != 0 && o.batch_stage_rows != 8 && o.batch_stage_rows != crk::kRS)
        return cleanup(create_error(CR_EINVAL, "batch_stage_rows must be 0 (autotuned), 8 or 16"));
    if (o.batch_stage_rows != 0) b->stage_rows = o.batch_stage_rows;
    cr_status s = (o.grid > 0) ? batch_plan(b, std::max(1, o.grid)) : batch_autotune(b, 8, o.batch_stage_rows);
    if (s == CR_OK && o.grid > 0) s = batch_reset(b);
    if (s != CR_OK) return cleanup(create_error(s, b->err.c_str()));
    *out = b;
    return CR_OK;
}

cr_status cr_batch_solve(cr_batch_handle b, double tol, int64_t max_iter, int64_t *converged)
{
    if (!b || max_iter < 0) return CR_EINVAL;
    if (converged) *converged = 0;
    const int check = std::max(1, (int)b->inst[0]->opt.kkt_every);
    long long done = 0;
    std::vector<int> act(b->B);
    int nact = b->B;
    while (done < max_iter && nact > 0) {
        const long long chunk = std::min<long long>(max_iter - done, 2000);
        CR_TRY(batch_launch(b, chunk, tol >= 0.0 ? check : 0, tol));
        CR_TRY(batch_sync_error(b));
        CR_BCUDA(b, cudaMemcpy(act.data(), b->d_active, sizeof(int) * b->B, cudaMemcpyDeviceToHost));
        nact = 0;
        for (int a : act) nact += a;
        done += chunk;
        b->iters += chunk;
    }
    // iteration counts of the instances (host view)
    for (int i = 0; i < b->B; ++i) {
        DevState st;
        CR_TRY(read_state(b->inst[i], &st));
        b->inst[i]->iters = st.iters_done;
    }
    if (converged) *converged = b->B - nact;
    return nact == 0 ? CR_OK : CR_NOT_CONVERGED;
}

cr_status cr_batch_iterate(cr_batch_handle b, int64_t k)
{
    if (!b || k < 0) return CR_EINVAL;
    long long done = 0;
    while (done < k) {
        const long long chunk = std::min<long long>(k - done, 2000);
        CR_TRY(batch_launch(b, chunk, 0, -1.0));
        done += chunk;
    }
    CR_TRY(batch_sync_error(b));
    b->iters += k;
    for (int i = 0; i < b->B; ++i) {
        DevState st;
        CR_TRY(read_state(b->inst[i], &st));
        b->inst[i]->iters = st.iters_done;
    }
    return CR_OK;
}

cr_status cr_batch_reset(cr_batch_handle b)
{
    if (!b) return CR_EINVAL;
    return batch_reset(b);
}

cr_status cr_batch_instance(cr_batch_handle b, int32_t i, cr_handle *h)
{
    if (!b || i < 0 || i >= b->B || !h) return CR_EINVAL;
    *h = b->inst[i];
    return CR_OK;
}

cr_status cr_batch_info(cr_batch_handle b, int32_t *factor, int32_t *grid, int64_t *iters)
{
    if (!b) return CR_EINVAL;
    if (factor) *factor = b->factor;
    if (grid) *grid = b->Gphys;
    if (iters) *iters = b->iters;
    return CR_OK;
}

cr_status cr_batch_stats(cr_batch_handle b, int32_t *graph_live, int64_t *graph_launches, int64_t *direct_launches,
                         int32_t *tuned, double *tune_ms)
{
    if (!b) return CR_EINVAL;
    if (graph_live) *graph_live = (b->graph_ok && b->gexec) ? 1 : 0;
    if (graph_launches) *graph_launches = b->graph_launches;
    if (direct_launches) *direct_launches = b->direct_launches;
    if (tuned) *tuned = (int32_t)b->tune_factor.size();
    if (tune_ms)
        for (size_t i = 0; i < b->tune_ms.size() && i < 8; ++i) tune_ms[i] = b->tune_ms[i];
    return CR_OK;
}

cr_status cr_batch_tuning(cr_batch_handle b, int32_t cap, int32_t *count, int32_t *stage_rows, int32_t *factor,
                          int32_t *cand_rows, int32_t *cand_factor, double *cand_ms)
{
    if (!b || cap < 0) return CR_EINVAL;
    if (stage_rows) *stage_rows = b->stage_rows;
    if (factor) *factor = b->factor;
    if (count) *count = (int32_t)b->tune_ms.size();
    for (size_t i = 0; i < b->tune_ms.size() && (int32_t)i < cap; ++i) {
        if (cand_rows) cand_rows[i] = b->tune_rows[i];
        if (cand_factor) cand_factor[i] = b->tune_factor[i];
        if (cand_ms) cand_ms[i] = b->tune_ms[i];
    }
    return CR_OK;
}

void cr_batch_destroy(cr_batch_handle b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    for (cr_handle h : b->inst) cr_destroy(h);
    for (void *p : b->allocs) cudaFree(p);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

const char *cr_batch_last_error(cr_batch_handle b) { return b ? b->err.c_str() : g_create_err.c_str(); }

}  // extern "C"
