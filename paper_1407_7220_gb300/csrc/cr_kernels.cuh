// cr_kernels.cuh -- device code of the GB300 P-APG convex-regression solver.
//
// Method: Aybat & Wang, arXiv:1407.7220, P-APG (Fig. 2) on the dual
// (lambda_dual) of problem (regularize) with every pairwise constraint of
// problem (original) dualized (K = N).  One iteration l is split into phases:
//
//   foldB(l)  Step 1 at theta^(2)_l by linearity of the closed form:
//             eta(theta^(2)_l) = (1+beta) eta(theta^(1)_{l-1}) - beta eta(theta^(1)_{l-2})
//             plus Step 2 for the y >= 0 rows (mu) and Steps 3-4 scalars (t, beta).
//   pair(l)   Step 2 for every pair p = (l1,l2): theta^(2) = cur + beta (cur - prev),
//             g = (C eta)_p, theta^(1)_l = max(0, theta^(2) - g / L), written over prev;
//             fused adjoint: row sums, column sums and theta^T X partials of the new array.
//   foldA(l)  FP64 reduction of the partials into A_1^T theta, A_2^T theta of theta^(1)_l,
//             the minimizer eta(theta^(1)_l) and the dual value g_gamma(theta^(1)_l).
//   kkt       KKT residual terms at theta^(1)_l (FP32 screen, FP64 confirmation).
//
// Layout (row-major): theta[b] is N x ld, theta[l1*ld + l2] = multiplier of pair (l1,l2);
// columns N..ld-1 and the diagonal hold 0.  The pair pass tiles the array in stripes of
// W = 256 columns; CTA c owns the contiguous range [c*U, (c+1)*U) of (stripe, row) units,
// stripe-major, so each CTA walks down at most a few stripes and keeps its column
// accumulators in registers.  Eight warps per CTA: 2 across a stripe x 4 row groups;
// each thread owns 4 adjacent columns (one 16-byte FP32 vector or 8-byte 16-bit vector).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace crk {

constexpr int kThreads = 256;   // 8 warps per CTA
constexpr int kCons = kThreads; // every warp consumes pair-pass stages; lane 0 of warp 0 also produces them
constexpr int kW = 256;         // stripe width (columns)
constexpr int kWR = 4;          // row groups of consumer warps (2 warps per row)
constexpr int kRS = 8;          // rows per pipeline stage
constexpr int kMaxStages = 16;
constexpr size_t kSmemBudget = 227 * 1024 - 2048;   // dynamic shared memory per CTA (static arrays excluded)

template <int NP> struct RecLayout {
    static constexpr int REC = ((NP + 1 + 3) / 4) * 4;   // floats per row record (16-byte multiple)
};

enum : int {
    ERR_BARRIER = 1,   // grid barrier wait exceeded its bound
    ERR_NUMERIC = 2,   // non-finite value in the fold
    ERR_PIPE = 3,      // a pipeline (mbarrier) wait exceeded its bound
};

// Per-iteration scalar state; two slots indexed by iteration parity so that the
// phase that writes slot (l & 1) never races with readers of slot ((l-1) & 1).
struct Scal {
    double t;          // t of Fig. 2 step 3 after this iteration's update
    double dual;       // g_gamma(theta^(1)) the restart test compares against
    double beta;       // momentum weight used to form theta^(2)_l
    long long restarts;
};

struct DevState {
    Scal scal[2];
    unsigned long long bar_count;  // monotone grid-barrier counter (reset before each launch)
    long long iters_done;          // written by the persistent kernel at exit
    int error;
    int converged;
    int pad[2];
    double kkt[8];      // last reduced KKT terms: 0 kkt,1 pri,2 comp,3 infeas,4 gap,5 screen
};

struct Params {
    CUtensorMap tmap[2];    // TMA descriptors of theta[0], theta[1]: N x N, box kRS x kW
    // sizes
    long long N;
    int n;
    int NP;             // padded n (template value, for host checks)
    long long ld;       // row stride of theta (elements)
    int S;              // stripes = ceil(N / kW)
    int G;              // CTAs of the grid
    int slots;          // column-partial slots per CTA
    long long total;    // S * N units
    // constants
    double gamma, inv_gamma, L, invL_d, shift, sigma;
    float invL;
    float st_scale, st_inv_scale;   // theta storage scale (FP16 only; 1 otherwise)
    int momentum, restart, sr;
    double restart_tol;
    unsigned int seed;
    unsigned long long bar_timeout_ns;   // bound of every grid-barrier wait
    int bar_extra;                       // test hook: extra arrivals a barrier waits for (0 in use)
    // arrays
    void *theta[2];
    const double *X64;      // N x n
    float *rowrec;          // N x REC row records {y(theta^(2)) - s, x_1..x_n, 0...} (FP32)
    const double *h;        // N, ybar + s
    float *ccol2, *xi2;     // column data at theta^(2): xi.x - (y - s), xi (N x NP)
    float *yrow1, *ccol1, *xi1;     // same at theta^(1) (KKT screen)
    double *y1, *xi1_64;            // eta(theta^(1)) in FP64 (y shifted)
    double *v[2];           // A_1^T theta^(1) of the two latest iterates (N)
    double *w[2];           // A_2^T theta^(1) (N x n)
    double *mu[2];          // multipliers of the y >= 0 rows (N)
    float *rowpart;         // [N][Q]: row sums per (stripe, column half), Q = ceil4(2S), padding 0
    int Q;
    float *colpart;         // [G][slots][NP+1][kW]
    double *foldpart;       // [G][8]
    double *kktpart;        // [G][8]
    DevState *st;
};

// ---------------------------------------------------------------------------
// storage types
// ---------------------------------------------------------------------------
template <typename TS> struct Store;

__device__ __forceinline__ uint32_t hash3(uint32_t a, uint32_t b, uint32_t c)
{
    // counter-based: a multiply-xor mix of the counters followed by the
    // "lowbias32" integer finalizer (C. Wellons' hash-prospector)
    uint32_t x = a * 0x9E3779B1u ^ (b * 0x85EBCA77u + 0x165667B1u) ^ (c * 0xC2B2AE3Du + 0x27D4EB2Fu);
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

template <> struct Store<float> {
    using Vec = float4;
    __device__ static __forceinline__ void unpack(const Vec &v, float (&o)[4], float)
    {
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    }
    // Projected update max(0, th2 - g/L) rounded to the stored type.  v = RN(th2 - g*invL);
    // with SR the rounding residual e (exact while th2 and v are within 2x) decides the
    // unbiased step to a neighbour: k = floor(e/ulp(v) + u), u uniform in [0,1) from 16 bits.
    template <bool SR>
    __device__ static __forceinline__ float round(float th2, float g, float invL, uint32_t rnd16, float)
    {
        const float v = fmaf(-g, invL, th2);
        float r = v;
        if (SR) {
            const float e = fmaf(-g, invL, th2 - v);
            const uint32_t b = __float_as_uint(v);
            const uint32_t ef = max(b & 0x7F800000u, 23u << 23);
            const float inv_ulp = __uint_as_float(0x8A800000u - ef);          // 2^(23 - exponent(v))
            const float u1 = __uint_as_float(0x3F800000u | (rnd16 << 7));     // 1 + u
            const int kk = __float2int_rd(fmaf(e, inv_ulp, u1));             // floor(e/ulp + u) + 1
            r = __uint_as_float(b + (uint32_t)kk - 1u);
        }
        return v > 0.0f ? r : 0.0f;
    }
    __device__ static __forceinline__ float encode(float v, float) { return v; }
    __device__ static __forceinline__ Vec pack(const float (&s)[4]) { return make_float4(s[0], s[1], s[2], s[3]); }
    __device__ static __forceinline__ float decoded(float s, float) { return s; }
};

template <> struct Store<__nv_bfloat16> {
    using Vec = uint2;  // 4 x bf16
    __device__ static __forceinline__ float b2f(uint32_t bits16) { return __uint_as_float(bits16 << 16); }
    __device__ static __forceinline__ void unpack(const Vec &v, float (&o)[4], float)
    {
        o[0] = b2f(v.x & 0xFFFFu); o[1] = b2f(v.x >> 16);
        o[2] = b2f(v.y & 0xFFFFu); o[3] = b2f(v.y >> 16);
    }
    // returns the value actually stored (as float); bf16 bits kept in the float's top half
    template <bool SR>
    __device__ static __forceinline__ float round(float th2, float g, float invL, uint32_t rnd16, float)
    {
        const float v = fmaf(-g, invL, th2);
        uint32_t b = __float_as_uint(v);
        if (SR) b += rnd16;                                        // stochastic: add uniform 16-bit noise, truncate
        else b += 0x7FFFu + ((b >> 16) & 1u);                      // round to nearest even
        b &= 0xFFFF0000u;
        return v > 0.0f ? __uint_as_float(b) : 0.0f;
    }
    __device__ static __forceinline__ Vec pack(const float (&s)[4])
    {
        Vec v;
        v.x = (__float_as_uint(s[0]) >> 16) | (__float_as_uint(s[1]) & 0xFFFF0000u);
        v.y = (__float_as_uint(s[2]) >> 16) | (__float_as_uint(s[3]) & 0xFFFF0000u);
        return v;
    }
    __device__ static __forceinline__ float decoded(float s, float) { return s; }
};

template <> struct Store<__half> {
    using Vec = uint2;  // 4 x fp16, value = half * inv_scale
    __device__ static __forceinline__ float h2f(uint32_t bits16, float inv_scale)
    {
        return __half2float(__ushort_as_half((unsigned short)bits16)) * inv_scale;
    }
    __device__ static __forceinline__ void unpack(const Vec &v, float (&o)[4], float inv_scale)
    {
        o[0] = h2f(v.x & 0xFFFFu, inv_scale); o[1] = h2f(v.x >> 16, inv_scale);
        o[2] = h2f(v.y & 0xFFFFu, inv_scale); o[3] = h2f(v.y >> 16, inv_scale);
    }
    // returns the scaled half value (as float, exactly representable in fp16)
    template <bool SR>
    __device__ static __forceinline__ float round(float th2, float g, float invL, uint32_t rnd16, float scale)
    {
        const float v = fmaf(-g, invL, th2);
        const float sv = fminf(fmaxf(v, 0.0f) * scale, 65504.0f);
        float r;
        if (SR) {
            const __half hz = __float2half_rz(sv);
            const float lo = __half2float(hz);
            const float hi = __half2float(__ushort_as_half((unsigned short)(__half_as_ushort(hz) + 1)));
            r = ((float)rnd16 * (hi - lo) < (sv - lo) * 65536.0f) ? hi : lo;
        } else {
            r = __half2float(__float2half_rn(sv));
        }
        return v > 0.0f ? r : 0.0f;
    }
    __device__ static __forceinline__ Vec pack(const float (&s)[4])
    {
        Vec v;
        v.x = (uint32_t)__half_as_ushort(__float2half_rn(s[0])) | ((uint32_t)__half_as_ushort(__float2half_rn(s[1])) << 16);
        v.y = (uint32_t)__half_as_ushort(__float2half_rn(s[2])) | ((uint32_t)__half_as_ushort(__float2half_rn(s[3])) << 16);
        return v;
    }
    __device__ static __forceinline__ float decoded(float s, float inv_scale) { return s * inv_scale; }
};

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// --- PTX wrappers: mbarrier, TMA, proxy fence, named barrier ---
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
// generic-proxy writes (earlier phases) ordered before async-proxy (TMA) reads
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.global;" ::: "memory"); }
__device__ __forceinline__ void named_barrier_sync(int id, int count)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Block reduction of K doubles (sum or max per component) into out[] of thread 0;
// fixed order, hence deterministic.  red: shared scratch of 8*K doubles.
template <int K>
__device__ __forceinline__ void block_reduce(double (&v)[K], const bool (&is_max)[K], double *red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < K; ++i) v[i] = is_max[i] ? warp_max(v[i]) : warp_sum(v[i]);
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < K; ++i) red[warp * K + i] = v[i];
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < K; ++i) {
            double a = red[i];
            for (int w = 1; w < kThreads / 32; ++w) a = is_max[i] ? fmax(a, red[w * K + i]) : a + red[w * K + i];
            v[i] = a;
        }
    }
    __syncthreads();
}

// Grid-wide barrier for a cooperative launch of G CTAs.  Monotone counter:
// barrier number b completes when the counter reaches (b+1)*G (+ extra, a test
// hook).  The wait is bounded by wall time; on timeout the error word is set and
// every CTA leaves.
__device__ __forceinline__ bool bounded_grid_barrier(unsigned long long *count, int *error, unsigned long long G,
                                                     unsigned long long extra, unsigned long long timeout_ns,
                                                     unsigned long long &bar_no)
{
    __syncthreads();
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();
        const unsigned long long target = (bar_no + 1ull) * G + extra;
        atomicAdd(count, 1ull);
        const unsigned long long t0 = globaltimer();
        while (true) {
            unsigned long long c;
            asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(c) : "l"(count) : "memory");
            if (c >= target) break;
            if (*((volatile int *)error) != 0) { ok = 0; break; }
            if (globaltimer() - t0 > timeout_ns) {
                atomicCAS(error, 0, ERR_BARRIER);
                ok = 0;
                break;
            }
            __nanosleep(40);
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    ++bar_no;
    return s_ok != 0;
}

__device__ __forceinline__ bool grid_barrier(const Params &P, unsigned long long &bar_no)
{
    return bounded_grid_barrier(&P.st->bar_count, &P.st->error, (unsigned long long)P.G,
                                (unsigned long long)P.bar_extra, P.bar_timeout_ns, bar_no);
}

// CTA c's unit range [u0, u1) of the stripe-major (stripe, row) order.
__device__ __forceinline__ long long unit_begin(const Params &P, long long c)
{
    return (long long)(((unsigned long long)c * (unsigned long long)P.total) / (unsigned long long)P.G);
}

// Bounded mbarrier phase wait: gives up (and sets the error word) after the
// barrier bound, or at once when another CTA already reported an error.
__device__ __forceinline__ bool mbar_wait(const Params &P, uint64_t *bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*((volatile int *)&P.st->error) != 0) return false;
        if (globaltimer() - t0 > P.bar_timeout_ns) {
            atomicCAS(&P.st->error, 0, ERR_PIPE);
            return false;
        }
    }
}

// ---------------------------------------------------------------------------
// foldB(l): Step 1 at theta^(2)_l (by linearity), mu update, Steps 3-4 scalars
// ---------------------------------------------------------------------------
template <int NP>
__device__ void phase_foldB(const Params &P, long long ell, double *red, long long vc)
{
    const int c = (int)((ell - 1) & 1), p = (int)(ell & 1);
    __shared__ double s_beta;
    if (threadIdx.x < 32) {
        // every CTA reduces the dual-value partials of foldA(l-1) in the same order
        double a = 0.0, b = 0.0, cc = 0.0;
        for (int i = threadIdx.x; i < P.G; i += 32) {
            a += __ldcg(P.foldpart + i * 8 + 0);
            b += __ldcg(P.foldpart + i * 8 + 1);
            cc += __ldcg(P.foldpart + i * 8 + 2);
        }
        a = warp_sum(a);
        b = warp_sum(b);
        cc = warp_sum(cc);
        if (threadIdx.x == 0) {
            Scal old;
            old.t = __ldcg(&P.st->scal[c].t);
            old.dual = __ldcg(&P.st->scal[c].dual);
            old.beta = __ldcg(&P.st->scal[c].beta);
            old.restarts = __ldcg(&P.st->scal[c].restarts);
            Scal nw = old;
            double beta = 0.0;
            if (ell >= 2) {
                // g_gamma(theta^(1)_{l-1}) = 1/2||u||^2 + gamma/2||xi||^2 - theta^T C eta,
                // theta^T C eta = u^T y + gamma||xi||^2, u = y - h (Eq. (eq:g_gamma))
                double dv = 0.5 * a - cc - 0.5 * P.gamma * b;
                double t = old.t;
                if (P.restart && dv < old.dual - P.restart_tol * fabs(old.dual)) {
                    t = 1.0;
                    nw.restarts = old.restarts + 1;
                }
                double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));   // Fig. 2 step 3
                beta = P.momentum ? (t - 1.0) / tn : 0.0;           // Fig. 2 step 4 weight
                nw.t = tn;
                nw.dual = dv;
            }
            nw.beta = beta;
            s_beta = beta;
            if (vc == 0) P.st->scal[p] = nw;
        }
    }
    __syncthreads();
    const double beta = s_beta, b1 = 1.0 + beta;
    const long long N = P.N;
    const int n = P.n;
    for (long long l = vc * kThreads + threadIdx.x; l < N; l += (long long)P.G * kThreads) {
        double v2 = b1 * __ldcg(P.v[c] + l) - beta * __ldcg(P.v[p] + l);
        double mu2 = b1 * __ldcg(P.mu[c] + l) - beta * __ldcg(P.mu[p] + l);
        double y2 = __ldg(P.h + l) + v2 + mu2;
        double mun = mu2 - y2 * P.invL_d;     // Step 2 on the y >= 0 rows of C
        P.mu[p][l] = mun > 0.0 ? mun : 0.0;
        double ys = y2 - P.shift;
        double d = 0.0;
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            float xf = 0.0f;
            if (k < n) {
                double xi = (b1 * __ldcg(P.w[c] + l * n + k) - beta * __ldcg(P.w[p] + l * n + k)) * P.inv_gamma;
                d += xi * __ldg(P.X64 + l * n + k);
                xf = (float)xi;
            }
            P.xi2[l * NP + k] = xf;
        }
        P.rowrec[l * RecLayout<NP>::REC] = (float)ys;
        P.ccol2[l] = (float)(d - ys);
    }
}

// ---------------------------------------------------------------------------
// pair(l): Step 2 over all pairs + fused adjoint partial sums
//
// Warp-specialized pipeline per CTA: warp 8 (one lane) is the producer -- for every
// stage of kRS rows of the current stripe it issues two tiled TMA loads
// (cp.async.bulk.tensor.2d) of the theta^(1)_{l-1} and theta^(1)_{l-2} tiles
// [kRS x 256] and one bulk copy of the kRS row records (y_row, x), completing on the
// stage's "full" mbarrier.  Warps 0-7 consume: each takes 2 rows x 128 columns of the
// stage from shared memory, writes theta^(1)_l straight to global memory (16-byte or
// 8-byte vector stores) and arrives on the stage's "empty" mbarrier.  Out-of-range
// rows/columns of a tile are zero-filled by the TMA unit.
// ---------------------------------------------------------------------------

template <typename TS, int NP> struct PairSmem {
    static constexpr int REC = RecLayout<NP>::REC;
    static constexpr size_t tile_bytes = (size_t)kRS * kW * sizeof(TS);
    static constexpr size_t rec_bytes = (size_t)kRS * REC * sizeof(float);
    static constexpr size_t stage_bytes = 2 * tile_bytes + rec_bytes;
    static constexpr size_t flush_bytes = (size_t)kWR * (NP + 1) * kW * sizeof(float);
    // as many stages as fit next to the column-partial buffer (more bytes in flight per SM)
    static constexpr int kFit = (int)((kSmemBudget - flush_bytes - 128) / stage_bytes);
    static constexpr int kStages = kFit < kMaxStages ? kFit : kMaxStages;
    static_assert(kStages >= 2, "pipeline needs at least two stages");
    static constexpr size_t bytes = kStages * stage_bytes + flush_bytes + 128;   // + base alignment slack
    static_assert(tile_bytes % 128 == 0 && rec_bytes % 128 == 0, "stage buffers must stay 128-byte aligned");
};

// The two rows (rg, rg + 4) of one pipeline stage for one consumer warp, 4 columns per
// lane.  MASK handles the diagonal (l1 == l2), columns >= N and rows past the segment;
// stages without any of these take the unmasked instantiation.  SR: stochastic rounding.
template <typename TS, int NP, bool MASK, bool SR>
__device__ __forceinline__ void pair_stage_rows(const TS *tcur, const TS *tprv, const float *rec, int rg, int cofs,
                                                long long r, long long r1, long long col0, long long N, long long ld,
                                                const float (&ccol)[4], const float (&xi)[4][NP], float (&acc)[4][NP],
                                                float (&csum)[4], float beta, float invL, uint32_t rseed, float scl,
                                                float iscl, TS *__restrict__ nxt, bool vec_ok, float &rs0, float &rs1)
{
    using St = Store<TS>;
    using Vec = typename St::Vec;
    constexpr int REC = RecLayout<NP>::REC;
    float rsv[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int rl = rg + i * kWR;
        const long long rr = r + rl;
        const bool valid = !MASK || rr < r1;
        float rv[REC];
#pragma unroll
        for (int q = 0; q < REC; q += 4) {
            const float4 t4 = *reinterpret_cast<const float4 *>(rec + rl * REC + q);
            rv[q] = t4.x; rv[q + 1] = t4.y; rv[q + 2] = t4.z; rv[q + 3] = t4.w;
        }
        float tc[4], tp[4], outv[4];
        St::unpack(*reinterpret_cast<const Vec *>(tcur + rl * kW + cofs), tc, iscl);
        St::unpack(*reinterpret_cast<const Vec *>(tprv + rl * kW + cofs), tp, iscl);
        uint32_t h = 0, h2 = 0;
        if (SR) {
            h = hash3((uint32_t)rr, (uint32_t)(col0 >> 2), rseed);
            h2 = (h ^ (h >> 15)) * 0x2C1B3C6Du;
        }
        const uint32_t rnd[4] = {h & 0xFFFFu, h >> 16, h2 & 0xFFFFu, h2 >> 16};
        float rs = 0.0f;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float th2 = fmaf(beta, tc[j] - tp[j], tc[j]);  // theta^(2) = theta^(1) + beta (theta^(1) - prev)
            // (C eta)_p = y_l1 - y_l2 + xi_l2.x_l2 - xi_l2.x_l1, summed in two chains
            float g0 = rv[0] + ccol[j], g1 = 0.0f;
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                if (k & 1) g1 = fmaf(-xi[j][k], rv[1 + k], g1);
                else g0 = fmaf(-xi[j][k], rv[1 + k], g0);
            }
            float sv = St::template round<SR>(th2, g0 + g1, invL, rnd[j], scl);   // Pi_{>=0}(theta^(2) - g/L)
            if (MASK) {
                if (!valid || col0 + j >= N || col0 + j == rr) sv = 0.0f;
            }
            outv[j] = sv;
            const float vv = St::decoded(sv, iscl);
            rs += vv;                                                // row sum    (A_1^T, + part)
            csum[j] += vv;                                           // column sum (A_1^T, - part)
#pragma unroll
            for (int k = 0; k < NP; ++k) acc[j][k] = fmaf(vv, rv[1 + k], acc[j][k]);   // theta^T X (A_2^T)
        }
        if (vec_ok && valid) *reinterpret_cast<Vec *>(nxt + rr * ld + col0) = St::pack(outv);
        rsv[i] = rs;
    }
    rs0 = rsv[0];
    rs1 = rsv[1];
}

// Row sums of a batch of up to 4 stages (8 rows per warp) reduced across the warp with a
// transposing butterfly: 9 shuffles leave the full sum of batch entry
// e = 4*bit4 + 2*bit3 + bit2 (of the lane id) in every lane.  Entry e is row
// r_last - kRS*(3 - e/2) + rg + kWR*(e & 1); only the nb most recent stages are written.
__device__ __forceinline__ void flush_row_sums(float (&v)[8], int nb, long long r_last, int rg, long long r1,
                                               float *rp, int Q, int lane)
{
    const unsigned full = 0xffffffffu;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const bool hi = lane & 16;
        const float send = hi ? v[i] : v[i + 4], keep = hi ? v[i + 4] : v[i];
        v[i] = keep + __shfl_xor_sync(full, send, 16);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const bool hi = lane & 8;
        const float send = hi ? v[i] : v[i + 2], keep = hi ? v[i + 2] : v[i];
        v[i] = keep + __shfl_xor_sync(full, send, 8);
    }
    {
        const bool hi = lane & 4;
        const float send = hi ? v[0] : v[1], keep = hi ? v[1] : v[0];
        v[0] = keep + __shfl_xor_sync(full, send, 4);
    }
    v[0] += __shfl_xor_sync(full, v[0], 2);
    v[0] += __shfl_xor_sync(full, v[0], 1);
    if ((lane & 3) == 0) {
        const int e = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
        const int sp = e >> 1;
        const long long row = r_last - (long long)kRS * (3 - sp) + rg + kWR * (e & 1);
        if (sp >= 4 - nb && row < r1) rp[row * Q] = v[0];
    }
}

// Producer cursor: walks the CTA's stages (kRS rows of one stripe) in consumption order.
struct StageCursor {
    long long u, uend, s, r0, r1, r;
    __device__ __forceinline__ void begin(long long u0, long long ue, long long N)
    {
        u = u0;
        uend = ue;
        r = -1;
        next_segment(N);
    }
    __device__ __forceinline__ void next_segment(long long N)
    {
        if (u >= uend) return;
        s = u / N;
        r0 = u - s * N;
        r1 = min(N, r0 + (uend - u));
        r = r0;
    }
    __device__ __forceinline__ void advance(long long N)
    {
        r += kRS;
        if (r >= r1) {
            u += r1 - r0;
            next_segment(N);
        }
    }
};

// Issue stage number k (global count) into its ring slot: wait until the slot's previous
// occupant (stage k - S) was released by all 8 warps, then two tiled TMA loads and one
// bulk copy complete on the slot's "full" barrier.
template <typename TS, int NP>
__device__ __forceinline__ bool produce_stage(const Params &P, unsigned char *stage0, uint64_t *full, uint64_t *empty,
                                              unsigned long long k, const StageCursor &cur, int c, int p)
{
    using L = PairSmem<TS, NP>;
    constexpr int S = L::kStages;
    const int slot = (int)(k % S);
    const unsigned long long round = k / S;
    if (round > 0 && !mbar_wait(P, &empty[slot], (uint32_t)((round - 1) & 1))) return false;
    const int nrows = (int)min((long long)kRS, cur.r1 - cur.r);
    unsigned char *st = stage0 + slot * L::stage_bytes;
    mbar_arrive_expect_tx(&full[slot], (uint32_t)(2 * L::tile_bytes + (size_t)nrows * L::REC * 4));
    tma_load_2d(st, &P.tmap[c], (int)(cur.s * kW), (int)cur.r, &full[slot]);
    tma_load_2d(st + L::tile_bytes, &P.tmap[p], (int)(cur.s * kW), (int)cur.r, &full[slot]);
    bulk_load(st + 2 * L::tile_bytes, P.rowrec + cur.r * L::REC, (uint32_t)(nrows * L::REC * 4), &full[slot]);
    return true;
}

template <typename TS, int NP>
__device__ void phase_pair(const Params &P, long long ell, unsigned char *smem, uint64_t *full, uint64_t *empty,
                           unsigned long long &kstage, long long vc)
{
    using St = Store<TS>;
    using L = PairSmem<TS, NP>;
    constexpr int S = L::kStages;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int p = (int)(ell & 1), c = 1 - p;
    const long long N = P.N, ld = P.ld;
    const long long ubeg = unit_begin(P, vc);
    const long long uend = unit_begin(P, vc + 1);
    unsigned char *stage0 = smem;
    float *flush = reinterpret_cast<float *>(smem + S * L::stage_bytes);

    // number of stages of this pass (identical in every thread)
    unsigned long long nst = 0;
    for (long long u = ubeg; u < uend;) {
        const long long s = u / N, r0 = u - s * N, r1 = min(N, r0 + (uend - u));
        nst += (unsigned long long)((r1 - r0 + kRS - 1) / kRS);
        u += r1 - r0;
    }
    const unsigned long long kend = kstage + nst;

    // producer (lane 0 of warp 0): prefill the ring
    const bool producer = (tid == 0);
    StageCursor pc;
    unsigned long long kprod = kstage;
    bool pok = true;
    if (producer) {
        fence_proxy_async();
        pc.begin(ubeg, uend, N);
        for (; kprod < kend && kprod < kstage + S && pok; ++kprod) {
            pok = produce_stage<TS, NP>(P, stage0, full, empty, kprod, pc, c, p);
            pc.advance(N);
        }
    }
    __syncwarp();

    const int wc = warp & 1, rg = warp >> 1;
    const float beta = (float)__ldcg(&P.st->scal[p].beta);
    const float invL = P.invL;
    const float scl = P.st_scale, iscl = P.st_inv_scale;
    const bool sr = P.sr != 0;
    const uint32_t rseed = P.seed ^ (uint32_t)ell * 0x632BE5ABu;
    TS *__restrict__ nxt = (TS *)P.theta[p];   // theta^(1)_{l-2} on entry, theta^(1)_l on exit
    const long long first_stripe = ubeg / N;
    unsigned long long k = kstage;
    bool ok = true;
    for (long long u = ubeg; u < uend;) {
        const long long s = u / N, r0 = u - s * N, r1 = min(N, r0 + (uend - u));
        const long long colw = s * kW + wc * 128;       // first column of this warp
        const long long col0 = colw + lane * 4;
        const bool vec_ok = col0 < ld;
        const bool ragged = (s * kW + kW) > N;
        float ccol[4], xi[4][NP];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const long long cj = col0 + j;
            const bool v = cj < N;
            ccol[j] = v ? __ldcg(P.ccol2 + cj) : 0.0f;
#pragma unroll
            for (int q = 0; q < NP; ++q) xi[j][q] = v ? __ldcg(P.xi2 + cj * NP + q) : 0.0f;
        }
        float acc[4][NP], csum[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            csum[j] = 0.0f;
#pragma unroll
            for (int q = 0; q < NP; ++q) acc[j][q] = 0.0f;
        }
        float *rp = P.rowpart + (s * 2 + wc);   // row r's partial at rp[r * Q]
        const int cofs = wc * 128 + lane * 4;
        float rsb[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) rsb[q] = 0.0f;
        int nb = 0;
        for (long long r = r0; r < r1; r += kRS, ++k) {
            const int slot = (int)(k % S);
            if (ok && !mbar_wait(P, &full[slot], (uint32_t)((k / S) & 1))) ok = false;
            float ra = 0.0f, rb = 0.0f;
            if (ok) {
                const unsigned char *st = stage0 + slot * L::stage_bytes;
                const TS *tcur = reinterpret_cast<const TS *>(st);
                const TS *tprv = reinterpret_cast<const TS *>(st + L::tile_bytes);
                const float *rec = reinterpret_cast<const float *>(st + 2 * L::tile_bytes);
                const bool fast = !ragged && (r + kRS <= r1) && !(r < colw + 128 && colw < r + kRS);
                if (sr) {
                    if (fast)
                        pair_stage_rows<TS, NP, false, true>(tcur, tprv, rec, rg, cofs, r, r1, col0, N, ld, ccol, xi,
                                                             acc, csum, beta, invL, rseed, scl, iscl, nxt, vec_ok,
                                                             ra, rb);
                    else
                        pair_stage_rows<TS, NP, true, true>(tcur, tprv, rec, rg, cofs, r, r1, col0, N, ld, ccol, xi,
                                                            acc, csum, beta, invL, rseed, scl, iscl, nxt, vec_ok,
                                                            ra, rb);
                } else {
                    if (fast)
                        pair_stage_rows<TS, NP, false, false>(tcur, tprv, rec, rg, cofs, r, r1, col0, N, ld, ccol,
                                                              xi, acc, csum, beta, invL, rseed, scl, iscl, nxt,
                                                              vec_ok, ra, rb);
                    else
                        pair_stage_rows<TS, NP, true, false>(tcur, tprv, rec, rg, cofs, r, r1, col0, N, ld, ccol,
                                                             xi, acc, csum, beta, invL, rseed, scl, iscl, nxt,
                                                             vec_ok, ra, rb);
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[slot]);
            if (producer && pok && kprod < kend) {   // refill this slot with stage k + S
                pok = produce_stage<TS, NP>(P, stage0, full, empty, kprod, pc, c, p);
                pc.advance(N);
                ++kprod;
            }
            __syncwarp();   // reconverge warp 0 after the producer lane
            // shift the row-sum batch (most recent stage in entries 6, 7)
#pragma unroll
            for (int q = 0; q < 6; ++q) rsb[q] = rsb[q + 2];
            rsb[6] = ra;
            rsb[7] = rb;
            ++nb;
            if (nb == 4 || r + kRS >= r1) {
                flush_row_sums(rsb, nb, r, rg, r1, rp, P.Q, lane);
#pragma unroll
                for (int q = 0; q < 8; ++q) rsb[q] = 0.0f;
                nb = 0;
            }
        }
        // column partials of this segment: reduce the 4 row groups in shared memory
        const int slotc = (int)(s - first_stripe);
        float *cp = P.colpart + (vc * P.slots + slotc) * (NP + 1) * kW;
        const int cl = wc * 128 + lane * 4;
        named_barrier_sync(1, kCons);
        *reinterpret_cast<float4 *>(flush + (rg * (NP + 1)) * kW + cl) = make_float4(csum[0], csum[1], csum[2], csum[3]);
#pragma unroll
        for (int q = 0; q < NP; ++q)
            *reinterpret_cast<float4 *>(flush + (rg * (NP + 1) + 1 + q) * kW + cl) =
                make_float4(acc[0][q], acc[1][q], acc[2][q], acc[3][q]);
        named_barrier_sync(1, kCons);
        for (int e = tid; e < (NP + 1) * kW; e += kCons) {
            float a = flush[e];
#pragma unroll
            for (int q = 1; q < kWR; ++q) a += flush[q * (NP + 1) * kW + e];
            cp[e] = a;
        }
        named_barrier_sync(1, kCons);
        u += r1 - r0;
    }
    kstage += nst;
    __syncthreads();
}

// ---------------------------------------------------------------------------
// foldA(l): reduce partials of theta^(1)_l in FP64; eta(theta^(1)_l); dual terms
// ---------------------------------------------------------------------------
template <int NP>
__device__ void phase_foldA(const Params &P, long long ell, double *red, long long vc)
{
    const int p = (int)(ell & 1);
    const long long N = P.N;
    const int n = P.n;
    const int Q4 = P.Q >> 2;   // row partials per row, in float4 units
    double a = 0.0, b = 0.0, cc = 0.0, mviol = 0.0, mcomp = 0.0, sviol = 0.0, smuy = 0.0;
    for (long long l = vc * kThreads + threadIdx.x; l < N; l += (long long)P.G * kThreads) {
        // row sum: the Q (>= 2S, zero padded) contiguous partials of row l, independent 16-byte loads
        const float4 *rp4 = reinterpret_cast<const float4 *>(P.rowpart + l * P.Q);
        double R = 0.0;
#pragma unroll 8
        for (int q = 0; q < Q4; ++q) {
            const float4 t = __ldcg(rp4 + q);
            R += ((double)t.x + (double)t.y) + ((double)t.z + (double)t.w);
        }
        const long long s = l / kW, cl = l - s * kW;
        // CTAs whose unit range intersects stripe s, ascending
        const long long ua = s * N, ub = s * N + N - 1;
        long long c0 = (long long)(((unsigned long long)ua * (unsigned long long)P.G) / (unsigned long long)P.total);
        while (c0 > 0 && unit_begin(P, c0) > ua) --c0;
        while (c0 + 1 < P.G && unit_begin(P, c0 + 1) <= ua) ++c0;
        double Cc = 0.0, TX[NP];
#pragma unroll
        for (int k = 0; k < NP; ++k) TX[k] = 0.0;
        long long ubg = unit_begin(P, c0);
        for (long long cta = c0; cta < P.G && ubg <= ub; ++cta) {
            const long long unx = unit_begin(P, cta + 1);
            if (unx > ubg) {
                const long long fs = ubg / N;
                const float *cp = P.colpart + ((cta * P.slots + (s - fs)) * (NP + 1)) * kW + cl;
                Cc += (double)__ldcg(cp);
#pragma unroll
                for (int k = 0; k < NP; ++k) TX[k] += (double)__ldcg(cp + (1 + k) * kW);
            }
            ubg = unx;
        }
        const double v = R - Cc;               // (A_1^T theta)_l = row sum - column sum
        P.v[p][l] = v;
        const double hl = __ldg(P.h + l), mu = __ldcg(P.mu[p] + l);
        const double y = hl + v + mu;          // Step 1 closed form
        const double ys = y - P.shift;
        double d = 0.0, xin = 0.0;
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            float xf = 0.0f;
            if (k < n) {
                const double xk = __ldg(P.X64 + l * n + k);
                const double wk = Cc * xk - TX[k];   // (A_2^T theta)_l = Cc_l x_l - (theta^T X)_l
                P.w[p][l * n + k] = wk;
                const double xi = wk * P.inv_gamma;
                P.xi1_64[l * n + k] = xi;
                d += xi * xk;
                xin += xi * xi;
                xf = (float)xi;
            }
            P.xi1[l * NP + k] = xf;
        }
        P.y1[l] = y;
        P.yrow1[l] = (float)ys;
        P.ccol1[l] = (float)(d - ys);
        const double uu = y - hl;
        a += uu * uu;
        b += xin;
        cc += uu * y;
        mviol = fmax(mviol, -y);
        mcomp = fmax(mcomp, mu * fabs(y));
        if (y < 0.0) sviol += y * y;
        smuy += mu * y;
        if (!isfinite(y) || !isfinite(d)) atomicCAS(&P.st->error, 0, ERR_NUMERIC);
    }
    double vals[7] = {a, b, cc, mviol, mcomp, sviol, smuy};
    const bool ismax[7] = {false, false, false, true, true, false, false};
    block_reduce<7>(vals, ismax, red);
    if (threadIdx.x == 0)
#pragma unroll
        for (int i = 0; i < 7; ++i) P.foldpart[vc * 8 + i] = vals[i];
}

// ---------------------------------------------------------------------------
// KKT pass at theta^(1)_l: per-pair g = (C eta)_p; FP32 (screen) or FP64
// ---------------------------------------------------------------------------
template <typename TS, int NP, bool F64>
__device__ void phase_kkt(const Params &P, long long ell, double *red, long long vc)
{
    using St = Store<TS>;
    using Vec = typename St::Vec;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wc = warp & 1, wr = warp >> 1;
    const int p = (int)(ell & 1);
    const TS *__restrict__ th = (const TS *)P.theta[p];
    const float iscl = P.st_inv_scale;
    const long long N = P.N, ld = P.ld;
    const int n = P.n;
    double mviol = 0.0, mcomp = 0.0, sviol = 0.0, sthg = 0.0;
    constexpr int REC = RecLayout<NP>::REC;

    long long u = unit_begin(P, vc);
    const long long uend = unit_begin(P, vc + 1);
    while (warp < kCons / 32 && u < uend) {
        const long long s = u / N;
        const long long r0 = u - s * N;
        const long long r1 = min(N, r0 + (uend - u));
        const long long col0 = s * kW + wc * 128 + lane * 4;
        const bool vec_ok = col0 < ld;
        bool colv[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) colv[j] = (col0 + j) < N;
        float tv_viol = 0.0f, tv_comp = 0.0f, tv_s2 = 0.0f, tv_tg = 0.0f;
        for (long long r = r0 + wr; r < r1; r += kWR) {
            if (!vec_ok) continue;
            float tc[4];
            St::unpack(__ldcg((const Vec *)(th + r * ld + col0)), tc, iscl);
            if (F64) {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const long long l2 = col0 + j;
                    if (!colv[j] || l2 == r) continue;
                    double g = __ldcg(P.y1 + r) - __ldcg(P.y1 + l2);
                    for (int k = 0; k < n; ++k) g -= __ldcg(P.xi1_64 + l2 * n + k) * (__ldg(P.X64 + r * n + k) - __ldg(P.X64 + l2 * n + k));
                    mviol = fmax(mviol, -g);
                    mcomp = fmax(mcomp, (double)tc[j] * fabs(g));
                    if (g < 0.0) sviol += g * g;
                    sthg += (double)tc[j] * g;
                }
            } else {
                const float yr = __ldcg(P.yrow1 + r);
                float xr[NP];
#pragma unroll
                for (int k = 0; k < NP; ++k) xr[k] = __ldcg(P.rowrec + r * REC + 1 + k);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const long long l2 = col0 + j;
                    if (!colv[j] || l2 == r) continue;
                    float g = yr + __ldcg(P.ccol1 + l2);
#pragma unroll
                    for (int k = 0; k < NP; ++k) g = fmaf(-__ldcg(P.xi1 + l2 * NP + k), xr[k], g);
                    tv_viol = fmaxf(tv_viol, -g);
                    tv_comp = fmaxf(tv_comp, tc[j] * fabsf(g));
                    if (g < 0.0f) tv_s2 = fmaf(g, g, tv_s2);
                    tv_tg = fmaf(tc[j], g, tv_tg);
                }
            }
        }
        if (!F64) {
            mviol = fmax(mviol, (double)tv_viol);
            mcomp = fmax(mcomp, (double)tv_comp);
            sviol += (double)tv_s2;
            sthg += (double)tv_tg;
        }
        u += (r1 - r0);
    }
    double vals[4] = {mviol, mcomp, sviol, sthg};
    const bool ismax[4] = {true, true, false, false};
    block_reduce<4>(vals, ismax, red);
    if (threadIdx.x == 0)
#pragma unroll
        for (int i = 0; i < 4; ++i) P.kktpart[vc * 8 + i] = vals[i];
}

// Combine the KKT partials (pairs) and the fold partials (y >= 0 rows) into the
// metrics of cr_kkt_residual; every CTA computes the same values.  out: 0 kkt,
// 1 pri, 2 comp, 3 infeas_norm, 4 gap_norm.
__device__ __forceinline__ void reduce_kkt(const Params &P, double sigma, double *out)
{
    // warp 0 of the calling CTA
    double mv = 0.0, mc = 0.0, s2 = 0.0, tg = 0.0;
    for (int i = threadIdx.x; i < P.G; i += 32) {
        mv = fmax(mv, fmax(__ldcg(P.kktpart + i * 8 + 0), __ldcg(P.foldpart + i * 8 + 3)));
        mc = fmax(mc, fmax(__ldcg(P.kktpart + i * 8 + 1), __ldcg(P.foldpart + i * 8 + 4)));
        s2 += __ldcg(P.kktpart + i * 8 + 2) + __ldcg(P.foldpart + i * 8 + 5);
        tg += __ldcg(P.kktpart + i * 8 + 3) + __ldcg(P.foldpart + i * 8 + 6);
    }
    mv = warp_max(mv);
    mc = warp_max(mc);
    s2 = warp_sum(s2);
    tg = warp_sum(tg);
    const double np = (double)P.N * (double)(P.N - 1);
    const double pri = mv / sigma, comp = mc / (sigma * sigma);
    out[0] = fmax(pri, comp);
    out[1] = pri;
    out[2] = comp;
    out[3] = sqrt(s2) / sqrt(np);
    out[4] = tg / np;
}

}  // namespace crk
