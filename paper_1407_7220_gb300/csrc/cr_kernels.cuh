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

#include <type_traits>

namespace crk {

constexpr int kThreads = 256;   // 8 warps per CTA
constexpr int kCons = kThreads; // every warp consumes pair-pass stages; lane 0 of warp 0 also produces them
constexpr int kW = 256;         // stripe width (columns)
constexpr int kWR = 4;          // row groups of consumer warps (2 warps per row)
constexpr int kRS = 16;         // rows per pipeline stage
constexpr int kRPW = kRS / kWR; // rows of a stage per consumer warp
constexpr int kSB = 8 / kRPW;   // stages per row-sum batch (8 row sums per warp)
static_assert(kRS % kWR == 0 && 8 % kRPW == 0, "row split of a stage");
// The CUDA-core pass is compiled for stages of RS rows (16 by default; the batched launch also
// has 8-row stages, a tile shape its autotuner may pick): RPW rows per consumer warp, row sums
// flushed every SB stages (8 per warp).
template <int RS> struct StageRows {
    static constexpr int RPW = RS / kWR;
    static constexpr int SB = 8 / RPW;
    static_assert(RS % kWR == 0 && RPW >= 1 && 8 % RPW == 0, "row split of a stage");
};
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
    double ball_c;     // finite B_theta: radial factor min(1, B_theta / ||lambda||_2) of this iterate
};

struct DevState {
    Scal scal[2];
    unsigned long long bar_count;  // monotone grid-barrier counter (reset before each launch)
    long long iters_done;          // written by the persistent kernel at exit
    int error;
    int converged;
    int pad[2];
    double kkt[8];      // last reduced KKT terms: 0 kkt,1 pri,2 comp,3 infeas,4 gap,5 screen
    // ALCC (Sec. II-D): progress of the current MAPG call, written at the end of every launch
    long long alcc_ell;  // MAPG iterations done
    int alcc_done;       // 1: MAPG returned and the outer step of Fig. `fig:alcc` was taken
    int alcc_pad;
    double alcc_t;       // t of the MAPG figure after alcc_ell iterations
};

struct Params {
    CUtensorMap tmap[2];    // TMA descriptors of theta[0], theta[1]: N x N, box kRS x kW
    CUtensorMap tmap32[2];  // the same with a box of 32 rows (tensor-core pass, 16-bit theta)
    CUtensorMap tmap8[2];   // the same with a box of 8 rows (8-row stages of the batched launch)
    // sizes
    long long N;
    int n;
    int NP;             // padded n (template value, for host checks)
    long long ld;       // row stride of theta (elements)
    int S;              // stripes = ceil(N / kW)
    int G;              // CTAs of the grid
    int slots;          // column-partial slots per CTA
    long long total;    // S * N units
    const long long *ubeg;  // G + 1 entries: first unit of every CTA (host-computed partition)
    const long long *cfs;   // G entries: first stripe of every CTA (-1: no units)
    const long long *sc0, *sc1;   // S entries each: CTAs [sc0[s], sc1[s]) meet stripe s
    // constants
    double gamma, inv_gamma, L, invL_d, shift, sigma;
    float invL;
    float st_scale, st_inv_scale;   // theta storage scale (FP16 only; 1 otherwise)
    float xmax;                     // max |x_lk| over the data
    float alcc_delta;               // ALCC passes: relative bound of the FP32 residual's error, (n + 4) 2^-23
    int momentum, restart, sr;
    int fuse;           // 1: foldA(l) also performs foldB(l+1) (plain P-APG: beta needs no reduction)
    int fold_stats;     // 1: foldA writes its objective / y >= 0 partial sums (foldpart); with P.fuse the
                        // drivers ask for them on check iterations and the last iteration of a call only
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
    double *dd[2];          // w_l . x_l of the two latest iterates (N): foldB's xi^(2).x by linearity
    double *mu[2];          // multipliers of the y >= 0 rows (N)
    float *rowpart;         // [N][Q]: row sums per (stripe, column half), Q = ceil4(2S), padding 0
    int Q;
    float *colpart;         // [G][slots][cgroups][NP+1][kW]: column partials per CTA, stripe slot and group
    int cgroups;            // column-partial groups per CTA segment: kWR row groups of warps, or 1
    // FP64 multipliers (theta_dtype F64): the pair pass runs in FP64 on FP64 copies of its
    // inputs and writes FP64 partials (same layouts as rowrec, ccol2, xi2, rowpart, colpart)
    int f64;
    // P-APG with K blocks (Sec. II-A): block id of every point; pair mask of the FP64 pass
    // (0 none, 1 pairs between blocks only, 2 pairs inside a block only); the inner problem's
    // subgradient offset (xi = xi_off + A_2^T theta / gamma) and no y >= 0 rows
    const int *blk;
    int blkmode;
    const long long *band;  // K blocks, pairs inside blocks (points sorted by block): rows [band[2s],
                            // band[2s+1]) of stripe s hold every such pair of its columns; nullptr: all rows
    const double *xi_off;
    int no_mu;
    // Q_2 with a finite ball ||lambda||_2 <= B_theta (Eq. (lambda_dual)): per-CTA partial sums
    // of squares of the clamped multipliers (pairs and y >= 0 rows)
    int ball;
    double B_theta;
    double *ballpart;   // [G]
    double *rec64, *ccol2_64, *xi2_64;
    double *rowpart64, *colpart64;
    int tc;                 // 1: the pair pass runs its two products on the tensor cores
    float *xi_tc;           // tensor-core operands (TF32 hi/lo): Xi per stripe, written by every foldB
    float *xr_tc, *xt_tc;   // X rows and [X | 1] transposed per 8-row block (constant)
    // ALCC (Sec. II-D) on the full problem; (y_k, xi_k) live in y1 and xi1_64, theta_k in theta[0]
    double *ay[2], *axi[2]; // (y, xi)^(1) of the two latest MAPG iterations (N, N x n; FP64)
    double *ay2, *axi2;     // the extrapolated point (y, xi)^(2) of MAPG steps 4-5
    double *foldpart;       // [G][8]
    double *kktpart;        // [G][8]
    DevState *st;
};

// ---------------------------------------------------------------------------
// storage types
// ---------------------------------------------------------------------------
template <typename TS> struct Store;

// Counter-based generator for the stochastic rounding: hash_col mixes the column group and the
// iteration seed (b, c) once per segment; hash_row then takes the row a with one multiply-add,
// one odd-constant multiply and one xor-shift (a single round of the multiply/xor-shift integer
// finalizers of C. Wellons' hash-prospector: the rounding needs 16-bit uniforms that vary from
// pair to pair and iteration to iteration, not a full avalanche, and the pair pass evaluates it
// once per row and lane); hash_next derives a second word from the first.
__device__ __forceinline__ uint32_t hash_col(uint32_t b, uint32_t c)
{
    return (b * 0x85EBCA77u + 0x165667B1u) ^ (c * 0xC2B2AE3Du + 0x27D4EB2Fu);
}
__device__ __forceinline__ uint32_t hash_row(uint32_t hcol, uint32_t a)
{
    const uint32_t x = (a * 0x9E3779B1u + hcol) * 0x2C1B3C6Du;
    return x ^ (x >> 15);
}
__device__ __forceinline__ uint32_t hash_next(uint32_t h) { return (h ^ (h >> 16)) * 0x85EBCA77u; }

// Packed FP32 pairs (the f32x2 arithmetic of sm_100 and later): one instruction performs
// two IEEE single-precision operations, each half rounded exactly as the scalar one, so a
// packed expression gives the same bits as the scalar expression in the same order.
typedef unsigned long long f2;
__device__ __forceinline__ f2 f2_make(float a, float b)
{
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void f2_split(f2 v, float &a, float &b) { asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v)); }
__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c)
{
    f2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ f2 f2_add(f2 a, f2 b)
{
    f2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 f2_sub(f2 a, f2 b)
{
    f2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b)
{
    f2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 f2_add_rm(f2 a, f2 b)
{
    f2 r;
    asm("add.rm.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
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

    // --- packed forms used by the pair pass (two adjacent columns per f2) ---
    __device__ static __forceinline__ void unpack2(const float *p, f2 (&o)[2], float)
    {
        const ulonglong2 t = *reinterpret_cast<const ulonglong2 *>(p);
        o[0] = t.x;
        o[1] = t.y;
    }
    // round<SR> on both halves: r = v + k ulp(v), k = floor(e/ulp(v) + u), u uniform in [0,1)
    // from 16 bits (the low half of rnd for the first value, the high half for the second).
    // The scaling s = 2^(1 - E) (E the exponent of |v|, |v| clamped below at 2^-100) is the
    // complemented exponent field of |v|, so e s = (e/ulp) 2^-22.  t = e s + U with
    // U = 2^-15 + u 2^-22 (the 16 bits of u are the low mantissa bits of U) carries e/ulp + u to
    // 2^-16; RD(t + 3 - 2^-15) lands in [2, 4), whose spacing is 2^-22, so its bit pattern minus
    // that of 3 is k (in {-1, 0, 1} since |e| <= ulp/2).
    template <bool SR>
    __device__ static __forceinline__ f2 round2(f2 th2, f2 g, f2 ninvL2, float, uint32_t rnd, float)
    {
        const f2 v = f2_fma(g, ninvL2, th2);
        float v0, v1;
        f2_split(v, v0, v1);
        float r0 = v0, r1 = v1;
        if (SR) {
            const f2 e = f2_fma(g, ninvL2, f2_sub(th2, v));
            const uint32_t b0 = __float_as_uint(v0), b1 = __float_as_uint(v1);
            const float s0 = __uint_as_float(~__float_as_uint(fmaxf(fabsf(v0), 0x1p-100f)) & 0x7F800000u);
            const float s1 = __uint_as_float(~__float_as_uint(fmaxf(fabsf(v1), 0x1p-100f)) & 0x7F800000u);
            const float u0 = __uint_as_float(__byte_perm(rnd, 0x38000000u, 0x7610u));   // U = 2^-15 + u 2^-22
            const float u1 = __uint_as_float(__byte_perm(rnd, 0x38000000u, 0x7632u));
            const f2 t = f2_fma(e, f2_make(s0, s1), f2_make(u0, u1));
            const f2 fl = f2_add_rm(t, f2_make(3.0f - 0x1p-15f, 3.0f - 0x1p-15f));
            float fl0, fl1;
            f2_split(fl, fl0, fl1);
            r0 = __uint_as_float(b0 + __float_as_uint(fl0) - 0x40400000u);   // b + k
            r1 = __uint_as_float(b1 + __float_as_uint(fl1) - 0x40400000u);
        }
        // projection on theta >= 0 as max(r, 0): for v > 0 the rounded r is >= 0; for v < 0 it is
        // negative, and for v = -0 or +0 it is 0, a NaN pattern (max gives 0) or, with SR, the
        // smallest denormal (a > 0 rounded up, as unbiased rounding asks)
        return f2_make(fmaxf(r0, 0.0f), fmaxf(r1, 0.0f));
    }
    __device__ static __forceinline__ Vec pack2(const f2 (&s)[2])
    {
        Vec v;
        f2_split(s[0], v.x, v.y);
        f2_split(s[1], v.z, v.w);
        return v;
    }
    __device__ static __forceinline__ f2 decoded2(f2 s, f2) { return s; }
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
        return fmaxf(__uint_as_float(b), 0.0f);   // the rounding keeps the sign: v <= 0 gives 0
    }
    __device__ static __forceinline__ Vec pack(const float (&s)[4])
    {
        // the top halves of two values in one byte permute
        Vec v;
        v.x = __byte_perm(__float_as_uint(s[0]), __float_as_uint(s[1]), 0x7632u);
        v.y = __byte_perm(__float_as_uint(s[2]), __float_as_uint(s[3]), 0x7632u);
        return v;
    }
    __device__ static __forceinline__ float decoded(float s, float) { return s; }

    __device__ static __forceinline__ void unpack2(const __nv_bfloat16 *p, f2 (&o)[2], float)
    {
        const uint2 t = *reinterpret_cast<const uint2 *>(p);
        o[0] = f2_make(b2f(t.x & 0xFFFFu), b2f(t.x >> 16));
        o[1] = f2_make(b2f(t.y & 0xFFFFu), b2f(t.y >> 16));
    }
    // round<SR> on both halves, the update as one packed FMA (g * (-1/L) + th2 is the value of
    // fmaf(-g, 1/L, th2) in each half)
    template <bool SR>
    __device__ static __forceinline__ f2 round2(f2 th2, f2 g, f2 ninvL2, float, uint32_t rnd, float)
    {
        float v0, v1;
        f2_split(f2_fma(g, ninvL2, th2), v0, v1);
        uint32_t b0 = __float_as_uint(v0), b1 = __float_as_uint(v1);
        if (SR) {
            b0 += rnd & 0xFFFFu;
            b1 += rnd >> 16;
        } else {
            b0 += 0x7FFFu + ((b0 >> 16) & 1u);
            b1 += 0x7FFFu + ((b1 >> 16) & 1u);
        }
        return f2_make(fmaxf(__uint_as_float(b0 & 0xFFFF0000u), 0.0f), fmaxf(__uint_as_float(b1 & 0xFFFF0000u), 0.0f));
    }
    // round2 with the packing and the projection in one conversion: after the 16-bit noise (or
    // the round-to-nearest-even increment) the bit patterns are truncated, i.e. converted toward
    // zero, by one packed cvt.rz.relu (negative values give 0); returns the stored values as
    // floats and, in bits, the packed BF16 pair (low half: the first value)
    template <bool SR>
    __device__ static __forceinline__ f2 round2_bits(f2 th2, f2 g, f2 ninvL2, uint32_t rnd, uint32_t &bits)
    {
        float v0, v1;
        f2_split(f2_fma(g, ninvL2, th2), v0, v1);
        uint32_t b0 = __float_as_uint(v0), b1 = __float_as_uint(v1);
        if (SR) {
            b0 += rnd & 0xFFFFu;
            b1 += rnd >> 16;
        } else {
            b0 += 0x7FFFu + ((b0 >> 16) & 1u);
            b1 += 0x7FFFu + ((b1 >> 16) & 1u);
        }
        uint32_t h;
        asm("cvt.rz.relu.bf16x2.f32 %0, %1, %2;" : "=r"(h) : "f"(__uint_as_float(b1)), "f"(__uint_as_float(b0)));
        bits = h;
        return f2_make(__uint_as_float(h << 16), __uint_as_float(h & 0xFFFF0000u));
    }
    __device__ static __forceinline__ Vec pack2(const f2 (&s)[2])
    {
        float a[4];
        f2_split(s[0], a[0], a[1]);
        f2_split(s[1], a[2], a[3]);
        return pack(a);
    }
    __device__ static __forceinline__ f2 decoded2(f2 s, f2) { return s; }
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
        return r;   // sv = 0 for v <= 0, and both roundings keep 0
    }
    __device__ static __forceinline__ Vec pack(const float (&s)[4])
    {
        Vec v;
        v.x = (uint32_t)__half_as_ushort(__float2half_rn(s[0])) | ((uint32_t)__half_as_ushort(__float2half_rn(s[1])) << 16);
        v.y = (uint32_t)__half_as_ushort(__float2half_rn(s[2])) | ((uint32_t)__half_as_ushort(__float2half_rn(s[3])) << 16);
        return v;
    }
    __device__ static __forceinline__ float decoded(float s, float inv_scale) { return s * inv_scale; }

    __device__ static __forceinline__ void unpack2(const __half *p, f2 (&o)[2], float inv_scale)
    {
        const uint2 t = *reinterpret_cast<const uint2 *>(p);
        o[0] = f2_make(h2f(t.x & 0xFFFFu, inv_scale), h2f(t.x >> 16, inv_scale));
        o[1] = f2_make(h2f(t.y & 0xFFFFu, inv_scale), h2f(t.y >> 16, inv_scale));
    }
    // round<SR> on both halves with packed conversions.  Stochastic rounding adds noise uniform
    // over one FP16 step and rounds toward zero: with p = the FP16 step at s (2^(max(E,-14) - 10),
    // E the exponent of s; the subnormal step below 2^-14), t = s + u p and the pair is
    // RZ_f16(t0, t1), which rounds up with probability (s - RZ(s)) / p (to within the 2^-13 p that
    // t's own rounding adds).  u p is formed as U q - 2^-15 q with U = 2^-15 (1 + X 2^-23), X the 16
    // random bits (one byte permute), and q = 2^22 p (both exact powers-of-two scalings).
    template <bool SR>
    __device__ static __forceinline__ f2 round2(f2 th2, f2 g, f2 ninvL2, float, uint32_t rnd, float scl)
    {
        float v0, v1;
        f2_split(f2_fma(g, ninvL2, th2), v0, v1);
        const float s0 = fminf(fmaxf(v0, 0.0f) * scl, 65504.0f);
        const float s1 = fminf(fmaxf(v1, 0.0f) * scl, 65504.0f);
        uint32_t h;
        if (SR) {
            float t0, t1;
            f2_split(sr_noise(s0, s1, rnd), t0, t1);
            asm("cvt.rz.f16x2.f32 %0, %1, %2;" : "=r"(h) : "f"(t1), "f"(t0));
        } else {
            asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(h) : "f"(s1), "f"(s0));
        }
        const __half2 hh = *reinterpret_cast<const __half2 *>(&h);
        return f2_make(__low2float(hh), __high2float(hh));   // sv = 0 for v <= 0 either way
    }
    // The same update with th2 and g already multiplied by the scale: v s = fma(g s, -1/L, th2 s)
    // exactly (a power-of-two factor commutes with each rounding).  The clamp to [0, 65504] is
    // the conversion's own (.relu: negative values give 0, and the noise cannot lift a negative
    // value above 0 since it stays below one FP16 step of it; .satfinite: 65504 above), so the
    // stored values are those of round2 for every |v s| < 2^116.  Returns the stored FP16 numbers
    // as floats (scaled) and, in h, the packed pair (low half: the first value).
    template <bool SR>
    __device__ static __forceinline__ f2 round2_scaled(f2 th2s, f2 gs, f2 ninvL2, uint32_t rnd, uint32_t &h)
    {
        float s0, s1;
        f2_split(f2_fma(gs, ninvL2, th2s), s0, s1);
        if (SR) {
            float t0, t1;
            f2_split(sr_noise(s0, s1, rnd), t0, t1);
            asm("cvt.rz.relu.satfinite.f16x2.f32 %0, %1, %2;" : "=r"(h) : "f"(t1), "f"(t0));
        } else {
            asm("cvt.rn.relu.satfinite.f16x2.f32 %0, %1, %2;" : "=r"(h) : "f"(s1), "f"(s0));
        }
        const __half2 hh = *reinterpret_cast<const __half2 *>(&h);
        return f2_make(__low2float(hh), __high2float(hh));
    }
    // t = s + u p of the stochastic rounding above, both halves
    __device__ static __forceinline__ f2 sr_noise(float s0, float s1, uint32_t rnd)
    {
        const float q0 = __uint_as_float(max(__float_as_uint(s0) & 0x7F800000u, 113u << 23) + (12u << 23));
        const float q1 = __uint_as_float(max(__float_as_uint(s1) & 0x7F800000u, 113u << 23) + (12u << 23));
        const float U0 = __uint_as_float(__byte_perm(rnd, 0x38000000u, 0x7610u));
        const float U1 = __uint_as_float(__byte_perm(rnd, 0x38000000u, 0x7632u));
        const f2 q = f2_make(q0, q1);
        const f2 c = f2_fma(f2_make(-0x1p-15f, -0x1p-15f), q, f2_make(s0, s1));   // s - 2^-15 q, exact
        return f2_fma(f2_make(U0, U1), q, c);
    }
    __device__ static __forceinline__ Vec pack2(const f2 (&s)[2])
    {
        // the values are FP16 numbers: one exact packed conversion per pair
        float a[4];
        f2_split(s[0], a[0], a[1]);
        f2_split(s[1], a[2], a[3]);
        Vec v;
        asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(v.x) : "f"(a[1]), "f"(a[0]));
        asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(v.y) : "f"(a[3]), "f"(a[2]));
        return v;
    }
    __device__ static __forceinline__ f2 decoded2(f2 s, f2 iscl2) { return f2_mul(s, iscl2); }
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
// Non-blocking probe of a phase (try_wait may suspend the thread for a while; test_wait does not).
__device__ __forceinline__ bool mbar_test_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
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
// L2 cache policy for the per-row vectors that are re-read for every stripe (evict last).
// (An evict-first policy on the multiplier tiles measured slower on a GB300: 1.03 vs 1.01 ms
// per pass at N = 20,000, so those loads keep the default policy.)
__device__ __forceinline__ uint64_t l2_evict_last()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ void bulk_load_hint(void *dst, const void *src, uint32_t bytes, uint64_t *bar,
                                               uint64_t policy)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
                 " [%0], [%1], %2, [%3], %4;" ::"r"(smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
                 : "memory");
}
// Stores of the per-iteration partial sums (read by the next fold) with an L2 evict-last policy:
// the pair pass streams the multiplier arrays (GBs) through L2 after the first partials are
// written, and with the default policy the fold found most of them evicted to DRAM.
__device__ __forceinline__ void st_keep(float *p, float v, uint64_t pol)
{
    asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(p), "f"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void st_keep(ulonglong2 *p, ulonglong2 v, uint64_t pol)
{
    asm volatile("st.global.L2::cache_hint.v2.u64 [%0], {%1, %2}, %3;" ::"l"(p), "l"(v.x), "l"(v.y), "l"(pol)
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

// Block reduction of K doubles (sum or max per component) into v[] of thread 0; fixed
// order, hence deterministic.  red: shared scratch of (warps + 1)*K doubles.  Every component starts
// at 0 in every thread and maxima are taken over non-negative terms, so 0 is the identity of
// each component: a warp whose values are all +0 contributes zeros without FP64 work (GB300's
// FP64 pipe is narrow, and at small N most warps hold no rows), and the final pass over the
// warps runs one component per thread.
template <int K>
__device__ __forceinline__ void block_reduce(double (&v)[K], const bool (&is_max)[K], double *red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    bool nz = false;
#pragma unroll
    for (int i = 0; i < K; ++i) nz |= __double_as_longlong(v[i]) != 0ll;
    if (__any_sync(0xffffffffu, nz)) {
#pragma unroll
        for (int i = 0; i < K; ++i) v[i] = is_max[i] ? warp_max(v[i]) : warp_sum(v[i]);
    }
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < K; ++i) red[warp * K + i] = v[i];
    __syncthreads();
    if (threadIdx.x < K) {
        const int i = threadIdx.x;
        double a = red[i];
        for (int w = 1; w < kThreads / 32; ++w) a = is_max[i] ? fmax(a, red[w * K + i]) : a + red[w * K + i];
        red[(kThreads / 32) * K + i] = a;
    }
    __syncthreads();
    if (threadIdx.x == 0)
#pragma unroll
        for (int i = 0; i < K; ++i) v[i] = red[(kThreads / 32) * K + i];
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
// First (stripe, row) unit of CTA c (c <= G): an even split of the S*N units, each segment
// starting on an 8-row boundary (whole 8-row blocks for the tensor-core operands).  The host
// computes the table once per partition (no 64-bit division on the device).
__device__ __forceinline__ long long unit_begin(const Params &P, long long c) { return __ldg(P.ubeg + c); }

// Rows of the per-row phases: chunks of 32 consecutive rows (one per warp, coalesced) dealt
// round-robin over the CTAs first, so that every SM gets a share even when N < G * kThreads.
struct RowIter {
    long long q, step, N;
    int lane;
    __device__ __forceinline__ RowIter(const Params &P, long long vc)
        : q((long long)(threadIdx.x >> 5) * P.G + vc), step((long long)P.G * (kThreads >> 5)), N(P.N),
          lane((int)(threadIdx.x & 31))
    {
    }
    __device__ __forceinline__ bool more() const { return q * 32 < N; }
    __device__ __forceinline__ long long row() const { return q * 32 + lane; }
    __device__ __forceinline__ void next() { q += step; }
};


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
// Per-row part of foldB (Step 1 at theta^(2) by linearity, Step 2 on the y >= 0 row): slot c
// holds the latest iterate's aggregates, slot p the previous one's; writes mu[p] and the
// column data of theta^(2) that the pair pass reads.
template <int NP>
__device__ __forceinline__ void foldB_row(const Params &P, int c, int p, long long l, double beta)
{
    const double b1 = 1.0 + beta;
    const double g1 = b1 * P.inv_gamma, g0 = beta * P.inv_gamma;
    const int n = P.n;
    double v2 = b1 * __ldcg(P.v[c] + l) - beta * __ldcg(P.v[p] + l);
    double mu2 = b1 * __ldcg(P.mu[c] + l) - beta * __ldcg(P.mu[p] + l);
    double y2 = __ldcg(P.h + l) + v2 + mu2;
    double mun = mu2 - y2 * P.invL_d;     // Step 2 on the y >= 0 rows of C
    P.mu[p][l] = (mun > 0.0 && !P.no_mu) ? mun : 0.0;
    double ys = y2 - P.shift;
    // xi^(2) = ((1 + beta) w_c - beta w_p) / gamma (+ the offset of the K-block inner problems),
    // and xi^(2).x_l by the same linearity from w.x of the two iterates
    double d = (b1 * __ldcg(P.dd[c] + l) - beta * __ldcg(P.dd[p] + l)) * P.inv_gamma;
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        float xf = 0.0f;
        double xi = 0.0;
        if (k < n) {
            xi = fma(g1, __ldcg(P.w[c] + l * n + k), -(g0 * __ldcg(P.w[p] + l * n + k)));
            if (P.xi_off) {
                const double o = __ldcg(P.xi_off + l * n + k);
                xi += o;
                d += o * __ldg(P.X64 + l * n + k);
            }
            xf = (float)xi;
        }
        P.xi2[l * NP + k] = xf;
        if (P.f64) P.xi2_64[l * NP + k] = xi;   // the FP64 pass reads the column data unrounded
    }
    P.rowrec[l * RecLayout<NP>::REC] = (float)ys;
    P.ccol2[l] = (float)(d - ys);
    if (P.f64) {
        P.rec64[l * RecLayout<NP>::REC] = ys;
        P.ccol2_64[l] = d - ys;
    }
    if (P.tc) {
        // Xi of column l as the A operand of the residual product: stripe l/256, column pair
        // (l%256)/2 = lane, even/odd column = MMA; TF32 hi and lo parts
        constexpr int KP = (NP + 7) / 8 * 8;
        const long long st = l / kW;
        const int cl = (int)(l - st * kW), eo = cl & 1, mm = cl >> 1;
        float *base = P.xi_tc + (size_t)st * (2 * 2 * 128 * KP);
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            const float xf = P.xi2[l * NP + k];
            uint32_t hb;
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hb) : "f"(xf));
            const float hi = __uint_as_float(hb);
            uint32_t lb;
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(lb) : "f"(xf - hi));
            const size_t o = ((size_t)(mm >> 3) * (KP / 4) + (k >> 2)) * 32 + (mm & 7) * 4 + (k & 3);
            base[(size_t)(eo * 2 + 0) * 128 * KP + o] = hi;
            base[(size_t)(eo * 2 + 1) * 128 * KP + o] = __uint_as_float(lb);
        }
    }
}

// Momentum scalars of iteration e without the dual-value test (plain P-APG): Fig. 2 steps 3-4.
__device__ __forceinline__ Scal next_scal_plain(const Params &P, long long e)
{
    Scal old;
    const int c = (int)((e - 1) & 1);
    old.t = __ldcg(&P.st->scal[c].t);
    old.dual = __ldcg(&P.st->scal[c].dual);
    old.beta = __ldcg(&P.st->scal[c].beta);
    old.restarts = __ldcg(&P.st->scal[c].restarts);
    Scal nw = old;
    double beta = 0.0;
    if (e >= 2) {
        const double t = old.t;
        const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));   // Fig. 2 step 3
        beta = P.momentum ? (t - 1.0) / tn : 0.0;                 // Fig. 2 step 4 weight
        nw.t = tn;
    }
    nw.beta = beta;
    return nw;
}

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
    const double beta = s_beta;
    const long long N = P.N;
    for (RowIter it(P, vc); it.more(); it.next()) {
        const long long l = it.row();
        if (l < N) foldB_row<NP>(P, c, p, l, beta);
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

// Pass modes: the P-APG step (two multiplier tiles in, theta^(1)_l out), and the two ALCC passes
// of Sec. II-D over one multiplier array: m = (A_1 y + A_2 xi - theta_k)_- with its adjoint and
// nothing stored (MAPG gradient), and theta <- a m stored in place (Fig. `fig:alcc` step 4).
enum PairMode : int { PM_PAPG = 0, PM_ALCC_GRAD = 1, PM_ALCC_UPDATE = 2 };

template <typename TS, int NP, int TILES = 2, int RS = kRS> struct PairSmem {
    static constexpr int REC = RecLayout<NP>::REC;
    static constexpr size_t tile_bytes = (size_t)RS * kW * sizeof(TS);
    static constexpr size_t rec_bytes = (size_t)RS * REC * sizeof(float);
    static constexpr size_t stage_bytes = TILES * tile_bytes + rec_bytes;
    // as many stages as fit (more bytes in flight per SM)
    static constexpr int kFit = (int)((kSmemBudget - 128) / stage_bytes);
    static constexpr int kStages = kFit < kMaxStages ? kFit : kMaxStages;
    static_assert(kStages >= 2, "pipeline needs at least two stages");
    static constexpr size_t bytes = kStages * stage_bytes + 128;   // + base alignment slack
    static_assert(tile_bytes % 128 == 0 && rec_bytes % 128 == 0, "stage buffers must stay 128-byte aligned");
};

// theta - g_p in FP64 for pair (l1, l2) from the folds' FP64 point (y, xi)^(2) and X: the ALCC
// passes take it for the pairs whose FP32 estimate of theta - g is close to 0, since the
// multiplier estimate mu_k (g - theta)_- multiplies any absolute error in it by mu_k.
// g = y_l1 + (xi_l2.x_l2 - y_l2) - xi_l2.x_l1 with the column's FP64 constant xi_l2.x_l2 - y_l2
// from the folds: n FMAs and 2n + 2 loads (the FP32 pass's expression, in FP64, where its
// rounding is ~2^-29 of the FP32 error that the window is drawn from).
static __device__ __noinline__ double alcc_exact_margin(const Params &P, long long l1, long long l2, float theta)
{
    const int n = P.n;
    double g = __ldcg(P.ay2 + l1) + __ldcg(P.ccol2_64 + l2);
    for (int k = 0; k < n; ++k) g = fma(-__ldcg(P.axi2 + l2 * n + k), __ldg(P.X64 + l1 * n + k), g);
    return (double)theta - g;
}

// The kRPW rows (rg, rg + kWR, ...) of one pipeline stage for one consumer warp, 4 columns per
// lane held as two f32x2 column pairs.  MASK handles the diagonal (l1 == l2), columns >= N
// and rows past the segment; stages without any of these take the unmasked instantiation.
// SR: stochastic rounding.  nxi = -xi of the lane's columns; ninvL2 = (-1/L, -1/L).
// The arithmetic of every pair is the scalar expression order of Step 2 (two chains of the
// xi.x product, even and odd k), so the residual and the projection mask are reproducible
// by a scalar evaluation.
template <typename TS, int NP, bool MASK, bool SR, int MODE, int RPW = kRPW>
__device__ __forceinline__ void pair_stage_rows(const TS *tcur, const TS *tprv, const float *rec, int rg, int cofs,
                                                long long r, long long r1, long long col0, long long N, long long ld,
                                                const f2 (&ccol)[2], const f2 (&nxi)[2][NP], f2 (&acc)[2][NP],
                                                f2 (&csum)[2], f2 beta2, f2 ninvL2, float invL, uint32_t hcol,
                                                float scl, float iscl, f2 iscl2, TS *__restrict__ nxt, bool vec_ok,
                                                float (&rsv)[RPW], const Params &Pm, const f2 (&cbnd)[2])
{
    using St = Store<TS>;
    using Vec = typename St::Vec;
    constexpr int REC = RecLayout<NP>::REC;
    const f2 zero2 = 0ull;
#pragma unroll
    for (int i = 0; i < RPW; ++i) {
        const int rl = rg + i * kWR;
        const long long rr = r + rl;
        const bool valid = !MASK || rr < r1;
        float rv[REC];
#pragma unroll
        for (int q = 0; q < REC; q += 4) {
            const float4 t4 = *reinterpret_cast<const float4 *>(rec + rl * REC + q);
            rv[q] = t4.x; rv[q + 1] = t4.y; rv[q + 2] = t4.z; rv[q + 3] = t4.w;
        }
        // a row past the segment has no record in the stage (the copy moves the segment's rows
        // only): whatever the slot holds must not reach the accumulators as 0 * x
        if (MASK && !valid)
#pragma unroll
            for (int q = 0; q < REC; ++q) rv[q] = 0.0f;
        f2 xb[NP];   // (x_k, x_k) of this row
#pragma unroll
        for (int k = 0; k < NP; ++k) xb[k] = f2_make(rv[1 + k], rv[1 + k]);
        const f2 yb = f2_make(rv[0], rv[0]);
        f2 tc[2], tp[2], outv[2];
        St::unpack2(tcur + rl * kW + cofs, tc, iscl);
        if (MODE == PM_PAPG) St::unpack2(tprv + rl * kW + cofs, tp, iscl);
        else tp[0] = tp[1] = zero2;   // one array: theta^(2) = (1 + beta) theta
        uint32_t hP[2] = {0u, 0u};
        if (SR) {
            hP[0] = hash_row(hcol, (uint32_t)rr);
            hP[1] = hash_next(hP[0]);   // 16 bits per column
        }
        f2 rs2;
#pragma unroll
        for (int P = 0; P < 2; ++P) {
            const f2 th2 = f2_fma(beta2, f2_sub(tc[P], tp[P]), tc[P]);   // theta^(2) = theta^(1) + beta (theta^(1) - prev)
            // (C eta)_p = y_l1 - y_l2 + xi_l2.x_l2 - xi_l2.x_l1, summed in two chains
            f2 g0 = f2_add(yb, ccol[P]), g1 = zero2;
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                if (k & 1) g1 = f2_fma(nxi[P][k], xb[k], g1);
                else g0 = f2_fma(nxi[P][k], xb[k], g0);
            }
            f2 sv;
            if (MODE == PM_PAPG) {
                sv = St::template round2<SR>(th2, f2_add(g0, g1), ninvL2, invL, hP[P], scl);   // Pi_{>=0}(theta^(2) - g/L)
            } else {
                // ALCC: invL * max(0, theta - g).  Where the FP32 estimate e = theta - g lies within
                // kNear error bounds of 0 (every active pair near the solution, where e ~ lambda/mu_k),
                // theta - g is taken in FP64; farther out e keeps at least 10 correct bits
                constexpr float kNear = 1024.0f;
                float t0, t1, q0, q1, b0, b1;
                f2_split(tc[P], t0, t1);
                f2_split(f2_add(g0, g1), q0, q1);
                f2_split(cbnd[P], b0, b1);
                const float ay = fabsf(rv[0]);
                const long long c = col0 + 2 * P;
                const float e0 = t0 - q0, e1 = t1 - q1;
                float s0 = fmaxf(e0, 0.0f) * invL, s1 = fmaxf(e1, 0.0f) * invL;
                if ((!MASK || (valid && c < N && c != rr)) && fabsf(e0) <= kNear * Pm.alcc_delta * (ay + b0))
                    s0 = (float)fmax(0.0, (double)invL * alcc_exact_margin(Pm, rr, c, t0));
                if ((!MASK || (valid && c + 1 < N && c + 1 != rr)) && fabsf(e1) <= kNear * Pm.alcc_delta * (ay + b1))
                    s1 = (float)fmax(0.0, (double)invL * alcc_exact_margin(Pm, rr, c + 1, t1));
                sv = f2_make(s0, s1);
            }
            if (MASK) {
                float s0, s1;
                f2_split(sv, s0, s1);
                const long long c = col0 + 2 * P;
                if (!valid || c >= N || c == rr) s0 = 0.0f;
                if (!valid || c + 1 >= N || c + 1 == rr) s1 = 0.0f;
                sv = f2_make(s0, s1);
            }
            outv[P] = sv;
            const f2 vv = St::decoded2(sv, iscl2);
            rs2 = P == 0 ? vv : f2_add(rs2, vv);                            // row sum    (A_1^T, + part)
            csum[P] = f2_add(csum[P], vv);                                  // column sum (A_1^T, - part)
#pragma unroll
            for (int k = 0; k < NP; ++k) acc[P][k] = f2_fma(vv, xb[k], acc[P][k]);   // theta^T X (A_2^T)
        }
        if (MODE != PM_ALCC_GRAD && vec_ok && valid) *reinterpret_cast<Vec *>(nxt + rr * ld + col0) = St::pack2(outv);
        float a, b;
        f2_split(rs2, a, b);
        rsv[i] = a + b;
    }
}

// Row sums of a batch of up to kSB stages (8 rows per warp) reduced across the warp with a
// transposing butterfly: 9 shuffles leave the full sum of batch entry
// e = 4*bit4 + 2*bit3 + bit2 (of the lane id) in every lane.  Entry e is row
// r_last - kRS*(kSB - 1 - e/kRPW) + rg + kWR*(e % kRPW); only the nb most recent stages are written.
template <int RS = kRS>
__device__ __forceinline__ void flush_row_sums(float (&v)[8], int nb, long long r_last, int rg, long long r1,
                                               float *rp, int Q, int lane, uint64_t pol)
{
    constexpr int RPW = StageRows<RS>::RPW, SB = StageRows<RS>::SB;
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
        const int sp = e / RPW;
        const long long row = r_last - (long long)RS * (SB - 1 - sp) + rg + kWR * (e % RPW);
        if (sp >= SB - nb && row < r1) st_keep(rp + row * Q, v[0], pol);
    }
}

// Producer cursor: walks the CTA's stages (RS rows of one stripe) in consumption order.
template <int RS> struct StageCursorT {
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
        r += RS;
        if (r >= r1) {
            u += r1 - r0;
            next_segment(N);
        }
    }
};
using StageCursor = StageCursorT<kRS>;

// Position of stage k in the ring of S slots: slot = k mod S and the parity of k / S,
// advanced one stage at a time without a division.
template <int S> struct RingPos {
    int slot;
    uint32_t phase;
    __device__ __forceinline__ void init(unsigned long long k)
    {
        slot = (int)(k % S);
        phase = (uint32_t)((k / S) & 1);
    }
    __device__ __forceinline__ void next()
    {
        if (++slot == S) {
            slot = 0;
            phase ^= 1u;
        }
    }
};

// Issue the stage at ring position pos: unless this is the slot's first use (reuse false),
// wait until its previous occupant (S stages earlier) was released by all 8 warps, then
// two tiled TMA loads and one bulk copy complete on the slot's "full" barrier.
template <typename TS, int NP, int MODE, int RS = kRS>
__device__ __forceinline__ bool produce_stage(const Params &P, unsigned char *stage0, uint64_t *full, uint64_t *empty,
                                              const RingPos<PairSmem<TS, NP, MODE == PM_PAPG ? 2 : 1, RS>::kStages> &pos,
                                              bool reuse, const StageCursorT<RS> &cur, int c, int p)
{
    constexpr int TILES = MODE == PM_PAPG ? 2 : 1;
    using L = PairSmem<TS, NP, TILES, RS>;
    const CUtensorMap *tm = RS == kRS ? P.tmap : P.tmap8;   // box of RS rows
    const int slot = pos.slot;
    if (reuse && !mbar_wait(P, &empty[slot], pos.phase ^ 1u)) return false;
    const int nrows = (int)min((long long)RS, cur.r1 - cur.r);
    unsigned char *st = stage0 + slot * L::stage_bytes;
    mbar_arrive_expect_tx(&full[slot], (uint32_t)(TILES * L::tile_bytes + (size_t)nrows * L::REC * 4));
    tma_load_2d(st, &tm[c], (int)(cur.s * kW), (int)cur.r, &full[slot]);
    if (TILES == 2) tma_load_2d(st + L::tile_bytes, &tm[p], (int)(cur.s * kW), (int)cur.r, &full[slot]);
    bulk_load(st + TILES * L::tile_bytes, P.rowrec + cur.r * L::REC, (uint32_t)(nrows * L::REC * 4), &full[slot]);
    return true;
}

// Step 2 with FP64 multipliers (cr_pair_f64.cuh).
template <int NP> __device__ void phase_pair_f64(const Params &P, long long ell, unsigned char *smem, long long vc);

// MODE = PM_PAPG: Step 2 of P-APG at iteration ell.  The ALCC modes read and write array 0 only;
// a = mu_k / mu_{k+1} scales the stored values of PM_ALCC_UPDATE.
template <typename TS, int NP, int MODE = PM_PAPG, int RS = kRS>
__device__ void phase_pair_stream(const Params &P, long long ell, unsigned char *smem, uint64_t *full,
                                  uint64_t *empty, unsigned long long &kstage, long long vc, float a = 1.0f);

template <typename TS, int NP, int MODE = PM_PAPG, int RS = kRS>
__device__ __forceinline__ void phase_pair(const Params &P, long long ell, unsigned char *smem, uint64_t *full,
                                           uint64_t *empty, unsigned long long &kstage, long long vc, float a = 1.0f)
{
    if constexpr (std::is_same<TS, double>::value) {
        static_assert(MODE == PM_PAPG, "FP64 multipliers: P-APG only");
        phase_pair_f64<NP>(P, ell, smem, vc);
    } else {
        phase_pair_stream<TS, NP, MODE, RS>(P, ell, smem, full, empty, kstage, vc, a);
    }
}

template <typename TS, int NP, int MODE, int RS>
__device__ void phase_pair_stream(const Params &P, long long ell, unsigned char *smem, uint64_t *full,
                                  uint64_t *empty, unsigned long long &kstage, long long vc, float a)
{
    using St = Store<TS>;
    constexpr int TILES = MODE == PM_PAPG ? 2 : 1;
    using L = PairSmem<TS, NP, TILES, RS>;
    constexpr int S = L::kStages;
    constexpr int RPW = StageRows<RS>::RPW, SB = StageRows<RS>::SB;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int p = MODE == PM_PAPG ? (int)(ell & 1) : 0, c = MODE == PM_PAPG ? 1 - p : 0;
    const long long N = P.N, ld = P.ld;
    const long long ubeg = unit_begin(P, vc);
    const long long uend = unit_begin(P, vc + 1);
    unsigned char *stage0 = smem;

    // number of stages of this pass (identical in every thread)
    unsigned long long nst = 0;
    for (long long u = ubeg; u < uend;) {
        const long long s = u / N, r0 = u - s * N, r1 = min(N, r0 + (uend - u));
        nst += (unsigned long long)((r1 - r0 + RS - 1) / RS);
        u += r1 - r0;
    }
    const unsigned long long kend = kstage + nst;

    // producer (lane 0 of warp 0): prefill the ring
    const bool producer = (tid == 0);
    StageCursorT<RS> pc;
    unsigned long long kprod = kstage;
    RingPos<S> ppos;
    bool pok = true;
    if (producer) {
        fence_proxy_async();
        pc.begin(ubeg, uend, N);
        ppos.init(kprod);
        for (; kprod < kend && kprod < kstage + S && pok; ++kprod) {
            pok = produce_stage<TS, NP, MODE, RS>(P, stage0, full, empty, ppos, kprod >= (unsigned long long)S, pc, c, p);
            pc.advance(N);
            ppos.next();
        }
    }
    __syncwarp();

    const int wc = warp & 1, rg = warp >> 1;
    // MAPG gradient: m = max(0, theta - g) (beta 0, step 1); update: a max(0, theta - g) as
    // max(0, (1 + (a - 1)) theta - a g)
    const float beta = MODE == PM_PAPG ? (float)__ldcg(&P.st->scal[p].beta) : MODE == PM_ALCC_UPDATE ? a - 1.0f : 0.0f;
    const float invL = MODE == PM_PAPG ? P.invL : MODE == PM_ALCC_UPDATE ? a : 1.0f;
    const float scl = P.st_scale, iscl = P.st_inv_scale;
    const f2 beta2 = f2_make(beta, beta), ninvL2 = f2_make(-invL, -invL), iscl2 = f2_make(iscl, iscl);
    const bool sr = MODE == PM_PAPG && P.sr != 0;
    const uint64_t keep = l2_evict_last();   // policy of the partial-sum stores
    const uint32_t rseed = P.seed ^ (uint32_t)ell * 0x632BE5ABu;
    TS *__restrict__ nxt = (TS *)P.theta[p];   // theta^(1)_{l-2} on entry, theta^(1)_l on exit
    const long long first_stripe = ubeg / N;
    RingPos<S> cpos;
    cpos.init(kstage);
    bool ok = true;
    for (long long u = ubeg; u < uend;) {
        const long long s = u / N, r0 = u - s * N, r1 = min(N, r0 + (uend - u));
        const long long colw = s * kW + wc * 128;       // first column of this warp
        const long long col0 = colw + lane * 4;
        const bool vec_ok = col0 < ld;
        const bool ragged = (s * kW + kW) > N;
        f2 ccol[2], nxi[2][NP];
#pragma unroll
        for (int P2 = 0; P2 < 2; ++P2) {
            const long long ca = col0 + 2 * P2, cb = ca + 1;
            const bool va = ca < N, vb = cb < N;
            ccol[P2] = f2_make(va ? __ldcg(P.ccol2 + ca) : 0.0f, vb ? __ldcg(P.ccol2 + cb) : 0.0f);
#pragma unroll
            for (int q = 0; q < NP; ++q)
                nxi[P2][q] = f2_make(va ? -__ldcg(P.xi2 + ca * NP + q) : 0.0f, vb ? -__ldcg(P.xi2 + cb * NP + q) : 0.0f);
        }
        // ALCC passes: |ccol| + max|x| ||xi||_1 of each column (with |y_l1|, the size of the terms of g)
        f2 cbnd[2];
#pragma unroll
        for (int P2 = 0; P2 < 2; ++P2) {
            cbnd[P2] = 0ull;
            if (MODE != PM_PAPG) {
                float ca, cb, sa = 0.0f, sb = 0.0f;
                f2_split(ccol[P2], ca, cb);
#pragma unroll
                for (int q = 0; q < NP; ++q) {
                    float xa, xb2;
                    f2_split(nxi[P2][q], xa, xb2);
                    sa += fabsf(xa);
                    sb += fabsf(xb2);
                }
                cbnd[P2] = f2_make(fabsf(ca) + P.xmax * sa, fabsf(cb) + P.xmax * sb);
            }
        }
        f2 acc[2][NP], csum[2];
#pragma unroll
        for (int P2 = 0; P2 < 2; ++P2) {
            csum[P2] = 0ull;
#pragma unroll
            for (int q = 0; q < NP; ++q) acc[P2][q] = 0ull;
        }
        const uint32_t hcol = hash_col((uint32_t)(col0 >> 2), rseed);
        float *rp = P.rowpart + (s * 2 + wc);   // row r's partial at rp[r * Q]
        const int cofs = wc * 128 + lane * 4;
        float rsb[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) rsb[q] = 0.0f;
        int nb = 0;
        for (long long r = r0; r < r1; r += RS, cpos.next()) {
            const int slot = cpos.slot;
            if (ok && !mbar_wait(P, &full[slot], cpos.phase)) ok = false;
            float rsn[RPW];
#pragma unroll
            for (int i = 0; i < RPW; ++i) rsn[i] = 0.0f;
            if (ok) {
                const unsigned char *st = stage0 + slot * L::stage_bytes;
                const TS *tcur = reinterpret_cast<const TS *>(st);
                const TS *tprv = reinterpret_cast<const TS *>(st + (TILES - 1) * L::tile_bytes);   // unused by the ALCC modes
                const float *rec = reinterpret_cast<const float *>(st + TILES * L::tile_bytes);
                const bool fast = !ragged && (r + RS <= r1) && !(r < colw + 128 && colw < r + RS);
                if (sr) {
                    if (fast)
                        pair_stage_rows<TS, NP, false, true, MODE, RPW>(tcur, tprv, rec, rg, cofs, r, r1, col0, N, ld, ccol, nxi, acc, csum, beta2, ninvL2, invL, hcol, scl, iscl, iscl2, nxt, vec_ok, rsn, P, cbnd);
                    else
                        pair_stage_rows<TS, NP, true, true, MODE, RPW>(tcur, tprv, rec, rg, cofs, r, r1, col0, N, ld, ccol, nxi, acc, csum, beta2, ninvL2, invL, hcol, scl, iscl, iscl2, nxt, vec_ok, rsn, P, cbnd);
                } else {
                    if (fast)
                        pair_stage_rows<TS, NP, false, false, MODE, RPW>(tcur, tprv, rec, rg, cofs, r, r1, col0, N, ld, ccol, nxi, acc, csum, beta2, ninvL2, invL, hcol, scl, iscl, iscl2, nxt, vec_ok, rsn, P, cbnd);
                    else
                        pair_stage_rows<TS, NP, true, false, MODE, RPW>(tcur, tprv, rec, rg, cofs, r, r1, col0, N, ld, ccol, nxi, acc, csum, beta2, ninvL2, invL, hcol, scl, iscl, iscl2, nxt, vec_ok, rsn, P, cbnd);
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[slot]);
            if (producer && pok && kprod < kend) {   // refill this slot with the stage S ahead
                pok = produce_stage<TS, NP, MODE, RS>(P, stage0, full, empty, ppos, kprod >= (unsigned long long)S, pc, c, p);
                pc.advance(N);
                ppos.next();
                ++kprod;
            }
            __syncwarp();   // reconverge warp 0 after the producer lane
            // shift the row-sum batch (most recent stage in the last RPW entries)
#pragma unroll
            for (int q = 0; q < 8 - RPW; ++q) rsb[q] = rsb[q + RPW];
#pragma unroll
            for (int i = 0; i < RPW; ++i) rsb[8 - RPW + i] = rsn[i];
            ++nb;
            if (nb == SB || r + RS >= r1) {
                flush_row_sums<RS>(rsb, nb, r, rg, r1, rp, P.Q, lane, keep);
#pragma unroll
                for (int q = 0; q < 8; ++q) rsb[q] = 0.0f;
                nb = 0;
            }
        }
        // column partials of this segment, one block per row group (summed in FP64 by foldA)
        const int slotc = (int)(s - first_stripe);
        float *cp = P.colpart + (((vc * P.slots + slotc) * kWR + rg) * (NP + 1)) * kW + wc * 128 + lane * 4;
        st_keep(reinterpret_cast<ulonglong2 *>(cp), make_ulonglong2(csum[0], csum[1]), keep);
#pragma unroll
        for (int q = 0; q < NP; ++q)
            st_keep(reinterpret_cast<ulonglong2 *>(cp + (1 + q) * kW), make_ulonglong2(acc[0][q], acc[1][q]), keep);
        u += r1 - r0;
    }
    kstage += nst;
    __syncthreads();
}

// Compensated FP32 accumulation: (hi, lo) with hi + lo the running sum; each FP32 term is
// added exactly to hi by Knuth's TwoSum and its rounding error collected in lo.  About 2^-48
// relative for the sums of FP32 partials here, on the FP32 pipe (GB300's FP64 pipe is ~30x
// narrower); read back as (double)hi + (double)lo.
__device__ __forceinline__ void ff_add(float &hi, float &lo, float b)
{
    const float s = hi + b;
    const float bb = s - hi;
    lo += (hi - (s - bb)) + (b - bb);
    hi = s;
}
__device__ __forceinline__ double ff_value(float hi, float lo) { return (double)hi + (double)lo; }

// Aggregates of the values the pair pass accumulated for row and column l, reduced from its
// partials in a fixed order (deterministic): R = row sum, Cc = column sum, TX = (Theta^T X)_l,
// with Theta the array of values the pass produced (theta^(1), or m in the ALCC passes).
template <int NP>
__device__ __forceinline__ void gather_adjoint64(const Params &P, long long l, double &R, double &Cc,
                                                 double (&TX)[NP]);

template <int NP>
__device__ __forceinline__ void gather_adjoint(const Params &P, long long l, double &R, double &Cc, double (&TX)[NP])
{
    if (P.f64) {
        gather_adjoint64<NP>(P, l, R, Cc, TX);
        return;
    }
    const int Q4 = P.Q >> 2;   // row partials per row, in float4 units
    // row sum: the Q (>= 2S, zero padded) contiguous partials of row l, independent 16-byte loads
    // issued 16 at a time (the fold is bound by the round trips to L2), summed in four
    // interleaved compensated chains (one per vector component) that are added at the end
    const float4 *rp4 = reinterpret_cast<const float4 *>(P.rowpart + l * P.Q);
    float rh[4] = {0.0f, 0.0f, 0.0f, 0.0f}, rl[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    int q = 0;
    for (; q + 16 <= Q4; q += 16) {
        float4 t[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) t[i] = __ldcg(rp4 + q + i);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            ff_add(rh[0], rl[0], t[i].x);
            ff_add(rh[1], rl[1], t[i].y);
            ff_add(rh[2], rl[2], t[i].z);
            ff_add(rh[3], rl[3], t[i].w);
        }
    }
    for (; q < Q4; ++q) {
        const float4 t = __ldcg(rp4 + q);
        ff_add(rh[0], rl[0], t.x);
        ff_add(rh[1], rl[1], t.y);
        ff_add(rh[2], rl[2], t.z);
        ff_add(rh[3], rl[3], t.w);
    }
    R = (ff_value(rh[0], rl[0]) + ff_value(rh[1], rl[1])) + (ff_value(rh[2], rl[2]) + ff_value(rh[3], rl[3]));
    const long long s = l / kW, cl = l - s * kW;
    // CTAs whose unit range meets stripe s, ascending (host table: no dependent search)
    const long long c0 = __ldg(P.sc0 + s), c1 = __ldg(P.sc1 + s);
    float ch = 0.0f, clo = 0.0f, th[NP], tl[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) th[k] = tl[k] = 0.0f;
#pragma unroll 2
    for (long long cta = c0; cta < c1; ++cta) {
        const long long fs = __ldg(P.cfs + cta);
        if (fs >= 0) {
            const float *cp0 = P.colpart + ((cta * P.slots + (s - fs)) * P.cgroups * (NP + 1)) * kW + cl;
            // all (group, component) loads of one segment are independent: issue them together
            auto add_groups = [&](auto G) {
                constexpr int NG = decltype(G)::value;
                float cv[NG], tv[NG][NP];
#pragma unroll
                for (int g = 0; g < NG; ++g) {
                    const float *cp = cp0 + g * (NP + 1) * kW;
                    cv[g] = __ldcg(cp);
#pragma unroll
                    for (int k = 0; k < NP; ++k) tv[g][k] = __ldcg(cp + (1 + k) * kW);
                }
#pragma unroll
                for (int g = 0; g < NG; ++g) {
                    ff_add(ch, clo, cv[g]);
#pragma unroll
                    for (int k = 0; k < NP; ++k) ff_add(th[k], tl[k], tv[g][k]);
                }
            };
            if (P.cgroups == kWR)
                add_groups(std::integral_constant<int, kWR>());
            else
                add_groups(std::integral_constant<int, 1>());
        }
    }
    Cc = ff_value(ch, clo);
#pragma unroll
    for (int k = 0; k < NP; ++k) TX[k] = ff_value(th[k], tl[k]);
}

// The same aggregates from the FP64 partials of the FP64 pass, added in FP64 in the same fixed order.
template <int NP>
__device__ __forceinline__ void gather_adjoint64(const Params &P, long long l, double &R, double &Cc,
                                                 double (&TX)[NP])
{
    const double *rp = P.rowpart64 + l * P.Q;
    double r = 0.0;
    for (int q = 0; q < P.Q; ++q) r += __ldcg(rp + q);
    R = r;
    const long long s = l / kW, cl = l - s * kW;
    const long long c0 = __ldg(P.sc0 + s), c1 = __ldg(P.sc1 + s);
    double cc = 0.0, tx[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) tx[k] = 0.0;
    // one pre-reduced block per CTA segment (the FP64 pass adds its row groups in shared memory)
    for (long long cta = c0; cta < c1; ++cta) {
        const long long fs = __ldg(P.cfs + cta);
        if (fs >= 0) {
            const double *cp = P.colpart64 + ((cta * P.slots + (s - fs)) * (NP + 1)) * kW + cl;
            cc += __ldcg(cp);
#pragma unroll
            for (int k = 0; k < NP; ++k) tx[k] += __ldcg(cp + (1 + k) * kW);
        }
    }
    Cc = cc;
#pragma unroll
    for (int k = 0; k < NP; ++k) TX[k] = tx[k];
}

// Four multipliers theta[idx .. idx+3] of the stored array (16-byte aligned), as doubles.
template <typename TS>
__device__ __forceinline__ void load_theta4(const TS *th, long long idx, float iscl, double (&o)[4])
{
    if constexpr (std::is_same<TS, double>::value) {
        const double2 a = __ldcg(reinterpret_cast<const double2 *>(th + idx));
        const double2 b = __ldcg(reinterpret_cast<const double2 *>(th + idx + 2));
        o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
    } else {
        using St = Store<TS>;
        float t[4];
        St::unpack(__ldcg(reinterpret_cast<const typename St::Vec *>(th + idx)), t, iscl);
#pragma unroll
        for (int j = 0; j < 4; ++j) o[j] = (double)t[j];
    }
}

// ---------------------------------------------------------------------------
// Finite ball in Q_2: sum of squares of the clamped multipliers of iteration l (the pairs this
// CTA's pair pass wrote, and the y >= 0 rows of its fold rows), and the radial scaling of the
// stored array once foldA(l) knows the factor.  FP64 sums; FP32 or FP64 storage.
// ---------------------------------------------------------------------------
template <typename TS, int NP>
__device__ void phase_ball_norm(const Params &P, long long ell, double *red, long long vc)
{
    const int p = (int)(ell & 1);
    const TS *__restrict__ th = (const TS *)P.theta[p];
    const long long N = P.N, ld = P.ld;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double ss = 0.0;
    long long u = unit_begin(P, vc);
    const long long uend = unit_begin(P, vc + 1);
    while (u < uend) {
        const long long s = u / N, r0 = u - s * N, r1 = min(N, r0 + (uend - u));
        const long long col0 = s * kW + (warp & 1) * 128 + lane * 4;
        if (col0 < ld)
            for (long long r = r0 + (warp >> 1); r < r1; r += kWR) {
                double t[4];
                load_theta4<TS>(th, r * ld + col0, P.st_inv_scale, t);
#pragma unroll
                for (int j = 0; j < 4; ++j) ss += t[j] * t[j];   // padding columns and diagonal hold 0
            }
        u += r1 - r0;
    }
    for (RowIter it(P, vc); it.more(); it.next()) {
        const long long l = it.row();
        if (l < N) {
            const double m = __ldcg(P.mu[p] + l);
            ss += m * m;
        }
    }
    double vals[1] = {ss};
    const bool ismax[1] = {false};
    block_reduce<1>(vals, ismax, red);
    if (threadIdx.x == 0) P.ballpart[vc] = vals[0];
}

template <typename TS>
__device__ void phase_ball_scale(const Params &P, long long ell, long long vc)
{
    const int p = (int)(ell & 1);
    const double c = __ldcg(&P.st->scal[p].ball_c);
    if (!(c < 1.0)) return;
    if constexpr (std::is_same<TS, float>::value || std::is_same<TS, double>::value) {
        TS *__restrict__ th = (TS *)P.theta[p];
        const long long N = P.N, ld = P.ld;
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        long long u = unit_begin(P, vc);
        const long long uend = unit_begin(P, vc + 1);
        while (u < uend) {
            const long long s = u / N, r0 = u - s * N, r1 = min(N, r0 + (uend - u));
            const long long col0 = s * kW + (warp & 1) * 128 + lane * 4;
            if (col0 < ld)
                for (long long r = r0 + (warp >> 1); r < r1; r += kWR)
#pragma unroll
                    for (int j = 0; j < 4; ++j) th[r * ld + col0 + j] = (TS)((double)th[r * ld + col0 + j] * c);
            u += r1 - r0;
        }
    }
}

// ---------------------------------------------------------------------------
// foldA(l): reduce partials of theta^(1)_l in FP64; eta(theta^(1)_l); dual terms
// ---------------------------------------------------------------------------
template <int NP>
__device__ void phase_foldA(const Params &P, long long ell, double *red, long long vc, bool stats = true)
{
    const int p = (int)(ell & 1);
    const long long N = P.N;
    const int n = P.n;
    // fused foldB(l+1): its momentum weight needs no reduction in plain P-APG
    __shared__ double s_nbeta;
    if (P.fuse) {
        if (threadIdx.x == 0) {
            const Scal nw = next_scal_plain(P, ell + 1);
            s_nbeta = nw.beta;
            if (vc == 0) P.st->scal[(ell + 1) & 1] = nw;
        }
        __syncthreads();
    }
    // finite ball: theta^(1)_l = c Pi_{>=0}(.), c = min(1, B_theta / ||(clamped pairs, clamped mu)||_2),
    // from the partial sums of squares of the norm phase, reduced in the same order by every CTA
    __shared__ double s_ballc;
    double ballc = 1.0;
    if (P.ball) {
        if (threadIdx.x < 32) {
            double ss = 0.0;
            for (int i = threadIdx.x; i < P.G; i += 32) ss += __ldcg(P.ballpart + i);
            ss = warp_sum(ss);
            if (threadIdx.x == 0) {
                const double nrm = sqrt(ss);
                s_ballc = nrm > P.B_theta ? P.B_theta / nrm : 1.0;
                if (vc == 0) P.st->scal[p].ball_c = s_ballc;
            }
        }
        __syncthreads();
        ballc = s_ballc;
    }
    double a = 0.0, b = 0.0, cc = 0.0, mviol = 0.0, mcomp = 0.0, sviol = 0.0, smuy = 0.0;
    for (RowIter it(P, vc); it.more(); it.next()) {
        const long long l = it.row();
        if (l >= N) continue;
        double R, Cc, TX[NP];
        gather_adjoint<NP>(P, l, R, Cc, TX);
        if (P.ball && ballc < 1.0) {
            R *= ballc;
            Cc *= ballc;
#pragma unroll
            for (int k = 0; k < NP; ++k) TX[k] *= ballc;
            P.mu[p][l] = __ldcg(P.mu[p] + l) * ballc;
        }
        const double v = R - Cc;               // (A_1^T theta)_l = row sum - column sum
        P.v[p][l] = v;
        const double hl = __ldcg(P.h + l), mu = __ldcg(P.mu[p] + l);
        const double y = hl + v + mu;          // Step 1 closed form
        const double ys = y - P.shift;
        double dw = 0.0, doff = 0.0, xin = 0.0;
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            float xf = 0.0f;
            if (k < n) {
                const double xk = __ldg(P.X64 + l * n + k);
                const double wk = Cc * xk - TX[k];   // (A_2^T theta)_l = Cc_l x_l - (theta^T X)_l
                P.w[p][l * n + k] = wk;
                double xi = wk * P.inv_gamma;
                if (P.xi_off) {
                    const double o = __ldcg(P.xi_off + l * n + k);
                    xi += o;
                    doff += o * xk;
                }
                P.xi1_64[l * n + k] = xi;
                dw += wk * xk;
                if (stats) xin += xi * xi;
                xf = (float)xi;
            }
            P.xi1[l * NP + k] = xf;
        }
        P.dd[p][l] = dw;
        const double d = dw * P.inv_gamma + doff;   // xi_l . x_l
        P.y1[l] = y;
        P.yrow1[l] = (float)ys;
        P.ccol1[l] = (float)(d - ys);
        if (stats) {
            const double uu = y - hl;
            a += uu * uu;
            b += xin;
            cc += uu * y;
            mviol = fmax(mviol, -y);
            mcomp = fmax(mcomp, mu * fabs(y));
            if (y < 0.0) sviol += y * y;
            smuy += mu * y;
        }
        if (!isfinite(y) || !isfinite(d)) atomicCAS(&P.st->error, 0, ERR_NUMERIC);
        if (P.fuse) foldB_row<NP>(P, p, p ^ 1, l, s_nbeta);   // this row of foldB(l+1)
    }
    if (!stats) return;   // the same value in every thread of the grid
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
// With FP64 multipliers the screen is the FP64 evaluation itself (F64X).
template <typename TS, int NP, bool F64>
__device__ void phase_kkt(const Params &P, long long ell, double *red, long long vc)
{
    constexpr bool F64X = F64 || std::is_same<TS, double>::value;
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
            double tc[4];
            load_theta4<TS>(th, r * ld + col0, iscl, tc);
            if (F64X) {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const long long l2 = col0 + j;
                    if (!colv[j] || l2 == r) continue;
                    double g = __ldcg(P.y1 + r) - __ldcg(P.y1 + l2);
                    for (int k = 0; k < n; ++k) g -= __ldcg(P.xi1_64 + l2 * n + k) * (__ldg(P.X64 + r * n + k) - __ldg(P.X64 + l2 * n + k));
                    mviol = fmax(mviol, -g);
                    mcomp = fmax(mcomp, tc[j] * fabs(g));
                    if (g < 0.0) sviol += g * g;
                    sthg += tc[j] * g;
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
                    const float t = (float)tc[j];
                    tv_viol = fmaxf(tv_viol, -g);
                    tv_comp = fmaxf(tv_comp, t * fabsf(g));
                    if (g < 0.0f) tv_s2 = fmaf(g, g, tv_s2);
                    tv_tg = fmaf(t, g, tv_tg);
                }
            }
        }
        if (!F64X) {
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
