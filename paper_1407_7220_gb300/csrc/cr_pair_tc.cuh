// cr_pair_tc.cuh -- the pair pass with its two dense products on the tensor cores (tcgen05).
//
// Step 2 of P-APG (Fig. 2) at K = N needs, for every pair p = (l1, l2) of a tile, the residual
//   g_p = (y_l1 - s) + ccol_l2 - xi_l2 . x_l1            (ccol = xi.x - (y - s), Step 1 closed form)
// and the fused adjoint needs, for every column l2, sum_l1 theta_p x_l1 and sum_l1 theta_p.
// Over the rows of a segment both are small dense products:
//   D1 = Xi_stripe (256 x n) . X_rows^T (n x 64)        -> residual dot products (MMA1, per 64 rows)
//   D2 += Theta^T (256 x 16) . [X_rows | 1] (16 x n+1)   -> Theta^T X and column sums (MMA2, per stage)
// Both run as tcgen05.mma kind::tf32 with M = 128 (one MMA for the even columns of the stripe,
// one for the odd columns), accumulators in tensor memory.  Three TF32 products per FP32
// product (hi*hi + hi*lo + lo*hi, hi = TF32 rounding, lo = TF32 rounding of the remainder) give
// close to FP32 accuracy; a 16-bit theta is exact in TF32 and needs no split.
//
// CUDA cores keep the element-wise part: theta^(2), the projection, stochastic rounding, the
// store of theta^(1)_l, and the row sums (A_1^T, + part).  Consumer thread (warp w < 16,
// lane t) owns the tensor-memory lane m = 32 (w & 3) + t, i.e. columns 2m and 2m + 1 of the
// stripe, and RPW = RS/4 consecutive rows of every stage of RS rows (RS = 32 for a 16-bit
// theta, 16 for FP32, where two 32-row stages would not fit).  Warp 16 loads (TMA),
// warp 17 issues MMA1, warp 18 issues MMA2; each of the three runs on its own lane 0.
//
// Operand layouts (tcgen05 canonical K-major, no swizzle: an 8-row x 16-byte core matrix is
// 128 contiguous bytes; LBO = stride between core matrices along K, SBO = along M/N):
//   Xi (per stripe, smem for a whole segment): [eo][hl][16 row groups][KP/4][8][4] floats
//   X rows (per 8-row block, global and stage): [hl][KP/4][8][4]
//   [X | 1] transposed (per 8-row block):         [hl][N2/8][2][8][4]  (feature-major, K = rows)
// The partition starts every segment on an 8-row boundary, so a stage's 16 rows and a
// group's 64 rows are whole 8-row blocks of the precomputed X arrays.
// A tcgen05.mma costs about the same for N = 16 as for N = 64 (measured), hence 64-row
// groups for MMA1; its shared-memory descriptors are built once per pass.
#pragma once

#include <type_traits>

#include "cr_kernels.cuh"

namespace crk {

constexpr int kTcWG = 4;                        // consumer warpgroups
constexpr int kTcWarps = 4 * kTcWG;             // consumer warps
constexpr int kTcThreads = (kTcWarps + 3) * 32; // + producer, MMA1 and MMA2 issuer warps

// ---------------------------------------------------------------------------
// tcgen05 / tensor-memory wrappers
// ---------------------------------------------------------------------------
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// whole warp; writes the tensor-memory base address to *dst (shared memory)
__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Shared-memory matrix descriptor: start address, leading/stride byte offsets, version 1, no swizzle.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}
// Instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B, both K-major, M x N.
__host__ __device__ constexpr uint32_t umma_idesc_tf32(int M, int N)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// D (tensor memory) (+)= A (shared) . B^T (shared)
__device__ __forceinline__ void umma_ss(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
                 "l"(a), "l"(b), "r"(idesc), "r"(acc)
                 : "memory");
}
// D (tensor memory) (+)= A (tensor memory) . B^T (shared)
__device__ __forceinline__ void umma_ts(uint32_t d, uint32_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d),
                 "r"(a), "l"(b), "r"(idesc), "r"(acc)
                 : "memory");
}
// the barrier receives one arrival once every tcgen05 operation issued so far by this thread is done
__device__ __forceinline__ void umma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8])
{
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float (&v)[4])
{
    uint32_t r[4];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_st4(uint32_t taddr, const float (&v)[4])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};" ::"r"(taddr), "f"(v[0]), "f"(v[1]),
                 "f"(v[2]), "f"(v[3])
                 : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v)
{
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                   "=r"(r[15])
                 : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const float (&v)[8])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), "f"(v[0]),
                 "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7])
                 : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_ldv(uint32_t t, float (&v)[4]) { tmem_ld4(t, v); }
__device__ __forceinline__ void tmem_ldv(uint32_t t, float (&v)[8]) { tmem_ld8(t, v); }
__device__ __forceinline__ void tmem_stv(uint32_t t, const float (&v)[4]) { tmem_st4(t, v); }
__device__ __forceinline__ void tmem_stv(uint32_t t, const float (&v)[8]) { tmem_st8(t, v); }
__device__ __forceinline__ float tf32_rna(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// ---------------------------------------------------------------------------
// shapes
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int tc_kp(int NP) { return (NP + 7) / 8 * 8; }          // K of MMA1 (TF32 K-step 8)
__host__ __device__ constexpr int tc_n2(int NP) { return (NP + 1 + 15) / 16 * 16; }   // N of MMA2 (features + ones)
__host__ __device__ constexpr size_t tc_xi_floats(int NP) { return (size_t)2 * 2 * 128 * tc_kp(NP); }   // per stripe
__host__ __device__ constexpr size_t tc_xr_floats(int NP) { return (size_t)2 * tc_kp(NP) * 8; }          // per 8-row block
__host__ __device__ constexpr size_t tc_xt_floats(int NP) { return (size_t)2 * tc_n2(NP) * 8; }          // per 8-row block

constexpr int kGR = 64;   // largest MMA1 group (rows); the X arrays carry kGR rows of padding

template <typename TS, int NP> struct TcShape {
    static constexpr int KP = tc_kp(NP);
    static constexpr int N2 = tc_n2(NP);
    static constexpr bool SPLIT = std::is_same<TS, float>::value;   // FP32 theta needs a hi/lo split
    // rows of a stage: 32 for a 16-bit theta; 16 for FP32 (two 32-row FP32 stages left too
    // shallow a ring: 1.07 vs 1.05 ms per pass at N = 20,000, n = 10)
    static constexpr int RS = SPLIT ? 16 : 32;
    static constexpr int RPW = RS / kTcWG;                            // rows of a stage per consumer warp
    // rows of one MMA1 group (N of MMA1): an MMA with N = 64 costs about what N = 16 does
    static constexpr int GR = kGR;
    static_assert(GR % RS == 0 && GR <= kGR && RS % 8 == 0 && (RPW == 4 || RPW == 8), "stage split");
    static constexpr int REC = RecLayout<NP>::REC;
    static constexpr size_t tile_bytes = (size_t)RS * kW * sizeof(TS);
    static constexpr size_t rec_bytes = (size_t)RS * REC * sizeof(float);
    static constexpr size_t xr_block = tc_xr_floats(NP) * 4;   // bytes of one 8-row block
    static constexpr size_t xt_block = tc_xt_floats(NP) * 4;
    static constexpr size_t off_rec = 2 * tile_bytes;
    static constexpr size_t off_xt = off_rec + rec_bytes;
    static constexpr size_t stage_bytes = off_xt + (RS / 8) * xt_block;
    static constexpr size_t xi_bytes = tc_xi_floats(NP) * 4;
    static constexpr size_t xg_bytes = (GR / 8) * xr_block;    // X rows of one group
    static constexpr size_t off_xg = xi_bytes;                  // 2 group buffers
    static constexpr size_t off_stage = xi_bytes + 2 * xg_bytes;
    static constexpr int kFit = (int)((kSmemBudget - 128 - off_stage) / stage_bytes);
    static constexpr int kStages = kFit < kMaxStages ? kFit : kMaxStages;
    static_assert(kStages >= 2, "tensor-core pipeline needs at least two stages");
    static_assert(stage_bytes % 128 == 0 && xi_bytes % 128 == 0 && xg_bytes % 128 == 0 && off_xt % 128 == 0,
                  "stage buffers must stay 128-byte aligned");
    static constexpr size_t bytes = off_stage + kStages * stage_bytes + 128;
    // D2 (the adjoint product) is accumulated by the tensor cores over chunks of 32 rows only:
    // their FP32 accumulation truncates (rounds toward zero), so a sum carried over a whole
    // segment (thousands of MMAs) drifts below the true column sums (measured: the dual value
    // 2e-4 low at N = 20,000).  Each chunk's D2 is added to FP32 registers (round to nearest)
    // by the consumer warps, a quarter of the columns per warpgroup.
    static constexpr int CH = 32 / RS;   // stages per D2 chunk
    static constexpr int H2 = N2 / 2;    // D2 columns per warpgroup
    // tensor-memory columns: D1 (2 group buffers x {even, odd} x 64 rows), A2 = theta^T
    // (NA2 buffers x {even hi, odd hi[, even lo, odd lo]} x RS), D2 (ND2 chunk buffers x {even, odd} x N2)
    static constexpr int A2W = (SPLIT ? 4 : 2) * RS;
    static constexpr int COL_A2 = 4 * GR;
    static constexpr int ND2 = (512 - COL_A2 - 4 * N2) / A2W >= 2 ? 2 : 1;
    static constexpr int NA2_FIT = (512 - COL_A2 - 2 * ND2 * N2) / A2W;
    static constexpr int NA2 = NA2_FIT > 4 ? 4 : NA2_FIT;   // theta^T buffers (what fits in 512 columns)
    static_assert(NA2 >= 2, "tensor memory");
    static_assert(H2 % 8 == 0 && 32 % RS == 0, "D2 chunk split");
    static constexpr int COL_D1 = 0, COL_D2 = COL_A2 + NA2 * A2W;
    static constexpr int COLS = COL_D2 + 2 * ND2 * N2;
    static constexpr uint32_t NCOLS = COLS <= 128 ? 128u : (COLS <= 256 ? 256u : 512u);
    static_assert(COLS <= 512, "tensor memory");
    static constexpr uint32_t IDESC1 = umma_idesc_tf32(128, GR);
    static constexpr uint32_t IDESC2 = umma_idesc_tf32(128, N2);
};

// Shared-memory barriers and the tensor-memory base of the tensor-core pair pass.
struct TcBars {
    uint64_t xgfull[2];              // X rows of a group landed
    uint64_t d1full[2], d1free[2];   // MMA1 of a group done / its D1 read by all consumer warps
    uint64_t a2full[4], a2free[4];   // theta^T of a stage written by all consumer warps / MMA2 of the stage done
    uint64_t d2done[2], d2free[2];   // a D2 chunk's MMA2 chain done / that D2 buffer read by all consumer warps
    uint64_t xifull;                 // Xi of the segment's stripe landed
    uint64_t drain[2];               // end of pass: every MMA of issuer 1 / issuer 2 done
    uint32_t tmem;
    uint32_t drain_parity[2];        // completions of drain[i] so far, mod 2 (its issuer only)
    float rowx[4][2][4][8];          // row sums of a stage per warpgroup, stage parity, 64-column slab
};

__device__ __forceinline__ void tc_init_bars(TcBars &B)
{
    if (threadIdx.x == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(&B.xgfull[i], 1);
            mbar_init(&B.d1full[i], 1);
            mbar_init(&B.d1free[i], kTcWarps);
        }
        for (int i = 0; i < 4; ++i) {
            mbar_init(&B.a2full[i], kTcWarps);
            mbar_init(&B.a2free[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&B.d2done[i], 1);
            mbar_init(&B.d2free[i], kTcWarps);
        }
        mbar_init(&B.xifull, 1);
        for (int i = 0; i < 2; ++i) {
            mbar_init(&B.drain[i], 1);
            B.drain_parity[i] = 0;
        }
        fence_mbar_init();
    }
}

// Stage ring of the tensor-core pass: the "empty" barrier of a slot counts the consumer
// warps and the commit of the MMA2 that read the slot's [X | 1] blocks.  (A per-slot barrier
// completes once per use of the slot, so the producer's parity wait cannot alias.)
__device__ __forceinline__ void tc_init_pipeline(uint64_t *full, uint64_t *empty)
{
    if (threadIdx.x == 0) {
        for (int i = 0; i < kMaxStages; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], kTcWarps + 1);
        }
        fence_mbar_init();
    }
}

// Tensor memory for the pass (warp 0), before the first use; the address is read by all.
template <typename TS, int NP> __device__ __forceinline__ void tc_alloc(TcBars &B)
{
    if ((threadIdx.x >> 5) == 0) tmem_alloc(&B.tmem, TcShape<TS, NP>::NCOLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}
template <typename TS, int NP> __device__ __forceinline__ void tc_free(TcBars &B)
{
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if ((threadIdx.x >> 5) == 0) tmem_dealloc(B.tmem, TcShape<TS, NP>::NCOLS);
}

// Two adjacent theta entries of a row (column index even, so the access is aligned).
template <typename TS> struct Pair2;
template <> struct Pair2<float> {
    __device__ static __forceinline__ f2 load(const float *p, float) { return *reinterpret_cast<const f2 *>(p); }
    __device__ static __forceinline__ void store(float *p, f2 s) { *reinterpret_cast<f2 *>(p) = s; }
};
template <> struct Pair2<__nv_bfloat16> {
    __device__ static __forceinline__ f2 load(const __nv_bfloat16 *p, float)
    {
        const uint32_t t = *reinterpret_cast<const uint32_t *>(p);
        return f2_make(__uint_as_float(t << 16), __uint_as_float(t & 0xFFFF0000u));
    }
    __device__ static __forceinline__ void store(__nv_bfloat16 *p, f2 s)
    {
        float a, b;
        f2_split(s, a, b);
        *reinterpret_cast<uint32_t *>(p) = __byte_perm(__float_as_uint(a), __float_as_uint(b), 0x7632u);
    }
    __device__ static __forceinline__ void store_bits(__nv_bfloat16 *p, uint32_t h) { *reinterpret_cast<uint32_t *>(p) = h; }
};
template <> struct Pair2<__half> {
    __device__ static __forceinline__ f2 load(const __half *p, float iscl)
    {
        const __half2 t = *reinterpret_cast<const __half2 *>(p);
        return f2_make(__low2float(t) * iscl, __high2float(t) * iscl);
    }
    __device__ static __forceinline__ void store(__half *p, f2 s)
    {
        float a, b;
        f2_split(s, a, b);
        *reinterpret_cast<__half2 *>(p) = __floats2half2_rn(a, b);
    }
    // the stored FP16 numbers as floats, without the inverse scale
    __device__ static __forceinline__ f2 load_scaled(const __half *p)
    {
        const __half2 t = *reinterpret_cast<const __half2 *>(p);
        return f2_make(__low2float(t), __high2float(t));
    }
    __device__ static __forceinline__ void store_bits(__half *p, uint32_t h) { *reinterpret_cast<uint32_t *>(p) = h; }
};

// Row sums of one stage (8 rows per warp) reduced across the warp with a transposing
// butterfly (9 shuffles); entry e = 4*bit4 + 2*bit3 + bit2 of the lane id is row r8 + e.  The
// four warps of a warpgroup (the four 64-column slabs of the stripe, q = 0..3) then add their
// sums through shared memory (xb: this warpgroup's [4][8] block for the stage's parity; named
// barrier 1 + wg), and warp q = 0 stores one partial per (stripe, row), adding in order of q and
// multiplying by osc (the inverse storage scale of FP16 multipliers, else 1).
__device__ __forceinline__ void tc_flush_rows(float (&v)[8], long long r8, long long r1, float *rp, int Q, int lane,
                                              float *xb, int q, int wg, float osc)
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
    const int e = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
    if ((lane & 3) == 0) xb[q * 8 + e] = v[0];
    named_barrier_sync(1 + wg, 128);
    if (q == 0 && (lane & 3) == 0) {
        const long long row = r8 + e;
        const float t = (((xb[e] + xb[8 + e]) + xb[16 + e]) + xb[24 + e]) * osc;
        if (row < r1) st_keep(rp + row * Q, t, l2_evict_last());
    }
}

// The same for 4 rows per warp (6 shuffles); entry e = 2*bit4 + bit3 is row r4 + e.
__device__ __forceinline__ void tc_flush_rows(float (&v)[4], long long r4, long long r1, float *rp, int Q, int lane,
                                              float *xb, int q, int wg, float osc)
{
    const unsigned full = 0xffffffffu;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const bool hi = lane & 16;
        const float send = hi ? v[i] : v[i + 2], keep = hi ? v[i + 2] : v[i];
        v[i] = keep + __shfl_xor_sync(full, send, 16);
    }
    {
        const bool hi = lane & 8;
        const float send = hi ? v[0] : v[1], keep = hi ? v[1] : v[0];
        v[0] = keep + __shfl_xor_sync(full, send, 8);
    }
    v[0] += __shfl_xor_sync(full, v[0], 4);
    v[0] += __shfl_xor_sync(full, v[0], 2);
    v[0] += __shfl_xor_sync(full, v[0], 1);
    const int e = ((lane >> 4) & 1) * 2 + ((lane >> 3) & 1);
    if ((lane & 7) == 0) xb[q * 8 + e] = v[0];
    named_barrier_sync(1 + wg, 128);
    if (q == 0 && (lane & 7) == 0) {
        const long long row = r4 + e;
        const float t = (((xb[e] + xb[8 + e]) + xb[16 + e]) + xb[24 + e]) * osc;
        if (row < r1) st_keep(rp + row * Q, t, l2_evict_last());
    }
}

// Step 2 on the RPW rows x 2 columns of one consumer thread in one stage.  MASK handles the
// diagonal, columns >= N and rows past the segment; SR: stochastic rounding.  nrow points at
// theta^(1)_l[first row][col0].  Outputs: theta^T for MMA2 (TF32 hi/lo when SPLIT), row sums.
template <typename TS, int NP, bool SR, bool MASK>
__device__ __forceinline__ void tc_rows(const TS *tcur, const TS *tprv, const float *rec, int rb, int m, long long r,
                                        long long r1, long long col0, bool va, bool vb, f2 ccol,
                                        const float (&de)[TcShape<TS, NP>::RPW], const float (&dd)[TcShape<TS, NP>::RPW],
                                        f2 beta2, f2 ninvL2, float invL, uint32_t hcol, float scl, float iscl,
                                        f2 iscl2, f2 scl2, TS *nrow, long long ld, float (&ae)[TcShape<TS, NP>::RPW],
                                        float (&ao)[TcShape<TS, NP>::RPW], float (&le)[TcShape<TS, NP>::RPW],
                                        float (&lo)[TcShape<TS, NP>::RPW], float (&rs)[TcShape<TS, NP>::RPW])
{
    using St = Store<TS>;
    using Sh = TcShape<TS, NP>;
    constexpr int REC = Sh::REC;
    // FP16 multipliers are stored as theta * 2^e: the step runs on scaled values (theta^(2) and g
    // times 2^e, exact), which gives the stored numbers of the unscaled step; the row sums and the
    // theta^T operand stay scaled and the caller unscales the sums
    constexpr bool SCALED = std::is_same<TS, __half>::value;
    constexpr bool BF16 = std::is_same<TS, __nv_bfloat16>::value;
#pragma unroll
    for (int i = 0; i < Sh::RPW; ++i) {
        const int rl = rb + i;
        const long long rr = r + rl;
        const float y = rec[rl * REC];
        f2 tc2, tp2;
        if constexpr (SCALED) {
            tc2 = Pair2<TS>::load_scaled(tcur + rl * kW + 2 * m);
            tp2 = Pair2<TS>::load_scaled(tprv + rl * kW + 2 * m);
        } else {
            tc2 = Pair2<TS>::load(tcur + rl * kW + 2 * m, iscl);
            tp2 = Pair2<TS>::load(tprv + rl * kW + 2 * m, iscl);
        }
        const f2 th2 = f2_fma(beta2, f2_sub(tc2, tp2), tc2);   // theta^(2)
        f2 g = f2_sub(f2_add(f2_make(y, y), ccol), f2_make(de[i], dd[i]));
        const uint32_t h = SR ? hash_row(hcol, (uint32_t)rr) : 0u;
        f2 sv;   // Pi_{>=0}(theta^(2) - g/L) as stored
        uint32_t bits = 0;
        if constexpr (SCALED) {
            g = f2_mul(g, scl2);
            sv = St::template round2_scaled<SR>(th2, g, ninvL2, h, bits);
        } else if constexpr (BF16) {
            sv = St::template round2_bits<SR>(th2, g, ninvL2, h, bits);
        } else {
            sv = St::template round2<SR>(th2, g, ninvL2, invL, h, scl);
        }
        if (MASK) {
            float s0, s1;
            f2_split(sv, s0, s1);
            const bool vr = rr < r1;
            if (!vr || !va || col0 == rr) s0 = 0.0f;
            if (!vr || !vb || col0 + 1 == rr) s1 = 0.0f;
            sv = f2_make(s0, s1);
            if (va && vr) Pair2<TS>::store(nrow + i * ld, sv);
        } else if constexpr (SCALED || BF16) {
            Pair2<TS>::store_bits(nrow + i * ld, bits);
        } else {
            Pair2<TS>::store(nrow + i * ld, sv);
        }
        const f2 vv = SCALED ? sv : St::decoded2(sv, iscl2);
        float v0, v1;
        f2_split(vv, v0, v1);
        rs[i] = v0 + v1;
        if (Sh::SPLIT) {
            ae[i] = tf32_rna(v0);
            ao[i] = tf32_rna(v1);
            le[i] = v0 - ae[i];
            lo[i] = v1 - ao[i];
        } else {
            ae[i] = v0;
            ao[i] = v1;
        }
    }
}

// Issue the loads of one stage: the two theta tiles (TMA), the row records and the two
// 8-row blocks of [X | 1] transposed (bulk copies); reuse: wait for the slot's previous occupant.
template <typename TS, int NP>
__device__ __forceinline__ bool tc_produce(const Params &P, unsigned char *stage0, uint64_t *full, uint64_t *empty,
                                           const RingPos<TcShape<TS, NP>::kStages> &pos, bool reuse,
                                           const StageCursorT<TcShape<TS, NP>::RS> &cur, int c, int p, bool blocking,
                                           bool &issued)
{
    using Sh = TcShape<TS, NP>;
    issued = false;
    const int slot = pos.slot;
    if (reuse) {
        if (blocking) {
            if (!mbar_wait(P, &empty[slot], pos.phase ^ 1u)) return false;
        } else if (!mbar_test_wait(&empty[slot], pos.phase ^ 1u)) {
            return true;
        }
    }
    const int nrows = (int)min((long long)Sh::RS, cur.r1 - cur.r);
    unsigned char *st = stage0 + slot * Sh::stage_bytes;
    const long long blk = cur.r >> 3;
    const CUtensorMap *tm = Sh::RS == kRS ? P.tmap : P.tmap32;   // box of RS rows
    mbar_arrive_expect_tx(&full[slot], (uint32_t)(2 * Sh::tile_bytes + (size_t)nrows * Sh::REC * 4 +
                                                  (Sh::RS / 8) * Sh::xt_block));
    const uint64_t keep = l2_evict_last();
    tma_load_2d(st, &tm[c], (int)(cur.s * kW), (int)cur.r, &full[slot]);
    tma_load_2d(st + Sh::tile_bytes, &tm[p], (int)(cur.s * kW), (int)cur.r, &full[slot]);
    bulk_load_hint(st + Sh::off_rec, P.rowrec + cur.r * Sh::REC, (uint32_t)(nrows * Sh::REC * 4), &full[slot], keep);
    bulk_load_hint(st + Sh::off_xt, P.xt_tc + blk * tc_xt_floats(NP), (uint32_t)((Sh::RS / 8) * Sh::xt_block),
                   &full[slot], keep);
    issued = true;
    return true;
}

// Shared-memory descriptors of the pass, built once (the start-address field is the low 14
// bits, in 16-byte units, so a byte offset o < 256 KB - base is added as o >> 4).
struct TcDesc {
    uint64_t xi[2][2];   // [even/odd][hi/lo]: A of MMA1, K-step 0
    uint64_t xg[2][2];   // [group buffer][hi/lo]: B of MMA1, K-step 0
    uint64_t xt[2];      // [hi/lo]: B of MMA2 in stage slot 0, K-step 0
};

template <typename TS, int NP>
__device__ __forceinline__ TcDesc tc_descs(const unsigned char *smem)
{
    using Sh = TcShape<TS, NP>;
    constexpr int KP = Sh::KP;
    TcDesc D;
    const uint32_t xi = smem_u32(smem), xg = smem_u32(smem + Sh::off_xg), xt = smem_u32(smem + Sh::off_stage + Sh::off_xt);
#pragma unroll
    for (int e = 0; e < 2; ++e) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            D.xi[e][h] = umma_desc(xi + (e * 2 + h) * 512 * KP, 128, 32 * KP);
            D.xg[e][h] = umma_desc(xg + e * (uint32_t)Sh::xg_bytes + h * 32 * KP, 128, (uint32_t)Sh::xr_block);
        }
        D.xt[e] = umma_desc(xt + e * 32 * Sh::N2, 128, 256);
    }
    return D;
}

// MMA1 of one group into D1 buffer b: for the even and the odd columns of the stripe,
// D1 (128 x 64 rows) = Xi_hi X_hi^T + Xi_hi X_lo^T + Xi_lo X_hi^T over KP/8 K-steps of 8.
template <typename TS, int NP>
__device__ __forceinline__ void tc_mma1(uint32_t tb, const TcDesc &D, int xb, int b, uint64_t *done)
{
    using Sh = TcShape<TS, NP>;
#pragma unroll
    for (int eo = 0; eo < 2; ++eo) {
        const uint32_t d = tb + Sh::COL_D1 + 2 * Sh::GR * b + Sh::GR * eo;
#pragma unroll
        for (int s = 0; s < Sh::KP / 8; ++s) {
            umma_ss(d, D.xi[eo][0] + 16 * s, D.xg[xb][0] + 16 * s, Sh::IDESC1, s > 0 ? 1u : 0u);
            umma_ss(d, D.xi[eo][0] + 16 * s, D.xg[xb][1] + 16 * s, Sh::IDESC1, 1u);
            umma_ss(d, D.xi[eo][1] + 16 * s, D.xg[xb][0] + 16 * s, Sh::IDESC1, 1u);
        }
    }
    umma_commit(done);
}

// MMA2 of one stage: D2 (+)= Theta^T [X | 1] for the even and the odd columns, K = RS rows
// (RS/8 blocks of 8); theta^T comes from tensor memory (A2 buffer b).
template <typename TS, int NP>
__device__ __forceinline__ void tc_mma2(uint32_t tb, const TcDesc &D, int slot, int b, bool first, int db)
{
    using Sh = TcShape<TS, NP>;
    constexpr int N2 = Sh::N2;
    const uint64_t so = (uint64_t)(slot * (uint32_t)(Sh::stage_bytes >> 4));
#pragma unroll
    for (int eo = 0; eo < 2; ++eo) {
        const uint32_t d = tb + Sh::COL_D2 + 2 * N2 * db + N2 * eo;
        const uint32_t a = tb + Sh::COL_A2 + Sh::A2W * b + Sh::RS * eo;
#pragma unroll
        for (int s = 0; s < Sh::RS / 8; ++s) {
            const uint64_t bh = D.xt[0] + so + s * (Sh::xt_block >> 4), bl = D.xt[1] + so + s * (Sh::xt_block >> 4);
            umma_ts(d, a + 8 * s, bh, Sh::IDESC2, (first && s == 0) ? 0u : 1u);
            umma_ts(d, a + 8 * s, bl, Sh::IDESC2, 1u);
            if (Sh::SPLIT) umma_ts(d, a + 2 * Sh::RS + 8 * s, bh, Sh::IDESC2, 1u);
        }
    }
}

// Walks the MMA1 groups (GR rows of one stripe) of a unit range in consumption order.
template <int GR> struct GroupCursor {
    long long u, uend, s, r0, r1, r;
    __device__ __forceinline__ void begin(long long u0, long long ue, long long N)
    {
        u = u0;
        uend = ue;
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
    __device__ __forceinline__ bool valid() const { return u < uend; }
    __device__ __forceinline__ void advance(long long N)
    {
        r += GR;
        if (r >= r1) {
            u += r1 - r0;
            next_segment(N);
        }
    }
};

// Producer (lane 0 of warp 16): the loads of every stage, in order, each into its ring slot
// once the slot's previous stage was released by the consumers and by its MMA2; Xi of a
// stripe once the MMA1s of the previous segment are done.
template <typename TS, int NP>
__device__ __forceinline__ void tc_producer(const Params &P, long long ubeg, long long uend, int c, int p,
                                            unsigned char *smem, uint64_t *full, uint64_t *empty, TcBars &B,
                                            unsigned long long k0, unsigned long long kend, unsigned long long g0)
{
    using Sh = TcShape<TS, NP>;
    constexpr int S = Sh::kStages;
    const long long N = P.N;
    unsigned char *stage0 = smem + Sh::off_stage;
    fence_proxy_async();
    StageCursorT<Sh::RS> pc;
    pc.begin(ubeg, uend, N);
    RingPos<S> ppos;
    ppos.init(k0);
    unsigned long long gseg = g0;   // first group of the current segment
    bool ok = true;
    for (unsigned long long k = k0; k < kend && ok; ++k) {
        if (pc.r == pc.r0) {
            if (k != k0) {
                // Xi is read by every MMA1 of the previous segment: wait for its last group
                const unsigned long long gl = gseg - 1;
                ok = mbar_wait(P, &B.d1full[gl & 1], (uint32_t)((gl >> 1) & 1));
            }
            if (ok) {
                mbar_arrive_expect_tx(&B.xifull, (uint32_t)Sh::xi_bytes);
                bulk_load(smem, P.xi_tc + (size_t)pc.s * tc_xi_floats(NP), (uint32_t)Sh::xi_bytes, &B.xifull);
            }
            gseg += (unsigned long long)((pc.r1 - pc.r0 + Sh::GR - 1) / Sh::GR);
        }
        bool issued;
        if (ok) ok = tc_produce<TS, NP>(P, stage0, full, empty, ppos, k >= (unsigned long long)S, pc, c, p, true, issued);
        pc.advance(N);
        ppos.next();
    }
}

// MMA1 issuer (lane 0 of warp 17): for every group, once its X rows landed and its D1 buffer
// was read by the consumers (two groups back), D1 = Xi X^T; loads the X rows one group ahead.
template <typename TS, int NP>
__device__ __forceinline__ void tc_issue_mma1(const Params &P, long long ubeg, long long uend, unsigned char *smem,
                                              TcBars &B, unsigned long long g0, unsigned long long seg0)
{
    using Sh = TcShape<TS, NP>;
    const long long N = P.N;
    const uint32_t tb = B.tmem;
    const TcDesc D = tc_descs<TS, NP>(smem);
    fence_proxy_async();
    GroupCursor<Sh::GR> gc, xc;   // group to compute, group whose X rows to load
    gc.begin(ubeg, uend, N);
    xc.begin(ubeg, uend, N);
    unsigned long long g = g0, gload = g0, seg = seg0;
    bool ok = true;
    auto load_x = [&]() {
        if (!ok || !xc.valid()) return;
        const int xb = (int)(gload & 1);
        // the buffer's previous group (two back) must have finished its MMA1
        if (gload >= g0 + 2) ok = mbar_wait(P, &B.d1full[xb], (uint32_t)(((gload >> 1) - 1) & 1));
        if (!ok) return;
        mbar_arrive_expect_tx(&B.xgfull[xb], (uint32_t)Sh::xg_bytes);
        bulk_load_hint(smem + Sh::off_xg + xb * Sh::xg_bytes, P.xr_tc + (size_t)(xc.r >> 3) * tc_xr_floats(NP),
                       (uint32_t)Sh::xg_bytes, &B.xgfull[xb], l2_evict_last());
        xc.advance(N);
        ++gload;
    };
    load_x();
    load_x();
    while (gc.valid() && ok) {
        const int b = (int)(g & 1);
        if (gc.r == gc.r0) ok = mbar_wait(P, &B.xifull, (uint32_t)(seg & 1));   // Xi of this segment
        if (ok) ok = mbar_wait(P, &B.xgfull[b], (uint32_t)((g >> 1) & 1));
        if (ok && g >= 2) ok = mbar_wait(P, &B.d1free[b], (uint32_t)(((g >> 1) - 1) & 1));
        if (ok) {
            tc_fence_after();
            tc_mma1<TS, NP>(tb, D, b, b, &B.d1full[b]);
        }
        load_x();
        const long long s_before = gc.s, u_before = gc.u;
        gc.advance(N);
        if (gc.valid() && (gc.s != s_before || gc.u != u_before)) ++seg;
        ++g;
    }
    umma_commit(&B.drain[0]);
    mbar_wait(P, &B.drain[0], B.drain_parity[0]);
    B.drain_parity[0] ^= 1u;
}

// MMA2 issuer (lane 0 of warp 18): for every stage, once all consumer warps stored their
// theta^T, D2 += Theta^T [X | 1]; releases the ring slot and the theta^T buffer by commits.
// D2 restarts at the first stage of every chunk (CH stages of a segment) in buffer
// chunk % ND2, once the consumers read that buffer's previous chunk.
template <typename TS, int NP>
__device__ __forceinline__ void tc_issue_mma2(const Params &P, long long ubeg, long long uend, unsigned char *smem,
                                              uint64_t *full, uint64_t *empty, TcBars &B, unsigned long long k0,
                                              unsigned long long kend, unsigned long long ch0)
{
    using Sh = TcShape<TS, NP>;
    constexpr int S = Sh::kStages;
    const long long N = P.N;
    const uint32_t tb = B.tmem;
    const TcDesc D = tc_descs<TS, NP>(smem);
    StageCursorT<Sh::RS> mc;
    mc.begin(ubeg, uend, N);
    RingPos<S> mpos;
    mpos.init(k0);
    unsigned long long ch = ch0;
    bool ok = true;
    for (unsigned long long k = k0; k < kend && ok; ++k) {
        const int slot = mpos.slot;
        const long long i = (mc.r - mc.r0) / Sh::RS;   // stage of the segment
        const bool cfirst = (i % Sh::CH) == 0;
        const bool clast = (i % Sh::CH) == Sh::CH - 1 || mc.r + Sh::RS >= mc.r1;
        const int b = (int)(k % Sh::NA2);
        const int db = (int)(ch % Sh::ND2);
        ok = mbar_wait(P, &full[slot], mpos.phase) && mbar_wait(P, &B.a2full[b], (uint32_t)((k / Sh::NA2) & 1));
        if (ok && cfirst && ch >= (unsigned long long)Sh::ND2)
            ok = mbar_wait(P, &B.d2free[db], (uint32_t)((ch / Sh::ND2 - 1) & 1));
        if (ok) {
            tc_fence_after();
            tc_mma2<TS, NP>(tb, D, slot, b, cfirst, db);
            umma_commit(&empty[slot]);
            umma_commit(&B.a2free[b]);
            if (clast) umma_commit(&B.d2done[db]);
        }
        if (clast) ++ch;
        mc.advance(N);
        mpos.next();
    }
    umma_commit(&B.drain[1]);
    mbar_wait(P, &B.drain[1], B.drain_parity[1]);
    B.drain_parity[1] ^= 1u;
}

// The pair pass of iteration l with the tensor-core products (same results contract as
// phase_pair: theta^(1)_l written over theta^(1)_{l-2}, row partials, column partials).
// Launched with kTcThreads threads: warps 0-15 consume stages, warp 16 leads.
// kstage / kseg count stages and segments across passes (barrier parities).
template <typename TS, int NP>
__device__ void phase_pair_tc(const Params &P, long long ell, unsigned char *smem, uint64_t *full, uint64_t *empty,
                              TcBars &B, unsigned long long &kstage, unsigned long long &kseg, unsigned long long &kgrp,
                              unsigned long long &kch, long long vc)
{
    using Sh = TcShape<TS, NP>;
    constexpr int S = Sh::kStages, N2 = Sh::N2;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wg = warp >> 2, q = warp & 3;
    const int m = q * 32 + lane;   // tensor-memory lane: columns 2m, 2m+1 of the stripe
    const int p = (int)(ell & 1), c = 1 - p;
    const long long N = P.N, ld = P.ld;
    const long long ubeg = unit_begin(P, vc);
    const long long uend = unit_begin(P, vc + 1);
    unsigned char *stage0 = smem + Sh::off_stage;
    const uint32_t tb = B.tmem;
    const uint32_t tq = tb + ((uint32_t)(32 * q) << 16);   // this warp's lane quarter

    unsigned long long nst = 0, nseg = 0, ngrp = 0, nch = 0;
    for (long long u = ubeg; u < uend;) {
        const long long s = u / N, r0 = u - s * N, r1 = min(N, r0 + (uend - u));
        const long long sst = (r1 - r0 + Sh::RS - 1) / Sh::RS;
        nst += (unsigned long long)sst;
        nch += (unsigned long long)((sst + Sh::CH - 1) / Sh::CH);
        ngrp += (unsigned long long)((r1 - r0 + Sh::GR - 1) / Sh::GR);
        ++nseg;
        u += r1 - r0;
    }
    const unsigned long long k0 = kstage, kend = kstage + nst;
    if (warp >= kTcWarps) {
        if (lane == 0 && nst > 0) {
            if (warp == kTcWarps)
                tc_producer<TS, NP>(P, ubeg, uend, c, p, smem, full, empty, B, k0, kend, kgrp);
            else if (warp == kTcWarps + 1)
                tc_issue_mma1<TS, NP>(P, ubeg, uend, smem, B, kgrp, kseg);
            else
                tc_issue_mma2<TS, NP>(P, ubeg, uend, smem, full, empty, B, k0, kend, kch);
        }
        __syncwarp();
    } else {
        const float beta = (float)__ldcg(&P.st->scal[p].beta);
        const float invL = P.invL;
        const float scl = P.st_scale, iscl = P.st_inv_scale;
        const f2 beta2 = f2_make(beta, beta), ninvL2 = f2_make(-invL, -invL), iscl2 = f2_make(iscl, iscl);
        const f2 scl2 = f2_make(scl, scl);
        // FP16 row sums and D2 come out scaled by 2^e (tc_rows): unscaled where they are stored
        const float osc = std::is_same<TS, __half>::value ? iscl : 1.0f;
        const bool sr = P.sr != 0;
        const uint32_t rseed = P.seed ^ (uint32_t)ell * 0x632BE5ABu;
        TS *__restrict__ nxt = (TS *)P.theta[p];
        const long long first_stripe = ubeg / N;
        constexpr int RS = Sh::RS, RPW = Sh::RPW;
        const int rb = RPW * wg;   // first stage row of this warp
        RingPos<S> cpos;
        cpos.init(k0);
        unsigned long long k = k0, seg = kseg, gj = kgrp, ch = kch;
        bool ok = true;
        // this warpgroup's share of D2: columns [h0, h0 + H2) of the even (eo = 0) or odd block
        constexpr int H2 = Sh::H2;
        const int eo = wg >> 1, h0 = (wg & 1) * H2;
        float d2acc[H2];
        bool pending = false;          // a D2 chunk whose MMAs were issued and that is not added yet
        unsigned long long pch = 0;
        // adds D2 chunk cc to d2acc (round to nearest) and hands its buffer back to the MMA2 issuer
        auto flush_d2 = [&](unsigned long long cc) {
            const int db = (int)(cc % Sh::ND2);
            if (ok) ok = mbar_wait(P, &B.d2done[db], (uint32_t)((cc / Sh::ND2) & 1));
            ok = __all_sync(0xffffffffu, ok);
            if (ok) {
                tc_fence_after();
#pragma unroll
                for (int j = 0; j < H2; j += 8) {
                    float v[8];
                    tmem_ld8(tq + Sh::COL_D2 + 2 * N2 * db + N2 * eo + h0 + j, v);
                    tmem_wait_ld();
#pragma unroll
                    for (int t = 0; t < 8; ++t) d2acc[j + t] += v[t];
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&B.d2free[db]);
        };
        for (long long u = ubeg; u < uend;) {
            const long long s = u / N, r0 = u - s * N, r1 = min(N, r0 + (uend - u));
            const long long col0 = s * kW + 2 * m;
            const bool va = col0 < N, vb = col0 + 1 < N;
            const f2 ccol = f2_make(va ? __ldcg(P.ccol2 + col0) : 0.0f, vb ? __ldcg(P.ccol2 + col0 + 1) : 0.0f);
            const uint32_t hcol = hash_col((uint32_t)(col0 >> 1), rseed);
            const bool ragged = (s * kW + kW) > N;
            float *rp = P.rowpart + s;   // one partial per (stripe, row), stored by warp q = 0
#pragma unroll
            for (int j = 0; j < H2; ++j) d2acc[j] = 0.0f;
            for (long long r = r0; r < r1; r += RS, ++k, cpos.next()) {
                const int slot = cpos.slot;
                const int b = (int)(k % Sh::NA2);   // theta^T buffer of this stage
                const int go = (int)((r - r0) % Sh::GR);       // row offset inside the MMA1 group
                const bool glast = go + RS == Sh::GR || r + RS >= r1;
                const int b1 = (int)(gj & 1);
                // --- residual dot products from tensor memory (MMA1 of the group) ---
                if (ok) ok = mbar_wait(P, &full[slot], cpos.phase);
                if (ok && go == 0) ok = mbar_wait(P, &B.d1full[b1], (uint32_t)((gj >> 1) & 1));
                ok = __all_sync(0xffffffffu, ok);   // tensor-memory loads and stores are warp-collective
                float de[RPW], dd[RPW];
                if (ok) {
                    tc_fence_after();
                    tmem_ldv(tq + Sh::COL_D1 + 2 * Sh::GR * b1 + go + rb, de);
                    tmem_ldv(tq + Sh::COL_D1 + 2 * Sh::GR * b1 + Sh::GR + go + rb, dd);
                    tmem_wait_ld();
                }
                if (glast) {
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&B.d1free[b1]);
                    ++gj;
                }
                if (ok && k >= (unsigned long long)Sh::NA2)
                    ok = mbar_wait(P, &B.a2free[b], (uint32_t)(((k / Sh::NA2) - 1) & 1));
                ok = __all_sync(0xffffffffu, ok);
                // --- element-wise Step 2 on 4 rows x 2 columns ---
                float ae[RPW], ao[RPW], le[RPW], lo[RPW], rs[RPW];
                if (ok) {
                    const unsigned char *st = stage0 + slot * Sh::stage_bytes;
                    const TS *tcur = reinterpret_cast<const TS *>(st);
                    const TS *tprv = reinterpret_cast<const TS *>(st + Sh::tile_bytes);
                    const float *rec = reinterpret_cast<const float *>(st + Sh::off_rec);
                    TS *nrow = nxt + (r + rb) * ld + col0;
                    const bool fast = !ragged && (r + RS <= r1) && !(r < s * kW + kW && s * kW < r + RS);
                    if (sr) {
                        if (fast)
                            tc_rows<TS, NP, true, false>(tcur, tprv, rec, rb, m, r, r1, col0, va, vb, ccol, de, dd,
                                                         beta2, ninvL2, invL, hcol, scl, iscl, iscl2, scl2, nrow, ld, ae, ao,
                                                         le, lo, rs);
                        else
                            tc_rows<TS, NP, true, true>(tcur, tprv, rec, rb, m, r, r1, col0, va, vb, ccol, de, dd,
                                                        beta2, ninvL2, invL, hcol, scl, iscl, iscl2, scl2, nrow, ld, ae, ao,
                                                        le, lo, rs);
                    } else {
                        if (fast)
                            tc_rows<TS, NP, false, false>(tcur, tprv, rec, rb, m, r, r1, col0, va, vb, ccol, de, dd,
                                                          beta2, ninvL2, invL, hcol, scl, iscl, iscl2, scl2, nrow, ld, ae,
                                                          ao, le, lo, rs);
                        else
                            tc_rows<TS, NP, false, true>(tcur, tprv, rec, rb, m, r, r1, col0, va, vb, ccol, de, dd,
                                                         beta2, ninvL2, invL, hcol, scl, iscl, iscl2, scl2, nrow, ld, ae, ao,
                                                         le, lo, rs);
                    }
                    // theta^T for MMA2 (column k of A = stage row)
                    const uint32_t a2 = tq + Sh::COL_A2 + Sh::A2W * b + rb;
                    tmem_stv(a2, ae);
                    tmem_stv(a2 + RS, ao);
                    if (Sh::SPLIT) {
                        tmem_stv(a2 + 2 * RS, le);
                        tmem_stv(a2 + 3 * RS, lo);
                    }
                    tmem_wait_st();
                } else {
#pragma unroll
                    for (int i = 0; i < RPW; ++i) rs[i] = 0.0f;
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(&B.a2full[b]);
                    mbar_arrive(&empty[slot]);
                }
                tc_flush_rows(rs, r + rb, ok ? r1 : r, rp, P.Q, lane, &B.rowx[wg][k & 1][0][0], q, wg, osc);
                // the previous D2 chunk (its MMAs had a stage to finish), then mark this one
                if (pending) {
                    flush_d2(pch);
                    pending = false;
                }
                const long long si = (r - r0) / RS;
                if ((si % Sh::CH) == Sh::CH - 1 || r + RS >= r1) {
                    pch = ch++;
                    pending = true;
                }
            }
            // --- segment end: the last chunk, then this warpgroup's share of the column partials
            // (D2 column j < n: (Theta^T X)_j, j = n: the column sums; n < j <= NP written as 0) ---
            if (pending) {
                flush_d2(pch);
                pending = false;
            }
            if (ok) {
                const int slotc = (int)(s - first_stripe);
                float *cp = P.colpart + ((vc * P.slots + slotc) * P.cgroups * (NP + 1)) * kW + 2 * m + eo;
                const int n = P.n;
                const uint64_t keep = l2_evict_last();
#pragma unroll
                for (int j = 0; j < H2; ++j) {
                    const int kk = h0 + j;
                    if (kk == n) st_keep(cp, d2acc[j] * osc, keep);
                    else if (kk < NP) st_keep(cp + (1 + kk) * kW, kk < n ? d2acc[j] * osc : 0.0f, keep);
                }
            }
            u += r1 - r0;
            ++seg;
        }
    }
    kstage = kend;
    kseg += nseg;
    kgrp += ngrp;
    kch += nch;
    __syncthreads();
}

}  // namespace crk
