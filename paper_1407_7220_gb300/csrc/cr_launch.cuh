// cr_launch.cuh -- __global__ entry points (persistent driver and per-phase kernels)
// and the table the host uses to reach them for a given (theta dtype, padded n).
#pragma once

#include "cr_kernels.cuh"
#include "cr_backward.cuh"
#include "cr_blocks.cuh"
#include "cr_pair_f64.cuh"
#include "cr_pair_tc.cuh"

namespace crk {

enum Phase : int {
    PH_FOLDB = 0, PH_PAIR = 1, PH_FOLDA = 2, PH_KKT32 = 3, PH_KKT64 = 4, PH_DECIDE32 = 5, PH_DECIDE64 = 6,
    PH_BALL_NORM = 7, PH_BALL_SCALE = 8   // finite B_theta: norm of the clamped iterate, radial scaling
};

// Dynamic shared memory of the pair pass (the larger of the CUDA-core and tensor-core layouts;
// the FP64 pass stages nothing in shared memory).
template <typename TS, int NP> constexpr size_t pair_smem_bytes()
{
    if constexpr (std::is_same<TS, double>::value) {
        return f64_smem_bytes<NP>();
    } else {
        return PairSmem<TS, NP>::bytes > TcShape<TS, NP>::bytes ? PairSmem<TS, NP>::bytes : TcShape<TS, NP>::bytes;
    }
}

// 128-byte aligned base of the dynamic shared memory (TMA destinations).
__device__ __forceinline__ unsigned char *aligned_smem(unsigned char *raw)
{
    const uint32_t a = smem_u32(raw);
    return raw + ((128u - (a & 127u)) & 127u);
}

__device__ __forceinline__ void init_pipeline(uint64_t *full, uint64_t *empty)
{
    if (threadIdx.x == 0) {
        for (int i = 0; i < kMaxStages; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], kCons / 32);
        }
        fence_mbar_init();
    }
    __syncthreads();
}

// Persistent driver: iterations ell0..ell1 in one cooperative launch (CUDA-core pair pass).  Phases are
// separated by bounded grid barriers; every CTA takes the same decisions from the
// same reduced values.  check_every > 0 enables the convergence test (FP32 screen,
// FP64 confirmation) every check_every iterations and at ell1.
template <typename TS, int NP>
__device__ __forceinline__ void persistent_body(const Params &P, long long ell0, long long ell1, int check_every,
                                                double tol, double sigma, int first_foldB, unsigned char *sm,
                                                double *red, double *s_m, uint64_t *full, uint64_t *empty)
{
    unsigned long long bar = 0, kstage = 0;
    if (first_foldB) {   // 0 when the previous foldA already performed it (P.fuse)
        phase_foldB<NP>(P, ell0, red, blockIdx.x);
        if (!grid_barrier(P, bar)) return;
    }
    for (long long ell = ell0; ell <= ell1; ++ell) {
        phase_pair<TS, NP>(P, ell, sm, full, empty, kstage, blockIdx.x);
        if (!grid_barrier(P, bar)) return;
        const bool check = check_every > 0 && ((ell % check_every) == 0 || ell == ell1);
        phase_foldA<NP>(P, ell, red, blockIdx.x, !P.fuse || check || ell == ell1);
        if (!grid_barrier(P, bar)) return;
        if (check) {
            phase_kkt<TS, NP, false>(P, ell, red, blockIdx.x);
            if (!grid_barrier(P, bar)) return;
            if (threadIdx.x < 32) {
                double m[5];
                reduce_kkt(P, sigma, m);
                if (threadIdx.x == 0) {
                    for (int i = 0; i < 5; ++i) s_m[i] = m[i];
                    s_m[5] = m[0];
                }
            }
            __syncthreads();
            bool stop = s_m[0] <= tol;
            const double screen = s_m[5];
            if (stop) {
                phase_kkt<TS, NP, true>(P, ell, red, blockIdx.x);
                if (!grid_barrier(P, bar)) return;
                if (threadIdx.x < 32) {
                    double m[5];
                    reduce_kkt(P, sigma, m);
                    if (threadIdx.x == 0)
                        for (int i = 0; i < 5; ++i) s_m[i] = m[i];
                }
                __syncthreads();
                stop = s_m[0] <= tol;
            }
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                for (int i = 0; i < 5; ++i) P.st->kkt[i] = s_m[i];
                P.st->kkt[5] = screen;
                if (stop) {
                    P.st->converged = 1;
                    P.st->iters_done = ell;
                }
            }
            if (stop) return;
        }
        if (ell < ell1 && !P.fuse) {
            phase_foldB<NP>(P, ell + 1, red, blockIdx.x);
            if (!grid_barrier(P, bar)) return;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) P.st->iters_done = ell1;
}

template <typename TS, int NP>
__global__ void __launch_bounds__(kThreads, 1)
k_persistent(const __grid_constant__ Params P, long long ell0, long long ell1, int check_every, double tol,
             double sigma, int first_foldB)
{
    extern __shared__ unsigned char sm_raw[];
    unsigned char *sm = aligned_smem(sm_raw);
    __shared__ double red[72];
    __shared__ double s_m[8];
    __shared__ __align__(8) uint64_t full[kMaxStages], empty[kMaxStages];
    init_pipeline(full, empty);
    persistent_body<TS, NP>(P, ell0, ell1, check_every, tol, sigma, first_foldB, sm, red, s_m, full, empty);
}

// One phase of one iteration (the CR_DRIVER_PHASES path and the stand-alone metric
// calls).  Every kernel is a no-op once the state says converged or failed.
// Launched as a programmatic dependent of the previous phase: its CTAs may be placed while the
// previous grid drains, and griddepcontrol.wait (before any access to the state) holds them
// until that grid has completed and its writes are visible; the next phase may then be
// launched early in turn.  Without a programmatic launch both instructions are no-ops.
template <typename TS, int NP>
__global__ void __launch_bounds__(kThreads, 1)
k_phase(const __grid_constant__ Params P, int phase, long long ell, double tol, double sigma)
{
    extern __shared__ unsigned char sm_raw[];
    __shared__ double red[72];
    __shared__ __align__(8) uint64_t full[kMaxStages], empty[kMaxStages];
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int conv = __ldcg(&P.st->converged), err = __ldcg(&P.st->error);
    if (err != 0) return;
    if (conv != 0 && phase != PH_KKT64 && phase != PH_DECIDE64) return;
    switch (phase) {
    case PH_FOLDB: phase_foldB<NP>(P, ell, red, blockIdx.x); break;
    case PH_PAIR: {
        unsigned long long kstage = 0;
        init_pipeline(full, empty);
        phase_pair<TS, NP>(P, ell, aligned_smem(sm_raw), full, empty, kstage, blockIdx.x);
        break;
    }
    case PH_FOLDA: phase_foldA<NP>(P, ell, red, blockIdx.x, P.fold_stats != 0); break;
    case PH_BALL_NORM: phase_ball_norm<TS, NP>(P, ell, red, blockIdx.x); break;
    case PH_BALL_SCALE: phase_ball_scale<TS>(P, ell, blockIdx.x); break;
    case PH_KKT32: phase_kkt<TS, NP, false>(P, ell, red, blockIdx.x); break;
    case PH_KKT64: phase_kkt<TS, NP, true>(P, ell, red, blockIdx.x); break;
    case PH_DECIDE32:
    case PH_DECIDE64:
        // single CTA: reduce the KKT partials; tol < 0 only records the metrics
        if (blockIdx.x == 0 && threadIdx.x < 32) {
            double m[5];
            reduce_kkt(P, sigma, m);
            if (threadIdx.x == 0) {
                if (phase == PH_DECIDE32) {
                    P.st->kkt[5] = m[0];
                    // the FP64 pass that follows runs only if the screen passed
                    P.st->kkt[6] = (tol >= 0.0 && m[0] <= tol) ? 1.0 : 0.0;
                } else {
                    for (int i = 0; i < 5; ++i) P.st->kkt[i] = m[i];
                    if (tol >= 0.0 && m[0] <= tol) {
                        P.st->converged = 1;
                        P.st->iters_done = ell;
                    }
                }
            }
        }
        break;
    }
}

// KKT64 pass that runs only if the preceding FP32 screen passed (phase path).
template <typename TS, int NP>
__global__ void __launch_bounds__(kThreads, 1)
k_kkt64_if_screened(const __grid_constant__ Params P, long long ell)
{
    __shared__ double red[72];
    if (__ldcg(&P.st->error) != 0 || __ldcg(&P.st->kkt[6]) == 0.0) return;
    phase_kkt<TS, NP, true>(P, ell, red, blockIdx.x);
}

// ---------------------------------------------------------------------------
// Batched persistent driver: many independent instances (one Params each, in
// device memory) advance together in one cooperative launch.  Physical CTA b
// owns the work items off[b]..off[b+1]-1; item j is virtual CTA item_vc[j] of
// instance item_inst[j].  The phases and their order are those of k_persistent;
// instances whose KKT test passed leave the work (active[i] = 0).  The first
// iteration index is read from *ell_base, which the launch advances, so the same
// launch can be replayed (CUDA graph) chunk after chunk.
// ---------------------------------------------------------------------------
struct BatchArgs {
    const Params *inst;
    const int *item_inst;
    const int *item_vc;
    const int *off;
    int *active;
    long long *ell_base;
    unsigned long long *bar_count;
    int *error;
    unsigned long long bar_timeout_ns;
    int Gphys;
    int B;
};

template <typename TS, int NP, int RS = kRS>
__global__ void __launch_bounds__(kThreads, 1)
k_batch(const __grid_constant__ BatchArgs A, long long chunk, int check_every, double tol)
{
    extern __shared__ unsigned char sm_raw[];
    unsigned char *sm = aligned_smem(sm_raw);
    __shared__ double red[72];
    __shared__ int s_flag;
    __shared__ __align__(8) uint64_t full[kMaxStages], empty[kMaxStages];
    unsigned long long bar = 0, kstage = 0;
    init_pipeline(full, empty);
    const int j0 = A.off[blockIdx.x], j1 = A.off[blockIdx.x + 1];
    const long long ell0 = __ldcg(A.ell_base) + 1, ell1 = ell0 + chunk - 1;
#define CR_BAR()                                                                                                \
    if (!bounded_grid_barrier(A.bar_count, A.error, (unsigned long long)A.Gphys, 0ull, A.bar_timeout_ns, bar)) \
        return;
#define CR_ITEMS(...)                                           \
    for (int j = j0; j < j1; ++j) {                             \
        const int i = A.item_inst[j];                           \
        const long long vc = A.item_vc[j];                      \
        if (__ldcg(A.active + i) == 0) continue;                \
        const Params &P = A.inst[i];                            \
        __VA_ARGS__;                                            \
    }

    CR_ITEMS(phase_foldB<NP>(P, ell0, red, vc));
    CR_BAR();
    for (long long ell = ell0; ell <= ell1; ++ell) {
        CR_ITEMS((phase_pair<TS, NP, PM_PAPG, RS>(P, ell, sm, full, empty, kstage, vc)));
        CR_BAR();
        CR_ITEMS(phase_foldA<NP>(P, ell, red, vc));
        CR_BAR();
        if (check_every > 0 && ((ell % check_every) == 0 || ell == ell1)) {
            CR_ITEMS(phase_kkt<TS, NP, false>(P, ell, red, vc));
            CR_BAR();
            // screen decision per instance (owner = the CTA with its virtual CTA 0)
            CR_ITEMS(if (vc == 0) {
                if (threadIdx.x < 32) {
                    double m[5];
                    reduce_kkt(P, P.sigma, m);
                    if (threadIdx.x == 0) {
                        P.st->kkt[5] = m[0];
                        P.st->kkt[6] = m[0] <= tol ? 1.0 : 0.0;
                    }
                }
                __syncthreads();
            });
            CR_BAR();
            CR_ITEMS(if (__ldcg(&P.st->kkt[6]) != 0.0) phase_kkt<TS, NP, true>(P, ell, red, vc));
            CR_BAR();
            CR_ITEMS(if (vc == 0 && __ldcg(&P.st->kkt[6]) != 0.0) {
                if (threadIdx.x < 32) {
                    double m[5];
                    reduce_kkt(P, P.sigma, m);
                    if (threadIdx.x == 0) {
                        for (int q = 0; q < 5; ++q) P.st->kkt[q] = m[q];
                        if (m[0] <= tol) {
                            P.st->converged = 1;
                            P.st->iters_done = ell;
                            A.active[i] = 0;
                        }
                    }
                }
                __syncthreads();
            });
            CR_BAR();
        }
        if (ell < ell1) {
            CR_ITEMS(phase_foldB<NP>(P, ell + 1, red, vc));
            CR_BAR();
        }
    }
    // record the iterations of the instances still running, then advance the base
    CR_ITEMS(if (vc == 0 && threadIdx.x == 0) P.st->iters_done = ell1);
    (void)s_flag;
    if (blockIdx.x == 0 && threadIdx.x == 0) *A.ell_base = ell1;
#undef CR_ITEMS
#undef CR_BAR
}

// The pair pass with its products on the tensor cores (phase driver): 16 consumer warps
// plus one leader warp.  No-op once the state says converged or failed.
template <typename TS, int NP>
__global__ void __launch_bounds__(kTcThreads, 1) k_pair_tc(const __grid_constant__ Params P, long long ell)
{
    extern __shared__ unsigned char sm_raw[];
    __shared__ __align__(8) uint64_t full[kMaxStages], empty[kMaxStages];
    __shared__ __align__(8) TcBars tcb;
    __shared__ int s_skip;
    if (threadIdx.x == 0) s_skip = (__ldcg(&P.st->error) != 0 || __ldcg(&P.st->converged) != 0) ? 1 : 0;
    __syncthreads();
    if (s_skip) return;   // block-uniform
    unsigned long long kstage = 0, kseg = 0, kgrp = 0, kch = 0;
    tc_init_pipeline(full, empty);
    tc_init_bars(tcb);
    tc_alloc<TS, NP>(tcb);   // includes a block barrier
    phase_pair_tc<TS, NP>(P, ell, aligned_smem(sm_raw), full, empty, tcb, kstage, kseg, kgrp, kch, blockIdx.x);
    tc_free<TS, NP>(tcb);
}

struct KernelSet {
    const void *persistent;
    const void *phase;
    const void *pair_tc;
    const void *kkt64_if;
    const void *batch;
    const void *batch8;                            // the batched launch with 8-row stages
    size_t smem, smem_batch8;
    int NP;
    BwdKernels bwd;
    const void *blocks_prepare, *blocks_records;   // K-block P-APG (FP64 multipliers only)
};

// dLoss/dybar = ubar + accumulated, dLoss/dX = accumulated (FP64 -> FP32 outputs)
__global__ void k_bwd_finish(long long N, int n, const float *ubar, const double *ybar_acc, const double *X_acc,
                             float *dybar, float *dX);

template <typename TS, int NP> KernelSet make_set()
{
    KernelSet k;
    k.persistent = (const void *)k_persistent<TS, NP>;
    k.phase = (const void *)k_phase<TS, NP>;
    k.kkt64_if = (const void *)k_kkt64_if_screened<TS, NP>;
    if constexpr (std::is_same<TS, double>::value) {
        k.pair_tc = nullptr;   // FP64 multipliers: CUDA cores only, single instances only
        k.batch = nullptr;
        k.batch8 = nullptr;
        k.blocks_prepare = (const void *)k_blocks_prepare<NP>;
        k.blocks_records = (const void *)k_blocks_records<NP>;
    } else {
        k.pair_tc = (const void *)k_pair_tc<TS, NP>;
        k.batch = (const void *)k_batch<TS, NP>;
        k.batch8 = (const void *)k_batch<TS, NP, 8>;
        k.blocks_prepare = nullptr;
        k.blocks_records = nullptr;
    }
    k.smem = pair_smem_bytes<TS, NP>();
    k.smem_batch8 = PairSmem<TS, NP, 2, 8>::bytes;
    k.NP = NP;
    k.bwd = make_bwd<TS, NP>();
    return k;
}

// padded n values compiled: n -> smallest NP >= n in this list
#define CR_NP_LIST(X) X(2) X(4) X(5) X(8) X(10) X(16) X(20) X(32)
constexpr int kMaxN = 32;

// padded n values compiled for FP64 multipliers (n <= 10: its per-lane FP64 accumulators)
#define CR_NP_LIST_F64(X) X(2) X(4) X(5) X(8) X(10)
constexpr int kMaxNF64 = 10;

KernelSet kernels_f32(int NP);
KernelSet kernels_bf16(int NP);
KernelSet kernels_f16(int NP);
KernelSet kernels_f64(int NP);

}  // namespace crk
