// cr_alcc.cuh -- ALCC with the MAPG inner solver (Sec. II-D, Fig. `fig:alcc` and the MAPG
// figure) on the full problem (regularize): every pairwise constraint in one block, the
// multipliers theta_k an N x N array (theta[0]).
//
// One cooperative launch runs a bounded range of MAPG iterations of outer iteration k and, once
// MAPG returns, the outer step: theta_{k+1} = (mu_k / mu_{k+1}) (A_1 y_k + A_2 xi_k - theta_k)_-
// (Fig. `fig:alcc` step 4) and the KKT residual of (regularize) at (y_k, xi_k) with the multiplier
// estimate lambda = mu_{k+1} theta_{k+1}.  The host keeps the schedule of mu, tau and the alphas
// (steps 1-2, 5-6) and passes the constants of outer iteration k in AlccStep.
//
// A MAPG iteration is three phases separated by grid barriers:
//   grad  pair pass: m = (A_1 y^(2) + A_2 xi^(2) - theta_k)_- per pair, nothing stored, its adjoint
//         A_1^T m, A_2^T m accumulated as in the P-APG pass (one multiplier read per pair);
//   fold1 per row: the gradient step of MAPG steps 1-2 before projection, and the squared
//         distances to the ball centres;
//   fold2 per row: the projections on Q_y and Q_xi, the momentum of steps 4-5 and the column data
//         of the next pair pass; the squared step lengths of step 6.
// Every CTA then takes the stopping decision of steps 6-9 from the same reduced values.
#pragma once

#include "cr_launch.cuh"

namespace crk {

struct AlccStep {
    double inv_mu, gamma_inv_mu;   // 1/mu_k, gamma/mu_k
    double mu_next;                // mu_{k+1} = c mu_k
    double inv_Ly, inv_Lxi;        // 1/L^y_k, 1/L^xi_k (Fig. `fig:alcc` step 1)
    double By, Bxi;                // radii of Q_y (centre ybar) and Q_xi (centre 0)
    double alpha_y, alpha_xi;      // MAPG stopping thresholds
    double res_rel;                // the thresholds are at least res_rel ||y^(1)|| and res_rel ||xi^(1)|| (0: off)
    double t0;                     // t of the MAPG figure before iteration ell0
    long long lmax;                // ell^max_k (Fig. `fig:alcc` step 2)
    long long ell0, ell1;          // MAPG iterations of this launch (ell1 <= lmax)
    float a;                       // mu_k / mu_{k+1}
};

// fold1 of MAPG iteration ell: unprojected steps of MAPG steps 1-2 into slot ell & 1.
//   grad_y P_k  = (y - ybar)/mu_k - A_1^T m,    (A_1^T m)_l = R_l - Cc_l
//   grad_xi P_k = gamma xi/mu_k - A_2^T m,      (A_2^T m)_l = Cc_l x_l - (m^T X)_l
template <int NP>
__device__ void phase_mapg_grad(const Params &P, const AlccStep &S, long long ell, double *red, long long vc)
{
    const int q = (int)(ell & 1);
    const long long N = P.N;
    const int n = P.n;
    double sy = 0.0, sx = 0.0;
    for (RowIter it(P, vc); it.more(); it.next()) {
        const long long l = it.row();
        if (l >= N) continue;
        double R, Cc, TX[NP];
        gather_adjoint<NP>(P, l, R, Cc, TX);
        const double yb = __ldg(P.h + l);
        const double y2 = __ldcg(P.ay2 + l);
        const double gy = (y2 - yb) * S.inv_mu - (R - Cc);
        const double yr = y2 - gy * S.inv_Ly;
        P.ay[q][l] = yr;
        sy += (yr - yb) * (yr - yb);
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            if (k < n) {
                const double xk = __ldg(P.X64 + l * n + k);
                const double x2 = __ldcg(P.axi2 + l * n + k);
                const double gx = x2 * S.gamma_inv_mu - (Cc * xk - TX[k]);
                const double xr = x2 - gx * S.inv_Lxi;
                P.axi[q][l * n + k] = xr;
                sx += xr * xr;
            }
        }
    }
    double vals[2] = {sy, sx};
    const bool ismax[2] = {false, false};
    block_reduce<2>(vals, ismax, red);
    if (threadIdx.x == 0) {
        P.foldpart[vc * 8 + 0] = vals[0];
        P.foldpart[vc * 8 + 1] = vals[1];
    }
}

// Sum of foldpart component i over the CTAs in a fixed order (warp 0; result in lane 0).
__device__ __forceinline__ double sum_part(const Params &P, int i)
{
    double a = 0.0;
    for (int c = threadIdx.x; c < P.G; c += 32) a += __ldcg(P.foldpart + c * 8 + i);
    return warp_sum(a);
}

// fold2 of MAPG iteration ell: projections (steps 1-2), momentum with weight w (steps 4-5),
// column data of (y, xi)^(2)_{ell+1} for the next pair pass, squared step lengths (step 6) and
// squared norms of (y, xi)^(1)_ell.
template <int NP>
__device__ void phase_mapg_step(const Params &P, const AlccStep &S, long long ell, double w, double *red,
                                long long vc)
{
    const int q = (int)(ell & 1), qp = q ^ 1;
    __shared__ double s_f[2];
    if (threadIdx.x < 32) {
        const double sy = sum_part(P, 0), sx = sum_part(P, 1);
        if (threadIdx.x == 0) {
            const double ny = sqrt(sy), nx = sqrt(sx);
            s_f[0] = ny > S.By ? S.By / ny : 1.0;
            s_f[1] = nx > S.Bxi ? S.Bxi / nx : 1.0;
        }
    }
    __syncthreads();
    const double fy = s_f[0], fx = s_f[1];
    const long long N = P.N;
    const int n = P.n;
    constexpr int REC = RecLayout<NP>::REC;
    double dy = 0.0, dx = 0.0, ny = 0.0, nx = 0.0;
    for (RowIter it(P, vc); it.more(); it.next()) {
        const long long l = it.row();
        if (l >= N) continue;
        const double yb = __ldg(P.h + l), yr = __ldcg(P.ay[q] + l);
        const double y1 = fy == 1.0 ? yr : yb + fy * (yr - yb);
        P.ay[q][l] = y1;
        const double y2 = __ldcg(P.ay2 + l);
        dy += (y1 - y2) * (y1 - y2);
        ny += y1 * y1;
        const double y2n = y1 + w * (y1 - __ldcg(P.ay[qp] + l));
        P.ay2[l] = y2n;
        double d = 0.0;
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            float xf = 0.0f;
            if (k < n) {
                const double xr = __ldcg(P.axi[q] + l * n + k);
                const double x1 = fx == 1.0 ? xr : fx * xr;
                P.axi[q][l * n + k] = x1;
                const double x2 = __ldcg(P.axi2 + l * n + k);
                dx += (x1 - x2) * (x1 - x2);
                nx += x1 * x1;
                const double x2n = x1 + w * (x1 - __ldcg(P.axi[qp] + l * n + k));
                P.axi2[l * n + k] = x2n;
                d += x2n * __ldg(P.X64 + l * n + k);
                xf = (float)x2n;
            }
            P.xi2[l * NP + k] = xf;
        }
        P.rowrec[l * REC] = (float)y2n;
        P.ccol2[l] = (float)(d - y2n);
        P.ccol2_64[l] = d - y2n;
        if (!isfinite(y2n) || !isfinite(d)) atomicCAS(&P.st->error, 0, ERR_NUMERIC);
    }
    double vals[4] = {dy, dx, ny, nx};
    const bool ismax[4] = {false, false, false, false};
    block_reduce<4>(vals, ismax, red);
    if (threadIdx.x == 0) {
        P.foldpart[vc * 8 + 2] = vals[0];
        P.foldpart[vc * 8 + 3] = vals[1];
        P.foldpart[vc * 8 + 6] = vals[2];
        P.foldpart[vc * 8 + 7] = vals[3];
    }
}

// MAPG steps 6-9: the same decision in every CTA.  The thresholds are taken no smaller than
// res_rel times the norms of y and xi: a shorter step cannot change the next gradient, whose
// active terms the pair pass evaluates from the FP64 point.
__device__ __forceinline__ bool mapg_returns(const Params &P, const AlccStep &S, long long ell, int *s_flag)
{
    if (threadIdx.x < 32) {
        const double dy = sum_part(P, 2), dx = sum_part(P, 3), ny = sum_part(P, 6), nx = sum_part(P, 7);
        if (threadIdx.x == 0) {
            const double ay = fmax(S.alpha_y, S.res_rel * sqrt(ny)), ax = fmax(S.alpha_xi, S.res_rel * sqrt(nx));
            *s_flag = ((sqrt(dy) <= ay && sqrt(dx) <= ax) || ell >= S.lmax) ? 1 : 0;
        }
    }
    __syncthreads();
    const bool r = *s_flag != 0;
    __syncthreads();
    return r;
}

// (y_k, xi_k) = (y, xi)^(1) of the returning iteration (slot q): kept in y1 / xi1_64, made the
// start (y, xi)^(1)_0 = (y, xi)^(2)_1 of the next MAPG call, and written as the column data the
// outer-step pass and the next gradient pass read.
template <int NP>
__device__ void phase_alcc_take(const Params &P, int q, long long vc)
{
    const long long N = P.N;
    const int n = P.n;
    constexpr int REC = RecLayout<NP>::REC;
    for (RowIter it(P, vc); it.more(); it.next()) {
        const long long l = it.row();
        if (l >= N) continue;
        const double y = __ldcg(P.ay[q] + l);
        P.y1[l] = y;
        P.ay[0][l] = y;
        P.ay2[l] = y;
        double d = 0.0;
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            float xf = 0.0f;
            if (k < n) {
                const double xi = __ldcg(P.axi[q] + l * n + k);
                P.xi1_64[l * n + k] = xi;
                P.axi[0][l * n + k] = xi;
                P.axi2[l * n + k] = xi;
                d += xi * __ldg(P.X64 + l * n + k);
                xf = (float)xi;
            }
            P.xi2[l * NP + k] = xf;
        }
        P.rowrec[l * REC] = (float)y;
        P.ccol2[l] = (float)(d - y);
        P.ccol2_64[l] = d - y;
    }
}

// Stationarity of (regularize) with lambda = mu_{k+1} theta_{k+1}: max |y - ybar - A_1^T lambda| and
// max |gamma xi - A_2^T lambda| from the adjoint partials of the outer-step pass.
template <int NP>
__device__ void phase_alcc_stat(const Params &P, const AlccStep &S, double *red, long long vc)
{
    const long long N = P.N;
    const int n = P.n;
    double ry = 0.0, rx = 0.0;
    for (RowIter it(P, vc); it.more(); it.next()) {
        const long long l = it.row();
        if (l >= N) continue;
        double R, Cc, TX[NP];
        gather_adjoint<NP>(P, l, R, Cc, TX);
        ry = fmax(ry, fabs(__ldcg(P.y1 + l) - __ldg(P.h + l) - S.mu_next * (R - Cc)));
#pragma unroll
        for (int k = 0; k < NP; ++k)
            if (k < n) {
                const double a2 = Cc * __ldg(P.X64 + l * n + k) - TX[k];
                rx = fmax(rx, fabs(P.gamma * __ldcg(P.xi1_64 + l * n + k) - S.mu_next * a2));
            }
    }
    double vals[2] = {ry, rx};
    const bool ismax[2] = {true, true};
    block_reduce<2>(vals, ismax, red);
    if (threadIdx.x == 0) {
        P.foldpart[vc * 8 + 4] = vals[0];
        P.foldpart[vc * 8 + 5] = vals[1];
    }
}

// The phases of k_alcc as separate functions: each gets its own register allocation instead of
// one allocation for the whole kernel (which spilled).
template <typename TS, int NP, int MODE>
__device__ __noinline__ void alcc_pair_pass(const Params &P, long long ell, unsigned char *sm, uint64_t *full,
                                            uint64_t *empty, unsigned long long &kstage, long long vc, float a)
{
    phase_pair<TS, NP, MODE>(P, ell, sm, full, empty, kstage, vc, a);
}
template <int NP>
__device__ __noinline__ void alcc_grad_fold(const Params &P, const AlccStep &S, long long ell, double *red, long long vc)
{
    phase_mapg_grad<NP>(P, S, ell, red, vc);
}
template <int NP>
__device__ __noinline__ void alcc_step_fold(const Params &P, const AlccStep &S, long long ell, double w, double *red,
                                            long long vc)
{
    phase_mapg_step<NP>(P, S, ell, w, red, vc);
}
template <typename TS, int NP>
__device__ __noinline__ void alcc_kkt_pass(const Params &P, double *red, long long vc)
{
    phase_kkt<TS, NP, true>(P, 0, red, vc);
}

template <typename TS, int NP>
__global__ void __launch_bounds__(kThreads, 1) k_alcc(const __grid_constant__ Params P, const AlccStep S)
{
    extern __shared__ unsigned char sm_raw[];
    unsigned char *sm = aligned_smem(sm_raw);
    __shared__ double red[72];
    __shared__ int s_flag;
    __shared__ __align__(8) uint64_t full[kMaxStages], empty[kMaxStages];
    init_pipeline(full, empty);
    unsigned long long bar = 0, kstage = 0;
    const long long vc = blockIdx.x;
    double t = S.t0;
    long long ell = S.ell0;
    bool ret = false;
    for (; ell <= S.ell1; ++ell) {
        alcc_pair_pass<TS, NP, PM_ALCC_GRAD>(P, ell, sm, full, empty, kstage, vc, 1.0f);
        if (!grid_barrier(P, bar)) return;
        alcc_grad_fold<NP>(P, S, ell, red, vc);
        if (!grid_barrier(P, bar)) return;
        const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));   // MAPG step 3
        alcc_step_fold<NP>(P, S, ell, (t - 1.0) / tn, red, vc);
        t = tn;
        if (!grid_barrier(P, bar)) return;
        ret = mapg_returns(P, S, ell, &s_flag);
        if (ret) break;
    }
    if (!ret) {   // the launch ends inside the MAPG call
        if (vc == 0 && threadIdx.x == 0) {
            P.st->alcc_t = t;
            P.st->alcc_ell = S.ell1;
            P.st->alcc_done = 0;
        }
        return;
    }
    phase_alcc_take<NP>(P, (int)(ell & 1), vc);
    if (!grid_barrier(P, bar)) return;
    alcc_pair_pass<TS, NP, PM_ALCC_UPDATE>(P, 0, sm, full, empty, kstage, vc, S.a);   // theta_{k+1}, in place
    if (!grid_barrier(P, bar)) return;
    phase_alcc_stat<NP>(P, S, red, vc);
    alcc_kkt_pass<TS, NP>(P, red, vc);   // (A_1 y_k + A_2 xi_k)_p in FP64 against theta_{k+1}
    if (!grid_barrier(P, bar)) return;
    if (vc == 0 && threadIdx.x < 32) {
        double ry = 0.0, rx = 0.0, mv = 0.0, mc = 0.0;
        for (int c = threadIdx.x; c < P.G; c += 32) {
            ry = fmax(ry, __ldcg(P.foldpart + c * 8 + 4));
            rx = fmax(rx, __ldcg(P.foldpart + c * 8 + 5));
            mv = fmax(mv, __ldcg(P.kktpart + c * 8 + 0));
            mc = fmax(mc, __ldcg(P.kktpart + c * 8 + 1));
        }
        ry = warp_max(ry);
        rx = warp_max(rx);
        mv = warp_max(mv);
        mc = warp_max(mc);
        if (threadIdx.x == 0) {
            const double sg = P.sigma;
            const double stat = fmax(ry, rx) / sg, pri = mv / sg, comp = S.mu_next * mc / (sg * sg);
            P.st->kkt[0] = fmax(stat, fmax(pri, comp));
            P.st->kkt[1] = stat;
            P.st->kkt[2] = pri;
            P.st->kkt[3] = comp;
            P.st->alcc_t = t;
            P.st->alcc_ell = ell;
            P.st->alcc_done = 1;
        }
    }
}

struct AlccKernel {
    const void *fn;
    size_t smem;
};

// k_alcc<float, NP> for a compiled padded width (FP32 multipliers only); fn = nullptr otherwise.
AlccKernel alcc_kernel(int NP);

}  // namespace crk
