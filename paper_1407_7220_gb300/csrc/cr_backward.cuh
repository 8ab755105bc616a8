// cr_backward.cuh -- reverse mode through unrolled P-APG iterations (FP32 multipliers).
//
// Forward iteration l (Fig. 2, K = N), with beta_l, L, gamma and the shift held fixed:
//   theta2 = theta1_{l-1} + beta_l (theta1_{l-1} - theta1_{l-2})
//   y2 = ybar + s + A_1^T theta2 + mu2,   xi2 = A_2(X)^T theta2 / gamma
//   g_p = y2_l1 - y2_l2 - xi2_l2 . (x_l1 - x_l2),   theta1_l = max(0, theta2 - g / L)
// Given A = dLoss/dtheta1_l (built from the two later steps' adjoints by the momentum
// weights), one reverse step is:
//   pass 1 (per pair): m = [theta2 - g/L > 0] (recomputed bit for bit as in the forward),
//          w = m A, gbar = -w / L; accumulate the fold of Gbar: row and column sums,
//          Gbar^T X (columns) and Gbar Xi2 (rows)
//   fold 1 (per point, FP64): ybar2 = A_1^T gbar - w_mu / L, xibar2 = A_2^T gbar,
//          Xbar += colsum(Gbar) xi2 - (Gbar Xi2), dLoss/dybar += ybar2
//   pass 2 (per pair): thetabar2 = w + ybar2_l1 - ybar2_l2 - (xibar2_l2/gamma).(x_l1 - x_l2);
//          accumulate colsum(Theta2) and Theta2 (xibar2/gamma) for the X terms of xi2
//   fold 2 (per point): Xbar += colsum(Theta2) xibar2/gamma - (Theta2 xibar2/gamma)
// Accumulation uses FP64 atomics (order-dependent only at FP64 rounding level).
// T = float reverses the FP32 pass (its two-chain residual); T = double reverses the FP64 pass
// of cr_pair_f64.cuh (one chain, FP64 storage and arithmetic), so that the masks recomputed
// here are the forward's in either case.
#pragma once

#include "cr_kernels.cuh"

namespace crk {

constexpr int kBRows = 64;     // rows per backward task
constexpr int kBCols = 128;    // columns per backward task (one warp width x 4)

template <typename T> struct BwdParamsT {
    long long N, ld;
    int n, S128, REC;
    T invL, beta, c1, c2;
    double invL_d, inv_gamma, shift;
    const T *thc, *thp;             // theta1_{l-1}, theta1_{l-2}
    const T *rowrec;                // N x REC {y2 - s, x}
    const T *ccol2, *xi2;           // forward column data of iteration l
    const T *b1, *b2;               // thetabar2_{l+1}, thetabar2_{l+2} (N x ld)
    const float *ubar;              // dLoss/dyhat (N) on the last iteration, else null
    const T *yb2, *ccolb, *xib;     // pass 2 inputs: ybar2 (rows), xibar2.x/gamma - ybar2, xibar2/gamma (cols)
    T *outb;                        // thetabar2_l (N x ld)
    double *acc_row, *acc_col;      // [N][NP+1] accumulators (zeroed by the folds)
    // fold inputs
    const double *X64, *h;
    const double *v1, *v2, *mu1, *mu2;   // v, mu of theta1_{l-1}, theta1_{l-2} (FP64)
    const double *mub1, *mub2;      // mubar2_{l+1}, mubar2_{l+2}
    double beta_d, c1_d, c2_d;
    double *mub_out;                // mubar2_l
    double *ybar_acc, *X_acc;       // dLoss/dybar (N), dLoss/dX (N x n), FP64
    T *yb2_out, *ccolb_out, *xib_out;
};
using BwdParams = BwdParamsT<float>;

template <typename T> struct Vec4Of;
template <> struct Vec4Of<float> {
    __device__ static __forceinline__ void load(const float *p, float (&o)[4])
    {
        const float4 t = *reinterpret_cast<const float4 *>(p);
        o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
    }
    __device__ static __forceinline__ void store(float *p, const float (&v)[4])
    {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
};
template <> struct Vec4Of<double> {
    __device__ static __forceinline__ void load(const double *p, double (&o)[4])
    {
        const double2 a = *reinterpret_cast<const double2 *>(p), b = *reinterpret_cast<const double2 *>(p + 2);
        o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
    }
    __device__ static __forceinline__ void store(double *p, const double (&v)[4])
    {
        *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
        *reinterpret_cast<double2 *>(p + 2) = make_double2(v[2], v[3]);
    }
};

template <typename T, int NP, int PASS>
__global__ void __launch_bounds__(256)
k_adj_pass(const BwdParamsT<T> B)
{
    constexpr int K1 = NP + 1;
    constexpr bool F64 = std::is_same<T, double>::value;
    // FP32: the row terms and the column terms of a task meet in shared memory (dynamic,
    // bwd_smem_bytes): rowbuf holds kBRows x K1 items of 32 lane partials, item e's value of
    // lane l at e * 32 + (l ^ (e & 31)) so that neither the lanes' stores nor the one-thread-per-
    // item sums conflict on a bank; red holds the 8 warps' column partials [8][K1][kBCols].
    // FP64: warp sums and one atomic per term, as before.
    extern __shared__ float bsm[];
    float *rowbuf = bsm;
    float *red = bsm + kBRows * K1 * 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long N = B.N, ld = B.ld;
    const int REC = B.REC;
    const long long ntask = (long long)B.S128 * ((N + kBRows - 1) / kBRows);
    for (long long task = blockIdx.x; task < ntask; task += gridDim.x) {
        const long long stripe = task % B.S128, rblk = task / B.S128;
        const long long col0 = stripe * kBCols + lane * 4;
        const bool vec_ok = col0 < ld;
        bool colv[4];
        T ccol[4], xi[4][NP], cb[4], xb[4][NP];
        float ub[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const long long c = col0 + j;
            colv[j] = c < N;
            ccol[j] = colv[j] ? B.ccol2[c] : 0.0f;
            ub[j] = (colv[j] && B.ubar) ? B.ubar[c] : 0.0f;
            cb[j] = (PASS == 2 && colv[j]) ? B.ccolb[c] : (T)0;
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                xi[j][k] = colv[j] ? B.xi2[c * NP + k] : (T)0;
                xb[j][k] = (PASS == 2 && colv[j]) ? B.xib[c * NP + k] : (T)0;
            }
        }
        T cacc[4][K1];
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int k = 0; k < K1; ++k) cacc[j][k] = (T)0;
        const long long r0 = rblk * kBRows, r1 = min(N, r0 + kBRows);
        for (long long r = r0 + warp; r < r1; r += 8) {
            T rv[1 + NP];
#pragma unroll
            for (int q = 0; q < 1 + NP; ++q) rv[q] = B.rowrec[r * REC + q];
            const float ur = B.ubar ? B.ubar[r] : 0.0f;
            const T ybr = PASS == 2 ? B.yb2[r] : (T)0;
            T tc[4] = {0, 0, 0, 0}, tp[4] = {0, 0, 0, 0}, a1[4] = {0, 0, 0, 0}, a2[4] = {0, 0, 0, 0};
            if (vec_ok) {
                Vec4Of<T>::load(B.thc + r * ld + col0, tc);
                Vec4Of<T>::load(B.thp + r * ld + col0, tp);
                if (B.b1) Vec4Of<T>::load(B.b1 + r * ld + col0, a1);
                if (B.b2) Vec4Of<T>::load(B.b2 + r * ld + col0, a2);
            }
            T racc[K1];
#pragma unroll
            for (int k = 0; k < K1; ++k) racc[k] = (T)0;
            T outv[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                outv[j] = (T)0;
                if (!colv[j] || col0 + j == r) continue;
                // the forward pair pass, operation for operation
                const T th2 = fma(B.beta, tc[j] - tp[j], tc[j]);
                T v;
                if constexpr (F64) {
                    T g = rv[0] + ccol[j];   // one chain, as the FP64 pass
#pragma unroll
                    for (int k = 0; k < NP; ++k) g = fma(-xi[j][k], rv[1 + k], g);
                    v = fma(-g, B.invL, th2);
                } else {
                    T g0 = rv[0] + ccol[j], g1 = 0.0f;   // two chains (even and odd k), as the FP32 pass
#pragma unroll
                    for (int k = 0; k < NP; ++k) {
                        if (k & 1) g1 = fmaf(-xi[j][k], rv[1 + k], g1);
                        else g0 = fmaf(-xi[j][k], rv[1 + k], g0);
                    }
                    v = fmaf(-(g0 + g1), B.invL, th2);
                }
                const T A = B.c1 * a1[j] + B.c2 * a2[j] + (T)(ur - ub[j]);
                const T w = v > (T)0 ? A : (T)0;
                if (PASS == 1) {
                    const T gb = -w * B.invL;
                    racc[0] += gb;
#pragma unroll
                    for (int k = 0; k < NP; ++k) racc[1 + k] = fma(gb, xi[j][k], racc[1 + k]);
                    cacc[j][0] += gb;
#pragma unroll
                    for (int k = 0; k < NP; ++k) cacc[j][1 + k] = fma(gb, rv[1 + k], cacc[j][1 + k]);
                } else {
                    T t = ybr + cb[j];
#pragma unroll
                    for (int k = 0; k < NP; ++k) t = fma(-xb[j][k], rv[1 + k], t);
                    outv[j] = w + t;
#pragma unroll
                    for (int k = 0; k < NP; ++k) racc[1 + k] = fma(th2, xb[j][k], racc[1 + k]);
                    cacc[j][0] += th2;
                }
            }
            if (PASS == 2 && vec_ok) Vec4Of<T>::store(B.outb + r * ld + col0, outv);
            if constexpr (F64) {
#pragma unroll
                for (int k = 0; k < K1; ++k) {
                    const T t = warp_sum(racc[k]);
                    if (lane == 0 && (PASS == 1 || k > 0) && t != (T)0) atomicAdd(B.acc_row + r * K1 + k, (double)t);
                }
            } else {
                const int rl = (int)(r - r0);
#pragma unroll
                for (int k = 0; k < K1; ++k) {
                    const int e = rl * K1 + k;
                    rowbuf[e * 32 + (lane ^ (e & 31))] = racc[k];
                }
            }
        }
        const int kmax = PASS == 1 ? K1 : 1;
        if constexpr (F64) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const long long c = col0 + j;
#pragma unroll
                for (int k = 0; k < K1; ++k)
                    if (c < N && k < kmax && cacc[j][k] != 0.0) atomicAdd(B.acc_col + c * K1 + k, cacc[j][k]);
            }
        } else {
            // column sums: reduce the 8 warps in shared memory, one atomic per column and term
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int k = 0; k < K1; ++k) red[(warp * K1 + k) * kBCols + lane * 4 + j] = cacc[j][k];
            __syncthreads();
            // row sums: one thread per (row, term) item adds the 32 lane partials
            const int nitem = (int)(r1 - r0) * K1;
            for (int e = threadIdx.x; e < nitem; e += 256) {
                const int rl = e / K1, k = e - rl * K1;
                if (PASS == 2 && k == 0) continue;   // pass 2 has no row term 0
                const float *it = rowbuf + e * 32;
                const int sw = e & 31;
                float a = 0.0f;
#pragma unroll
                for (int l = 0; l < 32; ++l) a += it[l ^ sw];
                if (a != 0.0f) atomicAdd(B.acc_row + (r0 + rl) * K1 + k, (double)a);
            }
            for (int e = threadIdx.x; e < K1 * kBCols; e += 256) {
                const int k = e / kBCols, cl = e % kBCols;
                float a = 0.0f;
#pragma unroll
                for (int w = 0; w < 8; ++w) a += red[(w * K1 + k) * kBCols + cl];
                const long long c = stripe * kBCols + cl;
                if (c < N && k < kmax && a != 0.0f) atomicAdd(B.acc_col + c * K1 + k, (double)a);
            }
            __syncthreads();
        }
    }
}

// Fold of the reverse step (FP64, one thread per point).
template <typename T, int NP, int PASS>
__global__ void __launch_bounds__(256)
k_adj_fold(const BwdParamsT<T> B)
{
    constexpr int K1 = NP + 1;
    const long long N = B.N;
    const int n = B.n;
    for (long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x; l < N; l += (long long)gridDim.x * blockDim.x) {
        if (PASS == 1) {
            // the y >= 0 rows of C: mask exactly as the forward fold formed mu1_l
            const double b1 = 1.0 + B.beta_d;
            const double v2 = b1 * B.v1[l] - B.beta_d * B.v2[l];
            const double m2 = b1 * B.mu1[l] - B.beta_d * B.mu2[l];
            const double y2 = B.h[l] + v2 + m2;
            const double mun = m2 - y2 * B.invL_d;
            double Amu = B.c1_d * (B.mub1 ? B.mub1[l] : 0.0) + B.c2_d * (B.mub2 ? B.mub2[l] : 0.0) +
                         (B.ubar ? (double)B.ubar[l] : 0.0);
            const double wmu = mun > 0.0 ? Amu : 0.0;
            const double R = B.acc_row[l * K1], Cc = B.acc_col[l * K1];
            const double yb2 = R - Cc - wmu * B.invL_d;          // A_1^T gbar + adjoint of mu's update
            B.ybar_acc[l] += yb2;
            B.mub_out[l] = wmu + yb2;                            // y2 = ... + mu2
            double d = 0.0;
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                T xf = (T)0;
                if (k < n) {
                    const double xk = B.X64[l * n + k];
                    const double xib = Cc * xk - B.acc_col[l * K1 + 1 + k];   // A_2^T gbar
                    // X terms of g: colsum(Gbar) xi2_l - (Gbar Xi2)_l
                    B.X_acc[l * n + k] += Cc * (double)B.xi2[l * NP + k] - B.acc_row[l * K1 + 1 + k];
                    const double xg = xib * B.inv_gamma;
                    d += xg * xk;
                    xf = (T)xg;
                }
                B.xib_out[l * NP + k] = xf;
            }
            B.yb2_out[l] = (T)yb2;
            B.ccolb_out[l] = (T)(d - yb2);
        } else {
            const double Cth = B.acc_col[l * K1];
#pragma unroll
            for (int k = 0; k < NP; ++k)
                if (k < n) B.X_acc[l * n + k] += Cth * (double)B.xib[l * NP + k] - B.acc_row[l * K1 + 1 + k];
        }
#pragma unroll
        for (int k = 0; k < K1; ++k) {
            B.acc_row[l * K1 + k] = 0.0;
            B.acc_col[l * K1 + k] = 0.0;
        }
    }
}

struct BwdKernels {
    const void *pass1, *pass2, *fold1, *fold2;
    size_t smem;   // dynamic shared memory of the passes
};

// dynamic shared memory of k_adj_pass: the FP32 row items and column partials, none in FP64
template <typename T, int NP> constexpr size_t bwd_smem_bytes()
{
    return std::is_same<T, double>::value ? 0 : (size_t)(kBRows * 32 + 8 * kBCols) * (NP + 1) * sizeof(float);
}

// reverse mode is compiled for n <= 10 (padded widths 2, 4, 5, 8, 10), FP32 or FP64 multipliers
template <typename TS, int NP> BwdKernels make_bwd()
{
    if constexpr (NP <= 10 && (std::is_same<TS, float>::value || std::is_same<TS, double>::value))
        return BwdKernels{(const void *)k_adj_pass<TS, NP, 1>, (const void *)k_adj_pass<TS, NP, 2>,
                          (const void *)k_adj_fold<TS, NP, 1>, (const void *)k_adj_fold<TS, NP, 2>,
                          bwd_smem_bytes<TS, NP>()};
    else
        return BwdKernels{nullptr, nullptr, nullptr, nullptr, 0};
}

}  // namespace crk
