// cr_blocks.cuh -- P-APG with the points partitioned into K blocks (Sec. II-A, Fig. 2).
//
// The pairwise constraints between blocks and the y >= 0 rows of C (Eq. (eq:C)) are dualized
// (the outer multipliers theta, mu); the constraints inside each block stay in the block's Step-1
// problem
//     min 1/2 ||y_i - a_i||^2 + gamma/2 ||xi_i - b_i||^2   s.t. the block's pairwise constraints,
// a = h + A_1^T theta^(2) + mu^(2),  b = A_2^T theta^(2) / gamma  (sums over the dualized rows),
// the projection of the closed-form point onto the block's constraint set.  The library solves
// all K block problems at once with an inner P-APG on their duals (the FP64 pass restricted to the
// pairs inside a block: the inner problems separate by block), warm-started from the previous
// call's inner multipliers with the momentum restarted, for a fixed number of inner iterations;
// the paper solves Step 1 inexactly as well (ALCC, Sedumi or Mosek, Sec. III).
//
// One outer iteration l:
//   k_blocks_prepare   Steps 3-4 scalars of l; a, b at theta^(2)_l from the outer aggregates
//   inner P-APG        M iterations (FP64 pass over the pairs inside the blocks)
//   k_blocks_records   Step 1's result eta_l = (y, xi) into the outer pass's FP64 row and column
//                      data; Step 2 on the y >= 0 rows: mu^(1)_l = max(0, mu^(2)_l - y / L)
//   outer pair pass    Step 2 on the pairs between blocks (FP64 pass, pairs inside blocks masked)
//   outer foldA        the outer aggregates A_1^T theta^(1)_l, A_2^T theta^(1)_l
#pragma once

#include "cr_kernels.cuh"

namespace crk {

// at_theta1 = 0: iteration ell's momentum scalars and a, b at theta^(2)_ell (the outer
// iteration's Step 1); at_theta1 = 1: a, b at theta^(1)_ell itself (the primal point reported
// after the iterations).  mu2 receives mu^(2) for k_blocks_records.
template <int NP>
__global__ void __launch_bounds__(256)
k_blocks_prepare(const __grid_constant__ Params O, double *a, double *b, double *mu2, long long ell, int at_theta1)
{
    double beta = 0.0;
    int c, p;
    if (at_theta1) {
        c = (int)(ell & 1);
        p = c ^ 1;
    } else {
        c = (int)((ell - 1) & 1);
        p = (int)(ell & 1);
        const Scal nw = next_scal_plain(O, ell);   // Fig. 2 steps 3-4, the same value in every thread
        beta = nw.beta;
        if (blockIdx.x == 0 && threadIdx.x == 0) O.st->scal[p] = nw;
    }
    const double b1 = 1.0 + beta;
    const int n = O.n;
    for (long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x; l < O.N; l += (long long)gridDim.x * blockDim.x) {
        const double v2 = b1 * __ldcg(O.v[c] + l) - beta * __ldcg(O.v[p] + l);
        const double m2 = b1 * __ldcg(O.mu[c] + l) - beta * __ldcg(O.mu[p] + l);
        a[l] = __ldcg(O.h + l) + v2 + m2;
        mu2[l] = m2;
        for (int k = 0; k < n; ++k)
            b[l * n + k] = (b1 * __ldcg(O.w[c] + l * n + k) - beta * __ldcg(O.w[p] + l * n + k)) * O.inv_gamma;
    }
}

// Step 1's result (the inner problems' minimizer at their current multipliers) into the outer
// FP64 pass's row records and column data, and Step 2 on the y >= 0 rows.
template <int NP>
__global__ void __launch_bounds__(256)
k_blocks_records(const __grid_constant__ Params O, const double *y, const double *xi, const double *mu2, long long ell)
{
    constexpr int REC = RecLayout<NP>::REC;
    const int n = O.n;
    const int p = (int)(ell & 1);
    for (long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x; l < O.N; l += (long long)gridDim.x * blockDim.x) {
        const double yl = __ldcg(y + l);
        const double ys = yl - O.shift;
        double d = 0.0;
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            double x = 0.0;
            if (k < n) {
                x = __ldcg(xi + l * n + k);
                d += x * __ldg(O.X64 + l * n + k);
            }
            O.xi2_64[l * NP + k] = x;
        }
        O.rec64[l * REC] = ys;
        O.ccol2_64[l] = d - ys;
        const double mun = __ldcg(mu2 + l) - yl * O.invL_d;
        O.mu[p][l] = mun > 0.0 ? mun : 0.0;
    }
}

}  // namespace crk
