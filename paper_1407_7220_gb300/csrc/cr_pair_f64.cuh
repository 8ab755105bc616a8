// cr_pair_f64.cuh -- Step 2 of P-APG (Fig. 2) with the multiplier array stored in FP64.
//
// FP32 multipliers stop resolving the iterates near theta ~ 1 once the updates g/L fall below
// an ulp (2^-24 relative), and FP32 partial sums of the adjoint carry errors of the same order
// relative to the row and column sums; both set a floor on the KKT residual.  This pass keeps
// the whole per-pair computation in FP64: theta^(2) = theta^(1) + beta (theta^(1) - prev),
// g = (C eta)_p = (y_l1 - s) + (xi_l2.x_l2 - (y_l2 - s)) - xi_l2.x_l1 from FP64 copies of the
// fold's row and column data, theta^(1)_l = max(0, theta^(2) - g/L), and the fused adjoint (row
// sums, column sums, Theta^T X) accumulated in FP64 into FP64 partials (the layouts of the FP32
// pass).  The problems it serves are small (their two arrays sit in L2), so the tiles are read
// with plain coalesced loads: the CTA partition into (stripe, row) units, the warp layout (2
// warps across a 256-column stripe, 4 row groups, 4 columns per lane) and the row partials are
// those of the streaming pass; the 4 row groups' column partials are added in shared memory
// (fixed order) so that the fold reads one block per CTA segment.  GB300's FP64 pipe is narrow,
// so the grid uses every SM.
#pragma once

#include "cr_kernels.cuh"

namespace crk {

// Shared memory of the pass: one (NP + 1) x 256 block of FP64 column partials.
template <int NP> constexpr size_t f64_smem_bytes() { return (size_t)(NP + 1) * kW * sizeof(double) + 128; }

template <int NP> __device__ void phase_pair_f64(const Params &P, long long ell, unsigned char *smem, long long vc)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wc = warp & 1, rg = warp >> 1;
    const int p = (int)(ell & 1), c = 1 - p;
    const long long N = P.N, ld = P.ld;
    const long long ubeg = unit_begin(P, vc), uend = unit_begin(P, vc + 1);
    const double beta = __ldcg(&P.st->scal[p].beta);
    const double invL = P.invL_d;
    const double *cur = (const double *)P.theta[c];   // theta^(1)_{l-1}
    double *nxt = (double *)P.theta[p];               // theta^(1)_{l-2} on entry, theta^(1)_l on exit
    constexpr int REC = RecLayout<NP>::REC;
    const long long first_stripe = ubeg / N;
    for (long long u = ubeg; u < uend;) {
        const long long s = u / N, r0 = u - s * N, r1 = min(N, r0 + (uend - u));
        const long long col0 = s * kW + wc * 128 + lane * 4;   // this lane's 4 columns
        const bool vec_ok = col0 < ld;                          // ld is a multiple of 16
        double ccol[4], nxi[4][NP], csum[4], acc[4][NP];
        int bcol[4] = {-1, -1, -1, -1};   // block ids of this lane's columns (K-block P-APG)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const long long cj = col0 + j;
            const bool v = cj < N;
            if (P.blkmode && v) bcol[j] = __ldg(P.blk + cj);
            ccol[j] = v ? __ldcg(P.ccol2_64 + cj) : 0.0;
            csum[j] = 0.0;
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                nxi[j][k] = v ? -__ldcg(P.xi2_64 + cj * NP + k) : 0.0;
                acc[j][k] = 0.0;
            }
        }
        double *rp = P.rowpart64 + (s * 2 + wc);   // row r's partial at rp[r * Q]
        // pairs inside the blocks only: the rows of the stripe's band (the other rows' partials
        // stay 0; the column partials of the segment are written either way)
        const long long rb0 = P.band ? max(r0, __ldg(P.band + 2 * s)) : r0;
        const long long rb1 = P.band ? min(r1, __ldg(P.band + 2 * s + 1)) : r1;
        for (long long r = rb0 + rg; r < rb1; r += kWR) {
            const int brow = P.blkmode ? __ldg(P.blk + r) : -2;
            const double *rec = P.rec64 + r * REC;
            const double yr = __ldcg(rec);
            double xr[NP];
#pragma unroll
            for (int k = 0; k < NP; ++k) xr[k] = __ldcg(rec + 1 + k);
            double tc[4] = {0.0, 0.0, 0.0, 0.0}, tp[4] = {0.0, 0.0, 0.0, 0.0};
            if (vec_ok) {
                const double2 a0 = __ldcg(reinterpret_cast<const double2 *>(cur + r * ld + col0));
                const double2 a1 = __ldcg(reinterpret_cast<const double2 *>(cur + r * ld + col0 + 2));
                const double2 b0 = __ldcg(reinterpret_cast<const double2 *>(nxt + r * ld + col0));
                const double2 b1 = __ldcg(reinterpret_cast<const double2 *>(nxt + r * ld + col0 + 2));
                tc[0] = a0.x; tc[1] = a0.y; tc[2] = a1.x; tc[3] = a1.y;
                tp[0] = b0.x; tp[1] = b0.y; tp[2] = b1.x; tp[3] = b1.y;
            }
            double out[4], rs = 0.0;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const long long cj = col0 + j;
                double g = yr + ccol[j];   // (C eta)_p = y_l1 - y_l2 + xi_l2.x_l2 - xi_l2.x_l1
#pragma unroll
                for (int k = 0; k < NP; ++k) g = fma(nxi[j][k], xr[k], g);
                const double th2 = fma(beta, tc[j] - tp[j], tc[j]);   // theta^(2)
                const double v = fma(-g, invL, th2);
                double nw = v > 0.0 ? v : 0.0;                         // projection on theta >= 0
                if (cj >= N || cj == r) nw = 0.0;                      // padding columns, diagonal
                // K blocks: the outer dual holds the pairs between blocks, the inner one those inside
                if ((P.blkmode == 1 && bcol[j] == brow) || (P.blkmode == 2 && bcol[j] != brow)) nw = 0.0;
                out[j] = nw;
                rs += nw;
                csum[j] += nw;
#pragma unroll
                for (int k = 0; k < NP; ++k) acc[j][k] = fma(nw, xr[k], acc[j][k]);
            }
            if (vec_ok) {
                *reinterpret_cast<double2 *>(nxt + r * ld + col0) = make_double2(out[0], out[1]);
                *reinterpret_cast<double2 *>(nxt + r * ld + col0 + 2) = make_double2(out[2], out[3]);
            }
            // row sum of this warp's 128 columns (fixed butterfly order)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) rs += __shfl_xor_sync(0xffffffffu, rs, o);
            if (lane == 0) rp[r * P.Q] = rs;
        }
        // column partials of this segment: the row groups added in order 0..3 in shared memory,
        // then one block to global memory (added in FP64 by foldA)
        double *red = reinterpret_cast<double *>(smem);
        const int cl = wc * 128 + lane * 4;
        for (int g = 0; g < kWR; ++g) {
            if (rg == g) {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    red[cl + j] = g == 0 ? csum[j] : red[cl + j] + csum[j];
#pragma unroll
                    for (int k = 0; k < NP; ++k)
                        red[(1 + k) * kW + cl + j] = g == 0 ? acc[j][k] : red[(1 + k) * kW + cl + j] + acc[j][k];
                }
            }
            __syncthreads();
        }
        const int slotc = (int)(s - first_stripe);
        double *cp = P.colpart64 + ((vc * P.slots + slotc) * (NP + 1)) * kW;
        for (int i = tid; i < (NP + 1) * kW; i += kThreads) cp[i] = red[i];
        __syncthreads();
        u += r1 - r0;
    }
    __syncthreads();
}

}  // namespace crk
