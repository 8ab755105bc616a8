/*
 * cr_oracle.c -- plain FP64 CPU oracle for the P-APG iteration of
 * Aybat & Wang, "A Parallel Method for Large Scale Convex Regression
 * Problems" (arXiv:1407.7220).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent reference that the
 * CUDA path is checked against.  Nothing in the product library links, loads
 * or calls it; only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark may.  It shares no code, header or helper with the CUDA path.
 *
 * What it computes (all FP64, round-to-nearest, no FMA contraction):
 *
 *   Problem (regularize), Sec. II-C:
 *       min_{y, xi}  1/2 ||y - ybar||^2 + gamma/2 ||xi||^2
 *       s.t.  y_{l1} - y_{l2} - xi_{l2}^T (x_{l1} - x_{l2}) >= 0,  l1 != l2   (problem (original))
 *   plus the rows y >= 0 of C in Eq. (eq:C), made inactive by shifting the
 *   observations up by s (the paragraph after Eq. (omega_primal)).
 *
 *   Every pairwise constraint is dualized: the partition of Sec. II-A is taken
 *   to singletons (K = N), so Q_1 of Eq. (omega_primal) is the whole space and
 *   Step 1 of P-APG (Fig. 2) has the closed form
 *       y  = h + A_1^T theta + mu,        h = ybar + s
 *       xi = A_2^T theta / gamma
 *   with (A_1^T theta)_l = sum_m theta[l][m] - sum_m theta[m][l]
 *        (A_2^T theta)_l = sum_m theta[m][l] (x_l - x_m)
 *   (row p = (l1,l2) of A_1 is e_{l1} - e_{l2}; of A_2 it is
 *    -(x_{l1} - x_{l2})^T placed in block l2 -- problem (original)).
 *
 *   The iteration is P-APG, Fig. 2, steps 1-4, with the dual gradient of
 *   Eq. (dual gradient), grad g = -C eta, and the projection onto
 *   Q_2 = {theta >= 0} (B_theta = infinity).
 *
 * Storage: X is N x n row-major; theta is N x N row-major with
 * theta[l1*N + l2] the multiplier of the constraint (l1, l2); the diagonal
 * is unused and kept at zero.
 *
 * Options that are not in the paper are marked as such where they are read:
 * `restart` (function-value adaptive restart of the momentum) and
 * `momentum = 0` (the paper's comparator, dual gradient ascent, Sec. III).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_API __attribute__((visibility("default")))

/* Loops over rows run on several threads only from this many points on: at smaller N a
 * parallel region costs more than the loop (the pins run millions of iterations at N = 20).
 * Scheduling only: every sum below walks its terms in the same order whatever the thread
 * count, except the reduction clauses of orc_metrics (FP64 sums, order of the partials). */
#define ORC_PAR_MIN 256

/* ------------------------------------------------------------------------ */
/* Problem constants                                                         */
/* ------------------------------------------------------------------------ */

/* Shift of the observations (the paragraph after Eq. (omega_primal)): the
 * paper only asks for "a sufficiently large quantity" so that y(gamma) >= 0.
 * Reading used here: s = max(0, -min ybar) + (max ybar - min ybar). */
ORC_API double orc_shift(const double *ybar, int64_t N)
{
    double lo = ybar[0], hi = ybar[0];
    for (int64_t l = 1; l < N; ++l) {
        if (ybar[l] < lo) lo = ybar[l];
        if (ybar[l] > hi) hi = ybar[l];
    }
    double s = (lo < 0.0 ? -lo : 0.0) + (hi - lo);
    return s;
}

/* Largest eigenvalue of a symmetric n x n matrix (row-major, destroyed) by the
 * cyclic Jacobi rotation method (Golub & Van Loan, Sec. 8.5). */
static double jacobi_max_eig(double *a, int n)
{
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                tot += a[i * n + j] * a[i * n + j];
                if (i != j) off += a[i * n + j] * a[i * n + j];
            }
        if (off <= 1e-30 * tot || off == 0.0) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                double apq = a[p * n + q];
                if (apq == 0.0) continue;
                double app = a[p * n + p], aqq = a[q * n + q];
                double tau = (aqq - app) / (2.0 * apq);
                double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
                /* A <- J^T A J with J the (p,q) rotation */
                for (int k = 0; k < n; ++k) {
                    double akp = a[k * n + p], akq = a[k * n + q];
                    a[k * n + p] = c * akp - s * akq;
                    a[k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {
                    double apk = a[p * n + k], aqk = a[q * n + k];
                    a[p * n + k] = c * apk - s * aqk;
                    a[q * n + k] = s * apk + c * aqk;
                }
            }
    }
    double mx = a[0];
    for (int i = 1; i < n; ++i)
        if (a[i * n + i] > mx) mx = a[i * n + i];
    return mx;
}

/* Lipschitz constant of grad g_gamma, Eq. (eq:lischitz): L_g = sigma_max(C)^2 / gamma.
 * The paper does not say how sigma_max(C) is obtained.  Reading used here: the
 * bound  sigma_max(C)^2 <= 1 + ||A_1||^2 + ||A_2||^2  with
 *   ||A_1||^2 = 2N          (A_1^T A_1 = 2(N I - 1 1^T), the complete-graph Laplacian x2)
 *   ||A_2||^2 = max_l lambda_max(M_l),  M_l = sum_{m != l} (x_m - x_l)(x_m - x_l)^T
 * (A_2^T A_2 is block diagonal with blocks M_l).  M_l is formed by its definition
 * and its largest eigenvalue found by Jacobi. */
ORC_API double orc_lipschitz(const double *X, int64_t N, int32_t n, double gamma)
{
    double lam2 = 0.0;
#pragma omp parallel if (N >= ORC_PAR_MIN)
    {
        double *M = (double *)malloc(sizeof(double) * n * n);
        double local = 0.0;
#pragma omp for schedule(static)
        for (int64_t l = 0; l < N; ++l) {
            memset(M, 0, sizeof(double) * n * n);
            for (int64_t m = 0; m < N; ++m) {
                if (m == l) continue;
                for (int i = 0; i < n; ++i) {
                    double di = X[m * n + i] - X[l * n + i];
                    for (int j = 0; j < n; ++j) M[i * n + j] += di * (X[m * n + j] - X[l * n + j]);
                }
            }
            double e = jacobi_max_eig(M, n);
            if (e > local) local = e;
        }
#pragma omp critical
        if (local > lam2) lam2 = local;
        free(M);
    }
    return (1.0 + 2.0 * (double)N + lam2) / gamma;
}

/* ------------------------------------------------------------------------ */
/* Step 1 of P-APG (Fig. 2) at K = N: the closed-form minimizer of the       */
/* Lagrangian in Eq. (eq:g_gamma).                                            */
/* ------------------------------------------------------------------------ */

/* y_l  = h_l + sum_{m!=l} theta[l][m] - sum_{m!=l} theta[m][l] + mu_l
 * xi_l = (1/gamma) sum_{m!=l} theta[m][l] (x_l - x_m)                        */
ORC_API void orc_eta(const double *theta, const double *mu, const double *X, const double *h,
                     int64_t N, int32_t n, double gamma, double *y, double *xi)
{
    /* row sums: (A_1^T theta) positive part */
#pragma omp parallel for schedule(static) if (N >= ORC_PAR_MIN)
    for (int64_t l = 0; l < N; ++l) {
        double r = 0.0;
        for (int64_t m = 0; m < N; ++m)
            if (m != l) r += theta[l * N + m];
        y[l] = r;
    }
    /* column sums and A_2^T theta; each thread owns a range of columns l and
     * walks the rows m in increasing order (row-major reads). */
#pragma omp parallel if (N >= ORC_PAR_MIN)
    {
        int nt = 1, tid = 0;
#ifdef _OPENMP
        nt = omp_get_num_threads();
        tid = omp_get_thread_num();
#endif
        int64_t l0 = N * tid / nt, l1 = N * (tid + 1) / nt;
        int64_t w = l1 - l0;
        double *col = (double *)calloc((size_t)(w > 0 ? w : 1), sizeof(double));
        double *ax = (double *)calloc((size_t)(w > 0 ? w : 1) * n, sizeof(double));
        for (int64_t m = 0; m < N; ++m) {
            const double *trow = theta + m * N;
            const double *xm = X + m * n;
            for (int64_t l = l0; l < l1; ++l) {
                if (l == m) continue;
                double t = trow[l];
                col[l - l0] += t;
                for (int k = 0; k < n; ++k) ax[(l - l0) * n + k] += t * (X[l * n + k] - xm[k]);
            }
        }
        for (int64_t l = l0; l < l1; ++l) {
            y[l] = h[l] + y[l] - col[l - l0] + mu[l];
            for (int k = 0; k < n; ++k) xi[l * n + k] = ax[(l - l0) * n + k] / gamma;
        }
        free(col);
        free(ax);
    }
}

/* Constraint row p = (l1, l2) of C eta (Eq. (eq:C) and problem (original)):
 *   (C eta)_p = y_{l1} - y_{l2} - xi_{l2}^T (x_{l1} - x_{l2}).               */
static inline double pair_row(const double *y, const double *xi, const double *X, int32_t n,
                              int64_t l1, int64_t l2)
{
    double v = y[l1] - y[l2];
    for (int k = 0; k < n; ++k) v -= xi[l2 * n + k] * (X[l1 * n + k] - X[l2 * n + k]);
    return v;
}

/* Full N x N array of (C eta)_p (diagonal set to 0); for tests at small N. */
ORC_API void orc_residual(const double *y, const double *xi, const double *X, int64_t N, int32_t n,
                          double *G)
{
#pragma omp parallel for schedule(static) if (N >= ORC_PAR_MIN)
    for (int64_t l1 = 0; l1 < N; ++l1)
        for (int64_t l2 = 0; l2 < N; ++l2) G[l1 * N + l2] = (l1 == l2) ? 0.0 : pair_row(y, xi, X, n, l1, l2);
}

/* ------------------------------------------------------------------------ */
/* Metrics at a dual point theta (with its minimizer eta = (y, xi))           */
/* ------------------------------------------------------------------------ */

/* out[] layout (all FP64):
 *  0 kkt      = max(pri, comp)
 *  1 pri      = max( max_p (-(C eta)_p)_+ , max_l (-y_l)_+ ) / sigma
 *  2 comp     = max( max_p theta_p |(C eta)_p| , max_l mu_l |y_l| ) / sigma^2
 *  3 infeas   = || (A_1 y + A_2 xi)_- ||_2 / sqrt(N^2 - N)       (Sec. III, normalized infeasibility)
 *  4 gap      = theta^T C eta / (N^2 - N)                        (Sec. III, normalized duality gap)
 *  5 primal   = 1/2 ||y - h||^2 + gamma/2 ||xi||^2              (objective of (regularize))
 *  6 dual     = g_gamma(theta), Eq. (eq:g_gamma)
 *  7 fit      = 1/2 ||y - h||^2   (the paper's reported objective 1/2||y - ybar||^2, shift removed)
 *  8 sum_check= sum_l (y_l - h_l - mu_l)  (identically zero since A_1 1 = 0)
 * sigma = max(1, max ybar - min ybar), the scale of the data (a reading: the
 * paper reports only normalized infeasibility and gap, Sec. III). */
ORC_API void orc_metrics(const double *theta, const double *mu, const double *y, const double *xi,
                         const double *X, const double *h, int64_t N, int32_t n, double gamma,
                         double sigma, double *out)
{
    double maxviol = 0.0, maxcomp = 0.0, sumviol2 = 0.0, thetaG = 0.0;
#pragma omp parallel for schedule(static) reduction(max : maxviol, maxcomp) reduction(+ : sumviol2, thetaG) if (N >= ORC_PAR_MIN)
    for (int64_t l1 = 0; l1 < N; ++l1) {
        for (int64_t l2 = 0; l2 < N; ++l2) {
            if (l1 == l2) continue;
            double g = pair_row(y, xi, X, n, l1, l2);
            double th = theta[l1 * N + l2];
            if (-g > maxviol) maxviol = -g;
            if (g < 0.0) sumviol2 += g * g;
            double c = th * fabs(g);
            if (c > maxcomp) maxcomp = c;
            thetaG += th * g;
        }
    }
    double fit = 0.0, xin = 0.0, muy = 0.0, sumchk = 0.0;
    for (int64_t l = 0; l < N; ++l) {
        double u = y[l] - h[l];
        fit += u * u;
        if (-y[l] > maxviol) maxviol = -y[l];
        if (y[l] < 0.0) sumviol2 += y[l] * y[l];
        double c = mu[l] * fabs(y[l]);
        if (c > maxcomp) maxcomp = c;
        muy += mu[l] * y[l];
        sumchk += u - mu[l];
        for (int k = 0; k < n; ++k) xin += xi[l * n + k] * xi[l * n + k];
    }
    double pri = maxviol / sigma, comp = maxcomp / (sigma * sigma);
    double npairs = (double)N * (double)(N - 1);
    double primal = 0.5 * fit + 0.5 * gamma * xin;
    double gap = thetaG + muy; /* theta^T C eta including the y >= 0 rows */
    out[0] = pri > comp ? pri : comp;
    out[1] = pri;
    out[2] = comp;
    out[3] = sqrt(sumviol2) / sqrt(npairs);
    out[4] = gap / npairs;
    out[5] = primal;
    out[6] = primal - gap;
    out[7] = 0.5 * fit;
    out[8] = sumchk;
}

/* Dual value g_gamma(theta) of Eq. (eq:g_gamma) from the minimizer only:
 * theta^T C eta = (A_1^T theta + mu)^T y + (A_2^T theta)^T xi = (y-h)^T y + gamma ||xi||^2,
 * so g_gamma = 1/2||y-h||^2 + gamma/2||xi||^2 - (y-h)^T y - gamma||xi||^2. */
static double dual_value(const double *y, const double *xi, const double *h, int64_t N, int32_t n,
                         double gamma)
{
    double a = 0.0, b = 0.0, c = 0.0;
    for (int64_t l = 0; l < N; ++l) {
        double u = y[l] - h[l];
        a += u * u;
        c += u * y[l];
        for (int k = 0; k < n; ++k) b += xi[l * n + k] * xi[l * n + k];
    }
    return 0.5 * a + 0.5 * gamma * b - c - gamma * b;
}

/* ------------------------------------------------------------------------ */
/* P-APG, Fig. 2                                                              */
/* ------------------------------------------------------------------------ */

/* Iteration state, owned by the caller:
 *   P   (N x N) = theta^(1)_{l-1}      muP (N) = its y >= 0 multipliers
 *   T2  (N x N) = theta^(2)_l          mu2 (N)
 *   scal[0] = t_l, scal[1] = l - 1 (iterations done), scal[2] = g_gamma(theta^(1)_{l-1})
 *             (used by the restart option), scal[3] = restarts so far.
 * Iteration 0 of Fig. 2 (theta^(1)_0 = theta^(2)_1 = 0, t_1 = 1) is the state
 * with P = T2 = 0, mu = 0, scal = {1, 0, -inf, 0}; orc_state_init sets it. */
ORC_API void orc_state_init(int64_t N, double *P, double *T2, double *muP, double *mu2, double *scal)
{
    memset(P, 0, sizeof(double) * (size_t)N * (size_t)N);
    memset(T2, 0, sizeof(double) * (size_t)N * (size_t)N);
    memset(muP, 0, sizeof(double) * (size_t)N);
    memset(mu2, 0, sizeof(double) * (size_t)N);
    scal[0] = 1.0;
    scal[1] = 0.0;
    scal[2] = -INFINITY;
    scal[3] = 0.0;
}

typedef struct {
    double gamma;     /* Tikhonov parameter of (regularize), > 0            */
    double L;         /* step constant L_g of Eq. (eq:lischitz)             */
    double sigma;     /* data scale used by the KKT metric                  */
    double tol;       /* stop when the KKT metric at theta^(1) is <= tol    */
    int32_t momentum; /* 1: P-APG (Fig. 2); 0: dual gradient ascent (Sec. III comparator) */
    int32_t restart;  /* NOT IN THE PAPER: 1 = reset t to 1 whenever g_gamma(theta^(1)_l) < g_gamma(theta^(1)_{l-1}) */
    int32_t check_every; /* evaluate the KKT metric every this many iterations (0 = never) */
    int32_t pad;
    double restart_tol;  /* restart only if the dual value fell by more than restart_tol * |previous| */
    double B_theta;      /* radius of the ball in Q_2 = {lambda >= 0, ||lambda||_2 <= B_theta} (Eq. (lambda_dual));
                            <= 0 or infinite: no ball (Q_2 = {lambda >= 0}) */
} orc_opts;

/* Runs up to max_iter iterations of P-APG from the given state.  After each
 * iteration l the state holds theta^(1)_l in P and theta^(2)_{l+1} in T2.
 * y, xi (outputs) are the minimizer at the last theta^(1) (Theorem 1 reads the
 * primal at the dual iterate), metrics (9 doubles, see orc_metrics) are taken
 * there too.  Returns the number of iterations run. */
ORC_API int64_t orc_papg(const double *X, const double *h, int64_t N, int32_t n, const orc_opts *o,
                         double *P, double *T2, double *muP, double *mu2, double *scal,
                         int64_t max_iter, double *y, double *xi, double *metrics)
{
    const double gamma = o->gamma, invL = 1.0 / o->L;
    double *yy = (double *)malloc(sizeof(double) * (size_t)N);
    double *xx = (double *)malloc(sizeof(double) * (size_t)N * n);
    double *mun = (double *)malloc(sizeof(double) * (size_t)N);
    int64_t it = 0;
    int have_eta1 = 0;
    for (it = 0; it < max_iter; ++it) {
        /* Step 1: eta_l = argmin of the Lagrangian at theta^(2)_l. */
        orc_eta(T2, mu2, X, h, N, n, gamma, yy, xx);

        /* Step 2: theta^(1)_l = Pi_{Q_2}(theta^(2)_l - (1/L) C eta_l), written over T2
         * (theta^(2)_l is not needed afterwards).  Q_2 = {theta >= 0}. */
#pragma omp parallel for schedule(static) if (N >= ORC_PAR_MIN)
        for (int64_t l1 = 0; l1 < N; ++l1) {
            for (int64_t l2 = 0; l2 < N; ++l2) {
                if (l1 == l2) continue;
                double g = pair_row(yy, xx, X, n, l1, l2);
                double v = T2[l1 * N + l2] - g * invL;
                T2[l1 * N + l2] = v > 0.0 ? v : 0.0;
            }
        }
        /* rows y >= 0 of C (the identity block in Eq. (eq:C)) */
        for (int64_t l = 0; l < N; ++l) {
            double v = mu2[l] - yy[l] * invL;
            mun[l] = v > 0.0 ? v : 0.0;
        }
        /* Q_2 with a finite ball: the projection onto {lambda >= 0} intersected with the ball
         * ||lambda||_2 <= B_theta centred at 0 is the projection onto the orthant (the clamp
         * above) followed by the radial scaling min(1, B_theta / ||lambda||_2), over all dual
         * variables lambda = (theta, mu) */
        if (o->B_theta > 0.0 && isfinite(o->B_theta)) {
            double ss = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : ss) if (N >= ORC_PAR_MIN)
            for (int64_t l1 = 0; l1 < N; ++l1)
                for (int64_t l2 = 0; l2 < N; ++l2) ss += T2[l1 * N + l2] * T2[l1 * N + l2];
            for (int64_t l = 0; l < N; ++l) ss += mun[l] * mun[l];
            const double nrm = sqrt(ss);
            if (nrm > o->B_theta) {
                const double c = o->B_theta / nrm;
#pragma omp parallel for schedule(static) if (N >= ORC_PAR_MIN)
                for (int64_t l1 = 0; l1 < N; ++l1)
                    for (int64_t l2 = 0; l2 < N; ++l2) T2[l1 * N + l2] *= c;
                for (int64_t l = 0; l < N; ++l) mun[l] *= c;
            }
        }

        double ell = scal[1] + 1.0;
        int need_eta1 = o->restart || (o->check_every > 0 && ((int64_t)ell % o->check_every) == 0) ||
                        it == max_iter - 1;
        have_eta1 = 0;
        if (need_eta1) {
            orc_eta(T2, mun, X, h, N, n, gamma, y, xi);
            have_eta1 = 1;
        }

        /* Step 3: t_{l+1} = (1 + sqrt(1 + 4 t_l^2)) / 2, momentum weight (t_l - 1)/t_{l+1}. */
        double t = scal[0];
        if (o->restart) {
            double dv = dual_value(y, xi, h, N, n, gamma);
            if (dv < scal[2] - o->restart_tol * fabs(scal[2])) {
                t = 1.0; /* restart: the weight below becomes 0 */
                scal[3] += 1.0;
            }
            scal[2] = dv;
        }
        double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
        double beta = o->momentum ? (t - 1.0) / tn : 0.0;
        scal[0] = tn;
        scal[1] = ell;

        /* Step 4: theta^(2)_{l+1} = theta^(1)_l + beta (theta^(1)_l - theta^(1)_{l-1}). */
#pragma omp parallel for schedule(static) if (N >= ORC_PAR_MIN)
        for (int64_t l1 = 0; l1 < N; ++l1) {
            for (int64_t l2 = 0; l2 < N; ++l2) {
                int64_t q = l1 * N + l2;
                double cur = T2[q];
                T2[q] = cur + beta * (cur - P[q]);
                P[q] = cur;
            }
        }
        for (int64_t l = 0; l < N; ++l) {
            double cur = mun[l];
            mu2[l] = cur + beta * (cur - muP[l]);
            muP[l] = cur;
        }

        if (o->check_every > 0 && ((int64_t)ell % o->check_every) == 0) {
            orc_metrics(P, muP, y, xi, X, h, N, n, gamma, o->sigma, metrics);
            if (metrics[0] <= o->tol) {
                ++it;
                break;
            }
        }
    }
    if (!have_eta1) orc_eta(P, muP, X, h, N, n, gamma, y, xi);
    orc_metrics(P, muP, y, xi, X, h, N, n, gamma, o->sigma, metrics);
    free(yy);
    free(xx);
    free(mun);
    return it;
}

/* ------------------------------------------------------------------------ */
/* Forward-mode derivative of K iterations of P-APG (Fig. 2) from Iteration 0 */
/* ------------------------------------------------------------------------ */

/* Tangent of the fitted values yhat = y(theta^(1)_K) - s along a direction
 * (dybar, dX) of the data, with gamma, L and the shift s held fixed and plain
 * P-APG momentum (no restart).  Every step of the loop is differentiated as
 * written: Step 1 (closed form, linear in theta and in X through A_2), Step 2
 * (the projection max(0, .) differentiates to its active indicator), Steps 3-4
 * (linear).  Returns yhat (N) and its tangent dyhat (N). */
ORC_API void orc_papg_jvp(const double *X, const double *ybar, int64_t N, int32_t n, double gamma, double L,
                          double s, int64_t K, const double *dybar, const double *dX, double *yhat,
                          double *dyhat)
{
    const size_t NN = (size_t)N * (size_t)N;
    double *P = (double *)calloc(NN, sizeof(double)), *T2 = (double *)calloc(NN, sizeof(double));
    double *dP = (double *)calloc(NN, sizeof(double)), *dT2 = (double *)calloc(NN, sizeof(double));
    double *muP = (double *)calloc(N, sizeof(double)), *mu2 = (double *)calloc(N, sizeof(double));
    double *dmuP = (double *)calloc(N, sizeof(double)), *dmu2 = (double *)calloc(N, sizeof(double));
    double *h = (double *)malloc(sizeof(double) * N), *y = (double *)malloc(sizeof(double) * N);
    double *dy = (double *)malloc(sizeof(double) * N), *xi = (double *)malloc(sizeof(double) * N * n);
    double *dxi = (double *)malloc(sizeof(double) * N * n);
    double *nw = (double *)malloc(sizeof(double) * NN), *dnw = (double *)malloc(sizeof(double) * NN);
    double *mun = (double *)malloc(sizeof(double) * N), *dmun = (double *)malloc(sizeof(double) * N);
    const double invL = 1.0 / L;
    for (int64_t l = 0; l < N; ++l) h[l] = ybar[l] + s;
    double t = 1.0;
    for (int64_t it = 0; it < K; ++it) {
        /* Step 1 and its tangent:
         *   y = h + sum_m T2[l][m] - sum_m T2[m][l] + mu2,       dy = dybar + (same with dT2) + dmu2
         *   gamma xi_l = sum_m T2[m][l] (x_l - x_m),
         *   gamma dxi_l = sum_m dT2[m][l] (x_l - x_m) + sum_m T2[m][l] (dx_l - dx_m) */
#pragma omp parallel for schedule(static) if (N >= ORC_PAR_MIN)
        for (int64_t l = 0; l < N; ++l) {
            double r = 0.0, dr = 0.0, c = 0.0, dc = 0.0;
            for (int64_t m = 0; m < N; ++m) {
                if (m == l) continue;
                r += T2[l * N + m] - T2[m * N + l];
                dr += dT2[l * N + m] - dT2[m * N + l];
            }
            (void)c;
            (void)dc;
            y[l] = h[l] + r + mu2[l];
            dy[l] = dybar[l] + dr + dmu2[l];
            for (int k = 0; k < n; ++k) {
                double a = 0.0, da = 0.0;
                for (int64_t m = 0; m < N; ++m) {
                    if (m == l) continue;
                    const double tm = T2[m * N + l], dtm = dT2[m * N + l];
                    a += tm * (X[l * n + k] - X[m * n + k]);
                    da += dtm * (X[l * n + k] - X[m * n + k]) + tm * (dX[l * n + k] - dX[m * n + k]);
                }
                xi[l * n + k] = a / gamma;
                dxi[l * n + k] = da / gamma;
            }
        }
        /* Step 2 and its tangent: new = max(0, T2 - g/L), g = y_l1 - y_l2 - xi_l2 (x_l1 - x_l2) */
#pragma omp parallel for schedule(static) if (N >= ORC_PAR_MIN)
        for (int64_t l1 = 0; l1 < N; ++l1) {
            for (int64_t l2 = 0; l2 < N; ++l2) {
                const size_t q = (size_t)l1 * N + l2;
                if (l1 == l2) {
                    nw[q] = 0.0;
                    dnw[q] = 0.0;
                    continue;
                }
                double g = y[l1] - y[l2], dg = dy[l1] - dy[l2];
                for (int k = 0; k < n; ++k) {
                    const double dx = X[l1 * n + k] - X[l2 * n + k];
                    g -= xi[l2 * n + k] * dx;
                    dg -= dxi[l2 * n + k] * dx + xi[l2 * n + k] * (dX[l1 * n + k] - dX[l2 * n + k]);
                }
                const double v = T2[q] - g * invL;
                nw[q] = v > 0.0 ? v : 0.0;
                dnw[q] = v > 0.0 ? dT2[q] - dg * invL : 0.0;
            }
        }
        for (int64_t l = 0; l < N; ++l) {
            const double v = mu2[l] - y[l] * invL;
            mun[l] = v > 0.0 ? v : 0.0;
            dmun[l] = v > 0.0 ? dmu2[l] - dy[l] * invL : 0.0;
        }
        /* Steps 3-4 */
        const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
        const double beta = (t - 1.0) / tn;
        t = tn;
#pragma omp parallel for schedule(static) if (N >= ORC_PAR_MIN)
        for (int64_t l1 = 0; l1 < N; ++l1)
            for (int64_t l2 = 0; l2 < N; ++l2) {
                const size_t q = (size_t)l1 * N + l2;
                T2[q] = nw[q] + beta * (nw[q] - P[q]);
                dT2[q] = dnw[q] + beta * (dnw[q] - dP[q]);
                P[q] = nw[q];
                dP[q] = dnw[q];
            }
        for (int64_t l = 0; l < N; ++l) {
            mu2[l] = mun[l] + beta * (mun[l] - muP[l]);
            dmu2[l] = dmun[l] + beta * (dmun[l] - dmuP[l]);
            muP[l] = mun[l];
            dmuP[l] = dmun[l];
        }
    }
    /* fitted values at theta^(1)_K = P: yhat = ybar + A_1^T P + muP */
#pragma omp parallel for schedule(static) if (N >= ORC_PAR_MIN)
    for (int64_t l = 0; l < N; ++l) {
        double r = 0.0, dr = 0.0;
        for (int64_t m = 0; m < N; ++m) {
            if (m == l) continue;
            r += P[l * N + m] - P[m * N + l];
            dr += dP[l * N + m] - dP[m * N + l];
        }
        yhat[l] = ybar[l] + r + muP[l];
        dyhat[l] = dybar[l] + dr + dmuP[l];
    }
    free(P); free(T2); free(dP); free(dT2); free(muP); free(mu2); free(dmuP); free(dmu2);
    free(h); free(y); free(dy); free(xi); free(dxi); free(nw); free(dnw); free(mun); free(dmun);
}

/* The same forward-mode derivative for ORC_JD = 8 directions at once (direction index innermost
 * in every tangent array, a fixed count so that the loops over directions vectorize), for sizes
 * where separate runs of orc_papg_jvp would be slow.  Each
 * step and each tangent formula is the one of orc_papg_jvp, evaluated in the same order per
 * (point, direction); only the loops run row-major (column sums walk the rows m in increasing
 * order, as in orc_eta).  dybar: N x 8, dX: N x n x 8 (row-major, directions innermost);
 * dyhat: N x 8. */
#define ORC_JD 8
ORC_API void orc_papg_jvp_multi(const double *X, const double *ybar, int64_t N, int32_t n, double gamma,
                                double L, double s, int64_t K, const double *dybar, const double *dX,
                                double *yhat, double *dyhat)
{
    const size_t NN = (size_t)N * (size_t)N;
    double *P = (double *)calloc(NN, sizeof(double)), *T2 = (double *)calloc(NN, sizeof(double));
    double *dP = (double *)calloc(NN * ORC_JD, sizeof(double)), *dT2 = (double *)calloc(NN * ORC_JD, sizeof(double));
    double *muP = (double *)calloc(N, sizeof(double)), *mu2 = (double *)calloc(N, sizeof(double));
    double *dmuP = (double *)calloc((size_t)N * ORC_JD, sizeof(double)), *dmu2 = (double *)calloc((size_t)N * ORC_JD, sizeof(double));
    double *h = (double *)malloc(sizeof(double) * N), *y = (double *)malloc(sizeof(double) * N);
    double *dy = (double *)malloc(sizeof(double) * N * ORC_JD), *xi = (double *)malloc(sizeof(double) * N * n);
    double *dxi = (double *)malloc(sizeof(double) * N * n * ORC_JD);
    double *rs = (double *)malloc(sizeof(double) * N), *drs = (double *)malloc(sizeof(double) * N * ORC_JD);
    const double invL = 1.0 / L;
    for (int64_t l = 0; l < N; ++l) h[l] = ybar[l] + s;
    double t = 1.0;
    for (int64_t it = 0; it < K; ++it) {
        /* Step 1: row sums of T2 and of its tangents */
#pragma omp parallel for schedule(static) if (N >= ORC_PAR_MIN)
        for (int64_t l = 0; l < N; ++l) {
            double r = 0.0;
            double *dr = drs + (size_t)l * ORC_JD;
            for (int d = 0; d < ORC_JD; ++d) dr[d] = 0.0;
            for (int64_t m = 0; m < N; ++m) {
                if (m == l) continue;
                r += T2[l * N + m];
                const double *dt = dT2 + ((size_t)l * N + m) * ORC_JD;
                for (int d = 0; d < ORC_JD; ++d) dr[d] += dt[d];
            }
            rs[l] = r;
        }
        /* column sums, A_2^T T2 and their tangents: each thread owns a range of columns l and
         * walks the rows m in increasing order */
#pragma omp parallel if (N >= ORC_PAR_MIN)
        {
            int nt = 1, tid = 0;
#ifdef _OPENMP
            nt = omp_get_num_threads();
            tid = omp_get_thread_num();
#endif
            int64_t l0 = N * tid / nt, l1 = N * (tid + 1) / nt;
            int64_t w = l1 - l0 > 0 ? l1 - l0 : 1;
            double *c = (double *)calloc((size_t)w, sizeof(double));
            double *dc = (double *)calloc((size_t)w * ORC_JD, sizeof(double));
            double *ax = (double *)calloc((size_t)w * n, sizeof(double));
            double *dax = (double *)calloc((size_t)w * n * ORC_JD, sizeof(double));
            for (int64_t m = 0; m < N; ++m) {
                const double *xm = X + m * n, *dxm = dX + (size_t)m * n * ORC_JD;
                for (int64_t l = l0; l < l1; ++l) {
                    if (l == m) continue;
                    const double tm = T2[m * N + l];
                    const double *dtm = dT2 + ((size_t)m * N + l) * ORC_JD;
                    const double *xl = X + l * n, *dxl = dX + (size_t)l * n * ORC_JD;
                    c[l - l0] += tm;
                    double *dcl = dc + (size_t)(l - l0) * ORC_JD;
                    for (int d = 0; d < ORC_JD; ++d) dcl[d] += dtm[d];
                    for (int k = 0; k < n; ++k) {
                        const double dxk = xl[k] - xm[k];
                        ax[(l - l0) * n + k] += tm * dxk;
                        double *da = dax + ((size_t)(l - l0) * n + k) * ORC_JD;
                        const double *dxlk = dxl + (size_t)k * ORC_JD, *dxmk = dxm + (size_t)k * ORC_JD;
                        for (int d = 0; d < ORC_JD; ++d) da[d] += dtm[d] * dxk + tm * (dxlk[d] - dxmk[d]);
                    }
                }
            }
            for (int64_t l = l0; l < l1; ++l) {
                y[l] = h[l] + (rs[l] - c[l - l0]) + mu2[l];
                for (int d = 0; d < ORC_JD; ++d)
                    dy[(size_t)l * ORC_JD + d] = dybar[(size_t)l * ORC_JD + d] + (drs[(size_t)l * ORC_JD + d] - dc[(size_t)(l - l0) * ORC_JD + d]) +
                                            dmu2[(size_t)l * ORC_JD + d];
                for (int k = 0; k < n; ++k) {
                    xi[l * n + k] = ax[(l - l0) * n + k] / gamma;
                    for (int d = 0; d < ORC_JD; ++d)
                        dxi[((size_t)l * n + k) * ORC_JD + d] = dax[((size_t)(l - l0) * n + k) * ORC_JD + d] / gamma;
                }
            }
            free(c);
            free(dc);
            free(ax);
            free(dax);
        }
        /* Steps 3-4 scalars (the weight is known before Step 2) */
        const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
        const double beta = (t - 1.0) / tn;
        t = tn;
        /* Step 2 and its tangent, then Step 4 element by element:
         *   new = max(0, T2 - g/L), dnew = [v > 0] (dT2 - dg/L), T2 <- new + beta (new - P), P <- new */
#pragma omp parallel for schedule(static) if (N >= ORC_PAR_MIN)
        for (int64_t l1 = 0; l1 < N; ++l1) {
            const double *dyl1 = dy + (size_t)l1 * ORC_JD, *dxl1 = dX + (size_t)l1 * n * ORC_JD;
            for (int64_t l2 = 0; l2 < N; ++l2) {
                const size_t q = (size_t)l1 * N + l2;
                double *dt2 = dT2 + q * ORC_JD, *dp = dP + q * ORC_JD;
                if (l1 == l2) continue;   /* diagonal: stays 0 with zero tangents */
                const double *dyl2 = dy + (size_t)l2 * ORC_JD, *dxl2 = dX + (size_t)l2 * n * ORC_JD;
                double g = y[l1] - y[l2];
                for (int k = 0; k < n; ++k) g -= xi[l2 * n + k] * (X[l1 * n + k] - X[l2 * n + k]);
                const double v = T2[q] - g * invL;
                const double nw = v > 0.0 ? v : 0.0;
                for (int d = 0; d < ORC_JD; ++d) {
                    double dg = dyl1[d] - dyl2[d];
                    for (int k = 0; k < n; ++k) {
                        const double dx = X[l1 * n + k] - X[l2 * n + k];
                        dg -= dxi[((size_t)l2 * n + k) * ORC_JD + d] * dx +
                              xi[l2 * n + k] * (dxl1[(size_t)k * ORC_JD + d] - dxl2[(size_t)k * ORC_JD + d]);
                    }
                    const double dnw = v > 0.0 ? dt2[d] - dg * invL : 0.0;
                    dt2[d] = dnw + beta * (dnw - dp[d]);
                    dp[d] = dnw;
                }
                T2[q] = nw + beta * (nw - P[q]);
                P[q] = nw;
            }
        }
        for (int64_t l = 0; l < N; ++l) {
            const double v = mu2[l] - y[l] * invL;
            const double nm = v > 0.0 ? v : 0.0;
            for (int d = 0; d < ORC_JD; ++d) {
                const size_t i = (size_t)l * ORC_JD + d;
                const double dnm = v > 0.0 ? dmu2[i] - dy[i] * invL : 0.0;
                dmu2[i] = dnm + beta * (dnm - dmuP[i]);
                dmuP[i] = dnm;
            }
            mu2[l] = nm + beta * (nm - muP[l]);
            muP[l] = nm;
        }
    }
    /* fitted values at theta^(1)_K = P: yhat = ybar + A_1^T P + muP, and their tangents */
#pragma omp parallel for schedule(static) if (N >= ORC_PAR_MIN)
    for (int64_t l = 0; l < N; ++l) {
        double r = 0.0;
        double *dr = dyhat + (size_t)l * ORC_JD;
        for (int d = 0; d < ORC_JD; ++d) dr[d] = 0.0;
        for (int64_t m = 0; m < N; ++m) {
            if (m == l) continue;
            r += P[l * N + m] - P[m * N + l];
            const double *a = dP + ((size_t)l * N + m) * ORC_JD, *b = dP + ((size_t)m * N + l) * ORC_JD;
            for (int d = 0; d < ORC_JD; ++d) dr[d] += a[d] - b[d];
        }
        yhat[l] = ybar[l] + r + muP[l];
        for (int d = 0; d < ORC_JD; ++d) dr[d] = dybar[(size_t)l * ORC_JD + d] + dr[d] + dmuP[(size_t)l * ORC_JD + d];
    }
    free(P); free(T2); free(dP); free(dT2); free(muP); free(mu2); free(dmuP); free(dmu2);
    free(h); free(y); free(dy); free(xi); free(dxi); free(rs); free(drs);
}

/* Threads of the parallel loops from here on (timing the oracle single-threaded); t >= 1. */
ORC_API void orc_set_num_threads(int t)
{
#ifdef _OPENMP
    if (t >= 1) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

ORC_API int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
