/*
 * FP64 CPU oracle of the EM algorithm for a one-dimensional Gaussian mixture
 * (Wang, Chen, Kang & Rahman, arXiv:1601.00704, Sec. 2.2, Eqs. 20-24), used
 * there to split a pore-size distribution into OM and IOM components.
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE (see glbm_oracle.c).
 *
 * One iteration, in the paper's order:
 *   E-step  (Eq. 20, 21): w_j(i) = g_j(x_i) Phi_j / sum_l g_l(x_i) Phi_l,
 *           g_j = exp(-(x - mu_j)^2 / (2 var_j)) / sqrt(2 pi var_j)
 *           (reading: Eq. 21 as printed lacks the minus sign of the exponent)
 *   M-step  (Eq. 22) Phi_j = (1/m) sum_i w_j(i)
 *           (Eq. 23) mu_j  = sum_i w_j(i) x_i / sum_i w_j(i)
 *           (Eq. 24) var_j = sum_i w_j(i) (x_i - mu_j)^2 / sum_i w_j(i),
 *                    with the mu_j just updated (reading).
 * Iterations stop after max_iter, or when the mean log-likelihood of the
 * data (evaluated in the E-step) changes by less than tol.
 *
 * Pins (tests/test_oracle_em.py): recovery of the two-cluster test mixture of
 * the paper's validation table within sampling error; one component reduces
 * to the sample mean and the biased variance; the log-likelihood never
 * decreases; the fractions sum to one.
 */
#include <math.h>
#include <stdlib.h>

static const double TWO_PI = 6.28318530717958647692;

/* Returns the number of iterations done; phi/mu/var hold the initial guess
 * on entry and the estimate on exit; loglik (may be NULL) receives the mean
 * log-likelihood of the last E-step.  -1 on bad arguments. */
int orc_em_gmm1d(const double *x, long m, int k, double *phi, double *mu,
                 double *var, int max_iter, double tol, double *loglik) {
    if (m < 1 || k < 1 || max_iter < 0) return -1;
    double *w = (double *)malloc(sizeof(double) * (size_t)m * k);
    if (!w) return -1;
    double prev = -INFINITY, ll = -INFINITY;
    int it = 0;
    for (; it < max_iter; ++it) {
        /* E-step */
        ll = 0.0;
        for (long i = 0; i < m; ++i) {
            double den = 0.0;
            for (int j = 0; j < k; ++j) {
                const double d = x[i] - mu[j];
                const double g = exp(-d * d / (2.0 * var[j])) / sqrt(TWO_PI * var[j]);
                w[i * k + j] = g * phi[j];
                den += w[i * k + j];
            }
            for (int j = 0; j < k; ++j) w[i * k + j] /= den;
            ll += log(den);
        }
        ll /= (double)m;
        /* M-step */
        for (int j = 0; j < k; ++j) {
            double sw = 0.0, swx = 0.0;
            for (long i = 0; i < m; ++i) {
                sw += w[i * k + j];
                swx += w[i * k + j] * x[i];
            }
            phi[j] = sw / (double)m;
            mu[j] = swx / sw;
            double swd = 0.0;
            for (long i = 0; i < m; ++i) {
                const double d = x[i] - mu[j];
                swd += w[i * k + j] * d * d;
            }
            var[j] = swd / sw;
        }
        if (tol > 0.0 && fabs(ll - prev) < tol) {
            ++it;
            break;
        }
        prev = ll;
    }
    free(w);
    if (loglik) *loglik = ll;
    return it;
}
