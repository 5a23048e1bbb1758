/*
 * irbc_oracle.c -- TEST INFRASTRUCTURE, NOT PRODUCT CODE.
 *
 * Plain FP64 CPU restatement of the smooth IRBC model's equilibrium
 * conditions (Eftekhari & Scheidegger, arXiv 2202.06555, Sec. 2.1: eq.
 * law_of_motion, eq. model1, eq. model2, Table 1) with the expectation taken
 * by a degree-3 monomial rule (the paper's footnote to Sec. 2.1 cites Judd's
 * monomial rules), evaluated through the oracle's own brute-force DDSG
 * interpolant (ddsg_oracle.c). Only tests/, smoke() and bench.py's CPU
 * baseline may use it.
 *
 * State x = (a_1..a_N, k_1..k_N); policy p(x) = (k'_1..k'_N, lambda).
 * Parameters prm[] = {beta, alpha, delta, sigma, rho, phi, A}; gamma[N], tau[N].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define KMAX 8

void orc_eval(int d, int m, int C, const int32_t *comp_k, const int32_t *comp_dims,
              const int64_t *comp_off, const uint8_t *levels, const uint32_t *indices,
              const double *alpha, const double *b, const double *lo, const double *hi,
              int form, int64_t n, const double *x, double *y, double *S,
              uint64_t *hash, int32_t *count);

/* Table 1: A = (1 - beta (1 - delta)) / (alpha beta); gamma_j = a + 0.75 (j-1)/(N-1)
 * (j = 1..N; gamma = a when N = 1); tau_j = A^(1/gamma_j). */
void orc_irbc_params(int N, double a_gamma, double beta, double alpha, double delta,
                     double *A, double *gamma, double *tau)
{
    *A = (1.0 - beta * (1.0 - delta)) / (alpha * beta);
    for (int j = 0; j < N; ++j) {
        gamma[j] = N > 1 ? a_gamma + 0.75 * (double)j / (double)(N - 1) : a_gamma;
        tau[j] = pow(*A, 1.0 / gamma[j]);
    }
}

/* Degree-3 monomial rule for n independent N(0,1) shocks: 2n nodes
 * +-sqrt(n) e_i, each with weight 1/(2n). nodes: 2n x n (node 2i is +, 2i+1 is -). */
void orc_monomial_nodes(int n, double *nodes, double *weights)
{
    const double h = sqrt((double)n);
    for (int q = 0; q < 2 * n; ++q) {
        for (int j = 0; j < n; ++j) nodes[q * n + j] = 0.0;
        nodes[q * n + q / 2] = (q % 2 == 0) ? h : -h;
        weights[q] = 1.0 / (2.0 * n);
    }
}

/*
 * Residuals of eq. model1 (N Euler equations) and eq. model2 (aggregate
 * resource constraint) at ns states for the policy guess (k', lambda), with
 * next-period policies interpolated from the DDSG tables (paper form 0 or
 * slice-free form 1). Next-period productivity by eq. law_of_motion at the
 * 2(N+1) monomial nodes (shocks e_1..e_N, e); the next state (a', k') is
 * clamped to the policy's domain by the interpolant only -- a' itself enters
 * the marginal product unclamped.
 *   resid: ns x (N+1). euler_err (nullable): ns x 2, the unit-free Euler error
 *   max_j |beta E_j / (lambda (1 + phi g_j)) - 1| and |resource| / sum_j Y_j.
 */
void orc_irbc_residual(int N, const double *prm, const double *gamma, const double *tau,
                       int C, const int32_t *comp_k, const int32_t *comp_dims,
                       const int64_t *comp_off, const uint8_t *levels, const uint32_t *indices,
                       const double *alpha_tab, const double *b, const double *lo,
                       const double *hi, int form, int64_t ns, const double *states,
                       const double *guess, double *resid, double *euler_err)
{
    const double beta = prm[0], alpha = prm[1], delta = prm[2], sigma = prm[3], rho = prm[4],
                 phi = prm[5], A = prm[6];
    const int d = 2 * N, m = N + 1, nq = 2 * (N + 1);
    double *nodes = (double *)malloc(sizeof(double) * (size_t)nq * (N + 1));
    double *wts = (double *)malloc(sizeof(double) * (size_t)nq);
    double *xq = (double *)malloc(sizeof(double) * (size_t)nq * d);
    double *pq = (double *)malloc(sizeof(double) * (size_t)nq * m);
    orc_monomial_nodes(N + 1, nodes, wts);
    for (int64_t s = 0; s < ns; ++s) {
        const double *a = &states[s * d];
        const double *k = &states[s * d + N];
        const double *kp = &guess[s * m];
        const double lam = guess[s * m + N];
        for (int q = 0; q < nq; ++q) {
            const double eg = nodes[q * (N + 1) + N];
            for (int j = 0; j < N; ++j) {
                xq[q * d + j] = exp(rho * log(a[j]) + sigma * (nodes[q * (N + 1) + j] + eg));
                xq[q * d + N + j] = kp[j];
            }
        }
        orc_eval(d, m, C, comp_k, comp_dims, comp_off, levels, indices, alpha_tab, b, lo, hi, form,
                 nq, xq, pq, NULL, NULL, NULL);
        double res = 0.0, ysum = 0.0, emax = 0.0;
        for (int j = 0; j < N; ++j) {
            const double g1 = kp[j] / k[j] - 1.0;
            double E = 0.0;
            for (int q = 0; q < nq; ++q) {
                const double g2 = pq[q * m + j] / kp[j] - 1.0;
                const double lamp = pq[q * m + N];
                E += wts[q] * lamp *
                     (xq[q * d + j] * A * alpha * pow(kp[j], alpha - 1.0) + (1.0 - delta) +
                      0.5 * phi * g2 * (g2 + 2.0));
            }
            const double lhs = lam * (1.0 + phi * g1);
            resid[s * m + j] = lhs - beta * E;
            const double e = fabs(beta * E / lhs - 1.0);
            if (e > emax) emax = e;
            const double Y = a[j] * A * pow(k[j], alpha);
            ysum += Y;
            res += Y + k[j] * ((1.0 - delta) - 0.5 * phi * g1 * g1) - kp[j] - pow(lam / tau[j], -gamma[j]);
        }
        resid[s * m + N] = res;
        if (euler_err) {
            euler_err[s * 2 + 0] = emax;
            euler_err[s * 2 + 1] = fabs(res) / ysum;
        }
    }
    free(nodes);
    free(wts);
    free(xq);
    free(pq);
}

/* Fischer-Burmeister function: zero iff a >= 0, b >= 0, a b = 0. */
static double fb(double a, double b) { return a + b - sqrt(a * a + b * b); }

/* Non-smooth IRBC (irreversible investment, eq. modelkink1 with the aggregate
 * resource constraint eq. model2). The policy maps x = (a, k) to
 * (k'_1..k'_N, mu_1..mu_N, lambda) (m = 2N+1); guess rows likewise.
 * Residual rows: j < N the Euler equation of country j,
 *   lambda (1 + phi g'_j) - mu_j - beta E[lambda' (a'_j A alpha k'^(alpha-1) + 1 - delta
 *        + phi/2 g''_j (g''_j + 2)) - (1 - delta) mu'_j],
 * N + j the complementarity 0 <= mu_j _|_ (k'_j - (1 - delta) k_j) >= 0 written
 * as FB(mu_j, k'_j - (1 - delta) k_j) = 0, and 2N the resource constraint.
 * euler_err (optional, ns x 2): max_j |beta E_j / (lambda (1 + phi g'_j) - mu_j) - 1|
 * and |resource| / sum_j Y_j. Next states are clamped to [lo, hi] inside the
 * interpolation, as in the smooth model. */
void orc_irbc_residual_irr(int N, const double *prm, const double *gamma, const double *tau,
                           int C, const int32_t *comp_k, const int32_t *comp_dims,
                           const int64_t *comp_off, const uint8_t *levels, const uint32_t *indices,
                           const double *alpha_tab, const double *b, const double *lo,
                           const double *hi, int form, int64_t ns, const double *states,
                           const double *guess, double *resid, double *euler_err)
{
    const double beta = prm[0], alpha = prm[1], delta = prm[2], sigma = prm[3], rho = prm[4],
                 phi = prm[5], A = prm[6];
    const int d = 2 * N, m = 2 * N + 1, nq = 2 * (N + 1);
    double *nodes = (double *)malloc(sizeof(double) * (size_t)nq * (N + 1));
    double *wts = (double *)malloc(sizeof(double) * (size_t)nq);
    double *xq = (double *)malloc(sizeof(double) * (size_t)nq * d);
    double *pq = (double *)malloc(sizeof(double) * (size_t)nq * m);
    orc_monomial_nodes(N + 1, nodes, wts);
    for (int64_t s = 0; s < ns; ++s) {
        const double *a = &states[s * d];
        const double *k = &states[s * d + N];
        const double *kp = &guess[s * m];
        const double *mu = &guess[s * m + N];
        const double lam = guess[s * m + 2 * N];
        for (int q = 0; q < nq; ++q) {
            const double eg = nodes[q * (N + 1) + N];
            for (int j = 0; j < N; ++j) {
                xq[q * d + j] = exp(rho * log(a[j]) + sigma * (nodes[q * (N + 1) + j] + eg));
                xq[q * d + N + j] = kp[j];
            }
        }
        orc_eval(d, m, C, comp_k, comp_dims, comp_off, levels, indices, alpha_tab, b, lo, hi, form,
                 nq, xq, pq, NULL, NULL, NULL);
        double res = 0.0, ysum = 0.0, emax = 0.0;
        for (int j = 0; j < N; ++j) {
            const double g1 = kp[j] / k[j] - 1.0;
            double E = 0.0;
            for (int q = 0; q < nq; ++q) {
                const double g2 = pq[q * m + j] / kp[j] - 1.0;
                const double lamp = pq[q * m + 2 * N];
                const double mup = pq[q * m + N + j];
                E += wts[q] * (lamp * (xq[q * d + j] * A * alpha * pow(kp[j], alpha - 1.0) + (1.0 - delta) +
                                       0.5 * phi * g2 * (g2 + 2.0)) -
                               (1.0 - delta) * mup);
            }
            const double lhs = lam * (1.0 + phi * g1) - mu[j];
            resid[s * m + j] = lhs - beta * E;
            resid[s * m + N + j] = fb(mu[j], kp[j] - (1.0 - delta) * k[j]);
            const double e = fabs(beta * E / lhs - 1.0);
            if (e > emax) emax = e;
            const double Y = a[j] * A * pow(k[j], alpha);
            ysum += Y;
            res += Y + k[j] * ((1.0 - delta) - 0.5 * phi * g1 * g1) - kp[j] - pow(lam / tau[j], -gamma[j]);
        }
        resid[s * m + 2 * N] = res;
        if (euler_err) {
            euler_err[s * 2 + 0] = emax;
            euler_err[s * 2 + 1] = fabs(res) / ysum;
        }
    }
    free(nodes);
    free(wts);
    free(xq);
    free(pq);
}

/* Dense LU with partial pivoting and solve (row-major n x n), in place.
 * Returns 0, or -1 if a pivot is exactly zero. */
int orc_lu_solve(int n, double *Amat, double *rhs)
{
    for (int c = 0; c < n; ++c) {
        int p = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(Amat[r * n + c]) > fabs(Amat[p * n + c])) p = r;
        if (Amat[p * n + c] == 0.0) return -1;
        if (p != c) {
            for (int j = 0; j < n; ++j) {
                double t = Amat[c * n + j];
                Amat[c * n + j] = Amat[p * n + j];
                Amat[p * n + j] = t;
            }
            double t = rhs[c];
            rhs[c] = rhs[p];
            rhs[p] = t;
        }
        for (int r = c + 1; r < n; ++r) {
            const double f = Amat[r * n + c] / Amat[c * n + c];
            Amat[r * n + c] = f;
            for (int j = c + 1; j < n; ++j) Amat[r * n + j] -= f * Amat[c * n + j];
            rhs[r] -= f * rhs[c];
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        double s = rhs[r];
        for (int j = r + 1; j < n; ++j) s -= Amat[r * n + j] * rhs[j];
        rhs[r] = s / Amat[r * n + r];
    }
    return 0;
}
