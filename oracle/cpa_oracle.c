/*
 * FP64 CPU oracle for CPA-based singular value shrinkage
 * (Onuki et al., "Fast Singular Value Shrinkage with Chebyshev Polynomial
 * Approximation Based on Signal Sparsity", arXiv 1705.07112).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant with the CUDA library; the product path never
 * calls it.
 *
 * Everything is plain FP64 with plain loops in the order the paper states the
 * steps: no blocking, no fusion, no reordering.  Matrices are row-major,
 * dense, with leading dimension equal to the column count.
 *
 * Notation (the paper's): B is the m x n input (called X here), g the scalar
 * shrinkage on singular values, h(x) = g(sqrt x)/sqrt x the filter on the
 * eigenvalues of the Gram matrix, alpha the number of Chebyshev terms
 * (k = 0..alpha-1), c_k the shifted Chebyshev coefficients, Lambda_max the
 * interval bound, B_hat = (2/Lambda_max) Phi - Id the shifted Gram matrix and
 * Psi_k(B_hat) the matrix Chebyshev polynomials.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846

#define ORC_HARD 0
#define ORC_SOFT 1
#define ORC_WSOFT 2

/* ------------------------------------------------------------------------- */
/* Shrinkage responses (Section IV-A, Eq. filter_response_ours).             */
/*                                                                           */
/* The generic response is h(x; W, tau) = (sqrt x - W)/sqrt x when           */
/* sqrt x > tau and 0 otherwise, with                                        */
/*   hard:          W = 0,        tau = tau_hard                             */
/*   soft:          W = tau,      tau = tau          (tau = 1/rho)           */
/*   weighted soft: W = w(x),     tau = w(x)                                 */
/* The weight of the weighted soft response is a function of x = sigma^2:    */
/*   w(x) = c / (sigma_est + eps),  sigma_est = sqrt(max(x - noise, 0)),     */
/* i.e. a weight inversely proportional to an estimate of the signal part of */
/* the singular value (noise = expected noise energy per singular value).    */
/* ------------------------------------------------------------------------- */
static void response_params(int kind, double tau, double c, double eps,
                            double noise, double x, double *W, double *thr)
{
    if (kind == ORC_HARD) {
        *W = 0.0;
        *thr = tau;
    } else if (kind == ORC_SOFT) {
        *W = tau;
        *thr = tau;
    } else {
        double s2 = x - noise;
        double sest = s2 > 0.0 ? sqrt(s2) : 0.0;
        double w = c / (sest + eps);
        *W = w;
        *thr = w;
    }
}

/* h(x) on the eigenvalue axis (x = sigma^2 >= 0). */
double orc_h(int kind, double tau, double c, double eps, double noise, double x)
{
    double W, thr;
    double r = x > 0.0 ? sqrt(x) : 0.0;
    response_params(kind, tau, c, eps, noise, x, &W, &thr);
    if (r > thr)
        return (r - W) / r;
    return 0.0;
}

/* g(sigma) = sigma * h(sigma^2): the singular-value shrinkage (Eq.
 * sing_shrink_from_eig_shrink, g(sqrt x) = sqrt x h(x)). */
double orc_g(int kind, double tau, double c, double eps, double noise, double sigma)
{
    if (sigma <= 0.0)
        return 0.0;
    return sigma * orc_h(kind, tau, c, eps, noise, sigma * sigma);
}

/* ------------------------------------------------------------------------- */
/* Chebyshev approximation (Section II-B).                                   */
/* ------------------------------------------------------------------------- */

/* Shifted Chebyshev coefficients, Eq. chebychev_coeff_shifted:
 *   c_k = (2/alpha) sum_{l=1}^{alpha} cos(k theta_l) h(lam/2 (cos theta_l + 1)),
 *   theta_l = pi (l - 1/2) / alpha,   k = 0..alpha-1. */
void orc_coeffs(int kind, double tau, double c, double eps, double noise,
                int alpha, double lam, double *ck)
{
    for (int k = 0; k < alpha; k++) {
        double s = 0.0;
        for (int l = 1; l <= alpha; l++) {
            double th = ORC_PI * ((double)l - 0.5) / (double)alpha;
            double x = 0.5 * lam * (cos(th) + 1.0);
            s += cos((double)k * th) * orc_h(kind, tau, c, eps, noise, x);
        }
        ck[k] = 2.0 / (double)alpha * s;
    }
}

/* Unshifted coefficients of a function given by its samples at the
 * Chebyshev nodes, Eq. chebychev_coeff_discrete: hs[l-1] = h(cos theta_l). */
void orc_coeffs_from_nodes(int alpha, const double *hs, double *ck)
{
    for (int k = 0; k < alpha; k++) {
        double s = 0.0;
        for (int l = 1; l <= alpha; l++) {
            double th = ORC_PI * ((double)l - 0.5) / (double)alpha;
            s += cos((double)k * th) * hs[l - 1];
        }
        ck[k] = 2.0 / (double)alpha * s;
    }
}

/* Truncated Chebyshev series on [-1,1], Eq. chebychev_series, with the
 * polynomials taken from their trigonometric definition, Eq.
 * chebychev_polynomial: psi_k(x) = cos(k arccos x). */
double orc_series_cos(const double *ck, int alpha, double x)
{
    double t = acos(x);
    double s = 0.5 * ck[0];
    for (int k = 1; k < alpha; k++)
        s += ck[k] * cos((double)k * t);
    return s;
}

/* The same series with the polynomials from the three-term recurrence,
 * Eq. chebyche2: psi_0 = 1, psi_1 = x, psi_k = 2 x psi_{k-1} - psi_{k-2}. */
double orc_series_rec(const double *ck, int alpha, double x)
{
    double pm2 = 1.0, pm1 = x;
    double s = 0.5 * ck[0];
    if (alpha > 1)
        s += ck[1] * pm1;
    for (int k = 2; k < alpha; k++) {
        double pk = 2.0 * x * pm1 - pm2;
        s += ck[k] * pk;
        pm2 = pm1;
        pm1 = pk;
    }
    return s;
}

/* Chebyshev polynomial psi_k(x) by the recurrence (for pin tests). */
double orc_cheb_T(int k, double x)
{
    if (k == 0)
        return 1.0;
    double pm2 = 1.0, pm1 = x;
    for (int j = 2; j <= k; j++) {
        double pk = 2.0 * x * pm1 - pm2;
        pm2 = pm1;
        pm1 = pk;
    }
    return pm1;
}

/* ------------------------------------------------------------------------- */
/* Dense helpers.                                                            */
/* ------------------------------------------------------------------------- */

/* C (M x N) = A (M x K) * B (K x N), plain loops, sum in k order. */
static void matmul(const double *A, const double *B, double *C, int M, int K, int N)
{
    for (int i = 0; i < M; i++) {
        double *ci = C + (size_t)i * N;
        for (int j = 0; j < N; j++)
            ci[j] = 0.0;
        for (int k = 0; k < K; k++) {
            double a = A[(size_t)i * K + k];
            const double *bk = B + (size_t)k * N;
            for (int j = 0; j < N; j++)
                ci[j] += a * bk[j];
        }
    }
}

static void transpose(const double *A, double *At, int M, int N)
{
    for (int i = 0; i < M; i++)
        for (int j = 0; j < N; j++)
            At[(size_t)j * M + i] = A[(size_t)i * N + j];
}

/* Gram matrix of the smaller side (the Gram step of Algorithm 1, T = Id):
 * m >= n: G = X^T X (n x n);  m < n: G = X X^T (m x m). */
void orc_gram(const double *X, int m, int n, double *G)
{
    if (m >= n) {
        for (int i = 0; i < n; i++)
            for (int j = 0; j < n; j++) {
                double s = 0.0;
                for (int r = 0; r < m; r++)
                    s += X[(size_t)r * n + i] * X[(size_t)r * n + j];
                G[(size_t)i * n + j] = s;
            }
    } else {
        for (int i = 0; i < m; i++)
            for (int j = 0; j < m; j++) {
                double s = 0.0;
                for (int r = 0; r < n; r++)
                    s += X[(size_t)i * n + r] * X[(size_t)j * n + r];
                G[(size_t)i * m + j] = s;
            }
    }
}

/* Transformed Gram matrix Phi = T G T^T of the smaller side (Eq.
 * sing_shrink_exact_sparse), before any entry threshold; T NULL = Id. */
void orc_phi(const double *X, int m, int n, const double *T, double *Phi)
{
    int p = m < n ? m : n;
    size_t pp = (size_t)p * p;
    orc_gram(X, m, n, Phi);
    if (T) {
        double *Tt = malloc(pp * sizeof(double));
        double *tmp = malloc(pp * sizeof(double));
        transpose(T, Tt, p, p);
        matmul(T, Phi, tmp, p, p, p);
        matmul(tmp, Tt, Phi, p, p, p);
        free(Tt);
        free(tmp);
    }
}

/* ------------------------------------------------------------------------- */
/* Algorithm 1: CPA-based singular value shrinkage, dense.                   */
/*                                                                           */
/* X: m x n.  T: optional p x p orthogonal (or masked) transform, NULL = Id. */
/* eps_thr: entry threshold of Eq. threshold_components (|Phi_ij| >= eps     */
/* kept); a negative value disables the thresholding.  lam: Lambda_max,      */
/* supplied by the caller.  Y: m x n output.  Hout (optional): the p x p     */
/* matrix H_hat(Phi_) of Eq. chebychev_series_matrix.                        */
/*                                                                           */
/* For m < n the paper's m > n statement is applied to X^T and transposed    */
/* back: G_hat(X) = T^T H_hat(T X X^T T^T) T X.                              */
/* ------------------------------------------------------------------------- */
static int cpa_scheme(const double *X, int m, int n, int kind, double tau, double c,
                      double eps, double noise, int alpha, double lam, const double *T,
                      double eps_thr, double *Y, double *Hout, int clenshaw);

int orc_cpa(const double *X, int m, int n, int kind, double tau, double c,
            double eps, double noise, int alpha, double lam, const double *T,
            double eps_thr, double *Y, double *Hout)
{
    return cpa_scheme(X, m, n, kind, tau, c, eps, noise, alpha, lam, T, eps_thr, Y, Hout, 0);
}

/* The same filter H_hat = c_0/2 Id + sum_{k>=1} c_k T_k(B_hat) summed by
 * Clenshaw's recurrence (Clenshaw, 1955) instead of the forward one:
 *   b_alpha = b_{alpha+1} = 0,  b_k = c_k Id + 2 B_hat b_{k+1} - b_{k+2}
 *   (k = alpha-1 .. 0),  H_hat = (b_0 - b_2) / 2.
 * Same number of products; the sum needs no running accumulator. */
int orc_cpa_clenshaw(const double *X, int m, int n, int kind, double tau, double c,
                     double eps, double noise, int alpha, double lam, const double *T,
                     double eps_thr, double *Y, double *Hout)
{
    return cpa_scheme(X, m, n, kind, tau, c, eps, noise, alpha, lam, T, eps_thr, Y, Hout, 1);
}

static int cpa_scheme(const double *X, int m, int n, int kind, double tau, double c,
                      double eps, double noise, int alpha, double lam, const double *T,
                      double eps_thr, double *Y, double *Hout, int clenshaw)
{
    if (alpha < 1 || !(lam > 0.0))
        return 1;
    int p = m < n ? m : n;
    size_t pp = (size_t)p * p;
    double *Phi = malloc(pp * sizeof(double));
    double *Bh = malloc(pp * sizeof(double));
    double *Pm2 = malloc(pp * sizeof(double));
    double *Pm1 = malloc(pp * sizeof(double));
    double *Pk = malloc(pp * sizeof(double));
    double *H = malloc(pp * sizeof(double));
    double *tmp = malloc(pp * sizeof(double));
    double *ck = malloc((size_t)alpha * sizeof(double));

    /* Gram step: Phi = T G T^T */
    orc_gram(X, m, n, Phi);
    if (T) {
        double *Tt = malloc(pp * sizeof(double));
        transpose(T, Tt, p, p);
        matmul(T, Phi, tmp, p, p, p);
        matmul(tmp, Tt, Phi, p, p, p);
        free(Tt);
    }
    /* sparsification: Phi_ by entry thresholding (Eq. threshold_components) */
    if (eps_thr >= 0.0)
        for (size_t e = 0; e < pp; e++)
            if (!(fabs(Phi[e]) >= eps_thr))
                Phi[e] = 0.0;
    /* interval bound: Lambda_max is the caller's lam */
    /* coefficients, Eq. chebychev_coeff_shifted */
    orc_coeffs(kind, tau, c, eps, noise, alpha, lam, ck);
    /* shift: B_hat = (2/Lambda_max) Phi_ - Id */
    for (int i = 0; i < p; i++)
        for (int j = 0; j < p; j++)
            Bh[(size_t)i * p + j] = 2.0 / lam * Phi[(size_t)i * p + j] - (i == j ? 1.0 : 0.0);
    if (!clenshaw) {
        /* initial polynomials: Psi_0 = Id, Psi_1 = B_hat */
        for (int i = 0; i < p; i++)
            for (int j = 0; j < p; j++)
                Pm2[(size_t)i * p + j] = (i == j ? 1.0 : 0.0);
        memcpy(Pm1, Bh, pp * sizeof(double));
        /* initial sum: H = c_0/2 Psi_0 + c_1 Psi_1 */
        for (size_t e = 0; e < pp; e++)
            H[e] = 0.5 * ck[0] * Pm2[e] + (alpha > 1 ? ck[1] * Pm1[e] : 0.0);
        /* recurrence (Eq. recurrence_our_method) with accumulation:
         * Psi_k = 2 B_hat Psi_{k-1} - Psi_{k-2};  H += c_k Psi_k,  k = 2..alpha-1 */
        for (int k = 2; k < alpha; k++) {
            matmul(Bh, Pm1, tmp, p, p, p);
            for (size_t e = 0; e < pp; e++) {
                Pk[e] = 2.0 * tmp[e] - Pm2[e];
                H[e] += ck[k] * Pk[e];
            }
            double *r = Pm2;
            Pm2 = Pm1;
            Pm1 = Pk;
            Pk = r;
        }
    } else {
        /* Clenshaw: Pm1 = b_{k+1}, Pm2 = b_{k+2}, both zero at k = alpha - 1 */
        for (size_t e = 0; e < pp; e++) {
            Pm1[e] = 0.0;
            Pm2[e] = 0.0;
        }
        for (int k = alpha - 1; k >= 0; k--) {
            matmul(Bh, Pm1, tmp, p, p, p);
            for (int i = 0; i < p; i++)
                for (int j = 0; j < p; j++) {
                    size_t e = (size_t)i * p + j;
                    Pk[e] = (i == j ? ck[k] : 0.0) + 2.0 * tmp[e] - Pm2[e];
                }
            double *r = Pm2;   /* b_{k+2} <- b_{k+1}, b_{k+1} <- b_k */
            Pm2 = Pm1;
            Pm1 = Pk;
            Pk = r;
        }
        /* now Pm1 = b_0, Pm2 = b_1: the closing step of Clenshaw's
         * recurrence, sum_k c_k T_k = b_0 - B_hat b_1, less c_0/2 Id for
         * the halved first term */
        matmul(Bh, Pm2, tmp, p, p, p);
        for (int i = 0; i < p; i++)
            for (int j = 0; j < p; j++) {
                size_t e = (size_t)i * p + j;
                H[e] = Pm1[e] - tmp[e] - (i == j ? 0.5 * ck[0] : 0.0);
            }
    }
    /* final product (Eq. SVD_fil): G_hat = B T^T H T  (m >= n);  T^T H T B  (m < n) */
    double *F = H;
    if (T) {
        double *Tt = malloc(pp * sizeof(double));
        transpose(T, Tt, p, p);
        matmul(Tt, H, tmp, p, p, p);
        matmul(tmp, T, Bh, p, p, p); /* Bh reused as T^T H T */
        F = Bh;
        free(Tt);
    }
    if (m >= n)
        matmul(X, F, Y, m, n, n);
    else
        matmul(F, X, Y, m, m, n);
    if (Hout)
        memcpy(Hout, F, pp * sizeof(double));

    free(Phi); free(Bh); free(Pm2); free(Pm1); free(Pk); free(H); free(tmp); free(ck);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Vector form of the same filter (Eq. prop_another_form):                   */
/*   out = H_hat(G) v  with G the Gram matrix of the smaller side,           */
/* computed by the same recurrence applied to v, G v formed as X^T (X v)     */
/* (m >= n) or X (X^T v) (m < n) without forming G.  Row i of X H_hat(X^T X) */
/* is (H_hat(X^T X) x_i)^T and column j of H_hat(X X^T) X is H_hat(X X^T) x_j,*/
/* so sampled outputs of Algorithm 1 at any size come from this function.    */
/* T = Id, no entry thresholding.                                            */
/* ------------------------------------------------------------------------- */
static void gram_vec(const double *X, int m, int n, const double *v, double *out, double *work)
{
    if (m >= n) { /* out = X^T (X v), v in R^n, work in R^m */
        for (int r = 0; r < m; r++) {
            double s = 0.0;
            for (int j = 0; j < n; j++)
                s += X[(size_t)r * n + j] * v[j];
            work[r] = s;
        }
        for (int j = 0; j < n; j++)
            out[j] = 0.0;
        for (int r = 0; r < m; r++)
            for (int j = 0; j < n; j++)
                out[j] += X[(size_t)r * n + j] * work[r];
    } else { /* out = X (X^T v), v in R^m, work in R^n */
        for (int j = 0; j < n; j++)
            work[j] = 0.0;
        for (int r = 0; r < m; r++)
            for (int j = 0; j < n; j++)
                work[j] += X[(size_t)r * n + j] * v[r];
        for (int r = 0; r < m; r++) {
            double s = 0.0;
            for (int j = 0; j < n; j++)
                s += X[(size_t)r * n + j] * work[j];
            out[r] = s;
        }
    }
}

int orc_cpa_vec(const double *X, int m, int n, int kind, double tau, double c,
                double eps, double noise, int alpha, double lam,
                const double *v, double *out)
{
    if (alpha < 1 || !(lam > 0.0))
        return 1;
    int p = m < n ? m : n;
    int q = m < n ? n : m;
    double *ck = malloc((size_t)alpha * sizeof(double));
    double *zm2 = malloc((size_t)p * sizeof(double));
    double *zm1 = malloc((size_t)p * sizeof(double));
    double *zk = malloc((size_t)p * sizeof(double));
    double *gz = malloc((size_t)p * sizeof(double));
    double *work = malloc((size_t)q * sizeof(double));
    orc_coeffs(kind, tau, c, eps, noise, alpha, lam, ck);
    /* z_0 = v, z_1 = B_hat v = (2/lam) G v - v */
    memcpy(zm2, v, (size_t)p * sizeof(double));
    gram_vec(X, m, n, zm2, gz, work);
    for (int i = 0; i < p; i++)
        zm1[i] = 2.0 / lam * gz[i] - zm2[i];
    for (int i = 0; i < p; i++)
        out[i] = 0.5 * ck[0] * zm2[i] + (alpha > 1 ? ck[1] * zm1[i] : 0.0);
    for (int k = 2; k < alpha; k++) {
        gram_vec(X, m, n, zm1, gz, work);
        for (int i = 0; i < p; i++) {
            double bz = 2.0 / lam * gz[i] - zm1[i]; /* B_hat z_{k-1} */
            zk[i] = 2.0 * bz - zm2[i];
            out[i] += ck[k] * zk[i];
        }
        double *r = zm2;
        zm2 = zm1;
        zm1 = zk;
        zk = r;
    }
    free(ck); free(zm2); free(zm1); free(zk); free(gz); free(work);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Lambda_max bound (the interval step of Algorithm 1; the paper names no   */
/* method for it).                                                           */
/*                                                                           */
/* Power iteration on the Gram matrix G of the smaller side from the start   */
/* vector v0 (p entries, need not be normalised): `iters` products           */
/* v <- G v / |G v|, then one more product w = G v giving the Rayleigh       */
/* quotient theta = v.w and the residual r = |w - theta v|.  The bound is    */
/*   lam = min((theta + r) (1 + margin), trace G),                           */
/* trace G = |X|_F^2 being a rigorous upper bound of the largest eigenvalue  */
/* of a PSD matrix.  out = {theta, r, trace, lam}.                           */
/* ------------------------------------------------------------------------- */
int orc_lambda_bound(const double *X, int m, int n, int iters, double margin,
                     const double *v0, double *out)
{
    int p = m < n ? m : n;
    int q = m < n ? n : m;
    double *v = malloc((size_t)p * sizeof(double));
    double *w = malloc((size_t)p * sizeof(double));
    double *work = malloc((size_t)q * sizeof(double));
    double nv = 0.0;
    for (int i = 0; i < p; i++)
        nv += v0[i] * v0[i];
    nv = sqrt(nv);
    if (!(nv > 0.0)) {
        free(v); free(w); free(work);
        return 1;
    }
    for (int i = 0; i < p; i++)
        v[i] = v0[i] / nv;
    for (int t = 0; t < iters; t++) {
        gram_vec(X, m, n, v, w, work);
        double nw = 0.0;
        for (int i = 0; i < p; i++)
            nw += w[i] * w[i];
        nw = sqrt(nw);
        if (!(nw > 0.0))
            break; /* v in the null space: keep v, theta will be 0 */
        for (int i = 0; i < p; i++)
            v[i] = w[i] / nw;
    }
    gram_vec(X, m, n, v, w, work);
    double th = 0.0;
    for (int i = 0; i < p; i++)
        th += v[i] * w[i];
    double r2 = 0.0;
    for (int i = 0; i < p; i++)
        r2 += (w[i] - th * v[i]) * (w[i] - th * v[i]);
    double tr = 0.0;
    for (size_t e = 0; e < (size_t)m * n; e++)
        tr += X[e] * X[e];
    double lam = (th + sqrt(r2)) * (1.0 + margin);
    if (lam > tr)
        lam = tr;
    out[0] = th;
    out[1] = sqrt(r2);
    out[2] = tr;
    out[3] = lam;
    free(v); free(w); free(work);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* One-sided Jacobi SVD (Hestenes).  X: m x n with m >= n (callers transpose */
/* otherwise).  On return W (m x n) holds X V, whose columns are sigma_i u_i,*/
/* V (n x n) the right singular vectors as columns, s the singular values    */
/* (column norms of W, unsorted).  Sweeps rotate every column pair (i,j)     */
/* until every pair is orthogonal to within tol relative to its norms.       */
/* Returns the number of sweeps, or -1 if max_sweeps was hit.                */
/* ------------------------------------------------------------------------- */
int orc_svd_jacobi(const double *X, int m, int n, double *W, double *V, double *s,
                   double tol, int max_sweeps)
{
    if (m < n)
        return -2;
    memcpy(W, X, (size_t)m * n * sizeof(double));
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++)
            V[(size_t)i * n + j] = (i == j ? 1.0 : 0.0);
    /* columns whose norm is at the rounding level of the whole matrix
     * (numerically zero singular values) are not rotated against each
     * other: their inner products are noise and never meet the relative
     * test */
    double fro2 = 0.0;
    for (size_t e = 0; e < (size_t)m * n; e++)
        fro2 += X[e] * X[e];
    const double negligible = tol * tol * fro2;
    int sweep;
    for (sweep = 1; sweep <= max_sweeps; sweep++) {
        int rotated = 0;
        for (int i = 0; i < n - 1; i++) {
            for (int j = i + 1; j < n; j++) {
                double a = 0.0, b = 0.0, g = 0.0;
                for (int r = 0; r < m; r++) {
                    double wi = W[(size_t)r * n + i], wj = W[(size_t)r * n + j];
                    a += wi * wi;
                    b += wj * wj;
                    g += wi * wj;
                }
                if (g == 0.0 || fabs(g) <= tol * sqrt(a * b) || a <= negligible || b <= negligible)
                    continue;
                rotated = 1;
                /* rotation that zeroes the (i,j) entry of W^T W */
                double zeta = (b - a) / (2.0 * g);
                double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                double cs = 1.0 / sqrt(1.0 + t * t);
                double sn = cs * t;
                for (int r = 0; r < m; r++) {
                    double wi = W[(size_t)r * n + i], wj = W[(size_t)r * n + j];
                    W[(size_t)r * n + i] = cs * wi - sn * wj;
                    W[(size_t)r * n + j] = sn * wi + cs * wj;
                }
                for (int r = 0; r < n; r++) {
                    double vi = V[(size_t)r * n + i], vj = V[(size_t)r * n + j];
                    V[(size_t)r * n + i] = cs * vi - sn * vj;
                    V[(size_t)r * n + j] = sn * vi + cs * vj;
                }
            }
        }
        if (!rotated)
            break;
    }
    for (int j = 0; j < n; j++) {
        double a = 0.0;
        for (int r = 0; r < m; r++)
            a += W[(size_t)r * n + j] * W[(size_t)r * n + j];
        s[j] = sqrt(a);
    }
    return sweep > max_sweeps ? -1 : sweep;
}

/* ------------------------------------------------------------------------- */
/* Cyclic Jacobi eigen-decomposition of a symmetric p x p matrix.            */
/* On return w holds the eigenvalues (unsorted) and V the eigenvectors as    */
/* columns.  Returns the number of sweeps or -1 if max_sweeps was hit.       */
/* ------------------------------------------------------------------------- */
int orc_eig_jacobi(const double *S, int p, double *w, double *V, double tol, int max_sweeps)
{
    double *A = malloc((size_t)p * p * sizeof(double));
    memcpy(A, S, (size_t)p * p * sizeof(double));
    for (int i = 0; i < p; i++)
        for (int j = 0; j < p; j++)
            V[(size_t)i * p + j] = (i == j ? 1.0 : 0.0);
    int sweep;
    for (sweep = 1; sweep <= max_sweeps; sweep++) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < p; i++)
            for (int j = 0; j < p; j++) {
                double a = A[(size_t)i * p + j];
                tot += a * a;
                if (i != j)
                    off += a * a;
            }
        if (off <= tol * tol * tot)
            break;
        for (int i = 0; i < p - 1; i++) {
            for (int j = i + 1; j < p; j++) {
                double aij = A[(size_t)i * p + j];
                if (aij == 0.0)
                    continue;
                double aii = A[(size_t)i * p + i], ajj = A[(size_t)j * p + j];
                double th = (ajj - aii) / (2.0 * aij);
                double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
                double cs = 1.0 / sqrt(t * t + 1.0);
                double sn = t * cs;
                /* A <- J^T A J with J the rotation in the (i,j) plane */
                for (int r = 0; r < p; r++) {
                    double ari = A[(size_t)r * p + i], arj = A[(size_t)r * p + j];
                    A[(size_t)r * p + i] = cs * ari - sn * arj;
                    A[(size_t)r * p + j] = sn * ari + cs * arj;
                }
                for (int r = 0; r < p; r++) {
                    double air = A[(size_t)i * p + r], ajr = A[(size_t)j * p + r];
                    A[(size_t)i * p + r] = cs * air - sn * ajr;
                    A[(size_t)j * p + r] = sn * air + cs * ajr;
                }
                for (int r = 0; r < p; r++) {
                    double vri = V[(size_t)r * p + i], vrj = V[(size_t)r * p + j];
                    V[(size_t)r * p + i] = cs * vri - sn * vrj;
                    V[(size_t)r * p + j] = sn * vri + cs * vrj;
                }
            }
        }
    }
    for (int i = 0; i < p; i++)
        w[i] = A[(size_t)i * p + i];
    free(A);
    return sweep > max_sweeps ? -1 : sweep;
}

/* ------------------------------------------------------------------------- */
/* Exact singular value shrinkage, Eq. sing_shrink_exact:                    */
/*   G(X) = U diag(g(sigma_i)) V^T = sum_i h(sigma_i^2) (X v_i) v_i^T,       */
/* from the Jacobi SVD (the SVD-based method of Section V, Experimental Conditions).                */
/* sv (optional, p entries) receives the singular values.                    */
/* ------------------------------------------------------------------------- */
int orc_shrink_exact(const double *X, int m, int n, int kind, double tau, double c,
                     double eps, double noise, double *Y, double *sv)
{
    int tr = m < n;
    int mm = tr ? n : m, nn = tr ? m : n; /* work on the tall orientation */
    double *Xt = malloc((size_t)m * n * sizeof(double));
    if (tr)
        transpose(X, Xt, m, n);
    else
        memcpy(Xt, X, (size_t)m * n * sizeof(double));
    double *W = malloc((size_t)mm * nn * sizeof(double));
    double *V = malloc((size_t)nn * nn * sizeof(double));
    double *s = malloc((size_t)nn * sizeof(double));
    /* convergence level proportional to m eps: the computed column inner
     * products carry rounding errors of that relative size (Demmel and
     * Veselic, 1992), so a fixed 1e-15 can stall on tall matrices */
    double tol = (double)mm * 2.220446049250313e-16;
    if (tol < 1e-15)
        tol = 1e-15;
    int sw = orc_svd_jacobi(Xt, mm, nn, W, V, s, tol, 60);
    double *R = malloc((size_t)mm * nn * sizeof(double));
    for (size_t e = 0; e < (size_t)mm * nn; e++)
        R[e] = 0.0;
    for (int i = 0; i < nn; i++) {
        double hi = orc_h(kind, tau, c, eps, noise, s[i] * s[i]);
        if (hi == 0.0)
            continue;
        for (int r = 0; r < mm; r++) {
            double wri = hi * W[(size_t)r * nn + i];
            for (int j = 0; j < nn; j++)
                R[(size_t)r * nn + j] += wri * V[(size_t)j * nn + i];
        }
    }
    if (tr)
        transpose(R, Y, mm, nn);
    else
        memcpy(Y, R, (size_t)m * n * sizeof(double));
    if (sv)
        memcpy(sv, s, (size_t)nn * sizeof(double));
    free(Xt); free(W); free(V); free(s); free(R);
    return sw < 0 ? 1 : 0;
}

/* Exact shrinkage by the EVD-based method (Eq. sing_shrink_exact_from_eig2):
 *   G(X) = X V diag(h(lambda_i)) V^T   with X^T X = V diag(lambda) V^T
 * (m >= n), or V diag(h(lambda_i)) V^T X with X X^T = V diag(lambda) V^T. */
int orc_shrink_exact_evd(const double *X, int m, int n, int kind, double tau, double c,
                         double eps, double noise, double *Y)
{
    int p = m < n ? m : n;
    size_t pp = (size_t)p * p;
    double *G = malloc(pp * sizeof(double));
    double *V = malloc(pp * sizeof(double));
    double *w = malloc((size_t)p * sizeof(double));
    double *H = malloc(pp * sizeof(double));
    orc_gram(X, m, n, G);
    int sw = orc_eig_jacobi(G, p, w, V, 1e-15, 60);
    for (int i = 0; i < p; i++)
        for (int j = 0; j < p; j++) {
            double s = 0.0;
            for (int l = 0; l < p; l++)
                s += V[(size_t)i * p + l] * orc_h(kind, tau, c, eps, noise, w[l]) * V[(size_t)j * p + l];
            H[(size_t)i * p + j] = s;
        }
    if (m >= n)
        matmul(X, H, Y, m, n, n);
    else
        matmul(H, X, Y, m, m, n);
    free(G); free(V); free(w); free(H);
    return sw < 0 ? 1 : 0;
}

/* ------------------------------------------------------------------------- */
/* Counter-based generator for the power-iteration start vector.  SplitMix64 */
/* (Steele, Lea and Flood, "Fast splittable pseudorandom number generators", */
/* OOPSLA 2014): state advanced by the golden-ratio increment, then the      */
/* published two-multiply finaliser.  Output i (i = 0, 1, ...) of the        */
/* generator seeded with `seed` is mix(seed + (i+1) * 0x9E3779B97F4A7C15).   */
/* v0_i = u_i - 1/2 with u_i the top 53 bits of output i scaled to [0,1).    */
/* ------------------------------------------------------------------------- */
static uint64_t splitmix64_output(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

void orc_start_vector(uint64_t seed, int p, double *v0)
{
    for (int i = 0; i < p; i++) {
        uint64_t z = splitmix64_output(seed, (uint64_t)i);
        v0[i] = (double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5;
    }
}
