/*
 * Oracle dense linear algebra (test infrastructure only; never linked into the
 * product library).
 *
 * Plain, slow, LAPACK-free FP64 building blocks used by the CPU oracle of the
 * multilevel spectral domain decomposition method:
 *   - dense Cholesky A = L L^T (Section 4.3 uses a sparse Cholesky as the
 *     subdomain solver; the oracle uses the textbook dense algorithm),
 *   - forward / backward substitution with several right-hand sides,
 *   - the cyclic Jacobi eigenvalue algorithm for a dense symmetric matrix
 *     (used to compute every eigenpair of the local generalized eigenproblems,
 *     Eq. (theGEVP) and Section 3.3, through a spectral transformation),
 *   - for the oracle's method mode: band Cholesky, band solves and the band
 *     LDL^T inertia count (storage described above those routines).
 *
 * Dense matrices are row-major, n x n, double precision.  Nothing is
 * blocked, fused or reordered: each routine is the textbook definition.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* A = L L^T.  Returns 0 on success, k+1 if the k-th pivot is not positive. */
int orc_cholesky(int n, const double *A, double *L)
{
    memset(L, 0, sizeof(double) * (size_t)n * (size_t)n);
    for (int j = 0; j < n; ++j) {
        double d = A[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) d -= L[(size_t)j * n + k] * L[(size_t)j * n + k];
        if (!(d > 0.0)) return j + 1;
        double ljj = sqrt(d);
        L[(size_t)j * n + j] = ljj;
        for (int i = j + 1; i < n; ++i) {
            double s = A[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) s -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
            L[(size_t)i * n + j] = s / ljj;
        }
    }
    return 0;
}

/* Solve L X = B in place (B is n x nrhs, row-major). */
void orc_forward(int n, int nrhs, const double *L, double *B)
{
    for (int i = 0; i < n; ++i) {
        for (int c = 0; c < nrhs; ++c) {
            double s = B[(size_t)i * nrhs + c];
            for (int k = 0; k < i; ++k) s -= L[(size_t)i * n + k] * B[(size_t)k * nrhs + c];
            B[(size_t)i * nrhs + c] = s / L[(size_t)i * n + i];
        }
    }
}

/* Solve L^T X = B in place (B is n x nrhs, row-major). */
void orc_backward(int n, int nrhs, const double *L, double *B)
{
    for (int i = n - 1; i >= 0; --i) {
        for (int c = 0; c < nrhs; ++c) {
            double s = B[(size_t)i * nrhs + c];
            for (int k = i + 1; k < n; ++k) s -= L[(size_t)k * n + i] * B[(size_t)k * nrhs + c];
            B[(size_t)i * nrhs + c] = s / L[(size_t)i * n + i];
        }
    }
}

/*
 * Cyclic Jacobi method for a symmetric matrix S (n x n, destroyed).
 * On return w holds the eigenvalues (unsorted, in diagonal order) and the
 * columns of V the orthonormal eigenvectors: S_in = V diag(w) V^T.
 * Each sweep visits every pair (p, q), p < q, in row order and annihilates
 * S[p][q] with the plane rotation J that does so, S <- J^T S J (the
 * classical two-sided update; the symmetric copy of rows p and q is written
 * back into columns p and q).  A pair whose off-diagonal entry is already
 * below rounding level relative to its diagonal entries is set to zero
 * without a rotation.  Stops when the off-diagonal Frobenius norm is below
 * tol * ||S||_F.  Returns the number of sweeps, or -1 if max_sweeps were not
 * enough.
 */
int orc_jacobi(int n, double *S, double *w, double *V, int max_sweeps, double tol)
{
    /* Vt holds V transposed so that the rotation of V touches two rows */
    double *Vt = (double *)malloc(sizeof(double) * (size_t)n * (size_t)n);
    if (!Vt) return -2;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) Vt[(size_t)i * n + j] = (i == j) ? 1.0 : 0.0;
    double fro = 0.0;
    for (size_t k = 0; k < (size_t)n * n; ++k) fro += S[k] * S[k];
    fro = sqrt(fro);
    int sweeps = 0;
    for (;;) {
        double off = 0.0;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) off += 2.0 * S[(size_t)p * n + q] * S[(size_t)p * n + q];
        off = sqrt(off);
        if (off <= tol * fro || fro == 0.0) break;
        if (sweeps == max_sweeps) { sweeps = -1; break; }
        for (int p = 0; p < n - 1; ++p) {
            for (int q = p + 1; q < n; ++q) {
                double *Sp = S + (size_t)p * n, *Sq = S + (size_t)q * n;
                double apq = Sp[q];
                if (apq == 0.0) continue;
                double app = Sp[p], aqq = Sq[q];
                if (fabs(apq) <= 1e-18 * sqrt(fabs(app * aqq))) {
                    Sp[q] = 0.0; Sq[p] = 0.0;
                    continue;
                }
                /* rotation angle: cot(2 phi) = (aqq - app) / (2 apq) */
                double theta = (aqq - app) / (2.0 * apq);
                double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {          /* rows p and q */
                    double spk = Sp[k], sqk = Sq[k];
                    Sp[k] = c * spk - s * sqk;
                    Sq[k] = s * spk + c * sqk;
                }
                for (int k = 0; k < n; ++k) {          /* columns = rows (symmetry) */
                    S[(size_t)k * n + p] = Sp[k];
                    S[(size_t)k * n + q] = Sq[k];
                }
                Sp[p] = app - t * apq;
                Sq[q] = aqq + t * apq;
                Sp[q] = 0.0;
                Sq[p] = 0.0;
                double *Vp = Vt + (size_t)p * n, *Vq = Vt + (size_t)q * n;
                for (int k = 0; k < n; ++k) {          /* V <- V J */
                    double vkp = Vp[k], vkq = Vq[k];
                    Vp[k] = c * vkp - s * vkq;
                    Vq[k] = s * vkp + c * vkq;
                }
            }
        }
        ++sweeps;
    }
    for (int i = 0; i < n; ++i) w[i] = S[(size_t)i * n + i];
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) V[(size_t)i * n + j] = Vt[(size_t)j * n + i];
    free(Vt);
    return sweeps;
}

/*
 * Inertia count of a symmetric matrix by the textbook LDL^T factorisation
 * without pivoting: returns the number of negative pivots d_k, or -1 if a
 * pivot is exactly zero.  By Sylvester's law of inertia this is the number of
 * negative eigenvalues whenever the factorisation exists.  A is not modified.
 */
int orc_ldlt_negative_count(int n, const double *A)
{
    double *W = (double *)malloc(sizeof(double) * (size_t)n * (size_t)n);
    if (!W) return -2;
    memcpy(W, A, sizeof(double) * (size_t)n * (size_t)n);
    int neg = 0;
    for (int k = 0; k < n; ++k) {
        double d = W[(size_t)k * n + k];
        if (d == 0.0) { free(W); return -1; }
        if (d < 0.0) ++neg;
        for (int i = k + 1; i < n; ++i) {
            double lik = W[(size_t)i * n + k] / d;
            if (lik == 0.0) continue;
            for (int j = k + 1; j <= i; ++j) W[(size_t)i * n + j] -= lik * W[(size_t)j * n + k];
        }
    }
    free(W);
    return neg;
}

/*
 * Band matrices (method mode of the oracle): a symmetric matrix of order n
 * and half-bandwidth b is held by its lower band, row-major by rows, entry
 * (i, j), i - b <= j <= i, at AB[i * (b + 1) + (j - i + b)] (the diagonal in
 * the last column of each row; entries with j < 0 are unused).
 */

/* In place A = L L^T on the lower band (the textbook column algorithm
 * restricted to the band).  Returns 0 on success, k+1 if pivot k is not
 * positive. */
int orc_band_cholesky(int n, int b, double *AB)
{
    const int w = b + 1;
    for (int j = 0; j < n; ++j) {
        const int k0 = j - b > 0 ? j - b : 0;
        double d = AB[(size_t)j * w + b];
        for (int k = k0; k < j; ++k) {
            const double ljk = AB[(size_t)j * w + (k - j + b)];
            d -= ljk * ljk;
        }
        if (!(d > 0.0)) return j + 1;
        const double ljj = sqrt(d);
        AB[(size_t)j * w + b] = ljj;
        const int iend = j + b < n - 1 ? j + b : n - 1;
        for (int i = j + 1; i <= iend; ++i) {
            const int ki = i - b > 0 ? i - b : 0;
            double s = AB[(size_t)i * w + (j - i + b)];
            for (int k = ki; k < j; ++k)
                s -= AB[(size_t)i * w + (k - i + b)] * AB[(size_t)j * w + (k - j + b)];
            AB[(size_t)i * w + (j - i + b)] = s / ljj;
        }
    }
    return 0;
}

/* Solve L L^T X = B in place with the band factor from orc_band_cholesky
 * (B is n x nrhs, row-major): forward then backward substitution. */
void orc_band_solve(int n, int b, const double *LB, int nrhs, double *X)
{
    const int w = b + 1;
    for (int i = 0; i < n; ++i) {
        const int k0 = i - b > 0 ? i - b : 0;
        for (int c = 0; c < nrhs; ++c) {
            double s = X[(size_t)i * nrhs + c];
            for (int k = k0; k < i; ++k) s -= LB[(size_t)i * w + (k - i + b)] * X[(size_t)k * nrhs + c];
            X[(size_t)i * nrhs + c] = s / LB[(size_t)i * w + b];
        }
    }
    for (int i = n - 1; i >= 0; --i) {
        const int kend = i + b < n - 1 ? i + b : n - 1;
        for (int c = 0; c < nrhs; ++c) {
            double s = X[(size_t)i * nrhs + c];
            for (int k = i + 1; k <= kend; ++k) s -= LB[(size_t)k * w + (i - k + b)] * X[(size_t)k * nrhs + c];
            X[(size_t)i * nrhs + c] = s / LB[(size_t)i * w + b];
        }
    }
}

/* Inertia count of a symmetric band matrix by LDL^T without pivoting on a
 * copy of the band (the band is preserved by the elimination): number of
 * negative pivots, or -1 if a pivot is exactly zero. */
int orc_band_negative_count(int n, int b, const double *AB)
{
    const int w = b + 1;
    double *W = (double *)malloc(sizeof(double) * (size_t)n * (size_t)w);
    if (!W) return -2;
    memcpy(W, AB, sizeof(double) * (size_t)n * (size_t)w);
    int neg = 0;
    for (int k = 0; k < n; ++k) {
        const double d = W[(size_t)k * w + b];
        if (d == 0.0) { free(W); return -1; }
        if (d < 0.0) ++neg;
        const int iend = k + b < n - 1 ? k + b : n - 1;
        for (int i = k + 1; i <= iend; ++i) {
            const double lik = W[(size_t)i * w + (k - i + b)] / d;
            if (lik == 0.0) continue;
            for (int j = k + 1; j <= i; ++j)
                W[(size_t)i * w + (j - i + b)] -= lik * W[(size_t)j * w + (k - j + b)];
        }
    }
    free(W);
    return neg;
}

/*
 * Regularised LDL^T of a symmetric positive semi-definite matrix K (n x n,
 * row-major, not modified), without pivoting, in the given order: pivot k
 * is a null pivot when d_k <= tau * K_kk (K_kk the original diagonal entry),
 * the epsilon-regularisation of Section 4.2 taken to its limit (D^+_k = 0):
 * then d_k = 0, column k of L is zero below the diagonal and the remaining
 * Schur complement is not updated by row k (the generator is dropped as
 * dependent on the earlier ones).  Outputs L (unit lower, n x n), d (n) and
 * null (n flags).  Returns the number of null pivots, or -2 on allocation
 * failure.
 */
int orc_ldlt_null(int n, const double *K, double tau, double *L, double *d, int *null)
{
    double *W = (double *)malloc(sizeof(double) * (size_t)n * (size_t)n);
    if (!W) return -2;
    memcpy(W, K, sizeof(double) * (size_t)n * (size_t)n);
    memset(L, 0, sizeof(double) * (size_t)n * (size_t)n);
    int nn = 0;
    for (int k = 0; k < n; ++k) {
        L[(size_t)k * n + k] = 1.0;
        const double dk = W[(size_t)k * n + k];
        if (!(dk > tau * K[(size_t)k * n + k])) {
            d[k] = 0.0;
            null[k] = 1;
            ++nn;
            continue;
        }
        d[k] = dk;
        null[k] = 0;
        for (int i = k + 1; i < n; ++i) L[(size_t)i * n + k] = W[(size_t)i * n + k] / dk;
        for (int i = k + 1; i < n; ++i) {
            const double lik = L[(size_t)i * n + k];
            if (lik == 0.0) continue;
            for (int j = k + 1; j <= i; ++j) W[(size_t)i * n + j] -= lik * W[(size_t)j * n + k];
        }
    }
    free(W);
    return nn;
}
