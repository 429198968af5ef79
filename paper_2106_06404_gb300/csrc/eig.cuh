// Batched block subspace iteration with Rayleigh-Ritz for the local GEVPs
//   abar(w, v) = lambda b(w, v)                     (Eq. theGEVP)
// through the spectral transformation with the shifted matrix
// K = Abar + sigma B (mu = 1 / (lambda + sigma), largest mu wanted; cf. the
// shift-invert use of Section 4.2/4.3 and the transformation in the proof of
// the non-defectiveness lemma of Section 3.3).
//
// One iteration for every unconverged problem i (X B-orthonormal Ritz vectors
// with Ritz values theta, AX = Abar X, BX = B X):
//   W = BX - (AX + sigma BX) diag(mu),      mu_k = 1 / (theta_k + sigma)
//   W <- K^{-1} W        (tile LDL^T solve, FP64 or FP32 factors)
//   Y = X diag(mu) + W   (= K^{-1} B X when the solve is exact)
//   AY, BY; H = Y^T AY, M = Y^T BY (FP64); Rayleigh-Ritz H c = theta M c
//   X = Y C, AX = AY C, BX = BY C; residuals |AX_k - theta_k BX_k| / ((theta_k + sigma) |BX_k|).
// The residual form lets an inexact (lower precision) K^{-1} still converge
// to the FP64 eigenpairs: its fixed point does not depend on the solve.
#pragma once
#include "common.cuh"
#include "tile_ldlt.cuh"

namespace msdd {

struct GevpBatch {
    int P = 0;
    int ldx = PMAX;                   // columns stored per row
    std::vector<int> p;               // block size per problem (<= PMAX)
    DevBuf<int> d_p;
    TileBatch K;                      // factor of Abar + sigma B (rows = problem size)
    DevBuf<double> X, AX, BX, Y, AY, BY, W;        // (total_rows x ldx)
    DevBuf<double> H, M, C, theta, res;            // per problem PMAX^2 / PMAX
    int gsplit = 1;                                // row splits of the Gram products
    DevBuf<double> Hp, Mp;                         // per (problem, split) PMAX^2 partial Grams
    DevBuf<double> partial;                        // per (problem, row block) sums
    DevBuf<int> done, m, rank, iters;   // done: 0 running, 1 converged, 2 maxit, 3 at noise floor
    DevBuf<double> best;                 // best worst-selected residual so far
    DevBuf<int> best_it;
    DevBuf<int> n_active;
    int nblk_max = 0;
    bool knorm = false;           // residual measured in the K^+-norm (coarse levels)
    void alloc(cudaStream_t s);
    // Non-owning view of problems [p0, p0 + np) with its own active counter
    // (group < 2): per-problem arrays offset, block vectors shared (they are
    // addressed by absolute row offsets).
    GevpBatch slice(int p0, int np, int group) const;
};

struct EigParams {
    double sigma = 1e-2;
    double tol = 1e-6;
    double eta = 0.3;
    int nev_max = 8;
    int maxit = 100;
    unsigned long long seed = 12345;
};

// Fill X with counter-based random numbers (rows < n_i, columns < p_i) and
// zero the rest; reset per-problem state.
void eig_init(GevpBatch& g, unsigned long long seed, cudaStream_t s);
// X[:, c] <- Wst rows (woff[i] + r), columns c < min(wc, p_i), for rows r < n_i
// (caller-provided start vectors; the remaining columns keep eig_init's).
void eig_load_start(GevpBatch& g, const double* Wst, int wc, const long long* d_woff, cudaStream_t s);
// W = BX - (AX + sigma BX) diag(mu) (first == true: W = BX).
void eig_form_rhs(GevpBatch& g, double sigma, bool first, cudaStream_t s);
// Y = X diag(mu) + W (first == true: Y = W).
void eig_form_y(GevpBatch& g, double sigma, bool first, cudaStream_t s);
// Y = X diag(mu) + W with the K^+-norm residual partial sums of X.
void eig_form_y_knorm(GevpBatch& g, double sigma, cudaStream_t s);
// Convergence test on the K^+-norm residuals (regularised coarse pencils).
void eig_check_knorm(GevpBatch& g, const EigParams& ep, int it, cudaStream_t s);
// FP32 start phase: X <- orthonormal basis of span(W) by Euclidean CholQR
// (Gram with FP32 products, FP64 Cholesky of the scaled p x p Gram).
void eig_cholqr32(GevpBatch& g, cudaStream_t s);
// H = Y^T AY, M = Y^T BY.
void eig_gram(GevpBatch& g, cudaStream_t s);
// Rayleigh-Ritz: theta ascending, C with C^T M C = I.
void eig_rayleigh_ritz(GevpBatch& g, cudaStream_t s);
// X = Y C, AX = AY C, BX = BY C, residual partial sums.
void eig_update(GevpBatch& g, cudaStream_t s);
// X = Y C only: with a cheap operator (stored stencils) AX and BX are applied
// afresh, together with the next right-hand side (apply_local_rhs).
void eig_update_x(GevpBatch& g, cudaStream_t s);
// Residuals, selection count m = min(nev_max, #{theta < eta}), convergence flags.
void eig_check(GevpBatch& g, const EigParams& ep, int it, cudaStream_t s);

// Dense operators for the coarse levels: Abar dense (problem i at aoff[i],
// leading dimension n_i); own generators are rows < nown[i] and B = X Abar X
// with X the indicator of the own rows (chi_{l,i} of Section 4.2).
void apply_dense_pencil(const double* Abar, const long long* d_aoff, const int* d_n, const int* d_nown,
                        const TileBatch& layout, const double* X, double* AX, double* BX, int ldx, int ncols,
                        const int* skip, int P, int nmax, cudaStream_t s);

}  // namespace msdd
