// Batched tile-band LDL^T factorisation and solves (declarations).
//
// Every local matrix of the method (fine-level Dirichlet matrices A_{l,i} of
// Eq. (dirichlet_space), the shifted Neumann pencils of the eigensolver, and
// the dense coarse-level matrices) is symmetric and banded with half-bandwidth
// b (dense: b = n - 1).  It is stored as NB x NB tiles: tile row R holds the
// tiles (R, C) for R - kb <= C <= R, kb = ceil(b / NB).  Factorisation writes
// K = L D L^T with L unit lower triangular; the diagonal tile (R, R) is then
// overwritten by T_R = L_RR^{-1}, the off-diagonal tiles by L_RC, and D^{-1}
// is kept per row.  A solve is a chain of small tile products
//   z_R = T_R (y_R - sum_J L_RJ z_J),   x_R = T_R^T (D_R^{-1} z_R - sum_I L_IR^T x_I).
// With `reg_tol` > 0 a pivot d_k <= reg_tol * K_kk (original diagonal) is a
// null pivot: D^{-1}_k = 0 and column k of L is zero, so the solve applies a
// regularised inverse that annihilates the common kernel (the ker A cap ker B
// treatment of Section 4.2, Eq. evp_reg).
#pragma once
#include "common.cuh"

namespace msdd {

struct TileBatch {
    int P = 0;
    int prec = 0;                 // 0: double tiles, 1: float tiles
    std::vector<int> n, kb, K, b; // host copies (b: half-bandwidth)
    std::vector<long long> toff, roff;
    long long total_tile_elems = 0, total_rows = 0;
    int max_K = 0;
    DevBuf<int> d_n, d_kb, d_K, d_b, d_status, d_nreg;
    DevBuf<long long> d_toff, d_roff;
    DevBuf<double> tiles_d, dinv_d;
    DevBuf<float> tiles_f, dinv_f;
    // TMA descriptor (opaque CUtensorMap) of the FP32 tiles viewed as a
    // [total_tile_elems / 32][32] matrix, built on first use for tiles_f.p
    alignas(64) mutable unsigned char tmap_tiles[128] = {};
    mutable const float* tmap_base = nullptr;

    // Layout from per-problem sizes and half-bandwidths.
    void layout(const std::vector<int>& n_, const std::vector<int>& b_, int precision, cudaStream_t s);
    // Non-owning view of problems [p0, p0 + np) (same tiles, rows and offsets).
    TileBatch slice(int p0, int np) const;
    void* tiles() const { return prec ? (void*)tiles_f.p : (void*)tiles_d.p; }
    size_t bytes() const {
        return (size_t)total_tile_elems * (prec ? 4 : 8) + (size_t)total_rows * (prec ? 4 : 8);
    }
};

// Zero all tiles (before assembly).
void tile_zero(TileBatch& tb, cudaStream_t s);
// Copy dense row-major matrices (problem i at src + soff[i], leading dim lds[i])
// into the tile layout.  src is double; converted to the batch precision.
void tile_from_dense(TileBatch& tb, const double* src, const long long* d_soff, const int* d_lds,
                     cudaStream_t s);
// In-place LDL^T of every problem; fills d_status (0 ok, k+1 = failing row) and d_nreg.
void tile_factor(TileBatch& tb, double reg_tol, cudaStream_t s);
// E (total_rows x lde) <- per problem the identity of order n[i] (zero elsewhere).
void tile_identity(const TileBatch& tb, double* E, int lde, cudaStream_t s);
// Solve K X = B in place.  X is double, row-major, problem i rows at
// (roff[i] + r) * ldx, columns 0..ncols-1 (any ncols <= ldx; blocks of 32
// columns go to separate CTAs).  `skip` (device, per problem, may be
// null) skips problems whose flag is non-zero; `gdone` (device, may be null)
// skips everything when non-zero.
void tile_solve(const TileBatch& tb, double* X, int ldx, int ncols, const int* skip, cudaStream_t s,
                const int* gdone = nullptr);
// Throws if a bounded wait in a solve kernel gave up (its error flag is
// reset); call after a synchronisation point.
void tile_check_waits();

}  // namespace msdd
