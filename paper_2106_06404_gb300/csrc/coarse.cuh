// Coarse-level algebra: Gram blocks of the fine coarse-basis functions over
// element patches (the volume patch matrices of Section 4.1 expressed in the
// coarse basis), their assembly into the Galerkin level matrix and the
// generating-system Neumann matrices of Section 4.2, batched small GEMMs, and
// the vector kernels of the preconditioner and of CG.
#pragma once
#include "common.cuh"
#include "q1.cuh"

namespace msdd {

// dst[doff + k * ld + k'] = sum over the contribution list of G[goff + k * mjj + k'].
struct SumItem {
    long long doff;
    int ld, rows, cols;
    int cbeg, cend;   // range in the contribution list
};
void block_sum(const SumItem* d_items, int nitems, const long long* d_contrib, const double* G, double* dst,
               cudaStream_t s);

// Batched C_b = alpha * op(A_b) op(B_b) + beta * C_b, FP64.  Nothing is done
// when *gdone != 0; item b is left alone when skip[b] != 0.
struct GemmItem {
    long long aoff, boff, coff;
    int m, n, k;
    int lda, ldb, ldc;
};
void gemm_batched(const GemmItem* d_items, int nitems, int transA, int transB, double alpha, const double* A,
                  const double* B, double beta, double* C, int max_m, int max_n, cudaStream_t s,
                  const int* gdone = nullptr, const int* skip = nullptr);

// Batched matrix-vector products with the GemmItem geometry (n = 1 implied):
// y[coff + r * ldc] = alpha * sum_k op(A)[r][k] x[boff + k * ldb] + beta * y[...].
void gemv_batched(const GemmItem* d_items, int nitems, int transA, double alpha, const double* A, const double* x,
                  double beta, double* y, int max_m, cudaStream_t s, const int* gdone = nullptr);

// dst = src with rows of the own block (rows < nown) scaled by (1 + sigma)
// on their own-own entries: K = Abar + sigma X Abar X for dense pencils.
void dense_shift(const double* Abar, double* Kd, const long long* d_aoff, const int* d_n, const int* d_nown,
                 double sigma, int P, int nmax, cudaStream_t s);

// ---- preconditioner / CG vector kernels
// Fine Dirichlet gather and coarse restriction: rhs_j = r on the Dirichlet box
// of j (solve-buffer layout), r1[c1off_j + k] = Phi_j^T rhs_j.
void fine_gather_restrict(const Geom& g, const ProbBox* d_fine, const long long* d_droff, const int* d_K,
                          const double* r, double* rhs, const double* Phi, const long long* d_phioff, int ldphi,
                          const int* d_m, const long long* d_c1off, double* r1, int P, const int* done,
                          cudaStream_t s);

// Per-axis lookup of fine subdomains whose Dirichlet range holds a coordinate.
struct CombineMaps {
    int parts[3];
    const int* first[3];   // per axis, per node coordinate: first block index (or -1)
    const int* last[3];
};
// z[u] = sum_{j : u in D_j} ( y_j[u] + Phi_j[u,:] . z1[c1off_j : c1off_j + m_j] ),
// and partial sums of r.z for the following dot product.
void fine_combine(const Geom& g, const CombineMaps& cm, const ProbBox* d_fine, const long long* d_droff,
                  const double* y, const double* Phi, const long long* d_phioff, int ldphi, const int* d_m,
                  const long long* d_c1off, const double* z1, double* z, const double* r, double* partial,
                  int nblocks, const int* done, cudaStream_t s, struct PcgScalars* sc = nullptr, int fin = 0);
// Modes of the combine: COMB_Y the fine local solutions, COMB_COARSE the
// prolongation Phi z1, COMB_RAS the local solutions weighted by chi = 1/N(x)
// (restricted additive Schwarz), COMB_ACC adds to z; partial (z . r per
// block) is skipped when NULL.
constexpr int COMB_Y = 1, COMB_COARSE = 2, COMB_RAS = 4, COMB_ACC = 8;
void fine_combine_mode(const Geom& g, const CombineMaps& cm, const ProbBox* d_fine, const long long* d_droff,
                       const double* y, const double* Phi, const long long* d_phioff, int ldphi, const int* d_m,
                       const long long* d_c1off, const double* z1, double* z, const double* r, double* partial,
                       int nblocks, const int* done, int mode, cudaStream_t s, struct PcgScalars* sc = nullptr,
                       int fin = 0);

// out[dst_off[i] + k] (+)= in[src_off[i] + k] for k < len[i]; mode 0: copy, 1: add.
void segment_copy(const long long* d_src_off, const long long* d_dst_off, const int* d_len, int P, int maxlen,
                  const double* in, double* out, int mode, const int* done, cudaStream_t s);

// Deterministic dot product: partial sums by `nblocks` CTAs then one CTA.
int dot_blocks(long long n);
void dot_partial(const double* x, const double* y, long long n, double* partial, int nblocks, cudaStream_t s);

}  // namespace msdd

namespace msdd {
// Strided block copies: dst[doff + r * ldd + c] = src[soff + r * lds + c].
struct CopyItem {
    long long soff, doff;
    int lds, ldd, rows, cols;
};
void copy_blocks(const CopyItem* d_items, int nitems, const double* src, double* dst, cudaStream_t s);
}  // namespace msdd
