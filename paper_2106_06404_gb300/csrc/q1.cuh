// Q1 finite elements on a structured box mesh: local matrix assembly into the
// tile-band format, matrix-free local Neumann operators, the global operator
// and the load vector.  Section 3.4: a_tau(u, v) = int_tau (K grad u) . grad v,
// abar_{l,i} = sum over tau in T_{h,l,i} (Eq. locala_cg), and
// b^1_{l,i}(u, v) = abar_{l,i}(chi u, chi v) (Eq. cg_rhs_blf).
#pragma once
#include "common.cuh"
#include "tile_ldlt.cuh"

namespace msdd {

// Global mesh description (plain values; passed by value to kernels).
struct Geom {
    int dim;
    int n[3];          // elements per axis (n[2] = 1 in 2D)
    int ulo[3], uhi[3];// box of unknown nodes, inclusive (Dirichlet faces removed)
    int ushape[3];     // uhi - ulo + 1
    int coeff_kind;    // 0 scalar per element, 1 symmetric tensor per element
    int ncomp;         // 1, 3 (2D tensor) or 6 (3D tensor)
    const double* coeff;
    int blf;           // fine GEVP right-hand side b^1, b^2 or b^3 (Section 3.4)
    const int* ecov[3];// b^2: per axis, fine element boxes holding each element index (device)
    double rscale;     // h_x^(dim-2): the element matrices are rscale times the reference matrices
};

// One local problem on the fine level: its overlapping element box
// [elo, ehi) and the inclusive node boxes of its Neumann space (all
// non-Dirichlet nodes of the closure) and its Dirichlet space (nodes whose
// hat function is supported in the closure).
struct ProbBox {
    int elo[3], ehi[3];
    int nlo[3], nhi[3];
    int dlo[3], dhi[3];
};

// ---- box index helpers (lexicographic, x fastest)
__host__ __device__ __forceinline__ bool in_box(const int lo[3], const int hi[3], const int x[3], int dim) {
    for (int d = 0; d < dim; ++d)
        if (x[d] < lo[d] || x[d] > hi[d]) return false;
    return true;
}

__host__ __device__ __forceinline__ long long unknown_index(const Geom& g, const int x[3]) {
    long long u = 0, stride = 1;
    for (int d = 0; d < g.dim; ++d) {
        u += (x[d] - g.ulo[d]) * stride;
        stride *= g.ushape[d];
    }
    return u;
}

__host__ __device__ __forceinline__ void box_coords(int r, const int lo[3], const int hi[3], int dim, int x[3]) {
    for (int d = 0; d < 3; ++d) {
        if (d >= dim) { x[d] = 0; continue; }
        int w = hi[d] - lo[d] + 1;
        x[d] = lo[d] + r % w;
        r /= w;
    }
}

__host__ __device__ __forceinline__ int box_index(const int lo[3], const int hi[3], const int x[3], int dim) {
    int r = 0, stride = 1;
    for (int d = 0; d < dim; ++d) {
        r += (x[d] - lo[d]) * stride;
        stride *= hi[d] - lo[d] + 1;
    }
    return r;
}

__host__ __device__ __forceinline__ int box_size(const int lo[3], const int hi[3], int dim) {
    int s = 1;
    for (int d = 0; d < dim; ++d) s *= (hi[d] >= lo[d]) ? hi[d] - lo[d] + 1 : 0;
    return s;
}


// Reference element matrices R_de[a][b] = int d_d phi_a d_e phi_b for the
// mesh's element size; uploaded once per set-up.
void upload_reference(const Geom& g);

// count[u] over unknowns: number of fine subdomains whose Dirichlet box holds u.
void pou_count(const Geom& g, const ProbBox* d_boxes, int P, int* d_count, cudaStream_t s);

// Assemble into zeroed tiles: mode 0 -> Dirichlet matrix on the Dirichlet box;
// mode 1 -> Abar + sigma * X Abar X on the Neumann box (X = diag(chi)).
void assemble_local_tiles(const Geom& g, const ProbBox* d_boxes, const int* d_count, TileBatch& tb,
                          int mode, double sigma, cudaStream_t s);

// AX = Abar X, BX = X Abar X applied to the first ncols columns (row-major,
// ldx, rows at roff[i]); problems with skip[i] != 0 are left untouched.
void apply_neumann(const Geom& g, const ProbBox* d_boxes, const int* d_count, const TileBatch& layout,
                   const double* X, double* AX, double* BX, int ldx, int ncols, const int* skip, cudaStream_t s);

// W = X Abar X applied to X in FP32 arithmetic (start phase of the
// eigensolver); padding rows of W are zeroed.
void apply_b32(const Geom& g, const ProbBox* d_boxes, const int* d_count, const TileBatch& layout, const double* X,
               double* W, int ldx, int ncols, cudaStream_t s);

// The local Neumann operators of the fine problems as stored 3^d-point
// stencils over the rows of the Neumann box (the layout of the GEVP
// vectors):  a[row][o] = abar(phi_{x+o}, phi_x) and
// b[row][o] = chi(x) a[row][o] chi(x+o)  (so that B = X Abar X), zero where
// x + o leaves the Neumann box and on padding rows; b32 is b rounded to FP32.
// Built once per set-up; the eigensolver's operator applications then read
// coefficients instead of recomputing element integrals and chi.
struct LocalStencil {
    int noff = 0;
    DevBuf<double> a, b;
    DevBuf<float> b32;
};
void build_local_stencil(const Geom& g, const ProbBox* d_boxes, const int* d_count, const TileBatch& layout,
                         LocalStencil& ls, cudaStream_t s);
// AX = Abar X, BX = X Abar X from the stored stencils (same contract as apply_neumann).
// With FP32 factors in `layout` (the chosen form) the products are accumulated
// in double-float, as in apply_local_rhs.
void apply_local(const LocalStencil& ls, const ProbBox* d_boxes, int dim, const TileBatch& layout, const double* X,
                 double* AX, double* BX, int ldx, int ncols, const int* skip, cudaStream_t s);
// W = BX - (AX + sigma BX) diag(1 / (theta + sigma)) with AX, BX from the
// stored stencils (zero on padding rows, columns < p_i), and the residual
// partial sums of X (layout of EIG_ROWBLK) for the problems with done == 0;
// theta is PMAX per problem, partial (P * nblk_max * 2 PMAX).
void apply_local_rhs(const LocalStencil& ls, const ProbBox* d_boxes, int dim, const TileBatch& layout,
                     const double* X, double* W, int ldx, const int* d_p, const double* theta, double sigma,
                     double* partial, int nblk_max, const int* done, cudaStream_t s);
// W = X Abar X X in FP32 arithmetic from b32 (same contract as apply_b32).
void apply_local_b32(const LocalStencil& ls, const ProbBox* d_boxes, int dim, const TileBatch& layout,
                     const double* X, double* W, int ldx, int ncols, cudaStream_t s);

// Stored 3^d-point stencil of the global operator: S[o * n + u] = A(u, u + o),
// offsets o lexicographic (x fastest) in {-1, 0, 1}^d, zero where u + o is
// not an unknown.  n * 3^d doubles.
void global_stencil(const Geom& g, double* S, cudaStream_t s);
// q = A p from the stored stencil and partial sums of p.q (nblocks CTAs).
// (sc != NULL: the kernel's last block also applies the finishing step `fin`
// of PcgFin to the summed partials, e.g. alpha = rho / p.q.)
void spmv_stencil_dot(const Geom& g, const double* S, const double* p, double* q, double* partial, int nblocks,
                      const int* done, cudaStream_t s, struct PcgScalars* sc = nullptr, int fin = 0);

// y = A x on the unknowns (Dirichlet nodes eliminated).
void apply_global(const Geom& g, const double* x, double* y, cudaStream_t s);

// Load vector l(v) = int f v for constant f.
void load_vector(const Geom& g, double f, double* b, cudaStream_t s);

// chi on the Dirichlet box of each problem times the first m columns of the
// Neumann-box vectors X: Phi[i] (rows dlo..dhi, ldphi columns).
void make_coarse_basis(const Geom& g, const ProbBox* d_boxes, const int* d_count, const TileBatch& nlayout,
                       const double* X, int ldx, const int* d_m, double* Phi, const long long* d_phioff,
                       int ldphi, int P, cudaStream_t s);

// One Gram block of the fine coarse-basis functions over an element box
// [elo, ehi) (a volume patch, Section 4.1):
//   G = sum_{tau in box} Phi_j(tau)^T A_tau Phi_jj(tau)      (m_j x m_jj, row-major at goff),
// Phi_j(tau) the values of phi_{j,k} = e chi_j w_{j,k} at the element's nodes
// (zero outside the Dirichlet box of j).
struct GramItem {
    int elo[3], ehi[3];
    int j, jj;
    long long goff;
};
void patch_gram(const Geom& g, const ProbBox* d_fine, const double* Phi, const long long* d_phioff, int ldphi,
                const int* d_m, const GramItem* d_items, int nitems, double* G, cudaStream_t s);

// q = A p on the unknowns and partial sums of p.q (nblocks CTAs).
void apply_global_dot(const Geom& g, const double* p, double* q, double* partial, int nblocks, const int* done,
                      cudaStream_t s);

}  // namespace msdd
