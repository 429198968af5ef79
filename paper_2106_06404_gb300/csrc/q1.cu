// Q1 assembly and matrix-free operators on the structured mesh.
#include "q1.cuh"
#include "pcg.cuh"

#include <cstring>
#include <mutex>

#include <cmath>

namespace msdd {

// R[d][e][a][b] = int_tau d_d phi_a d_e phi_b on the element tau scaled to
// x-edge 1 (edges 1, h_y / h_x, h_z / h_x), and the scalar-coefficient sum
// S[a][b] = sum_d R[d][d][a][b].  On the element of the mesh (edges h_x,
// h_y, h_z) the integrals are h_x^(dim-2) times these (Geom::rscale), so the
// constants depend on the element's shape only and are the same, bit for
// bit, for every mesh whose elements have that shape.
__constant__ double c_R[3][3][8][8];
__constant__ double c_S[8][8];

void upload_reference(const Geom& g) {
    double R[3][3][8][8];
    double S[8][8];
    memset(R, 0, sizeof(R));
    memset(S, 0, sizeof(S));
    const int dim = g.dim, nloc = 1 << dim;
    // h_d / h_x = n_x / n_d, a correctly rounded quotient: equal for equal shapes
    double h[3] = {1.0, (double)g.n[0] / g.n[1], dim == 3 ? (double)g.n[0] / g.n[2] : 1.0};
    // 2-point Gauss-Legendre on [0,1] per axis integrates the (bi/tri)quadratic
    // integrand exactly.
    const double gp[2] = {0.5 - 0.5 / std::sqrt(3.0), 0.5 + 0.5 / std::sqrt(3.0)};
    double vol = h[0] * h[1] * (dim == 3 ? h[2] : 1.0);
    int nq = 1 << dim;
    for (int q = 0; q < nq; ++q) {
        double xi[3] = {gp[q & 1], gp[(q >> 1) & 1], gp[(q >> 2) & 1]};
        double grad[8][3];
        for (int a = 0; a < nloc; ++a) {
            int bit[3] = {a & 1, (a >> 1) & 1, (a >> 2) & 1};
            double val[3];
            for (int d = 0; d < dim; ++d) val[d] = bit[d] ? xi[d] : 1.0 - xi[d];
            for (int d = 0; d < dim; ++d) {
                double gd = (bit[d] ? 1.0 : -1.0) / h[d];
                for (int e = 0; e < dim; ++e)
                    if (e != d) gd *= val[e];
                grad[a][d] = gd;
            }
        }
        double w = vol / nq;
        for (int d = 0; d < dim; ++d)
            for (int e = 0; e < dim; ++e)
                for (int a = 0; a < nloc; ++a)
                    for (int b = 0; b < nloc; ++b) R[d][e][a][b] += w * grad[a][d] * grad[b][e];
    }
    for (int d = 0; d < dim; ++d)
        for (int a = 0; a < nloc; ++a)
            for (int b = 0; b < nloc; ++b) S[a][b] += R[d][d][a][b];
    // the reference matrices live in constant memory shared by every
    // hierarchy of the process: upload only when they change (hierarchies
    // whose elements have the same shape share them)
    static std::mutex mu;
    static double last_R[3][3][8][8], last_S[8][8];
    static bool have = false;
    std::lock_guard<std::mutex> lk(mu);
    if (have && memcmp(last_R, R, sizeof(R)) == 0 && memcmp(last_S, S, sizeof(S)) == 0) return;
    MSDD_CUDA(cudaMemcpyToSymbol(c_R, R, sizeof(R)));
    MSDD_CUDA(cudaMemcpyToSymbol(c_S, S, sizeof(S)));
    memcpy(last_R, R, sizeof(R));
    memcpy(last_S, S, sizeof(S));
    have = true;
}

namespace {

__device__ __forceinline__ double elem_entry(const Geom& g, long long e, int a, int b) {
    if (g.coeff_kind == 0) return g.coeff[e] * (c_S[a][b] * g.rscale);
    const double* k = g.coeff + e * g.ncomp;
    double K[3][3];
    if (g.dim == 2) {
        K[0][0] = k[0]; K[1][1] = k[1]; K[0][1] = K[1][0] = k[2];
    } else {
        K[0][0] = k[0]; K[1][1] = k[1]; K[2][2] = k[2];
        K[1][2] = K[2][1] = k[3];
        K[0][2] = K[2][0] = k[4];
        K[0][1] = K[1][0] = k[5];
    }
    double v = 0.0;
    for (int d = 0; d < g.dim; ++d)
        for (int f = 0; f < g.dim; ++f) v += K[d][f] * c_R[d][f][a][b];
    return v * g.rscale;
}

// sum over elements tau of the element box containing nodes x and x + o of
// a_tau(phi_{x+o}, phi_x).
// Element l belongs to another fine subdomain as well: boxes are products of
// per-axis intervals, so the element lies in >= 2 boxes iff some axis does.
__device__ __forceinline__ bool overlap_element(const Geom& g, const int l[3]) {
    for (int d = 0; d < g.dim; ++d)
        if (g.ecov[d][l[d]] >= 2) return true;
    return false;
}

// ring: sum only the elements that belong to another subdomain too (b^2)
__device__ double stencil_coef(const Geom& g, const int* elo, const int* ehi, const int x[3], const int o[3],
                               bool ring = false) {
    int lo[3], cnt[3];
    for (int d = 0; d < 3; ++d) {
        if (d >= g.dim) { lo[d] = 0; cnt[d] = 1; continue; }
        if (o[d] < 0) { lo[d] = x[d] - 1; cnt[d] = 1; }
        else if (o[d] > 0) { lo[d] = x[d]; cnt[d] = 1; }
        else { lo[d] = x[d] - 1; cnt[d] = 2; }
    }
    double v = 0.0;
    for (int kz = 0; kz < cnt[2]; ++kz)
        for (int ky = 0; ky < cnt[1]; ++ky)
            for (int kx = 0; kx < cnt[0]; ++kx) {
                int l[3] = {lo[0] + kx, lo[1] + ky, lo[2] + kz};
                bool inside = true;
                for (int d = 0; d < g.dim; ++d)
                    if (l[d] < elo[d] || l[d] >= ehi[d]) inside = false;
                if (!inside || (ring && !overlap_element(g, l))) continue;
                int a = 0, b = 0;
                for (int d = 0; d < g.dim; ++d) {
                    a |= (x[d] - l[d]) << d;
                    b |= (x[d] + o[d] - l[d]) << d;
                }
                long long e = l[0] + (long long)g.n[0] * (l[1] + (long long)g.n[1] * l[2]);
                v += elem_entry(g, e, a, b);
            }
    return v;
}

__device__ __forceinline__ double chi_at(const Geom& g, const ProbBox& pb, const int* count, const int x[3]) {
    if (!in_box(pb.dlo, pb.dhi, x, g.dim)) return 0.0;
    return 1.0 / (double)count[unknown_index(g, x)];
}

__global__ void k_pou_count(Geom g, const ProbBox* __restrict__ boxes, int* __restrict__ count) {
    const ProbBox pb = boxes[blockIdx.y];
    int n = box_size(pb.dlo, pb.dhi, g.dim);
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        int x[3];
        box_coords(r, pb.dlo, pb.dhi, g.dim, x);
        atomicAdd(&count[unknown_index(g, x)], 1);
    }
}

template <typename T>
__global__ void k_assemble(Geom g, const ProbBox* __restrict__ boxes, const int* __restrict__ count, T* __restrict__ tiles,
                           const int* __restrict__ kb_, const long long* __restrict__ toff_, int mode, double sigma) {
    const int i = blockIdx.y;
    const ProbBox pb = boxes[i];
    const int* lo = mode == 0 ? pb.dlo : pb.nlo;
    const int* hi = mode == 0 ? pb.dhi : pb.nhi;
    const int n = box_size(lo, hi, g.dim);
    const int kb = kb_[i];
    const long long toff = toff_[i];
    const int noff = g.dim == 3 ? 27 : 9;
    for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < (long long)n * noff;
         w += (long long)gridDim.x * blockDim.x) {
        int r = (int)(w / noff), oi = (int)(w % noff);
        int o[3] = {oi % 3 - 1, (oi / 3) % 3 - 1, g.dim == 3 ? oi / 9 - 1 : 0};
        int x[3], y[3];
        box_coords(r, lo, hi, g.dim, x);
        for (int d = 0; d < 3; ++d) y[d] = x[d] + o[d];
        if (!in_box(lo, hi, y, g.dim)) continue;
        int c = box_index(lo, hi, y, g.dim);
        if (c > r) continue;   // lower triangle only
        double v = stencil_coef(g, pb.elo, pb.ehi, x, o);
        if (mode == 1) {
            // K = Abar + sigma B with B of the chosen right-hand side form
            const double cx = chi_at(g, pb, count, x), cy = chi_at(g, pb, count, y);
            if (g.blf == 3) v *= 1.0 + sigma * (1.0 - cx) * (1.0 - cy);
            else if (g.blf == 2) v += sigma * cx * stencil_coef(g, pb.elo, pb.ehi, x, o, true) * cy;
            else v *= 1.0 + sigma * cx * cy;
        }
        int R = r / NB, C = c / NB;
        tiles[toff + ((long long)R * (kb + 1) + (R - C)) * NB2 + (r % NB) * NB + (c % NB)] = (T)v;
    }
}

// One thread per (row, chunk of 8 columns).
__global__ void k_apply_neumann(Geom g, const ProbBox* __restrict__ boxes, const int* __restrict__ count,
                                const long long* __restrict__ roff_, const double* __restrict__ X,
                                double* __restrict__ AX, double* __restrict__ BX, int ldx, int ncols,
                                const int* __restrict__ skip) {
    const int i = blockIdx.y;
    if (skip && skip[i]) return;
    const ProbBox pb = boxes[i];
    const int n = box_size(pb.nlo, pb.nhi, g.dim);
    const int nchunk = (ncols + 7) / 8;
    const long long roff = roff_[i];
    const int noff = g.dim == 3 ? 27 : 9;
    for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < (long long)n * nchunk;
         w += (long long)gridDim.x * blockDim.x) {
        int r = (int)(w / nchunk), ch = (int)(w % nchunk);
        int c0 = ch * 8, c1 = min(ncols, c0 + 8);
        int x[3];
        box_coords(r, pb.nlo, pb.nhi, g.dim, x);
        double ax[8], bx[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) { ax[c] = 0.0; bx[c] = 0.0; }
        const double chix = chi_at(g, pb, count, x);
        for (int oi = 0; oi < noff; ++oi) {
            int o[3] = {oi % 3 - 1, (oi / 3) % 3 - 1, g.dim == 3 ? oi / 9 - 1 : 0};
            int y[3];
            for (int d = 0; d < 3; ++d) y[d] = x[d] + o[d];
            if (!in_box(pb.nlo, pb.nhi, y, g.dim)) continue;
            double a = stencil_coef(g, pb.elo, pb.ehi, x, o);
            if (a == 0.0) continue;
            double chiy = chi_at(g, pb, count, y);
            const double* xr = X + (roff + box_index(pb.nlo, pb.nhi, y, g.dim)) * ldx;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                if (c0 + c < c1) {
                    double v = xr[c0 + c];
                    ax[c] += a * v;
                    bx[c] += a * chiy * v;
                }
            }
        }
        double* ar = AX + (roff + r) * ldx;
        double* br = BX + (roff + r) * ldx;
#pragma unroll
        for (int c = 0; c < 8; ++c)
            if (c0 + c < c1) { ar[c0 + c] = ax[c]; br[c0 + c] = chix * bx[c]; }
    }
}

// FP32 versions of the element entries and stencil coefficients (used only
// by the FP32 start phase of the eigensolver).
__device__ __forceinline__ float elem_entry_f(const Geom& g, long long e, int a, int b) {
    if (g.coeff_kind == 0) return (float)g.coeff[e] * (float)(c_S[a][b] * g.rscale);
    return (float)elem_entry(g, e, a, b);
}

__device__ float stencil_coef_f(const Geom& g, const int* elo, const int* ehi, const int x[3], const int o[3]) {
    int lo[3], cnt[3];
    for (int d = 0; d < 3; ++d) {
        if (d >= g.dim) { lo[d] = 0; cnt[d] = 1; continue; }
        if (o[d] < 0) { lo[d] = x[d] - 1; cnt[d] = 1; }
        else if (o[d] > 0) { lo[d] = x[d]; cnt[d] = 1; }
        else { lo[d] = x[d] - 1; cnt[d] = 2; }
    }
    float v = 0.f;
    for (int kz = 0; kz < cnt[2]; ++kz)
        for (int ky = 0; ky < cnt[1]; ++ky)
            for (int kx = 0; kx < cnt[0]; ++kx) {
                int l[3] = {lo[0] + kx, lo[1] + ky, lo[2] + kz};
                bool inside = true;
                for (int d = 0; d < g.dim; ++d)
                    if (l[d] < elo[d] || l[d] >= ehi[d]) inside = false;
                if (!inside) continue;
                int a = 0, b = 0;
                for (int d = 0; d < g.dim; ++d) {
                    a |= (x[d] - l[d]) << d;
                    b |= (x[d] + o[d] - l[d]) << d;
                }
                long long e = l[0] + (long long)g.n[0] * (l[1] + (long long)g.n[1] * l[2]);
                v += elem_entry_f(g, e, a, b);
            }
    return v;
}

// W = X Abar X applied to X in FP32 arithmetic (one thread per row and chunk
// of 8 columns); rows beyond n are written as zero.
__global__ void k_apply_b32(Geom g, const ProbBox* __restrict__ boxes, const int* __restrict__ count,
                            const long long* __restrict__ roff_, const int* __restrict__ K_,
                            const double* __restrict__ X, double* __restrict__ W, int ldx, int ncols) {
    const int i = blockIdx.y;
    const ProbBox pb = boxes[i];
    const int n = box_size(pb.nlo, pb.nhi, g.dim);
    const int rows = K_[i] * NB;
    const int nchunk = (ncols + 7) / 8;
    const long long roff = roff_[i];
    const int noff = g.dim == 3 ? 27 : 9;
    for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < (long long)rows * nchunk;
         w += (long long)gridDim.x * blockDim.x) {
        int r = (int)(w / nchunk), c0 = (int)(w % nchunk) * 8;
        int c1 = min(ncols, c0 + 8);
        float bx[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) bx[c] = 0.f;
        float chix = 0.f;
        if (r < n) {
            int x[3];
            box_coords(r, pb.nlo, pb.nhi, g.dim, x);
            chix = (float)chi_at(g, pb, count, x);
            if (chix != 0.f) {
                for (int oi = 0; oi < noff; ++oi) {
                    int o[3] = {oi % 3 - 1, (oi / 3) % 3 - 1, g.dim == 3 ? oi / 9 - 1 : 0};
                    int y[3];
                    for (int d = 0; d < 3; ++d) y[d] = x[d] + o[d];
                    if (!in_box(pb.nlo, pb.nhi, y, g.dim)) continue;
                    float chiy = (float)chi_at(g, pb, count, y);
                    if (chiy == 0.f) continue;
                    float a = stencil_coef_f(g, pb.elo, pb.ehi, x, o) * chiy;
                    const double* xr = X + (roff + box_index(pb.nlo, pb.nhi, y, g.dim)) * ldx;
#pragma unroll
                    for (int c = 0; c < 8; ++c)
                        if (c0 + c < c1) bx[c] += a * (float)xr[c0 + c];
                }
            }
        }
        double* wr = W + (roff + r) * ldx;
#pragma unroll
        for (int c = 0; c < 8; ++c)
            if (c0 + c < c1) wr[c0 + c] = (double)(chix * bx[c]);
    }
}

// ---- stored local stencils
__global__ void k_local_stencil(Geom g, const ProbBox* __restrict__ boxes, const int* __restrict__ count,
                                const long long* __restrict__ roff_, const int* __restrict__ K_,
                                double* __restrict__ A, double* __restrict__ B, float* __restrict__ B32) {
    const int i = blockIdx.y;
    const ProbBox pb = boxes[i];
    const int n = box_size(pb.nlo, pb.nhi, g.dim);
    const int rows = K_[i] * NB;
    const int noff = g.dim == 3 ? 27 : 9;
    const long long base = roff_[i] * noff;
    for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < (long long)rows * noff;
         w += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(w / noff), oi = (int)(w % noff);
        double a = 0.0, b = 0.0;
        if (r < n) {
            int x[3], y[3];
            box_coords(r, pb.nlo, pb.nhi, g.dim, x);
            const int o[3] = {oi % 3 - 1, (oi / 3) % 3 - 1, g.dim == 3 ? oi / 9 - 1 : 0};
            for (int d = 0; d < 3; ++d) y[d] = x[d] + o[d];
            if (in_box(pb.nlo, pb.nhi, y, g.dim)) {
                a = stencil_coef(g, pb.elo, pb.ehi, x, o);
                if (g.blf == 3)
                    b = (1.0 - chi_at(g, pb, count, x)) * a * (1.0 - chi_at(g, pb, count, y));
                else if (g.blf == 2)
                    b = chi_at(g, pb, count, x) * stencil_coef(g, pb.elo, pb.ehi, x, o, true) * chi_at(g, pb, count, y);
                else
                    b = chi_at(g, pb, count, x) * a * chi_at(g, pb, count, y);
            }
        }
        A[base + w] = a;
        B[base + w] = b;
        B32[base + w] = (float)b;
    }
}

// row offset of neighbour oi in the lexicographic Neumann-box layout
__device__ __forceinline__ int nbr_offset(int oi, int w0, int w1, int dim) {
    return (oi % 3 - 1) + w0 * ((oi / 3) % 3 - 1) + (dim == 3 ? w0 * w1 * (oi / 9 - 1) : 0);
}

// One thread per (row, chunk of 8 columns).  A zero coefficient marks a
// neighbour outside the box (its row is not read).  DF: the products are
// accumulated in double-float (split_f64, df_fma) on the FP32 pipes.
template <bool DF>
__global__ void __launch_bounds__(128) k_apply_local(const ProbBox* __restrict__ boxes, int dim,
                                                     const long long* __restrict__ roff_, const double* __restrict__ A,
                                                     const double* __restrict__ B, const double* __restrict__ X,
                                                     double* __restrict__ AX, double* __restrict__ BX, int ldx,
                                                     int ncols, const int* __restrict__ skip) {
    const int i = blockIdx.y;
    if (skip && skip[i]) return;
    const ProbBox pb = boxes[i];
    const int n = box_size(pb.nlo, pb.nhi, dim);
    const int w0 = pb.nhi[0] - pb.nlo[0] + 1, w1 = dim >= 2 ? pb.nhi[1] - pb.nlo[1] + 1 : 1;
    const int noff = dim == 3 ? 27 : 9;
    const int nchunk = (ncols + 7) / 8;
    const long long roff = roff_[i];
    for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < (long long)n * nchunk;
         w += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(w / nchunk), c0 = (int)(w % nchunk) * 8;
        const int c1 = min(ncols, c0 + 8);
        double ax[8], bx[8];
        float axh[8], axl[8], bxh[8], bxl[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) { ax[c] = 0.0; bx[c] = 0.0; axh[c] = axl[c] = bxh[c] = bxl[c] = 0.f; }
        const double* ar = A + (roff + r) * noff;
        const double* br = B + (roff + r) * noff;
        for (int oi = 0; oi < noff; ++oi) {
            const double a = ar[oi], b = br[oi];
            if (a == 0.0 && b == 0.0) continue;
            const double* xr = X + (roff + r + nbr_offset(oi, w0, w1, dim)) * ldx;
            if constexpr (DF) {
                float ah, al, bh, bl;
                split_f64(a, ah, al);
                split_f64(b, bh, bl);
#pragma unroll
                for (int c = 0; c < 8; ++c)
                    if (c0 + c < c1) {
                        float vh, vl;
                        split_f64(xr[c0 + c], vh, vl);
                        df_fma(axh[c], axl[c], ah, al, vh, vl);
                        df_fma(bxh[c], bxl[c], bh, bl, vh, vl);
                    }
            } else {
#pragma unroll
                for (int c = 0; c < 8; ++c)
                    if (c0 + c < c1) {
                        const double v = xr[c0 + c];
                        ax[c] += a * v;
                        bx[c] += b * v;
                    }
            }
        }
        if constexpr (DF) {
#pragma unroll
            for (int c = 0; c < 8; ++c) { ax[c] = df_to_f64(axh[c], axl[c]); bx[c] = df_to_f64(bxh[c], bxl[c]); }
        }
        double* aw = AX + (roff + r) * ldx;
        double* bw = BX + (roff + r) * ldx;
#pragma unroll
        for (int c = 0; c < 8; ++c)
            if (c0 + c < c1) { aw[c0 + c] = ax[c]; bw[c0 + c] = bx[c]; }
    }
}

// AX = Abar X and BX = B X from the stored stencils, consumed at once:
// W = BX - (AX + sigma BX) diag(mu), mu_c = 1 / (theta_c + sigma) (the next
// right-hand side of the residual-correction subspace iteration; zero on
// padding rows) and, per 32-row block and column, the residual sums
// |AX - theta BX|^2 and |BX|^2 (EIG_ROWBLK layout).  Grid: (row blocks,
// problems); 128 threads = 32 rows x 4 groups of 4 columns.
// Since BX - (AX + sigma BX) mu = -(AX - theta BX) mu, W is one product of
// the residual R = AX - theta BX.  The squares are summed in FP32 (from
// integer-pipe conversions): they only feed the relative residual test, and
// the FP64 pipe is the bound of this kernel.  DF: the stencil products in
// double-float (split_f64, df_fma), R and W from their FP64 sums.
template <bool DF>
__global__ void __launch_bounds__(128) k_apply_rhs(const ProbBox* __restrict__ boxes, int dim,
                                                   const long long* __restrict__ roff_, const int* __restrict__ K_,
                                                   const double* __restrict__ A, const double* __restrict__ B,
                                                   const double* __restrict__ X, double* __restrict__ W, int ldx,
                                                   const int* __restrict__ p_, const double* __restrict__ theta,
                                                   double sigma, double* __restrict__ partial, int nblk_max,
                                                   const int* __restrict__ done) {
    static_assert(EIG_ROWBLK == NB, "row blocks are tile rows");
    __shared__ float sn[EIG_ROWBLK][PMAX + 1], sd[EIG_ROWBLK][PMAX + 1];
    __shared__ double sth[PMAX], smu[PMAX];
    const int i = blockIdx.y, blk = blockIdx.x;
    if (done[i]) return;
    const ProbBox pb = boxes[i];
    const int n = box_size(pb.nlo, pb.nhi, dim);
    const int rows = K_[i] * NB;
    const int r0 = blk * EIG_ROWBLK;
    if (r0 >= rows) return;   // rows is a multiple of NB = EIG_ROWBLK: every row of the block exists
    const int p = p_[i];
    const int w0 = pb.nhi[0] - pb.nlo[0] + 1, w1 = dim >= 2 ? pb.nhi[1] - pb.nlo[1] + 1 : 1;
    const int noff = dim == 3 ? 27 : 9;
    const long long roff = roff_[i];
    const int t = threadIdx.x, rr = t >> 2, cg = (t & 3) * 4;
    const int r = r0 + rr;
    if (t < p) {
        const double th = theta[i * PMAX + t];
        sth[t] = th;
        smu[t] = 1.0 / (th + sigma);
    }
    __syncthreads();
    for (int cb = cg; cb < p; cb += 16) {
        double ax[4] = {0.0, 0.0, 0.0, 0.0}, bx[4] = {0.0, 0.0, 0.0, 0.0};
        if (r < n) {
            float axh[4] = {0.f, 0.f, 0.f, 0.f}, axl[4] = {0.f, 0.f, 0.f, 0.f};
            float bxh[4] = {0.f, 0.f, 0.f, 0.f}, bxl[4] = {0.f, 0.f, 0.f, 0.f};
            const double* ar = A + (roff + r) * noff;
            const double* br = B + (roff + r) * noff;
            for (int oi = 0; oi < noff; ++oi) {
                const double a = ar[oi], b = br[oi];
                if (a == 0.0 && b == 0.0) continue;
                const double* xr = X + (roff + r + nbr_offset(oi, w0, w1, dim)) * ldx + cb;
                if constexpr (DF) {
                    float ah, al, bh, bl;
                    split_f64(a, ah, al);
                    split_f64(b, bh, bl);
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        if (cb + c < p) {
                            float vh, vl;
                            split_f64(xr[c], vh, vl);
                            df_fma(axh[c], axl[c], ah, al, vh, vl);
                            df_fma(bxh[c], bxl[c], bh, bl, vh, vl);
                        }
                } else {
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        if (cb + c < p) {
                            const double v = xr[c];
                            ax[c] += a * v;
                            bx[c] += b * v;
                        }
                }
            }
            if constexpr (DF) {
#pragma unroll
                for (int c = 0; c < 4; ++c) { ax[c] = df_to_f64(axh[c], axl[c]); bx[c] = df_to_f64(bxh[c], bxl[c]); }
            }
        }
        double* wr = W + (roff + r) * ldx + cb;
#pragma unroll
        for (int c = 0; c < 4; ++c)
            if (cb + c < p) {
                const double rv = ax[c] - sth[cb + c] * bx[c];
                wr[c] = r < n ? -rv * smu[cb + c] : 0.0;
                const float rf = f64_to_f32(rv), bf = f64_to_f32(bx[c]);
                sn[rr][cb + c] = rf * rf;
                sd[rr][cb + c] = bf * bf;
            }
    }
    __syncthreads();
    if (t < PMAX) {
        float a = 0.f, b = 0.f;
        for (int k = 0; t < p && k < EIG_ROWBLK; ++k) {
            a += sn[k][t];
            b += sd[k][t];
        }
        double* dst = partial + ((long long)i * nblk_max + blk) * 2 * PMAX;
        dst[t] = f32_to_f64(a);
        dst[PMAX + t] = f32_to_f64(b);
    }
}

// FP32 arithmetic, conversions on the integer pipe; padding rows zeroed.
__global__ void __launch_bounds__(128) k_apply_local_b32(const ProbBox* __restrict__ boxes, int dim,
                                                         const long long* __restrict__ roff_, const int* __restrict__ K_,
                                                         const float* __restrict__ B32, const double* __restrict__ X,
                                                         double* __restrict__ W, int ldx, int ncols) {
    const int i = blockIdx.y;
    const ProbBox pb = boxes[i];
    const int n = box_size(pb.nlo, pb.nhi, dim);
    const int rows = K_[i] * NB;
    const int w0 = pb.nhi[0] - pb.nlo[0] + 1, w1 = dim >= 2 ? pb.nhi[1] - pb.nlo[1] + 1 : 1;
    const int noff = dim == 3 ? 27 : 9;
    const int nchunk = (ncols + 7) / 8;
    const long long roff = roff_[i];
    for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < (long long)rows * nchunk;
         w += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(w / nchunk), c0 = (int)(w % nchunk) * 8;
        const int c1 = min(ncols, c0 + 8);
        float acc[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[c] = 0.f;
        if (r < n) {
            const float* br = B32 + (roff + r) * noff;
            for (int oi = 0; oi < noff; ++oi) {
                const float b = br[oi];
                if (b == 0.f) continue;
                const double* xr = X + (roff + r + nbr_offset(oi, w0, w1, dim)) * ldx;
#pragma unroll
                for (int c = 0; c < 8; ++c)
                    if (c0 + c < c1) acc[c] += b * f64_to_f32(xr[c0 + c]);
            }
        }
        double* wr = W + (roff + r) * ldx;
#pragma unroll
        for (int c = 0; c < 8; ++c)
            if (c0 + c < c1) wr[c0 + c] = f32_to_f64(acc[c]);
    }
}

// Stencil coefficients of the global operator: S[o * nun + u] = A(u, u + o)
// for the 3^d offsets o (zero where the neighbour is not an unknown).
__global__ void k_global_stencil(Geom g, double* __restrict__ S, long long nun) {
    int elo[3] = {0, 0, 0};
    int ehi[3] = {g.n[0], g.n[1], g.n[2]};
    const int noff = g.dim == 3 ? 27 : 9;
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < nun; u += (long long)gridDim.x * blockDim.x) {
        int xc[3];
        long long rem = u;
        for (int d = 0; d < 3; ++d) {
            if (d >= g.dim) { xc[d] = 0; continue; }
            xc[d] = g.ulo[d] + (int)(rem % g.ushape[d]);
            rem /= g.ushape[d];
        }
        for (int oi = 0; oi < noff; ++oi) {
            int o[3] = {oi % 3 - 1, (oi / 3) % 3 - 1, g.dim == 3 ? oi / 9 - 1 : 0};
            int yc[3];
            for (int d = 0; d < 3; ++d) yc[d] = xc[d] + o[d];
            S[(long long)oi * nun + u] = in_box(g.ulo, g.uhi, yc, g.dim) ? stencil_coef(g, elo, ehi, xc, o) : 0.0;
        }
    }
}

// q = A p from the stored stencil (one thread per unknown, neighbours of an
// x-row are contiguous), plus partial sums of p.q.
// q = S p over the unknowns with the stored 3^D-point stencil, and block
// partial sums of p.q.  Every neighbour index is clamped into [0, nun): a
// neighbour outside the unknown box has coefficient exactly 0 in S, so its
// term adds nothing and the loads need no branch.  1024 threads a block
// (the grid is the dot-product block count, a few blocks per SM).
template <int D>
__global__ void __launch_bounds__(1024) k_spmv_stencil_dot(Geom g, const double* __restrict__ S,
                                                           const double* __restrict__ p, double* __restrict__ q,
                                                           long long nun, double* __restrict__ partial,
                                                           const int* __restrict__ done, PcgScalars* sc, int fin) {
    __shared__ double red[1024];
    if (done && *done) return;
    constexpr int NOFF = D == 3 ? 27 : 9;
    const long long sy = g.ushape[0], sz = (long long)g.ushape[0] * g.ushape[1];
    double part = 0.0;
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < nun; u += (long long)gridDim.x * blockDim.x) {
        double acc = 0.0;
#pragma unroll
        for (int oi = 0; oi < NOFF; ++oi) {
            const double c = S[(long long)oi * nun + u];
            long long v = u + (oi % 3 - 1) + ((oi / 3) % 3 - 1) * sy + (D == 3 ? (oi / 9 - 1) * sz : 0);
            v = v < 0 ? 0 : (v >= nun ? nun - 1 : v);
            acc += c * p[v];
        }
        q[u] = acc;
        part += acc * p[u];
    }
    red[threadIdx.x] = part;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
    if (sc) pcg_last_block(sc, fin, partial);
}

__global__ void k_apply_global(Geom g, const double* __restrict__ x, double* __restrict__ y, long long nun) {
    int elo[3] = {0, 0, 0};
    int ehi[3] = {g.n[0], g.n[1], g.n[2]};
    const int noff = g.dim == 3 ? 27 : 9;
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < nun; u += (long long)gridDim.x * blockDim.x) {
        int xc[3];
        long long rem = u;
        for (int d = 0; d < 3; ++d) {
            if (d >= g.dim) { xc[d] = 0; continue; }
            xc[d] = g.ulo[d] + (int)(rem % g.ushape[d]);
            rem /= g.ushape[d];
        }
        double acc = 0.0;
        for (int oi = 0; oi < noff; ++oi) {
            int o[3] = {oi % 3 - 1, (oi / 3) % 3 - 1, g.dim == 3 ? oi / 9 - 1 : 0};
            int yc[3];
            for (int d = 0; d < 3; ++d) yc[d] = xc[d] + o[d];
            if (!in_box(g.ulo, g.uhi, yc, g.dim)) continue;
            acc += stencil_coef(g, elo, ehi, xc, o) * x[unknown_index(g, yc)];
        }
        y[u] = acc;
    }
}

__global__ void k_load_vector(Geom g, double f, double* __restrict__ b, long long nun) {
    double vol = 1.0;
    for (int d = 0; d < g.dim; ++d) vol /= g.n[d];
    const int nloc = 1 << g.dim;
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < nun; u += (long long)gridDim.x * blockDim.x) {
        long long rem = u;
        int cnt = 1;
        for (int d = 0; d < g.dim; ++d) {
            int xd = g.ulo[d] + (int)(rem % g.ushape[d]);
            rem /= g.ushape[d];
            cnt *= (xd > 0 ? 1 : 0) + (xd < g.n[d] ? 1 : 0);
        }
        b[u] = f * vol * cnt / nloc;
    }
}

__global__ void k_make_basis(Geom g, const ProbBox* __restrict__ boxes, const int* __restrict__ count,
                             const long long* __restrict__ roff_, const double* __restrict__ X, int ldx,
                             const int* __restrict__ m_, double* __restrict__ Phi, const long long* __restrict__ phioff,
                             int ldphi) {
    const int i = blockIdx.y;
    const ProbBox pb = boxes[i];
    const int nd = box_size(pb.dlo, pb.dhi, g.dim);
    const int m = m_[i];
    for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < nd * ldphi; w += gridDim.x * blockDim.x) {
        int r = w / ldphi, k = w % ldphi;
        int x[3];
        box_coords(r, pb.dlo, pb.dhi, g.dim, x);
        double v = 0.0;
        if (k < m) {
            int rn = box_index(pb.nlo, pb.nhi, x, g.dim);
            v = chi_at(g, pb, count, x) * X[(roff_[i] + rn) * ldx + k];
        }
        Phi[phioff[i] + (long long)r * ldphi + k] = v;
    }
}

}  // namespace

void pou_count(const Geom& g, const ProbBox* d_boxes, int P, int* d_count, cudaStream_t s) {
    long long nun = (long long)g.ushape[0] * g.ushape[1] * (g.dim == 3 ? g.ushape[2] : 1);
    MSDD_CUDA(cudaMemsetAsync(d_count, 0, nun * sizeof(int), s));
    dim3 grid(64, P);
    k_pou_count<<<grid, 256, 0, s>>>(g, d_boxes, d_count);
    MSDD_LAUNCH_CHECK();
}

void assemble_local_tiles(const Geom& g, const ProbBox* d_boxes, const int* d_count, TileBatch& tb, int mode,
                          double sigma, cudaStream_t s) {
    if (tb.P == 0) return;
    dim3 grid(128, tb.P);
    if (tb.prec)
        k_assemble<float><<<grid, 256, 0, s>>>(g, d_boxes, d_count, tb.tiles_f.p, tb.d_kb.p, tb.d_toff.p, mode, sigma);
    else
        k_assemble<double><<<grid, 256, 0, s>>>(g, d_boxes, d_count, tb.tiles_d.p, tb.d_kb.p, tb.d_toff.p, mode, sigma);
    MSDD_LAUNCH_CHECK();
}

void apply_neumann(const Geom& g, const ProbBox* d_boxes, const int* d_count, const TileBatch& layout,
                   const double* X, double* AX, double* BX, int ldx, int ncols, const int* skip, cudaStream_t s) {
    if (layout.P == 0) return;
    dim3 grid(64, layout.P);
    k_apply_neumann<<<grid, 128, 0, s>>>(g, d_boxes, d_count, layout.d_roff.p, X, AX, BX, ldx, ncols, skip);
    MSDD_LAUNCH_CHECK();
}

void apply_b32(const Geom& g, const ProbBox* d_boxes, const int* d_count, const TileBatch& layout, const double* X,
               double* W, int ldx, int ncols, cudaStream_t s) {
    if (layout.P == 0) return;
    dim3 grid(64, layout.P);
    k_apply_b32<<<grid, 128, 0, s>>>(g, d_boxes, d_count, layout.d_roff.p, layout.d_K.p, X, W, ldx, ncols);
    MSDD_LAUNCH_CHECK();
}

void build_local_stencil(const Geom& g, const ProbBox* d_boxes, const int* d_count, const TileBatch& layout,
                         LocalStencil& ls, cudaStream_t s) {
    ls.noff = g.dim == 3 ? 27 : 9;
    const size_t len = (size_t)layout.total_rows * ls.noff;
    ls.a.alloc(len);
    ls.b.alloc(len);
    ls.b32.alloc(len);
    if (layout.P == 0) return;
    dim3 grid(64, layout.P);
    k_local_stencil<<<grid, 256, 0, s>>>(g, d_boxes, d_count, layout.d_roff.p, layout.d_K.p, ls.a.p, ls.b.p, ls.b32.p);
    MSDD_LAUNCH_CHECK();
}

void apply_local(const LocalStencil& ls, const ProbBox* d_boxes, int dim, const TileBatch& layout, const double* X,
                 double* AX, double* BX, int ldx, int ncols, const int* skip, cudaStream_t s) {
    if (layout.P == 0) return;
    dim3 grid(64, layout.P);
    // the chosen form (FP32 factors) takes the double-float products
    if (layout.prec)
        k_apply_local<true><<<grid, 128, 0, s>>>(d_boxes, dim, layout.d_roff.p, ls.a.p, ls.b.p, X, AX, BX, ldx, ncols,
                                                 skip);
    else
        k_apply_local<false><<<grid, 128, 0, s>>>(d_boxes, dim, layout.d_roff.p, ls.a.p, ls.b.p, X, AX, BX, ldx, ncols,
                                                  skip);
    MSDD_LAUNCH_CHECK();
}

void apply_local_rhs(const LocalStencil& ls, const ProbBox* d_boxes, int dim, const TileBatch& layout,
                     const double* X, double* W, int ldx, const int* d_p, const double* theta, double sigma,
                     double* partial, int nblk_max, const int* done, cudaStream_t s) {
    if (layout.P == 0) return;
    dim3 grid(nblk_max, layout.P);
    if (layout.prec)
        k_apply_rhs<true><<<grid, 128, 0, s>>>(d_boxes, dim, layout.d_roff.p, layout.d_K.p, ls.a.p, ls.b.p, X, W, ldx,
                                               d_p, theta, sigma, partial, nblk_max, done);
    else
        k_apply_rhs<false><<<grid, 128, 0, s>>>(d_boxes, dim, layout.d_roff.p, layout.d_K.p, ls.a.p, ls.b.p, X, W, ldx,
                                                d_p, theta, sigma, partial, nblk_max, done);
    MSDD_LAUNCH_CHECK();
}

void apply_local_b32(const LocalStencil& ls, const ProbBox* d_boxes, int dim, const TileBatch& layout,
                     const double* X, double* W, int ldx, int ncols, cudaStream_t s) {
    if (layout.P == 0) return;
    dim3 grid(64, layout.P);
    k_apply_local_b32<<<grid, 128, 0, s>>>(d_boxes, dim, layout.d_roff.p, layout.d_K.p, ls.b32.p, X, W, ldx, ncols);
    MSDD_LAUNCH_CHECK();
}

void global_stencil(const Geom& g, double* S, cudaStream_t s) {
    long long nun = (long long)g.ushape[0] * g.ushape[1] * (g.dim == 3 ? g.ushape[2] : 1);
    unsigned blocks = (unsigned)std::min<long long>(ceil_div(nun, 256), 152 * 16);
    k_global_stencil<<<blocks, 256, 0, s>>>(g, S, nun);
    MSDD_LAUNCH_CHECK();
}

void spmv_stencil_dot(const Geom& g, const double* S, const double* p, double* q, double* partial, int nblocks,
                      const int* done, cudaStream_t s, PcgScalars* sc, int fin) {
    long long nun = (long long)g.ushape[0] * g.ushape[1] * (g.dim == 3 ? g.ushape[2] : 1);
    if (g.dim == 3)
        k_spmv_stencil_dot<3><<<nblocks, 1024, 0, s>>>(g, S, p, q, nun, partial, done, sc, fin);
    else
        k_spmv_stencil_dot<2><<<nblocks, 1024, 0, s>>>(g, S, p, q, nun, partial, done, sc, fin);
    MSDD_LAUNCH_CHECK();
}

void apply_global(const Geom& g, const double* x, double* y, cudaStream_t s) {
    long long nun = (long long)g.ushape[0] * g.ushape[1] * (g.dim == 3 ? g.ushape[2] : 1);
    unsigned blocks = (unsigned)std::min<long long>(ceil_div(nun, 256), 152 * 16);
    k_apply_global<<<blocks, 256, 0, s>>>(g, x, y, nun);
    MSDD_LAUNCH_CHECK();
}

void load_vector(const Geom& g, double f, double* b, cudaStream_t s) {
    long long nun = (long long)g.ushape[0] * g.ushape[1] * (g.dim == 3 ? g.ushape[2] : 1);
    unsigned blocks = (unsigned)std::min<long long>(ceil_div(nun, 256), 152 * 16);
    k_load_vector<<<blocks, 256, 0, s>>>(g, f, b, nun);
    MSDD_LAUNCH_CHECK();
}

void make_coarse_basis(const Geom& g, const ProbBox* d_boxes, const int* d_count, const TileBatch& nlayout,
                       const double* X, int ldx, const int* d_m, double* Phi, const long long* d_phioff, int ldphi,
                       int P, cudaStream_t s) {
    if (P == 0) return;
    dim3 grid(32, P);
    k_make_basis<<<grid, 256, 0, s>>>(g, d_boxes, d_count, nlayout.d_roff.p, X, ldx, d_m, Phi, d_phioff, ldphi);
    MSDD_LAUNCH_CHECK();
}

}  // namespace msdd

namespace msdd {
namespace {

constexpr int GCH = 16;   // elements staged per chunk in patch_gram

__global__ void __launch_bounds__(256) k_patch_gram(Geom g, const ProbBox* __restrict__ fine,
                                                    const double* __restrict__ Phi, const long long* __restrict__ phioff,
                                                    int ldphi, const int* __restrict__ m_,
                                                    const GramItem* __restrict__ items, double* __restrict__ G) {
    extern __shared__ double sm[];
    const GramItem it = items[blockIdx.x];
    const int nloc = 1 << g.dim;
    const int mj = m_[it.j], mjj = m_[it.jj];
    if (mj == 0 || mjj == 0) return;
    const ProbBox bj = fine[it.j], bjj = fine[it.jj];
    double* Pj = sm;
    double* Pjj = Pj + GCH * nloc * ldphi;
    double* Tm = Pjj + GCH * nloc * ldphi;
    int w[3] = {1, 1, 1};
    long long ne = 1;
    for (int d = 0; d < g.dim; ++d) { w[d] = it.ehi[d] - it.elo[d]; ne *= w[d]; }
    const int t = threadIdx.x;
    double acc[4] = {0, 0, 0, 0};
    const long long pj = phioff[it.j], pjj = phioff[it.jj];
    for (long long c0 = 0; c0 < ne; c0 += GCH) {
        __syncthreads();
        for (int e = t; e < GCH * nloc; e += blockDim.x) {
            long long el = c0 + e / nloc;
            int a = e % nloc;
            bool ok = el < ne;
            int x[3] = {0, 0, 0};
            if (ok) {
                long long rem = el;
                for (int d = 0; d < g.dim; ++d) {
                    x[d] = it.elo[d] + (int)(rem % w[d]) + ((a >> d) & 1);
                    rem /= w[d];
                }
            }
            bool inj = ok && in_box(bj.dlo, bj.dhi, x, g.dim);
            bool injj = ok && in_box(bjj.dlo, bjj.dhi, x, g.dim);
            int rj = inj ? box_index(bj.dlo, bj.dhi, x, g.dim) : 0;
            int rjj = injj ? box_index(bjj.dlo, bjj.dhi, x, g.dim) : 0;
            for (int k = 0; k < mj; ++k) Pj[e * ldphi + k] = inj ? Phi[pj + (long long)rj * ldphi + k] : 0.0;
            for (int k = 0; k < mjj; ++k) Pjj[e * ldphi + k] = injj ? Phi[pjj + (long long)rjj * ldphi + k] : 0.0;
        }
        __syncthreads();
        for (int e = t; e < GCH * nloc * mjj; e += blockDim.x) {
            int elc = e / (nloc * mjj), a = (e / mjj) % nloc, kk = e % mjj;
            long long el = c0 + elc;
            double v = 0.0;
            if (el < ne) {
                long long rem = el;
                int l[3] = {0, 0, 0};
                for (int d = 0; d < g.dim; ++d) { l[d] = it.elo[d] + (int)(rem % w[d]); rem /= w[d]; }
                long long E = l[0] + (long long)g.n[0] * (l[1] + (long long)g.n[1] * l[2]);
                for (int b = 0; b < nloc; ++b) v += elem_entry(g, E, a, b) * Pjj[(elc * nloc + b) * ldphi + kk];
            }
            Tm[(elc * nloc + a) * ldphi + kk] = v;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int e = t + q * blockDim.x;
            if (e >= mj * mjj) break;
            int k = e / mjj, kk = e % mjj;
            double s = 0.0;
            for (int ea = 0; ea < GCH * nloc; ++ea) s += Pj[ea * ldphi + k] * Tm[ea * ldphi + kk];
            acc[q] += s;
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        int e = t + q * blockDim.x;
        if (e < mj * mjj) G[it.goff + e] = acc[q];
    }
}

__global__ void k_apply_global_dot(Geom g, const double* __restrict__ x, double* __restrict__ y, long long nun,
                                   double* __restrict__ partial, const int* __restrict__ done) {
    __shared__ double red[256];
    if (done && *done) return;
    int elo[3] = {0, 0, 0};
    int ehi[3] = {g.n[0], g.n[1], g.n[2]};
    const int noff = g.dim == 3 ? 27 : 9;
    double part = 0.0;
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < nun; u += (long long)gridDim.x * blockDim.x) {
        int xc[3];
        long long rem = u;
        for (int d = 0; d < 3; ++d) {
            if (d >= g.dim) { xc[d] = 0; continue; }
            xc[d] = g.ulo[d] + (int)(rem % g.ushape[d]);
            rem /= g.ushape[d];
        }
        double acc = 0.0;
        for (int oi = 0; oi < noff; ++oi) {
            int o[3] = {oi % 3 - 1, (oi / 3) % 3 - 1, g.dim == 3 ? oi / 9 - 1 : 0};
            int yc[3];
            for (int d = 0; d < 3; ++d) yc[d] = xc[d] + o[d];
            if (!in_box(g.ulo, g.uhi, yc, g.dim)) continue;
            acc += stencil_coef(g, elo, ehi, xc, o) * x[unknown_index(g, yc)];
        }
        y[u] = acc;
        part += acc * x[u];
    }
    red[threadIdx.x] = part;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

}  // namespace

void patch_gram(const Geom& g, const ProbBox* d_fine, const double* Phi, const long long* d_phioff, int ldphi,
                const int* d_m, const GramItem* d_items, int nitems, double* G, cudaStream_t s) {
    if (nitems == 0) return;
    size_t smem = (size_t)3 * GCH * (1 << g.dim) * ldphi * sizeof(double);
    if (smem > 48 * 1024) raise_smem_limit(k_patch_gram, smem);
    k_patch_gram<<<nitems, 256, smem, s>>>(g, d_fine, Phi, d_phioff, ldphi, d_m, d_items, G);
    MSDD_LAUNCH_CHECK();
}

void apply_global_dot(const Geom& g, const double* p, double* q, double* partial, int nblocks, const int* done,
                      cudaStream_t s) {
    long long nun = (long long)g.ushape[0] * g.ushape[1] * (g.dim == 3 ? g.ushape[2] : 1);
    k_apply_global_dot<<<nblocks, 256, 0, s>>>(g, p, q, nun, partial, done);
    MSDD_LAUNCH_CHECK();
}

}  // namespace msdd
