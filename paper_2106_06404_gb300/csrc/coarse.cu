// Coarse-level assembly, batched small GEMMs and preconditioner vector kernels.
#include "coarse.cuh"
#include "pcg.cuh"

namespace msdd {

namespace {

constexpr int COMBINE_NT = 1024;

__global__ void k_block_sum(const SumItem* __restrict__ items, const long long* __restrict__ contrib,
                            const double* __restrict__ G, double* __restrict__ dst) {
    const SumItem it = items[blockIdx.x];
    const int n = it.rows * it.cols;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        double v = 0.0;
        for (int c = it.cbeg; c < it.cend; ++c) v += G[contrib[c] + e];
        dst[it.doff + (long long)(e / it.cols) * it.ld + e % it.cols] = v;
    }
}

constexpr int GT = 32;

// C tile of 32 rows x 8 NQ columns per CTA (NQ < 4 when the items are
// narrower than 32 columns: the FP64 pipe bounds this kernel, so padded
// columns cost as much as real ones).  skip[z] != 0 leaves item z alone.
template <int NQ>
__global__ void __launch_bounds__(256) k_gemm_batched(const GemmItem* __restrict__ items, int transA, int transB,
                                                      double alpha, const double* __restrict__ A,
                                                      const double* __restrict__ B, double beta,
                                                      double* __restrict__ C, const int* __restrict__ gdone,
                                                      const int* __restrict__ skip) {
    constexpr int TN = 8 * NQ;
    __shared__ double sA[GT][GT + 1], sB[GT][TN + 1];
    if (gdone && *gdone) return;
    if (skip && skip[blockIdx.z]) return;
    const GemmItem it = items[blockIdx.z];
    const int row0 = blockIdx.y * GT, col0 = blockIdx.x * TN;
    if (row0 >= it.m || col0 >= it.n) return;
    const int t = threadIdx.x;
    const int r = t >> 3, cb = t & 7;
    double acc[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[q] = 0.0;
    for (int k0 = 0; k0 < it.k; k0 += GT) {
        for (int e = t; e < GT * GT; e += 256) {
            int a = e / GT, b = e % GT;       // sA[a = row][b = k]
            int gr = row0 + a, gk = k0 + b;
            double va = 0.0;
            if (gr < it.m && gk < it.k)
                va = transA ? A[it.aoff + (long long)gk * it.lda + gr] : A[it.aoff + (long long)gr * it.lda + gk];
            sA[a][b] = va;
        }
        for (int e = t; e < GT * TN; e += 256) {
            int a = e / TN, b = e % TN;       // sB[a = k][b = col]
            int bk = k0 + a, bc = col0 + b;
            double vb = 0.0;
            if (bk < it.k && bc < it.n)
                vb = transB ? B[it.boff + (long long)bc * it.ldb + bk] : B[it.boff + (long long)bk * it.ldb + bc];
            sB[a][b] = vb;
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < GT; ++k) {
            double a = sA[r][k];
#pragma unroll
            for (int q = 0; q < NQ; ++q) acc[q] += a * sB[k][cb + 8 * q];
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        int gr = row0 + r, gc = col0 + cb + 8 * q;
        if (gr < it.m && gc < it.n) {
            double* dst = C + it.coff + (long long)gr * it.ldc + gc;
            *dst = alpha * acc[q] + (beta != 0.0 ? beta * *dst : 0.0);
        }
    }
}

// y_b = alpha * op(A_b) x_b + beta * y_b, one warp per output entry
// (row of A, or column when transposed), eight warps per CTA.
__global__ void __launch_bounds__(256) k_gemv_batched(const GemmItem* __restrict__ items, int transA, double alpha,
                                                      const double* __restrict__ A, const double* __restrict__ x,
                                                      double beta, double* __restrict__ y,
                                                      const int* __restrict__ gdone) {
    if (gdone && *gdone) return;
    const GemmItem it = items[blockIdx.y];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = blockIdx.x * 8 + warp;
    if (row >= it.m) return;
    double s = 0.0;
    if (transA) {
        for (int k = lane; k < it.k; k += 32) s += A[it.aoff + (long long)k * it.lda + row] * x[it.boff + (long long)k * it.ldb];
    } else {
        const double* a = A + it.aoff + (long long)row * it.lda;
        for (int k = lane; k < it.k; k += 32) s += a[k] * x[it.boff + (long long)k * it.ldb];
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
        double* dst = y + it.coff + (long long)row * it.ldc;
        *dst = alpha * s + (beta != 0.0 ? beta * *dst : 0.0);
    }
}

__global__ void k_dense_shift(const double* __restrict__ A, double* __restrict__ Kd, const long long* __restrict__ aoff,
                              const int* __restrict__ n_, const int* __restrict__ nown_, double sigma) {
    const int i = blockIdx.y;
    const int n = n_[i], nown = nown_[i];
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)n * n;
         e += (long long)gridDim.x * blockDim.x) {
        int a = (int)(e / n), b = (int)(e % n);
        double v = A[aoff[i] + e];
        if (a < nown && b < nown) v *= 1.0 + sigma;
        Kd[aoff[i] + e] = v;
    }
}

// One CTA of 512 threads per fine subdomain; templated on the dimension so
// that node coordinates and box bounds stay in registers.
template <int D>
__global__ void __launch_bounds__(512) k_fine_gather_restrict(
    Geom g, const ProbBox* __restrict__ fine, const long long* __restrict__ droff, const int* __restrict__ dK,
    const double* __restrict__ r, double* __restrict__ rhs, const double* __restrict__ Phi,
    const long long* __restrict__ phioff, int ldphi, const int* __restrict__ m_, const long long* __restrict__ c1off,
    double* __restrict__ r1, const int* __restrict__ done) {
    __shared__ double red[PMAX][16];
    if (done && *done) return;
    const int j = blockIdx.x;
    int dlo[3], wd[3];
    int n = 1;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        dlo[d] = d < D ? fine[j].dlo[d] : 0;
        const int hi = d < D ? fine[j].dhi[d] : 0;
        wd[d] = hi >= dlo[d] ? hi - dlo[d] + 1 : 0;
        if (d < D) n *= wd[d];
    }
    const int rows = dK[j] * NB;
    const int m = m_[j];
    const int t = threadIdx.x;
    const int lane = t & 31, warp = t >> 5;
    double acc[PMAX];
#pragma unroll
    for (int k = 0; k < PMAX; ++k) acc[k] = 0.0;
    for (int rr = t; rr < rows; rr += blockDim.x) {
        double v = 0.0;
        if (rr < n) {
            int rem = rr;
            long long u = 0, stride = 1;
#pragma unroll
            for (int d = 0; d < D; ++d) {
                const int xd = dlo[d] + rem % wd[d];
                rem /= wd[d];
                u += (xd - g.ulo[d]) * stride;
                stride *= g.ushape[d];
            }
            v = r[u];
            const double* ph = Phi + phioff[j] + (long long)rr * ldphi;
#pragma unroll
            for (int k = 0; k < PMAX; ++k)
                if (k < m) acc[k] += ph[k] * v;
        }
        rhs[droff[j] + rr] = v;
    }
#pragma unroll
    for (int k = 0; k < PMAX; ++k) {
        if (k >= m) break;
        double v = acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[k][warp] = v;
    }
    __syncthreads();
    if (t < m) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[t][w];
        r1[c1off[j] + t] = v;
    }
}

// Threads over the unknowns (the grid is the dot-product block count);
// templated on the dimension so that node coordinates and the covering
// subdomains' box bounds stay in registers.  32-bit coordinate divisions
// (the set-up rejects 2^31 unknowns or more).
template <int D>
__global__ void __launch_bounds__(COMBINE_NT, 1) k_fine_combine(
    Geom g, CombineMaps cm, const ProbBox* __restrict__ fine, const long long* __restrict__ droff,
    const double* __restrict__ y, const double* __restrict__ Phi, const long long* __restrict__ phioff, int ldphi,
    const int* __restrict__ m_, const long long* __restrict__ c1off, const double* __restrict__ z1,
    double* __restrict__ z, const double* __restrict__ r, double* __restrict__ partial, long long nun,
    const int* __restrict__ done, int mode, PcgScalars* sc, int fin) {
    __shared__ double red[COMBINE_NT];
    if (done && *done) return;
    double part = 0.0;
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < nun; u += (long long)gridDim.x * blockDim.x) {
        int x[3] = {0, 0, 0}, lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
        unsigned rem = (unsigned)u;
#pragma unroll
        for (int d = 0; d < D; ++d) {
            const unsigned sd = (unsigned)g.ushape[d];
            const unsigned q = rem / sd;
            x[d] = g.ulo[d] + (int)(rem - q * sd);
            rem = q;
            lo[d] = cm.first[d][x[d]];
            hi[d] = cm.last[d][x[d]];
        }
        double acc = 0.0;
        int ncov = 0;
        for (int pz = lo[2]; pz <= hi[2]; ++pz)
            for (int py = lo[1]; py <= hi[1]; ++py)
                for (int px = lo[0]; px <= hi[0]; ++px) {
                    const int j = px + cm.parts[0] * (py + cm.parts[1] * pz);
                    int loc = 0, stride = 1;
#pragma unroll
                    for (int d = 0; d < D; ++d) {
                        const int dl = fine[j].dlo[d];
                        loc += (x[d] - dl) * stride;
                        stride *= fine[j].dhi[d] - dl + 1;
                    }
                    double v = (mode & COMB_Y) ? y[droff[j] + loc] : 0.0;
                    if (mode & COMB_COARSE) {
                        const int m = m_[j];
                        const double* ph = Phi + phioff[j] + (long long)loc * ldphi;
                        const double* zz = z1 + c1off[j];
                        for (int k = 0; k < m; ++k) v += ph[k] * zz[k];
                    }
                    acc += v;
                    ++ncov;
                }
        // restricted: chi_j(x) = 1 / N(x) for every subdomain j holding x
        if (mode & COMB_RAS) acc *= 1.0 / (double)ncov;
        if (mode & COMB_ACC) acc += z[u];
        z[u] = acc;
        if (partial) part += acc * r[u];
    }
    if (!partial) return;
    red[threadIdx.x] = part;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
    if (sc) pcg_last_block(sc, fin, partial);
}

__global__ void k_segment_copy(const long long* __restrict__ so, const long long* __restrict__ dof,
                               const int* __restrict__ len, const double* __restrict__ in, double* __restrict__ out,
                               int mode, const int* __restrict__ done) {
    if (done && *done) return;
    const int i = blockIdx.y;
    const int n = len[i];
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        double v = in[so[i] + k];
        if (mode) out[dof[i] + k] += v;
        else out[dof[i] + k] = v;
    }
}

__global__ void k_dot_partial(const double* __restrict__ x, const double* __restrict__ y, long long n,
                              double* __restrict__ partial) {
    __shared__ double red[256];
    double part = 0.0;
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < n; u += (long long)gridDim.x * blockDim.x)
        part += x[u] * y[u];
    red[threadIdx.x] = part;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

}  // namespace

void block_sum(const SumItem* d_items, int nitems, const long long* d_contrib, const double* G, double* dst,
               cudaStream_t s) {
    if (nitems == 0) return;
    k_block_sum<<<nitems, 256, 0, s>>>(d_items, d_contrib, G, dst);
    MSDD_LAUNCH_CHECK();
}

void gemm_batched(const GemmItem* d_items, int nitems, int transA, int transB, double alpha, const double* A,
                  const double* B, double beta, double* C, int max_m, int max_n, cudaStream_t s,
                  const int* gdone, const int* skip) {
    if (nitems == 0 || max_m == 0 || max_n == 0) return;
    const int nq = max_n >= 32 ? 4 : (max_n + 7) / 8;
    dim3 grid(ceil_div(max_n, 8 * nq), ceil_div(max_m, GT), nitems);
    switch (nq) {
        case 1: k_gemm_batched<1><<<grid, 256, 0, s>>>(d_items, transA, transB, alpha, A, B, beta, C, gdone, skip); break;
        case 2: k_gemm_batched<2><<<grid, 256, 0, s>>>(d_items, transA, transB, alpha, A, B, beta, C, gdone, skip); break;
        case 3: k_gemm_batched<3><<<grid, 256, 0, s>>>(d_items, transA, transB, alpha, A, B, beta, C, gdone, skip); break;
        default: k_gemm_batched<4><<<grid, 256, 0, s>>>(d_items, transA, transB, alpha, A, B, beta, C, gdone, skip); break;
    }
    MSDD_LAUNCH_CHECK();
}

void fine_gather_restrict(const Geom& g, const ProbBox* d_fine, const long long* d_droff, const int* d_K,
                          const double* r, double* rhs, const double* Phi, const long long* d_phioff, int ldphi,
                          const int* d_m, const long long* d_c1off, double* r1, int P, const int* done,
                          cudaStream_t s) {
    if (P == 0) return;
    if (g.dim == 3)
        k_fine_gather_restrict<3><<<P, 512, 0, s>>>(g, d_fine, d_droff, d_K, r, rhs, Phi, d_phioff, ldphi, d_m, d_c1off, r1,
                                             done);
    else
        k_fine_gather_restrict<2><<<P, 512, 0, s>>>(g, d_fine, d_droff, d_K, r, rhs, Phi, d_phioff, ldphi, d_m, d_c1off, r1,
                                             done);
    MSDD_LAUNCH_CHECK();
}

void fine_combine(const Geom& g, const CombineMaps& cm, const ProbBox* d_fine, const long long* d_droff,
                  const double* y, const double* Phi, const long long* d_phioff, int ldphi, const int* d_m,
                  const long long* d_c1off, const double* z1, double* z, const double* r, double* partial,
                  int nblocks, const int* done, cudaStream_t s, PcgScalars* sc, int fin) {
    fine_combine_mode(g, cm, d_fine, d_droff, y, Phi, d_phioff, ldphi, d_m, d_c1off, z1, z, r, partial, nblocks, done,
                      COMB_Y | COMB_COARSE, s, sc, fin);
}

void fine_combine_mode(const Geom& g, const CombineMaps& cm, const ProbBox* d_fine, const long long* d_droff,
                       const double* y, const double* Phi, const long long* d_phioff, int ldphi, const int* d_m,
                       const long long* d_c1off, const double* z1, double* z, const double* r, double* partial,
                       int nblocks, const int* done, int mode, cudaStream_t s, PcgScalars* sc, int fin) {
    long long nun = (long long)g.ushape[0] * g.ushape[1] * (g.dim == 3 ? g.ushape[2] : 1);
    if (!partial) sc = nullptr;                      // no partials, nothing to finish
    if (g.dim == 3)
        k_fine_combine<3><<<nblocks, COMBINE_NT, 0, s>>>(g, cm, d_fine, d_droff, y, Phi, d_phioff, ldphi, d_m, d_c1off,
                                                         z1, z, r, partial, nun, done, mode, sc, fin);
    else
        k_fine_combine<2><<<nblocks, COMBINE_NT, 0, s>>>(g, cm, d_fine, d_droff, y, Phi, d_phioff, ldphi, d_m, d_c1off,
                                                         z1, z, r, partial, nun, done, mode, sc, fin);
    MSDD_LAUNCH_CHECK();
}

void segment_copy(const long long* d_src_off, const long long* d_dst_off, const int* d_len, int P, int maxlen,
                  const double* in, double* out, int mode, const int* done, cudaStream_t s) {
    if (P == 0 || maxlen == 0) return;
    dim3 grid(std::max(1u, std::min(ceil_div(maxlen, 256), 64u)), P);
    k_segment_copy<<<grid, 256, 0, s>>>(d_src_off, d_dst_off, d_len, in, out, mode, done);
    MSDD_LAUNCH_CHECK();
}

int dot_blocks(long long n) { return (int)std::max(1u, std::min(ceil_div(n, 1024), 152u * 4)); }

void dot_partial(const double* x, const double* y, long long n, double* partial, int nblocks, cudaStream_t s) {
    k_dot_partial<<<nblocks, 256, 0, s>>>(x, y, n, partial);
    MSDD_LAUNCH_CHECK();
}

void gemv_batched(const GemmItem* d_items, int nitems, int transA, double alpha, const double* A, const double* x,
                  double beta, double* y, int max_m, cudaStream_t s, const int* gdone) {
    if (nitems == 0 || max_m == 0) return;
    dim3 grid(ceil_div(max_m, 8), nitems);
    k_gemv_batched<<<grid, 256, 0, s>>>(d_items, transA, alpha, A, x, beta, y, gdone);
    MSDD_LAUNCH_CHECK();
}

void dense_shift(const double* Abar, double* Kd, const long long* d_aoff, const int* d_n, const int* d_nown,
                 double sigma, int P, int nmax, cudaStream_t s) {
    if (P == 0) return;
    dim3 grid(std::max(1u, std::min(ceil_div((long long)nmax * nmax, 256), 256u)), P);
    k_dense_shift<<<grid, 256, 0, s>>>(Abar, Kd, d_aoff, d_n, d_nown, sigma);
    MSDD_LAUNCH_CHECK();
}

}  // namespace msdd

namespace msdd {
namespace {
__global__ void k_copy_blocks(const CopyItem* __restrict__ items, const double* __restrict__ src,
                              double* __restrict__ dst) {
    const CopyItem it = items[blockIdx.x];
    for (int e = threadIdx.x; e < it.rows * it.cols; e += blockDim.x) {
        int r = e / it.cols, c = e % it.cols;
        dst[it.doff + (long long)r * it.ldd + c] = src[it.soff + (long long)r * it.lds + c];
    }
}
}  // namespace
void copy_blocks(const CopyItem* d_items, int nitems, const double* src, double* dst, cudaStream_t s) {
    if (nitems == 0) return;
    k_copy_blocks<<<nitems, 256, 0, s>>>(d_items, src, dst);
    MSDD_LAUNCH_CHECK();
}
}  // namespace msdd
