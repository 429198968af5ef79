// Device-resident PCG scalar and vector kernels (see pcg.cuh).
#include "pcg.cuh"

namespace msdd {

namespace {

__device__ double sum_partials(const double* partial, int nblocks) {
    // one warp, fixed order: lane-strided then a fixed shuffle tree
    double v = 0.0;
    for (int k = threadIdx.x; k < nblocks; k += 32) v += partial[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(1024) k_start(const double* __restrict__ b, double* __restrict__ x, double* __restrict__ r, long long n,
                        double* __restrict__ partial) {
    __shared__ double red[1024];
    double part = 0.0;
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < n; u += (long long)gridDim.x * blockDim.x) {
        double v = b[u];
        r[u] = v;
        x[u] = 0.0;
        part += v * v;
    }
    red[threadIdx.x] = part;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void k_fin_bb(PcgScalars* sc, const double* __restrict__ partial, int nblocks, double tol, int maxit) {
    double v = sum_partials(partial, nblocks);
    if (threadIdx.x == 0) {
        sc->bb = v;
        sc->rr = v;
        sc->tol2 = tol * tol;
        sc->iters = 0;
        sc->maxit = maxit;
        sc->done = (v == 0.0) ? 1 : 0;
    }
}

__global__ void k_fin_rho0(PcgScalars* sc, const double* __restrict__ partial, int nblocks) {
    double v = sum_partials(partial, nblocks);
    if (threadIdx.x == 0) sc->rho = v;
}

__global__ void k_copy(const double* __restrict__ z, double* __restrict__ p, long long n, const PcgScalars* sc) {
    if (sc->done) return;
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < n; u += (long long)gridDim.x * blockDim.x)
        p[u] = z[u];
}


// fin = PCG_FIN_RR: the last block applies the r.r test itself
__global__ void __launch_bounds__(1024) k_axpy(PcgScalars* sc, double* __restrict__ x, double* __restrict__ r,
                       const double* __restrict__ p, const double* __restrict__ q, long long n,
                       double* __restrict__ partial, int fin) {
    __shared__ double red[1024];
    if (sc->done) return;
    const double a = sc->alpha;
    double part = 0.0;
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < n; u += (long long)gridDim.x * blockDim.x) {
        x[u] += a * p[u];
        double rv = r[u] - a * q[u];
        r[u] = rv;
        part += rv * rv;
    }
    red[threadIdx.x] = part;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
    if (fin) pcg_last_block(sc, fin, partial);
}



__global__ void k_update_p(const PcgScalars* sc, const double* __restrict__ z, double* __restrict__ p, long long n) {
    if (sc->done) return;
    const double b = sc->beta;
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < n; u += (long long)gridDim.x * blockDim.x)
        p[u] = z[u] + b * p[u];
}

unsigned vec_blocks(long long n) { return (unsigned)std::max(1u, std::min(ceil_div(n, 256), 152u * 8)); }

// ---- GMRES building blocks (Arnoldi vectors V[k] = V + k * n)
// partial[k * gridDim.x + b] = block b's share of V[k] . w
__global__ void k_mdot(const double* __restrict__ V, const double* __restrict__ w, long long n,
                       double* __restrict__ partial, const int* __restrict__ done) {
    if (done && *done) return;
    __shared__ double red[256];
    const double* v = V + (long long)blockIdx.y * n;
    double part = 0.0;
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < n; u += (long long)gridDim.x * blockDim.x)
        part += v[u] * w[u];
    red[threadIdx.x] = part;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[(long long)blockIdx.y * gridDim.x + blockIdx.x] = red[0];
}

// w = (init ? 0 : w) + alpha * sum_k c[k] V[k]
__global__ void k_vcomb(double* __restrict__ w, const double* __restrict__ V, const double* __restrict__ c, int nvec,
                        long long n, double alpha, int init, const int* __restrict__ done) {
    if (done && *done) return;
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < n; u += (long long)gridDim.x * blockDim.x) {
        double a = 0.0;
        for (int k = 0; k < nvec; ++k) a += c[k] * V[(long long)k * n + u];
        w[u] = (init ? 0.0 : w[u]) + alpha * a;
    }
}

__global__ void k_scale_to(const double* __restrict__ x, double* __restrict__ y, double a, long long n) {
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < n; u += (long long)gridDim.x * blockDim.x)
        y[u] = a * x[u];
}

__global__ void k_sub(const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ c, long long n,
                      const int* __restrict__ done) {
    if (done && *done) return;
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < n; u += (long long)gridDim.x * blockDim.x)
        c[u] = a[u] - b[u];
}

// y = (*a) x
__global__ void k_scale_dev(const double* __restrict__ x, double* __restrict__ y, const double* __restrict__ a,
                            long long n, const int* __restrict__ done) {
    if (done && *done) return;
    const double s = *a;
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < n; u += (long long)gridDim.x * blockDim.x)
        y[u] = s * x[u];
}

// Gram-Schmidt coefficients c[i] = sum_b partial[i * nbd + b] (b in order),
// added to column col of H (row-major, m columns; set on the first pass).
__global__ void k_gs_coef(const double* __restrict__ partial, int nbd, int nvec, double* __restrict__ H, int m,
                          int col, double* __restrict__ c, int accumulate, const GmresState* st) {
    if (st->done) return;
    for (int i = threadIdx.x; i < nvec; i += blockDim.x) {
        double v = 0.0;
        for (int q = 0; q < nbd; ++q) v += partial[(long long)i * nbd + q];
        c[i] = v;
        double* h = H + (long long)i * m + col;
        *h = accumulate ? *h + v : v;
    }
}

// End of Arnoldi step k: H(k+1, k) = ||w|| (partials summed in order),
// 1 / H(k+1, k) for the next basis vector, the previous Givens rotations on
// column k, a new rotation that zeroes H(k+1, k), the rotated right-hand
// side g, and the stop test on the residual estimate |g[k+1]|.
__global__ void k_gm_fin(const double* __restrict__ partial, int nbd, double* __restrict__ H, int m, int k,
                         double* __restrict__ cs, double* __restrict__ sn, double* __restrict__ gv,
                         double* __restrict__ hinv, GmresState* st) {
    if (st->done || threadIdx.x != 0) return;
    double ss = 0.0;
    for (int q = 0; q < nbd; ++q) ss += partial[q];
    const double h = sqrt(ss);
    auto Hat = [&](int i, int j) -> double& { return H[(long long)i * m + j]; };
    Hat(k + 1, k) = h;
    *hinv = h > 0.0 ? 1.0 / h : 0.0;
    for (int i = 0; i < k; ++i) {
        const double a = cs[i] * Hat(i, k) + sn[i] * Hat(i + 1, k);
        Hat(i + 1, k) = -sn[i] * Hat(i, k) + cs[i] * Hat(i + 1, k);
        Hat(i, k) = a;
    }
    const double den = hypot(Hat(k, k), Hat(k + 1, k));
    cs[k] = Hat(k, k) / den;
    sn[k] = Hat(k + 1, k) / den;
    Hat(k, k) = den;
    Hat(k + 1, k) = 0.0;
    gv[k + 1] = -sn[k] * gv[k];
    gv[k] = cs[k] * gv[k];
    st->it += 1;
    st->kk = k + 1;
    if (fabs(gv[k + 1]) < st->tol_bn) st->done = 1;
    else if (st->it >= st->maxit) st->done = 2;
}

}  // namespace

void gm_gs_coef(const double* partial, int nbd, int nvec, double* H, int m, int col, double* c, bool accumulate,
                const GmresState* st, cudaStream_t s) {
    k_gs_coef<<<1, 256, 0, s>>>(partial, nbd, nvec, H, m, col, c, accumulate ? 1 : 0, st);
    MSDD_LAUNCH_CHECK();
}
void gm_fin(const double* partial, int nbd, double* H, int m, int k, double* cs, double* sn, double* gv, double* hinv,
            GmresState* st, cudaStream_t s) {
    k_gm_fin<<<1, 32, 0, s>>>(partial, nbd, H, m, k, cs, sn, gv, hinv, st);
    MSDD_LAUNCH_CHECK();
}
void vec_scale_dev(const double* x, double* y, const double* a, long long n, const int* done, cudaStream_t s) {
    k_scale_dev<<<vec_blocks(n), 256, 0, s>>>(x, y, a, n, done);
    MSDD_LAUNCH_CHECK();
}

void vec_mdot(const double* V, int nvec, const double* w, long long n, double* partial, int nblk, cudaStream_t s,
              const int* done) {
    k_mdot<<<dim3(nblk, nvec), 256, 0, s>>>(V, w, n, partial, done);
    MSDD_LAUNCH_CHECK();
}
void vec_comb(double* w, const double* V, const double* c, int nvec, long long n, double alpha, bool init,
              cudaStream_t s, const int* done) {
    k_vcomb<<<vec_blocks(n), 256, 0, s>>>(w, V, c, nvec, n, alpha, init ? 1 : 0, done);
    MSDD_LAUNCH_CHECK();
}
void vec_scale_to(const double* x, double* y, double a, long long n, cudaStream_t s) {
    k_scale_to<<<vec_blocks(n), 256, 0, s>>>(x, y, a, n);
    MSDD_LAUNCH_CHECK();
}
void vec_sub(const double* a, const double* b, double* c, long long n, cudaStream_t s, const int* done) {
    k_sub<<<vec_blocks(n), 256, 0, s>>>(a, b, c, n, done);
    MSDD_LAUNCH_CHECK();
}

void pcg_start(const double* b, double* x, double* r, long long n, double* partial, int nblocks, cudaStream_t s) {
    k_start<<<nblocks, 1024, 0, s>>>(b, x, r, n, partial);
    MSDD_LAUNCH_CHECK();
}
void pcg_fin_bb(PcgScalars* sc, const double* partial, int nblocks, double tol, int maxit, cudaStream_t s) {
    k_fin_bb<<<1, 32, 0, s>>>(sc, partial, nblocks, tol, maxit);
    MSDD_LAUNCH_CHECK();
}
void pcg_fin_rho0(PcgScalars* sc, const double* partial, int nblocks, const double* z, double* p, long long n,
                  cudaStream_t s) {
    k_fin_rho0<<<1, 32, 0, s>>>(sc, partial, nblocks);
    MSDD_LAUNCH_CHECK();
    k_copy<<<vec_blocks(n), 256, 0, s>>>(z, p, n, sc);
    MSDD_LAUNCH_CHECK();
}
void pcg_axpy(PcgScalars* sc, double* x, double* r, const double* p, const double* q, long long n, double* partial,
              int nblocks, cudaStream_t s, bool fuse_rr) {
    k_axpy<<<nblocks, 1024, 0, s>>>(sc, x, r, p, q, n, partial, fuse_rr ? PCG_FIN_RR : PCG_FIN_NONE);
    MSDD_LAUNCH_CHECK();
}
void pcg_update_p(PcgScalars* sc, const double* z, double* p, long long n, cudaStream_t s) {
    k_update_p<<<vec_blocks(n), 256, 0, s>>>(sc, z, p, n);
    MSDD_LAUNCH_CHECK();
}

}  // namespace msdd
