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

__global__ void k_start(const double* __restrict__ b, double* __restrict__ x, double* __restrict__ r, long long n,
                        double* __restrict__ partial) {
    __shared__ double red[256];
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

__global__ void k_fin_alpha(PcgScalars* sc, const double* __restrict__ partial, int nblocks) {
    if (sc->done) return;
    double v = sum_partials(partial, nblocks);
    if (threadIdx.x == 0) {
        sc->pq = v;
        if (!(v > 0.0)) { sc->done = 3; sc->alpha = 0.0; }
        else sc->alpha = sc->rho / v;
    }
}

__global__ void k_axpy(const PcgScalars* sc, double* __restrict__ x, double* __restrict__ r,
                       const double* __restrict__ p, const double* __restrict__ q, long long n,
                       double* __restrict__ partial) {
    __shared__ double red[256];
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
}

__global__ void k_fin_rr(PcgScalars* sc, const double* __restrict__ partial, int nblocks) {
    if (sc->done) return;
    double v = sum_partials(partial, nblocks);
    if (threadIdx.x == 0) {
        sc->rr = v;
        sc->iters += 1;
        if (v < sc->tol2 * sc->bb) sc->done = 1;
        else if (sc->iters >= sc->maxit) sc->done = 2;
    }
}

__global__ void k_fin_beta(PcgScalars* sc, const double* __restrict__ partial, int nblocks) {
    if (sc->done) return;
    double v = sum_partials(partial, nblocks);
    if (threadIdx.x == 0) {
        sc->rz = v;
        sc->beta = v / sc->rho;
        sc->rho = v;
    }
}

__global__ void k_update_p(const PcgScalars* sc, const double* __restrict__ z, double* __restrict__ p, long long n) {
    if (sc->done) return;
    const double b = sc->beta;
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < n; u += (long long)gridDim.x * blockDim.x)
        p[u] = z[u] + b * p[u];
}

unsigned vec_blocks(long long n) { return (unsigned)std::max(1u, std::min(ceil_div(n, 256), 152u * 8)); }

}  // namespace

void pcg_start(const double* b, double* x, double* r, long long n, double* partial, int nblocks, cudaStream_t s) {
    k_start<<<nblocks, 256, 0, s>>>(b, x, r, n, partial);
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
void pcg_fin_alpha(PcgScalars* sc, const double* partial, int nblocks, cudaStream_t s) {
    k_fin_alpha<<<1, 32, 0, s>>>(sc, partial, nblocks);
    MSDD_LAUNCH_CHECK();
}
void pcg_axpy(PcgScalars* sc, double* x, double* r, const double* p, const double* q, long long n, double* partial,
              int nblocks, cudaStream_t s) {
    k_axpy<<<nblocks, 256, 0, s>>>(sc, x, r, p, q, n, partial);
    MSDD_LAUNCH_CHECK();
}
void pcg_fin_rr(PcgScalars* sc, const double* partial, int nblocks, cudaStream_t s) {
    k_fin_rr<<<1, 32, 0, s>>>(sc, partial, nblocks);
    MSDD_LAUNCH_CHECK();
}
void pcg_fin_beta(PcgScalars* sc, const double* partial, int nblocks, cudaStream_t s) {
    k_fin_beta<<<1, 32, 0, s>>>(sc, partial, nblocks);
    MSDD_LAUNCH_CHECK();
}
void pcg_update_p(PcgScalars* sc, const double* z, double* p, long long n, cudaStream_t s) {
    k_update_p<<<vec_blocks(n), 256, 0, s>>>(sc, z, p, n);
    MSDD_LAUNCH_CHECK();
}

}  // namespace msdd
