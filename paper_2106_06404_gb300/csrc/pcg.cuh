// Device-resident preconditioned CG scalars and vector updates (Section 5:
// CG stopped when ||b - A x^m|| < tol ||b - A x^0||, x^0 = 0).  Every kernel
// reads the scalars from device memory and returns at once when `done` is
// set, so a fixed sequence of iterations can be captured in a CUDA graph and
// replayed until the host sees the flag.
#pragma once
#include "common.cuh"

namespace msdd {

struct PcgScalars {
    double rho, alpha, beta, bb, rr, pq, rz;
    double tol2;
    int done;      // 0 running, 1 converged, 2 maxit, 3 breakdown
    int iters;
    int maxit;
    int pad;
    unsigned ticket;   // blocks of a fused producer kernel that stored their partial (reset by the last)
    unsigned pad2;
};

// Finishing steps of a CG iteration that a producer kernel can apply itself
// (its last block to finish sums the block partials): alpha = rho / p.q,
// the r.r convergence test, beta = r.z / rho.
enum PcgFin { PCG_FIN_NONE = 0, PCG_FIN_ALPHA = 1, PCG_FIN_RR = 2, PCG_FIN_BETA = 3 };

#ifdef __CUDACC__
// the scalar updates of the finishing steps, given the summed partials v
__device__ __forceinline__ void pcg_fin_apply(PcgScalars* sc, int fin, double v) {
    if (fin == PCG_FIN_ALPHA) {
        sc->pq = v;
        if (!(v > 0.0)) { sc->done = 3; sc->alpha = 0.0; }
        else sc->alpha = sc->rho / v;
    } else if (fin == PCG_FIN_RR) {
        sc->rr = v;
        sc->iters += 1;
        if (v < sc->tol2 * sc->bb) sc->done = 1;
        else if (sc->iters >= sc->maxit) sc->done = 2;
    } else if (fin == PCG_FIN_BETA) {
        sc->rz = v;
        sc->beta = v / sc->rho;
        sc->rho = v;
    }
}
// Called by every thread of every block once thread 0 has stored
// partial[blockIdx.x]: the last block to arrive sums the gridDim.x partials
// (one warp, lane-strided then a fixed shuffle tree: a fixed order, so the
// result does not depend on which block arrives last) and applies `fin`.
__device__ __forceinline__ void pcg_last_block(PcgScalars* sc, int fin, const double* partial) {
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&sc->ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last || threadIdx.x >= 32) return;
    __threadfence();
    double v = 0.0;
    for (int k = threadIdx.x; k < (int)gridDim.x; k += 32) v += __ldcg(partial + k);
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) {
        pcg_fin_apply(sc, fin, v);
        sc->ticket = 0u;
    }
}
#endif

// r = b, x = 0, partial sums of b.b
void pcg_start(const double* b, double* x, double* r, long long n, double* partial, int nblocks, cudaStream_t s);
// bb = sum(partial); tol2 = tol^2; done = (bb == 0)
void pcg_fin_bb(PcgScalars* sc, const double* partial, int nblocks, double tol, int maxit, cudaStream_t s);
// rho = sum(partial) (r.z after the first preconditioner application); p = z
void pcg_fin_rho0(PcgScalars* sc, const double* partial, int nblocks, const double* z, double* p, long long n,
                  cudaStream_t s);
// x += alpha p, r -= alpha q, partial sums of r.r (fuse_rr: and the r.r
// convergence / maxit test, PCG_FIN_RR, applied by the kernel's last block)
void pcg_axpy(PcgScalars* sc, double* x, double* r, const double* p, const double* q, long long n, double* partial,
              int nblocks, cudaStream_t s, bool fuse_rr = false);
// p = z + beta p
void pcg_update_p(PcgScalars* sc, const double* z, double* p, long long n, cudaStream_t s);

// GMRES building blocks (Arnoldi vectors V[k] = V + k n, device).  Kernels
// given `done` return at once when it is set, so Arnoldi steps can be
// enqueued ahead of the host's convergence test.
// partial[k * nblk + b]: block b's share of V[k] . w, k < nvec.
void vec_mdot(const double* V, int nvec, const double* w, long long n, double* partial, int nblk, cudaStream_t s,
              const int* done = nullptr);
// w = (init ? 0 : w) + alpha sum_k c[k] V[k] (c device, nvec entries)
void vec_comb(double* w, const double* V, const double* c, int nvec, long long n, double alpha, bool init,
              cudaStream_t s, const int* done = nullptr);
void vec_scale_to(const double* x, double* y, double a, long long n, cudaStream_t s);   // y = a x
void vec_sub(const double* a, const double* b, double* c, long long n, cudaStream_t s,
             const int* done = nullptr);                                               // c = a - b
void vec_scale_dev(const double* x, double* y, const double* a, long long n, const int* done,
                   cudaStream_t s);                                                    // y = (*a) x

// Device state of one GMRES cycle.
struct GmresState {
    int done;      // 0 running, 1 residual estimate below tol_bn, 2 maxit
    int it;        // Arnoldi steps so far (all cycles)
    int maxit;
    int kk;        // steps of the current cycle
    double tol_bn; // tol * ||b||
};
// c[i] = sum_b partial[i * nbd + b], i < nvec; H(i, col) = c[i] (+= on later passes)
void gm_gs_coef(const double* partial, int nbd, int nvec, double* H, int m, int col, double* c, bool accumulate,
                const GmresState* st, cudaStream_t s);
// H(k+1, k) = sqrt(sum partial[0..nbd)), *hinv = 1 / H(k+1, k), Givens rotations, stop test
void gm_fin(const double* partial, int nbd, double* H, int m, int k, double* cs, double* sn, double* gv, double* hinv,
            GmresState* st, cudaStream_t s);

}  // namespace msdd
