// Batched subspace iteration with Rayleigh-Ritz (see eig.cuh).
#include "eig.cuh"

#include <cmath>

namespace msdd {

namespace {

constexpr int TPB = 256;
constexpr int LD = PMAX + 1;
constexpr int ROWBLK = 32;

__global__ void k_init(double* __restrict__ X, const int* __restrict__ n_, const int* __restrict__ K_,
                       const long long* __restrict__ roff_, const int* __restrict__ p_, int ldx,
                       unsigned long long seed, int* __restrict__ done, int* __restrict__ iters,
                       double* __restrict__ theta, double* __restrict__ best, int* __restrict__ best_it) {
    const int i = blockIdx.y;
    const int n = n_[i], p = p_[i];
    const long long rows = (long long)K_[i] * NB;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < rows * ldx;
         e += (long long)gridDim.x * blockDim.x) {
        int r = (int)(e / ldx), c = (int)(e % ldx);
        double v = 0.0;
        if (r < n && c < p) {
            uint64_t key = seed ^ ((uint64_t)i << 42) ^ ((uint64_t)r << 12) ^ (uint64_t)c;
            v = hash_uniform(key);
        }
        X[(roff_[i] + r) * ldx + c] = v;
    }
    if (blockIdx.x == 0 && threadIdx.x < PMAX) {
        theta[i * PMAX + threadIdx.x] = 0.0;
        if (threadIdx.x == 0) {
            done[i] = (n == 0 || p == 0) ? 1 : 0;
            iters[i] = 0;
            best[i] = 1e300;
            best_it[i] = 0;
        }
    }
}

__global__ void k_form_rhs(double* __restrict__ W, const double* __restrict__ AX, const double* __restrict__ BX,
                           const double* __restrict__ theta, const int* __restrict__ n_, const int* __restrict__ K_,
                           const long long* __restrict__ roff_, const int* __restrict__ p_, int ldx, double sigma,
                           int first, const int* __restrict__ done) {
    const int i = blockIdx.y;
    if (done[i]) return;
    const int n = n_[i], p = p_[i];
    const long long rows = (long long)K_[i] * NB;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < rows * ldx;
         e += (long long)gridDim.x * blockDim.x) {
        int r = (int)(e / ldx), c = (int)(e % ldx);
        long long idx = (roff_[i] + r) * ldx + c;
        double v = 0.0;
        if (r < n && c < p) {
            double bx = BX[idx];
            if (first) {
                v = bx;
            } else {
                double mu = 1.0 / (theta[i * PMAX + c] + sigma);
                v = bx - (AX[idx] + sigma * bx) * mu;
            }
        }
        W[idx] = v;
    }
}

__global__ void k_form_y(double* __restrict__ Y, const double* __restrict__ X, const double* __restrict__ W,
                         const double* __restrict__ theta, const int* __restrict__ n_, const int* __restrict__ K_,
                         const long long* __restrict__ roff_, const int* __restrict__ p_, int ldx, double sigma,
                         int first, const int* __restrict__ done) {
    const int i = blockIdx.y;
    if (done[i]) return;
    const int n = n_[i], p = p_[i];
    const long long rows = (long long)K_[i] * NB;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < rows * ldx;
         e += (long long)gridDim.x * blockDim.x) {
        int r = (int)(e / ldx), c = (int)(e % ldx);
        long long idx = (roff_[i] + r) * ldx + c;
        double v = 0.0;
        if (r < n && c < p) {
            v = W[idx];
            if (!first) v += X[idx] / (theta[i * PMAX + c] + sigma);
        }
        Y[idx] = v;
    }
}

// Y = X diag(mu) + W on a block of 32 rows, and per column the partial sums
// of W . R with R = BX - (AX + sigma BX) diag(mu) recomputed: W = K^+ R, so
// sum W.R = R^T K^+ R, the squared K^+-norm of the transformed residual.
__global__ void __launch_bounds__(TPB) k_form_y_knorm(double* __restrict__ Y, const double* __restrict__ X,
                                                      const double* __restrict__ W, const double* __restrict__ AX,
                                                      const double* __restrict__ BX, const double* __restrict__ theta,
                                                      const int* __restrict__ n_, const int* __restrict__ K_,
                                                      const long long* __restrict__ roff_, const int* __restrict__ p_,
                                                      int ldx, double sigma, double* __restrict__ partial,
                                                      int nblk_max, const int* __restrict__ done) {
    __shared__ double red[ROWBLK][LD];
    const int i = blockIdx.y, blk = blockIdx.x;
    if (done[i]) return;
    const int n = n_[i], p = p_[i];
    const long long rows = (long long)K_[i] * NB;
    const int r0 = blk * ROWBLK;
    if (r0 >= rows) return;
    const long long roff = roff_[i];
    const int t = threadIdx.x;
    const int rr = t >> 3, cb = t & 7;
    for (int q = 0; q < 4; ++q) {
        int c = cb + 8 * q;
        int r = r0 + rr;
        double v = 0.0, wr = 0.0;
        if (r < rows && c < ldx) {
            long long idx = (roff + r) * ldx + c;
            if (r < n && c < p) {
                double mu = 1.0 / (theta[i * PMAX + c] + sigma);
                double w = W[idx];
                double bx = BX[idx];
                double R = bx - (AX[idx] + sigma * bx) * mu;
                v = X[idx] * mu + w;
                wr = w * R;
            }
            Y[idx] = v;
        }
        red[rr][c] = wr;
    }
    __syncthreads();
    if (t < PMAX) {
        double a = 0.0;
        for (int k = 0; k < ROWBLK; ++k) a += red[k][t];
        partial[((long long)i * nblk_max + blk) * PMAX + t] = a;
    }
}

// H = Y^T AY, M = Y^T BY (symmetric, FP64), one CTA per problem.
__global__ void __launch_bounds__(TPB) k_gram(const double* __restrict__ Y, const double* __restrict__ AY,
                                              const double* __restrict__ BY, double* __restrict__ H,
                                              double* __restrict__ M, const int* __restrict__ n_,
                                              const long long* __restrict__ roff_, const int* __restrict__ p_,
                                              int ldx, const int* __restrict__ done) {
    __shared__ double sY[ROWBLK][LD], sA[ROWBLK][LD], sB[ROWBLK][LD];
    const int i = blockIdx.x;
    if (done[i]) return;
    const int n = n_[i], p = p_[i];
    const long long roff = roff_[i];
    const int npair = p * (p + 1) / 2;
    int pa[3], pb[3];
    double h[3] = {0, 0, 0}, m[3] = {0, 0, 0};
    for (int q = 0; q < 3; ++q) {
        int e = threadIdx.x + q * TPB;
        pa[q] = -1;
        if (e < npair) {
            // e -> (a, b) with a <= b
            int a = 0, rem = e;
            while (rem >= p - a) { rem -= p - a; ++a; }
            pa[q] = a;
            pb[q] = a + rem;
        }
    }
    for (int r0 = 0; r0 < n; r0 += ROWBLK) {
        __syncthreads();
        for (int e = threadIdx.x; e < ROWBLK * p; e += TPB) {
            int rr = e / p, c = e % p;
            int r = r0 + rr;
            long long idx = (roff + r) * ldx + c;
            bool ok = r < n;
            sY[rr][c] = ok ? Y[idx] : 0.0;
            sA[rr][c] = ok ? AY[idx] : 0.0;
            sB[rr][c] = ok ? BY[idx] : 0.0;
        }
        __syncthreads();
        for (int q = 0; q < 3; ++q) {
            if (pa[q] < 0) continue;
            int a = pa[q], b = pb[q];
            double hs = 0.0, ms = 0.0;
#pragma unroll 8
            for (int rr = 0; rr < ROWBLK; ++rr) {
                hs += sY[rr][a] * sA[rr][b];
                ms += sY[rr][a] * sB[rr][b];
            }
            h[q] += hs;
            m[q] += ms;
        }
    }
    for (int q = 0; q < 3; ++q) {
        if (pa[q] < 0) continue;
        int a = pa[q], b = pb[q];
        // symmetrise: average the two triangles' contributions is not needed, the
        // products Y^T AY are symmetric in exact arithmetic; keep (a,b) from a<=b.
        H[(long long)i * PMAX * PMAX + a * PMAX + b] = h[q];
        H[(long long)i * PMAX * PMAX + b * PMAX + a] = h[q];
        M[(long long)i * PMAX * PMAX + a * PMAX + b] = m[q];
        M[(long long)i * PMAX * PMAX + b * PMAX + a] = m[q];
    }
}

// ---- block-wide symmetric eigen-solver (parallel cyclic Jacobi, round robin)
template <typename T>
__device__ void rot_params(T app, T aqq, T apq, T& c, T& s) {
    const T tiny = sizeof(T) == 4 ? T(1e-9) : T(1e-18);
    if (apq == T(0) || fabs(apq) <= tiny * sqrt(fabs(app * aqq))) { c = T(1); s = T(0); return; }
    T th = (aqq - app) / (T(2) * apq);
    T t;
    if (fabs(th) > T(1e15)) t = T(0.5) / th;
    else t = (th >= T(0) ? T(1) : T(-1)) / (fabs(th) + sqrt(th * th + T(1)));
    c = T(1) / sqrt(t * t + T(1));
    s = t * c;
}

// S (q x q, q even) is overwritten by its eigenvalues on the diagonal; V =
// eigenvectors.  Sweeps stop when the off-diagonal mass falls below
// rel_tol^2 of the Frobenius mass, or after max_sweeps.
template <typename T>
__device__ void block_jacobi(T (*S)[LD], T (*V)[LD], int q, T* sc, T* ss, int* sa, int* sb, double* red,
                             double rel_tol2, int max_sweeps) {
    const int t = threadIdx.x;
    for (int e = t; e < q * q; e += TPB) V[e / q][e % q] = (e / q == e % q) ? T(1) : T(0);
    __syncthreads();
    double fro = 0.0;
    {
        double part = 0.0;
        for (int e = t; e < q * q; e += TPB) part += (double)S[e / q][e % q] * (double)S[e / q][e % q];
        red[t] = part;
        __syncthreads();
        for (int w = TPB / 2; w > 0; w >>= 1) {
            if (t < w) red[t] += red[t + w];
            __syncthreads();
        }
        fro = red[0];
        __syncthreads();
    }
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        double part = 0.0;
        for (int e = t; e < q * q; e += TPB) {
            int a = e / q, b = e % q;
            if (a != b) part += (double)S[a][b] * (double)S[a][b];
        }
        red[t] = part;
        __syncthreads();
        for (int w = TPB / 2; w > 0; w >>= 1) {
            if (t < w) red[t] += red[t + w];
            __syncthreads();
        }
        double off = red[0];
        __syncthreads();
        if (off <= rel_tol2 * fro || fro == 0.0) break;
        for (int step = 0; step < q - 1; ++step) {
            if (t < q / 2) {
                // circle method: position 0 fixed, the others rotate
                int pos1 = t, pos2 = q - 1 - t;
                int a = pos1 == 0 ? 0 : 1 + (pos1 - 1 + step) % (q - 1);
                int b = 1 + (pos2 - 1 + step) % (q - 1);
                if (a > b) { int tmp = a; a = b; b = tmp; }
                T c, s;
                rot_params<T>(S[a][a], S[b][b], S[a][b], c, s);
                sa[t] = a; sb[t] = b; sc[t] = c; ss[t] = s;
            }
            __syncthreads();
            for (int e = t; e < (q / 2) * q; e += TPB) {    // rows
                int j = e / q, k = e % q;
                if (ss[j] == T(0)) continue;
                int a = sa[j], b = sb[j];
                T x = S[a][k], y = S[b][k];
                S[a][k] = sc[j] * x - ss[j] * y;
                S[b][k] = ss[j] * x + sc[j] * y;
            }
            __syncthreads();
            for (int e = t; e < (q / 2) * q; e += TPB) {    // columns of S and V
                int j = e / q, k = e % q;
                if (ss[j] == T(0)) continue;
                int a = sa[j], b = sb[j];
                T x = S[k][a], y = S[k][b];
                S[k][a] = sc[j] * x - ss[j] * y;
                S[k][b] = ss[j] * x + sc[j] * y;
                T u = V[k][a], v = V[k][b];
                V[k][a] = sc[j] * u - ss[j] * v;
                V[k][b] = ss[j] * u + sc[j] * v;
            }
            __syncthreads();
        }
    }
}

// Eigen-decomposition of the symmetric q x q FP64 matrix S (overwritten by
// its eigenvalues on the diagonal, eigenvectors in V).  Most rotations are
// done in FP32 on a copy; the FP32 eigenvectors are re-orthonormalised in
// FP64 (modified Gram-Schmidt), S is transformed exactly in FP64 and FP64
// sweeps (quadratic convergence from the FP32 level, normally one or two)
// finish it.  W and U are FP64 scratch; U also holds the FP32 copies.
__device__ void mixed_jacobi(double (*S)[LD], double (*V)[LD], double (*W)[LD], double (*U)[LD], int q,
                             float* scf, float* ssf, double* sc, double* ss, double* coef, int* sa, int* sb,
                             double* red) {
    const int t = threadIdx.x;
    float (*G32)[LD] = reinterpret_cast<float (*)[LD]>(&U[0][0]);
    float (*V32)[LD] = G32 + PMAX;
    for (int e = t; e < q * q; e += TPB) G32[e / q][e % q] = (float)S[e / q][e % q];
    __syncthreads();
    block_jacobi<float>(G32, V32, q, scf, ssf, sa, sb, red, 1e-12, 12);
    for (int e = t; e < q * q; e += TPB) V[e / q][e % q] = (double)V32[e / q][e % q];
    __syncthreads();
    for (int k = 0; k < q; ++k) {
        if (t < 32) {
            double s2 = 0.0;
            for (int r = t; r < q; r += 32) s2 += V[r][k] * V[r][k];
            for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
            if (t == 0) red[0] = s2 > 0.0 ? 1.0 / sqrt(s2) : 0.0;
        }
        __syncthreads();
        const double inv = red[0];
        __syncthreads();
        for (int r = t; r < q; r += TPB) V[r][k] *= inv;
        __syncthreads();
        for (int j = k + 1 + t; j < q; j += TPB) {
            double d = 0.0;
            for (int r = 0; r < q; ++r) d += V[r][k] * V[r][j];
            coef[j] = d;
        }
        __syncthreads();
        for (int e = t; e < q * q; e += TPB) {
            int r = e / q, j = e % q;
            if (j > k) V[r][j] -= coef[j] * V[r][k];
        }
        __syncthreads();
    }
    // S <- V^T S V in FP64
    for (int e = t; e < q * q; e += TPB) {
        int a = e / q, b = e % q;
        double v = 0.0;
        for (int j = 0; j < q; ++j) v += S[a][j] * V[j][b];
        W[a][b] = v;
    }
    __syncthreads();
    for (int e = t; e < q * q; e += TPB) {
        int a = e / q, b = e % q;
        double v = 0.0;
        for (int j = 0; j < q; ++j) v += V[j][a] * W[j][b];
        U[a][b] = v;
    }
    __syncthreads();
    for (int e = t; e < q * q; e += TPB) {
        int a = e / q, b = e % q;
        S[a][b] = 0.5 * (U[a][b] + U[b][a]);
    }
    __syncthreads();
    block_jacobi<double>(S, W, q, sc, ss, sa, sb, red, 1e-30, 30);
    // V <- V W
    for (int e = t; e < q * q; e += TPB) {
        int a = e / q, b = e % q;
        double v = 0.0;
        for (int j = 0; j < q; ++j) v += V[a][j] * W[j][b];
        U[a][b] = v;
    }
    __syncthreads();
    for (int e = t; e < q * q; e += TPB) V[e / q][e % q] = U[e / q][e % q];
    __syncthreads();
}

// Rayleigh-Ritz on (H, M): column scaling D = diag(M)^{-1/2}, Cholesky of
// D M D (Jacobi-based pseudo-inverse square root if it is not numerically
// positive definite), Jacobi on the reduced standard problem.
__global__ void __launch_bounds__(TPB) k_rayleigh_ritz(const double* __restrict__ H, const double* __restrict__ M,
                                                       double* __restrict__ C, double* __restrict__ theta,
                                                       const int* __restrict__ p_, int* __restrict__ rank,
                                                       const int* __restrict__ done) {
    __shared__ double S[PMAX][LD], V[PMAX][LD], L[PMAX][LD], T[PMAX][LD], U[PMAX][LD];
    __shared__ double dsc[PMAX], sc[PMAX / 2], ss[PMAX / 2], red[TPB], th[PMAX], coef[PMAX];
    __shared__ float scf[PMAX / 2], ssf[PMAX / 2];
    __shared__ int sa[PMAX / 2], sb[PMAX / 2], perm[PMAX];
    __shared__ int s_fail;
    const int i = blockIdx.x;
    if (done[i]) return;
    const int p = p_[i];
    const int q = p + (p & 1);
    const int t = threadIdx.x;
    const double* Hi = H + (long long)i * PMAX * PMAX;
    const double* Mi = M + (long long)i * PMAX * PMAX;
    if (t < PMAX) {
        double mkk = t < p ? Mi[t * PMAX + t] : 0.0;
        dsc[t] = mkk > 0.0 ? 1.0 / sqrt(mkk) : 0.0;
    }
    if (t == 0) s_fail = 0;
    __syncthreads();
    // scaled M into L, scaled H into T (q x q, dummy rows zero)
    for (int e = t; e < q * q; e += TPB) {
        int a = e / q, b = e % q;
        bool ok = a < p && b < p;
        L[a][b] = ok ? dsc[a] * Mi[a * PMAX + b] * dsc[b] : 0.0;
        T[a][b] = ok ? dsc[a] * Hi[a * PMAX + b] * dsc[b] : 0.0;
    }
    __syncthreads();
    // Cholesky of L in place (lower), columns with dsc == 0 are dropped
    for (int k = 0; k < p; ++k) {
        if (t == 0) {
            double d = L[k][k];
            if (dsc[k] == 0.0) L[k][k] = 0.0;
            else if (!(d > 1e-13)) { s_fail = 1; L[k][k] = 0.0; }
            else L[k][k] = sqrt(d);
        }
        __syncthreads();
        double lkk = L[k][k];
        if (t > k && t < p) L[t][k] = lkk > 0.0 ? L[t][k] / lkk : 0.0;
        __syncthreads();
        for (int e = t; e < p * p; e += TPB) {
            int a = e / p, b = e % p;
            if (b > k && a >= b) L[a][b] -= L[a][k] * L[b][k];
        }
        __syncthreads();
    }
    int r = 0;
    if (!s_fail) {
        // G = L^{-1} T L^{-T}: first S = L^{-1} T (column-parallel forward substitution)
        for (int k = 0; k < p; ++k) {
            if (t < p) {
                double v = T[k][t];
                for (int j = 0; j < k; ++j) v -= L[k][j] * S[j][t];
                S[k][t] = L[k][k] > 0.0 ? v / L[k][k] : 0.0;
            }
            __syncthreads();
        }
        // V = L^{-1} S^T  -> G (symmetric); reuse V as temporary
        for (int k = 0; k < p; ++k) {
            if (t < p) {
                double v = S[t][k];
                for (int j = 0; j < k; ++j) v -= L[k][j] * V[j][t];
                V[k][t] = L[k][k] > 0.0 ? v / L[k][k] : 0.0;
            }
            __syncthreads();
        }
        for (int e = t; e < q * q; e += TPB) {
            int a = e / q, b = e % q;
            double v = (a < p && b < p) ? 0.5 * (V[a][b] + V[b][a]) : 0.0;
            if (a < p && b < p && (L[a][a] == 0.0 || L[b][b] == 0.0)) v = (a == b) ? 1e300 : 0.0;
            S[a][b] = v;
        }
        __syncthreads();
        mixed_jacobi(S, V, T, U, q, scf, ssf, sc, ss, coef, sa, sb, red);
        // C = D L^{-T} V  (backward substitution, column-parallel), into T
        for (int k = p - 1; k >= 0; --k) {
            if (t < q) {
                double v = V[k][t];
                for (int j = k + 1; j < p; ++j) v -= L[j][k] * T[j][t];
                T[k][t] = L[k][k] > 0.0 ? v / L[k][k] : 0.0;
            }
            __syncthreads();
        }
        for (int k = 0; k < p; ++k) r += L[k][k] > 0.0 ? 1 : 0;
    } else {
        // pseudo-inverse square root of D M D via its eigen-decomposition
        for (int e = t; e < q * q; e += TPB) {
            int a = e / q, b = e % q;
            S[a][b] = (a < p && b < p) ? dsc[a] * Mi[a * PMAX + b] * dsc[b] : 0.0;
        }
        __syncthreads();
        block_jacobi<double>(S, V, q, sc, ss, sa, sb, red, 1e-30, 30);   // S diag = s, V = U
        double smax = 0.0;
        for (int k = 0; k < p; ++k) smax = fmax(smax, S[k][k]);
        __syncthreads();
        if (t < PMAX) th[t] = (t < p && S[t][t] > 1e-13 * smax) ? 1.0 / sqrt(S[t][t]) : 0.0;
        // L <- U diag(th): reuse L as U_scaled
        __syncthreads();
        for (int e = t; e < q * q; e += TPB) {
            int a = e / q, b = e % q;
            L[a][b] = (a < p && b < p) ? V[a][b] * th[b] : 0.0;
        }
        __syncthreads();
        // G = L^T T L  (T holds scaled H);  S = T L first
        for (int e = t; e < q * q; e += TPB) {
            int a = e / q, b = e % q;
            double v = 0.0;
            for (int j = 0; j < p; ++j) v += T[a][j] * L[j][b];
            S[a][b] = v;
        }
        __syncthreads();
        for (int e = t; e < q * q; e += TPB) {
            int a = e / q, b = e % q;
            double v = 0.0;
            for (int j = 0; j < p; ++j) v += L[j][a] * S[j][b];
            V[a][b] = v;
        }
        __syncthreads();
        for (int e = t; e < q * q; e += TPB) {
            int a = e / q, b = e % q;
            double v = (a < p && b < p) ? 0.5 * (V[a][b] + V[b][a]) : 0.0;
            if (a < p && b < p && (th[a] == 0.0 || th[b] == 0.0)) v = (a == b) ? 1e300 : 0.0;
            S[a][b] = v;
        }
        __syncthreads();
        block_jacobi<double>(S, V, q, sc, ss, sa, sb, red, 1e-30, 30);
        // C = L V into T
        for (int e = t; e < q * q; e += TPB) {
            int a = e / q, b = e % q;
            double v = 0.0;
            for (int j = 0; j < p; ++j) v += L[a][j] * V[j][b];
            T[a][b] = v;
        }
        __syncthreads();
        for (int k = 0; k < p; ++k) r += th[k] > 0.0 ? 1 : 0;
    }
    // sort eigenvalues ascending; apply D to rows of C
    if (t < p) {
        double v = S[t][t];
        int rk = 0;
        for (int j = 0; j < p; ++j) {
            double w = S[j][j];
            if (w < v || (w == v && j < t)) ++rk;
        }
        perm[rk] = t;
    }
    __syncthreads();
    if (t < PMAX) theta[i * PMAX + t] = t < p ? S[perm[t]][perm[t]] : 1e300;
    for (int e = t; e < PMAX * PMAX; e += TPB) {
        int a = e / PMAX, k = e % PMAX;
        double v = 0.0;
        if (a < p && k < p) v = dsc[a] * T[a][perm[k]];
        if (k < p && S[perm[k]][perm[k]] >= 1e299) v = 0.0;
        C[(long long)i * PMAX * PMAX + e] = v;
    }
    if (t == 0) rank[i] = r;
}

// ---- Rayleigh-Ritz, one warp per problem (p <= 32), the same steps as
// k_rayleigh_ritz with __syncwarp in place of block barriers: column scaling
// D = diag(M)^{-1/2}, Cholesky D M D = L L^T, reduced matrix
// G = L^{-1} (D H D) L^{-T}, FP32 Jacobi sweeps on G, FP64 modified
// Gram-Schmidt of the eigenvectors V, exact FP64 V^T G V and FP64 sweeps to
// convergence, C = D L^{-T} V; the pseudo-inverse path when D M D is not
// numerically positive definite.
namespace wrr {

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename T>
__device__ void jacobi(T (*S)[LD], T (*V)[LD], int q, double rel_tol2, int max_sweeps, bool init_v) {
    __shared__ T sc[PMAX / 2], ss[PMAX / 2];
    __shared__ int sa[PMAX / 2], sb[PMAX / 2];
    const int lane = threadIdx.x & 31;
    if (init_v)
        for (int e = lane; e < q * q; e += 32) V[e / q][e % q] = (e / q == e % q) ? T(1) : T(0);
    __syncwarp();
    double fro = 0.0;
    for (int e = lane; e < q * q; e += 32) fro += (double)S[e / q][e % q] * (double)S[e / q][e % q];
    fro = warp_sum(fro);
    const int h = q / 2;
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        double off = 0.0;
        for (int e = lane; e < q * q; e += 32) {
            int a = e / q, b = e % q;
            if (a != b) off += (double)S[a][b] * (double)S[a][b];
        }
        off = warp_sum(off);
        if (off <= rel_tol2 * fro || fro == 0.0) break;
        for (int step = 0; step < q - 1; ++step) {
            // round-robin pairing: position 0 fixed, the others rotate
            if (lane < h) {
                int a = lane == 0 ? 0 : 1 + (lane - 1 + step) % (q - 1);
                int b = 1 + (q - 1 - lane - 1 + step) % (q - 1);
                if (a > b) { int tmp = a; a = b; b = tmp; }
                T c, s;
                rot_params<T>(S[a][a], S[b][b], S[a][b], c, s);
                sa[lane] = a; sb[lane] = b; sc[lane] = c; ss[lane] = s;
            }
            __syncwarp();
            for (int e = lane; e < h * q; e += 32) {    // rows a, b
                int j = e / q, k = e % q;
                T sj = ss[j];
                if (sj == T(0)) continue;
                int a = sa[j], b = sb[j];
                T cj = sc[j];
                T x = S[a][k], y = S[b][k];
                S[a][k] = cj * x - sj * y;
                S[b][k] = sj * x + cj * y;
            }
            __syncwarp();
            for (int e = lane; e < h * q; e += 32) {    // columns a, b of S and V
                int j = e / q, k = e % q;
                T sj = ss[j];
                if (sj == T(0)) continue;
                int a = sa[j], b = sb[j];
                T cj = sc[j];
                T x = S[k][a], y = S[k][b];
                S[k][a] = cj * x - sj * y;
                S[k][b] = sj * x + cj * y;
                T u = V[k][a], v = V[k][b];
                V[k][a] = cj * u - sj * v;
                V[k][b] = sj * u + cj * v;
            }
            __syncwarp();
        }
    }
}

}  // namespace wrr

__global__ void __launch_bounds__(32) k_rr_warp(const double* __restrict__ H, const double* __restrict__ M,
                                                double* __restrict__ C, double* __restrict__ theta,
                                                const int* __restrict__ p_, int* __restrict__ rank,
                                                const int* __restrict__ done) {
    __shared__ double L[PMAX][LD], Tm[PMAX][LD], S[PMAX][LD], V[PMAX][LD], W[PMAX][LD];
    __shared__ double dsc[PMAX], coef[PMAX];
    __shared__ int perm[PMAX];
    // the FP32 Jacobi works in W's storage (two float q x q arrays fit in one double array)
    float (*G32)[LD] = reinterpret_cast<float (*)[LD]>(&W[0][0]);
    float (*V32)[LD] = G32 + PMAX;
    const int i = blockIdx.x;
    if (done[i]) return;
    const int p = p_[i];
    const int q = p + (p & 1);
    const int lane = threadIdx.x;
    const double* Hi = H + (long long)i * PMAX * PMAX;
    const double* Mi = M + (long long)i * PMAX * PMAX;
    {
        double m = lane < p ? Mi[lane * PMAX + lane] : 0.0;
        dsc[lane] = m > 0.0 ? 1.0 / sqrt(m) : 0.0;
    }
    __syncwarp();
    for (int e = lane; e < q * q; e += 32) {
        int a = e / q, b = e % q;
        bool ok = a < p && b < p;
        L[a][b] = ok ? dsc[a] * Mi[a * PMAX + b] * dsc[b] : 0.0;
        Tm[a][b] = ok ? dsc[a] * Hi[a * PMAX + b] * dsc[b] : 0.0;
    }
    __syncwarp();
    // Cholesky of L in place (lower); lane a owns row a.  A column with
    // dsc == 0 is dropped; any other pivot <= 1e-13 sends the problem to
    // the pseudo-inverse path below.
    bool fail = false;
    for (int k = 0; k < p; ++k) {
        const double d = L[k][k];
        double lkk;
        if (dsc[k] == 0.0) lkk = 0.0;
        else if (!(d > 1e-13)) { fail = true; lkk = 0.0; }
        else lkk = sqrt(d);
        __syncwarp();
        if (lane == k) L[k][k] = lkk;
        if (lane > k && lane < p) L[lane][k] = lkk > 0.0 ? L[lane][k] / lkk : 0.0;
        __syncwarp();
        if (lane > k && lane < p)
            for (int b = k + 1; b <= lane; ++b) L[lane][b] -= L[lane][k] * L[b][k];
        __syncwarp();
    }
    int r = 0;
    if (!fail) {
        // S = L^{-1} Tm, then W = L^{-1} S^T = G (lane = column)
        if (lane < p)
            for (int k = 0; k < p; ++k) {
                double v = Tm[k][lane];
                for (int j = 0; j < k; ++j) v -= L[k][j] * S[j][lane];
                S[k][lane] = L[k][k] > 0.0 ? v / L[k][k] : 0.0;
            }
        __syncwarp();
        if (lane < p)
            for (int k = 0; k < p; ++k) {
                double v = S[lane][k];
                for (int j = 0; j < k; ++j) v -= L[k][j] * V[j][lane];
                V[k][lane] = L[k][k] > 0.0 ? v / L[k][k] : 0.0;
            }
        __syncwarp();
        for (int e = lane; e < q * q; e += 32) {
            int a = e / q, b = e % q;
            double v = (a < p && b < p) ? 0.5 * (V[a][b] + V[b][a]) : 0.0;
            if (a < p && b < p && (L[a][a] == 0.0 || L[b][b] == 0.0)) v = (a == b) ? 1e300 : 0.0;
            S[a][b] = v;
        }
        __syncwarp();
        for (int e = lane; e < q * q; e += 32) G32[e / q][e % q] = (float)S[e / q][e % q];
        __syncwarp();
        // FP32 sweeps, then FP64 modified Gram-Schmidt on the eigenvectors
        wrr::jacobi<float>(G32, V32, q, 1e-12, 12, true);
        for (int e = lane; e < q * q; e += 32) V[e / q][e % q] = (double)V32[e / q][e % q];
        __syncwarp();
        for (int k = 0; k < q; ++k) {
            double s2 = 0.0;
            for (int rr = lane; rr < q; rr += 32) s2 += V[rr][k] * V[rr][k];
            s2 = wrr::warp_sum(s2);
            const double inv = s2 > 0.0 ? 1.0 / sqrt(s2) : 0.0;
            if (lane < q) V[lane][k] *= inv;
            __syncwarp();
            if (lane > k && lane < q) {
                double d = 0.0;
                for (int rr = 0; rr < q; ++rr) d += V[rr][k] * V[rr][lane];
                coef[lane] = d;
            }
            __syncwarp();
            if (lane < q)
                for (int j = k + 1; j < q; ++j) V[lane][j] -= coef[j] * V[lane][k];
            __syncwarp();
        }
        // S <- V^T S V exactly in FP64 (W = S V, Tm = V^T W), then FP64 sweeps
        for (int e = lane; e < q * q; e += 32) {
            int a = e / q, b = e % q;
            double v = 0.0;
            for (int j = 0; j < q; ++j) v += S[a][j] * V[j][b];
            W[a][b] = v;
        }
        __syncwarp();
        for (int e = lane; e < q * q; e += 32) {
            int a = e / q, b = e % q;
            double v = 0.0;
            for (int j = 0; j < q; ++j) v += V[j][a] * W[j][b];
            Tm[a][b] = v;
        }
        __syncwarp();
        for (int e = lane; e < q * q; e += 32) {
            int a = e / q, b = e % q;
            S[a][b] = 0.5 * (Tm[a][b] + Tm[b][a]);
        }
        __syncwarp();
        wrr::jacobi<double>(S, W, q, 1e-30, 30, true);
        // Tm = V W (eigenvectors of G); W = L^{-T} Tm (lane = column)
        for (int e = lane; e < q * q; e += 32) {
            int a = e / q, b = e % q;
            double v = 0.0;
            for (int j = 0; j < q; ++j) v += V[a][j] * W[j][b];
            Tm[a][b] = v;
        }
        __syncwarp();
        if (lane < q)
            for (int k = p - 1; k >= 0; --k) {
                double v = Tm[k][lane];
                for (int j = k + 1; j < p; ++j) v -= L[j][k] * W[j][lane];
                W[k][lane] = L[k][k] > 0.0 ? v / L[k][k] : 0.0;
            }
        __syncwarp();
        for (int k = 0; k < p; ++k) r += L[k][k] > 0.0 ? 1 : 0;
    } else {
        // pseudo-inverse square root of D M D from its eigen-decomposition
        for (int e = lane; e < q * q; e += 32) {
            int a = e / q, b = e % q;
            S[a][b] = (a < p && b < p) ? dsc[a] * Mi[a * PMAX + b] * dsc[b] : 0.0;
        }
        __syncwarp();
        wrr::jacobi<double>(S, V, q, 1e-30, 30, true);
        double smax = 0.0;
        for (int k = 0; k < p; ++k) smax = fmax(smax, S[k][k]);
        coef[lane] = (lane < p && S[lane][lane] > 1e-13 * smax) ? 1.0 / sqrt(S[lane][lane]) : 0.0;
        __syncwarp();
        for (int e = lane; e < q * q; e += 32) {          // L = U diag(th)
            int a = e / q, b = e % q;
            L[a][b] = (a < p && b < p) ? V[a][b] * coef[b] : 0.0;
        }
        __syncwarp();
        for (int e = lane; e < q * q; e += 32) {          // S = Tm L
            int a = e / q, b = e % q;
            double v = 0.0;
            for (int j = 0; j < p; ++j) v += Tm[a][j] * L[j][b];
            S[a][b] = v;
        }
        __syncwarp();
        for (int e = lane; e < q * q; e += 32) {          // V = L^T S
            int a = e / q, b = e % q;
            double v = 0.0;
            for (int j = 0; j < p; ++j) v += L[j][a] * S[j][b];
            V[a][b] = v;
        }
        __syncwarp();
        for (int e = lane; e < q * q; e += 32) {
            int a = e / q, b = e % q;
            double v = (a < p && b < p) ? 0.5 * (V[a][b] + V[b][a]) : 0.0;
            if (a < p && b < p && (coef[a] == 0.0 || coef[b] == 0.0)) v = (a == b) ? 1e300 : 0.0;
            S[a][b] = v;
        }
        __syncwarp();
        wrr::jacobi<double>(S, V, q, 1e-30, 30, true);
        for (int e = lane; e < q * q; e += 32) {          // W = L V
            int a = e / q, b = e % q;
            double v = 0.0;
            for (int j = 0; j < p; ++j) v += L[a][j] * V[j][b];
            W[a][b] = v;
        }
        __syncwarp();
        for (int k = 0; k < p; ++k) r += coef[k] > 0.0 ? 1 : 0;
    }
    // ascending order; rows of C scaled by D
    if (lane < p) {
        double v = S[lane][lane];
        int rk = 0;
        for (int j = 0; j < p; ++j) {
            double w = S[j][j];
            if (w < v || (w == v && j < lane)) ++rk;
        }
        perm[rk] = lane;
    }
    __syncwarp();
    theta[i * PMAX + lane] = lane < p ? S[perm[lane]][perm[lane]] : 1e300;
    for (int e = lane; e < PMAX * PMAX; e += 32) {
        int a = e / PMAX, k = e % PMAX;
        double v = 0.0;
        if (a < p && k < p) v = dsc[a] * W[a][perm[k]];
        if (k < p && S[perm[k]][perm[k]] >= 1e299) v = 0.0;
        C[(long long)i * PMAX * PMAX + e] = v;
    }
    if (lane == 0) rank[i] = r;
}

// X = Y C, AX = AY C, BX = BY C on a block of 32 rows; residual partial sums.
// Outputs (row, column < p) are spread over the threads, at most 4 each.
__global__ void __launch_bounds__(TPB) k_update(const double* __restrict__ Y, const double* __restrict__ AY,
                                                const double* __restrict__ BY, double* __restrict__ X,
                                                double* __restrict__ AX, double* __restrict__ BX,
                                                const double* __restrict__ C, const double* __restrict__ theta,
                                                const int* __restrict__ n_, const int* __restrict__ K_,
                                                const long long* __restrict__ roff_, const int* __restrict__ p_,
                                                int ldx, double* __restrict__ partial, int nblk_max,
                                                const int* __restrict__ done) {
    __shared__ double sC[PMAX][LD], sY[ROWBLK][LD], sA[ROWBLK][LD], sB[ROWBLK][LD];
    const int i = blockIdx.y, blk = blockIdx.x;
    if (done[i]) return;
    const int n = n_[i], p = p_[i];
    const long long rows = (long long)K_[i] * NB;
    const int r0 = blk * ROWBLK;
    if (r0 >= rows) return;
    const long long roff = roff_[i];
    const int t = threadIdx.x;
    for (int e = t; e < p * p; e += TPB) sC[e / p][e % p] = C[(long long)i * PMAX * PMAX + (e / p) * PMAX + e % p];
    for (int e = t; e < ROWBLK * p; e += TPB) {
        int rr = e / p, c = e % p;
        int r = r0 + rr;
        bool ok = r < n;
        long long idx = (roff + r) * ldx + c;
        sY[rr][c] = ok ? Y[idx] : 0.0;
        sA[rr][c] = ok ? AY[idx] : 0.0;
        sB[rr][c] = ok ? BY[idx] : 0.0;
    }
    __syncthreads();
    double vnum[4] = {0, 0, 0, 0}, vden[4] = {0, 0, 0, 0};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int e = t + k * TPB;
        if (e >= ROWBLK * p) break;
        int rr = e / p, c = e % p;
        double x = 0.0, ax = 0.0, bx = 0.0;
        for (int j = 0; j < p; ++j) {
            double cj = sC[j][c];
            x += sY[rr][j] * cj;
            ax += sA[rr][j] * cj;
            bx += sB[rr][j] * cj;
        }
        int r = r0 + rr;
        if (r < rows) {
            long long idx = (roff + r) * ldx + c;
            X[idx] = x;
            AX[idx] = ax;
            BX[idx] = bx;
        }
        double rv = ax - theta[i * PMAX + c] * bx;
        vnum[k] = rv * rv;
        vden[k] = bx * bx;
    }
    __syncthreads();   // sY / sA are reused for the residual sums
    for (int e = t; e < ROWBLK * PMAX; e += TPB) { sY[e / PMAX][e % PMAX] = 0.0; sA[e / PMAX][e % PMAX] = 0.0; }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int e = t + k * TPB;
        if (e >= ROWBLK * p) break;
        sY[e / p][e % p] = vnum[k];
        sA[e / p][e % p] = vden[k];
    }
    __syncthreads();
    if (t < PMAX) {
        double a = 0.0, b = 0.0;
        for (int k = 0; k < ROWBLK; ++k) { a += sY[k][t]; b += sA[k][t]; }
        double* dst = partial + ((long long)i * nblk_max + blk) * 2 * PMAX;
        dst[t] = a;
        dst[PMAX + t] = b;
    }
}

__device__ void decide(int i, const double* sres, const double* theta, int p, double sigma, double tol, double eta,
                       int nev_max, int it, int maxit, bool may_stop, int* done, int* m_, int* iters, int* n_active,
                       double* best, int* best_it) {
    int count = 0;
    for (int k = 0; k < p; ++k) count += theta[i * PMAX + k] < eta ? 1 : 0;
    int m = count < nev_max ? count : nev_max;
    bool conv = may_stop;
    double worst = 0.0;
    for (int k = 0; k < m; ++k) {
        conv = conv && sres[k] <= tol;
        worst = fmax(worst, sres[k]);
    }
    if (m < nev_max && m < p) {
        double th = theta[i * PMAX + m];
        bool settled = sres[m] <= tol || sres[m] * (th + sigma) <= 0.1 * (th - eta);
        conv = conv && settled;
        if (!settled) worst = fmax(worst, sres[m]);
    }
    if (worst < 0.5 * best[i]) {
        best[i] = worst;
        best_it[i] = it;
    }
    bool stagnated = may_stop && it - best_it[i] >= 10 && worst <= sqrt(tol);
    m_[i] = m;
    iters[i] = it;
    if (conv) done[i] = 1;
    else if (stagnated) done[i] = 3;
    else if (it >= maxit) done[i] = 2;
    else atomicAdd(n_active, 1);
}

__global__ void k_check(const double* __restrict__ partial, const double* __restrict__ theta, double* __restrict__ res,
                        const int* __restrict__ K_, const int* __restrict__ p_, int nblk_max, double sigma, double tol,
                        double eta, int nev_max, int it, int maxit, int* __restrict__ done, int* __restrict__ m_,
                        int* __restrict__ iters, int* __restrict__ n_active, double* __restrict__ best,
                        int* __restrict__ best_it) {
    const int i = blockIdx.x;
    __shared__ double sres[PMAX];
    if (done[i]) return;
    const int p = p_[i];
    const int nblk = (int)ceil_div((long long)K_[i] * NB, ROWBLK);
    const int t = threadIdx.x;
    if (t < PMAX) {
        double a = 0.0, b = 0.0;
        for (int k = 0; k < nblk; ++k) {
            const double* src = partial + ((long long)i * nblk_max + k) * 2 * PMAX;
            a += src[t];
            b += src[PMAX + t];
        }
        double th = theta[i * PMAX + t];
        double rv = (t < p && b > 0.0) ? sqrt(a) / ((fabs(th) + sigma) * sqrt(b)) : 0.0;
        sres[t] = rv;
        res[i * PMAX + t] = rv;
    }
    __syncthreads();
    if (t == 0)
        decide(i, sres, theta, p, sigma, tol, eta, nev_max, it + 1, maxit, it >= 1, done, m_, iters, n_active, best,
               best_it);
}

__global__ void k_check_knorm(const double* __restrict__ partial, const double* __restrict__ theta,
                              double* __restrict__ res, const int* __restrict__ K_, const int* __restrict__ p_,
                              int nblk_max, double sigma, double tol, double eta, int nev_max, int it, int maxit,
                              int* __restrict__ done, int* __restrict__ m_, int* __restrict__ iters,
                              int* __restrict__ n_active, double* __restrict__ best, int* __restrict__ best_it) {
    const int i = blockIdx.x;
    __shared__ double sres[PMAX];
    if (done[i]) return;
    const int p = p_[i];
    const int nblk = (int)ceil_div((long long)K_[i] * NB, ROWBLK);
    const int t = threadIdx.x;
    if (t < PMAX) {
        double a = 0.0;
        for (int k = 0; k < nblk; ++k) a += partial[((long long)i * nblk_max + k) * PMAX + t];
        double th = theta[i * PMAX + t];
        double rv = t < p ? sqrt(fmax(a, 0.0) * (fabs(th) + sigma)) : 0.0;
        sres[t] = rv;
        res[i * PMAX + t] = rv;
    }
    __syncthreads();
    if (t == 0)
        decide(i, sres, theta, p, sigma, tol, eta, nev_max, it, maxit, true, done, m_, iters, n_active, best, best_it);
}

// ---- FP32 start phase: Euclidean CholQR of the block W (W = Q R, X <- Q).
// G = W^T W with FP32 products, one CTA per problem.
__global__ void __launch_bounds__(TPB) k_gram32(const double* __restrict__ W, double* __restrict__ G,
                                                const int* __restrict__ n_, const long long* __restrict__ roff_,
                                                const int* __restrict__ p_, int ldx) {
    __shared__ float sW[ROWBLK][LD];
    const int i = blockIdx.x;
    const int n = n_[i], p = p_[i];
    const long long roff = roff_[i];
    const int npair = p * (p + 1) / 2;
    int pa[3], pb[3];
    float acc[3] = {0.f, 0.f, 0.f};
    for (int q = 0; q < 3; ++q) {
        int e = threadIdx.x + q * TPB;
        pa[q] = -1;
        if (e < npair) {
            int a = 0, rem = e;
            while (rem >= p - a) { rem -= p - a; ++a; }
            pa[q] = a;
            pb[q] = a + rem;
        }
    }
    for (int r0 = 0; r0 < n; r0 += ROWBLK) {
        __syncthreads();
        for (int e = threadIdx.x; e < ROWBLK * p; e += TPB) {
            int rr = e / p, c = e % p;
            int r = r0 + rr;
            sW[rr][c] = r < n ? (float)W[(roff + r) * ldx + c] : 0.f;
        }
        __syncthreads();
        for (int q = 0; q < 3; ++q) {
            if (pa[q] < 0) continue;
            float s = 0.f;
#pragma unroll 8
            for (int rr = 0; rr < ROWBLK; ++rr) s += sW[rr][pa[q]] * sW[rr][pb[q]];
            acc[q] += s;
        }
    }
    for (int q = 0; q < 3; ++q) {
        if (pa[q] < 0) continue;
        G[(long long)i * PMAX * PMAX + pa[q] * PMAX + pb[q]] = acc[q];
        G[(long long)i * PMAX * PMAX + pb[q] * PMAX + pa[q]] = acc[q];
    }
}

// C = D R^{-1} with D = diag(G)^{-1/2} and D G D = R^T R (FP64 Cholesky, one
// warp per problem).  A column whose pivot falls below 1e-10 of its scaled
// diagonal is dependent on the previous ones: it is reset to its scaled self
// (R row e_k) so that the basis stays finite; the FP64 phase removes it.
__global__ void k_cholqr(const double* __restrict__ G, double* __restrict__ C, const int* __restrict__ p_) {
    __shared__ double R[PMAX][LD], Ri[PMAX][LD], d[PMAX];
    const int i = blockIdx.x;
    const int p = p_[i];
    const int t = threadIdx.x;
    const double* Gi = G + (long long)i * PMAX * PMAX;
    if (t < PMAX) {
        double g = t < p ? Gi[t * PMAX + t] : 0.0;
        d[t] = g > 0.0 ? 1.0 / sqrt(g) : 0.0;
    }
    __syncwarp();
    for (int e = t; e < PMAX * PMAX; e += 32) {
        int a = e / PMAX, b = e % PMAX;
        R[a][b] = (a < p && b < p) ? d[a] * Gi[a * PMAX + b] * d[b] : 0.0;
        Ri[a][b] = 0.0;
    }
    __syncwarp();
    // upper Cholesky in place: R <- U with D G D = U^T U
    for (int k = 0; k < p; ++k) {
        double piv = R[k][k];
        bool ok = piv > 1e-10;
        double u = ok ? sqrt(piv) : 1.0;
        __syncwarp();
        if (t == 0) R[k][k] = u;
        for (int j = k + 1 + t; j < p; j += 32) R[k][j] = ok ? R[k][j] / u : 0.0;
        __syncwarp();
        for (int e = t; e < p * p; e += 32) {
            int a = e / p, b = e % p;
            if (a > k && b >= a) R[a][b] -= R[k][a] * R[k][b];
        }
        __syncwarp();
    }
    // Ri = U^{-1} (upper), column-parallel back substitution
    if (t < p) {
        for (int r = t; r >= 0; --r) {
            double v = (r == t) ? 1.0 : 0.0;
            for (int j = r + 1; j <= t; ++j) v -= R[r][j] * Ri[j][t];
            Ri[r][t] = v / R[r][r];
        }
    }
    __syncwarp();
    for (int e = t; e < PMAX * PMAX; e += 32) {
        int a = e / PMAX, b = e % PMAX;
        C[(long long)i * PMAX * PMAX + e] = (a < p && b < p) ? d[a] * Ri[a][b] : 0.0;
    }
}

// X = W C in FP32 arithmetic, on blocks of 32 rows.
__global__ void __launch_bounds__(TPB) k_update32(const double* __restrict__ W, double* __restrict__ X,
                                                  const double* __restrict__ C, const int* __restrict__ n_,
                                                  const int* __restrict__ K_, const long long* __restrict__ roff_,
                                                  const int* __restrict__ p_, int ldx) {
    __shared__ float sC[PMAX][LD], sW[ROWBLK][LD];
    const int i = blockIdx.y, blk = blockIdx.x;
    const int n = n_[i], p = p_[i];
    const long long rows = (long long)K_[i] * NB;
    const int r0 = blk * ROWBLK;
    if (r0 >= rows) return;
    const long long roff = roff_[i];
    const int t = threadIdx.x;
    for (int e = t; e < p * p; e += TPB) sC[e / p][e % p] = (float)C[(long long)i * PMAX * PMAX + (e / p) * PMAX + e % p];
    for (int e = t; e < ROWBLK * p; e += TPB) {
        int rr = e / p, c = e % p;
        int r = r0 + rr;
        sW[rr][c] = r < n ? (float)W[(roff + r) * ldx + c] : 0.f;
    }
    __syncthreads();
    for (int e = t; e < ROWBLK * p; e += TPB) {
        int rr = e / p, c = e % p;
        if (r0 + rr >= rows) continue;
        float x = 0.f;
        for (int j = 0; j < p; ++j) x += sW[rr][j] * sC[j][c];
        X[(roff + r0 + rr) * ldx + c] = (double)x;
    }
}

__global__ void k_dense_pencil(const double* __restrict__ A, const long long* __restrict__ aoff,
                               const int* __restrict__ n_, const int* __restrict__ nown_,
                               const long long* __restrict__ roff_, const double* __restrict__ X,
                               double* __restrict__ AX, double* __restrict__ BX, int ldx, int ncols,
                               const int* __restrict__ skip) {
    const int i = blockIdx.y;
    if (skip && skip[i]) return;
    const int n = n_[i], nown = nown_[i];
    const int nchunk = (ncols + 7) / 8;
    const long long roff = roff_[i];
    const double* Ai = A + aoff[i];
    for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < (long long)n * nchunk;
         w += (long long)gridDim.x * blockDim.x) {
        int r = (int)(w / nchunk), c0 = (int)(w % nchunk) * 8;
        double so[8], sn[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) { so[c] = 0.0; sn[c] = 0.0; }
        const double* arow = Ai + (long long)r * n;
        for (int j = 0; j < n; ++j) {
            double a = arow[j];
            if (a == 0.0) continue;
            const double* xr = X + (roff + j) * ldx + c0;
            if (j < nown) {
#pragma unroll
                for (int c = 0; c < 8; ++c) if (c0 + c < ncols) so[c] += a * xr[c];
            } else {
#pragma unroll
                for (int c = 0; c < 8; ++c) if (c0 + c < ncols) sn[c] += a * xr[c];
            }
        }
        double* ar = AX + (roff + r) * ldx + c0;
        double* br = BX + (roff + r) * ldx + c0;
#pragma unroll
        for (int c = 0; c < 8; ++c)
            if (c0 + c < ncols) {
                ar[c] = so[c] + sn[c];
                br[c] = r < nown ? so[c] : 0.0;
            }
    }
}

}  // namespace

void GevpBatch::alloc(cudaStream_t s) {
    P = K.P;
    d_p.upload(p, s);
    size_t rows = (size_t)K.total_rows;
    for (DevBuf<double>* b : {&X, &AX, &BX, &Y, &AY, &BY, &W}) { b->alloc(rows * ldx); b->zero(s); }
    H.alloc((size_t)P * PMAX * PMAX);
    M.alloc((size_t)P * PMAX * PMAX);
    C.alloc((size_t)P * PMAX * PMAX);
    theta.alloc((size_t)P * PMAX);
    res.alloc((size_t)P * PMAX);
    nblk_max = (int)ceil_div((long long)K.max_K * NB, ROWBLK);
    partial.alloc((size_t)P * nblk_max * 2 * PMAX);
    done.alloc(P);
    best.alloc(P);
    best_it.alloc(P);
    m.alloc(P);
    rank.alloc(P);
    iters.alloc(P);
    n_active.alloc(1);
}

void eig_init(GevpBatch& g, unsigned long long seed, cudaStream_t s) {
    if (g.P == 0) return;
    dim3 grid(32, g.P);
    k_init<<<grid, 256, 0, s>>>(g.X.p, g.K.d_n.p, g.K.d_K.p, g.K.d_roff.p, g.d_p.p, g.ldx, seed, g.done.p, g.iters.p,
                                g.theta.p, g.best.p, g.best_it.p);
    MSDD_LAUNCH_CHECK();
}

void eig_form_rhs(GevpBatch& g, double sigma, bool first, cudaStream_t s) {
    dim3 grid(32, g.P);
    k_form_rhs<<<grid, 256, 0, s>>>(g.W.p, g.AX.p, g.BX.p, g.theta.p, g.K.d_n.p, g.K.d_K.p, g.K.d_roff.p, g.d_p.p,
                                    g.ldx, sigma, first ? 1 : 0, g.done.p);
    MSDD_LAUNCH_CHECK();
}

void eig_form_y(GevpBatch& g, double sigma, bool first, cudaStream_t s) {
    dim3 grid(32, g.P);
    k_form_y<<<grid, 256, 0, s>>>(g.Y.p, g.X.p, g.W.p, g.theta.p, g.K.d_n.p, g.K.d_K.p, g.K.d_roff.p, g.d_p.p, g.ldx,
                                  sigma, first ? 1 : 0, g.done.p);
    MSDD_LAUNCH_CHECK();
}

void eig_form_y_knorm(GevpBatch& g, double sigma, cudaStream_t s) {
    dim3 grid(g.nblk_max, g.P);
    k_form_y_knorm<<<grid, TPB, 0, s>>>(g.Y.p, g.X.p, g.W.p, g.AX.p, g.BX.p, g.theta.p, g.K.d_n.p, g.K.d_K.p,
                                        g.K.d_roff.p, g.d_p.p, g.ldx, sigma, g.partial.p, g.nblk_max, g.done.p);
    MSDD_LAUNCH_CHECK();
}

void eig_check_knorm(GevpBatch& g, const EigParams& ep, int it, cudaStream_t s) {
    k_check_knorm<<<g.P, 64, 0, s>>>(g.partial.p, g.theta.p, g.res.p, g.K.d_K.p, g.d_p.p, g.nblk_max, ep.sigma,
                                     ep.tol, ep.eta, ep.nev_max, it, ep.maxit, g.done.p, g.m.p, g.iters.p,
                                     g.n_active.p, g.best.p, g.best_it.p);
    MSDD_LAUNCH_CHECK();
}

void eig_cholqr32(GevpBatch& g, cudaStream_t s) {
    k_gram32<<<g.P, TPB, 0, s>>>(g.W.p, g.H.p, g.K.d_n.p, g.K.d_roff.p, g.d_p.p, g.ldx);
    MSDD_LAUNCH_CHECK();
    k_cholqr<<<g.P, 32, 0, s>>>(g.H.p, g.C.p, g.d_p.p);
    MSDD_LAUNCH_CHECK();
    dim3 grid(g.nblk_max, g.P);
    k_update32<<<grid, TPB, 0, s>>>(g.W.p, g.X.p, g.C.p, g.K.d_n.p, g.K.d_K.p, g.K.d_roff.p, g.d_p.p, g.ldx);
    MSDD_LAUNCH_CHECK();
}

void eig_gram(GevpBatch& g, cudaStream_t s) {
    k_gram<<<g.P, TPB, 0, s>>>(g.Y.p, g.AY.p, g.BY.p, g.H.p, g.M.p, g.K.d_n.p, g.K.d_roff.p, g.d_p.p, g.ldx, g.done.p);
    MSDD_LAUNCH_CHECK();
}

void eig_rayleigh_ritz(GevpBatch& g, cudaStream_t s) {
    k_rayleigh_ritz<<<g.P, TPB, 0, s>>>(g.H.p, g.M.p, g.C.p, g.theta.p, g.d_p.p, g.rank.p, g.done.p);
    MSDD_LAUNCH_CHECK();
}

void eig_update(GevpBatch& g, cudaStream_t s) {
    dim3 grid(g.nblk_max, g.P);
    k_update<<<grid, TPB, 0, s>>>(g.Y.p, g.AY.p, g.BY.p, g.X.p, g.AX.p, g.BX.p, g.C.p, g.theta.p, g.K.d_n.p,
                                  g.K.d_K.p, g.K.d_roff.p, g.d_p.p, g.ldx, g.partial.p, g.nblk_max, g.done.p);
    MSDD_LAUNCH_CHECK();
}

void eig_check(GevpBatch& g, const EigParams& ep, int it, cudaStream_t s) {
    k_check<<<g.P, 64, 0, s>>>(g.partial.p, g.theta.p, g.res.p, g.K.d_K.p, g.d_p.p, g.nblk_max, ep.sigma, ep.tol,
                               ep.eta, ep.nev_max, it, ep.maxit, g.done.p, g.m.p, g.iters.p, g.n_active.p, g.best.p,
                               g.best_it.p);
    MSDD_LAUNCH_CHECK();
}

void apply_dense_pencil(const double* Abar, const long long* d_aoff, const int* d_n, const int* d_nown,
                        const TileBatch& layout, const double* X, double* AX, double* BX, int ldx, int ncols,
                        const int* skip, int P, int nmax, cudaStream_t s) {
    if (P == 0) return;
    dim3 grid(std::max(1u, ceil_div((long long)nmax * ((ncols + 7) / 8), 128)), P);
    k_dense_pencil<<<grid, 128, 0, s>>>(Abar, d_aoff, d_n, d_nown, layout.d_roff.p, X, AX, BX, ldx, ncols, skip);
    MSDD_LAUNCH_CHECK();
}

}  // namespace msdd
