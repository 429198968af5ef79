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
__device__ void rot_params(double app, double aqq, double apq, double& c, double& s) {
    if (apq == 0.0 || fabs(apq) <= 1e-18 * sqrt(fabs(app * aqq))) { c = 1.0; s = 0.0; return; }
    double th = (aqq - app) / (2.0 * apq);
    double t;
    if (fabs(th) > 1e150) t = 0.5 / th;
    else t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
    c = 1.0 / sqrt(t * t + 1.0);
    s = t * c;
}

// S (q x q, q even) is overwritten by its eigenvalues on the diagonal; V = eigenvectors.
__device__ void block_jacobi(double (*S)[LD], double (*V)[LD], int q, double* sc, double* ss, int* sa, int* sb,
                             double* red) {
    const int t = threadIdx.x;
    for (int e = t; e < q * q; e += TPB) V[e / q][e % q] = (e / q == e % q) ? 1.0 : 0.0;
    __syncthreads();
    double fro = 0.0;
    {
        double part = 0.0;
        for (int e = t; e < q * q; e += TPB) part += S[e / q][e % q] * S[e / q][e % q];
        red[t] = part;
        __syncthreads();
        for (int w = TPB / 2; w > 0; w >>= 1) {
            if (t < w) red[t] += red[t + w];
            __syncthreads();
        }
        fro = red[0];
        __syncthreads();
    }
    for (int sweep = 0; sweep < 30; ++sweep) {
        double part = 0.0;
        for (int e = t; e < q * q; e += TPB) {
            int a = e / q, b = e % q;
            if (a != b) part += S[a][b] * S[a][b];
        }
        red[t] = part;
        __syncthreads();
        for (int w = TPB / 2; w > 0; w >>= 1) {
            if (t < w) red[t] += red[t + w];
            __syncthreads();
        }
        double off = red[0];
        __syncthreads();
        if (off <= 1e-30 * fro || fro == 0.0) break;
        for (int step = 0; step < q - 1; ++step) {
            if (t < q / 2) {
                // circle method: position 0 fixed, the others rotate
                int pos1 = t, pos2 = q - 1 - t;
                int a = pos1 == 0 ? 0 : 1 + (pos1 - 1 + step) % (q - 1);
                int b = 1 + (pos2 - 1 + step) % (q - 1);
                if (a > b) { int tmp = a; a = b; b = tmp; }
                double c, s;
                rot_params(S[a][a], S[b][b], S[a][b], c, s);
                sa[t] = a; sb[t] = b; sc[t] = c; ss[t] = s;
            }
            __syncthreads();
            for (int e = t; e < (q / 2) * q; e += TPB) {    // rows
                int j = e / q, k = e % q;
                if (ss[j] == 0.0) continue;
                int a = sa[j], b = sb[j];
                double x = S[a][k], y = S[b][k];
                S[a][k] = sc[j] * x - ss[j] * y;
                S[b][k] = ss[j] * x + sc[j] * y;
            }
            __syncthreads();
            for (int e = t; e < (q / 2) * q; e += TPB) {    // columns of S and V
                int j = e / q, k = e % q;
                if (ss[j] == 0.0) continue;
                int a = sa[j], b = sb[j];
                double x = S[k][a], y = S[k][b];
                S[k][a] = sc[j] * x - ss[j] * y;
                S[k][b] = ss[j] * x + sc[j] * y;
                double u = V[k][a], v = V[k][b];
                V[k][a] = sc[j] * u - ss[j] * v;
                V[k][b] = ss[j] * u + sc[j] * v;
            }
            __syncthreads();
        }
    }
}

// Rayleigh-Ritz on (H, M): column scaling D = diag(M)^{-1/2}, Cholesky of
// D M D (Jacobi-based pseudo-inverse square root if it is not numerically
// positive definite), Jacobi on the reduced standard problem.
__global__ void __launch_bounds__(TPB) k_rayleigh_ritz(const double* __restrict__ H, const double* __restrict__ M,
                                                       double* __restrict__ C, double* __restrict__ theta,
                                                       const int* __restrict__ p_, int* __restrict__ rank,
                                                       const int* __restrict__ done) {
    __shared__ double S[PMAX][LD], V[PMAX][LD], L[PMAX][LD], T[PMAX][LD];
    __shared__ double dsc[PMAX], sc[PMAX / 2], ss[PMAX / 2], red[TPB], th[PMAX];
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
        block_jacobi(S, V, q, sc, ss, sa, sb, red);
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
        block_jacobi(S, V, q, sc, ss, sa, sb, red);   // S diag = s, V = U
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
        block_jacobi(S, V, q, sc, ss, sa, sb, red);
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
