// Batched subspace iteration with Rayleigh-Ritz (see eig.cuh).
#include "eig.cuh"

#include <type_traits>

#include <cmath>

namespace msdd {

namespace {

constexpr int TPB = 256;
constexpr int LD = PMAX + 1;
constexpr int ROWBLK = EIG_ROWBLK;

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
    __shared__ double smu[PMAX];                       // 1 / (theta + sigma): one division per column
    const int i = blockIdx.y;
    if (done[i]) return;
    const int n = n_[i], p = p_[i];
    const long long rows = (long long)K_[i] * NB;
    if (threadIdx.x < p) smu[threadIdx.x] = first ? 0.0 : 1.0 / (theta[i * PMAX + threadIdx.x] + sigma);
    __syncthreads();
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < rows * ldx;
         e += (long long)gridDim.x * blockDim.x) {
        int r = (int)(e / ldx), c = (int)(e % ldx);
        long long idx = (roff_[i] + r) * ldx + c;
        double v = 0.0;
        if (r < n && c < p) {
            double bx = BX[idx];
            v = first ? bx : bx - (AX[idx] + sigma * bx) * smu[c];
        }
        W[idx] = v;
    }
}

__global__ void k_form_y(double* __restrict__ Y, const double* __restrict__ X, const double* __restrict__ W,
                         const double* __restrict__ theta, const int* __restrict__ n_, const int* __restrict__ K_,
                         const long long* __restrict__ roff_, const int* __restrict__ p_, int ldx, double sigma,
                         int first, const int* __restrict__ done) {
    __shared__ double smu[PMAX];                       // 1 / (theta + sigma): one division per column
    const int i = blockIdx.y;
    if (done[i]) return;
    const int n = n_[i], p = p_[i];
    const long long rows = (long long)K_[i] * NB;
    if (threadIdx.x < p) smu[threadIdx.x] = first ? 0.0 : 1.0 / (theta[i * PMAX + threadIdx.x] + sigma);
    __syncthreads();
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < rows * ldx;
         e += (long long)gridDim.x * blockDim.x) {
        int r = (int)(e / ldx), c = (int)(e % ldx);
        long long idx = (roff_[i] + r) * ldx + c;
        double v = 0.0;
        if (r < n && c < p) v = first ? W[idx] : fma(X[idx], smu[c], W[idx]);
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
    __shared__ double red[ROWBLK][LD], smu[PMAX];
    const int i = blockIdx.y, blk = blockIdx.x;
    if (done[i]) return;
    const int n = n_[i], p = p_[i];
    const long long rows = (long long)K_[i] * NB;
    const int r0 = blk * ROWBLK;
    if (r0 >= rows) return;
    if (threadIdx.x < p) smu[threadIdx.x] = 1.0 / (theta[i * PMAX + threadIdx.x] + sigma);
    __syncthreads();
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
                const double mu = smu[c];
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

// H = Y^T AY, M = Y^T BY as partial sums over `gsplit` row ranges of each
// problem (grid: problems x splits); each thread owns 2 x 2 blocks (bi <= bj)
// of the upper block triangle, read as pairs from shared row chunks.
// DF = false: FP64 arithmetic.  DF = true: the rows are split into FP32
// (hi, lo) pairs as they are staged and the products are accumulated in
// double-float (split_f64, df_fma), off the narrow FP64 pipe; the partials
// are stored as FP64.
constexpr int GR_T = 64, GR_ROWS = 32, GR_LD = 34;
template <bool DF>
__global__ void __launch_bounds__(GR_T) k_gram_split(const double* __restrict__ Y, const double* __restrict__ AY,
                                                     const double* __restrict__ BY, double* __restrict__ Hp,
                                                     double* __restrict__ Mp, const int* __restrict__ n_,
                                                     const long long* __restrict__ roff_, const int* __restrict__ p_,
                                                     int ldx, const int* __restrict__ done, int gsplit) {
    using V = std::conditional_t<DF, float, double>;
    constexpr int NA = DF ? 2 : 1;                       // FP64: value; DF: hi, lo
    __shared__ __align__(16) V sY[NA][GR_ROWS][GR_LD], sA[NA][GR_ROWS][GR_LD], sB[NA][GR_ROWS][GR_LD];
    const int i = blockIdx.x, sp = blockIdx.y, t = threadIdx.x;
    if (done[i]) return;
    const int n = n_[i], p = p_[i], q = p + (p & 1), nb = q / 2;
    const long long roff = roff_[i];
    const int rows_per = (n + gsplit - 1) / gsplit;
    const int r_lo = sp * rows_per, r_hi = min(n, r_lo + rows_per);
    const int nblk = nb * (nb + 1) / 2;
    constexpr int KMAX = (PMAX / 2 * (PMAX / 2 + 1) / 2 + GR_T - 1) / GR_T;
    int ba[KMAX], bb[KMAX];
    V h[KMAX][NA][4], m[KMAX][NA][4];
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
        const int e = t + k * GR_T;
        ba[k] = -1;
        bb[k] = 0;
        if (e < nblk) {
            int a = 0, rem = e;
            while (rem >= nb - a) { rem -= nb - a; ++a; }
            ba[k] = a;
            bb[k] = a + rem;
        }
#pragma unroll
        for (int z = 0; z < NA; ++z)
#pragma unroll
            for (int c = 0; c < 4; ++c) { h[k][z][c] = V(0); m[k][z][c] = V(0); }
    }
    for (int r0 = r_lo; r0 < r_hi; r0 += GR_ROWS) {
        __syncthreads();
        for (int e = t; e < GR_ROWS * q; e += GR_T) {
            const int rr = e / q, c = e % q, r = r0 + rr;
            const bool ok = r < r_hi && c < p;
            const long long idx = (roff + r) * ldx + c;
            const double y = ok ? Y[idx] : 0.0, av = ok ? AY[idx] : 0.0, bv = ok ? BY[idx] : 0.0;
            if constexpr (DF) {
                split_f64(y, sY[0][rr][c], sY[1][rr][c]);
                split_f64(av, sA[0][rr][c], sA[1][rr][c]);
                split_f64(bv, sB[0][rr][c], sB[1][rr][c]);
            } else {
                sY[0][rr][c] = y;
                sA[0][rr][c] = av;
                sB[0][rr][c] = bv;
            }
        }
        __syncthreads();
        const int nr = min(GR_ROWS, r_hi - r0);
#pragma unroll
        for (int k = 0; k < KMAX; ++k) {
            if (ba[k] < 0) continue;
            const int a0 = 2 * ba[k], b0 = 2 * bb[k];
            for (int rr = 0; rr < nr; ++rr) {
                if constexpr (DF) {
                    const float2 yh = *reinterpret_cast<const float2*>(&sY[0][rr][a0]);
                    const float2 yl = *reinterpret_cast<const float2*>(&sY[1][rr][a0]);
                    const float2 ah = *reinterpret_cast<const float2*>(&sA[0][rr][b0]);
                    const float2 al = *reinterpret_cast<const float2*>(&sA[1][rr][b0]);
                    const float2 bh = *reinterpret_cast<const float2*>(&sB[0][rr][b0]);
                    const float2 bl = *reinterpret_cast<const float2*>(&sB[1][rr][b0]);
                    df_fma(h[k][0][0], h[k][1][0], yh.x, yl.x, ah.x, al.x);
                    df_fma(h[k][0][1], h[k][1][1], yh.x, yl.x, ah.y, al.y);
                    df_fma(h[k][0][2], h[k][1][2], yh.y, yl.y, ah.x, al.x);
                    df_fma(h[k][0][3], h[k][1][3], yh.y, yl.y, ah.y, al.y);
                    df_fma(m[k][0][0], m[k][1][0], yh.x, yl.x, bh.x, bl.x);
                    df_fma(m[k][0][1], m[k][1][1], yh.x, yl.x, bh.y, bl.y);
                    df_fma(m[k][0][2], m[k][1][2], yh.y, yl.y, bh.x, bl.x);
                    df_fma(m[k][0][3], m[k][1][3], yh.y, yl.y, bh.y, bl.y);
                } else {
                    const double2 y = *reinterpret_cast<const double2*>(&sY[0][rr][a0]);
                    const double2 av = *reinterpret_cast<const double2*>(&sA[0][rr][b0]);
                    const double2 bv = *reinterpret_cast<const double2*>(&sB[0][rr][b0]);
                    h[k][0][0] += y.x * av.x; h[k][0][1] += y.x * av.y; h[k][0][2] += y.y * av.x; h[k][0][3] += y.y * av.y;
                    m[k][0][0] += y.x * bv.x; m[k][0][1] += y.x * bv.y; m[k][0][2] += y.y * bv.x; m[k][0][3] += y.y * bv.y;
                }
            }
        }
    }
    double* Hs = Hp + ((long long)i * gsplit + sp) * PMAX * PMAX;
    double* Ms = Mp + ((long long)i * gsplit + sp) * PMAX * PMAX;
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
        if (ba[k] < 0) continue;
        const int a0 = 2 * ba[k], b0 = 2 * bb[k];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int a = a0 + (c >> 1), b = b0 + (c & 1);
            if (a >= p || b >= p) continue;
            double hv, mv;
            if constexpr (DF) {
                hv = df_to_f64(h[k][0][c], h[k][1][c]);
                mv = df_to_f64(m[k][0][c], m[k][1][c]);
            } else {
                hv = h[k][0][c];
                mv = m[k][0][c];
            }
            Hs[a * PMAX + b] = hv;
            Ms[a * PMAX + b] = mv;
            if (a0 != b0) {                                 // mirror off-diagonal blocks
                Hs[b * PMAX + a] = hv;
                Ms[b * PMAX + a] = mv;
            }
        }
    }
}

// ---- block-wide symmetric eigen-solver (parallel cyclic Jacobi, round robin)
// FP64 divisions and square roots are long instruction sequences on the
// FP64 pipe; the kernels below take their reciprocal square roots from an
// FP32 seed refined by two Newton steps r <- r (3 - x r^2) / 2 (relative
// error ~1e-7 -> ~1e-14 -> rounding level).
__device__ __forceinline__ double rsqrt_nr(double x) {
    if (!(x > 1e-30 && x < 1e30)) return x > 0.0 ? 1.0 / sqrt(x) : 0.0;
    double r = f32_to_f64(rsqrtf(f64_to_f32(x)));
    r = r * (1.5 - 0.5 * x * r * r);
    r = r * (1.5 - 0.5 * x * r * r);
    return r;
}

// A pair (a, b) is rotated only while |S_ab| > rel_tol sqrt(|S_aa S_bb|)
// and |S_ab| > floor_abs (floor_abs is tied to the scale of S, so that
// pairs with a zero diagonal entry terminate).  The test is evaluated in
// FP32 for both precisions (a threshold test needs no more).
__device__ __forceinline__ bool pair_active_f(float app, float aqq, float apq, float rel_tol, float floor_abs) {
    const float a = fabsf(apq);
    return a > floor_abs && a > rel_tol * sqrtf(fabsf(app)) * sqrtf(fabsf(aqq));
}
template <typename T>
__device__ __forceinline__ bool pair_active(T app, T aqq, T apq, T rel_tol, T floor_abs);
template <>
__device__ __forceinline__ bool pair_active<float>(float app, float aqq, float apq, float rel_tol, float floor_abs) {
    return pair_active_f(app, aqq, apq, rel_tol, floor_abs);
}
template <>
__device__ __forceinline__ bool pair_active<double>(double app, double aqq, double apq, double rel_tol,
                                                    double floor_abs) {
    return pair_active_f(f64_to_f32(app), f64_to_f32(aqq), f64_to_f32(apq), f64_to_f32(rel_tol),
                         fmaxf(f64_to_f32(floor_abs), 1e-37f));
}

// FP32: the Jacobi angle with fast reciprocal / reciprocal square root (the
// pair is then zeroed explicitly; the FP32 sweeps only seed the FP64 ones).
__device__ __forceinline__ void rot_params(float app, float aqq, float apq, float& c, float& s) {
    const float th = __fdividef(aqq - app, 2.0f * apq);
    float t;
    if (!(fabsf(th) <= 1e15f)) {
        t = __fdividef(0.5f, th);
    } else {
        const float r2 = fmaf(th, th, 1.0f);
        t = copysignf(__fdividef(1.0f, fabsf(th) + r2 * rsqrtf(r2)), th);
    }
    c = rsqrtf(fmaf(t, t, 1.0f));
    s = t * c;
}
// FP64: the angle from FP32 arithmetic; c and s are then rescaled by
// (c^2 + s^2)^{-1/2} ~ 1 - d/2 + 3 d^2 / 8, d = c^2 + s^2 - 1 evaluated
// without rounding error by FP32 error-free products (c^2 - 1 and the sum
// with s^2 are exact by Sterbenz' lemma since c^2 >= 1/2), and stored as
// FP64 sums c + c (-d/2 + 3 d^2/8).  The rotation is orthogonal to FP64
// accuracy and reduces the pair by ~1e-7 instead of annihilating it (the
// pair is not zeroed; later sweeps finish it).
__device__ __forceinline__ void rot_params(double app, double aqq, double apq, double& c, double& s) {
    const float num = f64_to_f32(aqq - app), den = 2.0f * f64_to_f32(apq);
    if (!(den != 0.0f && isfinite(num) && isfinite(den))) {
        const double th = (aqq - app) / (2.0 * apq);
        const double t = (fabs(th) > 1e15) ? 0.5 / th : (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
        c = 1.0 / sqrt(1.0 + t * t);
        s = t * c;
        return;
    }
    float cf, sf;
    rot_params(0.0f, num, 0.5f * den, cf, sf);            // th = num / den
    const float c2h = cf * cf, c2l = fmaf(cf, cf, -c2h);
    const float s2h = sf * sf, s2l = fmaf(sf, sf, -s2h);
    const float d = ((c2h - 1.0f) + s2h) + (c2l + s2l);
    const float corr = d * fmaf(0.375f, d, -0.5f);
    c = f32_to_f64(cf) + f32_to_f64(cf * corr);
    s = f32_to_f64(sf) + f32_to_f64(sf * corr);
}

// S (q x q, q even) is overwritten by its eigenvalues on the diagonal; V =
// eigenvectors.  Stops after a check finds no active pair, or after
// max_sweeps sweeps.  Diagonal entries >= 1e299 mark dropped columns (their
// off-diagonal entries are zero) and are left out of the scale.
//
// One step of the round-robin ordering rotates q/2 disjoint pairs; the
// two-sided update J^T S J is done in one pass over the 2 x 2 blocks
// (pair j rows, pair jj columns), which the disjoint pairs cover exactly
// once, together with the column update of V.  The pair parameters are
// double-buffered, so a step in which no pair rotates costs one barrier.
template <typename T>
__device__ void block_jacobi(T (*S)[LD], T (*V)[LD], int q, T rel_tol, T floor_rel, int max_sweeps) {
    __shared__ T sc[2][PMAX / 2], ss[2][PMAX / 2];
    __shared__ int sa[2][PMAX / 2], sb[2][PMAX / 2], sr[2][PMAX / 2];
    __shared__ double s_scale;
    const int t = threadIdx.x, h = q / 2;
    for (int e = t; e < q * q; e += TPB) V[e / q][e % q] = (e / q == e % q) ? T(1) : T(0);
    if (t < 32) {
        double m = 0.0;
        for (int k = t; k < q; k += 32) {
            double v = fabs((double)S[k][k]);
            if (v < 1e299) m = fmax(m, v);
        }
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (t == 0) s_scale = m;
    }
    __syncthreads();
    const T floor_abs = fmax((T)(floor_rel * s_scale), sizeof(T) == 4 ? T(1e-30) : T(1e-290));
    int par = 0;
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        int active = 0;
        for (int e = t; e < q * q; e += TPB) {
            int a = e / q, b = e % q;
            if (a < b && pair_active<T>(S[a][a], S[b][b], S[a][b], rel_tol, floor_abs)) active = 1;
        }
        if (!__syncthreads_or(active)) break;
        for (int step = 0; step < q - 1; ++step, par ^= 1) {
            int rot = 0;
            if (t < h) {
                // circle method: position 0 fixed, the others rotate
                int pos1 = t, pos2 = q - 1 - t;
                int a = pos1 == 0 ? 0 : 1 + (pos1 - 1 + step) % (q - 1);
                int b = 1 + (pos2 - 1 + step) % (q - 1);
                if (a > b) { int tmp = a; a = b; b = tmp; }
                T c = T(1), s = T(0);
                rot = pair_active<T>(S[a][a], S[b][b], S[a][b], rel_tol, floor_abs) ? 1 : 0;
                if (rot) rot_params(S[a][a], S[b][b], S[a][b], c, s);
                sa[par][t] = a; sb[par][t] = b; sc[par][t] = c; ss[par][t] = s; sr[par][t] = rot;
            }
            // (integer flags: FP64 comparisons would occupy the narrow FP64 pipe)
            if (!__syncthreads_or(rot)) continue;
            const int nblk = h * h;
            for (int e = t; e < nblk + q * h; e += TPB) {
                if (e < nblk) {
                    const int j = e / h, jj = e % h;
                    if (!(sr[par][j] | sr[par][jj])) continue;
                    const T sj = ss[par][j], sjj = ss[par][jj];
                    const T cj = sc[par][j], cjj = sc[par][jj];
                    const int x1 = sa[par][j], x2 = sb[par][j], y1 = sa[par][jj], y2 = sb[par][jj];
                    const T b11 = S[x1][y1], b12 = S[x1][y2], b21 = S[x2][y1], b22 = S[x2][y2];
                    const T r11 = cj * b11 - sj * b21, r12 = cj * b12 - sj * b22;      // rows x1, x2
                    const T r21 = sj * b11 + cj * b21, r22 = sj * b12 + cj * b22;
                    T n11 = cjj * r11 - sjj * r12, n12 = sjj * r11 + cjj * r12;          // columns y1, y2
                    T n21 = cjj * r21 - sjj * r22, n22 = sjj * r21 + cjj * r22;
                    if (sizeof(T) == 4 && j == jj) { n12 = T(0); n21 = T(0); }        // exact angle: annihilated
                    S[x1][y1] = n11; S[x1][y2] = n12; S[x2][y1] = n21; S[x2][y2] = n22;
                } else {
                    const int e2 = e - nblk, k = e2 / h, jj = e2 % h;
                    if (!sr[par][jj]) continue;
                    const T sjj = ss[par][jj];
                    const T cjj = sc[par][jj];
                    const int y1 = sa[par][jj], y2 = sb[par][jj];
                    const T u = V[k][y1], v = V[k][y2];
                    V[k][y1] = cjj * u - sjj * v;
                    V[k][y2] = sjj * u + cjj * v;
                }
            }
            __syncthreads();
        }
    }
}

// D = E F for q x q blocks in shared memory (E transposed when tE); four
// partial sums per entry keep the dependent FP64 chains short.
__device__ __forceinline__ void smem_gemm(double (*D)[LD], const double (*E)[LD], const double (*F)[LD], int q,
                                          bool tE) {
    for (int e = threadIdx.x; e < q * q; e += TPB) {
        const int a = e / q, b = e % q;
        double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0;
        int j = 0;
        if (tE) {
            for (; j + 3 < q; j += 4) {
                v0 += E[j][a] * F[j][b];
                v1 += E[j + 1][a] * F[j + 1][b];
                v2 += E[j + 2][a] * F[j + 2][b];
                v3 += E[j + 3][a] * F[j + 3][b];
            }
            for (; j < q; ++j) v0 += E[j][a] * F[j][b];
        } else {
            for (; j + 3 < q; j += 4) {
                v0 += E[a][j] * F[j][b];
                v1 += E[a][j + 1] * F[j + 1][b];
                v2 += E[a][j + 2] * F[j + 2][b];
                v3 += E[a][j + 3] * F[j + 3][b];
            }
            for (; j < q; ++j) v0 += E[a][j] * F[j][b];
        }
        D[a][b] = (v0 + v1) + (v2 + v3);
    }
}

// Eigen-decomposition of the symmetric q x q FP64 matrix S (overwritten by
// its eigenvalues on the diagonal, eigenvectors in V).  Most rotations are
// done in FP32 on a copy; the FP32 eigenvectors are re-orthonormalised in
// FP64 by two Newton-Schulz steps V <- V (3 I - V^T V) / 2 (orthogonality
// error 1e-7 -> 1e-14 -> rounding level), S is transformed exactly in FP64
// and FP64 sweeps finish it (normally one).  W and U are FP64 scratch; U
// also holds the FP32 copies.
__device__ void mixed_jacobi(double (*S)[LD], double (*V)[LD], double (*W)[LD], double (*U)[LD], int q) {
    const int t = threadIdx.x;
    float (*G32)[LD] = reinterpret_cast<float (*)[LD]>(&U[0][0]);
    float (*V32)[LD] = G32 + PMAX;
    for (int e = t; e < q * q; e += TPB) G32[e / q][e % q] = f64_to_f32(S[e / q][e % q]);
    __syncthreads();
    block_jacobi<float>(G32, V32, q, 1e-6f, 1e-9f, 12);
    for (int e = t; e < q * q; e += TPB) V[e / q][e % q] = f32_to_f64(V32[e / q][e % q]);
    __syncthreads();
    for (int it = 0; it < 2; ++it) {
        smem_gemm(W, V, V, q, true);                 // W = V^T V
        __syncthreads();
        for (int e = t; e < q * q; e += TPB) W[e / q][e % q] = ((e / q == e % q) ? 1.5 : 0.0) - 0.5 * W[e / q][e % q];
        __syncthreads();
        smem_gemm(U, V, W, q, false);                // U = V (3 I - V^T V) / 2
        __syncthreads();
        for (int e = t; e < q * q; e += TPB) V[e / q][e % q] = U[e / q][e % q];
        __syncthreads();
    }
    // S <- V^T S V in FP64 (W = S V, U = V^T W)
    smem_gemm(W, S, V, q, false);
    __syncthreads();
    smem_gemm(U, V, W, q, true);
    __syncthreads();
    for (int e = t; e < q * q; e += TPB) {
        int a = e / q, b = e % q;
        S[a][b] = 0.5 * (U[a][b] + U[b][a]);
    }
    __syncthreads();
    block_jacobi<double>(S, W, q, 1e-10, 1e-15, 8);
    smem_gemm(U, V, W, q, false);                    // V <- V W
    __syncthreads();
    for (int e = t; e < q * q; e += TPB) V[e / q][e % q] = U[e / q][e % q];
    __syncthreads();
}


// D = op(E) op(F) for q x q FP32 blocks in shared memory (q even).
__device__ __forceinline__ void smem_gemm_f(float (*D)[LD], const float (*E)[LD], const float (*F)[LD], int q,
                                            bool tE, bool tF) {
    for (int e = threadIdx.x; e < q * q; e += TPB) {
        const int a = e / q, b = e % q;
        float v0 = 0.f, v1 = 0.f;
        for (int j = 0; j < q; j += 2) {
            const float e0 = tE ? E[j][a] : E[a][j], e1 = tE ? E[j + 1][a] : E[a][j + 1];
            const float f0 = tF ? F[b][j] : F[j][b], f1 = tF ? F[b][j + 1] : F[j + 1][b];
            v0 = fmaf(e0, f0, v0);
            v1 = fmaf(e1, f1, v1);
        }
        D[a][b] = v0 + v1;
    }
}

// Rayleigh-Ritz for a well-conditioned scaled pencil (Hs, Ms), FP32 first:
//   1. FP32 Cholesky Ms = L L^T and U = L^{-1} (warp 0), G = U Hs U^T and its
//      FP32 Jacobi eigenvectors V; Z = U^T V (so Z^T Ms Z ~ I, Z^T Hs Z ~
//      diagonal to FP32 accuracy);
//   2. FP64: Z <- Z P with P = I - E/2 + 3 E^2/8, E = Z^T Ms Z - I (the
//      second-order inverse square root of I + E: the error drops from |E|
//      to O(|E|^3)), repeated while |E| > 2e-6 (at most 3 times);
//   3. FP64 Jacobi on A = Z^T Hs Z (nearly diagonal), Z <- Z Q.
// Every serial chain runs in FP32 and the FP64 work is seven or so q x q
// products plus the finishing Jacobi steps.  Returns false (nothing of L and
// T changed but a unit dummy pivot) when an FP32 pivot is below 1e-3 or
// |E| > 0.05: the caller then takes the FP64 Cholesky path.  On success S
// holds theta on its diagonal and T the coefficients C' (rows scaled by D
// later).  L = Ms, T = Hs on entry (zero padded to q); S, V, U scratch.
__device__ bool rr_fast(double (*S)[LD], double (*V)[LD], double (*L)[LD], double (*T)[LD], double (*U)[LD], int p,
                        int q) {
    __shared__ float linv32[PMAX];
    __shared__ int s_fail32, s_emax;
    const int t = threadIdx.x;
    float (*L32)[LD] = reinterpret_cast<float (*)[LD]>(&U[0][0]);
    float (*U32)[LD] = L32 + PMAX;
    float (*T32)[LD] = reinterpret_cast<float (*)[LD]>(&S[0][0]);
    float (*G32)[LD] = T32 + PMAX;
    float (*V32)[LD] = reinterpret_cast<float (*)[LD]>(&V[0][0]);
    float (*W32)[LD] = V32 + PMAX;
    if (t == 0 && q > p) L[p][p] = 1.0;                 // odd p: a unit dummy pivot
    __syncthreads();
    for (int e = t; e < q * q; e += TPB) {
        const int a = e / q, b = e % q;
        L32[a][b] = f64_to_f32(L[a][b]);
        T32[a][b] = f64_to_f32(T[a][b]);
    }
    __syncthreads();
    if (t < 32) {
        const int lane = t;
        int fail = 0;
        for (int k = 0; k < q; ++k) {
            const float d = L32[k][k];
            float r = 0.f, lkk = 0.f;
            if (d > 1e-3f) {
                r = rsqrtf(d);
                r = r * fmaf(-0.5f * d * r, r, 1.5f);
                lkk = d * r;
            } else {
                fail = 1;
            }
            __syncwarp();
            if (lane == k) { L32[k][k] = lkk; linv32[k] = r; }
            if (lane > k && lane < q) L32[lane][k] *= r;
            __syncwarp();
            if (lane > k && lane < q)
                for (int b = k + 1; b <= lane; ++b) L32[lane][b] = fmaf(-L32[lane][k], L32[b][k], L32[lane][b]);
            __syncwarp();
        }
        if (lane < q) {
            const int c = lane;
            for (int r = 0; r < q; ++r) {
                float v = 0.f;
                if (r >= c) {
                    float a0 = (r == c) ? 1.f : 0.f, a1 = 0.f;
                    int j = c;
                    for (; j + 1 < r; j += 2) {
                        a0 = fmaf(-L32[r][j], U32[j][c], a0);
                        a1 = fmaf(-L32[r][j + 1], U32[j + 1][c], a1);
                    }
                    if (j < r) a0 = fmaf(-L32[r][j], U32[j][c], a0);
                    v = (a0 + a1) * linv32[r];
                }
                U32[r][c] = v;
            }
        }
        if (lane == 0) { s_fail32 = fail; s_emax = 0; }
    }
    __syncthreads();
    if (s_fail32) return false;
    smem_gemm_f(W32, U32, T32, q, false, false);        // W = U Hs
    __syncthreads();
    smem_gemm_f(G32, W32, U32, q, false, true);         // G = W U^T
    __syncthreads();
    for (int e = t; e < q * q; e += TPB) {
        const int a = e / q, b = e % q;
        if (a < b) {
            const float v = 0.5f * (G32[a][b] + G32[b][a]);
            G32[a][b] = v;
            G32[b][a] = v;
        }
    }
    __syncthreads();
    block_jacobi<float>(G32, V32, q, 1e-6f, 1e-9f, 12);
    __syncthreads();
    smem_gemm_f(L32, U32, V32, q, true, false);         // Z = U^T V (FP32), into the L32 slot
    __syncthreads();
    for (int e = t; e < q * q; e += TPB) S[e / q][e % q] = f32_to_f64(L32[e / q][e % q]);
    __syncthreads();
    // FP64 Ms-orthonormalisation of Z
    bool ok = false;
    for (int round = 0; round < 3; ++round) {
        smem_gemm(V, L, S, q, false);                    // W = Ms Z
        __syncthreads();
        smem_gemm(U, S, V, q, true);                     // Z^T W
        __syncthreads();
        float em = 0.f;
        for (int e = t; e < q * q; e += TPB) {
            const int a = e / q, b = e % q;
            double v = U[a][b];
            if (a == b) {
                v -= 1.0;
                U[a][b] = v;
            }
            const float av = fabsf(f64_to_f32(v));
            em = av != av ? 1e30f : fmaxf(em, av);        // NaN sends the problem to the FP64 path
        }
        for (int o = 16; o > 0; o >>= 1) em = fmaxf(em, __shfl_xor_sync(0xffffffffu, em, o));
        if ((t & 31) == 0) atomicMax(&s_emax, __float_as_int(em));     // non-negative: int order = float order
        __syncthreads();
        const float emax = __int_as_float(s_emax);
        if (!(emax <= 0.05f)) return false;
        if (emax == 0.f) { ok = true; break; }
        smem_gemm(V, U, U, q, false);                    // E^2
        __syncthreads();
        for (int e = t; e < q * q; e += TPB) {
            const int a = e / q, b = e % q;
            V[a][b] = fma(0.375, V[a][b], fma(-0.5, U[a][b], a == b ? 1.0 : 0.0));
        }
        __syncthreads();
        smem_gemm(U, S, V, q, false);                    // Z P
        __syncthreads();
        for (int e = t; e < q * q; e += TPB) S[e / q][e % q] = U[e / q][e % q];
        if (t == 0) s_emax = 0;
        __syncthreads();
        if (emax <= 2e-6f) { ok = true; break; }
    }
    if (!ok) return false;
    // A = Z^T Hs Z, then the FP64 Jacobi finish
    smem_gemm(V, T, S, q, false);                        // W = Hs Z
    __syncthreads();
    smem_gemm(U, S, V, q, true);                         // A = Z^T W
    __syncthreads();
    for (int e = t; e < q * q; e += TPB) {
        const int a = e / q, b = e % q;
        if (a < b) {
            const double v = 0.5 * (U[a][b] + U[b][a]);
            U[a][b] = v;
            U[b][a] = v;
        }
    }
    __syncthreads();
    block_jacobi<double>(U, V, q, 1e-10, 1e-15, 8);
    __syncthreads();
    smem_gemm(T, S, V, q, false);                        // C' = Z Q
    __syncthreads();
    for (int e = t; e < q * q; e += TPB) S[e / q][e % q] = U[e / q][e % q];
    __syncthreads();
    return true;
}

// Rayleigh-Ritz on (H, M): column scaling D = diag(M)^{-1/2}, Cholesky of
// D M D (Jacobi-based pseudo-inverse square root if it is not numerically
// positive definite), eigen-decomposition of the reduced standard problem.
// C = D L^{-T} V with theta ascending; columns of dropped (dependent)
// directions get theta = +inf and zero columns of C.
// H and M are first summed from the split partials of k_gram_split (in
// split order) and stored; the kernel then reads them back.
__global__ void __launch_bounds__(TPB) k_rayleigh_ritz(const double* __restrict__ Hp, const double* __restrict__ Mp,
                                                       int gsplit, double* __restrict__ H, double* __restrict__ M,
                                                       double* __restrict__ C, double* __restrict__ theta,
                                                       const int* __restrict__ p_, int* __restrict__ rank,
                                                       const int* __restrict__ done) {
    __shared__ double S[PMAX][LD], V[PMAX][LD], L[PMAX][LD], T[PMAX][LD], U[PMAX][LD];
    __shared__ double dsc[PMAX], th[PMAX], linv[PMAX];
    __shared__ int perm[PMAX];
    __shared__ int s_fail, s_zero;
    const int i = blockIdx.x;
    if (done[i]) return;
    const int p = p_[i];
    const int q = p + (p & 1);
    const int t = threadIdx.x;
    double* Hw = H + (long long)i * PMAX * PMAX;
    double* Mw = M + (long long)i * PMAX * PMAX;
    for (int e = t; e < p * p; e += TPB) {
        const int a = e / p, b = e % p;
        double hs = 0.0, ms = 0.0;
        for (int sp = 0; sp < gsplit; ++sp) {
            const long long o = ((long long)i * gsplit + sp) * PMAX * PMAX + a * PMAX + b;
            hs += Hp[o];
            ms += Mp[o];
        }
        Hw[a * PMAX + b] = hs;
        Mw[a * PMAX + b] = ms;
    }
    const double* Hi = Hw;
    const double* Mi = Mw;
    if (t == 0) s_zero = 0;
    __syncthreads();
    if (t < PMAX) {
        double mkk = t < p ? Mi[t * PMAX + t] : 0.0;
        dsc[t] = mkk > 0.0 ? rsqrt_nr(mkk) : 0.0;
        if (t < p && !(mkk > 0.0)) s_zero = 1;
    }
    __syncthreads();
    // scaled M into L, scaled H into T (q x q, dummy rows zero)
    for (int e = t; e < q * q; e += TPB) {
        int a = e / q, b = e % q;
        bool ok = a < p && b < p;
        L[a][b] = ok ? dsc[a] * Mi[a * PMAX + b] * dsc[b] : 0.0;
        T[a][b] = ok ? dsc[a] * Hi[a * PMAX + b] * dsc[b] : 0.0;
    }
    __syncthreads();
    int r = 0;
    if (!s_zero && rr_fast(S, V, L, T, U, p, q)) {
        r = p;
        goto sorted_output;
    }
    // warp 0: Cholesky of L in place (lane a owns row a), then U = L^{-1}
    // (lane c owns column c).  A column with dsc == 0 is dropped (linv = 0);
    // any other pivot <= 1e-13 sends the problem to the pseudo-inverse path.
    if (t < 32) {
        const int lane = t;
        int fail = 0;
        for (int k = 0; k < p; ++k) {
            const double d = L[k][k];
            double lkk = 0.0, r = 0.0;
            if (dsc[k] != 0.0) {
                if (d > 1e-13) { r = rsqrt_nr(d); lkk = d * r; }
                else fail = 1;
            }
            __syncwarp();
            if (lane == k) { L[k][k] = lkk; linv[k] = r; }
            if (lane > k && lane < p) L[lane][k] *= r;
            __syncwarp();
            if (lane > k && lane < p)
                for (int b = k + 1; b <= lane; ++b) L[lane][b] -= L[lane][k] * L[b][k];
            __syncwarp();
        }
        if (lane < q) {
            const int c = lane;
            for (int r = 0; r < q; ++r) {
                double v = 0.0;
                if (c < p && r >= c && r < p) {
                    double a0 = (r == c) ? 1.0 : 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
                    int j = c;
                    for (; j + 3 < r; j += 4) {
                        a0 -= L[r][j] * U[j][c];
                        a1 -= L[r][j + 1] * U[j + 1][c];
                        a2 -= L[r][j + 2] * U[j + 2][c];
                        a3 -= L[r][j + 3] * U[j + 3][c];
                    }
                    for (; j < r; ++j) a0 -= L[r][j] * U[j][c];
                    v = ((a0 + a1) + (a2 + a3)) * linv[r];
                }
                U[r][c] = v;
            }
        }
        if (lane == 0) s_fail = fail;
    }
    __syncthreads();
    if (!s_fail) {
        // G = U T U^T  (S = U T, then V = S U^T)
        smem_gemm(S, U, T, q, false);
        __syncthreads();
        for (int e = t; e < q * q; e += TPB) T[e % q][e / q] = U[e / q][e % q];   // T = U^T
        __syncthreads();
        smem_gemm(V, S, T, q, false);
        __syncthreads();
        for (int e = t; e < q * q; e += TPB) {
            int a = e / q, b = e % q;
            double v = (a < p && b < p) ? 0.5 * (V[a][b] + V[b][a]) : 0.0;
            if (a < p && b < p && (linv[a] == 0.0 || linv[b] == 0.0)) v = (a == b) ? 1e300 : 0.0;
            S[a][b] = v;
        }
        __syncthreads();
        mixed_jacobi(S, V, T, L, q);
        // C' = U^T V into T (the D scaling is applied on output)
        smem_gemm(T, U, V, q, true);
        __syncthreads();
        for (int k = 0; k < p; ++k) r += linv[k] > 0.0 ? 1 : 0;
    } else {
        // pseudo-inverse square root of D M D via its eigen-decomposition
        for (int e = t; e < q * q; e += TPB) {
            int a = e / q, b = e % q;
            S[a][b] = (a < p && b < p) ? dsc[a] * Mi[a * PMAX + b] * dsc[b] : 0.0;
        }
        __syncthreads();
        block_jacobi<double>(S, V, q, 1e-12, 1e-15, 30);   // S diag = s, V = U
        double smax = 0.0;
        for (int k = 0; k < p; ++k) smax = fmax(smax, S[k][k]);
        __syncthreads();
        if (t < PMAX) th[t] = (t < p && S[t][t] > 1e-13 * smax) ? rsqrt_nr(S[t][t]) : 0.0;
        __syncthreads();
        for (int e = t; e < q * q; e += TPB) {              // L = U diag(th)
            int a = e / q, b = e % q;
            L[a][b] = (a < p && b < p) ? V[a][b] * th[b] : 0.0;
        }
        __syncthreads();
        smem_gemm(S, T, L, q, false);                       // S = T L (T holds scaled H)
        __syncthreads();
        smem_gemm(V, L, S, q, true);                        // V = L^T S
        __syncthreads();
        for (int e = t; e < q * q; e += TPB) {
            int a = e / q, b = e % q;
            double v = (a < p && b < p) ? 0.5 * (V[a][b] + V[b][a]) : 0.0;
            if (a < p && b < p && (th[a] == 0.0 || th[b] == 0.0)) v = (a == b) ? 1e300 : 0.0;
            S[a][b] = v;
        }
        __syncthreads();
        block_jacobi<double>(S, V, q, 1e-12, 1e-15, 30);
        smem_gemm(T, L, V, q, false);                       // C' = L V
        __syncthreads();
        for (int k = 0; k < p; ++k) r += th[k] > 0.0 ? 1 : 0;
    }
sorted_output:
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
// FULL = false: X = Y C only (AX, BX, partial untouched).
// DF (with FULL = false, the chosen form's X-only update): the products in
// double-float (split_f64 while staging, df_fma), X stored as FP64.
template <bool FULL, bool DF = false>
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
    if constexpr (DF && !FULL) {
        // hi and lo halves of C and of the row block, as FP32 in the FP64 arrays' space
        float (*cH)[LD] = reinterpret_cast<float (*)[LD]>(&sC[0][0]);
        float (*cL)[LD] = cH + PMAX;
        float (*yH)[LD] = reinterpret_cast<float (*)[LD]>(&sY[0][0]);
        float (*yL)[LD] = yH + ROWBLK;
        for (int e = t; e < p * p; e += TPB)
            split_f64(C[(long long)i * PMAX * PMAX + (e / p) * PMAX + e % p], cH[e / p][e % p], cL[e / p][e % p]);
        for (int e = t; e < ROWBLK * p; e += TPB) {
            const int rr = e / p, c = e % p, r = r0 + rr;
            split_f64(r < n ? Y[(roff + r) * ldx + c] : 0.0, yH[rr][c], yL[rr][c]);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int e = t + k * TPB;
            if (e >= ROWBLK * p) break;
            const int rr = e / p, c = e % p;
            float xh = 0.f, xl = 0.f;
            for (int j = 0; j < p; ++j) df_fma(xh, xl, yH[rr][j], yL[rr][j], cH[j][c], cL[j][c]);
            const int r = r0 + rr;
            if (r < rows) X[(roff + r) * ldx + c] = df_to_f64(xh, xl);
        }
        return;
    }
    for (int e = t; e < p * p; e += TPB) sC[e / p][e % p] = C[(long long)i * PMAX * PMAX + (e / p) * PMAX + e % p];
    for (int e = t; e < ROWBLK * p; e += TPB) {
        int rr = e / p, c = e % p;
        int r = r0 + rr;
        bool ok = r < n;
        long long idx = (roff + r) * ldx + c;
        sY[rr][c] = ok ? Y[idx] : 0.0;
        if (FULL) {
            sA[rr][c] = ok ? AY[idx] : 0.0;
            sB[rr][c] = ok ? BY[idx] : 0.0;
        }
    }
    __syncthreads();
    if (!FULL) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int e = t + k * TPB;
            if (e >= ROWBLK * p) break;
            int rr = e / p, c = e % p;
            double x = 0.0;
            for (int j = 0; j < p; ++j) x += sY[rr][j] * sC[j][c];
            int r = r0 + rr;
            if (r < rows) X[(roff + r) * ldx + c] = x;
        }
        return;
    }
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
// Partial Grams over `gsplit` row ranges of each problem (grid: problems x
// splits), written to Gp[(i gsplit + s) PMAX^2]; k_cholqr sums them.
__global__ void __launch_bounds__(TPB) k_gram32(const double* __restrict__ W, double* __restrict__ Gp,
                                                const int* __restrict__ n_, const long long* __restrict__ roff_,
                                                const int* __restrict__ p_, int ldx, int gsplit) {
    __shared__ float sW[ROWBLK][LD];
    const int i = blockIdx.x, sp = blockIdx.y;
    const int n = n_[i], p = p_[i];
    const long long roff = roff_[i];
    const int rows_per = (n + gsplit - 1) / gsplit;
    const int r_lo = sp * rows_per, r_hi = min(n, r_lo + rows_per);
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
    for (int r0 = r_lo; r0 < r_hi; r0 += ROWBLK) {
        __syncthreads();
        for (int e = threadIdx.x; e < ROWBLK * p; e += TPB) {
            int rr = e / p, c = e % p;
            int r = r0 + rr;
            sW[rr][c] = r < r_hi ? f64_to_f32(W[(roff + r) * ldx + c]) : 0.f;
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
    double* G = Gp + ((long long)i * gsplit + sp) * PMAX * PMAX;
    for (int q = 0; q < 3; ++q) {
        if (pa[q] < 0) continue;
        G[pa[q] * PMAX + pb[q]] = f32_to_f64(acc[q]);
        G[pb[q] * PMAX + pa[q]] = f32_to_f64(acc[q]);
    }
}

// C = D R^{-1} with D = diag(G)^{-1/2} and D G D = R^T R (FP32 Cholesky, one
// warp per problem: G holds FP32 products and X = W C is formed in FP32, so
// FP64 here would only lengthen the serial chain).  A column whose pivot
// falls below 1e-10 of its scaled diagonal is dependent on the previous
// ones: it is reset to its scaled self (R row e_k) so that the basis stays
// finite; the FP64 phase removes it.
__device__ __forceinline__ float rsqrt_f32(float x) {
    const float r = rsqrtf(x);
    return r * fmaf(-0.5f * x * r, r, 1.5f);
}
__global__ void k_cholqr(const double* __restrict__ Gp, int gsplit, double* __restrict__ C,
                         const int* __restrict__ p_) {
    __shared__ float R[PMAX][LD], Ri[PMAX][LD], d[PMAX], d_inv[PMAX];
    const int i = blockIdx.x;
    const int p = p_[i];
    const int t = threadIdx.x;
    const double* Gi = Gp + (long long)i * gsplit * PMAX * PMAX;
    // G = sum of the row-range partials, by the whole block (their loads are
    // the long part); the factorisation below is one warp's
    for (int e = t; e < PMAX * PMAX; e += blockDim.x) {
        int a = e / PMAX, b = e % PMAX;
        float g = 0.f;
        if (a < p && b < p)
            for (int sp = 0; sp < gsplit; ++sp) g += f64_to_f32(Gi[(long long)sp * PMAX * PMAX + e]);
        R[a][b] = g;
        Ri[a][b] = 0.f;
    }
    __syncthreads();
    if (t >= 32) return;
    if (t < PMAX) {
        const float g = t < p ? R[t][t] : 0.f;
        d[t] = g > 0.f ? rsqrt_f32(g) : 0.f;
    }
    __syncwarp();
    for (int e = t; e < PMAX * PMAX; e += 32) {
        int a = e / PMAX, b = e % PMAX;
        R[a][b] = (a < p && b < p) ? d[a] * R[a][b] * d[b] : 0.f;
    }
    __syncwarp();
    // upper Cholesky in place: R <- U with D G D = U^T U
    for (int k = 0; k < p; ++k) {
        const float piv = R[k][k];
        const bool ok = piv > 1e-10f;
        const float ru = ok ? rsqrt_f32(piv) : 1.f;
        __syncwarp();
        if (t == 0) { R[k][k] = ok ? piv * ru : 1.f; d_inv[k] = ru; }
        for (int j = k + 1 + t; j < p; j += 32) R[k][j] = ok ? R[k][j] * ru : 0.f;
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
            float v = (r == t) ? 1.f : 0.f;
            for (int j = r + 1; j <= t; ++j) v -= R[r][j] * Ri[j][t];
            Ri[r][t] = v * d_inv[r];
        }
    }
    __syncwarp();
    for (int e = t; e < PMAX * PMAX; e += 32) {
        int a = e / PMAX, b = e % PMAX;
        C[(long long)i * PMAX * PMAX + e] = (a < p && b < p) ? f32_to_f64(d[a] * Ri[a][b]) : 0.0;
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
    for (int e = t; e < p * p; e += TPB) sC[e / p][e % p] = f64_to_f32(C[(long long)i * PMAX * PMAX + (e / p) * PMAX + e % p]);
    for (int e = t; e < ROWBLK * p; e += TPB) {
        int rr = e / p, c = e % p;
        int r = r0 + rr;
        sW[rr][c] = r < n ? f64_to_f32(W[(roff + r) * ldx + c]) : 0.f;
    }
    __syncthreads();
    for (int e = t; e < ROWBLK * p; e += TPB) {
        int rr = e / p, c = e % p;
        if (r0 + rr >= rows) continue;
        float x = 0.f;
        for (int j = 0; j < p; ++j) x += sW[rr][j] * sC[j][c];
        X[(roff + r0 + rr) * ldx + c] = f32_to_f64(x);
    }
}

// AX = Abar X and BX = X Abar X (X the indicator of the own generators, rows
// and columns < nown): one tiled product (32 rows x 8 NQ columns of the
// output per CTA, k-tiles of 32 staged in shared memory) whose k-sum is
// split at nown: AX = own part + rest, BX = own part on own rows.
template <int NQ>
__global__ void __launch_bounds__(256) k_dense_pencil(const double* __restrict__ A, const long long* __restrict__ aoff,
                                                      const int* __restrict__ n_, const int* __restrict__ nown_,
                                                      const long long* __restrict__ roff_,
                                                      const double* __restrict__ X, double* __restrict__ AX,
                                                      double* __restrict__ BX, int ldx, int ncols,
                                                      const int* __restrict__ skip) {
    constexpr int GT = 32, TN = 8 * NQ;
    __shared__ double sA[GT][GT + 1], sX[GT][TN + 1];
    const int i = blockIdx.z;
    if (skip && skip[i]) return;
    const int n = n_[i], nown = nown_[i];
    const int row0 = blockIdx.y * GT, col0 = blockIdx.x * TN;
    if (row0 >= n || col0 >= ncols) return;
    const long long roff = roff_[i];
    const double* Ai = A + aoff[i];
    const int t = threadIdx.x, r = t >> 3, cb = t & 7;
    double ao[NQ], an[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) { ao[q] = 0.0; an[q] = 0.0; }
    for (int k0 = 0; k0 < n; k0 += GT) {
        for (int e = t; e < GT * GT; e += 256) {
            const int a = e / GT, b = e % GT, gr = row0 + a, gk = k0 + b;
            sA[a][b] = (gr < n && gk < n) ? Ai[(long long)gr * n + gk] : 0.0;
        }
        for (int e = t; e < GT * TN; e += 256) {
            const int a = e / TN, b = e % TN, gk = k0 + a, gc = col0 + b;
            sX[a][b] = (gk < n && gc < ncols) ? X[(roff + gk) * ldx + gc] : 0.0;
        }
        __syncthreads();
        if (k0 + GT <= nown) {
#pragma unroll 8
            for (int k = 0; k < GT; ++k) {
                const double a = sA[r][k];
#pragma unroll
                for (int q = 0; q < NQ; ++q) ao[q] += a * sX[k][cb + 8 * q];
            }
        } else if (k0 >= nown) {
#pragma unroll 8
            for (int k = 0; k < GT; ++k) {
                const double a = sA[r][k];
#pragma unroll
                for (int q = 0; q < NQ; ++q) an[q] += a * sX[k][cb + 8 * q];
            }
        } else {
            for (int k = 0; k < GT; ++k) {
                const double a = sA[r][k];
                if (k0 + k < nown) {
#pragma unroll
                    for (int q = 0; q < NQ; ++q) ao[q] += a * sX[k][cb + 8 * q];
                } else {
#pragma unroll
                    for (int q = 0; q < NQ; ++q) an[q] += a * sX[k][cb + 8 * q];
                }
            }
        }
        __syncthreads();
    }
    const int gr = row0 + r;
    if (gr >= n) return;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const int gc = col0 + cb + 8 * q;
        if (gc < ncols) {
            AX[(roff + gr) * ldx + gc] = ao[q] + an[q];
            BX[(roff + gr) * ldx + gc] = gr < nown ? ao[q] : 0.0;
        }
    }
}

__global__ void k_load_start(double* __restrict__ X, const double* __restrict__ Wst, int wc,
                             const long long* __restrict__ woff, const int* __restrict__ n_,
                             const long long* __restrict__ roff_, const int* __restrict__ p_, int ldx) {
    const int i = blockIdx.y;
    const int n = n_[i], c1 = min(wc, p_[i]);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)n * c1;
         e += (long long)gridDim.x * blockDim.x) {
        const long long r = e / c1;
        const int c = (int)(e % c1);
        X[(roff_[i] + r) * ldx + c] = Wst[(woff[i] + r) * wc + c];
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
    // row splits: about 2048 CTAs in total, at least 64 rows per split (the
    // double-float Gram waits on its staging loads: more CTAs hide that)
    gsplit = (int)std::max<long long>(1, std::min<long long>(ceil_div(2048, std::max(P, 1)),
                                                                 ceil_div((long long)K.max_K * NB, 64)));
    Hp.alloc((size_t)P * gsplit * PMAX * PMAX);
    Mp.alloc((size_t)P * gsplit * PMAX * PMAX);
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
    n_active.alloc(2);
}

GevpBatch GevpBatch::slice(int p0, int np, int group) const {
    GevpBatch v;
    v.P = np;
    v.ldx = ldx;
    v.p.assign(p.begin() + p0, p.begin() + p0 + np);
    v.d_p = d_p.view(p0, np);
    v.K = K.slice(p0, np);
    for (auto pr : {std::make_pair(&v.X, &X), std::make_pair(&v.AX, &AX), std::make_pair(&v.BX, &BX),
                    std::make_pair(&v.Y, &Y), std::make_pair(&v.AY, &AY), std::make_pair(&v.BY, &BY),
                    std::make_pair(&v.W, &W)})
        *pr.first = pr.second->view(0, pr.second->n);
    const size_t q2 = (size_t)PMAX * PMAX;
    v.H = H.view(p0 * q2, np * q2); v.M = M.view(p0 * q2, np * q2); v.C = C.view(p0 * q2, np * q2);
    v.theta = theta.view((size_t)p0 * PMAX, (size_t)np * PMAX);
    v.res = res.view((size_t)p0 * PMAX, (size_t)np * PMAX);
    v.gsplit = gsplit;
    v.Hp = Hp.view(p0 * gsplit * q2, np * gsplit * q2);
    v.Mp = Mp.view(p0 * gsplit * q2, np * gsplit * q2);
    v.nblk_max = nblk_max;
    v.partial = partial.view((size_t)p0 * nblk_max * 2 * PMAX, (size_t)np * nblk_max * 2 * PMAX);
    v.done = done.view(p0, np); v.m = m.view(p0, np); v.rank = rank.view(p0, np); v.iters = iters.view(p0, np);
    v.best = best.view(p0, np); v.best_it = best_it.view(p0, np);
    v.n_active = n_active.view(group, 1);
    v.knorm = knorm;
    return v;
}

void eig_load_start(GevpBatch& g, const double* Wst, int wc, const long long* d_woff, cudaStream_t s) {
    if (g.P == 0 || !Wst || wc <= 0) return;
    dim3 grid(32, g.P);
    k_load_start<<<grid, 256, 0, s>>>(g.X.p, Wst, wc, d_woff, g.K.d_n.p, g.K.d_roff.p, g.d_p.p, g.ldx);
    MSDD_LAUNCH_CHECK();
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
    k_gram32<<<dim3(g.P, g.gsplit), TPB, 0, s>>>(g.W.p, g.Hp.p, g.K.d_n.p, g.K.d_roff.p, g.d_p.p, g.ldx, g.gsplit);
    MSDD_LAUNCH_CHECK();
    k_cholqr<<<g.P, 256, 0, s>>>(g.Hp.p, g.gsplit, g.C.p, g.d_p.p);
    MSDD_LAUNCH_CHECK();
    dim3 grid(g.nblk_max, g.P);
    k_update32<<<grid, TPB, 0, s>>>(g.W.p, g.X.p, g.C.p, g.K.d_n.p, g.K.d_K.p, g.K.d_roff.p, g.d_p.p, g.ldx);
    MSDD_LAUNCH_CHECK();
}

void eig_gram(GevpBatch& g, cudaStream_t s) {
    // the chosen form (FP32 fine factors) takes the double-float products
    if (g.K.prec)
        k_gram_split<true><<<dim3(g.P, g.gsplit), GR_T, 0, s>>>(g.Y.p, g.AY.p, g.BY.p, g.Hp.p, g.Mp.p, g.K.d_n.p,
                                                                g.K.d_roff.p, g.d_p.p, g.ldx, g.done.p, g.gsplit);
    else
        k_gram_split<false><<<dim3(g.P, g.gsplit), GR_T, 0, s>>>(g.Y.p, g.AY.p, g.BY.p, g.Hp.p, g.Mp.p, g.K.d_n.p,
                                                                 g.K.d_roff.p, g.d_p.p, g.ldx, g.done.p, g.gsplit);
    MSDD_LAUNCH_CHECK();
}

void eig_rayleigh_ritz(GevpBatch& g, cudaStream_t s) {
    k_rayleigh_ritz<<<g.P, TPB, 0, s>>>(g.Hp.p, g.Mp.p, g.gsplit, g.H.p, g.M.p, g.C.p, g.theta.p, g.d_p.p, g.rank.p,
                                        g.done.p);
    MSDD_LAUNCH_CHECK();
}

void eig_update(GevpBatch& g, cudaStream_t s) {
    dim3 grid(g.nblk_max, g.P);
    k_update<true><<<grid, TPB, 0, s>>>(g.Y.p, g.AY.p, g.BY.p, g.X.p, g.AX.p, g.BX.p, g.C.p, g.theta.p, g.K.d_n.p,
                                        g.K.d_K.p, g.K.d_roff.p, g.d_p.p, g.ldx, g.partial.p, g.nblk_max, g.done.p);
    MSDD_LAUNCH_CHECK();
}

void eig_update_x(GevpBatch& g, cudaStream_t s) {
    dim3 grid(g.nblk_max, g.P);
    if (g.K.prec)
        k_update<false, true><<<grid, TPB, 0, s>>>(g.Y.p, nullptr, nullptr, g.X.p, nullptr, nullptr, g.C.p, g.theta.p,
                                                   g.K.d_n.p, g.K.d_K.p, g.K.d_roff.p, g.d_p.p, g.ldx, nullptr,
                                                   g.nblk_max, g.done.p);
    else
        k_update<false><<<grid, TPB, 0, s>>>(g.Y.p, nullptr, nullptr, g.X.p, nullptr, nullptr, g.C.p, g.theta.p,
                                             g.K.d_n.p, g.K.d_K.p, g.K.d_roff.p, g.d_p.p, g.ldx, nullptr, g.nblk_max,
                                             g.done.p);
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
    if (P == 0 || nmax == 0 || ncols == 0) return;
    const int nq = ncols >= 32 ? 4 : (ncols + 7) / 8;
    dim3 grid(ceil_div(ncols, 8 * nq), ceil_div(nmax, 32), P);
    switch (nq) {
        case 1: k_dense_pencil<1><<<grid, 256, 0, s>>>(Abar, d_aoff, d_n, d_nown, layout.d_roff.p, X, AX, BX, ldx, ncols, skip); break;
        case 2: k_dense_pencil<2><<<grid, 256, 0, s>>>(Abar, d_aoff, d_n, d_nown, layout.d_roff.p, X, AX, BX, ldx, ncols, skip); break;
        case 3: k_dense_pencil<3><<<grid, 256, 0, s>>>(Abar, d_aoff, d_n, d_nown, layout.d_roff.p, X, AX, BX, ldx, ncols, skip); break;
        default: k_dense_pencil<4><<<grid, 256, 0, s>>>(Abar, d_aoff, d_n, d_nown, layout.d_roff.p, X, AX, BX, ldx, ncols, skip); break;
    }
    MSDD_LAUNCH_CHECK();
}

}  // namespace msdd
