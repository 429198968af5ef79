// Batched tile-band LDL^T factorisation and triangular solves (one CTA per
// local matrix).  See tile_ldlt.cuh for the storage format.
#include "tile_ldlt.cuh"

#include <cuda.h>
#include <cstring>
#include <mutex>
#include <type_traits>

namespace msdd {

namespace {

constexpr int TPB = 256;     // threads per CTA; each owns 4 entries of a 32 x 32 tile
constexpr int LDS = NB + 1;  // padded shared-memory row stride

__device__ __forceinline__ long long tile_index(long long toff, int kb, int R, int C) {
    return toff + ((long long)R * (kb + 1) + (R - C)) * NB2;
}

template <typename T>
__device__ __forceinline__ void load_tile(T (*dst)[LDS], const T* __restrict__ src) {
    for (int e = threadIdx.x; e < NB2; e += TPB) dst[e / NB][e % NB] = src[e];
}

template <typename T>
__device__ __forceinline__ void store_tile(T* __restrict__ dst, T (*src)[LDS]) {
    for (int e = threadIdx.x; e < NB2; e += TPB) dst[e] = src[e / NB][e % NB];
}

// ------------------------------------------------------------------ factor
// Dense LDL^T of the diagonal tile R held in W (lower triangle; rows >=
// rows_valid are padding): pivots d with d <= reg_tol * od (the original
// diagonal) are null pivots (D^{-1} = 0, counted in s_nreg), other
// non-positive pivots set s_status to the first failing row + 1.  T_R =
// L_RR^{-1} (unit lower) is built in Sa and stored to Tdst, D^{-1} to ddst.
template <typename T>
__device__ void factor_diag_tile(T (*W)[LDS], T (*Sa)[LDS], T* sd, const T* od, T& piv_inv, int rows_valid,
                                 double reg_tol, int R, int& s_status, int& s_nreg, T* __restrict__ Tdst,
                                 T* __restrict__ ddst) {
    const int t = threadIdx.x;
    for (int k = 0; k < NB; ++k) {
        if (t == 0) {
            T d = W[k][k];
            T dinv_k;
            if (k >= rows_valid) {
                dinv_k = T(1);
            } else if (reg_tol > 0.0 && !(d > T(reg_tol) * od[k])) {
                dinv_k = T(0);
                ++s_nreg;
            } else if (!(d > T(0))) {
                dinv_k = T(0);
                if (s_status == 0) s_status = R * NB + k + 1;
            } else {
                dinv_k = T(1) / d;
            }
            piv_inv = dinv_k;
            sd[k] = dinv_k;
        }
        __syncthreads();
        const T pinv = piv_inv;
        // trailing update W[a][b] -= W[a][k] W[b][k] / d for k < b <= a
        for (int e = t; e < NB2; e += TPB) {
            int a = e / NB, b = e % NB;
            if (b > k && a >= b) W[a][b] -= W[a][k] * W[b][k] * pinv;
        }
        __syncthreads();
        if (t > k && t < NB) W[t][k] = (k >= rows_valid || t >= rows_valid) ? T(0) : W[t][k] * pinv;
        __syncthreads();
    }
    for (int e = t; e < NB2; e += TPB) Sa[e / NB][e % NB] = (e / NB == e % NB) ? T(1) : T(0);
    __syncthreads();
    for (int k = 0; k < NB - 1; ++k) {
        for (int e = t; e < NB2; e += TPB) {
            int a = e / NB, b = e % NB;
            if (a > k && b <= k) Sa[a][b] -= W[a][k] * Sa[k][b];
        }
        __syncthreads();
    }
    store_tile(Tdst, Sa);
    if (t < NB) ddst[t] = sd[t];
}

template <typename T>
__global__ void __launch_bounds__(TPB) k_tile_factor(
    T* __restrict__ tiles, T* __restrict__ dinv, const int* __restrict__ n_, const int* __restrict__ kb_,
    const int* __restrict__ K_, const long long* __restrict__ toff_, const long long* __restrict__ roff_,
    int* __restrict__ status, int* __restrict__ nreg, double reg_tol)
{
    __shared__ T W[NB][LDS];
    __shared__ T Sa[NB][LDS];
    __shared__ T Sb[NB][LDS];
    __shared__ T sd[NB];
    __shared__ T od[NB];
    __shared__ T piv_inv;
    __shared__ int s_status, s_nreg;

    const int i = blockIdx.x;
    const int n = n_[i], kb = kb_[i], K = K_[i];
    const long long toff = toff_[i], roff = roff_[i];
    const int t = threadIdx.x;
    const int r = t >> 3, c0 = t & 7;
    if (t == 0) { s_status = 0; s_nreg = 0; }

    for (int R = 0; R < K; ++R) {
        const int Cmin = R - kb > 0 ? R - kb : 0;
        for (int C = Cmin; C <= R; ++C) {
            __syncthreads();
            load_tile(W, tiles + tile_index(toff, kb, R, C));
            __syncthreads();
            if (C == R && t < NB) od[t] = W[t][t];
            // W -= sum_J L_RJ D_J L_CJ^T
            const int Jmin = (C - kb > Cmin) ? C - kb : Cmin;
            T acc[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] = W[r][c0 + 8 * q];
            for (int J = Jmin; J < C; ++J) {
                __syncthreads();
                load_tile(Sa, tiles + tile_index(toff, kb, R, J));
                load_tile(Sb, tiles + tile_index(toff, kb, C, J));
                if (t < NB) {
                    T di = dinv[roff + (long long)J * NB + t];
                    sd[t] = di != T(0) ? T(1) / di : T(0);
                }
                __syncthreads();
#pragma unroll 8
                for (int k = 0; k < NB; ++k) {
                    T a = Sa[r][k] * sd[k];
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[q] -= a * Sb[c0 + 8 * q][k];
                }
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < 4; ++q) W[r][c0 + 8 * q] = acc[q];
            __syncthreads();
            if (C < R) {
                // L_RC = W T_C^T D_C^{-1}
                load_tile(Sb, tiles + tile_index(toff, kb, C, C));
                if (t < NB) sd[t] = dinv[roff + (long long)C * NB + t];
                __syncthreads();
                T out[4] = {0, 0, 0, 0};
#pragma unroll 8
                for (int k = 0; k < NB; ++k) {
                    T w = W[r][k];
#pragma unroll
                    for (int q = 0; q < 4; ++q) out[q] += w * Sb[c0 + 8 * q][k];
                }
                T* dst = tiles + tile_index(toff, kb, R, C);
#pragma unroll
                for (int q = 0; q < 4; ++q) dst[r * NB + c0 + 8 * q] = out[q] * sd[c0 + 8 * q];
            } else {
                factor_diag_tile<T>(W, Sa, sd, od, piv_inv, n - R * NB, reg_tol, R, s_status, s_nreg,
                                    tiles + tile_index(toff, kb, R, R), dinv + roff + (long long)R * NB);
            }
        }
    }
    __syncthreads();
    if (t == 0) { status[i] = s_status; nreg[i] = s_nreg; }
}

// ------------------------------------------------------------------ solve
// acc[r][c] for the 4 (row, column) pairs owned by a thread: row r = t>>3,
// columns c0 + 8q.
template <typename T>
__global__ void __launch_bounds__(TPB) k_tile_solve(
    const T* __restrict__ tiles, const T* __restrict__ dinv, const int* __restrict__ n_,
    const int* __restrict__ kb_, const int* __restrict__ K_, const long long* __restrict__ toff_,
    const long long* __restrict__ roff_, double* __restrict__ X, int ldx, int ncols,
    const int* __restrict__ skip, const int* __restrict__ gdone)
{
    __shared__ T Sa[NB][LDS];
    __shared__ T Sx[NB][LDS];   // operand block of X (rows x columns)
    __shared__ T Acc[NB][LDS];

    const int i = blockIdx.x;
    if (skip && skip[i]) return;
    if (gdone && *gdone) return;
    const int kb = kb_[i], K = K_[i];
    const long long toff = toff_[i], roff = roff_[i];
    const int t = threadIdx.x;
    const int r = t >> 3, c0 = t & 7;
    (void)n_;
    // this CTA handles the columns [32 * blockIdx.y, 32 * blockIdx.y + 32)
    const int c_lo = blockIdx.y * NB;
    X += c_lo;
    ncols = min(NB, ncols - c_lo);
    if (ncols <= 0) return;

    // forward: z_R = T_R (x_R - sum_J L_RJ z_J)
    for (int R = 0; R < K; ++R) {
        T acc[4];
        double* xr = X + (roff + (long long)R * NB) * ldx;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int c = c0 + 8 * q;
            acc[q] = c < ncols ? T(xr[(long long)r * ldx + c]) : T(0);
        }
        const int Jmin = R - kb > 0 ? R - kb : 0;
        for (int J = Jmin; J < R; ++J) {
            __syncthreads();
            load_tile(Sa, tiles + tile_index(toff, kb, R, J));
            const double* xj = X + (roff + (long long)J * NB) * ldx;
            for (int e = t; e < NB * NB; e += TPB) {
                int a = e / NB, c = e % NB;
                Sx[a][c] = c < ncols ? T(xj[(long long)a * ldx + c]) : T(0);
            }
            __syncthreads();
#pragma unroll 8
            for (int k = 0; k < NB; ++k) {
                T l = Sa[r][k];
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[q] -= l * Sx[k][c0 + 8 * q];
            }
        }
        __syncthreads();
        load_tile(Sa, tiles + tile_index(toff, kb, R, R));
#pragma unroll
        for (int q = 0; q < 4; ++q) Acc[r][c0 + 8 * q] = acc[q];
        __syncthreads();
        T out[4] = {0, 0, 0, 0};
        for (int k = 0; k <= r; ++k) {
            T l = Sa[r][k];
#pragma unroll
            for (int q = 0; q < 4; ++q) out[q] += l * Acc[k][c0 + 8 * q];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int c = c0 + 8 * q;
            if (c < ncols) xr[(long long)r * ldx + c] = (double)out[q];
        }
    }
    // backward: x_R = T_R^T (D_R^{-1} z_R - sum_I L_IR^T x_I)
    for (int R = K - 1; R >= 0; --R) {
        __syncthreads();
        T acc[4];
        double* xr = X + (roff + (long long)R * NB) * ldx;
        const T dr = dinv[roff + (long long)R * NB + r];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int c = c0 + 8 * q;
            acc[q] = c < ncols ? dr * T(xr[(long long)r * ldx + c]) : T(0);
        }
        const int Imax = R + kb < K - 1 ? R + kb : K - 1;
        for (int I = R + 1; I <= Imax; ++I) {
            __syncthreads();
            load_tile(Sa, tiles + tile_index(toff, kb, I, R));
            const double* xi = X + (roff + (long long)I * NB) * ldx;
            for (int e = t; e < NB * NB; e += TPB) {
                int a = e / NB, c = e % NB;
                Sx[a][c] = c < ncols ? T(xi[(long long)a * ldx + c]) : T(0);
            }
            __syncthreads();
#pragma unroll 8
            for (int k = 0; k < NB; ++k) {
                T l = Sa[k][r];
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[q] -= l * Sx[k][c0 + 8 * q];
            }
        }
        __syncthreads();
        load_tile(Sa, tiles + tile_index(toff, kb, R, R));
#pragma unroll
        for (int q = 0; q < 4; ++q) Acc[r][c0 + 8 * q] = acc[q];
        __syncthreads();
        T out[4] = {0, 0, 0, 0};
        for (int k = r; k < NB; ++k) {
            T l = Sa[k][r];
#pragma unroll
            for (int q = 0; q < 4; ++q) out[q] += l * Acc[k][c0 + 8 * q];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int c = c0 + 8 * q;
            if (c < ncols) xr[(long long)r * ldx + c] = (double)out[q];
        }
    }
}


// cp.async (16-byte global -> shared copies, completion by groups)
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait_n() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// ------------------------------------------------------------------ solve, one right-hand side
// The PCG local solves.  One CTA of 128 threads per matrix; the whole local
// vector lives in shared memory.  Forward sweep: thread (row r = t/4, chunk
// t%4) reads 8 contiguous entries of row r of each tile (coalesced) and the 4
// partial sums of a row are combined by warp shuffles.  Backward sweep uses
// the transposed tiles: thread (column c = lane, rows 8*warp..) reads tile
// rows contiguously across the warp, partial sums of the 4 warps are combined
// in shared memory.  For band matrices (kb <= KBP) the tiles of step R+1 are
// loaded into registers while step R computes.
// ------------------------------------------------------------------ factor, dense, right-looking
// Dense batches (kb >= K - 1: coarse-level matrices) are factored one tile
// column k per launch triple, so that many CTAs share each step instead of
// one CTA per matrix: the diagonal tile (one CTA per problem), the panel
// L_ik = A_ik T_k^T D_k^{-1} (one CTA per tile), and the trailing update
// A_ij -= L_ik D_k L_jk^T for k < j <= i (one CTA per tile).  Every tile sees
// the subtractions of k_tile_factor in the same order and in the same
// precision, so the factors are the same.  k_save_diag first parks the
// original diagonal (the null-pivot reference) in dinv and clears the status.
template <typename T>
__global__ void __launch_bounds__(TPB) k_save_diag(const T* __restrict__ tiles, T* __restrict__ dinv,
                                                   const int* __restrict__ kb_, const int* __restrict__ K_,
                                                   const long long* __restrict__ toff_,
                                                   const long long* __restrict__ roff_, int* __restrict__ status,
                                                   int* __restrict__ nreg) {
    const int i = blockIdx.x;
    const int kb = kb_[i], K = K_[i];
    const long long toff = toff_[i], roff = roff_[i];
    for (int e = threadIdx.x; e < K * NB; e += TPB) {
        const int R = e / NB, r = e % NB;
        dinv[roff + e] = tiles[tile_index(toff, kb, R, R) + r * NB + r];
    }
    if (threadIdx.x == 0) { status[i] = 0; nreg[i] = 0; }
}

template <typename T>
__global__ void __launch_bounds__(TPB) k_rl_diag(T* __restrict__ tiles, T* __restrict__ dinv,
                                                 const int* __restrict__ n_, const int* __restrict__ kb_,
                                                 const int* __restrict__ K_, const long long* __restrict__ toff_,
                                                 const long long* __restrict__ roff_, int* __restrict__ status,
                                                 int* __restrict__ nreg, double reg_tol, int k) {
    __shared__ T W[NB][LDS];
    __shared__ T Sa[NB][LDS];
    __shared__ T sd[NB];
    __shared__ T od[NB];
    __shared__ T piv_inv;
    __shared__ int s_status, s_nreg;
    const int i = blockIdx.x;
    const int K = K_[i];
    if (k >= K) return;
    const int kb = kb_[i], t = threadIdx.x;
    const long long toff = toff_[i], roff = roff_[i];
    if (t == 0) { s_status = status[i]; s_nreg = nreg[i]; }
    load_tile(W, tiles + tile_index(toff, kb, k, k));
    if (t < NB) od[t] = dinv[roff + (long long)k * NB + t];
    __syncthreads();
    factor_diag_tile<T>(W, Sa, sd, od, piv_inv, n_[i] - k * NB, reg_tol, k, s_status, s_nreg,
                        tiles + tile_index(toff, kb, k, k), dinv + roff + (long long)k * NB);
    __syncthreads();
    if (t == 0) { status[i] = s_status; nreg[i] = s_nreg; }
}

// grid.y: i = k + 1 + blockIdx.y
template <typename T>
__global__ void __launch_bounds__(TPB) k_rl_panel(T* __restrict__ tiles, const T* __restrict__ dinv,
                                                  const int* __restrict__ kb_, const int* __restrict__ K_,
                                                  const long long* __restrict__ toff_,
                                                  const long long* __restrict__ roff_, int k) {
    __shared__ T W[NB][LDS];
    __shared__ T Sb[NB][LDS];
    __shared__ T sd[NB];
    const int i = blockIdx.x, R = k + 1 + blockIdx.y;
    const int K = K_[i];
    if (R >= K) return;
    const int kb = kb_[i], t = threadIdx.x, r = t >> 3, c0 = t & 7;
    const long long toff = toff_[i], roff = roff_[i];
    T* dst = tiles + tile_index(toff, kb, R, k);
    load_tile(W, dst);
    load_tile(Sb, tiles + tile_index(toff, kb, k, k));
    if (t < NB) sd[t] = dinv[roff + (long long)k * NB + t];
    __syncthreads();
    T out[4] = {0, 0, 0, 0};
#pragma unroll 8
    for (int kk = 0; kk < NB; ++kk) {
        T w = W[r][kk];
#pragma unroll
        for (int q = 0; q < 4; ++q) out[q] += w * Sb[c0 + 8 * q][kk];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) dst[r * NB + c0 + 8 * q] = out[q] * sd[c0 + 8 * q];
}

// grid.y enumerates the tiles (i, j), k < j <= i < K, row by row
template <typename T>
__global__ void __launch_bounds__(TPB) k_rl_update(T* __restrict__ tiles, const T* __restrict__ dinv,
                                                   const int* __restrict__ kb_, const int* __restrict__ K_,
                                                   const long long* __restrict__ toff_,
                                                   const long long* __restrict__ roff_, int k) {
    __shared__ T Sa[NB][LDS];
    __shared__ T Sb[NB][LDS];
    __shared__ T sd[NB];
    const int i = blockIdx.x;
    const int K = K_[i];
    int e = blockIdx.y, R = k + 1;
    while (R < K && e >= R - k) { e -= R - k; ++R; }
    if (R >= K) return;
    const int C = k + 1 + e;
    const int kb = kb_[i], t = threadIdx.x, r = t >> 3, c0 = t & 7;
    const long long toff = toff_[i], roff = roff_[i];
    T* dst = tiles + tile_index(toff, kb, R, C);
    T acc[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] = dst[r * NB + c0 + 8 * q];
    load_tile(Sa, tiles + tile_index(toff, kb, R, k));
    load_tile(Sb, tiles + tile_index(toff, kb, C, k));
    if (t < NB) {
        T di = dinv[roff + (long long)k * NB + t];
        sd[t] = di != T(0) ? T(1) / di : T(0);
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < NB; ++kk) {
        T a = Sa[r][kk] * sd[kk];
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] -= a * Sb[c0 + 8 * q][kk];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) dst[r * NB + c0 + 8 * q] = acc[q];
}

// ------------------------------------------------------------------ factor, FP32, half-bandwidth <= 2 tiles
// The steps and the arithmetic of k_tile_factor<float> (same expressions in
// the same order), arranged for latency: the tiles of the last three tile
// rows (L, T and the pivots) stay in shared memory, so nothing the CTA
// produced is read back from global memory; the original tiles of row R + 1
// are copied with cp.async while row R is factored; the diagonal tiles are
// factored and inverted by one warp holding a row per lane in registers
// (shuffles instead of block barriers).
constexpr int FB_T = 256, FB_LD = NB + 1, FB_ROWS = 3;
constexpr size_t factor_band32_smem() {
    return sizeof(float) * ((size_t)2 * FB_ROWS * NB2 + (size_t)FB_ROWS * FB_ROWS * NB * FB_LD + (size_t)NB * FB_LD +
                            (size_t)2 * FB_ROWS * NB + NB) + 16;
}

__global__ void __launch_bounds__(FB_T) k_tile_factor_band32(
    float* __restrict__ tiles, float* __restrict__ dinv, const int* __restrict__ n_, const int* __restrict__ kb_,
    const int* __restrict__ K_, const long long* __restrict__ toff_, const long long* __restrict__ roff_,
    int* __restrict__ status, int* __restrict__ nreg, double reg_tol)
{
    extern __shared__ __align__(16) float fb_sm[];
    float* stg = fb_sm;                                                          // [2][3][32*32] original tiles
    float (*cache)[NB][FB_LD] = reinterpret_cast<float (*)[NB][FB_LD]>(stg + 2 * FB_ROWS * NB2);  // [row%3 * 3 + d]
    float (*Wsm)[FB_LD] = reinterpret_cast<float (*)[FB_LD]>(&cache[FB_ROWS * FB_ROWS][0][0]);
    float* cpiv = &Wsm[NB][0];                                                   // [3][32] D = 1 / D^{-1}
    float* cdinv = cpiv + FB_ROWS * NB;                                          // [3][32] D^{-1}
    float* od = cdinv + FB_ROWS * NB;                                            // original diagonal
    __shared__ int s_status, s_nreg;

    const int i = blockIdx.x;
    const int n = n_[i], kb = kb_[i], K = K_[i];
    const long long toff = toff_[i], roff = roff_[i];
    const int t = threadIdx.x;
    const int r = t >> 3, c0 = t & 7;
    if (t == 0) { s_status = 0; s_nreg = 0; }
    auto issue_row = [&](int R) {
        if (R < K) {
            const int Cmin = R - kb > 0 ? R - kb : 0;
            for (int C = Cmin; C <= R; ++C) {
                const float* src = tiles + tile_index(toff, kb, R, C);
                float* dst = stg + ((R & 1) * FB_ROWS + (R - C)) * NB2;
                for (int ch = t; ch < NB2 / 4; ch += FB_T) cp_async16(dst + ch * 4, src + ch * 4);
            }
        }
        cp_async_commit();
    };
    issue_row(0);
    for (int R = 0; R < K; ++R) {
        issue_row(R + 1);
        cp_async_wait_n<1>();                       // row R landed (row R + 1 may be in flight)
        __syncthreads();
        const int Cmin = R - kb > 0 ? R - kb : 0;
        const int rs = R % FB_ROWS;
        for (int C = Cmin; C <= R; ++C) {
            __syncthreads();                        // the previous step's cache and Wsm accesses are done
            const float* A = stg + ((R & 1) * FB_ROWS + (R - C)) * NB2;
            if (C == R && t < NB) od[t] = A[t * NB + t];
            float acc[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] = A[r * NB + c0 + 8 * q];
            // W -= sum_J L_RJ D_J L_CJ^T
            for (int J = Cmin; J < C; ++J) {
                const float (*LR)[FB_LD] = cache[rs * FB_ROWS + (R - J)];
                const float (*LC)[FB_LD] = cache[(C % FB_ROWS) * FB_ROWS + (C - J)];
                const float* Dj = cpiv + (J % FB_ROWS) * NB;
#pragma unroll 8
                for (int k = 0; k < NB; ++k) {
                    const float a = LR[r][k] * Dj[k];
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[q] -= a * LC[c0 + 8 * q][k];
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) Wsm[r][c0 + 8 * q] = acc[q];
            __syncthreads();
            if (C < R) {
                // L_RC = W T_C^T D_C^{-1}
                const float (*TC)[FB_LD] = cache[(C % FB_ROWS) * FB_ROWS];
                const float* dC = cdinv + (C % FB_ROWS) * NB;
                float out[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 8
                for (int k = 0; k < NB; ++k) {
                    const float w = Wsm[r][k];
#pragma unroll
                    for (int q = 0; q < 4; ++q) out[q] += w * TC[c0 + 8 * q][k];
                }
                float* dst = tiles + tile_index(toff, kb, R, C);
                float (*Lc)[FB_LD] = cache[rs * FB_ROWS + (R - C)];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float v = out[q] * dC[c0 + 8 * q];
                    Lc[r][c0 + 8 * q] = v;
                    dst[r * NB + c0 + 8 * q] = v;
                }
            } else if (t < 32) {
                // dense LDL^T of the diagonal tile by warp 0, lane a holding
                // row a of W in registers (W[b][k] by shuffle from lane b);
                // then T_R = L_RR^{-1}, lane a building row a of T
                const int lane = t;
                const int rows_valid = n - R * NB;
                float row[NB];
#pragma unroll
                for (int b = 0; b < NB; ++b) row[b] = Wsm[lane][b];
                float dl = 0.f;                     // D^{-1} of this lane's row
                int nr = 0, st = 0;
#pragma unroll
                for (int k = 0; k < NB; ++k) {
                    const float d = __shfl_sync(0xffffffffu, row[k], k);
                    float dinv_k;
                    if (k >= rows_valid) {
                        dinv_k = 1.f;
                    } else if (reg_tol > 0.0 && !(d > (float)reg_tol * od[k])) {
                        dinv_k = 0.f;
                        ++nr;
                    } else if (!(d > 0.f)) {
                        dinv_k = 0.f;
                        if (st == 0) st = R * NB + k + 1;
                    } else {
                        dinv_k = 1.f / d;
                    }
                    if (lane == k) dl = dinv_k;
                    const float pinv = dinv_k;
                    const float wak = row[k];
                    // W[a][b] -= W[a][k] W[b][k] / d for k < b <= a
#pragma unroll
                    for (int b = 0; b < NB; ++b) {
                        if (b > k) {
                            const float wbk = __shfl_sync(0xffffffffu, wak, b);
                            if (lane >= b) row[b] -= wak * wbk * pinv;
                        }
                    }
                    if (lane > k) row[k] = (k >= rows_valid || lane >= rows_valid) ? 0.f : wak * pinv;
                }
                float tr[NB];
#pragma unroll
                for (int b = 0; b < NB; ++b) tr[b] = (b == lane) ? 1.f : 0.f;
#pragma unroll
                for (int k = 0; k < NB - 1; ++k) {
                    const float lak = row[k];
#pragma unroll
                    for (int b = 0; b < NB; ++b) {
                        if (b <= k) {
                            const float tkb = __shfl_sync(0xffffffffu, tr[b], k);
                            if (lane > k) tr[b] -= lak * tkb;
                        }
                    }
                }
                float* dst = tiles + tile_index(toff, kb, R, R);
                float (*Tc)[FB_LD] = cache[rs * FB_ROWS];
#pragma unroll
                for (int b = 0; b < NB; ++b) {
                    Tc[lane][b] = tr[b];
                    dst[lane * NB + b] = tr[b];
                }
                cdinv[rs * NB + lane] = dl;
                cpiv[rs * NB + lane] = dl != 0.f ? 1.f / dl : 0.f;
                dinv[roff + (long long)R * NB + lane] = dl;
                if (lane == 0) { s_nreg += nr; if (s_status == 0 && st != 0) s_status = st; }
            }
        }
        __syncthreads();                            // row R complete before its stage is refilled
    }
    cp_async_wait_n<0>();
    __syncthreads();
    if (t == 0) { status[i] = s_status; nreg[i] = s_nreg; }
}

constexpr int S1T = 128;

constexpr int S1_STAGES = 4;

template <typename T, int KBP>
constexpr size_t solve1_ring_bytes() { return sizeof(T) * (size_t)S1_STAGES * (KBP + 1) * NB2; }

template <typename T, int KBP>
__global__ void __launch_bounds__(S1T) k_tile_solve1(
    const T* __restrict__ tiles, const T* __restrict__ dinv, const int* __restrict__ kb_, const int* __restrict__ K_,
    const long long* __restrict__ toff_, const long long* __restrict__ roff_, double* __restrict__ X,
    const int* __restrict__ gdone)
{
    // The tiles of step R + S1_STAGES - 1 are copied into a shared ring with
    // cp.async while step R computes; zs holds the whole local vector.
    constexpr int NST = S1_STAGES;
    extern __shared__ __align__(16) unsigned char zs_raw[];
    T* ring = reinterpret_cast<T*>(zs_raw);                       // [NST][KBP + 1][32 * 32]
    T* zs = ring + (size_t)NST * (KBP + 1) * NB2;                 // [K * 32]
    __shared__ T accs[NB];
    __shared__ T part[S1T / 32][NB + 1];
    if (gdone && *gdone) return;
    const int i = blockIdx.x;
    const int kb = kb_[i], K = K_[i];
    const long long toff = toff_[i], roff = roff_[i];
    const int t = threadIdx.x;
    auto stage = [&](int st, int d) { return ring + ((size_t)st * (KBP + 1) + d) * NB2; };
    auto issue = [&](int st, int R, bool fwd) {
        if (R >= 0 && R < K) {
            for (int d = 0; d <= KBP; ++d) {
                const int other = fwd ? R - d : R + d;
                if (d > kb || other < 0 || other >= K) continue;
                const T* src = tiles + (fwd ? tile_index(toff, kb, R, other) : tile_index(toff, kb, other, R));
                T* dst = stage(st, d);
                constexpr int PER = 16 / (int)sizeof(T);
                for (int ch = t; ch < NB2 / PER; ch += S1T) cp_async16(dst + ch * PER, src + ch * PER);
            }
        }
        cp_async_commit();
    };
    for (int k = 0; k < NST - 1; ++k) issue(k, k, true);
    for (int e = t; e < K * NB; e += S1T) zs[e] = from_f64<T>(X[roff + e]);

    // forward: z_R = T_R (x_R - sum_{J<R} L_RJ z_J); thread (row r = t/4,
    // columns c0..c0+7) with the 4 partial sums of a row combined by shuffles
    {
        const int r = t >> 2, c0 = (t & 3) * 8;
        for (int R = 0; R < K; ++R) {
            const int st = R % NST;
            cp_async_wait_n<NST - 2>();
            __syncthreads();
            issue((R + NST - 1) % NST, R + NST - 1, true);
            T acc = T(0);
#pragma unroll
            for (int d = 1; d <= KBP; ++d) {
                if (d > kb || R - d < 0) continue;
                const T* lt = stage(st, d) + r * NB + c0;
                const T* zj = zs + (R - d) * NB + c0;
#pragma unroll
                for (int q = 0; q < 8; ++q) acc += lt[q] * zj[q];
            }
            acc += __shfl_xor_sync(0xffffffffu, acc, 1);
            acc += __shfl_xor_sync(0xffffffffu, acc, 2);
            if ((t & 3) == 0) accs[r] = zs[R * NB + r] - acc;
            __syncthreads();
            const T* tt = stage(st, 0) + r * NB + c0;
            T s = T(0);
#pragma unroll
            for (int q = 0; q < 8; ++q) s += tt[q] * accs[c0 + q];
            s += __shfl_xor_sync(0xffffffffu, s, 1);
            s += __shfl_xor_sync(0xffffffffu, s, 2);
            if ((t & 3) == 0) zs[R * NB + r] = s;
        }
    }
    cp_async_wait_n<0>();
    __syncthreads();
    for (int k = 0; k < NST - 1; ++k) issue(k, K - 1 - k, false);
    for (int e = t; e < K * NB; e += S1T) zs[e] *= dinv[roff + e];
    // backward: x_R = T_R^T (D_R^{-1} z_R - sum_{I>R} L_IR^T x_I); thread
    // (column = lane, rows k0..k0+7 of the tile), warps combined in shared memory
    {
        const int lane = t & 31, warp = t >> 5, k0 = warp * 8;
        for (int R = K - 1, it = 0; R >= 0; --R, ++it) {
            const int st = it % NST;
            cp_async_wait_n<NST - 2>();
            __syncthreads();
            issue((it + NST - 1) % NST, R - (NST - 1), false);
            T s = T(0);
#pragma unroll
            for (int d = 1; d <= KBP; ++d) {
                if (d > kb || R + d >= K) continue;
                const T* lt = stage(st, d) + k0 * NB + lane;
                const T* xi = zs + (R + d) * NB + k0;
#pragma unroll
                for (int q = 0; q < 8; ++q) s += lt[q * NB] * xi[q];
            }
            part[warp][lane] = s;
            __syncthreads();
            if (warp == 0) {
                T v = T(0);
#pragma unroll
                for (int w = 0; w < S1T / 32; ++w) v += part[w][lane];
                accs[lane] = zs[R * NB + lane] - v;
            }
            __syncthreads();
            const T* tt = stage(st, 0) + k0 * NB + lane;
            T s2 = T(0);
#pragma unroll
            for (int q = 0; q < 8; ++q) s2 += tt[q * NB] * accs[k0 + q];
            part[warp][lane] = s2;
            __syncthreads();
            if (warp == 0) {
                T v = T(0);
#pragma unroll
                for (int w = 0; w < S1T / 32; ++w) v += part[w][lane];
                zs[R * NB + lane] = v;
            }
        }
    }
    cp_async_wait_n<0>();
    __syncthreads();
    for (int e = t; e < K * NB; e += S1T) X[roff + e] = to_f64(zs[e]);
}

// One right-hand side, any kb (dense coarse matrices): tiles are read as
// needed without prefetch; same thread mappings as above.
template <typename T>
__global__ void __launch_bounds__(S1T) k_tile_solve1_dense(
    const T* __restrict__ tiles, const T* __restrict__ dinv, const int* __restrict__ kb_, const int* __restrict__ K_,
    const long long* __restrict__ toff_, const long long* __restrict__ roff_, double* __restrict__ X,
    const int* __restrict__ gdone)
{
    extern __shared__ double zs[];
    __shared__ double accs[NB];
    __shared__ double part[S1T / 32][NB + 1];
    if (gdone && *gdone) return;
    const int i = blockIdx.x;
    const int kb = kb_[i], K = K_[i];
    const long long toff = toff_[i], roff = roff_[i];
    const int t = threadIdx.x;
    for (int e = t; e < K * NB; e += S1T) zs[e] = X[roff + e];
    __syncthreads();
    {
        const int r = t >> 2, c0 = (t & 3) * 8;
        for (int R = 0; R < K; ++R) {
            double acc = 0.0;
            for (int J = (R - kb > 0 ? R - kb : 0); J < R; ++J) {
                const T* src = tiles + tile_index(toff, kb, R, J) + r * NB + c0;
                const double* zj = zs + J * NB + c0;
#pragma unroll
                for (int q = 0; q < 8; ++q) acc += (double)src[q] * zj[q];
            }
            acc += __shfl_xor_sync(0xffffffffu, acc, 1);
            acc += __shfl_xor_sync(0xffffffffu, acc, 2);
            if ((t & 3) == 0) accs[r] = zs[R * NB + r] - acc;
            __syncthreads();
            const T* tr = tiles + tile_index(toff, kb, R, R) + r * NB + c0;
            double s = 0.0;
#pragma unroll
            for (int q = 0; q < 8; ++q) s += (double)tr[q] * accs[c0 + q];
            s += __shfl_xor_sync(0xffffffffu, s, 1);
            s += __shfl_xor_sync(0xffffffffu, s, 2);
            if ((t & 3) == 0) zs[R * NB + r] = s;
            __syncthreads();
        }
    }
    for (int e = t; e < K * NB; e += S1T) zs[e] *= (double)dinv[roff + e];
    __syncthreads();
    {
        const int lane = t & 31, warp = t >> 5, k0 = warp * 8;
        for (int R = K - 1; R >= 0; --R) {
            double s = 0.0;
            const int Imax = R + kb < K - 1 ? R + kb : K - 1;
            for (int I = R + 1; I <= Imax; ++I) {
                const T* src = tiles + tile_index(toff, kb, I, R);
                const double* xi = zs + I * NB + k0;
#pragma unroll
                for (int q = 0; q < 8; ++q) s += (double)src[(k0 + q) * NB + lane] * xi[q];
            }
            part[warp][lane] = s;
            __syncthreads();
            if (warp == 0) {
                double v = 0.0;
#pragma unroll
                for (int w = 0; w < S1T / 32; ++w) v += part[w][lane];
                accs[lane] = zs[R * NB + lane] - v;
            }
            __syncthreads();
            const T* tr = tiles + tile_index(toff, kb, R, R);
            double s2 = 0.0;
#pragma unroll
            for (int q = 0; q < 8; ++q) s2 += (double)tr[(k0 + q) * NB + lane] * accs[k0 + q];
            part[warp][lane] = s2;
            __syncthreads();
            if (warp == 0) {
                double v = 0.0;
#pragma unroll
                for (int w = 0; w < S1T / 32; ++w) v += part[w][lane];
                zs[R * NB + lane] = v;
            }
            __syncthreads();
        }
    }
    for (int e = t; e < K * NB; e += S1T) X[roff + e] = zs[e];
}


// ------------------------------------------------------------------ solve, several right-hand sides, band
// For kb <= 2, one 64-thread CTA per problem.  Step R needs the diagonal
// tile, the kb off-diagonal tiles of block row (forward) or block column
// (backward) R, the 32 x ncols block R of X and D_R^{-1}; these are copied
// into shared memory with cp.async BAND_STAGES - 1 steps ahead.  The last kb
// solution blocks stay in a shared ring.  Thread t owns the register block
// rows 4 (t >> 3) + i, i < 4, columns CPT (t & 7) + j, j < CPT.
//
// Tiles are stored in shared memory as 32 x 32 with the 4-element groups of
// a row permuted: group g of row r sits at position g ^ ((r >> 2) & 7).  The
// four rows 4 rg + i a warp reads together for one group (forward), and the
// four groups rg of one row (backward), then fall in distinct banks.
constexpr int BAND_STAGES = 3;
constexpr int BAND_SLOTS = 3;      // diagonal tile + at most 2 off-diagonal tiles per step

__device__ __forceinline__ int band_swz(int row) { return (row >> 2) & 7; }

// copy one 32 x 32 tile (row-major in global memory) into the permuted layout
template <typename T, int NT>
__device__ __forceinline__ void band_async_tile(T* dst, const T* __restrict__ src) {
    constexpr int PER = 16 / (int)sizeof(T);           // elements per 16-byte chunk
    for (int ch = threadIdx.x; ch < NB2 / PER; ch += NT) {
        const int e = ch * PER, r = e / NB, c = e % NB;
        const int g = c >> 2, within = c & 3;
        cp_async16(dst + r * NB + ((g ^ band_swz(r)) << 2) + within, src + e);
    }
}

// four consecutive elements of a permuted tile: row r, group g
template <typename T>
__device__ __forceinline__ void band_load4(const T* tile, int r, int g, T (&v)[4]);
template <>
__device__ __forceinline__ void band_load4<float>(const float* tile, int r, int g, float (&v)[4]) {
    const float4 x = *reinterpret_cast<const float4*>(tile + r * NB + ((g ^ band_swz(r)) << 2));
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
}
template <>
__device__ __forceinline__ void band_load4<double>(const double* tile, int r, int g, double (&v)[4]) {
    const double2* p = reinterpret_cast<const double2*>(tile + r * NB + ((g ^ band_swz(r)) << 2));
    const double2 a = p[0], b = p[1];
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

template <typename T, int CPT, int CG>
struct BandSmem {
    static constexpr int ZLD = CG * CPT;                // columns held in the ring and Acc
    static size_t bytes(int sxld) {
        return sizeof(T) * ((size_t)BAND_STAGES * BAND_SLOTS * NB2 + (size_t)BAND_STAGES * NB + (size_t)(BAND_SLOTS + 1) * NB * ZLD) +
               sizeof(double) * (size_t)BAND_STAGES * NB * sxld;
    }
};

template <typename T, int CPT, int CG>
__global__ void __launch_bounds__(8 * CG) k_tile_solve_band(
    const T* __restrict__ tiles, const T* __restrict__ dinv, const int* __restrict__ kb_, const int* __restrict__ K_,
    const long long* __restrict__ toff_, const long long* __restrict__ roff_, double* __restrict__ Xall, int ldx,
    int ncols_all, const int* __restrict__ skip, const int* __restrict__ gdone)
{
    // blockIdx.y selects a chunk of ZLD columns (an independent set of
    // right-hand sides solved by its own CTA)
    constexpr int NST = BAND_STAGES, ZLD = BandSmem<T, CPT, CG>::ZLD, NT = 8 * CG;
    const int cbase = blockIdx.y * ZLD;
    const int ncols = min(ZLD, ncols_all - cbase);
    double* __restrict__ X = Xall + cbase;
    const int sxld = ((ncols + 1) / 2) * 2;             // staged columns of X (whole 16-byte chunks)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* St = reinterpret_cast<T*>(smem_raw);                                   // [NST][SLOTS][32*32]
    T* Sd = St + (size_t)NST * BAND_SLOTS * NB2;                              // [NST][32]   D^{-1}
    T* Zr = Sd + (size_t)NST * NB;                                            // [SLOTS][32][ZLD]
    T* Acc = Zr + (size_t)BAND_SLOTS * NB * ZLD;                              // [32][ZLD]
    double* Sx = reinterpret_cast<double*>(Acc + (size_t)NB * ZLD);           // [NST][32][sxld]
    const int i = blockIdx.x;
    if (skip && skip[i]) return;
    if (gdone && *gdone) return;
    const int kb = kb_[i], K = K_[i];
    const long long toff = toff_[i], roff = roff_[i];
    const int t = threadIdx.x;
    const int rg = t / CG, cg = t % CG, warp = t >> 5;
    const int r0 = 4 * rg, c0 = CPT * cg;
    // rows of this warp: 4 * (32 warp / CG) ... 4 * ((32 warp + 31) / CG) + 3
    const int wrow_lo = 4 * ((32 * warp) / CG), wgrp_hi = (32 * warp + 31) / CG;
    auto stile = [&](int st, int slot) { return St + (size_t)(st * BAND_SLOTS + slot) * NB2; };
    auto issue = [&](int st, int R, bool fwd) {
        if (R >= 0 && R < K) {
            band_async_tile<T, NT>(stile(st, 0), tiles + tile_index(toff, kb, R, R));
            for (int d = 1; d <= kb; ++d) {
                const int o = fwd ? R - d : R + d;
                if (o < 0 || o >= K) continue;
                band_async_tile<T, NT>(stile(st, d), tiles + (fwd ? tile_index(toff, kb, R, o) : tile_index(toff, kb, o, R)));
            }
            if (!fwd) {
                constexpr int PER = 16 / (int)sizeof(T);
                for (int ch = t; ch < NB / PER; ch += NT)
                    cp_async16(Sd + st * NB + ch * PER, dinv + roff + (long long)R * NB + ch * PER);
            }
            const int cpr = sxld / 2;                    // 16-byte chunks per row
            const double* src = X + (roff + (long long)R * NB) * ldx;
            double* dst = Sx + (size_t)st * NB * sxld;
            for (int ch = t; ch < NB * cpr; ch += NT) {
                const int r = ch / cpr, c = (ch % cpr) * 2;
                cp_async16(dst + r * sxld + c, src + (long long)r * ldx + c);
            }
        }
        cp_async_commit();
    };
    auto finish = [&](T (&acc)[4][CPT], int R, const T* Tt, bool fwd) {
        // Acc <- acc; out = T_R acc (forward) or T_R^T acc (backward)
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int j = 0; j < CPT; ++j) Acc[(r0 + a) * ZLD + c0 + j] = acc[a][j];
        __syncthreads();
        T out[4][CPT];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int j = 0; j < CPT; ++j) out[a][j] = T(0);
        if (fwd) {
            // T_R is lower triangular with zeros above the diagonal: the
            // groups up to the warp's last row suffice
            const int gmax = wgrp_hi + 1;
#pragma unroll 4
            for (int g = 0; g < gmax; ++g) {
                T l[4][4];
#pragma unroll
                for (int a = 0; a < 4; ++a) band_load4<T>(Tt, r0 + a, g, l[a]);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const T* z = Acc + (4 * g + kk) * ZLD + c0;
#pragma unroll
                    for (int j = 0; j < CPT; ++j) {
                        const T zv = z[j];
#pragma unroll
                        for (int a = 0; a < 4; ++a) out[a][j] += l[a][kk] * zv;
                    }
                }
            }
        } else {
#pragma unroll 4
            for (int k = wrow_lo; k < NB; ++k) {
                T l[4];
                band_load4<T>(Tt, k, rg, l);
                const T* z = Acc + k * ZLD + c0;
#pragma unroll
                for (int j = 0; j < CPT; ++j) {
                    const T zv = z[j];
#pragma unroll
                    for (int a = 0; a < 4; ++a) out[a][j] += l[a] * zv;
                }
            }
        }
        T* Zw = Zr + (size_t)(R % BAND_SLOTS) * NB * ZLD;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            double* xw = X + (roff + (long long)R * NB + r0 + a) * ldx;
#pragma unroll
            for (int j = 0; j < CPT; ++j) {
                Zw[(r0 + a) * ZLD + c0 + j] = out[a][j];
                if (c0 + j < ncols) xw[c0 + j] = to_f64(out[a][j]);
            }
        }
    };

    // forward: z_R = T_R (x_R - sum_J L_RJ z_J)
    for (int k = 0; k < NST - 1; ++k) issue(k, k, true);
    for (int R = 0; R < K; ++R) {
        const int st = R % NST;
        cp_async_wait_n<NST - 2>();
        __syncthreads();
        issue((R + NST - 1) % NST, R + NST - 1, true);
        T acc[4][CPT];
        const double* xs = Sx + (size_t)st * NB * sxld;
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int j = 0; j < CPT; ++j) acc[a][j] = (c0 + j < ncols) ? from_f64<T>(xs[(r0 + a) * sxld + c0 + j]) : T(0);
        for (int d = 1; d <= kb; ++d) {
            if (R - d < 0) break;
            const T* L = stile(st, d);
            const T* Z = Zr + (size_t)((R - d) % BAND_SLOTS) * NB * ZLD;
#pragma unroll
            for (int g = 0; g < NB / 4; ++g) {
                T l[4][4];
#pragma unroll
                for (int a = 0; a < 4; ++a) band_load4<T>(L, r0 + a, g, l[a]);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const T* z = Z + (4 * g + kk) * ZLD + c0;
#pragma unroll
                    for (int j = 0; j < CPT; ++j) {
                        const T zv = z[j];
#pragma unroll
                        for (int a = 0; a < 4; ++a) acc[a][j] -= l[a][kk] * zv;
                    }
                }
            }
        }
        finish(acc, R, stile(st, 0), true);
    }
    cp_async_wait_n<0>();
    __syncthreads();
    // backward: x_R = T_R^T (D_R^{-1} z_R - sum_I L_IR^T x_I)
    for (int k = 0; k < NST - 1; ++k) issue(k, K - 1 - k, false);
    for (int R = K - 1, it = 0; R >= 0; --R, ++it) {
        const int st = it % NST;
        cp_async_wait_n<NST - 2>();
        __syncthreads();
        issue((it + NST - 1) % NST, R - (NST - 1), false);
        T acc[4][CPT];
        const double* xs = Sx + (size_t)st * NB * sxld;
        const T* dv = Sd + st * NB;
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int j = 0; j < CPT; ++j)
                acc[a][j] = (c0 + j < ncols) ? dv[r0 + a] * from_f64<T>(xs[(r0 + a) * sxld + c0 + j]) : T(0);
        for (int d = 1; d <= kb; ++d) {
            if (R + d >= K) break;
            const T* L = stile(st, d);
            const T* Z = Zr + (size_t)((R + d) % BAND_SLOTS) * NB * ZLD;
#pragma unroll 8
            for (int k = 0; k < NB; ++k) {
                T l[4];
                band_load4<T>(L, k, rg, l);
                const T* z = Z + k * ZLD + c0;
#pragma unroll
                for (int j = 0; j < CPT; ++j) {
                    const T zv = z[j];
#pragma unroll
                    for (int a = 0; a < 4; ++a) acc[a][j] -= l[a] * zv;
                }
            }
        }
        finish(acc, R, stile(st, 0), false);
    }
    cp_async_wait_n<0>();
}

// ---- TMA / mbarrier helpers of the FP32 band solve.  Every mbarrier wait is
// bounded; a kernel whose wait runs out records it in g_wait_timeouts.
__device__ int g_wait_timeouts;

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
constexpr long long kWaitTries = 1LL << 22;
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity) {
    for (long long k = 0; k < kWaitTries; ++k)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void tma_load_tile(void* dst, const CUtensorMap* map, int row, unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
            smem_u32(dst)),
        "l"(map), "r"(0), "r"(row), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }

// ---- FP32 band LDL^T with the panel updates on the tensor cores (3 <= kb <= 12)
// Left-looking by tile column C, one CTA (one warpgroup) per matrix.  The
// update of column C,
//   U_R = sum_{J} L_RJ D_J L_CJ^T,  R = C .. min(C + kb, K - 1),
//   J = max(C - kb, R - kb) .. C - 1,
// is a product D = A B^T with A = [L_RJ] (tile rows R stacked, 128-row
// blocks of four tile rows, tiles outside the band zero) and
// B = [L_CJ D_J] (32 x 32 per J), done by tcgen05.mma kind::tf32 into a
// TMEM accumulator (four 128 x 32 FP32 blocks).  FP32 accuracy from TF32
// operands by the three-product split x = hi + lo, hi = x with the low 13
// mantissa bits cleared: A_hi B_hi + A_hi B_lo + A_lo B_hi (the lo * lo
// term is below FP32 rounding).  The tensor cores of this GPU take a
// kind::tf32 operand as its top 19 bits (truncation, measured), so the FP32
// L tiles themselves serve as hi parts, and lo = x - hi of each L tile is
// written once, when the tile is computed, to a scratch array.  The A
// operands (hi from the tiles, lo from the scratch) are streamed by TMA
// (3-stage ring, one pair (block, J) per stage, tiles outside the band read
// as zeros from out-of-range coordinates); the B operands are scaled by D_J
// and split in shared memory.  Then, as in
// k_tile_factor: W_RC = A_RC - U_R, the diagonal tile is factored and
// inverted by warp 0 in registers (null pivots as there), and
// L_RC = W_RC T_C^T D_C^{-1}.  Operands are K-major with the 128-byte
// swizzle (row r of a tile at 128 r bytes, 16-byte chunk g at g ^ (r & 7)),
// descriptors: start >> 4, stride between 8-row groups 1024 B, the K step
// of 8 elements advances the start by 32 B.
constexpr int TF_NT = 128, TF_KBM = 12, TF_NS = 3;
constexpr int TF_MAXPAIRS = TF_KBM * ((TF_KBM + 1 + 3) / 4);
constexpr size_t tf_smem_bytes() {
    return 1024 + (size_t)TF_NS * 8 * NB2 * 4            // A stages: 4 hi + 4 lo tiles
           + (size_t)TF_KBM * 2 * NB2 * 4                // B_J hi and lo
           + (size_t)NB2 * 4 + NB * 4                    // T_C, D_C^{-1}
           + (size_t)TF_KBM * NB * 4                     // D_J of the B operands
           + 64 * (TF_NS * 2 + 3) + TF_MAXPAIRS * 4 + 64;
}

__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xffffe000u); }

__device__ __forceinline__ uint64_t umma_desc_sw128(unsigned saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);          // start address
    d |= (uint64_t)1 << 16;                             // leading byte offset (unused: K-major, 128 B rows)
    d |= (uint64_t)(1024 >> 4) << 32;                   // stride byte offset: 8 rows x 128 B
    d |= (uint64_t)1 << 46;                             // descriptor version
    d |= (uint64_t)2 << 61;                             // 128-byte swizzle
    return d;
}
__device__ __forceinline__ void umma_tf32(unsigned tmem, uint64_t a, uint64_t b, unsigned idesc, unsigned acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void umma_commit(unsigned long long* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tmem_ld32(unsigned taddr, float (&v)[32]) {
    unsigned r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
        "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int k = 0; k < 32; ++k) v[k] = __uint_as_float(r[k]);
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;\n" ::: "memory"); }

// lo: E floats (E = total tile elements), lo parts of the L tiles in the tile layout;
// tm_hi / tm_lo: [E / 32][32] tensor maps of the tiles and of lo
__global__ void __launch_bounds__(TF_NT) k_tile_factor_tc(
    const __grid_constant__ CUtensorMap tm_hi, const __grid_constant__ CUtensorMap tm_lo, float* __restrict__ tiles,
    float* __restrict__ lo, long long total_elems, float* __restrict__ dinv, const int* __restrict__ n_, const int* __restrict__ kb_,
    const int* __restrict__ K_, const long long* __restrict__ toff_, const long long* __restrict__ roff_,
    int* __restrict__ status, int* __restrict__ nreg, double reg_tol)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
    float* Ast = reinterpret_cast<float*>(base);                                   // [NS][8][1024]
    float* Bst = Ast + (size_t)TF_NS * 8 * NB2;                                     // [KBM][2][1024]
    float* Tc = Bst + (size_t)TF_KBM * 2 * NB2;                                     // [32][32]
    float* Dc = Tc + NB2;                                                           // [32]
    float* Dj = Dc + NB;                                                            // [KBM][32]
    unsigned long long* bars = reinterpret_cast<unsigned long long*>(Dj + TF_KBM * NB);  // full[NS], empty[NS], acc, b
    unsigned long long* full = bars;
    unsigned long long* empty = bars + TF_NS;
    unsigned long long* accb = bars + 2 * TF_NS;
    unsigned long long* bfull = bars + 2 * TF_NS + 1;
    int* pairs = reinterpret_cast<int*>(bars + 2 * TF_NS + 3);                     // (J << 8) | mb
    __shared__ unsigned s_tmem;
    __shared__ int s_status, s_nreg, s_abort, s_npairs, s_used;

    const int i = blockIdx.x;
    const int n = n_[i], kb = kb_[i], K = K_[i];
    const long long toff = toff_[i], roff = roff_[i];
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    if (kb > TF_KBM) {                                  // never launched so (host dispatch)
        if (t == 0) status[i] = -1;
        return;
    }
    const int oob_row = (int)(total_elems / NB);        // first row beyond both tensors: zero fill
    if (t == 0) {
        s_status = 0; s_nreg = 0; s_abort = 0;
        for (int s = 0; s < TF_NS; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        mbar_init(accb, 1);
        mbar_init(bfull, 1);
        fence_mbar_init();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;\n" ::"r"(smem_u32(&s_tmem)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = s_tmem;
    // D f32, A and B tf32, both K-major, N = 32, M = 128
    const unsigned idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);
    // parity bits: ph_full (product thread), ph_empty and par_issued (copy
    // thread), ph_acc (all threads); pair_base counts the ring's pairs so far
    unsigned ph_full = 0, ph_empty = 0, ph_acc = 0, par_issued = 0, ph_b = 0;
    int pair_base = 0;

    auto issue_pair = [&](int C, int Rend, int pr, int stage) {
        // A operand tiles of pair (J, mb): hi into slots 0..3, lo into 4..7
        const int J = pr >> 8, mb = pr & 0xff;
        float* dst = Ast + (size_t)stage * 8 * NB2;
        mbar_expect_tx(&full[stage], 8 * NB2 * 4);
        for (int q = 0; q < 4; ++q) {
            const int R = C + 4 * mb + q;
            const bool valid = R <= Rend && R - J <= kb;
            const long long ti = valid ? tile_index(toff, kb, R, J) : 0;
            const int row = valid ? (int)(ti / NB) : oob_row;
            tma_load_tile(dst + (size_t)q * NB2, &tm_hi, row, &full[stage]);
            tma_load_tile(dst + (size_t)(4 + q) * NB2, &tm_lo, row, &full[stage]);
        }
    };

    for (int C = 0; C < K && !s_abort; ++C) {
        const int Rend = min(C + kb, K - 1);
        const int J0 = max(0, C - kb);
        const int nJ = C - J0;
        const int nmb = (Rend - C + 1 + 3) / 4;
        // ---- pair list and B operands: B_J[n][j] = L_CJ[n][j] * D_J[j], split
        if (t == 0) {
            int np = 0, used = 0;
            for (int J = J0; J < C; ++J)
                for (int mb = 0; mb < nmb; ++mb) {
                    const int R0 = C + 4 * mb;
                    if (R0 <= Rend && R0 - J <= kb) {       // the block's first row has the most J's
                        pairs[np++] = (J << 8) | mb;
                        used |= 1 << mb;
                    }
                }
            s_npairs = np;
            s_used = used;
        }
        // raw tiles L_CJ by TMA into the lo slots, D_J into shared memory
        if (t == 32 && nJ > 0) {
            mbar_expect_tx(bfull, nJ * NB2 * 4);
            for (int jj = 0; jj < nJ; ++jj)
                tma_load_tile(Bst + (size_t)(2 * jj + 1) * NB2, &tm_hi,
                              (int)(tile_index(toff, kb, C, J0 + jj) / NB), bfull);
        }
        for (int e = t; e < nJ * NB; e += TF_NT) {
            const float di = dinv[roff + (long long)J0 * NB + e];
            Dj[e] = di != 0.f ? 1.f / di : 0.f;
        }
        __syncthreads();
        if (nJ > 0) {
            if (!mbar_wait_bounded(bfull, ph_b & 1u)) {
                if (atomicExch(&s_abort, 1) == 0) atomicAdd(&g_wait_timeouts, 1);
            } else {
                ph_b ^= 1u;
            }
        }
        for (int e = t; e < nJ * NB2; e += TF_NT) {
            // element (r, c) of tile jj; the same swizzled position in both slots
            const int jj = e / NB2, w = e % NB2, r = w / NB, c = w % NB;
            const int sidx = r * NB + ((((c >> 2) ^ (r & 7))) << 2) + (c & 3);
            float* lo_slot = Bst + (size_t)(2 * jj + 1) * NB2;
            const float b = lo_slot[sidx] * Dj[jj * NB + c];
            const float hi = tf32_hi(b);
            Bst[(size_t)(2 * jj) * NB2 + sidx] = hi;
            lo_slot[sidx] = b - hi;
        }
        fence_proxy_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        const int np = s_npairs, used = s_used;
        // ---- tensor-core update: lane 0 of warp 1 streams the A operands into the
        // ring, lane 0 of warp 0 issues the products (each side waits only for
        // the other: "full" when a stage's copies landed, "empty" when the
        // products that read a stage are done)
        if (t == 32 && np > 0) {
            for (int p = 0; p < np; ++p) {
                const int g = pair_base + p, st = g % TF_NS;
                if (g >= TF_NS) {
                    if (!mbar_wait_bounded(&empty[st], (ph_empty >> st) & 1u)) {
                        if (atomicExch(&s_abort, 1) == 0) atomicAdd(&g_wait_timeouts, 1);
                        break;
                    }
                    ph_empty ^= 1u << st;
                }
                if (*(volatile int*)&s_abort) break;
                issue_pair(C, Rend, pairs[p], st);
                par_issued = (par_issued & ~(1u << st)) | ((unsigned)((g / TF_NS) & 1) << st);
            }
        }
        if (t == 0 && np > 0) {
            unsigned started = 0;                       // M-blocks whose accumulator has been started
            for (int p = 0; p < np; ++p) {
                const int g = pair_base + p, st = g % TF_NS;
                if (!mbar_wait_bounded(&full[st], (ph_full >> st) & 1u)) {
                    if (atomicExch(&s_abort, 1) == 0) atomicAdd(&g_wait_timeouts, 1);
                    break;
                }
                ph_full ^= 1u << st;
                tc_fence_after();
                const int J = pairs[p] >> 8, mb = pairs[p] & 0xff, jj = J - J0;
                const unsigned a_hi = smem_u32(Ast + (size_t)st * 8 * NB2), a_lo = a_hi + 4 * NB2 * 4;
                const unsigned b_hi = smem_u32(Bst + (size_t)(2 * jj) * NB2), b_lo = b_hi + NB2 * 4;
                const unsigned d = tmem + 32u * mb;
                for (int k = 0; k < 4; ++k) {
                    const unsigned ko = 32u * k;
                    const unsigned acc = (started >> mb) & 1u;
                    umma_tf32(d, umma_desc_sw128(a_hi + ko), umma_desc_sw128(b_hi + ko), idesc, acc);
                    started |= 1u << mb;
                    umma_tf32(d, umma_desc_sw128(a_hi + ko), umma_desc_sw128(b_lo + ko), idesc, 1u);
                    umma_tf32(d, umma_desc_sw128(a_lo + ko), umma_desc_sw128(b_hi + ko), idesc, 1u);
                }
                umma_commit(&empty[st]);                // the stage is free once these products are done
            }
            umma_commit(accb);
        }
        pair_base += np;
        __syncthreads();
        if (s_abort) break;
        // ---- W_RC = A_RC - U_R for the rows of this thread: tile row C + 4 mb + warp, row lane
        if (np > 0) {
            if (!mbar_wait_bounded(accb, ph_acc & 1u)) {
                if (atomicExch(&s_abort, 1) == 0) atomicAdd(&g_wait_timeouts, 1);
            } else {
                ph_acc ^= 1u;                           // (on a timeout the phase stays pending)
            }
        }
        tc_fence_after();
        __syncthreads();
        if (s_abort) break;
        float w[4][NB];
#pragma unroll
        for (int mb = 0; mb < 4; ++mb) {
            const int R = C + 4 * mb + warp;
            if (mb < nmb && ((used >> mb) & 1)) {
                float u[NB];
                tmem_ld32(tmem + ((unsigned)(32 * warp) << 16) + 32u * mb, u);
                if (R <= Rend) {
                    const float* a = tiles + tile_index(toff, kb, R, C) + lane * NB;
#pragma unroll
                    for (int c = 0; c < NB; ++c) w[mb][c] = a[c] - u[c];
                }
            } else if (mb < nmb && R <= Rend) {
                const float* a = tiles + tile_index(toff, kb, R, C) + lane * NB;
#pragma unroll
                for (int c = 0; c < NB; ++c) w[mb][c] = a[c];
            }
        }
        tc_fence_before();
        // ---- diagonal tile (warp 0, mb 0: R = C): L D L^T in registers, T_C = L_CC^{-1}
        if (warp == 0) {
            const int rows_valid = n - C * NB;
            // original diagonal entry of this row (null-pivot reference)
            const float od_l = tiles[tile_index(toff, kb, C, C) + lane * NB + lane];
            float row[NB];
#pragma unroll
            for (int b = 0; b < NB; ++b) row[b] = w[0][b];
            float dl = 0.f;
            int nr = 0, stc = 0;
#pragma unroll
            for (int k = 0; k < NB; ++k) {
                const float d = __shfl_sync(0xffffffffu, row[k], k);
                const float odk = __shfl_sync(0xffffffffu, od_l, k);
                float dinv_k;
                if (k >= rows_valid) {
                    dinv_k = 1.f;
                } else if (reg_tol > 0.0 && !(d > (float)reg_tol * odk)) {
                    dinv_k = 0.f;
                    ++nr;
                } else if (!(d > 0.f)) {
                    dinv_k = 0.f;
                    if (stc == 0) stc = C * NB + k + 1;
                } else {
                    dinv_k = 1.f / d;
                }
                if (lane == k) dl = dinv_k;
                const float wak = row[k];
#pragma unroll
                for (int b = 0; b < NB; ++b) {
                    if (b > k) {
                        const float wbk = __shfl_sync(0xffffffffu, wak, b);
                        if (lane >= b) row[b] -= wak * wbk * dinv_k;
                    }
                }
                if (lane > k) row[k] = (k >= rows_valid || lane >= rows_valid) ? 0.f : wak * dinv_k;
            }
            float tr[NB];
#pragma unroll
            for (int b = 0; b < NB; ++b) tr[b] = (b == lane) ? 1.f : 0.f;
#pragma unroll
            for (int k = 0; k < NB - 1; ++k) {
                const float lak = row[k];
#pragma unroll
                for (int b = 0; b < NB; ++b) {
                    if (b <= k) {
                        const float tkb = __shfl_sync(0xffffffffu, tr[b], k);
                        if (lane > k) tr[b] -= lak * tkb;
                    }
                }
            }
            float* dst = tiles + tile_index(toff, kb, C, C) + lane * NB;
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                Tc[lane * NB + b] = tr[b];
                dst[b] = tr[b];
            }
            Dc[lane] = dl;
            dinv[roff + (long long)C * NB + lane] = dl;
            if (lane == 0) {
                s_nreg += nr;
                if (s_status == 0 && stc != 0) s_status = stc;
            }
        }
        __syncthreads();
        // ---- panel: L_RC = W_RC T_C^T D_C^{-1}, stored with its hi / lo parts for later columns
#pragma unroll
        for (int mb = 0; mb < 4; ++mb) {
            const int R = C + 4 * mb + warp;
            if (mb >= nmb || R <= C || R > Rend) continue;
            float out[NB];
#pragma unroll
            for (int c = 0; c < NB; ++c) {
                float s = 0.f;
#pragma unroll
                for (int g = 0; g < NB / 4; ++g) {
                    const float4 tv = *reinterpret_cast<const float4*>(Tc + c * NB + 4 * g);
                    s += w[mb][4 * g] * tv.x;
                    s += w[mb][4 * g + 1] * tv.y;
                    s += w[mb][4 * g + 2] * tv.z;
                    s += w[mb][4 * g + 3] * tv.w;
                }
                out[c] = s * Dc[c];
            }
            const long long ti = tile_index(toff, kb, R, C) + lane * NB;
#pragma unroll
            for (int c = 0; c < NB; ++c) {
                tiles[ti + c] = out[c];
                lo[ti + c] = out[c] - tf32_hi(out[c]);
            }
        }
        fence_proxy_async_global();                     // the next columns read these by TMA
        __syncthreads();
    }
    // ---- end: wait (bounded) for copies and products still in flight, free TMEM
    if (s_abort) {
        // copies still in flight land, and the products issued complete, before the CTA exits
        if (t == 32)
            for (int s = 0; s < TF_NS && s < pair_base; ++s) mbar_wait_bounded(&full[s], (par_issued >> s) & 1u);
        if (t == 0) mbar_wait_bounded(accb, ph_acc & 1u);  // a column's products, if their wait gave up
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;\n" ::"r"(tmem));
    if (t == 0) { status[i] = s_status; nreg[i] = s_nreg; }
}

// ---- the FP32 band solve with TMA tile loads, warp-specialised (kb <= 2)
// The steps and expressions of k_tile_solve_band<float> (forward z_R = T_R
// (x_R - sum_J L_RJ z_J), backward x_R = T_R^T (D_R^{-1} z_R - sum_I L_IR^T
// x_I), products summed in the same order), arranged so that no block
// barrier sits on the sweeps' chain: each
// of W consumer warps owns C right-hand-side columns and all 32 rows of a
// tile row (lane = row), so a step's data exchange is warp-internal
// (__syncwarp); a producer warp streams the tiles of each step and D^{-1}
// with TMA into an NST-stage ring ("full" mbarriers completed by the copies'
// byte counts, "empty" mbarriers released by each consumer warp after its
// last read of the stage).  Each lane prefetches its own row of the
// right-hand sides with cp.async, XD steps ahead.  Column k of tile
// L_{R,R-d} can be nonzero only where 32 d + r - k <= b (the band), so the
// forward products start at k = 32 d - b and the backward ones stop at
// k = b - 32 d + 31.  Every wait is bounded; on a timeout the CTA records it
// (g_wait_timeouts), the producer waits (bounded) for the copies it still
// has in flight, and the CTA returns.
template <int C>
__device__ __forceinline__ void ws_ld(const float* p, float (&v)[C]) {
    if constexpr (C == 4) {
        const float4 x = *reinterpret_cast<const float4*>(p);
        v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
    } else if constexpr (C == 2) {
        const float2 x = *reinterpret_cast<const float2*>(p);
        v[0] = x.x; v[1] = x.y;
    } else {
        v[0] = *p;
    }
}
template <int C>
__device__ __forceinline__ void ws_st(float* p, const float (&v)[C]) {
    if constexpr (C == 4) *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    else if constexpr (C == 2) *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
    else *p = v[0];
}
// element (row, col) of a 128-byte-swizzled 32 x 32 FP32 tile
__device__ __forceinline__ int swz(int row, int col) { return row * NB + ((((col >> 2) ^ (row & 7))) << 2) + (col & 3); }

// acc[c] += SIGN * sum_{K0 <= k < K1} tile[lane][k] V[k][c]  (row access of a
// swizzled tile; V: [32][C] floats, read by broadcast).  Fully unrolled so
// that all loads issue ahead of the products.
template <int C, int K0, int K1, int SIGN>
__device__ __forceinline__ void ws_row_product(const float* tile, const float* V, int lane, float (&acc)[C]) {
    float l[K1 - K0];
#pragma unroll
    for (int g = K0 / 4; g < K1 / 4; ++g) {
        const float4 x = *reinterpret_cast<const float4*>(tile + lane * NB + ((g ^ (lane & 7)) << 2));
        l[4 * g - K0] = x.x; l[4 * g - K0 + 1] = x.y; l[4 * g - K0 + 2] = x.z; l[4 * g - K0 + 3] = x.w;
    }
#pragma unroll
    for (int k = K0; k < K1; ++k) {
        float v[C];
        ws_ld<C>(V + k * C, v);
#pragma unroll
        for (int c = 0; c < C; ++c) {
            if (SIGN > 0) acc[c] += l[k - K0] * v[c];
            else acc[c] -= l[k - K0] * v[c];
        }
    }
}
// acc[c] += SIGN * sum_{0 <= k < K1} tile[k][lane] V[k][c]  (column access)
template <int C, int K1, int SIGN>
__device__ __forceinline__ void ws_col_product(const float* tile, const float* V, int lane, float (&acc)[C]) {
    float l[K1];
#pragma unroll
    for (int k = 0; k < K1; ++k) l[k] = tile[swz(k, lane)];
#pragma unroll
    for (int k = 0; k < K1; ++k) {
        float v[C];
        ws_ld<C>(V + k * C, v);
#pragma unroll
        for (int c = 0; c < C; ++c) {
            if (SIGN > 0) acc[c] += l[k] * v[c];
            else acc[c] -= l[k] * v[c];
        }
    }
}

// Wide-band forms of the two products: the loads are volatile shared
// loads issued eight k at a time ahead of their products (the compiler keeps
// their order), with two partial sums per column.  With 13 tiles a step the
// products dominate and this ordering is 2-12% faster; with 3 tiles the
// plain forms above are.
__device__ __forceinline__ float4 lds4_ordered(const float* p) {
    float4 r;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];\n"
                 : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
                 : "r"(smem_u32(p)));
    return r;
}
__device__ __forceinline__ float lds1_ordered(const float* p) {
    float r;
    asm volatile("ld.shared.f32 %0, [%1];\n" : "=f"(r) : "r"(smem_u32(p)));
    return r;
}
__device__ __forceinline__ float2 lds2_ordered(const float* p) {
    float2 r;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];\n" : "=f"(r.x), "=f"(r.y) : "r"(smem_u32(p)));
    return r;
}
template <int C>
__device__ __forceinline__ void ws_ld_ordered(const float* p, float (&v)[C]) {
    if constexpr (C == 4) {
        const float4 x = lds4_ordered(p);
        v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
    } else if constexpr (C == 2) {
        const float2 x = lds2_ordered(p);
        v[0] = x.x; v[1] = x.y;
    } else {
        ws_ld<C>(p, v);
    }
}
template <int C, int K0, int K1, int SIGN>
__device__ __forceinline__ void ws_row_product_wide(const float* tile, const float* V, int lane, float (&acc)[C]) {
    constexpr int NK = K1 - K0;
    static_assert(NK % 8 == 0, "k range in multiples of 8");
    float l[NK];
#pragma unroll
    for (int g = K0 / 4; g < K1 / 4; ++g) {
        const float4 x = lds4_ordered(tile + lane * NB + ((g ^ (lane & 7)) << 2));
        l[4 * g - K0] = x.x; l[4 * g - K0 + 1] = x.y; l[4 * g - K0 + 2] = x.z; l[4 * g - K0 + 3] = x.w;
    }
    float a0[C], a1[C];
#pragma unroll
    for (int c = 0; c < C; ++c) { a0[c] = acc[c]; a1[c] = 0.f; }
#pragma unroll
    for (int k8 = 0; k8 < NK; k8 += 8) {
        float v[8][C];
#pragma unroll
        for (int k = 0; k < 8; ++k) ws_ld_ordered<C>(V + (K0 + k8 + k) * C, v[k]);
#pragma unroll
        for (int k = 0; k < 8; k += 2)
#pragma unroll
            for (int c = 0; c < C; ++c) {
                if (SIGN > 0) { a0[c] += l[k8 + k] * v[k][c]; a1[c] += l[k8 + k + 1] * v[k + 1][c]; }
                else { a0[c] -= l[k8 + k] * v[k][c]; a1[c] -= l[k8 + k + 1] * v[k + 1][c]; }
            }
    }
#pragma unroll
    for (int c = 0; c < C; ++c) acc[c] = a0[c] + a1[c];
}
template <int C, int K1, int SIGN>
__device__ __forceinline__ void ws_col_product_wide(const float* tile, const float* V, int lane, float (&acc)[C]) {
    static_assert(K1 % 8 == 0, "k range in multiples of 8");
    float l[K1];
#pragma unroll
    for (int k = 0; k < K1; ++k) l[k] = lds1_ordered(tile + swz(k, lane));
    float a0[C], a1[C];
#pragma unroll
    for (int c = 0; c < C; ++c) { a0[c] = acc[c]; a1[c] = 0.f; }
#pragma unroll
    for (int k8 = 0; k8 < K1; k8 += 8) {
        float v[8][C];
#pragma unroll
        for (int k = 0; k < 8; ++k) ws_ld_ordered<C>(V + (k8 + k) * C, v[k]);
#pragma unroll
        for (int k = 0; k < 8; k += 2)
#pragma unroll
            for (int c = 0; c < C; ++c) {
                if (SIGN > 0) { a0[c] += l[k8 + k] * v[k][c]; a1[c] += l[k8 + k + 1] * v[k + 1][c]; }
                else { a0[c] -= l[k8 + k] * v[k][c]; a1[c] -= l[k8 + k + 1] * v[k + 1][c]; }
            }
    }
#pragma unroll
    for (int c = 0; c < C; ++c) acc[c] = a0[c] + a1[c];
}
// the form a configuration uses: ordered for wide bands (more than 2 tiles)
// with 2 or 4 columns a warp (the configurations that were measured)
template <bool WIDE, int C, int K0, int K1, int SIGN>
__device__ __forceinline__ void ws_rowp(const float* tile, const float* V, int lane, float (&acc)[C]) {
    if constexpr (WIDE) ws_row_product_wide<C, K0, K1, SIGN>(tile, V, lane, acc);
    else ws_row_product<C, K0, K1, SIGN>(tile, V, lane, acc);
}
template <bool WIDE, int C, int K1, int SIGN>
__device__ __forceinline__ void ws_colp(const float* tile, const float* V, int lane, float (&acc)[C]) {
    if constexpr (WIDE) ws_col_product_wide<C, K1, SIGN>(tile, V, lane, acc);
    else ws_col_product<C, K1, SIGN>(tile, V, lane, acc);
}

__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}

template <int KBP, int W, int C, int NST, int XD>
struct BandWs {
    // The backward sweep's first right-hand side read from X (block K-1-S,
    // written by forward step K-1-S) is issued XD - 1 steps ahead, at step
    // K - XD + 1: it must come after that write, so XD <= S + 1 = KBP + 2.
    static_assert(XD <= KBP + 2, "X prefetch deeper than the solution ring allows");
    static constexpr int SLOTS = KBP + 1;            // tiles per step; also the solution ring per warp
    static constexpr int NT = 32 * (W + 1);
    static constexpr int COLS = W * C;
    static constexpr size_t stage_bytes = (size_t)SLOTS * NB2 * sizeof(float);
    static constexpr size_t warp_bytes =
        sizeof(float) * ((size_t)SLOTS * NB * C + (size_t)NB * C) + sizeof(double) * (size_t)XD * NB * C;
    static constexpr size_t smem_bytes =
        1024 + (size_t)NST * stage_bytes + (size_t)NST * NB * sizeof(float) + 16 * (size_t)NST + (size_t)W * warp_bytes;
};

// Half-bandwidth b at most KBP tiles (kb <= KBP); a step needs the diagonal
// tile and kb off-diagonal tiles, and z_{R-1} .. z_{R-kb} (forward) or
// x_{R+1} .. x_{R+kb} (backward) from the warp's ring of KBP + 1 solution
// blocks.  When the backward sweep starts, the ring still holds z_R for the
// last KBP + 1 rows, so only the rows before those are read back from X.
template <int KBP, int W, int C, int NST, int XD>
__global__ void __launch_bounds__(32 * (W + 1)) k_tile_solve_band_ws(
    const __grid_constant__ CUtensorMap tmt, const float* __restrict__ dinv, const int* __restrict__ kb_,
    const int* __restrict__ K_, const int* __restrict__ b_, const long long* __restrict__ toff_,
    const long long* __restrict__ roff_, double* __restrict__ Xall, int ldx, int ncols_all,
    const int* __restrict__ skip, const int* __restrict__ gdone)
{
    using Cfg = BandWs<KBP, W, C, NST, XD>;
    constexpr int S = Cfg::SLOTS;
    static_assert(C == 1 || C == 2 || C == 4, "1, 2 or 4 columns per warp");
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
    float* St = reinterpret_cast<float*>(base);                                        // [NST][S][32*32]
    float* Sd = St + (size_t)NST * S * NB2;                                            // [NST][32]
    unsigned long long* full = reinterpret_cast<unsigned long long*>(Sd + (size_t)NST * NB);
    unsigned long long* empty = full + NST;
    unsigned char* wbase = reinterpret_cast<unsigned char*>(empty + NST);
    __shared__ int s_abort;

    const int i = blockIdx.x;
    if (skip && skip[i]) return;
    if (gdone && *gdone) return;
    const int kb = kb_[i], K = K_[i], bw = b_[i];
    if (kb > KBP) return;                            // never launched so (host dispatch)
    const long long toff = toff_[i], roff = roff_[i];
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    if (t == 0) {
        s_abort = 0;
        for (int s = 0; s < NST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], W);
        }
        fence_mbar_init();
    }
    __syncthreads();
    auto stile = [&](int st, int slot) { return St + (size_t)(st * S + slot) * NB2; };
    auto give_up = [&]() {
        if (atomicExch(&s_abort, 1) == 0) atomicAdd(&g_wait_timeouts, 1);
    };
    const int total = 2 * K;                         // steps of both sweeps

    if (warp == W) {
        // ---------------- producer: one lane issues every copy
        if (lane == 0) {
            unsigned pending = 0, par = 0;           // stages with copies in flight, their phase parity
            for (int it = 0; it < total; ++it) {
                const int st = it % NST;
                if (it >= NST) {
                    if (!mbar_wait_bounded(&empty[st], ((it / NST) - 1) & 1u)) { give_up(); break; }
                    pending &= ~(1u << st);
                }
                if (*(volatile int*)&s_abort) break;
                const bool fwd = it < K;
                const int R = fwd ? it : total - 1 - it;
                int nt = 1;
                for (int d = 1; d <= kb; ++d) {
                    const int o = fwd ? R - d : R + d;
                    if (o >= 0 && o < K) ++nt;
                }
                mbar_expect_tx(&full[st], nt * NB2 * 4 + (fwd ? 0 : NB * 4));
                tma_load_tile(stile(st, 0), &tmt, (int)(tile_index(toff, kb, R, R) / NB), &full[st]);
                for (int d = 1; d <= kb; ++d) {
                    const int o = fwd ? R - d : R + d;
                    if (o < 0 || o >= K) continue;
                    const long long ti = fwd ? tile_index(toff, kb, R, o) : tile_index(toff, kb, o, R);
                    tma_load_tile(stile(st, d), &tmt, (int)(ti / NB), &full[st]);
                }
                if (!fwd) bulk_load(Sd + st * NB, dinv + roff + (long long)R * NB, NB * 4, &full[st]);
                pending |= 1u << st;
                par = (par & ~(1u << st)) | (((unsigned)(it / NST) & 1u) << st);
            }
            // after an abort, copies still in flight must land before the CTA exits
            if (*(volatile int*)&s_abort)
                for (int s = 0; s < NST; ++s)
                    if (pending & (1u << s)) mbar_wait_bounded(&full[s], (par >> s) & 1u);
        }
        return;
    }

    // ---------------- consumer warp: columns [c_lo, c_lo + nc)
    const int c_lo = blockIdx.y * Cfg::COLS + warp * C;
    const int nc = max(0, min(C, ncols_all - c_lo));
    float* Zr = reinterpret_cast<float*>(wbase + (size_t)warp * Cfg::warp_bytes);     // [S][32][C]
    float* Acc = Zr + (size_t)S * NB * C;                                               // [32][C]
    double* Xs = reinterpret_cast<double*>(Acc + (size_t)NB * C);                      // [XD][32][C]
    double* X = Xall + c_lo;
    // loads of this lane's row: index q < K: forward step q (row q); q >= K:
    // backward row K - 1 - S - (q - K) (backward steps s >= S)
    const int nload = K + max(0, K - S);
    auto issue_load = [&](int q) {
        if (q < nload && nc > 0) {
            if (q >= K) __threadfence_block();       // rows written by this lane in the forward sweep
            const int R = q < K ? q : K - 1 - S - (q - K);
            const double* src = X + (roff + (long long)R * NB + lane) * ldx;
            double* dst = Xs + ((size_t)(q % XD) * NB + lane) * C;
            if constexpr (C == 1) {
                asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_u32(dst)), "l"(src));
            } else {
                cp_async16(dst, src);
                if (C == 4 && nc > 2) cp_async16(dst + 2, src + 2);
            }
        }
        cp_async_commit();
    };
    for (int q = 0; q < XD - 1; ++q) issue_load(q);
    int q_next = XD - 1, q_use = 0;
    for (int it = 0; it < total; ++it) {
        const int st = it % NST;
        const bool fwd = it < K;
        const int R = fwd ? it : total - 1 - it;
        float acc[C];
        // right-hand side of this step (own row)
        if (fwd || (it - K) >= S) {
            issue_load(q_next++);
            cp_async_wait_n<XD - 1>();
            const double* xs = Xs + ((size_t)(q_use % XD) * NB + lane) * C;
#pragma unroll
            for (int c = 0; c < C; ++c) acc[c] = c < nc ? f64_to_f32(xs[c]) : 0.f;
            ++q_use;
        } else {
            ws_ld<C>(Zr + ((size_t)(R % S) * NB + lane) * C, acc);
        }
        if (!mbar_wait_bounded(&full[st], (it / NST) & 1u)) { give_up(); break; }
        if (nc > 0) {
            if (!fwd) {
                const float dr = Sd[st * NB + lane];
#pragma unroll
                for (int c = 0; c < C; ++c) acc[c] *= dr;
            }
            for (int d = 1; d <= kb; ++d) {
                const int o = fwd ? R - d : R + d;
                if (o < 0 || o >= K) continue;
                const float* L = stile(st, d);
                const float* Z = Zr + (size_t)(o % S) * NB * C;
                if (fwd) {
                    // acc -= L_{R,o}[lane][k] z_o[k]; nonzero only for k >= 32 d - b
                    const int k0 = NB * d - bw;
                    if (k0 >= 24) ws_rowp<(KBP > 2 && C >= 2), C, 24, 32, -1>(L, Z, lane, acc);
                    else if (k0 >= 16) ws_rowp<(KBP > 2 && C >= 2), C, 16, 32, -1>(L, Z, lane, acc);
                    else ws_rowp<(KBP > 2 && C >= 2), C, 0, 32, -1>(L, Z, lane, acc);
                } else {
                    // acc -= L_{o,R}[k][lane] x_o[k]; nonzero only for k <= b - 32 d + 31
                    const int kend = bw - NB * d + NB;
                    if (kend <= 8) ws_colp<(KBP > 2 && C >= 2), C, 8, -1>(L, Z, lane, acc);
                    else if (kend <= 16) ws_colp<(KBP > 2 && C >= 2), C, 16, -1>(L, Z, lane, acc);
                    else ws_colp<(KBP > 2 && C >= 2), C, 32, -1>(L, Z, lane, acc);
                }
            }
            ws_st<C>(Acc + lane * C, acc);
            __syncwarp();
            const float* T = stile(st, 0);
            float out[C];
#pragma unroll
            for (int c = 0; c < C; ++c) out[c] = 0.f;
            if (fwd) ws_rowp<(KBP > 2 && C >= 2), C, 0, 32, 1>(T, Acc, lane, out);
            else ws_colp<(KBP > 2 && C >= 2), C, 32, 1>(T, Acc, lane, out);
            __syncwarp();                                   // Acc reads done before the next step's writes
            ws_st<C>(Zr + ((size_t)(R % S) * NB + lane) * C, out);
            double* xw = X + (roff + (long long)R * NB + lane) * ldx;
#pragma unroll
            for (int c = 0; c < C; ++c)
                if (c < nc) xw[c] = f32_to_f64(out[c]);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[st]);
    }
    cp_async_wait_n<0>();
}

// Launch of k_tile_solve_band_ws for one configuration.
template <int KBP, int W, int C, int NST, int XD>
void launch_band_ws(const TileBatch& tb, const CUtensorMap& tm, double* X, int ldx, int ncols, const int* skip,
                    cudaStream_t s, const int* gdone) {
    using Cfg = BandWs<KBP, W, C, NST, XD>;
    static_assert(Cfg::smem_bytes <= 227 * 1024, "shared memory per CTA");
    auto kern = k_tile_solve_band_ws<KBP, W, C, NST, XD>;
    raise_smem_limit(kern, Cfg::smem_bytes);
    kern<<<dim3(tb.P, (ncols + Cfg::COLS - 1) / Cfg::COLS), Cfg::NT, Cfg::smem_bytes, s>>>(
        tm, tb.dinv_f.p, tb.d_kb.p, tb.d_K.p, tb.d_b.p, tb.d_toff.p, tb.d_roff.p, X, ldx, ncols, skip, gdone);
    MSDD_LAUNCH_CHECK();
}

// ---- one right-hand side, wide bands: the off-diagonal tiles of a step split
// over warps.  With one column a step is a chain of kb tile products and the
// T_R product in one warp; here WS consumer warps each take the tiles d = w + 1,
// w + 1 + WS, ... of the step and store their partial sums, and warp 0 forms
// the right-hand side minus those sums and applies T_R (T_R^T backward), writes
// the step's solution to the ring and to X, under two named barriers of the
// consumer warps.  The producer warp streams the tiles as in
// k_tile_solve_band_ws; warp 0 alone releases a stage, after the barrier that
// ends every warp's reads of it.
template <int KBP, int WS, int NST, int XD>
struct BandSplit {
    static_assert(XD <= KBP + 2, "X prefetch deeper than the solution ring allows");
    static constexpr int S = KBP + 1;
    static constexpr int NT = 32 * (WS + 1);
    static constexpr size_t smem_bytes = 1024 + (size_t)NST * S * NB2 * sizeof(float) + (size_t)NST * NB * 4 +
                                         16 * (size_t)NST + (size_t)(S + WS + 1) * NB * 4 + 16 + (size_t)XD * NB * 8;
};

template <int KBP, int WS, int NST, int XD>
__global__ void __launch_bounds__(32 * (WS + 1)) k_tile_solve_band_split(
    const __grid_constant__ CUtensorMap tmt, const float* __restrict__ dinv, const int* __restrict__ kb_,
    const int* __restrict__ K_, const int* __restrict__ b_, const long long* __restrict__ toff_,
    const long long* __restrict__ roff_, double* __restrict__ X, const int* __restrict__ gdone)
{
    using Cfg = BandSplit<KBP, WS, NST, XD>;
    constexpr int S = Cfg::S;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
    float* St = reinterpret_cast<float*>(base);                                        // [NST][S][32*32]
    float* Sd = St + (size_t)NST * S * NB2;                                            // [NST][32]
    unsigned long long* full = reinterpret_cast<unsigned long long*>(Sd + (size_t)NST * NB);
    unsigned long long* empty = full + NST;
    float* Zr = reinterpret_cast<float*>(empty + NST);                                // [S][32] solutions
    float* Pp = Zr + (size_t)S * NB;                                                   // [WS][32] partial sums
    float* Acc = Pp + (size_t)WS * NB;                                                 // [32]
    double* Xs = reinterpret_cast<double*>(                                            // [XD][32]
        base + ((reinterpret_cast<unsigned char*>(Acc + NB) - base + 15) & ~(size_t)15));
    __shared__ int s_abort, s_stop;

    const int i = blockIdx.x;
    if (gdone && *gdone) return;
    const int kb = kb_[i], K = K_[i], bw = b_[i];
    if (kb > KBP) return;                            // never launched so (host dispatch)
    const long long toff = toff_[i], roff = roff_[i];
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    if (t == 0) {
        s_abort = 0;
        for (int s = 0; s < NST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        fence_mbar_init();
    }
    __syncthreads();
    auto stile = [&](int st, int slot) { return St + (size_t)(st * S + slot) * NB2; };
    auto give_up = [&]() {
        if (atomicExch(&s_abort, 1) == 0) atomicAdd(&g_wait_timeouts, 1);
    };
    const int total = 2 * K;

    if (warp == WS) {
        // ---------------- producer (as in k_tile_solve_band_ws)
        if (lane == 0) {
            unsigned pending = 0, par = 0;
            for (int it = 0; it < total; ++it) {
                const int st = it % NST;
                if (it >= NST) {
                    if (!mbar_wait_bounded(&empty[st], ((it / NST) - 1) & 1u)) { give_up(); break; }
                    pending &= ~(1u << st);
                }
                if (*(volatile int*)&s_abort) break;
                const bool fwd = it < K;
                const int R = fwd ? it : total - 1 - it;
                int nt = 1;
                for (int d = 1; d <= kb; ++d) {
                    const int o = fwd ? R - d : R + d;
                    if (o >= 0 && o < K) ++nt;
                }
                mbar_expect_tx(&full[st], nt * NB2 * 4 + (fwd ? 0 : NB * 4));
                tma_load_tile(stile(st, 0), &tmt, (int)(tile_index(toff, kb, R, R) / NB), &full[st]);
                for (int d = 1; d <= kb; ++d) {
                    const int o = fwd ? R - d : R + d;
                    if (o < 0 || o >= K) continue;
                    const long long ti = fwd ? tile_index(toff, kb, R, o) : tile_index(toff, kb, o, R);
                    tma_load_tile(stile(st, d), &tmt, (int)(ti / NB), &full[st]);
                }
                if (!fwd) bulk_load(Sd + st * NB, dinv + roff + (long long)R * NB, NB * 4, &full[st]);
                pending |= 1u << st;
                par = (par & ~(1u << st)) | (((unsigned)(it / NST) & 1u) << st);
            }
            if (*(volatile int*)&s_abort)
                for (int s = 0; s < NST; ++s)
                    if (pending & (1u << s)) mbar_wait_bounded(&full[s], (par >> s) & 1u);
        }
        return;
    }

    auto consumers_sync = [&]() { asm volatile("bar.sync 1, %0;\n" ::"r"(32 * WS) : "memory"); };
    // X prefetch of warp 0 (lane = row): index u < K forward block u; u >= K
    // backward block K - 1 - S - (u - K) (backward steps s >= S)
    const int nload = K + max(0, K - S);
    auto issue_load = [&](int u) {
        if (u < nload) {
            if (u >= K) __threadfence_block();       // rows written by this lane in the forward sweep
            const int R = u < K ? u : K - 1 - S - (u - K);
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_u32(Xs + (u % XD) * NB + lane)),
                         "l"(X + roff + (long long)R * NB + lane));
        }
        cp_async_commit();
    };
    if (warp == 0)
        for (int u = 0; u < XD - 1; ++u) issue_load(u);
    int u_next = XD - 1, u_use = 0;
    for (int it = 0; it < total; ++it) {
        const int st = it % NST;
        const bool fwd = it < K;
        const int R = fwd ? it : total - 1 - it;
        float rhs[1] = {0.f};
        if (warp == 0) {
            if (fwd || (it - K) >= S) {
                issue_load(u_next++);
                cp_async_wait_n<XD - 1>();
                rhs[0] = f64_to_f32(Xs[(u_use % XD) * NB + lane]);
                ++u_use;
            } else {
                rhs[0] = Zr[(R % S) * NB + lane];
            }
        }
        const bool ok = mbar_wait_bounded(&full[st], (it / NST) & 1u);
        if (!ok) give_up();
        float part[1] = {0.f};
        if (ok) {
            for (int d = warp + 1; d <= kb; d += WS) {
                const int o = fwd ? R - d : R + d;
                if (o < 0 || o >= K) continue;
                const float* L = stile(st, d);
                const float* Z = Zr + (size_t)(o % S) * NB;
                if (fwd) {
                    const int k0 = NB * d - bw;
                    if (k0 >= 24) ws_row_product<1, 24, 32, 1>(L, Z, lane, part);
                    else if (k0 >= 16) ws_row_product<1, 16, 32, 1>(L, Z, lane, part);
                    else ws_row_product<1, 0, 32, 1>(L, Z, lane, part);
                } else {
                    const int kend = bw - NB * d + NB;
                    if (kend <= 8) ws_col_product<1, 8, 1>(L, Z, lane, part);
                    else if (kend <= 16) ws_col_product<1, 16, 1>(L, Z, lane, part);
                    else ws_col_product<1, 32, 1>(L, Z, lane, part);
                }
            }
        }
        Pp[warp * NB + lane] = part[0];
        consumers_sync();                            // every partial is in Pp
        if (warp == 0) {
            if (ok) {
                float acc = fwd ? rhs[0] : rhs[0] * Sd[st * NB + lane];
                for (int w = 0; w < WS; ++w) acc -= Pp[w * NB + lane];
                Acc[lane] = acc;
                __syncwarp();
                float out[1] = {0.f};
                const float* T = stile(st, 0);
                if (fwd) ws_row_product<1, 0, 32, 1>(T, Acc, lane, out);
                else ws_col_product<1, 32, 1>(T, Acc, lane, out);
                Zr[(R % S) * NB + lane] = out[0];
                X[roff + (long long)R * NB + lane] = f32_to_f64(out[0]);
            }
            if (lane == 0) *(volatile int*)&s_stop = *(volatile int*)&s_abort;
        }
        consumers_sync();                            // the solution is in the ring; the stage and Pp are free
        if (warp == 0 && lane == 0) mbar_arrive(&empty[st]);
        if (*(volatile int*)&s_stop) break;          // sampled once by warp 0: every warp leaves after this step
    }
    if (warp == 0) cp_async_wait_n<0>();
}

template <int KBP, int WS, int NST, int XD>
void launch_band_split(const TileBatch& tb, const CUtensorMap& tm, double* X, cudaStream_t s, const int* gdone) {
    using Cfg = BandSplit<KBP, WS, NST, XD>;
    static_assert(Cfg::smem_bytes <= 227 * 1024, "shared memory per CTA");
    auto kern = k_tile_solve_band_split<KBP, WS, NST, XD>;
    raise_smem_limit(kern, Cfg::smem_bytes);
    kern<<<tb.P, Cfg::NT, Cfg::smem_bytes, s>>>(tm, tb.dinv_f.p, tb.d_kb.p, tb.d_K.p, tb.d_b.p, tb.d_toff.p,
                                                tb.d_roff.p, X, gdone);
    MSDD_LAUNCH_CHECK();
}

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

// [elems / 32][32] FP32 view of a tile array, 32 x 32 boxes, 128-byte swizzle.
bool encode_tile_map(const float* base, long long elems, CUtensorMap* m) {
    EncodeTiledFn enc = encode_tiled();
    if (!enc || !base || elems <= 0) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)NB, (cuuint64_t)(elems / NB)};
    const cuuint64_t strides[1] = {(cuuint64_t)NB * sizeof(float)};
    const cuuint32_t box[2] = {(cuuint32_t)NB, (cuuint32_t)NB};
    const cuuint32_t estr[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)base, dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The tile descriptor of an FP32 batch (built once per tiles_f allocation).
const CUtensorMap* tile_tensor_map(const TileBatch& tb) {
    if (!tb.prec || !tb.tiles_f.p || tb.total_tile_elems <= 0) return nullptr;
    if (tb.tmap_base == tb.tiles_f.p) return reinterpret_cast<const CUtensorMap*>(tb.tmap_tiles);
    CUtensorMap* m = reinterpret_cast<CUtensorMap*>(tb.tmap_tiles);
    if (!encode_tile_map(tb.tiles_f.p, tb.total_tile_elems, m)) return nullptr;
    tb.tmap_base = tb.tiles_f.p;
    return m;
}

template <typename T, int CPT, int CG>
void launch_band(const TileBatch& tb, const T* tiles, const T* dinv, double* X, int ldx, int ncols, const int* skip,
                 cudaStream_t s, const int* gdone) {
    constexpr int ZLD = BandSmem<T, CPT, CG>::ZLD;
    const int chunks = (ncols + ZLD - 1) / ZLD;
    const size_t b = BandSmem<T, CPT, CG>::bytes(((std::min(ncols, ZLD) + 1) / 2) * 2);
    raise_smem_limit(k_tile_solve_band<T, CPT, CG>, b);
    k_tile_solve_band<T, CPT, CG><<<dim3(tb.P, chunks), 8 * CG, b, s>>>(tiles, dinv, tb.d_kb.p, tb.d_K.p, tb.d_toff.p,
                                                                         tb.d_roff.p, X, ldx, ncols, skip, gdone);
    MSDD_LAUNCH_CHECK();
}

template <typename T>
void launch_band_cols(const TileBatch& tb, const T* tiles, const T* dinv, double* X, int ldx, int ncols,
                      const int* skip, cudaStream_t s, const int* gdone) {
    // chunks of 8 columns, one 64-thread CTA each (more independent
    // sequential sweeps in flight per SM than wider CTAs)
    launch_band<T, 1, 8>(tb, tiles, dinv, X, ldx, ncols, skip, s, gdone);
}

__global__ void k_fill_identity(double* __restrict__ E, const int* __restrict__ n_, const int* __restrict__ K_,
                                const long long* __restrict__ roff_, int lde) {
    const int i = blockIdx.y;
    const int n = n_[i];
    const long long rows = (long long)K_[i] * NB;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < rows * lde;
         e += (long long)gridDim.x * blockDim.x) {
        long long r = e / lde, c = e % lde;
        E[(roff_[i] + r) * lde + c] = (r == c && r < n) ? 1.0 : 0.0;
    }
}

template <typename T>
__global__ void k_tile_from_dense(T* __restrict__ tiles, const int* __restrict__ n_, const int* __restrict__ kb_,
                                  const int* __restrict__ K_, const long long* __restrict__ toff_,
                                  const int* __restrict__ b_, const double* __restrict__ src,
                                  const long long* __restrict__ soff, const int* __restrict__ lds)
{
    const int i = blockIdx.y;
    const int n = n_[i], kb = kb_[i], K = K_[i], bw = b_[i];
    const long long ntile = (long long)K * (kb + 1) * NB2;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < ntile;
         e += (long long)gridDim.x * blockDim.x) {
        long long tileno = e / NB2;
        int within = (int)(e % NB2);
        int R = (int)(tileno / (kb + 1)), d = (int)(tileno % (kb + 1));
        int C = R - d;
        int rr = R * NB + within / NB, cc = C * NB + within % NB;
        T v = 0;
        if (C >= 0 && rr < n && cc < n && cc >= 0 && cc <= rr && rr - cc <= bw)
            v = (T)src[soff[i] + (long long)rr * lds[i] + cc];
        tiles[toff_[i] + e] = v;
    }
}

}  // namespace

TileBatch TileBatch::slice(int p0, int np) const {
    TileBatch v;
    v.P = np;
    v.prec = prec;
    auto sub = [&](const auto& vec) { return std::decay_t<decltype(vec)>(vec.begin() + p0, vec.begin() + p0 + np); };
    v.n = sub(n); v.kb = sub(kb); v.K = sub(K); v.b = sub(b); v.toff = sub(toff); v.roff = sub(roff);
    v.total_tile_elems = total_tile_elems;
    v.total_rows = total_rows;
    v.max_K = 0;
    for (int k : v.K) v.max_K = std::max(v.max_K, k);
    v.d_n = d_n.view(p0, np); v.d_kb = d_kb.view(p0, np); v.d_K = d_K.view(p0, np); v.d_b = d_b.view(p0, np);
    v.d_status = d_status.view(p0, np); v.d_nreg = d_nreg.view(p0, np);
    v.d_toff = d_toff.view(p0, np); v.d_roff = d_roff.view(p0, np);
    v.tiles_d = tiles_d.view(0, tiles_d.n); v.dinv_d = dinv_d.view(0, dinv_d.n);
    v.tiles_f = tiles_f.view(0, tiles_f.n); v.dinv_f = dinv_f.view(0, dinv_f.n);
    tile_tensor_map(*this);                     // build the shared descriptor once, then copy it
    memcpy(v.tmap_tiles, tmap_tiles, sizeof(tmap_tiles));
    v.tmap_base = tmap_base;
    return v;
}

void TileBatch::layout(const std::vector<int>& n_, const std::vector<int>& b_, int precision, cudaStream_t s) {
    P = (int)n_.size();
    prec = precision;
    tmap_base = nullptr;
    n = n_;
    kb.resize(P);
    K.resize(P);
    b.resize(P);
    toff.resize(P);
    roff.resize(P);
    total_tile_elems = 0;
    total_rows = 0;
    max_K = 0;
    for (int i = 0; i < P; ++i) {
        K[i] = n[i] > 0 ? (int)ceil_div(n[i], NB) : 0;
        int bi = b_[i] < n[i] - 1 ? b_[i] : n[i] - 1;
        if (bi < 0) bi = 0;
        b[i] = bi;
        kb[i] = (int)ceil_div(bi, NB);
        if (kb[i] > K[i] - 1) kb[i] = K[i] > 0 ? K[i] - 1 : 0;
        toff[i] = total_tile_elems;
        roff[i] = total_rows;
        total_tile_elems += (long long)K[i] * (kb[i] + 1) * NB2;
        total_rows += (long long)K[i] * NB;
        if (K[i] > max_K) max_K = K[i];
    }
    d_n.upload(n, s);
    d_kb.upload(kb, s);
    d_b.upload(b, s);
    d_K.upload(K, s);
    d_toff.upload(toff, s);
    d_roff.upload(roff, s);
    d_status.alloc(P);
    d_nreg.alloc(P);
    if (prec) {
        tiles_f.alloc(total_tile_elems);
        dinv_f.alloc(total_rows);
        tiles_d.release();
        dinv_d.release();
    } else {
        tiles_d.alloc(total_tile_elems);
        dinv_d.alloc(total_rows);
        tiles_f.release();
        dinv_f.release();
    }
}

void tile_zero(TileBatch& tb, cudaStream_t s) {
    if (tb.prec) tb.tiles_f.zero(s); else tb.tiles_d.zero(s);
}

void tile_from_dense(TileBatch& tb, const double* src, const long long* d_soff, const int* d_lds, cudaStream_t s) {
    if (tb.P == 0) return;
    long long maxt = 0;
    for (int i = 0; i < tb.P; ++i) maxt = std::max(maxt, (long long)tb.K[i] * (tb.kb[i] + 1) * NB2);
    dim3 grid(std::min<long long>(ceil_div(maxt, 256), 1024), tb.P);
    if (tb.prec)
        k_tile_from_dense<float><<<grid, 256, 0, s>>>(tb.tiles_f.p, tb.d_n.p, tb.d_kb.p, tb.d_K.p, tb.d_toff.p, tb.d_b.p, src, d_soff, d_lds);
    else
        k_tile_from_dense<double><<<grid, 256, 0, s>>>(tb.tiles_d.p, tb.d_n.p, tb.d_kb.p, tb.d_K.p, tb.d_toff.p, tb.d_b.p, src, d_soff, d_lds);
    MSDD_LAUNCH_CHECK();
}

void tile_identity(const TileBatch& tb, double* E, int lde, cudaStream_t s) {
    if (tb.P == 0) return;
    dim3 grid(64, tb.P);
    k_fill_identity<<<grid, 256, 0, s>>>(E, tb.d_n.p, tb.d_K.p, tb.d_roff.p, lde);
    MSDD_LAUNCH_CHECK();
}

void tile_factor(TileBatch& tb, double reg_tol, cudaStream_t s) {
    if (tb.P == 0) return;
    int maxkb = 0;
    for (int v : tb.kb) maxkb = std::max(maxkb, v);
    bool dense = tb.max_K >= 3;
    for (int i = 0; i < tb.P && dense; ++i) dense = tb.kb[i] >= tb.K[i] - 1;
    if (dense) {
        auto run = [&](auto* tl, auto* dv) {
            using T = std::remove_pointer_t<decltype(tl)>;
            k_save_diag<T><<<tb.P, TPB, 0, s>>>(tl, dv, tb.d_kb.p, tb.d_K.p, tb.d_toff.p, tb.d_roff.p, tb.d_status.p,
                                               tb.d_nreg.p);
            MSDD_LAUNCH_CHECK();
            for (int k = 0; k < tb.max_K; ++k) {
                k_rl_diag<T><<<tb.P, TPB, 0, s>>>(tl, dv, tb.d_n.p, tb.d_kb.p, tb.d_K.p, tb.d_toff.p, tb.d_roff.p,
                                                 tb.d_status.p, tb.d_nreg.p, reg_tol, k);
                MSDD_LAUNCH_CHECK();
                const int m = tb.max_K - 1 - k;
                if (m == 0) break;
                k_rl_panel<T><<<dim3(tb.P, m), TPB, 0, s>>>(tl, dv, tb.d_kb.p, tb.d_K.p, tb.d_toff.p, tb.d_roff.p, k);
                MSDD_LAUNCH_CHECK();
                k_rl_update<T><<<dim3(tb.P, m * (m + 1) / 2), TPB, 0, s>>>(tl, dv, tb.d_kb.p, tb.d_K.p, tb.d_toff.p,
                                                                         tb.d_roff.p, k);
                MSDD_LAUNCH_CHECK();
            }
        };
        if (tb.prec) run(tb.tiles_f.p, tb.dinv_f.p);
        else run(tb.tiles_d.p, tb.dinv_d.p);
        return;
    }
    if (tb.prec && maxkb <= 2) {
        const size_t b = factor_band32_smem();
        raise_smem_limit(k_tile_factor_band32, b);
        k_tile_factor_band32<<<tb.P, FB_T, b, s>>>(tb.tiles_f.p, tb.dinv_f.p, tb.d_n.p, tb.d_kb.p, tb.d_K.p,
                                                  tb.d_toff.p, tb.d_roff.p, tb.d_status.p, tb.d_nreg.p, reg_tol);
        MSDD_LAUNCH_CHECK();
        return;
    }
    if (tb.prec && maxkb <= TF_KBM) {
        // 3 <= kb <= 12: panel updates on the tensor cores (lo parts of the factor in scratch)
        const CUtensorMap* thi = tile_tensor_map(tb);
        DevBuf<float> lo(tb.total_tile_elems);
        alignas(64) CUtensorMap tlo;
        if (thi && encode_tile_map(lo.p, tb.total_tile_elems, &tlo)) {
            const size_t b = tf_smem_bytes();
            raise_smem_limit(k_tile_factor_tc, b);
            k_tile_factor_tc<<<tb.P, TF_NT, b, s>>>(*thi, tlo, tb.tiles_f.p, lo.p, tb.total_tile_elems, tb.dinv_f.p,
                                                   tb.d_n.p, tb.d_kb.p, tb.d_K.p, tb.d_toff.p, tb.d_roff.p,
                                                   tb.d_status.p, tb.d_nreg.p, reg_tol);
            MSDD_LAUNCH_CHECK();
            return;
        }
    }
    if (tb.prec)
        k_tile_factor<float><<<tb.P, TPB, 0, s>>>(tb.tiles_f.p, tb.dinv_f.p, tb.d_n.p, tb.d_kb.p, tb.d_K.p,
                                                 tb.d_toff.p, tb.d_roff.p, tb.d_status.p, tb.d_nreg.p, reg_tol);
    else
        k_tile_factor<double><<<tb.P, TPB, 0, s>>>(tb.tiles_d.p, tb.dinv_d.p, tb.d_n.p, tb.d_kb.p, tb.d_K.p,
                                                  tb.d_toff.p, tb.d_roff.p, tb.d_status.p, tb.d_nreg.p, reg_tol);
    MSDD_LAUNCH_CHECK();
}

void tile_check_waits() {
    int n = 0;
    MSDD_CUDA(cudaMemcpyFromSymbol(&n, g_wait_timeouts, sizeof(int)));
    if (n) {
        const int zero = 0;
        MSDD_CUDA(cudaMemcpyToSymbol(g_wait_timeouts, &zero, sizeof(int)));
        throw WaitTimeout("a band solve gave up waiting for its tile copies (" + std::to_string(n) + " CTAs)");
    }
}

void tile_solve(const TileBatch& tb, double* X, int ldx, int ncols, const int* skip, cudaStream_t s,
                const int* gdone) {
    if (tb.P == 0) return;
    if (ncols > ldx) throw std::runtime_error("tile_solve: more columns than the leading dimension");
    const size_t zbytes = (size_t)tb.max_K * NB * sizeof(double);   // upper bound for both precisions
    if (ncols == 1 && ldx == 1 && skip == nullptr) {
        int maxkb = 0;
        for (int v : tb.kb) maxkb = std::max(maxkb, v);
        const size_t zt = (size_t)tb.max_K * NB * (tb.prec ? sizeof(float) : sizeof(double));
        const size_t ring_bytes = (tb.prec ? (maxkb <= 1 ? solve1_ring_bytes<float, 1>() : solve1_ring_bytes<float, 2>())
                                           : (maxkb <= 1 ? solve1_ring_bytes<double, 1>() : solve1_ring_bytes<double, 2>())) + zt;
        if (maxkb <= 2 && ring_bytes <= 200 * 1024) {
            if (tb.prec) {
                auto k = maxkb <= 1 ? k_tile_solve1<float, 1> : k_tile_solve1<float, 2>;
                raise_smem_limit(k, ring_bytes);
                k<<<tb.P, S1T, ring_bytes, s>>>(tb.tiles_f.p, tb.dinv_f.p, tb.d_kb.p, tb.d_K.p, tb.d_toff.p, tb.d_roff.p, X, gdone);
            } else {
                auto k = maxkb <= 1 ? k_tile_solve1<double, 1> : k_tile_solve1<double, 2>;
                raise_smem_limit(k, ring_bytes);
                k<<<tb.P, S1T, ring_bytes, s>>>(tb.tiles_d.p, tb.dinv_d.p, tb.d_kb.p, tb.d_K.p, tb.d_toff.p, tb.d_roff.p, X, gdone);
            }
            MSDD_LAUNCH_CHECK();
            return;
        }
        if (tb.prec && maxkb > 2 && maxkb <= 12) {
            // wide bands, one right-hand side (PCG local solves of 3D boxes):
            // the step's off-diagonal tiles split over 6 warps, two stages of 13 tiles
            const CUtensorMap* tm = tile_tensor_map(tb);
            if (tm) {
                launch_band_split<12, 6, 2, 4>(tb, *tm, X, s, gdone);
                return;
            }
        }
        if (maxkb > 2 && zbytes <= 160 * 1024) {
            if (zbytes > 48 * 1024) {
                raise_smem_limit(k_tile_solve1_dense<float>, zbytes);
                raise_smem_limit(k_tile_solve1_dense<double>, zbytes);
            }
            if (tb.prec) k_tile_solve1_dense<float><<<tb.P, S1T, zbytes, s>>>(tb.tiles_f.p, tb.dinv_f.p, tb.d_kb.p, tb.d_K.p, tb.d_toff.p, tb.d_roff.p, X, gdone);
            else k_tile_solve1_dense<double><<<tb.P, S1T, zbytes, s>>>(tb.tiles_d.p, tb.dinv_d.p, tb.d_kb.p, tb.d_K.p, tb.d_toff.p, tb.d_roff.p, X, gdone);
            MSDD_LAUNCH_CHECK();
            return;
        }
    }
    int maxkb = 0;
    for (int v : tb.kb) maxkb = std::max(maxkb, v);
    // the band kernels stage blocks of X with 16-byte copies
    const bool aligned = ldx % 2 == 0 && ((uintptr_t)X % 16) == 0;
    const CUtensorMap* tm = tb.prec && aligned && ncols <= NB ? tile_tensor_map(tb) : nullptr;
    if (tm && maxkb <= 2) {
        // 16 columns in 4 warps of 4, 6 stages.  8 warps of 2 with 3 stages
        // is 9% faster on its own (129 vs 139 us a launch) but no faster in
        // the set-up, where the other half's kernels share the SMs
        launch_band_ws<2, 4, 4, 6, 4>(tb, *tm, X, ldx, ncols, skip, s, gdone);
        return;
    }
    if (tm && maxkb <= 12) {
        // wide bands (3D boxes): 20 columns per CTA in 10 warps of 2, 2 stages
        // of 13 tiles (17% faster than 5 warps of 4 with 3 stages: the smaller
        // shared-memory carve-out leaves L1 to the right-hand-side rows)
        launch_band_ws<12, 10, 2, 2, 4>(tb, *tm, X, ldx, ncols, skip, s, gdone);
        return;
    }
    if (maxkb <= 2 && ncols <= NB && aligned) {
        if (tb.prec) launch_band_cols<float>(tb, tb.tiles_f.p, tb.dinv_f.p, X, ldx, ncols, skip, s, gdone);
        else launch_band_cols<double>(tb, tb.tiles_d.p, tb.dinv_d.p, X, ldx, ncols, skip, s, gdone);
        return;
    }
    const dim3 grid(tb.P, (ncols + NB - 1) / NB);
    if (tb.prec)
        k_tile_solve<float><<<grid, TPB, 0, s>>>(tb.tiles_f.p, tb.dinv_f.p, tb.d_n.p, tb.d_kb.p, tb.d_K.p,
                                                tb.d_toff.p, tb.d_roff.p, X, ldx, ncols, skip, gdone);
    else
        k_tile_solve<double><<<grid, TPB, 0, s>>>(tb.tiles_d.p, tb.dinv_d.p, tb.d_n.p, tb.d_kb.p, tb.d_K.p,
                                                 tb.d_toff.p, tb.d_roff.p, X, ldx, ncols, skip, gdone);
    MSDD_LAUNCH_CHECK();
}

}  // namespace msdd
