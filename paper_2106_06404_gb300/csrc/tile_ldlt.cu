// Batched tile-band LDL^T factorisation and triangular solves (one CTA per
// local matrix).  See tile_ldlt.cuh for the storage format.
#include "tile_ldlt.cuh"

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
                // dense LDL^T of the diagonal tile (lower triangle of W)
                const int rows_valid = n - R * NB;   // rows >= rows_valid are padding
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
                // T_R = L_RR^{-1} (unit lower), built in Sa
                for (int e = t; e < NB2; e += TPB) Sa[e / NB][e % NB] = (e / NB == e % NB) ? T(1) : T(0);
                __syncthreads();
                for (int k = 0; k < NB - 1; ++k) {
                    for (int e = t; e < NB2; e += TPB) {
                        int a = e / NB, b = e % NB;
                        if (a > k && b <= k) Sa[a][b] -= W[a][k] * Sa[k][b];
                    }
                    __syncthreads();
                }
                store_tile(tiles + tile_index(toff, kb, R, R), Sa);
                if (t < NB) dinv[roff + (long long)R * NB + t] = sd[t];
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


// ------------------------------------------------------------------ solve, one right-hand side
// The PCG local solves.  One CTA of 128 threads per matrix; the whole local
// vector lives in shared memory.  Forward sweep: thread (row r = t/4, chunk
// t%4) reads 8 contiguous entries of row r of each tile (coalesced) and the 4
// partial sums of a row are combined by warp shuffles.  Backward sweep uses
// the transposed tiles: thread (column c = lane, rows 8*warp..) reads tile
// rows contiguously across the warp, partial sums of the 4 warps are combined
// in shared memory.  For band matrices (kb <= KBP) the tiles of step R+1 are
// loaded into registers while step R computes.
constexpr int S1T = 128;

template <typename T, int KBP>
__device__ __forceinline__ void load_row_chunks(T (&v)[KBP + 1][8], const T* __restrict__ tiles, long long toff, int kb,
                                                int R, int K, int r, int c0, bool fwd) {
#pragma unroll
    for (int d = 0; d <= KBP; ++d) {
        int other = fwd ? R - d : R + d;   // fwd: tile (R, R-d); bwd: tile (R+d, R)
        bool ok = d <= kb && other >= 0 && other < K && R >= 0 && R < K;
        const T* src = ok ? tiles + (fwd ? tile_index(toff, kb, R, other) : tile_index(toff, kb, other, R)) : nullptr;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            // fwd: row r, columns c0..c0+7; bwd: rows c0..c0+7 (c0 = 8 * warp), column r (= lane)
            v[d][q] = ok ? (fwd ? src[r * NB + c0 + q] : src[(c0 + q) * NB + r]) : T(0);
        }
    }
}

template <typename T, int KBP>
__global__ void __launch_bounds__(S1T) k_tile_solve1(
    const T* __restrict__ tiles, const T* __restrict__ dinv, const int* __restrict__ kb_, const int* __restrict__ K_,
    const long long* __restrict__ toff_, const long long* __restrict__ roff_, double* __restrict__ X,
    const int* __restrict__ gdone)
{
    extern __shared__ __align__(16) unsigned char zs_raw[];
    T* zs = reinterpret_cast<T*>(zs_raw);
    __shared__ T accs[NB];
    __shared__ T part[S1T / 32][NB + 1];
    if (gdone && *gdone) return;
    const int i = blockIdx.x;
    const int kb = kb_[i], K = K_[i];
    const long long toff = toff_[i], roff = roff_[i];
    const int t = threadIdx.x;
    for (int e = t; e < K * NB; e += S1T) zs[e] = T(X[roff + e]);
    __syncthreads();

    // forward: z_R = T_R (x_R - sum_{J<R} L_RJ z_J)
    {
        const int r = t >> 2, c0 = (t & 3) * 8;
        T cur[KBP + 1][8], nxt[KBP + 1][8];
        load_row_chunks<T, KBP>(cur, tiles, toff, kb, 0, K, r, c0, true);
        for (int R = 0; R < K; ++R) {
            load_row_chunks<T, KBP>(nxt, tiles, toff, kb, R + 1, K, r, c0, true);
            T acc = T(0);
#pragma unroll
            for (int d = 1; d <= KBP; ++d) {
                if (d > kb || R - d < 0) continue;
                const T* zj = zs + (R - d) * NB + c0;
#pragma unroll
                for (int q = 0; q < 8; ++q) acc += cur[d][q] * zj[q];
            }
            acc += __shfl_xor_sync(0xffffffffu, acc, 1);
            acc += __shfl_xor_sync(0xffffffffu, acc, 2);
            if ((t & 3) == 0) accs[r] = zs[R * NB + r] - acc;
            __syncthreads();
            T s = T(0);
#pragma unroll
            for (int q = 0; q < 8; ++q) s += cur[0][q] * accs[c0 + q];
            s += __shfl_xor_sync(0xffffffffu, s, 1);
            s += __shfl_xor_sync(0xffffffffu, s, 2);
            if ((t & 3) == 0) zs[R * NB + r] = s;
            __syncthreads();
#pragma unroll
            for (int d = 0; d <= KBP; ++d)
#pragma unroll
                for (int q = 0; q < 8; ++q) cur[d][q] = nxt[d][q];
        }
    }
    for (int e = t; e < K * NB; e += S1T) zs[e] *= dinv[roff + e];
    __syncthreads();
    // backward: x_R = T_R^T (D_R^{-1} z_R - sum_{I>R} L_IR^T x_I)
    {
        const int lane = t & 31, warp = t >> 5, k0 = warp * 8;
        T cur[KBP + 1][8], nxt[KBP + 1][8];
        load_row_chunks<T, KBP>(cur, tiles, toff, kb, K - 1, K, lane, k0, false);
        for (int R = K - 1; R >= 0; --R) {
            load_row_chunks<T, KBP>(nxt, tiles, toff, kb, R - 1, K, lane, k0, false);
            T s = T(0);
#pragma unroll
            for (int d = 1; d <= KBP; ++d) {
                if (d > kb || R + d >= K) continue;
                const T* xi = zs + (R + d) * NB + k0;
#pragma unroll
                for (int q = 0; q < 8; ++q) s += cur[d][q] * xi[q];
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
            T s2 = T(0);
#pragma unroll
            for (int q = 0; q < 8; ++q) s2 += cur[0][q] * accs[k0 + q];
            part[warp][lane] = s2;
            __syncthreads();
            if (warp == 0) {
                T v = T(0);
#pragma unroll
                for (int w = 0; w < S1T / 32; ++w) v += part[w][lane];
                zs[R * NB + lane] = v;
            }
            __syncthreads();
#pragma unroll
            for (int d = 0; d <= KBP; ++d)
#pragma unroll
                for (int q = 0; q < 8; ++q) cur[d][q] = nxt[d][q];
        }
    }
    for (int e = t; e < K * NB; e += S1T) X[roff + e] = (double)zs[e];
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
// For kb <= KBR: the tiles of step R+1 are copied into shared memory with
// cp.async while step R computes, and the last kb solution blocks stay in a
// shared ring (no re-reading of earlier blocks from global memory).  Thread
// (row r = t/8, columns t%8 + 8q) owns up to 4 entries of a 32 x ncols block.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait_n() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }
constexpr int RING_STAGES = 3;

template <typename T>
struct RingLayout {
    static constexpr int LDT = sizeof(T) == 4 ? NB + 4 : NB + 2;   // 16-byte aligned padded rows
    static constexpr int LDZ = NB + 1;
};

template <typename T>
__device__ __forceinline__ void async_tile(T* dst, const T* __restrict__ src) {
    constexpr int PER = 16 / (int)sizeof(T);
    constexpr int LDT = RingLayout<T>::LDT;
    for (int ch = threadIdx.x; ch < NB2 / PER; ch += TPB) {
        int e = ch * PER;
        cp_async16(dst + (e / NB) * LDT + (e % NB), src + e);
    }
}

template <typename T, int KBR>
__global__ void __launch_bounds__(TPB) k_tile_solve_ring(
    const T* __restrict__ tiles, const T* __restrict__ dinv, const int* __restrict__ kb_, const int* __restrict__ K_,
    const long long* __restrict__ toff_, const long long* __restrict__ roff_, double* __restrict__ X, int ldx,
    int ncols, const int* __restrict__ skip, const int* __restrict__ gdone)
{
    // NST-stage cp.async pipeline: stage s holds the tiles of one step and the
    // 32 x ldx block of X (right-hand side in the forward sweep, z in the
    // backward sweep) it starts from; NST - 1 steps are in flight.
    constexpr int LDT = RingLayout<T>::LDT, LDZ = RingLayout<T>::LDZ, S = KBR + 1, NST = RING_STAGES;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* St = reinterpret_cast<T*>(smem_raw);                               // [NST][S][NB][LDT]
    double* Sx = reinterpret_cast<double*>(St + (size_t)NST * S * NB * LDT);  // [NST][NB][ldx]
    T* Zr = reinterpret_cast<T*>(Sx + (size_t)NST * NB * ldx);            // [S][NB][LDZ]
    T* Acc = Zr + S * NB * LDZ;                                           // [NB][LDZ]
    const int i = blockIdx.x;
    if (skip && skip[i]) return;
    if (gdone && *gdone) return;
    const int kb = kb_[i], K = K_[i];
    const long long toff = toff_[i], roff = roff_[i];
    const int t = threadIdx.x;
    const int r = t >> 3, cb = t & 7;
    const int qn = (ncols + 7) / 8;          // columns cb + 8q, q < qn, owned by this thread
    auto stage_tile = [&](int st, int slot) { return St + ((size_t)(st * S + slot) * NB) * LDT; };
    auto issue = [&](int st, int R, bool fwd) {
        if (R >= 0 && R < K) {
            async_tile(stage_tile(st, 0), tiles + tile_index(toff, kb, R, R));
            for (int d = 1; d <= kb; ++d) {
                int o = fwd ? R - d : R + d;
                if (o < 0 || o >= K) continue;
                async_tile(stage_tile(st, d), tiles + (fwd ? tile_index(toff, kb, R, o) : tile_index(toff, kb, o, R)));
            }
            const double* src = X + (roff + (long long)R * NB) * ldx;
            double* dst = Sx + (size_t)st * NB * ldx;
            for (int ch = t; ch < NB * ldx / 2; ch += TPB) cp_async16(dst + 2 * ch, src + 2 * ch);
        }
        cp_async_commit();
    };
    // forward: z_R = T_R (x_R - sum_J L_RJ z_J)
    for (int k = 0; k < NST - 1; ++k) issue(k, k, true);
    for (int R = 0; R < K; ++R) {
        const int st = R % NST;
        issue((R + NST - 1) % NST, R + NST - 1, true);
        cp_async_wait_n<NST - 1>();
        __syncthreads();
        T acc[4];
        const double* xr = Sx + (size_t)st * NB * ldx + r * ldx;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int c = cb + 8 * q;
            acc[q] = (q < qn && c < ncols) ? T(xr[c]) : T(0);
        }
        for (int d = 1; d <= kb; ++d) {
            if (R - d < 0) break;
            const T* L = stage_tile(st, d) + r * LDT;
            const T* Z = Zr + ((R - d) % S) * NB * LDZ;
#pragma unroll 8
            for (int k = 0; k < NB; ++k) {
                T l = L[k];
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (q < qn) acc[q] -= l * Z[k * LDZ + cb + 8 * q];
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) Acc[r * LDZ + cb + 8 * q] = acc[q];
        __syncthreads();
        const T* Tt = stage_tile(st, 0) + r * LDT;
        T out[4] = {0, 0, 0, 0};
        for (int k = 0; k <= r; ++k) {
            T l = Tt[k];
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (q < qn) out[q] += l * Acc[k * LDZ + cb + 8 * q];
        }
        T* Zw = Zr + (R % S) * NB * LDZ;
        double* xw = X + (roff + (long long)R * NB + r) * ldx;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int c = cb + 8 * q;
            Zw[r * LDZ + c] = out[q];
            if (q < qn && c < ncols) xw[c] = (double)out[q];
        }
        __syncthreads();
    }
    cp_async_wait_n<0>();
    __syncthreads();
    // backward: x_R = T_R^T (D_R^{-1} z_R - sum_I L_IR^T x_I)
    for (int k = 0; k < NST - 1; ++k) issue(k, K - 1 - k, false);
    for (int R = K - 1, it = 0; R >= 0; --R, ++it) {
        const int st = it % NST;
        issue((it + NST - 1) % NST, R - (NST - 1), false);
        cp_async_wait_n<NST - 1>();
        __syncthreads();
        T acc[4];
        const double* xr = Sx + (size_t)st * NB * ldx + r * ldx;
        const T dr = dinv[roff + (long long)R * NB + r];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int c = cb + 8 * q;
            acc[q] = (q < qn && c < ncols) ? dr * T(xr[c]) : T(0);
        }
        for (int d = 1; d <= kb; ++d) {
            if (R + d >= K) break;
            const T* L = stage_tile(st, d);
            const T* Z = Zr + ((R + d) % S) * NB * LDZ;
#pragma unroll 8
            for (int k = 0; k < NB; ++k) {
                T l = L[k * LDT + r];
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (q < qn) acc[q] -= l * Z[k * LDZ + cb + 8 * q];
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) Acc[r * LDZ + cb + 8 * q] = acc[q];
        __syncthreads();
        const T* Tt = stage_tile(st, 0);
        T out[4] = {0, 0, 0, 0};
        for (int k = r; k < NB; ++k) {
            T l = Tt[k * LDT + r];
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (q < qn) out[q] += l * Acc[k * LDZ + cb + 8 * q];
        }
        T* Zw = Zr + (R % S) * NB * LDZ;
        double* xw = X + (roff + (long long)R * NB + r) * ldx;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int c = cb + 8 * q;
            Zw[r * LDZ + c] = out[q];
            if (q < qn && c < ncols) xw[c] = (double)out[q];
        }
        __syncthreads();
    }
    cp_async_wait_n<0>();
}

template <typename T, int KBR>
size_t ring_smem_bytes(int ldx) {
    return sizeof(T) * ((size_t)RING_STAGES * (KBR + 1) * NB * RingLayout<T>::LDT + (size_t)(KBR + 2) * NB * RingLayout<T>::LDZ) +
           sizeof(double) * (size_t)RING_STAGES * NB * ldx;
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

void TileBatch::layout(const std::vector<int>& n_, const std::vector<int>& b_, int precision, cudaStream_t s) {
    P = (int)n_.size();
    prec = precision;
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
    if (tb.prec)
        k_tile_factor<float><<<tb.P, TPB, 0, s>>>(tb.tiles_f.p, tb.dinv_f.p, tb.d_n.p, tb.d_kb.p, tb.d_K.p,
                                                 tb.d_toff.p, tb.d_roff.p, tb.d_status.p, tb.d_nreg.p, reg_tol);
    else
        k_tile_factor<double><<<tb.P, TPB, 0, s>>>(tb.tiles_d.p, tb.dinv_d.p, tb.d_n.p, tb.d_kb.p, tb.d_K.p,
                                                  tb.d_toff.p, tb.d_roff.p, tb.d_status.p, tb.d_nreg.p, reg_tol);
    MSDD_LAUNCH_CHECK();
}

void tile_solve(const TileBatch& tb, double* X, int ldx, int ncols, const int* skip, cudaStream_t s,
                const int* gdone) {
    if (tb.P == 0) return;
    if (ncols > ldx) throw std::runtime_error("tile_solve: more columns than the leading dimension");
    const size_t zbytes = (size_t)tb.max_K * NB * sizeof(double);   // upper bound for both precisions
    if (ncols == 1 && ldx == 1 && skip == nullptr && zbytes <= 160 * 1024) {
        int maxkb = 0;
        for (int v : tb.kb) maxkb = std::max(maxkb, v);
        if (zbytes > 48 * 1024) {
            MSDD_CUDA(cudaFuncSetAttribute(k_tile_solve1<float, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zbytes));
            MSDD_CUDA(cudaFuncSetAttribute(k_tile_solve1<float, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zbytes));
            MSDD_CUDA(cudaFuncSetAttribute(k_tile_solve1<double, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zbytes));
            MSDD_CUDA(cudaFuncSetAttribute(k_tile_solve1<double, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zbytes));
            MSDD_CUDA(cudaFuncSetAttribute(k_tile_solve1_dense<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zbytes));
            MSDD_CUDA(cudaFuncSetAttribute(k_tile_solve1_dense<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zbytes));
        }
        if (tb.prec) {
            if (maxkb <= 1) k_tile_solve1<float, 1><<<tb.P, S1T, zbytes, s>>>(tb.tiles_f.p, tb.dinv_f.p, tb.d_kb.p, tb.d_K.p, tb.d_toff.p, tb.d_roff.p, X, gdone);
            else if (maxkb <= 2) k_tile_solve1<float, 2><<<tb.P, S1T, zbytes, s>>>(tb.tiles_f.p, tb.dinv_f.p, tb.d_kb.p, tb.d_K.p, tb.d_toff.p, tb.d_roff.p, X, gdone);
            else k_tile_solve1_dense<float><<<tb.P, S1T, zbytes, s>>>(tb.tiles_f.p, tb.dinv_f.p, tb.d_kb.p, tb.d_K.p, tb.d_toff.p, tb.d_roff.p, X, gdone);
        } else {
            if (maxkb <= 1) k_tile_solve1<double, 1><<<tb.P, S1T, zbytes, s>>>(tb.tiles_d.p, tb.dinv_d.p, tb.d_kb.p, tb.d_K.p, tb.d_toff.p, tb.d_roff.p, X, gdone);
            else if (maxkb <= 2) k_tile_solve1<double, 2><<<tb.P, S1T, zbytes, s>>>(tb.tiles_d.p, tb.dinv_d.p, tb.d_kb.p, tb.d_K.p, tb.d_toff.p, tb.d_roff.p, X, gdone);
            else k_tile_solve1_dense<double><<<tb.P, S1T, zbytes, s>>>(tb.tiles_d.p, tb.dinv_d.p, tb.d_kb.p, tb.d_K.p, tb.d_toff.p, tb.d_roff.p, X, gdone);
        }
        MSDD_LAUNCH_CHECK();
        return;
    }
    int maxkb = 0;
    for (int v : tb.kb) maxkb = std::max(maxkb, v);
    // the ring kernel stages whole 32 x ldx blocks of X with 16-byte copies
    const bool ring_ok = maxkb <= 2 && ncols <= NB && ldx <= NB && ldx % 2 == 0 &&
                         ((uintptr_t)X % 16) == 0;
    if (ring_ok) {
        if (tb.prec) {
            size_t b = ring_smem_bytes<float, 2>(ldx);
            MSDD_CUDA(cudaFuncSetAttribute(k_tile_solve_ring<float, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b));
            k_tile_solve_ring<float, 2><<<tb.P, TPB, b, s>>>(
                tb.tiles_f.p, tb.dinv_f.p, tb.d_kb.p, tb.d_K.p, tb.d_toff.p, tb.d_roff.p, X, ldx, ncols, skip, gdone);
        } else {
            size_t b = ring_smem_bytes<double, 2>(ldx);
            MSDD_CUDA(cudaFuncSetAttribute(k_tile_solve_ring<double, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b));
            k_tile_solve_ring<double, 2><<<tb.P, TPB, b, s>>>(
                tb.tiles_d.p, tb.dinv_d.p, tb.d_kb.p, tb.d_K.p, tb.d_toff.p, tb.d_roff.p, X, ldx, ncols, skip, gdone);
        }
        MSDD_LAUNCH_CHECK();
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
