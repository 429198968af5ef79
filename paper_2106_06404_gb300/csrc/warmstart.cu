// Learned warm start: patches, MLP forward/backward, loss, Adam, start
// vectors and training targets (see warmstart.cuh and include/msdd.h).
#include "warmstart.cuh"

namespace msdd {

namespace {

constexpr double NN_EPS = 1e-6;     // ridge of the least-squares fit in the loss

// round to the nearest bfloat16, ties to even (integer form of the definition)
__device__ __forceinline__ float bf16_rne(float x) {
    unsigned u = __float_as_uint(x);
    if ((u & 0x7f800000u) == 0x7f800000u) return x;
    u += 0x7fffu + ((u >> 16) & 1u);
    return __uint_as_float(u & 0xffff0000u);
}

// ---- patches: area average of log10 kappa over PATCH x PATCH equal cells of
// the element box, minus the patch mean, divided by 6
__global__ void __launch_bounds__(256) k_nn_patch(Geom g, const ProbBox* __restrict__ boxes, float* __restrict__ X) {
    __shared__ double red[256];
    const int i = blockIdx.x, t = threadIdx.x;
    const ProbBox b = boxes[i];
    const int w = b.ehi[0] - b.elo[0], h = b.ehi[1] - b.elo[1];
    double vals[(NN_IN + 255) / 256];
    double part = 0.0;
    int nc = 0;
    for (int c = t; c < NN_IN; c += 256, ++nc) {
        const int I = c / NN_PATCH, J = c % NN_PATCH;
        const double ya = (double)I * h / NN_PATCH, yb = (double)(I + 1) * h / NN_PATCH;
        const double xa = (double)J * w / NN_PATCH, xb = (double)(J + 1) * w / NN_PATCH;
        double s = 0.0;
        for (int ey = (int)floor(ya); ey < min(h, (int)ceil(yb)); ++ey) {
            const double oy = fmin(yb, ey + 1.0) - fmax(ya, (double)ey);
            if (!(oy > 0.0)) continue;
            for (int ex = (int)floor(xa); ex < min(w, (int)ceil(xb)); ++ex) {
                const double ox = fmin(xb, ex + 1.0) - fmax(xa, (double)ex);
                if (!(ox > 0.0)) continue;
                const long long e = (b.elo[0] + ex) + (long long)g.n[0] * (b.elo[1] + ey);
                s += ox * oy * log10(g.coeff[e]);
            }
        }
        vals[nc] = s / ((xb - xa) * (yb - ya));
        part += vals[nc];
    }
    red[t] = part;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (t < o) red[t] += red[t + o];
        __syncthreads();
    }
    const double mean = red[0] / NN_IN;
    nc = 0;
    for (int c = t; c < NN_IN; c += 256, ++nc) X[(long long)i * NN_IN + c] = (float)((vals[nc] - mean) / 6.0);
}

// ---- C[M][N] = epilogue(sum_k A(m,k) B(n,k)); A(m,k) = TA ? A[k lda + m] : A[m lda + k],
// B(n,k) = TB ? B[k ldb + n] : B[n ldb + k]; RB rounds B to bfloat16 (weights);
// EPI: 0 store, 1 add bias[n].
//
// BF16 tensor cores (mma.m16n8k16, FP32 accumulate).  An FP32 operand is
// split into three bfloat16 terms x = h + m + l (each the round-to-nearest
// of what the previous ones leave; together the 24 significand bits), so a
// product with a bfloat16 weight is formed exactly from three mma (h, m, l
// against the weight) and the arithmetic is that of FP32 products with the
// BF16-rounded weights.  Two FP32 operands (the weight gradients) take the
// six terms with index sum <= 2 (the rest are below 2^-24 of the product).
// 64 x 64 tile per CTA, 8 warps of 32 x 16 (2 x 2 mma tiles), k-steps of 16
// staged in shared memory as FP32.
__device__ __forceinline__ void bf16_split3(float x, unsigned (&t)[3]) {
    const float h = bf16_rne(x);
    const float r1 = __fsub_rn(x, h);
    const float m = bf16_rne(r1);
    const float l = bf16_rne(__fsub_rn(r1, m));
    t[0] = __float_as_uint(h) >> 16;
    t[1] = __float_as_uint(m) >> 16;
    t[2] = __float_as_uint(l) >> 16;
}
__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
    asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
template <bool TA, bool TB, bool RB, int EPI>
__global__ void __launch_bounds__(256) k_nn_gemm(int M, int N, int K, const float* __restrict__ A, int lda,
                                                 const float* __restrict__ B, int ldb, const float* __restrict__ bias,
                                                 float* __restrict__ C, int ldc) {
    __shared__ float As[16][65], Bs[16][65];
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31, g = lane >> 2, q = lane & 3;
    const int wm = (warp & 1) * 32, wn = (warp >> 1) * 16;       // this warp's 32 x 16 block of the tile
    float acc[2][2][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[i][j][c] = 0.f;
    constexpr int NB_TERMS = RB ? 1 : 3;
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int e = t; e < 16 * 64; e += 256) {
            const int kk = TA ? e / 64 : e % 16, mm = TA ? e % 64 : e / 16;
            const int m = m0 + mm, k = k0 + kk;
            As[kk][mm] = (m < M && k < K) ? (TA ? A[(long long)k * lda + m] : A[(long long)m * lda + k]) : 0.f;
            const int kb = TB ? e / 64 : e % 16, nb = TB ? e % 64 : e / 16;
            const int n = n0 + nb, k2 = k0 + kb;
            float bv = (n < N && k2 < K) ? (TB ? B[(long long)k2 * ldb + n] : B[(long long)n * ldb + k2]) : 0.f;
            Bs[kb][nb] = RB ? bf16_rne(bv) : bv;
        }
        __syncthreads();
        // fragments: A (16 x 16): (g, 2q..2q+1), (g + 8, ..), (g, 2q + 8..), (g + 8, 2q + 8..);
        // B (16 x 8): k 2q..2q+1 and 2q + 8..2q + 9 of column g; two bfloat16 a register, low = first
        unsigned af[2][3][4], bfr[2][3][2];
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int r = wm + 16 * i + g;
            const int rows[4] = {r, r + 8, r, r + 8}, ks[4] = {2 * q, 2 * q, 2 * q + 8, 2 * q + 8};
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                unsigned lo[3], hi[3];
                bf16_split3(As[ks[v]][rows[v]], lo);
                bf16_split3(As[ks[v] + 1][rows[v]], hi);
#pragma unroll
                for (int z = 0; z < 3; ++z) af[i][z][v] = lo[z] | (hi[z] << 16);
            }
        }
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int c = wn + 8 * j + g;
#pragma unroll
            for (int v = 0; v < 2; ++v) {
                const int kb = 2 * q + 8 * v;
                unsigned lo[3], hi[3];
                if (RB) {
                    lo[0] = __float_as_uint(Bs[kb][c]) >> 16;       // already bfloat16
                    hi[0] = __float_as_uint(Bs[kb + 1][c]) >> 16;
                } else {
                    bf16_split3(Bs[kb][c], lo);
                    bf16_split3(Bs[kb + 1][c], hi);
                }
#pragma unroll
                for (int z = 0; z < NB_TERMS; ++z) bfr[j][z][v] = lo[z] | (hi[z] << 16);
            }
        }
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                if (RB) {
                    // smallest terms first
                    mma_bf16(acc[i][j], af[i][2], bfr[j][0][0], bfr[j][0][1]);
                    mma_bf16(acc[i][j], af[i][1], bfr[j][0][0], bfr[j][0][1]);
                    mma_bf16(acc[i][j], af[i][0], bfr[j][0][0], bfr[j][0][1]);
                } else {
                    mma_bf16(acc[i][j], af[i][2], bfr[j][0][0], bfr[j][0][1]);
                    mma_bf16(acc[i][j], af[i][1], bfr[j][1][0], bfr[j][1][1]);
                    mma_bf16(acc[i][j], af[i][0], bfr[j][2][0], bfr[j][2][1]);
                    mma_bf16(acc[i][j], af[i][1], bfr[j][0][0], bfr[j][0][1]);
                    mma_bf16(acc[i][j], af[i][0], bfr[j][1][0], bfr[j][1][1]);
                    mma_bf16(acc[i][j], af[i][0], bfr[j][0][0], bfr[j][0][1]);
                }
            }
        __syncthreads();
    }
    // C fragments: (g, 2q), (g, 2q + 1), (g + 8, 2q), (g + 8, 2q + 1) of each 16 x 8 tile
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int m = m0 + wm + 16 * i + g + (c >> 1) * 8, n = n0 + wn + 8 * j + 2 * q + (c & 1);
                if (m >= M || n >= N) continue;
                float v = acc[i][j][c];
                if (EPI == 1) v += bias[n];
                C[(long long)m * ldc + n] = v;
            }
}

template <bool TA, bool TB, bool RB, int EPI>
void gemm(int M, int N, int K, const float* A, int lda, const float* B, int ldb, const float* bias, float* C, int ldc,
          cudaStream_t s) {
    dim3 grid((N + 63) / 64, (M + 63) / 64);
    k_nn_gemm<TA, TB, RB, EPI><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, bias, C, ldc);
    MSDD_LAUNCH_CHECK();
}

__global__ void k_nn_relu(const float* __restrict__ a, float* __restrict__ h, long long n) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        h[e] = fmaxf(a[e], 0.f);
}
// d <- d * (a > 0)
__global__ void k_nn_relu_back(const float* __restrict__ a, float* __restrict__ d, long long n) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        if (!(a[e] > 0.f)) d[e] = 0.f;
}
// db[n] = sum_m D[m][n] (fixed order)
__global__ void k_nn_colsum(const float* __restrict__ D, int M, int N, float* __restrict__ db) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.f;
    for (int m = 0; m < M; ++m) s += D[(long long)m * N + n];
    db[n] = s;
}

// ---- loss of one sample per CTA: Y (GRID^2 x NVEC) from the network output,
// T unit targets, C = (Y^T Y + eps I)^{-1} Y^T T, R = T - Y C,
// L = (|R|^2 + eps |C|^2) / m, dY = -2 R C^T / (m S)
__global__ void __launch_bounds__(128) k_nn_loss(const float* __restrict__ Yo, const float* __restrict__ T,
                                                 const int* __restrict__ mcnt, int S, double* __restrict__ lossv,
                                                 float* __restrict__ dY) {
    constexpr int NV = NN_NVEC, LDV = NN_NVEC + 1;
    __shared__ double Yd[NN_G2][LDV], Td[NN_G2][LDV];
    __shared__ double G[NV][LDV], Bm[NV][LDV], C[NV][LDV];
    __shared__ double red[128];
    const int s = blockIdx.x, t = threadIdx.x;
    const int m = min(mcnt[s], NV);
    for (int e = t; e < NN_G2 * NV; e += 128) {
        const int k = e / NN_G2, gi = e % NN_G2;
        Yd[gi][k] = Yo[(long long)s * NN_OUT + e];
        Td[gi][k] = k < m ? T[((long long)s * NV + k) * NN_G2 + gi] : 0.0;
    }
    __syncthreads();
    for (int e = t; e < 2 * NV * NV; e += 128) {
        const int which = e / (NV * NV), a = (e % (NV * NV)) / NV, b = e % NV;
        double v = 0.0;
        if (which == 0) {
            for (int gi = 0; gi < NN_G2; ++gi) v += Yd[gi][a] * Yd[gi][b];
            G[a][b] = v + (a == b ? NN_EPS : 0.0);
        } else {
            for (int gi = 0; gi < NN_G2; ++gi) v += Yd[gi][a] * Td[gi][b];
            Bm[a][b] = v;
        }
    }
    __syncthreads();
    if (t < 32) {
        const int lane = t;
        for (int k = 0; k < NV; ++k) {                       // Cholesky, lane = row
            const double lkk = sqrt(G[k][k]);
            __syncwarp();
            if (lane == k) G[k][k] = lkk;
            if (lane > k && lane < NV) G[lane][k] /= lkk;
            __syncwarp();
            if (lane > k && lane < NV)
                for (int b = k + 1; b <= lane; ++b) G[lane][b] -= G[lane][k] * G[b][k];
            __syncwarp();
        }
        if (lane < m) {                                      // C = G^{-1} Bm, lane = column
            for (int a = 0; a < NV; ++a) {
                double v = Bm[a][lane];
                for (int j = 0; j < a; ++j) v -= G[a][j] * C[j][lane];
                C[a][lane] = v / G[a][a];
            }
            for (int a = NV - 1; a >= 0; --a) {
                double v = C[a][lane];
                for (int j = a + 1; j < NV; ++j) v -= G[j][a] * C[j][lane];
                C[a][lane] = v / G[a][a];
            }
        }
    }
    __syncthreads();
    double part = 0.0;
    for (int e = t; e < NN_G2 * NV; e += 128) {              // R into Td
        const int gi = e / NV, b = e % NV;
        if (b >= m) continue;
        double r = Td[gi][b];
        for (int a = 0; a < NV; ++a) r -= Yd[gi][a] * C[a][b];
        Td[gi][b] = r;
        part += r * r;
    }
    for (int e = t; e < NV * NV; e += 128)
        if (e % NV < m) part += NN_EPS * C[e / NV][e % NV] * C[e / NV][e % NV];
    red[t] = part;
    __syncthreads();
    for (int o = 64; o > 0; o >>= 1) {
        if (t < o) red[t] += red[t + o];
        __syncthreads();
    }
    if (t == 0) lossv[s] = m > 0 ? red[0] / m : 0.0;
    const double sc = m > 0 ? -2.0 / ((double)m * S) : 0.0;
    for (int e = t; e < NN_G2 * NV; e += 128) {
        const int k = e / NN_G2, gi = e % NN_G2;
        double v = 0.0;
        for (int b = 0; b < m; ++b) v += Td[gi][b] * C[k][b];
        dY[(long long)s * NN_OUT + e] = (float)(sc * v);
    }
}

__global__ void k_nn_mean(const double* __restrict__ v, int S, double* __restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < S; ++i) s += v[i];
        *out = s / S;
    }
}

__global__ void k_nn_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m1,
                          float* __restrict__ m2, long long n, float lr, float c1, float c2) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const float gv = g[e];
        const float a = b1 * m1[e] + (1.f - b1) * gv;
        const float b = b2 * m2[e] + (1.f - b2) * gv * gv;
        m1[e] = a;
        m2[e] = b;
        p[e] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
    }
}

// ---- grid vectors -> node values of each box (x fastest), NVEC columns
__global__ void k_nn_start(const ProbBox* __restrict__ boxes, const long long* __restrict__ off, int dim,
                           const float* __restrict__ Y, double* __restrict__ out) {
    const int i = blockIdx.y;
    const ProbBox b = boxes[i];
    const int nx = b.nhi[0] - b.nlo[0] + 1, ny = dim >= 2 ? b.nhi[1] - b.nlo[1] + 1 : 1;
    const float* Yi = Y + (long long)i * NN_OUT;
    const int s = NN_GRID - 1;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nx * ny; r += gridDim.x * blockDim.x) {
        const int x = r % nx, y = r / nx;
        const double u = nx > 1 ? (double)x / (nx - 1) : 0.0, v = ny > 1 ? (double)y / (ny - 1) : 0.0;
        const double fx = u * s, fy = v * s;
        const int ix = min((int)floor(fx), s - 1), iy = min((int)floor(fy), s - 1);
        const double tx = fx - ix, ty = fy - iy;
        for (int k = 0; k < NN_NVEC; ++k) {
            const float* G = Yi + k * NN_G2;
            const double val = (1 - tx) * (1 - ty) * G[iy * NN_GRID + ix] + tx * (1 - ty) * G[iy * NN_GRID + ix + 1] +
                               (1 - tx) * ty * G[(iy + 1) * NN_GRID + ix] + tx * ty * G[(iy + 1) * NN_GRID + ix + 1];
            out[(off[i] + r) * NN_NVEC + k] = val;
        }
    }
}

// ---- targets: eigenvector k < m of box i sampled at the grid points by
// bilinear interpolation of its node grid, unit 2-norm
__global__ void __launch_bounds__(128) k_nn_targets(const ProbBox* __restrict__ boxes, const long long* __restrict__ roff,
                                                    const int* __restrict__ mm, int dim, const double* __restrict__ X,
                                                    int ldx, float* __restrict__ T, int* __restrict__ mout) {
    __shared__ double col[NN_G2];
    __shared__ double red[128];
    const int i = blockIdx.x, t = threadIdx.x;
    const ProbBox b = boxes[i];
    const int nx = b.nhi[0] - b.nlo[0] + 1, ny = dim >= 2 ? b.nhi[1] - b.nlo[1] + 1 : 1;
    const int m = min(mm[i], NN_NVEC);
    for (int k = 0; k < NN_NVEC; ++k) {
        float* Tk = T + ((long long)i * NN_NVEC + k) * NN_G2;
        if (k >= m) {
            for (int gi = t; gi < NN_G2; gi += 128) Tk[gi] = 0.f;
            continue;
        }
        double part = 0.0;
        for (int gi = t; gi < NN_G2; gi += 128) {
            const int gx = gi % NN_GRID, gy = gi / NN_GRID;
            const double fx = (double)gx / (NN_GRID - 1) * (nx - 1), fy = (double)gy / (NN_GRID - 1) * (ny - 1);
            const int ix = min((int)floor(fx), max(nx - 2, 0)), iy = min((int)floor(fy), max(ny - 2, 0));
            const double tx = fx - ix, ty = fy - iy;
            auto at = [&](int yy, int xx) { return X[(roff[i] + (long long)yy * nx + xx) * ldx + k]; };
            const double v = (1 - tx) * (1 - ty) * at(iy, ix) + tx * (1 - ty) * at(iy, ix + 1) +
                             (1 - tx) * ty * at(iy + 1, ix) + tx * ty * at(iy + 1, ix + 1);
            col[gi] = v;
            part += v * v;
        }
        red[t] = part;
        __syncthreads();
        for (int o = 64; o > 0; o >>= 1) {
            if (t < o) red[t] += red[t + o];
            __syncthreads();
        }
        const double inv = red[0] > 0.0 ? 1.0 / sqrt(red[0]) : 0.0;
        for (int gi = t; gi < NN_G2; gi += 128) Tk[gi] = (float)(col[gi] * inv);
        __syncthreads();
    }
    if (t == 0) mout[i] = m;
}

unsigned vblocks(long long n) { return (unsigned)std::max(1LL, std::min<long long>((n + 255) / 256, 152 * 8)); }

struct Work {
    float *a1, *h1, *a2, *h2, *y, *dy, *dh, *da;
    double* lossv;
};
Work carve(float* w, int S) {
    Work k;
    const long long sh = (long long)S * NN_H, so = (long long)S * NN_OUT;
    k.a1 = w; k.h1 = k.a1 + sh; k.a2 = k.h1 + sh; k.h2 = k.a2 + sh;
    k.y = k.h2 + sh; k.dy = k.y + so; k.dh = k.dy + so; k.da = k.dh + sh;
    // lossv: S doubles after da, 8-byte aligned
    long long off = (k.da + sh) - w;
    off = (off + 1) & ~1LL;
    k.lossv = reinterpret_cast<double*>(w + off);
    return k;
}

void forward_into(const float* P, int S, const float* X, Work& k, float* y, cudaStream_t s) {
    gemm<false, false, true, 1>(S, NN_H, NN_IN, X, NN_IN, P + NN_W1, NN_IN, P + NN_B1, k.a1, NN_H, s);
    k_nn_relu<<<vblocks((long long)S * NN_H), 256, 0, s>>>(k.a1, k.h1, (long long)S * NN_H);
    MSDD_LAUNCH_CHECK();
    gemm<false, false, true, 1>(S, NN_H, NN_H, k.h1, NN_H, P + NN_W2, NN_H, P + NN_B2, k.a2, NN_H, s);
    k_nn_relu<<<vblocks((long long)S * NN_H), 256, 0, s>>>(k.a2, k.h2, (long long)S * NN_H);
    MSDD_LAUNCH_CHECK();
    gemm<false, false, true, 1>(S, NN_OUT, NN_H, k.h2, NN_H, P + NN_W3, NN_H, P + NN_B3, y, NN_OUT, s);
}

}  // namespace

size_t nn_workspace_floats(int S) { return (size_t)6 * S * NN_H + (size_t)2 * S * NN_OUT + 2 * (size_t)S + 2; }

void nn_patches(const Geom& g, const ProbBox* d_boxes, int P, float* X, cudaStream_t s) {
    if (P == 0) return;
    k_nn_patch<<<P, 256, 0, s>>>(g, d_boxes, X);
    MSDD_LAUNCH_CHECK();
}

void nn_forward(const float* params, int S, const float* X, float* out, float* work, cudaStream_t s) {
    Work k = carve(work, S);
    forward_into(params, S, X, k, out, s);
}

void nn_loss_grad(const float* P, int S, const float* X, const float* T, const int* m, double* loss, float* grad,
                  float* work, cudaStream_t s) {
    Work k = carve(work, S);
    forward_into(P, S, X, k, k.y, s);
    k_nn_loss<<<S, 128, 0, s>>>(k.y, T, m, S, k.lossv, k.dy);
    MSDD_LAUNCH_CHECK();
    k_nn_mean<<<1, 32, 0, s>>>(k.lossv, S, loss);
    MSDD_LAUNCH_CHECK();
    // layer 3
    gemm<true, true, false, 0>(NN_OUT, NN_H, S, k.dy, NN_OUT, k.h2, NN_H, nullptr, grad + NN_W3, NN_H, s);
    k_nn_colsum<<<(NN_OUT + 255) / 256, 256, 0, s>>>(k.dy, S, NN_OUT, grad + NN_B3);
    MSDD_LAUNCH_CHECK();
    gemm<false, true, true, 0>(S, NN_H, NN_OUT, k.dy, NN_OUT, P + NN_W3, NN_H, nullptr, k.dh, NN_H, s);
    k_nn_relu_back<<<vblocks((long long)S * NN_H), 256, 0, s>>>(k.a2, k.dh, (long long)S * NN_H);
    MSDD_LAUNCH_CHECK();
    // layer 2 (k.dh = d a2)
    gemm<true, true, false, 0>(NN_H, NN_H, S, k.dh, NN_H, k.h1, NN_H, nullptr, grad + NN_W2, NN_H, s);
    k_nn_colsum<<<1, 256, 0, s>>>(k.dh, S, NN_H, grad + NN_B2);
    MSDD_LAUNCH_CHECK();
    gemm<false, true, true, 0>(S, NN_H, NN_H, k.dh, NN_H, P + NN_W2, NN_H, nullptr, k.da, NN_H, s);
    k_nn_relu_back<<<vblocks((long long)S * NN_H), 256, 0, s>>>(k.a1, k.da, (long long)S * NN_H);
    MSDD_LAUNCH_CHECK();
    // layer 1 (k.da = d a1)
    gemm<true, true, false, 0>(NN_H, NN_IN, S, k.da, NN_H, X, NN_IN, nullptr, grad + NN_W1, NN_IN, s);
    k_nn_colsum<<<1, 256, 0, s>>>(k.da, S, NN_H, grad + NN_B1);
    MSDD_LAUNCH_CHECK();
}

void nn_adam(float* params, const float* grad, float* m1, float* m2, int t, float lr, cudaStream_t s) {
    const float c1 = 1.f - powf(0.9f, (float)t), c2 = 1.f - powf(0.999f, (float)t);
    k_nn_adam<<<vblocks(NN_NPARAM), 256, 0, s>>>(params, grad, m1, m2, NN_NPARAM, lr, c1, c2);
    MSDD_LAUNCH_CHECK();
}

void nn_start_vectors(const ProbBox* d_boxes, const long long* d_off, int P, int dim, const float* Y, double* out,
                      cudaStream_t s) {
    if (P == 0) return;
    dim3 grid(8, P);
    k_nn_start<<<grid, 256, 0, s>>>(d_boxes, d_off, dim, Y, out);
    MSDD_LAUNCH_CHECK();
}

void nn_targets(const ProbBox* d_boxes, const long long* d_roff, const int* d_m, int P, int dim, const double* X,
                int ldx, float* T, int* mout, cudaStream_t s) {
    if (P == 0) return;
    k_nn_targets<<<P, 128, 0, s>>>(d_boxes, d_roff, d_m, dim, X, ldx, T, mout);
    MSDD_LAUNCH_CHECK();
}

}  // namespace msdd
