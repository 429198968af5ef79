// Test-only probe (built by tests/test_gpu_conversions.py on the GPU host):
// runs the library's integer-pipe conversions f64_to_f32 / f32_to_f64 and
// CUDA's own conversions on the same inputs and returns both bit patterns.
#include <cstdint>

#include "common.cuh"

__global__ void k_conv(const double* __restrict__ xd, const float* __restrict__ xf, int n, float* __restrict__ ours_f,
                       float* __restrict__ cuda_f, double* __restrict__ ours_d, double* __restrict__ cuda_d) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    ours_f[i] = msdd::f64_to_f32(xd[i]);
    cuda_f[i] = __double2float_rn(xd[i]);
    ours_d[i] = msdd::f32_to_f64(xf[i]);
    cuda_d[i] = (double)xf[i];
}

// all pointers device memory of n entries; returns a cudaError_t value
extern "C" int conv_probe(const double* xd, const float* xf, int n, float* ours_f, float* cuda_f, double* ours_d,
                          double* cuda_d) {
    if (n <= 0) return 0;
    k_conv<<<(n + 255) / 256, 256>>>(xd, xf, n, ours_f, cuda_f, ours_d, cuda_d);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return (int)e;
    return (int)cudaDeviceSynchronize();
}

// the double-float helpers: split_f64 of every input, and row dot products
// sum_j (a_rj)(b_rj) accumulated with df_fma (rows of length len)
__global__ void k_df(const double* __restrict__ x, int n, float* __restrict__ hi, float* __restrict__ lo,
                     const double* __restrict__ a, const double* __restrict__ b, int rows, int len,
                     double* __restrict__ dot) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) msdd::split_f64(x[i], hi[i], lo[i]);
    if (i < rows) {
        float sh = 0.f, sl = 0.f;
        for (int j = 0; j < len; ++j) {
            float ah, al, bh, bl;
            msdd::split_f64(a[(long long)i * len + j], ah, al);
            msdd::split_f64(b[(long long)i * len + j], bh, bl);
            msdd::df_fma(sh, sl, ah, al, bh, bl);
        }
        dot[i] = msdd::df_to_f64(sh, sl);
    }
}

extern "C" int df_probe(const double* x, int n, float* hi, float* lo, const double* a, const double* b, int rows,
                        int len, double* dot) {
    const int m = n > rows ? n : rows;
    if (m <= 0) return 0;
    k_df<<<(m + 255) / 256, 256>>>(x, n, hi, lo, a, b, rows, len, dot);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return (int)e;
    return (int)cudaDeviceSynchronize();
}
