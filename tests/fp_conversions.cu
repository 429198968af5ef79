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
