// Shared device/host helpers for the msdd CUDA library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <cstdio>
#include <stdexcept>
#include <string>
#include <vector>

namespace msdd {

// Tile edge of the tile-band LDL^T format (Section 4.3's subdomain solver is
// replaced by a batched blocked factorisation; see tile_ldlt.cu).
constexpr int NB = 32;
constexpr int NB2 = NB * NB;
// Maximum block size of the subspace iteration (columns of X, Y).
constexpr int PMAX = 32;

struct CudaError : std::runtime_error {
    explicit CudaError(const std::string& s) : std::runtime_error(s) {}
};

#define MSDD_CUDA(call)                                                                  \
    do {                                                                                 \
        cudaError_t err__ = (call);                                                      \
        if (err__ != cudaSuccess)                                                        \
            throw ::msdd::CudaError(std::string(#call) + ": " + cudaGetErrorString(err__)); \
    } while (0)

// Process-wide count of kernel launches issued by the library (a graph
// launch adds the number of kernels it holds).
long long& kernel_launch_counter();

#define MSDD_LAUNCH_CHECK()                 \
    do {                                    \
        ++::msdd::kernel_launch_counter();  \
        MSDD_CUDA(cudaGetLastError());      \
    } while (0)

// Owning device buffer (cudaMalloc / cudaFree), move-only.
template <typename T>
struct DevBuf {
    T* p = nullptr;
    size_t n = 0;
    DevBuf() = default;
    explicit DevBuf(size_t count) { alloc(count); }
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    DevBuf(DevBuf&& o) noexcept : p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
    DevBuf& operator=(DevBuf&& o) noexcept {
        if (this != &o) { release(); p = o.p; n = o.n; o.p = nullptr; o.n = 0; }
        return *this;
    }
    ~DevBuf() { release(); }
    void alloc(size_t count) {
        release();
        n = count;
        if (count) MSDD_CUDA(cudaMalloc(&p, count * sizeof(T)));
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    void upload(const std::vector<T>& h, cudaStream_t s) {
        alloc(h.size());
        if (n) MSDD_CUDA(cudaMemcpyAsync(p, h.data(), n * sizeof(T), cudaMemcpyHostToDevice, s));
    }
    void zero(cudaStream_t s) {
        if (n) MSDD_CUDA(cudaMemsetAsync(p, 0, n * sizeof(T), s));
    }
    std::vector<T> download(cudaStream_t s) const {
        std::vector<T> h(n);
        if (n) {
            MSDD_CUDA(cudaMemcpyAsync(h.data(), p, n * sizeof(T), cudaMemcpyDeviceToHost, s));
            MSDD_CUDA(cudaStreamSynchronize(s));
        }
        return h;
    }
};

__host__ __device__ inline unsigned ceil_div(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

// Counter-based uniform(-1, 1) numbers (splitmix64 finaliser of a 64-bit key).
__host__ __device__ inline double hash_uniform(uint64_t key) {
    uint64_t z = key + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    return (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

}  // namespace msdd
