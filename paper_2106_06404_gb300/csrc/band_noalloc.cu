// msdd_band_solve_noalloc: the batched band solve without any device
// allocation in the call.  Its staging buffer is a fixed file-scope device
// array instead of memory from cudaMalloc (declaration and contract in
// include/msdd.h).
#include <mutex>

#include "capi_types.cuh"

namespace {

// 2^21 doubles = 16 MiB, reserved on every device that loads the library.
constexpr long long kScratchDoubles = 1LL << 21;
__device__ __align__(256) double g_band_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
double* g_scratch_addr[kMaxDevices] = {};

// The device address of the scratch array on the current device; resolved
// once per device (host code cannot use the symbol itself as a pointer).
cudaError_t scratch_address(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_band_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

// stage <- X for every problem, padding rows of each problem zeroed.
__global__ void k_stage_in(const double* __restrict__ X, double* __restrict__ stage, const int* __restrict__ n_,
                           const int* __restrict__ K_, const long long* __restrict__ roff_, int nmax, int nrhs) {
    const int i = blockIdx.y;
    const int n = n_[i];
    const long long rows = (long long)K_[i] * msdd::NB;
    const long long base = roff_[i] * nrhs;
    const double* src = X + (long long)i * nmax * nrhs;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < rows * nrhs;
         e += (long long)gridDim.x * blockDim.x) {
        long long r = e / nrhs;
        stage[base + e] = r < n ? src[e] : 0.0;
    }
}

// X <- stage on the n[i] real rows of every problem.
__global__ void k_stage_out(double* __restrict__ X, const double* __restrict__ stage, const int* __restrict__ n_,
                            const long long* __restrict__ roff_, int nmax, int nrhs) {
    const int i = blockIdx.y;
    const long long len = (long long)n_[i] * nrhs;
    const long long base = roff_[i] * nrhs;
    double* dst = X + (long long)i * nmax * nrhs;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < len;
         e += (long long)gridDim.x * blockDim.x)
        dst[e] = stage[base + e];
}

msdd_status noalloc_fail(msdd_status s, const std::string& m) { return msdd::set_last_error(s, m); }

}  // namespace

extern "C" msdd_status msdd_band_solve_noalloc(const msdd_band_batch* bb, int nrhs, double* X, void* stream) {
    if (!bb || !X || nrhs < 1 || nrhs > msdd::PMAX)
        return noalloc_fail(MSDD_ERR_INVALID_ARG, "invalid band solve arguments");
    const long long need = bb->tb.total_rows * (long long)nrhs;
    if (need > kScratchDoubles)
        return noalloc_fail(MSDD_ERR_INVALID_ARG,
                            "batch needs " + std::to_string(need) + " doubles of scratch; the static limit is " +
                                std::to_string(kScratchDoubles) + " (use msdd_band_solve)");
    double* scratch = nullptr;
    cudaError_t e = scratch_address(&scratch);
    if (e != cudaSuccess) return noalloc_fail(MSDD_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    cudaStream_t st = (cudaStream_t)stream;
    try {
        const int P = bb->tb.P;
        dim3 grid(64, P);
        k_stage_in<<<grid, 256, 0, st>>>(X, scratch, bb->tb.d_n.p, bb->tb.d_K.p, bb->tb.d_roff.p, bb->nmax, nrhs);
        MSDD_LAUNCH_CHECK();
        msdd::tile_solve(bb->tb, scratch, nrhs, nrhs, nullptr, st);
        k_stage_out<<<grid, 256, 0, st>>>(X, scratch, bb->tb.d_n.p, bb->tb.d_roff.p, bb->nmax, nrhs);
        MSDD_LAUNCH_CHECK();
        MSDD_CUDA(cudaStreamSynchronize(st));
        msdd::tile_check_waits();
    } catch (const msdd::WaitTimeout& ex) {
        return noalloc_fail(MSDD_ERR_TIMEOUT, ex.what());
    } catch (const std::exception& ex) {
        return noalloc_fail(MSDD_ERR_CUDA, ex.what());
    }
    msdd::set_last_error(MSDD_OK, "");
    return MSDD_OK;
}
