// msdd_band_solve_noalloc: the batched band solve without any device
// allocation in the call.  Its staging buffer is a fixed file-scope device
// array instead of memory from cudaMalloc (declaration and contract in
// include/msdd.h).
#include <mutex>

#include "capi_types.cuh"

namespace {

// 2^21 doubles = 16 MiB on every device where the library's module is loaded.
constexpr long long kScratchDoubles = 1LL << 21;
__device__ __align__(256) double g_band_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
double* g_scratch_addr[kMaxDevices] = {};

// The device address of the scratch array on the current device, looked up
// once per device with that device current (host code cannot use the symbol
// itself as a pointer).  With lazy module loading the lookup is also what
// loads this file's module on the device, so the driver commits the array's
// memory here; an out-of-memory failure surfaces as a CudaError whose text
// the status mapping turns into MSDD_ERR_OOM.
double* scratch_address() {
    int dev = 0;
    MSDD_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices)
        throw msdd::MsddError(MSDD_ERR_UNSUPPORTED, "device index beyond the scratch table");
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        MSDD_CUDA(cudaGetSymbolAddress(&p, g_band_scratch));
        g_scratch_addr[dev] = static_cast<double*>(p);
    }
    return g_scratch_addr[dev];
}

// stage <- X for every problem (one CTA column per problem, blockIdx.x),
// padding rows of each problem zeroed.
__global__ void k_stage_in(const double* __restrict__ X, double* __restrict__ stage, const int* __restrict__ n_,
                           const int* __restrict__ K_, const long long* __restrict__ roff_, int nmax, int nrhs) {
    const int i = blockIdx.x;
    const int n = n_[i];
    const long long rows = (long long)K_[i] * msdd::NB;
    const long long base = roff_[i] * nrhs;
    const double* src = X + (long long)i * nmax * nrhs;
    for (long long e = threadIdx.x; e < rows * nrhs; e += blockDim.x) {
        long long r = e / nrhs;
        stage[base + e] = r < n ? src[e] : 0.0;
    }
}

// X <- stage on the n[i] real rows of every problem.
__global__ void k_stage_out(double* __restrict__ X, const double* __restrict__ stage, const int* __restrict__ n_,
                            const long long* __restrict__ roff_, int nmax, int nrhs) {
    const int i = blockIdx.x;
    const long long len = (long long)n_[i] * nrhs;
    const long long base = roff_[i] * nrhs;
    double* dst = X + (long long)i * nmax * nrhs;
    for (long long e = threadIdx.x; e < len; e += blockDim.x) dst[e] = stage[base + e];
}

struct SolveArgs {
    const msdd_band_batch* bb;
    int nrhs;
    double* X;
    void* stream;
};

msdd_status solve_noalloc(void* ctx) {
    const SolveArgs& a = *static_cast<const SolveArgs*>(ctx);
    const msdd_band_batch* bb = a.bb;
    if (!bb || !a.X || a.nrhs < 1 || a.nrhs > msdd::PMAX)
        return msdd::set_last_error(MSDD_ERR_INVALID_ARG, "invalid band solve arguments");
    const long long need = bb->tb.total_rows * (long long)a.nrhs;
    if (need > kScratchDoubles)
        return msdd::set_last_error(MSDD_ERR_INVALID_ARG,
                                    "batch needs " + std::to_string(need) + " doubles of scratch; the static limit is " +
                                        std::to_string(kScratchDoubles) + " (use msdd_band_solve)");
    double* scratch = scratch_address();
    cudaStream_t st = (cudaStream_t)a.stream;
    const int P = bb->tb.P;
    k_stage_in<<<P, 256, 0, st>>>(a.X, scratch, bb->tb.d_n.p, bb->tb.d_K.p, bb->tb.d_roff.p, bb->nmax, a.nrhs);
    MSDD_LAUNCH_CHECK();
    msdd::tile_solve(bb->tb, scratch, a.nrhs, a.nrhs, nullptr, st);
    k_stage_out<<<P, 256, 0, st>>>(a.X, scratch, bb->tb.d_n.p, bb->tb.d_roff.p, bb->nmax, a.nrhs);
    MSDD_LAUNCH_CHECK();
    MSDD_CUDA(cudaStreamSynchronize(st));
    msdd::tile_check_waits();
    return MSDD_OK;
}

}  // namespace

extern "C" msdd_status msdd_band_solve_noalloc(const msdd_band_batch* bb, int nrhs, double* X, void* stream) {
    SolveArgs a{bb, nrhs, X, stream};
    return msdd::classified_call(solve_noalloc, &a);
}
