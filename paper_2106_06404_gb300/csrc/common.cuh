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
// rows per block of the eigensolver's residual partial sums: entry
// ((i * nblk_max + blk) * 2 + {0, 1}) * PMAX + c holds, for rows
// [32 blk, 32 blk + 32) of problem i and column c, sum |AX - theta BX|^2 and
// sum |BX|^2
constexpr int EIG_ROWBLK = 32;

struct CudaError : std::runtime_error {
    explicit CudaError(const std::string& s) : std::runtime_error(s) {}
};

// A kernel's bounded wait ran out (it recorded the event and returned early).
struct WaitTimeout : std::runtime_error {
    explicit WaitTimeout(const std::string& s) : std::runtime_error(s) {}
};

#define MSDD_CUDA(call)                                                                  \
    do {                                                                                 \
        cudaError_t err__ = (call);                                                      \
        if (err__ != cudaSuccess)                                                        \
            throw ::msdd::CudaError(std::string(#call) + ": " + cudaGetErrorString(err__)); \
    } while (0)

// Count of kernel launches issued by the library from the calling host
// thread (a graph launch adds the number of kernels it holds);
// kernel_launch_flush adds a thread's count to the process total (batch
// workers call it when they end), kernel_launch_total is that total plus the
// calling thread's count.
long long& kernel_launch_counter();
void kernel_launch_flush();
long long kernel_launch_total();

#define MSDD_LAUNCH_CHECK()                                                                      \
    do {                                                                                         \
        ++::msdd::kernel_launch_counter();                                                       \
        const cudaError_t err__ = cudaGetLastError();                                            \
        if (err__ != cudaSuccess)                                                                \
            throw ::msdd::CudaError(std::string("kernel launch (") + ::msdd::base_name(__FILE__) + \
                                    ":" + std::to_string(__LINE__) + "): " + cudaGetErrorString(err__)); \
    } while (0)

// file name without its directories (for messages)
inline const char* base_name(const char* path) {
    const char* b = path;
    for (const char* c = path; *c; ++c)
        if (*c == '/' || *c == '\\') b = c + 1;
    return b;
}

// Caching device allocator (devcache.cu): dev_cache_release parks a block
// until the next dev_cache_collect, which synchronises the device once and
// makes parked blocks reusable by dev_cache_alloc of the same rounded size;
// dev_cache_trim returns everything to the driver.  The C API collects at
// the end of every call that released memory.
void* dev_cache_alloc(size_t bytes);
void dev_cache_release(void* p, size_t bytes);
void dev_cache_collect();
// Make the blocks that the calling thread released reusable without a device
// synchronisation.  Only for a thread that has synchronised every stream on
// which work using those blocks was issued (a batch worker between problems).
void dev_cache_collect_thread();
void dev_cache_trim();
size_t dev_cache_bytes();
// pinned host blocks, same rules (released blocks reusable after a collect)
void* pinned_cache_alloc(size_t bytes);
void pinned_cache_release(void* p, size_t bytes);
// CUDA events with timing, reused (put back only after they completed)
cudaEvent_t timing_event_get();
void timing_event_put(cudaEvent_t e);
// Raise a kernel's dynamic shared-memory limit to at least `bytes` (the
// limit is per function and device, shared by all host threads).  It is
// only ever raised, under a lock, so a launch that another thread sized
// for a smaller amount stays valid.
void raise_smem_limit(const void* func, size_t bytes);
template <class F>
void raise_smem_limit(F* func, size_t bytes) {
    raise_smem_limit(reinterpret_cast<const void*>(func), bytes);
}

// Device buffer (caching allocator above), move-only; borrow() makes a
// non-owning view of another buffer's memory (never freed by the view).
template <typename T>
struct DevBuf {
    T* p = nullptr;
    size_t n = 0;
    bool owned = true;
    DevBuf() = default;
    explicit DevBuf(size_t count) { alloc(count); }
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    DevBuf(DevBuf&& o) noexcept : p(o.p), n(o.n), owned(o.owned) { o.p = nullptr; o.n = 0; o.owned = true; }
    DevBuf& operator=(DevBuf&& o) noexcept {
        if (this != &o) {
            release();
            p = o.p; n = o.n; owned = o.owned;
            o.p = nullptr; o.n = 0; o.owned = true;
        }
        return *this;
    }
    ~DevBuf() { release(); }
    static DevBuf borrow(T* q, size_t count) {
        DevBuf v;
        v.p = q;
        v.n = count;
        v.owned = false;
        return v;
    }
    // view of elements [off, off + count) of this buffer
    DevBuf view(size_t off, size_t count) const { return borrow(p ? p + off : nullptr, count); }
    void alloc(size_t count) {
        release();
        if (count) p = static_cast<T*>(dev_cache_alloc(count * sizeof(T)));
        n = count;
    }
    void release() {
        if (p && owned) dev_cache_release(p, n * sizeof(T));
        p = nullptr;
        n = 0;
        owned = true;
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

// ---- FP64 <-> FP32 conversions on the integer pipe.  On this GPU the
// conversion instructions share the narrow FP64 pipe; these bit-level
// versions, written from the IEEE 754 binary64/binary32 formats, keep
// mixed-precision kernels off it.  Round to nearest even with gradual
// underflow (subnormal results and inputs are exact IEEE), overflow to
// infinity, NaN stays NaN (quiet).
#ifdef __CUDACC__
__device__ __forceinline__ float f64_to_f32(double x) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const unsigned hi = (unsigned)(u >> 32), lo = (unsigned)u;
    const unsigned sign = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7ffu);
    const int ef = e - 1023 + 127;
    const unsigned m = ((hi & 0x000fffffu) << 3) | (lo >> 29);   // leading 23 mantissa bits
    const unsigned rest = lo & 0x1fffffffu;                        // the 29 dropped bits
    unsigned v = ((unsigned)ef << 23) + m;
    v += (rest > 0x10000000u || (rest == 0x10000000u && (m & 1u))) ? 1u : 0u;   // a carry may give infinity
    if (ef <= 0) {
        // subnormal (or zero) result: the significand with its leading one,
        // in units of 2^-149, is sig >> (926 - e); a round-up to 2^23 is the
        // smallest normal number's encoding
        const unsigned long long sig = (1ull << 52) | (u & 0x000fffffffffffffull);
        const int sh = 926 - e;                                   // >= 30 here
        if (sh > 53 || e == 0) {
            v = 0u;
        } else {
            const unsigned long long q = sig >> sh, r = sig & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
            v = (unsigned)q + ((r > half || (r == half && (q & 1ull))) ? 1u : 0u);
        }
    }
    if (ef >= 255) v = (e == 0x7ff && ((hi & 0x000fffffu) | lo)) ? 0x7fc00000u : 0x7f800000u;
    return __uint_as_float(sign | v);
}
__device__ __forceinline__ double f32_to_f64(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned sign = u & 0x80000000u;
    const unsigned e = (u >> 23) & 0xffu;
    const unsigned m = u & 0x007fffffu;
    unsigned hi = sign | ((e + 896u) << 20) | (m >> 3);
    unsigned lo = m << 29;
    if (e == 0u) {
        if (m == 0u) {
            hi = sign;
            lo = 0u;
        } else {
            // subnormal input m 2^-149: leading one at bit p, exponent p - 149
            const unsigned p = 31u - (unsigned)__clz(m);
            const unsigned mn = (m << (23u - p)) & 0x007fffffu;
            hi = sign | ((p + 874u) << 20) | (mn >> 3);
            lo = mn << 29;
        }
    }
    if (e == 0xffu) { hi = sign | 0x7ff00000u | (m >> 3) | (m ? 0x00080000u : 0u); lo = m << 29; }
    return __hiloint2double((int)hi, (int)lo);
}
// ---- double-float arithmetic on the FP32 pipes (Dekker's error-free product
// via FMA, Knuth's two-sum).  A value is the unevaluated sum hi + lo of two
// FP32 numbers with |lo| <= 2^-23 |hi|, about 47 significant bits: enough for
// sums of products whose FP64 results only need ~1e-13 relative accuracy, at a
// dozen FP32 operations per multiply-add instead of one FP64 operation on the
// narrow FP64 pipe.  The _rn intrinsics keep the compiler from contracting
// the error-free steps into FMAs.
//
// FP64 x -> (hi, lo) from the bit fields: hi keeps the leading 24 significand
// bits (truncated, exact in FP32), lo is the remaining 29 bits rounded to FP32,
// so |x - hi - lo| <= 2^-47 |x|.  Exponents outside [2^-60, 2^100] fall back
// to (f64_to_f32(x), 0).
__device__ __forceinline__ void split_f64(double x, float& hi, float& lo) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const unsigned uh = (unsigned)(u >> 32), ul = (unsigned)u;
    const unsigned sign = uh & 0x80000000u;
    const int e = (int)((uh >> 20) & 0x7ffu);
    if (e < 1023 - 60 || e > 1023 + 100) {
        hi = f64_to_f32(x);
        lo = 0.f;
        return;
    }
    hi = __uint_as_float(sign | ((unsigned)(e - 1023 + 127) << 23) | ((uh & 0x000fffffu) << 3) | (ul >> 29));
    // lo = r 2^(e - 1075) with r the 29 dropped bits; the scale is a normal FP32 power of two here
    const float r = __uint2float_rn(ul & 0x1fffffffu);
    lo = __uint_as_float(__float_as_uint(__fmul_rn(r, __uint_as_float((unsigned)(e - 1075 + 127) << 23))) | sign);
}
// (sh, sl) += (ah + al)(bh + bl): the product of the leading parts exactly
// (p + e), the cross terms into e, p into sh by two-sum, the rest into sl
__device__ __forceinline__ void df_fma(float& sh, float& sl, float ah, float al, float bh, float bl) {
    const float p = __fmul_rn(ah, bh);
    float e = __fmaf_rn(ah, bh, -p);
    e = __fmaf_rn(ah, bl, e);
    e = __fmaf_rn(al, bh, e);
    const float s = __fadd_rn(sh, p);
    const float bb = __fsub_rn(s, sh);
    const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    sh = s;
    sl = __fadd_rn(sl, __fadd_rn(err, e));
}
__device__ __forceinline__ double df_to_f64(float hi, float lo) { return f32_to_f64(hi) + f32_to_f64(lo); }

// load a double as T / store a T as double
template <typename T> __device__ __forceinline__ T from_f64(double x);
template <> __device__ __forceinline__ double from_f64<double>(double x) { return x; }
template <> __device__ __forceinline__ float from_f64<float>(double x) { return f64_to_f32(x); }
__device__ __forceinline__ double to_f64(double x) { return x; }
__device__ __forceinline__ double to_f64(float x) { return f32_to_f64(x); }
#endif

}  // namespace msdd
