// Caching device allocator behind DevBuf (see common.cuh).
//
// A released block is not handed back to the driver: it waits in a pending
// list until the next safe point, where the device is synchronised once and
// pending blocks become free for reuse by allocations of the same rounded
// size.  Set-up and tear-down of a hierarchy therefore stop paying a
// cudaMalloc per buffer and a device-synchronising cudaFree per temporary
// once the sizes have been seen, and no block is ever reused while a kernel
// launched before its release may still read it.
#include "common.cuh"

#include <map>
#include <mutex>
#include <thread>
#include <utility>
#include <vector>

namespace msdd {

namespace {

// A parked block with the release order number and the releasing thread:
// a collect moves only blocks released before its device synchronisation
// began, so a block that another thread parks meanwhile (its kernels may
// still run) stays parked.
struct Parked {
    int device;          // -1 for pinned host blocks
    size_t bytes;        // rounded
    void* p;
    unsigned long long seq;
    std::thread::id owner;
};

struct Cache {
    std::mutex mu;
    std::map<std::pair<int, size_t>, std::vector<void*>> free_blocks;   // (device, rounded bytes)
    std::map<size_t, std::vector<void*>> free_host;                      // pinned host blocks
    std::vector<Parked> pending;
    unsigned long long seq = 0;
    size_t held = 0;                                                     // device bytes, free + parked
    std::vector<cudaEvent_t> events;                                     // completed timing events
};

Cache& cache() {
    static Cache* c = new Cache();   // never destroyed: blocks may be released during static destruction
    return *c;
}

// Size classes: multiples of 512 bytes up to 1 MiB; above that a quarter of
// the size's octave (1, 1.25, 1.5, 1.75 times a power of two), so that the
// buffers of problems of different sizes share blocks (at most 25% slack).
size_t rounded(size_t bytes) {
    if (bytes <= (size_t(1) << 20)) return (bytes + 511) & ~size_t(511);
    int top = 63;
    while (!((bytes >> top) & 1)) --top;
    const size_t step = size_t(1) << (top - 2);
    return (bytes + step - 1) & ~(step - 1);
}

int current_device() {
    int d = 0;
    cudaGetDevice(&d);
    return d;
}

}  // namespace

void* dev_cache_alloc(size_t bytes) {
    if (bytes == 0) return nullptr;
    const auto key = std::make_pair(current_device(), rounded(bytes));
    Cache& c = cache();
    {
        std::lock_guard<std::mutex> lk(c.mu);
        auto it = c.free_blocks.find(key);
        if (it != c.free_blocks.end() && !it->second.empty()) {
            void* p = it->second.back();
            it->second.pop_back();
            c.held -= key.second;
            return p;
        }
    }
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, key.second);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        dev_cache_trim();
        e = cudaMalloc(&p, key.second);
    }
    if (e != cudaSuccess) throw CudaError(std::string("cudaMalloc: ") + cudaGetErrorString(e));
    return p;
}

void dev_cache_release(void* p, size_t bytes) {
    if (!p) return;
    Cache& c = cache();
    const int dev = current_device();
    std::lock_guard<std::mutex> lk(c.mu);
    const size_t r = rounded(bytes);
    c.pending.push_back({dev, r, p, c.seq++, std::this_thread::get_id()});
    c.held += r;
}

void* pinned_cache_alloc(size_t bytes) {
    const size_t r = rounded(bytes);
    Cache& c = cache();
    {
        std::lock_guard<std::mutex> lk(c.mu);
        auto it = c.free_host.find(r);
        if (it != c.free_host.end() && !it->second.empty()) {
            void* p = it->second.back();
            it->second.pop_back();
            return p;
        }
    }
    void* p = nullptr;
    const cudaError_t e = cudaHostAlloc(&p, r, cudaHostAllocDefault);
    if (e != cudaSuccess) throw CudaError(std::string("cudaHostAlloc: ") + cudaGetErrorString(e));
    return p;
}

void pinned_cache_release(void* p, size_t bytes) {
    if (!p) return;
    Cache& c = cache();
    std::lock_guard<std::mutex> lk(c.mu);
    c.pending.push_back({-1, rounded(bytes), p, c.seq++, std::this_thread::get_id()});
}

namespace {

// move the parked blocks that `take` selects to the free lists (lock held)
template <class Pred>
void unpark(Cache& c, Pred take) {
    size_t keep = 0;
    for (size_t i = 0; i < c.pending.size(); ++i) {
        const Parked& e = c.pending[i];
        if (!take(e)) {
            c.pending[keep++] = e;
            continue;
        }
        if (e.device < 0) c.free_host[e.bytes].push_back(e.p);
        else c.free_blocks[{e.device, e.bytes}].push_back(e.p);
    }
    c.pending.resize(keep);
}

}  // namespace

void dev_cache_collect() {
    Cache& c = cache();
    unsigned long long upto;
    {
        std::lock_guard<std::mutex> lk(c.mu);
        if (c.pending.empty()) return;
        upto = c.seq;
    }
    cudaDeviceSynchronize();
    std::lock_guard<std::mutex> lk(c.mu);
    unpark(c, [&](const Parked& e) { return e.seq < upto; });
}

void dev_cache_collect_thread() {
    Cache& c = cache();
    const std::thread::id me = std::this_thread::get_id();
    std::lock_guard<std::mutex> lk(c.mu);
    unpark(c, [&](const Parked& e) { return e.owner == me; });
}

void dev_cache_trim() {
    Cache& c = cache();
    unsigned long long upto;
    {
        std::lock_guard<std::mutex> lk(c.mu);
        upto = c.seq;
    }
    cudaDeviceSynchronize();
    std::lock_guard<std::mutex> lk(c.mu);
    unpark(c, [&](const Parked& e) { return e.seq < upto; });
    size_t freed = 0;
    for (auto& kv : c.free_blocks)
        for (void* p : kv.second) {
            cudaFree(p);
            freed += kv.first.second;
        }
    c.free_blocks.clear();
    c.held -= freed;
    for (auto& kv : c.free_host)
        for (void* p : kv.second) cudaFreeHost(p);
    c.free_host.clear();
}

// timing events (default flags), reused across profiled intervals and hierarchies
cudaEvent_t timing_event_get() {
    Cache& c = cache();
    {
        std::lock_guard<std::mutex> lk(c.mu);
        if (!c.events.empty()) {
            cudaEvent_t e = c.events.back();
            c.events.pop_back();
            return e;
        }
    }
    cudaEvent_t e = nullptr;
    const cudaError_t r = cudaEventCreate(&e);
    if (r != cudaSuccess) throw CudaError(std::string("cudaEventCreate: ") + cudaGetErrorString(r));
    return e;
}

void timing_event_put(cudaEvent_t e) {
    if (!e) return;
    Cache& c = cache();
    std::lock_guard<std::mutex> lk(c.mu);
    c.events.push_back(e);
}

void raise_smem_limit(const void* func, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, size_t> limit;
    std::lock_guard<std::mutex> lk(mu);
    size_t& cur = limit[std::make_pair(current_device(), func)];
    if (bytes <= cur) return;
    if (bytes > 48 * 1024)
        MSDD_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    cur = bytes;
}

size_t dev_cache_bytes() {
    Cache& c = cache();
    std::lock_guard<std::mutex> lk(c.mu);
    return c.held;
}

}  // namespace msdd
