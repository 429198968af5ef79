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
#include <utility>
#include <vector>

namespace msdd {

namespace {

struct Cache {
    std::mutex mu;
    std::map<std::pair<int, size_t>, std::vector<void*>> free_blocks;   // (device, rounded bytes)
    std::vector<std::pair<std::pair<int, size_t>, void*>> pending;
    size_t held = 0;                                                     // bytes in both lists
    // pinned host blocks: same rules (device -1)
    std::map<size_t, std::vector<void*>> free_host;
    std::vector<std::pair<size_t, void*>> pending_host;
    std::vector<cudaEvent_t> events;                                     // completed timing events
};

Cache& cache() {
    static Cache* c = new Cache();   // never destroyed: blocks may be released during static destruction
    return *c;
}

size_t rounded(size_t bytes) { return (bytes + 511) & ~size_t(511); }

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
    std::lock_guard<std::mutex> lk(c.mu);
    const size_t r = rounded(bytes);
    c.pending.push_back({{current_device(), r}, p});
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
    c.pending_host.push_back({rounded(bytes), p});
}

void dev_cache_collect() {
    Cache& c = cache();
    {
        std::lock_guard<std::mutex> lk(c.mu);
        if (c.pending.empty() && c.pending_host.empty()) return;
    }
    cudaDeviceSynchronize();
    std::lock_guard<std::mutex> lk(c.mu);
    for (auto& e : c.pending) c.free_blocks[e.first].push_back(e.second);
    c.pending.clear();
    for (auto& e : c.pending_host) c.free_host[e.first].push_back(e.second);
    c.pending_host.clear();
}

void dev_cache_trim() {
    cudaDeviceSynchronize();
    Cache& c = cache();
    std::lock_guard<std::mutex> lk(c.mu);
    for (auto& e : c.pending) c.free_blocks[e.first].push_back(e.second);
    c.pending.clear();
    for (auto& kv : c.free_blocks)
        for (void* p : kv.second) cudaFree(p);
    c.free_blocks.clear();
    c.held = 0;
    for (auto& e : c.pending_host) c.free_host[e.first].push_back(e.second);
    c.pending_host.clear();
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

size_t dev_cache_bytes() {
    Cache& c = cache();
    std::lock_guard<std::mutex> lk(c.mu);
    return c.held;
}

}  // namespace msdd
