// Cache of large host buffers behind the instances' host arrays (the copy of
// the ILP each instance keeps, and the host plan's arrays).
//
// Large allocations come from fresh pages, and touching them for the first
// time costs page faults (writing 331 MB of fresh pages took 17-20 ms on one
// core of the GB300's host), and freeing them unmaps them again.  For the
// 327 MB copy of the 512x512 grid's ILP that every instance of it makes,
// creation spread over 16 host threads took 8-9 ms either way there, while
// destroying an instance went from 2.7 to 0.9 ms (on an 8-core x86 host,
// creation went from 40-50 ms to 20 ms).  Buffers freed by an
// instance are kept here, keyed by their size rounded up to 64 KB, and handed
// to the next allocation of that size.  Kept bytes are capped; what does not
// fit is returned to the system at once.  fdog_host_cache_release frees
// everything kept.
#include <cstdlib>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "fdog_internal.h"

namespace fdog {
namespace {

constexpr size_t kRound = size_t(64) << 10;

struct HostPool {
    std::mutex mu;
    std::map<size_t, std::vector<void*>> free_by_size;
    size_t kept = 0;
};

HostPool& pool() {
    // never destroyed: instances freed from static destructors may still return buffers
    static HostPool* p = new HostPool();
    return *p;
}

size_t rounded(size_t bytes) { return (bytes + kRound - 1) / kRound * kRound; }

}  // namespace

void* host_pool_get(size_t bytes) {
    const size_t sz = rounded(bytes);
    HostPool& hp = pool();
    {
        std::lock_guard<std::mutex> lk(hp.mu);
        auto it = hp.free_by_size.find(sz);
        if (it != hp.free_by_size.end() && !it->second.empty()) {
            void* p = it->second.back();
            it->second.pop_back();
            hp.kept -= sz;
            return p;
        }
    }
    void* p = std::aligned_alloc(64, sz);
    if (!p) throw std::bad_alloc();
    return p;
}

void host_pool_put(void* p, size_t bytes) noexcept {
    if (!p) return;
    const size_t sz = rounded(bytes);
    HostPool& hp = pool();
    {
        std::lock_guard<std::mutex> lk(hp.mu);
        if (hp.kept + sz <= kHostPoolCap) {
            try {
                hp.free_by_size[sz].push_back(p);
                hp.kept += sz;
                return;
            } catch (...) {
            }
        }
    }
    std::free(p);
}

size_t host_pool_release() noexcept {
    HostPool& hp = pool();
    std::map<size_t, std::vector<void*>> drop;
    size_t bytes = 0;
    {
        std::lock_guard<std::mutex> lk(hp.mu);
        drop.swap(hp.free_by_size);
        bytes = hp.kept;
        hp.kept = 0;
    }
    for (auto& [sz, v] : drop)
        for (void* p : v) std::free(p);
    return bytes;
}

}  // namespace fdog

extern "C" int fdog_host_cache_release(int64_t* bytes_freed) {
    const size_t b = fdog::host_pool_release();
    if (bytes_freed) *bytes_freed = static_cast<int64_t>(b);
    return FDOG_OK;
}
