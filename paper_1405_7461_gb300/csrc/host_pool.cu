// Page-locked host blocks for the result arrays a search hands to its caller
// (tdq_results), kept for reuse once the caller releases them.  A
// device-to-host copy into fresh pageable memory spends most of its time
// populating pages (on a GB300 node: a 54 MB result set takes ~2 ms into fresh
// malloc'd memory, ~0.3 ms into page-locked memory that is already mapped),
// and pinning a block is slower still, so blocks are pinned once and then
// recycled by size class.  Blocks still cached at exit are released with the
// process.
#include <map>
#include <mutex>
#include <unordered_map>

#include "tdq_internal.cuh"

namespace tdq {
namespace {

constexpr uint64_t kMinClassBytes = 1u << 16;
constexpr uint64_t kCacheBytes = 1ull << 30;  // page-locked bytes kept for reuse

std::mutex g_mu;
std::multimap<uint64_t, void *> g_free;        // size class -> cached block
std::unordered_map<void *, uint64_t> g_live;   // block handed out -> its size class
uint64_t g_cached = 0;

uint64_t size_class(uint64_t bytes)
{
    uint64_t c = kMinClassBytes;
    while (c < bytes) c <<= 1;
    return c;
}

}  // namespace

void *host_block_get(uint64_t bytes)
{
    const uint64_t c = size_class(bytes);
    {
        std::lock_guard<std::mutex> lock(g_mu);
        auto it = g_free.find(c);
        if (it != g_free.end()) {
            void *p = it->second;
            g_free.erase(it);
            g_cached -= c;
            g_live[p] = c;
            return p;
        }
    }
    void *p = nullptr;
    if (cudaHostAlloc(&p, c, cudaHostAllocPortable) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    g_live[p] = c;
    return p;
}

bool host_block_put(void *p)
{
    if (!p) return false;
    uint64_t c = 0;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        auto it = g_live.find(p);
        if (it == g_live.end()) return false;
        c = it->second;
        g_live.erase(it);
        if (g_cached + c <= kCacheBytes) {
            g_free.emplace(c, p);
            g_cached += c;
            return true;
        }
    }
    cudaFreeHost(p);
    return true;
}

}  // namespace tdq
