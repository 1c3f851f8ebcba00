// extern "C" handles on the serving loop's host bookkeeping (serve_pool.h)
// for the CPU tests in tests/test_serve_pool.py.
#include "../../paper_0901_1696_gb300/csrc/serve_pool.h"

using rfp::serve::Arena;
using rfp::serve::CacheEntry;
using rfp::serve::FactorCache;
using rfp::serve::Held;

extern "C" {
void *arena_new(size_t cap) { return new Arena(cap); }
void arena_free(void *a) { delete static_cast<Arena *>(a); }
int64_t arena_alloc(void *a, size_t bytes) { return static_cast<Arena *>(a)->alloc(bytes); }
int arena_release(void *a, int64_t off) { return static_cast<Arena *>(a)->release(off) ? 1 : 0; }
size_t arena_in_use(void *a) { return static_cast<Arena *>(a)->in_use(); }
size_t arena_largest_free(void *a) { return static_cast<Arena *>(a)->largest_free(); }
size_t arena_free_ranges(void *a) { return static_cast<Arena *>(a)->free_ranges(); }
size_t arena_capacity(void *a) { return static_cast<Arena *>(a)->capacity(); }

void *cache_new(void *a) { return new FactorCache(*static_cast<Arena *>(a)); }
void cache_free(void *c) { delete static_cast<FactorCache *>(c); }
// allocate (evicting) and insert an entry of `bytes` under key; -1 if impossible
int64_t cache_put(void *c, int64_t key, size_t bytes, int pinned)
{
    auto *fc = static_cast<FactorCache *>(c);
    const int64_t off = fc->alloc_evicting(bytes);
    if (off < 0) return -1;
    CacheEntry e{key, off, bytes, 1, 'N', 'L', Held::Factor64, pinned};
    fc->insert(e);
    return off;
}
int cache_has(void *c, int64_t key) { return static_cast<FactorCache *>(c)->find(key) ? 1 : 0; }
int cache_unpin(void *c, int64_t key)
{
    CacheEntry *e = static_cast<FactorCache *>(c)->find(key);
    if (!e || e->pins == 0) return 0;
    --e->pins;
    return 1;
}
int cache_erase(void *c, int64_t key) { return static_cast<FactorCache *>(c)->erase(key) ? 1 : 0; }
int64_t cache_evictions(void *c) { return static_cast<FactorCache *>(c)->evictions(); }
size_t cache_entries(void *c) { return static_cast<FactorCache *>(c)->entries(); }
size_t cache_bytes(void *c) { return static_cast<FactorCache *>(c)->bytes(); }
}
