// Host-side bookkeeping of the serving loop (serve.cu): a first-fit
// allocator over one device arena and the cache of resident RFP arrays.
// No CUDA here: the arena is a byte range [0, capacity) and the caller adds
// the device base address.  Not thread-safe: the serving loop's scheduler
// thread is its only user.
#pragma once

#include <cstddef>
#include <cstdint>
#include <iterator>
#include <list>
#include <map>
#include <unordered_map>

namespace rfp {
namespace serve {

constexpr size_t kAlign = 256;

inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// First-fit allocator with coalescing of neighbouring free ranges.
class Arena {
public:
    explicit Arena(size_t capacity) : capacity_(capacity / kAlign * kAlign)
    {
        if (capacity_) free_[0] = capacity_;
    }
    // Offset of a block of at least `bytes`, or -1 if no free range is large enough.
    int64_t alloc(size_t bytes)
    {
        const size_t need = align_up(bytes ? bytes : 1);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < need) continue;
            const size_t off = it->first, len = it->second;
            free_.erase(it);
            if (len > need) free_[off + need] = len - need;
            used_[off] = need;
            in_use_ += need;
            return (int64_t)off;
        }
        return -1;
    }
    // Returns false if off is not a live block.
    bool release(int64_t off)
    {
        auto u = used_.find((size_t)off);
        if (u == used_.end()) return false;
        size_t start = u->first, len = u->second;
        used_.erase(u);
        in_use_ -= len;
        auto next = free_.lower_bound(start);
        if (next != free_.end() && start + len == next->first) {   // merge with the following range
            len += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {                               // and with the preceding one
            auto prev = std::prev(next);
            if (prev->first + prev->second == start) {
                prev->second += len;
                return true;
            }
        }
        free_[start] = len;
        return true;
    }
    size_t capacity() const { return capacity_; }
    size_t in_use() const { return in_use_; }
    size_t largest_free() const
    {
        size_t m = 0;
        for (auto &f : free_) m = f.second > m ? f.second : m;
        return m;
    }
    size_t free_ranges() const { return free_.size(); }

private:
    size_t capacity_, in_use_ = 0;
    std::map<size_t, size_t> free_;   // offset -> length
    std::map<size_t, size_t> used_;   // offset -> length
};

// What a resident RFP array holds.
enum class Held : int32_t { Factor64 = 1, Matrix64 = 2 };

struct CacheEntry {
    int64_t key;
    int64_t offset;      // in the arena
    size_t bytes;
    int64_t n;
    char transr, uplo;
    Held held;
    int32_t pins;        // in-flight jobs using the entry
};

// Resident RFP arrays keyed by the caller's matrix key, least recently used
// first in `lru_`.  Pinned entries (used by in-flight work) are never evicted.
class FactorCache {
public:
    explicit FactorCache(Arena &arena) : arena_(arena) {}

    CacheEntry *find(int64_t key)
    {
        auto it = map_.find(key);
        if (it == map_.end()) return nullptr;
        lru_.splice(lru_.end(), lru_, it->second);   // most recently used
        return &*it->second;
    }
    // Insert an entry for a block already allocated in the arena; nullptr
    // (nothing inserted) if a pinned entry holds the key.
    CacheEntry *insert(const CacheEntry &e)
    {
        if (map_.count(e.key) && !erase(e.key)) return nullptr;
        lru_.push_back(e);
        auto it = std::prev(lru_.end());
        map_[e.key] = it;
        bytes_ += e.bytes;
        return &*it;
    }
    // Drop an entry and free its arena block (must not be pinned).
    bool erase(int64_t key)
    {
        auto it = map_.find(key);
        if (it == map_.end() || it->second->pins > 0) return false;
        arena_.release(it->second->offset);
        bytes_ -= it->second->bytes;
        lru_.erase(it->second);
        map_.erase(it);
        return true;
    }
    // Allocate `bytes`, evicting unpinned entries from the least recently
    // used end until the allocation succeeds; -1 if it cannot.
    int64_t alloc_evicting(size_t bytes)
    {
        if (align_up(bytes ? bytes : 1) > arena_.capacity()) return -1;   // never fits: evict nothing
        int64_t off = arena_.alloc(bytes);
        while (off < 0) {
            auto victim = lru_.begin();
            while (victim != lru_.end() && victim->pins > 0) ++victim;
            if (victim == lru_.end()) return -1;
            ++evictions_;
            erase(victim->key);
            off = arena_.alloc(bytes);
        }
        return off;
    }
    size_t entries() const { return map_.size(); }
    size_t bytes() const { return bytes_; }
    int64_t evictions() const { return evictions_; }

private:
    Arena &arena_;
    std::list<CacheEntry> lru_;
    std::unordered_map<int64_t, std::list<CacheEntry>::iterator> map_;
    size_t bytes_ = 0;
    int64_t evictions_ = 0;
};

}  // namespace serve
}  // namespace rfp
