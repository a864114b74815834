// rdct_arena.cu -- first-fit offset allocator with coalescing, used by the
// server to place request buffers inside its fixed device budget.  Host code
// only: it hands out offsets, the caller owns the memory they index.
#include <algorithm>
#include <cstdint>
#include <map>
#include <mutex>
#include <new>

#include "rdct_internal.h"

struct rdct_arena {
    int64_t size = 0, align = 256, used = 0;
    std::map<int64_t, int64_t> free_blocks;  // offset -> size
    std::map<int64_t, int64_t> live;         // offset -> size
    std::mutex mu;
};

using rdct::set_error;

extern "C" {

rdct_status rdct_arena_create(int64_t size, int64_t align, rdct_arena **arena) {
    if (!arena || size <= 0 || align <= 0 || (align & (align - 1)))
        return set_error(RDCT_ERR_ARG, "rdct_arena_create: size > 0 and a power-of-two alignment required");
    rdct_arena *a = new (std::nothrow) rdct_arena();
    if (!a) return set_error(RDCT_ERR_OOM, "rdct_arena_create: host allocation failed");
    a->size = size & ~(align - 1);
    a->align = align;
    if (a->size > 0) a->free_blocks[0] = a->size;
    *arena = a;
    return RDCT_OK;
}

rdct_status rdct_arena_alloc(rdct_arena *a, int64_t bytes, int64_t *offset) {
    if (!a || !offset || bytes <= 0) return set_error(RDCT_ERR_ARG, "rdct_arena_alloc: bad argument");
    const int64_t need = (bytes + a->align - 1) & ~(a->align - 1);
    std::lock_guard<std::mutex> lk(a->mu);
    for (auto it = a->free_blocks.begin(); it != a->free_blocks.end(); ++it) {
        if (it->second < need) continue;
        const int64_t off = it->first, rest = it->second - need;
        a->free_blocks.erase(it);
        if (rest > 0) a->free_blocks[off + need] = rest;
        a->live[off] = need;
        a->used += need;
        *offset = off;
        return RDCT_OK;
    }
    return set_error(RDCT_ERR_OOM, "rdct_arena_alloc: no free block large enough");
}

rdct_status rdct_arena_free(rdct_arena *a, int64_t offset) {
    if (!a) return set_error(RDCT_ERR_ARG, "rdct_arena_free: null arena");
    std::lock_guard<std::mutex> lk(a->mu);
    auto it = a->live.find(offset);
    if (it == a->live.end()) return set_error(RDCT_ERR_NOT_FOUND, "rdct_arena_free: not a live block");
    int64_t off = it->first, sz = it->second;
    a->live.erase(it);
    a->used -= sz;
    auto next = a->free_blocks.lower_bound(off);
    if (next != a->free_blocks.end() && off + sz == next->first) {  // merge with the following block
        sz += next->second;
        next = a->free_blocks.erase(next);
    }
    if (next != a->free_blocks.begin()) {  // merge with the preceding block
        auto prev = std::prev(next);
        if (prev->first + prev->second == off) {
            prev->second += sz;
            return RDCT_OK;
        }
    }
    a->free_blocks[off] = sz;
    return RDCT_OK;
}

int64_t rdct_arena_used(const rdct_arena *a) { return a ? a->used : 0; }

int64_t rdct_arena_largest_free(const rdct_arena *a) {
    if (!a) return 0;
    int64_t best = 0;
    for (const auto &kv : a->free_blocks) best = std::max(best, kv.second);
    return best;
}

rdct_status rdct_arena_destroy(rdct_arena *a) {
    delete a;
    return RDCT_OK;
}

}  // extern "C"
