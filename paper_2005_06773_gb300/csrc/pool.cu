// pool.cu -- first-fit allocator over a device buffer the caller owns (offsets only; no CUDA calls), used
// by the serving loop to admit requests by free device memory.  Blocks are multiples of 256 bytes; freed
// blocks merge with free neighbours.
#include <map>
#include <mutex>

#include "runtime.h"

using namespace mhc::host;

struct mhc_pool {
    size_t size = 0;
    std::map<size_t, size_t> free_;    // offset -> bytes
    std::map<size_t, size_t> used_;    // offset -> bytes
    size_t free_bytes = 0;
};

namespace mhc {
namespace host {

bool pool_alloc(mhc_pool *p, size_t bytes, size_t *offset) {
    bytes = align_up(bytes ? bytes : 1);
    for (auto it = p->free_.begin(); it != p->free_.end(); ++it) {
        if (it->second < bytes) continue;
        const size_t off = it->first, len = it->second;
        p->free_.erase(it);
        if (len > bytes) p->free_.emplace(off + bytes, len - bytes);
        p->used_.emplace(off, bytes);
        p->free_bytes -= bytes;
        *offset = off;
        return true;
    }
    return false;
}

bool pool_free(mhc_pool *p, size_t offset) {
    auto u = p->used_.find(offset);
    if (u == p->used_.end()) return false;
    size_t off = u->first, len = u->second;
    p->used_.erase(u);
    p->free_bytes += len;
    auto next = p->free_.lower_bound(off);
    if (next != p->free_.end() && off + len == next->first) {   // merge with the following block
        len += next->second;
        next = p->free_.erase(next);
    }
    if (next != p->free_.begin()) {                               // and with the preceding one
        auto prev = std::prev(next);
        if (prev->first + prev->second == off) {
            prev->second += len;
            return true;
        }
    }
    p->free_.emplace(off, len);
    return true;
}

size_t pool_largest(const mhc_pool *p) {
    size_t m = 0;
    for (const auto &f : p->free_) m = f.second > m ? f.second : m;
    return m;
}

size_t pool_free_bytes(const mhc_pool *p) { return p->free_bytes; }

mhc_pool *pool_new(size_t bytes) {
    mhc_pool *p = new mhc_pool();
    p->size = bytes & ~(kAlign - 1);
    if (p->size) p->free_.emplace(0, p->size);
    p->free_bytes = p->size;
    return p;
}

void pool_delete(mhc_pool *p) { delete p; }

}  // namespace host
}  // namespace mhc

extern "C" {

int mhc_pool_create(size_t bytes, mhc_pool **out) {
    if (!out) return fail(MHC_E_INVALID, "out is NULL");
    *out = nullptr;
    if (bytes < kAlign) return fail(MHC_E_INVALID, "a pool needs at least 256 bytes");
    *out = pool_new(bytes);
    return MHC_OK;
}

void mhc_pool_destroy(mhc_pool *p) { pool_delete(p); }

int mhc_pool_alloc(mhc_pool *p, size_t bytes, size_t *offset) {
    if (!p || !offset) return fail(MHC_E_INVALID, "pool and offset must be non-NULL");
    if (!pool_alloc(p, bytes, offset)) return fail(MHC_E_NOMEM, "no free block is large enough");
    return MHC_OK;
}

int mhc_pool_free(mhc_pool *p, size_t offset) {
    if (!p) return fail(MHC_E_INVALID, "pool is NULL");
    if (!pool_free(p, offset)) return fail(MHC_E_NOTFOUND, "no block starts at this offset");
    return MHC_OK;
}

int mhc_pool_info(mhc_pool *p, size_t *free_bytes, size_t *largest_free, int32_t *n_free_blocks) {
    if (!p) return fail(MHC_E_INVALID, "pool is NULL");
    if (free_bytes) *free_bytes = p->free_bytes;
    if (largest_free) *largest_free = pool_largest(p);
    if (n_free_blocks) *n_free_blocks = (int32_t)p->free_.size();
    return MHC_OK;
}

}  // extern "C"
