// Fixed-budget device-memory arena of the C ABI (host book-keeping over one cudaMalloc).
// Free ranges are kept by offset; allocation takes the first range that fits, freeing merges
// a range with its free neighbours.
#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <mutex>
#include <new>
#include <string>

#include "internal.h"

struct gabor_arena {
    char *base = nullptr;
    bool owned = true;                        // base came from cudaMalloc in gabor_arena_create
    int64_t capacity = 0;
    int64_t in_use = 0;
    std::map<int64_t, int64_t> free_ranges;   // offset -> size
    std::map<int64_t, int64_t> used;          // offset -> size
    std::mutex mu;
};

namespace {

constexpr int64_t kAlign = 256;

gb_status arena_fail(gb_status s, const std::string &msg)
{
    gb::set_last_error(msg.c_str());
    return s;
}

}  // namespace

extern "C" {

gb_status gabor_arena_create(gabor_arena_t *out, int64_t bytes)
{
    if (!out) return arena_fail(GB_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (bytes <= 0) return arena_fail(GB_ERR_INVALID_ARG, "arena size must be positive");
    bytes = (bytes + kAlign - 1) / kAlign * kAlign;
    gabor_arena *a = new (std::nothrow) gabor_arena();
    if (!a) return arena_fail(GB_ERR_OUT_OF_MEMORY, "host allocation failed");
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&a->base), (size_t)bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete a;
        return arena_fail(GB_ERR_OUT_OF_MEMORY, std::string("arena cudaMalloc: ") + cudaGetErrorString(e));
    }
    a->capacity = bytes;
    a->free_ranges[0] = bytes;
    *out = a;
    return GB_OK;
}

gb_status gabor_arena_wrap(gabor_arena_t *out, void *d_base, int64_t bytes)
{
    if (!out) return arena_fail(GB_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!d_base || bytes <= 0) return arena_fail(GB_ERR_INVALID_ARG, "NULL base or non-positive size");
    if (reinterpret_cast<uintptr_t>(d_base) % kAlign) return arena_fail(GB_ERR_INVALID_ARG, "base not 256-byte aligned");
    gabor_arena *a = new (std::nothrow) gabor_arena();
    if (!a) return arena_fail(GB_ERR_OUT_OF_MEMORY, "host allocation failed");
    a->base = static_cast<char *>(d_base);
    a->owned = false;
    a->capacity = bytes / kAlign * kAlign;
    if (a->capacity > 0) a->free_ranges[0] = a->capacity;
    *out = a;
    return GB_OK;
}

gb_status gabor_arena_alloc(gabor_arena_t a, int64_t bytes, void **d_ptr)
{
    if (!a || !d_ptr) return arena_fail(GB_ERR_INVALID_ARG, "NULL arena or output pointer");
    *d_ptr = nullptr;
    if (bytes <= 0) return arena_fail(GB_ERR_INVALID_ARG, "allocation size must be positive");
    const int64_t need = (bytes + kAlign - 1) / kAlign * kAlign;
    std::lock_guard<std::mutex> lock(a->mu);
    for (auto it = a->free_ranges.begin(); it != a->free_ranges.end(); ++it) {
        if (it->second < need) continue;
        const int64_t off = it->first, size = it->second;
        a->free_ranges.erase(it);
        if (size > need) a->free_ranges[off + need] = size - need;
        a->used[off] = need;
        a->in_use += need;
        *d_ptr = a->base + off;
        return GB_OK;
    }
    return arena_fail(GB_ERR_BUDGET, "arena: no free range of " + std::to_string(need) + " bytes");
}

gb_status gabor_arena_free(gabor_arena_t a, void *d_ptr)
{
    if (!a || !d_ptr) return arena_fail(GB_ERR_INVALID_ARG, "NULL arena or pointer");
    std::lock_guard<std::mutex> lock(a->mu);
    const int64_t off = static_cast<char *>(d_ptr) - a->base;
    auto u = a->used.find(off);
    if (u == a->used.end()) return arena_fail(GB_ERR_INVALID_ARG, "pointer is not an allocation of this arena");
    int64_t start = off, size = u->second;
    a->in_use -= size;
    a->used.erase(u);
    auto next = a->free_ranges.lower_bound(start);
    if (next != a->free_ranges.end() && next->first == start + size) {
        size += next->second;
        next = a->free_ranges.erase(next);
    }
    if (next != a->free_ranges.begin()) {
        auto prev = std::prev(next);
        if (prev->first + prev->second == start) {
            start = prev->first;
            size += prev->second;
            a->free_ranges.erase(prev);
        }
    }
    a->free_ranges[start] = size;
    return GB_OK;
}

gb_status gabor_arena_stats(gabor_arena_t a, int64_t *capacity, int64_t *in_use, int64_t *largest_free)
{
    if (!a) return arena_fail(GB_ERR_INVALID_ARG, "NULL arena");
    std::lock_guard<std::mutex> lock(a->mu);
    if (capacity) *capacity = a->capacity;
    if (in_use) *in_use = a->in_use;
    if (largest_free) {
        int64_t m = 0;
        for (const auto &kv : a->free_ranges) m = kv.second > m ? kv.second : m;
        *largest_free = m;
    }
    return GB_OK;
}

gb_status gabor_arena_destroy(gabor_arena_t a)
{
    if (!a) return GB_OK;
    if (a->base && a->owned) cudaFree(a->base);
    delete a;
    return GB_OK;
}

}  // extern "C"
