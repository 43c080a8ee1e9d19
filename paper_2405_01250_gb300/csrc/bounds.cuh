// Debug bounds checks, compiled in only with -DDIAQ_DEBUG_BOUNDS (the debug
// build of the library, libdiaq_gb300_dbg.so); in the normal build the
// check is the constant true and costs nothing.
//
// DIAQ_BOUNDS_OK(i, limit, site) is true when 0 <= i < limit. Otherwise it
// records the first failure of the translation unit - the site number and
// the index - in a device word, and the kernel skips that access (a load
// reads zero, a store is dropped), so a bad index is reported instead of
// touching memory. diaq_debug_bounds_check reads and clears every
// translation unit's word (without relocatable device code each .cu file has
// its own) and returns DIAQ_ERR_BOUNDS with the site and index.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace diaq {
// Sites, reported by number (diaq_debug_bounds_status names them).
enum BoundsSite : int {
    BS_APPLY_SMALL = 1,
    BS_APPLY_ROWS = 2,
    BS_APPLY_LARGE = 3,
    BS_APPLY_DIAG = 4,
    BS_STORED_VALUE = 5,
    BS_STORED_X = 6,
    BS_MATERIALISE = 7,
    BS_EXPECT = 8,
    BS_PAULI_APPLY = 9,
    BS_ROTATION = 10,
    BS_SAMPLE_TILES = 11,
    BS_SAMPLE_SEARCH = 12,
    BS_SHARD_MOVE = 13,
    BS_SPGEMM = 14,
    BS_WINDOW = 15,
    BS_SITES = 16
};
}  // namespace diaq

#if defined(DIAQ_DEBUG_BOUNDS) && defined(__CUDACC__)
static __device__ unsigned long long g_diaq_bounds_word;

__device__ __forceinline__ bool diaq_bounds_ok(int64_t i, int64_t limit, int site) {
    if (i >= 0 && i < limit) return true;
    const unsigned long long w = (1ull << 63) | (static_cast<unsigned long long>(site & 0x7fff) << 48) |
                                 (static_cast<unsigned long long>(i) & 0xffffffffffffull);
    atomicCAS(&g_diaq_bounds_word, 0ull, w);
    return false;
}
#define DIAQ_BOUNDS_OK(i, limit, site) ::diaq_bounds_ok(static_cast<int64_t>(i), static_cast<int64_t>(limit), (site))
#define DIAQ_BOUNDS_TU(name)                                                                     \
    namespace diaq {                                                                             \
    unsigned long long bounds_word_##name(bool clear) {                                          \
        unsigned long long w = 0;                                                                \
        if (cudaMemcpyFromSymbol(&w, g_diaq_bounds_word, sizeof(w)) != cudaSuccess) return ~0ull; \
        if (clear && w) {                                                                        \
            const unsigned long long z = 0;                                                      \
            cudaMemcpyToSymbol(g_diaq_bounds_word, &z, sizeof(z));                               \
        }                                                                                        \
        return w;                                                                                \
    }                                                                                            \
    }
#else
#define DIAQ_BOUNDS_OK(i, limit, site) true
#define DIAQ_BOUNDS_TU(name) \
    namespace diaq {         \
    unsigned long long bounds_word_##name(bool) { return 0; } \
    }
#endif
