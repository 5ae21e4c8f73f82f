// Launch wrappers of libspx's kernels (internal; called from api.cu).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace spx {

struct IndexView {
    const uint32_t *cell; // 4^g coarse words
    const uint32_t *fine; // blocks of 4^sub fine words
    const uint4 *ent;     // entries
    const int4 *edge;     // per-fine-row edge lists
    int sc;               // coarse shift: 30 - g
    int gc;               // g
    int sf;               // fine shift: 30 - g - sub
    int sb;               // sub
    uint32_t P;           // number of polygons
};

// Device status word bits (ORed into the ctx's persistent error word).
constexpr unsigned kErrTimeout = 1u;   // a bounded wait gave up
constexpr unsigned kErrInternal = 2u;  // an internal consistency check failed
constexpr unsigned kErrCopy = 4u;      // a bounded wait for a bulk copy gave up

// Per-ctx device counters, in this order.
enum { kStatPoints = 0, kStatTests = 1, kStatEscalations = 2, kStatPairs = 3, kStatCount = 4 };

struct JoinLaunch {
    IndexView ix;
    const int2 *pts;
    uint64_t n;
    uint2 *pairs;                 // may be null when cap == 0
    uint64_t cap;
    unsigned long long *counts;   // P entries or null; zeroed by the launcher
    unsigned long long *total;    // device total or null
    uint32_t *res;                // join pass 1 -> 3: per-point result (scratch)
    unsigned long long *tile_tot; // join: per-tile pair totals, then offsets (scratch)
    unsigned *tile_counter;       // tile claims (scratch)
    unsigned *err;                // persistent error word
    unsigned long long *stats;    // kStatCount counters
    int fp32;
};

// Scratch bytes the join needs for n points (per-point results, tile totals, counter).
size_t join_scratch_bytes(uint64_t n);
size_t plain_scratch_bytes(uint64_t n);

// scratch: device memory of join_scratch_bytes(n) bytes.  ev (may be null):
// four events recorded before pass 1, after pass 1 (resolve), after pass 2
// (scan) and after pass 3 (emit).
cudaError_t launch_join(const JoinLaunch &a, void *scratch, cudaStream_t s, cudaEvent_t *ev = nullptr);
cudaError_t launch_join_plain(const JoinLaunch &a, void *scratch, cudaStream_t s);
// scratch: at least 16 bytes of device memory (zeroed inside).
cudaError_t launch_aggregate(const JoinLaunch &a, void *scratch, cudaStream_t s, cudaEvent_t *ev = nullptr);

// Batched selection: per-query ascending point-id lists in ids (cap entries),
// offsets[q] / offsets[P] (device, P + 1 values; offsets[P] = total).  At most
// 1024 queries per index.  scratch: select_scratch_bytes(n, P, cap).
size_t select_scratch_bytes(uint64_t n, uint32_t P, uint64_t cap);
cudaError_t launch_select(const JoinLaunch &a, uint32_t *ids, uint64_t cap, unsigned long long *offsets,
                          void *scratch, cudaStream_t s);
constexpr uint32_t kSelectMaxQueries = 1024;

// dst[i] = src[i * (n / m)] for i < m (m <= n): the tuner's deterministic sample.
cudaError_t launch_gather_stride(const int2 *src, uint64_t n, int2 *dst, uint64_t m, cudaStream_t s);

int device_sm_count();

} // namespace spx
