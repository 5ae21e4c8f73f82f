// Internal interface between the ctx (api.cu) and the serving runtime
// (server.cu).
#pragma once

#include "kernels.h"
#include "spx.h"

#include <string>
#include <vector>

namespace spx {

// Device views of a point table and of some indexes of a ctx.
struct ServedData {
    int device = 0;
    const int2 *pts = nullptr;
    uint64_t n = 0;
    std::vector<IndexView> ix;
    std::vector<int> fp32;
};

// Fills out; on a bad handle returns SPX_EINVAL and sets ctx's message.
spx_status served_data(spx_ctx *ctx, spx_points points, const spx_index *indexes, uint32_t n, ServedData &out);
// Sets ctx's error message; returns st.
spx_status ctx_error(spx_ctx *ctx, spx_status st, const std::string &msg);
// Why a polygon set cannot be indexed (empty: it can).
std::string check_rings(const int32_t *xy, const uint64_t *ring_off, uint32_t P);
// Builds the index of a checked polygon set on the device one level coarser
// than the automatic grid (at least 5; sub_log2 3), on stream s with memory from `pool` (stream-ordered): view
// (its err pointer unset), its one allocation mem of `bytes` (the caller frees
// it with cudaFreeAsync).  The host waits on s alone.  0, or 1 (err: the
// input) or 2 (err: a CUDA error).
int device_grid_index(const int32_t *xy, const uint64_t *ring_off, uint32_t P, IndexView &view, void *&mem,
                      size_t &bytes, std::string &err, cudaStream_t s, cudaMemPool_t pool);

} // namespace spx
