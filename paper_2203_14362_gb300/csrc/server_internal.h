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

} // namespace spx
