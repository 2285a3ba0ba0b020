// Hooks of the context used by the request server (same library, not exported).
#pragma once

#include <cuda_runtime.h>

#include "../../include/berrywl.h"

namespace bw_internal {

// Gives the context a caller-owned device arena of `cap` bytes; calls that need more
// fail with BW_ENOMEM instead of allocating.  The context never frees it.
bw_status attach_arena(bw_ctx* ctx, void* base, size_t cap);
// Grows the context's pinned staging buffer to at least `bytes`.
bw_status reserve_staging(bw_ctx* ctx, size_t bytes);
// Clears the context's status word on stream s.
bw_status clear_status_async(bw_ctx* ctx, cudaStream_t s);
// Copies the context's status word (code, pad, k index, value: 24 bytes) to pinned host memory.
bw_status status_to_host_async(bw_ctx* ctx, void* pinned_dst, cudaStream_t s);
const char* last_error(const bw_ctx* ctx);

}  // namespace bw_internal
