// Internal declarations shared by the CUDA translation units of libscatter.
// Nothing here is part of the public ABI (include/scatter.h is).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include "scatter.h"

namespace scatter {

// Records a one-line failure description for scatter_last_error() and
// returns `st` so call sites can `return fail(...)`.
scatter_status fail(scatter_status st, const char* fmt, ...);

// Converts a CUDA error into SCATTER_ERR_CUDA with a message (or OK).
scatter_status cuda_status(cudaError_t e, const char* what);

bool log_enabled();

// Host-side fault injection for tests: with SCATTER_FAULT=alloc:N in the
// environment the N-th device allocation of plan building (counted since the
// variable last changed; plain "alloc" means the first) reports
// out-of-memory before any device call.  No device work is involved.
bool injected_alloc_failure();

}  // namespace scatter
