// Autotuner of the generic kernel's launch shape (threads, points per
// thread, split-K) with a JSON cache keyed by problem size and GPU.
#pragma once

#include "plan.h"

namespace scatter {

Tiling heuristic_tiling(const scatter_plan_s* p);
scatter_status apply_tiling(scatter_plan_s* p, const Tiling& t);
scatter_status autotune_generic(scatter_plan_s* p, const char* cache_path);
// Batched plans: (threads, points per thread) of the persistent kernel.
scatter_status autotune_batch(scatter_plan_s* p, const char* cache_path);

}  // namespace scatter
