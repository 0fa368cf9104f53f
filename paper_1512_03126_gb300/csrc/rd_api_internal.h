// Host-side helpers shared by the C-ABI translation units.
#pragma once
#include <cstddef>
#include <cstdint>

#include "rdsplit.h"

namespace rdapi {
int fail(int code, const char* fmt, ...);
void* dev_alloc(size_t bytes);
void dev_free(void* p);
int run_loop(rdsplit_mesh* h, double t_end, int64_t max_periods, uint64_t seed);
}  // namespace rdapi
