// Internal interface of the rank-k approximation (lowrank.cu).
#pragma once

#include "css_common.cuh"

size_t lowrank_workspace_bytes(int64_t n, int32_t l, int32_t k);
