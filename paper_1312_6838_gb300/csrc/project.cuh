// Internal interface of the random projection (project.cu).
#pragma once

#include "css_common.cuh"

size_t project_workspace_bytes(int dtype, int64_t m, int64_t n, int64_t r);
size_t project_random_workspace_bytes(int dtype, int64_t m, int64_t n, int64_t r);
size_t distributed_workspace_bytes(int dtype, int64_t m, int64_t n, int64_t r, int32_t k,
                                   int32_t k_block);
