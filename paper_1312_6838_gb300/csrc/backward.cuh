// Internal interface of the reconstruction-error adjoint (backward.cu).
#pragma once

#include "css_common.cuh"

size_t backward_workspace_bytes(int dtype, int64_t m, int64_t n, int32_t k);
