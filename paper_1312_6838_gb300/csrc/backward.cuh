// Internal interface of the embedding and the reconstruction-error adjoint
// (backward.cu).
#pragma once

#include "css_common.cuh"

size_t backward_workspace_bytes(int dtype, int64_t m, int64_t n, int32_t k);
size_t embed_workspace_bytes(int64_t m, int32_t l);
