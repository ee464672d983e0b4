// Internal interface of the initial-score kernels.
#pragma once

#include "css_common.cuh"

namespace css {

// Doubles of scratch the SIMT initial-score kernels need for their partials.
size_t css_f0_partial_doubles(int dtype, int m, int n);
size_t gcss_f0_partial_doubles(int dtype, int r, int n);

// CSS: C = A A^T (m x m, Acc type, leading dimension m) and
// f[i] = A_:i^T C A_:i.  A has dtype `dtype`.
cudaError_t css_f0_simt(int dtype, const void* A, long long lda, int m, int n, void* C,
                        double* partial, double* f, cudaStream_t s);

// GCSS: f[i] = ||B^T A_:i||^2, B (m x r, leading dimension ldb, Acc type).
cudaError_t gcss_f0_simt(int dtype, const void* A, long long lda, int m, int n, const void* B,
                         long long ldb, int r, double* partial, double* f, cudaStream_t s);

}  // namespace css
