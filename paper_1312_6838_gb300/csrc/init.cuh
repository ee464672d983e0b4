// Internal interface of the initial-score kernels.
#pragma once

#include "css_common.cuh"

namespace css {

// Doubles of scratch the SIMT initial-score kernels need for their partials.
size_t css_f0_partial_doubles(int dtype, int m, int n);
size_t gcss_f0_partial_doubles(int dtype, int r, int n);

// CSS: C = A A^T (m x m, Acc type, leading dimension ldc) and
// f[i] = A_:i^T C A_:i.  A has dtype `dtype`.
cudaError_t css_f0_simt(int dtype, const void* A, long long lda, int m, int n, void* C, long long ldc,
                        double* partial, double* f, cudaStream_t s);

// Many CSS problems at once (css_select_batched): the same computation as
// css_f0_simt for every item, in three launches whose blocks run over the
// concatenated tiles of all items.
struct F0Item {
  const void* A;
  long long lda;
  int m, n;
  void* C;           // m x m, Acc type, leading dimension ldc
  long long ldc;
  double* partial;   // css_f0_partial_doubles(dtype, m, n)
  double* f;         // n
};
struct F0Grid {
  int syrk = 0, colreduce = 0, sums = 0;   // blocks of the three launches
};
// Host: the first block of every item in each launch, three arrays of
// count + 1 ints back to back in `starts`; returns the grid sizes.
F0Grid css_f0_grouped_starts(int dtype, const int* m, const int* n, int count, int* starts);
// Device arrays: items[count], starts[3 * (count + 1)].
cudaError_t css_f0_grouped(int dtype, const F0Item* items, const int* starts, const F0Grid& grid,
                           int count, cudaStream_t s);

// GCSS: f[i] = ||B^T A_:i||^2, B (m x r, leading dimension ldb, Acc type).
cudaError_t gcss_f0_simt(int dtype, const void* A, long long lda, int m, int n, const void* B,
                         long long ldb, int r, double* partial, double* f, cudaStream_t s);

}  // namespace css
