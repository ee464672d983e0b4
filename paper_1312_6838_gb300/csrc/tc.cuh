// Internal interface of the tcgen05 GEMMs (tc_gemm.cu).
#pragma once

#include "css_common.cuh"

namespace css {
namespace tc {

// A (BF16, column-major, leading dimension lda) can feed the TMA path with a
// target width r (<= 512 columns in TMEM).
bool supported(const void* A, long long lda, int m, int r);

// Number of K slices of the projection for an m-row A on `sms` SMs (<= 32).
int project_slices(int m, int sms);

// partial[s][i + j*m] = sum over the columns l of slice s of A[i, l] Omega[l, j]
// (A m x n, Omega n x r, both BF16 column-major); FP32 accumulation in TMEM.
cudaError_t project_partials(const void* A, long long lda, int m, int n, const void* Om, long long ldo,
                             int r, int slices, float* partial, int* err, unsigned long long spin_ns,
                             cudaStream_t s);

// Bytes of scratch for the BF16 parts of B used by colnorms.
size_t colnorm_scratch_bytes(int m, int r);

// f[i] = ||B^T A_:i||^2 for the n columns of A (BF16, m x n) and B (FP32, m x r).
// stall != 0 is the test hook of css_opts::test_unmet_wait (a bounded wait
// that runs out).
cudaError_t colnorms(const void* A, long long lda, int m, int n, const float* B, long long ldb, int r,
                     void* scratch, double* f, int* err, unsigned long long spin_ns, cudaStream_t s,
                     int stall = 0);

// Scratch bytes of css_f0 (C in FP32, its BF16 parts, row-tile partials;
// f32: A's own BF16 parts too).
size_t css_f0_scratch_bytes(int m, int n, bool f32 = false);
// The tensor-map encoder is available (css_f0 for FP32 input needs no more).
bool supported_any();

// Algorithm 1's initial scores for BF16 A: C = A A^T on tensor cores (FP32
// accumulation of exact BF16 products), C split into two BF16 parts, and
// f[i] = A_:i^T C A_:i from the column dots of A with C A (FP64 sums).
// f32: A is FP32 (any alignment); it is split into two BF16 parts first and
// both GEMMs sum the four products of parts.
cudaError_t css_f0(const void* A, long long lda, int m, int n, void* scratch, double* f, int* err,
                   unsigned long long spin_ns, cudaStream_t s, int stall = 0, bool f32 = false);

}  // namespace tc
}  // namespace css
