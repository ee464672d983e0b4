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

// How css_f0 reads A: BF16 straight from A through TMA (supported()), BF16
// copied first to an aligned buffer (any other layout), FP32 split first
// into three BF16 parts (any layout; one that refuses 16-byte loads is also
// copied to an aligned FP32 buffer, for the greedy passes).
enum F0Source { kF0Bf16 = 0, kF0Bf16Staged = 1, kF0F32 = 2, kF0F32Staged = 3 };
int f0_source(bool f32, const void* A, long long lda, int m);
// kF0Bf16Staged, kF0F32Staged: the aligned copy of A that css_f0 leaves in its scratch
// (leading dimension a multiple of 8; it stays valid until the scratch is
// reused), so that later passes over A can take 16-byte loads.
bool f0_staged_copy(int m, int n, int src, void* scratch, const void** A, long long* lda);
// Scratch bytes of css_f0 (C in FP32, its BF16 parts, row-tile partials,
// A's parts or copy).  kF0Bf16Staged bounds every BF16 layout, kF0F32Staged
// every FP32 one.
size_t css_f0_scratch_bytes(int m, int n, int src);
// The tensor-map encoder is available (css_f0 for FP32 input needs no more).
bool supported_any();

// Algorithm 1's initial scores: C = A A^T on tensor cores (FP32
// accumulation of exact BF16 products, in K chunks added with compensated
// FP32 sums), C split into three BF16 parts (all of its FP32 bits), and
// f[i] = A_:i^T C A_:i from the column dots of A with C A (FP64 sums).  src = f0_source(...): for FP32
// A both GEMMs sum the six products of its parts down to 2^-16.
// pipe: column chunks of A that arrive one after another (a host copy split
// by the caller): chunk z holds columns [z * cols, (z + 1) * cols) and is in
// place once ready[z] has completed.  With src == kF0Bf16 and cols ==
// f0_chunk_cols(m, n), each K chunk of C = A A^T starts as soon as its
// columns are in; otherwise everything waits for all of them first.
struct F0Pipe {
  const cudaEvent_t* ready;
  int chunks, cols;
};
int f0_chunk_cols(int m, int n);
cudaError_t css_f0(const void* A, long long lda, int m, int n, void* scratch, double* f, int* err,
                   unsigned long long spin_ns, cudaStream_t s, int stall, int src,
                   const F0Pipe* pipe = nullptr);

// css_f0 for a group of problems (a batch): one launch per phase for all of
// them.  Problem i's scratch (css_f0_scratch_bytes(m[i], n[i], src[i])
// bytes, C first) is scratch[i]; its scores go to f[i].
struct GroupProb;
struct GroupTile;
struct GroupF0 {
  const GroupProb* probs;   // device: count descriptors
  const GroupTile* tiles2;  // device: the C = A A^T tiles of every problem
  const GroupTile* tiles3;  // device: the column-dot tiles
  int count, ntiles2, ntiles3, staged;
  int smem2, smem3;
};
// Bytes of device memory for the descriptors and tile lists.
size_t group_f0_desc_bytes(const int* m, const int* n, int count, bool f32);
// Writes the descriptors (tensor maps encoded on the host) to `desc` and
// fills `out`; synchronises `s` (the host lists end with the call).  All
// problems share one input type (src[i] = f0_source(...)); count <= 65535.
cudaError_t group_f0_prepare(int count, const void* const* A, const long long* lda, const int* m, const int* n,
                             void* const* scratch, double* const* f, const int* src, void* desc, int* err,
                             unsigned long long spin_ns, GroupF0* out, cudaStream_t s);
// Enqueues the phases (device work only: capturable).
cudaError_t group_f0_run(const GroupF0& g, cudaStream_t s);

}  // namespace tc
}  // namespace css
