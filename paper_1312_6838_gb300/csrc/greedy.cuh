// Internal interface of the persistent greedy kernel (greedy.cu).
#pragma once

#include "css_common.cuh"

namespace css {

// One greedy problem (Algorithm 1 when mode == 0, Algorithm 3 when mode == 1).
struct UnitDesc {
  const void* A;      // m x n, column-major, leading dimension lda
  long long lda;
  int m, n, k, mode;
  // CSS: T = C = A A^T (m x m, ld m, Acc type).  GCSS: T = B (m x r, ld ldt, Acc type).
  const void* T;
  long long ldt;
  int r, score_mode;
  double tau;
  // state
  double* f;          // numerator of the criterion, Theorem 2/4
  double* g;          // denominator (residual column norms)
  double* thr;        // candidate threshold tau * g_i^(0) (+inf where g_i^(0) = 0)
  unsigned char* selmask;
  double* Q;          // m x k orthonormal basis of the selected columns
  double* Z;          // CSS: C Q (m x k, ld m).  GCSS: B^T Q (r x k, ld r)
  double* W;          // k x n, row t = omega^(t)
  void* qv;           // Acc[m]  direction q (the omega of this step is A^T q)
  void* ypv;          // Acc[m]  (I - P) C q   or   (I - P) B B^T q
  double* e1;         // m
  double* e;          // m  (unnormalised new basis vector)
  double* y;          // m  (C e or B B^T e, unnormalised)
  double* coef;       // max(k, r) scratch coefficients
  double* ups;        // r  (B^T e, GCSS)
  // outputs
  int* sel;
  double* trace;
  int* n_sel;
  int* diag_argmax;
  unsigned long long* trace_ns;   // k * 8 phase timestamps or null
  double* diag_f;
  double* diag_g;
  const int* forced;
  int n_forced;
  int vec_ok;         // A and lda allow 16-byte vector loads
  int t_vec_ok;       // T (C or B) allows 16-byte vector loads
  int pad_;
};

struct TeamDesc {
  int cta0, ncta, u_begin, u_end;   // units order[u_begin .. u_end)
  uint32_t* bar;                    // word 0: the team barrier's arrival count
  double* part;                     // ncta * 4
  double* cand_val;                 // ncta
  int* cand_idx;                    // ncta
  uint32_t* tile_ctr;               // 2 words: fused-step tile counters (alternating)
  // the fused step's last tiles are cut into kSplitR row chunks; chunk sums
  // meet here (split_cap tiles x kSplitR x kSplitVals values, 8 bytes each)
  void* split_part;
  uint32_t* split_done;             // split_cap arrival counters (zero between uses)
  int split_cap;
  int pad_;
};

#ifndef CSS_SPLIT_ROWS
#define CSS_SPLIT_ROWS 4
#endif
constexpr int kSplitR = CSS_SPLIT_ROWS;   // row chunks of a split tile

constexpr int kSplitVals = 16;      // value slots per chunk (2 x the widest tile)
constexpr size_t kSplitSlotBytes = (size_t)kSplitR * kSplitVals * 8;

struct GreedyLaunch {
  const UnitDesc* units;
  const int* order;
  const TeamDesc* teams;
  const int* cta_team;
  DevStatus* st;
  int dtype;       // css_dtype of A
  int tile_cols;   // 2, 4 or 8
  int m_max, k_max, r_max;
  int grid;        // CTAs
  int threads;
  size_t smem;
};

// The kernel's two CTA shapes, both with 128 registers per thread: 512
// threads and one CTA per SM (the default), or 256 threads and two CTAs per
// SM, where teams of small problems gain from twice as many CTAs (Algorithm
// 4's column blocks).
constexpr int kGreedyThreads = 512;
constexpr int kGreedyThreadsPaired = 256;

#define CSS_GREEDY_SHAPE_API                                                     \
  /* Bytes of dynamic shared memory the kernel needs. */                        \
  size_t greedy_smem_bytes(int dtype, int m_max, int k_max, int r_max);         \
  /* Max co-resident CTAs per SM for the given configuration (0 on error). */   \
  int greedy_occupancy(int dtype, int tile_cols, size_t smem);                  \
  /* Enqueue the persistent kernel (cooperative launch). */                     \
  cudaError_t greedy_launch(const GreedyLaunch& L, cudaStream_t stream);
namespace one_per_sm { CSS_GREEDY_SHAPE_API }
namespace two_per_sm { CSS_GREEDY_SHAPE_API }
#undef CSS_GREEDY_SHAPE_API

// The same three calls for the shape with `threads` threads per CTA
// (kGreedyThreads or kGreedyThreadsPaired; GreedyLaunch::threads for the launch).
inline size_t greedy_smem_bytes(int dtype, int m_max, int k_max, int r_max, int threads) {
  return threads == kGreedyThreadsPaired ? two_per_sm::greedy_smem_bytes(dtype, m_max, k_max, r_max)
                                         : one_per_sm::greedy_smem_bytes(dtype, m_max, k_max, r_max);
}
inline int greedy_occupancy(int dtype, int tile_cols, size_t smem, int threads) {
  return threads == kGreedyThreadsPaired ? two_per_sm::greedy_occupancy(dtype, tile_cols, smem)
                                         : one_per_sm::greedy_occupancy(dtype, tile_cols, smem);
}
inline cudaError_t greedy_launch(const GreedyLaunch& L, cudaStream_t stream) {
  return L.threads == kGreedyThreadsPaired ? two_per_sm::greedy_launch(L, stream)
                                           : one_per_sm::greedy_launch(L, stream);
}
// Copies the basis Q of one unit (m x k, FP64 or double-float pairs) to `out`
// as FP64, zeroing columns t >= *n_sel (opts->basis).
cudaError_t export_basis(int dtype, const double* Q, int m, int k, const int* n_sel, double* out,
                         cudaStream_t stream);

}  // namespace css
