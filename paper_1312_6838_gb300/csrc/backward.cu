// Reconstruction at a fixed selected set S: the embedding Q = orth(A_S),
// W = Q^T A of Sec. 3.2 (css_embed), and the loss and gradient of the
// reconstruction error (css_residual_backward).
//
// Loss and gradient:
//   L(A) = ||A - P^(S) A||_F^2,  P^(S) = A_S (A_S^T A_S)^-1 A_S^T   (Eq. Projection)
//   T = (A_S^T A_S)^-1 A_S^T A,  R = A - A_S T
//   dL/dA = 2 R  (columns outside S),  dL/dA_S = -2 R T^T
//
// With the Cholesky factor A_S^T A_S = L L^T (recomputed here in FP64, not
// carried over from any forward pass) and Q = A_S L^-T (orthonormal):
//   W = Q^T A,  R = A - Q W,  T = L^-T W,  R T^T = (R W^T) L^-1.
// R is a small difference of large terms (the part of A outside span(A_S)),
// so W and R are accumulated in double-float arithmetic (pairs of FP32 values
// with error-free products and sums: Dekker's product by FMA and Knuth's
// TwoSum) when A is FP32/BF16; FP64 input uses FP64 throughout.  R W^T has no
// such cancellation and is accumulated in FP32 (FP64 for FP64 input).
#include <algorithm>
#include <vector>

#include "backward.cuh"
#include "df.cuh"

using namespace css;

namespace {

template <typename TA> __device__ __forceinline__ double to_d(TA v);
template <> __device__ __forceinline__ double to_d<double>(double v) { return v; }
template <> __device__ __forceinline__ double to_d<float>(float v) { return (double)v; }
template <> __device__ __forceinline__ double to_d<__nv_bfloat16>(__nv_bfloat16 v) {
  return (double)__uint_as_float(((uint32_t)__bfloat16_as_ushort(v)) << 16);
}
template <typename TA> __device__ __forceinline__ TA from_d(double v);
template <> __device__ __forceinline__ double from_d<double>(double v) { return v; }
template <> __device__ __forceinline__ float from_d<float>(double v) { return (float)v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_d<__nv_bfloat16>(double v) {
  return __float2bfloat16_rn((float)v);
}

// ------------------------------------------------------- small FP64 steps --
template <typename TA>
__global__ void gather_cols_kernel(const TA* __restrict__ A, long long lda, int m,
                                   const int* __restrict__ sel, int k, double* __restrict__ AS) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)m * k) return;
  const int i = (int)(idx % m), j = (int)(idx / m);
  AS[idx] = to_d<TA>(A[(long long)sel[j] * lda + i]);
}


// G = A_S^T A_S split over the m rows: block (pair, slice) forms the 32 x 32
// tile (ti >= tj) of one row slice, 2 x 2 outputs per thread; gram_fin then
// adds the slices in order and mirrors (bit-reproducible).  Enough blocks to
// fill the GPU even for small k, where one block per output tile would not.
constexpr int kGT = 32, kGK = 32;

struct GramPlan {
  int tiles, npairs, nslices, slice;
};

GramPlan gram_plan(int m, int k) {
  GramPlan g{};
  g.tiles = (k + kGT - 1) / kGT;
  g.npairs = g.tiles * (g.tiles + 1) / 2;
  const int want = std::max(1, (2 * 148 + g.npairs - 1) / g.npairs);
  g.nslices = std::max(1, std::min(want, (m + 127) / 128));
  g.slice = (m + g.nslices - 1) / g.nslices;
  return g;
}

__global__ void __launch_bounds__(256) gram_part_kernel(const double* __restrict__ AS, int m, int k, int slice,
                                                        int npairs, double* __restrict__ part) {
  __shared__ double xa[kGT][kGK + 1], xb[kGT][kGK + 1];
  const int pidx = blockIdx.x, sl = blockIdx.y;
  int ti = (int)((sqrtf(8.f * pidx + 1.f) - 1.f) * 0.5f);
  while (ti * (ti + 1) / 2 > pidx) --ti;
  while ((ti + 1) * (ti + 2) / 2 <= pidx) ++ti;
  const int tj = pidx - ti * (ti + 1) / 2;
  const int a0 = ti * kGT, b0 = tj * kGT;
  const int rb = sl * slice, re = min(m, rb + slice);
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double acc00 = 0.0, acc01 = 0.0, acc10 = 0.0, acc11 = 0.0;
  for (int r0 = rb; r0 < re; r0 += kGK) {
    for (int e = threadIdx.x; e < kGT * kGK; e += 256) {
      const int col = e / kGK, rr = e % kGK;
      const bool okr = r0 + rr < re;
      xa[col][rr] = (okr && a0 + col < k) ? AS[(long long)(a0 + col) * m + r0 + rr] : 0.0;
      xb[col][rr] = (okr && b0 + col < k) ? AS[(long long)(b0 + col) * m + r0 + rr] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < kGK; ++kk) {
      const double u0 = xa[ty * 2][kk], u1 = xa[ty * 2 + 1][kk];
      const double v0 = xb[tx * 2][kk], v1 = xb[tx * 2 + 1][kk];
      acc00 = fma(u0, v0, acc00);
      acc01 = fma(u0, v1, acc01);
      acc10 = fma(u1, v0, acc10);
      acc11 = fma(u1, v1, acc11);
    }
    __syncthreads();
  }
  double* out = part + ((long long)sl * npairs + pidx) * (kGT * kGT);
  out[(ty * 2) * kGT + tx * 2] = acc00;
  out[(ty * 2) * kGT + tx * 2 + 1] = acc01;
  out[(ty * 2 + 1) * kGT + tx * 2] = acc10;
  out[(ty * 2 + 1) * kGT + tx * 2 + 1] = acc11;
}

__global__ void gram_fin_kernel(const double* __restrict__ part, int nslices, int npairs, int k,
                                double* __restrict__ G) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)k * k) return;
  const int r = (int)(idx % k), c = (int)(idx / k);
  const int a = max(r, c), b = min(r, c);
  const int pidx = (a / kGT) * (a / kGT + 1) / 2 + b / kGT;
  const int off = (a % kGT) * kGT + (b % kGT);
  double s = 0.0;
  for (int q = 0; q < nslices; ++q) s += part[((long long)q * npairs + pidx) * (kGT * kGT) + off];
  G[idx] = s;
}

size_t gram_part_doubles(int m, int k) {
  const GramPlan g = gram_plan(m, k);
  return (size_t)g.nslices * g.npairs * kGT * kGT;
}

void gram(const double* AS, int m, int k, double* part, double* G, cudaStream_t s) {
  const GramPlan g = gram_plan(m, k);
  gram_part_kernel<<<dim3(g.npairs, g.nslices), 256, 0, s>>>(AS, m, k, g.slice, g.npairs, part);
  gram_fin_kernel<<<(unsigned)(((long long)k * k + 255) / 256), 256, 0, s>>>(part, g.nslices, g.npairs, k, G);
}

// Cholesky G = L L^T in place (lower triangle of the column-major k x k G).
// For k > kCholSmemK (G too large for one block's shared memory) it runs
// blocked right-looking, kCb columns a panel, as stream-ordered launches:
//   chol_block_kernel: one warp factors the panel's diagonal block D in
//     shared memory and writes it back;
//   chol_rows_kernel: each CTA solves kCb of the rows below it, L_i = G_i D^-T;
//   chol_update_kernel: one CTA per 32 x 32 tile of the trailing lower
//     triangle subtracts the panel's outer product, G_IJ -= L_I L_J^T.
// FP64 runs at two lanes per clock per SM on this part, so the k^3 / 6
// multiply-adds are spread over many SMs instead of one.  A pivot at or below
// 1e-12 of its column's initial squared norm (diag0, saved first) means the
// selected columns are linearly dependent to working precision: the pivot
// is replaced by 1 and status[0] = 1.
constexpr int kCb = 32;

__global__ void chol_diag_kernel(const double* __restrict__ G, int k, double* __restrict__ diag0) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < k) diag0[j] = G[(long long)j * k + j];
}

__global__ void __launch_bounds__(32) chol_block_kernel(double* __restrict__ G, int k, int j0,
                                                        const double* __restrict__ diag0,
                                                        int* __restrict__ status) {
  __shared__ double D[kCb][kCb + 1];   // rows x columns of the diagonal block
  const int lane = threadIdx.x;
  const int b = min(kCb, k - j0);
  for (int c = 0; c < b; ++c)
    if (lane >= c && lane < b) D[lane][c] = G[(long long)(j0 + c) * k + j0 + lane];
  __syncwarp();
  bool bad = false;
  for (int c = 0; c < b; ++c) {
    const double dd = D[c][c];
    const bool ok = dd > 1e-12 * diag0[j0 + c];
    const double d = ok ? sqrt(dd) : 1.0;
    bad |= !ok;
    __syncwarp();
    if (lane == c) D[c][c] = d;
    if (lane > c && lane < b) D[lane][c] /= d;
    __syncwarp();
    if (lane > c && lane < b) {
      const double lrc = D[lane][c];
      for (int q = c + 1; q <= lane; ++q) D[lane][q] -= lrc * D[q][c];
    }
    __syncwarp();
  }
  for (int c = 0; c < b; ++c)
    if (lane >= c && lane < b) G[(long long)(j0 + c) * k + j0 + lane] = D[lane][c];
  if (lane == 0 && bad) status[0] = 1;
}

// The rows below the factored diagonal block (kCb rows a CTA): row i of L
// solves x D^T = g by forward substitution over the block's columns.
__global__ void __launch_bounds__(32) chol_rows_kernel(double* __restrict__ G, int k, int j0) {
  __shared__ double D[kCb][kCb + 1];
  __shared__ double dinv[kCb];
  const int lane = threadIdx.x;
  const int b = min(kCb, k - j0);
  for (int c = 0; c < b; ++c)
    if (lane >= c && lane < b) D[lane][c] = G[(long long)(j0 + c) * k + j0 + lane];
  __syncwarp();
  if (lane < b) dinv[lane] = 1.0 / D[lane][lane];
  __syncwarp();
  const int i = j0 + b + blockIdx.x * kCb + lane;
  if (i >= k) return;
  double x[kCb];
#pragma unroll
  for (int c = 0; c < kCb; ++c) x[c] = c < b ? G[(long long)(j0 + c) * k + i] : 0.0;
#pragma unroll
  for (int c = 0; c < kCb; ++c) {
    if (c < b) {
      double v = x[c];
#pragma unroll
      for (int q = 0; q < c; ++q) v = fma(-x[q], D[c][q], v);
      x[c] = v * dinv[c];
    }
  }
#pragma unroll
  for (int c = 0; c < kCb; ++c)
    if (c < b) G[(long long)(j0 + c) * k + i] = x[c];
}

// Trailing update after the panel at j0 (width b): rows and columns from
// t0 = j0 + b on, lower tiles (ti >= tj) of 32 x 32, four outputs a thread.
__global__ void __launch_bounds__(256) chol_update_kernel(double* __restrict__ G, int k, int j0, int b) {
  __shared__ double PI[32][kCb + 1], PJ[32][kCb + 1];
  const int t0 = j0 + b;
  int ti = (int)((sqrtf(8.f * blockIdx.x + 1.f) - 1.f) * 0.5f);
  while (ti * (ti + 1) / 2 > (int)blockIdx.x) --ti;
  while ((ti + 1) * (ti + 2) / 2 <= (int)blockIdx.x) ++ti;
  const int tj = blockIdx.x - ti * (ti + 1) / 2;
  const int r0 = t0 + ti * 32, c0 = t0 + tj * 32;
  for (int e = threadIdx.x; e < 32 * kCb; e += 256) {
    const int r = e % 32, c = e / 32;
    const bool okc = c < b;
    PI[r][c] = (okc && r0 + r < k) ? G[(long long)(j0 + c) * k + r0 + r] : 0.0;
    PJ[r][c] = (okc && c0 + r < k) ? G[(long long)(j0 + c) * k + c0 + r] : 0.0;
  }
  __syncthreads();
  const int r = threadIdx.x % 32;
  const int i = r0 + r;
  if (i >= k) return;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int cl = threadIdx.x / 32 + 8 * q;
    const int l = c0 + cl;
    if (l >= k || l > i) continue;
    double acc = 0.0;
#pragma unroll 8
    for (int c = 0; c < b; ++c) acc = fma(PI[r][c], PJ[cl][c], acc);
    G[(long long)l * k + i] -= acc;
  }
}

// Linv = L^-1 by forward substitution L x = e_j, one warp per column j: the
// sum over the already known x_l is split across the lanes and the column
// is kept in shared memory.
constexpr int kLinvWarps = 8;
__global__ void __launch_bounds__(kLinvWarps * 32) linv_kernel(const double* __restrict__ G, int k,
                                                                double* __restrict__ Linv) {
  extern __shared__ double xs[];   // kLinvWarps x k
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int j = blockIdx.x * kLinvWarps + w;
  if (j >= k) return;
  double* x = xs + (size_t)w * k;
  for (int i = lane; i < j; i += 32) Linv[(long long)j * k + i] = 0.0;
  for (int i = j; i < k; ++i) {
    double part = 0.0;
    for (int l = j + lane; l < i; l += 32) part = fma(G[(long long)l * k + i], x[l], part);
    part = warp_sum(part);
    if (lane == 0) {
      const double v = ((i == j) ? 1.0 : 0.0) - part;
      x[i] = v / G[(long long)i * k + i];
    }
    __syncwarp();
  }
  for (int i = j + lane; i < k; i += 32) Linv[(long long)j * k + i] = x[i];
}

// For k <= kCholSmemK one block factors G held in shared memory (one launch;
// faster than the blocked form at these sizes): the k steps of the unblocked
// right-looking update read shared memory; L is written back over G.
constexpr int kCholSmemK = 128;
__global__ void __launch_bounds__(1024) chol_smem_kernel(double* __restrict__ Gg, int k, int* __restrict__ status) {
  extern __shared__ double G[];   // k x k, column-major
  __shared__ int bad;
  __shared__ double diag0[kCholSmemK];
  if (threadIdx.x == 0) bad = 0;
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) G[e] = Gg[e];
  __syncthreads();
  for (int j = threadIdx.x; j < k; j += blockDim.x) diag0[j] = G[j * k + j];
  __syncthreads();
  for (int j = 0; j < k; ++j) {
    if (threadIdx.x == 0) {
      // a pivot at or below 1e-12 of its column's squared norm: the selected
      // columns are linearly dependent to working precision
      const double d = G[j * k + j];
      const bool ok = d > 1e-12 * diag0[j];
      if (!ok) bad = 1;
      G[j * k + j] = ok ? sqrt(d) : 1.0;
    }
    __syncthreads();
    const double d = G[j * k + j];
    for (int i = j + 1 + threadIdx.x; i < k; i += blockDim.x) G[j * k + i] /= d;
    __syncthreads();
    const int rem = k - j - 1;
    for (int e = threadIdx.x; e < rem * rem; e += blockDim.x) {
      const int i = j + 1 + e % rem, l = j + 1 + e / rem;
      if (l <= i) G[l * k + i] -= G[j * k + i] * G[j * k + l];
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) Gg[e] = G[e];
  if (threadIdx.x == 0 && bad) status[0] = 1;
}

// Cholesky of the k x k matrix in G (overwritten by L) and L^-1 into Linv
// (status[0] = 1 for a rank-deficient G).
void chol_inv(double* G, int k, double* Linv, int* status, cudaStream_t s) {
  if (k <= kCholSmemK) {
    const size_t smem = (size_t)k * k * sizeof(double);
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(chol_smem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    chol_smem_kernel<<<1, 1024, smem, s>>>(G, k, status);
  } else {
    // the initial diagonal is kept in Linv, which is written only afterwards
    double* diag0 = Linv;
    chol_diag_kernel<<<(k + 255) / 256, 256, 0, s>>>(G, k, diag0);
    for (int j0 = 0; j0 < k; j0 += kCb) {
      const int b = std::min(kCb, k - j0);
      const int below = k - j0 - b;
      chol_block_kernel<<<1, 32, 0, s>>>(G, k, j0, diag0, status);
      if (below > 0) {
        chol_rows_kernel<<<(below + kCb - 1) / kCb, 32, 0, s>>>(G, k, j0);
        const int T = (below + 31) / 32;
        chol_update_kernel<<<T * (T + 1) / 2, 256, 0, s>>>(G, k, j0, b);
      }
    }
  }
  const size_t smem = (size_t)kLinvWarps * k * sizeof(double);
  if (smem > 48 * 1024) cudaFuncSetAttribute(linv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  linv_kernel<<<(k + kLinvWarps - 1) / kLinvWarps, kLinvWarps * 32, smem, s>>>(G, k, Linv);
}

// Q = A_S L^-T (m x k): Q[i, j] = sum_{l <= j} A_S[i, l] Linv[j, l]; the
// double-float split of Q is stored alongside.
__global__ void q_kernel(const double* __restrict__ AS, const double* __restrict__ Linv, int m, int k,
                         double* __restrict__ Q, float* __restrict__ Qh, float* __restrict__ Ql) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)m * k) return;
  const int i = (int)(idx % m), j = (int)(idx / m);
  double acc = 0.0;
  for (int l = 0; l <= j; ++l) acc = fma(AS[(long long)l * m + i], Linv[(long long)l * k + j], acc);
  Q[idx] = acc;
  float h, lo;
  df_split(acc, h, lo);
  Qh[idx] = h;
  Ql[idx] = lo;
}

// --------------------------------------------------- W = Q^T A  (k x n) -----
// 32 (k) x 64 (n) outputs per block, 2 x 4 per thread, K = m in chunks of 16.
// Element (j, c) of W goes to W[j * wj + c * wc]; the double-float split to
// Wh / Wl (same positions) when those are not null.
template <typename TA>
__global__ void __launch_bounds__(256) w_kernel(const float* __restrict__ Qh, const float* __restrict__ Ql,
                                                const double* __restrict__ Q, const TA* __restrict__ A,
                                                long long lda, int m, int n, int k,
                                                double* __restrict__ W, long long wj, long long wc,
                                                float* __restrict__ Wh, float* __restrict__ Wl) {
  constexpr int BK = 16;
  __shared__ float qh[BK][33], ql[BK][33];
  __shared__ double qd[BK][33];
  __shared__ float as[BK][65];
  __shared__ double ad[BK][65];
  const int j0 = blockIdx.y * 32, c0 = blockIdx.x * 64;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;  // ty: 16 rows of j (x2), tx: 16 cols (x4)
  constexpr bool F64 = sizeof(TA) == 8;
  DF acc[2][4];
  double accd[2][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) { acc[a][b] = DF{0.f, 0.f}; accd[a][b] = 0.0; }
  for (int r0 = 0; r0 < m; r0 += BK) {
    for (int e = threadIdx.x; e < BK * 32; e += 256) {
      const int rr = e % BK, jj = e / BK;
      const bool ok = r0 + rr < m && j0 + jj < k;
      const long long o = (long long)(j0 + jj) * m + r0 + rr;
      if (F64) qd[rr][jj] = ok ? Q[o] : 0.0;
      else { qh[rr][jj] = ok ? Qh[o] : 0.f; ql[rr][jj] = ok ? Ql[o] : 0.f; }
    }
    for (int e = threadIdx.x; e < BK * 64; e += 256) {
      const int rr = e % BK, cc = e / BK;
      const bool ok = r0 + rr < m && c0 + cc < n;
      const double v = ok ? to_d<TA>(A[(long long)(c0 + cc) * lda + r0 + rr]) : 0.0;
      if (F64) ad[rr][cc] = v;
      else as[rr][cc] = (float)v;
    }
    __syncthreads();
#pragma unroll 4
    for (int rr = 0; rr < BK; ++rr) {
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          if (F64) accd[a][b] = fma(qd[rr][ty * 2 + a], ad[rr][tx * 4 + b], accd[a][b]);
          else df_fma(acc[a][b], as[rr][tx * 4 + b], qh[rr][ty * 2 + a], ql[rr][ty * 2 + a]);
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int j = j0 + ty * 2 + a, c = c0 + tx * 4 + b;
      if (j < k && c < n) {
        const double v = F64 ? accd[a][b] : (double)acc[a][b].s + (double)acc[a][b].c;
        const long long o = (long long)j * wj + (long long)c * wc;
        W[o] = v;
        if (Wh) {
          float h, lo;
          df_split(v, h, lo);
          Wh[o] = h;
          Wl[o] = lo;
        }
      }
    }
}

// The FP32/BF16 (double-float) form of w_kernel: 64 x 64 outputs per block,
// 4 x 4 per thread, so that each K step reads three 16-byte vectors of shared
// memory for 16 double-float multiply-adds; K chunks of 16 double-buffered
// through registers.  Each output's terms are added in the same order as in
// w_kernel, so the result is bit-identical.
constexpr int kDT = 64, kDK = 16, kDP = kDT + 4;

template <typename TA>
__global__ void __launch_bounds__(256) w_df_kernel(const float* __restrict__ Qh, const float* __restrict__ Ql,
                                                   const TA* __restrict__ A, long long lda, int m, int n, int k,
                                                   double* __restrict__ W, long long wj, long long wc,
                                                   float* __restrict__ Wh, float* __restrict__ Wl) {
  __shared__ __align__(16) float sq[2][2][kDK][kDP];   // [buffer][hi, lo][row of the chunk][j]
  __shared__ __align__(16) float sa[2][kDK][kDP];      // [buffer][row of the chunk][column]
  const int j0 = blockIdx.y * kDT, c0 = blockIdx.x * kDT;
  const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
  const int rr = tid % kDK, cq = tid / kDK;   // staging: row rr, columns cq + 16 v
  float rh[4], rl[4], ra[4];
  DF acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = DF{0.f, 0.f};
  auto fetch = [&](int r0) {
    const int r = r0 + rr;
    const bool okr = r < m;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int x = cq + 16 * v;
      const bool okq = okr && j0 + x < k, oka = okr && c0 + x < n;
      rh[v] = okq ? Qh[(long long)(j0 + x) * m + r] : 0.f;
      rl[v] = okq ? Ql[(long long)(j0 + x) * m + r] : 0.f;
      ra[v] = oka ? (float)to_d<TA>(A[(long long)(c0 + x) * lda + r]) : 0.f;
    }
  };
  auto stage = [&](int b) {
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      sq[b][0][rr][cq + 16 * v] = rh[v];
      sq[b][1][rr][cq + 16 * v] = rl[v];
      sa[b][rr][cq + 16 * v] = ra[v];
    }
  };
  fetch(0);
  stage(0);
  __syncthreads();
  int buf = 0;
  for (int r0 = 0; r0 < m; r0 += kDK) {
    const bool more = r0 + kDK < m;
    if (more) fetch(r0 + kDK);
#pragma unroll 4
    for (int kk = 0; kk < kDK; ++kk) {
      const float4 qh4 = *reinterpret_cast<const float4*>(&sq[buf][0][kk][ty * 4]);
      const float4 ql4 = *reinterpret_cast<const float4*>(&sq[buf][1][kk][ty * 4]);
      const float4 a4 = *reinterpret_cast<const float4*>(&sa[buf][kk][tx * 4]);
      const float qh[4] = {qh4.x, qh4.y, qh4.z, qh4.w}, ql[4] = {ql4.x, ql4.y, ql4.z, ql4.w};
      const float av[4] = {a4.x, a4.y, a4.z, a4.w};
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) df_fma(acc[a][b], av[b], qh[a], ql[a]);
    }
    if (more) stage(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int j = j0 + ty * 4 + a, c = c0 + tx * 4 + b;
      if (j < k && c < n) {
        const double v = (double)acc[a][b].s + (double)acc[a][b].c;
        const long long o = (long long)j * wj + (long long)c * wc;
        W[o] = v;
        if (Wh) {
          float h, lo;
          df_split(v, h, lo);
          Wh[o] = h;
          Wl[o] = lo;
        }
      }
    }
}

// W = Q^T A launch: FP64 A on w_kernel, FP32/BF16 A on w_df_kernel.
template <typename TA>
void launch_w(const float* Qh, const float* Ql, const double* Q, const TA* A, long long lda, int m, int n, int k,
              double* W, long long wj, long long wc, float* Wh, float* Wl, cudaStream_t s) {
  if constexpr (sizeof(TA) == 8)
    w_kernel<TA><<<dim3((n + 63) / 64, (k + 31) / 32), 256, 0, s>>>(Qh, Ql, Q, A, lda, m, n, k, W, wj, wc, Wh, Wl);
  else
    w_df_kernel<TA><<<dim3((n + kDT - 1) / kDT, (k + kDT - 1) / kDT), 256, 0, s>>>(Qh, Ql, A, lda, m, n, k, W, wj,
                                                                                 wc, Wh, Wl);
}

// ------------------------------------ R = A - Q W (m x n) with epilogues -----
// 64 x 64 outputs per block, 4 x 4 per thread, K = k in chunks of 16.
// Writes R (FP32, or FP64 for FP64 input) when Rout != null, dA = 2 g R when
// dA != null, and a per-block partial of ||R||^2.
template <typename TA>
__global__ void __launch_bounds__(256) r_kernel(const float* __restrict__ Qh, const float* __restrict__ Ql,
                                                const double* __restrict__ Q, const float* __restrict__ Wh,
                                                const float* __restrict__ Wl, const double* __restrict__ W,
                                                const TA* __restrict__ A, long long lda, int m, int n, int k,
                                                void* __restrict__ Rout, TA* __restrict__ dA, long long ldda,
                                                double g2, double* __restrict__ loss_part) {
  constexpr int BK = 16;
  constexpr bool F64 = sizeof(TA) == 8;
  __shared__ float qh[BK][65], ql[BK][65], wh[BK][65], wl[BK][65];
  __shared__ double qd[BK][65], wd[BK][65];
  __shared__ double red[8];
  const int i0 = blockIdx.x * 64, c0 = blockIdx.y * 64;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  DF acc[4][4];
  double accd[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) { acc[a][b] = DF{0.f, 0.f}; accd[a][b] = 0.0; }
  for (int j0 = 0; j0 < k; j0 += BK) {
    for (int e = threadIdx.x; e < BK * 64; e += 256) {
      const int ii = e % 64, jj = e / 64;   // Q: rows contiguous
      const bool okq = i0 + ii < m && j0 + jj < k;
      const long long oq = (long long)(j0 + jj) * m + i0 + ii;
      const int jj2 = e % BK, cc = e / BK;  // W: k contiguous per column
      const bool okw = j0 + jj2 < k && c0 + cc < n;
      const long long ow = (long long)(c0 + cc) * k + j0 + jj2;
      if (F64) {
        qd[jj][ii] = okq ? Q[oq] : 0.0;
        wd[jj2][cc] = okw ? W[ow] : 0.0;
      } else {
        qh[jj][ii] = okq ? Qh[oq] : 0.f;
        ql[jj][ii] = okq ? Ql[oq] : 0.f;
        wh[jj2][cc] = okw ? Wh[ow] : 0.f;
        wl[jj2][cc] = okw ? Wl[ow] : 0.f;
      }
    }
    __syncthreads();
#pragma unroll 2
    for (int jj = 0; jj < BK; ++jj) {
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          if (F64) accd[a][b] = fma(qd[jj][ty * 4 + a], wd[jj][tx * 4 + b], accd[a][b]);
          else df_fma2(acc[a][b], qh[jj][ty * 4 + a], ql[jj][ty * 4 + a], wh[jj][tx * 4 + b],
                       wl[jj][tx * 4 + b]);
        }
    }
    __syncthreads();
  }
  double sq = 0.0;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int i = i0 + ty * 4 + a, c = c0 + tx * 4 + b;
      if (i < m && c < n) {
        const double av = to_d<TA>(A[(long long)c * lda + i]);
        // a - (s + c) in double: the pair carries the product to ~2^-48
        const double r = F64 ? av - accd[a][b] : (av - (double)acc[a][b].s) - (double)acc[a][b].c;
        sq += r * r;
        if (Rout) {
          if (F64) ((double*)Rout)[(long long)c * m + i] = r;
          else ((float*)Rout)[(long long)c * m + i] = (float)r;
        }
        if (dA) dA[(long long)c * ldda + i] = from_d<TA>(g2 * r);
      }
    }
  sq = warp_sum(sq);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sq;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    loss_part[(long long)blockIdx.y * gridDim.x + blockIdx.x] = t;
  }
}

// The FP32/BF16 (double-float) form of r_kernel: the same 64 x 64 tile and
// 4 x 4 outputs per thread, with Q and W staged so that each K step reads
// four 16-byte vectors of shared memory for 16 double-float multiply-adds,
// and K chunks double-buffered through registers.  Same order of terms and
// of the loss partial sums as r_kernel, so the results are bit-identical.
template <typename TA>
__global__ void __launch_bounds__(256) r_df_kernel(const float* __restrict__ Qh, const float* __restrict__ Ql,
                                                   const float* __restrict__ Wh, const float* __restrict__ Wl,
                                                   const TA* __restrict__ A, long long lda, int m, int n, int k,
                                                   float* __restrict__ Rout, TA* __restrict__ dA, long long ldda,
                                                   double g2, double* __restrict__ loss_part) {
  __shared__ __align__(16) float sq[2][2][kDK][kDP];   // [buffer][hi, lo][j of the chunk][row]
  __shared__ __align__(16) float sw[2][2][kDK][kDP];   // [buffer][hi, lo][j of the chunk][column]
  __shared__ double red[8];
  const int i0 = blockIdx.x * kDT, c0 = blockIdx.y * kDT;
  const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
  // staging: Q rows ii = tid % 64 of chunk entries jq + 4 v; W entries jw = tid % 16 of columns cw + 16 v
  const int ii = tid % kDT, jq = tid / kDT;
  const int jw = tid % kDK, cw = tid / kDK;
  float qh_r[4], ql_r[4], wh_r[4], wl_r[4];
  DF acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = DF{0.f, 0.f};
  auto fetch = [&](int jb) {
    const bool oki = i0 + ii < m;
    const bool okw = jb + jw < k;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int j = jb + jq + 4 * v;
      const bool okq = oki && j < k;
      qh_r[v] = okq ? Qh[(long long)j * m + i0 + ii] : 0.f;
      ql_r[v] = okq ? Ql[(long long)j * m + i0 + ii] : 0.f;
      const int c = c0 + cw + 16 * v;
      const bool ok = okw && c < n;
      wh_r[v] = ok ? Wh[(long long)c * k + jb + jw] : 0.f;
      wl_r[v] = ok ? Wl[(long long)c * k + jb + jw] : 0.f;
    }
  };
  auto stage = [&](int b) {
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      sq[b][0][jq + 4 * v][ii] = qh_r[v];
      sq[b][1][jq + 4 * v][ii] = ql_r[v];
      sw[b][0][jw][cw + 16 * v] = wh_r[v];
      sw[b][1][jw][cw + 16 * v] = wl_r[v];
    }
  };
  fetch(0);
  stage(0);
  __syncthreads();
  int buf = 0;
  for (int jb = 0; jb < k; jb += kDK) {
    const bool more = jb + kDK < k;
    if (more) fetch(jb + kDK);
#pragma unroll 2
    for (int jj = 0; jj < kDK; ++jj) {
      const float4 qh4 = *reinterpret_cast<const float4*>(&sq[buf][0][jj][ty * 4]);
      const float4 ql4 = *reinterpret_cast<const float4*>(&sq[buf][1][jj][ty * 4]);
      const float4 wh4 = *reinterpret_cast<const float4*>(&sw[buf][0][jj][tx * 4]);
      const float4 wl4 = *reinterpret_cast<const float4*>(&sw[buf][1][jj][tx * 4]);
      const float qh[4] = {qh4.x, qh4.y, qh4.z, qh4.w}, ql[4] = {ql4.x, ql4.y, ql4.z, ql4.w};
      const float wh[4] = {wh4.x, wh4.y, wh4.z, wh4.w}, wl[4] = {wl4.x, wl4.y, wl4.z, wl4.w};
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) df_fma2(acc[a][b], qh[a], ql[a], wh[b], wl[b]);
    }
    if (more) stage(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }
  double sq_sum = 0.0;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int i = i0 + ty * 4 + a, c = c0 + tx * 4 + b;
      if (i < m && c < n) {
        const double av = to_d<TA>(A[(long long)c * lda + i]);
        // a - (s + c) in double: the pair carries the product to ~2^-48
        const double r = (av - (double)acc[a][b].s) - (double)acc[a][b].c;
        sq_sum += r * r;
        if (Rout) Rout[(long long)c * m + i] = (float)r;
        if (dA) dA[(long long)c * ldda + i] = from_d<TA>(g2 * r);
      }
    }
  sq_sum = warp_sum(sq_sum);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sq_sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    loss_part[(long long)blockIdx.y * gridDim.x + blockIdx.x] = t;
  }
}

__global__ void sum_kernel(const double* __restrict__ part, long long cnt, double scale,
                           double* __restrict__ out) {
  __shared__ double red[32];
  double a = 0.0;
  for (long long i = threadIdx.x; i < cnt; i += blockDim.x) a += part[i];
  a = block_sum(a, red);
  if (threadIdx.x == 0) out[0] = a * scale;
}

// ------------------------------ P = R W^T (m x k), split over column slices --
// partial[s][i + j*m] = sum over columns c of slice s of R[i, c] W[j, c].
template <typename TR>
__global__ void __launch_bounds__(256) rwt_kernel(const TR* __restrict__ R, const double* __restrict__ W,
                                                  int m, int n, int k, int slice,
                                                  TR* __restrict__ partial) {
  constexpr int BK = 16;
  __shared__ TR rs[BK][65];
  __shared__ TR ws[BK][33];
  const int i0 = blockIdx.x * 64, j0 = blockIdx.y * 32, sl = blockIdx.z;
  const int cb = sl * slice, ce = min(n, cb + slice);
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  TR acc[4][2];
#pragma unroll
  for (int a = 0; a < 4; ++a) { acc[a][0] = TR(0); acc[a][1] = TR(0); }
  for (int c0 = cb; c0 < ce; c0 += BK) {
    for (int e = threadIdx.x; e < BK * 64; e += 256) {
      const int ii = e % 64, cc = e / 64;
      rs[cc][ii] = (c0 + cc < ce && i0 + ii < m) ? R[(long long)(c0 + cc) * m + i0 + ii] : TR(0);
    }
    for (int e = threadIdx.x; e < BK * 32; e += 256) {
      const int jj = e % 32, cc = e / 32;
      ws[cc][jj] = (c0 + cc < ce && j0 + jj < k) ? (TR)W[(long long)(c0 + cc) * k + j0 + jj] : TR(0);
    }
    __syncthreads();
#pragma unroll 4
    for (int cc = 0; cc < BK; ++cc)
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        acc[a][0] = fma(rs[cc][ty * 4 + a], ws[cc][tx * 2 + 0], acc[a][0]);
        acc[a][1] = fma(rs[cc][ty * 4 + a], ws[cc][tx * 2 + 1], acc[a][1]);
      }
    __syncthreads();
  }
  TR* out = partial + (long long)sl * m * k;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int i = i0 + ty * 4 + a, j = j0 + tx * 2 + b;
      if (i < m && j < k) out[(long long)j * m + i] = acc[a][b];
    }
}

// FP32 form of rwt_kernel: 64 x 64 outputs per block, 4 x 4 per thread, two
// 16-byte shared-memory reads per K step for 16 FMAs, K chunks
// double-buffered through registers; same order of terms (bit-identical).
__global__ void __launch_bounds__(256) rwt_f32_kernel(const float* __restrict__ R, const double* __restrict__ W,
                                                      int m, int n, int k, int slice, float* __restrict__ partial) {
  __shared__ __align__(16) float rs[2][kDK][kDP];
  __shared__ __align__(16) float ws[2][kDK][kDP];
  const int i0 = blockIdx.x * kDT, j0 = blockIdx.y * kDT, sl = blockIdx.z;
  const int cb = sl * slice, ce = min(n, cb + slice);
  const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
  const int xi = tid % kDT, kq = tid / kDT;   // staging: row / entry xi of chunk columns kq + 4 v
  float rr[4], wr[4];
  float acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
  auto fetch = [&](int c0) {
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int c = c0 + kq + 4 * v;
      const bool okc = c < ce;
      rr[v] = (okc && i0 + xi < m) ? R[(long long)c * m + i0 + xi] : 0.f;
      wr[v] = (okc && j0 + xi < k) ? (float)W[(long long)c * k + j0 + xi] : 0.f;
    }
  };
  auto stage = [&](int b) {
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      rs[b][kq + 4 * v][xi] = rr[v];
      ws[b][kq + 4 * v][xi] = wr[v];
    }
  };
  if (cb < ce) {
    fetch(cb);
    stage(0);
  }
  __syncthreads();
  int buf = 0;
  for (int c0 = cb; c0 < ce; c0 += kDK) {
    const bool more = c0 + kDK < ce;
    if (more) fetch(c0 + kDK);
#pragma unroll 4
    for (int kk = 0; kk < kDK; ++kk) {
      const float4 r4 = *reinterpret_cast<const float4*>(&rs[buf][kk][ty * 4]);
      const float4 w4 = *reinterpret_cast<const float4*>(&ws[buf][kk][tx * 4]);
      const float ra[4] = {r4.x, r4.y, r4.z, r4.w}, wa[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(ra[a], wa[b], acc[a][b]);
    }
    if (more) stage(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }
  float* out = partial + (long long)sl * m * k;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int i = i0 + ty * 4 + a, j = j0 + tx * 4 + b;
      if (i < m && j < k) out[(long long)j * m + i] = acc[a][b];
    }
}

// P = R W^T (m x k) from the slices, added in slice order, in FP64.
template <typename TR>
__global__ void sum_slices_kernel(const TR* __restrict__ partial, int S, long long mk, double* __restrict__ P) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= mk) return;
  double p = 0.0;
  for (int s = 0; s < S; ++s) p += (double)partial[(long long)s * mk + idx];
  P[idx] = p;
}

// dA[:, S[j]] = -2 g sum_{l >= j} P[i, l] Linv[l, j].
template <typename TA>
__global__ void das_kernel(const double* __restrict__ P, const double* __restrict__ Linv, int m, int k,
                           const int* __restrict__ sel, double g2, TA* __restrict__ dA, long long ldda) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)m * k) return;
  const int i = (int)(idx % m), j = (int)(idx / m);
  double acc = 0.0;
  for (int l = j; l < k; ++l) acc += P[(long long)l * m + i] * Linv[(long long)j * k + l];
  dA[(long long)sel[j] * ldda + i] = from_d<TA>(-g2 * acc);
}

constexpr int kSlices = 16;

struct BwLayout {
  int* status;
  double *AS, *G, *gpart, *Linv, *Q, *W;
  float *Qh, *Ql, *Wh, *Wl;
  void* R;
  void* P;
  double* Psum;
  double* loss_part;
  double* loss_tmp;
  size_t bytes;
};

BwLayout bw_layout(void* ws, size_t cap, int dt, int64_t m, int64_t n, int32_t k, bool grad) {
  WsCarver c(ws, cap);
  BwLayout L{};
  L.status = c.take<int>(64);
  L.AS = c.take<double>((size_t)m * k);
  L.G = c.take<double>((size_t)k * k);
  L.gpart = c.take<double>(gram_part_doubles((int)m, k));
  L.Linv = c.take<double>((size_t)k * k);
  L.Q = c.take<double>((size_t)m * k);
  L.Qh = c.take<float>((size_t)m * k);
  L.Ql = c.take<float>((size_t)m * k);
  L.W = c.take<double>((size_t)k * n);
  L.Wh = c.take<float>((size_t)k * n);
  L.Wl = c.take<float>((size_t)k * n);
  const size_t rs = dt == CSS_F64 ? 8 : 4;
  L.R = grad ? (void*)c.take<char>((size_t)m * n * rs) : nullptr;
  L.P = grad ? (void*)c.take<char>((size_t)kSlices * m * k * rs) : nullptr;
  L.Psum = grad ? c.take<double>((size_t)m * k) : nullptr;
  L.loss_part = c.take<double>((size_t)((m + 63) / 64) * ((n + 63) / 64));
  L.loss_tmp = c.take<double>(1);
  L.bytes = c.off;
  return L;
}

template <typename TA>
css_status run_backward(const TA* A, int m, int n, long long lda, const int* sel, int k,
                        double grad_out, TA* dA, long long ldda, double* loss, const BwLayout& L,
                        const css_opts& o, cudaStream_t s) {
  using TR = typename AccOf<TA>::type;
  cudaMemsetAsync(L.status, 0, sizeof(int), s);
  const long long mk = (long long)m * k;
  gather_cols_kernel<TA><<<(unsigned)((mk + 255) / 256), 256, 0, s>>>(A, lda, m, sel, k, L.AS);
  gram(L.AS, m, k, L.gpart, L.G, s);
  chol_inv(L.G, k, L.Linv, L.status, s);
  q_kernel<<<(unsigned)((mk + 255) / 256), 256, 0, s>>>(L.AS, L.Linv, m, k, L.Q, L.Qh, L.Ql);
  launch_w<TA>(L.Qh, L.Ql, L.Q, A, lda, m, n, k, L.W, 1, k, L.Wh, L.Wl, s);
  const dim3 rg((m + 63) / 64, (n + 63) / 64);
  if constexpr (sizeof(TA) == 8)
    r_kernel<TA><<<rg, 256, 0, s>>>(L.Qh, L.Ql, L.Q, L.Wh, L.Wl, L.W, A, lda, m, n, k, dA ? L.R : nullptr,
                                    dA, ldda, 2.0 * grad_out, L.loss_part);
  else
    r_df_kernel<TA><<<rg, 256, 0, s>>>(L.Qh, L.Ql, L.Wh, L.Wl, A, lda, m, n, k,
                                       dA ? (float*)L.R : nullptr, dA, ldda, 2.0 * grad_out, L.loss_part);
  if (loss) sum_kernel<<<1, 512, 0, s>>>(L.loss_part, (long long)rg.x * rg.y, 1.0, loss);
  if (dA) {
    const int slice = (n + kSlices - 1) / kSlices;
    if constexpr (sizeof(TR) == 4)
      rwt_f32_kernel<<<dim3((m + kDT - 1) / kDT, (k + kDT - 1) / kDT, kSlices), 256, 0, s>>>(
          (const float*)L.R, L.W, m, n, k, slice, (float*)L.P);
    else
      rwt_kernel<TR><<<dim3((m + 63) / 64, (k + 31) / 32, kSlices), 256, 0, s>>>((const TR*)L.R, L.W, m, n,
                                                                                k, slice, (TR*)L.P);
    sum_slices_kernel<TR><<<(unsigned)((mk + 255) / 256), 256, 0, s>>>((const TR*)L.P, kSlices, mk, L.Psum);
    das_kernel<TA><<<(unsigned)((mk + 255) / 256), 256, 0, s>>>(L.Psum, L.Linv, m, k, sel, 2.0 * grad_out, dA,
                                                               ldda);
  }
  if (cudaGetLastError() != cudaSuccess) return CSS_ERR_CUDA;
  if (o.sync) {
    int st = 0;
    if (cudaMemcpyAsync(&st, L.status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return CSS_ERR_CUDA;
    if (st) return CSS_ERR_INVALID_ARG;   // A_S is rank deficient
  }
  return CSS_OK;
}

// ------------------------------------------------ embedding (Sec. 3.2) -----
// Copy of an m x l FP64 matrix to a caller buffer with leading dimension ld.
__global__ void copy_cols_kernel(const double* __restrict__ src, int m, int l, double* __restrict__ dst,
                                 long long ld) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)m * l) return;
  const int i = (int)(idx % m), j = (int)(idx / m);
  dst[(long long)j * ld + i] = src[idx];
}

struct EmbLayout {
  int* status;
  double *AS, *G, *gpart, *Linv, *Q1, *Q;
  float *Qh, *Ql;
  size_t bytes;
};

EmbLayout emb_layout(void* ws, size_t cap, int64_t m, int32_t l) {
  WsCarver c(ws, cap);
  EmbLayout L{};
  L.status = c.take<int>(64);
  L.AS = c.take<double>((size_t)m * l);
  L.G = c.take<double>((size_t)l * l);
  L.gpart = c.take<double>(gram_part_doubles((int)m, l));
  L.Linv = c.take<double>((size_t)l * l);
  L.Q1 = c.take<double>((size_t)m * l);
  L.Q = c.take<double>((size_t)m * l);
  L.Qh = c.take<float>((size_t)m * l);
  L.Ql = c.take<float>((size_t)m * l);
  L.bytes = c.off;
  return L;
}

// CholeskyQR2: A_S^T A_S = L1 L1^T, Q1 = A_S L1^-T; Q1^T Q1 = L2 L2^T,
// Q = Q1 L2^-T.  Then W = Q^T A (row t at W + t * ldw).
template <typename TA>
css_status run_embed(const TA* A, int m, int n, long long lda, const int* sel, int l, double* Qout,
                     long long ldq, double* W, long long ldw, const EmbLayout& L, const css_opts& o,
                     cudaStream_t s) {
  cudaMemsetAsync(L.status, 0, sizeof(int), s);
  const long long ml = (long long)m * l;
  const unsigned gb = (unsigned)((ml + 255) / 256);
  gather_cols_kernel<TA><<<gb, 256, 0, s>>>(A, lda, m, sel, l, L.AS);
  gram(L.AS, m, l, L.gpart, L.G, s);
  chol_inv(L.G, l, L.Linv, L.status, s);
  q_kernel<<<gb, 256, 0, s>>>(L.AS, L.Linv, m, l, L.Q1, L.Qh, L.Ql);
  gram(L.Q1, m, l, L.gpart, L.G, s);
  chol_inv(L.G, l, L.Linv, L.status, s);
  q_kernel<<<gb, 256, 0, s>>>(L.Q1, L.Linv, m, l, L.Q, L.Qh, L.Ql);
  if (W)
    launch_w<TA>(L.Qh, L.Ql, L.Q, A, lda, m, n, l, W, ldw, 1, nullptr, nullptr, s);
  if (Qout) copy_cols_kernel<<<gb, 256, 0, s>>>(L.Q, m, l, Qout, ldq);
  if (cudaGetLastError() != cudaSuccess) return CSS_ERR_CUDA;
  if (o.sync) {
    int st = 0;
    if (cudaMemcpyAsync(&st, L.status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return CSS_ERR_CUDA;
    if (st) return CSS_ERR_INVALID_ARG;   // A_S is rank deficient
  }
  return CSS_OK;
}

// The selected indices are device memory the caller wrote on `s`: read back
// in stream order (one synchronisation) and checked on the host.
css_status check_selection(const int32_t* sel, int32_t k, int64_t n, cudaStream_t s) {
  std::vector<int32_t> h(k);
  if (cudaMemcpyAsync(h.data(), sel, sizeof(int32_t) * k, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return CSS_ERR_CUDA;
  std::vector<char> seen(n, 0);
  for (int32_t v : h) {
    if (v < 0 || v >= n || seen[v]) return CSS_ERR_INVALID_ARG;
    seen[v] = 1;
  }
  return CSS_OK;
}

}  // namespace

size_t embed_workspace_bytes(int64_t m, int32_t l) { return emb_layout(nullptr, (size_t)-1, m, l).bytes; }

extern "C" css_status css_embed(const void* A, css_dtype dtype, int64_t m, int64_t n, int64_t lda,
                                const int32_t* sel, int32_t l, double* Q, int64_t ldq, double* W,
                                int64_t ldw, void* ws, size_t ws_bytes, const css_opts* opts,
                                css_stream_t stream) {
  css_opts o;
  css_opts_default(&o);
  if (opts) o = *opts;
  if (!A || !sel || (!Q && !W)) return CSS_ERR_INVALID_ARG;
  if (dtype != CSS_F64 && dtype != CSS_F32 && dtype != CSS_BF16) return CSS_ERR_INVALID_ARG;
  if (m < 1 || n < 1 || lda < m || l < 1 || l > 1024 || l > m || l > n) return CSS_ERR_INVALID_ARG;
  if (m > INT32_MAX || n > INT32_MAX) return CSS_ERR_INVALID_ARG;
  if ((Q && ldq < m) || (W && ldw < n)) return CSS_ERR_INVALID_ARG;
  if (!ws || ((uintptr_t)ws % kWsAlign) != 0) return CSS_ERR_WORKSPACE;
  EmbLayout L = emb_layout(ws, ws_bytes, m, l);
  if (L.bytes > ws_bytes) return CSS_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  css_status cs = check_selection(sel, l, n, s);
  if (cs != CSS_OK) return cs;
  switch (dtype) {
    case CSS_F64:
      return run_embed<double>((const double*)A, (int)m, (int)n, lda, sel, l, Q, ldq, W, ldw, L, o, s);
    case CSS_F32:
      return run_embed<float>((const float*)A, (int)m, (int)n, lda, sel, l, Q, ldq, W, ldw, L, o, s);
    default:
      return run_embed<__nv_bfloat16>((const __nv_bfloat16*)A, (int)m, (int)n, lda, sel, l, Q, ldq, W, ldw,
                                      L, o, s);
  }
}

size_t backward_workspace_bytes(int dtype, int64_t m, int64_t n, int32_t k) {
  return bw_layout(nullptr, (size_t)-1, dtype, m, n, k, true).bytes;
}

extern "C" css_status css_residual_backward(const void* A, css_dtype dtype, int64_t m, int64_t n,
                                            int64_t lda, const int32_t* sel, int32_t k,
                                            double grad_out, void* dA, int64_t ldda, double* loss,
                                            void* ws, size_t ws_bytes, const css_opts* opts,
                                            css_stream_t stream) {
  css_opts o;
  css_opts_default(&o);
  if (opts) o = *opts;
  if (!A || !sel || (!dA && !loss)) return CSS_ERR_INVALID_ARG;
  if (dtype != CSS_F64 && dtype != CSS_F32 && dtype != CSS_BF16) return CSS_ERR_INVALID_ARG;
  if (m < 1 || n < 1 || lda < m || k < 1 || k > 1024 || k > m || k > n) return CSS_ERR_INVALID_ARG;
  if (dA && ldda < m) return CSS_ERR_INVALID_ARG;
  if (m > INT32_MAX || n > INT32_MAX) return CSS_ERR_INVALID_ARG;
  if (!ws || ((uintptr_t)ws % kWsAlign) != 0) return CSS_ERR_WORKSPACE;
  BwLayout L = bw_layout(ws, ws_bytes, dtype, m, n, k, dA != nullptr);
  if (L.bytes > ws_bytes) return CSS_ERR_WORKSPACE;
  // the selected indices: in range and distinct (a small stream-ordered copy)
  cudaStream_t s = (cudaStream_t)stream;
  const css_status cs = check_selection(sel, k, n, s);
  if (cs != CSS_OK) return cs;
  switch (dtype) {
    case CSS_F64:
      return run_backward<double>((const double*)A, (int)m, (int)n, lda, sel, k, grad_out,
                                  (double*)dA, ldda, loss, L, o, s);
    case CSS_F32:
      return run_backward<float>((const float*)A, (int)m, (int)n, lda, sel, k, grad_out,
                                 (float*)dA, ldda, loss, L, o, s);
    default:
      return run_backward<__nv_bfloat16>((const __nv_bfloat16*)A, (int)m, (int)n, lda, sel, k,
                                         grad_out, (__nv_bfloat16*)dA, ldda, loss, L, o, s);
  }
}
