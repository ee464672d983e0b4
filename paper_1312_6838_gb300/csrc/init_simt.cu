// Initial scores on CUDA cores (the initialisation of Algorithms 1 and 3).
//
//   CSS :  f_i^(0) = ||A^T A_:i||^2 = A_:i^T C A_:i  with  C = A A^T
//          (the n x n matrix A^T A is never formed)
//   GCSS:  f_i^(0) = ||B^T A_:i||^2
//
// Both are register-tiled SIMT GEMMs with column-reduction epilogues; the
// product tile is never stored.  Partial sums over row tiles are written in
// FP64 and added in a fixed order, so results do not depend on scheduling.
#include "init.cuh"

namespace css {
namespace {

template <typename TA> __device__ __forceinline__ typename AccOf<TA>::type cvt_in(TA v);
template <> __device__ __forceinline__ double cvt_in<double>(double v) { return v; }
template <> __device__ __forceinline__ float cvt_in<float>(float v) { return v; }
template <> __device__ __forceinline__ float cvt_in<__nv_bfloat16>(__nv_bfloat16 v) {
  return __uint_as_float(((uint32_t)__bfloat16_as_ushort(v)) << 16);
}

// ---------------------------------------------------------------- SYRK ------
// C = A A^T (m x m, leading dimension m).  Only tile pairs bi <= bj are
// computed; the lower tile is written by mirroring.  TT x TT outputs per
// thread, 16 x 16 threads, K chunks of KC columns of A.
template <typename TA, int TT, int KC>
__device__ __forceinline__ void syrk_tile(const TA* __restrict__ A, long long lda, int m, int n,
                                          typename AccOf<TA>::type* __restrict__ C, long long ldc, int tile) {
  using Acc = typename AccOf<TA>::type;
  constexpr int BT = 16 * TT;
  __shared__ __align__(16) Acc As[KC][BT];
  __shared__ __align__(16) Acc Bs[KC][BT];
  const int nt = (m + BT - 1) / BT;
  // decode the linear index into (bi, bj), bi <= bj
  int idx = tile, bi = 0;
  while (idx >= nt - bi) { idx -= nt - bi; ++bi; }
  const int bj = bi + idx;
  const int i0 = bi * BT, j0 = bj * BT;
  const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
  Acc acc[TT][TT];
#pragma unroll
  for (int a = 0; a < TT; ++a)
#pragma unroll
    for (int b = 0; b < TT; ++b) acc[a][b] = Acc(0);
  for (int l0 = 0; l0 < n; l0 += KC) {
    for (int e = tid; e < KC * BT; e += 256) {
      const int kk = e / BT, rr = e % BT;
      const int l = l0 + kk;
      As[kk][rr] = (l < n && i0 + rr < m) ? cvt_in<TA>(A[(long long)l * lda + i0 + rr]) : Acc(0);
      Bs[kk][rr] = (l < n && j0 + rr < m) ? cvt_in<TA>(A[(long long)l * lda + j0 + rr]) : Acc(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < KC; ++kk) {
      Acc a[TT], b[TT];
#pragma unroll
      for (int q = 0; q < TT; ++q) { a[q] = As[kk][ty * TT + q]; b[q] = Bs[kk][tx * TT + q]; }
#pragma unroll
      for (int q = 0; q < TT; ++q)
#pragma unroll
        for (int w = 0; w < TT; ++w) acc[q][w] = fma(a[q], b[w], acc[q][w]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < TT; ++q) {
    const int i = i0 + ty * TT + q;
#pragma unroll
    for (int w = 0; w < TT; ++w) {
      const int j = j0 + tx * TT + w;
      if (i < m && j < m) {
        C[(long long)j * ldc + i] = acc[q][w];
        if (bi != bj) C[(long long)i * ldc + j] = acc[q][w];
      }
    }
  }
}

// ------------------------------------------- FP32-accumulating tiles -------
// FP32 or BF16 A: 128 x 128 outputs per block, 8 x 8 per thread as two 4 x 4
// quadrants (rows ty*4 + {0..3} and 64 + ty*4 + {0..3}, columns likewise with
// tx), so that each K step reads four 16-byte vectors from shared memory for
// 64 FMAs without bank conflicts.  K advances in chunks of 16 through two
// shared-memory buffers: the next chunk's global loads are in registers while
// the current chunk is multiplied.
constexpr int kFT = 128;            // tile edge
constexpr int kFK = 16;             // K chunk
constexpr int kFP = kFT + 4;        // row stride of the K-major operands (16-byte aligned)
constexpr int kFV = kFT * kFK / 256;  // elements each thread stages per operand

struct F32Acc {
  float v[8][8];
};

__device__ __forceinline__ void f32_zero(F32Acc& a) {
#pragma unroll
  for (int q = 0; q < 8; ++q)
#pragma unroll
    for (int w = 0; w < 8; ++w) a.v[q][w] = 0.f;
}

// acc += X[kk][rows] (x) Y[kk][cols] for the kFK steps of one staged chunk
template <int LD>
__device__ __forceinline__ void f32_chunk(const float* __restrict__ X, const float* __restrict__ Y, int ty,
                                          int tx, F32Acc& acc) {
#pragma unroll
  for (int kk = 0; kk < kFK; ++kk) {
    const float4 a0 = *reinterpret_cast<const float4*>(X + kk * LD + ty * 4);
    const float4 a1 = *reinterpret_cast<const float4*>(X + kk * LD + 64 + ty * 4);
    const float4 b0 = *reinterpret_cast<const float4*>(Y + kk * LD + tx * 4);
    const float4 b1 = *reinterpret_cast<const float4*>(Y + kk * LD + 64 + tx * 4);
    const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
    const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
    for (int q = 0; q < 8; ++q)
#pragma unroll
      for (int w = 0; w < 8; ++w) acc.v[q][w] = fmaf(a[q], b[w], acc.v[q][w]);
  }
}

// row (or column) index of this thread's q-th output within the tile
__device__ __forceinline__ int f32_idx(int t, int q) { return (q < 4 ? 0 : 64) + t * 4 + (q & 3); }

// C = A A^T for tile pair (bi, bj), bi <= bj (see syrk_tile).  The staged
// operands are A's rows i0.., j0.. over 16 consecutive columns: column-major
// A makes each of them a contiguous run.
template <typename TA>
__device__ __forceinline__ void syrk_tile_f32(const TA* __restrict__ A, long long lda, int m, int n,
                                              float* __restrict__ C, long long ldc, int tile) {
  __shared__ __align__(16) float sm[2][2][kFK][kFT];
  const int nt = (m + kFT - 1) / kFT;
  int idx = tile, bi = 0;
  while (idx >= nt - bi) { idx -= nt - bi; ++bi; }
  const int bj = bi + idx;
  const int i0 = bi * kFT, j0 = bj * kFT;
  const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
  F32Acc acc;
  f32_zero(acc);
  float ra[kFV], rb[kFV];
  // thread tid stages row rr = tid % 128 of columns l0 + tid / 128 + 2 v
  const int rr = tid % kFT, kk0 = tid / kFT;
  const bool oka = i0 + rr < m, okb = j0 + rr < m;
  const TA* pa = A + (long long)kk0 * lda + i0 + rr;
  const TA* pb = A + (long long)kk0 * lda + j0 + rr;
  const long long step = 2 * lda;
  auto fetch = [&](int l0) {
    const long long off = (long long)l0 * lda;
#pragma unroll
    for (int v = 0; v < kFV; ++v) {
      const bool okl = l0 + kk0 + 2 * v < n;
      ra[v] = (okl && oka) ? cvt_in<TA>(pa[off + v * step]) : 0.f;
      rb[v] = (okl && okb) ? cvt_in<TA>(pb[off + v * step]) : 0.f;
    }
  };
  auto stage = [&](int buf) {
#pragma unroll
    for (int v = 0; v < kFV; ++v) {
      sm[buf][0][kk0 + 2 * v][rr] = ra[v];
      sm[buf][1][kk0 + 2 * v][rr] = rb[v];
    }
  };
  fetch(0);
  stage(0);
  __syncthreads();
  int buf = 0;
  for (int l0 = 0; l0 < n; l0 += kFK) {
    const bool more = l0 + kFK < n;
    if (more) fetch(l0 + kFK);
    f32_chunk<kFT>(&sm[buf][0][0][0], &sm[buf][1][0][0], ty, tx, acc);
    if (more) stage(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int i = i0 + f32_idx(ty, q);
#pragma unroll
    for (int w = 0; w < 8; ++w) {
      const int j = j0 + f32_idx(tx, w);
      if (i < m && j < m) {
        C[(long long)j * ldc + i] = acc.v[q][w];
        if (bi != bj) C[(long long)i * ldc + j] = acc.v[q][w];
      }
    }
  }
}

// Column reduction (see colreduce_tile) with FP32 accumulation.  X and Y are
// K-contiguous, so 16 consecutive threads read 16 consecutive K entries of
// one row and write them transposed into the K-major staging buffers (row
// stride kFP keeps those writes to two-way bank conflicts).
template <typename TX, typename TA, int EPI>
__device__ __forceinline__ void colreduce_tile_f32(const TX* __restrict__ X, long long ldx,
                                                   const TA* __restrict__ Y, long long ldy, int K, int M,
                                                   int N, double* __restrict__ partial, int mb, int nb) {
  __shared__ __align__(16) float sm[2][2][kFK][kFP];
  const int r0 = mb * kFT, c0 = nb * kFT;
  const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
  F32Acc acc;
  f32_zero(acc);
  float rx[kFV], ry[kFV];
  // thread tid stages K entry kk of rows rr0 + 16 v.  FP32 Y: in a warp, 8
  // lanes read 8 consecutive K entries (32 bytes) of one of 4 rows, and the
  // transposed writes (bank 4 kk + rr mod 32 with the kFP stride) fall in 32
  // distinct banks.  BF16 Y: 16 lanes per row, so that each row's read is
  // still a whole 32-byte sector (the writes then pair up on banks).
  const int lane = tid & 31, wrp = tid >> 5;
  constexpr bool k16 = sizeof(TA) == 2;
  const int kk = k16 ? tid % kFK : (lane & 7) + 8 * (wrp & 1);
  const int rr0 = k16 ? tid / kFK : (lane >> 3) + 4 * (wrp >> 1);
  const int vx = (M - r0 - rr0 + kFK - 1) / kFK, vy = (N - c0 - rr0 + kFK - 1) / kFK;   // valid rows
  const TX* px = X + (long long)(r0 + rr0) * ldx + kk;
  const TA* py = Y + (long long)(c0 + rr0) * ldy + kk;
  const long long sx = kFK * ldx, sy = kFK * ldy;
  auto fetch = [&](int k0) {
    const bool okk = k0 + kk < K;
#pragma unroll
    for (int v = 0; v < kFV; ++v) {
      rx[v] = (okk && v < vx) ? (float)px[k0 + v * sx] : 0.f;
      ry[v] = (okk && v < vy) ? cvt_in<TA>(py[k0 + v * sy]) : 0.f;
    }
  };
  auto stage = [&](int buf) {
#pragma unroll
    for (int v = 0; v < kFV; ++v) {
      sm[buf][0][kk][rr0 + kFK * v] = rx[v];
      sm[buf][1][kk][rr0 + kFK * v] = ry[v];
    }
  };
  fetch(0);
  stage(0);
  __syncthreads();
  int buf = 0;
  for (int k0 = 0; k0 < K; k0 += kFK) {
    const bool more = k0 + kFK < K;
    if (more) fetch(k0 + kFK);
    f32_chunk<kFP>(&sm[buf][0][0][0], &sm[buf][1][0][0], ty, tx, acc);
    if (more) stage(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }
  // epilogue: per column, this thread's 8 rows summed in FP64, then the 16
  // row groups added in a fixed order (the staging buffers are free now)
  double* red = reinterpret_cast<double*>(&sm[0][0][0][0]);   // [16][kFT]
#pragma unroll
  for (int w = 0; w < 8; ++w) {
    const int cl = f32_idx(tx, w), i = c0 + cl;
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int r = r0 + f32_idx(ty, q);
      if (r < M && i < N) {
        const double d = (double)acc.v[q][w];
        if (EPI == 0) s += d * (double)cvt_in<TA>(Y[(long long)i * ldy + r]);
        else s += d * d;
      }
    }
    red[ty * kFT + cl] = s;
  }
  __syncthreads();
  for (int c = tid; c < kFT; c += 256) {
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < 16; ++q) s += red[q * kFT + c];
    if (c0 + c < N) partial[(long long)mb * N + c0 + c] = s;
  }
}

template <typename TA, int TT, int KC>
__global__ void __launch_bounds__(256, 2) syrk_kernel(const TA* __restrict__ A, long long lda, int m,
                                                   int n, typename AccOf<TA>::type* __restrict__ C,
                                                   long long ldc) {
  if constexpr (sizeof(typename AccOf<TA>::type) == 4) syrk_tile_f32<TA>(A, lda, m, n, C, ldc, blockIdx.x);
  else syrk_tile<TA, TT, KC>(A, lda, m, n, C, ldc, blockIdx.x);
}

// ------------------------------------------------------ column reduction ----
// D = X^T Y with X (K x M, ldx) and Y (K x N, ldy) both K-contiguous.
// partial[mb * n + i] = sum over the rows r of M-tile mb of
//     EPI == 0 :  D[r, i] * Y[r, i]       (CSS: C A dotted with A, needs M == K)
//     EPI == 1 :  D[r, i]^2               (GCSS: ||B^T a_i||^2)
template <typename TX, typename TA, int TT, int KC, int EPI>
__device__ __forceinline__ void colreduce_tile(const TX* __restrict__ X, long long ldx,
                                               const TA* __restrict__ Y, long long ldy, int K, int M,
                                               int N, double* __restrict__ partial, int mb, int nb) {
  using Acc = typename AccOf<TA>::type;
  constexpr int BT = 16 * TT;
  __shared__ __align__(16) Acc Xs[KC][BT + 1];
  __shared__ __align__(16) Acc Ys[KC][BT + 1];
  __shared__ double red[16][BT];
  const int r0 = mb * BT, c0 = nb * BT;
  const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
  Acc acc[TT][TT];
#pragma unroll
  for (int a = 0; a < TT; ++a)
#pragma unroll
    for (int b = 0; b < TT; ++b) acc[a][b] = Acc(0);
  for (int k0 = 0; k0 < K; k0 += KC) {
    for (int e = tid; e < KC * BT; e += 256) {
      const int rr = e / KC, kk = e % KC;  // consecutive threads walk K (contiguous)
      const int k = k0 + kk;
      Xs[kk][rr] = (k < K && r0 + rr < M) ? (Acc)X[(long long)(r0 + rr) * ldx + k] : Acc(0);
      Ys[kk][rr] = (k < K && c0 + rr < N) ? cvt_in<TA>(Y[(long long)(c0 + rr) * ldy + k]) : Acc(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < KC; ++kk) {
      Acc a[TT], b[TT];
#pragma unroll
      for (int q = 0; q < TT; ++q) { a[q] = Xs[kk][ty * TT + q]; b[q] = Ys[kk][tx * TT + q]; }
#pragma unroll
      for (int q = 0; q < TT; ++q)
#pragma unroll
        for (int w = 0; w < TT; ++w) acc[q][w] = fma(a[q], b[w], acc[q][w]);
    }
    __syncthreads();
  }
  // epilogue: per column, sum over this thread's TT rows in FP64
#pragma unroll
  for (int w = 0; w < TT; ++w) {
    const int i = c0 + tx * TT + w;
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < TT; ++q) {
      const int r = r0 + ty * TT + q;
      if (r < M && i < N) {
        const double d = (double)acc[q][w];
        if (EPI == 0) s += d * (double)cvt_in<TA>(Y[(long long)i * ldy + r]);
        else s += d * d;
      }
    }
    red[ty][tx * TT + w] = s;
  }
  __syncthreads();
  for (int c = tid; c < BT; c += 256) {
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < 16; ++q) s += red[q][c];
    if (c0 + c < N) partial[(long long)mb * N + c0 + c] = s;
  }
}

template <typename TX, typename TA, int TT, int KC, int EPI>
__global__ void __launch_bounds__(256) colreduce_kernel(const TX* __restrict__ X, long long ldx,
                                                       const TA* __restrict__ Y, long long ldy, int K,
                                                       int M, int N, double* __restrict__ partial) {
  if constexpr (sizeof(typename AccOf<TA>::type) == 4)
    colreduce_tile_f32<TX, TA, EPI>(X, ldx, Y, ldy, K, M, N, partial, blockIdx.y, blockIdx.x);
  else
    colreduce_tile<TX, TA, TT, KC, EPI>(X, ldx, Y, ldy, K, M, N, partial, blockIdx.y, blockIdx.x);
}

__global__ void sum_partials_kernel(const double* __restrict__ partial, int nblk, int n,
                                    double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += partial[(long long)b * n + i];
  out[i] = s;
}

template <typename TA> struct Tiles { static constexpr int TT = 8, KC = 16; };
template <> struct Tiles<double> { static constexpr int TT = 4, KC = 16; };

template <typename TA>
cudaError_t css_f0_simt_t(const void* A_, long long lda, int m, int n, void* C_, long long ldc,
                          double* partial, double* f, cudaStream_t s) {
  using Acc = typename AccOf<TA>::type;
  constexpr int TT = Tiles<TA>::TT, KC = Tiles<TA>::KC, BT = 16 * TT;
  const TA* A = reinterpret_cast<const TA*>(A_);
  Acc* C = reinterpret_cast<Acc*>(C_);
  const int nt = (m + BT - 1) / BT;
  syrk_kernel<TA, TT, KC><<<nt * (nt + 1) / 2, 256, 0, s>>>(A, lda, m, n, C, ldc);
  dim3 grid((n + BT - 1) / BT, nt);
  colreduce_kernel<Acc, TA, TT, KC, 0><<<grid, 256, 0, s>>>(C, ldc, A, lda, m, m, n, partial);
  sum_partials_kernel<<<(n + 255) / 256, 256, 0, s>>>(partial, nt, n, f);
  return cudaGetLastError();
}

template <typename TA>
cudaError_t gcss_f0_simt_t(const void* A_, long long lda, int m, int n, const void* B_,
                           long long ldb, int r, double* partial, double* f, cudaStream_t s) {
  using Acc = typename AccOf<TA>::type;
  constexpr int TT = Tiles<TA>::TT, KC = Tiles<TA>::KC, BT = 16 * TT;
  const TA* A = reinterpret_cast<const TA*>(A_);
  const Acc* B = reinterpret_cast<const Acc*>(B_);
  const int mt = (r + BT - 1) / BT;
  dim3 grid((n + BT - 1) / BT, mt);
  colreduce_kernel<Acc, TA, TT, KC, 1><<<grid, 256, 0, s>>>(B, ldb, A, lda, m, r, n, partial);
  sum_partials_kernel<<<(n + 255) / 256, 256, 0, s>>>(partial, mt, n, f);
  return cudaGetLastError();
}

// ------------------------------------------------------------ grouped -------
// One launch for the initial scores of many CSS problems: blockIdx.x runs
// over the concatenated tiles of all problems; start[g] is the first block of
// problem g (start[count] = grid).
__device__ __forceinline__ int group_of(const int* __restrict__ start, int count, int b) {
  int lo = 0, hi = count;   // start[lo] <= b < start[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (start[mid] <= b) lo = mid;
    else hi = mid;
  }
  return lo;
}

template <typename TA, int TT, int KC>
__global__ void __launch_bounds__(256, 2) syrk_grouped(const F0Item* __restrict__ items,
                                                    const int* __restrict__ start, int count) {
  using Acc = typename AccOf<TA>::type;
  const int g = group_of(start, count, blockIdx.x);
  const F0Item it = items[g];
  if constexpr (sizeof(Acc) == 4)
    syrk_tile_f32<TA>(reinterpret_cast<const TA*>(it.A), it.lda, it.m, it.n, reinterpret_cast<Acc*>(it.C),
                      it.ldc, blockIdx.x - start[g]);
  else
    syrk_tile<TA, TT, KC>(reinterpret_cast<const TA*>(it.A), it.lda, it.m, it.n,
                          reinterpret_cast<Acc*>(it.C), it.ldc, blockIdx.x - start[g]);
}

template <typename TA, int TT, int KC>
__global__ void __launch_bounds__(256) colreduce_grouped(const F0Item* __restrict__ items,
                                                         const int* __restrict__ start, int count) {
  using Acc = typename AccOf<TA>::type;
  constexpr int BT = 16 * TT;
  const int g = group_of(start, count, blockIdx.x);
  const F0Item it = items[g];
  const int local = blockIdx.x - start[g];
  const int nbs = (it.n + BT - 1) / BT;
  if constexpr (sizeof(Acc) == 4)
    colreduce_tile_f32<Acc, TA, 0>(reinterpret_cast<const Acc*>(it.C), it.ldc,
                                   reinterpret_cast<const TA*>(it.A), it.lda, it.m, it.m, it.n, it.partial,
                                   local / nbs, local % nbs);
  else
    colreduce_tile<Acc, TA, TT, KC, 0>(reinterpret_cast<const Acc*>(it.C), it.ldc,
                                       reinterpret_cast<const TA*>(it.A), it.lda, it.m, it.m, it.n,
                                       it.partial, local / nbs, local % nbs);
}

template <int BT>
__global__ void sum_partials_grouped(const F0Item* __restrict__ items, const int* __restrict__ start,
                                     int count) {
  const int g = group_of(start, count, blockIdx.x);
  const F0Item it = items[g];
  const int i = (blockIdx.x - start[g]) * blockDim.x + threadIdx.x;
  if (i >= it.n) return;
  const int nblk = (it.m + BT - 1) / BT;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += it.partial[(long long)b * it.n + i];
  it.f[i] = s;
}

template <typename TA>
cudaError_t css_f0_grouped_t(const F0Item* items, const int* starts, const F0Grid& grid, int count,
                             cudaStream_t s) {
  constexpr int TT = Tiles<TA>::TT, KC = Tiles<TA>::KC, BT = 16 * TT;
  syrk_grouped<TA, TT, KC><<<grid.syrk, 256, 0, s>>>(items, starts, count);
  colreduce_grouped<TA, TT, KC><<<grid.colreduce, 256, 0, s>>>(items, starts + (count + 1), count);
  sum_partials_grouped<BT><<<grid.sums, 256, 0, s>>>(items, starts + 2 * (count + 1), count);
  return cudaGetLastError();
}

}  // namespace

F0Grid css_f0_grouped_starts(int dtype, const int* m, const int* n, int count, int* starts) {
  const int BT = (dtype == CSS_F64) ? 64 : 128;
  F0Grid G{};
  int* s0 = starts;
  int* s1 = starts + (count + 1);
  int* s2 = starts + 2 * (count + 1);
  for (int g = 0; g < count; ++g) {
    const int nt = (m[g] + BT - 1) / BT;
    s0[g] = G.syrk;
    s1[g] = G.colreduce;
    s2[g] = G.sums;
    G.syrk += nt * (nt + 1) / 2;
    G.colreduce += nt * ((n[g] + BT - 1) / BT);
    G.sums += (n[g] + 255) / 256;
  }
  s0[count] = G.syrk;
  s1[count] = G.colreduce;
  s2[count] = G.sums;
  return G;
}

cudaError_t css_f0_grouped(int dtype, const F0Item* items, const int* starts, const F0Grid& grid,
                           int count, cudaStream_t s) {
  switch (dtype) {
    case CSS_F64: return css_f0_grouped_t<double>(items, starts, grid, count, s);
    case CSS_F32: return css_f0_grouped_t<float>(items, starts, grid, count, s);
    default: return css_f0_grouped_t<__nv_bfloat16>(items, starts, grid, count, s);
  }
}

size_t css_f0_partial_doubles(int dtype, int m, int n) {
  const int BT = (dtype == CSS_F64) ? 64 : 128;
  return (size_t)((m + BT - 1) / BT) * (size_t)n;
}
size_t gcss_f0_partial_doubles(int dtype, int r, int n) {
  const int BT = (dtype == CSS_F64) ? 64 : 128;
  return (size_t)((r + BT - 1) / BT) * (size_t)n;
}

cudaError_t css_f0_simt(int dtype, const void* A, long long lda, int m, int n, void* C, long long ldc,
                        double* partial, double* f, cudaStream_t s) {
  switch (dtype) {
    case CSS_F64: return css_f0_simt_t<double>(A, lda, m, n, C, ldc, partial, f, s);
    case CSS_F32: return css_f0_simt_t<float>(A, lda, m, n, C, ldc, partial, f, s);
    default: return css_f0_simt_t<__nv_bfloat16>(A, lda, m, n, C, ldc, partial, f, s);
  }
}

cudaError_t gcss_f0_simt(int dtype, const void* A, long long lda, int m, int n, const void* B,
                         long long ldb, int r, double* partial, double* f, cudaStream_t s) {
  switch (dtype) {
    case CSS_F64: return gcss_f0_simt_t<double>(A, lda, m, n, B, ldb, r, partial, f, s);
    case CSS_F32: return gcss_f0_simt_t<float>(A, lda, m, n, B, ldb, r, partial, f, s);
    default: return gcss_f0_simt_t<__nv_bfloat16>(A, lda, m, n, B, ldb, r, partial, f, s);
  }
}

}  // namespace css
