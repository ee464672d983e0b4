// Random projection B = A Omega (Sec. 5.1, Algorithm 2).
//
// Algorithm 2 has every mapper keep an in-memory partial sum
// Bbar = sum_{i in block} A_:i Omega_i: over its columns and the reducers add
// the c partials row by row.  Here the column range is split into S slices;
// each slice's partial product is one tile grid of the GEMM, and a second
// kernel adds the S partials in a fixed order (reproducible results).
#include "project.cuh"
#include "tc.cuh"

#include <algorithm>
#include <cstring>

using namespace css;

namespace {

template <typename TA> __device__ __forceinline__ typename AccOf<TA>::type cvt(TA v);
template <> __device__ __forceinline__ double cvt<double>(double v) { return v; }
template <> __device__ __forceinline__ float cvt<float>(float v) { return v; }
template <> __device__ __forceinline__ float cvt<__nv_bfloat16>(__nv_bfloat16 v) {
  return __uint_as_float(((uint32_t)__bfloat16_as_ushort(v)) << 16);
}

constexpr int kSlices = 8;

// partial[s][i + j*m] = sum over columns l of slice s of A[i, l] * Omega[l, j]
template <typename TA, int TT, int KC>
__global__ void __launch_bounds__(256) project_simt_kernel(const TA* __restrict__ A, long long lda,
                                                          const TA* __restrict__ Om, long long ldo,
                                                          int m, int n, int r, int slice_len,
                                                          typename AccOf<TA>::type* __restrict__ partial) {
  using Acc = typename AccOf<TA>::type;
  constexpr int BT = 16 * TT;
  __shared__ __align__(16) Acc As[KC][BT];
  __shared__ __align__(16) Acc Os[KC][BT + 1];
  const int i0 = blockIdx.x * BT, j0 = blockIdx.y * BT, sl = blockIdx.z;
  const int l_begin = sl * slice_len, l_end = min(n, l_begin + slice_len);
  const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
  Acc acc[TT][TT];
#pragma unroll
  for (int a = 0; a < TT; ++a)
#pragma unroll
    for (int b = 0; b < TT; ++b) acc[a][b] = Acc(0);
  for (int l0 = l_begin; l0 < l_end; l0 += KC) {
    for (int e = tid; e < KC * BT; e += 256) {
      const int kk = e / BT, rr = e % BT;           // A: rows contiguous
      const int l = l0 + kk;
      As[kk][rr] = (l < l_end && i0 + rr < m) ? cvt<TA>(A[(long long)l * lda + i0 + rr]) : Acc(0);
      const int jj = e / KC, k2 = e % KC;           // Omega: columns of length n contiguous
      const int l2 = l0 + k2;
      Os[k2][jj] = (l2 < l_end && j0 + jj < r) ? cvt<TA>(Om[(long long)(j0 + jj) * ldo + l2]) : Acc(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < KC; ++kk) {
      Acc a[TT], b[TT];
#pragma unroll
      for (int q = 0; q < TT; ++q) { a[q] = As[kk][ty * TT + q]; b[q] = Os[kk][tx * TT + q]; }
#pragma unroll
      for (int q = 0; q < TT; ++q)
#pragma unroll
        for (int w = 0; w < TT; ++w) acc[q][w] = fma(a[q], b[w], acc[q][w]);
    }
    __syncthreads();
  }
  Acc* out = partial + (long long)sl * m * r;
#pragma unroll
  for (int q = 0; q < TT; ++q)
#pragma unroll
    for (int w = 0; w < TT; ++w) {
      const int i = i0 + ty * TT + q, j = j0 + tx * TT + w;
      if (i < m && j < r) out[(long long)j * m + i] = acc[q][w];
    }
}

// Reducers: B[i, j] = sum_s partial[s][i, j], slices in order.
template <typename Acc>
__global__ void project_reduce_kernel(const Acc* __restrict__ partial, int S, int m, int r,
                                      Acc* __restrict__ B, long long ldb) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)m * r) return;
  const int i = (int)(idx % m), j = (int)(idx / m);
  Acc s = Acc(0);
  for (int q = 0; q < S; ++q) s += partial[(long long)q * m * r + idx];
  B[(long long)j * ldb + i] = s;
}

template <typename TA>
cudaError_t project_simt(const void* A, long long lda, const void* Om, long long ldo, int m, int n,
                         int r, void* B, long long ldb, void* partial, cudaStream_t s) {
  using Acc = typename AccOf<TA>::type;
  constexpr int TT = sizeof(Acc) == 8 ? 4 : 4, KC = 16, BT = 16 * TT;
  const int S = kSlices;
  const int slice_len = (n + S - 1) / S;
  dim3 grid((m + BT - 1) / BT, (r + BT - 1) / BT, S);
  project_simt_kernel<TA, TT, KC><<<grid, 256, 0, s>>>((const TA*)A, lda, (const TA*)Om, ldo, m, n,
                                                      r, slice_len, (Acc*)partial);
  const long long tot = (long long)m * r;
  project_reduce_kernel<Acc><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>((const Acc*)partial, S, m, r,
                                                                         (Acc*)B, ldb);
  return cudaGetLastError();
}

size_t accsz(int dt) { return dt == CSS_F64 ? 8 : 4; }

}  // namespace

constexpr int kMaxTcSlices = 32;

size_t project_workspace_bytes(int dtype, int64_t m, int64_t n, int64_t r) {
  (void)n;
  const size_t sl = std::max(kSlices, kMaxTcSlices);
  return kStatusBytes + align_up((size_t)sl * m * r * accsz(dtype));
}

extern "C" css_status css_project(const void* A, css_dtype dtype, int64_t m, int64_t n, int64_t lda,
                                  const void* Omega, int64_t r, int64_t ldo, void* Bout, int64_t ldb,
                                  void* ws, size_t ws_bytes, const css_opts* opts,
                                  css_stream_t stream) {
  (void)opts;
  if (!A || !Omega || !Bout) return CSS_ERR_INVALID_ARG;
  if (dtype != CSS_F64 && dtype != CSS_F32 && dtype != CSS_BF16) return CSS_ERR_INVALID_ARG;
  if (m < 1 || n < 1 || r < 1 || lda < m || ldo < n || ldb < m) return CSS_ERR_INVALID_ARG;
  if (m > INT32_MAX || n > INT32_MAX || r > INT32_MAX) return CSS_ERR_INVALID_ARG;
  if (!ws || ((uintptr_t)ws % kWsAlign) != 0) return CSS_ERR_WORKSPACE;
  if (ws_bytes < project_workspace_bytes(dtype, m, n, r)) return CSS_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  void* partial = (char*)ws + kStatusBytes;
  int* err = (int*)ws;
  css_opts o0;
  css_opts_default(&o0);
  const css_opts& oo = opts ? *opts : o0;
  cudaError_t e;
  // BF16 input: tcgen05 split-K GEMM (Algorithm 2's per-block partial sums in
  // TMEM), then the same fixed-order reduction as the SIMT path
  if (dtype == CSS_BF16 && oo.init_path != 1 && css::tc::supported(A, lda, (int)m, (int)r) &&
      css::tc::supported(Omega, ldo, (int)n, (int)r)) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int slices = std::min(kMaxTcSlices, css::tc::project_slices((int)m, sms > 0 ? sms : 1));
    if ((e = cudaMemsetAsync(err, 0, sizeof(int), s)) != cudaSuccess) return CSS_ERR_CUDA;
    e = css::tc::project_partials(A, lda, (int)m, (int)n, Omega, ldo, (int)r, slices, (float*)partial, err,
                                  oo.spin_budget_ns ? oo.spin_budget_ns : 2000000000ull, s);
    if (e != cudaSuccess) return CSS_ERR_CUDA;
    const long long tot = m * r;
    project_reduce_kernel<float><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(
        (const float*)partial, slices, (int)m, (int)r, (float*)Bout, ldb);
    if ((e = cudaGetLastError()) != cudaSuccess) return CSS_ERR_CUDA;
    if (oo.sync) {
      int h = 0;
      if (cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess)
        return CSS_ERR_CUDA;
      if (h) return (css_status)h;
    }
    return CSS_OK;
  }
  switch (dtype) {
    case CSS_F64: e = project_simt<double>(A, lda, Omega, ldo, (int)m, (int)n, (int)r, Bout, ldb, partial, s); break;
    case CSS_F32: e = project_simt<float>(A, lda, Omega, ldo, (int)m, (int)n, (int)r, Bout, ldb, partial, s); break;
    default: e = project_simt<__nv_bfloat16>(A, lda, Omega, ldo, (int)m, (int)n, (int)r, Bout, ldb, partial, s); break;
  }
  if (e != cudaSuccess) return CSS_ERR_CUDA;
  const css_opts o = [&] { css_opts t; css_opts_default(&t); return opts ? *opts : t; }();
  if (o.sync) {
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return CSS_ERR_CUDA;
  }
  return CSS_OK;
}
