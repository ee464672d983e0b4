// The random matrix Omega of Sec. 5.1 drawn on the device, and the random
// projection B = A Omega with a generated Omega (Algorithm 2).
//
// Entry (i, j) of Omega comes from one block of the counter-based generator
// Philox4x32-10 (Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as
// easy as 1, 2, 3", SC 2011) at counter (i, j, 0, 0) under key (seed mod 2^32,
// seed >> 32), so any entry can be drawn anywhere without a stream of state:
//   Gaussian     Box-Muller on the first two words, scaled to variance 1/r;
//   sparse sign  nonzero when the first word is below floor(2^32 / sqrt n)
//                (probability 1/sqrt n), +1 or -1 by the lowest bit of the
//                second word: the sparse random sign matrix of Sec. 5.1.
// With the sparse sign matrix the projection is formed without Omega: each
// column of B gathers the (about sqrt n) columns of A that its column of Omega
// selects, in increasing row order, so the sums are reproducible.
#include <algorithm>
#include <cmath>

#include "css_common.cuh"
#include "project.cuh"

namespace css {
namespace {

constexpr uint32_t kM0 = 0xD2511F53u, kM1 = 0xCD9E8D57u;   // round multipliers
constexpr uint32_t kW0 = 0x9E3779B9u, kW1 = 0xBB67AE85u;   // key increments

__device__ __forceinline__ uint4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                        uint32_t k1) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const uint32_t lo0 = kM0 * c0, hi0 = __umulhi(kM0, c0);
    const uint32_t lo1 = kM1 * c2, hi1 = __umulhi(kM1, c2);
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += kW0;
    k1 += kW1;
  }
  return make_uint4(c0, c1, c2, c3);
}

template <typename TA> struct Vec;
template <> struct Vec<double> {
  __device__ __forceinline__ static void unpack(const uint4& r, double (&a)[2]) {
    a[0] = __hiloint2double((int)r.y, (int)r.x);
    a[1] = __hiloint2double((int)r.w, (int)r.z);
  }
};
template <> struct Vec<float> {
  __device__ __forceinline__ static void unpack(const uint4& r, float (&a)[4]) {
    a[0] = __uint_as_float(r.x); a[1] = __uint_as_float(r.y);
    a[2] = __uint_as_float(r.z); a[3] = __uint_as_float(r.w);
  }
};
template <> struct Vec<__nv_bfloat16> {
  __device__ __forceinline__ static void unpack(const uint4& r, float (&a)[8]) {
    const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      a[2 * i] = __uint_as_float(w[i] << 16);
      a[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
    }
  }
};

template <typename T> __device__ __forceinline__ T from_f64(double v);
template <> __device__ __forceinline__ double from_f64<double>(double v) { return v; }
template <> __device__ __forceinline__ float from_f64<float>(double v) { return (float)v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_f64<__nv_bfloat16>(double v) {
  return __float2bfloat16_rn((float)v);
}

// Omega (n x r, leading dimension ldo).  Gaussian entries are formed in FP64
// for FP64 output and in FP32 otherwise.
template <typename T>
__global__ void omega_kernel(int n, int r, int dist, uint32_t thr, uint32_t k0, uint32_t k1, float inv_sqrt_r,
                             T* __restrict__ Om, long long ldo) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int j = blockIdx.y; j < r; j += gridDim.y) {
  const uint4 x = philox((uint32_t)i, (uint32_t)j, 0u, 0u, k0, k1);
  T v;
  if (dist == CSS_OMEGA_SPARSE_SIGN) {
    const float s = (x.x < thr) ? ((x.y & 1u) ? -1.f : 1.f) : 0.f;
    v = from_f64<T>((double)s);
  } else if constexpr (sizeof(T) == 8) {
    const double u1 = ((double)x.x + 1.0) * 2.3283064365386963e-10;   // 2^-32
    const double u2 = (double)x.y * 2.3283064365386963e-10;
    v = from_f64<T>(sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2) / sqrt((double)r));
  } else {
    // ln u1 with u1 = (w0 + 1) / 2^32: directly below 1/2; above it through
    // the exact integer complement, 1 - u1 = (2^32 - 1 - w0) / 2^32, so that
    // a float conversion never rounds u1 itself to 1
    const float lnu1 = (x.x < 0x80000000u) ? logf(((float)x.x + 1.f) * 2.3283064365386963e-10f)
                                           : log1pf(-(float)(~x.x) * 2.3283064365386963e-10f);
    const float u2 = (float)x.y * 2.3283064365386963e-10f;
    v = from_f64<T>((double)(sqrtf(-2.f * lnu1) * cospif(2.f * u2) * inv_sqrt_r));
  }
  Om[(long long)j * ldo + i] = v;
  }
}

// B[:, j] = sum over the rows i of Omega's column j with Omega_ij != 0 of
// Omega_ij A[:, i], for the sparse sign matrix.  Block (j, row block): every
// thread scans 32 consecutive rows of a window of Omega, the hits are packed
// in row order through a block prefix sum, then every thread adds the hit
// columns for its rows.
constexpr int kSpThreads = 256;
constexpr int kSpRowsPerThread = 8;
constexpr int kSpWindow = kSpThreads * 32;

template <typename TA, typename Acc>
__global__ void __launch_bounds__(kSpThreads) project_sparse_kernel(const TA* __restrict__ A, long long lda,
                                                                    int m, int n, uint32_t thr, uint32_t k0,
                                                                    uint32_t k1, Acc* __restrict__ B,
                                                                    long long ldb, bool vec_ok) {
  __shared__ int s_hit[kSpWindow];   // (row << 1) | negative
  __shared__ int s_off[kSpThreads];
  __shared__ int s_total;
  const int j = blockIdx.x;
  const int tid = threadIdx.x;
  const int row0 = blockIdx.y * kSpThreads * kSpRowsPerThread;
  Acc acc[kSpRowsPerThread];
#pragma unroll
  for (int q = 0; q < kSpRowsPerThread; ++q) acc[q] = Acc(0);
  for (int w0 = 0; w0 < n; w0 += kSpWindow) {
    uint32_t bits = 0u, neg = 0u;
    const int i0 = w0 + tid * 32;
    for (int q = 0; q < 32; ++q) {
      const int i = i0 + q;
      if (i < n) {
        const uint4 x = philox((uint32_t)i, (uint32_t)j, 0u, 0u, k0, k1);
        if (x.x < thr) {
          bits |= 1u << q;
          if (x.y & 1u) neg |= 1u << q;
        }
      }
    }
    // exclusive prefix sum of the hit counts (fixed order: thread order)
    const int cnt = __popc(bits);
    int v = cnt;
    const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += t;
    }
    if (lane == 31) s_off[warp] = v;
    __syncthreads();
    if (tid == 0) {
      int run = 0;
      for (int w = 0; w < kSpThreads / 32; ++w) {
        const int c = s_off[w];
        s_off[w] = run;
        run += c;
      }
      s_total = run;
    }
    __syncthreads();
    int off = s_off[warp] + v - cnt;
    for (uint32_t b = bits; b; b &= b - 1u) {
      const int q = __ffs(b) - 1;
      s_hit[off++] = ((i0 + q) << 1) | (int)((neg >> q) & 1u);
    }
    __syncthreads();
    const int total = s_total;
    // this thread's rows: kSpRowsPerThread consecutive ones, read with
    // 16-byte loads when the whole group lies in A and is aligned
    const int rb = row0 + tid * kSpRowsPerThread;
    constexpr int VPL = 16 / (int)sizeof(TA);   // elements per 16-byte load
    const bool vec = vec_ok && rb + kSpRowsPerThread <= m;
    for (int h = 0; h < total; ++h) {
      const int code = s_hit[h];
      const TA* col = A + (long long)(code >> 1) * lda + rb;
      const bool minus = (code & 1) != 0;
      if (vec) {
#pragma unroll
        for (int q0 = 0; q0 < kSpRowsPerThread; q0 += VPL) {
          const uint4 raw = __ldg(reinterpret_cast<const uint4*>(col + q0));
          Acc a[VPL];
          Vec<TA>::unpack(raw, a);
#pragma unroll
          for (int e = 0; e < VPL; ++e) acc[q0 + e] = minus ? acc[q0 + e] - a[e] : acc[q0 + e] + a[e];
        }
      } else {
#pragma unroll
        for (int q = 0; q < kSpRowsPerThread; ++q) {
          if (rb + q < m) {
            const Acc a = load_elem<TA>(col + q);
            acc[q] = minus ? acc[q] - a : acc[q] + a;
          }
        }
      }
    }
    __syncthreads();
  }
  const int rb = row0 + tid * kSpRowsPerThread;
#pragma unroll
  for (int q = 0; q < kSpRowsPerThread; ++q)
    if (rb + q < m) B[(long long)j * ldb + rb + q] = acc[q];
}

uint32_t sparse_threshold(int64_t n) {
  const double t = std::floor(4294967296.0 / std::sqrt((double)n));
  return t >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)t;
}

size_t esz(int dt) { return dt == CSS_F64 ? 8 : dt == CSS_F32 ? 4 : 2; }
int64_t omega_ld(int64_t n) { return (n + 7) / 8 * 8; }

cudaError_t generate(int64_t n, int64_t r, uint64_t seed, int dist, int dt, void* Om, int64_t ldo,
                     cudaStream_t s) {
  const dim3 blocks((unsigned)((n + 255) / 256), (unsigned)std::min<int64_t>(r, 65535));
  const uint32_t thr = sparse_threshold(n), k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  const float isr = 1.0f / std::sqrt((float)r);
  switch (dt) {
    case CSS_F64: omega_kernel<double><<<blocks, 256, 0, s>>>((int)n, (int)r, dist, thr, k0, k1, isr, (double*)Om, ldo); break;
    case CSS_F32: omega_kernel<float><<<blocks, 256, 0, s>>>((int)n, (int)r, dist, thr, k0, k1, isr, (float*)Om, ldo); break;
    default: omega_kernel<__nv_bfloat16><<<blocks, 256, 0, s>>>((int)n, (int)r, dist, thr, k0, k1, isr, (__nv_bfloat16*)Om, ldo); break;
  }
  return cudaGetLastError();
}

}  // namespace
}  // namespace css

using namespace css;

size_t project_random_workspace_bytes(int dtype, int64_t m, int64_t n, int64_t r) {
  const size_t om = ((size_t)omega_ld(n) * r * esz(dtype) + 255) / 256 * 256;
  return om + project_workspace_bytes(dtype, m, n, r);
}

extern "C" {

css_status css_random_omega(int64_t n, int64_t r, uint64_t seed, css_omega dist, css_dtype dtype, void* Omega,
                            int64_t ldo, css_stream_t stream) {
  // one thread per entry: at most 2^38 entries keeps the grid within 2^30 blocks
  if (!Omega || n < 1 || r < 1 || ldo < n || n > INT32_MAX || r > INT32_MAX || (int64_t)n * r > (1ll << 38))
    return CSS_ERR_INVALID_ARG;
  if (dist != CSS_OMEGA_GAUSSIAN && dist != CSS_OMEGA_SPARSE_SIGN) return CSS_ERR_INVALID_ARG;
  if (dtype != CSS_F64 && dtype != CSS_F32 && dtype != CSS_BF16) return CSS_ERR_INVALID_ARG;
  return generate(n, r, seed, dist, dtype, Omega, ldo, (cudaStream_t)stream) == cudaSuccess ? CSS_OK
                                                                                            : CSS_ERR_CUDA;
}

css_status css_project_random(const void* A, css_dtype dtype, int64_t m, int64_t n, int64_t lda, int64_t r,
                              uint64_t seed, css_omega dist, void* Bout, int64_t ldb, void* ws, size_t ws_bytes,
                              const css_opts* opts, css_stream_t stream) {
  if (!A || !Bout) return CSS_ERR_INVALID_ARG;
  if (dtype != CSS_F64 && dtype != CSS_F32 && dtype != CSS_BF16) return CSS_ERR_INVALID_ARG;
  if (dist != CSS_OMEGA_GAUSSIAN && dist != CSS_OMEGA_SPARSE_SIGN) return CSS_ERR_INVALID_ARG;
  if (m < 1 || n < 1 || r < 1 || lda < m || ldb < m || m > INT32_MAX || n > INT32_MAX || r > INT32_MAX)
    return CSS_ERR_INVALID_ARG;
  // row indices are packed with their sign bit; blocks per column of B < 2^16
  if (n >= (1ll << 30) || r >= (1ll << 31) || (int64_t)n * r > (1ll << 38) ||
      m > 65535ll * kSpThreads * kSpRowsPerThread)
    return CSS_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  css_opts o;
  css_opts_default(&o);
  if (opts) o = *opts;
  if (dist == CSS_OMEGA_SPARSE_SIGN) {
    // no workspace: the columns of Omega are drawn where they are used
    const dim3 grid((unsigned)r, (unsigned)((m + kSpThreads * kSpRowsPerThread - 1) / (kSpThreads * kSpRowsPerThread)));
    const uint32_t thr = sparse_threshold(n), k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    // 16-byte loads of a thread's rows need A and every column start aligned
    const bool vec_ok = ((uintptr_t)A % 16 == 0) && ((lda * (int64_t)esz(dtype)) % 16 == 0);
    switch (dtype) {
      case CSS_F64:
        project_sparse_kernel<double, double><<<grid, kSpThreads, 0, s>>>((const double*)A, lda, (int)m, (int)n, thr,
                                                                         k0, k1, (double*)Bout, ldb, vec_ok);
        break;
      case CSS_F32:
        project_sparse_kernel<float, float><<<grid, kSpThreads, 0, s>>>((const float*)A, lda, (int)m, (int)n, thr, k0,
                                                                       k1, (float*)Bout, ldb, vec_ok);
        break;
      default:
        project_sparse_kernel<__nv_bfloat16, float><<<grid, kSpThreads, 0, s>>>(
            (const __nv_bfloat16*)A, lda, (int)m, (int)n, thr, k0, k1, (float*)Bout, ldb, vec_ok);
        break;
    }
    if (cudaGetLastError() != cudaSuccess) return CSS_ERR_CUDA;
    if (o.sync && cudaStreamSynchronize(s) != cudaSuccess) return CSS_ERR_CUDA;
    return CSS_OK;
  }
  // Gaussian: Omega into the workspace (A's dtype, so BF16 A keeps the tensor
  // cores), then the projection of css_project
  if (!ws || ((uintptr_t)ws % kWsAlign) != 0) return CSS_ERR_WORKSPACE;
  if (ws_bytes < project_random_workspace_bytes(dtype, m, n, r)) return CSS_ERR_WORKSPACE;
  const int64_t ldo = omega_ld(n);
  const size_t om = ((size_t)ldo * r * esz(dtype) + 255) / 256 * 256;
  if (generate(n, r, seed, dist, dtype, ws, ldo, s) != cudaSuccess) return CSS_ERR_CUDA;
  return css_project(A, dtype, m, n, lda, ws, r, ldo, Bout, ldb, (char*)ws + om, ws_bytes - om, &o, stream);
}

}  // extern "C"
