// Internal device/host helpers shared by the libcss translation units.
// Nothing here is part of the C ABI (include/css.h).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/css.h"

namespace css {

// ---------------------------------------------------------------- status ----
// Device-side status block at the start of every workspace (256 bytes).
struct DevStatus {
  int32_t code;            // 0 = ok, else a css_status error value
  int32_t rank_exhausted;  // number of units that stopped early
  int32_t where;           // id of the wait that timed out (diagnostic)
  int32_t stall_where;     // test hook: this barrier id waits for one arrival too many (0 = none)
  uint64_t spin_budget_ns;
};

constexpr size_t kWsAlign = 256;
constexpr size_t kStatusBytes = 256;

inline size_t align_up(size_t x, size_t a = kWsAlign) { return (x + a - 1) / a * a; }

// Host-side bump allocator over a caller-provided workspace.
// Leading dimension of the m x m matrix C = A A^T held in the workspace
// (elements of acc_bytes each): a multiple of 16 bytes, so that every row of
// C starts on a 16-byte boundary and takes vector loads.
inline long long c_ld(long long m, int acc_bytes) {
  const long long v = 16 / acc_bytes;
  return (m + v - 1) / v * v;
}

struct WsCarver {
  char* base;
  size_t off;
  size_t cap;
  bool overflow;
  WsCarver(void* b, size_t c) : base((char*)b), off(0), cap(c), overflow(false) {}
  template <typename T>
  T* take(size_t count) {
    size_t bytes = align_up(count * sizeof(T));
    char* p = base ? base + off : nullptr;
    off += bytes;
    if (off > cap) overflow = true;
    return (T*)p;
  }
};

// ------------------------------------------------------------ element io ----
template <typename T> struct AccOf { using type = float; };
template <> struct AccOf<double> { using type = double; };

__device__ __forceinline__ float bf16_lo(uint32_t v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t v) { return __uint_as_float(v & 0xffff0000u); }

template <typename T> __device__ __forceinline__ typename AccOf<T>::type load_elem(const T* p);
template <> __device__ __forceinline__ double load_elem<double>(const double* p) { return __ldg(p); }
template <> __device__ __forceinline__ float load_elem<float>(const float* p) { return __ldg(p); }
template <> __device__ __forceinline__ float load_elem<__nv_bfloat16>(const __nv_bfloat16* p) {
  return __uint_as_float(((uint32_t)__ldg((const unsigned short*)p)) << 16);
}

// 16-byte streaming load of read-only data: L1 no-allocate, L2 evict-first.
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ uint4 ldg_stream16(const void* p, uint64_t pol) {
  uint4 v;
  asm volatile(
      "ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
      : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
      : "l"(p), "l"(pol));
  return v;
}

// Loads of data written by other CTAs of the same launch: bypass L1.
__device__ __forceinline__ double ldcg(const double* p) { return __ldcg(p); }
__device__ __forceinline__ float ldcg(const float* p) { return __ldcg(p); }
__device__ __forceinline__ int ldcg(const int* p) { return __ldcg(p); }

// ----------------------------------------------------------------- timing ---
__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t atom_add_acqrel_u32(uint32_t* p, uint32_t v) {
  uint32_t old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ int32_t ld_volatile_i32(const int32_t* p) {
  return *(volatile const int32_t*)p;
}

__device__ __forceinline__ void set_error(DevStatus* st, int32_t code, int32_t where) {
  if (atomicCAS(&st->code, 0, code) == 0) st->where = where;
}

__device__ __forceinline__ void red_release_add_u32(uint32_t* p, uint32_t v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Barrier over the `ncta` CTAs of one team.  bar[0] counts arrivals over the
// whole launch (zeroed before it); `epoch` (thread 0's count of this team's
// barriers so far) gives the value that completes this one.  Arrival is a
// release reduction that needs no reply, so the barrier costs one trip of the
// last arrival to L2 and one poll.  Every wait is bounded by the workspace's
// spin budget; on expiry (or when another CTA already flagged an error) it
// records CSS_ERR_TIMEOUT and returns false.  All CTAs of the team are
// co-resident (the persistent kernel is launched cooperatively).
__device__ __forceinline__ bool team_barrier(uint32_t* bar, int ncta, DevStatus* st, int where,
                                             uint32_t* epoch) {
  __shared__ int s_ok;
  __syncthreads();
  if (ncta <= 1) return ld_volatile_i32(&st->code) == 0;
  if (threadIdx.x == 0) {
    int ok = 1;
    *epoch += 1u;
    // (the test hook asks one barrier for an arrival that never comes)
    const uint32_t target = *epoch * (uint32_t)ncta + (st->stall_where == where ? 1u : 0u);
    red_release_add_u32(bar, 1u);
    uint64_t t0 = globaltimer_ns();
    const uint64_t budget = st->spin_budget_ns;
    uint32_t spins = 0;
    while ((int32_t)(ld_acquire_u32(bar) - target) < 0) {
      if ((++spins & 63u) == 0u) {
        if (ld_volatile_i32(&st->code) != 0) { ok = 0; break; }
        if (globaltimer_ns() - t0 > budget) {
          set_error(st, (int32_t)CSS_ERR_TIMEOUT, where);
          ok = 0;
          break;
        }
      }
      if (spins > 256u) __nanosleep(64);
    }
    if (ok && ld_volatile_i32(&st->code) != 0) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// ------------------------------------------------------------- reductions ---
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Exact float -> double by integer operations: conversions to FP64 issue at
// the FP64 rate on this part, integer operations at the full rate.  Subnormal
// floats (rare) take the hardware conversion.
__device__ __forceinline__ double to_f64(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xffu;
  const uint32_t frac = u & 0x7fffffu;
  const uint64_t sign = (uint64_t)(u >> 31) << 63;
  if (e == 0u) {
    if (frac == 0u) return __longlong_as_double((long long)sign);
    return (double)f;
  }
  const uint64_t ex = (e == 0xffu) ? 0x7ffull : (uint64_t)(e + 896u);   // 1023 - 127
  return __longlong_as_double((long long)(sign | (ex << 52) | ((uint64_t)frac << 29)));
}
__device__ __forceinline__ double to_f64(double d) { return d; }

// Candidate scores are non-negative doubles, whose IEEE-754 bit patterns
// (sign cleared, so that -0 and +0 agree) order like the values: the argmax
// compares these keys with integer instructions, because FP64 compares issue
// at a small fraction of the integer rate on this part.
__device__ __forceinline__ long long score_key(double v) {
  return __double_as_longlong(v) & 0x7fffffffffffffffLL;
}

// (key, index) ordering of the argmax: larger key wins, equal keys go to the
// lower index; index < 0 means "no candidate".
__device__ __forceinline__ bool better(long long k1, int i1, long long k2, int i2) {
  if (i1 < 0) return false;
  if (i2 < 0) return true;
  return (k1 > k2) || (k1 == k2 && i1 < i2);
}

__device__ __forceinline__ void warp_argmax(long long& k, int& i) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    long long k2 = __shfl_xor_sync(0xffffffffu, k, o);
    int i2 = __shfl_xor_sync(0xffffffffu, i, o);
    if (better(k2, i2, k, i)) { k = k2; i = i2; }
  }
}

// Block-wide FP64 sum in thread 0 only: the threads' values go through shared
// memory and warp 0 adds them (NW + 5 FP64 adds in one warp, instead of five
// in every warp).  `red` holds blockDim.x values; fixed order.
template <typename T>
__device__ __forceinline__ T block_sum_to0(T v, T* red) {
  const int lane = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  red[threadIdx.x] = v;
  __syncthreads();
  T s = T(0);
  if (threadIdx.x < 32) {
    for (int w = 0; w < nw; ++w) s += red[w * 32 + lane];
    s = warp_sum(s);
  }
  return s;
}

// Block-wide sum; every thread gets the result.  `red` holds >= 32 values.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  T s = (threadIdx.x < (unsigned)nw) ? red[threadIdx.x] : T(0);
  if (w == 0) s = warp_sum(s);
  if (threadIdx.x == 0) red[0] = s;
  __syncthreads();
  T r = red[0];
  return r;
}

}  // namespace css
