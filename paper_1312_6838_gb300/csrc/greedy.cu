// Persistent greedy kernel: Algorithm 1 (CSS) and Algorithm 3 (GCSS) of
// Farahat et al. (arXiv:1312.6838), every iteration on the device.
//
// Teams of co-resident CTAs each own a list of problems ("units"); a team
// synchronises with its own bounded barrier, so independent problems (the
// column blocks of Algorithm 4, or a batch of instances) run side by side in
// one cooperative launch.  A single large problem uses one team = the grid.
//
// Per iteration t (p = column picked at t):
//   pivot     e = (I - Q Q^T) a_p, one Gram-Schmidt pass with the coefficients
//             c = Q^T a_p formed exactly (FP64, or double-float for BF16/FP32
//             input); delta_p = ||e||^2, q = e / ||e|| (Eq. delta_omega:
//             omega = A^T q).
//   target    CSS:  y = C q with C = A A^T;  GCSS: upsilon = B^T q, y = B upsilon.
//             s = q^T y (= ||omega||^2, Theorem 2) or ||upsilon||^2 (Theorem 4).
//             y' = (I - Q Q^T) y = (y - Q d) with d = Z^T e / ||e||, Z = C Q,
//             so that A^T y' = G omega (CSS) or
//             A^T B upsilon - sum_r (upsilon^(r)^T upsilon) omega^(r) (GCSS).
//   fused     one pass over A: omega_i = a_i . q and h_i = a_i . y' per column,
//             f_i <- f_i - 2 omega_i h_i + s omega_i^2, g_i <- g_i - omega_i^2,
//             W[t, i] = omega_i, then the masked argmax of f_i / g_i.
//   trace     F <- F - f_p / g_p (Theorems 1 and 3).
//
// Two CTA shapes are built from this file: 512 threads with one CTA per SM
// (this translation unit, the defaults below) and 256 threads with two CTAs
// per SM (greedy_pair.cu), both with the same 128 registers per thread.
#include "greedy.cuh"

#ifndef CSS_GREEDY_NT
#define CSS_GREEDY_NT 512           // threads per CTA
#define CSS_GREEDY_CTAS_PER_SM 1    // co-resident CTAs the registers are budgeted for
#define CSS_GREEDY_SHAPE one_per_sm // namespace of this shape's host entry points
#define CSS_GREEDY_EXPORT_BASIS 1   // export_basis is built once, here
#endif

namespace css {
namespace {

constexpr int NT = CSS_GREEDY_NT;
constexpr int NW = NT / 32;
constexpr int NS = 2 * NW;  // half-warp streams of the row GEMVs
constexpr int RB = 16;      // rows per row tile

template <typename T> __device__ __forceinline__ T ld_cg(const T* p) { return __ldcg(p); }

// ---------------------------------------------------------------- context ---
template <typename Acc>
struct Ctx {
  int rank, ncta, tid, lane, warp;
  DevStatus* st;
  const TeamDesc* team;
  Acc* sq;       // K1: q           (aliases buf)
  Acc* sy;       // K1: y'          (aliases buf)
  double* se64;  // pivot phases: FP64 vector (aliases buf)
  Acc* seacc;    // pivot phases: same vector in Acc precision (aliases buf)
  double* scoef; // coefficients (FP64)
  Acc* sups;     // upsilon in Acc precision
  double* sred;  // NS * RB partials
  uint32_t* epoch;  // thread 0: barriers of the team passed so far
};

// ------------------------------------------------------------- transpose ----
// Sum NV per-lane values over the warp.  Lane L ends up with value index
// L >> (5 - log2 NV).  Costs NV - 1 + 5 - log2 NV shuffles.
template <int NV> struct Log2 { static constexpr int v = (NV >= 32) ? 5 : (NV >= 16) ? 4 : (NV >= 8) ? 3 : (NV >= 4) ? 2 : (NV >= 2) ? 1 : 0; };

template <int NV, typename T>
__device__ __forceinline__ T transpose_reduce(T (&v)[NV], int lane) {
  constexpr int LOG = Log2<NV>::v;
#pragma unroll
  for (int s = 0; s < LOG; ++s) {
    const int mask = 16 >> s;
    const int half = NV >> (s + 1);
    const bool up = (lane & mask) != 0;
#pragma unroll
    for (int j = 0; j < half; ++j) {
      T send = up ? v[j] : v[j + half];
      T keep = up ? v[j + half] : v[j];
      v[j] = keep + __shfl_xor_sync(0xffffffffu, send, mask);
    }
  }
  T r = v[0];
#pragma unroll
  for (int s = LOG; s < 5; ++s) r += __shfl_xor_sync(0xffffffffu, r, 16 >> s);
  return r;
}

// ------------------------------------------------------------ vector io -----
template <typename TA> struct Vec;
template <> struct Vec<double> {
  static constexpr int V = 2;
  __device__ __forceinline__ static void unpack(const uint4& r, double (&a)[2]) {
    a[0] = __hiloint2double((int)r.y, (int)r.x);
    a[1] = __hiloint2double((int)r.w, (int)r.z);
  }
};
template <> struct Vec<float> {
  static constexpr int V = 4;
  __device__ __forceinline__ static void unpack(const uint4& r, float (&a)[4]) {
    a[0] = __uint_as_float(r.x); a[1] = __uint_as_float(r.y);
    a[2] = __uint_as_float(r.z); a[3] = __uint_as_float(r.w);
  }
};
template <> struct Vec<__nv_bfloat16> {
  static constexpr int V = 8;
  __device__ __forceinline__ static void unpack(const uint4& r, float (&a)[8]) {
    a[0] = bf16_lo(r.x); a[1] = bf16_hi(r.x); a[2] = bf16_lo(r.y); a[3] = bf16_hi(r.y);
    a[4] = bf16_lo(r.z); a[5] = bf16_hi(r.z); a[6] = bf16_lo(r.w); a[7] = bf16_hi(r.w);
  }
};

template <typename Acc, int V>
__device__ __forceinline__ void lds_vec(const Acc* p, Acc (&a)[V]) {
  if constexpr (sizeof(Acc) == 4) {
#pragma unroll
    for (int i = 0; i < V; i += 4) {
      float4 t = *reinterpret_cast<const float4*>(p + i);
      a[i] = t.x; a[i + 1] = t.y; a[i + 2] = t.z; a[i + 3] = t.w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < V; i += 2) {
      double2 t = *reinterpret_cast<const double2*>(p + i);
      a[i] = t.x; a[i + 1] = t.y;
    }
  }
}

// ------------------------------------------------------------- row GEMV -----
// For every row i < m of the team's rows: fin(i, sum_{j<nj} M[i + j ldm] c[j], pv)
// with c in shared memory and pv = pre(i), which the finishing thread calls
// before the products so that the loads it makes overlap them.  Rows are split
// in tiles of RB rows, dealt round-robin to the team's CTAs; inside a CTA the
// j-range of a tile is split over half-warp streams when the CTA has few
// tiles.  Deterministic for a fixed team size.
struct NoPre {
  __device__ int operator()(int) const { return 0; }
};

template <typename TS, typename TM, typename TC, typename Acc, typename Pre, typename Fin>
__device__ void row_gemv(const Ctx<Acc>& x, int m, int nj, const TM* M, long long ldm,
                         const TC* c, Pre pre, Fin fin) {
  const int G = (m + RB - 1) / RB;
  const int my_tiles = (G > x.rank) ? (G - x.rank + x.ncta - 1) / x.ncta : 0;
  const int TP = (G + x.ncta - 1) / x.ncta;
  int SP = NS;
  while (SP > 1 && SP * TP > NS) SP >>= 1;
  const int slots = NS / SP;
  const int s = x.warp * 2 + (x.lane >> 4);
  const int slot = s / SP, sub = s % SP;
  const int r16 = x.lane & (RB - 1);
  TS* red = reinterpret_cast<TS*>(x.sred);
  for (int base = 0; base < my_tiles; base += slots) {
    const int ti = base + slot;
    // the finishing thread of this round and its row
    const int sl = x.tid / RB, rr = x.tid % RB;
    const int tj = base + sl;
    const int frow = (x.tid < slots * RB && tj < my_tiles) ? (x.rank + tj * x.ncta) * RB + rr : m;
    decltype(pre(0)) pv{};
    if (frow < m) pv = pre(frow);
    TS acc = TS(0);
    if (ti < my_tiles) {
      const int row = (x.rank + ti * x.ncta) * RB + r16;
      if (row < m) {
        const TM* mp = M + row;
        int j = sub;
        // eight loads in flight per trip: these phases are bound by L2 latency
        for (; j + 7 * SP < nj; j += 8 * SP) {
          TS a[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) a[q] = (TS)ld_cg(mp + (long long)(j + q * SP) * ldm);
#pragma unroll
          for (int q = 0; q < 8; ++q) acc += a[q] * (TS)c[j + q * SP];
        }
        for (; j < nj; j += SP) acc += (TS)ld_cg(mp + (long long)j * ldm) * (TS)c[j];
      }
    }
    red[s * RB + r16] = acc;
    __syncthreads();
    if (frow < m) {
      TS sum = TS(0);
      for (int q = 0; q < SP; ++q) sum += red[(sl * SP + q) * RB + rr];
      fin(frow, (double)sum, pv);
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------ column dots ---
// fin(j, sum_{i<len} M[i + j ldm] v[i]) for j < nj, v in shared memory.
template <typename TS, typename TM, typename TV, typename Acc, typename Fin>
__device__ void col_dots(const Ctx<Acc>& x, int len, int nj, const TM* M, long long ldm,
                         const TV* v, Fin fin) {
  const int per_cta = (nj + x.ncta - 1) / x.ncta;
  if (per_cta >= NW / 2) {
    for (int j = x.rank * NW + x.warp; j < nj; j += x.ncta * NW) {
      const TM* col = M + (long long)j * ldm;
      TS acc = TS(0);
#pragma unroll 8
      for (int i = x.lane; i < len; i += 32) acc += (TS)ld_cg(col + i) * (TS)v[i];
      acc = warp_sum(acc);
      if (x.lane == 0) fin(j, (double)acc);
    }
  } else {
    for (int j = x.rank; j < nj; j += x.ncta) {
      const TM* col = M + (long long)j * ldm;
      TS acc = TS(0);
#pragma unroll 8
      for (int i = x.tid; i < len; i += NT) acc += (TS)ld_cg(col + i) * (TS)v[i];
      acc = block_sum_to0(acc, reinterpret_cast<TS*>(x.sred));
      if (x.tid == 0) fin(j, (double)acc);
    }
  }
}

// col_dots for an FP32 matrix whose columns start on 16-byte boundaries (ldm
// a multiple of 4) and len a multiple of 4: one warp per column, four floats
// per lane per load, eight loads in flight (the GCSS pivot's B^T e).
template <typename Acc, typename Fin>
__device__ void col_dots_f4(const Ctx<Acc>& x, int len, int nj, const float* M, long long ldm, const float* v,
                            Fin fin) {
  const int len4 = len / 4;
  const float4* v4 = reinterpret_cast<const float4*>(v);
  for (int j = x.rank * NW + x.warp; j < nj; j += x.ncta * NW) {
    const float4* col = reinterpret_cast<const float4*>(M + (long long)j * ldm);
    float acc = 0.f;
#pragma unroll 8
    for (int i = x.lane; i < len4; i += 32) {
      const float4 a = ld_cg(col + i), b = v4[i];
      acc = fmaf(a.x, b.x, acc);
      acc = fmaf(a.y, b.y, acc);
      acc = fmaf(a.z, b.z, acc);
      acc = fmaf(a.w, b.w, acc);
    }
    acc = warp_sum(acc);
    if (x.lane == 0) fin(j, (double)acc);
  }
}

// ------------------------------------------------ double-float products ----
// The Gram-Schmidt products of the BF16/FP32 path (Q^T a_p, Q c, Z^T e, Q d:
// m x t multiply-adds each) run in double-float arithmetic: every FP64 value
// of Q, Z, e and the coefficients is held as an unevaluated sum hi + lo of two
// floats (48 significant bits), products are made exact with an FMA (Dekker's
// product) and the running sum keeps its rounding errors (Knuth's TwoSum) --
// the compensated dot product of Ogita, Rump and Oishi, as accurate as an
// evaluation in twice the float precision.  About eleven FP32 operations per
// term instead of one FP64 multiply-add, which issues some fifty times slower
// on this part.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
// (sh, sl) += (xh + xl) * (yh + yl)
__device__ __forceinline__ void df_fma(float& sh, float& sl, float xh, float xl, float yh, float yl) {
  const float p = xh * yh;
  float e = fmaf(xh, yh, -p);
  e = fmaf(xh, yl, e);
  e = fmaf(xl, yh, e);
  float s, err;
  two_sum(sh, p, s, err);
  sh = s;
  sl += err + e;
}
// (ah, al) += (bh, bl), renormalised
__device__ __forceinline__ void df_add(float& ah, float& al, float bh, float bl) {
  float s, e;
  two_sum(ah, bh, s, e);
  e += al + bl;
  ah = s + e;
  al = e - (ah - s);
}
__device__ __forceinline__ float2 df_norm(float h, float l) {
  float s, e;
  two_sum(h, l, s, e);
  return make_float2(s, e);
}
__device__ __forceinline__ double df_to_f64(float2 v) { return to_f64(v.x) + to_f64(v.y); }
// FP64 -> hi + lo (three FP64 operations; only where a vector element is formed)
__device__ __forceinline__ float2 f64_to_df(double v) {
  const float h = __double2float_rn(v);
  return make_float2(h, __double2float_rn(v - to_f64(h)));
}
__device__ __forceinline__ float2 df_of(float v) { return make_float2(v, 0.f); }
__device__ __forceinline__ float2 df_of(float2 v) { return v; }

__device__ __forceinline__ void warp_df_sum(float& h, float& l) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float bh = __shfl_xor_sync(0xffffffffu, h, o);
    const float bl = __shfl_xor_sync(0xffffffffu, l, o);
    df_add(h, l, bh, bl);
  }
}

// row_gemv in double-float: fin(i, sum_j M[i, j] c[j] as hi + lo, pre(i)),
// M and c held as float2 (hi, lo).  Same row and stream split as row_gemv.
template <typename Acc, typename Pre, typename Fin>
__device__ void row_gemv_df(const Ctx<Acc>& x, int m, int nj, const float2* M, long long ldm,
                            const float2* c, Pre pre, Fin fin) {
  const int G = (m + RB - 1) / RB;
  const int my_tiles = (G > x.rank) ? (G - x.rank + x.ncta - 1) / x.ncta : 0;
  const int TP = (G + x.ncta - 1) / x.ncta;
  int SP = NS;
  while (SP > 1 && SP * TP > NS) SP >>= 1;
  const int slots = NS / SP;
  const int s = x.warp * 2 + (x.lane >> 4);
  const int slot = s / SP, sub = s % SP;
  const int r16 = x.lane & (RB - 1);
  float2* red = reinterpret_cast<float2*>(x.sred);
  for (int base = 0; base < my_tiles; base += slots) {
    const int ti = base + slot;
    const int sl = x.tid / RB, rr = x.tid % RB;
    const int tj = base + sl;
    const int frow = (x.tid < slots * RB && tj < my_tiles) ? (x.rank + tj * x.ncta) * RB + rr : m;
    decltype(pre(0)) pv{};
    if (frow < m) pv = pre(frow);
    float ah = 0.f, al = 0.f;
    if (ti < my_tiles) {
      const int row = (x.rank + ti * x.ncta) * RB + r16;
      if (row < m) {
        const float2* mp = M + row;
        int j = sub;
        for (; j + 7 * SP < nj; j += 8 * SP) {
          float2 a[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) a[q] = ld_cg(mp + (long long)(j + q * SP) * ldm);
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const float2 cv = c[j + q * SP];
            df_fma(ah, al, a[q].x, a[q].y, cv.x, cv.y);
          }
        }
        for (; j < nj; j += SP) {
          const float2 a = ld_cg(mp + (long long)j * ldm);
          const float2 cv = c[j];
          df_fma(ah, al, a.x, a.y, cv.x, cv.y);
        }
      }
    }
    red[s * RB + r16] = df_norm(ah, al);
    __syncthreads();
    if (frow < m) {
      float h = 0.f, l = 0.f;
      for (int q = 0; q < SP; ++q) {
        const float2 v = red[(sl * SP + q) * RB + rr];
        df_add(h, l, v.x, v.y);
      }
      fin(frow, make_float2(h, l), pv);
    }
    __syncthreads();
  }
}

// col_dots in double-float: fin(j, sum_i M[i, j] v[i] as hi + lo), M as float2,
// v as float (exact values) or float2, in shared memory.
template <typename Acc, typename TV, typename Fin>
__device__ void col_dots_df(const Ctx<Acc>& x, int len, int nj, const float2* M, long long ldm,
                            const TV* v, Fin fin) {
  const int per_cta = (nj + x.ncta - 1) / x.ncta;
  if (per_cta >= NW / 2) {
    for (int j = x.rank * NW + x.warp; j < nj; j += x.ncta * NW) {
      const float2* col = M + (long long)j * ldm;
      float h = 0.f, l = 0.f;
#pragma unroll 8
      for (int i = x.lane; i < len; i += 32) {
        const float2 a = ld_cg(col + i);
        const float2 b = df_of(v[i]);
        df_fma(h, l, a.x, a.y, b.x, b.y);
      }
      const float2 n0 = df_norm(h, l);
      h = n0.x;
      l = n0.y;
      warp_df_sum(h, l);
      if (x.lane == 0) fin(j, make_float2(h, l));
    }
  } else {
    float2* red = reinterpret_cast<float2*>(x.sred);
    for (int j = x.rank; j < nj; j += x.ncta) {
      const float2* col = M + (long long)j * ldm;
      float h = 0.f, l = 0.f;
#pragma unroll 8
      for (int i = x.tid; i < len; i += NT) {
        const float2 a = ld_cg(col + i);
        const float2 b = df_of(v[i]);
        df_fma(h, l, a.x, a.y, b.x, b.y);
      }
      const float2 n0 = df_norm(h, l);
      h = n0.x;
      l = n0.y;
      warp_df_sum(h, l);
      __syncthreads();
      if (x.lane == 0) red[x.warp] = make_float2(h, l);
      __syncthreads();
      if (x.warp == 0) {
        float2 w = (x.lane < NW) ? red[x.lane] : make_float2(0.f, 0.f);
        h = w.x;
        l = w.y;
        warp_df_sum(h, l);
        if (x.lane == 0) fin(j, make_float2(h, l));
      }
    }
  }
}

// ------------------------------------------------------------- CTA argmax ---
// Publishes the CTA's best candidate and returns its index (every thread).
template <typename Acc>
__device__ int cta_argmax_publish(const Ctx<Acc>& x, long long bv, int bi) {
  __shared__ long long s_v[NW];
  __shared__ int s_i[NW];
  __shared__ int s_best;
  warp_argmax(bv, bi);
  if (x.lane == 0) { s_v[x.warp] = bv; s_i[x.warp] = bi; }
  __syncthreads();
  if (x.warp == 0) {
    long long v = (x.lane < NW) ? s_v[x.lane] : -1LL;
    int i = (x.lane < NW) ? s_i[x.lane] : -1;
    warp_argmax(v, i);
    if (x.lane == 0) {
      x.team->cand_val[x.rank] = __longlong_as_double(v);
      x.team->cand_idx[x.rank] = i;
      s_best = i;
    }
  }
  __syncthreads();
  return s_best;
}

// Warms L2 with column `col` of A: the team's next pivot is one of its CTAs'
// candidates, and the pivot phase reads that column first.
template <typename TA>
__device__ __forceinline__ void prefetch_column(const UnitDesc& u, int col) {
  const unsigned bytes = (unsigned)((size_t)u.m * sizeof(TA)) & ~15u;
  if (col < 0 || !u.vec_ok || bytes == 0u) return;
  const TA* p = reinterpret_cast<const TA*>(u.A) + (long long)col * u.lda;
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

template <typename Acc>
__device__ int team_argmax(const Ctx<Acc>& x) {
  __shared__ int s_p;
  if (x.warp == 0) {
    long long v = -1;
    int i = -1;
    for (int r = x.lane; r < x.ncta; r += 32) {
      long long v2 = __double_as_longlong(ld_cg(x.team->cand_val + r));
      int i2 = ld_cg(x.team->cand_idx + r);
      if (better(v2, i2, v, i)) { v = v2; i = i2; }
    }
    warp_argmax(v, i);
    if (x.lane == 0) s_p = i;
  }
  __syncthreads();
  return s_p;
}

// Sum of part[r * 4 + slot] over the team's CTAs, in a fixed order (every CTA
// gets the same bits).  Warp 0 reads the partials in parallel.
template <typename Acc>
__device__ double team_sum(const Ctx<Acc>& x, int slot) {
  __shared__ double s_sum;
  if (x.warp == 0) {
    double a = 0.0;
    for (int r = x.lane; r < x.ncta; r += 32) a += ld_cg(x.team->part + r * 4 + slot);
    a = warp_sum(a);
    if (x.lane == 0) s_sum = a;
  }
  __syncthreads();
  const double v = s_sum;
  __syncthreads();
  return v;
}

// --------------------------------------------------------- fused step (K1) --
// Work units come from a team-wide counter: first whole tiles of CW columns,
// then the last `nsplit` tiles (one per warp of the team at most) cut into
// kSplitR row chunks, so that the step ends with short units instead of
// warps idling behind a few long ones.  The chunk sums of a split tile meet
// in the team's split area; the warp that adds the last chunk sums them in
// chunk order (the result does not depend on which warp that is).
//
// The per-column update is FP64, and FP64 issues at a small fraction of the
// FP32 rate on this part, so it is not run per tile (where only CW lanes of
// the warp would hold results): each lane collects the (omega, h) of one column
// and the warp applies the update to 32 columns at once, every 32 / CW tiles.
template <typename TA, int CW>
__device__ void fused_step(const Ctx<typename AccOf<TA>::type>& x, const UnitDesc& u, int t,
                           int p, double s, uint64_t pol, long long& bv, int& bi) {
  using Acc = typename AccOf<TA>::type;
  constexpr int V = Vec<TA>::V;
  constexpr int NV = 2 * CW;
  constexpr int SH = 5 - Log2<NV>::v;
  constexpr int TPB = 32 / CW;  // tiles per epilogue batch
  static_assert(NV <= kSplitVals, "split slots hold 2 x CW values");
  const int n = u.n, m = u.m;
  const int ntiles = (n + CW - 1) / CW;
  const int nsplit = min(ntiles, x.team->split_cap);
  const int nbulk = ntiles - nsplit;
  const int nunits = nbulk + nsplit * kSplitR;
  // rows per chunk: a multiple of one warp-wide vector step
  const int rch = ((m + kSplitR - 1) / kSplitR + 32 * V - 1) / (32 * V) * (32 * V);
  const int m_vec = u.vec_ok ? (m / V) * V : 0;
  const TA* A = reinterpret_cast<const TA*>(u.A);
  Acc* split_part = reinterpret_cast<Acc*>(x.team->split_part);
  // slots are sized for 8-byte values; FP32 sums use the first half of each
  constexpr int SLOT = kSplitR * kSplitVals * 8 / (int)sizeof(Acc);
  // this lane's column within a tile, and where its omega and h sit after
  // the transpose-reduce (lane L holds value L >> SH)
  const int my_c = x.lane % CW;
  const int src_w = (2 * my_c) << SH, src_h = (2 * my_c + 1) << SH;
  const int my_slot = x.lane / CW;
  const bool val_lane = (x.lane & ((1 << SH) - 1)) == 0;
  Acc bw = Acc(0), bh = Acc(0);
  int bcol = -1, slot = 0;
  uint32_t* ctr = x.team->tile_ctr + (t & 1);
  int unit = 0;
  if (x.lane == 0) unit = (int)atomicAdd(ctr, 1u);
  unit = __shfl_sync(0xffffffffu, unit, 0);
  // short columns (at most 2 KB): a tile's loads are one or two dependent
  // memory round trips, so the warp asks L2 for the columns of its next unit
  // as soon as it draws it (one bulk prefetch per column).  Measured on the
  // batched workload (one CTA per problem, every SM streaming): the greedy
  // launch 4-7 % shorter; with 4 KB columns (the distributed blocks, 2048
  // rows) it was 5 % longer, so those are left alone
  const bool pf_next = u.vec_ok && (size_t)m * sizeof(TA) <= 2048 && (size_t)m * sizeof(TA) >= 16;
  while (unit < nunits) {
    int next = 0;
    if (x.lane == 0) next = (int)atomicAdd(ctr, 1u);
    if (pf_next) {
      const int nx = __shfl_sync(0xffffffffu, next, 0);
      if (nx < nunits && x.lane < CW) {
        const int nt = nx < nbulk ? nx : nbulk + (nx - nbulk) / kSplitR;
        const int col = nt * CW + x.lane;
        if (col < n)
          asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(A + (long long)col * u.lda),
                       "r"((unsigned)((size_t)m * sizeof(TA)) & ~15u)
                       : "memory");
      }
    }
    int tile = unit, sidx = -1, chunk = 0, r_lo = 0, r_hi = m;
    if (unit >= nbulk) {
      sidx = (unit - nbulk) / kSplitR;
      chunk = (unit - nbulk) - sidx * kSplitR;
      tile = nbulk + sidx;
      r_lo = min(m, chunk * rch);
      r_hi = (chunk == kSplitR - 1) ? m : min(m, r_lo + rch);
    }
    const int c0 = tile * CW;
    const TA* colp[CW];
#pragma unroll
    for (int c = 0; c < CW; ++c) colp[c] = A + (long long)min(c0 + c, n - 1) * u.lda;
    Acc v[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = Acc(0);
    const int v_hi = min(r_hi, m_vec);
#pragma unroll 4
    for (int r = r_lo + x.lane * V; r < v_hi; r += 32 * V) {
      uint4 raw[CW];
#pragma unroll
      for (int c = 0; c < CW; ++c) raw[c] = ldg_stream16(colp[c] + r, pol);
      Acc qa[V], ya[V];
      lds_vec<Acc, V>(x.sq + r, qa);
      lds_vec<Acc, V>(x.sy + r, ya);
#pragma unroll
      for (int c = 0; c < CW; ++c) {
        Acc a[V];
        Vec<TA>::unpack(raw[c], a);
        Acc tw = a[0] * qa[0], th = a[0] * ya[0];
#pragma unroll
        for (int e = 1; e < V; ++e) { tw = fma(a[e], qa[e], tw); th = fma(a[e], ya[e], th); }
        v[2 * c] += tw;
        v[2 * c + 1] += th;
      }
    }
    for (int r = max(r_lo, m_vec) + x.lane; r < r_hi; r += 32) {
      const Acc qa = x.sq[r], ya = x.sy[r];
#pragma unroll
      for (int c = 0; c < CW; ++c) {
        const Acc a = load_elem<TA>(colp[c] + r);
        v[2 * c] = fma(a, qa, v[2 * c]);
        v[2 * c + 1] = fma(a, ya, v[2 * c + 1]);
      }
    }
    Acc red = transpose_reduce<NV>(v, x.lane);
    bool have = true;
    if (sidx >= 0) {
      Acc* sp = split_part + (size_t)sidx * SLOT;
      if (val_lane) __stcg(sp + chunk * kSplitVals + (x.lane >> SH), red);
      __syncwarp();
      uint32_t old = 0;
      if (x.lane == 0) old = atom_add_acqrel_u32(x.team->split_done + sidx, 1u);
      old = __shfl_sync(0xffffffffu, old, 0);
      have = old == (uint32_t)(kSplitR - 1);
      if (have) {
        __syncwarp();   // lane 0's acquire orders the other lanes' loads
        if (val_lane) {
          Acc sum = Acc(0);
#pragma unroll
          for (int c = 0; c < kSplitR; ++c) sum += ld_cg(sp + c * kSplitVals + (x.lane >> SH));
          red = sum;
        }
        // every chunk has arrived: the counter is free for the next step
        if (x.lane == 0) x.team->split_done[sidx] = 0u;
      }
    }
    if (have) {
      const Acc wv = __shfl_sync(0xffffffffu, red, src_w);
      const Acc hv = __shfl_sync(0xffffffffu, red, src_h);
      if (my_slot == slot && c0 + my_c < n) { bw = wv; bh = hv; bcol = c0 + my_c; }
      ++slot;
    }
    unit = __shfl_sync(0xffffffffu, next, 0);
    if (slot == TPB || unit >= nunits) {
      if (bcol >= 0) {
        const int col = bcol;
        double fi = ld_cg(u.f + col), gi = ld_cg(u.g + col);
        const double thr = ld_cg(u.thr + col);
        bool selected = __ldcg(u.selmask + col) != 0;
        const double w = to_f64(bw), h = to_f64(bh);
        // Theorem 2 / Theorem 4: f - 2 omega o x + s (omega o omega), g - omega o omega
        fi = fi - 2.0 * w * h + s * (w * w);
        gi = gi - w * w;
        u.f[col] = fi;
        u.g[col] = gi;
        if (u.W) u.W[(long long)t * n + col] = w;
        if (col == p) { u.selmask[col] = 1; selected = true; }
        if (!selected && gi > thr) {
          const double sc = u.score_mode ? gi : fmax(fi, 0.0) / gi;
          const long long sk = score_key(sc);
          if (better(sk, col, bv, bi)) { bv = sk; bi = col; }
        }
      }
      slot = 0;
      bcol = -1;
    }
  }
}

// ------------------------------------------ initialisation (Algorithms 1, 3) -
// g_i^(0) = ||a_i||^2 (f^(0) was written by the initial-score kernels), the
// non-finite check, F^(0) partial sums and the first argmax.
template <typename TA>
__device__ void init_pass(const Ctx<typename AccOf<TA>::type>& x, const UnitDesc& u,
                          uint64_t pol, long long& bv, int& bi, double& fsum, int& bad) {
  using Acc = typename AccOf<TA>::type;
  constexpr int V = Vec<TA>::V;
  const int n = u.n, m = u.m;
  const int m_vec = u.vec_ok ? (m / V) * V : 0;
  const TA* A = reinterpret_cast<const TA*>(u.A);
  for (int col = x.rank * NW + x.warp; col < n; col += x.ncta * NW) {
    const TA* cp = A + (long long)col * u.lda;
    Acc acc = Acc(0);
    for (int r = x.lane * V; r < m_vec; r += 32 * V) {
      Acc a[V];
      Vec<TA>::unpack(ldg_stream16(cp + r, pol), a);
      Acc tt = a[0] * a[0];
#pragma unroll
      for (int e = 1; e < V; ++e) tt = fma(a[e], a[e], tt);
      acc += tt;
    }
    for (int r = m_vec + x.lane; r < m; r += 32) {
      const Acc a = load_elem<TA>(cp + r);
      acc = fma(a, a, acc);
    }
    acc = warp_sum(acc);
    if (x.lane == 0) {
      const double g0 = to_f64(acc);
      const double f0 = ld_cg(u.f + col);
      // columns with g_i <= tau g_i^(0) are no longer candidates
      u.thr[col] = (g0 > 0.0) ? u.tau * g0 : __longlong_as_double(0x7ff0000000000000LL);
      u.g[col] = g0;
      u.selmask[col] = 0;
      if (!isfinite(g0) || !isfinite(f0)) bad = 1;
      if (u.mode == 0) fsum += g0;
      if (g0 > 0.0) {
        const double sc = u.score_mode ? g0 : fmax(f0, 0.0) / g0;
        const long long sk = score_key(sc);
          if (better(sk, col, bv, bi)) { bv = sk; bi = col; }
      }
    }
  }
  if (u.mode == 1) {
    // ||B||_F^2, the starting value of Theorem 3's recursion
    const Acc* B = reinterpret_cast<const Acc*>(u.T);
    for (int j = x.rank * NW + x.warp; j < u.r; j += x.ncta * NW) {
      const Acc* cp = B + (long long)j * u.ldt;
      double acc = 0.0;
      for (int r = x.lane; r < m; r += 32) { const double b = (double)cp[r]; acc += b * b; }
      acc = warp_sum(acc);
      if (x.lane == 0) {
        if (!isfinite(acc)) bad = 1;
        fsum += acc;
      }
    }
  }
}

// --------------------------------------------------------------- the unit ---
template <typename TA, int CW>
__device__ void run_unit(const Ctx<typename AccOf<TA>::type>& x, const UnitDesc& u) {
  using Acc = typename AccOf<TA>::type;
  // BF16/FP32 input: Q, Z (CSS), e and the coefficients are held as float
  // pairs and their products run in double-float (see row_gemv_df)
  constexpr bool kDF = sizeof(Acc) == 4;
  __shared__ double s_scal[4];
  const uint64_t pol_stream = policy_evict_first();
  const uint64_t pol_keep = policy_evict_last();
  const TeamDesc& tm = *x.team;
  const int m = u.m, n = u.n;
  float2* const Q2 = reinterpret_cast<float2*>(u.Q);
  float2* const Z2 = reinterpret_cast<float2*>(u.Z);
  float2* const coef2 = reinterpret_cast<float2*>(u.coef);
  float2* const e2 = reinterpret_cast<float2*>(u.e1);
  float2* const scoef2 = reinterpret_cast<float2*>(x.scoef);
  float2* const se2 = reinterpret_cast<float2*>(x.se64);

  // ---- initialisation: g^(0), F^(0), first argmax
  long long bv = -1;
  double fsum = 0.0;
  int bi = -1, bad = 0;
  init_pass<TA>(x, u, pol_stream, bv, bi, fsum, bad);
  if (__syncthreads_or(bad)) set_error(x.st, (int32_t)CSS_ERR_NONFINITE, 100);
  fsum = block_sum(fsum, x.sred);
  if (x.tid == 0) tm.part[x.rank * 4 + 2] = fsum;
  // both fused-step tile counters start at zero for this unit (the previous
  // unit of the team finished before its closing barrier)
  if (x.rank == 0 && x.tid == 0) {
    tm.tile_ctr[0] = 0u;
    tm.tile_ctr[1] = 0u;
  }
  const int cb0 = cta_argmax_publish(x, bv, bi);
  if (x.tid == 0) prefetch_column<TA>(u, cb0);
  if (!team_barrier(tm.bar, x.ncta, x.st, 1, x.epoch)) return;

  double F = team_sum(x, 2);  // meaningful in rank 0, thread 0
  if (x.rank == 0 && x.tid == 0) u.trace[0] = F;

  const bool tracing = u.trace_ns != nullptr && x.rank == 0 && x.tid == 0;
  int t = 0;
  auto mark = [&](int j) {
    if (tracing) u.trace_ns[(long long)t * 16 + j] = globaltimer_ns();
  };
  for (; t < u.k; ++t) {
    mark(0);
    // ---- Phase A: pivot p, outputs; c = Q_t^T a_p (FP64 Gram-Schmidt coefficients)
    int p = team_argmax(x);
    mark(1);
    const int p_arg = p;
    if (t < u.n_forced) p = u.forced[t];
    if (p < 0) break;
    // f_p, g_p for the error trace: loaded now, used after the staging below
    double fp = 0.0, gp = 1.0;
    if (x.rank == 0 && x.tid == 0) {
      fp = ld_cg(u.f + p);
      gp = ld_cg(u.g + p);
      // counter of the next iteration's fused step; its last user finished
      // before the previous iteration's final barrier
      tm.tile_ctr[(t + 1) & 1] = 0u;
      if (u.diag_argmax) u.diag_argmax[t] = p_arg;
      u.sel[t] = p;
    }
    const TA* ap = reinterpret_cast<const TA*>(u.A) + (long long)p * u.lda;
    if constexpr (kDF) {
      // a_p is exact in float
#pragma unroll 8
      for (int i = x.tid; i < m; i += NT) x.seacc[i] = load_elem<TA>(ap + i);
      __syncthreads();
      col_dots_df(x, m, t, Q2, (long long)m, x.seacc, [&](int j, float2 v) { coef2[j] = v; });
    } else {
#pragma unroll 8
      for (int i = x.tid; i < m; i += NT) x.se64[i] = to_f64(load_elem<TA>(ap + i));
      __syncthreads();
      col_dots<double>(x, m, t, u.Q, (long long)m, x.se64, [&](int j, double v) { u.coef[j] = v; });
    }
    if (x.rank == 0 && x.tid == 0) {
      F = F - fp / gp;   // Theorem 1 / Theorem 3
      u.trace[t + 1] = F;
    }
    mark(2);
    if (!team_barrier(tm.bar, x.ncta, x.st, 2, x.epoch)) return;
    mark(3);

    // ---- Phase C: e = a_p - Q_t c, ||e||^2 partials (delta_p of Eq. delta_omega)
    double nrm_part = 0.0;
    if constexpr (kDF) {
      for (int j = x.tid; j < t; j += NT) scoef2[j] = ld_cg(coef2 + j);
      __syncthreads();
      row_gemv_df(x, m, t, Q2, (long long)m, scoef2, NoPre{}, [&](int i, float2 sum, int) {
        const double ei = to_f64(x.seacc[i]) - df_to_f64(sum);   // a_p is still staged
        u.e[i] = ei;
        e2[i] = f64_to_df(ei);   // e as hi + lo, formed once
        nrm_part += ei * ei;
      });
    } else {
      for (int j = x.tid; j < t; j += NT) x.scoef[j] = ld_cg(u.coef + j);
      __syncthreads();
      row_gemv<double>(x, m, t, u.Q, (long long)m, x.scoef, NoPre{}, [&](int i, double sum, int) {
        const double ei = x.se64[i] - sum;   // a_p is still staged in se64
        u.e[i] = ei;
        nrm_part += ei * ei;
      });
    }
    mark(4);
    nrm_part = block_sum_to0(nrm_part, x.sred);
    if (x.tid == 0) tm.part[x.rank * 4 + 0] = nrm_part;
    if (!team_barrier(tm.bar, x.ncta, x.st, 4, x.epoch)) return;
    mark(5);

    // ---- Phase D: y_un = C e (CSS) or B (B^T e) (GCSS); d = Z^T e
    // stage e and reduce ||e||^2 over the team's partials (the same order as
    // team_sum) with both sets of loads in flight together
    double nrm_acc = 0.0;
    if (x.warp == 0)
      for (int r = x.lane; r < x.ncta; r += 32) nrm_acc += ld_cg(tm.part + r * 4 + 0);
    if constexpr (kDF) {
#pragma unroll 8
      for (int i = x.tid; i < m; i += NT) {
        const float2 ev = ld_cg(e2 + i);
        se2[i] = ev;
        x.seacc[i] = ev.x;
      }
    } else {
#pragma unroll 8
      for (int i = x.tid; i < m; i += NT) {
        const double ei = ld_cg(u.e + i);
        x.se64[i] = ei;
        x.seacc[i] = (Acc)ei;
      }
    }
    if (x.warp == 0) {
      nrm_acc = warp_sum(nrm_acc);
      // 1 / ||e||, once per CTA (FP64 square roots and divisions are slow)
      if (x.lane == 0) { s_scal[0] = nrm_acc; s_scal[1] = 1.0 / sqrt(nrm_acc); }
    }
    __syncthreads();
    const double nrm2 = s_scal[0];
    mark(6);
    double s_un = 0.0;
    if (u.mode == 0) {
      const Acc* C = reinterpret_cast<const Acc*>(u.T);
      constexpr int VC = 16 / sizeof(Acc);
      const int m_vec = u.t_vec_ok ? (m / VC) * VC : 0;
      double ey = 0.0;
      constexpr int UC = 16;  // 16-byte loads in flight per lane
      // the CTA's row results go through shared memory so that one warp, not
      // all sixteen, issues their FP64 conversions and the FP64 dot e^T y
      Acc* srow = reinterpret_cast<Acc*>(x.sred);
      const int rows_per_warp = (m + x.ncta * NW - 1) / (x.ncta * NW);
      const bool gather = rows_per_warp * NW <= NS * RB * (int)(sizeof(double) / sizeof(Acc));
      int kr = 0;
      for (int i = x.rank * NW + x.warp; i < m; i += x.ncta * NW, ++kr) {
        const Acc* cp = C + (long long)i * u.ldt;
        Acc accs[UC];
#pragma unroll
        for (int q = 0; q < UC; ++q) accs[q] = Acc(0);
        int l = x.lane * VC;
        for (; l + (UC - 1) * 32 * VC < m_vec; l += UC * 32 * VC) {
          uint4 raw[UC];
#pragma unroll
          for (int q = 0; q < UC; ++q) raw[q] = ldg_stream16(cp + l + q * 32 * VC, pol_keep);
#pragma unroll
          for (int q = 0; q < UC; ++q) {
            Acc cv[VC], ev[VC];
            if constexpr (sizeof(Acc) == 4) Vec<float>::unpack(raw[q], cv);
            else Vec<double>::unpack(raw[q], cv);
            lds_vec<Acc, VC>(x.seacc + l + q * 32 * VC, ev);
#pragma unroll
            for (int e = 0; e < VC; ++e) accs[q] = fma(cv[e], ev[e], accs[q]);
          }
        }
        for (; l < m_vec; l += 32 * VC) {
          Acc cv[VC], ev[VC];
          if constexpr (sizeof(Acc) == 4) Vec<float>::unpack(ldg_stream16(cp + l, pol_keep), cv);
          else Vec<double>::unpack(ldg_stream16(cp + l, pol_keep), cv);
          lds_vec<Acc, VC>(x.seacc + l, ev);
#pragma unroll
          for (int e = 0; e < VC; ++e) accs[0] = fma(cv[e], ev[e], accs[0]);
        }
        Acc acc = Acc(0);
#pragma unroll
        for (int q = 0; q < UC; ++q) acc += accs[q];
        for (int l2 = m_vec + x.lane; l2 < m; l2 += 32) acc = fma(__ldg(cp + l2), x.seacc[l2], acc);
        acc = warp_sum(acc);
        if (x.lane == 0) {
          if (gather) {
            srow[kr * NW + x.warp] = acc;
          } else {
            u.y[i] = (double)acc;
            ey += (kDF ? df_to_f64(se2[i]) : x.se64[i]) * (double)acc;
          }
        }
      }
      if (gather) {
        __syncthreads();
        if (x.warp == 0) {
          for (int idx = x.lane; idx < rows_per_warp * NW; idx += 32) {
            const int i = x.rank * NW + (idx % NW) + (idx / NW) * x.ncta * NW;
            if (i < m) {
              const double yi = (double)srow[idx];
              u.y[i] = yi;
              ey += (kDF ? df_to_f64(se2[i]) : x.se64[i]) * yi;
            }
          }
        }
      }
      mark(7);
      if constexpr (kDF)
        col_dots_df(x, m, t, Z2, (long long)m, se2, [&](int j, float2 v) { coef2[j] = v; });
      else
        col_dots<double>(x, m, t, u.Z, (long long)m, x.se64, [&](int j, double v) { u.coef[j] = v; });
      mark(8);
      ey = block_sum_to0(ey, x.sred);
      if (x.tid == 0) tm.part[x.rank * 4 + 1] = ey;
      if (!team_barrier(tm.bar, x.ncta, x.st, 5, x.epoch)) return;
      mark(9);
    } else {
      const Acc* B = reinterpret_cast<const Acc*>(u.T);
      if constexpr (kDF) {
        if (u.t_vec_ok && m % 4 == 0)
          col_dots_f4(x, m, u.r, B, u.ldt, x.seacc, [&](int j, double v) { u.ups[j] = v; });
        else
          col_dots<Acc>(x, m, u.r, B, u.ldt, x.seacc, [&](int j, double v) { u.ups[j] = v; });
      } else {
        col_dots<Acc>(x, m, u.r, B, u.ldt, x.seacc, [&](int j, double v) { u.ups[j] = v; });
      }
      if (!team_barrier(tm.bar, x.ncta, x.st, 5, x.epoch)) return;
      for (int j = x.tid; j < u.r; j += NT) {
        const double v = ld_cg(u.ups + j);
        x.scoef[j] = v;
        x.sups[j] = (Acc)v;
      }
      __syncthreads();
      row_gemv<Acc>(x, m, u.r, B, u.ldt, x.sups, NoPre{}, [&](int i, double sum, int) { u.y[i] = sum; });
      col_dots<double>(x, u.r, t, u.Z, (long long)u.r, x.scoef, [&](int j, double v) {
        if constexpr (kDF) coef2[j] = f64_to_df(v);
        else u.coef[j] = v;
      });
      double ss = 0.0;
      for (int j = x.tid; j < u.r; j += NT) ss += x.scoef[j] * x.scoef[j];
      s_un = block_sum_to0(ss, x.sred);
      if (x.tid == 0) s_scal[2] = s_un / nrm2;   // Theorem 4's ||upsilon||^2 for unit q
      if (x.rank == 0) {
        // upsilon^(t) = B^T q, column t of Z (read by later iterations only)
        const double inv = s_scal[1];
        for (int j = x.tid; j < u.r; j += NT) u.Z[(long long)t * u.r + j] = x.scoef[j] * inv;
      }
      if (!team_barrier(tm.bar, x.ncta, x.st, 6, x.epoch)) return;
      mark(9);
    }

    // ---- Phase E: q, y = y_un / ||e||, y' = y - Q (Q^T y), s
    double s;
    {
      // CSS: s = e^T y / ||e||^2 from the team's partials (team_sum's order),
      // by one thread; the coefficient loads are in flight meanwhile
      double ey_acc = 0.0;
      if (u.mode == 0 && x.warp == 0)
        for (int r = x.lane; r < x.ncta; r += 32) ey_acc += ld_cg(tm.part + r * 4 + 1);
      if constexpr (kDF) {
        for (int j = x.tid; j < t; j += NT) scoef2[j] = ld_cg(coef2 + j);
      } else {
        for (int j = x.tid; j < t; j += NT) x.scoef[j] = ld_cg(u.coef + j);
      }
      if (u.mode == 0 && x.warp == 0) {
        ey_acc = warp_sum(ey_acc);
        if (x.lane == 0) s_scal[2] = ey_acc / nrm2;
      }
      __syncthreads();
      const double inv = s_scal[1];
      s = s_scal[2];
      Acc* qv = reinterpret_cast<Acc*>(u.qv);
      Acc* ypv = reinterpret_cast<Acc*>(u.ypv);
      auto pre = [&](int i) { return make_double2(ld_cg(u.y + i), ld_cg(u.e + i)); };
      if constexpr (kDF) {
        row_gemv_df(x, m, t, Q2, (long long)m, scoef2, pre, [&](int i, float2 sum, double2 ye) {
          const double yi = ye.x * inv;
          const double qi = ye.y * inv;
          const float2 q2 = f64_to_df(qi);
          Q2[(long long)t * m + i] = q2;
          if (u.mode == 0) Z2[(long long)t * m + i] = f64_to_df(yi);
          qv[i] = q2.x;
          ypv[i] = (Acc)(yi - df_to_f64(sum) * inv);
        });
      } else {
        row_gemv<double>(x, m, t, u.Q, (long long)m, x.scoef, pre, [&](int i, double sum, double2 ye) {
          const double yi = ye.x * inv;
          const double qi = ye.y * inv;
          u.Q[(long long)t * m + i] = qi;
          if (u.mode == 0) u.Z[(long long)t * m + i] = yi;
          qv[i] = (Acc)qi;
          ypv[i] = (Acc)(yi - sum * inv);
        });
      }
    }
    mark(10);
    if (!team_barrier(tm.bar, x.ncta, x.st, 7, x.epoch)) return;
    mark(11);

    // ---- fused step over A
    {
      const Acc* qv = reinterpret_cast<const Acc*>(u.qv);
      const Acc* ypv = reinterpret_cast<const Acc*>(u.ypv);
#pragma unroll 4
      for (int i = x.tid; i < m; i += NT) {
        x.sq[i] = ld_cg(qv + i);
        x.sy[i] = ld_cg(ypv + i);
      }
      __syncthreads();
      mark(12);
      long long bv2 = -1;
      int bi2 = -1;
      fused_step<TA, CW>(x, u, t, p, s, pol_stream, bv2, bi2);
      mark(13);
      const int cb = cta_argmax_publish(x, bv2, bi2);
      if (x.tid == 0) prefetch_column<TA>(u, cb);
      mark(15);
    }
    if (!team_barrier(tm.bar, x.ncta, x.st, 8, x.epoch)) return;
    mark(14);
  }

  if (x.rank == 0 && x.tid == 0) {
    *u.n_sel = t;
    if (t < u.k) atomicAdd(&x.st->rank_exhausted, 1);
  }
  if (u.diag_f) {
    for (int i = (x.rank * NT + x.tid); i < n; i += x.ncta * NT) {
      u.diag_f[i] = ld_cg(u.f + i);
      u.diag_g[i] = ld_cg(u.g + i);
    }
  }
  team_barrier(tm.bar, x.ncta, x.st, 9, x.epoch);
}

template <typename TA, int CW>
__global__ void __launch_bounds__(NT, CSS_GREEDY_CTAS_PER_SM) greedy_kernel(GreedyLaunch L) {
  using Acc = typename AccOf<TA>::type;
  extern __shared__ __align__(16) unsigned char smem[];
  const int team_id = L.cta_team[blockIdx.x];
  const TeamDesc& tm = L.teams[team_id];
  Ctx<Acc> x;
  x.rank = blockIdx.x - tm.cta0;
  x.ncta = tm.ncta;
  x.tid = threadIdx.x;
  x.lane = threadIdx.x & 31;
  x.warp = threadIdx.x >> 5;
  x.st = L.st;
  x.team = &tm;
  // shared memory carve (see greedy_smem_bytes)
  const size_t mp = ((size_t)L.m_max + 3) & ~(size_t)3;  // keeps every sub-buffer 16-byte aligned
  size_t buf = mp * (sizeof(double) + sizeof(Acc));
  if (2 * mp * sizeof(Acc) > buf) buf = 2 * mp * sizeof(Acc);
  unsigned char* p = smem;
  x.sq = reinterpret_cast<Acc*>(p);
  x.sy = reinterpret_cast<Acc*>(p) + mp;
  x.se64 = reinterpret_cast<double*>(p);
  x.seacc = reinterpret_cast<Acc*>(p + mp * sizeof(double));
  p += buf;
  const size_t nco = (size_t)max(L.k_max, L.r_max);
  x.scoef = reinterpret_cast<double*>(p);
  p += (nco * sizeof(double) + 15) & ~(size_t)15;
  x.sups = reinterpret_cast<Acc*>(p);
  p += ((size_t)L.r_max * sizeof(Acc) + 15) & ~(size_t)15;
  x.sred = reinterpret_cast<double*>(p);
  __shared__ uint32_t s_epoch;
  if (threadIdx.x == 0) s_epoch = 0u;   // used by thread 0 only
  x.epoch = &s_epoch;

  for (int ui = tm.u_begin; ui < tm.u_end; ++ui) {
    const UnitDesc u = L.units[L.order[ui]];
    run_unit<TA, CW>(x, u);
    if (ld_volatile_i32(&L.st->code) != 0) return;
  }
}

template <typename TA, int CW>
void* kernel_ptr() { return (void*)greedy_kernel<TA, CW>; }

void* pick_kernel(int dtype, int cw) {
  switch (dtype) {
    case CSS_F64:
      return cw == 2 ? kernel_ptr<double, 2>() : cw == 8 ? kernel_ptr<double, 8>() : kernel_ptr<double, 4>();
    case CSS_F32:
      return cw == 2 ? kernel_ptr<float, 2>() : cw == 8 ? kernel_ptr<float, 8>() : kernel_ptr<float, 4>();
    default:
      return cw == 2 ? kernel_ptr<__nv_bfloat16, 2>() : cw == 8 ? kernel_ptr<__nv_bfloat16, 8>()
                     : kernel_ptr<__nv_bfloat16, 4>();
  }
}

}  // namespace

namespace CSS_GREEDY_SHAPE {

size_t greedy_smem_bytes(int dtype, int m_max, int k_max, int r_max) {
  const size_t sa = (dtype == CSS_F64) ? 8 : 4;
  const size_t mp = ((size_t)m_max + 3) & ~(size_t)3;
  size_t buf = mp * (8 + sa);
  if (2 * mp * sa > buf) buf = 2 * mp * sa;
  const size_t nco = (size_t)(k_max > r_max ? k_max : r_max);
  size_t b = buf + ((nco * 8 + 15) & ~(size_t)15) + (((size_t)r_max * sa + 15) & ~(size_t)15);
  b += (size_t)NS * RB * sizeof(double);
  return b;
}

int greedy_occupancy(int dtype, int tile_cols, size_t smem) {
  void* k = pick_kernel(dtype, tile_cols);
  if (smem > 48 * 1024) {
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return 0;
  }
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, NT, smem) != cudaSuccess) return 0;
  return occ;
}

cudaError_t greedy_launch(const GreedyLaunch& L, cudaStream_t stream) {
  // the plan (team sizes, split slots) was made for this shape's CTAs
  if (L.threads != NT) return cudaErrorInvalidConfiguration;
  void* k = pick_kernel(L.dtype, L.tile_cols);
  if (L.smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem);
    if (e != cudaSuccess) return e;
  }
  GreedyLaunch arg = L;
  void* args[] = {&arg};
  return cudaLaunchCooperativeKernel(k, dim3(L.grid), dim3(NT), args, L.smem, stream);
}

}  // namespace CSS_GREEDY_SHAPE

#ifdef CSS_GREEDY_EXPORT_BASIS

// Q (FP64, or double-float pairs for FP32/BF16 input) to a caller buffer as
// FP64; columns at or beyond the number selected become zero.
__global__ void export_basis_kernel(const double* __restrict__ Q, int df, int m, int k,
                                    const int* __restrict__ n_sel, double* __restrict__ out) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)m * k) return;
  const int t = (int)(idx / m);
  double v = 0.0;
  if (t < *n_sel) {
    if (df) {
      const float2 q2 = reinterpret_cast<const float2*>(Q)[idx];
      v = (double)q2.x + (double)q2.y;
    } else {
      v = Q[idx];
    }
  }
  out[idx] = v;
}

cudaError_t export_basis(int dtype, const double* Q, int m, int k, const int* n_sel, double* out,
                         cudaStream_t stream) {
  const long long total = (long long)m * k;
  export_basis_kernel<<<(unsigned)((total + 255) / 256), 256, 0, stream>>>(Q, dtype != CSS_F64, m, k, n_sel,
                                                                           out);
  return cudaGetLastError();
}

#endif  // CSS_GREEDY_EXPORT_BASIS

}  // namespace css
