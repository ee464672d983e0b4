// Tensor-core GEMMs (tcgen05 + TMA) for the two dense contractions of the
// distributed variant:
//
//   projection   B = A Omega (Sec. 5.1, Algorithm 2).  D = A[rows, K] Omega[K, :]
//                per row tile of A and per slice of the K = n columns (the
//                slices are Algorithm 2's per-mapper partial sums; a second
//                kernel adds them in a fixed order).  A is M-major (column-
//                major A), Omega is K-major.
//   norms        f_i = ||B^T a_i||^2 (Algorithm 3's initial scores).  D = A^T B
//                per tile of 128 columns of A, both operands K-major; B (FP32)
//                is split into two BF16 parts B1 + B2 (16 significant bits)
//                that accumulate into the same TMEM tile; the epilogue sums
//                squares of each row in FP64.  A third part would carry B's
//                last 8 bits, but the tensor cores' own accumulation error is
//                larger than that part: measured against the FP64 oracle at
//                2048 x 65536, r = 400, the initial scores are within 2.9 u
//                sqrt(m) with two parts and 4.5 u sqrt(m) with three.
//
// One CTA = 6 warps: warp 0 lane 0 issues TMA loads into a 3-stage shared
// memory ring (128-byte swizzle), warp 1 owns the TMEM allocation and its lane
// 0 issues tcgen05.mma (BF16 x BF16 -> FP32, M = 128, up to two MMAs of
// N <= 256 side by side in TMEM), warps 2-5 read the accumulator back with
// tcgen05.ld (each warp its 32-lane quarter of TMEM).  Every mbarrier wait is
// bounded; on expiry an error flag is set and the CTA tears down.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "tc.cuh"
#include "css_common.cuh"

namespace css {
namespace tc {
namespace {

constexpr int BM = 128;
constexpr int BK = 64;        // K elements per stage: one 128-byte swizzle row
constexpr int STAGES = 4;     // ring depth, at most (Params::stages picks 1..4)
constexpr int kSmemMax = 227 * 1024;   // dynamic shared memory of one CTA
constexpr int kThreads = 192;
constexpr int kTmemCols = 512;
// BF16 parts of an FP32 operand (B of the GCSS norms, U' of the CSS scores):
// hi + lo carry 16 significant bits
constexpr int kParts = 2;

struct Params {
  int mode;          // 0 projection partials, 1 squared row norms, 2 C = A A^T, 3 column dots
  int M;             // rows of D (projection: m; norms: n; syrk, column dots: m)
  int N;             // useful columns of D (r; syrk: m; column dots: n)
  int n_half;        // columns per MMA (multiple of 16, <= 256)
  int halves;        // 1 or 2
  int n_tile;        // syrk / column dots: columns of D per CTA (blockIdx.y tiles)
  int kb_total;      // K blocks of 64 over the whole contraction
  int kb_per_cta;    // projection: K blocks per slice
  int nparts;        // BF16 parts summed into the accumulator
  int a_part_stride; // column offset between parts in A's tensor map
  int b_part_stride; // column offset between parts in B's tensor map
  int stage_bytes;
  float* out;        // projection: [slice][M x N] partials; syrk: C (ld M)
  double* f;         // norms: f[M]; column dots: partial[M-tile][N]
  const void* Acol;  // column dots: the matrix dotted with D's columns (BF16, or FP32 if acol_f32)
  long long lda_col;
  int acol_f32;
  int* err;
  unsigned long long spin_ns;
  // symmetric use of C = A A^T: mode 2 computes only the tiles that touch
  // the lower triangle (rows >= columns); mode 3 multiplies by the upper
  // triangle U' of C (diagonal halved), so M-tile J starts at K = 128 J
  int tri;
  // group: one ring stage holds the distinct tiles of every part for one K
  // block (a tile shared by all parts is loaded once), and the parts' MMAs
  // run back to back on it; otherwise each (K block, part) is its own stage
  int group;
  int stages;        // ring depth (1..STAGES)
  int stall;         // test hook: the epilogue also waits on a phase nothing completes
  // modes 2 and 3: K blocks per blockIdx.z chunk.  The tensor cores' FP32
  // accumulation loses up to about one unit in the last place of the running
  // sum per addition, always toward zero, so the error of a TMEM accumulation
  // grows with its length: K is cut into chunks whose sums are added
  // afterwards in FP64 (mode 2: per chunk partial tiles; mode 3: partial dots)
  int kb_chunk;
  int tiles_lower;   // mode 2: tiles per chunk (those touching the lower triangle)
  // part pairs (FP32 operands split into BF16 parts on both sides): when
  // npairs > 0 every (K block, pair) is its own stage and pair q multiplies
  // part pair_a[q] of A by part pair_b[q] of B, all into one accumulator.
  // An M- or N-major operand's parts sit a_kpart / b_kpart columns apart in
  // K; a K-major operand's parts use a_part_stride / b_part_stride.
  int npairs;
  int pair_a[4];
  int pair_b[4];
  int a_kpart;
  int b_kpart;
  // pair q accumulates into TMEM columns acc2_col * pair_acc[q] onwards.
  // The tensor cores' accumulation truncates by up to one unit of the
  // running sum per MMA, so the small cross products (hi lo, lo hi) go to a
  // second accumulator whose sum, and so its truncation, is 2^8 smaller; the
  // epilogue adds the two.  acc2_col = 0: one accumulator.
  int pair_acc[4];
  int acc2_col;
};

// Mode 2 tiles (BM rows x 256 columns) that touch the lower triangle: tile
// (bx, by) does when bx * 128 + 127 >= by * 256, i.e. by <= bx / 2.  Their
// index in row-tile order.
__host__ __device__ __forceinline__ int lower_tile_index(int bx, int by) {
  // sum over b < bx of (b / 2 + 1)
  const int q = bx / 2;
  const int before = bx + ((bx & 1) ? q * q : q * (q - 1));
  return before + by;
}
__host__ __device__ __forceinline__ int lower_tile_count(int mtiles) { return lower_tile_index(mtiles, 0); }

// ------------------------------------------------------------- PTX glue -----
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait for the phase with the given parity.  false: timed out (the
// error flag is set) or another role already failed.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err,
                                          unsigned long long budget) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = gtimer();
  while (true) {
#pragma unroll 1
    for (int i = 0; i < 32; ++i)
      if (mbar_try_wait(bar, parity)) return true;
    if (*(volatile int*)err != 0) return false;
    if (gtimer() - t0 > budget) {
      atomicCAS(err, 0, (int)CSS_ERR_TIMEOUT);
      return false;
    }
  }
}
// Wait used on the way out of a failed CTA: the copies and MMAs this CTA
// issued always complete, so it waits for them whatever the error flag says
// (a fixed bound of 1 s; it returns in microseconds in practice), so that no
// copy lands in, and no MMA reads, the shared memory or TMEM of an exited CTA.
__device__ __forceinline__ void mbar_drain(uint32_t bar, uint32_t parity) {
  const uint64_t t0 = gtimer();
  while (!mbar_try_wait(bar, parity))
    if (gtimer() - t0 > 1000000000ull) return;
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int c0,
                                            int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], "
      "[%2];" ::"r"(dst),
      "l"((uint64_t)map), "r"(bar), "r"(c0), "r"(c1)
      : "memory");
}
// Shared-memory matrix descriptor, 128-byte swizzle (sm_100 format).
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
// Instruction descriptor: kind::f16, BF16 x BF16 -> FP32.
__device__ __forceinline__ uint32_t make_idesc(int N, int M, bool a_mn, bool b_mn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void umma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                     uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}
__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// Double-float sums for the epilogues: products of two floats are exact as
// p + e (Dekker, by FMA) and sums keep their rounding error (Knuth's TwoSum),
// 48 significant bits without FP64 instructions (which issue ~50x slower than
// FP32 on this part).
__device__ __forceinline__ void df_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void df_add2(float& ah, float& al, float bh, float bl) {
  float s, e;
  df_two_sum(ah, bh, s, e);
  e += al + bl;
  ah = s + e;
  al = e - (ah - s);
}
__device__ __forceinline__ void df_acc_prod(float& sh, float& sl, float a, float b) {
  const float p = a * b;
  const float e = fmaf(a, b, -p);
  float s, err;
  df_two_sum(sh, p, s, err);
  sh = s;
  sl += err + e;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
      "[%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// v += the second accumulator's 16 columns at taddr (when acc2_col != 0),
// rounded to nearest once
__device__ __forceinline__ void add_acc2(uint32_t taddr, int acc2_col, float (&v)[16]) {
  if (acc2_col == 0) return;
  float w[16];
  tmem_ld16(taddr, w);
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] += w[i];
}

template <bool A_MN, bool B_MN>
__global__ void __launch_bounds__(kThreads, 1)
    tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, Params P) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int a_bytes = BM * BK * 2;
  const int NSTG = P.stages;
  uint8_t* bars_base = smem + NSTG * P.stage_bytes;
  uint64_t* full = (uint64_t*)bars_base;
  uint64_t* empty = full + STAGES;
  uint64_t* done = empty + STAGES;
  uint64_t* never = done + 1;   // test hook: a phase that nothing completes
  uint32_t* s_tmem = (uint32_t*)(never + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // work of this CTA
  const int tile0 = blockIdx.x * BM;
  int kb_begin = 0, kb_end = P.kb_total;
  int ntile0 = 0;
  if (P.mode == 0) {
    kb_begin = blockIdx.y * P.kb_per_cta;
    kb_end = min(P.kb_total, kb_begin + P.kb_per_cta);
  } else if (P.mode >= 2) {
    ntile0 = blockIdx.y * P.n_tile;
    kb_begin = blockIdx.z * P.kb_chunk;
    kb_end = min(P.kb_total, kb_begin + P.kb_chunk);
  }
  // strictly upper tile of C: not needed (the lower triangle is mirrored)
  if (P.tri && P.mode == 2 && tile0 + BM - 1 < ntile0) return;
  // U' rows of this tile are zero left of column tile0
  if (P.tri && P.mode == 3) {
    kb_begin = max(kb_begin, tile0 / BK);
    if (kb_begin >= kb_end) {
      // nothing of this K chunk meets the tile: its partial dots are zero
      for (int j = threadIdx.x; j < P.n_tile; j += blockDim.x) {
        const int c = ntile0 + j;
        if (c < P.N) P.f[((long long)blockIdx.x * gridDim.z + blockIdx.z) * P.N + c] = 0.0;
      }
      return;
    }
  }
  const int parts = P.nparts;
  // group mode: tiles per stage (a part stride of 0 means one shared tile)
  const int nA = (P.group && P.a_part_stride != 0) ? parts : 1;
  const int nB = (P.group && P.b_part_stride != 0) ? parts : 1;
  const int b_tile_bytes = P.halves * P.n_half * BK * 2;
  // stages per K block: one (group), one per pair, or one per part
  const int per_kb = P.group ? 1 : (P.npairs > 0 ? P.npairs : parts);
  const int n_it = max(0, kb_end - kb_begin) * per_kb;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NSTG; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    mbar_init(smem_u32(done), 1);
    mbar_init(smem_u32(never), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_tmem)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *s_tmem;

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------------------ producer
    int issued = 0;
    for (int it = 0; it < n_it; ++it) {
      const int s = it % NSTG;
      const uint32_t ph = (uint32_t)((it / NSTG) & 1);
      if (!mbar_wait(smem_u32(&empty[s]), ph ^ 1u, P.err, P.spin_ns)) break;
      const int kb = kb_begin + it / per_kb;
      const int q_it = it % per_kb;
      const int part_a0 = P.group ? 0 : (P.npairs > 0 ? P.pair_a[q_it] : q_it);
      const int part_b0 = P.group ? 0 : (P.npairs > 0 ? P.pair_b[q_it] : q_it);
      const int k0 = kb * BK;
      uint8_t* sa = smem + s * P.stage_bytes;
      uint8_t* sb = sa + nA * a_bytes;
      const uint32_t fb = smem_u32(&full[s]);
      mbar_expect_tx(fb, (uint32_t)(nA * a_bytes + nB * b_tile_bytes));
      for (int pa = 0; pa < nA; ++pa) {
        const int part = part_a0 + pa;
        uint8_t* ta = sa + pa * a_bytes;
        if (A_MN) {
          const int ka = part * P.a_kpart + k0;
          tma_load_2d(smem_u32(ta), &tmA, fb, tile0, ka);
          tma_load_2d(smem_u32(ta + 64 * BK * 2), &tmA, fb, tile0 + 64, ka);
        } else {
          tma_load_2d(smem_u32(ta), &tmA, fb, k0, part * P.a_part_stride + tile0);
        }
      }
      for (int pb = 0; pb < nB; ++pb) {
        const int part = part_b0 + pb;
        uint8_t* tb = sb + pb * b_tile_bytes;
        if (B_MN) {
          // N-major B: 64-row boxes stacked 8 KB apart (the descriptor's LBO)
          for (int q = 0; q < P.halves * P.n_half / 64; ++q)
            tma_load_2d(smem_u32(tb + q * 64 * BK * 2), &tmB, fb, ntile0 + 64 * q, part * P.b_kpart + k0);
        } else {
          for (int h = 0; h < P.halves; ++h)
            tma_load_2d(smem_u32(tb + h * P.n_half * BK * 2), &tmB, fb, k0,
                        ntile0 + part * P.b_part_stride + h * P.n_half);
        }
      }
      issued = it + 1;
    }
    // the copies issued last (one per stage) have landed before the CTA
    // exits, also when a wait failed and the MMA issuer stopped consuming
    for (int it = max(0, issued - NSTG); it < issued; ++it) {
      const int s = it % NSTG;
      mbar_drain(smem_u32(&full[s]), (uint32_t)((it / NSTG) & 1));
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------------------------------------------------- MMA issuer
    const uint32_t idesc = make_idesc(P.n_half, BM, A_MN, B_MN);
    // MMAs that share one stage: group mode runs every part on it; otherwise
    // a stage is one part or one pair
    const int pg = P.group ? parts : 1;
    for (int it = 0; it < n_it; ++it) {
      const int s = it % NSTG;
      const uint32_t ph = (uint32_t)((it / NSTG) & 1);
      if (!mbar_wait(smem_u32(&full[s]), ph, P.err, P.spin_ns)) break;
      fence_after();
      const uint32_t sa0 = smem_u32(smem + s * P.stage_bytes);
      const uint32_t sb0 = sa0 + nA * a_bytes;
#pragma unroll
      for (int ks = 0; ks < BK / 16; ++ks) {
        for (int pp = 0; pp < pg; ++pp) {
          // the stage's tiles, its accumulator, and whether this MMA is the
          // first into that accumulator (its input is then ignored)
          const int ia = nA > 1 ? pp : 0, ib = nB > 1 ? pp : 0;
          uint32_t acc = 0;
          bool first = it == 0 && ks == 0 && pp == 0;
          if (P.npairs > 0) {
            const int q = it % per_kb;
            acc = (uint32_t)(P.pair_acc[q] * P.acc2_col);
            first = it / per_kb == 0 && ks == 0;
            for (int q2 = 0; q2 < q; ++q2)
              if (P.pair_acc[q2] == P.pair_acc[q]) first = false;
          }
          const uint32_t sa = sa0 + ia * a_bytes;
          const uint32_t sb = sb0 + ib * b_tile_bytes;
          // A: M-major -> 16 K rows of 128 bytes per step; K-major -> 32 bytes
          const uint64_t ad = A_MN ? make_desc(sa + ks * 2048, 64 * BK * 2, 1024)
                                   : make_desc(sa + ks * 32, 16, 1024);
          for (int h = 0; h < P.halves; ++h) {
            const uint64_t bd = B_MN ? make_desc(sb + h * P.n_half * BK * 2 + ks * 2048, 64 * BK * 2, 1024)
                                     : make_desc(sb + h * P.n_half * BK * 2 + ks * 32, 16, 1024);
            umma(tmem + acc + h * P.n_half, ad, bd, idesc, first ? 0u : 1u);
          }
        }
      }
      umma_commit(smem_u32(&empty[s]));
    }
    umma_commit(smem_u32(done));
    // every MMA issued has finished before TMEM is released at the end
    mbar_drain(smem_u32(done), 0u);
  } else if (warp >= 2) {
    // ------------------------------------------------------------ epilogue
    const int q = warp & 3;                  // TMEM lane quarter of this warp
    const int row = tile0 + q * 32 + lane;
    bool ok = mbar_wait(smem_u32(done), 0u, P.err, P.spin_ns) && *(volatile int*)P.err == 0;
    if (ok && P.stall) ok = mbar_wait(smem_u32(never), 0u, P.err, P.spin_ns);
    // one decision for all four epilogue warps (tcgen05.ld is warp-collective
    // and the column-dot epilogue synchronises the four warps)
    {
      uint32_t all;
      asm volatile(
          "{\n .reg .pred pa, pb;\n setp.ne.u32 pa, %1, 0;\n"
          " barrier.red.and.pred pb, 1, 128, pa;\n selp.u32 %0, 1, 0, pb;\n}"
          : "=r"(all)
          : "r"((uint32_t)ok)
          : "memory");
      ok = all != 0;
    }
    fence_after();
    if (ok && n_it == 0) {
      // empty K slice: its partial product is zero (TMEM was never written)
      if (P.mode == 0 && row < P.M)
        for (int j = 0; j < P.N; ++j) P.out[(long long)blockIdx.y * P.M * P.N + (long long)j * P.M + row] = 0.f;
      if (P.mode == 1 && row < P.M) P.f[row] = 0.0;
    } else if (ok && P.mode == 3) {
      // column dots: partial[M-tile][c] = sum over this tile's rows r of
      // Acol[r, c] * D[r, c]; rows are TMEM lanes, so each 16-column chunk is
      // reduced across the warp (transpose reduction) and then across warps
      // (products exact as hi + lo, sums in double-float, one FP64 add per
      // column at the end)
      __shared__ float2 cred[4][16];
      const int ncols = P.halves * P.n_half;
      for (int j0 = 0; j0 < ncols; j0 += 16) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)j0, v);
        add_acc2(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(P.acc2_col + j0), P.acc2_col, v);
        float ph[16], pl[16];
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) {
          const int c = ntile0 + j0 + jj;
          ph[jj] = 0.f;
          pl[jj] = 0.f;
          if (row < P.M && c < P.N) {
            const long long ai = (long long)c * P.lda_col + row;
            const float a = P.acol_f32 ? reinterpret_cast<const float*>(P.Acol)[ai]
                                       : __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(P.Acol)[ai]);
            ph[jj] = a * v[jj];
            pl[jj] = fmaf(a, v[jj], -ph[jj]);
          }
        }
        // 16 values over 32 lanes: lane L ends with the warp sum of index L >> 1
#pragma unroll
        for (int st = 0; st < 4; ++st) {
          const int mask = 16 >> st, half = 8 >> st;
          const bool up = (lane & mask) != 0;
#pragma unroll
          for (int jj = 0; jj < half; ++jj) {
            const float sh = up ? ph[jj] : ph[jj + half], sl = up ? pl[jj] : pl[jj + half];
            const float kh = up ? ph[jj + half] : ph[jj], kl = up ? pl[jj + half] : pl[jj];
            const float oh = __shfl_xor_sync(0xffffffffu, sh, mask);
            const float ol = __shfl_xor_sync(0xffffffffu, sl, mask);
            ph[jj] = kh;
            pl[jj] = kl;
            df_add2(ph[jj], pl[jj], oh, ol);
          }
        }
        {
          const float oh = __shfl_xor_sync(0xffffffffu, ph[0], 1);
          const float ol = __shfl_xor_sync(0xffffffffu, pl[0], 1);
          df_add2(ph[0], pl[0], oh, ol);
        }
        if ((lane & 1) == 0) cred[q][lane >> 1] = make_float2(ph[0], pl[0]);
        asm volatile("bar.sync 1, 128;" ::: "memory");
        if (q == 0 && lane < 16) {
          const int c = ntile0 + j0 + lane;
          if (c < P.N) {
            float h = cred[0][lane].x, l = cred[0][lane].y;
            for (int w = 1; w < 4; ++w) df_add2(h, l, cred[w][lane].x, cred[w][lane].y);
            P.f[((long long)blockIdx.x * gridDim.z + blockIdx.z) * P.N + c] = to_f64(h) + to_f64(l);
          }
        }
        asm volatile("bar.sync 1, 128;" ::: "memory");
      }
    } else if (ok) {
      float sh = 0.f, sl = 0.f;   // mode 1: sum of squares in double-float
      float* tile_out = nullptr;
      if (P.mode == 2)
        tile_out = P.out + ((long long)blockIdx.z * P.tiles_lower + lower_tile_index(blockIdx.x, blockIdx.y)) *
                               (long long)(BM * P.n_tile);
      const int ncols = P.halves * P.n_half;
      for (int j0 = 0; j0 < ncols; j0 += 16) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)j0, v);
        add_acc2(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(P.acc2_col + j0), P.acc2_col, v);
        if (row < P.M) {
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) {
            const int j = j0 + jj;
            if (P.mode == 2) {
              // chunk z's partial of this tile: tile_out holds BM x n_tile
              // values, column-major
              const int c = ntile0 + j;
              if (c < P.N) tile_out[(long long)j * BM + (row - tile0)] = v[jj];
            } else if (j < P.N) {
              if (P.mode == 0)
                P.out[(long long)blockIdx.y * P.M * P.N + (long long)j * P.M + row] = v[jj];
              else
                df_acc_prod(sh, sl, v[jj], v[jj]);
            }
          }
        }
      }
      if (P.mode == 1 && row < P.M) P.f[row] = to_f64(sh) + to_f64(sl);
    }
    fence_before();
  }
  __syncthreads();
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols)
                 : "memory");
  }
}

// B (FP32, m x r, ldb) -> kParts BF16 parts B1 + B2 (m x rpad each, ld mpad),
// laid out side by side: part p, column j at Bp[(p * rpad + j) * mpad + i].
// tri: B is the symmetric C with only its lower triangle valid, and the parts
// hold U' (column j, row i: C[i, j] for i > j, C[j, j] / 2 on the diagonal,
// 0 above), so that a_i^T C a_i = 2 a_i^T U' a_i.
__global__ void split_parts_kernel(const float* __restrict__ B, long long ldb, int m, int r, int mpad,
                                   int rpad, __nv_bfloat16* __restrict__ Bp, int tri) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long tot = (long long)mpad * rpad;
  if (idx >= tot) return;
  const int i = (int)(idx % mpad), j = (int)(idx / mpad);
  float v = (i < m && j < r && (!tri || i >= j)) ? B[(long long)j * ldb + i] : 0.f;
  if (tri && i == j) v *= 0.5f;
#pragma unroll
  for (int p = 0; p < kParts; ++p) {
    const __nv_bfloat16 b = __float2bfloat16_rn(v);
    v -= __bfloat162float(b);
    Bp[(long long)(p * rpad + j) * mpad + i] = b;
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

// 2-D BF16 tensor map: dim0 (contiguous) x dim1 with row pitch ld elements,
// box {64, box1}, 128-byte swizzle, zero fill outside the tensor.
bool make_map(CUtensorMap* map, const void* base, uint64_t dim0, uint64_t dim1, uint64_t ld,
              uint32_t box1) {
  auto fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t gdim[2] = {dim0, dim1};
  const cuuint64_t gstride[1] = {ld * 2};
  const cuuint32_t box[2] = {64, box1};
  const cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), gdim, gstride, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

void halves_for(int r, int& n_half, int& halves) {
  if (r <= 256) {
    halves = 1;
    n_half = (r + 15) / 16 * 16;
  } else {
    halves = 2;
    n_half = ((r + 1) / 2 + 15) / 16 * 16;
  }
}

size_t smem_for(int stage_bytes, int stages) { return (size_t)stages * stage_bytes + 256 + 1024; }

// Deepest ring (up to `want` stages) that fits in one CTA's shared memory.
int fit_stages(int stage_bytes, int want) {
  int st = want;
  while (st > 1 && smem_for(stage_bytes, st) > (size_t)kSmemMax) --st;
  return st;
}

}  // namespace

bool supported(const void* A, long long lda, int m, int r) {
  if (r < 1 || r > 512 || m < 1) return false;
  if (((uintptr_t)A & 15u) != 0 || (lda % 8) != 0) return false;
  return encode_fn() != nullptr;
}

int project_slices(int m, int sms) {
  const int mt = (m + BM - 1) / BM;
  return std::max(1, sms / mt);
}

cudaError_t project_partials(const void* A, long long lda, int m, int n, const void* Om, long long ldo,
                             int r, int slices, float* partial, int* err, unsigned long long spin_ns,
                             cudaStream_t s) {
  CUtensorMap ta, tb;
  int n_half, halves;
  halves_for(r, n_half, halves);
  if (!make_map(&ta, A, (uint64_t)m, (uint64_t)n, (uint64_t)lda, BK)) return cudaErrorInvalidValue;
  if (!make_map(&tb, Om, (uint64_t)n, (uint64_t)r, (uint64_t)ldo, (uint32_t)n_half))
    return cudaErrorInvalidValue;
  Params P{};
  P.mode = 0;
  P.M = m;
  P.N = r;
  P.n_half = n_half;
  P.halves = halves;
  P.kb_total = (n + BK - 1) / BK;
  P.kb_per_cta = (P.kb_total + slices - 1) / slices;
  P.nparts = 1;
  P.stage_bytes = BM * BK * 2 + halves * n_half * BK * 2;
  P.stages = fit_stages(P.stage_bytes, STAGES);
  P.out = partial;
  P.err = err;
  P.spin_ns = spin_ns;
  const size_t smem = smem_for(P.stage_bytes, P.stages);
  cudaError_t e = cudaFuncSetAttribute(tc_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((m + BM - 1) / BM, slices);
  tc_kernel<true, false><<<grid, kThreads, smem, s>>>(ta, tb, P);
  return cudaGetLastError();
}

size_t colnorm_scratch_bytes(int m, int r) {
  const int mpad = (m + 7) / 8 * 8;
  const int rpad = (r + 15) / 16 * 16;
  return (size_t)mpad * kParts * rpad * 2;
}

cudaError_t colnorms(const void* A, long long lda, int m, int n, const float* B, long long ldb, int r,
                     void* scratch, double* f, int* err, unsigned long long spin_ns, cudaStream_t s,
                     int stall) {
  const int mpad = (m + 7) / 8 * 8;
  const int rpad = (r + 15) / 16 * 16;
  __nv_bfloat16* Bp = (__nv_bfloat16*)scratch;
  const long long tot = (long long)mpad * rpad;
  split_parts_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(B, ldb, m, r, mpad, rpad, Bp, 0);
  CUtensorMap ta, tb;
  int n_half, halves;
  halves_for(r, n_half, halves);
  if (!make_map(&ta, A, (uint64_t)m, (uint64_t)n, (uint64_t)lda, BM)) return cudaErrorInvalidValue;
  if (!make_map(&tb, Bp, (uint64_t)mpad, (uint64_t)(kParts * rpad), (uint64_t)mpad, (uint32_t)n_half))
    return cudaErrorInvalidValue;
  Params P{};
  P.mode = 1;
  P.M = n;
  P.N = r;
  P.n_half = n_half;
  P.halves = halves;
  P.kb_total = (m + BK - 1) / BK;
  P.kb_per_cta = P.kb_total;
  P.nparts = kParts;
  P.b_part_stride = rpad;
  P.stage_bytes = BM * BK * 2 + halves * n_half * BK * 2;
  P.stages = fit_stages(P.stage_bytes, STAGES);
  P.f = f;
  P.err = err;
  P.spin_ns = spin_ns;
  P.stall = stall;
  const size_t smem = smem_for(P.stage_bytes, P.stages);
  cudaError_t e = cudaFuncSetAttribute(tc_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((n + BM - 1) / BM, 1);
  tc_kernel<false, false><<<grid, kThreads, smem, s>>>(ta, tb, P);
  return cudaGetLastError();
}

__global__ void sum_rows_kernel(const double* __restrict__ partial, int nblk, int n,
                                double* __restrict__ out, double scale) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += partial[(long long)b * n + i];
  out[i] = scale * s;
}

// C = sum over the K chunks of their partial tiles (FP64 sums in chunk
// order, rounded once to FP32), written to both triangles of C (ld m)
// through 32 x 32 shared-memory tiles, so reads and writes are coalesced.
// Only the 32 x 32 tiles on or below the diagonal run; each lies inside one
// chunk tile of 128 x 256.
__global__ void reduce_lower_kernel(const float* __restrict__ parts, int chunks, int tiles_lower, int m,
                                    float* __restrict__ C) {
  __shared__ float tile[32][33];
  const int bi = blockIdx.x, bj = blockIdx.y;   // rows bi*32.., columns bj*32..
  if (bi < bj) return;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int r = bi * 32 + tx;
  const int bx = (bi * 32) / BM, by = (bj * 32) / 256;
  const long long chunk_stride = (long long)tiles_lower * BM * 256;
  const float* src = parts + (long long)lower_tile_index(bx, by) * BM * 256;
  for (int k = ty; k < 32; k += blockDim.y) {
    const int c = bj * 32 + k;
    float v = 0.f;
    if (r < m && c < m && r >= c) {
      const long long local = (long long)(c - by * 256) * BM + (r - bx * BM);
      double sum = 0.0;
      for (int z = 0; z < chunks; ++z) sum += (double)src[z * chunk_stride + local];
      v = (float)sum;
      C[(long long)c * m + r] = v;
    }
    tile[k][tx] = v;
  }
  __syncthreads();
  // C[c, r] = C[r, c] for r > c
  for (int k = ty; k < 32; k += blockDim.y) {
    const int c = bj * 32 + tx, r2 = bi * 32 + k;
    if (r2 < m && c < m && r2 > c) C[(long long)r2 * m + c] = tile[tx][k];
  }
}

// K chunking of the initial-score GEMMs (see Params::kb_chunk): C = A A^T
// accumulates at most 4096 products per TMEM sum (chunks capped at 32, so
// very wide A gets longer chunks), U' A likewise (one chunk for m <= 4096:
// at the 4096 x 65536 size shorter chunks cut the initial scores' error from
// 4.8 to 3.2 u sqrt(m) but cost 2.8 ms).
constexpr int kSyrkChunkKb = 64;
constexpr int kSyrkMaxChunks = 32;
constexpr int kDotsChunkKb = 64;
int syrk_chunk_kb(int n) {
  const int kb = (n + BK - 1) / BK;
  return std::max(kSyrkChunkKb, (kb + kSyrkMaxChunks - 1) / kSyrkMaxChunks);
}
int syrk_chunks(int n) {
  const int kb = (n + BK - 1) / BK, c = syrk_chunk_kb(n);
  return (kb + c - 1) / c;
}
int dots_chunks(int m) { return ((m + BK - 1) / BK + kDotsChunkKb - 1) / kDotsChunkKb; }

// Scratch of css_f0: C (FP32, m x m), then one region used first for the
// K-chunk partial tiles of C and afterwards for U' in BF16 parts and
// the column-dot partials.
// FP32 input: A's BF16 parts, side by side, each padded to whole K blocks
// (part p, column j at Ap[(p * npad + j) * mpad + i], zero beyond m and n).
int f32_npad(int n) { return (n + BK - 1) / BK * BK; }

size_t css_f0_scratch_bytes(int m, int n, bool f32) {
  const int mpad = (m + 7) / 8 * 8;
  const int rpad = (m + 15) / 16 * 16;
  const int mtiles = (m + BM - 1) / BM;
  const size_t c = align_up((size_t)m * m * 4);
  const size_t chunks = align_up((size_t)syrk_chunks(n) * lower_tile_count(mtiles) * BM * 256 * 4);
  const size_t parts = align_up((size_t)mpad * kParts * rpad * 2);
  const size_t part = align_up((size_t)mtiles * dots_chunks(m) * n * 8);
  const size_t a_parts = f32 ? align_up((size_t)mpad * kParts * f32_npad(n) * 2) : 0;
  return c + std::max(chunks, parts + part) + a_parts;
}

cudaError_t css_f0(const void* A, long long lda, int m, int n, void* scratch, double* f, int* err,
                   unsigned long long spin_ns, cudaStream_t s, int stall, bool f32) {
  const int mpad = (m + 7) / 8 * 8;
  const int rpad = (m + 15) / 16 * 16;
  const int mtiles = (m + BM - 1) / BM;
  const int npad = f32_npad(n);
  float* C = (float*)scratch;
  float* chunk_tiles = (float*)((char*)scratch + align_up((size_t)m * m * 4));
  __nv_bfloat16* Cp = (__nv_bfloat16*)chunk_tiles;
  double* partial = (double*)((char*)Cp + align_up((size_t)mpad * kParts * rpad * 2));
  const int nchunk = syrk_chunks(n), ndots = dots_chunks(m);
  const int tiles_lower = lower_tile_count(mtiles);
  // FP32 A: its BF16 parts after the C / chunk / U' region (see css_f0_scratch_bytes)
  __nv_bfloat16* Ap = nullptr;
  if (f32) {
    const size_t c = align_up((size_t)m * m * 4);
    const size_t chunks = align_up((size_t)nchunk * tiles_lower * BM * 256 * 4);
    const size_t parts = align_up((size_t)mpad * kParts * rpad * 2);
    const size_t part = align_up((size_t)mtiles * ndots * n * 8);
    Ap = (__nv_bfloat16*)((char*)scratch + c + std::max(chunks, parts + part));
  }
  // the operand pairs of the FP32 path: (hi, hi), (hi, lo), (lo, hi); lo lo
  // is below 2^-32 of the product, under the FP32 accumulation's own rounding
  constexpr int kPairs = 3;
  const int kPairA[kPairs] = {0, 0, 1}, kPairB[kPairs] = {0, 1, 0};
  cudaError_t e;
  if (f32) {
    const long long tot = (long long)mpad * npad;
    split_parts_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>((const float*)A, lda, m, n, mpad, npad, Ap, 0);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  // C = A A^T: both operands are A, row-major in K (= the column index)
  {
    CUtensorMap ta;
    const bool ok = f32 ? make_map(&ta, Ap, (uint64_t)mpad, (uint64_t)kParts * npad, (uint64_t)mpad, BK)
                        : make_map(&ta, A, (uint64_t)m, (uint64_t)n, (uint64_t)lda, BK);
    if (!ok) return cudaErrorInvalidValue;
    Params P{};
    P.mode = 2;
    P.tri = 1;
    P.M = m;
    P.N = m;
    P.n_half = 256;
    P.halves = 1;
    P.n_tile = 256;
    P.kb_total = (n + BK - 1) / BK;
    P.kb_per_cta = P.kb_total;
    P.kb_chunk = syrk_chunk_kb(n);
    P.tiles_lower = tiles_lower;
    P.nparts = 1;
    if (f32) {
      // C = (A1 + A2)(A1 + A2)^T, the pairs of parts into one accumulator
      P.npairs = kPairs;
      for (int q = 0; q < kPairs; ++q) {
        P.pair_a[q] = kPairA[q];
        P.pair_b[q] = kPairB[q];
        P.pair_acc[q] = q > 0;
      }
      P.acc2_col = 256;
      P.a_kpart = npad;
      P.b_kpart = npad;
    }
    P.stage_bytes = BM * BK * 2 + 256 * BK * 2;
    P.stages = fit_stages(P.stage_bytes, STAGES);
    P.out = chunk_tiles;
    P.err = err;
    P.spin_ns = spin_ns;
    P.stall = stall;
    const size_t smem = smem_for(P.stage_bytes, P.stages);
    if ((e = cudaFuncSetAttribute(tc_kernel<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
      return e;
    dim3 grid(mtiles, (m + 255) / 256, nchunk);
    tc_kernel<true, true><<<grid, kThreads, smem, s>>>(ta, ta, P);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  // C = the chunks' sum, both triangles (the greedy iterations read whole rows)
  reduce_lower_kernel<<<dim3((m + 31) / 32, (m + 31) / 32), dim3(32, 8), 0, s>>>(chunk_tiles, nchunk,
                                                                                 tiles_lower, m, C);
  // U' (upper triangle of C, diagonal halved) = U1 + U2 in BF16
  {
    const long long tot = (long long)mpad * rpad;
    split_parts_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(C, m, m, m, mpad, rpad, Cp, 1);
  }
  // partial[M-tile][i] = sum over the tile's rows r of A[r, i] (U' A)[r, i];
  // U' is zero left of the diagonal, so M-tile J contracts over K >= 128 J only
  // (half of the products of C A)
  {
    CUtensorMap ta, tb;
    if (!make_map(&ta, Cp, (uint64_t)mpad, (uint64_t)(kParts * rpad), (uint64_t)mpad, BM)) return cudaErrorInvalidValue;
    const bool ok = f32 ? make_map(&tb, Ap, (uint64_t)mpad, (uint64_t)kParts * npad, (uint64_t)mpad, 256)
                        : make_map(&tb, A, (uint64_t)m, (uint64_t)n, (uint64_t)lda, 256);
    if (!ok) return cudaErrorInvalidValue;
    Params P{};
    P.mode = 3;
    P.tri = 1;
    P.M = m;
    P.N = n;
    P.n_half = 256;
    P.halves = f32 ? 1 : 2;
    P.n_tile = P.halves * 256;
    P.kb_total = (m + BK - 1) / BK;
    P.kb_per_cta = P.kb_total;
    P.kb_chunk = kDotsChunkKb;
    P.a_part_stride = rpad;
    if (f32) {
      // one stage per (K block, pair), 256 columns per CTA (the cross
      // products take the other half of TMEM): 48 KB per stage
      P.group = 0;
      P.nparts = 1;
      P.npairs = kPairs;
      for (int q = 0; q < kPairs; ++q) {
        P.pair_a[q] = kPairA[q];
        P.pair_b[q] = kPairB[q];
        P.pair_acc[q] = q > 0;
      }
      P.acc2_col = 256;
      P.b_part_stride = npad;
      P.stage_bytes = BM * BK * 2 + 256 * BK * 2;
      P.stages = fit_stages(P.stage_bytes, STAGES);
    } else {
      // 512 columns per CTA (two MMAs of N = 256, the whole TMEM) and one
      // stage per K block holding the U' parts and the single shared A tile:
      // 96 KB per stage
      P.group = 1;
      P.nparts = kParts;
      P.b_part_stride = 0;
      P.stage_bytes = kParts * BM * BK * 2 + 512 * BK * 2;
      P.stages = 2;
    }
    P.f = partial;
    P.Acol = A;
    P.acol_f32 = f32 ? 1 : 0;
    P.lda_col = lda;
    P.err = err;
    P.spin_ns = spin_ns;
    P.stall = stall;
    const size_t smem = smem_for(P.stage_bytes, P.stages);
    if ((e = cudaFuncSetAttribute(tc_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
      return e;
    dim3 grid(mtiles, (n + P.n_tile - 1) / P.n_tile, ndots);
    tc_kernel<false, false><<<grid, kThreads, smem, s>>>(ta, tb, P);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  // f_i = a_i^T C a_i = 2 a_i^T U' a_i
  sum_rows_kernel<<<(n + 255) / 256, 256, 0, s>>>(partial, mtiles * ndots, n, f, 2.0);
  return cudaGetLastError();
}

bool supported_any() { return encode_fn() != nullptr; }

}  // namespace tc
}  // namespace css
