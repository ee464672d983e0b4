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
//                is split into three BF16 parts (all 24 bits) that accumulate
//                into the same TMEM tile; the epilogue sums squares of each
//                row in FP64.
//   initial CSS scores (css_f0): C = A A^T, U' = its upper triangle in
//                three BF16 parts, and the column dots of A with U' A.
//
// The number of parts of an FP32 operand: two (16 bits) leave every entry
// with a relative error of 2^-17.  That hardly moves the initial scores (f0
// within 2.9 u sqrt(m) of the oracle's at 2048 x 65536 for the norms) but
// moves the late, small scores: on small problems with k close to the rank
// the final errors were 5-25 (GCSS) and 20-80 (CSS) times the oracle's, and
// 0.8-1.05 with three parts.
//
// One CTA = 6 warps: warp 0 lane 0 issues TMA loads into a shared
// memory ring (128-byte swizzle), warp 1 owns the TMEM allocation and its lane
// 0 issues tcgen05.mma (BF16 x BF16 -> FP32, M = 128, up to two MMAs of
// N <= 256 side by side in TMEM), warps 2-5 read the accumulator back with
// tcgen05.ld (each warp its 32-lane quarter of TMEM).  Every mbarrier wait is
// bounded; on expiry an error flag is set and the CTA tears down.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <vector>

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
constexpr int kTmemCols = 512;   // TMEM columns a CTA takes unless Params::tmem_cols says fewer
// The initial-score GEMMs of BF16 A take 256 TMEM columns and two 48 KB ring
// stages per CTA, so that two CTAs share an SM and one's epilogue overlaps
// the other's MMAs (instead of 512 columns and 96-112 KB stages, one CTA per SM)
constexpr bool kSyrk2Cta = true;
constexpr bool kDots2Cta = true;
// FP32 A's column-dot GEMM: columns per CTA (its two accumulators take
// twice that of TMEM; 128 lets two CTAs share an SM)
constexpr int kDotsF32Cols = 128;
// BF16 parts of an FP32 operand (B of the GCSS norms, U' of the CSS scores,
// FP32 A): three, all 24 bits of it (see the top of the file).
constexpr int kParts = 3;

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
  int acol_vec;      // Acol and lda_col allow 16-byte loads
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
  int pair_a[8];
  int pair_b[8];
  int a_kpart;
  int b_kpart;
  // pair q accumulates into TMEM columns acc2_col * pair_acc[q] onwards.
  // The tensor cores' accumulation truncates by up to one unit of the
  // running sum per MMA, so the small cross products (hi lo, lo hi) go to a
  // second accumulator whose sum, and so its truncation, is 2^8 smaller; the
  // epilogue adds the two.  acc2_col = 0: one accumulator.
  int pair_acc[8];
  int acc2_col;
  int bz_off;        // added to blockIdx.z (a launch of some of the K chunks)
  int tmem_cols;     // TMEM columns to allocate (0: kTmemCols); a power of 2 >= 32
};

}  // namespace

// One problem of a group (see group_f0_prepare).  Tensor maps first: they
// must sit on 64-byte boundaries in device memory.
struct GroupProb {
  CUtensorMap mapA2;   // C = A A^T: A (or its parts), box {64, BK}
  CUtensorMap mapU;    // U' parts, box {64, BM}
  CUtensorMap mapA3;   // column dots: A (or its parts), box {64, 256}
  Params p2, p3;       // the two GEMMs (f0_params_syrk, f0_params_dots)
  const void* A;
  long long lda;
  int m, n, mpad, npad, rpad, src;   // src: F0Source
  long long ldc;                      // C's leading dimension
  int nchunk, ndots, mtiles, tiles_lower, tw;
  float* C;
  float* chunk_tiles;
  __nv_bfloat16* Cp;
  __nv_bfloat16* Ap;
  float* Acopy;
  double* partial;
  double* f;
};
// One CTA of a grouped GEMM launch: problem, row tile, column tile, K chunk.
struct GroupTile {
  int prob, bx, by, bz;
};

namespace {

// Mode 2 tiles (BM rows x tw columns, tw = 256 or 128) that touch the lower
// triangle: tile (bx, by) does when bx * 128 + 127 >= by * tw, i.e. by <= bx
// / 2 (tw = 256) or by <= bx (tw = 128).  Their index in row-tile order.
__host__ __device__ __forceinline__ int lower_tile_index(int bx, int by, int tw) {
  if (tw == 128) return bx * (bx + 1) / 2 + by;
  // sum over b < bx of (b / 2 + 1)
  const int q = bx / 2;
  const int before = bx + ((bx & 1) ? q * q : q * (q - 1));
  return before + by;
}
__host__ __device__ __forceinline__ int lower_tile_count(int mtiles, int tw) {
  return lower_tile_index(mtiles, 0, tw);
}

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

// One CTA's tile: rows bx * BM.., column tile by (modes 2, 3) or K slice by
// (mode 0), K chunk bz of gz.  The tensor maps are generic addresses (kernel
// parameters, or global memory for a group of problems).
template <bool A_MN, bool B_MN>
__device__ __forceinline__ void tc_body(const Params& P, const CUtensorMap* mapA, const CUtensorMap* mapB,
                                        int bx, int by, int bz, int gz) {
  const CUtensorMap& tmA = *mapA;
  const CUtensorMap& tmB = *mapB;
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
  const uint32_t tcols = P.tmem_cols ? (uint32_t)P.tmem_cols : (uint32_t)kTmemCols;
  // work of this CTA
  const int tile0 = bx * BM;
  int kb_begin = 0, kb_end = P.kb_total;
  int ntile0 = 0;
  if (P.mode == 0) {
    kb_begin = by * P.kb_per_cta;
    kb_end = min(P.kb_total, kb_begin + P.kb_per_cta);
  } else if (P.mode >= 2) {
    ntile0 = by * P.n_tile;
    kb_begin = bz * P.kb_chunk;
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
        if (c < P.N) P.f[((long long)bx * gz + bz) * P.N + c] = 0.0;
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
                 "r"(tcols)
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
        for (int j = 0; j < P.N; ++j) P.out[(long long)by * P.M * P.N + (long long)j * P.M + row] = 0.f;
      if (P.mode == 1 && row < P.M) P.f[row] = 0.0;
    } else if (ok && P.mode == 3) {
      // column dots: partial[M-tile][c] = sum over this tile's rows r of
      // Acol[r, c] * D[r, c]; rows are TMEM lanes, so each 16-column chunk is
      // reduced across the warp (transpose reduction) and then across warps
      // (products exact as hi + lo, sums in double-float, one FP64 add per
      // column at the end)
      __shared__ float2 cred[4][16];
      const int ncols = P.halves * P.n_half;
      // this tile of Acol (BM rows x ncols columns in its own type,
      // column-major, zero outside the matrix) into the ring, which every MMA
      // has finished reading: a few batches of independent coalesced loads
      // instead of a dependent round trip per 16-column chunk
      float* sacol_f = reinterpret_cast<float*>(smem);
      __nv_bfloat16* sacol_b = reinterpret_cast<__nv_bfloat16*>(smem);
      {
        const int et = threadIdx.x - 64;   // 0..127 over the epilogue warps
        const int esz = P.acol_f32 ? 4 : 2;
        if (P.acol_vec) {
          // 16-byte vectors; a column's last partial vector element by element
          // (nothing past row M is read)
          const int epv = 16 / esz, vpc = BM / epv;
          const char* base = reinterpret_cast<const char*>(P.Acol);
          uint4* sv = reinterpret_cast<uint4*>(smem);
#pragma unroll 16
          for (int idx = et; idx < ncols * vpc; idx += 128) {
            const int j = idx / vpc, vv = idx - j * vpc;
            const int c = ntile0 + j, rw = tile0 + vv * epv;
            uint4 val = make_uint4(0u, 0u, 0u, 0u);
            if (c < P.N && rw < P.M) {
              const char* src = base + ((long long)c * P.lda_col + rw) * esz;
              if (rw + epv <= P.M) {
                val = __ldg(reinterpret_cast<const uint4*>(src));
              } else {
                uint32_t w[4] = {0u, 0u, 0u, 0u};
                for (int e = 0; rw + e < P.M; ++e) {
                  const uint32_t x = esz == 4 ? reinterpret_cast<const uint32_t*>(src)[e]
                                              : (uint32_t)reinterpret_cast<const unsigned short*>(src)[e];
                  w[e * esz / 4] |= x << ((e * esz * 8) & 31);
                }
                val = make_uint4(w[0], w[1], w[2], w[3]);
              }
            }
            sv[idx] = val;
          }
        } else if (P.acol_f32) {
          const float* Ac = reinterpret_cast<const float*>(P.Acol);
#pragma unroll 16
          for (int idx = et; idx < ncols * BM; idx += 128) {
            const int j = idx / BM, rr = idx - j * BM;
            const int c = ntile0 + j, rw = tile0 + rr;
            sacol_f[idx] = (rw < P.M && c < P.N) ? __ldg(Ac + (long long)c * P.lda_col + rw) : 0.f;
          }
        } else {
          const __nv_bfloat16* Ab = reinterpret_cast<const __nv_bfloat16*>(P.Acol);
#pragma unroll 16
          for (int idx = et; idx < ncols * BM; idx += 128) {
            const int j = idx / BM, rr = idx - j * BM;
            const int c = ntile0 + j, rw = tile0 + rr;
            sacol_b[idx] = (rw < P.M && c < P.N) ? Ab[(long long)c * P.lda_col + rw] : __float2bfloat16_rn(0.f);
          }
        }
        asm volatile("bar.sync 1, 128;" ::: "memory");
      }
      for (int j0 = 0; j0 < ncols; j0 += 16) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)j0, v);
        add_acc2(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(P.acc2_col + j0), P.acc2_col, v);
        float ph[16], pl[16];
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) {
          // zero outside the matrix (see the staging above)
          const int si = (j0 + jj) * BM + q * 32 + lane;
          const float a = P.acol_f32 ? sacol_f[si] : __bfloat162float(sacol_b[si]);
          ph[jj] = a * v[jj];
          pl[jj] = fmaf(a, v[jj], -ph[jj]);
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
            P.f[((long long)bx * gz + bz) * P.N + c] = to_f64(h) + to_f64(l);
          }
        }
        asm volatile("bar.sync 1, 128;" ::: "memory");
      }
    } else if (ok) {
      float sh = 0.f, sl = 0.f;   // mode 1: sum of squares in double-float
      float* tile_out = nullptr;
      if (P.mode == 2)
        tile_out = P.out + ((long long)bz * P.tiles_lower + lower_tile_index(bx, by, P.n_tile)) *
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
                P.out[(long long)by * P.M * P.N + (long long)j * P.M + row] = v[jj];
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
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols)
                 : "memory");
  }
}

template <bool A_MN, bool B_MN>
__global__ void __launch_bounds__(kThreads, 1)
    tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
              const __grid_constant__ Params P) {
  tc_body<A_MN, B_MN>(P, &tmA, &tmB, blockIdx.x, blockIdx.y, blockIdx.z + P.bz_off, gridDim.z + P.bz_off);
}

// B (FP32, m x r, ldb) -> np BF16 parts B1 + B2 (+ B3) (m x rpad each, ld
// mpad), laid out side by side: part p, column j at Bp[(p * rpad + j) * mpad + i].
// tri: B is the symmetric C with only its lower triangle valid, and the parts
// hold U' (column j, row i: C[i, j] for i > j, C[j, j] / 2 on the diagonal,
// 0 above), so that a_i^T C a_i = 2 a_i^T U' a_i.
__device__ __forceinline__ void split_one(const float* __restrict__ B, long long ldb, int m, int r, int mpad,
                                          int rpad, __nv_bfloat16* __restrict__ Bp, int tri, int np,
                                          long long idx) {
  const int i = (int)(idx % mpad), j = (int)(idx / mpad);
  float v = (i < m && j < r && (!tri || i >= j)) ? B[(long long)j * ldb + i] : 0.f;
  if (tri && i == j) v *= 0.5f;
#pragma unroll 3
  for (int p = 0; p < np; ++p) {
    const __nv_bfloat16 b = __float2bfloat16_rn(v);
    v -= __bfloat162float(b);
    Bp[(long long)(p * rpad + j) * mpad + i] = b;
  }
}
__global__ void split_parts_kernel(const float* __restrict__ B, long long ldb, int m, int r, int mpad,
                                   int rpad, __nv_bfloat16* __restrict__ Bp, int tri, int np) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < (long long)mpad * rpad) split_one(B, ldb, m, r, mpad, rpad, Bp, tri, np, idx);
}

// BF16 A (m x n, any leading dimension) -> an exact copy with leading
// dimension mpad, zero beyond m (element idx of mpad x npad).
__device__ __forceinline__ void stage_one(const __nv_bfloat16* __restrict__ A, long long lda, int m, int n,
                                          int mpad, __nv_bfloat16* __restrict__ Ap, long long idx) {
  const int i = (int)(idx % mpad), j = (int)(idx / mpad);
  Ap[idx] = (i < m && j < n) ? A[(long long)j * lda + i] : __float2bfloat16_rn(0.f);
}
__global__ void stage_kernel(const __nv_bfloat16* __restrict__ A, long long lda, int m, int n, int mpad, int npad,
                             __nv_bfloat16* __restrict__ Ap) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < (long long)mpad * npad) stage_one(A, lda, m, n, mpad, Ap, idx);
}
// FP32 A (any leading dimension) -> an exact copy with leading dimension
// mpad, zero beyond m (element idx of mpad x n).
__device__ __forceinline__ void stage_f32_one(const float* __restrict__ A, long long lda, int m, int mpad,
                                              float* __restrict__ Ac, long long idx) {
  const int i = (int)(idx % mpad), j = (int)(idx / mpad);
  Ac[idx] = i < m ? A[(long long)j * lda + i] : 0.f;
}
__global__ void stage_f32_kernel(const float* __restrict__ A, long long lda, int m, int n, int mpad,
                                 float* __restrict__ Ac) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < (long long)mpad * n) stage_f32_one(A, lda, m, mpad, Ac, idx);
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
  split_parts_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(B, ldb, m, r, mpad, rpad, Bp, 0, kParts);
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

namespace {

__device__ __forceinline__ double sum_row(const double* __restrict__ partial, int nblk, int n, int i) {
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += partial[(long long)b * n + i];
  return s;
}
__global__ void sum_rows_kernel(const double* __restrict__ partial, int nblk, int n,
                                double* __restrict__ out, double scale) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = scale * sum_row(partial, nblk, n, i);
}

// C = sum over the K chunks of their partial tiles (compensated sums in
// chunk order, rounded once to FP32), written to both triangles of C (ld ldc)
// through 32 x 32 shared-memory tiles, so reads and writes are coalesced.
// Only the 32 x 32 tiles on or below the diagonal run (bi >= bj); each lies
// inside one chunk tile of 128 x 256.  Block-wide (32 x 8 threads).
__device__ __forceinline__ void reduce_lower_block(const float* __restrict__ parts, int chunks, int tiles_lower,
                                                   int tw, int m, long long ldc, float* __restrict__ C, int bi,
                                                   int bj, float (&tile)[32][33]) {
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int r = bi * 32 + tx;
  const int bx = (bi * 32) / BM, by = (bj * 32) / tw;
  const long long chunk_stride = (long long)tiles_lower * BM * tw;
  const float* src = parts + (long long)lower_tile_index(bx, by, tw) * BM * tw;
  for (int k = ty; k < 32; k += blockDim.y) {
    const int c = bj * 32 + k;
    float v = 0.f;
    if (r < m && c < m && r >= c) {
      const long long local = (long long)(c - by * tw) * BM + (r - bx * BM);
      // compensated FP32 sum (TwoSum): within a unit of the exact sum
      // before the final rounding, like an FP64 sum, at FP32 rates (FP64
      // additions, at two per clock per SM, made this kernel their bound)
      float sh = 0.f, sl = 0.f;
      for (int z = 0; z < chunks; ++z) {
        float s_, e_;
        df_two_sum(sh, src[z * chunk_stride + local], s_, e_);
        sh = s_;
        sl += e_;
      }
      v = sh + sl;
      C[(long long)c * ldc + r] = v;
    }
    tile[k][tx] = v;
  }
  __syncthreads();
  // C[c, r] = C[r, c] for r > c
  for (int k = ty; k < 32; k += blockDim.y) {
    const int c = bj * 32 + tx, r2 = bi * 32 + k;
    if (r2 < m && c < m && r2 > c) C[(long long)r2 * ldc + c] = tile[tx][k];
  }
  __syncthreads();   // the tile is free for the block's next use
}
__global__ void reduce_lower_kernel(const float* __restrict__ parts, int chunks, int tiles_lower, int tw, int m,
                                    long long ldc, float* __restrict__ C) {
  __shared__ float tile[32][33];
  if (blockIdx.x < blockIdx.y) return;
  reduce_lower_block(parts, chunks, tiles_lower, tw, m, ldc, C, blockIdx.x, blockIdx.y, tile);
}

// K chunking of the initial-score GEMMs (see Params::kb_chunk).  A TMEM sum
// of L products is biased by about L / 32 units of its last place (one
// truncation per MMA of K = 16, half a unit on average), a bias that C
// passes on to every initial score; the round-to-nearest FMAs of a SIMT dot
// product err by about sqrt(m) units.  So C = A A^T is summed in chunks of
// about 64 sqrt(m) products (4 to 64 K blocks of 64: 2 sqrt(m) units), at
// most 32 chunks (very wide A gets longer ones), added with compensated
// FP32 sums.  U' A likewise, in chunks of 2048 (at 4096 x 65536: f0 within
// 4.2 u sqrt(m) of the oracle's instead of 5.5 for 0.33 ms more, and the
// selection then agrees with the oracle's at every iteration; chunks of
// 1024: 3.5 u sqrt(m), 1.2 ms more).
constexpr int kSyrkMaxChunks = 32;
constexpr int kDotsChunkKb = 32;
int syrk_chunk_kb(int m, int n) {
  const int kb = (n + BK - 1) / BK;
  int c = 4;
  while (c < 64 && (c + 1) * (c + 1) <= m) ++c;   // floor(sqrt(m)), in [4, 64]
  return std::max(c, (kb + kSyrkMaxChunks - 1) / kSyrkMaxChunks);
}
int syrk_chunks(int m, int n) {
  const int kb = (n + BK - 1) / BK, c = syrk_chunk_kb(m, n);
  return (kb + c - 1) / c;
}
int dots_chunks(int m) { return ((m + BK - 1) / BK + kDotsChunkKb - 1) / kDotsChunkKb; }

// Scratch of css_f0: C (FP32, m x m, leading dimension c_ld(m, 4)), then
// one region used first for the
// K-chunk partial tiles of C and afterwards for U' in BF16 parts and
// the column-dot partials.
// Then, unless A feeds the TMA path in place: A's BF16 parts (FP32 input:
// two; BF16 input with a layout TMA refuses: one, an exact copy), side by
// side, each padded to whole K blocks (part p, column j at
// Ap[(p * npad + j) * mpad + i], zero beyond m and n).
// Columns per tile of C = A A^T: FP32 A (two accumulators for its part
// pairs) takes 128 so that the two fit in 256 TMEM columns and two CTAs
// share an SM; BF16 takes 256.
constexpr int kSyrkF32Cols = 128;
int syrk_tile_cols(bool f32) { return f32 ? kSyrkF32Cols : 256; }

struct F0Layout {
  int mpad, rpad, npad, mtiles, nchunk, ndots, tiles_lower;
  int tw;          // columns of C = A A^T per tile (syrk_tile_cols)
  long long ldc;   // C's leading dimension (c_ld)
  size_t bytes;
  float* C;
  float* chunk_tiles;
  __nv_bfloat16* Cp;
  double* partial;
  __nv_bfloat16* Ap;
  float* Acopy;
};
bool is_f32(int src) { return src == kF0F32 || src == kF0F32Staged; }
int a_parts(int src) { return is_f32(src) ? kParts : src == kF0Bf16Staged ? 1 : 0; }

F0Layout f0_layout(int m, int n, int src, void* scratch) {
  F0Layout L{};
  L.mpad = (m + 7) / 8 * 8;
  L.rpad = (m + 15) / 16 * 16;
  L.npad = (n + BK - 1) / BK * BK;
  L.mtiles = (m + BM - 1) / BM;
  L.nchunk = syrk_chunks(m, n);
  L.ndots = dots_chunks(m);
  L.tw = syrk_tile_cols(is_f32(src));
  L.tiles_lower = lower_tile_count(L.mtiles, L.tw);
  L.ldc = c_ld(m, 4);
  const size_t c = align_up((size_t)m * L.ldc * 4);
  const size_t chunks = align_up((size_t)L.nchunk * L.tiles_lower * BM * L.tw * 4);
  const size_t parts = align_up((size_t)L.mpad * kParts * L.rpad * 2);
  const size_t part = align_up((size_t)L.mtiles * L.ndots * n * 8);
  const size_t ap = align_up((size_t)L.mpad * a_parts(src) * L.npad * 2);
  // kF0F32Staged: an FP32 copy of A with leading dimension mpad after the parts
  const size_t acopy = src == kF0F32Staged ? align_up((size_t)L.mpad * n * 4) : 0;
  L.bytes = c + std::max(chunks, parts + part) + ap + acopy;
  char* b = (char*)scratch;
  L.C = (float*)b;
  L.chunk_tiles = (float*)(b + c);
  L.Cp = (__nv_bfloat16*)(b + c);
  L.partial = (double*)(b + c + parts);
  L.Ap = src != kF0Bf16 ? (__nv_bfloat16*)(b + c + std::max(chunks, parts + part)) : nullptr;
  L.Acopy = src == kF0F32Staged ? (float*)(b + c + std::max(chunks, parts + part) + ap) : nullptr;
  return L;
}

// the operand pairs of FP32 A (parts 0, 1, 2 of 8 bits each): every pair
// whose product is at least 2^-16 of the leading one; the three dropped
// pairs are near 2^-24 of it, the FP32 accumulation's own rounding.  The
// cross products accumulate apart (Params::pair_acc).
constexpr int kPairs = 6;
constexpr int kPairA[kPairs] = {0, 0, 1, 0, 1, 2}, kPairB[kPairs] = {0, 1, 0, 2, 1, 0};
void set_pairs(Params& P) {
  P.npairs = kPairs;
  for (int q = 0; q < kPairs; ++q) {
    P.pair_a[q] = kPairA[q];
    P.pair_b[q] = kPairB[q];
    P.pair_acc[q] = q > 0;
  }
  P.acc2_col = 256;
}

// Columns of D per CTA of the column-dot GEMM.
int dots_n_tile(bool f32) { return f32 ? kDotsF32Cols : kDots2Cta ? 256 : 512; }

// Tensor maps of the two GEMMs: C = A A^T (both operands A, or its parts,
// row-major in K = the column index), and U' A (U' parts K-major; A, or its
// parts, K-major in the rows).
bool f0_maps(const F0Layout& L, const void* A, long long lda, int m, int n, int src, CUtensorMap* mA2,
             CUtensorMap* mU, CUtensorMap* mA3) {
  if (src != kF0Bf16) {
    const uint64_t cols = (uint64_t)a_parts(src) * L.npad;
    if (!make_map(mA2, L.Ap, (uint64_t)L.mpad, cols, (uint64_t)L.mpad, BK)) return false;
    if (!make_map(mA3, L.Ap, (uint64_t)L.mpad, cols, (uint64_t)L.mpad, (uint32_t)std::min(256, dots_n_tile(is_f32(src)))))
      return false;
  } else {
    if (!make_map(mA2, A, (uint64_t)m, (uint64_t)n, (uint64_t)lda, BK)) return false;
    if (!make_map(mA3, A, (uint64_t)m, (uint64_t)n, (uint64_t)lda, 256)) return false;
  }
  return make_map(mU, L.Cp, (uint64_t)L.mpad, (uint64_t)(kParts * L.rpad), (uint64_t)L.mpad, BM);
}

// C = A A^T: the tiles touching the lower triangle, grid (mtiles, ceil(m /
// 256), nchunk), chunk partial tiles to L.chunk_tiles
Params f0_params_syrk(const F0Layout& L, int m, int n, int src, int* err, unsigned long long spin_ns,
                      int stall) {
  const bool f32 = is_f32(src);
  Params P{};
  P.mode = 2;
  P.tri = 1;
  P.M = m;
  P.N = m;
  P.n_half = L.tw;
  P.halves = 1;
  P.n_tile = L.tw;
  P.kb_total = (n + BK - 1) / BK;
  P.kb_per_cta = P.kb_total;
  P.kb_chunk = syrk_chunk_kb(m, n);
  P.tiles_lower = L.tiles_lower;
  P.nparts = 1;
  if (f32) {
    // C = (A1 + A2 + A3)(A1 + A2 + A3)^T: one ring stage per (K block, pair)
    set_pairs(P);
    P.acc2_col = L.tw;
    P.a_kpart = L.npad;
    P.b_kpart = L.npad;
  }
  P.stage_bytes = BM * BK * 2 + L.tw * BK * 2;
  P.stages = fit_stages(P.stage_bytes, STAGES);
  if (kSyrk2Cta && !f32) {
    P.stages = 2;
    P.tmem_cols = 256;
  }
  if (f32 && L.tw == 128) {
    // two accumulators of 128 columns: 256 TMEM columns, three 32 KB stages
    P.stages = 3;
    P.tmem_cols = 256;
  }
  P.out = L.chunk_tiles;
  P.err = err;
  P.spin_ns = spin_ns;
  P.stall = stall;
  return P;
}

// partial[M-tile][i] = sum over the tile's rows r of A[r, i] (U' A)[r, i];
// U' is zero left of the diagonal, so M-tile J contracts over K >= 128 J only
// (half of the products of C A).  Grid (mtiles, ceil(n / n_tile), ndots).
Params f0_params_dots(const F0Layout& L, const void* A, long long lda, int m, int n, int src, int* err,
                      unsigned long long spin_ns, int stall) {
  const bool f32 = is_f32(src);
  Params P{};
  P.mode = 3;
  P.tri = 1;
  P.M = m;
  P.N = n;
  P.n_half = std::min(256, dots_n_tile(f32));
  P.halves = dots_n_tile(f32) / P.n_half;
  P.n_tile = P.halves * P.n_half;
  P.kb_total = (m + BK - 1) / BK;
  P.kb_per_cta = P.kb_total;
  P.kb_chunk = kDotsChunkKb;
  P.a_part_stride = L.rpad;
  if (f32) {
    // U' parts times A parts, one stage per (K block, pair), 256 columns
    // per CTA (the cross products take the other half of TMEM): 48 KB per
    // stage
    P.group = 0;
    P.nparts = 1;
    set_pairs(P);
    P.acc2_col = P.n_tile;
    P.tmem_cols = 2 * P.n_tile;
    P.b_part_stride = L.npad;
    P.stage_bytes = BM * BK * 2 + P.n_tile * BK * 2;
    P.stages = P.n_tile < 256 ? 3 : fit_stages(P.stage_bytes, STAGES);
  } else if (kDots2Cta) {
    // 256 columns per CTA, one stage per (K block, U' part) holding that
    // part's tile and the A tile (48 KB), two stages: two CTAs per SM
    P.group = 0;
    P.nparts = kParts;
    P.b_part_stride = 0;
    P.stage_bytes = BM * BK * 2 + 256 * BK * 2;
    P.stages = 2;
    P.tmem_cols = 256;
  } else {
    // 512 columns per CTA (two MMAs of N = 256, the whole TMEM) and one
    // stage per K block holding the U' parts and the single shared A tile:
    // 112 KB per stage
    P.group = 1;
    P.nparts = kParts;
    P.b_part_stride = 0;
    P.stage_bytes = kParts * BM * BK * 2 + 512 * BK * 2;
    P.stages = 2;
  }
  // the epilogue stages the tile's Acol (BM x n_tile, BF16 or FP32) in the ring
  static_assert(BM * 512 * 2 <= 2 * (kParts * BM * BK * 2 + 512 * BK * 2), "BF16 ring holds the Acol tile");
  static_assert(2 * (kParts * BM * BK * 2 + 512 * BK * 2) + 256 + 1024 <= kSmemMax, "BF16 ring fits");
  static_assert(BM * 256 * 4 <= 3 * (BM * BK * 2 + 256 * BK * 2), "FP32 ring holds the Acol tile");
  static_assert(BM * 256 * 2 <= 2 * (BM * BK * 2 + 256 * BK * 2), "two-stage BF16 ring holds the Acol tile");
  P.f = L.partial;
  // the outer factor a_i of the column dots: A itself, or its aligned copy
  // (same values) when one is made, so that the epilogue's staging takes
  // 16-byte loads
  const void* Ac = src == kF0Bf16Staged ? (const void*)L.Ap : src == kF0F32Staged ? (const void*)L.Acopy : A;
  const long long ldac = Ac == A ? lda : L.mpad;
  P.Acol = Ac;
  P.acol_f32 = f32 ? 1 : 0;
  P.acol_vec = ((uintptr_t)Ac % 16 == 0 && (ldac * (f32 ? 4 : 2)) % 16 == 0) ? 1 : 0;
  P.lda_col = ldac;
  P.err = err;
  P.spin_ns = spin_ns;
  P.stall = stall;
  return P;
}

template <bool A_MN, bool B_MN>
cudaError_t set_smem(const Params& P) {
  cudaError_t e = cudaFuncSetAttribute(tc_kernel<A_MN, B_MN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem_for(P.stage_bytes, P.stages));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(tc_kernel<A_MN, B_MN>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  return e;
}

// ------------------------------------------------------ groups of problems -
// The initial scores of many independent problems (a batch) in one launch
// per phase.  Every problem's descriptors and tensor maps sit in device
// memory; a CTA of the GEMM phases takes one entry of a tile list, a block of
// the elementwise phases takes problem blockIdx.y.
constexpr int kGroupBlocks = 32;   // blocks per problem in the elementwise phases

__global__ void group_split_kernel(const GroupProb* __restrict__ probs, int which) {
  const GroupProb& g = probs[blockIdx.y];
  // which 0: A -> its parts (FP32) or its aligned copy (BF16 staged); 1: C -> U' parts
  if (which == 0 && g.src == kF0Bf16) return;
  if (which == 0 && g.src == kF0F32Staged) {
    const long long tot = (long long)g.mpad * g.n;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < tot;
         idx += (long long)gridDim.x * blockDim.x)
      stage_f32_one((const float*)g.A, g.lda, g.m, g.mpad, g.Acopy, idx);
  }
  if (which == 0 && g.src == kF0Bf16Staged) {
    const long long tot = (long long)g.mpad * g.npad;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < tot;
         idx += (long long)gridDim.x * blockDim.x)
      stage_one((const __nv_bfloat16*)g.A, g.lda, g.m, g.n, g.mpad, g.Ap, idx);
    return;
  }
  const float* B = which ? g.C : (const float*)g.A;
  const long long ldb = which ? g.ldc : g.lda;
  const int r = which ? g.m : g.n, cols = which ? g.rpad : g.npad;
  __nv_bfloat16* out = which ? g.Cp : g.Ap;
  const long long tot = (long long)g.mpad * cols;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < tot;
       idx += (long long)gridDim.x * blockDim.x)
    split_one(B, ldb, g.m, r, g.mpad, cols, out, which, kParts, idx);
}

__global__ void group_reduce_kernel(const GroupProb* __restrict__ probs) {
  __shared__ float tile[32][33];
  const GroupProb& g = probs[blockIdx.y];
  const int nb = (g.m + 31) / 32;
  for (int q = blockIdx.x; q < nb * nb; q += gridDim.x) {
    const int bi = q % nb, bj = q / nb;
    if (bi >= bj) reduce_lower_block(g.chunk_tiles, g.nchunk, g.tiles_lower, g.tw, g.m, g.ldc, g.C, bi, bj, tile);
  }
}

__global__ void group_sum_rows_kernel(const GroupProb* __restrict__ probs) {
  const GroupProb& g = probs[blockIdx.y];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.n; i += gridDim.x * blockDim.x)
    g.f[i] = 2.0 * sum_row(g.partial, g.mtiles * g.ndots, g.n, i);
}

template <bool A_MN, bool B_MN>
__global__ void __launch_bounds__(kThreads, 1)
    tc_group_kernel(const GroupProb* __restrict__ probs, const GroupTile* __restrict__ tiles, int mode) {
  const GroupTile w = tiles[blockIdx.x];
  const GroupProb& g = probs[w.prob];
  const Params P = mode == 2 ? g.p2 : g.p3;
  const CUtensorMap* mA = mode == 2 ? &g.mapA2 : &g.mapU;
  const CUtensorMap* mB = mode == 2 ? &g.mapA2 : &g.mapA3;
  if (threadIdx.x == 0) {
    // the maps were written to global memory by a copy before the launch
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"((uint64_t)mA) : "memory");
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"((uint64_t)mB) : "memory");
  }
  tc_body<A_MN, B_MN>(P, mA, mB, w.bx, w.by, w.bz, mode == 2 ? g.nchunk : g.ndots);
}

}  // namespace

size_t css_f0_scratch_bytes(int m, int n, int src) { return f0_layout(m, n, src, nullptr).bytes; }

bool f0_staged_copy(int m, int n, int src, void* scratch, const void** A, long long* lda) {
  if (src != kF0Bf16Staged && src != kF0F32Staged) return false;
  const F0Layout L = f0_layout(m, n, src, scratch);
  *A = src == kF0F32Staged ? (const void*)L.Acopy : (const void*)L.Ap;
  *lda = L.mpad;
  return true;
}

int f0_source(bool f32, const void* A, long long lda, int m) {
  const bool aligned = ((uintptr_t)A & 15u) == 0 && (lda * (f32 ? 4 : 2)) % 16 == 0;
  if (f32) return aligned ? kF0F32 : kF0F32Staged;
  return supported(A, lda, m, 256) ? kF0Bf16 : kF0Bf16Staged;
}

int f0_chunk_cols(int m, int n) { return syrk_chunk_kb(m, n) * BK; }

cudaError_t css_f0(const void* A, long long lda, int m, int n, void* scratch, double* f, int* err,
                   unsigned long long spin_ns, cudaStream_t s, int stall, int src, const F0Pipe* pipe) {
  const F0Layout L = f0_layout(m, n, src, scratch);
  CUtensorMap mA2, mU, mA3;
  if (!f0_maps(L, A, lda, m, n, src, &mA2, &mU, &mA3)) return cudaErrorInvalidValue;
  cudaError_t e;
  // chunks of A arriving: per K chunk of C = A A^T, or all before anything
  const bool per_chunk = pipe && src == kF0Bf16 && pipe->cols == f0_chunk_cols(m, n) && pipe->chunks == L.nchunk;
  if (pipe && !per_chunk)
    for (int z = 0; z < pipe->chunks; ++z)
      if ((e = cudaStreamWaitEvent(s, pipe->ready[z], 0)) != cudaSuccess) return e;
  if (src != kF0Bf16) {
    const long long tot = (long long)L.mpad * L.npad;
    if (src == kF0F32Staged)
      stage_f32_kernel<<<(unsigned)(((long long)L.mpad * n + 255) / 256), 256, 0, s>>>((const float*)A, lda, m, n,
                                                                                      L.mpad, L.Acopy);
    if (is_f32(src))
      split_parts_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>((const float*)A, lda, m, n, L.mpad,
                                                                         L.npad, L.Ap, 0, kParts);
    else
      stage_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>((const __nv_bfloat16*)A, lda, m, n, L.mpad,
                                                                   L.npad, L.Ap);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  const Params P2 = f0_params_syrk(L, m, n, src, err, spin_ns, stall);
  if ((e = set_smem<true, true>(P2)) != cudaSuccess) return e;
  if (per_chunk) {
    // one launch per K chunk, each after its columns have arrived
    for (int z = 0; z < L.nchunk; ++z) {
      if ((e = cudaStreamWaitEvent(s, pipe->ready[z], 0)) != cudaSuccess) return e;
      Params Pz = P2;
      Pz.bz_off = z;
      tc_kernel<true, true><<<dim3(L.mtiles, (m + L.tw - 1) / L.tw, 1), kThreads, smem_for(P2.stage_bytes, P2.stages),
                              s>>>(mA2, mA2, Pz);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
  } else {
    tc_kernel<true, true><<<dim3(L.mtiles, (m + L.tw - 1) / L.tw, L.nchunk), kThreads,
                            smem_for(P2.stage_bytes, P2.stages), s>>>(mA2, mA2, P2);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  // C = the chunks' sum, both triangles (the greedy iterations read whole rows)
  reduce_lower_kernel<<<dim3((m + 31) / 32, (m + 31) / 32), dim3(32, 8), 0, s>>>(L.chunk_tiles, L.nchunk,
                                                                                 L.tiles_lower, L.tw, m, L.ldc, L.C);
  // U' (upper triangle of C, diagonal halved) = U1 + U2 + U3 in BF16
  {
    const long long tot = (long long)L.mpad * L.rpad;
    split_parts_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(L.C, L.ldc, m, m, L.mpad, L.rpad, L.Cp, 1,
                                                                       kParts);
  }
  const Params P3 = f0_params_dots(L, A, lda, m, n, src, err, spin_ns, stall);
  if ((e = set_smem<false, false>(P3)) != cudaSuccess) return e;
  tc_kernel<false, false><<<dim3(L.mtiles, (n + P3.n_tile - 1) / P3.n_tile, L.ndots), kThreads,
                            smem_for(P3.stage_bytes, P3.stages), s>>>(mU, mA3, P3);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // f_i = a_i^T C a_i = 2 a_i^T U' a_i
  sum_rows_kernel<<<(n + 255) / 256, 256, 0, s>>>(L.partial, L.mtiles * L.ndots, n, f, 2.0);
  return cudaGetLastError();
}

bool supported_any() { return encode_fn() != nullptr; }

// Tile lists of a problem: the C = A A^T tiles that touch the lower
// triangle (every chunk), and every column-dot tile.
void group_tile_counts(int m, int n, bool f32, int* t2, int* t3) {
  const F0Layout L = f0_layout(m, n, f32 ? kF0F32 : kF0Bf16, nullptr);   // (tile counts only)
  const int n_tile = dots_n_tile(f32);
  *t2 = L.tiles_lower * L.nchunk;
  *t3 = L.mtiles * ((n + n_tile - 1) / n_tile) * L.ndots;
}

size_t group_f0_desc_bytes(const int* m, const int* n, int count, bool f32) {
  size_t t2 = 0, t3 = 0;
  for (int i = 0; i < count; ++i) {
    int a, b;
    group_tile_counts(m[i], n[i], f32, &a, &b);
    t2 += a;
    t3 += b;
  }
  return align_up(sizeof(GroupProb) * (size_t)count) + align_up(sizeof(GroupTile) * std::max<size_t>(t2, 1)) +
         align_up(sizeof(GroupTile) * std::max<size_t>(t3, 1));
}

cudaError_t group_f0_prepare(int count, const void* const* A, const long long* lda, const int* m, const int* n,
                             void* const* scratch, double* const* f, const int* src, void* desc, int* err,
                             unsigned long long spin_ns, GroupF0* out, cudaStream_t s) {
  if (count < 1 || count > 65535) return cudaErrorInvalidValue;
  std::vector<GroupProb> probs(count);
  std::vector<GroupTile> t2, t3;
  std::vector<long long> c2, c3;   // work of each tile (K blocks), for the order
  for (int i = 0; i < count; ++i) {
    if (is_f32(src[i]) != is_f32(src[0])) return cudaErrorInvalidValue;   // one input type
    const F0Layout L = f0_layout(m[i], n[i], src[i], scratch[i]);
    GroupProb& g = probs[i];
    g = GroupProb{};
    if (!f0_maps(L, A[i], lda[i], m[i], n[i], src[i], &g.mapA2, &g.mapU, &g.mapA3)) return cudaErrorInvalidValue;
    g.p2 = f0_params_syrk(L, m[i], n[i], src[i], err, spin_ns, 0);
    g.p3 = f0_params_dots(L, A[i], lda[i], m[i], n[i], src[i], err, spin_ns, 0);
    g.A = A[i];
    g.lda = lda[i];
    g.m = m[i];
    g.n = n[i];
    g.mpad = L.mpad;
    g.npad = L.npad;
    g.rpad = L.rpad;
    g.src = src[i];
    g.nchunk = L.nchunk;
    g.ndots = L.ndots;
    g.mtiles = L.mtiles;
    g.tiles_lower = L.tiles_lower;
    g.tw = L.tw;
    g.C = L.C;
    g.ldc = L.ldc;
    g.chunk_tiles = L.chunk_tiles;
    g.Cp = L.Cp;
    g.Ap = L.Ap;
    g.Acopy = L.Acopy;
    g.partial = L.partial;
    g.f = f[i];
    const Params& P2 = g.p2;
    for (int bz = 0; bz < L.nchunk; ++bz)
      for (int bx = 0; bx < L.mtiles; ++bx)
        for (int by = 0; by <= (L.tw == 256 ? bx / 2 : bx); ++by) {
          t2.push_back(GroupTile{i, bx, by, bz});
          c2.push_back((long long)std::min(P2.kb_chunk, P2.kb_total - bz * P2.kb_chunk) * std::max(1, P2.npairs));
        }
    const Params& P3 = g.p3;
    for (int bz = 0; bz < L.ndots; ++bz)
      for (int by = 0; by < (n[i] + P3.n_tile - 1) / P3.n_tile; ++by)
        for (int bx = 0; bx < L.mtiles; ++bx) {
          const int kb0 = std::max(bz * P3.kb_chunk, bx * BM / BK);
          const int kb1 = std::min(P3.kb_total, (bz + 1) * P3.kb_chunk);
          t3.push_back(GroupTile{i, bx, by, bz});
          c3.push_back((long long)std::max(0, kb1 - kb0) * std::max(1, P3.npairs));
        }
  }
  // longest tiles first, so that the last wave is made of short ones
  auto order = [](std::vector<GroupTile>& t, const std::vector<long long>& c) {
    std::vector<int> ix(t.size());
    for (size_t i = 0; i < ix.size(); ++i) ix[i] = (int)i;
    std::stable_sort(ix.begin(), ix.end(), [&](int a, int b) { return c[a] > c[b]; });
    std::vector<GroupTile> o(t.size());
    for (size_t i = 0; i < ix.size(); ++i) o[i] = t[ix[i]];
    t.swap(o);
  };
  order(t2, c2);
  order(t3, c3);
  char* d = (char*)desc;
  GroupProb* dprobs = (GroupProb*)d;
  GroupTile* dt2 = (GroupTile*)(d + align_up(sizeof(GroupProb) * (size_t)count));
  GroupTile* dt3 = (GroupTile*)((char*)dt2 + align_up(sizeof(GroupTile) * std::max<size_t>(t2.size(), 1)));
  cudaError_t e;
  if ((e = cudaMemcpyAsync(dprobs, probs.data(), sizeof(GroupProb) * count, cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return e;
  if ((e = cudaMemcpyAsync(dt2, t2.data(), sizeof(GroupTile) * t2.size(), cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return e;
  if ((e = cudaMemcpyAsync(dt3, t3.data(), sizeof(GroupTile) * t3.size(), cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return e;
  // the host vectors end with this call
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  *out = GroupF0{};
  out->probs = dprobs;
  out->tiles2 = dt2;
  out->tiles3 = dt3;
  out->count = count;
  out->ntiles2 = (int)t2.size();
  out->ntiles3 = (int)t3.size();
  out->staged = 0;
  for (int i = 0; i < count; ++i) out->staged |= src[i] != kF0Bf16;
  out->smem2 = (int)smem_for(probs[0].p2.stage_bytes, probs[0].p2.stages);
  out->smem3 = (int)smem_for(probs[0].p3.stage_bytes, probs[0].p3.stages);
  return cudaSuccess;
}

cudaError_t group_f0_run(const GroupF0& g, cudaStream_t s) {
  cudaError_t e;
  const dim3 eg(kGroupBlocks, g.count);
  if (g.staged) group_split_kernel<<<eg, 256, 0, s>>>(g.probs, 0);
  if ((e = cudaFuncSetAttribute(tc_group_kernel<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, g.smem2)) !=
          cudaSuccess ||
      (e = cudaFuncSetAttribute(tc_group_kernel<true, true>, cudaFuncAttributePreferredSharedMemoryCarveout, 100)) !=
          cudaSuccess)
    return e;
  tc_group_kernel<true, true><<<g.ntiles2, kThreads, g.smem2, s>>>(g.probs, g.tiles2, 2);
  group_reduce_kernel<<<eg, dim3(32, 8), 0, s>>>(g.probs);
  group_split_kernel<<<eg, 256, 0, s>>>(g.probs, 1);
  if ((e = cudaFuncSetAttribute(tc_group_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                g.smem3)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(tc_group_kernel<false, false>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                100)) != cudaSuccess)
    return e;
  tc_group_kernel<false, false><<<g.ntiles3, kThreads, g.smem3, s>>>(g.probs, g.tiles3, 3);
  group_sum_rows_kernel<<<eg, 256, 0, s>>>(g.probs);
  return cudaGetLastError();
}

}  // namespace tc
}  // namespace css
