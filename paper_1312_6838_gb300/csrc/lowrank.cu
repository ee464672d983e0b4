// Rank-k approximation and approximate SVD from an embedding (Sec. 3.2):
//
//   W = U^(W) Sigma^(W) V^(W)^T,   A~_{S,k} = Q W~_k,
//   U~ = Q U^(W)_k,  Sigma~ = Sigma^(W)_k,  V~ = V^(W)_k   (Eq. ApproxSVD).
//
// W is short and wide (l x n, l <= 1024), so its SVD goes through the l x l
// Gram matrix G = W W^T = U^(W) (Sigma^(W))^2 U^(W)^T:
//   1. gram_rows_kernel: G in FP64 over lower 32 x 32 tiles, the n columns cut
//      into slices whose partial tiles gram_reduce_kernel adds in a fixed
//      order (bitwise reproducible).
//   2. jacobi_kernel: the eigenvalues of G by two-sided cyclic Jacobi
//      rotations (Golub and Van Loan, Matrix Computations, Sec. 8.5) in the
//      parallel round-robin ordering of Brent and Luk (1985): each round
//      rotates l/2 disjoint index pairs at once.  One cooperative kernel, one
//      CTA per chunk pair (x <= y) of a g x g grid, one grid barrier per
//      round; CTA (x, y) updates the 2 x 2 blocks whose row pair lies in pair
//      chunk x and column pair in chunk y and writes each to its mirror image
//      too, so it needs the rotations of two chunks only.  The rounds'
//      rotations are logged for the eigenvectors.
//   3. order_kernel: eigenvalues sorted descending, sigma, the tail sum and
//      the 1 / sigma scaling of V~; replay_columns_kernel forms only the k
//      wanted eigenvectors from the rotation log, off the barrier-bound path,
//      and signs them (U^(W)_k).
//   4. gemm_nn_df_kernel: U~ = Q U^(W)_k and V~ = W^T U^(W)_k Sigma_k^-1,
//      products in double-float (df.cuh) on the FP32 pipe.
//
// Steps 1-3 are FP64: on this part FP64 runs at 1/64 of the FP32 rate, so
// the Gram matrix (l^2 n / 2 multiply-adds) is bound by the FP64 pipe, and
// each Jacobi round by latency: one dependent L2 trip, a short chain of FP64
// arithmetic and a grid barrier.  The products of step 4 (l k (m + n)
// multiply-adds) need no more than double-float's 48 bits: their results
// are a singular basis, accurate to the Gram route's resolution anyway.
#include <algorithm>
#include <cmath>
#include <vector>

#include "css_common.cuh"
#include "lowrank.cuh"
#include "df.cuh"

using namespace css;

namespace {

constexpr int kGT = 32;          // Gram tile
constexpr int kGK = 32;          // columns per staged chunk
constexpr int kMaxL = 1024;
constexpr int kMaxSweeps = 40;
constexpr int kJacobiThreads = 256;
constexpr int kMaxGridDim = 16;  // at most 16 * 17 / 2 = 136 CTAs (<= one per SM)

// ----------------------------------------------------------- 1. G = W W^T --
// Block (pair, slice): output tile (ti, tj), ti >= tj, over the columns of one
// slice; 2 x 2 outputs per thread.
__global__ void __launch_bounds__(256) gram_rows_kernel(const double* __restrict__ W, long long ldw, int l,
                                                        int n, int slice, int npairs,
                                                        double* __restrict__ part) {
  __shared__ double xa[kGT][kGK + 1], xb[kGT][kGK + 1];
  const int pidx = blockIdx.x, sl = blockIdx.y;
  int ti = (int)((sqrtf(8.f * pidx + 1.f) - 1.f) * 0.5f);
  while (ti * (ti + 1) / 2 > pidx) --ti;
  while ((ti + 1) * (ti + 2) / 2 <= pidx) ++ti;
  const int tj = pidx - ti * (ti + 1) / 2;
  const int a0 = ti * kGT, b0 = tj * kGT;
  const int cb = sl * slice, ce = min(n, cb + slice);
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double acc00 = 0.0, acc01 = 0.0, acc10 = 0.0, acc11 = 0.0;
  for (int c0 = cb; c0 < ce; c0 += kGK) {
    for (int e = threadIdx.x; e < kGT * kGK; e += 256) {
      const int row = e / kGK, col = e % kGK;
      const bool okc = c0 + col < ce;
      xa[row][col] = (okc && a0 + row < l) ? W[(long long)(a0 + row) * ldw + c0 + col] : 0.0;
      xb[row][col] = (okc && b0 + row < l) ? W[(long long)(b0 + row) * ldw + c0 + col] : 0.0;
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

// G (lp x lp, column-major, zero padding row/column when l is odd) from the
// slices' partial tiles, added in slice order.
__global__ void gram_reduce_kernel(const double* __restrict__ part, int nslices, int npairs, int l, int lp,
                                   double* __restrict__ G) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)lp * lp) return;
  const int r = (int)(idx % lp), c = (int)(idx / lp);
  if (r >= l || c >= l) {
    G[idx] = 0.0;
    return;
  }
  const int a = max(r, c), b = min(r, c);
  const int ti = a / kGT, tj = b / kGT;
  const int pidx = ti * (ti + 1) / 2 + tj;
  const int off = (a % kGT) * kGT + (b % kGT);
  double s = 0.0;
  for (int q = 0; q < nslices; ++q) s += part[((long long)q * npairs + pidx) * (kGT * kGT) + off];
  G[idx] = s;
}

// ------------------------------------------------------------- 2. Jacobi --
struct JacobiArgs {
  double* G0;
  double* G1;
  double2* rotlog;    // (c, s) of every pair of every round, for the V replay
  long long max_rounds;
  int lp;
  int gdim;
  int chunk;          // pairs per chunk
  uint32_t* bar;
  int* flags;         // [kMaxSweeps + 1]: some pair still needs a rotation
  int* info;          // [0] sweeps, [1] buffer holding the final G, [2] rounds
  DevStatus* st;
};

// Pair j of round r of the round-robin tournament on lp indices: index lp-1
// stays, the others turn one step per round (every pair meets once in lp-1
// rounds).
__device__ __forceinline__ void rr_pair(int r, int j, int lp, int& p, int& q) {
  int a, b;
  if (j == 0) {
    a = r;
    b = lp - 1;
  } else {
    a = (r + j) % (lp - 1);
    b = (r + lp - 1 - j) % (lp - 1);
  }
  p = min(a, b);
  q = max(a, b);
}

// One plane rotation applied to a pair (a, b): (c a - s b, s a + c b), in one
// fixed instruction order so that mirrored elements come out bitwise equal.
__device__ __forceinline__ void rot(double c, double s, double a, double b, double& x, double& y) {
  x = fma(c, a, -(s * b));
  y = fma(s, a, c * b);
}

// A pair is rotated unless |g_pq| <= 1e-15 sqrt(g_pp g_qq) (the relative test
// of Demmel and Veselic) or |g_pq| <= 1e-17 trace(G), far below the Gram
// matrix's own rounding.  Evaluated in FP32 on the entries scaled by
// 1 / trace(G) (all of magnitude <= 1 for a PSD G).
__device__ __forceinline__ bool needs_rot(double gpp, double gqq, double gpq, double inv_tr) {
  const float ps = (float)(gpp * inv_tr), qs = (float)(gqq * inv_tr), xs = fabsf((float)(gpq * inv_tr));
  return xs > 1e-17f && xs * xs > 1e-30f * fabsf(ps * qs);
}

// The rotation that annihilates g_pq: t = tan(theta), the smaller root of
// t^2 + 2 tau t - 1 = 0 with tau = (g_qq - g_pp) / (2 g_pq), i.e.
// t = sgn(d) 2 g_pq / (|d| + sqrt(d^2 + 4 g_pq^2)), d = g_qq - g_pp (taken in
// FP64, then scaled by 1 / trace(G)), formed in FP32: t only has to be close.
// c = 1 / sqrt(1 + t^2) then comes from that t to FP64 precision (the FP32
// reciprocal square root refined by two Newton-Raphson steps
// y <- y (3/2 - x y^2 / 2)), and s = t c, so the rotation is orthogonal to
// FP64 precision.
__device__ __forceinline__ void rot_angle(double gpp, double gqq, double gpq, double inv_tr, double& c,
                                          double& sn) {
  const float df = (float)((gqq - gpp) * inv_tr), gf = 2.f * (float)(gpq * inv_tr);
  const float tf = copysignf(1.f, df) * gf / (fabsf(df) + sqrtf(fmaf(df, df, gf * gf)));
  const double t = (double)tf;
  const double x = fma(t, t, 1.0), hx = -0.5 * x;
  double y = (double)rsqrtf((float)x);
  y = y * fma(hx, y * y, 1.5);
  y = y * fma(hx, y * y, 1.5);
  c = y;
  sn = t * y;
}

__global__ void __launch_bounds__(kJacobiThreads) jacobi_kernel(JacobiArgs A) {
  __shared__ double s_c[kMaxL / 2], s_s[kMaxL / 2];
  __shared__ double s_red[32];
  __shared__ uint32_t s_epoch;
  __shared__ int s_any;
  const int lp = A.lp, h = lp / 2, NT = kJacobiThreads, tid = threadIdx.x;
  // CTA -> chunk pair (cx <= cy) of the upper triangle of a gdim x gdim grid
  int cx = 0, cb = blockIdx.x;
  while (cb >= A.gdim - cx) { cb -= A.gdim - cx; ++cx; }
  const int cy = cx + cb;
  const int xb = cx * A.chunk, xe = min(h, xb + A.chunk);
  const int yb = cy * A.chunk, ye = min(h, yb + A.chunk);
  const int ncta = gridDim.x;
  if (tid == 0) s_epoch = 0u;
  // trace(G) = ||W||_F^2, the same sum in every CTA
  double tr = 0.0;
  for (int i = tid; i < lp; i += NT) tr += A.G0[(long long)i * lp + i];
  tr = block_sum(tr, s_red);
  if (!isfinite(tr)) {
    if (blockIdx.x == 0 && tid == 0) set_error(A.st, (int32_t)CSS_ERR_NONFINITE, 0);
    return;
  }
  const double inv_tr = tr > 0.0 ? 1.0 / tr : 0.0;
  const int nx = xe - xb, ny = ye - yb;
  const int nang = nx + (cx == cy ? 0 : ny);
  // blocks (jr, jc), jr in chunk x, jc in chunk y; on a diagonal chunk pair
  // only jr <= jc (the other half is the mirror image)
  const bool diag = cx == cy;
  const int nblk = diag ? nx * (nx + 1) / 2 : nx * ny;
  auto block_of = [diag, xb, yb, nx](int e) -> int2 {
    if (diag) {
      int b = (int)((sqrtf(8.f * e + 1.f) - 1.f) * 0.5f);
      while (b * (b + 1) / 2 > e) --b;
      while ((b + 1) * (b + 2) / 2 <= e) ++b;
      return make_int2(xb + (e - b * (b + 1) / 2), xb + b);
    }
    return make_int2(xb + e % nx, yb + e / nx);
  };
  const long long tot = (long long)lp * lp;
  const long long per = (tot + ncta - 1) / ncta;
  const long long cbeg = (long long)blockIdx.x * per, cend = min(tot, cbeg + per);
  int cur = 0, sweep = 0;
  long long rg = 0;
  bool conv = false;
  for (sweep = 0; sweep <= kMaxSweeps; ++sweep) {
    // Does any pair of the current G still need a rotation?  (Checked on
    // the whole matrix, so no sweep without rotations is needed to stop.)
    {
      const double* Gc = cur ? A.G1 : A.G0;
      int bad = 0;
      for (long long idx = cbeg + tid; idx < cend; idx += NT) {
        const int p = (int)(idx % lp), q = (int)(idx / lp);
        if (p >= q) continue;
        const double gpq = __ldcg(Gc + idx);
        const double gpp = __ldcg(Gc + (long long)p * lp + p), gqq = __ldcg(Gc + (long long)q * lp + q);
        bad |= needs_rot(gpp, gqq, gpq, inv_tr) ? 1 : 0;
      }
      if (__syncthreads_or(bad) && tid == 0) atomicOr(A.flags + sweep, 1);
      if (!team_barrier(A.bar, ncta, A.st, 40, &s_epoch)) return;
      if (tid == 0) s_any = __ldcg(A.flags + sweep);
      __syncthreads();
      if (!s_any) {
        conv = true;
        break;
      }
      if (sweep == kMaxSweeps || rg + (lp - 1) > A.max_rounds) break;
    }
    for (int r = 0; r < lp - 1; ++r, ++rg) {
      const double* Gc = cur ? A.G1 : A.G0;
      double* Gn = cur ? A.G0 : A.G1;
      // this thread's first 2 x 2 block: its loads go out together with the
      // rotations' inputs (both only need the round's pairs)
      int f_r0 = 0, f_r1 = 0, f_c0 = 0, f_c1 = 0;
      double f00 = 0.0, f10 = 0.0, f01 = 0.0, f11 = 0.0;
      if (tid < nblk) {
        const int2 fj = block_of(tid);
        rr_pair(r, fj.x, lp, f_r0, f_r1);
        rr_pair(r, fj.y, lp, f_c0, f_c1);
        f00 = __ldcg(Gc + (long long)f_c0 * lp + f_r0);
        f10 = __ldcg(Gc + (long long)f_c0 * lp + f_r1);
        f01 = __ldcg(Gc + (long long)f_c1 * lp + f_r0);
        f11 = __ldcg(Gc + (long long)f_c1 * lp + f_r1);
      }
      for (int e = tid; e < nang; e += NT) {
        const int j = e < nx ? xb + e : yb + (e - nx);
        int p, q;
        rr_pair(r, j, lp, p, q);
        const double gpp = __ldcg(Gc + (long long)p * lp + p);
        const double gqq = __ldcg(Gc + (long long)q * lp + q);
        const double gpq = __ldcg(Gc + (long long)q * lp + p);
        double c = 1.0, sn = 0.0;
        if (needs_rot(gpp, gqq, gpq, inv_tr)) rot_angle(gpp, gqq, gpq, inv_tr, c, sn);
        s_c[j] = c;
        s_s[j] = sn;
        // the CTA on the diagonal of chunk x logs the chunk's rotations
        if (cx == cy) A.rotlog[rg * h + j] = make_double2(c, sn);
      }
      __syncthreads();
      // 2 x 2 blocks: rows of pair jr, columns of pair jc, jr <= jc; each is
      // written to both its own place and its mirror image, so G stays
      // exactly symmetric and half the rotations' FP64 work is saved.
      for (int e = tid; e < nblk; e += NT) {
        const int2 jj = block_of(e);
        const int jr = jj.x, jc = jj.y;
        int r0, r1, c0, c1;
        double b00, b10, b01, b11;
        if (e == tid) {
          r0 = f_r0; r1 = f_r1; c0 = f_c0; c1 = f_c1;
          b00 = f00; b10 = f10; b01 = f01; b11 = f11;
        } else {
          rr_pair(r, jr, lp, r0, r1);
          rr_pair(r, jc, lp, c0, c1);
          b00 = __ldcg(Gc + (long long)c0 * lp + r0);
          b10 = __ldcg(Gc + (long long)c0 * lp + r1);
          b01 = __ldcg(Gc + (long long)c1 * lp + r0);
          b11 = __ldcg(Gc + (long long)c1 * lp + r1);
        }
        const double cr = s_c[jr], sr = s_s[jr], cc = s_c[jc], sc = s_s[jc];
        double x00, x10, x01, x11, o00, o01, o10, o11;
        rot(cr, sr, b00, b10, x00, x10);     // rows
        rot(cr, sr, b01, b11, x01, x11);
        rot(cc, sc, x00, x01, o00, o01);     // columns
        rot(cc, sc, x10, x11, o10, o11);
        if (jr == jc) {
          // the pair's own 2 x 2 block: g_pq = g_qp
          Gn[(long long)r0 * lp + r0] = o00;
          Gn[(long long)r1 * lp + r0] = o01;
          Gn[(long long)r0 * lp + r1] = o01;
          Gn[(long long)r1 * lp + r1] = o11;
        } else {
          Gn[(long long)c0 * lp + r0] = o00;
          Gn[(long long)c1 * lp + r0] = o01;
          Gn[(long long)c0 * lp + r1] = o10;
          Gn[(long long)c1 * lp + r1] = o11;
          Gn[(long long)r0 * lp + c0] = o00;
          Gn[(long long)r0 * lp + c1] = o01;
          Gn[(long long)r1 * lp + c0] = o10;
          Gn[(long long)r1 * lp + c1] = o11;
        }
      }
      if (!team_barrier(A.bar, ncta, A.st, 41, &s_epoch)) return;
      cur ^= 1;
    }
  }
  if (blockIdx.x == 0 && tid == 0) {
    A.info[0] = sweep;
    A.info[1] = cur;
    A.info[2] = (int)rg;
    if (!conv) set_error(A.st, (int32_t)CSS_ERR_NOT_CONVERGED, 42);
  }
}

// Eigenvector ord[r] of G is column ord[r] of V = J_1 J_2 ... J_R, the product
// of every round's rotations: V e = J_1 (J_2 (... (J_R e))).  Block r replays
// the logged rounds backwards on that one column, kept in shared memory (the
// round's pairs are disjoint, so one thread a pair), then signs it so that
// its entry of largest magnitude (lowest index on ties) is positive and
// writes it as column r of U^(W)_k.  Only the k wanted columns are formed.
__global__ void __launch_bounds__(512) replay_columns_kernel(const double2* __restrict__ rotlog,
                                                             const int* __restrict__ info,
                                                             const int* __restrict__ ord, int l, int lp,
                                                             double* __restrict__ Uw) {
  extern __shared__ double col[];
  __shared__ double s_best[16];
  __shared__ int s_bi[16];
  const int h = lp / 2, j = threadIdx.x;   // blockDim.x: h rounded up to whole warps
  const int c0 = ord[blockIdx.x];
  for (int i = threadIdx.x; i < lp; i += blockDim.x) col[i] = (i == c0) ? 1.0 : 0.0;
  __syncthreads();
  const long long R = info[2];
  const bool act = j < h;
  int r = R > 0 ? (int)((R - 1) % (lp - 1)) : 0;
  double2 cs = (act && R > 0) ? __ldcg(rotlog + (R - 1) * h + j) : make_double2(1.0, 0.0);
  for (long long g = R - 1; g >= 0; --g) {
    const double2 nxt = (act && g > 0) ? __ldcg(rotlog + (g - 1) * h + j) : make_double2(1.0, 0.0);
    if (act) {
      int p, q;
      rr_pair(r, j, lp, p, q);
      const double vp = col[p], vq = col[q];
      // (J v)_p = c v_p + s v_q,  (J v)_q = -s v_p + c v_q
      col[p] = fma(cs.x, vp, cs.y * vq);
      col[q] = fma(cs.x, vq, -(cs.y * vp));
    }
    __syncthreads();
    cs = nxt;
    if (--r < 0) r = lp - 2;
  }
  // sign rule: block-wide argmax of |v_i| (lowest index on ties)
  double best = -1.0;
  int bi = l;
  for (int i = threadIdx.x; i < l; i += blockDim.x) {
    const double a = fabs(col[i]);
    if (a > best) { best = a; bi = i; }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if (lane == 0) { s_best[wid] = best; s_bi[wid] = bi; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < nw; ++w)
      if (s_best[w] > best || (s_best[w] == best && s_bi[w] < bi)) { best = s_best[w]; bi = s_bi[w]; }
    s_bi[0] = bi;
  }
  __syncthreads();
  bi = s_bi[0];
  const double sg = (bi < l && col[bi] < 0.0) ? -1.0 : 1.0;
  for (int i = threadIdx.x; i < l; i += blockDim.x) Uw[(long long)blockIdx.x * l + i] = sg * col[i];
}

// --------------------------------------------------- 3. order and signs --
// One block.  lam_i = G_ii; rank by (lambda descending, index ascending).
__global__ void __launch_bounds__(1024) order_kernel(const double* __restrict__ G0, const double* __restrict__ G1,
                                                     const int* __restrict__ info, int l, int lp, int k, long long n,
                                                     double* __restrict__ sigma, double* __restrict__ scale,
                                                     double* __restrict__ tail, int* __restrict__ ord_out) {
  __shared__ double lam[kMaxL];
  __shared__ int ord[kMaxL];
  __shared__ double red[32];
  const double* G = info[1] ? G1 : G0;
  for (int i = threadIdx.x; i < l; i += blockDim.x) lam[i] = G[(long long)i * lp + i];
  __syncthreads();
  double tr = 0.0;
  for (int i = threadIdx.x; i < l; i += blockDim.x) {
    const double v = lam[i];
    int rk = 0;
    for (int j = 0; j < l; ++j) rk += (lam[j] > v) || (lam[j] == v && j < i);
    ord[rk] = i;
    tr += fmax(v, 0.0);
  }
  tr = block_sum(tr, red);   // ||W||_F^2
  double tl = 0.0;
  for (int r = k + threadIdx.x; r < l; r += blockDim.x) tl += fmax(lam[ord[r]], 0.0);
  tl = block_sum(tl, red);
  if (threadIdx.x == 0 && tail) tail[0] = tl;
  // resolution of the Gram route: (n + l) 2^-52 ||W||_F^2
  const double thr = (double)(n + l) * 0x1p-52 * tr;
  for (int r = threadIdx.x; r < k; r += blockDim.x) {
    const double lv = fmax(lam[ord[r]], 0.0);
    const double sv = sqrt(lv);
    sigma[r] = sv;
    scale[r] = (lv > thr && sv > 0.0) ? 1.0 / sv : 0.0;
    ord_out[r] = ord[r];
  }
}

// ----------------------------------- 4. C = A B diag(scale), double-float --
// A: M x K (lda), B: K x N (ldb), C: M x N (ldc), all column-major FP64.
// 64 x 64 outputs per block, 4 x 4 per thread (rows tx + 16 a, columns
// ty + 16 b).  The operands are split into hi + lo floats as they are staged
// and the products accumulate in double-float (df.cuh): about 2^-46 relative
// per term against FP64's 2^-53, on the FP32 pipe.  When a_bound is given
// (a device value >= every |A_ij|), A is first scaled by 2^-(e+1), where
// 2^e <= a_bound < 2^(e+1), so its entries stay inside FP32's range; the
// scaling is exact and is undone on the output.  B's entries must lie in
// FP32's range (here: orthonormal columns, entries <= 1).
__global__ void __launch_bounds__(256) gemm_nn_df_kernel(const double* __restrict__ A, long long lda,
                                                         const double* __restrict__ B, long long ldb,
                                                         const double* __restrict__ scale,
                                                         const double* __restrict__ a_bound,
                                                         double* __restrict__ C, long long ldc, long long M,
                                                         int N, int K) {
  constexpr int BK = 16;
  __shared__ float2 as[BK][64], bs[BK][65];
  const long long m0 = (long long)blockIdx.x * 64;
  const int n0 = blockIdx.y * 64;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double sa = 1.0, inv_sa = 1.0;
  if (a_bound) {
    const double ab = *a_bound;
    if (ab > 0.0 && isfinite(ab)) {
      const int e = ilogb(ab) + 1;
      sa = ldexp(1.0, -e);
      inv_sa = ldexp(1.0, e);
    }
  }
  DF acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = DF{0.f, 0.f};
  for (int k0 = 0; k0 < K; k0 += BK) {
    for (int e = threadIdx.x; e < BK * 64; e += 256) {
      const int i = e % 64, kk = e / 64;
      float2 va = make_float2(0.f, 0.f), vb = make_float2(0.f, 0.f);
      if (m0 + i < M && k0 + kk < K) df_split(A[(long long)(k0 + kk) * lda + m0 + i] * sa, va.x, va.y);
      as[kk][i] = va;
      const int kk2 = e % BK, j = e / BK;
      if (n0 + j < N && k0 + kk2 < K) df_split(B[(long long)(n0 + j) * ldb + k0 + kk2], vb.x, vb.y);
      bs[kk2][j] = vb;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < BK; ++kk) {
      float2 av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = as[kk][tx + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = bs[kk][ty + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) df_fma2(acc[a][b], av[a].x, av[a].y, bv[b].x, bv[b].y);
    }
    __syncthreads();
  }
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const int j = n0 + ty + 16 * b;
    if (j >= N) continue;
    const double sc = (scale ? scale[j] : 1.0) * inv_sa;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const long long i = m0 + tx + 16 * a;
      if (i < M) C[(long long)j * ldc + i] = ((double)acc[a][b].s + (double)acc[a][b].c) * sc;
    }
  }
}

// ------------------------------------------------------------ host side --
struct LrLayout {
  DevStatus* st;
  int* info;
  int* flags;
  uint32_t* bar;
  double *part, *G0, *G1, *Uw, *scale;
  int* ord;
  double2* rotlog;
  long long max_rounds;
  int nslices, npairs, slice;
  size_t bytes;
};

int gram_tiles(int l) { return (l + kGT - 1) / kGT; }

LrLayout lr_layout(void* ws, size_t cap, int64_t n, int32_t l, int32_t k, int sms) {
  WsCarver c(ws, cap);
  LrLayout L{};
  L.st = (DevStatus*)c.take<char>(kStatusBytes);   // first: css_read_status reads it
  L.info = c.take<int>(64);
  L.flags = c.take<int>(kMaxSweeps + 4);
  L.bar = c.take<uint32_t>(64);
  const int t = gram_tiles(l);
  L.npairs = t * (t + 1) / 2;
  // about twelve (pair, slice) blocks per SM, so that the uneven last share
  // of blocks costs little; slices of >= 256 columns
  const int want = std::max(1, (12 * std::max(sms, 1) + L.npairs - 1) / L.npairs);
  const int cap_slices = (int)std::max<int64_t>(1, (n + 255) / 256);
  L.nslices = std::min({want, cap_slices, 256});
  L.slice = (int)((n + L.nslices - 1) / L.nslices);
  L.part = c.take<double>((size_t)L.nslices * L.npairs * kGT * kGT);
  const int lp = l + (l & 1);
  L.G0 = c.take<double>((size_t)lp * lp);
  L.G1 = c.take<double>((size_t)lp * lp);
  L.ord = c.take<int>(k);
  L.max_rounds = (long long)kMaxSweeps * (lp - 1);
  L.rotlog = c.take<double2>((size_t)L.max_rounds * (lp / 2));
  L.Uw = c.take<double>((size_t)l * k);
  L.scale = c.take<double>(k);
  L.bytes = c.off;
  return L;
}

int device_sms() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return n;
}

// The Gram slices are sized for 152 SMs whatever the device, so that
// css_workspace_size needs no device and the launch carves the same layout.
constexpr int kLayoutSms = 152;

}  // namespace

size_t lowrank_workspace_bytes(int64_t n, int32_t l, int32_t k) {
  return lr_layout(nullptr, (size_t)-1, n, l, k, kLayoutSms).bytes;
}

extern "C" css_status css_lowrank(const double* W, int64_t ldw, const double* Q, int64_t ldq, int64_t m,
                                  int64_t n, int32_t l, int32_t k, double* sigma, double* U, int64_t ldu,
                                  double* V, int64_t ldv, double* Uw, double* tail, void* ws, size_t ws_bytes,
                                  const css_opts* opts, css_stream_t stream) {
  css_opts o;
  css_opts_default(&o);
  if (opts) o = *opts;
  if (!W || !sigma) return CSS_ERR_INVALID_ARG;
  if (n < 1 || n > INT32_MAX || ldw < n || l < 1 || l > kMaxL || k < 1 || k > l) return CSS_ERR_INVALID_ARG;
  if (U && (!Q || m < 1 || m > INT32_MAX || ldq < m || ldu < m)) return CSS_ERR_INVALID_ARG;
  if (V && ldv < n) return CSS_ERR_INVALID_ARG;
  if (!ws || ((uintptr_t)ws % kWsAlign) != 0) return CSS_ERR_WORKSPACE;
  LrLayout L = lr_layout(ws, ws_bytes, n, l, k, kLayoutSms);
  if (L.bytes > ws_bytes) return CSS_ERR_WORKSPACE;
  int dev = 0, major = 0, minor = 0, coop = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CSS_ERR_CUDA;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (major != 10 || minor != 3 || !coop) return CSS_ERR_UNSUPPORTED;
  cudaStream_t s = (cudaStream_t)stream;
  const int lp = l + (l & 1), h = lp / 2;
  // Jacobi grid: the g (g + 1) / 2 chunk pairs of the upper triangle,
  // chunks of about 8 pairs, g <= 16, no more CTAs than SMs
  int gdim = std::max(1, std::min(kMaxGridDim, h / 8));
  const int sms = device_sms();
  while (gdim > 1 && gdim * (gdim + 1) / 2 > sms) --gdim;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, jacobi_kernel, kJacobiThreads, 0) != cudaSuccess ||
      occ < 1)
    return CSS_ERR_CUDA;
  const int chunk = (h + gdim - 1) / gdim;

  DevStatus hs{};
  hs.spin_budget_ns = o.spin_budget_ns ? o.spin_budget_ns : 2000000000ull;
  cudaError_t e = cudaMemcpyAsync(L.st, &hs, sizeof(hs), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(L.flags, 0, sizeof(int) * (kMaxSweeps + 4), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(L.bar, 0, sizeof(uint32_t) * 64, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(L.info, 0, sizeof(int) * 64, s);
  if (e != cudaSuccess) return CSS_ERR_CUDA;
  // opts->timing_ms (sync mode): Gram, eigendecomposition, products, sweeps
  const bool timed = o.timing_ms != nullptr && o.sync;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  if (timed)
    for (auto& x : ev)
      if (cudaEventCreate(&x) != cudaSuccess) return CSS_ERR_CUDA;
  struct EvGuard {
    cudaEvent_t* e;
    ~EvGuard() {
      for (int i = 0; i < 4; ++i)
        if (e[i]) cudaEventDestroy(e[i]);
    }
  } guard{ev};
  if (timed) cudaEventRecord(ev[0], s);
  gram_rows_kernel<<<dim3(L.npairs, L.nslices), 256, 0, s>>>(W, ldw, l, (int)n, L.slice, L.npairs, L.part);
  gram_reduce_kernel<<<(unsigned)(((long long)lp * lp + 255) / 256), 256, 0, s>>>(L.part, L.nslices, L.npairs,
                                                                                   l, lp, L.G0);
  if (cudaGetLastError() != cudaSuccess) return CSS_ERR_CUDA;
  if (timed) cudaEventRecord(ev[1], s);
  JacobiArgs ja{L.G0, L.G1, L.rotlog, L.max_rounds, lp, gdim, chunk, L.bar, L.flags, L.info, L.st};
  void* args[] = {&ja};
  e = cudaLaunchCooperativeKernel((const void*)jacobi_kernel, dim3(gdim * (gdim + 1) / 2), dim3(kJacobiThreads),
                                  args, 0, s);
  if (e != cudaSuccess) return CSS_ERR_CUDA;
  double* uw = Uw ? Uw : L.Uw;
  order_kernel<<<1, 1024, 0, s>>>(L.G0, L.G1, L.info, l, lp, k, (long long)n, sigma, L.scale, tail, L.ord);
  replay_columns_kernel<<<k, (h + 31) / 32 * 32, lp * sizeof(double), s>>>(L.rotlog, L.info, L.ord, l, lp, uw);
  if (timed) cudaEventRecord(ev[2], s);
  // |W_ij| <= ||W||_2 = sigma_1 bounds W's entries for the FP32 split
  if (U)
    gemm_nn_df_kernel<<<dim3((unsigned)((m + 63) / 64), (k + 63) / 64), 256, 0, s>>>(Q, ldq, uw, l, nullptr, nullptr,
                                                                                      U, ldu, m, k, l);
  if (V)
    gemm_nn_df_kernel<<<dim3((unsigned)((n + 63) / 64), (k + 63) / 64), 256, 0, s>>>(W, ldw, uw, l, L.scale, sigma,
                                                                                      V, ldv, n, k, l);
  if (cudaGetLastError() != cudaSuccess) return CSS_ERR_CUDA;
  if (timed) cudaEventRecord(ev[3], s);
  if (!o.sync) return CSS_OK;
  DevStatus st{};
  int info[2] = {0, 0};
  e = cudaMemcpyAsync(&st, L.st, sizeof(st), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(info, L.info, sizeof(info), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return CSS_ERR_CUDA;
  if (timed) {
    float ms[3] = {0.f, 0.f, 0.f};
    for (int i = 0; i < 3; ++i) cudaEventElapsedTime(&ms[i], ev[i], ev[i + 1]);
    for (int i = 0; i < 3; ++i) o.timing_ms[i] = ms[i];
    o.timing_ms[3] = info[0];
  }
  return st.code != 0 ? (css_status)st.code : CSS_OK;
}
