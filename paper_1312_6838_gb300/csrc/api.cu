// C ABI of libcss (include/css.h): argument checks, workspace layout and the
// launch sequence of every entry point.  All device work is in greedy.cu,
// init_simt.cu, project.cu and backward.cu.
#include <algorithm>
#include <cstring>
#include <type_traits>
#include <mutex>
#include <numeric>
#include <vector>

#include "greedy.cuh"
#include "init.cuh"
#include "tc.cuh"
#include "project.cuh"
#include "tune.cuh"
#include "backward.cuh"
#include "lowrank.cuh"

using namespace css;

namespace {

constexpr int kMaxK = 1024;          // columns selected per problem
constexpr int kMaxCtas = 1024;       // descriptor space reserved per call
constexpr uint64_t kDefaultSpinNs = 2000000000ull;
constexpr double kPivotColumnEquiv = 1500.0;  // planner default: one pivot step in streamed columns
constexpr int kDefaultSplitShare = 2;        // fused step: split tail tiles for half of the warps

size_t esize(int dt) { return dt == CSS_F64 ? 8 : dt == CSS_F32 ? 4 : 2; }
size_t accsize(int dt) { return dt == CSS_F64 ? 8 : 4; }
bool valid_dtype(int dt) { return dt == CSS_F64 || dt == CSS_F32 || dt == CSS_BF16; }

css_opts defaults() {
  css_opts o;
  std::memset(&o, 0, sizeof(o));
  o.tau_rel = -1.0;
  o.sync = 1;
  return o;
}

double tau_of(const css_opts& o, int dt) {
  if (o.tau_rel >= 0.0) return o.tau_rel;
  return dt == CSS_F64 ? 1e-12 : 1e-6;
}

// Per-problem device state (see UnitDesc in greedy.cuh).
struct UnitState {
  double *f = nullptr, *g = nullptr, *thr = nullptr;
  unsigned char* selmask = nullptr;
  double *Q = nullptr, *Z = nullptr, *W = nullptr;
  void *qv = nullptr, *ypv = nullptr;
  double *e1 = nullptr, *e = nullptr, *y = nullptr, *coef = nullptr, *ups = nullptr;
};

void carve_scores(WsCarver& c, int n, UnitState& s) {
  s.f = c.take<double>(n);
  s.g = c.take<double>(n);
  s.thr = c.take<double>(n);
  s.selmask = c.take<unsigned char>(n);
}

void carve_rest(WsCarver& c, int dt, int m, int n, int k, int r, int mode, bool need_W,
                UnitState& s) {
  s.Q = c.take<double>((size_t)m * k);
  s.Z = c.take<double>((size_t)(mode == 0 ? m : r) * k);
  // W (the omega rows) is an optional output only; nothing reads it back
  (void)need_W;
  (void)n;
  s.qv = c.take<char>((size_t)m * accsize(dt));
  s.ypv = c.take<char>((size_t)m * accsize(dt));
  s.e1 = c.take<double>(m);
  s.e = c.take<double>(m);
  s.y = c.take<double>(m);
  s.coef = c.take<double>(std::max(k, r) + 1);
  s.ups = c.take<double>(std::max(r, 1));
}

// Launch-wide descriptor region.
struct Header {
  DevStatus* st;
  DevStatus* st_init;   // the status a launch starts from (copied into st)
  UnitDesc* units;
  TeamDesc* teams;
  int* order;
  int* cta_team;
  uint32_t* bars;
  double* part;
  double* cand_val;
  int* cand_idx;
  uint32_t* tile_ctr;
  int* aux_err;   // error flag of the tensor-core initial-score kernel
  void* split_part;
  uint32_t* split_done;
  int split_slots;
};

// Split-tile slots for units with `split_cols` columns in total: a team never
// splits more tiles than it has warps or than its widest unit has tiles
// (tiles are at least two columns wide).
int split_slots_for(int64_t split_cols) {
  const int64_t per_grid = (int64_t)kMaxCtas * (kGreedyThreads / 32);
  return (int)std::min<int64_t>(per_grid, (split_cols + 1) / 2 + 1);
}

// Byte offset, inside the 256-byte status slot at the start of every
// workspace, of the tensor-core initial-score kernel's error flag.  The
// greedy launch resets only the DevStatus at offset 0, so the flag survives
// until css_read_status or finish() reads it.
constexpr size_t kAuxErrOffset = 128;
static_assert(sizeof(DevStatus) <= kAuxErrOffset && kAuxErrOffset + sizeof(int) <= kStatusBytes,
              "the flag sits in the status slot, after the DevStatus");

void carve_header(WsCarver& c, int max_units, Header& h, int64_t split_cols) {
  h.st = c.take<DevStatus>(1);
  h.aux_err = h.st ? reinterpret_cast<int*>(reinterpret_cast<char*>(h.st) + kAuxErrOffset) : nullptr;
  h.st_init = c.take<DevStatus>(1);
  h.units = c.take<UnitDesc>(max_units);
  h.teams = c.take<TeamDesc>(kMaxCtas);
  h.order = c.take<int>(max_units);
  h.cta_team = c.take<int>(kMaxCtas);
  h.bars = c.take<uint32_t>(2 * kMaxCtas);
  h.part = c.take<double>(4 * kMaxCtas);
  h.cand_val = c.take<double>(kMaxCtas);
  h.cand_idx = c.take<int>(kMaxCtas);
  h.tile_ctr = c.take<uint32_t>(2 * kMaxCtas);
  h.split_slots = split_slots_for(split_cols);
  h.split_part = c.take<char>((size_t)h.split_slots * kSplitSlotBytes);
  h.split_done = c.take<uint32_t>(h.split_slots);
}

css_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return CSS_OK;
  if (e == cudaErrorMemoryAllocation) return CSS_ERR_NO_MEMORY;
  return CSS_ERR_CUDA;
}

int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return n;
}

bool device_ok() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  int major = 0, minor = 0;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  return major == 10 && minor == 3;
}

// One team per entry of `team_units`; CTAs split proportionally to `work`.
struct Plan {
  std::vector<TeamDesc> teams;
  std::vector<int> order;
  std::vector<int> cta_team;
  int grid = 0;
};

// Assign units to teams.  units_per_team == 0: one team per unit, with CTA
// counts proportional to the unit's work (at least one CTA each) when the
// grid has more CTAs than units; otherwise longest-processing-time-first
// assignment of units to single-CTA teams.
Plan make_plan(const std::vector<double>& work, int grid) {
  Plan P;
  const int nu = (int)work.size();
  std::vector<int> idx(nu);
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return work[a] > work[b]; });
  if (nu <= grid) {
    double tot = 0.0;
    for (double w : work) tot += w;
    std::vector<int> cnt(nu, 1);
    int left = grid - nu;
    // largest remainder over the spare CTAs
    std::vector<double> share(nu);
    for (int u = 0; u < nu; ++u) share[u] = tot > 0 ? work[u] / tot * left : 0.0;
    int used = 0;
    for (int u = 0; u < nu; ++u) { int a = (int)share[u]; cnt[u] += a; used += a; }
    std::vector<int> rem(nu);
    std::iota(rem.begin(), rem.end(), 0);
    std::stable_sort(rem.begin(), rem.end(), [&](int a, int b) {
      return (share[a] - (int)share[a]) > (share[b] - (int)share[b]);
    });
    for (int q = 0; q < left - used && q < nu; ++q) cnt[rem[q]] += 1;
    int cta = 0;
    for (int q = 0; q < nu; ++q) {
      const int u = idx[q];
      TeamDesc t{};
      t.cta0 = cta;
      t.ncta = cnt[u];
      t.u_begin = q;
      t.u_end = q + 1;
      P.order.push_back(u);
      for (int c = 0; c < cnt[u]; ++c) P.cta_team.push_back((int)P.teams.size());
      cta += cnt[u];
      P.teams.push_back(t);
    }
    P.grid = cta;
  } else {
    std::vector<double> load(grid, 0.0);
    std::vector<std::vector<int>> lists(grid);
    for (int q = 0; q < nu; ++q) {
      const int u = idx[q];
      int best = (int)(std::min_element(load.begin(), load.end()) - load.begin());
      lists[best].push_back(u);
      load[best] += work[u];
    }
    for (int t = 0; t < grid; ++t) {
      TeamDesc d{};
      d.cta0 = t;
      d.ncta = 1;
      d.u_begin = (int)P.order.size();
      for (int u : lists[t]) P.order.push_back(u);
      d.u_end = (int)P.order.size();
      P.teams.push_back(d);
      P.cta_team.push_back(t);
    }
    P.grid = grid;
  }
  return P;
}

// A persistent launch in two parts: prepare_units plans the teams and copies
// every descriptor into the workspace; start_units resets the status, the
// barriers and the counters from device-side values and launches, so that
// it can be repeated (or captured in a CUDA graph) without host data.
struct LaunchInfo {
  GreedyLaunch L;
  int split_used;
  uint32_t* bars;
  uint32_t* tile_ctr;
  uint32_t* split_done;
  DevStatus* st;
  DevStatus* st_init;
  // false: the launch keeps the status an earlier launch of the same call
  // left (Algorithm 4's union launch reports the block launch's errors too)
  bool reset_status;
};

css_status prepare_units(const Header& h, std::vector<UnitDesc>& units, const std::vector<double>& work,
                         int dt, int grid_max, int tile_cols, uint64_t spin_ns, cudaStream_t s,
                         LaunchInfo& info, int stall_where = 0, int split_share = kDefaultSplitShare,
                         int threads = kGreedyThreads) {
  int m_max = 1, k_max = 1, r_max = 1;
  for (auto& u : units) {
    m_max = std::max(m_max, u.m);
    k_max = std::max(k_max, u.k);
    r_max = std::max(r_max, u.r);
  }
  const size_t smem = greedy_smem_bytes(dt, m_max, k_max, r_max, threads);
  if (smem > 227 * 1024) return CSS_ERR_UNSUPPORTED;
  const int occ = greedy_occupancy(dt, tile_cols, smem, threads);
  const int sms = sm_count();
  if (occ <= 0 || sms <= 0) return CSS_ERR_CUDA;
  int grid = std::min(grid_max > 0 ? grid_max : sms * occ, sms * occ);
  grid = std::min(grid, kMaxCtas);
  Plan P = make_plan(work, grid);
  int split_used = 0;
  for (size_t t = 0; t < P.teams.size(); ++t) {
    TeamDesc& d = P.teams[t];
    d.bar = h.bars + 2 * d.cta0;
    d.part = h.part + 4 * d.cta0;
    d.cand_val = h.cand_val + d.cta0;
    d.cand_idx = h.cand_idx + d.cta0;
    d.tile_ctr = h.tile_ctr + 2 * d.cta0;
    // split the last tiles of each fused step: at most one per warp of the team
    int widest = 0;
    for (int q = d.u_begin; q < d.u_end; ++q)
      widest = std::max(widest, (units[P.order[q]].n + tile_cols - 1) / tile_cols);
    const int cap = std::min({widest, d.ncta * (threads / 32) / std::max(1, split_share),
                              h.split_slots - split_used});
    d.split_cap = std::max(cap, 0);
    d.split_part = static_cast<char*>(h.split_part) + (size_t)split_used * kSplitSlotBytes;
    d.split_done = h.split_done + split_used;
    split_used += d.split_cap;
  }
  DevStatus st{};
  st.spin_budget_ns = spin_ns ? spin_ns : kDefaultSpinNs;
  st.stall_where = stall_where;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(h.st_init, &st, sizeof(st), cudaMemcpyHostToDevice, s)) != cudaSuccess) return cuda_status(e);
  if ((e = cudaMemcpyAsync(h.units, units.data(), units.size() * sizeof(UnitDesc), cudaMemcpyHostToDevice, s)) != cudaSuccess) return cuda_status(e);
  if ((e = cudaMemcpyAsync(h.teams, P.teams.data(), P.teams.size() * sizeof(TeamDesc), cudaMemcpyHostToDevice, s)) != cudaSuccess) return cuda_status(e);
  if ((e = cudaMemcpyAsync(h.order, P.order.data(), P.order.size() * sizeof(int), cudaMemcpyHostToDevice, s)) != cudaSuccess) return cuda_status(e);
  if ((e = cudaMemcpyAsync(h.cta_team, P.cta_team.data(), P.cta_team.size() * sizeof(int), cudaMemcpyHostToDevice, s)) != cudaSuccess) return cuda_status(e);
  GreedyLaunch L{};
  L.units = h.units;
  L.order = h.order;
  L.teams = h.teams;
  L.cta_team = h.cta_team;
  L.st = h.st;
  L.dtype = dt;
  L.tile_cols = tile_cols;
  L.m_max = m_max;
  L.k_max = k_max;
  L.r_max = r_max;
  L.grid = P.grid;
  L.threads = threads;
  L.smem = smem;
  info.L = L;
  info.split_used = split_used;
  info.bars = h.bars;
  info.tile_ctr = h.tile_ctr;
  info.split_done = h.split_done;
  info.st = h.st;
  info.st_init = h.st_init;
  info.reset_status = true;
  return CSS_OK;
}

css_status start_units(const LaunchInfo& info, cudaStream_t s) {
  cudaError_t e;
  if (info.reset_status &&
      (e = cudaMemcpyAsync(info.st, info.st_init, sizeof(DevStatus), cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
    return cuda_status(e);
  if ((e = cudaMemsetAsync(info.bars, 0, 2 * sizeof(uint32_t) * info.L.grid, s)) != cudaSuccess) return cuda_status(e);
  if ((e = cudaMemsetAsync(info.tile_ctr, 0, 2 * sizeof(uint32_t) * info.L.grid, s)) != cudaSuccess)
    return cuda_status(e);
  if (info.split_used > 0 &&
      (e = cudaMemsetAsync(info.split_done, 0, sizeof(uint32_t) * info.split_used, s)) != cudaSuccess)
    return cuda_status(e);
  return cuda_status(greedy_launch(info.L, s));
}

css_status launch_units(const Header& h, std::vector<UnitDesc>& units, const std::vector<double>& work,
                        int dt, int grid_max, int tile_cols, uint64_t spin_ns, cudaStream_t s,
                        int stall_where = 0, int split_share = kDefaultSplitShare) {
  LaunchInfo info{};
  css_status cs = prepare_units(h, units, work, dt, grid_max, tile_cols, spin_ns, s, info, stall_where,
                                split_share);
  if (cs != CSS_OK) return cs;
  return start_units(info, s);
}

css_status finish(const Header& h, const css_opts& o, cudaStream_t s) {
  if (!o.sync) return CSS_OK;
  DevStatus st{};
  int aux = 0;
  cudaError_t e = cudaMemcpyAsync(&st, h.st, sizeof(st), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&aux, h.aux_err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_status(e);
  if (aux != 0) return (css_status)aux;
  if (st.code != 0) return (css_status)st.code;
  return st.rank_exhausted ? CSS_RANK_EXHAUSTED : CSS_OK;
}

// CUDA-event phase timer for opts->timing_ms (sync mode only).
struct PhaseTimer {
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  bool on = false;
  PhaseTimer(const css_opts& o) : on(o.timing_ms != nullptr && o.sync) {
    if (on)
      for (auto& e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) on = false;
  }
  ~PhaseTimer() {
    for (auto& e : ev)
      if (e) cudaEventDestroy(e);
  }
  void mark(int i, cudaStream_t s) {
    if (on) cudaEventRecord(ev[i], s);
  }
  void report(const css_opts& o) {
    if (!on) return;
    float a = 0.f, b = 0.f;
    if (cudaEventSynchronize(ev[2]) != cudaSuccess) return;
    cudaEventElapsedTime(&a, ev[0], ev[1]);
    cudaEventElapsedTime(&b, ev[1], ev[2]);
    o.timing_ms[0] = a;
    o.timing_ms[1] = b;
  }
};

// Columns per fused-step tile: 8 keeps the most 16-byte loads in flight per
// warp (measured fastest for BF16 and FP32 at m = 4096); the split tail keeps
// the last, long tiles from idling the team.
// Columns per fused-step tile: the caller's choice, else the autotuner's
// (css_autotune_select, css_tile_cache_load) for this device and shape
// bucket, else 8, which keeps the most 16-byte loads in flight per warp and
// measured fastest for BF16 and FP32 at m = 4096.
int pick_tile(const css_opts& o, int dt, int64_t m, int64_t n) {
  if (o.tile_cols == 2 || o.tile_cols == 4 || o.tile_cols == 8) return o.tile_cols;
  const int t = tuned_tile(dt, m, n);
  return t ? t : 8;
}

// The forced prefix is device memory the caller wrote on `s`: it is read back
// in stream order (one synchronisation, forced prefixes only) and checked.
// Split share of the fused step: the caller's, else the tuned value for this
// device and shape bucket, else the default.
int pick_split_share(const css_opts& o, int dt, int64_t m, int64_t n) {
  if (o.split_share == 1 || o.split_share == 2 || o.split_share == 4 || o.split_share == 8) return o.split_share;
  const int t = tuned_knob(dt, m, n, 1);
  return t > 0 ? t : kDefaultSplitShare;
}

// Algorithm 4's planner pivot cost in streamed columns: the caller's, else the
// tuned value, else the default.
double pick_pivot_cost(const css_opts& o, int dt, int64_t m, int64_t n) {
  if (o.pivot_cost > 0) return (double)o.pivot_cost;
  const int t = tuned_knob(dt, m, n, 2);
  return t >= 0 ? (double)t : kPivotColumnEquiv;
}

bool valid_knobs(const css_opts& o) {
  return (o.split_share == 0 || o.split_share == 1 || o.split_share == 2 || o.split_share == 4 ||
          o.split_share == 8) &&
         o.pivot_cost >= 0 && o.pivot_cost <= 1000000;
}

css_status check_forced(const css_opts& o, int n, int k, cudaStream_t s) {
  if (o.n_forced <= 0) return CSS_OK;
  if (!o.forced || o.n_forced > k) return CSS_ERR_INVALID_ARG;
  std::vector<int32_t> h(o.n_forced);
  if (cudaMemcpyAsync(h.data(), o.forced, sizeof(int32_t) * o.n_forced, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return CSS_ERR_CUDA;
  std::vector<char> seen(n, 0);
  for (int32_t v : h) {
    if (v < 0 || v >= n || seen[v]) return CSS_ERR_INVALID_ARG;
    seen[v] = 1;
  }
  return CSS_OK;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// opts->test_unmet_wait: 1 -> the greedy kernel's barrier 2 (the first of
// the first iteration) waits for an arrival no CTA makes; 2 -> the
// tensor-core kernels wait on an mbarrier phase nothing completes.
constexpr int kStallBarrier = 2;
bool valid_test_hook(const css_opts& o) { return o.test_unmet_wait >= 0 && o.test_unmet_wait <= 2; }
int stall_barrier(const css_opts& o) { return o.test_unmet_wait == 1 ? kStallBarrier : 0; }
int stall_mbarrier(const css_opts& o) { return o.test_unmet_wait == 2 ? 1 : 0; }

// ---------------------------------------------------------- css_select ------
struct SelectLayout {
  Header h;
  UnitState s;
  void* C;
  double* partial;
  size_t bytes;
};

SelectLayout select_layout(void* ws, size_t cap, int dt, int64_t m, int64_t n, int32_t k, bool need_W) {
  WsCarver c(ws, cap);
  SelectLayout L{};
  carve_header(c, 1, L.h, n);
  carve_scores(c, (int)n, L.s);
  carve_rest(c, dt, (int)m, (int)n, k, 0, 0, need_W, L.s);
  // C = A A^T (m x m) first; for BF16 and FP32 input the tensor-core path
  // needs its BF16 parts and row-tile partials (and A's parts or aligned
  // copy) right behind it
  size_t cbytes = (size_t)m * c_ld(m, (int)accsize(dt)) * accsize(dt);
  if (dt != CSS_F64)
    cbytes = std::max(cbytes, tc::css_f0_scratch_bytes((int)m, (int)n, dt == CSS_F32 ? tc::kF0F32Staged : tc::kF0Bf16Staged));
  L.C = c.take<char>(cbytes);
  L.partial = c.take<double>(css_f0_partial_doubles(dt, (int)m, (int)n));
  L.bytes = c.off;
  return L;
}

struct GcssLayout {
  Header h;
  UnitState s;
  double* partial;
  void* tc_scratch;
  size_t bytes;
};

GcssLayout gcss_layout(void* ws, size_t cap, int dt, int64_t m, int64_t n, int64_t r, int32_t k,
                       bool need_W) {
  WsCarver c(ws, cap);
  GcssLayout L{};
  carve_header(c, 1, L.h, n);
  carve_scores(c, (int)n, L.s);
  carve_rest(c, dt, (int)m, (int)n, k, (int)r, 1, need_W, L.s);
  L.partial = c.take<double>(gcss_f0_partial_doubles(dt, (int)r, (int)n));
  L.tc_scratch = c.take<char>(tc::colnorm_scratch_bytes((int)m, (int)r));
  L.bytes = c.off;
  return L;
}

UnitDesc make_unit(const void* A, int dt, int64_t m, int64_t n, int64_t lda, int32_t k, int mode,
                   const void* T, int64_t ldt, int64_t r, const UnitState& s, double* W,
                   int32_t* sel, double* trace, int32_t* n_sel, const css_opts& o) {
  UnitDesc u{};
  u.A = A;
  u.lda = lda;
  u.m = (int)m;
  u.n = (int)n;
  u.k = k;
  u.mode = mode;
  u.T = T;
  u.ldt = ldt;
  u.r = (int)r;
  u.score_mode = o.score_mode;
  u.tau = tau_of(o, dt);
  u.f = s.f;
  u.g = s.g;
  u.thr = s.thr;
  u.selmask = s.selmask;
  u.Q = s.Q;
  u.Z = s.Z;
  u.W = W;
  u.qv = s.qv;
  u.ypv = s.ypv;
  u.e1 = s.e1;
  u.e = s.e;
  u.y = s.y;
  u.coef = s.coef;
  u.ups = s.ups;
  u.sel = sel;
  u.trace = trace;
  u.n_sel = n_sel;
  u.diag_argmax = o.diag_argmax;
  u.trace_ns = (unsigned long long*)o.trace_ns;
  u.diag_f = o.diag_f;
  u.diag_g = o.diag_g;
  u.forced = o.forced;
  u.n_forced = o.forced ? o.n_forced : 0;
  u.vec_ok = aligned16(A) && ((lda * (int64_t)esize(dt)) % 16 == 0);
  u.t_vec_ok = aligned16(T) && ((ldt * (int64_t)accsize(dt)) % 16 == 0);
  return u;
}

size_t host_out_bytes(int32_t k) {
  return align_up(align_up(sizeof(int32_t) * (k + 1), 8) + sizeof(double) * (k + 1));
}

// f_i^(0) = ||B^T a_i||^2 (Algorithm 3's initialisation): tcgen05 for BF16 A
// (B split into three BF16 parts), register-tiled SIMT otherwise.
cudaError_t gcss_f0(int dt, const void* A, int64_t lda, int64_t m, int64_t n, const void* B, int64_t ldb,
                    int64_t r, double* partial, void* tc_scratch, double* f, const Header& h,
                    const css_opts& o, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(h.aux_err, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  if (dt == CSS_BF16 && o.init_path != 1 && tc_scratch && tc::supported(A, lda, (int)m, (int)r))
    return tc::colnorms(A, lda, (int)m, (int)n, (const float*)B, ldb, (int)r, tc_scratch, f, h.aux_err,
                        o.spin_budget_ns ? o.spin_budget_ns : kDefaultSpinNs, s, stall_mbarrier(o));
  return gcss_f0_simt(dt, A, lda, (int)m, (int)n, B, ldb, (int)r, partial, f, s);
}

int team_ctas_for(int64_t n, int64_t m) {
  // enough CTAs to keep the column stream and the FP64 pivot work spread out
  int64_t a = (n + 127) / 128;
  int64_t b = (m + 15) / 16;
  return (int)std::max<int64_t>(1, std::max(a, b));
}

// RndGreedyCSS (Sec. 7): B = A Omega with Omega n x l drawn on the device,
// then Algorithm 3 for the target B.  Workspace: gcss_select's first (so that
// css_read_status reads its status), then B, then css_project_random's.
size_t randomized_parts(int dtype, int64_t m, int64_t n, int32_t l, size_t& g, size_t& bb) {
  g = align_up(gcss_layout(nullptr, (size_t)-1, dtype, m, n, l, l, true).bytes);
  bb = align_up((size_t)m * l * accsize(dtype));
  return g + bb + project_random_workspace_bytes(dtype, m, n, l);
}

}  // namespace

extern "C" {

void css_opts_default(css_opts* opts) {
  if (opts) *opts = defaults();
}

const char* css_status_string(css_status s) {
  switch (s) {
    case CSS_OK: return "CSS_OK";
    case CSS_RANK_EXHAUSTED: return "CSS_RANK_EXHAUSTED: fewer than k columns above the rank threshold";
    case CSS_ERR_INVALID_ARG: return "CSS_ERR_INVALID_ARG";
    case CSS_ERR_CUDA: return "CSS_ERR_CUDA: a CUDA runtime call failed";
    case CSS_ERR_NO_MEMORY: return "CSS_ERR_NO_MEMORY";
    case CSS_ERR_WORKSPACE: return "CSS_ERR_WORKSPACE: workspace missing, misaligned or too small";
    case CSS_ERR_TIMEOUT: return "CSS_ERR_TIMEOUT: a bounded device wait ran out";
    case CSS_ERR_NONFINITE: return "CSS_ERR_NONFINITE: input holds NaN or Inf";
    case CSS_ERR_UNSUPPORTED: return "CSS_ERR_UNSUPPORTED";
    case CSS_ERR_NOT_CONVERGED: return "CSS_ERR_NOT_CONVERGED: the eigenvalue iteration hit its sweep limit";
  }
  return "unknown css_status";
}

const char* css_version(void) { return "libcss 0.1 (sm_103a)"; }

size_t css_workspace_size(css_op op, css_dtype dtype, int64_t m, int64_t n, int64_t r, int32_t k,
                          int32_t k_block, const css_opts* opts) {
  (void)opts;
  if (op == CSS_OP_LOWRANK) {
    // m may be 0 here (U not requested); r is the embedding dimension l
    if (n <= 0 || n > (int64_t)INT32_MAX || r < 1 || r > 1024 || k < 1 || k > r) return 0;
    return lowrank_workspace_bytes(n, (int32_t)r, k);
  }
  if (!valid_dtype(dtype) || m <= 0 || n <= 0) return 0;
  switch (op) {
    case CSS_OP_SELECT:
    case CSS_OP_HOST_SELECT: {
      if (k <= 0) return 0;
      size_t b = select_layout(nullptr, (size_t)-1, dtype, m, n, k, true).bytes;
      return op == CSS_OP_HOST_SELECT ? b + host_out_bytes(k) : b;
    }
    case CSS_OP_GCSS:
      if (k <= 0 || r <= 0) return 0;
      return gcss_layout(nullptr, (size_t)-1, dtype, m, n, r, k, true).bytes;
    case CSS_OP_DISTRIBUTED:
      if (k <= 0 || r <= 0 || k_block <= 0) return 0;
      return distributed_workspace_bytes(dtype, m, n, r, k, k_block);
    case CSS_OP_PROJECT:
      if (r <= 0) return 0;
      return project_workspace_bytes(dtype, m, n, r);
    case CSS_OP_PROJECT_RANDOM:
      if (r <= 0) return 0;
      return project_random_workspace_bytes(dtype, m, n, r);
    case CSS_OP_RANDOMIZED: {
      if (k <= 0) return 0;
      size_t g = 0, bb = 0;
      return randomized_parts(dtype, m, n, k, g, bb);
    }
    case CSS_OP_BACKWARD:
      if (k <= 0) return 0;
      return backward_workspace_bytes(dtype, m, n, k);
    case CSS_OP_EMBED:
      if (k <= 0 || k > 1024 || k > m || k > n) return 0;
      return embed_workspace_bytes(m, k);
    default:
      break;
  }
  return 0;
}

}  // extern "C"

namespace {

// css_select; pipe: A's columns arrive in chunks (css_select_host).
css_status select_impl(const void* A, css_dtype dtype, int64_t m, int64_t n, int64_t lda, int32_t k,
                       int32_t* sel, double* trace, int32_t* n_sel, double* W, void* ws,
                       size_t ws_bytes, const css_opts* opts, css_stream_t stream, const tc::F0Pipe* pipe) {
  const css_opts o = opts ? *opts : defaults();
  cudaStream_t s = (cudaStream_t)stream;
  if (!A || !sel || !trace || !n_sel || !valid_dtype(dtype)) return CSS_ERR_INVALID_ARG;
  if (m < 1 || n < 1 || lda < m || k < 1 || k > kMaxK || k > m || k > n) return CSS_ERR_INVALID_ARG;
  if (n > (int64_t)INT32_MAX || m > (int64_t)INT32_MAX) return CSS_ERR_INVALID_ARG;
  if (o.score_mode != 0 && o.score_mode != 1) return CSS_ERR_INVALID_ARG;
  if (!valid_test_hook(o) || !valid_knobs(o)) return CSS_ERR_INVALID_ARG;
  if (!ws || ((uintptr_t)ws % kWsAlign) != 0) return CSS_ERR_WORKSPACE;
  SelectLayout L = select_layout(ws, ws_bytes, dtype, m, n, k, W == nullptr);
  if (L.bytes > ws_bytes) return CSS_ERR_WORKSPACE;
  if (!device_ok()) return CSS_ERR_UNSUPPORTED;
  css_status cs = check_forced(o, (int)n, k, s);
  if (cs != CSS_OK) return cs;
  PhaseTimer tm(o);
  tm.mark(0, s);
  if (cudaMemsetAsync(L.h.aux_err, 0, sizeof(int), s) != cudaSuccess) return CSS_ERR_CUDA;
  cudaError_t e;
  const unsigned long long spin = o.spin_budget_ns ? o.spin_budget_ns : kDefaultSpinNs;
  // the greedy iterations stream A; a BF16 A whose layout refuses 16-byte
  // loads is read from the aligned copy the initial scores made of it
  const void* As = A;
  long long ldas = lda;
  if (dtype != CSS_F64 && o.init_path != 1 && tc::supported_any()) {
    const int src = tc::f0_source(dtype == CSS_F32, A, lda, (int)m);
    e = tc::css_f0(A, lda, (int)m, (int)n, L.C, L.s.f, L.h.aux_err, spin, s, stall_mbarrier(o), src, pipe);
    tc::f0_staged_copy((int)m, (int)n, src, L.C, &As, &ldas);
  } else {
    e = cudaSuccess;
    for (int z = 0; pipe && z < pipe->chunks && e == cudaSuccess; ++z) e = cudaStreamWaitEvent(s, pipe->ready[z], 0);
    if (e == cudaSuccess)
      e = css_f0_simt(dtype, A, lda, (int)m, (int)n, L.C, c_ld(m, (int)accsize(dtype)), L.partial, L.s.f, s);
  }
  if (e != cudaSuccess) return cuda_status(e);
  tm.mark(1, s);
  std::vector<UnitDesc> units{make_unit(As, dtype, m, n, ldas, k, 0, L.C, c_ld(m, (int)accsize(dtype)), 0, L.s, W,
                                        sel, trace, n_sel, o)};
  const int tile = pick_tile(o, dtype, m, n);
  int gmax = o.grid_ctas > 0 ? o.grid_ctas : team_ctas_for(n, m);
  cs = launch_units(L.h, units, {1.0}, dtype, gmax, tile, o.spin_budget_ns, s, stall_barrier(o),
                    pick_split_share(o, dtype, m, n));
  if (cs != CSS_OK) return cs;
  tm.mark(2, s);
  if (o.basis && (e = export_basis(dtype, L.s.Q, (int)m, k, n_sel, o.basis, s)) != cudaSuccess)
    return cuda_status(e);
  cs = finish(L.h, o, s);
  tm.report(o);
  return cs;
}

// A copy stream and arrival events for css_select_host, one set per device,
// made on first use and kept for the life of the process.
constexpr int kMaxHostChunks = 32;
struct HostPipe {
  cudaStream_t copy = nullptr;
  cudaEvent_t start = nullptr;
  cudaEvent_t ready[kMaxHostChunks] = {};
  bool ok = false;
};
std::mutex g_pipe_mu;
HostPipe* host_pipe() {
  static HostPipe pipes[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(g_pipe_mu);
  HostPipe& p = pipes[dev];
  if (!p.ok) {
    bool good = cudaStreamCreateWithFlags(&p.copy, cudaStreamNonBlocking) == cudaSuccess &&
                cudaEventCreateWithFlags(&p.start, cudaEventDisableTiming) == cudaSuccess;
    for (int z = 0; good && z < kMaxHostChunks; ++z)
      good = cudaEventCreateWithFlags(&p.ready[z], cudaEventDisableTiming) == cudaSuccess;
    if (!good) return nullptr;
    p.ok = true;
  }
  return &p;
}

}  // namespace

extern "C" {

css_status css_select(const void* A, css_dtype dtype, int64_t m, int64_t n, int64_t lda, int32_t k,
                      int32_t* sel, double* trace, int32_t* n_sel, double* W, void* ws,
                      size_t ws_bytes, const css_opts* opts, css_stream_t stream) {
  return select_impl(A, dtype, m, n, lda, k, sel, trace, n_sel, W, ws, ws_bytes, opts, stream, nullptr);
}

css_status gcss_select(const void* A, css_dtype dtype, int64_t m, int64_t n, int64_t lda,
                       const void* B, int64_t r, int64_t ldb, int32_t k, int32_t* sel, double* trace,
                       int32_t* n_sel, double* W, void* ws, size_t ws_bytes, const css_opts* opts,
                       css_stream_t stream) {
  const css_opts o = opts ? *opts : defaults();
  cudaStream_t s = (cudaStream_t)stream;
  if (!A || !B || !sel || !trace || !n_sel || !valid_dtype(dtype)) return CSS_ERR_INVALID_ARG;
  if (m < 1 || n < 1 || r < 1 || lda < m || ldb < m || k < 1 || k > kMaxK || k > m || k > n)
    return CSS_ERR_INVALID_ARG;
  if (o.score_mode != 0 && o.score_mode != 1) return CSS_ERR_INVALID_ARG;
  if (!valid_test_hook(o) || !valid_knobs(o)) return CSS_ERR_INVALID_ARG;
  if (!ws || ((uintptr_t)ws % kWsAlign) != 0) return CSS_ERR_WORKSPACE;
  GcssLayout L = gcss_layout(ws, ws_bytes, dtype, m, n, r, k, W == nullptr);
  if (L.bytes > ws_bytes) return CSS_ERR_WORKSPACE;
  if (!device_ok()) return CSS_ERR_UNSUPPORTED;
  css_status cs = check_forced(o, (int)n, k, s);
  if (cs != CSS_OK) return cs;
  PhaseTimer tm(o);
  tm.mark(0, s);
  cudaError_t e = gcss_f0(dtype, A, lda, m, n, B, ldb, r, L.partial, L.tc_scratch, L.s.f, L.h, o, s);
  if (e != cudaSuccess) return cuda_status(e);
  tm.mark(1, s);
  std::vector<UnitDesc> units{make_unit(A, dtype, m, n, lda, k, 1, B, ldb, r, L.s, W, sel, trace,
                                        n_sel, o)};
  const int tile = pick_tile(o, dtype, m, n);
  int gmax = o.grid_ctas > 0 ? o.grid_ctas : team_ctas_for(n, m);
  cs = launch_units(L.h, units, {1.0}, dtype, gmax, tile, o.spin_budget_ns, s, stall_barrier(o),
                    pick_split_share(o, dtype, m, n));
  if (cs != CSS_OK) return cs;
  tm.mark(2, s);
  if (o.basis && (e = export_basis(dtype, L.s.Q, (int)m, k, n_sel, o.basis, s)) != cudaSuccess)
    return cuda_status(e);
  cs = finish(L.h, o, s);
  tm.report(o);
  return cs;
}

css_status css_select_randomized(const void* A, css_dtype dtype, int64_t m, int64_t n, int64_t lda, int32_t l,
                                 uint64_t seed, css_omega dist, int32_t* sel, double* trace, int32_t* n_sel,
                                 void* ws, size_t ws_bytes, const css_opts* opts, css_stream_t stream) {
  if (!A || !sel || !trace || !n_sel || !valid_dtype(dtype)) return CSS_ERR_INVALID_ARG;
  if (m < 1 || n < 1 || lda < m || l < 1 || l > kMaxK || l > m || l > n) return CSS_ERR_INVALID_ARG;
  if (!ws || ((uintptr_t)ws % kWsAlign) != 0) return CSS_ERR_WORKSPACE;
  size_t g = 0, bb = 0;
  const size_t need = randomized_parts(dtype, m, n, l, g, bb);
  if (ws_bytes < need) return CSS_ERR_WORKSPACE;
  css_opts po = opts ? *opts : defaults();
  po.sync = 0;            // the selection below reports the status
  po.timing_ms = nullptr;
  void* B = (char*)ws + g;
  css_status cs = css_project_random(A, dtype, m, n, lda, l, seed, dist, B, m, (char*)B + bb, ws_bytes - g - bb,
                                     &po, stream);
  if (cs != CSS_OK) return cs;
  return gcss_select(A, dtype, m, n, lda, B, l, m, l, sel, trace, n_sel, nullptr, ws, g, opts, stream);
}

css_status css_read_status(const void* ws, css_stream_t stream) {
  if (!ws) return CSS_ERR_WORKSPACE;
  DevStatus st{};
  int aux = 0;
  cudaError_t e = cudaMemcpyAsync(&st, ws, sizeof(st), cudaMemcpyDeviceToHost, (cudaStream_t)stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&aux, (const char*)ws + kAuxErrOffset, sizeof(int), cudaMemcpyDeviceToHost,
                        (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_status(e);
  if (aux != 0) return (css_status)aux;
  if (st.code != 0) return (css_status)st.code;
  return st.rank_exhausted ? CSS_RANK_EXHAUSTED : CSS_OK;
}

css_status css_select_host(const void* A_host, css_dtype dtype, int64_t m, int64_t n, int64_t lda,
                           int32_t k, int32_t* sel, double* trace, int32_t* n_sel, void* A_dev,
                           void* ws, size_t ws_bytes, const css_opts* opts, css_stream_t stream) {
  if (!A_host || !A_dev || !sel || !trace || !n_sel || !valid_dtype(dtype)) return CSS_ERR_INVALID_ARG;
  if (m < 1 || n < 1 || lda < m || k < 1) return CSS_ERR_INVALID_ARG;
  if (!ws || ((uintptr_t)ws % kWsAlign) != 0 || ws_bytes < kWsAlign) return CSS_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  // outputs live in the first 256-byte slot... too small for k; carve after the select workspace
  const size_t need = select_layout(nullptr, (size_t)-1, dtype, m, n, k, true).bytes;
  const size_t out_bytes = host_out_bytes(k);
  if (ws_bytes < need + out_bytes) return CSS_ERR_WORKSPACE;
  char* outs = (char*)ws + need;
  int32_t* d_sel = (int32_t*)outs;
  int32_t* d_nsel = d_sel + k;
  double* d_trace = (double*)(outs + align_up(sizeof(int32_t) * (k + 1), 8));
  css_opts o = opts ? *opts : defaults();
  o.sync = 1;
  // A goes over in column chunks on a copy stream, so that the initial
  // scores' C = A A^T works on the chunks already in while later ones are in
  // flight (host-to-device copies run at about 210 GB/s on this part, under
  // a thirtieth of HBM).  The chunks follow C's K chunks.
  const size_t col_bytes = (size_t)lda * esize(dtype);
  const int cols = std::max(1, tc::f0_chunk_cols((int)m, (int)n));
  const int chunks = (int)((n + cols - 1) / cols);
  HostPipe* hp = (dtype != CSS_F64 && chunks <= kMaxHostChunks) ? host_pipe() : nullptr;
  cudaError_t e;
  css_status cs;
  if (hp) {
    // the copy waits for the stream's earlier work on A_dev
    if ((e = cudaEventRecord(hp->start, s)) != cudaSuccess) return cuda_status(e);
    if ((e = cudaStreamWaitEvent(hp->copy, hp->start, 0)) != cudaSuccess) return cuda_status(e);
    for (int z = 0; z < chunks; ++z) {
      const int64_t c0 = (int64_t)z * cols, nc = std::min<int64_t>(cols, n - c0);
      if ((e = cudaMemcpyAsync((char*)A_dev + c0 * col_bytes, (const char*)A_host + c0 * col_bytes, nc * col_bytes,
                               cudaMemcpyHostToDevice, hp->copy)) != cudaSuccess ||
          (e = cudaEventRecord(hp->ready[z], hp->copy)) != cudaSuccess) {
        cudaStreamSynchronize(hp->copy);
        return cuda_status(e);
      }
    }
    const tc::F0Pipe pipe{hp->ready, chunks, cols};
    cs = select_impl(A_dev, dtype, m, n, lda, k, d_sel, d_trace, d_nsel, nullptr, ws, need, &o, stream, &pipe);
    if (cs < 0) {
      cudaStreamSynchronize(hp->copy);
      return cs;
    }
  } else {
    if ((e = cudaMemcpyAsync(A_dev, A_host, (size_t)lda * n * esize(dtype), cudaMemcpyHostToDevice, s)) != cudaSuccess)
      return cuda_status(e);
    cs = css_select(A_dev, dtype, m, n, lda, k, d_sel, d_trace, d_nsel, nullptr, ws, need, &o, stream);
    if (cs < 0) return cs;
  }
  e = cudaMemcpyAsync(sel, d_sel, sizeof(int32_t) * k, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(trace, d_trace, sizeof(double) * (k + 1), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(n_sel, d_nsel, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_status(e);
  return cs;
}

}  // extern "C"

// ----------------------------------------------- batched and distributed ----
namespace {

__global__ void gather_columns_kernel(const char* __restrict__ A, long long lda_bytes, int m_bytes,
                                      const int* __restrict__ ids, const int* __restrict__ count,
                                      char* __restrict__ A0, long long lda0_bytes) {
  const int U = *count;
  for (int j = blockIdx.y; j < U; j += gridDim.y) {
    const char* src = A + (long long)ids[j] * lda_bytes;
    char* dst = A0 + (long long)j * lda0_bytes;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < m_bytes; b += gridDim.x * blockDim.x)
      dst[b] = src[b];
  }
}

__global__ void gather_f_kernel(const double* __restrict__ f0, const int* __restrict__ ids,
                                const int* __restrict__ count, int umax, double* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < umax && j < *count) out[j] = f0[ids[j]];
}

// Final picks (indices into the union) -> global column ids; -1 past n_sel.
__global__ void map_sel_kernel(const int* __restrict__ local, const int* __restrict__ ids, int k,
                               const int* __restrict__ n_sel, int* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < k) out[j] = (j < *n_sel) ? ids[local[j]] : -1;
}

// Algorithm 4's reduce step, on the device: the union's first slot for each
// block (exclusive prefix sum of the blocks' pick counts, in block order),
// its size U written into the union unit's column count, and the block
// launch's rank-exhaustion count cleared (a block that picks fewer than
// l_block columns is not an error of the call; the union launch reports its
// own).  One block of 1024 threads; the status code is kept.
__global__ void union_scan_kernel(const int* __restrict__ bnsel, int nb, int* __restrict__ first,
                                  int* __restrict__ count, UnitDesc* __restrict__ unit, DevStatus* st) {
  __shared__ int s_carry;
  __shared__ int s_warp[32];
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int base = 0; base < nb; base += blockDim.x) {
    const int b = base + threadIdx.x;
    const int v = b < nb ? bnsel[b] : 0;
    int x = v;   // inclusive scan within the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[w] = x;
    __syncthreads();
    if (w == 0) {
      int t = s_warp[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += y;
      }
      s_warp[lane] = t;
    }
    __syncthreads();
    const int before = s_carry + (w > 0 ? s_warp[w - 1] : 0) + x - v;
    if (b < nb) first[b] = before;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) s_carry = before + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *count = s_carry;
    unit->n = s_carry;
    st->rank_exhausted = 0;
  }
}

// Block-local picks -> global column ids, in place in block_sel (-1 past a
// block's count), and the union's id list in block order, then selection
// order within each block.
__global__ void union_ids_kernel(int* __restrict__ bsel, const int* __restrict__ bnsel,
                                 const int* __restrict__ first, const long long* __restrict__ offs, int nb,
                                 int lb, int* __restrict__ ids) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)nb * lb) return;
  const int b = (int)(idx / lb), j = (int)(idx - (long long)b * lb);
  if (j < bnsel[b]) {
    const int g = (int)(offs[b] + bsel[idx]);
    bsel[idx] = g;
    ids[first[b] + j] = g;
  } else {
    bsel[idx] = -1;
  }
}

struct DistLayout {
  Header h;                // block launch (its status is the call's status)
  Header hu;               // union launch (descriptors only)
  UnitState sc;            // f, g, thr, selmask over all n columns
  double* f0_saved;
  std::vector<UnitState> blk;
  int* bsel;
  double* btrace;
  int* bnsel;
  double* partial;
  void* tc_scratch;
  long long* offs;         // block offsets on the device
  int* first;              // union slot of each block's first pick
  int* count;              // union size U
  // union step
  char* A0;
  int64_t lda0;
  int* ids;
  UnitState us;
  int* usel;
  size_t bytes;
};

DistLayout dist_layout(void* ws, size_t cap, int dt, int64_t m, int64_t n, int64_t r, int32_t k,
                       int32_t lb, const int64_t* offs, int nb) {
  WsCarver c(ws, cap);
  DistLayout L{};
  int64_t umax = 0;
  for (int b = 0; b < nb; ++b) {
    const int64_t w = offs ? offs[b + 1] - offs[b] : (n + nb - 1) / nb;
    umax += std::min<int64_t>(lb, w);
  }
  carve_header(c, std::max(nb, 1), L.h, n + 2 * (int64_t)nb);
  carve_header(c, 1, L.hu, umax);
  carve_scores(c, (int)n, L.sc);
  L.f0_saved = c.take<double>(n);
  L.blk.resize(nb);
  for (int b = 0; b < nb; ++b) {
    const int64_t w = offs ? offs[b + 1] - offs[b] : (n + nb - 1) / nb;
    const int kb = (int)std::min<int64_t>(lb, w);
    carve_rest(c, dt, (int)m, (int)w, kb, (int)r, 1, true, L.blk[b]);
  }
  L.bsel = c.take<int>((size_t)nb * lb);
  L.btrace = c.take<double>((size_t)nb * (lb + 1));
  L.bnsel = c.take<int>(nb);
  L.partial = c.take<double>(gcss_f0_partial_doubles(dt, (int)r, (int)n));
  L.tc_scratch = c.take<char>(tc::colnorm_scratch_bytes((int)m, (int)r));
  L.offs = c.take<long long>(nb + 1);
  L.first = c.take<int>(nb);
  L.count = c.take<int>(1);
  L.lda0 = (m + 7) / 8 * 8;
  L.A0 = c.take<char>((size_t)L.lda0 * umax * esize(dt));
  L.ids = c.take<int>(umax);
  carve_scores(c, (int)umax, L.us);
  carve_rest(c, dt, (int)m, (int)umax, std::max(1, k), (int)r, 1, true, L.us);
  L.usel = c.take<int>(std::max(1, k));
  L.bytes = c.off;
  return L;
}

// Host side of a prepared Algorithm 4 call, kept in the caller's
// css_distributed_plan: both launches' descriptors are in the workspace.
struct DistPlanImpl {
  uint64_t magic;
  void* ws;
  int dtype, nb, lb, k, umax, init_path, use_tc, pad_;
  const void* A;
  const void* B;
  long long lda, ldb;
  int64_t m, n, r;
  uint64_t spin_ns;
  int32_t* sel;
  int32_t* n_sel;
  int* bsel;
  int* bnsel;
  int* first;
  int* count;
  int* ids;
  long long* offs;
  double* f;
  double* f0_saved;
  double* uf;
  double* partial;
  void* tc_scratch;
  char* A0;
  long long lda0;
  int* usel;
  int* aux_err;
  UnitDesc* union_unit;
  DevStatus* st;
  LaunchInfo blocks;
  LaunchInfo uni;
};
constexpr uint64_t kDistMagic = 0x4353534450504c4eull;   // "CSSDPPLN"
static_assert(sizeof(DistPlanImpl) <= sizeof(css_distributed_plan), "css_distributed_plan too small");
static_assert(std::is_trivially_copyable<DistPlanImpl>::value, "the plan is copied as bytes");

css_status dist_prepare(const void* A, css_dtype dtype, int64_t m, int64_t n, int64_t lda, const void* B,
                        int64_t r, int64_t ldb, const int64_t* block_offsets, int32_t nblocks, int32_t l_block,
                        int32_t k, int32_t* sel, double* trace, int32_t* n_sel, int32_t* block_sel, void* ws,
                        size_t ws_bytes, const css_opts& o, DistPlanImpl& P, cudaStream_t s) {
  if (!A || !B || !sel || !trace || !n_sel || !block_offsets || !valid_dtype(dtype))
    return CSS_ERR_INVALID_ARG;
  if (m < 1 || n < 1 || r < 1 || lda < m || ldb < m || nblocks < 1 || l_block < 1 || k < 1 ||
      k > kMaxK || l_block > kMaxK || nblocks > kMaxCtas * 64)
    return CSS_ERR_INVALID_ARG;
  if (n > (int64_t)INT32_MAX || m > (int64_t)INT32_MAX) return CSS_ERR_INVALID_ARG;
  if (block_offsets[0] != 0 || block_offsets[nblocks] != n) return CSS_ERR_INVALID_ARG;
  int64_t umax = 0;
  for (int b = 0; b < nblocks; ++b) {
    if (block_offsets[b + 1] <= block_offsets[b]) return CSS_ERR_INVALID_ARG;
    umax += std::min<int64_t>(l_block, block_offsets[b + 1] - block_offsets[b]);
  }
  if (k > umax || k > m) return CSS_ERR_INVALID_ARG;
  if (o.n_forced || o.test_unmet_wait || !valid_knobs(o)) return CSS_ERR_INVALID_ARG;
  if (!ws || ((uintptr_t)ws % kWsAlign) != 0) return CSS_ERR_WORKSPACE;
  DistLayout L = dist_layout(ws, ws_bytes, dtype, m, n, r, k, l_block, block_offsets, nblocks);
  if (L.bytes > ws_bytes) return CSS_ERR_WORKSPACE;
  if (!device_ok()) return CSS_ERR_UNSUPPORTED;
  cudaError_t e;
  std::vector<long long> offs(block_offsets, block_offsets + nblocks + 1);
  if ((e = cudaMemcpyAsync(L.offs, offs.data(), sizeof(long long) * offs.size(), cudaMemcpyHostToDevice, s)) !=
      cudaSuccess)
    return cuda_status(e);
  int* bsel = block_sel ? block_sel : L.bsel;
  css_opts ob = o;
  ob.diag_argmax = nullptr;
  ob.diag_f = ob.diag_g = nullptr;
  ob.trace_ns = nullptr;
  ob.basis = nullptr;
  // map phase: one unit per block, all in one persistent launch
  std::vector<UnitDesc> units;
  std::vector<double> work;
  const double pivot_cost = pick_pivot_cost(o, dtype, m, n);
  const int share = pick_split_share(o, dtype, m, n);
  for (int b = 0; b < nblocks; ++b) {
    const int64_t off = block_offsets[b], w = block_offsets[b + 1] - off;
    const int kb = (int)std::min<int64_t>(l_block, w);
    UnitState st = L.blk[b];
    st.f = L.sc.f + off;
    st.g = L.sc.g + off;
    st.thr = L.sc.thr + off;
    st.selmask = L.sc.selmask + off;
    const void* Ab = (const char*)A + off * lda * (int64_t)esize(dtype);
    units.push_back(make_unit(Ab, dtype, m, w, lda, kb, 1, B, ldb, r, st, nullptr,
                              bsel + (size_t)b * l_block, L.btrace + (size_t)b * (l_block + 1),
                              L.bnsel + b, ob));
    // a block's cost: kb iterations, each a streaming pass over its w columns
    // plus the pivot, whose latency-bound cost is charged as a fixed number
    // of column-equivalents (default 1500, swept on the 2048 x 262144
    // workload with the blocks in the two-CTAs-per-SM shape: 100 / 300 / 700
    // / 1500 / 3000 gave the blocks' launch 34.8 / 27.8 / 26.6 / 24.8 / 27.9
    // ms; css_autotune_distributed tunes it)
    work.push_back((double)kb * ((double)w + pivot_cost));
  }
  const int tile = pick_tile(o, dtype, m, n);
  P = DistPlanImpl{};
  // the blocks run in the kernel's two-CTAs-per-SM shape: each block's team
  // of a few CTAs gets twice as many (measured on 2048 x 262144 BF16, 64
  // blocks: the blocks' launch 27.9 -> 26.3 ms; the single-problem and
  // batched launches are faster in the one-CTA shape)
  css_status cs = prepare_units(L.h, units, work, dtype, o.grid_ctas, tile, o.spin_budget_ns, s, P.blocks, 0,
                                share, kGreedyThreadsPaired);
  if (cs != CSS_OK) return cs;
  // reduce phase: the union unit is planned for its largest size; the union
  // scan writes its actual column count into the descriptor on the device
  const int ku = (int)std::min<int64_t>(k, umax);
  std::vector<UnitDesc> uu{make_unit(L.A0, dtype, m, umax, L.lda0, ku, 1, B, ldb, r, L.us, nullptr, L.usel,
                                     trace, n_sel, ob)};
  cs = prepare_units(L.hu, uu, {1.0}, dtype, o.grid_ctas > 0 ? o.grid_ctas : team_ctas_for(umax, m), tile,
                     o.spin_budget_ns, s, P.uni, 0, share);
  if (cs != CSS_OK) return cs;
  // the union launch reports into the block launch's status (kept, not reset)
  P.uni.L.st = L.h.st;
  P.uni.st = L.h.st;
  P.uni.reset_status = false;
  // the descriptors came from host vectors that end with this call
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_status(e);
  P.magic = kDistMagic;
  P.ws = ws;
  P.dtype = dtype;
  P.nb = nblocks;
  P.lb = l_block;
  P.k = k;
  P.umax = (int)umax;
  P.init_path = o.init_path;
  P.A = A;
  P.B = B;
  P.lda = lda;
  P.ldb = ldb;
  P.m = m;
  P.n = n;
  P.r = r;
  P.spin_ns = o.spin_budget_ns ? o.spin_budget_ns : kDefaultSpinNs;
  P.sel = sel;
  P.n_sel = n_sel;
  P.bsel = bsel;
  P.bnsel = L.bnsel;
  P.first = L.first;
  P.count = L.count;
  P.ids = L.ids;
  P.offs = L.offs;
  P.f = L.sc.f;
  P.f0_saved = L.f0_saved;
  P.uf = L.us.f;
  P.partial = L.partial;
  P.tc_scratch = L.tc_scratch;
  P.A0 = L.A0;
  P.lda0 = L.lda0;
  P.usel = L.usel;
  P.aux_err = L.h.aux_err;
  P.union_unit = L.hu.units;
  P.st = L.h.st;
  return CSS_OK;
}

// The whole of Algorithm 4 as device work on `s` (no host copy, no
// synchronisation): initial scores, the block launch, the union built on the
// device, the union launch and the mapping of its picks to global ids.
css_status dist_run(const DistPlanImpl& P, cudaStream_t s, PhaseTimer* tm = nullptr) {
  Header h{};
  h.aux_err = P.aux_err;
  css_opts o = defaults();
  o.init_path = P.init_path;
  o.spin_budget_ns = P.spin_ns;
  cudaError_t e;
  if (tm) tm->mark(0, s);
  if ((e = gcss_f0(P.dtype, P.A, P.lda, P.m, P.n, P.B, P.ldb, P.r, P.partial, P.tc_scratch, P.f, h, o, s)) !=
      cudaSuccess)
    return cuda_status(e);
  // f^(0) of every column, kept for the union step (it depends on a_i and B only)
  if ((e = cudaMemcpyAsync(P.f0_saved, P.f, sizeof(double) * P.n, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
    return cuda_status(e);
  if ((e = cudaMemsetAsync(P.bsel, 0xff, sizeof(int) * (size_t)P.nb * P.lb, s)) != cudaSuccess)
    return cuda_status(e);
  if (tm) tm->mark(1, s);
  css_status cs = start_units(P.blocks, s);
  if (cs != CSS_OK) return cs;
  if (tm) tm->mark(2, s);
  union_scan_kernel<<<1, 1024, 0, s>>>(P.bnsel, P.nb, P.first, P.count, P.union_unit, P.st);
  const long long tot = (long long)P.nb * P.lb;
  union_ids_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(P.bsel, P.bnsel, P.first, P.offs, P.nb, P.lb,
                                                                 P.ids);
  {
    const int es = (int)esize(P.dtype);
    dim3 grid((unsigned)std::max<int64_t>(1, std::min<int64_t>(8, (P.m * es + 1023) / 1024)),
              (unsigned)std::min(P.umax, 65535));
    gather_columns_kernel<<<grid, 256, 0, s>>>((const char*)P.A, P.lda * es, (int)(P.m * es), P.ids, P.count,
                                               P.A0, P.lda0 * es);
    gather_f_kernel<<<(P.umax + 255) / 256, 256, 0, s>>>(P.f0_saved, P.ids, P.count, P.umax, P.uf);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e);
  }
  cs = start_units(P.uni, s);
  if (cs != CSS_OK) return cs;
  map_sel_kernel<<<(P.k + 255) / 256, 256, 0, s>>>(P.usel, P.ids, P.k, P.n_sel, P.sel);
  return cuda_status(cudaGetLastError());
}

}  // namespace

size_t distributed_workspace_bytes(int dtype, int64_t m, int64_t n, int64_t r, int32_t k,
                                   int32_t k_block) {
  // sized for the worst case of the block partition: blocks of at least
  // k_block columns, each selecting k_block
  const int nb = (int)std::max<int64_t>(1, n / std::max(1, k_block));
  return dist_layout(nullptr, (size_t)-1, dtype, m, n, r, k, k_block, nullptr, nb).bytes;
}

extern "C" {

size_t gcss_distributed_workspace_size(css_dtype dtype, int64_t m, int64_t n, int64_t r,
                                       const int64_t* block_offsets, int32_t nblocks,
                                       int32_t l_block, int32_t k) {
  if (!valid_dtype(dtype) || !block_offsets || nblocks < 1 || m < 1 || n < 1 || r < 1 ||
      l_block < 1 || k < 1)
    return 0;
  if (block_offsets[0] != 0 || block_offsets[nblocks] != n) return 0;
  for (int b = 0; b < nblocks; ++b)
    if (block_offsets[b + 1] <= block_offsets[b]) return 0;
  return dist_layout(nullptr, (size_t)-1, dtype, m, n, r, k, l_block, block_offsets, nblocks).bytes;
}

css_status gcss_distributed(const void* A, css_dtype dtype, int64_t m, int64_t n, int64_t lda,
                            const void* B, int64_t r, int64_t ldb, const int64_t* block_offsets,
                            int32_t nblocks, int32_t l_block, int32_t k, int32_t* sel,
                            double* trace, int32_t* n_sel, int32_t* block_sel, void* ws,
                            size_t ws_bytes, const css_opts* opts, css_stream_t stream) {
  const css_opts o = opts ? *opts : defaults();
  cudaStream_t s = (cudaStream_t)stream;
  DistPlanImpl P;
  css_status cs = dist_prepare(A, dtype, m, n, lda, B, r, ldb, block_offsets, nblocks, l_block, k, sel, trace,
                               n_sel, block_sel, ws, ws_bytes, o, P, s);
  if (cs != CSS_OK) return cs;
  PhaseTimer tm(o);
  cs = dist_run(P, s, &tm);
  if (cs != CSS_OK) return cs;
  Header h{};
  h.st = P.st;
  h.aux_err = P.aux_err;
  cs = finish(h, o, s);
  tm.report(o);
  return cs;
}

css_status gcss_distributed_prepare(const void* A, css_dtype dtype, int64_t m, int64_t n, int64_t lda,
                                    const void* B, int64_t r, int64_t ldb, const int64_t* block_offsets,
                                    int32_t nblocks, int32_t l_block, int32_t k, int32_t* sel, double* trace,
                                    int32_t* n_sel, int32_t* block_sel, void* ws, size_t ws_bytes,
                                    const css_opts* opts, css_distributed_plan* plan, css_stream_t stream) {
  if (!plan) return CSS_ERR_INVALID_ARG;
  const css_opts o = opts ? *opts : defaults();
  std::memset(plan, 0, sizeof(*plan));
  DistPlanImpl P;
  css_status cs = dist_prepare(A, dtype, m, n, lda, B, r, ldb, block_offsets, nblocks, l_block, k, sel, trace,
                               n_sel, block_sel, ws, ws_bytes, o, P, (cudaStream_t)stream);
  if (cs != CSS_OK) return cs;
  std::memcpy(static_cast<void*>(plan), static_cast<const void*>(&P), sizeof(P));
  return CSS_OK;
}

css_status gcss_distributed_run(const css_distributed_plan* plan, void* ws, css_stream_t stream) {
  if (!plan) return CSS_ERR_INVALID_ARG;
  DistPlanImpl P;
  std::memcpy(static_cast<void*>(&P), static_cast<const void*>(plan), sizeof(P));
  if (P.magic != kDistMagic || P.ws != ws || !ws) return CSS_ERR_INVALID_ARG;
  return dist_run(P, (cudaStream_t)stream);
}

}  // extern "C"

namespace {

struct BatchLayout {
  Header h;
  std::vector<UnitState> st;
  std::vector<void*> C;
  std::vector<double*> partial;
  F0Item* items;   // initial-score work list, count entries
  int* starts;     // 3 * (count + 1) first blocks (css_f0_grouped_starts)
  void* gdesc;     // tensor-core path: descriptors and tile lists of the group
  size_t bytes;
};

BatchLayout batch_layout(void* ws, size_t cap, const css_problem* probs, int count, int dt) {
  WsCarver c(ws, cap);
  BatchLayout L{};
  int64_t cols = 0;
  for (int i = 0; i < count; ++i) cols += probs[i].n + 2;   // + 2: ceil of each half
  carve_header(c, std::max(count, 1), L.h, cols);
  L.st.resize(count);
  L.C.resize(count);
  L.partial.resize(count);
  for (int i = 0; i < count; ++i) {
    const css_problem& p = probs[i];
    carve_scores(c, (int)p.n, L.st[i]);
    carve_rest(c, dt, (int)p.m, (int)p.n, p.k, 0, 0, p.W == nullptr, L.st[i]);
    // C first; for BF16 and FP32 input the tensor-core path's scratch
    // (tc::css_f0_scratch_bytes) starts with C
    size_t cbytes = (size_t)p.m * c_ld(p.m, (int)accsize(dt)) * accsize(dt);
    if (dt != CSS_F64)
      cbytes = std::max(cbytes, tc::css_f0_scratch_bytes((int)p.m, (int)p.n,
                                                         dt == CSS_F32 ? tc::kF0F32Staged : tc::kF0Bf16Staged));
    L.C[i] = c.take<char>(cbytes);
    L.partial[i] = c.take<double>(css_f0_partial_doubles(dt, (int)p.m, (int)p.n));
  }
  L.items = c.take<F0Item>(std::max(count, 1));
  L.starts = c.take<int>(3 * (std::max(count, 1) + 1));
  if (dt != CSS_F64) {
    std::vector<int> ms(count), ns(count);
    for (int i = 0; i < count; ++i) {
      ms[i] = (int)probs[i].m;
      ns[i] = (int)probs[i].n;
    }
    L.gdesc = c.take<char>(tc::group_f0_desc_bytes(ms.data(), ns.data(), count, dt == CSS_F32));
  }
  L.bytes = c.off;
  return L;
}

// Host side of a prepared batch, kept in the caller's css_batched_plan.
struct BatchedPlanImpl {
  uint64_t magic;
  void* ws;
  int count, dtype;
  int simt_count;  // problems whose initial scores take the SIMT kernels (items)
  int use_tc;      // the others: grouped tensor-core launches (tcg)
  tc::GroupF0 tcg;
  F0Grid grid;
  const F0Item* items;
  const int* starts;
  int* aux_err;
  LaunchInfo info;
};
constexpr uint64_t kPlanMagic = 0x43535342504c414eull;   // "CSSBPLAN"
static_assert(sizeof(BatchedPlanImpl) <= sizeof(css_batched_plan), "css_batched_plan too small");
static_assert(std::is_trivially_copyable<BatchedPlanImpl>::value, "the plan is copied as bytes");

css_status batched_prepare(const css_problem* probs, int32_t count, css_dtype dtype, void* ws,
                           size_t ws_bytes, const css_opts& o, BatchedPlanImpl& P, cudaStream_t s) {
  if (!probs || count < 1 || !valid_dtype(dtype)) return CSS_ERR_INVALID_ARG;
  if (o.n_forced || o.diag_argmax || o.diag_f || o.trace_ns || o.test_unmet_wait || !valid_knobs(o))
    return CSS_ERR_INVALID_ARG;
  for (int i = 0; i < count; ++i) {
    const css_problem& p = probs[i];
    if (!p.A || !p.sel || !p.trace || !p.n_sel) return CSS_ERR_INVALID_ARG;
    if (p.m < 1 || p.n < 1 || p.lda < p.m || p.k < 1 || p.k > kMaxK || p.k > p.m || p.k > p.n)
      return CSS_ERR_INVALID_ARG;
  }
  if (!ws || ((uintptr_t)ws % kWsAlign) != 0) return CSS_ERR_WORKSPACE;
  BatchLayout L = batch_layout(ws, ws_bytes, probs, count, dtype);
  if (L.bytes > ws_bytes) return CSS_ERR_WORKSPACE;
  if (!device_ok()) return CSS_ERR_UNSUPPORTED;
  std::vector<UnitDesc> units;
  std::vector<double> work;
  // initial scores: tensor cores for BF16 / FP32 problems (one grouped
  // launch per phase), the SIMT kernels for FP64 or with init_path = 1
  std::vector<F0Item> items;
  std::vector<int> ms, ns, starts;
  std::vector<const void*> tA;
  std::vector<long long> tlda;
  std::vector<int> tm_, tn;
  std::vector<void*> tscr;
  std::vector<double*> tf;
  std::vector<int> tsrc;
  const bool tc_ok = dtype != CSS_F64 && o.init_path != 1 && count <= 65535 && tc::supported_any();
  for (int i = 0; i < count; ++i) {
    const css_problem& p = probs[i];
    const void* As = p.A;   // see css_select: the aligned copy of a BF16 A, if one is made
    long long ldas = p.lda;
    if (tc_ok) {
      tsrc.push_back(tc::f0_source(dtype == CSS_F32, p.A, p.lda, (int)p.m));
      tc::f0_staged_copy((int)p.m, (int)p.n, tsrc.back(), L.C[i], &As, &ldas);
      tA.push_back(p.A);
      tlda.push_back(p.lda);
      tm_.push_back((int)p.m);
      tn.push_back((int)p.n);
      tscr.push_back(L.C[i]);
      tf.push_back(L.st[i].f);
    } else {
      items.push_back(F0Item{p.A, p.lda, (int)p.m, (int)p.n, L.C[i], c_ld(p.m, (int)accsize(dtype)), L.partial[i],
                             L.st[i].f});
      ms.push_back((int)p.m);
      ns.push_back((int)p.n);
    }
    units.push_back(make_unit(As, dtype, p.m, p.n, ldas, p.k, 0, L.C[i], c_ld(p.m, (int)accsize(dtype)), 0,
                              L.st[i], p.W, p.sel, p.trace, p.n_sel, o));
    work.push_back((double)p.k * p.m * p.n + 4.0 * p.m * p.k * p.k);
  }
  P = BatchedPlanImpl{};
  P.simt_count = (int)items.size();
  cudaError_t e;
  if (P.simt_count > 0) {
    starts.resize(3 * (items.size() + 1));
    P.grid = css_f0_grouped_starts(dtype, ms.data(), ns.data(), P.simt_count, starts.data());
    if ((e = cudaMemcpyAsync(L.items, items.data(), sizeof(F0Item) * items.size(), cudaMemcpyHostToDevice, s)) !=
        cudaSuccess)
      return cuda_status(e);
    if ((e = cudaMemcpyAsync(L.starts, starts.data(), sizeof(int) * starts.size(), cudaMemcpyHostToDevice, s)) !=
        cudaSuccess)
      return cuda_status(e);
  }
  if (!tA.empty()) {
    const unsigned long long spin = o.spin_budget_ns ? o.spin_budget_ns : kDefaultSpinNs;
    if ((e = tc::group_f0_prepare((int)tA.size(), tA.data(), tlda.data(), tm_.data(), tn.data(), tscr.data(),
                                  tf.data(), tsrc.data(), L.gdesc, L.h.aux_err, spin, &P.tcg, s)) !=
        cudaSuccess)
      return cuda_status(e);
    P.use_tc = 1;
  }
  int64_t m_big = 0, n_big = 0;
  for (int i = 0; i < count; ++i)
    if (probs[i].m * probs[i].n > m_big * n_big) { m_big = probs[i].m; n_big = probs[i].n; }
  const int tile = pick_tile(o, dtype, m_big, n_big);
  css_status cs = prepare_units(L.h, units, work, dtype, o.grid_ctas, tile, o.spin_budget_ns, s, P.info, 0,
                                pick_split_share(o, dtype, m_big, n_big));
  if (cs != CSS_OK) return cs;
  // the descriptors come from host vectors that end with this call
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_status(e);
  P.magic = kPlanMagic;
  P.ws = ws;
  P.count = count;
  P.dtype = dtype;
  P.items = L.items;
  P.starts = L.starts;
  P.aux_err = L.h.aux_err;
  return CSS_OK;
}

// Initial scores of every problem (grouped launches: SIMT and/or tensor
// cores), then the persistent launch: device work only, so the sequence can
// be captured.
css_status batched_run(const BatchedPlanImpl& P, cudaStream_t s, PhaseTimer* tm) {
  if (cudaMemsetAsync(P.aux_err, 0, sizeof(int), s) != cudaSuccess) return CSS_ERR_CUDA;
  if (tm) tm->mark(0, s);
  cudaError_t e;
  if (P.simt_count > 0 && (e = css_f0_grouped(P.dtype, P.items, P.starts, P.grid, P.simt_count, s)) != cudaSuccess)
    return cuda_status(e);
  if (P.use_tc && (e = tc::group_f0_run(P.tcg, s)) != cudaSuccess) return cuda_status(e);
  if (tm) tm->mark(1, s);
  css_status cs = start_units(P.info, s);
  if (tm) tm->mark(2, s);
  return cs;
}

}  // namespace

extern "C" {

size_t css_batched_workspace_size(const css_problem* probs, int32_t count, css_dtype dtype,
                                  const css_opts* opts) {
  (void)opts;
  if (!probs || count < 1 || !valid_dtype(dtype)) return 0;
  for (int i = 0; i < count; ++i)
    if (probs[i].m < 1 || probs[i].n < 1 || probs[i].k < 1) return 0;
  return batch_layout(nullptr, (size_t)-1, probs, count, dtype).bytes;
}

css_status css_select_batched(const css_problem* probs, int32_t count, css_dtype dtype, void* ws,
                              size_t ws_bytes, const css_opts* opts, css_stream_t stream) {
  const css_opts o = opts ? *opts : defaults();
  cudaStream_t s = (cudaStream_t)stream;
  BatchedPlanImpl P;
  css_status cs = batched_prepare(probs, count, dtype, ws, ws_bytes, o, P, s);
  if (cs != CSS_OK) return cs;
  PhaseTimer tm(o);
  cs = batched_run(P, s, &tm);
  if (cs != CSS_OK) return cs;
  cs = finish(batch_layout(ws, ws_bytes, probs, count, dtype).h, o, s);
  tm.report(o);
  return cs;
}

css_status css_select_batched_prepare(const css_problem* probs, int32_t count, css_dtype dtype,
                                      void* workspace, size_t workspace_bytes, const css_opts* opts,
                                      css_batched_plan* plan, css_stream_t stream) {
  if (!plan) return CSS_ERR_INVALID_ARG;
  const css_opts o = opts ? *opts : defaults();
  std::memset(plan, 0, sizeof(*plan));
  BatchedPlanImpl P;
  css_status cs = batched_prepare(probs, count, dtype, workspace, workspace_bytes, o, P,
                                  (cudaStream_t)stream);
  if (cs != CSS_OK) return cs;
  std::memcpy(static_cast<void*>(plan), static_cast<const void*>(&P), sizeof(P));
  return CSS_OK;
}

css_status css_select_batched_run(const css_batched_plan* plan, void* workspace, css_stream_t stream) {
  if (!plan) return CSS_ERR_INVALID_ARG;
  BatchedPlanImpl P;
  std::memcpy(static_cast<void*>(&P), static_cast<const void*>(plan), sizeof(P));
  if (P.magic != kPlanMagic || P.ws != workspace || !workspace) return CSS_ERR_INVALID_ARG;
  return batched_run(P, (cudaStream_t)stream, nullptr);
}

}  // extern "C"
