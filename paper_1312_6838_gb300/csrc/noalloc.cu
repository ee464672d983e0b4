// css_select_noalloc: greedy CSS with its scratch memory in a fixed device
// array owned by the library, for callers that cannot allocate device memory.
//
// Such callers include services whose device memory is fully pre-reserved by
// the host application (every byte belongs to its own pool, so a cudaMalloc
// from a library would fail or steal from it), plugins whose host framework
// forbids allocation calls, and latency-sensitive code that must not call
// cudaMalloc/cudaFree because those calls can synchronise the whole device.
// They pass A and the output buffers; the workspace that css_select would
// take from the caller lives in g_css_scratch below.
#include <mutex>

#include "css_common.cuh"

namespace {

// One copy per device that loads the library; it stays allocated until the
// process exits.  Size: CSS_NOALLOC_SCRATCH_BYTES (include/css.h).
static __device__ __align__(256) unsigned char g_css_scratch[CSS_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_ptr[kMaxDevices] = {nullptr};

// Device address of g_css_scratch on the current device.  The host-side
// symbol is only a stand-in: the address must come from
// cudaGetSymbolAddress, once per device, with that device current.  The
// address is kept for the life of the process, so a device reset after the
// first call is not supported.
css_status scratch_for_current_device(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CSS_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return CSS_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_css_scratch) != cudaSuccess || !p) return CSS_ERR_CUDA;
    g_ptr[dev] = p;
  }
  *out = g_ptr[dev];
  return CSS_OK;
}

}  // namespace

extern "C" css_status css_select_noalloc(const void* A, css_dtype dtype, int64_t m, int64_t n,
                                         int64_t lda, int32_t k, int32_t* sel, double* trace,
                                         int32_t* n_sel, double* W, const css_opts* opts,
                                         css_stream_t stream) {
  css_opts o;
  css_opts_default(&o);
  if (opts) o = *opts;
  // options that would make the call allocate (events) are not taken here;
  // the device status sits in the library's array, which the caller cannot
  // pass to css_read_status, so the call always synchronises and reports it
  if (o.timing_ms || !o.sync) return CSS_ERR_INVALID_ARG;
  const size_t need = css_workspace_size(CSS_OP_SELECT, dtype, m, n, 0, k, 0, &o);
  if (need == 0) return CSS_ERR_INVALID_ARG;
  if (need > (size_t)CSS_NOALLOC_SCRATCH_BYTES) return CSS_ERR_WORKSPACE;
  void* ws = nullptr;
  css_status s = scratch_for_current_device(&ws);
  if (s != CSS_OK) return s;
  // css_select writes every scratch word it reads before reading it (status
  // block, barrier counters and descriptors are rewritten per call), so the
  // previous call's contents need no clearing.
  return css_select(A, dtype, m, n, lda, k, sel, trace, n_sel, W, ws,
                    (size_t)CSS_NOALLOC_SCRATCH_BYTES, &o, stream);
}
