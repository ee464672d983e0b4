// Adjoint of the reconstruction error at a fixed selected set.
#include "backward.cuh"

size_t backward_workspace_bytes(int dtype, int64_t m, int64_t n, int32_t k) {
  (void)dtype; (void)m; (void)n; (void)k;
  return css::kStatusBytes;
}

extern "C" css_status css_residual_backward(const void* A, css_dtype dtype, int64_t m, int64_t n,
                                            int64_t lda, const int32_t* sel, int32_t k,
                                            double grad_out, void* dA, int64_t ldda, double* loss,
                                            void* ws, size_t ws_bytes, const css_opts* opts,
                                            css_stream_t stream) {
  (void)A; (void)dtype; (void)m; (void)n; (void)lda; (void)sel; (void)k; (void)grad_out;
  (void)dA; (void)ldda; (void)loss; (void)ws; (void)ws_bytes; (void)opts; (void)stream;
  return CSS_ERR_UNSUPPORTED;
}
