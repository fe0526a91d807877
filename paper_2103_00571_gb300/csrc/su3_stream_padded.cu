// The staged AOS kernels for arrays whose sites are wider than their links (the paper's 640-byte
// FP64 Site and any other 16-byte multiple): a and c move as 2-D tensors through the TMA engine,
// so the bytes after each site's links are neither read nor written. Compiled apart from the
// packed-stride kernels so that the two halves build in parallel.
#include "su3_stream.cuh"

namespace su3 {

su3_status launch_mult_padded(const Form& f, const LaunchCfg& cfg, const void* a, const double* b, void* c,
                              const LaunchCtx& ctx) {
  return mult_dispatch<true>(f, cfg, a, b, c, ctx);
}

su3_status launch_adjacent_padded(int which, const Form& f, const LaunchCfg& cfg, const void* a, const double* bv,
                                  void* c, const LaunchCtx& ctx) {
  return adjacent_dispatch<true>(which, f, cfg, a, bv, c, ctx);
}

}  // namespace su3
