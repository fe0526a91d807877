// The staged AOS kernels for arrays whose sites are wider than their links (the paper's 640-byte
// FP64 Site and any other 16-byte multiple): a and c move as 2-D tensors through the TMA engine,
// so the bytes after each site's links are neither read nor written. Compiled apart from the
// packed-stride kernels so that the two halves build in parallel.
#include "su3_stream.cuh"

namespace su3 {

// cuTensorMapEncodeTiled, reached through the runtime's driver entry point (no link to libcuda).
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_tiled() {
  static const EncodeTiledFn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return (EncodeTiledFn) nullptr;
    return reinterpret_cast<EncodeTiledFn>(f);
  }();
  return fn;
}

// An AOS array as a 2-D tensor for the TMA engine: n_sites rows `stride` bytes apart, each row the
// site's `row_bytes` of links as 8-byte elements (the bytes after the links lie outside the tensor,
// so no copy reads or writes them); a box is `rows` whole rows.
su3_status encode_sites(CUtensorMap* m, const void* base, long long n_sites, long long stride, long long row_bytes,
                        long long rows, const LaunchCtx& ctx) {
  const EncodeTiledFn enc = encode_tiled();
  if (!enc) {
    *ctx.err = "cuTensorMapEncodeTiled is not available from the CUDA driver";
    return SU3_ERR_CUDA;
  }
  const cuuint64_t dim[2] = {(cuuint64_t)(row_bytes / 8), (cuuint64_t)n_sites};
  const cuuint64_t pitch[1] = {(cuuint64_t)stride};
  const cuuint32_t box[2] = {(cuuint32_t)(row_bytes / 8), (cuuint32_t)rows};
  const cuuint32_t estride[2] = {1, 1};
  const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<void*>(base), dim, pitch, box, estride,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    *ctx.err = "cuTensorMapEncodeTiled failed (error " + std::to_string((int)r) + ")";
    return SU3_ERR_CUDA;
  }
  return SU3_OK;
}

su3_status launch_mult_padded(const Form& f, const LaunchCfg& cfg, const void* a, const double* b, void* c,
                              const LaunchCtx& ctx) {
  return mult_dispatch<true>(f, cfg, a, b, c, ctx);
}

su3_status launch_adjacent_padded(int which, const Form& f, const LaunchCfg& cfg, const void* a, const double* bv,
                                  void* c, const LaunchCtx& ctx) {
  return adjacent_dispatch<true>(which, f, cfg, a, bv, c, ctx);
}

}  // namespace su3
