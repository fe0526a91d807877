// The streaming kernels for packed site strides (every layout), the failure-path self test and
// the default launch configurations; the kernels themselves are in su3_stream.cuh.
#include "su3_stream.cuh"

namespace su3 {

// ---- failure-path self test ------------------------------------------------------------------

// One CTA waits on an mbarrier that expects two arrivals but gets one, with a short limit; the
// bounded wait gives up, the kernel records the timeout and returns.
__global__ void su3_selftest_wait_kernel(unsigned* status, unsigned long long limit_ns) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 2);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bar)) : "memory");
  const bool ok = mbar_wait_bounded(&bar, 0u, limit_ns);
  if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicOr(status, kDevErrTimeout);
}

su3_status launch_selftest_wait(int limit_ms, const LaunchCtx& ctx) {
  su3_selftest_wait_kernel<<<1, 32, 0, ctx.stream>>>(ctx.status, (unsigned long long)limit_ms * 1000000ull);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    *ctx.err = std::string("su3_selftest_wait_kernel launch: ") + cudaGetErrorString(e);
    return SU3_ERR_CUDA;
  }
  ++*ctx.launches;
  return SU3_OK;
}

// ---- host launchers -----------------------------------------------------------------------------

LaunchCfg default_cfg(const Form& f) {
  LaunchCfg c;
  if (f.layout == SU3_LAYOUT_AOS) {
    c.block = 128;
    // ~18 KB per tile for FP64 full sites, ~9-18 KB for the narrower forms
    const int64_t site_in = f.a_stride;
    int ts = (int)std::max<int64_t>(32, std::min<int64_t>(128, 18432 / std::max<int64_t>(site_in, 1)));
    c.tile_sites = ts;
    c.stages = 4;
    c.ctas_per_sm = 2;
  } else {
    c.block = 256;
    c.tile_sites = f.dtype == SU3_F64 ? 1 : f.dtype == SU3_F32 ? 2 : 4;  // links per thread
    c.stages = 0;
    c.ctas_per_sm = 4;
  }
  c.native_permille = f.arith == SU3_ARITH_HYBRID ? 125 : 0;
  if (f.arith == SU3_ARITH_HYBRID) {
    c.block = 256;  // 8 warps, one of them native
    if (f.layout == SU3_LAYOUT_AOS) {
      c.tile_sites = 64;  // 256 links: one per thread and tile
      c.stages = 3;       // two such CTAs fit in one SM's shared memory
    }
  }
  return c;
}

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

su3_status encode_2d(CUtensorMap* m, const void* base, long long inner, long long rows, long long pitch,
                     long long box_inner, long long box_rows, const LaunchCtx& ctx) {
  const EncodeTiledFn enc = encode_tiled();
  if (!enc) {
    *ctx.err = "cuTensorMapEncodeTiled is not available from the CUDA driver";
    return SU3_ERR_CUDA;
  }
  const cuuint64_t dim[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
  const cuuint64_t stride[1] = {(cuuint64_t)pitch};
  const cuuint32_t box[2] = {(cuuint32_t)box_inner, (cuuint32_t)box_rows};
  const cuuint32_t estride[2] = {1, 1};
  const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<void*>(base), dim, stride, box, estride,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    *ctx.err = "cuTensorMapEncodeTiled failed (error " + std::to_string((int)r) + ")";
    return SU3_ERR_CUDA;
  }
  return SU3_OK;
}

// AOS arrays whose a or c sites are wider than their links go to the padded kernels.
static bool padded_sites(const Form& f, long long link_in, long long link_out) {
  return f.layout == SU3_LAYOUT_AOS && (f.a_stride != 4 * link_in || f.c_stride != 4 * link_out);
}

su3_status launch_mult(const Form& f, const LaunchCfg& cfg, const void* a, const double* b, void* c,
                       const LaunchCtx& ctx) {
  if (padded_sites(f, link_bytes(f.dtype, f.repr_in), link_bytes(f.dtype, f.repr_out)))
    return launch_mult_padded(f, cfg, a, b, c, ctx);
  return mult_dispatch<false>(f, cfg, a, b, c, ctx);
}

su3_status launch_adjacent(int which, const Form& f, const LaunchCfg& cfg, const void* a, const double* bv, void* c,
                           const LaunchCtx& ctx) {
  // output link: a 3x3 matrix (a^dagger b) or a colour vector of 3 complex numbers (a v, a^dagger v)
  const long long out = which == 0 ? link_bytes(f.dtype, SU3_REPR_FULL18) : 3 * 2 * real_bytes(f.dtype);
  if (padded_sites(f, link_bytes(f.dtype, f.repr_in), out)) return launch_adjacent_padded(which, f, cfg, a, bv, c, ctx);
  return adjacent_dispatch<false>(which, f, cfg, a, bv, c, ctx);
}

}  // namespace su3
