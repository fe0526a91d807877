// The SU3_Bench link multiply (arXiv 2103.00571, §Background "SU3_Bench") with a and c left in
// host memory: the kernel itself streams a in and c out over the host link (NVLink-C2C on GB300),
// with no staging copy in HBM.
//
// The host link is the bound here (measured on GB300: about 211 GB/s host-to-device, 194 GB/s
// device-to-host and 343 GB/s both ways at once, the same for the copy engines and for loads and
// stores issued by the SMs), and even the FP64-pipe-bound FP64 kernel computes five times faster
// than that. So the design keeps every byte moving once over the link and nothing else:
//  * each warp owns a shared-memory slot of 8 sites and walks tiles of 8 sites;
//  * its lanes load the tile's link bytes with coalesced 16-byte loads straight from host memory
//    (no bulk copies: they only ever touch device memory in this library), each lane multiplies
//    one link in the slot with the same per-link op as the HBM kernels, and the lanes write the
//    result links back to host memory with coalesced 16-byte streaming stores;
//  * warps are independent (no CTA barrier after b is staged), so many tiles' loads are in flight.
// AOS only, any site stride (pad bytes of a site are neither read nor written).
#include <cuda_runtime.h>

#include <algorithm>

#include "su3_device.cuh"
#include "su3_internal.h"

namespace su3 {

constexpr int kHostTileSites = 8;  // sites per warp tile: 32 links, one per lane

template <typename A>
struct HostArgs {
  const unsigned char* a;  // device-usable address of a in host memory
  unsigned char* c;
  long long n_sites;
  long long a_stride;  // bytes between sites
  long long c_stride;
  int native_warps;
  BMat<A> b;
};

__device__ __forceinline__ double2 ld_stream_16(const void* p) {
  double2 v;
  asm volatile("ld.global.cs.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "l"(p));
  return v;
}

template <class Op>
__global__ void __launch_bounds__(256) su3_host_kernel(const __grid_constant__ HostArgs<typename Op::BArg> p) {
  using V = typename Op::V;
  constexpr int NE_IN = Op::kNeIn, NE_OUT = Op::kNeOut;
  constexpr bool kInPlace = (NE_OUT == NE_IN);
  constexpr int kSiteIn = 4 * NE_IN * (int)sizeof(V);    // link bytes of one site of a
  constexpr int kSiteOut = 4 * NE_OUT * (int)sizeof(V);  // link bytes of one site of c
  static_assert(kSiteIn % 16 == 0 && kSiteOut % 16 == 0, "sites are whole 16-byte words");
  constexpr int kWordsIn = kSiteIn / 16, kWordsOut = kSiteOut / 16;
  constexpr int kSlot = kHostTileSites * (kSiteIn + (kInPlace ? 0 : kSiteOut));

  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ typename Op::BArg bsh[72];
  Op op;
  load_b_op(p.b, bsh, op, p.native_warps);  // the only CTA barrier

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, warps = blockDim.x >> 5;
  unsigned char* in = smem + (size_t)warp * kSlot;
  unsigned char* out = kInPlace ? in : in + kHostTileSites * kSiteIn;
  const long long n_tiles = (p.n_sites + kHostTileSites - 1) / kHostTileSites;
  const long long step = (long long)gridDim.x * warps;
  int k = 0;
  for (long long t = (long long)blockIdx.x * warps + warp; t < n_tiles; t += step, ++k) {
    const long long first = t * kHostTileSites;
    const int nt = (int)min((long long)kHostTileSites, p.n_sites - first);
    for (int w = lane; w < nt * kWordsIn; w += 32) {
      const int site = w / kWordsIn, word = w - site * kWordsIn;
      reinterpret_cast<double2*>(in)[w] = ld_stream_16(p.a + (first + site) * p.a_stride + 16 * word);
    }
    __syncwarp();
    op.begin_tile(k);
    if (lane < 4 * nt)  // link `lane` of the tile: direction lane % 4 = tid % 4
      op.apply(reinterpret_cast<const V*>(in) + lane * NE_IN, reinterpret_cast<V*>(out) + lane * NE_OUT);
    __syncwarp();
    for (int w = lane; w < nt * kWordsOut; w += 32) {
      const int site = w / kWordsOut, word = w - site * kWordsOut;
      stg_stream(reinterpret_cast<double2*>(p.c + (first + site) * p.c_stride + 16 * word),
                 reinterpret_cast<const double2*>(out)[w]);
    }
    __syncwarp();  // the slot is reloaded only after every lane has stored from it
  }
}

template <class Op>
static su3_status run_host(const Form& f, const LaunchCfg& cfg, const void* a, const double* b, void* c,
                           const LaunchCtx& ctx) {
  using V = typename Op::V;
  constexpr bool kInPlace = (Op::kNeOut == Op::kNeIn);
  const int block = 256;
  const size_t smem = (size_t)(block / 32) * kHostTileSites * 4 * sizeof(V) * (Op::kNeIn + (kInPlace ? 0 : Op::kNeOut));
  HostArgs<typename Op::BArg> p;
  p.a = static_cast<const unsigned char*>(a);
  p.c = static_cast<unsigned char*>(c);
  p.n_sites = f.n_sites;
  p.a_stride = f.a_stride;
  p.c_stride = f.c_stride;
  LaunchCfg hc = cfg;
  hc.block = block;
  p.native_warps = native_warps(f, hc);
  p.b = make_b<typename Op::BArg>(b);
  auto kern = su3_host_kernel<Op>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 0;
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block, smem);
  if (e != cudaSuccess) {
    *ctx.err = std::string("su3_host_kernel set-up: ") + cudaGetErrorString(e);
    return SU3_ERR_CUDA;
  }
  const long long tiles = (f.n_sites + kHostTileSites - 1) / kHostTileSites;
  const long long want = (tiles + block / 32 - 1) / (block / 32);
  const int grid = (int)std::max<long long>(1, std::min<long long>(want, (long long)ctx.num_sms * std::max(per_sm, 1)));
  kern<<<grid, block, smem, ctx.stream>>>(p);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    *ctx.err = std::string("su3_host_kernel launch: ") + cudaGetErrorString(e);
    return SU3_ERR_CUDA;
  }
  ++*ctx.launches;
  return SU3_OK;
}

template <int DT>
static su3_status run_host_repr(const Form& f, const LaunchCfg& cfg, const void* a, const double* b, void* c,
                                const LaunchCtx& ctx) {
  if (f.repr_in == SU3_REPR_FULL18) return run_host<NativeOp<DT, 9, 3>>(f, cfg, a, b, c, ctx);
  if (f.repr_out == SU3_REPR_TWOROW12) return run_host<NativeOp<DT, 6, 2>>(f, cfg, a, b, c, ctx);
  return run_host<NativeOp<DT, 6, 3>>(f, cfg, a, b, c, ctx);
}

su3_status launch_mult_host_direct(const Form& f, const LaunchCfg& cfg, const void* a, const double* b, void* c,
                                   const LaunchCtx& ctx) {
  if (f.layout != SU3_LAYOUT_AOS) return SU3_ERR_UNSUPPORTED;
  if (f.arith == SU3_ARITH_F32PAIR || f.arith == SU3_ARITH_HYBRID) {
    if (f.dtype != SU3_F64) return SU3_ERR_UNSUPPORTED;
    const bool hyb = f.arith == SU3_ARITH_HYBRID;
    if (f.repr_in == SU3_REPR_FULL18)
      return hyb ? run_host<HybridF64Op<9, 3>>(f, cfg, a, b, c, ctx) : run_host<PairF64Op<9, 3>>(f, cfg, a, b, c, ctx);
    if (f.repr_out == SU3_REPR_TWOROW12)
      return hyb ? run_host<HybridF64Op<6, 2>>(f, cfg, a, b, c, ctx) : run_host<PairF64Op<6, 2>>(f, cfg, a, b, c, ctx);
    return hyb ? run_host<HybridF64Op<6, 3>>(f, cfg, a, b, c, ctx) : run_host<PairF64Op<6, 3>>(f, cfg, a, b, c, ctx);
  }
  switch (f.dtype) {
    case SU3_F64: return run_host_repr<kF64>(f, cfg, a, b, c, ctx);
    case SU3_F32: return run_host_repr<kF32>(f, cfg, a, b, c, ctx);
    case SU3_F16: return run_host_repr<kF16>(f, cfg, a, b, c, ctx);
    case SU3_BF16: return run_host_repr<kBF16>(f, cfg, a, b, c, ctx);
  }
  return SU3_ERR_UNSUPPORTED;
}

}  // namespace su3
