// Streaming kernels of the SU3_Bench link multiply (arXiv 2103.00571, §Background "SU3_Bench"):
// c[i].link[j] = a[i].link[j] x b[j] for every site i and link j.
//
// The paper's own analysis (§Background) puts the time in streaming A in and C out with no reuse
// and B cache-resident. On GB300 that means: move a and c between HBM and shared memory with
// 1-D bulk async copies (the TMA engine), keep b in registers (each thread always serves the same
// link direction j), and spend the SM only on the 108 FMAs of each link.
//
//  * The staged kernel (every layout): a persistent CTA streams tiles of `tile_sites` sites through
//    a `stages`-deep ring of shared-memory buffers. Each tile arrives by bulk copies completing on
//    one mbarrier: one copy of whole sites (AOS; padded sites: one 2-D tensor copy of the tile's
//    links), one copy of whole 32-link blocks (AOSOA32), or the element planes into plane slots
//    of 256 links (SOA: one 2-D tensor copy of all planes for 64-site tiles of 4- or 8-byte
//    elements, one copy per plane otherwise). Each thread multiplies work
//    items q = tid, tid+block, ... of the tile: whole links, or single output rows when
//    threads_per_link is 3, and writes the result back in place (two-row in, full out: into a
//    3-deep ring of output buffers in the same layout). Warp 0 then bulk-stores the tile and
//    refills the ring. Inside a tile a link's elements sit 1 (AOS), 32 (AOSOA32) or 256 (SOA)
//    storage vectors apart; the element-major layouts put consecutive links in consecutive
//    vectors, so a warp's shared-memory accesses are conflict-free. AOS site bytes past the four
//    links (the paper's coordinates, index, parity and pad) are neither read nor written: with
//    such a stride the array is a 2-D tensor for the TMA engine (rows = sites, a row = the four
//    links, the row pitch = the stride), so one tensor copy brings a tile's links in, packed in
//    shared memory (a 640-byte stride, a multiple of the 128-byte bank width, would otherwise
//    put every site on the same banks), and one writes them out. A tile too large for the
//    requested CTAs per SM is shrunk.
//  * The direct kernel (SOA / AOSOA32 with stages = 0): the element-major layouts are coalesced as
//    they stand, so a thread loads its links straight from global memory with 8/16-byte
//    no-L1-allocate loads and writes with streaming stores.
#pragma once
#include <cuda.h>  // CUtensorMap and its encoder's types (the encoder is reached through the runtime)
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>

#include "su3_device.cuh"
#include "su3_internal.h"

namespace su3 {

template <typename A>
struct AosArgs {
  const unsigned char* a;
  unsigned char* c;
  long long n_sites;
  long long a_stride;  // AOS: bytes between sites of a
  long long c_stride;  // AOS: bytes between sites of c
  long long n_links;   // SOA: links per element plane in global memory (4 * n_sites)
  int tile_sites;
  int stages;
  int n_tiles;
  unsigned stage_bytes;  // bytes reserved per input stage (multiple of 128)
  unsigned out_bytes;    // bytes per output buffer (separate-output forms)
  int native_warps;      // HYBRID: warps [0, native_warps) of every CTA compute natively
  unsigned* status;
  int a_padded;       // AOS: a's sites are wider than their links; tiles arrive through SiteMaps::a
  int c_padded;       // AOS: c's sites are wider than their links; tiles leave through SiteMaps::c
  int soa_tensor;     // SOA: a tile's element planes move as one 2-D tensor copy each way
  BMat<A> b;
};

// Tensor maps of a and c for the TMA engine: padded AOS arrays (rows = sites, a row = the site's
// links as 8-byte elements, a box = tile_sites rows), or SOA arrays (rows = element planes, a box
// = the 256 links of one tile in every plane). A kernel parameter of their own: the copies take
// their address, and the other arguments stay plain constants.
struct SiteMaps {
  CUtensorMap a;
  CUtensorMap c;
};

constexpr int kSmemHeader = 1024;    // mbarriers (<= 8 x 8 B) + b (<= 576 B), then 128-aligned data
constexpr int kSoaPlaneLinks = 256;  // links per element plane of an SOA tile in shared memory

// Distance, in storage vectors, between consecutive elements of one link inside a staged tile.
template <int LAYOUT>
__host__ __device__ constexpr int tile_elem_stride() {
  return LAYOUT == SU3_LAYOUT_AOS ? 1 : LAYOUT == SU3_LAYOUT_AOSOA32 ? 32 : kSoaPlaneLinks;
}

// Element 0 of tile link q (element-major layouts), in storage vectors from the tile start.
template <int LAYOUT, int NE>
__device__ __forceinline__ int tile_link_base(int q) {
  return LAYOUT == SU3_LAYOUT_AOSOA32 ? (q >> 5) * NE * 32 + (q & 31) : q;
}

// The staged streaming kernel. Op::kNeIn complex elements per input link (9 full, 6 two-row),
// Op::kNeOut per output link. In place (kNeOut == kNeIn): the result overwrites the input tile in
// shared memory. Otherwise (two-row in, full out) results go to a ring of 3 output buffers.
// TPL threads per link: 1 (a thread computes whole links), or one thread per output row. The work
// items of a tile are then ordered row-major over (row, link), so that item q's link direction is
// still q % 4 = tid % 4 and each thread keeps one b[j] in registers.
// Tiles: AOS any number of sites; AOSOA32 a multiple of 8 sites (whole 32-link blocks; the last
// block of an array is padded, so it is always read whole); SOA at most 64 sites (256 links).
// PADDED (AOS only): a's or c's sites are wider than their links, and `maps` holds their tensor
// maps; otherwise `maps` is read only by SOA tensor copies. One instantiation per PADDED value, so
// the packed kernels keep their own code.
template <class Op, int TPL, int LAYOUT, bool PADDED>
__global__ void __launch_bounds__(256) su3_aos_kernel(const __grid_constant__ AosArgs<typename Op::BArg> p,
                                                      const __grid_constant__ SiteMaps maps) {
  using V = typename Op::V;
  using BA = typename Op::BArg;
  constexpr int NE_IN = Op::kNeIn, NE_OUT = Op::kNeOut;
  constexpr bool kInPlace = (NE_OUT == NE_IN);
  // FP64 two-row in, full out, packed AoS sites, one thread per link: each warp stages its 32
  // consecutive links' results (4.6 KB) in a double-buffered slot of its own and drains it with one
  // bulk copy, instead of the CTA filling a ring of 3 whole-tile output buffers. A CTA then needs
  // about half the shared memory, so a third one fits on an SM (FP32-pair form: 4.34 -> 4.60 G
  // site/s at L=48). Narrower outputs keep the ring: for matrix x vector products (0.8-1.5 KB per
  // warp copy) per-warp copies measured up to 2.3x slower; FP32/FP16 storage keeps it too.
  constexpr bool kWarpOut = !kInPlace && LAYOUT == SU3_LAYOUT_AOS && TPL == 1 && !PADDED && NE_IN == 6 &&
                            NE_OUT == 9 && sizeof(V) == 16;
  constexpr int kVec = (int)sizeof(V);
  constexpr int kLinkIn = NE_IN * kVec;
  constexpr int kLinkOut = NE_OUT * kVec;
  constexpr int ES = tile_elem_stride<LAYOUT>();

  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);
  BA* bsh = reinterpret_cast<BA*>(smem + 64);
  unsigned char* stage0 = smem + kSmemHeader;
  unsigned char* out0 = stage0 + (size_t)p.stages * p.stage_bytes;

  const int tid = threadIdx.x;
  const int S_ = p.stages;
  if (tid == 0) {
    for (int s = 0; s < S_; ++s) mbar_init(&full[s], 1);
    fence_mbar_init();
  }
  Op op;
  load_b_op(p.b, bsh, op, p.native_warps);  // contains __syncthreads (also publishes the mbarrier init)

  const uint64_t pol = policy_evict_first();
  const int my_tiles = p.n_tiles > (int)blockIdx.x ? (p.n_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  auto tile_of = [&](int k) { return (int)blockIdx.x + k * (int)gridDim.x; };
  auto tile_nsites = [&](int t) {
    long long first = (long long)t * p.tile_sites;
    long long rest = p.n_sites - first;
    return (int)(rest < p.tile_sites ? rest : p.tile_sites);
  };
  // thread 0: the copies of tile k into stage k % S. AOS tiles are packed (4 links per site) in
  // shared memory whatever a's stride: padded sites (e.g. the paper's 640-byte FP64 Site) arrive by
  // one 2-D tensor copy of the tile's links, so the fields after the links are never read.
  auto issue_load = [&](int k) {
    const int t = tile_of(k);
    const int s = k % S_;
    const int nt = tile_nsites(t);
    const long long first = (long long)t * p.tile_sites;
    unsigned char* dst = stage0 + (size_t)s * p.stage_bytes;
    if constexpr (LAYOUT == SU3_LAYOUT_AOS) {
      if constexpr (PADDED) {
        if (p.a_padded) {
          // the box is always tile_sites rows (rows past the array arrive as zeros and count)
          mbar_arrive_expect_tx(&full[s], (unsigned)(p.tile_sites * 4 * kLinkIn));
          tma_load_2d(dst, &maps.a, 0, (int)first, &full[s], pol);
          return;
        }
      }
      const unsigned bytes = (unsigned)((long long)nt * p.a_stride);
      mbar_arrive_expect_tx(&full[s], bytes);
      bulk_g2s(dst, p.a + first * p.a_stride, bytes, &full[s], pol);
    } else if constexpr (LAYOUT == SU3_LAYOUT_AOSOA32) {
      const unsigned bytes = (unsigned)((4 * nt + 31) / 32 * 32 * kLinkIn);
      mbar_arrive_expect_tx(&full[s], bytes);
      bulk_g2s(dst, p.a + 4 * first * kLinkIn, bytes, &full[s], pol);
    } else {
      if (p.soa_tensor) {
        // the tile's 256 links of every element plane in one 2-D tensor copy (links past the
        // array arrive as zeros and count); x in 8-byte elements
        mbar_arrive_expect_tx(&full[s], (unsigned)(NE_IN * kSoaPlaneLinks * kVec));
        tma_load_2d(dst, &maps.a, (int)(4 * first * kVec / 8), 0, &full[s], pol);
        return;
      }
      const unsigned plane = (unsigned)(4 * nt * kVec);
      mbar_arrive_expect_tx(&full[s], plane * NE_IN);
#pragma unroll 1
      for (int e = 0; e < NE_IN; ++e)
        bulk_g2s(dst + (size_t)e * kSoaPlaneLinks * kVec, p.a + ((long long)e * p.n_links + 4 * first) * kVec, plane,
                 &full[s], pol);
    }
  };

  const int prefetch = kInPlace ? S_ - 1 : S_;
  if (tid == 0)
    for (int k = 0; k < prefetch && k < my_tiles; ++k) issue_load(k);

  // packed kernel: one copy of a whole tile of c. Its per-site branch below (a c stride wider
  // than the tile's) serves no launch, since padded strides take the PADDED kernel, but two
  // variants of the kernel without it measured 5-11 % slower on the narrow (FP32/FP16/BF16)
  // forms, a code-generation effect, so it stays.
  const bool packed_store = kInPlace ? (p.a_stride == 4 * kLinkIn && p.c_stride == 4 * kLinkOut)
                                     : (p.c_stride == 4 * kLinkOut);
  int issued = my_tiles < prefetch ? my_tiles : prefetch;  // loads issued so far (thread 0's view)
  int kfail = -1;
  int wpar = 0;  // kWarpOut: which of the warp's two output slots is next

  for (int k = 0; k < my_tiles; ++k) {
    const int s = k % S_;
    const int t = tile_of(k);
    const int nt = tile_nsites(t);
    const bool ok = mbar_wait_bounded(&full[s], (unsigned)((k / S_) & 1));
    unsigned char* in = stage0 + (size_t)s * p.stage_bytes;
    unsigned char* out = kInPlace ? in : out0 + (size_t)(k % 3) * p.out_bytes;
    if (ok && kWarpOut) {
      op.begin_tile(k);
      const int links = 4 * nt, lane = tid & 31;
      const long long first = (long long)t * p.tile_sites;
      for (int base = tid - lane; base < links; base += blockDim.x) {  // warp-uniform
        unsigned char* slot = out0 + ((size_t)(tid >> 5) * 2 + wpar) * 32 * kLinkOut;
        if (lane == 0) bulk_wait_read<1>();  // the store issued two slots back has read this slot
        __syncwarp();
        const int link = base + lane;
        if (link < links) {
          const int site = link >> 2, j = link & 3;
          op.template apply<ES, ES>(reinterpret_cast<const V*>(in + (size_t)site * p.a_stride + j * kLinkIn),
                                    reinterpret_cast<V*>(slot + (size_t)lane * kLinkOut));
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) {  // links base .. base + n - 1 of the tile are contiguous in packed c
          const int n = links - base < 32 ? links - base : 32;
          bulk_s2g(p.c + (4 * first + base) * kLinkOut, slot, (unsigned)(n * kLinkOut), pol);
          bulk_commit();
        }
        wpar ^= 1;
      }
    } else if (ok) {
      op.begin_tile(k);
      const int links = 4 * nt;
      for (int q = tid; q < TPL * links; q += blockDim.x) {
        int row = 0;
        if (TPL >= 2 && q >= links) row = 1;
        if (TPL >= 3 && q >= 2 * links) row = 2;
        const int link = q - row * links;
        const V* src;
        V* dst;
        if constexpr (LAYOUT == SU3_LAYOUT_AOS) {
          if constexpr (PADDED) {  // tiles of padded sites are packed in shared memory
            src = reinterpret_cast<const V*>(in + (size_t)link * kLinkIn);
          } else {
            const int site = link >> 2, j = link & 3;
            src = reinterpret_cast<const V*>(in + (size_t)site * p.a_stride + j * kLinkIn);
          }
          dst = kInPlace ? const_cast<V*>(src) : reinterpret_cast<V*>(out + (size_t)link * kLinkOut);
        } else {
          src = reinterpret_cast<const V*>(in) + tile_link_base<LAYOUT, NE_IN>(link);
          dst = kInPlace ? const_cast<V*>(src) : reinterpret_cast<V*>(out) + tile_link_base<LAYOUT, NE_OUT>(link);
        }
        if constexpr (TPL == 1) op.template apply<ES, ES>(src, dst);
        else op.template apply_row<ES, ES>(src, dst, row);
      }
    }
    fence_proxy_async_smem();
    if (!kInPlace && !kWarpOut && tid < 32) bulk_wait_read<1>();  // store(k-2) done reading out[(k+1)%3]
    if (__syncthreads_or(!ok)) {
      kfail = k;
      break;
    }
    if (kWarpOut) {  // the warps stored their own links; stage s has been read by all of them
      if (tid == 0 && issued < my_tiles) issue_load(issued++);
    } else if (tid < 32) {
      // store tile k
      const long long first = (long long)t * p.tile_sites;
      if constexpr (LAYOUT == SU3_LAYOUT_AOS) {
        if constexpr (PADDED) {
          // the packed tile in one copy; padded c: one 2-D tensor copy of the links (rows past the
          // array are not written, nor are the bytes after each site's links)
          if (tid == 0) {
            if (p.c_padded) tma_store_2d(&maps.c, 0, (int)first, out, pol);
            else bulk_s2g(p.c + first * p.c_stride, out, (unsigned)(nt * 4 * kLinkOut), pol);
          }
        } else if (packed_store) {
          if (tid == 0) bulk_s2g(p.c + first * p.c_stride, out, (unsigned)(nt * 4 * kLinkOut), pol);
        } else {
          const long long src_stride = kInPlace ? p.a_stride : 4 * kLinkOut;
          for (int i = tid; i < nt; i += 32)
            bulk_s2g(p.c + (first + i) * p.c_stride, out + (size_t)i * src_stride, (unsigned)(4 * kLinkOut), pol);
        }
      } else if constexpr (LAYOUT == SU3_LAYOUT_AOSOA32) {
        // whole blocks in one copy; a partial last block (only at the end of the array) one
        // element row at a time, so that c's padding links are never written
        const int links = 4 * nt, whole = links / 32, rem = links % 32;
        unsigned char* cblk = p.c + 4 * first * kLinkOut;
        if (tid == 0 && whole) bulk_s2g(cblk, out, (unsigned)(whole * 32 * kLinkOut), pol);
        if (rem && tid < NE_OUT) {
          const size_t off = ((size_t)whole * NE_OUT * 32 + (size_t)tid * 32) * kVec;
          bulk_s2g(cblk + off, out + off, (unsigned)(rem * kVec), pol);
        }
      } else if (p.soa_tensor) {  // every element plane in one tensor copy (links past the array are not written)
        if (tid == 0) tma_store_2d(&maps.c, (int)(4 * first * kVec / 8), 0, out, pol);
      } else {
        if (tid < NE_OUT)
          bulk_s2g(p.c + ((long long)tid * p.n_links + 4 * first) * kVec, out + (size_t)tid * kSoaPlaneLinks * kVec,
                   (unsigned)(4 * nt * kVec), pol);
      }
      bulk_commit();
      if (kInPlace) {
        bulk_wait_read<1>();  // store(k-1) has read stage (k-1) % S
        __syncwarp();
        if (tid == 0 && issued < my_tiles) issue_load(issued++);
      } else if (tid == 0 && issued < my_tiles) {
        issue_load(issued++);  // stage s was fully read before the barrier
      }
    }
  }

  if (kfail >= 0 && tid == 0) {
    atomicOr(p.status, kDevErrTimeout);
    // let the loads still in flight land before shared memory is released (bounded)
    for (int k = kfail; k < issued; ++k) mbar_wait_bounded(&full[k % S_], (unsigned)((k / S_) & 1));
  }
  if (kWarpOut ? (tid & 31) == 0 : tid < 32) bulk_wait_all<0>();
}

// ---- SOA / AOSOA32: direct coalesced loads ----------------------------------------------------

template <typename A>
struct DirectArgs {
  const void* a;
  void* c;
  long long n_links;
  int native_warps;       // HYBRID: warps [0, native_warps) of every CTA compute natively
  BMat<A> b;
};

template <int LAYOUT, int NE>
__device__ __forceinline__ long long elem_index(long long q, int e, long long n_links) {
  if (LAYOUT == SU3_LAYOUT_SOA) return (long long)e * n_links + q;
  return ((q >> 5) * NE + e) * 32 + (q & 31);  // AOSOA32
}

template <class Op, int LAYOUT, int LPT>
__global__ void __launch_bounds__(256) su3_direct_kernel(const __grid_constant__ DirectArgs<typename Op::BArg> p) {
  using V = typename Op::V;
  constexpr int NE_IN = Op::kNeIn, NE_OUT = Op::kNeOut;
  __shared__ typename Op::BArg bsh[72];
  const long long q_end = p.n_links;
  Op op;
  load_b_op(p.b, bsh, op, p.native_warps);
  const V* a = reinterpret_cast<const V*>(p.a);
  V* c = reinterpret_cast<V*>(p.c);
  const long long T = (long long)gridDim.x * blockDim.x;  // a multiple of 4: j stays tid % 4
  int it = 0;
  for (long long base = (long long)blockIdx.x * blockDim.x + threadIdx.x; base < q_end; base += LPT * T, ++it) {
    op.begin_tile(it);
    V buf[LPT][NE_IN];
#pragma unroll
    for (int u = 0; u < LPT; ++u) {
      const long long q = base + u * T;
      if (q < q_end) {
#pragma unroll
        for (int e = 0; e < NE_IN; ++e) buf[u][e] = ldg_stream(a + elem_index<LAYOUT, NE_IN>(q, e, p.n_links));
      }
    }
#pragma unroll
    for (int u = 0; u < LPT; ++u) {
      const long long q = base + u * T;
      if (q < q_end) {
        V res[NE_OUT];
        op.apply(buf[u], res);
#pragma unroll
        for (int e = 0; e < NE_OUT; ++e) stg_stream(c + elem_index<LAYOUT, NE_OUT>(q, e, p.n_links), res[e]);
      }
    }
  }
}

// ---- host launchers (templates: each translation unit instantiates its own kind of stride) ----

inline su3_status cuda_fail(const LaunchCtx& ctx, const char* what, cudaError_t e) {
  *ctx.err = std::string(what) + ": " + cudaGetErrorString(e);
  return SU3_ERR_CUDA;
}

// Max rows (sites) of one tensor-copy box.
constexpr long long kMaxBoxRows = 256;

// A 2-D tensor map for the TMA engine over 8-byte elements: `rows` rows of `inner` elements,
// `pitch` bytes apart (a multiple of 16); a box is box_rows rows of box_inner elements.
su3_status encode_2d(CUtensorMap* m, const void* base, long long inner, long long rows, long long pitch,
                     long long box_inner, long long box_rows, const LaunchCtx& ctx);

// An AOS array of padded sites: n_sites rows `stride` bytes apart, each row the site's row_bytes
// of links (the bytes after the links lie outside the tensor, so no copy reads or writes them); a
// box is `rows` whole rows.
inline su3_status encode_sites(CUtensorMap* m, const void* base, long long n_sites, long long stride,
                               long long row_bytes, long long rows, const LaunchCtx& ctx) {
  return encode_2d(m, base, row_bytes / 8, n_sites, stride, row_bytes / 8, rows, ctx);
}

// The same dispatch over forms, instantiated once per kind of site stride (each in its own
// translation unit, so that they compile in parallel).
su3_status launch_mult_padded(const Form& f, const LaunchCfg& cfg, const void* a, const double* b, void* c,
                              const LaunchCtx& ctx);
su3_status launch_adjacent_padded(int which, const Form& f, const LaunchCfg& cfg, const void* a, const double* bv,
                                  void* c, const LaunchCtx& ctx);

// The staged kernel for one layout. Tile geometry: AOS tile_sites whole sites; AOSOA32 tile_sites
// a multiple of 8 (whole 32-link blocks); SOA at most 64 sites, each element plane in a slot of
// 256 links, so an SOA stage is NE x 256 storage vectors whatever tile_sites is.
template <class Op, int LAYOUT, bool PADDED>
static su3_status run_aos(const Form& f, const LaunchCfg& cfg_in, const void* a, const double* b, void* c,
                          const LaunchCtx& ctx) {
  LaunchCfg cfg = cfg_in;  // the launch may narrow its block for a small array (below)
  using BA = typename Op::BArg;
  using V = typename Op::V;
  constexpr bool kInPlace = (Op::kNeOut == Op::kNeIn);
  constexpr long long kVec = (long long)sizeof(V);
  constexpr long long kLinkIn = Op::kNeIn * kVec, kLinkOut = Op::kNeOut * kVec;
  const long long quantum = LAYOUT == SU3_LAYOUT_AOSOA32 ? 8 : 1;
  auto r128 = [](long long x) { return (x + 127) / 128 * 128; };
  auto in_bytes = [&](long long ts) {
    if (LAYOUT == SU3_LAYOUT_AOS) return r128(ts * 4 * kLinkIn);  // packed sites, whatever the stride
    if (LAYOUT == SU3_LAYOUT_AOSOA32) return r128(ts * 4 * kLinkIn);
    return r128(Op::kNeIn * kSoaPlaneLinks * kVec);
  };
  auto out_bytes = [&](long long ts) {
    if (kInPlace) return 0LL;
    if (LAYOUT == SU3_LAYOUT_SOA) return r128(Op::kNeOut * kSoaPlaneLinks * kVec);
    return r128(ts * 4 * kLinkOut);
  };
  // separate outputs: two slots of 32 links per warp (the kernel's kWarpOut case), else a ring of
  // 3 whole-tile buffers
  const bool warp_out = !kInPlace && LAYOUT == SU3_LAYOUT_AOS && !PADDED && cfg.threads_per_link == 1 &&
                        Op::kNeIn == 6 && Op::kNeOut == 9 && kVec == 16;
  auto smem_of = [&](long long ts) {
    return kSmemHeader + cfg.stages * in_bytes(ts) + (warp_out ? cfg.block / 32 * 2 * 32 * kLinkOut : 3 * out_bytes(ts));
  };

  long long ts = cfg.tile_sites;
  // padded AOS sites move through tensor copies whose box holds at most 256 rows
  const bool a_pad = LAYOUT == SU3_LAYOUT_AOS && f.a_stride != 4 * kLinkIn;
  const bool c_pad = LAYOUT == SU3_LAYOUT_AOS && f.c_stride != 4 * kLinkOut;
  if ((a_pad || c_pad) != PADDED) {
    *ctx.err = "internal: site strides do not match the kernel chosen";
    return SU3_ERR_INVALID_ARG;
  }
  if ((a_pad || c_pad) && f.n_sites > 0x7fffffffLL) {
    *ctx.err = "arrays of padded AOS sites hold at most 2^31 - 1 sites";
    return SU3_ERR_INVALID_ARG;
  }
  if (a_pad || c_pad) ts = std::min(ts, kMaxBoxRows);
  if (LAYOUT == SU3_LAYOUT_AOSOA32 && ts % 8) {
    *ctx.err = "AOSOA32 tiles must be a multiple of 8 sites (whole 32-link blocks)";
    return SU3_ERR_INVALID_ARG;
  }
  if (LAYOUT == SU3_LAYOUT_SOA && ts > kSoaPlaneLinks / 4) {
    *ctx.err = "SOA tiles hold at most 64 sites (256 links per element plane)";
    return SU3_ERR_INVALID_ARG;
  }
  if (LAYOUT != SU3_LAYOUT_SOA) {
    // the two-row -> full form shares its configuration with two-row -> two-row but also needs a
    // 3-deep output ring: shrink the tile until both fit in shared memory
    if (!kInPlace)
      while (ts > quantum && smem_of(ts) > 227 * 1024) ts = std::max(quantum, (ts + 1) / 2 / quantum * quantum);
    // keep ctas_per_sm CTAs resident: shrink the tile (to a multiple of 8 sites) until that many
    // CTAs fit in one SM's shared memory instead of silently running fewer
    if (ctx.smem_per_sm > 0) {
      const long long per_cta = ctx.smem_per_sm / cfg.ctas_per_sm - ctx.smem_reserved;
      if (smem_of(ts) > per_cta) {
        while (ts > quantum && smem_of(ts) > per_cta) ts -= quantum;
        if (ts >= 8) ts &= ~7LL;
      }
    }
  }
  // an array with fewer tiles than SMs: narrower tiles, in CTAs just wide enough for them, spread
  // it over more SMs, so that its warps do not queue on a few SMs' pipes (every launch shape gives
  // the same bits; this only shortens small launches)
  if (f.n_sites > 0 && (f.n_sites + ts - 1) / ts < ctx.num_sms) {
    long long t2 = (f.n_sites + ctx.num_sms - 1) / ctx.num_sms;
    t2 = std::max(quantum, (t2 + quantum - 1) / quantum * quantum);
    if (t2 < ts) {
      ts = t2;
      const long long items = ts * 4 * (cfg.threads_per_link == 1 ? 1 : (Op::kRowSplit ? Op::kNeOut / 3 : 1));
      cfg.block = (int)std::min<long long>(cfg.block, std::max<long long>(32, (items + 31) / 32 * 32));
    }
  }
  AosArgs<BA> p;
  p.a = static_cast<const unsigned char*>(a);
  p.c = static_cast<unsigned char*>(c);
  p.n_sites = f.n_sites;
  p.a_stride = f.a_stride;
  p.c_stride = f.c_stride;
  p.n_links = 4 * f.n_sites;
  p.tile_sites = (int)ts;
  p.stages = cfg.stages;
  const long long n_tiles = (f.n_sites + ts - 1) / ts;
  if (n_tiles > 0x7fffffffLL) {
    *ctx.err = "too many tiles for one launch: use a larger tile_sites";
    return SU3_ERR_INVALID_ARG;
  }
  p.n_tiles = (int)n_tiles;
  p.stage_bytes = (unsigned)in_bytes(ts);
  p.out_bytes = warp_out ? 0u : (unsigned)out_bytes(ts);
  p.native_warps = native_warps(f, cfg);
  const int grid = (int)std::min<long long>(p.n_tiles, (long long)ctx.num_sms * cfg.ctas_per_sm);
  p.status = ctx.status;
  p.a_padded = a_pad ? 1 : 0;
  p.c_padded = c_pad ? 1 : 0;
  p.b = make_b<BA>(b);
  const size_t smem = (size_t)smem_of(ts);
  if (smem > 227 * 1024) {
    *ctx.err = "launch configuration needs " + std::to_string(smem) + " B of shared memory (max 232448)";
    return SU3_ERR_INVALID_ARG;
  }
  constexpr int kRows = Op::kNeOut / 3;
  constexpr int kTplRows = Op::kRowSplit ? kRows : 1;
  if (cfg.threads_per_link != 1 && (!Op::kRowSplit || cfg.threads_per_link != 3)) {
    *ctx.err = "threads_per_link must be 1, or 3 (one thread per output row) for the link products";
    return SU3_ERR_INVALID_ARG;
  }
  const bool rows = cfg.threads_per_link != 1;  // one thread per output row
  auto start = [&](auto kern, const auto&... args) -> su3_status {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(ctx, "cudaFuncSetAttribute", e);
    kern<<<grid, cfg.block, smem, ctx.stream>>>(args...);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, "su3_aos_kernel launch", e);
    ++*ctx.launches;
    return SU3_OK;
  };
  SiteMaps maps;
  memset(&maps, 0, sizeof(maps));  // read by the padded kernels and the SOA tensor copies only
  // SOA tiles of exactly 256 links whose plane rows fit one box (at most 256 8-byte elements, so
  // 4- and 8-byte complex elements) move as one tensor copy each way
  p.soa_tensor = LAYOUT == SU3_LAYOUT_SOA && ts == kSoaPlaneLinks / 4 && kVec <= 8 ? 1 : 0;
  if (p.soa_tensor) {
    const long long row = p.n_links * kVec;  // one element plane, bytes (a multiple of 16)
    su3_status st = encode_2d(&maps.a, a, row / 8, Op::kNeIn, row, kSoaPlaneLinks * kVec / 8, Op::kNeIn, ctx);
    if (st == SU3_OK) st = encode_2d(&maps.c, c, row / 8, Op::kNeOut, row, kSoaPlaneLinks * kVec / 8, Op::kNeOut, ctx);
    if (st != SU3_OK) return st;
  }
  if constexpr (PADDED) {
    if (a_pad) {
      const su3_status st = encode_sites(&maps.a, a, f.n_sites, f.a_stride, 4 * kLinkIn, ts, ctx);
      if (st != SU3_OK) return st;
    }
    if (c_pad) {
      const su3_status st = encode_sites(&maps.c, c, f.n_sites, f.c_stride, 4 * kLinkOut, ts, ctx);
      if (st != SU3_OK) return st;
    }
  }
  return rows ? start(su3_aos_kernel<Op, kTplRows, LAYOUT, PADDED>, p, maps)
              : start(su3_aos_kernel<Op, 1, LAYOUT, PADDED>, p, maps);
}

template <class Op, int LAYOUT>
static su3_status run_direct(const Form& f, const LaunchCfg& cfg, const void* a, const double* b, void* c,
                             const LaunchCtx& ctx) {
  DirectArgs<typename Op::BArg> p;
  p.a = a;
  p.c = c;
  p.n_links = 4 * f.n_sites;
  p.b = make_b<typename Op::BArg>(b);
  const int lpt = cfg.tile_sites;
  const long long per_cta = (long long)cfg.block * lpt;
  p.native_warps = native_warps(f, cfg);
  const int grid = (int)std::max<long long>(1, std::min<long long>((p.n_links + per_cta - 1) / per_cta,
                                                                    (long long)ctx.num_sms * cfg.ctas_per_sm));
  switch (lpt) {
    case 1: su3_direct_kernel<Op, LAYOUT, 1><<<grid, cfg.block, 0, ctx.stream>>>(p); break;
    case 2: su3_direct_kernel<Op, LAYOUT, 2><<<grid, cfg.block, 0, ctx.stream>>>(p); break;
    case 4: su3_direct_kernel<Op, LAYOUT, 4><<<grid, cfg.block, 0, ctx.stream>>>(p); break;
    default:
      *ctx.err = "links per thread (tile_sites) must be 1, 2 or 4 for SOA/AOSOA32";
      return SU3_ERR_INVALID_ARG;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, "su3_direct_kernel launch", e);
  ++*ctx.launches;
  return SU3_OK;
}

template <class Op, bool PADDED>
static su3_status run_layout(const Form& f, const LaunchCfg& cfg, const void* a, const double* b, void* c,
                             const LaunchCtx& ctx) {
  if constexpr (PADDED) {
    return run_aos<Op, SU3_LAYOUT_AOS, true>(f, cfg, a, b, c, ctx);  // only AOS sites have a stride
  } else {
    switch (f.layout) {
      case SU3_LAYOUT_AOS: return run_aos<Op, SU3_LAYOUT_AOS, false>(f, cfg, a, b, c, ctx);
      // element-major layouts: staged tiles when the configuration has stages, direct loads otherwise
      case SU3_LAYOUT_AOSOA32:
        return cfg.stages ? run_aos<Op, SU3_LAYOUT_AOSOA32, false>(f, cfg, a, b, c, ctx)
                          : run_direct<Op, SU3_LAYOUT_AOSOA32>(f, cfg, a, b, c, ctx);
      case SU3_LAYOUT_SOA:
        return cfg.stages ? run_aos<Op, SU3_LAYOUT_SOA, false>(f, cfg, a, b, c, ctx)
                          : run_direct<Op, SU3_LAYOUT_SOA>(f, cfg, a, b, c, ctx);
    }
    return SU3_ERR_UNSUPPORTED;
  }
}

template <int DT, bool PADDED>
static su3_status run_repr(const Form& f, const LaunchCfg& cfg, const void* a, const double* b, void* c,
                           const LaunchCtx& ctx) {
  if (f.repr_in == SU3_REPR_FULL18) return run_layout<NativeOp<DT, 9, 3>, PADDED>(f, cfg, a, b, c, ctx);
  if (f.repr_out == SU3_REPR_TWOROW12) return run_layout<NativeOp<DT, 6, 2>, PADDED>(f, cfg, a, b, c, ctx);
  return run_layout<NativeOp<DT, 6, 3>, PADDED>(f, cfg, a, b, c, ctx);
}

template <bool PADDED>
static su3_status mult_dispatch(const Form& f, const LaunchCfg& cfg, const void* a, const double* b, void* c,
                                const LaunchCtx& ctx) {
  if (f.arith == SU3_ARITH_F32PAIR || f.arith == SU3_ARITH_HYBRID) {
    if (f.dtype != SU3_F64) return SU3_ERR_UNSUPPORTED;
    const bool hyb = f.arith == SU3_ARITH_HYBRID;
    if (f.repr_in == SU3_REPR_FULL18)
      return hyb ? run_layout<HybridF64Op<9, 3>, PADDED>(f, cfg, a, b, c, ctx) : run_layout<PairF64Op<9, 3>, PADDED>(f, cfg, a, b, c, ctx);
    if (f.repr_out == SU3_REPR_TWOROW12)
      return hyb ? run_layout<HybridF64Op<6, 2>, PADDED>(f, cfg, a, b, c, ctx) : run_layout<PairF64Op<6, 2>, PADDED>(f, cfg, a, b, c, ctx);
    return hyb ? run_layout<HybridF64Op<6, 3>, PADDED>(f, cfg, a, b, c, ctx) : run_layout<PairF64Op<6, 3>, PADDED>(f, cfg, a, b, c, ctx);
  }
  switch (f.dtype) {
    case SU3_F64: return run_repr<kF64, PADDED>(f, cfg, a, b, c, ctx);
    case SU3_F32: return run_repr<kF32, PADDED>(f, cfg, a, b, c, ctx);
    case SU3_F16: return run_repr<kF16, PADDED>(f, cfg, a, b, c, ctx);
    case SU3_BF16: return run_repr<kBF16, PADDED>(f, cfg, a, b, c, ctx);
  }
  return SU3_ERR_UNSUPPORTED;
}

// a^dagger x b (which = 0), a v (1) and a^dagger v (2) over an AOS FULL18 array (NATIVE
// arithmetic, or FP32 pairs for FP64 storage). For the matrix x vector forms `bv` holds v[j] at bv[18*j .. 18*j+5] and c is the
// packed array of output colour vectors (4 per site).
template <bool PADDED>
static su3_status adjacent_dispatch(int which, const Form& f, const LaunchCfg& cfg, const void* a,
                                    const double* bv, void* c, const LaunchCtx& ctx) {
  const bool pair = f.arith == SU3_ARITH_F32PAIR && f.dtype == SU3_F64;
  if (f.layout != SU3_LAYOUT_AOS || f.repr_in != SU3_REPR_FULL18 || (f.arith != SU3_ARITH_NATIVE && !pair)) {
    *ctx.err = "adjacent operations take AOS FULL18 arrays with NATIVE arithmetic (or F32PAIR for F64)";
    return SU3_ERR_UNSUPPORTED;
  }
  if (pair) {
    if (which == 0) return run_aos<PairAnOp, SU3_LAYOUT_AOS, PADDED>(f, cfg, a, bv, c, ctx);
    if (which == 1) return run_aos<PairMatVecOp<false>, SU3_LAYOUT_AOS, PADDED>(f, cfg, a, bv, c, ctx);
    return run_aos<PairMatVecOp<true>, SU3_LAYOUT_AOS, PADDED>(f, cfg, a, bv, c, ctx);
  }
#define SU3_ADJ_CASES(DT)                                                             \
  case DT:                                                                            \
    if (which == 0) return run_aos<AnOp<DT>, SU3_LAYOUT_AOS, PADDED>(f, cfg, a, bv, c, ctx);                  \
    if (which == 1) return run_aos<MatVecOp<DT, false>, SU3_LAYOUT_AOS, PADDED>(f, cfg, a, bv, c, ctx);       \
    return run_aos<MatVecOp<DT, true>, SU3_LAYOUT_AOS, PADDED>(f, cfg, a, bv, c, ctx);
  switch (f.dtype) {
    SU3_ADJ_CASES(kF64)
    SU3_ADJ_CASES(kF32)
    SU3_ADJ_CASES(kF16)
    SU3_ADJ_CASES(kBF16)
  }
#undef SU3_ADJ_CASES
  return SU3_ERR_UNSUPPORTED;
}

}  // namespace su3
