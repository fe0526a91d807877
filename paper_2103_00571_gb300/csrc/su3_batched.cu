// Batched SU3_Bench link multiply: many independent lattices (uneven extents, FP64 or FP32
// storage, each with its own four b matrices) in ONE persistent launch.
//
// The tiles of all lattices form one global work list (lattice l owns tiles
// first_tile[l] .. first_tile[l+1]-1). A tile is one shared-memory stage of bytes: tile_sites FP64
// sites or 2 * tile_sites FP32 sites. Each CTA strides over that list with the same shared-memory
// bulk-copy ring as the single-lattice AOS kernel; the thread issuing a tile's copy looks its
// lattice up (a galloping search forward from the previous tile's lattice, since a CTA's tiles
// come in increasing order) and leaves (lattice, first site, sites) next to the stage, where the
// computing threads read it after the stage's mbarrier completes. Each tile's link products use
// that lattice's b (read through the L1 cache; FP32 lattices round it to FP32 once per load); a
// thread computes whole links, or single output rows when the launch has threads_per_link 3.
#include <cuda_runtime.h>

#include <string.h>

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <mutex>

#include "su3_device.cuh"
#include "su3_internal.h"

namespace su3 {

struct TileInfo {
  int lattice;
  int nt;  // sites in this tile
  long long first_site;
};

struct BatchArgs {
  float unit;  // 1.0 for FP32-pair arithmetic (a parameter, so the compiler cannot fold it)
  const BatchDesc* descs;
  int n;
  int total_tiles;
  int tile_sites;
  int stages;
  unsigned stage_bytes;
  unsigned* status;
};

constexpr int kBatchHeader = 1024;  // mbarriers (<= 8) + TileInfo per stage (<= 8 x 16 B)

// Work item q of a tile with `links` links and TPL threads per link (1, or 3 = one per row): the
// items are ordered row-major over (row, link), so an item's direction j = q % 4 = tid % 4.
template <int TPL>
__device__ __forceinline__ void batch_item(int q, int links, int& row, int& link) {
  row = 0;
  if (TPL >= 2 && q >= links) row = 1;
  if (TPL >= 3 && q >= 2 * links) row = 2;
  link = q - row * links;
}

template <int DT, int TPL>
__device__ __forceinline__ void batch_tile_compute(unsigned char* in, int nt, const BatchDesc& d) {
  using S = Storage<DT>;
  using A = typename S::acc;
  using V = typename S::vec;
  constexpr int kLink = 9 * (int)sizeof(V);
  const int j = threadIdx.x & 3;
  A bre[9], bim[9];
#pragma unroll
  for (int e = 0; e < 9; ++e) {
    bre[e] = (A)__ldg(&d.b[18 * j + 2 * e]);
    bim[e] = (A)__ldg(&d.b[18 * j + 2 * e + 1]);
  }
  const int links = 4 * nt;
  for (int q = threadIdx.x; q < TPL * links; q += blockDim.x) {
    int row, link;
    batch_item<TPL>(q, links, row, link);
    V* p = reinterpret_cast<V*>(in + (size_t)link * kLink);
    if constexpr (TPL == 1) {
      Link<A> la, lc;
#pragma unroll
      for (int e = 0; e < 9; ++e) S::unpack(p[e], la.re[e], la.im[e]);
      link_mult<3>(la, bre, bim, lc);
#pragma unroll
      for (int e = 0; e < 9; ++e) p[e] = S::pack(lc.re[e], lc.im[e]);
    } else {
      A are[3], aim[3], cre[3], cim[3];
#pragma unroll
      for (int m = 0; m < 3; ++m) S::unpack(p[3 * row + m], are[m], aim[m]);
      row_mult(are, aim, bre, bim, cre, cim);
#pragma unroll
      for (int l = 0; l < 3; ++l) p[3 * row + l] = S::pack(cre[l], cim[l]);
    }
  }
}

// FP64 lattice in FP32-pair arithmetic: b comes pre-split in the descriptor.
template <int TPL>
__device__ __forceinline__ void batch_tile_compute_pair(unsigned char* in, int nt, const BatchDesc& d, float unit) {
  PairF64Op<9, 3> op;
  op.init_pre(d.bpair + 36 * (threadIdx.x & 3));
  op.set_unit(unit);
  const int links = 4 * nt;
  for (int q = threadIdx.x; q < TPL * links; q += blockDim.x) {
    int row, link;
    batch_item<TPL>(q, links, row, link);
    double2* p = reinterpret_cast<double2*>(in + (size_t)link * 144);
    if constexpr (TPL == 1) op.apply(p, p);
    else op.apply_row(p, p, row);
  }
}

template <int TPL>
__global__ void __launch_bounds__(256) su3_batched_kernel(const __grid_constant__ BatchArgs p) {
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);
  TileInfo* info = reinterpret_cast<TileInfo*>(smem + 128);
  unsigned char* stage0 = smem + kBatchHeader;
  const int tid = threadIdx.x;
  const int S_ = p.stages;
  if (tid == 0) {
    for (int s = 0; s < S_; ++s) mbar_init(&full[s], 1);
    fence_mbar_init();
  }
  __syncthreads();
  const uint64_t pol = policy_evict_first();
  const int my_tiles =
      p.total_tiles > (int)blockIdx.x ? (p.total_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

  // thread 0 only: find the tile's lattice, record it beside the stage, start the copy
  int cur = 0;  // lattice of the previous tile (thread 0's state): tiles come in increasing order
  auto issue_load = [&](int k) {
    const int t = (int)blockIdx.x + k * (int)gridDim.x;
    // last lattice with first_tile <= t: gallop forward from cur, then bisect
    int lo = cur, step = 1;
    while (lo + step < p.n && p.descs[lo + step].first_tile <= t) {
      lo += step;
      step <<= 1;
    }
    int hi = min(lo + step, p.n) - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (p.descs[mid].first_tile <= t) lo = mid; else hi = mid - 1;
    }
    cur = lo;
    const BatchDesc& d = p.descs[lo];
    const int ts = batch_tile_sites(d.dtype, p.tile_sites);
    const long long first = (long long)(t - d.first_tile) * ts;
    long long rest = d.n_sites - first;
    const int nt = (int)(rest < ts ? rest : ts);
    const int s = k % S_;
    info[s].lattice = lo;
    info[s].nt = nt > 0 ? nt : 0;
    info[s].first_site = first;
    const long long site_bytes = d.dtype == SU3_F64 ? 576 : 288;
    const unsigned bytes = (unsigned)(info[s].nt * site_bytes);
    mbar_arrive_expect_tx(&full[s], bytes);
    if (bytes) bulk_g2s(stage0 + (size_t)s * p.stage_bytes, static_cast<const unsigned char*>(d.a) + first * site_bytes,
                        bytes, &full[s], pol);
  };

  const int prefetch = S_ - 1;
  int issued = my_tiles < prefetch ? my_tiles : prefetch;
  if (tid == 0)
    for (int k = 0; k < issued; ++k) issue_load(k);

  int kfail = -1;
  for (int k = 0; k < my_tiles; ++k) {
    const int s = k % S_;
    const bool ok = mbar_wait_bounded(&full[s], (unsigned)((k / S_) & 1));
    unsigned char* in = stage0 + (size_t)s * p.stage_bytes;
    const TileInfo ti = info[s];
    const BatchDesc& d = p.descs[ti.lattice];
    const int dtype = d.dtype;
    if (ok) {
      if (dtype == SU3_F64) {
        if (d.arith == SU3_ARITH_F32PAIR) batch_tile_compute_pair<TPL>(in, ti.nt, d, p.unit);
        else batch_tile_compute<kF64, TPL>(in, ti.nt, d);
      } else {
        batch_tile_compute<kF32, TPL>(in, ti.nt, d);
      }
    }
    fence_proxy_async_smem();
    if (__syncthreads_or(!ok)) {
      kfail = k;
      break;
    }
    if (tid < 32) {
      if (tid == 0 && ti.nt > 0) {
        const long long site_bytes = dtype == SU3_F64 ? 576 : 288;
        bulk_s2g(static_cast<unsigned char*>(d.c) + ti.first_site * site_bytes, in, (unsigned)(ti.nt * site_bytes), pol);
      }
      bulk_commit();
      bulk_wait_read<1>();
      __syncwarp();
      if (tid == 0 && issued < my_tiles) issue_load(issued++);
    }
  }
  if (kfail >= 0 && tid == 0) {
    atomicOr(p.status, kDevErrTimeout);
    // let the loads still in flight land before shared memory is released (bounded)
    for (int k = kfail; k < issued; ++k) mbar_wait_bounded(&full[k % S_], (unsigned)((k / S_) & 1));
  }
  if (tid < 32) bulk_wait_all<0>();
}

BatchCfg default_batch_cfg() {
  // measured best on GB300 for the 96-lattice FP64/FP32 mix (and for its FP32-pair variant):
  // four 64-thread CTAs per SM, 32-site (18 KB) stages, three deep
  BatchCfg c;
  c.block = 64;
  c.tile_sites = 32;
  c.stages = 3;
  c.ctas_per_sm = 4;
  return c;
}

int batch_tile_count(long long n_sites, int dtype, int tile_sites) {
  const int ts = batch_tile_sites(dtype, tile_sites);
  return (int)((n_sites + ts - 1) / ts);
}

static size_t batch_smem(const BatchCfg& cfg) {
  return kBatchHeader + (size_t)cfg.stages * (((size_t)cfg.tile_sites * 576 + 127) / 128 * 128);
}

su3_status prepare_batched(const BatchCfg& cfg, std::string* err) {
  const size_t smem = batch_smem(cfg);
  if (smem > 227 * 1024 || cfg.stages < 2 || cfg.stages > 8 || cfg.tile_sites < 1 || cfg.block < 32 ||
      cfg.block > 256 || cfg.block % 32) {
    *err = "batched launch configuration exceeds shared memory, stage or block limits";
    return SU3_ERR_INVALID_ARG;
  }
  if (cfg.threads_per_link != 1 && cfg.threads_per_link != 3) {
    *err = "batched threads_per_link must be 1 or 3";
    return SU3_ERR_INVALID_ARG;
  }
  cudaError_t e = cudaFuncSetAttribute(cfg.threads_per_link == 3 ? su3_batched_kernel<3> : su3_batched_kernel<1>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) {
    *err = std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e);
    return SU3_ERR_CUDA;
  }
  return SU3_OK;
}

su3_status launch_batched(const BatchDesc* descs_dev, int n, int total_tiles, const BatchCfg& cfg,
                          const LaunchCtx& ctx) {
  if (total_tiles == 0) return SU3_OK;
  BatchArgs p;
  p.unit = 1.0f;
  p.descs = descs_dev;
  p.n = n;
  p.total_tiles = total_tiles;
  p.tile_sites = cfg.tile_sites;
  p.stages = cfg.stages;
  p.stage_bytes = (unsigned)(((long long)cfg.tile_sites * 576 + 127) / 128 * 128);
  p.status = ctx.status;
  const size_t smem = batch_smem(cfg);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(ctx.stream, &cs);
  if (cs == cudaStreamCaptureStatusNone) {
    su3_status s = prepare_batched(cfg, ctx.err);
    if (s != SU3_OK) return s;
  }
  cudaError_t e;
  const int grid = std::min(total_tiles, ctx.num_sms * cfg.ctas_per_sm);
  if (cfg.threads_per_link == 3) su3_batched_kernel<3><<<grid, cfg.block, smem, ctx.stream>>>(p);
  else su3_batched_kernel<1><<<grid, cfg.block, smem, ctx.stream>>>(p);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    *ctx.err = std::string("su3_batched_kernel launch: ") + cudaGetErrorString(e);
    return SU3_ERR_CUDA;
  }
  ++*ctx.launches;
  return SU3_OK;
}

}  // namespace su3

// ---- su3_mult_batched_static: the batched launch without any device allocation -----------------
//
// The descriptor table and the status word live in a file-scope device array instead of handle
// memory. Layout: bytes [0, 256) hold the status word (first 4 bytes), then up to
// SU3_STATIC_MAX_LATTICES BatchDesc entries. Host code never uses the array's name as an address:
// it asks the runtime for the device address once per device (cudaGetSymbolAddress, with that
// device current) and passes that pointer to the kernel.

namespace su3 {

static_assert(sizeof(BatchDesc) == 1192, "the static area's documented size assumes 1192-byte descriptors");
constexpr size_t kStaticHeader = 256;
constexpr size_t kStaticBytes = kStaticHeader + (size_t)SU3_STATIC_MAX_LATTICES * sizeof(BatchDesc);

static __device__ __align__(256) unsigned char g_su3_static_area[kStaticBytes];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_static_mu;    // guards the per-device addresses below
std::mutex g_static_call;  // held for a whole call: the host table is reused by the next call
unsigned char* g_static_addr[kMaxDevices] = {};
int g_static_sms[kMaxDevices] = {};
// Host copy of the descriptor table: filled completely, uploaded with one copy, and kept alive
// (under g_static_call) until the call has waited for its stream, so the copy never reads a
// source that changes under it, whether or not the driver staged it.
BatchDesc g_static_host[SU3_STATIC_MAX_LATTICES];
}  // namespace

// Device address of the static area on the current device (looked up once per device).
static cudaError_t static_area(int dev, unsigned char** addr, int* sms) {
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_su3_static_area);
    if (e != cudaSuccess) return e;
    int n = 0;
    e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    g_static_addr[dev] = static_cast<unsigned char*>(p);
    g_static_sms[dev] = n;
  }
  *addr = g_static_addr[dev];
  *sms = g_static_sms[dev];
  return cudaSuccess;
}

}  // namespace su3

namespace su3 {
static su3_status mult_batched_static_impl(int32_t n, const su3_batch_item* items, void* stream);
}  // namespace su3

extern "C" su3_status su3_mult_batched_static(int32_t n, const su3_batch_item* items, void* stream) {
  using namespace su3;
  nvtxRangePushA("su3_mult_batched_static");
  const su3_status s = mult_batched_static_impl(n, items, stream);
  nvtxRangePop();
  return s;
}

namespace su3 {

static su3_status mult_batched_static_impl(int32_t n, const su3_batch_item* items, void* stream) {
  if (n < 0 || (n > 0 && !items)) return SU3_ERR_INVALID_ARG;
  // validate everything and count tiles before touching the GPU
  const BatchCfg cfg = default_batch_cfg();
  int m = 0;
  long long tiles = 0;
  for (int i = 0; i < n; ++i) {
    const su3_desc& d = items[i].desc;
    if (su3_check_desc(&d) != SU3_OK) return SU3_ERR_INVALID_ARG;
    if ((d.dtype != SU3_F64 && d.dtype != SU3_F32) || d.repr != SU3_REPR_FULL18 || d.layout != SU3_LAYOUT_AOS ||
        (d.arith != SU3_ARITH_NATIVE && !(d.arith == SU3_ARITH_F32PAIR && d.dtype == SU3_F64)) ||
        (d.site_stride_bytes != 0 && d.site_stride_bytes != 4 * link_bytes(d.dtype, d.repr)))
      return SU3_ERR_UNSUPPORTED;
    if (d.n_sites == 0) continue;
    const void* a = items[i].a_dev;
    const void* c = items[i].c_dev;
    if (!a || !c || ((uintptr_t)a & 15u) || ((uintptr_t)c & 15u)) return SU3_ERR_INVALID_ARG;
    const uintptr_t nb = (uintptr_t)(d.n_sites * 4 * link_bytes(d.dtype, d.repr));
    if (a != c && (uintptr_t)a < (uintptr_t)c + nb && (uintptr_t)c < (uintptr_t)a + nb) return SU3_ERR_INVALID_ARG;
    ++m;
    tiles += batch_tile_count(d.n_sites, d.dtype, cfg.tile_sites);
  }
  if (m > SU3_STATIC_MAX_LATTICES || tiles > (1ll << 30)) return SU3_ERR_INVALID_ARG;
  if (m == 0) return SU3_OK;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SU3_ERR_CUDA;
  unsigned char* area = nullptr;
  int sms = 0;
  if (static_area(dev, &area, &sms) != cudaSuccess) return SU3_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)stream;

  // one call at a time in this process: the host table and the device area are shared
  std::lock_guard<std::mutex> call_lock(g_static_call);
  BatchDesc* host = g_static_host;
  int filled = 0, first_tile = 0;
  for (int i = 0; i < n; ++i) {
    const su3_batch_item& it = items[i];
    if (it.desc.n_sites == 0) continue;
    BatchDesc& o = host[filled++];
    o.a = it.a_dev;
    o.c = it.c_dev;
    o.n_sites = it.desc.n_sites;
    o.dtype = it.desc.dtype;
    o.first_tile = first_tile;
    o.arith = it.desc.arith;
    o.reserved = 0;
    memcpy(o.b, it.b, sizeof(o.b));
    split_b_pairs(&it.b[0][0][0][0], o.bpair);
    first_tile += batch_tile_count(it.desc.n_sites, it.desc.dtype, cfg.tile_sites);
  }
  // clear the status word, then upload the whole table in one copy
  if (cudaMemsetAsync(area, 0, sizeof(unsigned), st) != cudaSuccess) return SU3_ERR_CUDA;
  BatchDesc* table = reinterpret_cast<BatchDesc*>(area + kStaticHeader);
  if (cudaMemcpyAsync(table, host, sizeof(BatchDesc) * filled, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return SU3_ERR_CUDA;
  std::string err;
  int64_t launches = 0;
  LaunchCtx ctx;
  ctx.stream = st;
  ctx.status = reinterpret_cast<unsigned*>(area);
  ctx.num_sms = sms;
  ctx.launches = &launches;
  ctx.err = &err;
  su3_status s = launch_batched(table, m, first_tile, cfg, ctx);
  // wait even when the launch failed: the table copy must be done before the lock is released
  const cudaError_t se = cudaStreamSynchronize(st);
  if (s != SU3_OK) return s;
  if (se != cudaSuccess) return SU3_ERR_CUDA;
  unsigned word = 0;
  if (cudaMemcpy(&word, area, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess) return SU3_ERR_CUDA;
  return word ? SU3_ERR_TIMEOUT : SU3_OK;
}

}  // namespace su3
