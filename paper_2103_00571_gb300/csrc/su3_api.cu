// libsu3 C ABI: handle, argument validation, dispatch, completion and error reporting, the
// host-buffer path and the batched/graph path. The operation itself is the SU3_Bench link multiply
// (arXiv 2103.00571, §Background "SU3_Bench"); the kernels live in su3_stream.cu,
// su3_batched.cu and su3_pack.cu.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <map>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "su3.h"
#include "su3_internal.h"

using namespace su3;

namespace su3 {
// Times `grid` CTAs of 256 threads, each thread running 8 independent FP64 FMA chains of `steps`
// FMAs (diagnostic: the device's sustained FP64 FMA rate); out_dev holds grid * 256 doubles.
// Defined in su3_diag.cu.
su3_status measure_dfma_rate(int steps, double* out_dev, int grid, const LaunchCtx& ctx, float* ms);
}  // namespace su3

namespace {

// NVTX range over one entry point: names the call in Nsight timelines and in ncu's NVTX
// filters; the header-only NVTX3 calls do nothing unless a profiling tool is attached.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Runs one entry point on the handle's device and gives the calling thread its current device
// back afterwards (a no-op when the handle's device is already current).
struct DeviceScope {
  int prev = -1;
  explicit DeviceScope(int dev) {
    int cur = -1;
    if (cudaGetDevice(&cur) == cudaSuccess && cur != dev && cudaSetDevice(dev) == cudaSuccess) prev = cur;
  }
  ~DeviceScope() {
    if (prev >= 0) cudaSetDevice(prev);
  }
  DeviceScope(const DeviceScope&) = delete;
  DeviceScope& operator=(const DeviceScope&) = delete;
};

enum FaultPoint { kFaultNone = 0, kFaultLaunch = 1, kFaultAlloc = 2, kFaultCopy = 4, kFaultSync = 8 };

int parse_fault_env() {
  const char* v = getenv("SU3_FAULT_INJECT");
  if (!v) return kFaultNone;
  int f = 0;
  std::string s(v);
  if (s.find("launch") != std::string::npos) f |= kFaultLaunch;
  if (s.find("alloc") != std::string::npos) f |= kFaultAlloc;
  if (s.find("copy") != std::string::npos) f |= kFaultCopy;
  if (s.find("sync") != std::string::npos) f |= kFaultSync;
  return f;
}

constexpr int kHostBuffers = 3;

}  // namespace

struct su3_handle {
  int device = 0;
  int num_sms = 0;
  int smem_per_sm = 0, smem_reserved = 0;
  unsigned* status_dev = nullptr;
  int64_t launches = 0;
  std::string err;
  int fault = 0;
  std::map<std::tuple<int, int, int, int, int, int>, LaunchCfg> cfgs;  // CfgKey
  // batched, direct mode
  BatchDesc* bdesc_dev = nullptr;
  BatchDesc* bdesc_host = nullptr;  // pinned
  int bcap = 0;
  cudaEvent_t bcopy_done = nullptr;   // the last upload has read the pinned host table
  bool bcopy_pending = false;
  cudaEvent_t bkern_done = nullptr;   // the last direct-mode kernel has finished with bdesc_dev
  bool bkern_pending = false;
  // batched, graph mode (its own descriptor buffers: a replay re-reads them)
  BatchDesc* gdesc_dev = nullptr;
  BatchDesc* gdesc_host = nullptr;
  int gcap = 0;
  cudaGraphExec_t gexec = nullptr;
  std::vector<char> gkey;
  cudaStream_t cap_stream = nullptr;
  BatchCfg bcfg;
  // host-buffer path
  unsigned char* hbuf_dev[kHostBuffers] = {nullptr, nullptr, nullptr};
  size_t hbuf_bytes = 0;
  cudaStream_t s_h2d = nullptr, s_comp = nullptr, s_d2h = nullptr;
  cudaEvent_t ev_h2d[kHostBuffers] = {}, ev_comp[kHostBuffers] = {}, ev_d2h[kHostBuffers] = {};
  cudaEvent_t ev_start = nullptr;
  int host_path = SU3_HOST_AUTO;  // su3_set_host_path
  int host_path_used = 0;         // the path the last su3_mult_host call took
  bool pageable_access = false;   // the device reads pageable host memory coherently
};

namespace {

su3_status fail(su3_handle* h, su3_status s, const std::string& msg) {
  if (h) h->err = msg;
  return s;
}

su3_status cuda_err(su3_handle* h, const char* what, cudaError_t e) {
  return fail(h, SU3_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

LaunchCtx ctx_of(su3_handle* h, cudaStream_t st) {
  LaunchCtx c;
  c.stream = st;
  c.status = h->status_dev;
  c.num_sms = h->num_sms;
  c.smem_per_sm = h->smem_per_sm;
  c.smem_reserved = h->smem_reserved;
  c.launches = &h->launches;
  c.err = &h->err;
  return c;
}

// Launch configurations are kept per (dtype, repr of a, repr of c, layout, arith, padded): an AOS
// site stride wider than the links (the paper's 640-byte FP64 site) moves each site's links in
// bulk copies of their own and gets its own configuration, and so does two-row in, full out (its kernel also keeps an
// output ring and, in FP32 pairs, needs more registers than two-row in and out).
using CfgKey = std::tuple<int, int, int, int, int, int>;
CfgKey form_key(const su3_desc* d, int repr_out) {
  const bool padded = d->layout == SU3_LAYOUT_AOS && d->site_stride_bytes != 0 &&
                      d->site_stride_bytes != 4 * link_bytes(d->dtype, d->repr);
  return std::make_tuple((int)d->dtype, (int)d->repr, repr_out, (int)d->layout, (int)d->arith, padded ? 1 : 0);
}
CfgKey form_key(const su3_desc* d) { return form_key(d, d->repr); }

int64_t resolved_stride(const su3_desc* d) {
  if (d->layout != SU3_LAYOUT_AOS) return 0;
  return d->site_stride_bytes ? d->site_stride_bytes : 4 * link_bytes(d->dtype, d->repr);
}

su3_status check_cfg(su3_handle* h, const Form& f, const LaunchCfg& c) {
  if (c.block < 32 || c.block > 256 || c.block % 32)
    return fail(h, SU3_ERR_INVALID_ARG, "block must be a multiple of 32 in [32, 256]");
  if (c.ctas_per_sm < 1 || c.ctas_per_sm > 32) return fail(h, SU3_ERR_INVALID_ARG, "ctas_per_sm must be in [1, 32]");
  if (c.native_permille < 0 || c.native_permille > 1000)
    return fail(h, SU3_ERR_INVALID_ARG, "native_permille must be in [0, 1000]");
  if (f.layout == SU3_LAYOUT_AOS || c.stages != 0) {  // the staged kernel
    if (c.threads_per_link != 1 && c.threads_per_link != 3)
      return fail(h, SU3_ERR_INVALID_ARG, "threads_per_link must be 1 (per link) or 3 (one thread per output row)");
    if (c.stages < 2 || c.stages > 8) return fail(h, SU3_ERR_INVALID_ARG, "stages must be in [2, 8]");
    if (c.tile_sites < 1 || c.tile_sites > 1024) return fail(h, SU3_ERR_INVALID_ARG, "tile_sites must be in [1, 1024]");
    const int64_t site_bytes = f.layout == SU3_LAYOUT_AOS ? f.a_stride : 4 * link_bytes(f.dtype, f.repr_in);
    if ((int64_t)c.tile_sites * site_bytes > (1 << 20))
      return fail(h, SU3_ERR_INVALID_ARG, "a tile may not exceed 1 MiB");
    if (f.layout == SU3_LAYOUT_AOSOA32 && c.tile_sites % 8)
      return fail(h, SU3_ERR_INVALID_ARG, "AOSOA32 tiles must be a multiple of 8 sites (whole 32-link blocks)");
    if (f.layout == SU3_LAYOUT_SOA && c.tile_sites > 64)
      return fail(h, SU3_ERR_INVALID_ARG, "SOA tiles hold at most 64 sites (256 links per element plane)");
  } else if (c.tile_sites != 1 && c.tile_sites != 2 && c.tile_sites != 4) {  // direct loads
    return fail(h, SU3_ERR_INVALID_ARG, "links per thread (tile_sites) must be 1, 2 or 4 for SOA/AOSOA32 direct loads");
  } else if (c.threads_per_link != 1) {
    return fail(h, SU3_ERR_INVALID_ARG, "threads_per_link must be 1 for SOA/AOSOA32 direct loads");
  }
  return SU3_OK;
}

// The configuration of the (a, c) repr pair, else that of a's repr in and out, else the default.
LaunchCfg cfg_for(su3_handle* h, const su3_desc* d, const Form& f) {
  auto it = h->cfgs.find(form_key(d, f.repr_out));
  if (it == h->cfgs.end() && f.repr_out != d->repr) it = h->cfgs.find(form_key(d));
  if (it != h->cfgs.end()) return it->second;
  return default_cfg(f);
}

// Validates an (a, c) descriptor pair into a Form.
su3_status make_form(su3_handle* h, const su3_desc* ad, const su3_desc* cd, Form* f) {
  su3_status s = su3_check_desc(ad);
  if (s != SU3_OK) return fail(h, s, "invalid a descriptor (dtype/repr/layout/arith/n_sites/stride)");
  s = su3_check_desc(cd);
  if (s != SU3_OK) return fail(h, s, "invalid c descriptor (dtype/repr/layout/arith/n_sites/stride)");
  if (ad->dtype != cd->dtype || ad->layout != cd->layout || ad->arith != cd->arith || ad->n_sites != cd->n_sites)
    return fail(h, SU3_ERR_INVALID_ARG, "a and c must share dtype, layout, arith and n_sites");
  if (ad->repr == SU3_REPR_FULL18 && cd->repr != SU3_REPR_FULL18)
    return fail(h, SU3_ERR_UNSUPPORTED, "FULL18 input needs FULL18 output");
  f->dtype = ad->dtype;
  f->repr_in = ad->repr;
  f->repr_out = cd->repr;
  f->layout = ad->layout;
  f->arith = ad->arith;
  f->n_sites = ad->n_sites;
  f->a_stride = resolved_stride(ad);
  f->c_stride = resolved_stride(cd);
  return SU3_OK;
}

bool ranges_overlap(const void* a, int64_t an, const void* b, int64_t bn) {
  const uintptr_t a0 = (uintptr_t)a, b0 = (uintptr_t)b;
  return a0 < b0 + (uintptr_t)bn && b0 < a0 + (uintptr_t)an;
}

}  // namespace

extern "C" {

int32_t su3_abi_version(void) { return SU3_ABI_VERSION; }

const char* su3_status_string(su3_status s) {
  switch (s) {
    case SU3_OK: return "SU3_OK";
    case SU3_ERR_INVALID_ARG: return "SU3_ERR_INVALID_ARG";
    case SU3_ERR_UNSUPPORTED: return "SU3_ERR_UNSUPPORTED";
    case SU3_ERR_CUDA: return "SU3_ERR_CUDA";
    case SU3_ERR_NOT_INITIALIZED: return "SU3_ERR_NOT_INITIALIZED";
    case SU3_ERR_TIMEOUT: return "SU3_ERR_TIMEOUT";
    case SU3_ERR_FAULT_INJECTED: return "SU3_ERR_FAULT_INJECTED";
  }
  return "SU3_ERR_UNKNOWN";
}

const char* su3_last_error(const su3_handle* h) { return h ? h->err.c_str() : "null handle"; }

int64_t su3_launch_count(const su3_handle* h) { return h ? h->launches : 0; }

int64_t su3_link_bytes(int32_t dtype, int32_t repr) {
  if (dtype < SU3_F64 || dtype > SU3_BF16 || repr < SU3_REPR_FULL18 || repr > SU3_REPR_TWOROW12) return 0;
  return link_bytes(dtype, repr);
}

su3_status su3_check_desc(const su3_desc* d) {
  if (!d) return SU3_ERR_INVALID_ARG;
  if (d->dtype < SU3_F64 || d->dtype > SU3_BF16) return SU3_ERR_INVALID_ARG;
  if (d->repr < SU3_REPR_FULL18 || d->repr > SU3_REPR_TWOROW12) return SU3_ERR_INVALID_ARG;
  if (d->layout < SU3_LAYOUT_AOS || d->layout > SU3_LAYOUT_SOA) return SU3_ERR_INVALID_ARG;
  if (d->arith < SU3_ARITH_NATIVE || d->arith > SU3_ARITH_HYBRID) return SU3_ERR_INVALID_ARG;
  if (d->arith != SU3_ARITH_NATIVE && d->dtype != SU3_F64) return SU3_ERR_INVALID_ARG;
  if (d->n_sites < 0 || d->n_sites > ((int64_t)1 << 36)) return SU3_ERR_INVALID_ARG;
  const int64_t lb = link_bytes(d->dtype, d->repr);
  if (d->layout == SU3_LAYOUT_AOS) {
    if (d->site_stride_bytes != 0 && (d->site_stride_bytes < 4 * lb || d->site_stride_bytes % 16 != 0))
      return SU3_ERR_INVALID_ARG;
  } else if (d->site_stride_bytes != 0) {
    return SU3_ERR_INVALID_ARG;
  }
  return SU3_OK;
}

int64_t su3_array_bytes(const su3_desc* d) {
  if (su3_check_desc(d) != SU3_OK) return -1;
  const int64_t lb = link_bytes(d->dtype, d->repr);
  switch (d->layout) {
    case SU3_LAYOUT_AOS: return d->n_sites * resolved_stride(d);
    case SU3_LAYOUT_SOA: return 4 * d->n_sites * lb;
    case SU3_LAYOUT_AOSOA32: return (4 * d->n_sites + 31) / 32 * 32 * lb;
  }
  return -1;
}

su3_status su3_init(int device, su3_handle** out) {
  if (!out) return SU3_ERR_INVALID_ARG;
  *out = nullptr;
  su3_handle* h = new su3_handle();
  h->fault = parse_fault_env();
  h->device = device;
  h->bcfg = default_batch_cfg();
  if (h->fault & kFaultAlloc) {
    delete h;
    return SU3_ERR_FAULT_INJECTED;
  }
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&h->smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&h->smem_reserved, cudaDevAttrReservedSharedMemoryPerBlock, device);
  if (e == cudaSuccess) {
    int pma = 0;
    e = cudaDeviceGetAttribute(&pma, cudaDevAttrPageableMemoryAccess, device);
    h->pageable_access = (e == cudaSuccess && pma != 0);
  }
  if (e == cudaSuccess) e = cudaMalloc((void**)&h->status_dev, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemset(h->status_dev, 0, sizeof(unsigned));
  if (e != cudaSuccess) {
    if (h->status_dev) cudaFree(h->status_dev);
    delete h;
    cudaGetLastError();
  } else {
    *out = h;
  }
  if (prev >= 0 && prev != device) cudaSetDevice(prev);
  return e == cudaSuccess ? SU3_OK : SU3_ERR_CUDA;
}

su3_status su3_finalize(su3_handle* h) {
  if (!h) return SU3_OK;
  DeviceScope scope(h->device);
  cudaDeviceSynchronize();
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  cudaFree(h->bdesc_dev);
  cudaFreeHost(h->bdesc_host);
  cudaFree(h->gdesc_dev);
  cudaFreeHost(h->gdesc_host);
  if (h->bcopy_done) cudaEventDestroy(h->bcopy_done);
  if (h->bkern_done) cudaEventDestroy(h->bkern_done);
  for (int i = 0; i < kHostBuffers; ++i) {
    cudaFree(h->hbuf_dev[i]);
    if (h->ev_h2d[i]) cudaEventDestroy(h->ev_h2d[i]);
    if (h->ev_comp[i]) cudaEventDestroy(h->ev_comp[i]);
    if (h->ev_d2h[i]) cudaEventDestroy(h->ev_d2h[i]);
  }
  if (h->ev_start) cudaEventDestroy(h->ev_start);
  if (h->s_h2d) cudaStreamDestroy(h->s_h2d);
  if (h->s_comp) cudaStreamDestroy(h->s_comp);
  if (h->s_d2h) cudaStreamDestroy(h->s_d2h);
  cudaFree(h->status_dev);
  delete h;
  return SU3_OK;
}

namespace {

// The Form a configuration for (a_form -> repr_out) is validated against.
su3_status cfg_form(su3_handle* h, const su3_desc* form, int repr_out, Form* f) {
  if (su3_check_desc(form) != SU3_OK) return fail(h, SU3_ERR_INVALID_ARG, "invalid form descriptor");
  if (repr_out != SU3_REPR_FULL18 && repr_out != SU3_REPR_TWOROW12)
    return fail(h, SU3_ERR_INVALID_ARG, "invalid c representation");
  if (form->repr == SU3_REPR_FULL18 && repr_out != SU3_REPR_FULL18)
    return fail(h, SU3_ERR_UNSUPPORTED, "FULL18 input needs FULL18 output");
  *f = Form{};
  f->dtype = form->dtype;
  f->repr_in = form->repr;
  f->repr_out = repr_out;
  f->layout = form->layout;
  f->arith = form->arith;
  f->n_sites = form->n_sites;
  f->a_stride = f->c_stride = resolved_stride(form);
  return SU3_OK;
}

su3_status set_cfg(su3_handle* h, const su3_desc* form, int repr_out, const su3_launch_cfg* cfg) {
  if (!h) return SU3_ERR_NOT_INITIALIZED;
  if (!form || !cfg) return fail(h, SU3_ERR_INVALID_ARG, "null form or cfg");
  Form f;
  su3_status s = cfg_form(h, form, repr_out, &f);
  if (s != SU3_OK) return s;
  LaunchCfg c = default_cfg(f);
  if (cfg->block) c.block = cfg->block;
  if (cfg->tile_sites) c.tile_sites = cfg->tile_sites;
  if (cfg->stages) c.stages = cfg->stages;
  if (cfg->ctas_per_sm) c.ctas_per_sm = cfg->ctas_per_sm;
  if (cfg->native_permille) c.native_permille = cfg->native_permille;
  if (cfg->threads_per_link) c.threads_per_link = cfg->threads_per_link;
  s = check_cfg(h, f, c);
  if (s != SU3_OK) return s;
  h->cfgs[form_key(form, repr_out)] = c;
  return SU3_OK;
}

su3_status get_cfg(su3_handle* h, const su3_desc* form, int repr_out, su3_launch_cfg* cfg) {
  if (!h) return SU3_ERR_NOT_INITIALIZED;
  if (!form || !cfg) return fail(h, SU3_ERR_INVALID_ARG, "null form or cfg");
  Form f;
  su3_status s = cfg_form(h, form, repr_out, &f);
  if (s != SU3_OK) return s;
  LaunchCfg c = cfg_for(h, form, f);
  cfg->block = c.block;
  cfg->tile_sites = c.tile_sites;
  cfg->stages = c.stages;
  cfg->ctas_per_sm = c.ctas_per_sm;
  cfg->native_permille = c.native_permille;
  cfg->threads_per_link = c.threads_per_link;
  return SU3_OK;
}

}  // namespace

su3_status su3_set_launch_cfg(su3_handle* h, const su3_desc* form, const su3_launch_cfg* cfg) {
  return set_cfg(h, form, form ? form->repr : 0, cfg);
}

su3_status su3_get_launch_cfg(su3_handle* h, const su3_desc* form, su3_launch_cfg* cfg) {
  return get_cfg(h, form, form ? form->repr : 0, cfg);
}

su3_status su3_set_launch_cfg_for(su3_handle* h, const su3_desc* a_form, const su3_desc* c_form,
                                  const su3_launch_cfg* cfg) {
  if (h && !c_form) return fail(h, SU3_ERR_INVALID_ARG, "null c form");
  return set_cfg(h, a_form, c_form ? c_form->repr : 0, cfg);
}

su3_status su3_get_launch_cfg_for(su3_handle* h, const su3_desc* a_form, const su3_desc* c_form,
                                  su3_launch_cfg* cfg) {
  if (h && !c_form) return fail(h, SU3_ERR_INVALID_ARG, "null c form");
  return get_cfg(h, a_form, c_form ? c_form->repr : 0, cfg);
}

su3_status su3_set_batched_cfg(su3_handle* h, const su3_launch_cfg* cfg) {
  if (!h) return SU3_ERR_NOT_INITIALIZED;
  if (!cfg) return fail(h, SU3_ERR_INVALID_ARG, "null cfg");
  BatchCfg c = h->bcfg;
  if (cfg->block) c.block = cfg->block;
  if (cfg->tile_sites) c.tile_sites = cfg->tile_sites;
  if (cfg->stages) c.stages = cfg->stages;
  if (cfg->ctas_per_sm) c.ctas_per_sm = cfg->ctas_per_sm;
  if (cfg->threads_per_link) c.threads_per_link = cfg->threads_per_link;
  if (c.block < 32 || c.block > 256 || c.block % 32 || c.stages < 2 || c.stages > 8 || c.tile_sites < 1 ||
      c.tile_sites > 256 || c.ctas_per_sm < 1 || c.ctas_per_sm > 32 ||
      (c.threads_per_link != 1 && c.threads_per_link != 3))
    return fail(h, SU3_ERR_INVALID_ARG, "batched cfg out of range (block 32..256 step 32, stages 2..8, "
                                        "tile_sites 1..256, ctas_per_sm 1..32, threads_per_link 1 or 3)");
  h->bcfg = c;
  h->gkey.clear();  // the next graph-mode call captures a new graph
  return SU3_OK;
}

su3_status su3_get_batched_cfg(su3_handle* h, su3_launch_cfg* cfg) {
  if (!h) return SU3_ERR_NOT_INITIALIZED;
  if (!cfg) return fail(h, SU3_ERR_INVALID_ARG, "null cfg");
  cfg->block = h->bcfg.block;
  cfg->tile_sites = h->bcfg.tile_sites;
  cfg->stages = h->bcfg.stages;
  cfg->ctas_per_sm = h->bcfg.ctas_per_sm;
  cfg->native_permille = 0;
  cfg->threads_per_link = h->bcfg.threads_per_link;
  return SU3_OK;
}

su3_status su3_mult(su3_handle* h, const su3_desc* a_desc, const void* a_dev, const double* b,
                    const su3_desc* c_desc, void* c_dev, void* stream) {
  NvtxRange nvtx_range("su3_mult");
  if (!h) return SU3_ERR_NOT_INITIALIZED;
  DeviceScope scope(h->device);
  if (!a_desc || !b) return fail(h, SU3_ERR_INVALID_ARG, "null descriptor or b");
  if (!c_desc) c_desc = a_desc;
  Form f;
  su3_status s = make_form(h, a_desc, c_desc, &f);
  if (s != SU3_OK) return s;
  if (f.n_sites == 0) return SU3_OK;
  if (!a_dev || !c_dev) return fail(h, SU3_ERR_INVALID_ARG, "null a or c");
  if (!aligned16(a_dev) || !aligned16(c_dev)) return fail(h, SU3_ERR_INVALID_ARG, "a and c must be 16-byte aligned");
  const int64_t an = su3_array_bytes(a_desc), cn = su3_array_bytes(c_desc);
  if (a_dev == c_dev) {
    if (a_desc->repr != c_desc->repr || f.a_stride != f.c_stride)
      return fail(h, SU3_ERR_INVALID_ARG, "in-place operation needs identical a and c descriptors");
  } else if (ranges_overlap(a_dev, an, c_dev, cn)) {
    return fail(h, SU3_ERR_INVALID_ARG, "a and c overlap without being the same array");
  }
  if (h->fault & kFaultLaunch) return fail(h, SU3_ERR_FAULT_INJECTED, "fault injected at launch");
  LaunchCfg cfg = cfg_for(h, a_desc, f);
  s = check_cfg(h, f, cfg);
  if (s != SU3_OK) return s;
  return launch_mult(f, cfg, a_dev, b, c_dev, ctx_of(h, (cudaStream_t)stream));
}

su3_status su3_mult_op(su3_handle* h, int32_t op, const su3_desc* a_desc, const void* a_dev, const double* b,
                       const su3_desc* c_desc, void* c_dev, void* stream) {
  NvtxRange nvtx_range("su3_mult_op");
  if (!h) return SU3_ERR_NOT_INITIALIZED;
  DeviceScope scope(h->device);
  if (op == SU3_OP_NN) return su3_mult(h, a_desc, a_dev, b, c_desc, c_dev, stream);
  if (!b) return fail(h, SU3_ERR_INVALID_ARG, "null b");
  if (op == SU3_OP_NA) {
    double bd[72];  // b^dagger: bd[j][k][l] = conj(b[j][l][k]) (exact)
    for (int j = 0; j < 4; ++j)
      for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) {
          bd[18 * j + 6 * k + 2 * l] = b[18 * j + 6 * l + 2 * k];
          bd[18 * j + 6 * k + 2 * l + 1] = -b[18 * j + 6 * l + 2 * k + 1];
        }
    return su3_mult(h, a_desc, a_dev, bd, c_desc, c_dev, stream);
  }
  if (op != SU3_OP_AN) return fail(h, SU3_ERR_INVALID_ARG, "op must be SU3_OP_NN, SU3_OP_NA or SU3_OP_AN");
  if (!a_desc) return fail(h, SU3_ERR_INVALID_ARG, "null descriptor");
  if (!c_desc) c_desc = a_desc;
  Form f;
  su3_status s = make_form(h, a_desc, c_desc, &f);
  if (s != SU3_OK) return s;
  if (f.layout != SU3_LAYOUT_AOS || f.repr_in != SU3_REPR_FULL18 || f.repr_out != SU3_REPR_FULL18 ||
      (f.arith != SU3_ARITH_NATIVE && !(f.arith == SU3_ARITH_F32PAIR && f.dtype == SU3_F64)))
    return fail(h, SU3_ERR_UNSUPPORTED, "a^dagger b takes AOS FULL18 arrays with NATIVE arithmetic (or F32PAIR for F64)");
  if (f.n_sites == 0) return SU3_OK;
  if (!a_dev || !c_dev || !aligned16(a_dev) || !aligned16(c_dev))
    return fail(h, SU3_ERR_INVALID_ARG, "null or misaligned a or c");
  const int64_t an = su3_array_bytes(a_desc), cn = su3_array_bytes(c_desc);
  if (a_dev == c_dev) {
    if (f.a_stride != f.c_stride) return fail(h, SU3_ERR_INVALID_ARG, "in-place operation needs identical strides");
  } else if (ranges_overlap(a_dev, an, c_dev, cn)) {
    return fail(h, SU3_ERR_INVALID_ARG, "a and c overlap without being the same array");
  }
  if (h->fault & kFaultLaunch) return fail(h, SU3_ERR_FAULT_INJECTED, "fault injected at launch");
  LaunchCfg cfg = cfg_for(h, a_desc, f);
  cfg.threads_per_link = 1;  // row k of a^dagger b reads column k of a: no row split
  s = check_cfg(h, f, cfg);
  if (s != SU3_OK) return s;
  return launch_adjacent(0, f, cfg, a_dev, b, c_dev, ctx_of(h, (cudaStream_t)stream));
}

su3_status su3_mat_vec(su3_handle* h, int32_t adjoint, const su3_desc* a_desc, const void* a_dev, const double* v,
                       void* w_dev, void* stream) {
  NvtxRange nvtx_range("su3_mat_vec");
  if (!h) return SU3_ERR_NOT_INITIALIZED;
  DeviceScope scope(h->device);
  if (!a_desc || !v) return fail(h, SU3_ERR_INVALID_ARG, "null descriptor or v");
  Form f;
  su3_status s = make_form(h, a_desc, a_desc, &f);
  if (s != SU3_OK) return s;
  if (f.layout != SU3_LAYOUT_AOS || f.repr_in != SU3_REPR_FULL18 ||
      (f.arith != SU3_ARITH_NATIVE && !(f.arith == SU3_ARITH_F32PAIR && f.dtype == SU3_F64)))
    return fail(h, SU3_ERR_UNSUPPORTED, "matrix x vector takes AOS FULL18 arrays with NATIVE arithmetic (or F32PAIR for F64)");
  if (f.n_sites == 0) return SU3_OK;
  f.c_stride = 12 * 2 * real_bytes(f.dtype);  // 4 packed colour vectors per site
  if (!a_dev || !w_dev || !aligned16(a_dev) || !aligned16(w_dev))
    return fail(h, SU3_ERR_INVALID_ARG, "null or misaligned a or w");
  if (ranges_overlap(a_dev, su3_array_bytes(a_desc), w_dev, f.n_sites * f.c_stride))
    return fail(h, SU3_ERR_INVALID_ARG, "a and w overlap");
  if (h->fault & kFaultLaunch) return fail(h, SU3_ERR_FAULT_INJECTED, "fault injected at launch");
  LaunchCfg cfg = cfg_for(h, a_desc, f);
  cfg.threads_per_link = 1;  // one output vector per link
  s = check_cfg(h, f, cfg);
  if (s != SU3_OK) return s;
  double vb[72] = {0};
  for (int j = 0; j < 4; ++j)
    for (int q = 0; q < 6; ++q) vb[18 * j + q] = v[6 * j + q];
  return launch_adjacent(adjoint ? 2 : 1, f, cfg, a_dev, vb, w_dev, ctx_of(h, (cudaStream_t)stream));
}

su3_status su3_pack(su3_handle* h, const double* src, const su3_desc* dst, void* dst_dev, void* stream) {
  NvtxRange nvtx_range("su3_pack");
  if (!h) return SU3_ERR_NOT_INITIALIZED;
  DeviceScope scope(h->device);
  if (!dst || su3_check_desc(dst) != SU3_OK) return fail(h, SU3_ERR_INVALID_ARG, "invalid destination descriptor");
  if (dst->n_sites == 0) return SU3_OK;
  if (!src || !dst_dev || !aligned16(src) || !aligned16(dst_dev))
    return fail(h, SU3_ERR_INVALID_ARG, "null or misaligned pointer");
  if (ranges_overlap(src, dst->n_sites * 576, dst_dev, su3_array_bytes(dst)))
    return fail(h, SU3_ERR_INVALID_ARG, "source and destination overlap");
  if (h->fault & kFaultLaunch) return fail(h, SU3_ERR_FAULT_INJECTED, "fault injected at launch");
  Form f{};
  f.dtype = dst->dtype;
  f.repr_in = f.repr_out = dst->repr;
  f.layout = dst->layout;
  f.n_sites = dst->n_sites;
  f.a_stride = f.c_stride = resolved_stride(dst);
  return launch_pack(f, src, dst_dev, ctx_of(h, (cudaStream_t)stream));
}

su3_status su3_unpack(su3_handle* h, const su3_desc* src, const void* src_dev, double* dst, void* stream) {
  NvtxRange nvtx_range("su3_unpack");
  if (!h) return SU3_ERR_NOT_INITIALIZED;
  DeviceScope scope(h->device);
  if (!src || su3_check_desc(src) != SU3_OK) return fail(h, SU3_ERR_INVALID_ARG, "invalid source descriptor");
  if (src->n_sites == 0) return SU3_OK;
  if (!src_dev || !dst || !aligned16(src_dev) || !aligned16(dst))
    return fail(h, SU3_ERR_INVALID_ARG, "null or misaligned pointer");
  if (ranges_overlap(dst, src->n_sites * 576, src_dev, su3_array_bytes(src)))
    return fail(h, SU3_ERR_INVALID_ARG, "source and destination overlap");
  if (h->fault & kFaultLaunch) return fail(h, SU3_ERR_FAULT_INJECTED, "fault injected at launch");
  Form f{};
  f.dtype = src->dtype;
  f.repr_in = f.repr_out = src->repr;
  f.layout = src->layout;
  f.n_sites = src->n_sites;
  f.a_stride = f.c_stride = resolved_stride(src);
  return launch_unpack(f, src_dev, dst, ctx_of(h, (cudaStream_t)stream));
}

su3_status su3_sync(su3_handle* h, void* stream, int32_t timeout_ms) {
  NvtxRange nvtx_range("su3_sync");
  if (!h) return SU3_ERR_NOT_INITIALIZED;
  DeviceScope scope(h->device);
  if (h->fault & kFaultSync) return fail(h, SU3_ERR_FAULT_INJECTED, "fault injected at sync");
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e;
  if (timeout_ms < 0) {
    e = cudaStreamSynchronize(st);
  } else {
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms);
    for (;;) {
      e = cudaStreamQuery(st);
      if (e != cudaErrorNotReady) break;
      if (std::chrono::steady_clock::now() > deadline)
        return fail(h, SU3_ERR_TIMEOUT, "work on the stream did not finish within the host deadline");
      std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
  }
  if (e != cudaSuccess) return cuda_err(h, "asynchronous CUDA error", e);
  unsigned st_word = 0;
  e = cudaMemcpy(&st_word, h->status_dev, sizeof(unsigned), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_err(h, "reading the device status word", e);
  if (st_word) {
    cudaMemset(h->status_dev, 0, sizeof(unsigned));
    if (st_word & kDevErrTimeout)
      return fail(h, SU3_ERR_TIMEOUT, "a device-side bounded wait (mbarrier) ran out; results are incomplete");
    return fail(h, SU3_ERR_CUDA, "device status word reported an error");
  }
  return SU3_OK;
}

su3_status su3_measure_fp64_rate(su3_handle* h, int32_t steps, double* tflops) {
  NvtxRange nvtx_range("su3_measure_fp64_rate");
  if (!h) return SU3_ERR_NOT_INITIALIZED;
  DeviceScope scope(h->device);
  if (!tflops || steps < 1 || steps > (1 << 24)) return fail(h, SU3_ERR_INVALID_ARG, "steps must be in [1, 2^24]");
  const int grid = h->num_sms * 8;  // 2,048 threads per SM
  double* out = nullptr;
  cudaError_t e = cudaMalloc((void**)&out, sizeof(double) * (size_t)grid * 256);
  if (e != cudaSuccess) return cuda_err(h, "cudaMalloc", e);
  cudaStream_t st = nullptr;
  e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    cudaFree(out);
    return cuda_err(h, "cudaStreamCreate", e);
  }
  float ms = 0.f;
  su3_status s = measure_dfma_rate(steps, out, grid, ctx_of(h, st), &ms);  // warm-up
  if (s == SU3_OK) s = measure_dfma_rate(steps, out, grid, ctx_of(h, st), &ms);
  cudaStreamDestroy(st);
  cudaFree(out);
  if (s != SU3_OK) return s;
  // 8 chains per thread, 2 flop per FMA
  *tflops = 2.0 * 8.0 * (double)grid * 256.0 * (double)steps / (ms * 1e-3) / 1e12;
  return SU3_OK;
}

su3_status su3_selftest_wait_timeout(su3_handle* h, int32_t limit_ms, void* stream) {
  if (!h) return SU3_ERR_NOT_INITIALIZED;
  DeviceScope scope(h->device);
  if (limit_ms < 1 || limit_ms > 2000) return fail(h, SU3_ERR_INVALID_ARG, "limit_ms must be in [1, 2000]");
  return launch_selftest_wait(limit_ms, ctx_of(h, (cudaStream_t)stream));
}

// ---- host-buffer path ---------------------------------------------------------------------------

namespace {

// Device address of the host range [p, p + n) when the device can address all of it directly:
// both ends inside pinned, mapped host memory, mapped contiguously. Null otherwise (pageable
// memory, a range that leaves its allocation, or no mapping).
void* mapped_view(const void* p, size_t n) {
  if (n == 0) return nullptr;
  cudaPointerAttributes a0, a1;
  if (cudaPointerGetAttributes(&a0, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  const char* last = static_cast<const char*>(p) + (n - 1);
  if (cudaPointerGetAttributes(&a1, last) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a0.type != cudaMemoryTypeHost || a1.type != cudaMemoryTypeHost || !a0.devicePointer || !a1.devicePointer)
    return nullptr;
  if (static_cast<const char*>(a1.devicePointer) - static_cast<const char*>(a0.devicePointer) != (ptrdiff_t)(n - 1))
    return nullptr;
  return a0.devicePointer;
}

// p itself when it is ordinary (unregistered, pageable) host memory, which a device with coherent
// pageable-memory access reads and writes through the host's page tables; else nullptr.
void* pageable_view(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeUnregistered ? const_cast<void*>(p) : nullptr;
}

}  // namespace

int32_t su3_host_pageable_access(const su3_handle* h) { return h && h->pageable_access ? 1 : 0; }

su3_status su3_set_host_path(su3_handle* h, int32_t path) {
  if (!h) return SU3_ERR_NOT_INITIALIZED;
  if (path != SU3_HOST_AUTO && path != SU3_HOST_DIRECT && path != SU3_HOST_STAGED)
    return fail(h, SU3_ERR_INVALID_ARG, "host path must be SU3_HOST_AUTO, SU3_HOST_DIRECT or SU3_HOST_STAGED");
  h->host_path = path;
  return SU3_OK;
}

int32_t su3_last_host_path(const su3_handle* h) { return h ? h->host_path_used : 0; }

su3_status su3_mult_host(su3_handle* h, const su3_desc* a_desc, const void* a_host, const double* b,
                         const su3_desc* c_desc, void* c_host, void* stream) {
  NvtxRange nvtx_range("su3_mult_host");
  if (!h) return SU3_ERR_NOT_INITIALIZED;
  DeviceScope scope(h->device);
  if (!a_desc || !b) return fail(h, SU3_ERR_INVALID_ARG, "null descriptor or b");
  if (!c_desc) c_desc = a_desc;
  Form f;
  su3_status s = make_form(h, a_desc, c_desc, &f);
  if (s != SU3_OK) return s;
  if (f.n_sites == 0) return SU3_OK;
  if (f.layout != SU3_LAYOUT_AOS)
    return fail(h, SU3_ERR_UNSUPPORTED, "the host-buffer path takes AOS arrays (chunks are whole sites)");
  if (!a_host || !c_host) return fail(h, SU3_ERR_INVALID_ARG, "null a or c");
  if (a_host != c_host && ranges_overlap(a_host, su3_array_bytes(a_desc), c_host, su3_array_bytes(c_desc)))
    return fail(h, SU3_ERR_INVALID_ARG, "a and c overlap without being the same array");
  if (h->fault & kFaultCopy) return fail(h, SU3_ERR_FAULT_INJECTED, "fault injected at copy");
  LaunchCfg cfg = cfg_for(h, a_desc, f);
  s = check_cfg(h, f, cfg);
  if (s != SU3_OK) return s;
  cudaError_t e;
  cudaStream_t user = (cudaStream_t)stream;
  if (h->host_path != SU3_HOST_STAGED) {
    // direct: the kernel streams a and c over the host link itself, no staging copies
    void* a_view = mapped_view(a_host, (size_t)su3_array_bytes(a_desc));
    void* c_view = mapped_view(c_host, (size_t)su3_array_bytes(c_desc));
    if (h->pageable_access) {
      // a device that reads pageable host memory coherently streams ordinary buffers as they
      // stand (measured on GB300: 2x the staged path's copies from pageable memory)
      if (!a_view) a_view = pageable_view(a_host);
      if (!c_view) c_view = pageable_view(c_host);
    }
    // the kernel moves 16-byte words: other buffers take the staged path (copies of any alignment)
    const bool aligned = aligned16(a_host) && aligned16(c_host) && aligned16(a_view) && aligned16(c_view);
    if (a_view && c_view && aligned) {
      h->host_path_used = SU3_HOST_DIRECT;
      s = launch_mult_host_direct(f, cfg, a_view, b, c_view, ctx_of(h, user));
      if (s != SU3_OK) return s;
      return su3_sync(h, user, -1);
    }
    if (h->host_path == SU3_HOST_DIRECT)
      return fail(h, SU3_ERR_INVALID_ARG,
                  !aligned ? "the direct host path needs 16-byte aligned a and c"
                  : h->pageable_access
                      ? "the direct host path needs a and c in host memory (pinned, mapped or pageable)"
                      : "the direct host path needs a and c each inside one pinned, mapped host allocation "
                        "(this device does not read pageable host memory)");
  }
  h->host_path_used = SU3_HOST_STAGED;
  if (!h->s_h2d) {
    for (cudaStream_t* p : {&h->s_h2d, &h->s_comp, &h->s_d2h}) {
      e = cudaStreamCreateWithFlags(p, cudaStreamNonBlocking);
      if (e != cudaSuccess) return cuda_err(h, "cudaStreamCreate", e);
    }
    for (int i = 0; i < kHostBuffers; ++i) {
      for (cudaEvent_t* p : {&h->ev_h2d[i], &h->ev_comp[i], &h->ev_d2h[i]}) {
        e = cudaEventCreateWithFlags(p, cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_err(h, "cudaEventCreate", e);
      }
    }
    e = cudaEventCreateWithFlags(&h->ev_start, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_err(h, "cudaEventCreate", e);
  }
  // chunks of whole sites, a multiple of the kernel tile, ~64 MB of input each
  const int64_t a_site = f.a_stride, c_site = f.c_stride;
  const int64_t c_links = 4 * link_bytes(f.dtype, f.repr_out);  // link bytes of one site of c
  int64_t chunk = std::max<int64_t>(cfg.tile_sites, (64ll << 20) / a_site / cfg.tile_sites * cfg.tile_sites);
  chunk = std::min<int64_t>(chunk, f.n_sites);
  const size_t a_bytes = (size_t)(chunk * a_site), c_bytes = (size_t)(chunk * c_site);
  const size_t need = (a_bytes + 255) / 256 * 256 + c_bytes;
  if (need > h->hbuf_bytes) {
    if (h->fault & kFaultAlloc) return fail(h, SU3_ERR_FAULT_INJECTED, "fault injected at alloc");
    cudaDeviceSynchronize();
    for (int i = 0; i < kHostBuffers; ++i) {
      cudaFree(h->hbuf_dev[i]);
      h->hbuf_dev[i] = nullptr;
    }
    h->hbuf_bytes = 0;
    for (int i = 0; i < kHostBuffers; ++i) {
      e = cudaMalloc((void**)&h->hbuf_dev[i], need);
      if (e != cudaSuccess) return cuda_err(h, "cudaMalloc (host-path staging)", e);
    }
    h->hbuf_bytes = need;
  }
  e = cudaEventRecord(h->ev_start, user);
  if (e != cudaSuccess) return cuda_err(h, "cudaEventRecord", e);
  for (cudaStream_t st : {h->s_h2d, h->s_comp, h->s_d2h}) cudaStreamWaitEvent(st, h->ev_start, 0);
  const size_t c_off = (a_bytes + 255) / 256 * 256;
  const int64_t n_chunks = (f.n_sites + chunk - 1) / chunk;
  for (int64_t i = 0; i < n_chunks; ++i) {
    const int bi = (int)(i % kHostBuffers);
    const int64_t first = i * chunk;
    const int64_t ns = std::min<int64_t>(chunk, f.n_sites - first);
    unsigned char* abuf = h->hbuf_dev[bi];
    unsigned char* cbuf = h->hbuf_dev[bi] + c_off;
    if (i >= kHostBuffers) cudaStreamWaitEvent(h->s_h2d, h->ev_d2h[bi], 0);  // buffer free again
    e = cudaMemcpyAsync(abuf, (const unsigned char*)a_host + first * a_site, (size_t)(ns * a_site),
                        cudaMemcpyHostToDevice, h->s_h2d);
    if (e != cudaSuccess) return cuda_err(h, "cudaMemcpyAsync H2D", e);
    cudaEventRecord(h->ev_h2d[bi], h->s_h2d);
    cudaStreamWaitEvent(h->s_comp, h->ev_h2d[bi], 0);
    Form fc = f;
    fc.n_sites = ns;
    s = launch_mult(fc, cfg, abuf, b, cbuf, ctx_of(h, h->s_comp));
    if (s != SU3_OK) return s;
    cudaEventRecord(h->ev_comp[bi], h->s_comp);
    cudaStreamWaitEvent(h->s_d2h, h->ev_comp[bi], 0);
    if (c_site == c_links) {
      e = cudaMemcpyAsync((unsigned char*)c_host + first * c_site, cbuf, (size_t)(ns * c_site),
                          cudaMemcpyDeviceToHost, h->s_d2h);
    } else {  // padded sites: only the link bytes of each site go back, c's pad bytes stay untouched
      e = cudaMemcpy2DAsync((unsigned char*)c_host + first * c_site, (size_t)c_site, cbuf, (size_t)c_site,
                            (size_t)c_links, (size_t)ns, cudaMemcpyDeviceToHost, h->s_d2h);
    }
    if (e != cudaSuccess) return cuda_err(h, "cudaMemcpyAsync D2H", e);
    cudaEventRecord(h->ev_d2h[bi], h->s_d2h);
  }
  e = cudaStreamSynchronize(h->s_d2h);
  if (e != cudaSuccess) return cuda_err(h, "host-path completion", e);
  return su3_sync(h, h->s_comp, -1);
}

// ---- batched --------------------------------------------------------------------------------

// Validates the items and writes the descriptors of the non-empty lattices; *m = their number.
static su3_status fill_batch(su3_handle* h, int32_t n, const su3_batch_item* items, BatchDesc* out, int* total,
                             int* m_out) {
  int tiles = 0, m = 0;
  for (int i = 0; i < n; ++i) {
    const su3_batch_item& it = items[i];
    const su3_desc& d = it.desc;
    if (su3_check_desc(&d) != SU3_OK) return fail(h, SU3_ERR_INVALID_ARG, "invalid descriptor in batch item " + std::to_string(i));
    if ((d.dtype != SU3_F64 && d.dtype != SU3_F32) || d.repr != SU3_REPR_FULL18 || d.layout != SU3_LAYOUT_AOS ||
        (d.arith != SU3_ARITH_NATIVE && !(d.arith == SU3_ARITH_F32PAIR && d.dtype == SU3_F64)) ||
        (d.site_stride_bytes != 0 && d.site_stride_bytes != 4 * link_bytes(d.dtype, d.repr)))
      return fail(h, SU3_ERR_UNSUPPORTED,
                  "batched items must be F64 or F32, FULL18, packed AOS, NATIVE (or F32PAIR for F64)");
    if (d.n_sites == 0) continue;
    if (!it.a_dev || !it.c_dev || !aligned16(it.a_dev) || !aligned16(it.c_dev))
      return fail(h, SU3_ERR_INVALID_ARG, "null or misaligned pointer in batch item " + std::to_string(i));
    const int64_t nb = su3_array_bytes(&d);
    if (it.a_dev != it.c_dev && ranges_overlap(it.a_dev, nb, it.c_dev, nb))
      return fail(h, SU3_ERR_INVALID_ARG, "a and c overlap in batch item " + std::to_string(i));
    BatchDesc& o = out[m++];
    o.a = it.a_dev;
    o.c = it.c_dev;
    o.n_sites = d.n_sites;
    o.dtype = d.dtype;
    o.first_tile = tiles;
    o.arith = d.arith;
    o.reserved = 0;
    memcpy(o.b, it.b, sizeof(o.b));
    split_b_pairs(&it.b[0][0][0][0], o.bpair);
    const int64_t t = batch_tile_count(d.n_sites, d.dtype, h->bcfg.tile_sites);
    if ((int64_t)tiles + t > (1ll << 30)) return fail(h, SU3_ERR_INVALID_ARG, "batch too large");
    tiles += (int)t;
  }
  *total = tiles;
  *m_out = m;
  return SU3_OK;
}

static su3_status ensure_batch_buffers(su3_handle* h, int n, bool graph) {
  BatchDesc** dv = graph ? &h->gdesc_dev : &h->bdesc_dev;
  BatchDesc** hv = graph ? &h->gdesc_host : &h->bdesc_host;
  int* cap = graph ? &h->gcap : &h->bcap;
  if (n <= *cap) return SU3_OK;
  if (h->fault & kFaultAlloc) return fail(h, SU3_ERR_FAULT_INJECTED, "fault injected at alloc");
  cudaDeviceSynchronize();
  cudaFree(*dv);
  cudaFreeHost(*hv);
  *dv = nullptr;
  *hv = nullptr;
  *cap = 0;
  const int want = std::max(n, 128);
  cudaError_t e = cudaMalloc((void**)dv, sizeof(BatchDesc) * want);
  if (e == cudaSuccess) e = cudaMallocHost((void**)hv, sizeof(BatchDesc) * want);
  if (e != cudaSuccess) return cuda_err(h, "allocating the batched workspace", e);
  *cap = want;
  return SU3_OK;
}

su3_status su3_mult_batched(su3_handle* h, int32_t n, const su3_batch_item* items, void* stream, int32_t use_graph) {
  NvtxRange nvtx_range("su3_mult_batched");
  if (!h) return SU3_ERR_NOT_INITIALIZED;
  DeviceScope scope(h->device);
  if (n < 0 || (n > 0 && !items)) return fail(h, SU3_ERR_INVALID_ARG, "bad item count or null items");
  if (n == 0) return SU3_OK;
  if (h->fault & kFaultLaunch) return fail(h, SU3_ERR_FAULT_INJECTED, "fault injected at launch");
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e;
  if (!use_graph) {
    su3_status s = ensure_batch_buffers(h, n, false);
    if (s != SU3_OK) return s;
    if (h->bcopy_pending) {  // the previous upload must have left the pinned buffer
      cudaEventSynchronize(h->bcopy_done);
      h->bcopy_pending = false;
    }
    int total = 0, m = 0;
    std::vector<BatchDesc> tmp(n);
    s = fill_batch(h, n, items, tmp.data(), &total, &m);
    if (s != SU3_OK) return s;
    if (total == 0) return SU3_OK;
    memcpy(h->bdesc_host, tmp.data(), sizeof(BatchDesc) * m);
    if (h->fault & kFaultCopy) return fail(h, SU3_ERR_FAULT_INJECTED, "fault injected at copy");
    if (!h->bcopy_done) {
      e = cudaEventCreateWithFlags(&h->bcopy_done, cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->bkern_done, cudaEventDisableTiming);
      if (e != cudaSuccess) return cuda_err(h, "cudaEventCreate", e);
    }
    // the previous call's kernel may still read bdesc_dev on another stream: the upload that
    // overwrites it waits for that kernel on the GPU
    if (h->bkern_pending) {
      e = cudaStreamWaitEvent(st, h->bkern_done, 0);
      if (e != cudaSuccess) return cuda_err(h, "cudaStreamWaitEvent", e);
    }
    e = cudaMemcpyAsync(h->bdesc_dev, h->bdesc_host, sizeof(BatchDesc) * m, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_err(h, "uploading batch descriptors", e);
    cudaEventRecord(h->bcopy_done, st);
    h->bcopy_pending = true;
    s = launch_batched(h->bdesc_dev, m, total, h->bcfg, ctx_of(h, st));
    if (s != SU3_OK) return s;
    e = cudaEventRecord(h->bkern_done, st);
    if (e != cudaSuccess) return cuda_err(h, "cudaEventRecord", e);
    h->bkern_pending = true;
    return SU3_OK;
  }
  // graph mode: key = the raw item list; rebuild the graph when it changes
  std::vector<char> key((const char*)items, (const char*)items + sizeof(su3_batch_item) * n);
  if (!h->gexec || key != h->gkey) {
    su3_status s = ensure_batch_buffers(h, n, true);
    if (s != SU3_OK) return s;
    int total = 0, m = 0;
    std::vector<BatchDesc> tmp(n);
    s = fill_batch(h, n, items, tmp.data(), &total, &m);
    if (s != SU3_OK) return s;
    if (total == 0) return SU3_OK;
    s = prepare_batched(h->bcfg, &h->err);  // kernel attributes are set outside the capture
    if (s != SU3_OK) return s;
    cudaDeviceSynchronize();  // earlier replays may still read the descriptor buffers
    if (h->gexec) {
      cudaGraphExecDestroy(h->gexec);
      h->gexec = nullptr;
    }
    memcpy(h->gdesc_host, tmp.data(), sizeof(BatchDesc) * m);
    if (!h->cap_stream) {
      e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking);
      if (e != cudaSuccess) return cuda_err(h, "cudaStreamCreate", e);
    }
    cudaGraph_t g;
    e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_err(h, "cudaStreamBeginCapture", e);
    cudaMemcpyAsync(h->gdesc_dev, h->gdesc_host, sizeof(BatchDesc) * m, cudaMemcpyHostToDevice, h->cap_stream);
    const int64_t before = h->launches;
    s = launch_batched(h->gdesc_dev, m, total, h->bcfg, ctx_of(h, h->cap_stream));
    h->launches = before;  // counted at replay
    e = cudaStreamEndCapture(h->cap_stream, &g);
    if (s != SU3_OK) return s;
    if (e != cudaSuccess) return cuda_err(h, "cudaStreamEndCapture", e);
    e = cudaGraphInstantiate(&h->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_err(h, "cudaGraphInstantiate", e);
    h->gkey.swap(key);
  }
  e = cudaGraphLaunch(h->gexec, st);
  if (e != cudaSuccess) return cuda_err(h, "cudaGraphLaunch", e);
  ++h->launches;
  return SU3_OK;
}

}  // extern "C"
