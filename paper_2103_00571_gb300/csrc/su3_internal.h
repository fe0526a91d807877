// Host-side internals shared by the libsu3 translation units (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "su3.h"

namespace su3 {

// Device status word bits (the handle's status word; su3_sync reads and clears it).
enum : unsigned { kDevErrTimeout = 1u };

// A fully validated form: what a kernel instantiation is selected by.
struct Form {
  int dtype;      // su3_dtype
  int repr_in;    // su3_repr of a
  int repr_out;   // su3_repr of c
  int layout;     // su3_layout
  int arith;      // su3_arith
  int64_t n_sites;
  int64_t a_stride;  // AOS: bytes between sites of a (resolved, never 0)
  int64_t c_stride;  // AOS: bytes between sites of c
};

struct LaunchCfg {
  int block;
  int tile_sites;
  int stages;
  int ctas_per_sm;
  int native_permille;  // HYBRID: share of tiles on the FP64 pipe
  int threads_per_link = 1;  // AOS: 1, or 3 = one thread per output row (2 per link for two-row output)
};

// Everything a launcher needs from the handle.
struct LaunchCtx {
  cudaStream_t stream;
  unsigned* status;  // device status word
  int num_sms;
  int smem_per_sm = 0;    // shared memory per SM in bytes (0: unknown, no fitting)
  int smem_reserved = 0;  // shared memory the system reserves per CTA
  int64_t* launches;  // incremented per kernel launch
  std::string* err;
};

inline int real_bytes(int dtype) { return dtype == SU3_F64 ? 8 : dtype == SU3_F32 ? 4 : 2; }
inline int n_elem(int repr) { return repr == SU3_REPR_FULL18 ? 9 : 6; }
inline int64_t link_bytes(int dtype, int repr) { return (int64_t)n_elem(repr) * 2 * real_bytes(dtype); }

// Default launch configuration of a form (used until the autotuner sets one).
LaunchCfg default_cfg(const Form& f);

// HYBRID: warps per CTA on the FP64 pipe, the nearest to native_permille of the CTA's warps.
inline int native_warps(const Form& f, const LaunchCfg& cfg) {
  if (f.arith != SU3_ARITH_HYBRID) return 0;
  const int warps = cfg.block / 32;
  const int n = (warps * cfg.native_permille + 500) / 1000;
  return n < warps ? n : warps;
}

// c = a x b over one lattice (the streaming kernels). b is FP64 on the host.
su3_status launch_mult(const Form& f, const LaunchCfg& cfg, const void* a, const double* b, void* c,
                       const LaunchCtx& ctx);

// c = a x b with a and c in host memory the device can address (pinned, or any host memory on a
// device with pageable-memory access): the kernel streams both over the host link itself.
su3_status launch_mult_host_direct(const Form& f, const LaunchCfg& cfg, const void* a, const double* b, void* c,
                                   const LaunchCtx& ctx);

// a^dagger b (which 0), a v (1), a^dagger v (2): AOS FULL18 NATIVE; v[j] at bv[18*j .. 18*j+5].
su3_status launch_adjacent(int which, const Form& f, const LaunchCfg& cfg, const void* a, const double* bv, void* c,
                           const LaunchCtx& ctx);

// One CTA whose bounded mbarrier wait runs out after limit_ms (failure-path self test).
su3_status launch_selftest_wait(int limit_ms, const LaunchCtx& ctx);

// Packed FP64 AOS <-> the form's storage.
su3_status launch_pack(const Form& dst, const double* src, void* dst_dev, const LaunchCtx& ctx);
su3_status launch_unpack(const Form& src, const void* src_dev, double* dst, const LaunchCtx& ctx);

// Device descriptor of one lattice in a batched launch.
struct BatchDesc {
  const void* a;
  void* c;
  long long n_sites;
  int dtype;           // SU3_F64 or SU3_F32
  int first_tile;      // exclusive prefix sum of tile counts
  int arith;           // SU3_ARITH_NATIVE, or SU3_ARITH_F32PAIR for F64 lattices
  int reserved;
  double b[72];        // FP64 b (F32 lattices round it in the kernel)
  float bpair[144];    // F32PAIR: b[j][e] split as (re_hi, im_hi, re_lo, im_lo), [j][e][4]
};

// Fills BatchDesc::bpair from the FP64 b (hi = b rounded to FP32, lo = the rest rounded to FP32).
inline void split_b_pairs(const double* b, float* out) {
  for (int q = 0; q < 36; ++q) {
    const double r = b[2 * q], i = b[2 * q + 1];
    const float rh = (float)r, ih = (float)i;
    out[4 * q] = rh;
    out[4 * q + 1] = ih;
    out[4 * q + 2] = (float)(r - (double)rh);
    out[4 * q + 3] = (float)(i - (double)ih);
  }
}

struct BatchCfg {
  int block;
  int tile_sites;
  int stages;
  int ctas_per_sm;
  int threads_per_link = 1;  // 1, or 3: one thread per output row
};

BatchCfg default_batch_cfg();
// Tiles are sized in bytes: tile_sites FP64 sites, or 2 * tile_sites FP32 sites (576 B vs 288 B each).
__host__ __device__ inline int batch_tile_sites(int dtype, int tile_sites) { return dtype == SU3_F64 ? tile_sites : 2 * tile_sites; }
int batch_tile_count(long long n_sites, int dtype, int tile_sites);

// Validates a batched configuration and sets the kernel's shared-memory attribute.
su3_status prepare_batched(const BatchCfg& cfg, std::string* err);

// One persistent launch over `n` lattices whose descriptors are already in device memory.
su3_status launch_batched(const BatchDesc* descs_dev, int n, int total_tiles, const BatchCfg& cfg,
                          const LaunchCtx& ctx);

}  // namespace su3
