// Layout and precision conversion between the benchmark's packed FP64 Site array and the reduced
// forms (outside the timed path). Unpack stages tiles of 256 links through shared memory, so that
// the form's side and the FP64 side are each read and written in their own memory order.
// Pack rounds each real once, to nearest even, straight from FP64 (cvt.rn.{f32,f16,bf16}.f64: no
// FP64 -> FP32 -> FP16 double rounding); unpack widens exactly and rebuilds row 2 of a two-row
// link as conj(row0 x row1) in FP64.
#include <cuda_runtime.h>

#include <algorithm>

#include "su3_device.cuh"
#include "su3_internal.h"

namespace su3 {

__device__ __forceinline__ float f64_to_f32_rn(double x) {
  float r;
  asm("cvt.rn.f32.f64 %0, %1;" : "=f"(r) : "d"(x));
  return r;
}
__device__ __forceinline__ unsigned short f64_to_f16_rn(double x) {
  unsigned short r;
  asm("cvt.rn.f16.f64 %0, %1;" : "=h"(r) : "d"(x));
  return r;
}
__device__ __forceinline__ unsigned short f64_to_bf16_rn(double x) {
  unsigned short r;
  asm("cvt.rn.bf16.f64 %0, %1;" : "=h"(r) : "d"(x));
  return r;
}
__device__ __forceinline__ double f16_to_f64(unsigned short h) {
  double r;
  asm("cvt.f64.f16 %0, %1;" : "=d"(r) : "h"(h));
  return r;
}

// Complex element e of link q in the form's storage: byte offset.
struct Addr {
  int layout;
  int ne;            // complex elements per link in this array
  int vec_bytes;     // bytes of one complex element
  long long stride;  // AOS: bytes between sites
  long long n_links;
  __device__ __forceinline__ long long off(long long q, int e) const {
    if (layout == SU3_LAYOUT_AOS) return (q >> 2) * stride + ((q & 3) * ne + e) * (long long)vec_bytes;
    if (layout == SU3_LAYOUT_SOA) return ((long long)e * n_links + q) * vec_bytes;
    return (((q >> 5) * ne + e) * 32 + (q & 31)) * (long long)vec_bytes;
  }
  // Number of work items of a tile of `tl` links (tiles start at multiples of 32 links): tl x ne,
  // or for AOSOA32 whole blocks of 32 links, whose items past tl the caller skips.
  __device__ __forceinline__ int items(int tl) const {
    return (layout == SU3_LAYOUT_AOSOA32 ? (tl + 31) / 32 * 32 : tl) * ne;
  }
  // The i-th element of the tile in the form's memory order (so that consecutive threads touch
  // consecutive addresses): AOS link-major, SOA element-major, AOSOA32 by blocks of 32 links,
  // element-major inside a block. Returns the tile-relative link (>= tl: skip) and the element.
  __device__ __forceinline__ void item(int i, int tl, int& ql, int& e) const {
    if (layout == SU3_LAYOUT_AOS) {
      ql = i / ne;
      e = i - ql * ne;
    } else if (layout == SU3_LAYOUT_SOA) {
      e = i / tl;
      ql = i - e * tl;
    } else {
      const int blk = i / (32 * ne), rem = i - blk * 32 * ne;
      e = rem >> 5;
      ql = blk * 32 + (rem & 31);
    }
  }
};

constexpr int kPackTile = 256;  // unpack: links per tile, 36 KB of FP64 links in shared memory

__device__ __forceinline__ void store_elem(unsigned char* d, int dtype, double re, double im) {
  if (dtype == SU3_F64) {
    *reinterpret_cast<double2*>(d) = make_double2(re, im);
  } else if (dtype == SU3_F32) {
    *reinterpret_cast<float2*>(d) = make_float2(f64_to_f32_rn(re), f64_to_f32_rn(im));
  } else if (dtype == SU3_F16) {
    *reinterpret_cast<unsigned*>(d) = (unsigned)f64_to_f16_rn(re) | ((unsigned)f64_to_f16_rn(im) << 16);
  } else {
    *reinterpret_cast<unsigned*>(d) = (unsigned)f64_to_bf16_rn(re) | ((unsigned)f64_to_bf16_rn(im) << 16);
  }
}

// Exact FP32 -> FP64 widening. Normal numbers and zeros are re-encoded with integer operations
// (same value, same bits as the hardware conversion, without the FP64 pipe); subnormals,
// infinities and NaNs (none in SU(3) data) take the hardware conversion.
__device__ __forceinline__ double widen_f32(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned e8 = (b >> 23) & 0xFFu;
  if (e8 - 1u < 254u) {
    const unsigned hi = (b & 0x80000000u) | ((e8 + 896u) << 20) | ((b & 0x7FFFFFu) >> 3);
    return __hiloint2double((int)hi, (int)(b << 29));
  }
  if ((b & 0x7FFFFFFFu) == 0u) return __hiloint2double((int)(b & 0x80000000u), 0);
  return (double)f;
}

__device__ __forceinline__ double2 load_elem(const unsigned char* s, int dtype) {
  if (dtype == SU3_F64) return *reinterpret_cast<const double2*>(s);
  if (dtype == SU3_F32) {
    const float2 v = *reinterpret_cast<const float2*>(s);
    return make_double2(widen_f32(v.x), widen_f32(v.y));
  }
  const unsigned w = *reinterpret_cast<const unsigned*>(s);
  if (dtype == SU3_F16) {
    // binary16 -> binary32 is exact (the half conversion unit), then widened as above
    const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&w));
    return make_double2(widen_f32(f.x), widen_f32(f.y));
  }
  return make_double2(widen_f32(__uint_as_float(w << 16)), widen_f32(__uint_as_float(w & 0xffff0000u)));
}

// FP64 packed AoS links -> the form, one thread per link: its 18 doubles come through the L1
// cache, each element is rounded and written at the form's address. Used for the element-major
// layouts and two-row AOS, where it measured faster on GB300 than the staged kernel below
// (6.3 vs 4.3 TB/s for FP64 AoSoA32, 5.7 vs 3.4 for two-row FP16 AOS).
__global__ void __launch_bounds__(256) su3_pack_kernel(const double* __restrict__ src, unsigned char* __restrict__ dst,
                                                       Addr ad, int dtype) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= ad.n_links) return;
  const double* s = src + q * 18;
  for (int e = 0; e < ad.ne; ++e) store_elem(dst + ad.off(q, e), dtype, s[2 * e], s[2 * e + 1]);
}

constexpr int kPackStageTile = 128;  // staged pack: links per tile, 18 KB of FP64 links

// FP64 packed AoS links -> a FULL18 AOS form, staged: a tile of links comes in with consecutive
// 16-byte loads into shared memory and leaves element by element in the form's order (for a
// packed stride, consecutive addresses). Measured faster than the per-link kernel for these
// forms: FP32 4.96 vs 4.54 TB/s, FP16 4.36 vs 3.73.
__global__ void __launch_bounds__(256) su3_pack_staged_kernel(const double2* __restrict__ src,
                                                              unsigned char* __restrict__ dst, Addr ad, int dtype) {
  __shared__ double2 tile[kPackStageTile * 9];
  const long long n_tiles = (ad.n_links + kPackStageTile - 1) / kPackStageTile;
  for (long long t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    const long long q0 = t * kPackStageTile;
    const int tl = (int)min((long long)kPackStageTile, ad.n_links - q0);
    for (int i = threadIdx.x; i < tl * 9; i += blockDim.x) tile[i] = src[q0 * 9 + i];
    __syncthreads();
    for (int i = threadIdx.x; i < ad.items(tl); i += blockDim.x) {
      int ql, e;
      ad.item(i, tl, ql, e);
      if (ql >= tl) continue;
      const double2 v = tile[ql * 9 + e];
      store_elem(dst + ad.off(q0 + ql, e), dtype, v.x, v.y);
    }
    __syncthreads();
  }
}

// The form -> FP64 packed AoS links: elements come in in the form's memory order, widened
// exactly into shared memory; two-row links get row 2 = conj(row0 x row1) there; then the FP64
// links leave with consecutive 16-byte stores.
__global__ void __launch_bounds__(256) su3_unpack_kernel(const unsigned char* __restrict__ src, double2* __restrict__ dst,
                                                         Addr ad, int dtype) {
  __shared__ double2 tile[kPackTile * 9];
  const long long n_tiles = (ad.n_links + kPackTile - 1) / kPackTile;
  for (long long t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    const long long q0 = t * kPackTile;
    const int tl = (int)min((long long)kPackTile, ad.n_links - q0);
    for (int i = threadIdx.x; i < ad.items(tl); i += blockDim.x) {
      int ql, e;
      ad.item(i, tl, ql, e);
      if (ql >= tl) continue;
      tile[ql * 9 + e] = load_elem(src + ad.off(q0 + ql, e), dtype);
    }
    __syncthreads();
    if (ad.ne == 6) {
      for (int ql = threadIdx.x; ql < tl; ql += blockDim.x) {
        double r0re[3], r0im[3], r1re[3], r1im[3], ore[3], oim[3];
        for (int m = 0; m < 3; ++m) {
          r0re[m] = tile[ql * 9 + m].x;
          r0im[m] = tile[ql * 9 + m].y;
          r1re[m] = tile[ql * 9 + 3 + m].x;
          r1im[m] = tile[ql * 9 + 3 + m].y;
        }
        rebuild_row2_elems(r0re, r0im, r1re, r1im, ore, oim);
        for (int m = 0; m < 3; ++m) tile[ql * 9 + 6 + m] = make_double2(ore[m], oim[m]);
      }
      __syncthreads();
    }
    for (int i = threadIdx.x; i < tl * 9; i += blockDim.x) dst[q0 * 9 + i] = tile[i];
    __syncthreads();
  }
}

static Addr make_addr(const Form& f) {
  Addr a;
  a.layout = f.layout;
  a.ne = n_elem(f.repr_in);
  a.vec_bytes = 2 * real_bytes(f.dtype);
  a.stride = f.a_stride;
  a.n_links = 4 * f.n_sites;
  return a;
}

static int unpack_grid(const Addr& ad, const LaunchCtx& ctx) {
  const long long n_tiles = (ad.n_links + kPackTile - 1) / kPackTile;
  return (int)std::max<long long>(1, std::min<long long>(n_tiles, (long long)ctx.num_sms * 6));
}

su3_status launch_pack(const Form& dst, const double* src, void* dst_dev, const LaunchCtx& ctx) {
  Addr ad = make_addr(dst);
  if (ad.layout == SU3_LAYOUT_AOS && ad.ne == 9) {
    const long long n_tiles = (ad.n_links + kPackStageTile - 1) / kPackStageTile;
    const int grid = (int)std::max<long long>(1, std::min<long long>(n_tiles, (long long)ctx.num_sms * 8));
    su3_pack_staged_kernel<<<grid, 256, 0, ctx.stream>>>(reinterpret_cast<const double2*>(src),
                                                         static_cast<unsigned char*>(dst_dev), ad, dst.dtype);
  } else {
    const long long grid = (ad.n_links + 255) / 256;
    su3_pack_kernel<<<(unsigned)grid, 256, 0, ctx.stream>>>(src, static_cast<unsigned char*>(dst_dev), ad, dst.dtype);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    *ctx.err = std::string("su3_pack_kernel launch: ") + cudaGetErrorString(e);
    return SU3_ERR_CUDA;
  }
  ++*ctx.launches;
  return SU3_OK;
}

su3_status launch_unpack(const Form& src, const void* src_dev, double* dst, const LaunchCtx& ctx) {
  Addr ad = make_addr(src);
  su3_unpack_kernel<<<unpack_grid(ad, ctx), 256, 0, ctx.stream>>>(static_cast<const unsigned char*>(src_dev),
                                                                reinterpret_cast<double2*>(dst), ad, src.dtype);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    *ctx.err = std::string("su3_unpack_kernel launch: ") + cudaGetErrorString(e);
    return SU3_ERR_CUDA;
  }
  ++*ctx.launches;
  return SU3_OK;
}

}  // namespace su3
