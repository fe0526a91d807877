// Layout and precision conversion between the benchmark's packed FP64 Site array and the reduced
// forms (outside the timed path). Pack rounds each real once, to nearest even, straight from FP64
// (cvt.rn.{f32,f16,bf16}.f64: no FP64 -> FP32 -> FP16 double rounding); unpack widens exactly and
// rebuilds row 2 of a two-row link as conj(row0 x row1) in FP64.
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
__device__ __forceinline__ double bf16_to_f64(unsigned short h) {
  return (double)__uint_as_float((unsigned)h << 16);
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
};

__global__ void su3_pack_kernel(const double* __restrict__ src, unsigned char* __restrict__ dst, Addr ad,
                                int dtype) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= ad.n_links) return;
  const double* s = src + q * 18;
  for (int e = 0; e < ad.ne; ++e) {
    const double re = s[2 * e], im = s[2 * e + 1];
    unsigned char* d = dst + ad.off(q, e);
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
}

__global__ void su3_unpack_kernel(const unsigned char* __restrict__ src, double* __restrict__ dst, Addr ad,
                                  int dtype) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= ad.n_links) return;
  Link<double> l;
  for (int e = 0; e < ad.ne; ++e) {
    const unsigned char* s = src + ad.off(q, e);
    if (dtype == SU3_F64) {
      double2 v = *reinterpret_cast<const double2*>(s);
      l.re[e] = v.x;
      l.im[e] = v.y;
    } else if (dtype == SU3_F32) {
      float2 v = *reinterpret_cast<const float2*>(s);
      l.re[e] = (double)v.x;
      l.im[e] = (double)v.y;
    } else {
      const unsigned w = *reinterpret_cast<const unsigned*>(s);
      const unsigned short lo = (unsigned short)(w & 0xffffu), hi = (unsigned short)(w >> 16);
      l.re[e] = dtype == SU3_F16 ? f16_to_f64(lo) : bf16_to_f64(lo);
      l.im[e] = dtype == SU3_F16 ? f16_to_f64(hi) : bf16_to_f64(hi);
    }
  }
  if (ad.ne == 6) rebuild_row2(l);
  double* d = dst + q * 18;
  for (int e = 0; e < 9; ++e) {
    d[2 * e] = l.re[e];
    d[2 * e + 1] = l.im[e];
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

su3_status launch_pack(const Form& dst, const double* src, void* dst_dev, const LaunchCtx& ctx) {
  Addr ad = make_addr(dst);
  const int block = 256;
  const long long grid = (ad.n_links + block - 1) / block;
  su3_pack_kernel<<<(unsigned)grid, block, 0, ctx.stream>>>(src, static_cast<unsigned char*>(dst_dev), ad,
                                                             dst.dtype);
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
  const int block = 256;
  const long long grid = (ad.n_links + block - 1) / block;
  su3_unpack_kernel<<<(unsigned)grid, block, 0, ctx.stream>>>(static_cast<const unsigned char*>(src_dev), dst,
                                                               ad, src.dtype);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    *ctx.err = std::string("su3_unpack_kernel launch: ") + cudaGetErrorString(e);
    return SU3_ERR_CUDA;
  }
  ++*ctx.launches;
  return SU3_OK;
}

}  // namespace su3
