// Device-side building blocks of libsu3 (sm_103a): PTX wrappers for mbarriers, bulk async copies
// and cache-hinted vector memory operations, storage conversions, and the 3x3 complex link
// product of the SU3_Bench kernel (arXiv 2103.00571, §Background "SU3_Bench").
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace su3 {

// Upper bound on any spin-wait, in globaltimer nanoseconds.
constexpr unsigned long long kWaitLimitNs = 4000000000ull;

enum Dtype { kF64 = 0, kF32 = 1, kF16 = 2, kBF16 = 3 };

// ---- PTX wrappers -----------------------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Waits for phase `parity` of an mbarrier; gives up after `limit_ns` and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity,
                                                  unsigned long long limit_ns = kWaitLimitNs) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer_ns();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (globaltimer_ns() - t0 > limit_ns) return false;
  }
}

// 1-D bulk async copy global -> this CTA's shared memory, completing `bytes` on `bar`.
// Both addresses 16-byte aligned, bytes a multiple of 16 (checked by the callers' invariants).
__device__ __forceinline__ void bulk_g2s(void* sdst, const void* gsrc, unsigned bytes, uint64_t* bar,
                                         uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], "
      "%2, [%3], %4;" ::"r"(smem_u32(sdst)),
      "l"(gsrc), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
      : "memory");
}

// 1-D bulk async copy shared -> global, tracked by this thread's bulk groups.
__device__ __forceinline__ void bulk_s2g(void* gdst, const void* ssrc, unsigned bytes, uint64_t policy) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group.L2::cache_hint [%0], [%1], %2, %3;" ::"l"(gdst),
               "r"(smem_u32(ssrc)), "r"(bytes), "l"(policy)
               : "memory");
}

// 2-D tensor copies (the TMA engine reading a tensor map): the box at element coordinates (x, y)
// of the map. Load: global -> this CTA's shared memory, completing the box's bytes on `bar` (rows
// past the tensor's end arrive as zeros and count like the rest). Store: shared -> global, tracked
// by this thread's bulk groups; rows past the tensor's end are not written. The map is a
// __grid_constant__ kernel parameter (its generic address); shared memory 128-byte aligned.
__device__ __forceinline__ void tma_load_2d(void* sdst, const void* tmap, int x, int y, uint64_t* bar,
                                            uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint [%0], "
      "[%1, {%2, %3}], [%4], %5;" ::"r"(smem_u32(sdst)),
      "l"(tmap), "r"(x), "r"(y), "r"(smem_u32(bar)), "l"(policy)
      : "memory");
}

__device__ __forceinline__ void tma_store_2d(const void* tmap, int x, int y, const void* ssrc, uint64_t policy) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group.L2::cache_hint [%0, {%1, %2}], [%3], %4;" ::"l"(
                   tmap),
               "r"(x), "r"(y), "r"(smem_u32(ssrc)), "l"(policy)
               : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}

template <int N>
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group %0;" ::"n"(N) : "memory");
}

// Orders this thread's generic-proxy shared-memory writes before later async-proxy reads.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

// ---- streaming global loads/stores (read once: no L1 allocation; write once: evict-first) ----

__device__ __forceinline__ double2 ldg_stream(const double2* p) {
  double2 v;
  asm volatile("ld.global.nc.L1::no_allocate.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "l"(p));
  return v;
}
__device__ __forceinline__ float2 ldg_stream(const float2* p) {
  float2 v;
  asm volatile("ld.global.nc.L1::no_allocate.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
  return v;
}
__device__ __forceinline__ uint32_t ldg_stream(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.global.nc.L1::no_allocate.b32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ void stg_stream(double2* p, double2 v) {
  asm volatile("st.global.cs.v2.f64 [%0], {%1, %2};" ::"l"(p), "d"(v.x), "d"(v.y) : "memory");
}
__device__ __forceinline__ void stg_stream(float2* p, float2 v) {
  asm volatile("st.global.cs.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(v.x), "f"(v.y) : "memory");
}
__device__ __forceinline__ void stg_stream(uint32_t* p, uint32_t v) {
  asm volatile("st.global.cs.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// ---- storage <-> arithmetic conversions --------------------------------------------------------
// A "complex element" of storage type T is stored as one vector: double2 (F64), float2 (F32),
// or a 32-bit word holding two 16-bit reals (F16/BF16), re in the low half.

template <int DT>
struct Storage;

template <>
struct Storage<kF64> {
  using real = double;   // storage real
  using vec = double2;   // one complex element in memory
  using acc = double;    // arithmetic type
  static constexpr int real_bytes = 8;
  __device__ static __forceinline__ void unpack(vec v, acc& re, acc& im) { re = v.x; im = v.y; }
  __device__ static __forceinline__ vec pack(acc re, acc im) { return make_double2(re, im); }
};

template <>
struct Storage<kF32> {
  using real = float;
  using vec = float2;
  using acc = float;
  static constexpr int real_bytes = 4;
  __device__ static __forceinline__ void unpack(vec v, acc& re, acc& im) { re = v.x; im = v.y; }
  __device__ static __forceinline__ vec pack(acc re, acc im) { return make_float2(re, im); }
};

template <>
struct Storage<kF16> {
  using real = __half;
  using vec = uint32_t;
  using acc = float;
  static constexpr int real_bytes = 2;
  __device__ static __forceinline__ void unpack(vec v, acc& re, acc& im) {
    __half2 h = *reinterpret_cast<__half2*>(&v);
    float2 f = __half22float2(h);
    re = f.x;
    im = f.y;
  }
  __device__ static __forceinline__ vec pack(acc re, acc im) {
    __half2 h = __floats2half2_rn(re, im);  // both halves rounded to nearest even
    return *reinterpret_cast<uint32_t*>(&h);
  }
};

template <>
struct Storage<kBF16> {
  using real = __nv_bfloat16;
  using vec = uint32_t;
  using acc = float;
  static constexpr int real_bytes = 2;
  __device__ static __forceinline__ void unpack(vec v, acc& re, acc& im) {
    re = __uint_as_float(v << 16);          // a bfloat16 is the top half of a binary32
    im = __uint_as_float(v & 0xffff0000u);
  }
  __device__ static __forceinline__ vec pack(acc re, acc im) {
    __nv_bfloat162 h = __floats2bfloat162_rn(re, im);
    return *reinterpret_cast<uint32_t*>(&h);
  }
};

// ---- b in the kernel parameters ---------------------------------------------------------------

// The four b matrices by value in a kernel's parameter block: b[j][row][col][re/im], plus the
// constant 1.0 that FP32-pair arithmetic multiplies by (see dot_pair2: as a kernel parameter its
// value is unknown to the compiler, so no multiply can be folded into the FMA that uses it).
template <typename A>
struct BMat {
  A v[72];
  float unit;
};

template <typename A>
inline BMat<A> make_b(const double* b) {
  BMat<A> m;
  for (int i = 0; i < 72; ++i) m.v[i] = (A)b[i];
  m.unit = 1.0f;
  return m;
}

// Stages b (72 reals) in shared memory and lets each thread's op take its direction j = tid % 4.
template <class Op>
__device__ __forceinline__ void load_b_op(const BMat<typename Op::BArg>& b, typename Op::BArg* bsh, Op& op,
                                          int native_warps) {
  for (int i = threadIdx.x; i < 72; i += blockDim.x) bsh[i] = b.v[i];
  __syncthreads();
  op.init(bsh + 18 * (threadIdx.x & 3), native_warps);
  op.set_unit(b.unit);
}

// ---- the link product -------------------------------------------------------------------------

// A link in registers: up to 9 complex elements, row major (e = 3*row + col).
template <typename T>
struct Link {
  T re[9], im[9];
};

// Row 2 of an SU(3) matrix from rows 0 and 1: conj(row0 x row1), with
// (u x v)_k = u_p v_q - u_q v_p, (p, q) = (k+1, k+2) mod 3. r0/r1 hold rows 0 and 1 (re, im).
template <typename T>
__device__ __forceinline__ void rebuild_row2_elems(const T (&r0re)[3], const T (&r0im)[3], const T (&r1re)[3],
                                                   const T (&r1im)[3], T (&ore)[3], T (&oim)[3]) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int p = (k + 1) % 3, q = (k + 2) % 3;
    T xr = r0re[p] * r1re[q];
    xr = fma(-r0im[p], r1im[q], xr);
    xr = fma(-r0re[q], r1re[p], xr);
    xr = fma(r0im[q], r1im[p], xr);
    T xi = r0re[p] * r1im[q];
    xi = fma(r0im[p], r1re[q], xi);
    xi = fma(-r0re[q], r1im[p], xi);
    xi = fma(-r0im[q], r1re[p], xi);
    ore[k] = xr;
    oim[k] = -xi;
  }
}

template <typename T>
__device__ __forceinline__ void rebuild_row2(Link<T>& a) {
  T r0re[3], r0im[3], r1re[3], r1im[3], ore[3], oim[3];
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    r0re[m] = a.re[m];
    r0im[m] = a.im[m];
    r1re[m] = a.re[3 + m];
    r1im[m] = a.im[3 + m];
  }
  rebuild_row2_elems(r0re, r0im, r1re, r1im, ore, oim);
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    a.re[6 + m] = ore[m];
    a.im[6 + m] = oim[m];
  }
}

// One output row: c[l] = sum_m a[m] b[m][l] (the SU3_Bench kernel's inner l, m loops for one k;
// 4 real FMAs per complex multiply-accumulate).
template <typename T>
__device__ __forceinline__ void row_mult(const T (&are)[3], const T (&aim)[3], const T (&bre)[9], const T (&bim)[9],
                                         T (&cre)[3], T (&cim)[3]) {
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    T re = are[0] * bre[l];
    T im = are[0] * bim[l];
    re = fma(-aim[0], bim[l], re);
    im = fma(aim[0], bre[l], im);
#pragma unroll
    for (int m = 1; m < 3; ++m) {
      re = fma(are[m], bre[3 * m + l], re);
      re = fma(-aim[m], bim[3 * m + l], re);
      im = fma(are[m], bim[3 * m + l], im);
      im = fma(aim[m], bre[3 * m + l], im);
    }
    cre[l] = re;
    cim[l] = im;
  }
}

// c[k][l] = sum_m a[k][m] b[m][l] for rows k < ROWS.
template <int ROWS, typename T>
__device__ __forceinline__ void link_mult(const Link<T>& a, const T (&bre)[9], const T (&bim)[9],
                                          Link<T>& c) {
#pragma unroll
  for (int k = 0; k < ROWS; ++k) {
    T are[3], aim[3], cre[3], cim[3];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      are[m] = a.re[3 * k + m];
      aim[m] = a.im[3 * k + m];
    }
    row_mult(are, aim, bre, bim, cre, cim);
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      c.re[3 * k + l] = cre[l];
      c.im[3 * k + l] = cim[l];
    }
  }
}

// ---- per-link operations used by the streaming kernels ----------------------------------------
// An op owns this thread's copy of b[j] (j = tid % 4) and turns one input link (NE_IN complex
// storage elements) into one output link (3*ROWS_OUT elements). `src` and `dst` may alias.
// Element e of the input link is src[e * ES_IN] and of the output link dst[e * ES_OUT]: 1 for a
// link stored contiguously (AOS), 32 inside an AOSOA32 block, the plane stride inside an SOA tile.
// Ops with kRowSplit also compute a single output row (apply_row), with the same operations as
// apply(), for launches with one thread per output row.

template <int DT, int NE_IN, int ROWS_OUT>
struct NativeOp {
  using S = Storage<DT>;
  using A = typename S::acc;   // FP64 for F64 storage, FP32 otherwise
  using V = typename S::vec;
  using BArg = A;              // precision of b in the kernel parameters
  static constexpr int kNeIn = NE_IN, kNeOut = 3 * ROWS_OUT;
  static constexpr bool kRowSplit = true;  // has apply_row: one thread per output row is possible
  A bre[9], bim[9];
  __device__ __forceinline__ void begin_tile(int) {}
  __device__ __forceinline__ void set_unit(float) {}
  __device__ __forceinline__ void init(const BArg* bj, int /*native_warps*/) {
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      bre[e] = bj[2 * e];
      bim[e] = bj[2 * e + 1];
    }
  }
  template <int ES_IN = 1, int ES_OUT = 1>
  __device__ __forceinline__ void apply(const V* src, V* dst) const {
    Link<A> la, lc;
#pragma unroll
    for (int e = 0; e < NE_IN; ++e) S::unpack(src[e * ES_IN], la.re[e], la.im[e]);
    if (NE_IN == 6 && ROWS_OUT == 3) rebuild_row2(la);
    link_mult<ROWS_OUT>(la, bre, bim, lc);
#pragma unroll
    for (int e = 0; e < 3 * ROWS_OUT; ++e) dst[e * ES_OUT] = S::pack(lc.re[e], lc.im[e]);
  }
  // Output row k alone (row split: one thread per output row). Reads input row k only, except
  // that a rebuilt row 2 reads rows 0 and 1; the arithmetic is exactly that of apply().
  template <int ES_IN = 1, int ES_OUT = 1>
  __device__ __forceinline__ void apply_row(const V* src, V* dst, int k) const {
    A are[3], aim[3], cre[3], cim[3];
    if (NE_IN == 6 && ROWS_OUT == 3 && k == 2) {
      A r0re[3], r0im[3], r1re[3], r1im[3];
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        S::unpack(src[m * ES_IN], r0re[m], r0im[m]);
        S::unpack(src[(3 + m) * ES_IN], r1re[m], r1im[m]);
      }
      rebuild_row2_elems(r0re, r0im, r1re, r1im, are, aim);
    } else {
#pragma unroll
      for (int m = 0; m < 3; ++m) S::unpack(src[(3 * k + m) * ES_IN], are[m], aim[m]);
    }
    row_mult(are, aim, bre, bim, cre, cim);
#pragma unroll
    for (int l = 0; l < 3; ++l) dst[(3 * k + l) * ES_OUT] = S::pack(cre[l], cim[l]);
  }
};

// ---- adjacent SU(3) operations ----------------------------------------------------------------
// The other per-link SU(3) products of lattice-QCD codes next to the benchmark's a x b: a^dagger x b (MILC's
// mult_su3_an) and the matrix x colour-vector products a v and a^dagger v (mult_su3_mat_vec and
// its adjoint), with b or v fixed per link direction exactly as in the SU3_Bench kernel.
// (a x b^dagger needs no kernel of its own: b^dagger is formed exactly on the host.)

template <int DT>
struct AnOp {  // c[k][l] = sum_m conj(a[m][k]) b[m][l]
  using S = Storage<DT>;
  using A = typename S::acc;
  using V = typename S::vec;
  using BArg = A;
  static constexpr int kNeIn = 9, kNeOut = 9;
  static constexpr bool kRowSplit = false;  // row k of a^dagger b reads column k of a
  A bre[9], bim[9];
  __device__ __forceinline__ void begin_tile(int) {}
  __device__ __forceinline__ void set_unit(float) {}
  __device__ __forceinline__ void init(const BArg* bj, int) {
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      bre[e] = bj[2 * e];
      bim[e] = bj[2 * e + 1];
    }
  }
  template <int ES_IN = 1, int ES_OUT = 1>
  __device__ __forceinline__ void apply(const V* src, V* dst) const {
    Link<A> la;
#pragma unroll
    for (int e = 0; e < 9; ++e) S::unpack(src[e * ES_IN], la.re[e], la.im[e]);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
#pragma unroll
      for (int l = 0; l < 3; ++l) {
        // conj(a) = (ar, -ai): re += ar br + ai bi, im += ar bi - ai br
        A re = la.re[k] * bre[l];
        A im = la.re[k] * bim[l];
        re = fma(la.im[k], bim[l], re);
        im = fma(-la.im[k], bre[l], im);
#pragma unroll
        for (int m = 1; m < 3; ++m) {
          re = fma(la.re[3 * m + k], bre[3 * m + l], re);
          re = fma(la.im[3 * m + k], bim[3 * m + l], re);
          im = fma(la.re[3 * m + k], bim[3 * m + l], im);
          im = fma(-la.im[3 * m + k], bre[3 * m + l], im);
        }
        dst[(3 * k + l) * ES_OUT] = S::pack(re, im);
      }
    }
  }
};

template <int DT, bool ADJ>
struct MatVecOp {  // w[k] = sum_m a[k][m] v[m]   (ADJ: sum_m conj(a[m][k]) v[m])
  using S = Storage<DT>;
  using A = typename S::acc;
  using V = typename S::vec;
  using BArg = A;
  static constexpr int kNeIn = 9, kNeOut = 3;
  static constexpr bool kRowSplit = false;  // one output vector per link
  A vre[3], vim[3];
  __device__ __forceinline__ void begin_tile(int) {}
  __device__ __forceinline__ void set_unit(float) {}
  __device__ __forceinline__ void init(const BArg* vj, int) {
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      vre[m] = vj[2 * m];
      vim[m] = vj[2 * m + 1];
    }
  }
  template <int ES_IN = 1, int ES_OUT = 1>
  __device__ __forceinline__ void apply(const V* src, V* dst) const {
    Link<A> la;
#pragma unroll
    for (int e = 0; e < 9; ++e) S::unpack(src[e * ES_IN], la.re[e], la.im[e]);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      A re = 0, im = 0;
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        const int e = ADJ ? 3 * m + k : 3 * k + m;
        const A ai = ADJ ? -la.im[e] : la.im[e];
        re = fma(la.re[e], vre[m], re);
        re = fma(-ai, vim[m], re);
        im = fma(la.re[e], vim[m], im);
        im = fma(ai, vre[m], im);
      }
      dst[k * ES_OUT] = S::pack(re, im);
    }
  }
};

// ---- FP64 storage with FP32-pair ("double-float") arithmetic ----------------------------------
// GB300 issues FP64 FMAs at 1/64 of the FP32 rate, and even double<->float conversions run on the
// FP64 pipe. This op keeps FP64 in memory but computes with unevaluated pairs of FP32 numbers:
//  * split: a double x becomes hi + lo, hi = x truncated to 24 significant bits (integer bit
//    operations on the exponent and mantissa), lo = the remaining 29 mantissa bits, converted with
//    one rounding (I2F) and scaled by 2^(e-52). |x - hi - lo| <= 2^-48 |x|. Valid for
//    2^-74 <= |x| < 2^127; smaller magnitudes (including 0) are replaced by a value below 2^-73.
//  * each real output is a 6-term dot product (Ogita, Rump and Oishi's Dot2 scheme, SIAM J. Sci.
//    Comput. 26 (2005)): products x_hi*y_hi are split exactly into p + e by an FMA (TwoProduct),
//    the p's are summed with Knuth's TwoSum, and every error term (e, the TwoSum errors and the
//    cross products x_hi*y_lo + x_lo*y_hi) is accumulated in a second FP32 number;
//  * the real and imaginary parts of each complex output run as the two lanes of Blackwell's
//    packed FP32x2 add/mul/fma, halving the FP32 instruction count;
//  * the pair (s, L) becomes a double by building both halves' FP64 bit patterns with integer
//    operations (exact for normal floats) and one FP64 add. (Assembling it with integer
//    operations only, to leave the FP64 pipe idle, measured slower: the extra integer work costs
//    more issue slots than the FP64 add.)
// Measured error against the FP64 oracle on random SU(3) data: max ~3e-14, RMS ~2e-15.

struct FF {
  float h, l;
};

__device__ __forceinline__ FF split_f64(double x) {
  const unsigned H = (unsigned)__double2hiint(x);
  const unsigned Lw = (unsigned)__double2loint(x);
  unsigned ax = H & 0x7FFFFFFFu;
  ax = max(ax, (949u << 20));  // |x| >= 2^-74 keeps every exponent below in range
  const unsigned hb = __funnelshift_l(Lw, ax - (896u << 20), 3) | (H & 0x80000000u);
  const unsigned sb = (hb & 0xFF800000u) - (52u << 23);  // sign | 2^(e-52)
  FF r;
  r.h = __uint_as_float(hb);
  r.l = __uint2float_rn(Lw & 0x1FFFFFFFu) * __uint_as_float(sb);
  return r;
}

// Exact FP64 value of a normal float, built from its bits (zero maps to 2^-127). The arithmetic
// shift copies the sign into bits 28-31; the mask keeps bit 31 and the exponent and mantissa in
// bits 0-27, and adding the exponent bias difference (1023 - 127) << 20 cannot carry into the
// sign. Four integer operations (one fewer than or-ing the sign back in: 1.3 % faster measured).
__device__ __forceinline__ double f32_bits_to_f64(float f) {
  const int b = __float_as_int(f);
  const unsigned hi = ((unsigned)(b >> 3) & 0x8FFFFFFFu) + (896u << 20);
  return __hiloint2double((int)hi, (int)((unsigned)b << 29));
}

// Packed FP32x2 arithmetic (Blackwell's add/mul/fma.f32x2: two independent, individually
// rounded FP32 operations per instruction). a - b is computed as fma(b, -1, a), which rounds
// exactly like a subtraction.
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }

// The real and imaginary parts of one complex output as two lanes of FP32x2 operations:
// sum_{t<N} x_t * y_t with x = (xh, xl) broadcast to both lanes and y = (yh, yl) per lane, in the
// manner of Ogita, Rump and Oishi's Dot2. Per term t: the product p = fl(xh*yh), Knuth's TwoSum
// s2 = s + p with its two exact error parts t1 (s's share) and t2 = p - z (p's share, z = s2 - s),
// and the product error e = xh*yh - p. Since e and t2 are always added together and
// e + t2 = xh*yh - z exactly, one FMA gives their sum with a single rounding of a value of size
// ~ulp(s2) (so ~2^-48 of the sum); t1 and that FMA go to one error accumulator, the cross
// products xh*yl + xl*yh to another. That is 10 FP32x2 operations per term instead of 12.
// The add s + p is written as fma(p, unit, s) with unit = 1.0 passed as a kernel parameter: p's
// only use is then inside an FMA's multiplicand, which the compiler cannot merge with p's multiply.
// (As a plain add of a single-use product it was contracted into fma(xh, yh, s), which rounds
// s2 differently from the TwoSum's p and loses the error term: ~2^-24 results, measured.)
// The result is the unevaluated pair s + L per lane.
template <int N>
__device__ __forceinline__ void dot_pair2(const float (&xh)[N], const float (&xl)[N], const float2 (&yh)[N],
                                          const float2 (&yl)[N], float2 one, float2& s_out, float2& L_out) {
  float2 x0h = make_float2(xh[0], xh[0]), x0l = make_float2(xl[0], xl[0]);
  float2 s = mul2(x0h, yh[0]);
  float2 Lt = fma2(x0h, yh[0], make_float2(-s.x, -s.y));  // e of the first product
  float2 Lc = fma2(x0h, yl[0], mul2(x0l, yh[0]));
#pragma unroll
  for (int t = 1; t < N; ++t) {
    const float2 xth = make_float2(xh[t], xh[t]), xtl = make_float2(xl[t], xl[t]);
    const float2 p = mul2(xth, yh[t]);
    const float2 s2 = fma2(p, one, s);
    const float2 z = sub2(s2, s);
    const float2 t1 = sub2(s, sub2(s2, z));
    s = s2;
    Lt = add2(Lt, t1);
    Lt = add2(Lt, fma2(xth, yh[t], make_float2(-z.x, -z.y)));  // e + t2 in one rounding
    Lc = fma2(xth, yl[t], Lc);
    Lc = fma2(xtl, yh[t], Lc);
  }
  s_out = s;
  L_out = add2(Lt, Lc);
}

// One complex output of the product: the 6-term pair dot product, assembled into FP64.
__device__ __forceinline__ double2 dot6_pair2(const float (&xh)[6], const float (&xl)[6], const float2 (&yh)[6],
                                              const float2 (&yl)[6], float2 one) {
  float2 s, L;
  dot_pair2<6>(xh, xl, yh, yl, one, s, L);
  return make_double2(f32_bits_to_f64(s.x) + f32_bits_to_f64(L.x), f32_bits_to_f64(s.y) + f32_bits_to_f64(L.y));
}

// Row 2 of a two-row link, conj(u x v) with u = row 0 and v = row 1, in FP32-pair arithmetic: from
// the pair splits of the two rows (terms 2m = re, 2m+1 = im of element m) to the pair (wh, wl)
// of each real of row 2. Element k is conj(u_p v_q - u_q v_p), (p, q) = (k+1, k+2) mod 3; its
// (re, im) lanes are one 4-term dot product with a's row-0 reals broadcast and row-1 reals,
// negated or swapped, per lane:
//   re = up.re vq.re - up.im vq.im - uq.re vp.re + uq.im vp.im
//   im = -up.re vq.im - up.im vq.re + uq.re vp.im + uq.im vp.re
// The pair (s, L) of a Dot2 is itself a split of the value (s carries 24 bits, L the rest), so
// row 2 goes into the product with no FP64 operation.
__device__ __forceinline__ void rebuild_row2_pair(const float (&uh)[6], const float (&ul)[6], const float (&vh)[6],
                                                  const float (&vl)[6], float2 one, float (&wh)[6], float (&wl)[6]) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int p = (k + 1) % 3, q = (k + 2) % 3;
    const float xh[4] = {uh[2 * p], uh[2 * p + 1], uh[2 * q], uh[2 * q + 1]};
    const float xl[4] = {ul[2 * p], ul[2 * p + 1], ul[2 * q], ul[2 * q + 1]};
    const float2 yh[4] = {make_float2(vh[2 * q], -vh[2 * q + 1]), make_float2(-vh[2 * q + 1], -vh[2 * q]),
                          make_float2(-vh[2 * p], vh[2 * p + 1]), make_float2(vh[2 * p + 1], vh[2 * p])};
    const float2 yl[4] = {make_float2(vl[2 * q], -vl[2 * q + 1]), make_float2(-vl[2 * q + 1], -vl[2 * q]),
                          make_float2(-vl[2 * p], vl[2 * p + 1]), make_float2(vl[2 * p + 1], vl[2 * p])};
    float2 sv, Lv;
    dot_pair2<4>(xh, xl, yh, yl, one, sv, Lv);
    wh[2 * k] = sv.x;
    wl[2 * k] = Lv.x;
    wh[2 * k + 1] = sv.y;
    wl[2 * k + 1] = Lv.y;
  }
}

template <int NE_IN, int ROWS_OUT>
struct PairF64Op {
  using V = double2;
  using BArg = double;
  static constexpr int kNeIn = NE_IN, kNeOut = 3 * ROWS_OUT;
  static constexpr bool kRowSplit = true;
  // b[j] split once per thread, as lane pairs for the two terms of each (m, l):
  // (re, im) lanes of ar*(br, bi) and of ai*(-bi, br), high and low parts.
  float2 ya[9], yb[9], yla[9], ylb[9];
  float2 one;  // (1, 1), from the kernel parameters (dot_pair2)
  __device__ __forceinline__ void begin_tile(int) {}
  __device__ __forceinline__ void set_unit(float u) { one = make_float2(u, u); }
  __device__ __forceinline__ void init(const double* bj, int /*native_warps*/) {
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      const double r = bj[2 * e], i = bj[2 * e + 1];
      const float rh = __double2float_rn(r), ih = __double2float_rn(i);
      const float rl = __double2float_rn(r - (double)rh), il = __double2float_rn(i - (double)ih);
      ya[e] = make_float2(rh, ih);
      yb[e] = make_float2(-ih, rh);
      yla[e] = make_float2(rl, il);
      ylb[e] = make_float2(-il, rl);
    }
  }
  // The same constants from a host-side split: pre[4e..4e+3] = (re_hi, im_hi, re_lo, im_lo).
  __device__ __forceinline__ void init_pre(const float* pre) {
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      const float rh = __ldg(pre + 4 * e), ih = __ldg(pre + 4 * e + 1);
      const float rl = __ldg(pre + 4 * e + 2), il = __ldg(pre + 4 * e + 3);
      ya[e] = make_float2(rh, ih);
      yb[e] = make_float2(-ih, rh);
      yla[e] = make_float2(rl, il);
      ylb[e] = make_float2(-il, rl);
    }
  }
  // The pair split of input row r (terms 2m: re, 2m+1: im of element m).
  template <int ES_IN>
  __device__ __forceinline__ void split_row(const V* src, int r, float (&xh)[6], float (&xl)[6]) const {
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      const double2 v = src[(3 * r + m) * ES_IN];
      const FF re = split_f64(v.x), im = split_f64(v.y);
      xh[2 * m] = re.h;
      xl[2 * m] = re.l;
      xh[2 * m + 1] = im.h;
      xl[2 * m + 1] = im.l;
    }
  }
  // Output row k from the pair split (xh, xl) of the input row.
  template <int ES_OUT>
  __device__ __forceinline__ void row_out(const float (&xh)[6], const float (&xl)[6], V* dst, int k) const {
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      float2 yh[6], yl[6];
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        yh[2 * m] = ya[3 * m + l];
        yl[2 * m] = yla[3 * m + l];
        yh[2 * m + 1] = yb[3 * m + l];
        yl[2 * m + 1] = ylb[3 * m + l];
      }
      dst[(3 * k + l) * ES_OUT] = dot6_pair2(xh, xl, yh, yl, one);
    }
  }
  // Output row k: reads input row k and writes output row k (so src and dst may alias). Row 2 of
  // a two-row input is first rebuilt from rows 0 and 1 in pair arithmetic (rebuild_row2_pair).
  template <int ES_IN = 1, int ES_OUT = 1>
  __device__ __forceinline__ void apply_row(const V* src, V* dst, int k) const {
    float xh[6], xl[6];
    if (NE_IN == 6 && ROWS_OUT == 3 && k == 2) {
      float uh[6], ul[6], vh[6], vl[6];
      split_row<ES_IN>(src, 0, uh, ul);
      split_row<ES_IN>(src, 1, vh, vl);
      rebuild_row2_pair(uh, ul, vh, vl, one, xh, xl);
    } else {
      split_row<ES_IN>(src, k, xh, xl);
    }
    row_out<ES_OUT>(xh, xl, dst, k);
  }
  template <int ES_IN = 1, int ES_OUT = 1>
  __device__ __forceinline__ void apply(const V* src, V* dst) const {
    if constexpr (NE_IN == 6 && ROWS_OUT == 3) {
      // two-row in, full out (never in place): rows 0 and 1 are split once and serve both their
      // own outputs and the rebuild of row 2 (the same operations as apply_row, so the same bits)
      float uh[6], ul[6], vh[6], vl[6], wh[6], wl[6];
      split_row<ES_IN>(src, 0, uh, ul);
      split_row<ES_IN>(src, 1, vh, vl);
      rebuild_row2_pair(uh, ul, vh, vl, one, wh, wl);
      row_out<ES_OUT>(uh, ul, dst, 0);
      row_out<ES_OUT>(vh, vl, dst, 1);
      row_out<ES_OUT>(wh, wl, dst, 2);
    } else {
#pragma unroll
      for (int k = 0; k < ROWS_OUT; ++k) apply_row<ES_IN, ES_OUT>(src, dst, k);
    }
  }
};


// The adjacent products in FP32-pair arithmetic (FP64 storage, FP64-accurate results):
// a^dagger b, whose output row k is the product's row routine applied to column k of a
// conjugated (the imaginary parts' splits change sign, exactly), with the same b pairs.
struct PairAnOp {
  using V = double2;
  using BArg = double;
  static constexpr int kNeIn = 9, kNeOut = 9;
  static constexpr bool kRowSplit = false;  // row k of a^dagger b reads column k of a
  PairF64Op<9, 3> pair;                     // b as FP32 pairs and the row routine
  __device__ __forceinline__ void begin_tile(int) {}
  __device__ __forceinline__ void set_unit(float u) { pair.set_unit(u); }
  __device__ __forceinline__ void init(const double* bj, int w) { pair.init(bj, w); }
  template <int ES_IN = 1, int ES_OUT = 1>
  __device__ __forceinline__ void apply(const V* src, V* dst) const {
    double2 a[9];  // all of a first: the output may overwrite it (in place)
#pragma unroll
    for (int e = 0; e < 9; ++e) a[e] = src[e * ES_IN];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      float xh[6], xl[6];  // conj(a[m][k]), terms 2m: re, 2m+1: im
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        const FF re = split_f64(a[3 * m + k].x), im = split_f64(a[3 * m + k].y);
        xh[2 * m] = re.h;
        xl[2 * m] = re.l;
        xh[2 * m + 1] = -im.h;
        xl[2 * m + 1] = -im.l;
      }
      pair.template row_out<ES_OUT>(xh, xl, dst, k);
    }
  }
};

// a v and a^dagger v in FP32-pair arithmetic: each output element is one 6-term pair dot product
// of row k of a (ADJ: column k, conjugated) with v[j] held as FP32 pairs.
template <bool ADJ>
struct PairMatVecOp {
  using V = double2;
  using BArg = double;
  static constexpr int kNeIn = 9, kNeOut = 3;
  static constexpr bool kRowSplit = false;  // one output vector per link
  float2 ya[3], yb[3], yla[3], ylb[3];      // v[m]: (re, im), (-im, re), and their low parts
  float2 one;
  __device__ __forceinline__ void begin_tile(int) {}
  __device__ __forceinline__ void set_unit(float u) { one = make_float2(u, u); }
  __device__ __forceinline__ void init(const double* vj, int) {
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      const double r = vj[2 * m], i = vj[2 * m + 1];
      const float rh = __double2float_rn(r), ih = __double2float_rn(i);
      const float rl = __double2float_rn(r - (double)rh), il = __double2float_rn(i - (double)ih);
      ya[m] = make_float2(rh, ih);
      yb[m] = make_float2(-ih, rh);
      yla[m] = make_float2(rl, il);
      ylb[m] = make_float2(-il, rl);
    }
  }
  template <int ES_IN = 1, int ES_OUT = 1>
  __device__ __forceinline__ void apply(const V* src, V* dst) const {
    const float2 yh[6] = {ya[0], yb[0], ya[1], yb[1], ya[2], yb[2]};
    const float2 yl[6] = {yla[0], ylb[0], yla[1], ylb[1], yla[2], ylb[2]};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      float xh[6], xl[6];
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        const double2 v = src[(ADJ ? 3 * m + k : 3 * k + m) * ES_IN];
        const FF re = split_f64(v.x), im = split_f64(v.y);
        xh[2 * m] = re.h;
        xl[2 * m] = re.l;
        xh[2 * m + 1] = ADJ ? -im.h : im.h;
        xl[2 * m + 1] = ADJ ? -im.l : im.l;
      }
      dst[k * ES_OUT] = dot6_pair2(xh, xl, yh, yl, one);
    }
  }
};

// HYBRID: per tile, warp w uses the FP64 pipe (NATIVE) when (tile + w) % period == 0 and FP32
// pairs otherwise, period = warps / native_warps. The native work rotates over all warps, so it
// is spread over every SM sub-partition's FP64 unit. Each thread keeps both forms of its b[j].
template <int NE_IN, int ROWS_OUT>
struct HybridF64Op {
  using V = double2;
  using BArg = double;
  static constexpr int kNeIn = NE_IN, kNeOut = 3 * ROWS_OUT;
  static constexpr bool kRowSplit = true;
  NativeOp<kF64, NE_IN, ROWS_OUT> nat;
  PairF64Op<NE_IN, ROWS_OUT> pair;
  int period;  // 0: never native
  bool native;
  __device__ __forceinline__ void init(const double* bj, int native_warps) {
    nat.init(bj, 0);
    pair.init(bj, 0);
    const int warps = (int)(blockDim.x >> 5);
    period = native_warps > 0 ? max(1, warps / native_warps) : 0;
    native = false;
  }
  __device__ __forceinline__ void begin_tile(int k) {
    native = period > 0 && ((k + (int)(threadIdx.x >> 5)) % period) == 0;
  }
  __device__ __forceinline__ void set_unit(float u) { pair.set_unit(u); }
  template <int ES_IN = 1, int ES_OUT = 1>
  __device__ __forceinline__ void apply(const V* src, V* dst) const {
    if (native) nat.template apply<ES_IN, ES_OUT>(src, dst);
    else pair.template apply<ES_IN, ES_OUT>(src, dst);
  }
  template <int ES_IN = 1, int ES_OUT = 1>
  __device__ __forceinline__ void apply_row(const V* src, V* dst, int k) const {
    if (native) nat.template apply_row<ES_IN, ES_OUT>(src, dst, k);
    else pair.template apply_row<ES_IN, ES_OUT>(src, dst, k);
  }
};

}  // namespace su3
