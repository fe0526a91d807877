/*
 * CPU oracle for the SU3_Bench link multiply (arXiv 2103.00571). TEST INFRASTRUCTURE ONLY:
 * the tests, the smoke check, and the benchmark's CPU-baseline leg and reference arm call it; the
 * product path never does. It shares no source with the CUDA library.
 *
 * Everything is plain FP64 with no contraction into FMA (built with -ffp-contract=off), in the
 * order the definitions state, so that a reader can check it against the paper by eye.
 *
 * Data layout (paper §Background, the su3_matrix and Site structures): a complex number is
 * (re, im) interleaved; an su3_matrix is 3x3 complex, row major, e[k][l]: 18 doubles; a site
 * holds link[4] su3_matrix at offset 0. Sites follow each other every `site_stride` doubles
 * (72 for the packed 576-byte site, 80 for the paper's padded 640-byte FP64 site); the doubles
 * after the four links are never read or written.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

/*
 * The SU3_Bench kernel (§Background, "SU3_Bench", the core-kernel figure as the prose describes
 * it): for every site i and link j, a 3x3x3 complex matrix product in which the inner m loop is a
 * dot product of row k of A[i].link[j] with column l of B[j]:
 *     C[i].link[j].e[k][l] = sum_{m=0..2} A[i].link[j].e[k][m] * B[j].e[m][l].
 * Each complex product-accumulate is 4 multiplies and 4 adds (the paper's 864 flop per site).
 * The i loop is parallel over OpenMP threads (the paper's "VersionX": a plain parallel for over
 * sites, §Performance on Xeon); every site is independent, so the thread count never changes a
 * result.
 */
void su3o_mult(int64_t n_sites, int64_t site_stride, const double* a, const double* b, double* c) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n_sites; ++i) {
    for (int j = 0; j < 4; ++j) {
      const double* A = a + i * site_stride + 18 * j;
      const double* B = b + 18 * j;
      double* C = c + i * site_stride + 18 * j;
      for (int k = 0; k < 3; ++k) {
        for (int l = 0; l < 3; ++l) {
          double re = 0.0, im = 0.0;
          for (int m = 0; m < 3; ++m) {
            double ar = A[6 * k + 2 * m], ai = A[6 * k + 2 * m + 1];
            double br = B[6 * m + 2 * l], bi = B[6 * m + 2 * l + 1];
            re = re + ar * br;
            re = re - ai * bi;
            im = im + ar * bi;
            im = im + ai * br;
          }
          C[6 * k + 2 * l] = re;
          C[6 * k + 2 * l + 1] = im;
        }
      }
    }
  }
}

/*
 * The same kernel on selected sites only (for sampled checks of lattices too large to recompute
 * whole): a_sel[n][72] are the input sites, c_sel[n][72] receive the products.
 */
void su3o_mult_sites(int64_t n, const double* a_sel, const double* b, double* c_sel) {
  su3o_mult(n, 72, a_sel, b, c_sel);
}

/*
 * Two-row (12-real) representation of an SU(3) matrix (the MILC-style compression named by the
 * benchmark's reduced-storage form; the paper itself stores all 18 reals): rows 0 and 1 are kept,
 * and row 2 is rebuilt as conj(row0 x row1), with the cross product
 *     (u x v)_0 = u1 v2 - u2 v1,  (u x v)_1 = u2 v0 - u0 v2,  (u x v)_2 = u0 v1 - u1 v0.
 * This holds for every special unitary 3x3 matrix: its rows are orthonormal and det = 1.
 * in12[n][12] -> out18[n][18].
 */
void su3o_tworow_expand(int64_t n, const double* in12, double* out18) {
#pragma omp parallel for schedule(static)
  for (int64_t t = 0; t < n; ++t) {
    const double* u = in12 + 12 * t;     /* row 0 */
    const double* v = in12 + 12 * t + 6; /* row 1 */
    double* o = out18 + 18 * t;
    for (int q = 0; q < 12; ++q) o[q] = in12[12 * t + q];
    for (int k = 0; k < 3; ++k) {
      int p = (k + 1) % 3, q = (k + 2) % 3;
      /* (u x v)_k = u_p v_q - u_q v_p */
      double upr = u[2 * p], upi = u[2 * p + 1], uqr = u[2 * q], uqi = u[2 * q + 1];
      double vpr = v[2 * p], vpi = v[2 * p + 1], vqr = v[2 * q], vqi = v[2 * q + 1];
      double xr = (upr * vqr - upi * vqi) - (uqr * vpr - uqi * vpi);
      double xi = (upr * vqi + upi * vqr) - (uqr * vpi + uqi * vpr);
      o[12 + 2 * k] = xr;
      o[12 + 2 * k + 1] = -xi;
    }
  }
}

/* Drops row 2: in18[n][18] -> out12[n][12]. */
void su3o_tworow_compress(int64_t n, const double* in18, double* out12) {
  for (int64_t t = 0; t < n; ++t)
    for (int q = 0; q < 12; ++q) out12[12 * t + q] = in18[18 * t + q];
}

/*
 * Unitarity and determinant of n matrices m[n][18]: writes max over the matrices of
 * max_{k,l} |(M M^dagger)_{kl} - delta_{kl}| to out[0] and max |det M - 1| to out[1]
 * (complex moduli). det M is expanded along row 0 (the Leibniz formula for 3x3).
 */
void su3o_unitarity(int64_t n, const double* m, double out[2]) {
  double worst_u = 0.0, worst_d = 0.0;
  for (int64_t t = 0; t < n; ++t) {
    const double* M = m + 18 * t;
    for (int k = 0; k < 3; ++k) {
      for (int l = 0; l < 3; ++l) {
        double re = 0.0, im = 0.0;
        for (int q = 0; q < 3; ++q) {
          /* M[k][q] * conj(M[l][q]) */
          double xr = M[6 * k + 2 * q], xi = M[6 * k + 2 * q + 1];
          double yr = M[6 * l + 2 * q], yi = -M[6 * l + 2 * q + 1];
          re = re + (xr * yr - xi * yi);
          im = im + (xr * yi + xi * yr);
        }
        if (k == l) re = re - 1.0;
        double e = sqrt(re * re + im * im);
        if (e > worst_u) worst_u = e;
      }
    }
    /* det = m00 (m11 m22 - m12 m21) - m01 (m10 m22 - m12 m20) + m02 (m10 m21 - m11 m20) */
#define RE(k, l) M[6 * (k) + 2 * (l)]
#define IM(k, l) M[6 * (k) + 2 * (l) + 1]
    double dr = 0.0, di = 0.0;
    for (int l = 0; l < 3; ++l) {
      int p = (l + 1) % 3, q = (l + 2) % 3;
      /* cofactor of (0, l) with cyclic sign: m1p m2q - m1q m2p */
      double cr = (RE(1, p) * RE(2, q) - IM(1, p) * IM(2, q)) - (RE(1, q) * RE(2, p) - IM(1, q) * IM(2, p));
      double ci = (RE(1, p) * IM(2, q) + IM(1, p) * RE(2, q)) - (RE(1, q) * IM(2, p) + IM(1, q) * RE(2, p));
      dr = dr + (RE(0, l) * cr - IM(0, l) * ci);
      di = di + (RE(0, l) * ci + IM(0, l) * cr);
    }
#undef RE
#undef IM
    double e = sqrt((dr - 1.0) * (dr - 1.0) + di * di);
    if (e > worst_d) worst_d = e;
  }
  out[0] = worst_u;
  out[1] = worst_d;
}

/*
 * Storage rounding for the reduced-precision forms. Each real is rounded once, straight from
 * FP64, to nearest with ties to even (IEEE 754 roundTiesToEven), with no intermediate FP32 step.
 * The bit patterns are built from the definition: the kept significand bits, the discarded
 * remainder compared with half an ulp, and a tie going to the even neighbour.
 */
static uint64_t bits64(double x) {
  uint64_t u;
  memcpy(&u, &x, 8);
  return u;
}

/* binary16: 1 sign, 5 exponent (bias 15), 10 fraction bits; subnormals below 2^-14. */
static uint16_t round_to_half(double x) {
  uint64_t u = bits64(x);
  uint16_t sign = (uint16_t)((u >> 48) & 0x8000u);
  double ax = fabs(x);
  if (isnan(x)) return (uint16_t)(sign | 0x7e00u);
  if (ax >= 65520.0) return (uint16_t)(sign | 0x7c00u); /* rounds to infinity */
  if (ax == 0.0) return sign;
  /* the value in units of the binary16 ulp of its binade: q = ax / ulp, ulp = 2^(e-10), e >= -14 */
  int e;
  frexp(ax, &e); /* ax = f * 2^e, f in [0.5, 1): binade exponent is e-1 */
  int be = e - 1;
  if (be < -14) be = -14; /* subnormal range shares the ulp 2^-24 */
  double q = ldexp(ax, 10 - be); /* exact: scaling by a power of two */
  double fl = floor(q);
  double rem = q - fl; /* exact */
  uint64_t n = (uint64_t)fl;
  if (rem > 0.5 || (rem == 0.5 && (n & 1u))) n += 1;
  /* n = significand with the leading one (for normals) in units of 2^(be-10) */
  uint32_t bits;
  if (n == 0) return sign;
  if (be == -14 && n < 1024u) {
    bits = (uint32_t)n; /* subnormal */
  } else {
    if (n == 2048u) { /* rounding carried into the next binade */
      n = 1024u;
      be += 1;
    }
    if (be > 15) return (uint16_t)(sign | 0x7c00u);
    bits = ((uint32_t)(be + 15) << 10) | (uint32_t)(n - 1024u);
  }
  return (uint16_t)(sign | bits);
}

/* bfloat16: 1 sign, 8 exponent (bias 127), 7 fraction bits. */
static uint16_t round_to_bf16(double x) {
  uint64_t u = bits64(x);
  uint16_t sign = (uint16_t)((u >> 48) & 0x8000u);
  double ax = fabs(x);
  if (isnan(x)) return (uint16_t)(sign | 0x7fc0u);
  if (isinf(x)) return (uint16_t)(sign | 0x7f80u);
  if (ax == 0.0) return sign;
  int e;
  frexp(ax, &e);
  int be = e - 1;
  if (be < -126) be = -126;
  double q = ldexp(ax, 7 - be);
  double fl = floor(q);
  double rem = q - fl;
  uint64_t n = (uint64_t)fl;
  if (rem > 0.5 || (rem == 0.5 && (n & 1u))) n += 1;
  if (n == 0) return sign;
  uint32_t bits;
  if (be == -126 && n < 128u) {
    bits = (uint32_t)n;
  } else {
    if (n == 256u) {
      n = 128u;
      be += 1;
    }
    if (be > 127) return (uint16_t)(sign | 0x7f80u);
    bits = ((uint32_t)(be + 127) << 7) | (uint32_t)(n - 128u);
  }
  return (uint16_t)(sign | bits);
}

void su3o_round_half(int64_t n, const double* x, uint16_t* out) {
  for (int64_t t = 0; t < n; ++t) out[t] = round_to_half(x[t]);
}

void su3o_round_bf16(int64_t n, const double* x, uint16_t* out) {
  for (int64_t t = 0; t < n; ++t) out[t] = round_to_bf16(x[t]);
}

/* Round to binary32 (the C conversion, which rounds to nearest even). */
void su3o_round_float(int64_t n, const double* x, float* out) {
  for (int64_t t = 0; t < n; ++t) out[t] = (float)x[t];
}

/* Exact widening of binary16 / bfloat16 bit patterns back to FP64. */
void su3o_widen_half(int64_t n, const uint16_t* h, double* out) {
  for (int64_t t = 0; t < n; ++t) {
    uint32_t s = (h[t] >> 15) & 1u, ex = (h[t] >> 10) & 0x1fu, fr = h[t] & 0x3ffu;
    double v;
    if (ex == 0)
      v = ldexp((double)fr, -24);
    else if (ex == 31)
      v = fr ? NAN : INFINITY;
    else
      v = ldexp((double)(fr + 1024u), (int)ex - 25);
    out[t] = s ? -v : v;
  }
}

void su3o_widen_bf16(int64_t n, const uint16_t* h, double* out) {
  for (int64_t t = 0; t < n; ++t) {
    uint32_t s = (h[t] >> 15) & 1u, ex = (h[t] >> 7) & 0xffu, fr = h[t] & 0x7fu;
    double v;
    if (ex == 0)
      v = ldexp((double)fr, -133);
    else if (ex == 255)
      v = fr ? NAN : INFINITY;
    else
      v = ldexp((double)(fr + 128u), (int)ex - 134);
    out[t] = s ? -v : v;
  }
}

/* Max abs and root-mean-square difference over n reals (the error report of each form). */
void su3o_error(int64_t n, const double* x, const double* ref, double out[2]) {
  double mx = 0.0, ss = 0.0;
  for (int64_t t = 0; t < n; ++t) {
    double d = fabs(x[t] - ref[t]);
    if (isnan(d)) d = INFINITY; /* a NaN anywhere fails every tolerance */
    if (d > mx) mx = d;
    ss += d * d;
  }
  out[0] = mx;
  out[1] = n > 0 ? sqrt(ss / (double)n) : 0.0;
}

/* Number of OpenMP threads the parallel loops above use. */
#ifdef _OPENMP
#include <omp.h>
#endif
int su3o_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Sets the number of OpenMP threads of the parallel loops above (for single-core timing). */
void su3o_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/*
 * Adjacent SU(3) operations of the same lattice shape (the paper's introduction places SU(3)
 * products with matrices and with colour vectors at the core of lattice-QCD codes such as MILC;
 * these are their plain definitions, one link at a time, b or v fixed per link direction j as in
 * the SU3_Bench kernel):
 *   su3o_mult_an: c[i][j][k][l] = sum_m conj(a[i][j][m][k]) * b[j][m][l]      (a^dagger b)
 *   su3o_mult_na: c[i][j][k][l] = sum_m a[i][j][k][m] * conj(b[j][l][m])      (a b^dagger)
 *   su3o_mat_vec: w[i][j][k]    = sum_m a[i][j][k][m] * v[j][m]               (a v)
 *                 or, with adjoint != 0, sum_m conj(a[i][j][m][k]) * v[j][m]  (a^dagger v)
 * v holds four colour vectors (4 x 3 complex = 24 doubles); w[n][4][3][2] is packed.
 */
void su3o_mult_an(int64_t n_sites, int64_t site_stride, const double* a, const double* b, double* c) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n_sites; ++i) {
    for (int j = 0; j < 4; ++j) {
      const double* A = a + i * site_stride + 18 * j;
      const double* B = b + 18 * j;
      double* C = c + i * site_stride + 18 * j;
      for (int k = 0; k < 3; ++k) {
        for (int l = 0; l < 3; ++l) {
          double re = 0.0, im = 0.0;
          for (int m = 0; m < 3; ++m) {
            double ar = A[6 * m + 2 * k], ai = -A[6 * m + 2 * k + 1]; /* conj(a[m][k]) */
            double br = B[6 * m + 2 * l], bi = B[6 * m + 2 * l + 1];
            re = re + ar * br;
            re = re - ai * bi;
            im = im + ar * bi;
            im = im + ai * br;
          }
          C[6 * k + 2 * l] = re;
          C[6 * k + 2 * l + 1] = im;
        }
      }
    }
  }
}

void su3o_mult_na(int64_t n_sites, int64_t site_stride, const double* a, const double* b, double* c) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n_sites; ++i) {
    for (int j = 0; j < 4; ++j) {
      const double* A = a + i * site_stride + 18 * j;
      const double* B = b + 18 * j;
      double* C = c + i * site_stride + 18 * j;
      for (int k = 0; k < 3; ++k) {
        for (int l = 0; l < 3; ++l) {
          double re = 0.0, im = 0.0;
          for (int m = 0; m < 3; ++m) {
            double ar = A[6 * k + 2 * m], ai = A[6 * k + 2 * m + 1];
            double br = B[6 * l + 2 * m], bi = -B[6 * l + 2 * m + 1]; /* conj(b[l][m]) */
            re = re + ar * br;
            re = re - ai * bi;
            im = im + ar * bi;
            im = im + ai * br;
          }
          C[6 * k + 2 * l] = re;
          C[6 * k + 2 * l + 1] = im;
        }
      }
    }
  }
}

void su3o_mat_vec(int64_t n_sites, int64_t site_stride, int adjoint, const double* a, const double* v, double* w) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n_sites; ++i) {
    for (int j = 0; j < 4; ++j) {
      const double* A = a + i * site_stride + 18 * j;
      const double* X = v + 6 * j;
      double* W = w + i * 24 + 6 * j;
      for (int k = 0; k < 3; ++k) {
        double re = 0.0, im = 0.0;
        for (int m = 0; m < 3; ++m) {
          double ar, ai;
          if (adjoint) {
            ar = A[6 * m + 2 * k];
            ai = -A[6 * m + 2 * k + 1]; /* conj(a[m][k]) */
          } else {
            ar = A[6 * k + 2 * m];
            ai = A[6 * k + 2 * m + 1];
          }
          double xr = X[2 * m], xi = X[2 * m + 1];
          re = re + ar * xr;
          re = re - ai * xi;
          im = im + ar * xi;
          im = im + ai * xr;
        }
        W[2 * k] = re;
        W[2 * k + 1] = im;
      }
    }
  }
}
