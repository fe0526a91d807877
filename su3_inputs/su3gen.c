/*
 * Seeded synthetic inputs for the SU3_Bench link multiply: random SU(3) matrices.
 *
 * This module only builds input matrices. It holds none of the multiply's arithmetic and is
 * shared, as bytes, by the CPU oracle and by the CUDA path.
 *
 * Recipe (per matrix; the paper's lattices are synthetic L^4 site arrays, §Background):
 *   1. draw 12 N(0,1) doubles, in the order v0[0].re, v0[0].im, v0[1].re, ..., v1[2].im;
 *   2. row0 = v0 / |v0|;
 *   3. w = v1 - <row0, v1> row0 (complex inner product, conjugate on row0); row1 = w / |w|;
 *   4. row2 = conj(row0 x row1), with (u x v)_0 = u1 v2 - u2 v1, (u x v)_1 = u2 v0 - u0 v2,
 *      (u x v)_2 = u0 v1 - u1 v0.
 * The result is unitary with determinant exactly 1 up to rounding.
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
 * as 1, 2, 3", SC'11), written from its published definition. Key = the 64-bit seed; counter =
 * (matrix id low word, matrix id high word, lattice id, draw index). Each draw gives four 32-bit
 * words = two uniforms in (0,1] with 53 random bits = two normals by Box-Muller. A matrix whose
 * |v0| or |w| falls below 1e-12 is redrawn with draw indices shifted by 6 (probability ~0).
 * Every matrix depends only on (seed, lattice id, matrix id), never on the thread count.
 *
 * Matrix ids of one lattice of V sites: 0 .. 4V-1 are the links a[i][j] (id = 4 i + j, site
 * major); 4V .. 4V+3 are the four fixed matrices b[0..3].
 *
 * Layout: a matrix is 9 complex numbers, row major, each (re, im) interleaved: 18 doubles.
 * A site is 4 such matrices (72 doubles = 576 bytes).
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void su3gen_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)PHILOX_M0 * c0;
    uint64_t p1 = (uint64_t)PHILOX_M1 * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += PHILOX_W0;
    k1 += PHILOX_W1;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

/* Uniform in (0, 1] from two 32-bit words: 53 bits, plus one so that 0 never occurs. */
static double uniform53(uint32_t w0, uint32_t w1) {
  uint64_t x = ((uint64_t)w0 << 21) ^ (uint64_t)(w1 >> 11);
  x &= (((uint64_t)1) << 53) - 1;
  return ((double)x + 1.0) * (1.0 / 9007199254740992.0);
}

static void draw_normals12(uint64_t seed, uint32_t lattice, uint64_t id, uint32_t attempt,
                           double z[12]) {
  const double two_pi = 6.283185307179586476925286766559;
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (uint32_t d = 0; d < 6; ++d) {
    uint32_t ctr[4] = {(uint32_t)id, (uint32_t)(id >> 32), lattice, attempt * 6u + d};
    uint32_t w[4];
    su3gen_philox4x32_10(ctr, key, w);
    double u1 = uniform53(w[0], w[1]);
    double u2 = uniform53(w[2], w[3]);
    double r = sqrt(-2.0 * log(u1));
    z[2 * d] = r * cos(two_pi * u2);
    z[2 * d + 1] = r * sin(two_pi * u2);
  }
}

/* Builds one SU(3) matrix (18 doubles) from (seed, lattice, id). Returns the attempt used. */
static int make_su3(uint64_t seed, uint32_t lattice, uint64_t id, double m[18]) {
  for (uint32_t attempt = 0;; ++attempt) {
    double z[12];
    draw_normals12(seed, lattice, id, attempt, z);
    double v0r[3], v0i[3], v1r[3], v1i[3];
    for (int k = 0; k < 3; ++k) {
      v0r[k] = z[2 * k];
      v0i[k] = z[2 * k + 1];
      v1r[k] = z[6 + 2 * k];
      v1i[k] = z[6 + 2 * k + 1];
    }
    double n0 = 0.0;
    for (int k = 0; k < 3; ++k) n0 += v0r[k] * v0r[k] + v0i[k] * v0i[k];
    n0 = sqrt(n0);
    if (n0 < 1e-12) continue;
    double r0r[3], r0i[3];
    for (int k = 0; k < 3; ++k) {
      r0r[k] = v0r[k] / n0;
      r0i[k] = v0i[k] / n0;
    }
    /* p = <row0, v1> = sum_k conj(row0_k) v1_k */
    double pr = 0.0, pi = 0.0;
    for (int k = 0; k < 3; ++k) {
      pr += r0r[k] * v1r[k] + r0i[k] * v1i[k];
      pi += r0r[k] * v1i[k] - r0i[k] * v1r[k];
    }
    double wr[3], wi[3];
    for (int k = 0; k < 3; ++k) {
      wr[k] = v1r[k] - (pr * r0r[k] - pi * r0i[k]);
      wi[k] = v1i[k] - (pr * r0i[k] + pi * r0r[k]);
    }
    double n1 = 0.0;
    for (int k = 0; k < 3; ++k) n1 += wr[k] * wr[k] + wi[k] * wi[k];
    n1 = sqrt(n1);
    if (n1 < 1e-12) continue;
    double r1r[3], r1i[3];
    for (int k = 0; k < 3; ++k) {
      r1r[k] = wr[k] / n1;
      r1i[k] = wi[k] / n1;
    }
    /* x = row0 x row1 (complex products), row2 = conj(x) */
    static const int P[3] = {1, 2, 0}, Q[3] = {2, 0, 1};
    double r2r[3], r2i[3];
    for (int k = 0; k < 3; ++k) {
      int p = P[k], q = Q[k];
      double xr = (r0r[p] * r1r[q] - r0i[p] * r1i[q]) - (r0r[q] * r1r[p] - r0i[q] * r1i[p]);
      double xi = (r0r[p] * r1i[q] + r0i[p] * r1r[q]) - (r0r[q] * r1i[p] + r0i[q] * r1r[p]);
      r2r[k] = xr;
      r2i[k] = -xi;
    }
    for (int k = 0; k < 3; ++k) {
      m[0 * 6 + 2 * k] = r0r[k];
      m[0 * 6 + 2 * k + 1] = r0i[k];
      m[1 * 6 + 2 * k] = r1r[k];
      m[1 * 6 + 2 * k + 1] = r1i[k];
      m[2 * 6 + 2 * k] = r2r[k];
      m[2 * 6 + 2 * k + 1] = r2i[k];
    }
    return (int)attempt;
  }
}

/* The raw 12 normals of matrix `id` (first attempt); exposed for distribution tests. */
void su3gen_normals(uint64_t seed, uint32_t lattice, uint64_t id, double z[12]) {
  draw_normals12(seed, lattice, id, 0u, z);
}

/* Matrices with ids first_id .. first_id+count-1 into out[count][18]. */
void su3gen_matrices(uint64_t seed, uint32_t lattice, uint64_t first_id, int64_t count,
                     double* out) {
#pragma omp parallel for schedule(static)
  for (int64_t t = 0; t < count; ++t) make_su3(seed, lattice, first_id + (uint64_t)t, out + 18 * t);
}

/*
 * Sites first_site .. first_site+n-1 of a lattice of n_total sites (all 4 links each), written
 * with `stride_doubles` doubles between consecutive sites (>= 72; the extra doubles of each site
 * are left untouched). The four b matrices of that lattice are ids 4*n_total .. 4*n_total+3 and
 * come from su3gen_matrices.
 */
void su3gen_sites(uint64_t seed, uint32_t lattice, int64_t first_site, int64_t n,
                  int64_t stride_doubles, double* out) {
#pragma omp parallel for schedule(static)
  for (int64_t s = 0; s < n; ++s) {
    for (int j = 0; j < 4; ++j)
      make_su3(seed, lattice, 4 * (uint64_t)(first_site + s) + (uint64_t)j,
               out + stride_doubles * s + 18 * j);
  }
}

/* Sites at arbitrary indices (for sampled checks of large lattices): out[n][72]. */
void su3gen_sites_at(uint64_t seed, uint32_t lattice, const int64_t* idx, int64_t n, double* out) {
#pragma omp parallel for schedule(static)
  for (int64_t s = 0; s < n; ++s) {
    for (int j = 0; j < 4; ++j)
      make_su3(seed, lattice, 4 * (uint64_t)idx[s] + (uint64_t)j, out + 72 * s + 18 * j);
  }
}

/*
 * Extents (Lx, Ly, Lz, Lt) of n lattices, each drawn uniformly from {4, 6, ..., 24}: one Philox
 * draw per lattice (counter = (k, 0, 0x5eed, 0xe7e7)), word mod 11 (bias < 3e-9).
 */
void su3gen_extents(uint64_t seed, int32_t n, int32_t* out) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (int32_t k = 0; k < n; ++k) {
    uint32_t ctr[4] = {(uint32_t)k, 0u, 0x5eedu, 0xe7e7u};
    uint32_t w[4];
    su3gen_philox4x32_10(ctr, key, w);
    for (int d = 0; d < 4; ++d) out[4 * k + d] = 4 + 2 * (int32_t)(w[d] % 11u);
  }
}
