/*
 * A plain C99 caller of libsu3, with no Python and no PyTorch in the process: the SU3_Bench
 * product (§Background, c[i].link[j] = a[i].link[j] x b[j]) through su3_mult on device buffers
 * and through su3_mult_host on pageable host buffers (the path the library picks, then the staged
 * path) and on pinned ones, in FP64 with NATIVE and with F32PAIR arithmetic, each checked against
 * the FP64 oracle within the FP64 form's 1e-13.
 *
 * Test infrastructure: it links the oracle and the seeded input generator beside libsu3 only to
 * compare. Usage: su3_c_caller [L]  (an L^4 lattice, default 8). Exit 0 when every check passed.
 */
#include <cuda_runtime_api.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "su3.h"

/* the seeded SU(3) input generator and the FP64 oracle (their own libraries) */
void su3gen_sites(uint64_t seed, uint32_t lattice, int64_t first_site, int64_t n, int64_t stride_doubles,
                  double* out);
void su3gen_matrices(uint64_t seed, uint32_t lattice, uint64_t first_id, int64_t count, double* out);
void su3o_mult(int64_t n_sites, int64_t site_stride, const double* a, const double* b, double* c);

static su3_handle* h = NULL;

static double max_abs_diff(const double* x, const double* y, int64_t n) {
  double m = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    const double d = fabs(x[i] - y[i]);
    if (!(d <= m)) m = d; /* a NaN difference wins */
  }
  return m;
}

static int su3_ok(su3_status s, const char* what) {
  if (s == SU3_OK) return 1;
  fprintf(stderr, "%s: %s (%s)\n", what, su3_status_string(s), h ? su3_last_error(h) : "");
  return 0;
}

static int cuda_ok(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return 1;
  fprintf(stderr, "%s: %s\n", what, cudaGetErrorString(e));
  return 0;
}

static int check(const char* what, const double* c, const double* ref, int64_t n) {
  const double err = max_abs_diff(c, ref, n);
  printf("%-34s max abs err %.3e\n", what, err);
  if (err <= 1e-13) return 1;
  fprintf(stderr, "%s: error %.3e above 1e-13\n", what, err);
  return 0;
}

int main(int argc, char** argv) {
  const int64_t L = argc > 1 ? atoll(argv[1]) : 8;
  const int64_t V = L * L * L * L, n = 72 * V;
  const size_t bytes = (size_t)n * sizeof(double);
  const uint64_t seed = 2103;
  double b[72];
  double* a = (double*)malloc(bytes);
  double* c = (double*)malloc(bytes);
  double* ref = (double*)malloc(bytes);
  if (!a || !c || !ref) return 2;
  su3gen_sites(seed, 0, 0, V, 72, a);
  su3gen_matrices(seed, 0, (uint64_t)(4 * V), 4, b); /* the lattice's four b matrices */
  su3o_mult(V, 72, a, b, ref);

  if (!su3_ok(su3_init(0, &h), "su3_init")) return 1;
  printf("pageable host access: %d\n", (int)su3_host_pageable_access(h));
  double *a_dev = NULL, *c_dev = NULL, *a_pin = NULL, *c_pin = NULL;
  if (!cuda_ok(cudaMalloc((void**)&a_dev, bytes), "cudaMalloc a") ||
      !cuda_ok(cudaMalloc((void**)&c_dev, bytes), "cudaMalloc c") ||
      !cuda_ok(cudaMallocHost((void**)&a_pin, bytes), "cudaMallocHost a") ||
      !cuda_ok(cudaMallocHost((void**)&c_pin, bytes), "cudaMallocHost c") ||
      !cuda_ok(cudaMemcpy(a_dev, a, bytes, cudaMemcpyHostToDevice), "copy a"))
    return 1;
  memcpy(a_pin, a, bytes);

  int ok = 1;
  const int32_t ariths[2] = {SU3_ARITH_NATIVE, SU3_ARITH_F32PAIR};
  const char* names[2] = {"native", "f32pair"};
  for (int t = 0; t < 2 && ok; ++t) {
    su3_desc d = {SU3_F64, SU3_REPR_FULL18, SU3_LAYOUT_AOS, ariths[t], V, 0};
    char what[64];

    /* device buffers, asynchronous on the default stream, errors surfacing at su3_sync */
    ok = ok && cuda_ok(cudaMemset(c_dev, 0, bytes), "memset c");
    ok = ok && su3_ok(su3_mult(h, &d, a_dev, b, &d, c_dev, NULL), "su3_mult");
    ok = ok && su3_ok(su3_sync(h, NULL, -1), "su3_sync");
    ok = ok && cuda_ok(cudaMemcpy(c, c_dev, bytes, cudaMemcpyDeviceToHost), "copy c");
    snprintf(what, sizeof what, "su3_mult device %s", names[t]);
    ok = ok && check(what, c, ref, n);

    /* pageable host buffers: streamed by the kernel on a device that reads them coherently,
       else copied through HBM */
    const int32_t want_path = su3_host_pageable_access(h) ? SU3_HOST_DIRECT : SU3_HOST_STAGED;
    memset(c, 0, bytes);
    ok = ok && su3_ok(su3_mult_host(h, &d, a, b, &d, c, NULL), "su3_mult_host pageable");
    snprintf(what, sizeof what, "su3_mult_host pageable %s", names[t]);
    ok = ok && check(what, c, ref, n);
    if (ok && su3_last_host_path(h) != want_path) {
      fprintf(stderr, "pageable buffers took path %d, not %d\n", (int)su3_last_host_path(h), (int)want_path);
      ok = 0;
    }

    /* pageable host buffers forced through the staged path */
    memset(c, 0, bytes);
    ok = ok && su3_ok(su3_set_host_path(h, SU3_HOST_STAGED), "su3_set_host_path");
    ok = ok && su3_ok(su3_mult_host(h, &d, a, b, &d, c, NULL), "su3_mult_host pageable staged");
    snprintf(what, sizeof what, "su3_mult_host pageable staged %s", names[t]);
    ok = ok && check(what, c, ref, n);
    if (ok && su3_last_host_path(h) != SU3_HOST_STAGED) {
      fprintf(stderr, "SU3_HOST_STAGED took path %d\n", (int)su3_last_host_path(h));
      ok = 0;
    }
    ok = su3_ok(su3_set_host_path(h, SU3_HOST_AUTO), "su3_set_host_path") && ok;

    /* pinned host buffers: the kernel streams them over the host link */
    memset(c_pin, 0, bytes);
    ok = ok && su3_ok(su3_mult_host(h, &d, a_pin, b, &d, c_pin, NULL), "su3_mult_host pinned");
    snprintf(what, sizeof what, "su3_mult_host pinned %s", names[t]);
    ok = ok && check(what, c_pin, ref, n);
    if (ok && su3_last_host_path(h) != SU3_HOST_DIRECT) {
      fprintf(stderr, "pinned buffers took path %d, not the direct path\n", (int)su3_last_host_path(h));
      ok = 0;
    }
  }

  cudaFree(a_dev);
  cudaFree(c_dev);
  cudaFreeHost(a_pin);
  cudaFreeHost(c_pin);
  ok = su3_ok(su3_finalize(h), "su3_finalize") && ok;
  free(a);
  free(c);
  free(ref);
  if (ok) printf("c caller ok: L=%lld, %lld sites\n", (long long)L, (long long)V);
  return ok ? 0 : 1;
}
