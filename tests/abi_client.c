/* A plain C consumer of include/wavelet.h: builds a wavelet matrix of a small
 * sequence on the current GPU, once from a device copy (wm_build) and once
 * from the host array itself (wm_build_host, pageable memory), and answers
 * rank queries on both, using only the C ABI and the CUDA runtime for device
 * memory.  The CPU test suite compiles it as
 * C99 and as C++ and links it against the library (every call it makes must
 * resolve); it is not run there.  Run on a GPU it prints "abi client ok" and
 * exits 0 when every rank answer of both equals a count on the host. */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime_api.h>

#include "wavelet.h"

#define N 100000u
#define SIGMA 300u
#define Q 64u

static int fail(const char* what, int s) {
  fprintf(stderr, "%s: %d (%s)\n", what, s, wt_status_str((wt_status)s));
  return 1;
}

int main(void) {
  uint16_t* h_seq = (uint16_t*)malloc(N * sizeof(uint16_t));
  uint64_t h_i[Q], h_out[Q], h_out2[Q];
  uint32_t h_c[Q];
  void *d_seq = NULL, *d_i = NULL, *d_c = NULL, *d_out = NULL;
  wt_handle h = NULL, h2 = NULL;
  wt_status s;
  uint32_t x = 12345u, q;
  uint64_t k;
  int bad = 0;
  if (!h_seq) return 1;
  for (k = 0; k < N; k++) {  /* a fixed linear congruential sequence */
    x = x * 1664525u + 1013904223u;
    h_seq[k] = (uint16_t)((x >> 8) % SIGMA);
  }
  for (q = 0; q < Q; q++) {
    h_i[q] = (uint64_t)q * (N / Q) + q;
    h_c[q] = h_seq[(q * 977u) % N];
  }
  if (cudaMalloc(&d_seq, N * sizeof(uint16_t)) != cudaSuccess ||
      cudaMalloc(&d_i, sizeof h_i) != cudaSuccess || cudaMalloc(&d_c, sizeof h_c) != cudaSuccess ||
      cudaMalloc(&d_out, sizeof h_out) != cudaSuccess)
    return fail("cudaMalloc", 0);
  cudaMemcpy(d_seq, h_seq, N * sizeof(uint16_t), cudaMemcpyHostToDevice);
  cudaMemcpy(d_i, h_i, sizeof h_i, cudaMemcpyHostToDevice);
  cudaMemcpy(d_c, h_c, sizeof h_c, cudaMemcpyHostToDevice);

  s = wm_build(d_seq, N, SIGMA, 2, NULL, NULL, &h);
  if (s != WT_OK) return fail("wm_build", s);
  s = wt_rank(h, (const uint32_t*)d_c, (const uint64_t*)d_i, Q, (uint64_t*)d_out, NULL);
  if (s != WT_OK) return fail("wt_rank", s);
  s = wt_sync(h);
  if (s != WT_OK) return fail("wt_sync", s);
  if (wt_memcpy_d2h(h_out, d_out, sizeof h_out) != WT_OK) return fail("wt_memcpy_d2h", 0);
  s = wm_build_host(h_seq, N, SIGMA, 2, NULL, NULL, &h2);
  if (s != WT_OK) return fail("wm_build_host", s);
  s = wt_rank(h2, (const uint32_t*)d_c, (const uint64_t*)d_i, Q, (uint64_t*)d_out, NULL);
  if (s != WT_OK) return fail("wt_rank (host build)", s);
  s = wt_sync(h2);
  if (s != WT_OK) return fail("wt_sync (host build)", s);
  if (wt_memcpy_d2h(h_out2, d_out, sizeof h_out2) != WT_OK) return fail("wt_memcpy_d2h", 0);
  for (q = 0; q < Q; q++) {  /* rank(c, i): occurrences of c in S[0..i] */
    uint64_t cnt = 0;
    for (k = 0; k <= h_i[q]; k++) cnt += h_seq[k] == h_c[q];
    if (cnt != h_out[q]) bad++;
    if (cnt != h_out2[q]) bad++;
  }
  wt_free(h);
  wt_free(h2);
  cudaFree(d_seq);
  cudaFree(d_i);
  cudaFree(d_c);
  cudaFree(d_out);
  free(h_seq);
  if (bad) {
    fprintf(stderr, "%d rank answers differ\n", bad);
    return 1;
  }
  printf("abi client ok\n");
  return 0;
}
