/*
 * gen.c -- seeded synthetic inputs shared by the tests, the bench and the
 * oracle comparisons.  It holds no wavelet-tree arithmetic: only random
 * number generation and the workload distributions.
 *
 * PRNG: xoshiro256** (Blackman & Vigna, 2018) seeded through splitmix64.
 * Sequences are generated in chunks of 2^24 symbols; chunk c draws from the
 * stream seeded with seed ^ splitmix64(c), so chunks are independent and the
 * output does not depend on the number of threads.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define CHUNK ((uint64_t)1 << 24)

typedef struct { uint64_t s[4]; } rng_t;

static uint64_t splitmix64_next(uint64_t* x) {
  uint64_t z = (*x += 0x9e3779b97f4a7c15ULL);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

static uint64_t mix(uint64_t v) { uint64_t x = v; return splitmix64_next(&x); }

static void rng_seed(rng_t* r, uint64_t seed) {
  uint64_t x = seed;
  for (int i = 0; i < 4; i++) r->s[i] = splitmix64_next(&x);
}

static uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static uint64_t rng_next(rng_t* r) {
  uint64_t* s = r->s;
  uint64_t result = rotl(s[1] * 5, 7) * 9;
  uint64_t t = s[1] << 17;
  s[2] ^= s[0];
  s[3] ^= s[1];
  s[1] ^= s[2];
  s[0] ^= s[3];
  s[2] ^= t;
  s[3] = rotl(s[3], 45);
  return result;
}

/* uniform integer in [0, m), m <= 2^32 (multiply-shift) */
static uint64_t rng_below(rng_t* r, uint64_t m) { return ((rng_next(r) >> 32) * m) >> 32; }
/* uniform double in [0, 1) with 53 bits */
static double rng_unit(rng_t* r) { return (double)(rng_next(r) >> 11) * (1.0 / 9007199254740992.0); }

static void store(void* out, int width, uint64_t i, uint64_t v) {
  if (width == 1) ((uint8_t*)out)[i] = (uint8_t)v;
  else if (width == 2) ((uint16_t*)out)[i] = (uint16_t)v;
  else ((uint32_t*)out)[i] = (uint32_t)v;
}

/* i.i.d. uniform symbols in [0, sigma) */
void syn_uniform(uint64_t seed, uint64_t n, uint32_t sigma, int width, void* out) {
  int64_t nch = (int64_t)((n + CHUNK - 1) / CHUNK);
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t c = 0; c < nch; c++) {
    rng_t r;
    rng_seed(&r, seed ^ mix((uint64_t)c));
    uint64_t lo = (uint64_t)c * CHUNK, hi = lo + CHUNK < n ? lo + CHUNK : n;
    for (uint64_t i = lo; i < hi; i++) store(out, width, i, rng_below(&r, sigma));
  }
}

/* Seeded Fisher-Yates permutation of [0, sigma). */
void syn_permutation(uint64_t seed, uint32_t sigma, uint32_t* perm) {
  rng_t r;
  rng_seed(&r, seed ^ 0x7065726d75746531ULL);
  for (uint32_t i = 0; i < sigma; i++) perm[i] = i;
  for (uint32_t i = sigma; i > 1; i--) {
    uint32_t j = (uint32_t)rng_below(&r, i);
    uint32_t t = perm[i - 1]; perm[i - 1] = perm[j]; perm[j] = t;
  }
}

/* Zipf(s) over ranks 1..sigma by inverse CDF (cumulative doubles, binary
 * search on a 53-bit uniform), rank r mapped to symbol perm[r-1]. */
int syn_zipf(uint64_t seed, uint64_t n, uint32_t sigma, double s, int width, void* out) {
  double* cdf = (double*)malloc((size_t)sigma * sizeof(double));
  uint32_t* perm = (uint32_t*)malloc((size_t)sigma * sizeof(uint32_t));
  if (!cdf || !perm) { free(cdf); free(perm); return -1; }
  double acc = 0.0;
  for (uint32_t k = 0; k < sigma; k++) { acc += pow((double)(k + 1), -s); cdf[k] = acc; }
  for (uint32_t k = 0; k < sigma; k++) cdf[k] /= acc;
  cdf[sigma - 1] = 1.0;
  syn_permutation(seed, sigma, perm);
  int64_t nch = (int64_t)((n + CHUNK - 1) / CHUNK);
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t c = 0; c < nch; c++) {
    rng_t r;
    rng_seed(&r, seed ^ mix((uint64_t)c));
    uint64_t lo = (uint64_t)c * CHUNK, hi = lo + CHUNK < n ? lo + CHUNK : n;
    for (uint64_t i = lo; i < hi; i++) {
      double u = rng_unit(&r);
      uint32_t a = 0, b = sigma - 1; /* first k with cdf[k] > u */
      while (a < b) { uint32_t m = a + (b - a) / 2; if (cdf[m] > u) b = m; else a = m + 1; }
      store(out, width, i, perm[a]);
    }
  }
  free(cdf); free(perm);
  return 0;
}

/* Standard normal by Marsaglia's polar method. */
static double rng_normal(rng_t* r) {
  for (;;) {
    double u = 2.0 * rng_unit(r) - 1.0, v = 2.0 * rng_unit(r) - 1.0;
    double q = u * u + v * v;
    if (q > 0.0 && q < 1.0) return u * sqrt(-2.0 * log(q) / q);
  }
}

/* Gamma(a), a >= 1, by Marsaglia & Tsang (2000). */
static double rng_gamma_ge1(rng_t* r, double a) {
  double d = a - 1.0 / 3.0, c = 1.0 / sqrt(9.0 * d);
  for (;;) {
    double x = rng_normal(r), v = 1.0 + c * x;
    if (v <= 0.0) continue;
    v = v * v * v;
    double u = rng_unit(r);
    if (u <= 0.0) continue;
    if (log(u) < 0.5 * x * x + d - d * v + d * log(v)) return d * v;
  }
}

/* Gamma(a) for 0 < a < 1 by the boost Gamma(a+1) * U^(1/a). */
static double rng_gamma(rng_t* r, double a) {
  if (a >= 1.0) return rng_gamma_ge1(r, a);
  double g = rng_gamma_ge1(r, a + 1.0);
  double u;
  do { u = rng_unit(r); } while (u <= 0.0);
  return g * pow(u, 1.0 / a);
}

/* Order-3 Markov transition rows over {A,C,G,T} = 0..3: 64 contexts, each
 * row Dirichlet(alpha).  Row-major cumulative probabilities, 64 x 4. */
void syn_markov_table(uint64_t seed, double alpha, double* cum) {
  rng_t r;
  rng_seed(&r, seed ^ 0x6d61726b6f763321ULL);
  for (int ctx = 0; ctx < 64; ctx++) {
    double g[4], t = 0.0;
    for (int k = 0; k < 4; k++) { g[k] = rng_gamma(&r, alpha); t += g[k]; }
    double a = 0.0;
    for (int k = 0; k < 4; k++) { a += g[k] / t; cum[4 * ctx + k] = a; }
    cum[4 * ctx + 3] = 1.0;
  }
}

/* Genome-like text: order-3 chain (context = last three emitted symbols),
 * every draw repeated R ~ Geometric(p_burst) times on {1,2,...}; each chunk
 * starts from a context of three uniform draws (not emitted); symbol 4 (the
 * sentinel) is written at position n-1.  u8 output. */
void syn_genome(uint64_t seed, uint64_t n, double alpha, double p_burst, uint8_t* out) {
  double cum[256];
  syn_markov_table(seed, alpha, cum);
  int64_t nch = (int64_t)((n + CHUNK - 1) / CHUNK);
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t c = 0; c < nch; c++) {
    rng_t r;
    rng_seed(&r, seed ^ mix((uint64_t)c));
    uint64_t lo = (uint64_t)c * CHUNK, hi = lo + CHUNK < n ? lo + CHUNK : n;
    uint32_t ctx = 0;
    for (int k = 0; k < 3; k++) ctx = ((ctx << 2) | (uint32_t)rng_below(&r, 4)) & 63u;
    uint64_t i = lo;
    while (i < hi) {
      double u = rng_unit(&r);
      uint32_t x = 0;
      while (x < 3 && u >= cum[4 * ctx + x]) x++;
      /* geometric burst length on {1,2,...}: count failures before success */
      uint64_t R = 1;
      while (rng_unit(&r) >= p_burst) R++;
      for (uint64_t k = 0; k < R && i < hi; k++, i++) {
        out[i] = (uint8_t)x;
        ctx = ((ctx << 2) | x) & 63u;
      }
    }
  }
  if (n > 0) out[n - 1] = 4;
}

/* Batched workload plan: m sequences with lengths log-uniform in
 * [2^lo_log2, 2^hi_log2]; if their sum exceeds cap, every length is scaled
 * by cap/sum, floored, clamped to >= 2^lo_log2, then the largest is
 * decremented until the sum fits.  sigma from sigmas[0..nsig) uniformly;
 * zipf flag by a fair coin; per-sequence seeds.  Returns the total. */
uint64_t syn_batch_plan(uint64_t seed, uint32_t m, int lo_log2, int hi_log2, uint64_t cap,
                        const uint32_t* sigmas, uint32_t nsig, uint64_t* len,
                        uint32_t* sigma, uint8_t* zipf, uint64_t* seq_seed) {
  rng_t r;
  rng_seed(&r, seed ^ 0x6261746368706c6eULL);
  uint64_t lo = (uint64_t)1 << lo_log2, hi = (uint64_t)1 << hi_log2;
  uint64_t total = 0;
  for (uint32_t i = 0; i < m; i++) {
    double e = (double)lo_log2 + rng_unit(&r) * (double)(hi_log2 - lo_log2);
    uint64_t v = (uint64_t)floor(pow(2.0, e));
    if (v < lo) v = lo;
    if (v > hi) v = hi;
    len[i] = v;
    total += v;
    sigma[i] = sigmas[rng_below(&r, nsig)];
    zipf[i] = (uint8_t)(rng_next(&r) >> 63);
    seq_seed[i] = rng_next(&r);
  }
  if (total > cap) {
    uint64_t t2 = 0;
    for (uint32_t i = 0; i < m; i++) {
      uint64_t v = (uint64_t)floor((double)len[i] * ((double)cap / (double)total));
      if (v < lo) v = lo;
      len[i] = v;
      t2 += v;
    }
    /* repeated "decrement the largest (first on ties)", taken in steps that
     * keep the same element the largest */
    while (t2 > cap) {
      uint32_t big = 0;
      for (uint32_t i = 1; i < m; i++) if (len[i] > len[big]) big = i;
      uint64_t second = 0;
      for (uint32_t i = 0; i < m; i++) if (i != big && len[i] > second) second = len[i];
      uint64_t step = len[big] > second ? len[big] - second : 1;
      if (step > t2 - cap) step = t2 - cap;
      len[big] -= step;
      t2 -= step;
    }
    total = t2;
  }
  return total;
}

/* Uniform random 64-bit words (query arguments, bitvectors). */
void syn_words(uint64_t seed, uint64_t n, uint64_t* out) {
  int64_t nch = (int64_t)((n + CHUNK - 1) / CHUNK);
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t c = 0; c < nch; c++) {
    rng_t r;
    rng_seed(&r, seed ^ mix((uint64_t)c) ^ 0x776f726473ULL);
    uint64_t lo = (uint64_t)c * CHUNK, hi = lo + CHUNK < n ? lo + CHUNK : n;
    for (uint64_t i = lo; i < hi; i++) out[i] = rng_next(&r);
  }
}
