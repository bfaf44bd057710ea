/*
 * wt_oracle.c -- the CPU oracle (TEST INFRASTRUCTURE; see oracle.h).
 *
 * Plain definitions, written out step by step, single-threaded.  Each
 * function names the passage of Shun's paper it follows.  Nothing here is
 * tuned; it must stay readable against the paper.
 */
#include "oracle.h"

#include <stdlib.h>
#include <string.h>

#define NONE UINT64_MAX

static int getbit(const uint64_t* w, uint64_t i) { return (int)((w[i >> 6] >> (i & 63)) & 1u); }
static void setbit(uint64_t* w, uint64_t i) { w[i >> 6] |= (uint64_t)1 << (i & 63); }
static uint32_t xbit(uint32_t x, int k) { return (x >> k) & 1u; }

uint32_t orc_levels(uint32_t sigma) {
  /* Root range [0, 2^ceil(log sigma) - 1] (§2): ceil(log2 sigma) levels. */
  uint32_t L = 0;
  while (L < 32 && ((uint64_t)1 << L) < (uint64_t)sigma) L++;
  return L == 0 ? 1 : L; /* sigma = 1: one all-zero level (reading) */
}

uint64_t orc_level_words(uint64_t nbits) { return ((nbits + 2047) / 2048) * 32; }

/* ---------------------------------------------------------------------- */
/* Balanced wavelet tree (§2).  Node [a,b] stores 0 for symbols in its left */
/* half and 1 otherwise; children hold the left/right halves.  Levelwise:   */
/* level l lists the nodes of depth l left to right, i.e. T_l = S stably    */
/* ordered by the top l bits, and its bit is bit L-1-l.  T_{l+1} is built   */
/* from T_l by a stable 0/1 partition inside every node segment.            */
/* ---------------------------------------------------------------------- */
int orc_wt_build(const uint32_t* S, uint64_t n, uint32_t sigma, uint64_t* bits) {
  uint32_t L = orc_levels(sigma);
  uint64_t W = orc_level_words(n);
  memset(bits, 0, (size_t)(L * W) * sizeof(uint64_t));
  if (n == 0) return 0;
  uint32_t* T = (uint32_t*)malloc(n * sizeof(uint32_t));
  uint32_t* U = (uint32_t*)malloc(n * sizeof(uint32_t));
  if (!T || !U) { free(T); free(U); return -1; }
  memcpy(T, S, n * sizeof(uint32_t));
  for (uint32_t l = 0; l < L; l++) {
    int k = (int)(L - 1 - l);
    uint64_t* B = bits + (uint64_t)l * W;
    for (uint64_t i = 0; i < n; i++)
      if (xbit(T[i], k)) setbit(B, i);
    /* node segments of T_l: maximal runs of equal prefix x >> (L - l) */
    uint64_t s = 0;
    while (s < n) {
      uint64_t e = s + 1;
      uint64_t pref = (l == 0) ? 0 : ((uint64_t)T[s] >> (L - l));
      while (e < n && ((l == 0) ? 0 : ((uint64_t)T[e] >> (L - l))) == pref) e++;
      uint64_t o = s;
      for (uint64_t i = s; i < e; i++)
        if (!xbit(T[i], k)) U[o++] = T[i];
      for (uint64_t i = s; i < e; i++)
        if (xbit(T[i], k)) U[o++] = T[i];
      s = e;
    }
    uint32_t* t = T; T = U; U = t;
  }
  free(T); free(U);
  return 0;
}

/* ---------------------------------------------------------------------- */
/* Wavelet matrix (§4.3): level l holds bit l (counted from the top) of the */
/* sequence T_l; T_{l+1} puts the elements of T_l whose bit is 0 first and  */
/* those with 1 after, each group in T_l order.  zeros[l] = number of 0s.   */
/* ---------------------------------------------------------------------- */
int orc_wm_build(const uint32_t* S, uint64_t n, uint32_t sigma, uint64_t* bits,
                 uint64_t* zeros) {
  uint32_t L = orc_levels(sigma);
  uint64_t W = orc_level_words(n);
  memset(bits, 0, (size_t)(L * W) * sizeof(uint64_t));
  for (uint32_t l = 0; l < L; l++) zeros[l] = 0;
  if (n == 0) return 0;
  uint32_t* T = (uint32_t*)malloc(n * sizeof(uint32_t));
  uint32_t* U = (uint32_t*)malloc(n * sizeof(uint32_t));
  if (!T || !U) { free(T); free(U); return -1; }
  memcpy(T, S, n * sizeof(uint32_t));
  for (uint32_t l = 0; l < L; l++) {
    int k = (int)(L - 1 - l);
    uint64_t* B = bits + (uint64_t)l * W;
    uint64_t o = 0;
    for (uint64_t i = 0; i < n; i++) {
      if (xbit(T[i], k)) setbit(B, i);
      else U[o++] = T[i];
    }
    zeros[l] = o;
    for (uint64_t i = 0; i < n; i++)
      if (xbit(T[i], k)) U[o++] = T[i];
    uint32_t* t = T; T = U; U = t;
  }
  free(T); free(U);
  return 0;
}

/* ---------------------------------------------------------------------- */
/* Rank directory (§5.1 rank: only the rank of 0 is stored; ranges and     */
/* sub-ranges with absolute and relative counts).  Written as: walk the    */
/* bits once, keep the running count of zeros, and read it off at every    */
/* 2048-bit and 512-bit boundary (clamped to nbits).                       */
/* ---------------------------------------------------------------------- */
void orc_rank_dir(const uint64_t* bits, uint64_t nbits, uint64_t* rec) {
  uint64_t nsb = (nbits + 2047) / 2048;
  uint64_t z = 0; /* zeros in [0, p) */
  uint64_t p = 0;
  for (uint64_t s = 0; s < nsb; s++) {
    uint64_t zb = z;
    uint64_t relw = 0;
    for (uint32_t b = 0; b < 4; b++) {
      uint64_t boundary = 2048 * s + 512 * (uint64_t)b;
      if (boundary > nbits) boundary = nbits;
      while (p < boundary) { if (!getbit(bits, p)) z++; p++; }
      relw |= (uint64_t)(z - zb) << (16 * b);
    }
    rec[2 * s] = zb;
    rec[2 * s + 1] = relw;
    uint64_t end = 2048 * (s + 1);
    if (end > nbits) end = nbits;
    while (p < end) { if (!getbit(bits, p)) z++; p++; }
  }
  rec[2 * nsb] = z;
  rec[2 * nsb + 1] = 0;
}

/* Sampled select (§5.1 select keeps the position of every (log n loglog n)- */
/* th 1; here every 4096th occurrence of b, counting from occurrence 0).   */
/* element p of a sequence of width-bit values packed LSB first into u64
   words (width 1: a bitvector; width 2: a digit level of the 4-ary tree) */
static uint32_t elem(const uint64_t* w, uint64_t p, int width) {
  uint64_t b = p * (uint64_t)width;
  return (uint32_t)((w[b >> 6] >> (b & 63)) & ((1u << width) - 1u));
}

static uint64_t samples_w(const uint64_t* w, uint64_t n, int width, uint32_t v,
                          uint64_t* samp) {
  uint64_t cnt = 0, ns = 0;
  for (uint64_t p = 0; p < n; p++) {
    if (elem(w, p, width) == v) {
      if (cnt % 4096 == 0) samp[ns++] = p;
      cnt++;
    }
  }
  return ns;
}

uint64_t orc_select_samples(const uint64_t* bits, uint64_t nbits, uint32_t b,
                            uint64_t* samp) {
  return samples_w(bits, nbits, 1, b, samp);
}

uint64_t orc_digit_samples(const uint64_t* dig, uint64_t ndig, uint32_t d, uint64_t* samp) {
  return samples_w(dig, ndig, 2, d, samp);
}

/* ---------------------------------------------------------------------- */
/* Clark-style select directory (§5.1 select), as defined in oracle.h.      */
/* ---------------------------------------------------------------------- */
static int clark_w(const uint64_t* bits, uint64_t nbits, int width, uint32_t b,
                   uint64_t huge_min, uint64_t sparse_min, uint64_t* nranges, uint64_t* nhuge,
                   uint64_t* nsparse, uint64_t* desc, uint32_t* sub, uint32_t* sparse,
                   uint64_t* huge) {
  /* pass 1: the positions of occurrences 0, 256, 512, ... */
  uint64_t cnt = 0;
  for (uint64_t p = 0; p < nbits; p++)
    if (elem(bits, p, width) == b) cnt++;
  uint64_t M = (cnt + 255) / 256, R = (cnt + 4095) / 4096;
  uint64_t* p256 = (uint64_t*)malloc((M + 1) * sizeof(uint64_t));
  if (!p256) return -1;
  uint64_t c = 0;
  for (uint64_t p = 0; p < nbits; p++) {
    if (elem(bits, p, width) == b) {
      if (c % 256 == 0) p256[c / 256] = p;
      c++;
    }
  }
  /* ranges: range k starts at occurrence 4096k and ends where range k+1
     starts (the last one at the end of the bitvector) */
  uint64_t nh = 0, ns = 0;
  for (uint64_t k = 0; k < R; k++) {
    uint64_t S1 = p256[16 * k];
    uint64_t e = (k + 1 < R) ? p256[16 * (k + 1)] : nbits;
    int is_huge = (e - S1) >= huge_min;
    uint32_t mask = 0;
    for (uint64_t i = 0; i < 16; i++) {
      uint64_t m = 16 * k + i;
      if (sub) sub[m] = is_huge ? 0u : (m < M ? (uint32_t)(p256[m] - S1) : 0xffffffffu);
      if (is_huge || m >= M) continue;
      uint64_t end = (i + 1 < 16 && m + 1 < M) ? p256[m + 1] : e;
      if (end - p256[m] >= sparse_min) mask |= 1u << i;
    }
    if (desc) {
      if (is_huge) desc[k] = ((uint64_t)1 << 63) | (4096 * nh);
      else desc[k] = ns | ((uint64_t)mask << 40);
    }
    /* pass 2 for this range: every occurrence it stores explicitly */
    if (is_huge) {
      if (huge) {
        uint64_t j = 0;
        for (uint64_t p = S1; p < e && j < 4096; p++)
          if (elem(bits, p, width) == b) huge[4096 * nh + j++] = p;
        for (; j < 4096; j++) huge[4096 * nh + j] = NONE;
      }
      nh++;
    } else {
      for (uint64_t i = 0; i < 16; i++) {
        if (!((mask >> i) & 1u)) continue;
        if (sparse) {
          uint64_t m = 16 * k + i, j = 0;
          for (uint64_t p = p256[m]; p < nbits && j < 256; p++)
            if (elem(bits, p, width) == b) sparse[256 * ns + j++] = (uint32_t)(p - S1);
          for (; j < 256; j++) sparse[256 * ns + j] = 0xffffffffu;
        }
        ns++;
      }
    }
  }
  free(p256);
  if (nranges) *nranges = R;
  if (nhuge) *nhuge = nh;
  if (nsparse) *nsparse = ns;
  return 0;
}

int orc_clark_build(const uint64_t* bits, uint64_t nbits, uint32_t b, uint64_t huge_min,
                    uint64_t sparse_min, uint64_t* nranges, uint64_t* nhuge, uint64_t* nsparse,
                    uint64_t* desc, uint32_t* sub, uint32_t* sparse, uint64_t* huge) {
  return clark_w(bits, nbits, 1, b, huge_min, sparse_min, nranges, nhuge, nsparse, desc, sub,
                 sparse, huge);
}

int orc_clark_digits(const uint64_t* dig, uint64_t ndig, uint32_t d, uint64_t huge_min,
                     uint64_t sparse_min, uint64_t* nranges, uint64_t* nhuge, uint64_t* nsparse,
                     uint64_t* desc, uint32_t* sub, uint32_t* sparse, uint64_t* huge) {
  return clark_w(dig, ndig, 2, d, huge_min, sparse_min, nranges, nhuge, nsparse, desc, sub,
                 sparse, huge);
}

/* ---------------------------------------------------------------------- */
/* Huffman code lengths (§4.3: the tree shape is given by codewords; the    */
/* Huffman shape is the example the paper names).                          */
/* ---------------------------------------------------------------------- */
typedef struct { uint64_t w; uint64_t id; } hnode;

static int hless(hnode a, hnode b) { return a.w < b.w || (a.w == b.w && a.id < b.id); }

static void hpush(hnode* h, uint64_t* sz, hnode x) {
  uint64_t i = (*sz)++;
  h[i] = x;
  while (i > 0) {
    uint64_t p = (i - 1) / 2;
    if (!hless(h[i], h[p])) break;
    hnode t = h[i]; h[i] = h[p]; h[p] = t; i = p;
  }
}

static hnode hpop(hnode* h, uint64_t* sz) {
  hnode top = h[0];
  h[0] = h[--(*sz)];
  uint64_t i = 0;
  for (;;) {
    uint64_t l = 2 * i + 1, r = l + 1, m = i;
    if (l < *sz && hless(h[l], h[m])) m = l;
    if (r < *sz && hless(h[r], h[m])) m = r;
    if (m == i) break;
    hnode t = h[i]; h[i] = h[m]; h[m] = t; i = m;
  }
  return top;
}

/* Package-merge (Larmore & Hirschberg 1990) for lengths <= cap.  Leaves are
 * ordered by (weight, symbol); in each merged list a leaf precedes a package
 * of equal weight.  Lists are built from depth cap up to depth 1, the first
 * 2m-2 items of the depth-1 list are taken, and a leaf's length is the number
 * of lists in which it is among the taken items. */
static void package_merge(const uint64_t* w, const uint32_t* sym, uint32_t m,
                          uint32_t cap, uint8_t* len) {
  /* lists[d] for d = 1..cap, each up to 2m items: weight and is-leaf flag */
  uint64_t cap2 = 2 * (uint64_t)m;
  uint64_t** lw = (uint64_t**)calloc(cap + 1, sizeof(uint64_t*));
  uint8_t** lf = (uint8_t**)calloc(cap + 1, sizeof(uint8_t*));
  uint64_t* lsz = (uint64_t*)calloc(cap + 1, sizeof(uint64_t));
  for (uint32_t d = 1; d <= cap; d++) {
    lw[d] = (uint64_t*)malloc(cap2 * sizeof(uint64_t));
    lf[d] = (uint8_t*)malloc(cap2);
  }
  /* depth cap: the leaves alone */
  for (uint32_t i = 0; i < m; i++) { lw[cap][i] = w[i]; lf[cap][i] = 1; }
  lsz[cap] = m;
  for (uint32_t d = cap; d > 1; d--) {
    /* packages of list d: pairs of consecutive items */
    uint64_t np = lsz[d] / 2;
    uint64_t i = 0, j = 0, o = 0;
    while (i < m || j < np) {
      uint64_t pw = (j < np) ? lw[d][2 * j] + lw[d][2 * j + 1] : 0;
      if (i < m && (j >= np || w[i] <= pw)) { lw[d - 1][o] = w[i]; lf[d - 1][o] = 1; i++; }
      else { lw[d - 1][o] = pw; lf[d - 1][o] = 0; j++; }
      o++;
    }
    lsz[d - 1] = o;
  }
  for (uint32_t i = 0; i < m; i++) len[sym[i]] = 0;
  uint64_t take = 2 * (uint64_t)m - 2;
  for (uint32_t d = 1; d <= cap && take > 0; d++) {
    uint64_t leaves = 0, packs = 0;
    for (uint64_t i = 0; i < take; i++) {
      if (lf[d][i]) leaves++; else packs++;
    }
    for (uint64_t i = 0; i < leaves; i++) len[sym[i]]++;
    take = 2 * packs;
  }
  for (uint32_t d = 1; d <= cap; d++) { free(lw[d]); free(lf[d]); }
  free(lw); free(lf); free(lsz);
}

uint32_t orc_huffman_lengths(const uint64_t* hist, uint32_t sigma, uint32_t cap,
                             uint8_t* len) {
  memset(len, 0, sigma);
  uint32_t m = 0;
  for (uint32_t s = 0; s < sigma; s++) if (hist[s]) m++;
  if (m == 0) return 0;
  if (m == 1) {
    for (uint32_t s = 0; s < sigma; s++) if (hist[s]) len[s] = 1;
    return 1;
  }
  uint64_t nn = 2 * (uint64_t)m - 1;
  hnode* h = (hnode*)malloc(nn * sizeof(hnode));
  uint64_t* parent = (uint64_t*)malloc(((uint64_t)sigma + m) * sizeof(uint64_t));
  uint64_t sz = 0;
  for (uint32_t s = 0; s < sigma; s++) {
    if (hist[s]) { hnode x = { hist[s], s }; hpush(h, &sz, x); }
  }
  uint64_t next = sigma;
  while (sz > 1) {
    hnode a = hpop(h, &sz), b = hpop(h, &sz);
    parent[a.id] = next;
    parent[b.id] = next;
    hnode c = { a.w + b.w, next };
    next++;
    hpush(h, &sz, c);
  }
  uint64_t root = next - 1;
  uint32_t maxlen = 0;
  for (uint32_t s = 0; s < sigma; s++) {
    if (!hist[s]) continue;
    uint32_t d = 0;
    uint64_t v = s;
    while (v != root) { v = parent[v]; d++; }
    len[s] = (uint8_t)(d > 255 ? 255 : d);
    if (d > maxlen) maxlen = d;
  }
  free(h); free(parent);
  if (maxlen <= cap) return maxlen;
  /* length-limited: leaves sorted by (weight, symbol) */
  uint64_t* w = (uint64_t*)malloc(m * sizeof(uint64_t));
  uint32_t* sym = (uint32_t*)malloc(m * sizeof(uint32_t));
  uint32_t k = 0;
  for (uint32_t s = 0; s < sigma; s++) if (hist[s]) { sym[k] = s; w[k] = hist[s]; k++; }
  /* insertion sort is fine for an oracle only on small inputs; use a plain
   * merge sort on (w, sym) to stay O(m log m). */
  {
    uint64_t* tw = (uint64_t*)malloc(m * sizeof(uint64_t));
    uint32_t* ts = (uint32_t*)malloc(m * sizeof(uint32_t));
    for (uint64_t width = 1; width < m; width *= 2) {
      for (uint64_t lo = 0; lo < m; lo += 2 * width) {
        uint64_t mid = lo + width < m ? lo + width : m;
        uint64_t hi = lo + 2 * width < m ? lo + 2 * width : m;
        uint64_t a = lo, b = mid, o = lo;
        while (a < mid || b < hi) {
          int takea = b >= hi || (a < mid && (w[a] < w[b] || (w[a] == w[b] && sym[a] < sym[b])));
          if (takea) { tw[o] = w[a]; ts[o] = sym[a]; a++; }
          else { tw[o] = w[b]; ts[o] = sym[b]; b++; }
          o++;
        }
      }
      memcpy(w, tw, m * sizeof(uint64_t));
      memcpy(sym, ts, m * sizeof(uint32_t));
    }
    free(tw); free(ts);
  }
  package_merge(w, sym, m, cap, len);
  maxlen = 0;
  for (uint32_t i = 0; i < m; i++) if (len[sym[i]] > maxlen) maxlen = len[sym[i]];
  free(w); free(sym);
  return maxlen;
}

void orc_canonical_codes(const uint8_t* len, uint32_t sigma, uint32_t* code) {
  /* order by (len, symbol): a counting pass over lengths 1..255 */
  uint32_t code_val = 0;
  uint32_t prev_len = 0;
  int first = 1;
  for (uint32_t s = 0; s < sigma; s++) code[s] = 0;
  for (uint32_t ln = 1; ln <= 255; ln++) {
    for (uint32_t s = 0; s < sigma; s++) {
      if (len[s] != ln) continue;
      if (first) { code_val = 0; first = 0; }
      else { code_val = (code_val + 1) << (ln - prev_len); }
      prev_len = ln;
      code[s] = code_val;
    }
  }
}

void orc_huff_level_sizes(const uint32_t* S, uint64_t n, const uint8_t* len,
                          uint32_t maxlen, uint64_t* nl) {
  for (uint32_t l = 0; l < maxlen; l++) nl[l] = 0;
  for (uint64_t i = 0; i < n; i++)
    for (uint32_t l = 0; l < maxlen; l++)
      if (len[S[i]] > l) nl[l]++;
}

/* Code bit l of symbol x (MSB first, §4.3 codeword definition). */
static uint32_t cbit(const uint8_t* len, const uint32_t* code, uint32_t x, uint32_t l) {
  return (code[x] >> (len[x] - 1 - l)) & 1u;
}
static uint64_t cprefix(const uint8_t* len, const uint32_t* code, uint32_t x, uint32_t l) {
  return l == 0 ? 0 : ((uint64_t)code[x] >> (len[x] - l));
}

int orc_huff_wt_build(const uint32_t* S, uint64_t n, const uint8_t* len,
                      const uint32_t* code, uint32_t maxlen,
                      const uint64_t* woff, uint64_t* bits) {
  if (n == 0 || maxlen == 0) return 0;
  uint32_t* T = (uint32_t*)malloc(n * sizeof(uint32_t));
  uint32_t* U = (uint32_t*)malloc(n * sizeof(uint32_t));
  if (!T || !U) { free(T); free(U); return -1; }
  memcpy(T, S, n * sizeof(uint32_t));
  uint64_t m = n; /* current level length */
  for (uint32_t l = 0; l < maxlen; l++) {
    uint64_t* B = bits + woff[l];
    memset(B, 0, (size_t)orc_level_words(m) * sizeof(uint64_t));
    for (uint64_t i = 0; i < m; i++)
      if (cbit(len, code, T[i], l)) setbit(B, i);
    /* next level: stable partition inside each node (equal l-bit prefix),
     * then drop the elements whose codeword ends at this level */
    uint64_t s = 0, o = 0;
    while (s < m) {
      uint64_t e = s + 1;
      uint64_t pref = cprefix(len, code, T[s], l);
      while (e < m && cprefix(len, code, T[e], l) == pref) e++;
      for (uint64_t i = s; i < e; i++)
        if (!cbit(len, code, T[i], l) && len[T[i]] > l + 1) U[o++] = T[i];
      for (uint64_t i = s; i < e; i++)
        if (cbit(len, code, T[i], l) && len[T[i]] > l + 1) U[o++] = T[i];
      s = e;
    }
    m = o;
    uint32_t* t = T; T = U; U = t;
  }
  free(T); free(U);
  return 0;
}

/* ---------------------------------------------------------------------- */
/* 4-ary wavelet tree (§4.3 multiary): keep the sequences of the binary     */
/* nodes at levels beta*log d; each stores the log d bits below its level.  */
/* ---------------------------------------------------------------------- */
int orc_mwt_build(const uint32_t* S, uint64_t n, uint32_t sigma, uint64_t* dig) {
  uint32_t L = orc_levels(sigma);
  uint32_t D = (L + 1) / 2;
  uint64_t W = orc_level_words(2 * n);
  memset(dig, 0, (size_t)(D * W) * sizeof(uint64_t));
  if (n == 0) return 0;
  uint32_t* T = (uint32_t*)malloc(n * sizeof(uint32_t));
  uint32_t* U = (uint32_t*)malloc(n * sizeof(uint32_t));
  if (!T || !U) { free(T); free(U); return -1; }
  memcpy(T, S, n * sizeof(uint32_t));
  for (uint32_t l = 0; l < L; l++) {
    int k = (int)(L - 1 - l);
    if (l % 2 == 0) {
      uint64_t* Dg = dig + (uint64_t)(l / 2) * W;
      for (uint64_t i = 0; i < n; i++) {
        uint64_t d = (l + 1 < L) ? ((xbit(T[i], k) << 1) | xbit(T[i], k - 1)) : xbit(T[i], k);
        Dg[i >> 5] |= d << (2 * (i & 31));
      }
    }
    /* binary level l -> l+1 as in orc_wt_build */
    uint64_t s = 0;
    while (s < n) {
      uint64_t e = s + 1;
      uint64_t pref = (l == 0) ? 0 : ((uint64_t)T[s] >> (L - l));
      while (e < n && ((l == 0) ? 0 : ((uint64_t)T[e] >> (L - l))) == pref) e++;
      uint64_t o = s;
      for (uint64_t i = s; i < e; i++) if (!xbit(T[i], k)) U[o++] = T[i];
      for (uint64_t i = s; i < e; i++) if (xbit(T[i], k)) U[o++] = T[i];
      s = e;
    }
    uint32_t* t = T; T = U; U = t;
  }
  free(T); free(U);
  return 0;
}

void orc_mwt_dir(const uint64_t* dig, uint64_t ndig, uint64_t* rec) {
  uint64_t nsb = (ndig + 1023) / 1024;
  uint64_t cnt[4] = {0, 0, 0, 0};
  uint64_t p = 0;
  for (uint64_t s = 0; s < nsb; s++) {
    uint64_t base[4] = {cnt[0], cnt[1], cnt[2], cnt[3]};
    for (int v = 0; v < 4; v++) rec[8 * s + v] = base[v];
    for (uint32_t b = 0; b < 4; b++) {
      uint64_t boundary = 1024 * s + 256 * (uint64_t)b;
      if (boundary > ndig) boundary = ndig;
      while (p < boundary) { cnt[(dig[p >> 5] >> (2 * (p & 31))) & 3u]++; p++; }
      uint64_t w = 0;
      for (int v = 0; v < 4; v++) w |= (cnt[v] - base[v]) << (16 * v);
      rec[8 * s + 4 + b] = w;
    }
    uint64_t end = 1024 * (s + 1);
    if (end > ndig) end = ndig;
    while (p < end) { cnt[(dig[p >> 5] >> (2 * (p & 31))) & 3u]++; p++; }
  }
  for (int v = 0; v < 4; v++) rec[8 * nsb + v] = cnt[v];
  for (int b = 0; b < 4; b++) rec[8 * nsb + 4 + b] = 0;
}

/* ---------------------------------------------------------------------- */
/* Queries by definition (§2).  Positions of each symbol are gathered once  */
/* with a counting pass so that each answer is a lookup.                    */
/* ---------------------------------------------------------------------- */
void orc_access(const uint32_t* S, uint64_t n, const uint64_t* i, uint64_t q,
                uint64_t* out) {
  for (uint64_t t = 0; t < q; t++) out[t] = (i[t] < n) ? (uint64_t)S[i[t]] : NONE;
}

typedef struct { uint64_t* off; uint64_t* pos; } poslist;

static int build_poslist(const uint32_t* S, uint64_t n, uint32_t sigma, poslist* P) {
  P->off = (uint64_t*)calloc((uint64_t)sigma + 1, sizeof(uint64_t));
  P->pos = (uint64_t*)malloc((n ? n : 1) * sizeof(uint64_t));
  if (!P->off || !P->pos) return -1;
  for (uint64_t i = 0; i < n; i++) if (S[i] < sigma) P->off[S[i] + 1]++;
  for (uint32_t c = 0; c < sigma; c++) P->off[c + 1] += P->off[c];
  uint64_t* fill = (uint64_t*)malloc(((uint64_t)sigma + 1) * sizeof(uint64_t));
  memcpy(fill, P->off, ((uint64_t)sigma + 1) * sizeof(uint64_t));
  for (uint64_t i = 0; i < n; i++) if (S[i] < sigma) P->pos[fill[S[i]]++] = i;
  free(fill);
  return 0;
}

void orc_rank(const uint32_t* S, uint64_t n, uint32_t sigma, const uint32_t* c,
              const uint64_t* i, uint64_t q, uint64_t* out) {
  poslist P;
  if (build_poslist(S, n, sigma, &P)) return;
  for (uint64_t t = 0; t < q; t++) {
    if (i[t] >= n || c[t] >= sigma) { out[t] = NONE; continue; }
    /* number of positions of c that are <= i */
    uint64_t lo = P.off[c[t]], hi = P.off[c[t] + 1];
    while (lo < hi) {
      uint64_t mid = lo + (hi - lo) / 2;
      if (P.pos[mid] <= i[t]) lo = mid + 1; else hi = mid;
    }
    out[t] = lo - P.off[c[t]];
  }
  free(P.off); free(P.pos);
}

void orc_select(const uint32_t* S, uint64_t n, uint32_t sigma, const uint32_t* c,
                const uint64_t* k, uint64_t q, uint64_t* out) {
  poslist P;
  if (build_poslist(S, n, sigma, &P)) return;
  for (uint64_t t = 0; t < q; t++) {
    if (c[t] >= sigma || k[t] == 0) { out[t] = NONE; continue; }
    uint64_t cnt = P.off[c[t] + 1] - P.off[c[t]];
    out[t] = (k[t] <= cnt) ? P.pos[P.off[c[t]] + k[t] - 1] : NONE;
  }
  free(P.off); free(P.pos);
}
