// ddmerge.cu -- domain-decomposition merge (Section 4.2): the levels of one
// sequence from the structures of its consecutive parts S_0 S_1 ... S_{R-1}.
//
// Every level of the whole sequence lists its nodes in order (balanced
// tree: the top-l-bit prefixes; wavelet matrix: the classes of the reversed
// top l bits) and each node's elements in sequence order, i.e. part by part.
// So the level bitmap of the whole is, node by node, the concatenation of the
// parts' bit runs of that node, placed at offsets given by prefix sums of the
// node sizes over nodes and parts (the paper's merge of the K sub-problems).
//
// Steps, all on the device:
//   1. node sizes and starts of every level of every part, level by level:
//      a node's children are its zeros and its ones (rank queries on the
//      part's directory at the node's two ends);
//   2. destination of every (part, node) run: exclusive scan of the node
//      totals over the nodes of a level, plus the runs of the earlier parts;
//   3. the runs' destinations cut at multiples of 32768 bits, the run of
//      every piece written out, then one warp per piece, 16 destination
//      words per lane: whole words are stored, words shared with a
//      neighbouring run are ORed into the zeroed level buffer.
// On one GPU the parts' bits are read in place.  Across GPUs, a rank's runs
// go to the rank owning their destination positions (the routing is planned
// in paper_1610_03524_gb300/dist.py).
#include <algorithm>
#include <cstdio>
#include <vector>

#include "wt_host.h"
#include "wt_internal.cuh"

namespace wtk {

wt_status scan_excl_u64_pub(const uint64_t* in, uint64_t* out, uint64_t n, uint64_t* scratch,
                            cudaStream_t st);
uint64_t scan_scratch_pub(uint64_t n);

#define CK(x)                                                                   \
  do {                                                                          \
    cudaError_t e_ = (x);                                                       \
    if (e_ != cudaSuccess) {                                                    \
      fprintf(stderr, "wavelet: %s -> %s\n", #x, cudaGetErrorString(e_));      \
      return e_ == cudaErrorMemoryAllocation ? WT_ERR_NO_MEMORY : WT_ERR_CUDA; \
    }                                                                           \
  } while (0)

constexpr uint32_t DD_PIECE = 32768;  // bits per piece of a run: 16 words per lane

// one level of one part
struct DdLevel {
  const uint64_t* bits;  // the level's words
  const uint64_t* dir;   // its rank directory (2 u64 per 2048-bit superblock + total)
  uint64_t n;            // bits on the level
};

// zeros in [0, x) of a binary level, x <= n (the directory's record layout:
// u64 zeros before the superblock, 4 x u16 zeros before each 512-bit block)
__device__ uint64_t dd_rank0(const DdLevel& v, uint64_t x) {
  const uint64_t s = x >> 11;
  const uint32_t b = (uint32_t)((x >> 9) & 3);
  uint64_t r = v.dir[2 * s] + ((v.dir[2 * s + 1] >> (16 * b)) & 0xffffull);
  const uint64_t wend = x >> 6;
  for (uint64_t w = 32 * s + 8 * b; w < wend; w++) r += 64 - __popcll(v.bits[w]);
  const uint32_t rem = (uint32_t)(x & 63);
  if (rem) r += rem - __popcll(v.bits[wend] & ((1ull << rem) - 1ull));
  return r;
}

// level 0 of every part: one node, the whole part
__global__ void k_dd_init(const DdLevel* lv, int L, uint32_t R, uint64_t stride, uint64_t* cnt) {
  const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < R) cnt[(uint64_t)p * stride] = lv[(uint64_t)p * L].n;
}

// level l -> l + 1 of every part: sizes and starts of the children of every
// node.  Node (l, c) of part p sits at p * stride + 2^l - 1 + c.
__global__ void k_dd_children(const DdLevel* lv, int L, int l, uint32_t R, int wm,
                              uint64_t stride, uint64_t* cnt, uint64_t* cs) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t nn = (uint64_t)1 << l;
  if (i >= (uint64_t)R * nn) return;
  const uint64_t p = i >> l, c = i & (nn - 1);
  const DdLevel v = lv[p * L + l];
  const uint64_t at = p * stride + nn - 1 + c, nb = p * stride + 2 * nn - 1;
  const uint64_t s = cs[at], k = cnt[at];
  const uint64_t r0 = dd_rank0(v, s);
  const uint64_t z = k ? dd_rank0(v, s + k) - r0 : 0;
  if (wm) {
    // zeros of the whole level first, classes in order in both halves
    const uint64_t Z = v.dir[2 * ((v.n + 2047) >> 11)];
    cnt[nb + c] = z;
    cnt[nb + c + nn] = k - z;
    cs[nb + c] = r0;
    cs[nb + c + nn] = Z + (s - r0);
  } else {
    cnt[nb + 2 * c] = z;
    cnt[nb + 2 * c + 1] = k - z;
    cs[nb + 2 * c] = s;
    cs[nb + 2 * c + 1] = s + z;
  }
}

// node totals over the parts
__global__ void k_dd_totals(const uint64_t* cnt, uint32_t R, uint64_t stride, uint64_t* tot) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= stride) return;
  uint64_t t = 0;
  for (uint32_t p = 0; p < R; p++) t += cnt[(uint64_t)p * stride + i];
  tot[i] = t;
}

__device__ __forceinline__ int dd_level_of(uint64_t i) { return 63 - __clzll(i + 1); }

// destination of every run (in its level) and its piece count
__global__ void k_dd_dest(const uint64_t* cnt, const uint64_t* X, uint32_t R, uint64_t stride,
                          uint64_t* dst, uint64_t* npc) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= stride) return;
  const int l = dd_level_of(i);
  uint64_t d = X[i] - X[((uint64_t)1 << l) - 1];
  for (uint32_t p = 0; p < R; p++) {
    const uint64_t g = (uint64_t)p * stride + i, k = cnt[g];
    dst[g] = d;
    // pieces: the run's destination cut at multiples of DD_PIECE bits
    npc[g] = k ? ((d % DD_PIECE) + k + DD_PIECE - 1) / DD_PIECE : 0;
    d += k;
  }
}

// The copy stores the words a run covers whole and ORs the others, so the
// words a run shares (its first and last when not word-aligned) and every
// level's words from its last partial one on start at zero: one thread per
// run, and per level the words [n / 64, W).
__global__ void k_dd_zero_edges(const uint64_t* cnt, const uint64_t* dst, uint64_t nseg,
                                uint64_t stride, uint64_t* out, uint64_t W, int L, uint64_t n) {
  const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g < nseg) {
    const uint64_t k = cnt[g];
    if (k) {
      uint64_t* const ol = out + (uint64_t)dd_level_of(g % stride) * W;
      const uint64_t d = dst[g];
      if (d & 63) ol[d >> 6] = 0;
      if ((d + k) & 63) ol[(d + k - 1) >> 6] = 0;
    }
  }
  const uint64_t pw = W - (n >> 6);
  if (g < (uint64_t)L * pw) out[(g / pw) * W + (n >> 6) + g % pw] = 0;
}

// run of every piece: one warp per run writes its index over its pieces
__global__ void k_dd_map(const uint64_t* PS, uint64_t nseg, uint32_t* map) {
  const int lane = threadIdx.x & 31;
  const uint64_t g = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (g >= nseg) return;
  const uint64_t a = PS[g], b = PS[g + 1];
  for (uint64_t t = a + lane; t < b; t += 32) map[t] = (uint32_t)g;
}

// one warp per piece, the grid covering every piece: each warp's reads of
// its run's table entries are independent of every other warp's
__global__ void k_dd_copy(const DdLevel* lv, int L, uint64_t stride, const uint32_t* map,
                          const uint64_t* cnt, const uint64_t* cs, const uint64_t* dst,
                          const uint64_t* PS, uint64_t npieces, uint64_t* out,
                          uint64_t out_level_words, uint32_t* err) {
  const int lane = threadIdx.x & 31;
  const uint64_t j = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (j >= npieces) return;
  const uint64_t g = map[j];
  {
    const uint64_t p = g / stride, i = g - p * stride;
    const int l = dd_level_of(i);
    const DdLevel v = lv[p * L + l];
    // piece j - PS[g] of the run: destination bits [D, E) inside one aligned
    // block of DD_PIECE bits, source bits from S
    const uint64_t D0 = dst[g], E0 = D0 + cnt[g];
    const uint64_t blk = (D0 / DD_PIECE + (j - PS[g])) * DD_PIECE;
    const uint64_t D = max(blk, D0), E = min(blk + DD_PIECE, E0);
    const uint64_t S = cs[g] + (D - D0);
    uint64_t* const ol = out + (uint64_t)l * out_level_words;
#pragma unroll
    for (int u = 0; u < (int)(DD_PIECE / 2048); u++) {
      const uint64_t w = (blk >> 6) + 32 * u + lane;  // destination words, 32 apart
      if ((w << 6) < E && (w << 6) + 64 > D) {
        const uint64_t a = max(w << 6, D), b = min((w << 6) + 64, E);
        const uint64_t sp = S + (a - D), nb = b - a;
        const uint64_t sw = sp >> 6;
        const uint32_t sh = (uint32_t)(sp & 63);
        if (sp + nb > v.n || w >= out_level_words) {  // never for consistent sizes
          atomicOr(err, ERR_INTERNAL);
          continue;
        }
        uint64_t x = v.bits[sw] >> sh;
        if (sh && ((sp + nb - 1) >> 6) > sw) x |= v.bits[sw + 1] << (64 - sh);
        if (nb < 64) x &= (1ull << nb) - 1ull;
        const uint32_t at = (uint32_t)(a - (w << 6));
        if (nb == 64) ol[w] = x;
        else atomicOr((unsigned long long*)(ol + w), (unsigned long long)(x << at));
      }
    }
  }
}

// parts: structures of S_0 .. S_{R-1} (same kind, WM or WT, same sigma, with
// directories, streams synchronised); h: the new handle, kind/L/levels/n set
wt_status dd_merge(wt_struct* const* parts, uint32_t R, wt_struct* h) {
  cudaStream_t st = h->stream;
  const int L = (int)h->L;
  const uint64_t n = h->n;
  const int wm = h->kind == WT_KIND_WM;
  h->bpe = 1;
  h->level_len.assign(L, n);
  h->level_off.assign(L + 1, 0);
  const uint64_t W = ((n + 2047) / 2048) * 32;
  for (int l = 0; l < L; l++) h->level_off[l + 1] = h->level_off[l] + W;
  CK(dmalloc((void**)&h->d_bits, std::max<uint64_t>(W * L, 1) * 8, st));
  h->d_bits_ro = h->d_bits;
  CK(dmalloc((void**)&h->d_zeros, std::max(L, 1) * 8, st));
  // zero counts: the parts' sums
  h->zeros.assign(L, 0);
  for (uint32_t p = 0; p < R; p++)
    for (int l = 0; l < L; l++) h->zeros[l] += parts[p]->zeros[l];
  h->zeros_valid = true;
  TRY(upload(h->d_zeros, h->zeros.data(), L * 8, st));
  // the parts' levels
  std::vector<DdLevel> hl((size_t)R * L);
  for (uint32_t p = 0; p < R; p++)
    for (int l = 0; l < L; l++) {
      const wt_struct* q = parts[p];
      hl[(size_t)p * L + l] = DdLevel{q->d_bits_ro + q->level_off[l], q->d_dir + q->dir_off[l],
                                      q->level_len[l]};
    }
  const uint64_t stride = ((uint64_t)1 << L) - 1;  // nodes of levels 0 .. L-1
  const uint64_t nseg = (uint64_t)R * stride;
  Work wk{st, {}};
  DdLevel* d_lv;
  uint64_t *cnt, *cs, *dst, *npc, *tot, *X, *PS, *scr;
  TRY(wk.get(&d_lv, hl.size()));
  TRY(wk.get(&cnt, nseg));
  TRY(wk.get(&cs, nseg));
  TRY(wk.get(&dst, nseg));
  TRY(wk.get(&npc, nseg));
  TRY(wk.get(&tot, stride));
  TRY(wk.get(&X, stride + 1));
  TRY(wk.get(&PS, nseg + 1));
  TRY(wk.get(&scr, scan_scratch_pub(std::max(nseg, stride))));
  TRY(upload(d_lv, hl.data(), hl.size() * sizeof(DdLevel), st));
  // level 0: one node per part, the whole part (the part sizes ride in the
  // level table)
  CK(cudaMemsetAsync(cs, 0, nseg * 8, st));
  k_dd_init<<<(R + 255) / 256, 256, 0, st>>>(d_lv, L, R, stride, cnt);
  count_launch();
  for (int l = 0; l + 1 < L; l++) {
    const uint64_t th = (uint64_t)R << l;
    k_dd_children<<<(unsigned)((th + 255) / 256), 256, 0, st>>>(d_lv, L, l, R, wm, stride, cnt, cs);
    count_launch();
  }
  k_dd_totals<<<(unsigned)((stride + 255) / 256), 256, 0, st>>>(cnt, R, stride, tot);
  count_launch();
  wt_status s = scan_excl_u64_pub(tot, X, stride, scr, st);
  if (s == WT_OK) {
    k_dd_dest<<<(unsigned)((stride + 255) / 256), 256, 0, st>>>(cnt, X, R, stride, dst, npc);
    count_launch();
    const uint64_t nz = std::max<uint64_t>(nseg, (uint64_t)L * (W - (n >> 6)));
    if (nz) {
      k_dd_zero_edges<<<(unsigned)((nz + 255) / 256), 256, 0, st>>>(cnt, dst, nseg, stride,
                                                                    h->d_bits, W, L, n);
      count_launch();
    }
    s = scan_excl_u64_pub(npc, PS, nseg, scr, st);
  }
  uint64_t npieces = 0;
  if (s == WT_OK) {
    CK(cudaMemcpyAsync(&npieces, PS + nseg, 8, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
  }
  if (s == WT_OK && npieces) {
    uint32_t* map;
    TRY(wk.get(&map, npieces));
    k_dd_map<<<(unsigned)((nseg * 32 + 255) / 256), 256, 0, st>>>(PS, nseg, map);
    count_launch();
    k_dd_copy<<<(unsigned)((npieces * 32 + 255) / 256), 256, 0, st>>>(
        d_lv, L, stride, map, cnt, cs, dst, PS, npieces, h->d_bits, W, h->d_err);
    count_launch();
  }
  cudaError_t e = cudaGetLastError();
  if (s != WT_OK) return s;
  if (e != cudaSuccess) return WT_ERR_CUDA;
  if (h->flags & WT_FLAG_NO_DIRECTORY) return WT_OK;
  return build_directories(h);
}

}  // namespace wtk
