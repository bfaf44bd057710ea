// k_pass.cuh -- the level-group partition kernel (one pass = t levels).
//
// One CTA processes one tile of T_a at a time (tiles taken from an atomic
// ticket; no CTA waits on another).  A whole, aligned tile arrives by one
// bulk copy (TMA) into shared memory, issued while the previous tile is still
// being processed.  For a tile it computes, in shared memory:
//   * the tile's bits of levels a..a+t-1, each in the order that level has
//     inside the tile, by t stable 1-bit splits of the tile (Section 4.1: the
//     descendants' sub-sequences are a stable integer sort on the next tau
//     bits; Section 4.3: for the wavelet matrix the key is the reversed
//     digit, i.e. the splits run from the level-a bit up).  Level j's bits
//     are the ballot words of b_j in the order after j splits;
//   * the element count of every class (node) of every level, folded from
//     the tile's digit counts.
// The tile's digit counts and those of all earlier tiles of its sequence or
// node come from prefix sums, taken before the pass, of every tile's digit
// counts: the domain decomposition of Section 4.2 with K = number of tiles
// and per-node offsets by prefix sums across the K sub-problems.  The
// tile's level bits leave as runs, one per (level, class); the runs' output
// words form one list, written by lanes in windows of 32 consecutive
// entries.  Words copied whole are stored; the "boundary" words that several
// tiles or nodes share (Section 4.2) are merged with atomicOr into the level
// buffer, which is zero before the pass (in a wavelet-matrix build each tile
// zeroes its share of the next pass's levels).  Finally the tile scatters its
// elements, narrowed to the bits still needed, to T_{a+t}: the stable
// partition on the t-bit digit (big nodes, Section 3).
#pragma once
#include <type_traits>

#include "wt_internal.cuh"

namespace wtk {

__device__ __forceinline__ int cls_idx(int j, int k) { return (1 << j) - 1 + k; }

__device__ __forceinline__ uint32_t load_elem(const void* p, int w, uint64_t i) {
  if (w == 1) return ((const uint8_t*)p)[i];
  if (w == 2) return ((const uint16_t*)p)[i];
  return ((const uint32_t*)p)[i];
}

__device__ __forceinline__ void store_elem(void* p, int w, uint64_t i, uint32_t v) {
  if (w == 1) ((uint8_t*)p)[i] = (uint8_t)v;
  else if (w == 2) ((uint16_t*)p)[i] = (uint16_t)v;
  else ((uint32_t*)p)[i] = v;
}

// Batched builds: tile ti's sequence, the last segment with tile0 <= ti.
__device__ __forceinline__ const SegDesc& seg_of(const PassParams& P0, uint32_t ti) {
  uint32_t lo = 0, hi = P0.nsegs - 1;
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (P0.segs[mid].tile0 <= ti) lo = mid;
    else hi = mid - 1;
  }
  return P0.segs[lo];
}

// Batched builds: the part of the parameters that belongs to tile ti's
// sequence into D.
__device__ __forceinline__ void fill_seg(PassParams& D, const PassParams& P0, uint32_t ti) {
  const SegDesc& d = seg_of(P0, ti);
  D.in = d.in;
  D.in_w = d.in_w;
  D.out = d.out;
  D.out_w = d.out_w;
  D.L = d.L;
  D.a = d.a;
  D.t = d.t;
  D.rbits = d.rbits;
  D.bits = d.bits;
  D.lvl_off = d.lvl_off;
  D.lvl_len = d.lvl_len;
  D.wm_cls = d.wm_cls;
  D.err = d.err;
  D.n_in = d.n;
  D.tile0 = d.tile0;
  D.sigma = d.sigma;
}

// Global class range [cs, ce) of level a+j, class k (k = the tile-local key
// whose bit i is digit bit i, i.e. the LSD order of the splits), for a tile
// inside node `node` of level a.  `dead` marks Huffman prefixes that are not
// internal nodes at that level (their elements have left the tree).
__device__ __forceinline__ void class_range(const PassParams& P, int j, uint32_t k,
                                            uint32_t node, uint64_t& cs, uint64_t& ce,
                                            bool& dead) {
  dead = false;
  if (P.shape == SHAPE_WM) {
    const uint64_t* z = P.wm_cls + ((1u << j) - 1u + (uint32_t)j);
    cs = z[k];
    ce = z[k + 1];
    return;
  }
  const int l = P.a + j;
  const uint64_t q = ((uint64_t)node << j) | rev_bits(k, j);
  if (P.shape == SHAPE_WT) {
    const int sh = P.L - l;
    cs = P.wt_C[q << sh];
    ce = P.wt_C[(q + 1) << sh];
    return;
  }
  const uint64_t off = P.hf_lvl[3 * l], first = P.hf_lvl[3 * l + 1], num = P.hf_lvl[3 * l + 2];
  if (q < first || q >= first + num) {
    dead = true;
    cs = ce = 0;
    return;
  }
  cs = P.hf_node[off + (q - first)];
  ce = P.hf_node[off + (q - first) + 1];
}

// store the low sizeof(E) bytes of v at shared-memory byte address a
template <typename E>
__device__ __forceinline__ void st_shared(uint32_t a, uint32_t v) {
  if (sizeof(E) == 2) asm volatile("st.shared.u16 [%0], %1;" ::"r"(a), "h"((unsigned short)v));
  else asm volatile("st.shared.u32 [%0], %1;" ::"r"(a), "r"(v));
}

__device__ __forceinline__ uint64_t spread32(uint32_t v) {
  uint64_t x = v;
  x = (x | (x << 16)) & 0x0000FFFF0000FFFFull;
  x = (x | (x << 8)) & 0x00FF00FF00FF00FFull;
  x = (x | (x << 4)) & 0x0F0F0F0F0F0F0F0Full;
  x = (x | (x << 2)) & 0x3333333333333333ull;
  x = (x | (x << 1)) & 0x5555555555555555ull;
  return x;
}

template <int TW>
__device__ __forceinline__ uint32_t get32(const uint32_t* pl, int e) {
  const int w = e >> 5, o = e & 31;
  const uint32_t lo = (w >= 0 && w < TW) ? pl[w] : 0u;
  const uint32_t hi = (w + 1 >= 0 && w + 1 < TW) ? pl[w + 1] : 0u;
  return o ? __funnelshift_r(lo, hi, o) : lo;
}

// the same over the ballot halves of a level's row words
template <int TW>
__device__ __forceinline__ uint32_t get32q(const uint2* pl, int e) {
  const int w = e >> 5, o = e & 31;
  const uint32_t lo = (w >= 0 && w < TW) ? pl[w].x : 0u;
  const uint32_t hi = (w + 1 >= 0 && w + 1 < TW) ? pl[w + 1].x : 0u;
  return o ? __funnelshift_r(lo, hi, o) : lo;
}

template <typename E, int T, int NT, bool DIG>
struct PassSmem {
  static constexpr int TW = T / 32;
  static constexpr size_t off_buf = 0;                                        // 2 x T elements
  static constexpr size_t off_lbits = off_buf + 2 * (size_t)T * sizeof(E);   // row words per level
  static constexpr int TWS = TW + 2;  // row words per level, two zero words after them
  static constexpr size_t off_pb1 = off_lbits + (size_t)TAU_MAX * TWS * 8;   // second digit bits
  static constexpr size_t off_ccnt = off_pb1 + (DIG ? (size_t)(TAU_MAX / 2) * TW * 4 : 0);
  static constexpr size_t off_cstart = off_ccnt + (size_t)NCLS * 4;
  static constexpr size_t off_excnt = off_cstart + (size_t)NCLS * 4;  // 8-aligned
  static constexpr size_t off_clscs = off_excnt + (size_t)NCLS * 8;
  static constexpr size_t bytes = off_clscs + (size_t)(1 << TAU_MAX) * 8;
};

// resident CTAs per SM the register budget is sized for: 5 for 16-bit
// elements (40 registers a thread at 288 threads a CTA; batched passes keep
// their per-sequence state in shared memory and spill 12 bytes at 40, which
// costs less than a fifth of the CTAs would); 4 for 32-bit elements, whose
// buffers let only 4 CTAs share an SM's shared memory (56 registers); 2 for
// the 8192-symbol tile (544 threads a CTA).  And whether a split keeps its
// elements in registers between its two phases (else it reads them from
// shared memory again).
#ifndef WT_PASS_MIN_CTAS
#define WT_PASS_MIN_CTAS 5
#endif
template <typename E, int T, bool BATCH>
struct PassCtas {
  static constexpr int value = T >= 8192 ? 2 : sizeof(E) == 4 ? 4 : WT_PASS_MIN_CTAS;
};
#ifndef WT_PASS_KEEP_X
#define WT_PASS_KEEP_X 1
#endif

template <typename E, int T, int NT, bool DIG, bool BATCH>
__global__ void __launch_bounds__(NT + 32, PassCtas<E, T, BATCH>::value) k_pass(const __grid_constant__ PassParams P0) {
  __shared__ PassParams s_P;
  const PassParams& P = BATCH ? s_P : P0;
  constexpr int W = NT / 32, PW = T / W, EPW = PW / 32, TW = T / 32, NB = NT + 32, CW = W;
  constexpr int TWS = TW + 2;
  static_assert(EPW >= 1 && EPW <= 32, "iterations per warp must fit a warp");
  static_assert(T % 64 == 0 && NT >= (1 << TAU_MAX), "tile geometry");
  using SM = PassSmem<E, T, NT, DIG>;
  extern __shared__ __align__(16) unsigned char smem[];
  E* const buf0 = (E*)(smem + SM::off_buf);
  E* const buf1 = buf0 + T;
  // per level and row: (ballot of the level's bit = the level's bits in its
  // order, ones before the row inside its warp)
  uint2* const rowq = (uint2*)(smem + SM::off_lbits);
  uint32_t* const pb1 = (uint32_t*)(smem + SM::off_pb1);      // b_j+1 plane of pair rounds
  uint32_t* const ccnt = (uint32_t*)(smem + SM::off_ccnt);
  uint32_t* const cstart = (uint32_t*)(smem + SM::off_cstart);
  uint64_t* const ex_cnt = (uint64_t*)(smem + SM::off_excnt);
  uint64_t* const cls_cs = (uint64_t*)(smem + SM::off_clscs);
  uint64_t* const sbase = cls_cs;  // reused by the scatter

  __shared__ uint32_t s_tile;
  // the buffer holding this tile's elements as loaded (0: the first of the
  // two) and whether they came by a bulk copy that completes on s_bar; the
  // same for the next tile (set during this one)
  __shared__ int s_ib, s_stg, s_nib, s_nstg, s_stall;
  __shared__ uint32_t s_phase, s_nxt;           // s_bar's open phase; the next tile
  __shared__ const unsigned char* s_nsrc;       // its elements if copied in bulk
  __shared__ int s_niw;                         // and their width
  __shared__ __align__(8) uint64_t s_bar;
  __shared__ int s_ones[W];
  __shared__ int s_scan[W + 1];
  __shared__ int wst[1 << TAU_MAX];
  __shared__ uint32_t s_dead[(1 << TAU_MAX) / 32];
  __shared__ int s_bad;
  __shared__ int s_oob;
  // the writer's flattened list of run words, in windows of 32 entries
  constexpr int WMAX = TAU_MAX * (2 * T / 64) + 2 * (1 << TAU_MAX);
  constexpr int WWIN = (WMAX + 31) / 32;
  __shared__ uint8_t s_g0[1 << TAU_MAX];
  __shared__ uint32_t s_wstart[WWIN];
  __shared__ uint8_t s_runid[WWIN * 32];
  __shared__ uint8_t s_winrun[WWIN];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int bpe = DIG ? 2 : 1;
  const uint32_t ntiles = P0.tiles ? *P0.ntiles_dev : P0.ntiles;
  if (BATCH && tid == 0) s_P = P0;
  const uint32_t lt = lanemask_lt();
  const int wbase = warp * PW;
  // the two words after each level's rows stay zero (the writer reads past
  // a level's last row without a bounds check)
  for (int i = tid; i < 2 * TAU_MAX; i += NB) rowq[(i >> 1) * TWS + TW + (i & 1)] = make_uint2(0u, 0u);

  auto bar_workers = [&]() { asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory"); };
  // block-wide exclusive scan of one int per thread
  auto block_scan = [&](int v, int& total) -> int {
    int si = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(FULL, si, o);
      if (lane >= o) si += y;
    }
    if (lane == 31) s_scan[warp] = si;
    __syncthreads();
    const int x = lane <= W ? s_scan[lane] : 0;
    const int base = __reduce_add_sync(FULL, lane < warp ? x : 0);
    total = __reduce_add_sync(FULL, x);
    __syncthreads();
    return base + si - v;
  };

  // Tile loads by the bulk-copy unit (TMA): tile ti+1's elements are copied
  // into the buffer tile ti no longer reads while tile ti is still being
  // processed, so a tile's load latency hides behind the previous tile.
  // Used for whole tiles at 16-byte aligned addresses whose elements have the
  // buffer's width (copied as they are) or are bytes in 16-bit buffers
  // (copied into the buffer's upper half, where the first split reads them
  // as bytes); other tiles are loaded by the threads.
  // tile nx's elements if they can come by one bulk copy, else nullptr
  // (and its element width into iw)
  auto stage_src = [&](uint32_t nx, int& iw) -> const unsigned char* {
    if (nx >= ntiles || P0.code_map) return nullptr;
    const void* in = P0.in;
    iw = P0.in_w;
    uint64_t s0;
    if (BATCH) {
      const SegDesc& sd = seg_of(P0, nx);
      in = sd.in;
      iw = sd.in_w;
      s0 = (uint64_t)(nx - sd.tile0) * T;
      if (s0 + T > sd.n) return nullptr;
    } else if (P0.tiles) {
      const TileDesc d = P0.tiles[nx];
      if (d.count != (uint32_t)T) return nullptr;
      s0 = d.start;
    } else {
      s0 = (uint64_t)(nx - P0.tile0) * T;
      if (s0 + T > P0.n_in) return nullptr;
    }
    if (!(iw == (int)sizeof(E) || (iw == 1 && sizeof(E) == 2))) return nullptr;
    const unsigned char* src = (const unsigned char*)in + s0 * (uint64_t)iw;
    return ((uintptr_t)src & 15) ? nullptr : src;
  };
  // copy them into buffer X (bytes narrower than E into its upper part)
  auto stage = [&](const unsigned char* src, int iw, E* X) {
    bulk_load((unsigned char*)X + (size_t)T * (sizeof(E) - iw), src, (uint32_t)(T * iw), &s_bar);
  };
  if (tid == 0) {
    s_stall = 0;
    s_nib = 0;
    s_phase = 0;
    const uint32_t nx = atomicAdd(P0.ticket, 1u);
    s_nxt = nx;
    mbar_init1(&s_bar);
    int iw;
    const unsigned char* src = stage_src(nx, iw);
    if (src) stage(src, iw, buf0);
    s_nstg = src != nullptr;
  }

  for (;;) {
    if (tid == 0) {
      const uint32_t nx = s_nxt;
      s_tile = nx;
      s_ib = s_nib;
      s_stg = s_nstg;
      if (BATCH && nx < ntiles) fill_seg(s_P, P0, nx);
    }
    __syncthreads();
    const uint32_t ti = s_tile;
    if (ti >= ntiles) break;
    // the tile's elements as loaded (k = 0) and the other buffer (k = 1),
    // both from one register: the byte offset of the first of them
    const uint32_t boff = s_ib ? (uint32_t)(T * sizeof(E)) : 0u;
    auto buf = [&](int k) -> E* {
      return (E*)((unsigned char*)buf0 + (boff ^ (k ? (uint32_t)(T * sizeof(E)) : 0u)));
    };
    // this tile's share of the zeroing of a later pass's levels (stores that
    // use the DRAM bandwidth the tile's compute leaves idle)
    if (!BATCH && P0.clear) clear_share(P0.clear, P0.clear_units, P0.clear_per, ti, tid, NB);
    const int t = P.t;
    const int ntl = (1 << t) - 1;
    uint64_t ts;
    int cnt;
    uint32_t node, seg0;  // seg0: first tile of the tile's sequence or node
    if (P.tiles) {
      const TileDesc d = P.tiles[ti];
      ts = d.start;
      cnt = (int)d.count;
      node = d.node;
      seg0 = d.seg0;
    } else {
      ts = (uint64_t)(ti - P.tile0) * T;
      const uint64_t rem = P.n_in - ts;
      cnt = (int)(rem < (uint64_t)T ? rem : (uint64_t)T);
      node = 0;
      seg0 = P.tile0;
    }
    const bool full = cnt == T;

    // ---- 1. load the tile (its digit counts were taken before the pass) --
    if (s_stg) {
      if (!mbar_wait(&s_bar, s_phase)) s_stall = 1;
    } else {
      E* const bufA = buf(0);
      if (P.code_map) {
        for (int i = tid; i < cnt; i += NB) bufA[i] = (E)P.code_map[load_elem(P.in, P.in_w, ts + i)];
      } else if (P.in_w == 2 && sizeof(E) == 2 && full &&
                 (((uintptr_t)P.in + 2 * ts) & 15) == 0) {
        const uint4* src = (const uint4*)((const uint16_t*)P.in + ts);
        uint4* dst = (uint4*)bufA;
        for (int i = tid; i < T / 8; i += NB) dst[i] = __ldcs(src + i);
      } else if (P.in_w == 1 && sizeof(E) == 2 && full && (((uintptr_t)P.in + ts) & 15) == 0) {
        const uint4* src = (const uint4*)((const uint8_t*)P.in + ts);
        for (int i = tid; i < T / 16; i += NB) {
          const uint4 q = __ldcs(src + i);
          const uint32_t w4[4] = {q.x, q.y, q.z, q.w};
          uint4* d = (uint4*)(bufA + 16 * i);
          uint32_t o[8];
#pragma unroll
          for (int k = 0; k < 4; k++) {
            o[2 * k] = __byte_perm(w4[k], 0, 0x4140);
            o[2 * k + 1] = __byte_perm(w4[k], 0, 0x4342);
          }
          d[0] = make_uint4(o[0], o[1], o[2], o[3]);
          d[1] = make_uint4(o[4], o[5], o[6], o[7]);
        }
      } else {
        for (int i = tid; i < cnt; i += NB) bufA[i] = (E)load_elem(P.in, P.in_w, ts + i);
      }
    }
    __syncthreads();
    if (s_stall) {  // uniform: a bulk copy that never completed
      if (tid == 0) atomicOr(P.err, ERR_STALL);
      return;
    }

    int cur;
    if (warp == CW) {
      // ---- 3 (control warp). class counts of every level from the tile's
      //      digit counts; counts of all earlier tiles from their prefix
      //      sums; exclusive counts of every level -------------------------
      // the CTA's next tile, taken now so that its latency hides behind
      // this tile's work, and where its elements are
      const uint32_t nx = lane == 0 ? atomicAdd(P0.ticket, 1u) : 0u;
      const int nd = 1 << t;
      // this tile's count of every digit value in the earlier tiles of its
      // sequence or node: the prefix sums of the per-tile counts (Section
      // 4.2, prefix sums across the K sub-problems), taken before the pass
      // (the tables are exclusive inside chunks of TCHUNK tiles, with the
      // chunks' exclusive prefixes and their total after the last chunk: the
      // tile's own digit counts are the difference to the next tile, or to
      // the next chunk for the last tile of a chunk)
      uint64_t* const exd = ex_cnt + cls_idx(t, 0);  // exclusive digit counts
      {
        const uint32_t ch = ti / TCHUNK;
        const uint32_t S = P0.tcs;
        const uint64_t* ca = P0.tchunk + (uint64_t)ch * S;
        const uint64_t* cb = P0.tchunk + (uint64_t)(seg0 / TCHUNK) * S;
        const uint32_t* ta = P0.tcnt + (uint64_t)ti * S;
        const uint32_t* tb = P0.tcnt + (uint64_t)seg0 * S;
        const bool last = (ti + 1) % TCHUNK == 0 || ti + 1 >= ntiles;
        uint32_t sum = 0;
        for (int r = lane; r < nd; r += 32) {
          const uint32_t a = ta[r];
          const uint32_t c = last ? (uint32_t)(ca[S + r] - ca[r]) - a : ta[S + r] - a;
          exd[r] = (ca[r] + a) - (cb[r] + tb[r]);
          ccnt[cls_idx(t, r)] = c;
          sum += c;
        }
        // a table that disagrees with the tile would misplace its bits: flag
        // it and leave the tile's outputs alone
        const bool bad = __reduce_add_sync(FULL, sum) != (uint32_t)cnt;
        if (lane == 0) {
          s_bad = bad;
          if (bad) atomicOr(P.err, ERR_INTERNAL);
        }
      }
      // class counts and tile-local class starts
      // level j classes are the digit values mod 2^j: level t holds the
      // digit counts, level j-1 class k sums classes k and k + 2^(j-1)
      __syncwarp();
      for (int j = t - 1; j >= 0; j--) {
        for (int k = lane; k < (1 << j); k += 32)
          ccnt[cls_idx(j, k)] = ccnt[cls_idx(j + 1, k)] + ccnt[cls_idx(j + 1, k + (1 << j))];
        __syncwarp();
      }
      // tile-local class starts: exclusive scan of each level's counts
      for (int j = 0; j <= t; j++) {
        uint32_t carry = 0;
        for (int k0 = 0; k0 < (1 << j); k0 += 32) {
          const int k = k0 + lane;
          const uint32_t c = k < (1 << j) ? ccnt[cls_idx(j, k)] : 0u;
          uint32_t ci = c;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, ci, o);
            if (lane >= o) ci += y;
          }
          if (k < (1 << j)) cstart[cls_idx(j, k)] = carry + ci - c;
          carry += __shfl_sync(FULL, ci, 31);
        }
      }
      __syncwarp();
      // exclusive counts of every level from the exclusive digit counts
      for (int j = t - 1; j >= 0; j--) {
        for (int k = lane; k < (1 << j); k += 32)
          ex_cnt[cls_idx(j, k)] = ex_cnt[cls_idx(j + 1, k)] + ex_cnt[cls_idx(j + 1, k + (1 << j))];
        __syncwarp();
      }
      if (lane == 0) {
        s_nxt = nx;
        int iw;
        s_nsrc = stage_src(nx, iw);
        s_niw = iw;
      }
    } else {
      // ---- 4 (worker warps). t stable 1-bit splits in shared memory -------
      // Warp w holds rows 16w..16w+15 of the tile (row = 32 consecutive
      // positions, one per lane).  Each level: one ballot per row gives the
      // level's bits in the current order (stored as they are) and, because
      // every lane sees every ballot of its warp, the ones before each row
      // are a running sum in uniform registers.  After one exchange of the
      // warps' one counts, an element at position p with k ones before it
      // goes to Z + k if its bit is 1 and to p - k otherwise.
      // a staged tile of bytes bound for a 16-bit buffer sits, as bytes, in
      // the buffer's upper half; the first split reads it there
      const bool bytes0 = sizeof(E) == 2 && s_stg && P.in_w == 1;
      auto splits = [&](auto full_c) {
        constexpr bool F = decltype(full_c)::value;
        const int nmove = P.out != nullptr ? t : t - 1;
        for (int j = 0; j < t; j++) {
          const E* src = buf(j & 1);
          E* dst = buf((j & 1) ^ 1);
          const uint32_t m = 1u << (P.rbits - 1 - j);
          const bool two = DIG && (((P.a + j) & 1) == 0) && (P.a + j + 1 < P.L);
          uint2* const Rw = rowq + j * TWS + warp * EPW;
#if WT_PASS_KEEP_X
          uint32_t xr[EPW];
#endif
          int ones = 0;
          // ballots of the level's bit over the warp's rows, reading the
          // elements through sp (bytes for a staged byte tile's first split)
          auto phase1 = [&](auto* sp) {
#pragma unroll
            for (int e = 0; e < EPW; e++) {
              const int p = wbase + e * 32 + lane;
              const uint32_t x = (F || p < cnt) ? (uint32_t)sp[p] : 0u;
#if WT_PASS_KEEP_X
              xr[e] = x;
#endif
              const uint32_t B = __ballot_sync(FULL, x & m);
              if (lane == 0) Rw[e] = make_uint2(B, (uint32_t)ones);
              ones += (int)sizeof(E) * __popc(B);
              if (DIG && two) {
                const uint32_t B2 = __ballot_sync(FULL, x & (m >> 1));
                if (lane == 0) pb1[(j >> 1) * TW + warp * EPW + e] = B2;
              }
            }
          };
          if (sizeof(E) == 2 && j == 0 && bytes0)
            phase1((const uint8_t*)src + T);
          else
            phase1(src);
          if (j < nmove) {
            if (lane == 0) s_ones[warp] = ones;
            bar_workers();
            const int v = lane < W ? s_ones[lane] : 0;
            const int T1 = __reduce_add_sync(FULL, v);
            const int ob = __reduce_add_sync(FULL, lane < warp ? v : 0);
            // shared-memory byte addresses: of this warp's first one's
            // destination, and of the lane's position minus the ones before
            // the warp
            const uint32_t ds = smem_addr(dst);
            const uint32_t zb = ds + (uint32_t)((int)sizeof(E) * cnt - T1 + ob);
            const uint32_t pl = ds + (uint32_t)((int)sizeof(E) * (wbase + lane) - ob);
#pragma unroll
            for (int e = 0; e < EPW; e++) {
              const uint2 R = Rw[e];
              const uint32_t q = R.y + (uint32_t)sizeof(E) * __popc(R.x & lt);
#if WT_PASS_KEEP_X
              const uint32_t x = xr[e];
#else
              const uint32_t x = (F || wbase + e * 32 + lane < cnt) ? (uint32_t)src[wbase + e * 32 + lane] : 0u;
#endif
              const uint32_t dest = (x & m) ? zb + q : pl + (uint32_t)(sizeof(E) * 32 * e) - q;
              if (F || wbase + e * 32 + lane < cnt) st_shared<E>(dest, x);
            }
            bar_workers();
          }
        }
      };
      if (full) splits(std::true_type{});
      else splits(std::false_type{});
    }
    fence_async_smem();  // the splits' accesses before the next bulk copy
    __syncthreads();
    // the final element order is in buf(1) after an odd number of moves
    cur = (P.out != nullptr ? t : t - 1) & 1;
    // the next tile goes to the buffer that does not hold the final order;
    // a bulk copy consumed by this tile has closed s_bar's phase
    if (tid == 0) {
      const int nib = cur ? s_ib : 1 - s_ib;
      const unsigned char* src = s_nsrc;
      s_phase ^= (uint32_t)s_stg;
      s_nib = nib;
      s_nstg = src != nullptr;
      if (src) stage(src, s_niw, nib ? buf1 : buf0);
    }

    if (s_bad) continue;  // uniform: read after the barrier above

    // ---- 5. level bitmaps: whole words stored, shared words ORed ----------
    auto emitted = [&](int j) -> bool { return !DIG || (((P.a + j) & 1) == 0); };
    // 64 local bits of level j starting at local bit position bp
    auto get64 = [&](int j, int bp) -> uint64_t {
      if (!DIG) {
        // bp >= 0 and bp < T: words bp/32 .. bp/32 + 2 exist (zero pads)
        const uint2* r = rowq + j * TWS + (bp >> 5);
        const int o = bp & 31;
        const uint32_t w0 = r[0].x, w1 = r[1].x, w2 = r[2].x;
        const uint32_t lo = __funnelshift_r(w0, w1, o), hi = __funnelshift_r(w1, w2, o);
        return ((uint64_t)hi << 32) | lo;
      }
      const int e = bp >> 1;
      const uint32_t b0 = get32q<TW>(rowq + j * TWS, e);
      if (P.a + j + 1 < P.L) {
        const uint32_t b1 = get32<TW>(pb1 + (j >> 1) * TW, e);
        return (spread32(b0) << 1) | spread32(b1);
      }
      return spread32(b0);
    };
    // words of every (level, class) of this tile, one flattened list: per
    // run its output word pointer, first bit in that word and word count
    uint64_t* const cls_wp = cls_cs;
    int nw = 0;
    if (tid < ntl) {
      const int j = 31 - __clz(tid + 1);
      uint64_t cs = 0, ce = 0;
      bool dead = true;
      if (emitted(j) && ccnt[tid]) class_range(P, j, (uint32_t)(tid + 1 - (1 << j)), node, cs, ce, dead);
      if (!dead) {
        const uint64_t G0 = (cs + ex_cnt[tid]) * bpe;
        const uint64_t G1 = G0 + (uint64_t)ccnt[tid] * bpe;
        const int lo_ = DIG ? ((P.a + j) >> 1) : (P.a + j);
        if (G1 > P.lvl_len[lo_] * (uint64_t)bpe) {
          atomicOr(P.err, ERR_INTERNAL);  // never for consistent tables
        } else {
          nw = (int)(((G1 - 1) >> 6) - (G0 >> 6) + 1);
          cls_wp[tid] = (uint64_t)(P.bits + P.lvl_off[lo_] + (G0 >> 6));
          s_g0[tid] = (uint8_t)(G0 & 63);
        }
      }
    }
    // the list in windows of 32 entries: a bit per run start, the run of
    // each start, and the run in force at each window's first entry
    if (tid < WWIN) s_wstart[tid] = 0u;
    int wtot;
    const int wex = block_scan(nw, wtot);  // its barriers order the zeroing
    if (tid < ntl) {
      wst[tid] = wex;
      if (nw > 0 && wex + nw <= WMAX) {
        atomicOr(&s_wstart[wex >> 5], 1u << (wex & 31));
        s_runid[wex] = (uint8_t)tid;
        for (int w = (wex + 31) >> 5; (w << 5) < wex + nw; w++) s_winrun[w] = (uint8_t)tid;
      }
    }
    __syncthreads();
    if (wtot > WMAX) {
      if (tid == 0) atomicOr(P.err, ERR_INTERNAL);  // never: bounded by the tile geometry
    } else {
      const uint32_t le = lt | (1u << lane);
      for (int win = warp; (win << 5) < wtot; win += NB / 32) {
        const int x = (win << 5) + lane;
        const uint32_t mb = s_wstart[win] & le;
        const int ci = mb ? (int)s_runid[(win << 5) + 31 - __clz(mb)] : (int)s_winrun[win];
        if (x < wtot) {
          const int k = x - wst[ci];  // word of the run
          const int j = 31 - __clz(ci + 1);
          uint64_t* const wp = (uint64_t*)cls_wp[ci];
          const int g0 = s_g0[ci];
          const int nbits = (int)ccnt[ci] * bpe, lb0 = (int)cstart[ci] * bpe;
          const int lo = k ? 0 : g0;           // first bit of the word that is the run's
          const int r0 = k ? 64 * k - g0 : 0;  // its index in the run
          const int nb = min(64 - lo, nbits - r0);
          uint64_t v = get64(j, lb0 + r0);
          if (nb < 64) v &= (1ull << nb) - 1ull;
          // stored when the run holds the whole word, else ORed
          if (nb == 64) wp[k] = v;
          else atomicOr((unsigned long long*)(wp + k), (unsigned long long)(v << lo));
        }
      }
    }
    __syncthreads();

    // ---- 6. scatter T_{a+t}, narrowed ------------------------------------
    if (P.out) {
      const E* fin = buf(cur);
      if (tid < 8) s_dead[tid] = 0;
      if (tid == 0) s_oob = 0;
      __syncthreads();
      // per digit value d (the t bits above the ones still needed, i.e. the
      // class key reversed): the byte address that tile-local position 0
      // would have in d's output range, so that position p goes to that
      // address + p * width (modular arithmetic: the base itself may lie
      // outside the output)
      for (int r = tid; r < (1 << t); r += NB) {
        uint64_t cs, ce;
        bool dead;
        class_range(P, t, (uint32_t)r, node, cs, ce, dead);
        const int ci = cls_idx(t, r);
        const uint32_t d = rev_bits((uint32_t)r, t);
        const uint64_t b0 = cs + ex_cnt[ci];
        sbase[d] = (uint64_t)(uintptr_t)P.out + (b0 - cstart[ci]) * (uint64_t)P.out_w;
        if (dead) atomicOr(&s_dead[d >> 5], 1u << (d & 31));
        else if (ccnt[ci] && b0 + ccnt[ci] > P.n_in) s_oob = 1;  // never for consistent tables
      }
      __syncthreads();
      const int nb = P.rbits - t;
      const uint32_t mask = nb >= 32 ? 0xffffffffu : ((1u << nb) - 1u);
      const uint32_t dmask = (1u << t) - 1u;
      // only Huffman trees have dead classes (elements leaving the tree)
      auto scatter = [&](auto out_t, auto huff_c) {
        using O = decltype(out_t);
        constexpr bool HF = decltype(huff_c)::value;
        auto one = [&](int p) {
          const uint32_t x = fin[p];
          const uint32_t d = (x >> nb) & dmask;
          if (HF && ((s_dead[d >> 5] >> (d & 31)) & 1u)) return;
          *(O*)(uintptr_t)(sbase[d] + (uint64_t)p * sizeof(O)) = (O)(x & mask);
        };
        if (full) {
          // a whole tile: T / NT elements per worker thread, unrolled
          if (tid < NT) {
#pragma unroll
            for (int k = 0; k < T / NT; k++) one(tid + k * NT);
          }
        } else {
          for (int p = tid; p < cnt; p += NB) one(p);
        }
      };
      if (s_oob) {
        if (tid == 0) atomicOr(P.err, ERR_INTERNAL);
      } else if (P.shape == SHAPE_HUFF) {
        if (P.out_w == 1) scatter(uint8_t{}, std::true_type{});
        else if (P.out_w == 2) scatter(uint16_t{}, std::true_type{});
        else scatter(uint32_t{}, std::true_type{});
      } else {
        if (P.out_w == 1) scatter(uint8_t{}, std::false_type{});
        else if (P.out_w == 2) scatter(uint16_t{}, std::false_type{});
        else scatter(uint32_t{}, std::false_type{});
      }
    }
    __syncthreads();
  }
}

}  // namespace wtk
