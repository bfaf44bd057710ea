// k_pass.cuh -- the level-group partition kernel (one pass = t levels).
//
// One CTA processes one tile of T_a at a time (tiles taken in order from an
// atomic ticket, so every wait below is on a tile that is already running).
// For a tile it computes, in shared memory:
//   * the tile's bits of levels a..a+t-1, each in the order that level has
//     inside the tile (t stable 1-bit splits; Section 4.1: the sub-sequences
//     of the descendants are a stable integer sort on the next tau bits, and
//     Section 4.3: for the wavelet matrix the key is the reversed digit);
//   * the tile's element count of every class (node) of every level, from the
//     zero counts of the split bits (prefix sums, Section 2);
//   * the last <= 64 bits the tile contributes to each class ("tails").
// It then runs a decoupled look-back (single-pass chained scan) over the
// tiles to get, for each class, the count of elements and the last 64 bits
// of all earlier tiles.  This is the domain decomposition of Section 4.2:
// K = number of tiles, per-node offsets by prefix sums across the K
// sub-problems, words copied whole, and the "boundary" words that several
// sub-problems share merged specially -- here the earlier tiles' tail bits
// travel with the prefix, so every word inside a node is stored once, whole,
// by the tile holding its last bit, and only words that straddle a node
// boundary are merged with atomicOr (into words zeroed by the plan step).
// Finally the tile scatters its elements, narrowed to the bits still needed,
// to T_{a+t}: a stable partition on the t-bit digit (big nodes, Section 3).
#pragma once
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

template <typename E, int T, int NT, bool DIG>
struct PassSmem {
  static constexpr int TW = T / 32;
  static constexpr size_t off_buf = 0;
  static constexpr size_t off_lbits = off_buf + 2 * (size_t)T * sizeof(E);
  static constexpr size_t off_lplane = off_lbits + (size_t)TAU_MAX * TW * 4;
  static constexpr size_t off_zpw = off_lplane + (DIG ? (size_t)(TAU_MAX / 2) * TW * 4 : 0);
  static constexpr size_t off_ccnt = off_zpw + (size_t)TW * 4;
  static constexpr size_t off_cstart = off_ccnt + (size_t)NCLS * 4;
  static constexpr size_t off_owntail = off_cstart + (size_t)NCLS * 4;  // 8-aligned
  static constexpr size_t off_extail = off_owntail + (size_t)NTAIL * 8;
  static constexpr size_t off_excnt = off_extail + (size_t)NTAIL * 8;
  static constexpr size_t off_clsce = off_excnt + (size_t)NCLS * 8;
  static constexpr size_t bytes = off_clsce + (size_t)NTAIL * 8;
};

template <typename E, int T, int NT, bool DIG>
__global__ void __launch_bounds__(NT) k_pass(const PassParams P) {
  constexpr int W = NT / 32, PW = T / W, EPW = PW / 32, TW = T / 32;
  static_assert(EPW >= 1 && EPW <= 32, "iterations per warp must fit a warp");
  static_assert(T % 64 == 0 && NT >= (1 << TAU_MAX), "tile geometry");
  using SM = PassSmem<E, T, NT, DIG>;
  extern __shared__ __align__(16) unsigned char smem[];
  E* const bufA = (E*)(smem + SM::off_buf);
  E* const bufB = bufA + T;
  uint32_t* const lbits = (uint32_t*)(smem + SM::off_lbits);
  uint32_t* const lplane = (uint32_t*)(smem + SM::off_lplane);
  uint32_t* const zpw = (uint32_t*)(smem + SM::off_zpw);
  uint32_t* const ccnt = (uint32_t*)(smem + SM::off_ccnt);
  uint32_t* const cstart = (uint32_t*)(smem + SM::off_cstart);
  uint64_t* const own_tail = (uint64_t*)(smem + SM::off_owntail);
  uint64_t* const ex_tail = (uint64_t*)(smem + SM::off_extail);
  uint64_t* const ex_cnt = (uint64_t*)(smem + SM::off_excnt);
  uint64_t* const cls_ce = (uint64_t*)(smem + SM::off_clsce);
  uint64_t* const cls_cs = own_tail;  // reused once the inclusive state is published
  uint64_t* const sbase = own_tail;   // reused again by the scatter

  __shared__ uint32_t s_tile;
  __shared__ int s_stat, s_stop;
  __shared__ int wst[1 << TAU_MAX];
  __shared__ uint32_t s_dead[(1 << TAU_MAX) / 32];
  __shared__ int s_warp[W];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int t = P.t;
  const int bpe = DIG ? 2 : 1;
  const int ncl = (2 << t) - 1, ntl = (1 << t) - 1;
  const uint32_t ntiles = P.tiles ? *P.ntiles_dev : P.ntiles;

  for (;;) {
    if (tid == 0) {
      uint32_t ti = atomicAdd(P.ticket, 1u);
      if (ld_volatile_u32(P.abort_flag)) ti = 0xffffffffu;
      s_tile = ti;
    }
    __syncthreads();
    const uint32_t ti = s_tile;
    if (ti >= ntiles) break;
    uint64_t ts;
    int cnt;
    uint32_t node;
    bool first;
    if (P.tiles) {
      const TileDesc d = P.tiles[ti];
      ts = d.start;
      cnt = (int)d.count;
      node = d.node;
      first = d.first != 0;
    } else {
      ts = (uint64_t)ti * T;
      const uint64_t rem = P.n_in - ts;
      cnt = (int)(rem < (uint64_t)T ? rem : (uint64_t)T);
      node = 0;
      first = (ti == 0);
    }

    // ---- 1. load the tile -------------------------------------------------
    if (P.code_map) {
      for (int i = tid; i < cnt; i += NT)
        bufA[i] = (E)P.code_map[load_elem(P.in, P.in_w, ts + i)];
    } else if (P.in_w == 2 && sizeof(E) == 2 && cnt == T && (ts & 7) == 0) {
      const uint4* src = (const uint4*)((const uint16_t*)P.in + ts);
      uint4* dst = (uint4*)bufA;
      for (int i = tid; i < T / 8; i += NT) dst[i] = __ldcs(src + i);
    } else {
      for (int i = tid; i < cnt; i += NT) bufA[i] = (E)load_elem(P.in, P.in_w, ts + i);
    }
    if (tid == 0) {
      ccnt[0] = (uint32_t)cnt;
      cstart[0] = 0;
    }
    __syncthreads();

    // ---- 2. t stable 1-bit splits ----------------------------------------
    const uint32_t lt = lanemask_lt();
    for (int j = 0; j < t; j++) {
      const E* src = (j & 1) ? bufB : bufA;
      E* dst = (j & 1) ? bufA : bufB;
      const bool move = (j < t - 1) || (P.out != nullptr);
      const int sh = P.rbits - 1 - j;
      const bool two = DIG && (((P.a + j) & 1) == 0) && (P.a + j + 1 < P.L);
      const int wbase = warp * PW;
      uint32_t xr[EPW], br[EPW];
      uint32_t myb = 0, myb2 = 0;
#pragma unroll
      for (int e = 0; e < EPW; e++) {
        const int p = wbase + e * 32 + lane;
        const bool v = p < cnt;
        const uint32_t x = v ? (uint32_t)src[p] : 0u;
        xr[e] = x;
        const uint32_t b = __ballot_sync(FULL, v && ((x >> sh) & 1u));
        br[e] = b;
        if (lane == e) myb = b;
        if (DIG && two) {
          const uint32_t b2 = __ballot_sync(FULL, v && ((x >> (sh - 1)) & 1u));
          if (lane == e) myb2 = b2;
        }
      }
      if (lane < EPW) {
        lbits[j * TW + warp * EPW + lane] = myb;
        if (DIG && two) lplane[(j >> 1) * TW + warp * EPW + lane] = myb2;
      }
      const int vstart = wbase + lane * 32;
      const int vc = min(max(cnt - vstart, 0), 32);
      const int z = (lane < EPW) ? vc - __popc(myb) : 0;
      int zi = z;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, zi, o);
        if (lane >= o) zi += y;
      }
      if (lane == 31) s_warp[warp] = zi;
      __syncthreads();
      int wz = 0, Zt = 0;
#pragma unroll
      for (int w2 = 0; w2 < W; w2++) {
        const int v2 = s_warp[w2];
        wz += (w2 < warp) ? v2 : 0;
        Zt += v2;
      }
      const int zpre = wz + zi - z;
      if (lane < EPW) zpw[warp * EPW + lane] = zpre;
      if (move) {
#pragma unroll
        for (int e = 0; e < EPW; e++) {
          const int zb = __shfl_sync(FULL, zpre, e);
          const int p = wbase + e * 32 + lane;
          if (p < cnt) {
            const uint32_t b = br[e];
            const int r1 = __popc(b & lt);
            const int pos0 = wbase + e * 32;
            const int dest = ((b >> lane) & 1u) ? (Zt + (pos0 - zb) + r1) : (zb + (lane - r1));
            dst[dest] = (E)xr[e];
          }
        }
      }
      __syncthreads();
      // class counts of level j+1: zeros inside each class run of level j
      const int nk = 1 << j;
      for (int k = tid; k < nk; k += NT) {
        const int s = (int)cstart[cls_idx(j, k)], c = (int)ccnt[cls_idx(j, k)];
        auto zb4 = [&](int p) -> int {
          if (p >= cnt) return Zt;
          const int w = p >> 5;
          return (int)zpw[w] + __popc(~lbits[j * TW + w] & ((1u << (p & 31)) - 1u));
        };
        const int zc = zb4(s + c) - zb4(s);
        ccnt[cls_idx(j + 1, k)] = (uint32_t)zc;
        ccnt[cls_idx(j + 1, k + nk)] = (uint32_t)(c - zc);
      }
      __syncthreads();
      // class starts of level j+1 (2nk <= NT classes): block exclusive scan
      {
        const int m = 2 * nk;
        const int v = (tid < m) ? (int)ccnt[cls_idx(j + 1, tid)] : 0;
        int si = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(FULL, si, o);
          if (lane >= o) si += y;
        }
        if (lane == 31) s_warp[warp] = si;
        __syncthreads();
        int base = 0;
        for (int w2 = 0; w2 < warp; w2++) base += s_warp[w2];
        if (tid < m) cstart[cls_idx(j + 1, tid)] = (uint32_t)(base + si - v);
        __syncthreads();
      }
    }

    // ---- 3. own tails of every emitted level ------------------------------
    auto emitted = [&](int j) -> bool { return !DIG || (((P.a + j) & 1) == 0); };
    // 64 local bits of level j starting at local bit position bp
    auto get64 = [&](int j, int bp) -> uint64_t {
      if (!DIG) {
        const uint32_t lo = get32<TW>(lbits + j * TW, bp);
        const uint32_t hi = get32<TW>(lbits + j * TW, bp + 32);
        return ((uint64_t)hi << 32) | lo;
      }
      const int e = bp >> 1;
      const uint32_t b0 = get32<TW>(lbits + j * TW, e);
      if (P.a + j + 1 < P.L) {
        const uint32_t b1 = get32<TW>(lplane + (j >> 1) * TW, e);
        return (spread32(b0) << 1) | spread32(b1);
      }
      return spread32(b0);
    };
    for (int i = tid; i < ntl; i += NT) {
      int j = 31 - __clz(i + 1);
      const int k = i + 1 - (1 << j);
      uint64_t tl = 0;
      if (emitted(j)) {
        const int c = (int)ccnt[i] * bpe;
        if (c > 0) {
          const int end = ((int)cstart[i] + (int)ccnt[i]) * bpe;
          tl = get64(j, end - 64);
          if (c < 64) tl &= ~0ull << (64 - c);
        }
      }
      (void)k;
      own_tail[i] = tl;
    }
    __syncthreads();

    // ---- 4. publish the aggregate, look back, publish the inclusive state --
    uint64_t* const slot = P.ring + (uint64_t)(ti & P.ring_mask) * SLOT_U64;
    uint64_t* const agg = slot + 8;
    uint64_t* const inc = agg + SLOT_STATE;
    const uint64_t myseq = P.seq_base + ti;
    {
      uint64_t* dstate = first ? inc : agg;
      for (int i = tid; i < ncl; i += NT) dstate[i] = ccnt[i];
      for (int i = tid; i < ntl; i += NT) dstate[NCLS + i] = own_tail[i];
      for (int i = tid; i < ncl; i += NT) ex_cnt[i] = 0;
      for (int i = tid; i < ntl; i += NT) ex_tail[i] = 0;
      __threadfence();
      __syncthreads();
      if (tid == 0) st_release_u64(slot, (myseq << 2) | (first ? 2u : 1u));
    }
    if (!first) {
      // Windowed look-back: warp 0 polls the flags of the 32 nearest
      // predecessors at once; the block then folds the whole window (up to the
      // nearest inclusive state) into the exclusive state in one sweep.
      uint32_t base = ti;
      for (;;) {
        if (warp == 0) {
          const int64_t p = (int64_t)base - 1 - lane;
          const bool exists = p >= 0;
          const uint64_t* f = P.ring + (uint64_t)((uint32_t)p & P.ring_mask) * SLOT_U64;
          const uint64_t want = P.seq_base + (uint64_t)p;
          const uint32_t exist_m = __ballot_sync(FULL, exists);
          uint64_t spins = 0;
          int nwin = -1, stop = 0;
          for (;;) {
            int st = 0;
            if (exists) {
              const uint64_t v = ld_acquire_u64(f);
              if ((v >> 2) == want) st = (int)(v & 3u);
            }
            const uint32_t ready = __ballot_sync(FULL, st != 0);
            const uint32_t incl = __ballot_sync(FULL, st == 2);
            uint32_t need = exist_m;
            if (incl) {
              const int fl = __ffs(incl) - 1;
              need = fl == 31 ? FULL : ((2u << fl) - 1u);
            }
            if ((ready & need) == need) {
              nwin = __popc(need);
              stop = incl != 0;
              break;
            }
            int ab = 0;
            if (lane == 0) ab = (++spins > P.spin_limit) || ld_volatile_u32(P.abort_flag);
            if (__shfl_sync(FULL, ab, 0)) break;
            if (spins > 8) __nanosleep(64);
          }
          if (lane == 0) {
            s_stat = nwin;
            s_stop = stop;
          }
        }
        __syncthreads();
        const int nwin = s_stat, stop = s_stop;
        if (nwin < 0) {
          if (tid == 0) {
            atomicOr(P.err, ERR_TIMEOUT);
            atomicExch(P.abort_flag, 1u);
          }
          return;
        }
        for (int i = tid; i < ncl; i += NT) {
          uint64_t c = ex_cnt[i];
          uint64_t tl = i < ntl ? ex_tail[i] : 0;
          for (int l = 0; l < nwin; l++) {
            const uint64_t* ps = P.ring + (uint64_t)((base - 1 - l) & P.ring_mask) * SLOT_U64 + 8 +
                                 ((stop && l == nwin - 1) ? SLOT_STATE : 0);
            if (i < ntl) tl = tail_combine(__ldcg(ps + NCLS + i), tl, c * bpe);
            c += __ldcg(ps + i);
          }
          ex_cnt[i] = c;
          if (i < ntl) ex_tail[i] = tl;
        }
        __syncthreads();
        if (stop) break;
        base -= 32;
      }
      for (int i = tid; i < ncl; i += NT) {
        if (i < ntl) inc[NCLS + i] = tail_combine(ex_tail[i], own_tail[i], (uint64_t)ccnt[i] * bpe);
        inc[i] = ex_cnt[i] + ccnt[i];
      }
      __threadfence();
      __syncthreads();
      if (tid == 0) st_release_u64(slot, (myseq << 2) | 2u);
    }

    // ---- 5. level bitmaps: each word stored once by the tile holding its
    //         last bit of the class; words shared by two classes are ORed ---
    // class ranges of every emitted (level, class), loaded once
    for (int i = tid; i < ntl; i += NT) {
      const int j = 31 - __clz(i + 1);
      uint64_t cs = 0, ce = 0;
      bool dead = true;
      if (emitted(j) && ccnt[i]) class_range(P, j, (uint32_t)(i + 1 - (1 << j)), node, cs, ce, dead);
      cls_cs[i] = dead ? ~0ull : cs;
      cls_ce[i] = ce;
    }
    __syncthreads();
    for (int j = 0; j < t; j++) {
      if (!emitted(j)) continue;
      const int lo_ = DIG ? ((P.a + j) >> 1) : (P.a + j);
      const uint64_t nlb = P.lvl_len[lo_] * (uint64_t)bpe;
      uint64_t* const lb = P.bits + P.lvl_off[lo_];
      const int nk = 1 << j;
      // words owned by this tile in class k: [first_w, last_w]
      auto owned_range = [&](int k, uint64_t& fw, uint64_t& lw) -> bool {
        const int ci = cls_idx(j, k);
        const uint64_t cs = cls_cs[ci];
        if (cs == ~0ull) return false;
        const uint64_t G0 = (cs + ex_cnt[ci]) * bpe, G1 = G0 + (uint64_t)ccnt[ci] * bpe;
        const uint64_t CE = cls_ce[ci] * bpe;
        const uint64_t w0 = G0 >> 6, w1 = (G1 - 1) >> 6;
        const bool own0 = (w0 * 64 + 63 < G1) || (CE == G1);
        const bool own1 = (w1 * 64 + 63 == G1 - 1) || (CE == G1);
        fw = own0 ? w0 : w0 + 1;
        lw = (w1 == w0) ? (own0 ? w0 : w0) : (own1 ? w1 : w1 - 1);
        if (w1 == w0 && !own0) return false;
        return lw + 1 > fw;
      };
      int nw = 0;
      if (tid < nk) {
        uint64_t fw, lw;
        if (owned_range(tid, fw, lw)) nw = (int)(lw - fw + 1);
      }
      // exclusive scan of the word counts over the classes
      int si = nw;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, si, o);
        if (lane >= o) si += y;
      }
      if (lane == 31) s_warp[warp] = si;
      __syncthreads();
      int wbase = 0, wtot = 0;
#pragma unroll
      for (int w2 = 0; w2 < W; w2++) {
        const int v2 = s_warp[w2];
        wbase += (w2 < warp) ? v2 : 0;
        wtot += v2;
      }
      if (tid < nk) wst[tid] = wbase + si - nw;
      __syncthreads();
      for (int x = tid; x < wtot; x += NT) {
        // class of word x: last k with wst[k] <= x
        int lo = 0, hi = nk - 1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (wst[mid] <= x) lo = mid;
          else hi = mid - 1;
        }
        const int k = lo;
        const int ci = cls_idx(j, k);
        uint64_t fw, lw;
        owned_range(k, fw, lw);
        const uint64_t w = fw + (uint64_t)(x - wst[k]);
        const uint64_t cs = cls_cs[ci];
        const uint64_t G0 = (cs + ex_cnt[ci]) * bpe, G1 = G0 + (uint64_t)ccnt[ci] * bpe;
        const uint64_t CS = cs * bpe, CE = cls_ce[ci] * bpe;
        const int LS = (int)cstart[ci] * bpe;
        const uint64_t wb = w << 6;
        const uint64_t lo2 = wb > G0 ? wb : G0;
        const uint64_t hi2 = (wb + 64 < G1) ? wb + 64 : G1;
        uint64_t v = get64(j, LS + (int)(lo2 - G0));
        const int nb = (int)(hi2 - lo2);
        if (nb < 64) v &= (1ull << nb) - 1ull;
        v <<= (int)(lo2 - wb);
        if (lo2 == G0) {
          const uint64_t cl = wb > CS ? wb : CS;
          const int nc = (int)(G0 - cl);
          if (nc > 0) v |= (ex_tail[ci] >> (64 - nc)) << (int)(G0 - (uint64_t)nc - wb);
        }
        const bool mixed = (wb < CS) || (CE < wb + 64 && CE < nlb);
        if (mixed) atomicOr((unsigned long long*)(lb + w), (unsigned long long)v);
        else lb[w] = v;
      }
      __syncthreads();
    }

    // ---- 6. scatter T_{a+t}, narrowed ------------------------------------
    if (P.out) {
      const E* fin = (t & 1) ? bufB : bufA;
      __syncthreads();  // own_tail (aliased by sbase) no longer read
      if (tid < 8) s_dead[tid] = 0;
      __syncthreads();
      for (int r = tid; r < (1 << t); r += NT) {
        uint64_t cs, ce;
        bool dead;
        class_range(P, t, (uint32_t)r, node, cs, ce, dead);
        const int ci = cls_idx(t, r);
        // modular base: cs + ex - cstart may wrap; dead classes are flagged apart
        sbase[r] = cs + ex_cnt[ci] - cstart[ci];
        if (dead) atomicOr(&s_dead[r >> 5], 1u << (r & 31));
      }
      __syncthreads();
      const int nb = P.rbits - t;
      const uint32_t mask = nb >= 32 ? 0xffffffffu : ((1u << nb) - 1u);
      const uint32_t rmask = (1u << t) - 1u;
      const int rsh = 32 - P.rbits;
      for (int p = tid; p < cnt; p += NT) {
        const uint32_t x = fin[p];
        const uint32_t r = (__brev(x) >> rsh) & rmask;
        if (!((s_dead[r >> 5] >> (r & 31)) & 1u)) store_elem(P.out, P.out_w, sbase[r] + p, x & mask);
      }
    }
    __syncthreads();
  }
}

}  // namespace wtk
