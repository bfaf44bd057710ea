// wm_cpu.cpp -- a multi-threaded CPU construction of the wavelet matrix, its
// rank directories and select samples: the timed CPU comparison of the
// benchmark, stronger than the single-threaded oracle.  Not part of the
// library and never called by it.
//
// Two constructions.  cpu_wm_build is levelwise (Sections 4.1-4.2): level l
// of the matrix holds bit L-1-l of T_l,
// and T_{l+1} is the stable split of T_l by that bit, zeros first.  Each level
// is built by P threads over P chunks of T_l (chunk starts on 64-element
// boundaries, so every thread writes whole words of the level): a pass that
// writes the chunk's bits and counts its zeros, the prefix sums of the counts,
// and a pass that moves every element to its place in T_{l+1}.  The rank
// directory and the select samples use the layouts of the library (2048-bit
// superblocks with 512-bit blocks; every 4096th occurrence of each bit value).
// cpu_wm_build_short follows Section 3's packed short lists and Theorem 4.1's
// parallel form: big levels every tau = 4 levels hold the symbols and are
// computed by a parallel stable counting sort on the tau-bit digit; the tau
// levels in between come from a short list of 4-bit integers packed 16 to a
// word, split four elements at a time by one table lookup (the block's level
// bits and its packed sub-lists of zeros and ones), the sub-lists of the
// threads' chunks concatenated at prefix-summed offsets.
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <thread>
#include <vector>

namespace {

template <typename F>
void parallel(int P, F f) {
  std::vector<std::thread> th;
  for (int p = 1; p < P; p++) th.emplace_back(f, p);
  f(0);
  for (auto& t : th) t.join();
}

uint64_t words_of(uint64_t nbits) { return ((nbits + 2047) / 2048) * 32; }

int nth_set(uint64_t w, int r) {  // position of the r-th (0-based) set bit
  for (int i = 0; i < 64; i++)
    if ((w >> i) & 1u) {
      if (r == 0) return i;
      r--;
    }
  return 63;
}

// Rank directories and select samples of the L levels, levels one after
// another, the superblocks of a level split among the threads.
void build_dirs(const uint64_t* bits, uint64_t n, int L, int P, uint64_t* dir, uint64_t* samp) {
  const uint64_t W = words_of(n), nsb = (n + 2047) / 2048, cap = n / 4096 + 1;
  for (int l = 0; l < L; l++) {
    const uint64_t* lb = bits + (uint64_t)l * W;
    uint64_t* ld = dir + (uint64_t)l * 2 * (nsb + 1);
    std::vector<uint64_t> sz(nsb + 1, 0);
    parallel(P, [&](int c) {
      for (uint64_t s = nsb * c / P; s < nsb * (c + 1) / P; s++) {
        uint64_t zc = 0, rel = 0;
        for (int blk = 0; blk < 4; blk++) {
          if (blk) rel |= zc << (16 * blk);
          for (int w = 0; w < 8; w++) {
            const uint64_t i0 = 2048 * s + 512 * blk + 64 * w;
            if (i0 >= n) break;
            const uint64_t nb = std::min<uint64_t>(64, n - i0);
            const uint64_t m = nb == 64 ? ~0ull : ((1ull << nb) - 1);
            zc += nb - (uint64_t)__builtin_popcountll(lb[i0 >> 6] & m);
          }
        }
        sz[s] = zc;
        ld[2 * s + 1] = rel;
      }
    });
    uint64_t acc = 0;
    for (uint64_t s = 0; s < nsb; s++) {
      ld[2 * s] = acc;
      acc += sz[s];
    }
    ld[2 * nsb] = acc;
    ld[2 * nsb + 1] = 0;
    uint64_t* s0 = samp + (uint64_t)l * 2 * cap;
    uint64_t* s1 = s0 + cap;
    parallel(P, [&](int c) {
      for (uint64_t s = nsb * c / P; s < nsb * (c + 1) / P; s++) {
        const uint64_t zb = ld[2 * s], ob = 2048 * s - zb;
        uint64_t zi = zb, oi = ob;
        for (int w = 0; w < 32; w++) {
          const uint64_t i0 = 2048 * s + 64 * w;
          if (i0 >= n) break;
          const uint64_t nb = std::min<uint64_t>(64, n - i0);
          const uint64_t m = nb == 64 ? ~0ull : ((1ull << nb) - 1);
          const uint64_t one = lb[i0 >> 6] & m, zero = ~lb[i0 >> 6] & m;
          const uint64_t co = (uint64_t)__builtin_popcountll(one), cz = nb - co;
          // occurrences 4096k inside this word
          uint64_t k = (zi + 4095) / 4096;
          if (4096 * k < zi + cz) s0[k] = i0 + nth_set(zero, (int)(4096 * k - zi));
          k = (oi + 4095) / 4096;
          if (4096 * k < oi + co) s1[k] = i0 + nth_set(one, (int)(4096 * k - oi));
          zi += cz;
          oi += co;
        }
      }
    });
  }
}

}  // namespace

extern "C" {

// S: n symbols < 2^L (uint16).  bits: L * words_of(n) words, zeroed by the
// caller; zeros: L.  dir: L * 2 * (ceil(n/2048) + 1) u64 (the library's
// records); samp: L * 2 * (n / 4096 + 1) u64 (zero samples then one samples
// per level, capacity n / 4096 + 1 each).  Returns 0.
int cpu_wm_build(const uint16_t* S, uint64_t n, int L, int P, uint64_t* bits, uint64_t* zeros,
                 uint64_t* dir, uint64_t* samp) {
  if (P < 1) P = 1;
  const uint64_t W = words_of(n);
  std::vector<uint16_t> a(S, S + n), b(n);
  // chunk c: elements [lo(c), lo(c+1)), starts rounded to 64
  auto lo = [&](int c) -> uint64_t { return std::min<uint64_t>(n, ((n * c / P) + 63) / 64 * 64); };
  std::vector<uint64_t> z(P + 1);
  for (int l = 0; l < L; l++) {
    const int sh = L - 1 - l;
    uint64_t* lb = bits + (uint64_t)l * W;
    parallel(P, [&](int c) {
      uint64_t zc = 0;
      for (uint64_t i = lo(c); i < lo(c + 1); i++) {
        const uint64_t bit = (a[i] >> sh) & 1u;
        lb[i >> 6] |= bit << (i & 63);
        zc += bit ^ 1u;
      }
      z[c] = zc;
    });
    uint64_t Z = 0;
    std::vector<uint64_t> zb(P);
    for (int c = 0; c < P; c++) {
      zb[c] = Z;
      Z += z[c];
    }
    zeros[l] = Z;
    parallel(P, [&](int c) {
      uint64_t zp = zb[c], op = Z + (lo(c) - zb[c]);
      for (uint64_t i = lo(c); i < lo(c + 1); i++) {
        if ((a[i] >> sh) & 1u) b[op++] = a[i];
        else b[zp++] = a[i];
      }
    });
    a.swap(b);
  }
  build_dirs(bits, n, L, P, dir, samp);
  return 0;
}

}  // extern "C"

namespace {

// Short-list table: for a block of four 4-bit integers x (integer i at bits
// 4i..4i+3) and a bit position t (bit 3 - t of each integer, the first level
// of the group at t = 0): the block's four level bits, the number of
// integers whose bit is 0, and the packed sub-lists of those integers and of
// the others, each in block order.
struct ShortTable {
  std::vector<uint64_t> e;  // [t][x]: bits | n0 << 4 | L0 << 8 | L1 << 24
  ShortTable() : e(4 * 65536) {
    for (int t = 0; t < 4; t++)
      for (uint32_t x = 0; x < 65536; x++) {
        uint64_t bits = 0, l0 = 0, l1 = 0;
        int n0 = 0, n1 = 0;
        for (int i = 0; i < 4; i++) {
          const uint64_t v = (x >> (4 * i)) & 15u;
          const uint64_t b = (v >> (3 - t)) & 1u;
          bits |= b << i;
          if (b) l1 |= v << (4 * n1++);
          else l0 |= v << (4 * n0++);
        }
        e[(size_t)t * 65536 + x] = bits | (uint64_t)n0 << 4 | l0 << 8 | l1 << 24;
      }
  }
};

const ShortTable& short_table() {
  static const ShortTable t;
  return t;
}

// append m 4-bit integers (packed from bit 0 of src's words) at integer
// offset o of dst; dst words shared with another thread are ORed atomically,
// dst must be zero where it is written
void put_nibbles(uint64_t* dst, uint64_t o, const uint64_t* src, uint64_t m) {
  if (!m) return;
  const uint64_t first = o >> 4, last = (o + m - 1) >> 4;
  const int sh = (int)(o & 15) * 4;
  auto orw = [&](uint64_t w, uint64_t v) {
    if (!v) return;
    if (w == first || w == last)
      __atomic_fetch_or(dst + w, v, __ATOMIC_RELAXED);
    else
      dst[w] |= v;
  };
  const uint64_t nw = (m + 15) / 16;
  for (uint64_t k = 0; k < nw; k++) {
    uint64_t v = src[k];
    if (k == nw - 1 && (m & 15)) v &= (1ull << (4 * (m & 15))) - 1;
    orw(first + k, v << sh);
    if (sh && first + k + 1 <= last) orw(first + k + 1, v >> (64 - sh));
  }
}

}  // namespace

extern "C" {

// The same outputs as cpu_wm_build, by big levels every four levels and
// short lists in between (see the head of this file).  Returns 0.
int cpu_wm_build_short(const uint16_t* S, uint64_t n, int L, int P, uint64_t* bits,
                       uint64_t* zeros, uint64_t* dir, uint64_t* samp) {
  if (P < 1) P = 1;
  constexpr int TAU = 4;
  const ShortTable& tab = short_table();
  const uint64_t W = words_of(n);
  const uint64_t nsw = (n + 15) / 16;  // short-list words
  std::vector<uint16_t> a(S, S + n), b(n);
  std::vector<uint64_t> sl(nsw + 1), sl2(nsw + 1);
  // chunk c: elements [lo(c), lo(c+1)), starts rounded to 64 (whole level
  // words and whole short-list words per thread)
  auto lo = [&](int c) -> uint64_t { return std::min<uint64_t>(n, ((n * c / P) + 63) / 64 * 64); };
  std::vector<std::vector<uint64_t>> L0(P), L1(P);
  std::vector<uint64_t> z(P), zb(P);
  for (int A = 0; A < L; A += TAU) {
    const int t = std::min(TAU, L - A);
    // the short list of this group: bits L-1-A .. L-A-t of every symbol of
    // the big level, as the top t bits of a 4-bit integer
    parallel(P, [&](int c) {
      const uint64_t i0 = lo(c), i1 = lo(c + 1);
      for (uint64_t w = i0 / 16; w < (i1 + 15) / 16; w++) {
        uint64_t v = 0;
        for (int k = 0; k < 16; k++) {
          const uint64_t i = 16 * w + k;
          if (i < i1) v |= (uint64_t)(((a[i] >> (L - A - t)) & ((1u << t) - 1)) << (4 - t)) << (4 * k);
        }
        sl[w] = v;
      }
    });
    for (int j = 0; j < t; j++) {
      const uint64_t* T = tab.e.data() + (size_t)j * 65536;
      uint64_t* lb = bits + (uint64_t)(A + j) * W;
      parallel(P, [&](int c) {
        const uint64_t i0 = lo(c), i1 = lo(c + 1);
        std::vector<uint64_t>& l0 = L0[c];
        std::vector<uint64_t>& l1 = L1[c];
        l0.resize((i1 - i0) / 16 + 2);
        l1.resize((i1 - i0) / 16 + 2);
        // sub-lists built in registers, a word written when full
        uint64_t a0 = 0, a1 = 0, w0 = 0, w1 = 0, m0 = 0;
        int f0 = 0, f1 = 0;
        auto push = [](uint64_t* d, uint64_t& acc, int& f, uint64_t& w, uint64_t v, int k) {
          if (!k) return;
          acc |= v << (4 * f);
          f += k;
          if (f >= 16) {
            d[w++] = acc;
            f -= 16;
            acc = f ? (v >> (4 * (k - f))) : 0;
          }
        };
        uint64_t lw = 0;
        for (uint64_t i = i0; i < i1; i += 4) {
          const uint64_t x = (sl[i >> 4] >> (4 * (i & 15))) & 0xffffu;
          const uint64_t e = T[x];
          const int cnt = (int)std::min<uint64_t>(4, i1 - i);
          // elements past the sequence's end are padding (zero integers, bit
          // 0): they count among the block's zeros, after the real ones
          const int z0 = (int)((e >> 4) & 7) - (4 - cnt);
          lw |= (e & 15) << (i & 63);
          if ((i & 63) == 60 || i + 4 >= i1) {
            lb[i >> 6] = lw;
            lw = 0;
          }
          push(l0.data(), a0, f0, w0, (e >> 8) & 0xffffu, z0);
          push(l1.data(), a1, f1, w1, (e >> 24) & 0xffffu, cnt - z0);
          m0 += z0;
        }
        if (f0) l0[w0] = a0;
        if (f1) l1[w1] = a1;
        z[c] = m0;
      });
      uint64_t Z = 0;
      for (int c = 0; c < P; c++) {
        zb[c] = Z;
        Z += z[c];
      }
      zeros[A + j] = Z;
      std::fill(sl2.begin(), sl2.end(), 0ull);
      parallel(P, [&](int c) {
        const uint64_t m = lo(c + 1) - lo(c);
        put_nibbles(sl2.data(), zb[c], L0[c].data(), z[c]);
        put_nibbles(sl2.data(), Z + (lo(c) - zb[c]), L1[c].data(), m - z[c]);
      });
      sl.swap(sl2);
    }
    if (A + t >= L) break;
    // the next big level: the stable sort of this one by the group's t bits
    // read backwards (the matrix's order after t more levels), by counting
    const int D = 1 << t;
    std::vector<uint64_t> cnt((size_t)P * D, 0);
    uint8_t rev[16];
    for (uint32_t d = 0; d < (1u << t); d++) {
      uint32_t r = 0;
      for (int i = 0; i < t; i++) r |= ((d >> (t - 1 - i)) & 1u) << i;
      rev[d] = (uint8_t)r;
    }
    // digit bit t-1 = level A; the sort key has level A as its lowest bit
    auto key = [&](uint16_t x) { return rev[(x >> (L - A - t)) & ((1u << t) - 1)]; };
    parallel(P, [&](int c) {
      for (uint64_t i = lo(c); i < lo(c + 1); i++) cnt[(size_t)c * D + key(a[i])]++;
    });
    uint64_t acc = 0;
    for (int d = 0; d < D; d++)
      for (int c = 0; c < P; c++) {
        const uint64_t v = cnt[(size_t)c * D + d];
        cnt[(size_t)c * D + d] = acc;
        acc += v;
      }
    parallel(P, [&](int c) {
      uint64_t* off = cnt.data() + (size_t)c * D;
      for (uint64_t i = lo(c); i < lo(c + 1); i++) b[off[key(a[i])]++] = a[i];
    });
    a.swap(b);
  }
  build_dirs(bits, n, L, P, dir, samp);
  return 0;
}

}  // extern "C"
