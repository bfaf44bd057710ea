// wm_cpu.cpp -- a multi-threaded CPU construction of the wavelet matrix, its
// rank directories and select samples: the timed CPU comparison of the
// benchmark, stronger than the single-threaded oracle.  Not part of the
// library and never called by it.
//
// Levelwise (Sections 4.1-4.2): level l of the matrix holds bit L-1-l of T_l,
// and T_{l+1} is the stable split of T_l by that bit, zeros first.  Each level
// is built by P threads over P chunks of T_l (chunk starts on 64-element
// boundaries, so every thread writes whole words of the level): a pass that
// writes the chunk's bits and counts its zeros, the prefix sums of the counts,
// and a pass that moves every element to its place in T_{l+1}.  The rank
// directory and the select samples use the layouts of the library (2048-bit
// superblocks with 512-bit blocks; every 4096th occurrence of each bit value).
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

}  // namespace

extern "C" {

// S: n symbols < 2^L (uint16).  bits: L * words_of(n) words, zeroed by the
// caller; zeros: L.  dir: L * 2 * (ceil(n/2048) + 1) u64 (the library's
// records); samp: L * 2 * (n / 4096 + 1) u64 (zero samples then one samples
// per level, capacity n / 4096 + 1 each).  Returns 0.
int cpu_wm_build(const uint16_t* S, uint64_t n, int L, int P, uint64_t* bits, uint64_t* zeros,
                 uint64_t* dir, uint64_t* samp) {
  if (P < 1) P = 1;
  const uint64_t W = words_of(n), nsb = (n + 2047) / 2048, cap = n / 4096 + 1;
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
  // rank directories and select samples, levels one after another, the
  // superblocks of a level split among the threads
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
  return 0;
}

}  // extern "C"
