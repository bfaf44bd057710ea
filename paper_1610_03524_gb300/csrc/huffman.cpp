// huffman.cpp -- host-side Huffman code construction for the arbitrarily
// shaped (Huffman) wavelet tree (paper Section 4.3: the tree shape comes as
// codewords; codeword bit i is 0 when the path turns left).  Off the device
// path: O(sigma log sigma) on the histogram.
//
// Lengths: Huffman's greedy merge with the two lightest nodes taken first,
// ties broken by node id (leaf id = symbol, internal id = sigma + creation
// order).  If a length exceeds `cap`, lengths come from package-merge
// (Larmore & Hirschberg 1990) limited to `cap`, leaves ordered by
// (weight, symbol) and a leaf placed before a package of equal weight.
// Codes: canonical -- symbols ordered by (length, symbol) get consecutive
// code values, shifted left when the length grows.
#include <stdint.h>

#include <algorithm>
#include <vector>

namespace wtk {

namespace {

void limited_lengths(const std::vector<uint64_t>& w, const std::vector<uint32_t>& sym,
                     uint32_t cap, uint8_t* len) {
  const size_t m = w.size();
  // lists from depth cap (leaves only) up to depth 1
  std::vector<std::vector<uint64_t>> lw(cap + 1);
  std::vector<std::vector<char>> leaf(cap + 1);
  lw[cap] = w;
  leaf[cap].assign(m, 1);
  for (uint32_t d = cap; d > 1; d--) {
    const std::vector<uint64_t>& cur = lw[d];
    const size_t np = cur.size() / 2;
    std::vector<uint64_t>& nw = lw[d - 1];
    std::vector<char>& nl = leaf[d - 1];
    nw.reserve(m + np);
    nl.reserve(m + np);
    size_t i = 0, j = 0;
    while (i < m || j < np) {
      const uint64_t pw = j < np ? cur[2 * j] + cur[2 * j + 1] : 0;
      if (i < m && (j >= np || w[i] <= pw)) {
        nw.push_back(w[i++]);
        nl.push_back(1);
      } else {
        nw.push_back(pw);
        nl.push_back(0);
        j++;
      }
    }
  }
  for (size_t i = 0; i < m; i++) len[sym[i]] = 0;
  size_t take = 2 * m - 2;
  for (uint32_t d = 1; d <= cap && take > 0; d++) {
    size_t leaves = 0;
    for (size_t i = 0; i < take; i++) leaves += leaf[d][i] ? 1 : 0;
    for (size_t i = 0; i < leaves; i++) len[sym[i]]++;
    take = 2 * (take - leaves);
  }
}

}  // namespace

// Scratch arrays of one call.  A thread keeps them between calls for
// alphabets of up to KEEP_MAX symbols: on a 2^20 alphabet the first touch of
// freshly allocated arrays cost more than the merge itself.  Seven u32 and
// four u64 arrays of at most KEEP_MAX entries each: at most about 126 MB per
// calling thread, kept until the thread exits.  Larger alphabets allocate
// per call.
struct HuffScratch {
  std::vector<uint32_t> present, leaf, big, cnt, pl, pi, depth;
  std::vector<uint64_t> lw, iw, key, tmp;
};
constexpr uint32_t KEEP_MAX = 1u << 21;

uint32_t huffman_lengths(const uint64_t* hist, uint32_t sigma, uint32_t cap, uint8_t* len) {
  std::fill(len, len + sigma, (uint8_t)0);
  thread_local HuffScratch kept;
  HuffScratch fresh;
  HuffScratch& sc = sigma <= KEEP_MAX ? kept : fresh;
  std::vector<uint32_t>& present = sc.present;
  present.clear();
  present.reserve(sigma);
  for (uint32_t s = 0; s < sigma; s++)
    if (hist[s]) present.push_back(s);
  if (present.empty()) return 0;
  if (present.size() == 1) {
    len[present[0]] = 1;
    return 1;
  }
  // Two-queue form of the (weight, id) min-heap merge: leaves sorted by
  // (weight, symbol) in one queue, internal nodes in creation order in a
  // second one (their weights never decrease, and every internal id exceeds
  // every leaf id, so both queues stay sorted by (weight, id) and the smaller
  // head is exactly the heap's minimum).  Nodes are numbered by queue
  // position (sorted leaf rank, creation order), which keeps every array
  // below sequential in memory.
  const size_t m = present.size();
  std::vector<uint32_t>& leaf = sc.leaf;  // symbols by (weight, symbol)
  std::vector<uint64_t>& lw = sc.lw;      // their weights
  leaf.resize(m);
  lw.resize(m);
  {
    // `present` is in symbol order, so a stable sort on the weight alone
    // gives (weight, symbol): a counting sort when most weights are below
    // 2^16, else an LSD radix sort (13-bit digits) on packed
    // (weight << 24 | symbol) keys, or a comparison sort past 40-bit weights
    uint64_t wmax = 0;
    size_t nbig = 0;
    constexpr uint64_t K = 1u << 16;
    for (uint32_t x : present) {
      wmax = std::max(wmax, hist[x]);
      nbig += hist[x] >= K;
    }
    if (nbig <= m / 8) {
      // mostly small weights: one counting pass below K, the few heavier
      // leaves sorted apart and placed after them
      std::vector<uint32_t>& cnt = sc.cnt;
      std::vector<uint32_t>& big = sc.big;
      cnt.assign(K + 1, 0);
      big.clear();
      big.reserve(nbig);
      for (uint32_t x : present) {
        if (hist[x] < K) cnt[hist[x] + 1]++;
        else big.push_back(x);
      }
      for (uint64_t b = 0; b < K; b++) cnt[b + 1] += cnt[b];
      for (uint32_t x : present)
        if (hist[x] < K) {
          const uint32_t at = cnt[hist[x]]++;
          leaf[at] = x;
          lw[at] = hist[x];
        }
      std::stable_sort(big.begin(), big.end(),
                       [&](uint32_t a, uint32_t b) { return hist[a] < hist[b]; });
      const size_t s0 = m - big.size();
      for (size_t i = 0; i < big.size(); i++) {
        leaf[s0 + i] = big[i];
        lw[s0 + i] = hist[big[i]];
      }
    } else if (wmax < (1ull << 40)) {
      std::vector<uint64_t>& key = sc.key;
      std::vector<uint64_t>& tmp = sc.tmp;
      key.resize(m);
      tmp.resize(m);
      for (size_t i = 0; i < m; i++) key[i] = (hist[present[i]] << 24) | present[i];
      int wbits = 1;
      while (wbits < 40 && (wmax >> wbits)) wbits++;
      constexpr int D = 13;
      std::vector<size_t> cnt((1u << D) + 1);
      for (int sh = 24; sh < 24 + wbits; sh += D) {
        std::fill(cnt.begin(), cnt.end(), 0);
        for (uint64_t k : key) cnt[((k >> sh) & ((1u << D) - 1)) + 1]++;
        for (uint32_t b = 0; b < (1u << D); b++) cnt[b + 1] += cnt[b];
        for (uint64_t k : key) tmp[cnt[(k >> sh) & ((1u << D) - 1)]++] = k;
        key.swap(tmp);
      }
      for (size_t i = 0; i < m; i++) {
        leaf[i] = (uint32_t)(key[i] & 0xffffffu);
        lw[i] = key[i] >> 24;
      }
    } else {
      leaf.assign(present.begin(), present.end());
      std::stable_sort(leaf.begin(), leaf.end(),
                       [&](uint32_t a, uint32_t b) { return hist[a] < hist[b]; });
      for (size_t i = 0; i < m; i++) lw[i] = hist[leaf[i]];
    }
  }
  // parents: of sorted leaf i at pl[i], of internal node k at pi[k]; an
  // internal parent k is stored as k (leaves and internal nodes apart)
  std::vector<uint32_t>& pl = sc.pl;
  std::vector<uint32_t>& pi = sc.pi;
  std::vector<uint64_t>& iw = sc.iw;  // weight of internal node k
  pl.resize(m);
  pi.resize(m - 1);
  iw.resize(m - 1);
  size_t li = 0, qi = 0, nint = 0;
  // take the lighter head; equal weight: the leaf (its id is smaller)
  auto take = [&](uint64_t& w, bool& is_leaf, size_t& idx) {
    is_leaf = li < m && (qi >= nint || lw[li] <= iw[qi]);
    if (is_leaf) {
      w = lw[li];
      idx = li++;
    } else {
      w = iw[qi];
      idx = qi++;
    }
  };
  for (size_t k = 0; k + 1 < m; k++) {
    uint64_t wa, wb;
    bool la, lb;
    size_t ia, ib;
    take(wa, la, ia);
    take(wb, lb, ib);
    (la ? pl[ia] : pi[ia]) = (uint32_t)k;
    (lb ? pl[ib] : pi[ib]) = (uint32_t)k;
    iw[nint++] = wa + wb;
  }
  // depths: an internal node is created after its children, so walking the
  // creation order downwards from the root gives every parent's depth first
  std::vector<uint32_t>& depth = sc.depth;
  depth.resize(m - 1);
  depth[m - 2] = 0;  // the root
  for (size_t v = m - 2; v-- > 0;) depth[v] = depth[pi[v]] + 1;
  uint32_t maxlen = 0;
  for (size_t i = 0; i < m; i++) {
    const uint32_t d = depth[pl[i]] + 1;
    len[leaf[i]] = (uint8_t)std::min<uint32_t>(d, 255);
    maxlen = std::max(maxlen, d);
  }
  if (maxlen <= cap) return maxlen;
  if (cap < 32 && m > ((size_t)1 << cap)) {
    // no prefix code of at most cap bits has m codewords
    std::fill(len, len + sigma, (uint8_t)0);
    return 0;
  }
  std::vector<uint32_t> sym = present;
  std::sort(sym.begin(), sym.end(), [&](uint32_t a, uint32_t b) {
    return hist[a] != hist[b] ? hist[a] < hist[b] : a < b;
  });
  std::vector<uint64_t> w(sym.size());
  for (size_t i = 0; i < sym.size(); i++) w[i] = hist[sym[i]];
  limited_lengths(w, sym, cap, len);
  maxlen = 0;
  for (uint32_t s : present) maxlen = std::max<uint32_t>(maxlen, len[s]);
  return maxlen;
}

void canonical_codes(const uint8_t* len, uint32_t sigma, uint32_t* code) {
  // symbols ordered by (length, symbol): a counting sort on the length
  size_t cnt[256] = {0};
  for (uint32_t s = 0; s < sigma; s++) {
    code[s] = 0;
    if (len[s]) cnt[len[s]]++;
  }
  size_t pos[257] = {0};  // pos[l]: symbols shorter than l (l >= 1)
  for (int l = 2; l <= 256; l++) pos[l] = pos[l - 1] + cnt[l - 1];
  std::vector<uint32_t> order(pos[256]);
  for (uint32_t s = 0; s < sigma; s++)
    if (len[s]) order[pos[len[s]]++] = s;
  uint64_t c = 0;
  for (size_t i = 0; i < order.size(); i++) {
    if (i) c = (c + 1) << (len[order[i]] - len[order[i - 1]]);
    code[order[i]] = (uint32_t)c;
  }
}

}  // namespace wtk
