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

uint32_t huffman_lengths(const uint64_t* hist, uint32_t sigma, uint32_t cap, uint8_t* len) {
  std::fill(len, len + sigma, (uint8_t)0);
  std::vector<uint32_t> present;
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
  // head is exactly the heap's minimum).
  const size_t m = present.size();
  std::vector<uint32_t> leaf(m);
  {
    // leaves sorted by (weight, symbol): LSD radix sort of the packed keys
    // weight * 2^24 + symbol (11-bit digits), or a comparison sort when the
    // weights do not fit 40 bits
    uint64_t wmax = 0;
    for (uint32_t x : present) wmax = std::max(wmax, hist[x]);
    if (wmax < (1ull << 40)) {
      std::vector<uint64_t> key(m), tmp(m);
      for (size_t i = 0; i < m; i++) key[i] = (hist[present[i]] << 24) | present[i];
      int bits = 24;
      while (bits < 64 && (wmax >> (bits - 24))) bits++;
      for (int sh = 0; sh < bits; sh += 11) {
        std::vector<size_t> cnt(2049, 0);
        for (uint64_t k : key) cnt[((k >> sh) & 2047) + 1]++;
        for (int b = 0; b < 2048; b++) cnt[b + 1] += cnt[b];
        for (uint64_t k : key) tmp[cnt[(k >> sh) & 2047]++] = k;
        key.swap(tmp);
      }
      for (size_t i = 0; i < m; i++) leaf[i] = (uint32_t)(key[i] & 0xffffffu);
    } else {
      leaf = present;
      std::sort(leaf.begin(), leaf.end(), [&](uint32_t a, uint32_t b) {
        return hist[a] != hist[b] ? hist[a] < hist[b] : a < b;
      });
    }
  }
  std::vector<uint64_t> parent((size_t)sigma + m, 0);
  std::vector<uint64_t> iw(m);  // weights of internal node sigma + k
  size_t li = 0, qi = 0, nint = 0;
  auto take = [&](uint64_t& w, uint64_t& id) {
    const bool use_leaf =
        li < m && (qi >= nint || hist[leaf[li]] <= iw[qi]);  // equal weight: leaf id is smaller
    if (use_leaf) {
      w = hist[leaf[li]];
      id = leaf[li++];
    } else {
      w = iw[qi];
      id = sigma + qi++;
    }
  };
  uint64_t next = sigma;
  for (size_t k = 0; k + 1 < m; k++) {
    uint64_t wa, ida, wb, idb;
    take(wa, ida);
    take(wb, idb);
    parent[ida] = next;
    parent[idb] = next;
    iw[nint++] = wa + wb;
    next++;
  }
  // depths: internal nodes are created after their children, so walking ids
  // downwards from the root gives every parent's depth before its children
  const uint64_t root = next - 1;
  std::vector<uint32_t> depth((size_t)sigma + present.size(), 0);
  for (uint64_t v = root; v-- > sigma;) depth[v] = depth[parent[v]] + 1;
  uint32_t maxlen = 0;
  for (uint32_t s : present) {
    const uint32_t d = depth[parent[s]] + 1;
    len[s] = (uint8_t)std::min<uint32_t>(d, 255);
    maxlen = std::max(maxlen, d);
  }
  if (maxlen <= cap) return maxlen;
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
