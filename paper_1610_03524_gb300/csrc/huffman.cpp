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
#include <functional>
#include <queue>
#include <vector>

namespace wtk {

namespace {

struct HNode {
  uint64_t w;
  uint64_t id;
  bool operator>(const HNode& o) const { return w != o.w ? w > o.w : id > o.id; }
};

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
  std::priority_queue<HNode, std::vector<HNode>, std::greater<HNode>> pq;
  for (uint32_t s : present) pq.push({hist[s], s});
  std::vector<uint64_t> parent((size_t)sigma + present.size(), 0);
  uint64_t next = sigma;
  while (pq.size() > 1) {
    const HNode a = pq.top();
    pq.pop();
    const HNode b = pq.top();
    pq.pop();
    parent[a.id] = next;
    parent[b.id] = next;
    pq.push({a.w + b.w, next});
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
  std::vector<uint32_t> order;
  for (uint32_t s = 0; s < sigma; s++) {
    code[s] = 0;
    if (len[s]) order.push_back(s);
  }
  std::stable_sort(order.begin(), order.end(),
                   [&](uint32_t a, uint32_t b) { return len[a] < len[b]; });
  uint64_t c = 0;
  for (size_t i = 0; i < order.size(); i++) {
    if (i) c = (c + 1) << (len[order[i]] - len[order[i - 1]]);
    code[order[i]] = (uint32_t)c;
  }
}

}  // namespace wtk
