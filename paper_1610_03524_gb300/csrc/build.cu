// build.cu -- construction of wavelet matrices, balanced / Huffman-shaped /
// 4-ary wavelet trees on one GPU.
//
// Pipeline of one build (all on one stream, no host synchronisation except
// the Huffman code construction):
//   1. histogram + validation pass over S (Section 4.1: counting for the
//      integer sort; for the wavelet matrix one digit histogram per pass,
//      since a histogram does not depend on the order of the elements);
//   2. plan: node/class start offsets of every level by prefix sums
//      (Section 4.2), zero counts z_l (Section 4.3), tile ticket reset;
//   3. one partition pass per tau levels (k_pass.cuh), each after the
//      per-tile digit counts and their prefix sums across the tiles;
//   4. rank/select directories on every level (dirq.cu).
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <thread>
#include <vector>

#include "k_pass.cuh"
#include "wt_host.h"

namespace wtk {


#define CK(x)                                                   \
  do {                                                          \
    cudaError_t e_ = (x);                                       \
    if (e_ != cudaSuccess) {                                    \
      fprintf(stderr, "wavelet: %s -> %s\n", #x, cudaGetErrorString(e_)); \
      return e_ == cudaErrorMemoryAllocation ? WT_ERR_NO_MEMORY : WT_ERR_CUDA; \
    }                                                           \
  } while (0)

// Device memory comes from the device's stream-ordered pool.  The pool keeps
// up to POOL_KEEP bytes of freed memory reserved instead of returning it to
// the driver at every synchronisation, so repeated builds do not map and
// unmap their multi-GB buffers each time.  It reuses memory freed on another
// stream only once that free has completed (or the allocating stream already
// waits for it): it never makes one stream wait for another's work to hand
// memory over, which would serialise builds and copies queued on different
// streams; it takes more memory from the device instead.
constexpr uint64_t POOL_KEEP = 32ull << 30;

cudaError_t dmalloc(void** p, size_t bytes, cudaStream_t s) {
  static std::mutex mu;
  static bool done[64] = {false};
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64) {
    std::lock_guard<std::mutex> g(mu);
    if (!done[dev]) {
      cudaMemPool_t pool;
      if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t keep = POOL_KEEP;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        int no = 0;
        cudaMemPoolSetAttribute(pool, cudaMemPoolReuseAllowInternalDependencies, &no);
      }
      done[dev] = true;
    }
  }
  if (bytes == 0) bytes = 16;
  return cudaMallocAsync(p, bytes, s);
}
void dfree(void* p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

Prof& prof() {
  static Prof p;
  return p;
}

uint32_t num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return (uint32_t)sms;
}

static uint32_t levels_of(uint32_t sigma) {
  uint32_t L = 0;
  while (L < 32 && ((uint64_t)1 << L) < (uint64_t)sigma) L++;
  return L == 0 ? 1 : L;
}
static uint64_t level_words(uint64_t nbits) { return ((nbits + 2047) / 2048) * 32; }
static int width_for_bits(int b) { return b <= 8 ? 1 : (b <= 16 ? 2 : 4); }

// ---------------------------------------------------------------------------
// 1. histogram / validation
// ---------------------------------------------------------------------------
template <int WB, typename F>
__device__ __forceinline__ void for_each_symbol(const void* seq, uint64_t n, uint64_t gtid,
                                                uint64_t gstride, F&& f) {
  using T = typename std::conditional<WB == 1, uint8_t,
                                      typename std::conditional<WB == 2, uint16_t, uint32_t>::type>::type;
  const T* s = (const T*)seq;
  constexpr int PER = 16 / WB;
  const bool aligned = (((uintptr_t)seq) & 15) == 0;
  uint64_t nvec = aligned ? n / PER : 0;
  const uint4* v = (const uint4*)seq;
  for (uint64_t i = gtid; i < nvec; i += gstride) {
    const uint4 q = __ldcs(v + i);
    const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int k = 0; k < 4; k++) {
      if (WB == 1) {
#pragma unroll
        for (int b = 0; b < 4; b++) f((w[k] >> (8 * b)) & 0xffu);
      } else if (WB == 2) {
        f(w[k] & 0xffffu);
        f(w[k] >> 16);
      } else {
        f(w[k]);
      }
    }
  }
  for (uint64_t i = nvec * PER + gtid; i < n; i += gstride) f((uint32_t)s[i]);
}

// Digit counts of the wavelet matrix's passes: pass g covers levels
// a = g*tau .. a+t-1; its digit is the t bits below level a, its sort key the
// digit reversed (Section 4.3: the reverse of the tau bits).
// Validation and the first pass's digit counts, walked tile by tile (tiles
// of `tile` symbols, as the first partition pass sees them): each tile's
// counts of the first pass's reversed digit, and their sums, the first
// pass's histogram, from the one read of the sequence.  The later passes
// take their counts from their own tiles (k_tile_counts).
template <int WB>
__global__ void __launch_bounds__(256) k_hist_digits_tiles(const void* seq, uint64_t n,
                                                           uint32_t sigma, int L, int t0,
                                                           uint64_t* hist, uint32_t* err,
                                                           uint32_t* tcnt, uint32_t tcs,
                                                           uint32_t tile, uint4* clear,
                                                           uint64_t clear_units,
                                                           uint64_t clear_per) {
  using T = typename std::conditional<WB == 1, uint8_t,
                                      typename std::conditional<WB == 2, uint16_t, uint32_t>::type>::type;
  __shared__ uint32_t th[2][TC_STRIDE];
  const int tid = threadIdx.x;
  th[0][tid] = 0;
  th[1][tid] = 0;
  uint32_t own = 0;  // this thread's reversed digit, summed over the block's tiles
  __syncthreads();
  const uint32_t rmask = (1u << t0) - 1u;
  const int rsh = 32 - L;
  const uint64_t ntiles = (n + tile - 1) / tile;
  const T* s = (const T*)seq;
  const bool vec = (((uintptr_t)seq) & 15) == 0;
  bool bad = false;
  int buf = 0;
  auto count = [&](uint32_t x) {
    bad |= x >= sigma;
    atomicAdd(&th[buf][(__brev(x) >> rsh) & rmask], 1u);
  };
  for (uint64_t ti = blockIdx.x; ti < ntiles; ti += gridDim.x) {
    // the first pass's levels start at zero: this tile's share of them
    if (clear) clear_share(clear, clear_units, clear_per, ti, tid, blockDim.x);
    const uint64_t i0 = ti * tile;
    const uint64_t i1 = i0 + tile < n ? i0 + tile : n;
    if (vec && i1 - i0 == tile) {
      constexpr int PER = 16 / WB;
      const uint4* v = (const uint4*)(s + i0);
      for (int k = tid; k < (int)(tile / PER); k += blockDim.x) {
        const uint4 q = __ldcs(v + k);
        const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int m = 0; m < 4; m++) {
          if (WB == 1) {
#pragma unroll
            for (int b = 0; b < 4; b++) count((w[m] >> (8 * b)) & 0xffu);
          } else if (WB == 2) {
            count(w[m] & 0xffffu);
            count(w[m] >> 16);
          } else {
            count(w[m]);
          }
        }
      }
    } else {
      for (uint64_t i = i0 + tid; i < i1; i += blockDim.x) count((uint32_t)s[i]);
    }
    __syncthreads();
    // the other buffer was written out one tile ago; this one now
    const uint32_t c = th[buf][tid];
    if (tid < (int)tcs) tcnt[ti * tcs + tid] = c;
    own += c;
    th[buf][tid] = 0;
    buf ^= 1;
  }
  if (bad) atomicOr(err, ERR_SYMBOL);
  // first pass: digit value = the reverse of this thread's t0-bit key
  if (tid <= (int)rmask && own)
    atomicAdd((unsigned long long*)&hist[__brev((uint32_t)tid) >> (32 - t0)], (unsigned long long)own);
}


// Histogram of a byte sequence over sigma = NV + 1 <= 8 values, four bytes
// at a time in a 32-bit word: a byte equals v exactly when w ^ (v x
// 0x01010101) has a zero byte there, which ((t & 0x7F7F7F7F) + 0x7F7F7F7F)
// finds without carries between bytes; the count of the last value is the
// bytes seen minus the others.  No atomics per symbol.
template <int NV>
__device__ __forceinline__ void hist_bytes_swar(const void* seq, uint64_t n, uint64_t* hist,
                                                uint32_t* err) {
  constexpr uint32_t sigma = NV + 1;
  uint32_t cnt[NV > 0 ? NV : 1] = {};
  uint64_t seen = 0;
  bool bad = false;
  constexpr uint32_t ge = (0x80u - sigma) * 0x01010101u;  // + low 7 bits: bit 7 iff byte >= sigma
  auto word = [&](uint32_t w) {
    bad |= ((((w & 0x7F7F7F7Fu) + ge) | w) & 0x80808080u) != 0u;
#pragma unroll
    for (int v = 0; v < NV; v++) {
      const uint32_t t = w ^ ((uint32_t)v * 0x01010101u);
      const uint32_t y = (t & 0x7F7F7F7Fu) + 0x7F7F7F7Fu;
      cnt[v] += __popc(~(y | t) & 0x80808080u);
    }
  };
  const uint8_t* sb = (const uint8_t*)seq;
  const uint64_t gt = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t gs = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t nvec = ((((uintptr_t)seq) & 15) == 0) ? n / 16 : 0;
  const uint4* vp = (const uint4*)seq;
  for (uint64_t i = gt; i < nvec; i += gs) {
    const uint4 q = __ldcs(vp + i);
    word(q.x);
    word(q.y);
    word(q.z);
    word(q.w);
    seen += 16;
  }
  for (uint64_t i = nvec * 16 + gt; i < n; i += gs) {
    const uint32_t x = sb[i];
    bad |= x >= sigma;
#pragma unroll
    for (int v = 0; v < NV; v++) cnt[v] += x == (uint32_t)v ? 1u : 0u;
    seen++;
  }
  if (bad) atomicOr(err, ERR_SYMBOL);
  const int lane = threadIdx.x & 31;
  uint64_t rest = seen;
#pragma unroll
  for (int v = 0; v < NV; v++) rest -= cnt[v];
#pragma unroll
  for (int v = 0; v <= NV; v++) {
    uint64_t c = v < NV ? (uint64_t)cnt[v] : rest;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(FULL, c, o);
    if (lane == 0 && c) atomicAdd((unsigned long long*)&hist[v], (unsigned long long)c);
  }
}

// Full symbol histogram (balanced / Huffman / 4-ary trees).
// (large alphabets: block b adds into copy b % ncopy of the histogram, at
// (b % ncopy) * sigma, so that the frequent symbols of a skewed alphabet
// spread their atomics over several addresses; the copies are summed
// afterwards.  The copies are 32-bit (hist32) while no count can reach
// 2^32, so that 16 copies of a 2^20-symbol alphabet, 64 MB, stay in L2: as
// 64-bit copies they took 128 MB and their atomics went to DRAM)
template <int WB>
__global__ void k_hist_full(const void* seq, uint64_t n, uint32_t sigma, uint64_t* hist,
                            uint32_t* err, int use_smem, uint32_t ncopy = 1,
                            uint32_t* hist32 = nullptr) {
  extern __shared__ uint32_t shh[];
  if (use_smem) {
    for (uint32_t i = threadIdx.x; i < sigma; i += blockDim.x) shh[i] = 0;
    __syncthreads();
  }
  bool bad = false;
  const int lane = threadIdx.x & 31;
  if (WB == 1 && sigma <= 8) {
    // byte sequences over tiny alphabets (DNA-like text)
    switch (sigma) {
      case 1: hist_bytes_swar<0>(seq, n, hist, err); return;
      case 2: hist_bytes_swar<1>(seq, n, hist, err); return;
      case 3: hist_bytes_swar<2>(seq, n, hist, err); return;
      case 4: hist_bytes_swar<3>(seq, n, hist, err); return;
      case 5: hist_bytes_swar<4>(seq, n, hist, err); return;
      case 6: hist_bytes_swar<5>(seq, n, hist, err); return;
      case 7: hist_bytes_swar<6>(seq, n, hist, err); return;
      default: hist_bytes_swar<7>(seq, n, hist, err); return;
    }
  }
  for_each_symbol<WB>(seq, n, (uint64_t)blockIdx.x * blockDim.x + threadIdx.x,
                      (uint64_t)gridDim.x * blockDim.x, [&](uint32_t x) {
                        const bool ok = x < sigma;
                        bad |= !ok;
                        if (use_smem) {
                          if (ok) atomicAdd(&shh[x], 1u);
                        } else {
                          // lanes holding the same symbol add once (skewed
                          // alphabets put many lanes on the frequent ones)
                          const uint32_t act = __activemask();
                          const uint32_t peers = __match_any_sync(act, x);
                          if (ok && lane == __ffs(peers) - 1) {
                            const uint64_t at = (uint64_t)(blockIdx.x % ncopy) * sigma + x;
                            if (hist32) atomicAdd(&hist32[at], (uint32_t)__popc(peers));
                            else atomicAdd((unsigned long long*)&hist[at], (unsigned long long)__popc(peers));
                          }
                        }
                      });
  if (bad) atomicOr(err, ERR_SYMBOL);
  if (use_smem) {
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < sigma; i += blockDim.x)
      if (shh[i]) atomicAdd((unsigned long long*)&hist[i], (unsigned long long)shh[i]);
  }
}

template <typename C>
__global__ void k_hist_sum_copies(const C* copies, uint32_t sigma, uint32_t ncopy, uint64_t* hist) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < sigma;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t a = 0;
    for (uint32_t c = 0; c < ncopy; c++) a += copies[(uint64_t)c * sigma + i];
    hist[i] += a;
  }
}

#ifndef WT_HIST_COPY_MB
#define WT_HIST_COPY_MB 64
#endif
constexpr uint64_t HIST_COPY_BYTES = (uint64_t)WT_HIST_COPY_MB << 20;

static wt_status launch_hist_full(const void* seq, int w, uint64_t n, uint32_t sigma,
                                  uint64_t* hist, uint32_t* err, cudaStream_t st) {
  if (n == 0) return WT_OK;
  const int use_smem = sigma <= 12288;
  const size_t shb = use_smem ? sigma * 4 : 0;
  const uint32_t blocks = std::min<uint64_t>(num_sms() * 4, (n + 4095) / 4096 + 1);
  // global counters: up to 16 copies (32-bit while no count can reach 2^32),
  // taking at most HIST_COPY_BYTES so that they stay in L2
  uint32_t ncopy = 1;
  uint64_t* dst = hist;
  uint32_t* dst32 = nullptr;
  Work wk{st, {}};
  const bool narrow = n < (1ull << 32);
  if (!use_smem) {
    const uint64_t c32 = HIST_COPY_BYTES / (4ull * sigma);
    if (narrow && c32 >= 2) {
      ncopy = (uint32_t)std::min<uint64_t>(16, c32);
      TRY(wk.get(&dst32, (size_t)ncopy * sigma));
      CK(cudaMemsetAsync(dst32, 0, (size_t)ncopy * sigma * 4, st));
    } else if ((ncopy = (uint32_t)std::max<uint64_t>(
                    1, std::min<uint64_t>(16, HIST_COPY_BYTES / (8ull * sigma)))) > 1) {
      TRY(wk.get(&dst, (size_t)ncopy * sigma));
      CK(cudaMemsetAsync(dst, 0, (size_t)ncopy * sigma * 8, st));
    }
  }
  if (w == 1) k_hist_full<1><<<blocks, 512, shb, st>>>(seq, n, sigma, dst, err, use_smem, ncopy, dst32);
  else if (w == 2) k_hist_full<2><<<blocks, 512, shb, st>>>(seq, n, sigma, dst, err, use_smem, ncopy, dst32);
  else k_hist_full<4><<<blocks, 512, shb, st>>>(seq, n, sigma, dst, err, use_smem, ncopy, dst32);
  count_launch();
  CK(cudaGetLastError());
  const unsigned sg = (unsigned)std::min<uint64_t>((sigma + 255) / 256, (uint64_t)num_sms() * 8);
  if (dst32) {
    k_hist_sum_copies<uint32_t><<<sg, 256, 0, st>>>(dst32, sigma, ncopy, hist);
    count_launch();
    CK(cudaGetLastError());
  } else if (ncopy > 1) {
    k_hist_sum_copies<uint64_t><<<sg, 256, 0, st>>>(dst, sigma, ncopy, hist);
    count_launch();
    CK(cudaGetLastError());
  }
  return WT_OK;
}

// ---------------------------------------------------------------------------
// exclusive scan of u64 (n entries -> n+1 outputs); reduce, scan, add
// ---------------------------------------------------------------------------
constexpr int SCAN_BT = 1024, SCAN_PER = 4, SCAN_CH = SCAN_BT * SCAN_PER;

__device__ uint64_t block_scan_excl_u64(uint64_t v, uint64_t* total) {
  __shared__ uint64_t ws[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint64_t x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t y = __shfl_up_sync(FULL, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[warp] = x;
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    uint64_t s = lane < nw ? ws[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(FULL, s, o);
      if (lane >= o) s += y;
    }
    if (lane < nw) ws[lane] = s;
  }
  __syncthreads();
  const uint64_t base = warp ? ws[warp - 1] : 0;
  if (total) *total = ws[(blockDim.x >> 5) - 1];
  __syncthreads();
  return base + x - v;
}

__global__ void k_scan_reduce(const uint64_t* in, uint64_t n, uint64_t* bsum) {
  const uint64_t b0 = (uint64_t)blockIdx.x * SCAN_CH;
  uint64_t s = 0;
  for (int k = 0; k < SCAN_PER; k++) {
    const uint64_t i = b0 + (uint64_t)k * SCAN_BT + threadIdx.x;
    if (i < n) s += in[i];
  }
  uint64_t tot;
  block_scan_excl_u64(s, &tot);
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void k_scan_top(uint64_t* bsum, uint64_t nb) {
  __shared__ uint64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (uint64_t c0 = 0; c0 < nb; c0 += blockDim.x) {
    const uint64_t i = c0 + threadIdx.x;
    const uint64_t v = i < nb ? bsum[i] : 0;
    uint64_t tot;
    const uint64_t ex = block_scan_excl_u64(v, &tot);
    if (i < nb) bsum[i] = carry + ex;
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) bsum[nb] = carry;
}

__global__ void k_scan_down(const uint64_t* in, uint64_t n, const uint64_t* bsum, uint64_t* out) {
  const uint64_t b0 = (uint64_t)blockIdx.x * SCAN_CH;
  const uint64_t i0 = b0 + (uint64_t)threadIdx.x * SCAN_PER;
  uint64_t v[SCAN_PER], s = 0;
  for (int k = 0; k < SCAN_PER; k++) {
    v[k] = (i0 + k < n) ? in[i0 + k] : 0;
    s += v[k];
  }
  uint64_t ex = block_scan_excl_u64(s, nullptr) + bsum[blockIdx.x];
  for (int k = 0; k < SCAN_PER; k++) {
    if (i0 + k < n) out[i0 + k] = ex;
    ex += v[k];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = bsum[gridDim.x];
}

// out[0..n] = exclusive prefix of in[0..n); scratch >= n/4096 + 2 entries
static wt_status scan_excl_u64(const uint64_t* in, uint64_t* out, uint64_t n, uint64_t* scratch,
                               cudaStream_t st) {
  const uint64_t nb = (n + SCAN_CH - 1) / SCAN_CH;
  if (nb == 0) {
    CK(cudaMemsetAsync(out, 0, sizeof(uint64_t), st));
    return WT_OK;
  }
  k_scan_reduce<<<(unsigned)nb, SCAN_BT, 0, st>>>(in, n, scratch);
  count_launch();
  k_scan_top<<<1, SCAN_BT, 0, st>>>(scratch, nb);
  count_launch();
  k_scan_down<<<(unsigned)nb, SCAN_BT, 0, st>>>(in, n, scratch, out);
  count_launch();
  CK(cudaGetLastError());
  return WT_OK;
}
static uint64_t scan_scratch(uint64_t n) { return n / SCAN_CH + 2; }

// ---------------------------------------------------------------------------
// 2. plans
// ---------------------------------------------------------------------------
struct PassGeom {
  int a, t, rbits, in_w, out_w;
  bool wide;  // 32-bit working elements
};

// bytes per element of the widest intermediate sequence
static int max_out_w(const std::vector<PassGeom>& ps) {
  int w = 1;
  for (const PassGeom& p : ps) w = std::max(w, p.out_w);
  return w;
}

static std::vector<PassGeom> make_passes(int L, int tau, int first_w) {
  std::vector<PassGeom> ps;
  for (int a = 0; a < L; a += tau) {
    PassGeom p;
    p.a = a;
    p.t = std::min(tau, L - a);
    p.rbits = L - a;
    p.in_w = a == 0 ? first_w : width_for_bits(L - a);
    p.out_w = (a + p.t < L) ? width_for_bits(L - a - p.t) : 0;
    p.wide = p.rbits > 16;
    ps.push_back(p);
  }
  return ps;
}

// Class starts of every level of every pass of one wavelet matrix, by one
// block (classes of level a+j are the values of the low j bits of the
// reversed digit r: prefix sums over the histogram, read at digit rev(r),
// folded mod 2^j), and
// the zero count of every level (the class-0 size after its split).
// One pass (levels a .. a+t-1): counts of the t-bit digits, given by digit
// value (by_key = 0) or by reversed digit, the key of the splits (by_key = 1).
__device__ void plan_wm_pass(const uint64_t* h, int by_key, int a, int t, uint64_t* cls,
                             uint64_t* zeros) {
  __shared__ uint64_t cnt[512];
  __shared__ uint64_t st[512];
  for (int j = 0; j <= t; j++) {
    const int nk = 1 << j;
    for (int k = threadIdx.x; k < nk; k += blockDim.x) {
      uint64_t s = 0;
      for (int r = k; r < (1 << t); r += nk) s += h[by_key ? r : rev_bits((uint32_t)r, t)];
      cnt[k] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      uint64_t acc = 0;
      for (int k = 0; k < nk; k++) {
        st[k] = acc;
        acc += cnt[k];
      }
      st[nk] = acc;
    }
    __syncthreads();
    uint64_t* c = cls + (nk - 1 + j);
    for (int k = threadIdx.x; k <= nk; k += blockDim.x) c[k] = st[k];
    if (j >= 1 && threadIdx.x == 0) zeros[a + j - 1] = st[nk >> 1];
    __syncthreads();
  }
}

__device__ void plan_wm_classes(const uint64_t* hist, int L, int tau, int G, uint64_t* cls,
                                uint64_t* zeros) {
  int hoff = 0, coff = 0;
  for (int g = 0; g < G; g++) {
    const int a = g * tau, t = min(tau, L - a);
    plan_wm_pass(hist + hoff, 0, a, t, cls + coff, zeros);
    hoff += 1 << t;
    coff += (2 << t) + t + 1;
  }
}

// the plan of one later pass from the totals of its tiles' digit counts
// (indexed by reversed digit: the last row of the scanned chunk table)
__global__ void k_plan_wm_pass(const uint64_t* totals, int a, int t, uint64_t* cls,
                               uint64_t* zeros) {
  plan_wm_pass(totals, 1, a, t, cls, zeros);
}

// Batched builds, one block per sequence of the launch: the plan of its pass
// from the totals of its own tiles' digit counts, i.e. the difference of the
// scanned tables' prefixes at its last and first tile (tcnt exclusive
// within chunks of TCHUNK tiles, tchunk the chunks' exclusive prefixes with
// the total after the last chunk).
__global__ void k_plan_batch_pass(const SegDesc* segs, const uint32_t* tcnt,
                                  const uint64_t* tchunk, uint32_t tcs, uint32_t ntiles) {
  __shared__ uint64_t tot[TC_STRIDE];
  const SegDesc& d = segs[blockIdx.x];
  const uint32_t t0 = d.tile0, t1 = t0 + (uint32_t)((d.n + PASS_T - 1) / PASS_T);
  const uint64_t last = (uint64_t)((ntiles + TCHUNK - 1) / TCHUNK) * tcs;
  auto prefix = [&](uint32_t ti, uint32_t r) -> uint64_t {
    if (ti >= ntiles) return tchunk[last + r];
    return tchunk[(uint64_t)(ti / TCHUNK) * tcs + r] + tcnt[(uint64_t)ti * tcs + r];
  };
  for (uint32_t r = threadIdx.x; r < (1u << d.t); r += blockDim.x) tot[r] = prefix(t1, r) - prefix(t0, r);
  __syncthreads();
  plan_wm_pass(tot, 1, d.a, d.t, d.wm_cls, d.zeros);
}

// Wavelet-matrix plan, one block: class starts and zero counts; reset of the
// tile tickets.
__global__ void k_plan_wm(const uint64_t* hist, int L, int tau, int G, uint64_t* cls,
                          uint64_t* zeros, uint32_t* tickets) {
  plan_wm_classes(hist, L, tau, G, cls, zeros);
  for (int g = threadIdx.x; g < 32; g += blockDim.x) tickets[g] = 0;
}

// Balanced-tree helpers over C (C[v] = number of symbols < v, v in [0, 2^L]).
// Zero counts: z_l = sum over nodes q of level l of the size of the left child.
__global__ void k_wt_zeros(const uint64_t* C, int L, uint64_t* zeros) {
  // one block per level
  const int l = blockIdx.x;
  const int sh = L - l - 1;
  uint64_t s = 0;
  for (uint64_t q = threadIdx.x; q < ((uint64_t)1 << l); q += blockDim.x)
    s += C[(2 * q + 1) << sh] - C[(2 * q) << sh];
  uint64_t tot;
  block_scan_excl_u64(s, &tot);
  if (threadIdx.x == 0) zeros[l] = tot;
}

// Zero the words that hold the start of a node (not word aligned) on every
// output level; and the padding words.  digits: only even binary levels are
// output (digit level l/2), 2 bits per element.
__global__ void k_wt_zero_words(const uint64_t* C, int L, uint64_t n, uint64_t* bits,
                                const uint64_t* lvl_off, int digits) {
  const uint64_t gid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t total = ((uint64_t)1 << L);  // sum over levels l < L of 2^l = 2^L - 1
  if (gid >= total - 1) return;
  // level l holds gids [2^l - 1, 2^{l+1} - 1)
  const int l = 63 - __clzll(gid + 1);
  const uint64_t q = gid + 1 - ((uint64_t)1 << l);
  if (q == 0) return;
  if (digits && (l & 1)) return;
  const uint64_t s = C[q << (L - l)];
  const uint64_t bp = digits ? 2 * s : s;
  if ((bp & 63) && s < n) bits[lvl_off[digits ? l / 2 : l] + (bp >> 6)] = 0;
}

__global__ void k_zero_padding(uint64_t* bits, const uint64_t* lvl_off, const uint64_t* lvl_len,
                               int nlev, int bpe) {
  const int l = blockIdx.x;
  if (l >= nlev) return;
  const uint64_t used = (lvl_len[l] * bpe + 63) >> 6;
  const uint64_t W = lvl_off[l + 1] - lvl_off[l];
  for (uint64_t w = used + threadIdx.x; w < W; w += blockDim.x) bits[lvl_off[l] + w] = 0;
}

__global__ void k_reset_tickets(uint32_t* tickets) {
  for (int g = threadIdx.x; g < 32; g += blockDim.x) tickets[g] = 0;
}

// Node-aligned tiles over T_a: node p spans [bnd[p*stride], bnd[(p+1)*stride]).
__global__ void k_tiles_count(const uint64_t* bnd, uint64_t stride, uint64_t nn, uint32_t T,
                              uint64_t* tcnt) {
  const uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nn) return;
  const uint64_t sz = bnd[(p + 1) * stride] - bnd[p * stride];
  tcnt[p] = (sz + T - 1) / T;
}

// One thread per tile: tile i belongs to the node p with toff[p] <= i <
// toff[p+1] (nodes without tiles share their toff with the next node, so the
// last p with toff[p] <= i is the right one).
__global__ void k_tiles_write(const uint64_t* bnd, uint64_t stride, uint64_t nn, uint32_t T,
                              uint64_t node_base, const uint64_t* toff, TileDesc* tiles,
                              uint32_t* ntiles, uint64_t max_tiles) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t total = toff[nn];
  if (i == 0) *ntiles = (uint32_t)total;
  if (i >= total || i >= max_tiles) return;
  uint64_t lo = 0, hi = nn - 1;
  while (lo < hi) {
    const uint64_t mid = (lo + hi + 1) >> 1;
    if (toff[mid] <= i) lo = mid;
    else hi = mid - 1;
  }
  const uint64_t p = lo, k = i - toff[p];
  const uint64_t s = bnd[p * stride] + k * T, e = bnd[(p + 1) * stride];
  TileDesc d;
  d.start = s;
  d.count = (uint32_t)std::min<uint64_t>(T, e - s);
  d.node = (uint32_t)(node_base + p);
  d.first = (k == 0);
  d.seg0 = (uint32_t)toff[p];
  tiles[i] = d;
}

// ---------------------------------------------------------------------------
// 3. pass launch
// ---------------------------------------------------------------------------
#ifndef WT_PASS_NT
#define WT_PASS_NT 256
#endif
constexpr int PT = PASS_T, PNT = WT_PASS_NT;

// Digit counts of every tile of a pass (the K sub-problems' per-class counts
// of Section 4.2): one block per tile, the same tiles and digits as k_pass.
template <typename E, bool BATCH>
__global__ void __launch_bounds__(256) k_tile_counts(const __grid_constant__ PassParams P0,
                                                     uint32_t* tcnt, uint32_t tile) {
  __shared__ uint32_t h[TC_STRIDE];
  __shared__ PassParams s_P;
  const PassParams& P = BATCH ? s_P : P0;
  const uint32_t ntiles = P0.tiles ? *P0.ntiles_dev : P0.ntiles;
  const int tid = threadIdx.x;
  if (BATCH && tid == 0) s_P = P0;
  for (uint32_t ti = blockIdx.x; ti < ntiles; ti += gridDim.x) {
    if (BATCH && tid == 0) fill_seg(s_P, P0, ti);
    h[tid] = 0;
    __syncthreads();
    uint64_t ts;
    int cnt;
    if (P.tiles) {
      const TileDesc d = P.tiles[ti];
      ts = d.start;
      cnt = (int)d.count;
    } else {
      ts = (uint64_t)(ti - P.tile0) * tile;
      const uint64_t rem = P.n_in - ts;
      cnt = (int)(rem < (uint64_t)tile ? rem : (uint64_t)tile);
    }
    const uint32_t rmask = (1u << P.t) - 1u;
    const int rsh = 32 - P.rbits;
    // batched first passes also check the symbols (the single builds check
    // them in their histogram kernel)
    const uint32_t sigma = BATCH ? P.sigma : 0u;
    bool bad = false;
    auto count = [&](uint32_t x) {
      if (BATCH) bad |= sigma != 0u && x >= sigma;
      atomicAdd(&h[(__brev(x) >> rsh) & rmask], 1u);
    };
    const uintptr_t a = (uintptr_t)P.in + ts * (uint64_t)P.in_w;
    if (P.code_map) {
      for (int i = tid; i < cnt; i += 256) count(P.code_map[load_elem(P.in, P.in_w, ts + i)]);
    } else if (P.in_w == 2 && cnt == (int)tile && (a & 15) == 0) {
      const uint4* src = (const uint4*)a;
      for (int i = tid; i < (int)tile / 8; i += 256) {
        const uint4 q = __ldcs(src + i);
        const uint32_t w4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int k = 0; k < 4; k++) {
          count(w4[k] & 0xffffu);
          count(w4[k] >> 16);
        }
      }
    } else if (P.in_w == 1 && cnt == (int)tile && (a & 15) == 0) {
      const uint4* src = (const uint4*)a;
      for (int i = tid; i < (int)tile / 16; i += 256) {
        const uint4 q = __ldcs(src + i);
        const uint32_t w4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int k = 0; k < 4; k++)
#pragma unroll
          for (int b = 0; b < 4; b++) count((w4[k] >> (8 * b)) & 0xffu);
      }
    } else {
      for (int i = tid; i < cnt; i += 256) count(load_elem(P.in, P.in_w, ts + i));
    }
    if (BATCH && bad) atomicOr(P.err, ERR_SYMBOL);
    __syncthreads();
    if (tid < (int)P0.tcs) tcnt[(uint64_t)ti * P0.tcs + tid] = h[tid];
    __syncthreads();
  }
}

// Prefix sums of the tiles' counts, per digit value: exclusive inside each
// chunk of TCHUNK tiles (in place, u32), and the chunks' totals.
__global__ void __launch_bounds__(256) k_tile_scan_chunk(uint32_t* tcnt, const uint32_t* ntiles_dev,
                                                         uint32_t ntiles_host, uint64_t* tchunk) {
  const uint32_t nt = ntiles_dev ? *ntiles_dev : ntiles_host;
  const uint32_t c = blockIdx.x, r = threadIdx.x, S = blockDim.x;  // one thread per digit
  const uint64_t t0 = (uint64_t)c * TCHUNK;
  const uint64_t t1 = t0 + TCHUNK < nt ? t0 + TCHUNK : nt;
  uint32_t run = 0;
  // sixteen loads in flight before their stores (in place: the stores
  // would otherwise wait for each load in turn)
  constexpr int B = 16;
  for (uint64_t ti = t0; ti < t1; ti += B) {
    uint32_t v[B];
#pragma unroll
    for (int k = 0; k < B; k++) v[k] = ti + k < t1 ? tcnt[(ti + k) * S + r] : 0u;
#pragma unroll
    for (int k = 0; k < B; k++) {
      if (ti + k < t1) tcnt[(ti + k) * S + r] = run;
      run += v[k];
    }
  }
  tchunk[(uint64_t)c * S + r] = run;
}

// ... and the exclusive prefix of the chunks' totals (u64), with the grand
// total after the last chunk: one warp per digit value, 32 chunks per step
__global__ void __launch_bounds__(32) k_tile_scan_top(uint64_t* tchunk, uint32_t nchunk) {
  const uint32_t r = blockIdx.x, lane = threadIdx.x, S = gridDim.x;  // one warp per digit
  uint64_t carry = 0;
  for (uint32_t c0 = 0; c0 < nchunk; c0 += 32) {
    const uint32_t c = c0 + lane;
    const uint64_t v = c < nchunk ? tchunk[(uint64_t)c * S + r] : 0ull;
    uint64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(FULL, x, o);
      if ((int)lane >= o) x += y;
    }
    if (c < nchunk) tchunk[(uint64_t)c * S + r] = carry + x - v;
    carry += __shfl_sync(FULL, x, 31);
  }
  if (lane == 0) tchunk[(uint64_t)nchunk * S + r] = carry;
}

// A wavelet-matrix pass planned from its own tiles' digit counts: class
// starts of its levels into cls, their zero counts into zeros.
struct PassPlan {
  uint64_t* cls;
  uint64_t* zeros;
};

// tcnt_pre: the tiles' digit counts when already taken (else counted here);
// plan: the pass's plan, made here from the totals of those counts
template <typename E, bool DIG, bool BATCH = false, int TT = PT, int TNT = PNT>
static wt_status launch_pass_t(const PassParams& P, uint64_t max_tiles, const wt_build_opts* o,
                               cudaStream_t st, uint32_t* tcnt_pre = nullptr,
                               const PassPlan* plan = nullptr) {
  using SM = PassSmem<E, TT, TNT, DIG>;
  auto kern = k_pass<E, TT, TNT, DIG, BATCH>;
  static bool attr = false;
  static int occ = 0;
  if (!attr) {
    CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::bytes));
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, TNT + 32, SM::bytes));
    if (occ < 1) occ = 1;
    attr = true;
  }
  int per_sm = occ;
  if (o && o->ctas_per_sm) per_sm = std::min<int>(occ, (int)o->ctas_per_sm);
  uint64_t grid = (uint64_t)num_sms() * per_sm;
  if (grid > max_tiles) grid = std::max<uint64_t>(max_tiles, 1);
  // every tile's digit counts and their prefix sums across the tiles
  const uint64_t mt = std::max<uint64_t>(max_tiles, 1);
  const uint32_t nchunk = (uint32_t)((mt + TCHUNK - 1) / TCHUNK);
  PassParams Q = P;
  Q.tcs = P.tcs ? P.tcs : tc_stride(P.t);  // batched passes give the widest digit's
  Work wk{st, {}};
  uint32_t* tcnt = tcnt_pre;
  uint64_t* tchunk = nullptr;
  if (!tcnt) {
    TRY(wk.get(&tcnt, mt * Q.tcs));
    k_tile_counts<E, BATCH><<<(unsigned)std::min<uint64_t>(mt, (uint64_t)num_sms() * 16), 256, 0,
                              st>>>(Q, tcnt, (uint32_t)TT);
    count_launch();
  }
  TRY(wk.get(&tchunk, ((uint64_t)nchunk + 1) * Q.tcs));
  k_tile_scan_chunk<<<nchunk, Q.tcs, 0, st>>>(tcnt, P.tiles ? P.ntiles_dev : nullptr, P.ntiles,
                                              tchunk);
  count_launch();
  k_tile_scan_top<<<Q.tcs, 32, 0, st>>>(tchunk, nchunk);
  count_launch();
  if (plan) {
    k_plan_wm_pass<<<1, 256, 0, st>>>(tchunk + (uint64_t)nchunk * Q.tcs, P.a, P.t, plan->cls,
                                      plan->zeros);
    count_launch();
  }
  if (BATCH) {
    k_plan_batch_pass<<<P.nsegs, 256, 0, st>>>(P.segs, tcnt, tchunk, Q.tcs, (uint32_t)mt);
    count_launch();
  }
  Q.tcnt = tcnt;
  Q.tchunk = tchunk;
  Prof& pf = prof();
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (pf.on) {
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, st);
  }
  kern<<<(unsigned)grid, TNT + 32, SM::bytes, st>>>(Q);
  CK(cudaGetLastError());
  count_launch();
  if (pf.on) {
    cudaEventRecord(e1, st);
    std::lock_guard<std::mutex> g(pf.mu);
    pf.ev.push_back(e0);
    pf.ev.push_back(e1);
    pf.pass_launches++;
  }
  return WT_OK;
}

// tile: symbols per tile (PT for the trees; 2048, 4096 or 8192 for the
// wavelet matrix, the 8192-symbol tile with 512 worker threads)
static wt_status launch_pass(const PassParams& P, bool wide, bool dig, uint64_t max_tiles,
                             const wt_build_opts* o, cudaStream_t st,
                             uint32_t* tcnt_pre = nullptr, const PassPlan* plan = nullptr,
                             uint32_t tile = PT) {
  if (dig) return wide ? launch_pass_t<uint32_t, true>(P, max_tiles, o, st, tcnt_pre, plan)
                       : launch_pass_t<uint16_t, true>(P, max_tiles, o, st, tcnt_pre, plan);
  if (tile == 2048)
    return wide ? launch_pass_t<uint32_t, false, false, 2048, 256>(P, max_tiles, o, st, tcnt_pre, plan)
                : launch_pass_t<uint16_t, false, false, 2048, 256>(P, max_tiles, o, st, tcnt_pre, plan);
  if (tile == 8192)
    return wide ? launch_pass_t<uint32_t, false, false, 8192, 512>(P, max_tiles, o, st, tcnt_pre, plan)
                : launch_pass_t<uint16_t, false, false, 8192, 512>(P, max_tiles, o, st, tcnt_pre, plan);
  return wide ? launch_pass_t<uint32_t, false>(P, max_tiles, o, st, tcnt_pre, plan)
              : launch_pass_t<uint16_t, false>(P, max_tiles, o, st, tcnt_pre, plan);
}

// Batched wavelet matrices: one launch over the tiles of every sequence in
// P.segs (P.ntiles tiles in total).
wt_status launch_pass_batch(const PassParams& P, bool wide, const wt_build_opts* o,
                            cudaStream_t st) {
  return wide ? launch_pass_t<uint32_t, false, true>(P, P.ntiles, o, st)
              : launch_pass_t<uint16_t, false, true>(P, P.ntiles, o, st);
}

static int pick_tau(const wt_build_opts* o, int L, bool even, uint64_t n = 0) {
  int tau = (o && o->tau) ? (int)o->tau : (even ? 8 : tuned_tau((uint32_t)L, n));
  if (tau < 1) tau = 1;
  if (tau > TAU_MAX) tau = TAU_MAX;
  if (even && (tau & 1)) tau = tau > 1 ? tau - 1 : 2;
  (void)L;
  return tau;
}

// common workspace of a build

// zero_bits: false when the build's own kernels zero the level buffer
static wt_status alloc_outputs(wt_struct* h, uint64_t total_words, bool zero_bits = true) {
  CK(dmalloc((void**)&h->d_bits, total_words * 8, h->stream));
  h->d_bits_ro = h->d_bits;
  // the partition passes store whole words and OR the words shared by
  // several tiles or nodes, so the level buffer starts at zero
  if (zero_bits) CK(cudaMemsetAsync(h->d_bits, 0, total_words * 8, h->stream));
  CK(dmalloc((void**)&h->d_zeros, std::max<uint32_t>(h->levels, 1) * 8, h->stream));
  CK(cudaMemsetAsync(h->d_zeros, 0, std::max<uint32_t>(h->levels, 1) * 8, h->stream));
  return WT_OK;
}

static void set_uniform_levels(wt_struct* h, uint64_t elems_per_level) {
  h->level_len.assign(h->levels, elems_per_level);
  h->level_off.assign(h->levels + 1, 0);
  for (uint32_t l = 0; l < h->levels; l++)
    h->level_off[l + 1] = h->level_off[l] + level_words(elems_per_level * h->bpe);
}

static PassParams base_params(wt_struct* h, Work& wk, uint32_t* tickets,
                              const uint64_t* d_lvl_off, const uint64_t* d_lvl_len) {
  PassParams P;
  memset(&P, 0, sizeof(P));
  P.bits = h->d_bits;
  P.lvl_off = d_lvl_off;
  P.lvl_len = d_lvl_len;
  P.ticket = tickets;
  P.err = h->d_err;
  (void)wk;
  return P;
}

// Host tables reach the device without a copy engine: a host-to-device copy
// would queue behind whatever large copy the caller has in flight (the next
// input, in a pipelined loop) and stall the build.  Tables up to 32 KB go as
// kernel parameters.
constexpr size_t UPLOAD_MAX = 3968, UPLOAD_BIG = 32000;
struct UploadBlock {
  uint8_t b[UPLOAD_MAX];
};
struct UploadBigBlock {
  uint8_t b[UPLOAD_BIG];
};

__global__ void k_upload(uint8_t* dst, const __grid_constant__ UploadBlock blk, uint32_t bytes) {
  for (uint32_t i = threadIdx.x; i < bytes; i += blockDim.x) dst[i] = blk.b[i];
}

__global__ void k_upload_big(uint8_t* dst, const __grid_constant__ UploadBigBlock blk,
                             uint32_t bytes) {
  for (uint32_t i = threadIdx.x; i < bytes; i += blockDim.x) dst[i] = blk.b[i];
}

// Larger tables: a pinned, device-mapped staging buffer that the host fills
// and a kernel copies into device memory, reading it over the host link (no
// copy engine).  Buffers are kept per device and reused once the event
// recorded after their copy kernel has completed.
struct Stage {
  uint8_t* p = nullptr;
  size_t bytes = 0;
  cudaEvent_t ev = nullptr;
};
constexpr size_t STAGE_MIN = 8u << 20;

__global__ void k_gather_host(uint8_t* dst, const uint8_t* src, size_t bytes) {
  const size_t i0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  if ((((uintptr_t)dst | (uintptr_t)src) & 15) == 0) {
    const size_t nv = bytes / 16;
    for (size_t i = i0; i < nv; i += stride) ((uint4*)dst)[i] = ((const uint4*)src)[i];
    for (size_t i = nv * 16 + i0; i < bytes; i += stride) dst[i] = src[i];
  } else {
    for (size_t i = i0; i < bytes; i += stride) dst[i] = src[i];
  }
}

static wt_status upload_staged(void* d_dst, const void* h_src, size_t bytes, cudaStream_t st) {
  static std::mutex mu;
  static std::vector<Stage> stages[64];
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return WT_ERR_CUDA;
  std::lock_guard<std::mutex> g(mu);
  std::vector<Stage>& v = stages[dev];
  Stage* s = nullptr;
  for (Stage& x : v)
    if (x.bytes >= bytes && cudaEventQuery(x.ev) == cudaSuccess) {
      s = &x;
      break;
    }
  // a busy buffer answers cudaErrorNotReady: a status, not an error to keep
  if (cudaPeekAtLastError() == cudaErrorNotReady) cudaGetLastError();
  if (!s) {
    Stage n;
    n.bytes = std::max(bytes, STAGE_MIN);
    CK(cudaHostAlloc((void**)&n.p, n.bytes, cudaHostAllocMapped | cudaHostAllocPortable));
    if (cudaEventCreateWithFlags(&n.ev, cudaEventDisableTiming) != cudaSuccess) {
      cudaFreeHost(n.p);
      return WT_ERR_CUDA;
    }
    v.push_back(n);
    s = &v.back();
  }
  memcpy(s->p, h_src, bytes);
  const unsigned grid = (unsigned)std::min<size_t>((bytes / 16 + 255) / 256 + 1, 4 * (size_t)num_sms());
  k_gather_host<<<grid, 256, 0, st>>>((uint8_t*)d_dst, s->p, bytes);
  count_launch();
  CK(cudaGetLastError());
  CK(cudaEventRecord(s->ev, st));
  return WT_OK;
}

wt_status upload(void* d_dst, const void* h_src, size_t bytes, cudaStream_t st) {
  if (bytes == 0) return WT_OK;
  if (bytes > UPLOAD_BIG) return upload_staged(d_dst, h_src, bytes, st);
  if (bytes <= UPLOAD_MAX) {
    UploadBlock blk;
    memcpy(blk.b, h_src, bytes);
    k_upload<<<1, 256, 0, st>>>((uint8_t*)d_dst, blk, (uint32_t)bytes);
    count_launch();
    CK(cudaGetLastError());
    return WT_OK;
  }
  static thread_local UploadBigBlock big;
  memcpy(big.b, h_src, bytes);
  k_upload_big<<<1, 1024, 0, st>>>((uint8_t*)d_dst, big, (uint32_t)bytes);
  count_launch();
  CK(cudaGetLastError());
  return WT_OK;
}

// ---------------------------------------------------------------------------
// wavelet matrix
// ---------------------------------------------------------------------------
wt_status build_wm(const void* d_seq, uint64_t n, uint32_t sigma, int w, const wt_build_opts* o,
                   wt_struct* h) {
  cudaStream_t st = h->stream;
  const int L = (int)levels_of(sigma);
  h->kind = WT_KIND_WM;
  h->L = h->levels = (uint32_t)L;
  h->bpe = 1;
  set_uniform_levels(h, n);
  const uint64_t W = level_words(n);
  // the level buffer is zeroed by the build's kernels (the histogram kernel
  // the first pass's levels, each pass the next pass's), not by a memset
  TRY(alloc_outputs(h, W * L, n == 0));
  Work wk{st, {}};
  if (n == 0) return build_directories(h);
  // levels per pass, symbols per tile and CTAs per SM: the caller's, else
  // the autotuner's for (L, ceil(log2 n)), else 8 / 4096 / the occupancy limit
  const TuneConfig tc = tuned_config((uint32_t)L, n);
  wt_build_opts eo = o ? *o : wt_build_opts{};
  if (!eo.tau) eo.tau = (uint32_t)tc.tau;
  if (!eo.tile_symbols) eo.tile_symbols = tc.tile;
  if (!eo.ctas_per_sm) eo.ctas_per_sm = tc.ctas;
  o = &eo;
  const int tau = pick_tau(o, L, false, n);
  std::vector<PassGeom> ps = make_passes(L, tau, w);
  const int G = (int)ps.size();
  const uint32_t T = o->tile_symbols;
  uint64_t *hist, *cls, *d_off, *d_len;
  uint32_t* tickets;
  int nh = 0, ncls = 0;
  for (auto& p : ps) {
    nh += 1 << p.t;
    ncls += (2 << p.t) + p.t + 1;
  }
  TRY(wk.get(&hist, nh));
  TRY(wk.get(&cls, ncls));
  TRY(wk.get(&tickets, 32));
  TRY(wk.get(&d_off, L + 1));
  TRY(wk.get(&d_len, L));
  TRY(upload(d_off, h->level_off.data(), (L + 1) * 8, st));
  TRY(upload(d_len, h->level_len.data(), L * 8, st));
  CK(cudaMemsetAsync(hist, 0, nh * 8, st));
  // the first pass's digit histogram and per-tile counts (with validation)
  uint32_t* tcnt0;
  const uint64_t ntiles0 = (n + T - 1) / T;
  TRY(wk.get(&tcnt0, (size_t)ntiles0 * tc_stride(ps[0].t)));
  {
    const uint32_t blocks = (uint32_t)std::min<uint64_t>((uint64_t)num_sms() * 8, ntiles0);
    const int t0 = ps[0].t;
    // the first pass's levels: W * t0 words, a share per tile
    uint4* const cl0 = (uint4*)h->d_bits;
    const uint64_t cu0 = W * (uint64_t)t0 / 2, cp0 = (cu0 + ntiles0 - 1) / ntiles0;
    if (w == 1)
      k_hist_digits_tiles<1><<<blocks, 256, 0, st>>>(d_seq, n, sigma, L, t0, hist, h->d_err, tcnt0,
                                                     tc_stride(t0), T, cl0, cu0, cp0);
    else if (w == 2)
      k_hist_digits_tiles<2><<<blocks, 256, 0, st>>>(d_seq, n, sigma, L, t0, hist, h->d_err, tcnt0,
                                                     tc_stride(t0), T, cl0, cu0, cp0);
    else
      k_hist_digits_tiles<4><<<blocks, 256, 0, st>>>(d_seq, n, sigma, L, t0, hist, h->d_err, tcnt0,
                                                     tc_stride(t0), T, cl0, cu0, cp0);
    count_launch();
    CK(cudaGetLastError());
  }
  // pass 0 planned from the histogram; the later passes from their own
  // tiles' digit counts, just before they run
  k_plan_wm<<<1, 1024, 0, st>>>(hist, L, tau, 1, cls, h->d_zeros, tickets);
  count_launch();
  CK(cudaGetLastError());
  // intermediate sequences
  void* seqbuf[2] = {nullptr, nullptr};
  for (int g = 0; g + 1 < G; g++) {
    if (!seqbuf[g & 1]) {
      uint8_t* b;
      TRY(wk.get(&b, (size_t)n * max_out_w(ps)));
      seqbuf[g & 1] = b;
    }
  }
  const void* in = d_seq;
  int coff = 0;
  const uint64_t ntiles = (n + T - 1) / T;
  for (int g = 0; g < G; g++) {
    const PassGeom& pg = ps[g];
    PassParams P = base_params(h, wk, tickets + g, d_off, d_len);
    P.in = in;
    P.in_w = pg.in_w;
    P.out = (g + 1 < G) ? seqbuf[g & 1] : nullptr;
    P.out_w = pg.out_w;
    P.L = L;
    P.a = pg.a;
    P.t = pg.t;
    P.rbits = pg.rbits;
    P.shape = SHAPE_WM;
    P.wm_cls = cls + coff;
    P.ntiles = (uint32_t)ntiles;
    P.n_in = n;
    if (g + 1 < G) {
      P.clear = (uint4*)(h->d_bits + W * (uint64_t)ps[g + 1].a);
      P.clear_units = W * (uint64_t)ps[g + 1].t / 2;
      P.clear_per = (P.clear_units + ntiles - 1) / ntiles;
    }
    const PassPlan plan{cls + coff, h->d_zeros};
    TRY(launch_pass(P, pg.wide, false, ntiles, o, st, g == 0 ? tcnt0 : nullptr,
                    g == 0 ? nullptr : &plan, T));
    coff += (2 << pg.t) + pg.t + 1;
    in = P.out;
  }
  if (o && (o->flags & WT_FLAG_NO_DIRECTORY)) return WT_OK;
  return build_directories(h);
}

// ---------------------------------------------------------------------------
// balanced wavelet tree and its 4-ary variant
// ---------------------------------------------------------------------------
wt_status build_wt(const void* d_seq, uint64_t n, uint32_t sigma, int w, const wt_build_opts* o,
                   wt_struct* h, bool multiary) {
  cudaStream_t st = h->stream;
  const int L = (int)levels_of(sigma);
  if (L > 24) return WT_ERR_UNSUPPORTED;
  h->kind = multiary ? WT_KIND_MULTI : WT_KIND_WT;
  h->L = (uint32_t)L;
  h->levels = multiary ? (uint32_t)((L + 1) / 2) : (uint32_t)L;
  h->bpe = multiary ? 2 : 1;
  set_uniform_levels(h, n);
  TRY(alloc_outputs(h, h->level_off.back()));
  Work wk{st, {}};
  if (n == 0) return build_directories(h);
  const int tau = pick_tau(o, L, multiary);
  std::vector<PassGeom> ps = make_passes(L, tau, w);
  const int G = (int)ps.size();
  const uint32_t T = PT;
  const uint64_t V = (uint64_t)1 << L;
  uint64_t *hist, *C, *scr, *d_off, *d_len, *tcnt, *toff;
  uint32_t *tickets, *d_ntiles;
  TileDesc* tiles;
  uint64_t max_nodes = (uint64_t)1 << ps.back().a;
  const uint64_t max_tiles = (n + T - 1) / T + max_nodes + 1;
  TRY(wk.get(&hist, V));
  TRY(wk.get(&C, V + 1));
  TRY(wk.get(&scr, scan_scratch(std::max(V, max_nodes))));
  TRY(wk.get(&tickets, 32));
  TRY(wk.get(&d_off, h->levels + 1));
  TRY(wk.get(&d_len, h->levels));
  TRY(wk.get(&tcnt, max_nodes));
  TRY(wk.get(&toff, max_nodes + 1));
  TRY(wk.get(&tiles, max_tiles));
  TRY(wk.get(&d_ntiles, 1));
  TRY(upload(d_off, h->level_off.data(), (h->levels + 1) * 8, st));
  TRY(upload(d_len, h->level_len.data(), h->levels * 8, st));
  CK(cudaMemsetAsync(hist, 0, V * 8, st));
  TRY(launch_hist_full(d_seq, w, n, sigma, hist, h->d_err, st));
  TRY(scan_excl_u64(hist, C, V, scr, st));
  if (!multiary) {
    k_wt_zeros<<<L, 1024, 0, st>>>(C, L, h->d_zeros);
    count_launch();
    CK(cudaGetLastError());
  }
  k_reset_tickets<<<1, 32, 0, st>>>(tickets);
  count_launch();
  CK(cudaGetLastError());
  void* seqbuf[2] = {nullptr, nullptr};
  for (int g = 0; g + 1 < G; g++) {
    if (!seqbuf[g & 1]) {
      uint8_t* b;
      TRY(wk.get(&b, (size_t)n * max_out_w(ps)));
      seqbuf[g & 1] = b;
    }
  }
  const void* in = d_seq;
  for (int g = 0; g < G; g++) {
    const PassGeom& pg = ps[g];
    const uint64_t nn = (uint64_t)1 << pg.a;
    const uint64_t stride = (uint64_t)1 << (L - pg.a);
    k_tiles_count<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(C, stride, nn, T, tcnt);
    count_launch();
    TRY(scan_excl_u64(tcnt, toff, nn, scr, st));
    {
      const uint64_t mt = (n + T - 1) / T + nn;
      k_tiles_write<<<(unsigned)((mt + 255) / 256), 256, 0, st>>>(C, stride, nn, T, 0, toff, tiles,
                                                                 d_ntiles, mt);
      count_launch();
    }
    CK(cudaGetLastError());
    PassParams P = base_params(h, wk, tickets + g, d_off, d_len);
    P.in = in;
    P.in_w = pg.in_w;
    P.out = (g + 1 < G) ? seqbuf[g & 1] : nullptr;
    P.out_w = pg.out_w;
    P.L = L;
    P.a = pg.a;
    P.t = pg.t;
    P.rbits = pg.rbits;
    P.shape = SHAPE_WT;
    P.digits = multiary ? 1 : 0;
    P.wt_C = C;
    P.tiles = tiles;
    P.ntiles_dev = d_ntiles;
    P.n_in = n;
    const uint64_t mt = (n + T - 1) / T + nn;
    TRY(launch_pass(P, pg.wide, multiary, mt, o, st));
    in = P.out;
  }
  if (o && (o->flags & WT_FLAG_NO_DIRECTORY)) return WT_OK;
  return build_directories(h);
}

// ---------------------------------------------------------------------------
// Huffman-shaped wavelet tree
// ---------------------------------------------------------------------------
__global__ void k_clear_words(uint64_t* bits, const uint64_t* idx, uint64_t m) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) bits[idx[i]] = 0;
}

uint32_t huffman_lengths(const uint64_t* hist, uint32_t sigma, uint32_t cap, uint8_t* len);
void canonical_codes(const uint8_t* len, uint32_t sigma, uint32_t* code);

wt_status build_huff(const void* d_seq, uint64_t n, uint32_t sigma, int w, const uint8_t* h_len,
                     const wt_build_opts* o, wt_struct* h) {
  cudaStream_t st = h->stream;
  if (sigma > (1u << 24)) return WT_ERR_UNSUPPORTED;
  h->kind = WT_KIND_HUFF;
  h->bpe = 1;
  Work wk{st, {}};
  uint64_t* hist;
  TRY(wk.get(&hist, sigma));
  CK(cudaMemsetAsync(hist, 0, (size_t)sigma * 8, st));
  TRY(launch_hist_full(d_seq, w, n, sigma, hist, h->d_err, st));
  std::vector<uint64_t> hh(sigma);
  uint32_t err = 0;
  CK(cudaMemcpyAsync(hh.data(), hist, (size_t)sigma * 8, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&err, h->d_err, 4, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (err & ERR_SYMBOL) return WT_ERR_SYMBOL_GE_SIGMA;
  h->code_len.assign(sigma, 0);
  h->code.assign(sigma, 0);
  uint32_t maxlen = 0;
  if (h_len) {
    // caller lengths: every present symbol needs a code, Kraft sum <= 1
    double kraft = 0;
    uint32_t present = 0;
    for (uint32_t s = 0; s < sigma; s++) {
      h->code_len[s] = h_len[s];
      if (h_len[s] > 32) return WT_ERR_INVALID_ARG;
      if (hh[s] && !h_len[s]) return WT_ERR_INVALID_ARG;
      if (h_len[s]) {
        kraft += std::ldexp(1.0, -(int)h_len[s]);
        maxlen = std::max<uint32_t>(maxlen, h_len[s]);
        present++;
      }
    }
    if (kraft > 1.0 + 1e-12) return WT_ERR_INVALID_ARG;
    (void)present;
  } else {
    maxlen = huffman_lengths(hh.data(), sigma, 32, h->code_len.data());
  }
  h->max_code_len = maxlen;
  const int Lm = (int)maxlen;
  h->L = h->levels = (uint32_t)Lm;
  // The sweeps below run on up to 16 host threads, each over a contiguous
  // chunk of symbols (or of `order`), with per-thread partial results
  // combined in a fixed order, so the result does not depend on the thread
  // count.
  const uint32_t hw = std::max(1u, std::thread::hardware_concurrency());
  auto par = [&](uint64_t items, auto&& f) {
    const int nt = (int)std::max<uint64_t>(1, std::min<uint64_t>({16, hw, items / 65536 + 1}));
    std::vector<std::thread> th;
    for (int t = 1; t < nt; t++) th.emplace_back(f, t, nt);
    f(0, nt);
    for (auto& x : th) x.join();
    return nt;
  };
  auto chunk = [](uint64_t items, int t, int nt, uint64_t& b, uint64_t& e) {
    b = items * (uint64_t)t / (uint64_t)nt;
    e = items * (uint64_t)(t + 1) / (uint64_t)nt;
  };
  constexpr int MAXT = 16;
  // symbols in canonical order (= order of the left-aligned codewords):
  // by (length, symbol), a counting sort on the length, stable across the
  // threads' symbol ranges
  std::vector<uint32_t> order;
  uint64_t lcount[34] = {0};
  uint64_t lpos[34] = {0};  // first index in `order` of each length
  {
    uint64_t tc[MAXT][34] = {};
    const int nt = par(sigma, [&](int t, int n_t) {
      uint64_t b, e;
      chunk(sigma, t, n_t, b, e);
      for (uint64_t s = b; s < e; s++) tc[t][h->code_len[s]]++;
    });
    for (int t = 0; t < nt; t++)
      for (int ln = 0; ln <= 33; ln++) lcount[ln] += tc[t][ln];
    for (int ln = 2; ln <= 33; ln++) lpos[ln] = lpos[ln - 1] + (ln - 1 >= 1 ? lcount[ln - 1] : 0);
    // each thread's first slot per length: after the earlier threads'
    uint64_t at[MAXT][34];
    for (int ln = 1; ln <= 33; ln++) {
      uint64_t p0 = lpos[ln];
      for (int t = 0; t < nt; t++) {
        at[t][ln] = p0;
        p0 += tc[t][ln];
      }
    }
    order.resize(lpos[33]);
    par(sigma, [&](int t, int n_t) {
      uint64_t b, e;
      chunk(sigma, t, n_t, b, e);
      uint64_t* w = at[t];
      for (uint64_t s = b; s < e; s++)
        if (h->code_len[s]) order[w[h->code_len[s]]++] = (uint32_t)s;
    });
  }
  // level sizes, internal nodes of every level and their start positions,
  // and zero counts.  `order` is sorted by length, so the elements still on
  // level l (length > l) are a suffix of it, starting at first_gt[l]; their
  // l-bit prefixes (top bits of the left-aligned codewords) never decrease
  // along it and, the codes being canonical, grow by at most one from one
  // symbol to the next (the next codeword adds 2^(Lm - len) to the left-
  // aligned value, len > l).  So symbol i opens a node on level l exactly
  // when l < len(i) and l exceeds the common prefix of codewords i-1 and i
  // (every level below len(0) for i = 0); that node's index on level l is
  // its prefix minus the level's first one, and it starts at the elements
  // before i on that level: S[i] - S[first_gt[l]], S = prefix sums of the
  // symbol counts along `order`.
  const size_t np = order.size();
  const int Lw = std::max(Lm, 1);
  // canonical codes: consecutive values within a length, the first of each
  // length the last of the previous length plus one, shifted left
  uint64_t fcode[34] = {0};
  {
    uint64_t c = 0;
    int prev = 0;
    for (int ln = 1; ln <= 33; ln++) {
      if (!lcount[ln]) continue;
      if (prev) c = (c + lcount[prev]) << (ln - prev);
      fcode[ln] = c;
      prev = ln;
    }
  }
  auto lcode = [&](uint64_t i, int& ln_i) -> uint64_t {  // left-aligned code of order[i]
    ln_i = h->code_len[order[i]];
    return (fcode[ln_i] + (i - lpos[ln_i])) << (Lm - ln_i);
  };
  auto first_open = [&](uint64_t i, uint64_t lci) -> int {  // first level symbol i opens a node on
    if (i == 0) return 0;
    int lp;
    const uint64_t prev = lcode(i - 1, lp);
    return __builtin_clzll((prev ^ lci) << (64 - Lm)) + 1;
  };
  std::vector<uint64_t> S(np + 1, 0);
  std::vector<uint64_t> nn(Lw, 0);
  {
    // chunk sums of the counts, then the prefix sums, the codes and the
    // nodes opened per level
    uint64_t csum[MAXT + 1] = {0};
    uint64_t topen[MAXT][33] = {};
    const int nt = par(np, [&](int t, int n_t) {
      uint64_t b, e, acc = 0;
      chunk(np, t, n_t, b, e);
      for (uint64_t i = b; i < e; i++) acc += hh[order[i]];
      csum[t + 1] = acc;
    });
    for (int t = 0; t < nt; t++) csum[t + 1] += csum[t];
    par(np, [&](int t, int n_t) {
      uint64_t b, e;
      chunk(np, t, n_t, b, e);
      uint64_t acc = csum[t];
      for (uint64_t i = b; i < e; i++) {
        const uint32_t sy = order[i];
        int ln_i;
        const uint64_t lci = lcode(i, ln_i);
        h->code[sy] = (uint32_t)(lci >> (Lm - ln_i));
        S[i] = acc;
        acc += hh[sy];
        for (int l = first_open(i, lci); l < ln_i; l++) topen[t][l]++;
      }
      if (t + 1 == n_t) S[np] = acc;
    });
    for (int t = 0; t < nt; t++)
      for (int l = 0; l < Lm; l++) nn[l] += topen[t][l];
  }
  std::vector<uint64_t> first_gt(Lw + 1, np);
  {
    uint64_t acc = 0;
    for (int l = 0; l <= Lw; l++) {
      first_gt[l] = acc;  // symbols with length <= l come first
      if (l + 1 <= 33) acc += lcount[std::min(l + 1, 33)];
    }
    for (int l = 0; l <= Lw; l++) first_gt[l] = std::min<uint64_t>(first_gt[l], np);
  }
  h->level_len.assign(Lm, 0);
  std::vector<uint64_t> node_lvl(3 * (size_t)Lw, 0);
  std::vector<uint64_t> zc(Lw, 0);
  std::vector<uint64_t> node;
  {
    uint64_t tot = 0;
    for (int l = 0; l < Lm; l++) {
      int lf;
      node_lvl[3 * l] = tot;
      node_lvl[3 * l + 1] = first_gt[l] < np ? lcode(first_gt[l], lf) >> (Lm - l) : 0;
      node_lvl[3 * l + 2] = nn[l];
      tot += nn[l] + 1;  // with the sentinel
      h->level_len[l] = S[np] - S[first_gt[l]];
    }
    node.resize(tot);
  }
  // node starts at their indices, the ones of every level (the counts of the
  // symbols whose code bit l is 1), and the left-aligned codes the first
  // pass maps the symbols to
  std::vector<uint32_t> left(sigma, 0u);
  std::vector<uint64_t> ones(Lw, 0);
  {
    uint64_t tones[MAXT][33] = {};
    int tbad[MAXT] = {0};
    const int nt = par(np, [&](int t, int n_t) {
      uint64_t b, e;
      chunk(np, t, n_t, b, e);
      for (uint64_t i = b; i < e; i++) {
        const uint32_t sy = order[i];
        int ln_i;
        const uint64_t lci = lcode(i, ln_i);
        left[sy] = (uint32_t)lci;
        const uint64_t w = hh[sy];
        for (int l = first_open(i, lci); l < ln_i; l++) {
          const uint64_t k = (lci >> (Lm - l)) - node_lvl[3 * l + 1];
          if (k >= nn[l]) {  // never for a prefix code
            tbad[t] = 1;
            continue;
          }
          node[node_lvl[3 * l] + k] = S[i] - S[first_gt[l]];
        }
        for (int l = 0; l < ln_i; l++)
          if ((lci >> (Lm - 1 - l)) & 1u) tones[t][l] += w;
      }
    });
    for (int t = 0; t < nt; t++) {
      if (tbad[t]) return WT_ERR_INVALID_ARG;  // not a prefix code
      for (int l = 0; l < Lm; l++) ones[l] += tones[t][l];
    }
  }
  for (int l = 0; l < Lm; l++) {
    zc[l] = h->level_len[l] - ones[l];
    node[node_lvl[3 * l] + nn[l]] = h->level_len[l];  // sentinel = level length
  }
  h->level_off.assign(Lm + 1, 0);
  for (int l = 0; l < Lm; l++) h->level_off[l + 1] = h->level_off[l] + level_words(h->level_len[l]);
  TRY(alloc_outputs(h, std::max<uint64_t>(h->level_off.back(), 1)));
  // zero counts per level: elements whose code bit l is 0
  h->zeros.assign(zc.begin(), zc.begin() + Lm);
  if (Lm) CK(cudaMemcpyAsync(h->d_zeros, h->zeros.data(), Lm * 8, cudaMemcpyHostToDevice, st));
  h->zeros_valid = true;
  // device tables
  // per length: first canonical code, its index in `order`, symbol count
  std::vector<uint64_t> lentab(3 * 34, 0);
  {
    uint64_t idx = 0;
    for (uint32_t ln = 1; ln <= 32; ln++) {
      lentab[34 + ln] = idx;
      lentab[68 + ln] = lcount[ln];
      if (lcount[ln]) lentab[ln] = h->code[order[idx]];
      idx += lcount[ln];
    }
  }
  CK(dmalloc((void**)&h->d_code, (size_t)sigma * 4, st));
  CK(dmalloc((void**)&h->d_len, sigma, st));
  CK(dmalloc((void**)&h->d_sym_by_rank, std::max<size_t>(order.size(), 1) * 4, st));
  CK(dmalloc((void**)&h->d_len_tab, lentab.size() * 8, st));
  CK(dmalloc((void**)&h->d_node, std::max<size_t>(node.size(), 1) * 8, st));
  CK(dmalloc((void**)&h->d_node_lvl, node_lvl.size() * 8, st));
  uint32_t* d_left;
  TRY(wk.get(&d_left, sigma));
  CK(cudaMemcpyAsync(h->d_code, h->code.data(), (size_t)sigma * 4, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(h->d_len, h->code_len.data(), sigma, cudaMemcpyHostToDevice, st));
  if (!order.empty())
    CK(cudaMemcpyAsync(h->d_sym_by_rank, order.data(), order.size() * 4, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(h->d_len_tab, lentab.data(), lentab.size() * 8, cudaMemcpyHostToDevice, st));
  if (!node.empty())
    CK(cudaMemcpyAsync(h->d_node, node.data(), node.size() * 8, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(h->d_node_lvl, node_lvl.data(), node_lvl.size() * 8, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d_left, left.data(), (size_t)sigma * 4, cudaMemcpyHostToDevice, st));
  CK(cudaStreamSynchronize(st));  // host vectors above are pageable and local
  if (n == 0 || Lm == 0) return build_directories(h);
  // the pass kernel wants hf_lvl as [off, first] pairs plus the count; use a
  // 3-wide table and read [3l], [3l+1], [3l+2]
  const int tau = pick_tau(o, Lm, false);
  std::vector<PassGeom> ps = make_passes(Lm, tau, 4);
  const int G = (int)ps.size();
  const uint32_t T = PT;
  uint64_t *d_off, *d_len, *scr, *tcnt, *toff;
  uint32_t *tickets, *d_ntiles;
  TileDesc* tiles;
  uint64_t max_nodes = 1;
  for (int l = 0; l < Lm; l++) max_nodes = std::max<uint64_t>(max_nodes, node_lvl[3 * l + 2]);
  const uint64_t max_tiles = (n + T - 1) / T + max_nodes + 1;
  TRY(wk.get(&tickets, 32));
  TRY(wk.get(&d_off, Lm + 1));
  TRY(wk.get(&d_len, Lm));
  TRY(wk.get(&scr, scan_scratch(max_nodes)));
  TRY(wk.get(&tcnt, max_nodes));
  TRY(wk.get(&toff, max_nodes + 1));
  TRY(wk.get(&tiles, max_tiles));
  TRY(wk.get(&d_ntiles, 1));
  TRY(upload(d_off, h->level_off.data(), (Lm + 1) * 8, st));
  TRY(upload(d_len, h->level_len.data(), Lm * 8, st));
  k_reset_tickets<<<1, 32, 0, st>>>(tickets);
  count_launch();
  CK(cudaGetLastError());
  void* seqbuf[2] = {nullptr, nullptr};
  for (int g = 0; g + 1 < G; g++) {
    if (!seqbuf[g & 1]) {
      uint8_t* b;
      TRY(wk.get(&b, (size_t)n * max_out_w(ps)));
      seqbuf[g & 1] = b;
    }
  }
  const void* in = d_seq;
  for (int g = 0; g < G; g++) {
    const PassGeom& pg = ps[g];
    const uint64_t nn = node_lvl[3 * pg.a + 2];
    if (nn) {
      const uint64_t* bnd = h->d_node + node_lvl[3 * pg.a];
      k_tiles_count<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(bnd, 1, nn, T, tcnt);
      count_launch();
      TRY(scan_excl_u64(tcnt, toff, nn, scr, st));
      const uint64_t mtw = (h->level_len[pg.a] + T - 1) / T + nn;
      k_tiles_write<<<(unsigned)((mtw + 255) / 256), 256, 0, st>>>(
          bnd, 1, nn, T, node_lvl[3 * pg.a + 1], toff, tiles, d_ntiles, mtw);
      count_launch();
    } else {
      CK(cudaMemsetAsync(d_ntiles, 0, 4, st));
    }
    CK(cudaGetLastError());
    PassParams P = base_params(h, wk, tickets + g, d_off, d_len);
    P.in = in;
    P.in_w = g == 0 ? w : pg.in_w;
    P.code_map = g == 0 ? d_left : nullptr;
    P.out = (g + 1 < G) ? seqbuf[g & 1] : nullptr;
    P.out_w = pg.out_w;
    P.L = Lm;
    P.a = pg.a;
    P.t = pg.t;
    P.rbits = pg.rbits;
    P.shape = SHAPE_HUFF;
    P.hf_node = h->d_node;
    P.hf_lvl = h->d_node_lvl;
    P.tiles = tiles;
    P.ntiles_dev = d_ntiles;
    P.n_in = h->level_len[pg.a];
    const uint64_t mt = (P.n_in + T - 1) / T + nn;
    TRY(launch_pass(P, pg.wide, false, mt, o, st));
    in = P.out;
  }
  if (o && (o->flags & WT_FLAG_NO_DIRECTORY)) return WT_OK;
  return build_directories(h);
}


}  // namespace wtk

namespace wtk {
wt_status scan_excl_u64_pub(const uint64_t* in, uint64_t* out, uint64_t n, uint64_t* scratch,
                            cudaStream_t st) {
  return scan_excl_u64(in, out, n, scratch, st);
}
uint64_t scan_scratch_pub(uint64_t n) { return scan_scratch(n); }
}  // namespace wtk
