// wt_host.h -- host-side internals of the library (handle layout, launch
// helpers shared between translation units).  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/wavelet.h"

namespace wtk {

// One device allocation shared by the handles of a batched build; freed when
// the last of them is freed.
struct Arena {
  void* base = nullptr;
  std::atomic<int> refs{0};
  uint64_t bytes = 0;
};

// Per-level metadata used by the query kernels (device copy in the handle).
struct LevelMeta {
  uint64_t bit_off;   // word offset of the level in bits
  uint64_t dir_off;   // u64 offset of the level's directory records
  uint64_t s0_off;    // u64 offset of the zero samples
  uint64_t s1_off;    // u64 offset of the one samples
  uint64_t n;         // elements (bits or digits) on the level
  uint64_t nsb;       // superblocks
};

// Constant-time select directory of one level (offsets, in elements, into
// the handle's two arrays: ck64 = descriptors | long-range positions,
// ck32 = sub-sample offsets | long-sub-range offsets), per bit value.
// per level, per bit value (binary levels: 0, 1) or digit value (4-ary
// digit levels: 0..3)
struct ClarkMeta {
  uint64_t nr[4], nh[4], ns[4];
  uint64_t desc[4], huge[4];    // in ck64
  uint64_t sub[4], sparse[4];   // in ck32
};

// Huffman query tables (device): symbols in canonical order, per length the
// first code and the offset into that order; per level the internal nodes.
struct HuffQuery {
  const uint32_t* code;     // [sigma]
  const uint8_t* len;       // [sigma]
  const uint32_t* sym_by_rank;  // present symbols sorted by (len, symbol)
  const uint64_t* len_first;    // [34]: first canonical code of each length
  const uint64_t* len_base;     // [34]: index in sym_by_rank of that code
  const uint64_t* len_count;    // [34]: symbols of each length
  const uint64_t* node;         // internal-node starts, per level + sentinel
  const uint64_t* node_lvl;     // per level: offset, first prefix, count
};

}  // namespace wtk

struct wt_struct {
  int kind = 0;
  uint64_t n = 0;
  uint32_t sigma = 0;
  uint32_t levels = 0;      // output levels (digit levels for MULTI)
  uint32_t L = 0;           // binary levels (code length bound for HUFF)
  uint32_t bpe = 1;
  cudaStream_t stream = nullptr;
  int device = 0;
  // device arrays owned by the handle
  uint64_t* d_bits = nullptr;
  const uint64_t* d_bits_ro = nullptr;  // == d_bits, or the caller's bitvector (RS)
  uint64_t* d_dir = nullptr;
  uint64_t* d_samp = nullptr;
  uint64_t* d_zeros = nullptr;   // [levels]
  uint32_t* d_err = nullptr;     // device error word
  wtk::LevelMeta* d_meta = nullptr;
  // Huffman tables (device)
  uint32_t* d_code = nullptr;
  uint8_t* d_len = nullptr;
  uint32_t* d_sym_by_rank = nullptr;
  uint64_t* d_len_tab = nullptr;   // len_first | len_base | len_count (3 x 34)
  uint64_t* d_node = nullptr;
  uint64_t* d_node_lvl = nullptr;
  // host mirrors
  std::vector<uint64_t> level_len, level_off, dir_off, samp_off, zeros;
  std::vector<wtk::LevelMeta> meta;
  std::vector<uint8_t> code_len;
  std::vector<uint32_t> code;
  uint32_t max_code_len = 0;
  bool zeros_valid = false;
  wt_status deferred = WT_OK;
  // constant-time select directory (WT_FLAG_SELECT_O1)
  uint32_t flags = 0;
  uint64_t* d_ck64 = nullptr;
  uint32_t* d_ck32 = nullptr;
  wtk::ClarkMeta* d_cmeta = nullptr;
  std::vector<wtk::ClarkMeta> cmeta;
  // batched builds: the shared allocation holding every device array above
  wtk::Arena* arena = nullptr;
  // asynchronous builds (huff_wt_build): the library thread that builds the
  // code on the host and enqueues the rest of the build on `stream` (then
  // the handle's own stream), and the event recorded after its last work
  std::thread* worker = nullptr;
  cudaEvent_t built = nullptr;
  bool own_stream = false;
};

namespace wtk {

// a handle built asynchronously (huff_wt_build): wait for its library thread
// and, with order, make st wait for everything the build enqueued; returns
// the handle's deferred status
wt_status join_build(wt_struct* h, cudaStream_t st, bool order);

// device memory helpers (stream-ordered pools)
cudaError_t dmalloc(void** p, size_t bytes, cudaStream_t s);
void dfree(void* p, cudaStream_t s);

// directories and select samples for all levels of a handle whose bitmaps,
// level_len/level_off/meta are set.  bpe == 1 binary; bpe == 2 digits.
wt_status build_directories(wt_struct* h);

// upload h->meta into h->d_meta (allocating it)
wt_status upload_meta(wt_struct* h);

uint32_t num_sms();

// Temporary device buffers of one call, returned to the pool (in stream
// order) when the call ends, on every path.
struct Work {
  cudaStream_t st;
  std::vector<void*> bufs;
  ~Work() {
    for (void* p : bufs) dfree(p, st);
  }
  template <typename T>
  wt_status get(T** p, size_t count) {
    void* q = nullptr;
    cudaError_t e = dmalloc(&q, count * sizeof(T), st);
    if (e != cudaSuccess) return WT_ERR_NO_MEMORY;
    bufs.push_back(q);
    *p = (T*)q;
    return WT_OK;
  }
};

#define TRY(x)                     \
  do {                             \
    wt_status s_ = (x);            \
    if (s_ != WT_OK) return s_;    \
  } while (0)

// Host -> device copy of a small table through a kernel's parameters (no
// copy engine: a small copy would otherwise queue behind large transfers of
// other streams); larger tables by cudaMemcpyAsync.
wt_status upload(void* d_dst, const void* h_src, size_t bytes, cudaStream_t st);

// Launch accounting (all kernels of the library) and optional CUDA-event
// timing of the partition-pass launches, for the benchmark's roofline.
struct Prof {
  std::atomic<bool> on{false};
  std::atomic<uint64_t> launches{0};
  std::atomic<uint64_t> pass_launches{0};
  std::mutex mu;                 // guards ev (library threads record too)
  std::vector<cudaEvent_t> ev;  // pairs: before, after each pass launch
};
Prof& prof();
inline void count_launch(uint64_t k = 1) { prof().launches += k; }

}  // namespace wtk

namespace wtk {
wt_status build_wm(const void* d_seq, uint64_t n, uint32_t sigma, int w, const wt_build_opts* o,
                   wt_struct* h);
wt_status build_wt(const void* d_seq, uint64_t n, uint32_t sigma, int w, const wt_build_opts* o,
                   wt_struct* h, bool multiary);
wt_status build_huff(const void* d_seq, uint64_t n, uint32_t sigma, int w, const uint8_t* h_len,
                     const wt_build_opts* o, wt_struct* h);
wt_status launch_query(wt_struct* h, int op, const uint32_t* c, const uint64_t* x, uint64_t q,
                       uint64_t* out, cudaStream_t st);
uint32_t huffman_lengths(const uint64_t* hist, uint32_t sigma, uint32_t cap, uint8_t* len);
void canonical_codes(const uint8_t* len, uint32_t sigma, uint32_t* code);
wt_status launch_query_multi(wt_struct* const* hs, uint32_t nh, const uint32_t* sid,
                             const uint8_t* op, const uint32_t* c, const uint64_t* x, uint64_t q,
                             uint64_t* out, cudaStream_t st);
// configuration of a wavelet-matrix build recorded by the autotuner for
// (L, ceil(log2 n)): levels per pass (8 if none), symbols per tile (PASS_T if
// none) and CTAs per SM (0 = as many as fit)
struct TuneConfig {
  int tau;
  uint32_t tile;
  uint32_t ctas;
};
TuneConfig tuned_config(uint32_t L, uint64_t n);
int tuned_tau(uint32_t L, uint64_t n);
// bytes a batched wavelet-matrix build keeps for one sequence
uint64_t wm_resident_bytes(uint64_t n, uint32_t sigma);
// domain-decomposition merge of the structures of consecutive parts into
// h (kind, L, levels, n, sigma, flags set)
wt_status dd_merge(wt_struct* const* parts, uint32_t R, wt_struct* h);
// final status of the m handles of one batched build (after its stream is
// synchronised), read with one copy of the batch's error words
void batch_status(wt_handle* hs, uint32_t m, wt_status* st);
}  // namespace wtk
