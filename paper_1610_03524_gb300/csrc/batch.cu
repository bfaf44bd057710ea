// batch.cu -- many wavelet matrices built by one set of launches, and the
// autotuner that picks the levels per pass.
//
// Section 4.2 splits one sequence into K sub-sequences and combines the
// per-node counts of the pieces by prefix sums.  A batch applies the same
// decomposition across sequences: the tiles of every sequence form one work
// list, each tile carries its sequence's parameters, and the per-tile class
// counts are chained only between tiles of the same sequence.  So a batch of
// m sequences costs one histogram launch, one planning launch, one partition
// launch per pass index (two if some sequences need 32-bit working
// elements), and one set of directory launches over all levels of all
// sequences, instead of m times that.  Every device array of the batch sits
// in one allocation (the arena) shared by the m handles.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "wt_host.h"
#include "wt_internal.cuh"

namespace wtk {

wt_status launch_pass_batch(const PassParams& P, bool wide, const wt_build_opts* o,
                            cudaStream_t st);
wt_status dir_build_levels(const uint64_t* bits, const LevelMeta* d_meta, uint32_t nlev,
                           const std::vector<uint64_t>& sb_first, uint64_t* dir, uint64_t* samp,
                           uint64_t* zeros, int write_zeros, cudaStream_t st,
                           const LevelMeta* h_meta = nullptr);

#define CK(x)                                                   \
  do {                                                          \
    cudaError_t e_ = (x);                                       \
    if (e_ != cudaSuccess) {                                    \
      fprintf(stderr, "wavelet: %s -> %s\n", #x, cudaGetErrorString(e_)); \
      return e_ == cudaErrorMemoryAllocation ? WT_ERR_NO_MEMORY : WT_ERR_CUDA; \
    }                                                           \
  } while (0)

// ---------------------------------------------------------------------------
// autotuner table: (L, ceil(log2 n)) -> levels per pass, tile, CTAs per SM
// ---------------------------------------------------------------------------
namespace {
struct TuneEntry {
  uint8_t tau;      // 0 = not tuned
  uint8_t tile_lg;  // log2 of the tile's symbols, 0 = default
  uint8_t ctas;     // 0 = as many as fit
};
std::mutex g_tune_mu;
TuneEntry g_tune[33][65];

int log2_ceil(uint64_t n) {
  int k = 0;
  while (k < 64 && ((uint64_t)1 << k) < n) k++;
  return k;
}

uint32_t levels_of_b(uint32_t sigma) {
  uint32_t L = 0;
  while (L < 32 && ((uint64_t)1 << L) < (uint64_t)sigma) L++;
  return L == 0 ? 1 : L;
}

uint64_t level_words_b(uint64_t nbits) { return ((nbits + 2047) / 2048) * 32; }
int width_for_bits_b(int b) { return b <= 8 ? 1 : (b <= 16 ? 2 : 4); }
uint64_t up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }
}  // namespace

TuneConfig tuned_config(uint32_t L, uint64_t n) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  const int k = log2_ceil(n);
  const TuneEntry e = (L <= 32 && k <= 64) ? g_tune[L][k] : TuneEntry{0, 0, 0};
  return TuneConfig{e.tau ? (int)e.tau : TAU_MAX, e.tile_lg ? 1u << e.tile_lg : (uint32_t)PASS_T,
                    (uint32_t)e.ctas};
}

int tuned_tau(uint32_t L, uint64_t n) { return tuned_config(L, n).tau; }

static void record_config(uint32_t L, uint64_t n, int tau, uint32_t tile, uint32_t ctas) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  const int k = log2_ceil(n);
  int lg = 0;
  while (tile > 1u && (1u << lg) < tile) lg++;
  if (L <= 32 && k <= 64)
    g_tune[L][k] = TuneEntry{(uint8_t)tau, (uint8_t)(tile ? lg : 0), (uint8_t)ctas};
}

// ---------------------------------------------------------------------------
// batch layout
// ---------------------------------------------------------------------------
namespace {

struct Pass1 {
  int a, t, rbits, in_w, out_w;
  bool wide;
};

struct SeqPlan {
  uint64_t n;
  uint32_t sigma;
  int w, L, tau, G;
  std::vector<Pass1> ps;
  uint64_t W, nsb, cap;      // words per level, superblocks per level, samples per value
  // arena offsets (u64 units inside each region)
  uint64_t bits_base, dir_base, samp_base, zeros_base, meta_base;
  // workspace offsets
  uint64_t cls_off, lvl_base, seq_off;  // seq_off: bytes in each ping-pong buffer
  uint64_t seq_bytes;
};

void plan_seq(SeqPlan& p, const wt_build_opts* o) {
  p.L = (int)levels_of_b(p.sigma);
  p.tau = (o && o->tau) ? (int)std::min<uint32_t>(o->tau, TAU_MAX) : tuned_tau(p.L, p.n);
  if (p.tau < 1) p.tau = 1;
  p.ps.clear();
  for (int a = 0; a < p.L; a += p.tau) {
    Pass1 q;
    q.a = a;
    q.t = std::min(p.tau, p.L - a);
    q.rbits = p.L - a;
    q.in_w = a == 0 ? p.w : width_for_bits_b(p.L - a);
    q.out_w = (a + q.t < p.L) ? width_for_bits_b(p.L - a - q.t) : 0;
    q.wide = q.rbits > 16;
    p.ps.push_back(q);
  }
  p.G = (int)p.ps.size();
  p.W = level_words_b(p.n);
  p.nsb = (p.n + 2047) / 2048;
  p.cap = p.n / 4096 + 1;
  int ow = 0;
  for (const Pass1& q : p.ps) ow = std::max(ow, q.out_w);
  p.seq_bytes = up(p.n * (uint64_t)ow, 256);
}

// bytes of the arena regions of one sequence
uint64_t bits_u64(const SeqPlan& p) { return (uint64_t)p.L * p.W; }
uint64_t dir_u64(const SeqPlan& p) { return up((uint64_t)p.L * 2 * (p.nsb + 1), 32); }
uint64_t samp_u64(const SeqPlan& p) { return up((uint64_t)p.L * 2 * p.cap, 32); }

}  // namespace

uint64_t wm_resident_bytes(uint64_t n, uint32_t sigma) {
  SeqPlan p{};
  p.n = n;
  p.sigma = sigma;
  p.w = 2;
  plan_seq(p, nullptr);
  return 8 * (bits_u64(p) + dir_u64(p) + samp_u64(p) + (uint64_t)p.L) +
         (uint64_t)p.L * sizeof(LevelMeta) + 8;
}

// Builds m wavelet matrices with directories; outs[i] receives handle i.
wt_status batch_build_wm(const wt_batch_item* items, uint32_t m, const wt_build_opts* o,
                         cudaStream_t st, wt_struct** hs) {
  std::vector<SeqPlan> sp(m);
  uint64_t nbits = 0, ndir = 0, nsamp = 0, nzeros = 0, nmeta = 0;
  uint64_t ncls = 0, nlvl = 0, nseq = 0;
  uint64_t nlev_tot = 0;
  int Gmax = 0;
  for (uint32_t i = 0; i < m; i++) {
    SeqPlan& p = sp[i];
    p.n = items[i].n;
    p.sigma = items[i].sigma;
    p.w = (int)items[i].width_bytes;
    plan_seq(p, o);
    p.bits_base = nbits;
    p.dir_base = ndir;
    p.samp_base = nsamp;
    p.zeros_base = nzeros;
    p.meta_base = nmeta;
    nbits += bits_u64(p);
    ndir += dir_u64(p);
    nsamp += samp_u64(p);
    nzeros += p.L;
    nmeta += p.L;
    p.cls_off = ncls;
    for (const Pass1& q : p.ps) ncls += (2u << q.t) + q.t + 1;
    p.lvl_base = nlvl;
    nlvl += 2 * (uint64_t)p.L + 1;  // L+1 word offsets, then L lengths
    p.seq_off = nseq;
    nseq += p.G > 1 ? p.seq_bytes : 0;
    nlev_tot += p.L;
    Gmax = std::max(Gmax, p.n ? p.G : 0);
  }
  // ---- arena: bits | dir | samp | zeros | meta | err[m] -----------------
  const uint64_t off_dir = 8 * nbits;
  const uint64_t off_samp = off_dir + 8 * ndir;
  const uint64_t off_zeros = off_samp + 8 * nsamp;
  const uint64_t off_meta = up(off_zeros + 8 * nzeros, 256);
  const uint64_t off_err = up(off_meta + sizeof(LevelMeta) * nmeta, 256);
  const uint64_t arena_bytes = off_err + up(4 * (uint64_t)m, 256);
  Arena* ar = new Arena();
  ar->bytes = arena_bytes;
  {
    cudaError_t e = dmalloc(&ar->base, arena_bytes, st);
    if (e != cudaSuccess) {
      delete ar;
      return WT_ERR_NO_MEMORY;
    }
  }
  uint8_t* A = (uint8_t*)ar->base;
  uint64_t* a_bits = (uint64_t*)A;
  uint64_t* a_dir = (uint64_t*)(A + off_dir);
  uint64_t* a_samp = (uint64_t*)(A + off_samp);
  uint64_t* a_zeros = (uint64_t*)(A + off_zeros);
  LevelMeta* a_meta = (LevelMeta*)(A + off_meta);
  uint32_t* a_err = (uint32_t*)(A + off_err);
  // level l of a sequence inside its own arrays
  auto meta_of = [](const SeqPlan& p, int l) {
    LevelMeta mt{};
    mt.bit_off = (uint64_t)l * p.W;
    mt.dir_off = (uint64_t)l * 2 * (p.nsb + 1);
    mt.s0_off = (uint64_t)(2 * l) * p.cap;
    mt.s1_off = (uint64_t)(2 * l + 1) * p.cap;
    mt.n = p.n;
    mt.nsb = p.nsb;
    return mt;
  };
  // handles own the arena from here on (a failure below frees it through
  // them); their host-side tables are filled once the work is enqueued
  for (uint32_t i = 0; i < m; i++) {
    wt_struct* h = hs[i];
    const SeqPlan& p = sp[i];
    h->arena = ar;
    ar->refs++;
    h->kind = WT_KIND_WM;
    h->n = p.n;
    h->sigma = p.sigma;
    h->L = h->levels = (uint32_t)p.L;
    h->bpe = 1;
    h->stream = st;
    h->d_bits = a_bits + p.bits_base;
    h->d_bits_ro = h->d_bits;
    h->d_dir = a_dir + p.dir_base;
    h->d_samp = a_samp + p.samp_base;
    h->d_zeros = a_zeros + p.zeros_base;
    h->d_meta = a_meta + p.meta_base;
    h->d_err = a_err + i;
  }
  // ---- workspace ----------------------------------------------------------
  uint64_t nsegs_tot = 0;
  for (int g = 0; g < Gmax; g++)
    for (uint32_t i = 0; i < m; i++)
      if (sp[i].n && g < sp[i].G) nsegs_tot++;
  const uint64_t w_cls = 0;
  const uint64_t w_lvl = up(w_cls + 8 * ncls, 256);
  const uint64_t w_gmeta = up(w_lvl + 8 * nlvl, 256);
  const uint64_t w_sseg = up(w_gmeta + sizeof(LevelMeta) * nlev_tot, 256);
  const uint64_t w_tab_end = up(w_sseg + sizeof(SegDesc) * std::max<uint64_t>(nsegs_tot, 1), 256);
  const uint64_t w_tick = w_tab_end;
  const uint64_t w_seq0 = up(w_tick + 4 * 64, 256);
  const uint64_t w_seq1 = up(w_seq0 + nseq, 256);
  const uint64_t ws_bytes = up(w_seq1 + nseq, 256);
  void* wsv = nullptr;
  CK(dmalloc(&wsv, ws_bytes, st));
  uint8_t* Wd = (uint8_t*)wsv;
  uint64_t* d_cls = (uint64_t*)(Wd + w_cls);
  uint64_t* d_lvl = (uint64_t*)(Wd + w_lvl);
  LevelMeta* d_gmeta = (LevelMeta*)(Wd + w_gmeta);
  SegDesc* d_sseg = (SegDesc*)(Wd + w_sseg);
  uint32_t* d_tick = (uint32_t*)(Wd + w_tick);
  uint8_t* d_seq[2] = {Wd + w_seq0, Wd + w_seq1};

  // host image of the tables [w_lvl, w_tab_end)
  std::vector<uint8_t> img(w_tab_end - w_lvl, 0);
  auto at = [&](uint64_t off) { return img.data() + (off - w_lvl); };
  uint64_t* h_lvl = (uint64_t*)at(w_lvl);
  LevelMeta* h_gmeta = (LevelMeta*)at(w_gmeta);
  SegDesc* h_sseg = (SegDesc*)at(w_sseg);
  std::vector<uint64_t> sb_first(nlev_tot + 1, 0);
  std::vector<LevelMeta> h_meta_all(nmeta);
  {
    uint64_t lev = 0;
    for (uint32_t i = 0; i < m; i++) {
      const SeqPlan& p = sp[i];
      uint64_t* lo = h_lvl + p.lvl_base;
      uint64_t* ll = lo + p.L + 1;
      for (int l = 0; l <= p.L; l++) lo[l] = (uint64_t)l * p.W;
      for (int l = 0; l < p.L; l++) ll[l] = p.n;
      for (int l = 0; l < p.L; l++, lev++) {
        LevelMeta mt = meta_of(p, l);
        h_meta_all[p.meta_base + l] = mt;
        mt.bit_off += p.bits_base;
        mt.dir_off += p.dir_base;
        mt.s0_off += p.samp_base;
        mt.s1_off += p.samp_base;
        h_gmeta[lev] = mt;
        sb_first[lev + 1] = sb_first[lev] + p.nsb;
      }
    }
  }
  // per-launch segment lists: pass g, narrow (E = u16) then wide (E = u32)
  struct Launch {
    uint64_t first;
    uint32_t nsegs, ntiles;
    bool wide;
    int tmax;  // widest digit of its segments
  };
  std::vector<Launch> launches;
  {
    uint64_t k = 0;
    for (int g = 0; g < Gmax; g++) {
      for (int wide = 0; wide < 2; wide++) {
        Launch L0{k, 0, 0, wide != 0, 1};
        uint32_t tiles = 0;
        for (uint32_t i = 0; i < m; i++) {
          const SeqPlan& p = sp[i];
          if (!p.n || g >= p.G || p.ps[g].wide != (wide != 0)) continue;
          const Pass1& q = p.ps[g];
          uint64_t coff = p.cls_off;
          for (int g2 = 0; g2 < g; g2++) coff += (2u << p.ps[g2].t) + p.ps[g2].t + 1;
          SegDesc& d = h_sseg[k++];
          d.in = g == 0 ? items[i].d_seq : (const void*)(d_seq[(g - 1) & 1] + p.seq_off);
          d.out = (g + 1 < p.G) ? (void*)(d_seq[g & 1] + p.seq_off) : nullptr;
          d.bits = a_bits + p.bits_base;
          d.lvl_off = d_lvl + p.lvl_base;
          d.lvl_len = d_lvl + p.lvl_base + p.L + 1;
          d.wm_cls = d_cls + coff;
          d.zeros = a_zeros + p.zeros_base;
          d.err = a_err + i;
          d.n = p.n;
          d.tile0 = tiles;
          d.sigma = g == 0 ? p.sigma : 0u;
          d.in_w = q.in_w;
          d.out_w = q.out_w;
          d.L = p.L;
          d.a = q.a;
          d.t = q.t;
          d.rbits = q.rbits;
          tiles += (uint32_t)((p.n + PASS_T - 1) / PASS_T);
          L0.nsegs++;
          L0.tmax = std::max(L0.tmax, q.t);
        }
        L0.ntiles = tiles;
        if (L0.nsegs) launches.push_back(L0);
      }
    }
  }
  // ---- uploads and launches -------------------------------------------------
  if (nbits) CK(cudaMemsetAsync(a_bits, 0, 8 * nbits, st));
  CK(cudaMemsetAsync(a_err, 0, 4 * (uint64_t)m, st));
  if (nzeros) CK(cudaMemsetAsync(a_zeros, 0, 8 * nzeros, st));  // empty sequences plan nothing
  CK(cudaMemsetAsync(d_tick, 0, 4 * 64, st));
  wt_status s = nmeta ? upload(a_meta, h_meta_all.data(), sizeof(LevelMeta) * nmeta, st) : WT_OK;
  if (s == WT_OK) s = upload(Wd + w_lvl, img.data(), img.size(), st);
  for (size_t li = 0; li < launches.size() && s == WT_OK; li++) {
    const Launch& L0 = launches[li];
    PassParams P;
    memset(&P, 0, sizeof(P));
    P.shape = SHAPE_WM;
    P.ticket = d_tick + li;
    P.err = a_err;  // replaced per tile by the sequence's own word
    P.ntiles = L0.ntiles;
    P.segs = d_sseg + L0.first;
    P.nsegs = L0.nsegs;
    P.tcs = tc_stride(L0.tmax);
    s = launch_pass_batch(P, L0.wide, o, st);
  }
  if (s == WT_OK && !(o && (o->flags & WT_FLAG_NO_DIRECTORY)))
    s = dir_build_levels(a_bits, d_gmeta, (uint32_t)nlev_tot, sb_first, a_dir, a_samp, nullptr,
                         0, st);
  dfree(wsv, st);
  if (s != WT_OK) return s;
  CK(cudaGetLastError());
  // the handles' host-side tables, while the device works
  for (uint32_t i = 0; i < m; i++) {
    wt_struct* h = hs[i];
    const SeqPlan& p = sp[i];
    h->level_len.assign(p.L, p.n);
    h->level_off.resize(p.L + 1);
    h->dir_off.resize(p.L + 1);
    h->samp_off.resize(2 * p.L + 1);
    h->meta.resize(p.L);
    for (int l = 0; l <= p.L; l++) {
      const LevelMeta mt = meta_of(p, l);
      h->level_off[l] = mt.bit_off;
      h->dir_off[l] = mt.dir_off;
      h->samp_off[2 * l] = mt.s0_off;
      if (l < p.L) {
        h->samp_off[2 * l + 1] = mt.s1_off;
        h->meta[l] = mt;
      }
    }
  }
  return WT_OK;
}

void batch_status(wt_handle* hs, uint32_t m, wt_status* st) {
  // the batch's error words are consecutive in its arena
  // on the batch's own stream (the legacy stream would wait for every other
  // blocking stream, e.g. a caller's copy of the next input)
  std::vector<uint32_t> err((size_t)m, 0);
  const bool ok = m &&
                  cudaMemcpyAsync(err.data(), hs[0]->d_err, 4 * (size_t)m, cudaMemcpyDeviceToHost,
                                  hs[0]->stream) == cudaSuccess &&
                  cudaStreamSynchronize(hs[0]->stream) == cudaSuccess;
  for (uint32_t i = 0; i < m; i++) {
    wt_status s = WT_OK;
    if (!ok) s = WT_ERR_CUDA;
    else if (err[i] & ERR_SYMBOL) s = WT_ERR_SYMBOL_GE_SIGMA;
    else if (err[i]) s = WT_ERR_CUDA;
    if (s != WT_OK) hs[i]->deferred = s;
    st[i] = s;
  }
}

// ---------------------------------------------------------------------------
// autotuner
// ---------------------------------------------------------------------------
wt_status build_wm(const void* d_seq, uint64_t n, uint32_t sigma, int w, const wt_build_opts* o,
                   wt_struct* h);

}  // namespace wtk

using namespace wtk;

namespace {
void free_handle_partial(wt_struct* h) {
  // handles of a failed batch: release the arena reference, nothing else
  if (h->arena && h->arena->refs.fetch_sub(1) == 1) {
    dfree(h->arena->base, h->stream);
    delete h->arena;
  }
  h->arena = nullptr;
  delete h;
}
}  // namespace

extern "C" wt_status wm_batch_build(const wt_batch_item* items, uint32_t m,
                                    const wt_build_opts* opts, wt_stream stream, wt_handle* outs) {
  if (!outs || (m && !items)) return WT_ERR_INVALID_ARG;
  for (uint32_t i = 0; i < m; i++) outs[i] = nullptr;
  if (opts) {
    if (opts->tau > 8) return WT_ERR_INVALID_ARG;
    if (opts->select_sample != 0 && opts->select_sample != 4096) return WT_ERR_UNSUPPORTED;
    if (opts->tile_symbols != 0 && opts->tile_symbols != (uint32_t)PASS_T) return WT_ERR_UNSUPPORTED;
    if (opts->k_chunks != 0) return WT_ERR_UNSUPPORTED;
    if (opts->flags & WT_FLAG_SELECT_O1) return WT_ERR_UNSUPPORTED;
  }
  for (uint32_t i = 0; i < m; i++) {
    const wt_batch_item& it = items[i];
    if ((!it.d_seq && it.n) || it.sigma == 0) return WT_ERR_INVALID_ARG;
    if (it.width_bytes != 1 && it.width_bytes != 2 && it.width_bytes != 4)
      return WT_ERR_INVALID_ARG;
    if (it.n >= ((uint64_t)1 << 40)) return WT_ERR_UNSUPPORTED;
  }
  if (m == 0) return WT_OK;
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<wt_struct*> hs(m, nullptr);
  int dev = 0;
  cudaGetDevice(&dev);
  for (uint32_t i = 0; i < m; i++) {
    hs[i] = new (std::nothrow) wt_struct();
    if (!hs[i]) {
      for (uint32_t j = 0; j < i; j++) delete hs[j];
      return WT_ERR_NO_MEMORY;
    }
    hs[i]->device = dev;
    hs[i]->stream = st;
  }
  wt_status s = batch_build_wm(items, m, opts, st, hs.data());
  if (s == WT_OK && cudaGetLastError() != cudaSuccess) s = WT_ERR_CUDA;
  if (s != WT_OK) {
    cudaStreamSynchronize(st);
    for (uint32_t i = 0; i < m; i++) free_handle_partial(hs[i]);
    cudaStreamSynchronize(st);
    return s;
  }
  for (uint32_t i = 0; i < m; i++) outs[i] = hs[i];
  return WT_OK;
}

struct wt_batch_s {
  std::vector<wt_handle> hs;
  cudaStream_t st = nullptr;
};

extern "C" wt_status wm_batch_build_one(const wt_batch_item* items, uint32_t m,
                                        const wt_build_opts* opts, wt_stream stream,
                                        wt_batch* out) {
  if (!out) return WT_ERR_INVALID_ARG;
  *out = nullptr;
  wt_batch b = new (std::nothrow) wt_batch_s();
  if (!b) return WT_ERR_NO_MEMORY;
  b->hs.assign(m, nullptr);
  b->st = (cudaStream_t)stream;
  const wt_status s = wm_batch_build(items, m, opts, stream, b->hs.data());
  if (s != WT_OK) {
    delete b;
    return s;
  }
  *out = b;
  return WT_OK;
}

extern "C" wt_handle wt_batch_handle(wt_batch b, uint32_t i) {
  return (b && i < b->hs.size()) ? b->hs[i] : nullptr;
}

extern "C" wt_status wt_batch_sync(wt_batch b, wt_status* st) {
  if (!b) return WT_ERR_INVALID_ARG;
  if (cudaStreamSynchronize(b->st) != cudaSuccess) return WT_ERR_CUDA;
  const uint32_t m = (uint32_t)b->hs.size();
  std::vector<wt_status> s(m, WT_OK);
  if (m) batch_status(b->hs.data(), m, s.data());
  wt_status first = WT_OK;
  for (uint32_t i = 0; i < m; i++) {
    if (st) st[i] = s[i];
    if (first == WT_OK) first = s[i];
  }
  return first;
}

extern "C" wt_status wt_batch_free(wt_batch b) {
  if (!b) return WT_ERR_INVALID_ARG;
  // one wait for the batch's queued work, then every handle's reference to
  // the shared arena is dropped; the last returns it to the pool
  cudaError_t e = cudaStreamSynchronize(b->st);
  for (wt_handle h : b->hs) {
    if (!h) continue;
    if (h->arena && h->arena->refs.fetch_sub(1) == 1) {
      dfree(h->arena->base, b->st);
      delete h->arena;
    }
    h->arena = nullptr;
    delete h;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
  delete b;
  return e == cudaSuccess ? WT_OK : WT_ERR_CUDA;
}

extern "C" wt_status wm_autotune(const void* d_seq, uint64_t n, uint32_t sigma,
                                 uint32_t width_bytes, wt_stream stream, uint32_t* best_tau,
                                 float* ms_out) {
  if ((!d_seq && n) || sigma == 0 || !best_tau) return WT_ERR_INVALID_ARG;
  if (width_bytes != 1 && width_bytes != 2 && width_bytes != 4) return WT_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const uint32_t L = levels_of_b(sigma);
  const uint32_t tmax = std::min<uint32_t>(L, TAU_MAX);
  if (ms_out)
    for (int i = 0; i < TAU_MAX; i++) ms_out[i] = 0.f;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float best = 0.f;
  uint32_t bt = tmax;
  wt_status s = WT_OK;
  for (uint32_t tau = 1; tau <= tmax && s == WT_OK; tau++) {
    // one untimed build, then the best of two timed ones
    float t_best = 0.f;
    for (int r = 0; r < 3 && s == WT_OK; r++) {
      wt_build_opts o{};
      o.tau = tau;
      o.flags = WT_FLAG_NO_DIRECTORY;
      wt_handle h = nullptr;
      cudaEventRecord(e0, st);
      s = wm_build(d_seq, n, sigma, width_bytes, &o, stream, &h);
      cudaEventRecord(e1, st);
      if (s != WT_OK) break;
      s = wt_sync(h);
      wt_free(h);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (r > 0 && (t_best == 0.f || ms < t_best)) t_best = ms;
    }
    if (s != WT_OK) break;
    if (ms_out) ms_out[tau - 1] = t_best;
    if (best == 0.f || t_best < best) {
      best = t_best;
      bt = tau;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != WT_OK) return s;
  *best_tau = bt;
  record_config(L, n, (int)bt, 0, 0);
  return WT_OK;
}

namespace {
// one untimed build, then the best of two timed ones (no directories)
wt_status time_wm(const void* d_seq, uint64_t n, uint32_t sigma, uint32_t width,
                  cudaStream_t st, uint32_t tau, uint32_t tile, uint32_t ctas, cudaEvent_t e0,
                  cudaEvent_t e1, float* best) {
  *best = 0.f;
  for (int r = 0; r < 3; r++) {
    wt_build_opts o{};
    o.tau = tau;
    o.tile_symbols = tile;
    o.ctas_per_sm = ctas;
    o.flags = WT_FLAG_NO_DIRECTORY;
    wt_handle h = nullptr;
    cudaEventRecord(e0, st);
    wt_status s = wm_build(d_seq, n, sigma, width, &o, (wt_stream)st, &h);
    cudaEventRecord(e1, st);
    if (s != WT_OK) return s;
    s = wt_sync(h);
    wt_free(h);
    if (s != WT_OK) return s;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (r > 0 && (*best == 0.f || ms < *best)) *best = ms;
  }
  return WT_OK;
}
}  // namespace

extern "C" wt_status wm_autotune_config(const void* d_seq, uint64_t n, uint32_t sigma,
                                        uint32_t width_bytes, wt_stream stream, wt_tuning* out) {
  if ((!d_seq && n) || sigma == 0 || !out) return WT_ERR_INVALID_ARG;
  if (width_bytes != 1 && width_bytes != 2 && width_bytes != 4) return WT_ERR_INVALID_ARG;
  if (n >= ((uint64_t)1 << 40)) return WT_ERR_UNSUPPORTED;
  cudaStream_t st = (cudaStream_t)stream;
  const uint32_t L = levels_of_b(sigma);
  const uint32_t tmax = std::min<uint32_t>(L, TAU_MAX);
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  wt_status s = WT_OK;
  // levels per pass first, at the default tile and occupancy; then tile
  // size and CTAs per SM at the best two of them
  float tms[TAU_MAX + 1] = {0};
  for (uint32_t tau = 1; tau <= tmax && s == WT_OK; tau++)
    s = time_wm(d_seq, n, sigma, width_bytes, st, tau, 0, 0, e0, e1, &tms[tau]);
  uint32_t t1 = tmax, t2 = 0;
  for (uint32_t tau = 1; tau <= tmax; tau++)
    if (tms[tau] < tms[t1]) t1 = tau;
  for (uint32_t tau = 1; tau <= tmax; tau++)
    if (tau != t1 && (t2 == 0 || tms[tau] < tms[t2])) t2 = tau;
  wt_tuning best{};
  best.tau = t1;
  best.tile_symbols = (uint32_t)PASS_T;
  best.ms = tms[t1];
  const uint32_t tiles[3] = {2048, 4096, 8192};
  const uint32_t ctas[3] = {0, 4, 3};
  for (uint32_t tau : {t1, t2}) {
    if (tau == 0) continue;
    for (uint32_t tile : tiles)
      for (uint32_t c : ctas) {
        if (s != WT_OK) break;
        if (tile == (uint32_t)PASS_T && c == 0) continue;  // timed above
        float ms = 0.f;
        s = time_wm(d_seq, n, sigma, width_bytes, st, tau, tile, c, e0, e1, &ms);
        if (s == WT_OK && ms < best.ms) {
          best.tau = tau;
          best.tile_symbols = tile;
          best.ctas_per_sm = c;
          best.ms = ms;
        }
      }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != WT_OK) return s;
  best.k_chunks = (n + best.tile_symbols - 1) / best.tile_symbols;
  *out = best;
  record_config(L, n, (int)best.tau, best.tile_symbols, best.ctas_per_sm);
  return WT_OK;
}

extern "C" wt_status wm_tuning(uint64_t n, uint32_t sigma, wt_tuning* out) {
  if (!out || sigma == 0) return WT_ERR_INVALID_ARG;
  const TuneConfig c = tuned_config(levels_of_b(sigma), n);
  *out = wt_tuning{};
  out->tau = std::min<uint32_t>((uint32_t)c.tau, levels_of_b(sigma));
  out->tile_symbols = c.tile;
  out->ctas_per_sm = c.ctas;
  out->k_chunks = (n + c.tile - 1) / c.tile;
  return WT_OK;
}

extern "C" void wm_autotune_clear(void) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  memset(g_tune, 0, sizeof(g_tune));
}

extern "C" wt_status wt_query_multi(const wt_handle* hs, uint32_t nh, const uint32_t* d_sid,
                                    const uint8_t* d_op, const uint32_t* d_c,
                                    const uint64_t* d_x, uint64_t q, uint64_t* d_out,
                                    wt_stream stream) {
  if ((nh && !hs) || (q && (!d_sid || !d_op || !d_c || !d_x || !d_out))) return WT_ERR_INVALID_ARG;
  for (uint32_t i = 0; i < nh; i++) {
    if (!hs[i]) return WT_ERR_INVALID_ARG;
    const wt_status s = join_build(hs[i], (cudaStream_t)stream, true);
    if (s != WT_OK) return s;
  }
  return launch_query_multi(hs, nh, d_sid, d_op, d_c, d_x, q, d_out, (cudaStream_t)stream);
}
