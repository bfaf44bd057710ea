// api.cu -- the C ABI (include/wavelet.h): argument checks, handle lifetime,
// export.  Every computational step runs in the kernels of build.cu and
// dirq.cu.
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>

#include "wt_host.h"
#include "wt_internal.cuh"

using namespace wtk;

namespace {

bool valid_width(uint32_t w) { return w == 1 || w == 2 || w == 4; }

wt_status check_opts(const wt_build_opts* o) {
  if (!o) return WT_OK;
  if (o->tau > 8) return WT_ERR_INVALID_ARG;
  if (o->select_sample != 0 && o->select_sample != 4096) return WT_ERR_UNSUPPORTED;
  // tiles of 2048, 4096 or 8192 symbols (wavelet matrix; the trees take
  // PASS_T only, checked by the caller); K = ceil(n / tile) follows from n
  if (o->tile_symbols != 0 && o->tile_symbols != 2048 && o->tile_symbols != 4096 &&
      o->tile_symbols != 8192)
    return WT_ERR_UNSUPPORTED;
  if (o->k_chunks != 0) return WT_ERR_UNSUPPORTED;
  return WT_OK;
}

// sync: first wait for the work queued on the handle's stream (queries on
// other streams included, through the caller's ordering), as wt_free does
void free_arrays(wt_struct* h, bool sync = false) {
  cudaStream_t st = h->stream;
  if (h->arena) {
    // the last handle of a batch returns the shared allocation
    if (h->arena->refs.fetch_sub(1) == 1) {
      if (sync) cudaStreamSynchronize(st);
      dfree(h->arena->base, st);
      delete h->arena;
      // the memory is back in the pool, for allocations on any stream
      if (sync) cudaStreamSynchronize(st);
    }
    h->arena = nullptr;
    return;
  }
  if (sync) cudaStreamSynchronize(st);
  dfree(h->d_bits, st);
  dfree(h->d_dir, st);
  dfree(h->d_samp, st);
  dfree(h->d_zeros, st);
  dfree(h->d_err, st);
  dfree(h->d_meta, st);
  dfree(h->d_code, st);
  dfree(h->d_len, st);
  dfree(h->d_sym_by_rank, st);
  dfree(h->d_len_tab, st);
  dfree(h->d_node, st);
  dfree(h->d_node_lvl, st);
  dfree(h->d_ck64, st);
  dfree(h->d_ck32, st);
  dfree(h->d_cmeta, st);
}

wt_status new_handle(wt_stream stream, uint64_t n, uint32_t sigma, wt_struct** out) {
  wt_struct* h = new (std::nothrow) wt_struct();
  if (!h) return WT_ERR_NO_MEMORY;
  h->stream = (cudaStream_t)stream;
  h->n = n;
  h->sigma = sigma;
  cudaGetDevice(&h->device);
  if (dmalloc((void**)&h->d_err, 8, h->stream) != cudaSuccess) {
    free_arrays(h);
    delete h;
    return WT_ERR_NO_MEMORY;
  }
  cudaMemsetAsync(h->d_err, 0, 8, h->stream);
  *out = h;
  return WT_OK;
}

wt_status finish(wt_struct* h, wt_status s, wt_handle* out) {
  if (s == WT_OK) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) s = WT_ERR_CUDA;
  }
  if (s != WT_OK) {
    cudaStreamSynchronize(h->stream);
    free_arrays(h);
    cudaStreamSynchronize(h->stream);
    delete h;
    *out = nullptr;
    return s;
  }
  *out = h;
  return WT_OK;
}

wt_status sync_handle(wt_struct* h) {
  if (h->deferred != WT_OK) return h->deferred;
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return h->deferred = WT_ERR_CUDA;
  // small reads on the handle's own stream (not the legacy stream, which
  // would wait for every other blocking stream of the device)
  uint32_t err = 0;
  e = cudaMemcpyAsync(&err, h->d_err, 4, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return h->deferred = WT_ERR_CUDA;
  if (err & ERR_SYMBOL) return h->deferred = WT_ERR_SYMBOL_GE_SIGMA;
  // ERR_INTERNAL (a table disagreed with a tile) or ERR_STALL (a tile load
  // that did not complete in time)
  if (err) return h->deferred = WT_ERR_CUDA;
  if (!h->zeros_valid) {
    h->zeros.assign(h->levels, 0);
    if (h->levels && h->bpe == 1) {
      e = cudaMemcpyAsync(h->zeros.data(), h->d_zeros, h->levels * 8, cudaMemcpyDeviceToHost,
                          h->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
      if (e != cudaSuccess) return h->deferred = WT_ERR_CUDA;
    }
    h->zeros_valid = true;
  }
  return WT_OK;
}

// A handle built asynchronously: wait for its library thread, then (with
// st given) order st after everything the build enqueued.  Returns the
// handle's deferred status.
wt_status join_build_impl(wt_struct* h, cudaStream_t st, bool order) {
  if (h->worker) {
    h->worker->join();
    delete h->worker;
    h->worker = nullptr;
  }
  if (order && h->built && st != h->stream) cudaStreamWaitEvent(st, h->built, 0);
  return h->deferred;
}

__global__ void k_copy_bytes(uint8_t* dst, const uint8_t* src, uint64_t bytes) {
  const uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  if ((((uintptr_t)dst | (uintptr_t)src) & 15) == 0) {
    const uint64_t nv = bytes / 16;
    for (uint64_t i = i0; i < nv; i += stride) ((uint4*)dst)[i] = ((const uint4*)src)[i];
    for (uint64_t i = nv * 16 + i0; i < bytes; i += stride) dst[i] = src[i];
  } else {
    for (uint64_t i = i0; i < bytes; i += stride) dst[i] = src[i];
  }
}

// Huffman-shaped tree, asynchronous: the call enqueues a copy of the input on
// the caller's stream (the input is borrowed only until that stream reaches
// the copy) and returns; a library thread builds the code on the host from
// the histogram and enqueues the build on the handle's own stream, which
// starts after the copy.  Every later call on the handle first waits for
// that thread and orders its own stream after the build (join_build).
wt_status huff_async(const void* d_seq, uint64_t n, uint32_t sigma, uint32_t width,
                     const uint8_t* h_len, const wt_build_opts* opts, wt_stream stream,
                     wt_handle* out) {
  cudaStream_t cs = (cudaStream_t)stream;
  wt_struct* h = nullptr;
  wt_status s = new_handle(stream, n, sigma, &h);
  if (s != WT_OK) return s;
  h->flags = opts ? opts->flags : 0u;
  h->kind = WT_KIND_HUFF;
  cudaStream_t own = nullptr;
  cudaEvent_t ready = nullptr;
  void* copy = nullptr;
  const uint64_t bytes = n * (uint64_t)width;
  bool ok = cudaStreamCreateWithFlags(&own, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&h->built, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) == cudaSuccess &&
            dmalloc(&copy, bytes, cs) == cudaSuccess;
  if (ok && bytes) {
    const unsigned grid = (unsigned)std::min<uint64_t>((bytes / 16 + 255) / 256 + 1, 4096);
    k_copy_bytes<<<grid, 256, 0, cs>>>((uint8_t*)copy, (const uint8_t*)d_seq, bytes);
    count_launch();
  }
  ok = ok && cudaEventRecord(ready, cs) == cudaSuccess &&
       cudaStreamWaitEvent(own, ready, 0) == cudaSuccess && cudaGetLastError() == cudaSuccess;
  if (ready) cudaEventDestroy(ready);
  if (!ok) {
    if (copy) dfree(copy, cs);
    cudaStreamSynchronize(cs);
    free_arrays(h);
    cudaStreamSynchronize(cs);
    if (h->built) cudaEventDestroy(h->built);
    if (own) cudaStreamDestroy(own);
    delete h;
    return WT_ERR_CUDA;
  }
  h->stream = own;
  h->own_stream = true;
  std::vector<uint8_t> lens;
  if (h_len) lens.assign(h_len, h_len + sigma);
  const wt_build_opts oc = opts ? *opts : wt_build_opts{};
  const int dev = h->device;
  h->worker = new std::thread([h, copy, n, sigma, width, lens, oc, dev]() {
    cudaSetDevice(dev);
    wt_status st = build_huff(copy, n, sigma, (int)width, lens.empty() ? nullptr : lens.data(),
                              &oc, h);
    dfree(copy, h->stream);
    if (st == WT_OK && cudaGetLastError() != cudaSuccess) st = WT_ERR_CUDA;
    if (st != WT_OK) h->deferred = st;
    cudaEventRecord(h->built, h->stream);
  });
  *out = h;
  return WT_OK;
}

// One stream per device for the copies of host-memory builds, created on
// first use and kept for the life of the process.
cudaError_t host_copy_stream(cudaStream_t* out) {
  static std::mutex mu;
  static cudaStream_t streams[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> g(mu);
  if (!streams[dev]) {
    e = cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      streams[dev] = nullptr;
      return e;
    }
  }
  *out = streams[dev];
  return cudaSuccess;
}

wt_status seq_build(int kind, const void* d_seq, uint64_t n, uint32_t sigma, uint32_t width,
                    const uint8_t* h_len, uint32_t degree, const wt_build_opts* opts,
                    wt_stream stream, wt_handle* out) {
  if (!out) return WT_ERR_INVALID_ARG;
  *out = nullptr;
  if ((!d_seq && n) || sigma == 0 || !valid_width(width)) return WT_ERR_INVALID_ARG;
  wt_status s = check_opts(opts);
  if (s != WT_OK) return s;
  if (kind == WT_KIND_MULTI && degree != 4) return WT_ERR_UNSUPPORTED;
  if (kind != WT_KIND_WM && opts && opts->tile_symbols != 0 &&
      opts->tile_symbols != (uint32_t)PASS_T)
    return WT_ERR_UNSUPPORTED;
  // the constant-time select directory packs 40-bit offsets; tile indices are 32-bit
  if (n >= ((uint64_t)1 << 40)) return WT_ERR_UNSUPPORTED;
  if ((kind == WT_KIND_WT || kind == WT_KIND_MULTI || kind == WT_KIND_HUFF) && sigma > (1u << 24))
    return WT_ERR_UNSUPPORTED;
  if (kind == WT_KIND_HUFF) return huff_async(d_seq, n, sigma, width, h_len, opts, stream, out);
  wt_struct* h = nullptr;
  s = new_handle(stream, n, sigma, &h);
  if (s != WT_OK) return s;
  h->flags = opts ? opts->flags : 0u;
  switch (kind) {
    case WT_KIND_WM: s = build_wm(d_seq, n, sigma, (int)width, opts, h); break;
    case WT_KIND_WT: s = build_wt(d_seq, n, sigma, (int)width, opts, h, false); break;
    case WT_KIND_MULTI: s = build_wt(d_seq, n, sigma, (int)width, opts, h, true); break;
    default: s = build_huff(d_seq, n, sigma, (int)width, h_len, opts, h); break;
  }
  return finish(h, s, out);
}

}  // namespace

namespace wtk {
wt_status join_build(wt_struct* h, cudaStream_t st, bool order) {
  return join_build_impl(h, st, order);
}
}  // namespace wtk

extern "C" {

wt_status wt_build(const void* d_seq, uint64_t n, uint32_t sigma, uint32_t width_bytes,
                   const wt_build_opts* opts, wt_stream stream, wt_handle* out) {
  return seq_build(WT_KIND_WT, d_seq, n, sigma, width_bytes, nullptr, 2, opts, stream, out);
}

wt_status wm_build(const void* d_seq, uint64_t n, uint32_t sigma, uint32_t width_bytes,
                   const wt_build_opts* opts, wt_stream stream, wt_handle* out) {
  return seq_build(WT_KIND_WM, d_seq, n, sigma, width_bytes, nullptr, 2, opts, stream, out);
}

wt_status wm_build_host(const void* h_seq, uint64_t n, uint32_t sigma, uint32_t width_bytes,
                        const wt_build_opts* opts, wt_stream stream, wt_handle* out) {
  if (!out) return WT_ERR_INVALID_ARG;
  *out = nullptr;
  if ((!h_seq && n) || sigma == 0 || !valid_width(width_bytes)) return WT_ERR_INVALID_ARG;
  wt_status s = check_opts(opts);
  if (s != WT_OK) return s;
  if (n >= ((uint64_t)1 << 40)) return WT_ERR_UNSUPPORTED;
  cudaStream_t cs = (cudaStream_t)stream;
  const uint64_t bytes = n * (uint64_t)width_bytes;
  void* d = nullptr;
  if (bytes) {
    // the copy goes on the device's host-copy stream, so that the copies of
    // calls on different streams follow one another at the link's full rate
    // (each while earlier builds run) instead of sharing it; the caller's
    // stream waits for it
    cudaStream_t xs = nullptr;
    cudaEvent_t copied = nullptr;
    if (host_copy_stream(&xs) != cudaSuccess) {
      cudaGetLastError();
      return WT_ERR_CUDA;
    }
    if (dmalloc(&d, bytes, xs) != cudaSuccess) {
      cudaGetLastError();
      return WT_ERR_NO_MEMORY;
    }
    const bool ok = cudaMemcpyAsync(d, h_seq, bytes, cudaMemcpyHostToDevice, xs) == cudaSuccess &&
                    cudaEventCreateWithFlags(&copied, cudaEventDisableTiming) == cudaSuccess &&
                    cudaEventRecord(copied, xs) == cudaSuccess &&
                    cudaStreamWaitEvent(cs, copied, 0) == cudaSuccess;
    if (copied) cudaEventDestroy(copied);
    if (!ok) {
      dfree(d, xs);
      cudaGetLastError();
      return WT_ERR_CUDA;
    }
  }
  s = seq_build(WT_KIND_WM, d, n, sigma, width_bytes, nullptr, 2, opts, stream, out);
  // every step of the build is on `stream`: the release follows them
  if (d) dfree(d, cs);
  return s;
}

wt_status huff_wt_build(const void* d_seq, uint64_t n, uint32_t sigma, uint32_t width_bytes,
                        const uint8_t* h_code_len, const wt_build_opts* opts, wt_stream stream,
                        wt_handle* out) {
  return seq_build(WT_KIND_HUFF, d_seq, n, sigma, width_bytes, h_code_len, 2, opts, stream, out);
}

wt_status multiary_build(const void* d_seq, uint64_t n, uint32_t sigma, uint32_t width_bytes,
                         uint32_t degree, const wt_build_opts* opts, wt_stream stream,
                         wt_handle* out) {
  return seq_build(WT_KIND_MULTI, d_seq, n, sigma, width_bytes, nullptr, degree, opts, stream,
                   out);
}

wt_status rs_build(const uint64_t* d_bits, uint64_t nbits, const wt_build_opts* opts,
                   wt_stream stream, wt_handle* out) {
  if (!out) return WT_ERR_INVALID_ARG;
  *out = nullptr;
  if (!d_bits && nbits) return WT_ERR_INVALID_ARG;
  wt_status s = check_opts(opts);
  if (s != WT_OK) return s;
  wt_struct* h = nullptr;
  s = new_handle(stream, nbits, 2, &h);
  if (s != WT_OK) return s;
  h->flags = opts ? opts->flags : 0u;
  h->kind = WT_KIND_RS;
  h->levels = h->L = 1;
  h->bpe = 1;
  h->d_bits_ro = d_bits;
  h->level_len.assign(1, nbits);
  h->level_off.assign(2, 0);
  h->level_off[1] = ((nbits + 2047) / 2048) * 32;
  if (dmalloc((void**)&h->d_zeros, 8, h->stream) != cudaSuccess) s = WT_ERR_NO_MEMORY;
  if (s == WT_OK) s = build_directories(h);
  return finish(h, s, out);
}

wt_status wt_dd_merge(const wt_handle* parts, uint32_t r, const wt_build_opts* opts,
                      wt_stream stream, wt_handle* out) {
  if (!out) return WT_ERR_INVALID_ARG;
  *out = nullptr;
  if (!parts || r == 0) return WT_ERR_INVALID_ARG;
  wt_status s = check_opts(opts);
  if (s != WT_OK) return s;
  for (uint32_t p = 0; p < r; p++)
    if (parts[p]) join_build(parts[p], parts[p]->stream, false);
  const wt_struct* p0 = parts[0];
  if (!p0 || (p0->kind != WT_KIND_WM && p0->kind != WT_KIND_WT)) return WT_ERR_INVALID_ARG;
  uint64_t n = 0;
  for (uint32_t p = 0; p < r; p++) {
    wt_struct* q = parts[p];
    if (!q || q->kind != p0->kind || q->sigma != p0->sigma || q->L != p0->L || q->bpe != 1 ||
        (q->flags & WT_FLAG_NO_DIRECTORY))
      return WT_ERR_INVALID_ARG;
    s = sync_handle(q);  // the parts' bits, directories and zero counts are final
    if (s != WT_OK) return s;
    n += q->n;
  }
  // node tables of R x 2^L entries; 40-bit offsets as for every build
  if (p0->L > 20 || ((uint64_t)r << p0->L) > ((uint64_t)1 << 26)) return WT_ERR_UNSUPPORTED;
  if (n >= ((uint64_t)1 << 40)) return WT_ERR_UNSUPPORTED;
  wt_struct* h = nullptr;
  s = new_handle(stream, n, p0->sigma, &h);
  if (s != WT_OK) return s;
  h->flags = opts ? opts->flags : 0u;
  h->kind = p0->kind;
  h->L = h->levels = p0->L;
  s = dd_merge(parts, r, h);
  return finish(h, s, out);
}

wt_status wt_access(wt_handle h, const uint64_t* d_i, uint64_t q, uint64_t* d_out,
                    wt_stream stream) {
  if (!h || (q && (!d_i || !d_out))) return WT_ERR_INVALID_ARG;
  const wt_status s = join_build(h, (cudaStream_t)stream, true);
  if (s != WT_OK) return s;
  return launch_query(h, 0, nullptr, d_i, q, d_out, (cudaStream_t)stream);
}

wt_status wt_rank(wt_handle h, const uint32_t* d_c, const uint64_t* d_i, uint64_t q,
                  uint64_t* d_out, wt_stream stream) {
  if (!h || (q && (!d_c || !d_i || !d_out))) return WT_ERR_INVALID_ARG;
  const wt_status s = join_build(h, (cudaStream_t)stream, true);
  if (s != WT_OK) return s;
  return launch_query(h, 1, d_c, d_i, q, d_out, (cudaStream_t)stream);
}

wt_status wt_select(wt_handle h, const uint32_t* d_c, const uint64_t* d_k, uint64_t q,
                    uint64_t* d_out, wt_stream stream) {
  if (!h || (q && (!d_c || !d_k || !d_out))) return WT_ERR_INVALID_ARG;
  const wt_status s = join_build(h, (cudaStream_t)stream, true);
  if (s != WT_OK) return s;
  return launch_query(h, 2, d_c, d_k, q, d_out, (cudaStream_t)stream);
}

wt_status wt_sync(wt_handle h) {
  if (!h) return WT_ERR_INVALID_ARG;
  join_build(h, h->stream, false);
  return sync_handle(h);
}

wt_status wt_export(wt_handle h, wt_export_view* out) {
  if (!h || !out) return WT_ERR_INVALID_ARG;
  join_build(h, h->stream, false);
  wt_status s = sync_handle(h);
  if (s != WT_OK) return s;
  memset(out, 0, sizeof(*out));
  out->kind = (uint32_t)h->kind;
  out->levels = h->levels;
  out->n = h->n;
  out->sigma = h->sigma;
  out->bits_per_elem = h->bpe;
  out->dir_words_per_rec = h->bpe == 2 ? 8 : 2;
  out->max_code_len = h->max_code_len;
  out->bits = h->d_bits_ro;
  out->dir = h->d_dir;
  out->samp = h->d_samp;
  out->level_len = h->level_len.data();
  out->level_off = h->level_off.data();
  out->dir_off = h->dir_off.data();
  out->samp_off = h->samp_off.data();
  out->zeros = h->zeros.data();
  out->code_len = h->code_len.empty() ? nullptr : h->code_len.data();
  out->code = h->code.empty() ? nullptr : h->code.data();
  return WT_OK;
}

wt_status wt_free(wt_handle h) {
  if (!h) return WT_ERR_INVALID_ARG;
  // memory goes back in stream order after the handle's queued work; a
  // handle of a batch that is not the last one frees nothing and waits for
  // nothing
  join_build(h, h->stream, false);
  const bool owner = !h->arena;
  free_arrays(h, true);
  // the memory is back in the pool, for allocations on any stream
  const cudaError_t e = owner ? cudaStreamSynchronize(h->stream) : cudaGetLastError();
  if (h->built) cudaEventDestroy(h->built);
  if (h->own_stream) cudaStreamDestroy(h->stream);
  delete h;
  return e == cudaSuccess ? WT_OK : WT_ERR_CUDA;
}

wt_status wt_export_select(wt_handle h, uint32_t level, uint32_t bit, wt_select_view* out) {
  if (!h || !out || bit > 3) return WT_ERR_INVALID_ARG;
  join_build(h, h->stream, false);
  wt_status s = sync_handle(h);
  if (s != WT_OK) return s;
  if (!(h->flags & WT_FLAG_SELECT_O1) || level >= h->cmeta.size() || bit > (h->bpe == 2 ? 3u : 1u))
    return WT_ERR_INVALID_ARG;
  const ClarkMeta& m = h->cmeta[level];
  memset(out, 0, sizeof(*out));
  out->nranges = m.nr[bit];
  out->nhuge = m.nh[bit];
  out->nsparse = m.ns[bit];
  out->desc = h->d_ck64 + m.desc[bit];
  out->huge = h->d_ck64 + m.huge[bit];
  out->sub = h->d_ck32 + m.sub[bit];
  out->sparse = h->d_ck32 + m.sparse[bit];
  return WT_OK;
}

uint64_t wt_symbol_levels(wt_handle h) {
  if (!h) return 0;
  join_build(h, h->stream, false);
  uint64_t s = 0;
  for (uint64_t v : h->level_len) s += v;
  return h->bpe == 2 ? s * 2 : s;
}

const char* wt_status_str(wt_status s) {
  switch (s) {
    case WT_OK: return "ok";
    case WT_ERR_INVALID_ARG: return "invalid argument";
    case WT_ERR_SYMBOL_GE_SIGMA: return "symbol >= sigma";
    case WT_ERR_NO_MEMORY: return "out of device memory";
    case WT_ERR_CUDA: return "CUDA error";
    case WT_ERR_TIMEOUT: return "not finished yet";
    case WT_ERR_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

wt_status wt_memcpy_d2h(void* h_dst, const void* d_src, uint64_t bytes) {
  if (!bytes) return WT_OK;
  if (!h_dst || !d_src) return WT_ERR_INVALID_ARG;
  return cudaMemcpy(h_dst, d_src, bytes, cudaMemcpyDeviceToHost) == cudaSuccess ? WT_OK
                                                                                : WT_ERR_CUDA;
}

void wt_prof_enable(int on) {
  Prof& p = prof();
  std::lock_guard<std::mutex> g(p.mu);
  p.on = on != 0;
  p.launches = 0;
  p.pass_launches = 0;
  for (cudaEvent_t e : p.ev) cudaEventDestroy(e);
  p.ev.clear();
}

wt_status wt_prof_read(uint64_t* launches, uint64_t* pass_launches, double* pass_ms) {
  Prof& p = prof();
  std::lock_guard<std::mutex> g(p.mu);
  double ms = 0;
  wt_status s = WT_OK;
  for (size_t i = 0; i + 1 < p.ev.size(); i += 2) {
    if (cudaEventSynchronize(p.ev[i + 1]) != cudaSuccess) s = WT_ERR_CUDA;
    float f = 0;
    if (cudaEventElapsedTime(&f, p.ev[i], p.ev[i + 1]) == cudaSuccess) ms += f;
  }
  if (launches) *launches = p.launches;
  if (pass_launches) *pass_launches = p.pass_launches;
  if (pass_ms) *pass_ms = ms;
  for (cudaEvent_t e : p.ev) cudaEventDestroy(e);
  p.ev.clear();
  p.launches = 0;
  p.pass_launches = 0;
  return s;
}

uint32_t wt_huffman_lengths(const uint64_t* h_hist, uint32_t sigma, uint32_t cap,
                            uint8_t* h_len) {
  // the radix path packs (weight << 24 | symbol): the alphabet limit of
  // huff_wt_build keeps every symbol within 24 bits
  if (!h_hist || !h_len || cap == 0 || cap > 64 || sigma > (1u << 24)) return 0;
  return huffman_lengths(h_hist, sigma, cap, h_len);
}

void wt_canonical_codes(const uint8_t* h_len, uint32_t sigma, uint32_t* h_code) {
  if (!h_len || !h_code) return;
  canonical_codes(h_len, sigma, h_code);
}

}  // extern "C"
