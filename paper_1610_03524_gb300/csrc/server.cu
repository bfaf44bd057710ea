// server.cu -- a serving loop over the batched build and the multi-structure
// query kernel: requests arrive at any time from any thread; a build worker
// admits pending builds under a device-memory budget and builds all admitted
// ones with one batched build; a query worker gathers every pending query
// request whose structures are ready into one launch (continuous batching).
// Host-side orchestration only: every computational step runs in the
// library's kernels (wm_batch_build, wt_query_multi).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "wt_host.h"

namespace {

uint64_t now_ns() {
  return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

enum ReqKind : uint32_t { REQ_BUILD = 1, REQ_QUERY = 2 };

struct Request {
  uint64_t id = 0;
  uint32_t kind = 0;
  uint64_t submit_ns = 0, done_ns = 0;
  bool done = false;
  wt_status status = WT_OK;
  // build
  std::vector<uint8_t> seq;
  uint64_t n = 0;
  uint32_t sigma = 0, width = 0;
  uint64_t need = 0;  // bytes the build holds while it runs and after
  // queries
  uint64_t q = 0;
  std::vector<uint64_t> sid, x, out;
  std::vector<uint64_t> uniq;  // the distinct structures the queries name
  std::vector<uint8_t> op;
  std::vector<uint32_t> c;
};

// one batched build's shared allocation, released with its last structure
struct BatchRec {
  uint64_t bytes = 0;
  int live = 0;
};

struct Structure {
  wt_handle h = nullptr;
  std::shared_ptr<BatchRec> batch;
  bool ready = false;
  bool failed = false;
  int inflight = 0;  // query launches using the handle
};

// Host buffer in page-locked memory, grown on demand.
struct Pinned {
  void* p = nullptr;
  size_t cap = 0;
  ~Pinned() {
    if (p) cudaFreeHost(p);
  }
  bool reserve(size_t n) {
    if (n <= cap) return true;
    if (p) cudaFreeHost(p);
    p = nullptr;
    cap = 0;
    size_t c = std::max<size_t>(n, 1 << 20);
    if (cudaHostAlloc(&p, c, cudaHostAllocDefault) != cudaSuccess) return false;
    cap = c;
    return true;
  }
};

}  // namespace

struct wt_server_s {
  wt_server_opts opts{};
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_build, cv_query, cv_done;
  bool stop = false;
  uint64_t next_id = 1;
  std::map<uint64_t, std::shared_ptr<Request>> reqs;
  std::deque<std::shared_ptr<Request>> pend_build, pend_query;
  std::map<uint64_t, Structure> structs;  // by build request id
  uint64_t used = 0;                      // resident bytes + bytes held by running builds
  uint64_t build_gen = 0;                 // bumped on a new build or memory given back
  uint64_t n_build_batches = 0, n_query_launches = 0;
  cudaStream_t s_build = nullptr, s_query = nullptr;
  std::thread t_build, t_query;

  void build_loop();
  void query_loop();
  void finish(const std::shared_ptr<Request>& r, wt_status s) {
    r->status = s;
    r->done_ns = now_ns();
    r->done = true;
  }
};

namespace {

// device bytes a build of (n, sigma, width) holds: the structure, plus while
// it runs the device copy of the sequence, its intermediate sequences and its
// tiles' digit counts (1 KB per 4096-symbol tile)
uint64_t build_need(uint64_t n, uint32_t sigma, uint32_t width) {
  return wtk::wm_resident_bytes(n, sigma) + n * (uint64_t)width + 2 * n * 2 + n / 4 + 8192;
}

// bytes a batched build holds besides its sequences' needs (tile counts,
// tables, directory scratch)
constexpr uint64_t BATCH_OVERHEAD = 16ull << 20;

}  // namespace

void wt_server_s::build_loop() {
  cudaSetDevice(device);
  Pinned pin;
  for (;;) {
    std::vector<std::shared_ptr<Request>> take;
    {
      std::unique_lock<std::mutex> lk(mu);
      cv_build.wait(lk, [&] { return stop || !pend_build.empty(); });
      if (stop) return;
      // admission in arrival order while the budget allows
      uint64_t add = BATCH_OVERHEAD;
      while (!pend_build.empty() && take.size() < opts.max_batch_builds) {
        auto& r = pend_build.front();
        if (r->need + BATCH_OVERHEAD > opts.budget_bytes) {
          finish(r, WT_ERR_NO_MEMORY);
          structs[r->id].failed = true;
          pend_build.pop_front();
          cv_done.notify_all();
          continue;
        }
        if (used + add + r->need > opts.budget_bytes) break;
        add += r->need;
        take.push_back(r);
        pend_build.pop_front();
      }
      if (take.empty()) {
        // nothing admissible: wait for a new build or for memory given back
        const uint64_t g0 = build_gen;
        cv_build.wait(lk, [&] { return stop || build_gen != g0; });
        if (stop) return;
        continue;
      }
      used += add;
    }
    // one batched build of every admitted sequence
    const uint32_t m = (uint32_t)take.size();
    uint64_t in_bytes = 0;
    std::vector<uint64_t> off(m);
    for (uint32_t i = 0; i < m; i++) {
      off[i] = in_bytes;
      in_bytes += (take[i]->seq.size() + 255) / 256 * 256;
    }
    wt_status s = WT_OK;
    void* d_in = nullptr;
    if (!pin.reserve(std::max<uint64_t>(in_bytes, 1))) s = WT_ERR_NO_MEMORY;
    if (s == WT_OK && wtk::dmalloc(&d_in, std::max<uint64_t>(in_bytes, 1), s_build) != cudaSuccess)
      s = WT_ERR_NO_MEMORY;
    std::vector<wt_batch_item> items(m);
    std::vector<wt_handle> hs(m, nullptr);
    if (s == WT_OK) {
      for (uint32_t i = 0; i < m; i++)
        if (!take[i]->seq.empty())
          memcpy((uint8_t*)pin.p + off[i], take[i]->seq.data(), take[i]->seq.size());
      if (in_bytes &&
          cudaMemcpyAsync(d_in, pin.p, in_bytes, cudaMemcpyHostToDevice, s_build) != cudaSuccess)
        s = WT_ERR_CUDA;
      for (uint32_t i = 0; i < m; i++) {
        items[i].d_seq = (uint8_t*)d_in + off[i];
        items[i].n = take[i]->n;
        items[i].sigma = take[i]->sigma;
        items[i].width_bytes = take[i]->width;
      }
    }
    if (s == WT_OK) s = wm_batch_build(items.data(), m, nullptr, s_build, hs.data());
    if (cudaStreamSynchronize(s_build) != cudaSuccess && s == WT_OK) s = WT_ERR_CUDA;
    if (d_in) wtk::dfree(d_in, s_build);
    cudaStreamSynchronize(s_build);
    std::vector<wt_status> st(m, s);
    if (s == WT_OK) wtk::batch_status(hs.data(), m, st.data());
    auto rec = std::make_shared<BatchRec>();
    uint64_t arena = 0;
    if (s == WT_OK && m) arena = hs[0]->arena ? hs[0]->arena->bytes : 0;
    {
      std::lock_guard<std::mutex> lk(mu);
      uint64_t need = BATCH_OVERHEAD;
      for (auto& r : take) need += r->need;
      used -= need;
      build_gen++;
      if (s == WT_OK) {
        used += arena;
        rec->bytes = arena;
        rec->live = (int)m;
      }
      for (uint32_t i = 0; i < m; i++) {
        Structure& S = structs[take[i]->id];
        if (s == WT_OK) {
          S.h = hs[i];
          S.batch = rec;
        }
        S.ready = st[i] == WT_OK;
        S.failed = st[i] != WT_OK;
        finish(take[i], st[i]);
      }
      n_build_batches++;
    }
    cv_done.notify_all();
    cv_query.notify_all();
  }
}

void wt_server_s::query_loop() {
  cudaSetDevice(device);
  Pinned pin_in, pin_out;
  void* d_buf = nullptr;
  size_t d_cap = 0;
  std::vector<uint32_t> dense;
  for (;;) {
    std::vector<std::shared_ptr<Request>> take;
    std::vector<wt_handle> tab;
    std::map<uint64_t, uint32_t> slot;  // structure id -> table index
    std::vector<std::shared_ptr<Request>> failed;
    {
      std::unique_lock<std::mutex> lk(mu);
      for (;;) {
        if (stop) {
          if (d_buf) {
            wtk::dfree(d_buf, s_query);
            cudaStreamSynchronize(s_query);
          }
          return;
        }
        // every pending request whose structures are all built (or failed)
        uint64_t qtot = 0;
        for (auto it = pend_query.begin(); it != pend_query.end();) {
          auto& r = *it;
          bool ready = true;
          for (uint64_t id : r->uniq) {
            auto f = structs.find(id);
            if (f != structs.end() && !f->second.ready && !f->second.failed) {
              ready = false;
              break;
            }
          }
          if (!ready || (qtot && qtot + r->q > opts.max_batch_queries)) {
            ++it;
            continue;
          }
          qtot += r->q;
          take.push_back(r);
          it = pend_query.erase(it);
        }
        if (!take.empty()) break;
        cv_query.wait(lk);
      }
      for (auto& r : take)
        for (uint64_t id : r->uniq) {
          auto f = structs.find(id);
          if (f == structs.end() || !f->second.ready) continue;
          if (slot.emplace(id, (uint32_t)tab.size()).second) tab.push_back(f->second.h);
        }
      // the handles stay valid: wt_server_release waits for this launch
      for (auto& kv : slot) structs[kv.first].inflight++;
    }
    uint64_t q = 0;
    for (auto& r : take) q += r->q;
    // pack (sid, op, c, x) into one host staging buffer
    const size_t b_sid = 0, b_op = b_sid + 4 * q, b_c = (b_op + q + 7) / 8 * 8, b_x = b_c + 4 * q,
                 b_end = b_x + 8 * q, b_out = (b_end + 255) / 256 * 256, d_need = b_out + 8 * q;
    wt_status s = WT_OK;
    if (!pin_in.reserve(b_end) || !pin_out.reserve(8 * q)) s = WT_ERR_NO_MEMORY;
    if (s == WT_OK && d_cap < d_need) {
      if (d_buf) wtk::dfree(d_buf, s_query);
      d_buf = nullptr;
      d_cap = 0;
      if (wtk::dmalloc(&d_buf, d_need, s_query) != cudaSuccess) s = WT_ERR_NO_MEMORY;
      else d_cap = d_need;
    }
    if (s == WT_OK) {
      uint8_t* P = (uint8_t*)pin_in.p;
      uint32_t* hsid = (uint32_t*)(P + b_sid);
      uint8_t* hop = P + b_op;
      uint32_t* hc = (uint32_t*)(P + b_c);
      uint64_t* hx = (uint64_t*)(P + b_x);
      // structure id -> table index in a flat array over the ids in use
      // (ids are small consecutive request numbers)
      const uint64_t top = slot.empty() ? 0 : slot.rbegin()->first + 1;
      dense.assign(top, 0xffffffffu);
      for (auto& kv : slot) dense[kv.first] = kv.second;
      uint64_t k = 0;
      for (auto& r : take) {
        const uint64_t* rs = r->sid.data();
        for (uint64_t i = 0; i < r->q; i++, k++)
          hsid[k] = rs[i] < top ? dense[rs[i]] : 0xffffffffu;  // unknown -> UINT64_MAX
        memcpy(hop + (k - r->q), r->op.data(), r->q);
        memcpy(hc + (k - r->q), r->c.data(), 4 * r->q);
        memcpy(hx + (k - r->q), r->x.data(), 8 * r->q);
      }
      uint8_t* D = (uint8_t*)d_buf;
      if (cudaMemcpyAsync(D, P, b_end, cudaMemcpyHostToDevice, s_query) != cudaSuccess)
        s = WT_ERR_CUDA;
      if (s == WT_OK)
        s = wt_query_multi(tab.data(), (uint32_t)tab.size(), (const uint32_t*)(D + b_sid), D + b_op,
                           (const uint32_t*)(D + b_c), (const uint64_t*)(D + b_x), q,
                           (uint64_t*)(D + b_out), s_query);
      if (s == WT_OK && cudaMemcpyAsync(pin_out.p, D + b_out, 8 * q, cudaMemcpyDeviceToHost,
                                        s_query) != cudaSuccess)
        s = WT_ERR_CUDA;
      if (cudaStreamSynchronize(s_query) != cudaSuccess && s == WT_OK) s = WT_ERR_CUDA;
    }
    {
      std::lock_guard<std::mutex> lk(mu);
      for (auto& kv : slot) structs[kv.first].inflight--;
      uint64_t k = 0;
      for (auto& r : take) {
        if (s == WT_OK) {
          r->out.assign((uint64_t*)pin_out.p + k, (uint64_t*)pin_out.p + k + r->q);
        }
        k += r->q;
        finish(r, s);
      }
      n_query_launches++;
    }
    cv_done.notify_all();
  }
}

extern "C" {

wt_status wt_server_create(const wt_server_opts* opts, wt_server* out) {
  if (!out || !opts || opts->budget_bytes == 0) return WT_ERR_INVALID_ARG;
  *out = nullptr;
  wt_server_s* s = new (std::nothrow) wt_server_s();
  if (!s) return WT_ERR_NO_MEMORY;
  s->opts = *opts;
  if (!s->opts.max_batch_builds) s->opts.max_batch_builds = 4096;
  if (!s->opts.max_batch_queries) s->opts.max_batch_queries = 1u << 22;
  cudaGetDevice(&s->device);
  // queries on the highest-priority stream: when both streams have work
  // waiting, the query kernels' blocks are scheduled first
  int prio_least = 0, prio_greatest = 0;
  cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest);
  if (cudaStreamCreateWithFlags(&s->s_build, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithPriority(&s->s_query, cudaStreamNonBlocking, prio_greatest) !=
          cudaSuccess) {
    if (s->s_build) cudaStreamDestroy(s->s_build);
    delete s;
    return WT_ERR_CUDA;
  }
  s->t_build = std::thread([s] { s->build_loop(); });
  s->t_query = std::thread([s] { s->query_loop(); });
  *out = s;
  return WT_OK;
}

wt_status wt_server_submit_build(wt_server s, const void* h_seq, uint64_t n, uint32_t sigma,
                                 uint32_t width_bytes, uint64_t* req) {
  if (!s || !req || (!h_seq && n) || sigma == 0) return WT_ERR_INVALID_ARG;
  if (width_bytes != 1 && width_bytes != 2 && width_bytes != 4) return WT_ERR_INVALID_ARG;
  auto r = std::make_shared<Request>();
  r->kind = REQ_BUILD;
  r->n = n;
  r->sigma = sigma;
  r->width = width_bytes;
  r->need = build_need(n, sigma, width_bytes);
  r->seq.assign((const uint8_t*)h_seq, (const uint8_t*)h_seq + n * width_bytes);
  r->submit_ns = now_ns();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    r->id = s->next_id++;
    s->reqs[r->id] = r;
    s->structs[r->id] = Structure{};
    s->pend_build.push_back(r);
    s->build_gen++;
  }
  *req = r->id;
  s->cv_build.notify_one();
  return WT_OK;
}

wt_status wt_server_submit_queries(wt_server s, uint64_t q, const uint64_t* h_sid,
                                   const uint8_t* h_op, const uint32_t* h_c, const uint64_t* h_x,
                                   uint64_t* req) {
  if (!s || !req || (q && (!h_sid || !h_op || !h_c || !h_x))) return WT_ERR_INVALID_ARG;
  auto r = std::make_shared<Request>();
  r->kind = REQ_QUERY;
  r->q = q;
  r->sid.assign(h_sid, h_sid + q);
  r->op.assign(h_op, h_op + q);
  r->c.assign(h_c, h_c + q);
  r->x.assign(h_x, h_x + q);
  r->submit_ns = now_ns();
  // the distinct structures named (a flat marker over the ids when they are
  // small, as request ids are; else a sort)
  {
    uint64_t mx = 0;
    for (uint64_t i = 0; i < q; i++) mx = std::max(mx, h_sid[i]);
    if (mx < (1ull << 24)) {
      std::vector<uint8_t> seen(mx + 1, 0);
      for (uint64_t i = 0; i < q; i++)
        if (!seen[h_sid[i]]) {
          seen[h_sid[i]] = 1;
          r->uniq.push_back(h_sid[i]);
        }
    } else {
      r->uniq = r->sid;
      std::sort(r->uniq.begin(), r->uniq.end());
      r->uniq.erase(std::unique(r->uniq.begin(), r->uniq.end()), r->uniq.end());
    }
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    r->id = s->next_id++;
    s->reqs[r->id] = r;
    if (q == 0) {
      s->finish(r, WT_OK);
    } else {
      s->pend_query.push_back(r);
    }
  }
  *req = r->id;
  s->cv_query.notify_one();
  s->cv_done.notify_all();
  return WT_OK;
}

wt_status wt_server_poll(wt_server s, uint64_t req, int wait, uint64_t* h_out,
                         wt_request_info* info) {
  if (!s) return WT_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto f = s->reqs.find(req);
  if (f == s->reqs.end()) return WT_ERR_INVALID_ARG;
  auto r = f->second;
  if (!r->done) {
    if (!wait) {
      if (info) {
        memset(info, 0, sizeof(*info));
        info->kind = r->kind;
        info->submit_ns = r->submit_ns;
      }
      return WT_ERR_TIMEOUT;  // not finished yet
    }
    s->cv_done.wait(lk, [&] { return r->done; });
  }
  if (info) {
    info->status = r->status;
    info->kind = r->kind;
    info->submit_ns = r->submit_ns;
    info->done_ns = r->done_ns;
  }
  if (r->kind == REQ_QUERY && h_out && r->status == WT_OK && r->q)
    memcpy(h_out, r->out.data(), 8 * r->q);
  // a finished query request is forgotten once read
  if (r->kind == REQ_QUERY) s->reqs.erase(f);
  return WT_OK;
}

wt_status wt_server_handle(wt_server s, uint64_t sid, wt_handle* out) {
  if (!s || !out) return WT_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto f = s->structs.find(sid);
  if (f == s->structs.end() || !f->second.ready) return WT_ERR_INVALID_ARG;
  *out = f->second.h;
  return WT_OK;
}

wt_status wt_server_release(wt_server s, uint64_t sid) {
  if (!s) return WT_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto f = s->structs.find(sid);
  if (f == s->structs.end()) return WT_ERR_INVALID_ARG;
  if (!f->second.ready && !f->second.failed) return WT_ERR_INVALID_ARG;  // still building
  // wait for any query launch that uses it
  s->cv_done.wait(lk, [&] {
    auto g = s->structs.find(sid);
    return g == s->structs.end() || g->second.inflight == 0;
  });
  f = s->structs.find(sid);
  if (f == s->structs.end()) return WT_ERR_INVALID_ARG;
  Structure S = f->second;
  s->structs.erase(f);
  s->reqs.erase(sid);
  if (S.batch && --S.batch->live == 0) s->used -= S.batch->bytes;
  s->build_gen++;
  lk.unlock();
  if (S.h) wt_free(S.h);
  s->cv_build.notify_all();
  return WT_OK;
}

wt_status wt_server_stats(wt_server s, wt_server_stats_t* out) {
  if (!s || !out) return WT_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  out->used_bytes = s->used;
  out->budget_bytes = s->opts.budget_bytes;
  out->build_batches = s->n_build_batches;
  out->query_launches = s->n_query_launches;
  out->pending_builds = s->pend_build.size();
  out->pending_queries = s->pend_query.size();
  out->structures = 0;
  for (auto& kv : s->structs) out->structures += kv.second.ready ? 1 : 0;
  return WT_OK;
}

wt_status wt_server_destroy(wt_server s) {
  if (!s) return WT_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_build.notify_all();
  s->cv_query.notify_all();
  s->cv_done.notify_all();
  if (s->t_build.joinable()) s->t_build.join();
  if (s->t_query.joinable()) s->t_query.join();
  {
    // requests still waiting end with an error (pollers are woken)
    std::lock_guard<std::mutex> lk(s->mu);
    for (auto& kv : s->reqs)
      if (!kv.second->done) s->finish(kv.second, WT_ERR_INVALID_ARG);
  }
  s->cv_done.notify_all();
  for (auto& kv : s->structs)
    if (kv.second.h) wt_free(kv.second.h);
  cudaStreamDestroy(s->s_build);
  cudaStreamDestroy(s->s_query);
  delete s;
  return WT_OK;
}

}  // extern "C"
