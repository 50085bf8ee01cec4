// hc_server.cu -- served search: a request loop with continuous batching.
//
// Texts are registered once and stay resident in device memory.  Requests
// (a pattern against one resident text) are queued by any host thread; one
// worker thread of the server assembles batches from the queue and runs each
// as a batched search (device preprocessing, persistent scan, emit) on one of
// `max_inflight` streams, so that requests arriving while earlier batches are
// on the GPU are launched as soon as a stream and memory are free and their
// work overlaps with the earlier batches' on the device.
//
// Admission: the device bytes of resident texts plus those of every admitted
// request (filter, pattern, launch tables, scan workspace) stay within
// `mem_limit`; a request waits in the queue until enough admitted memory has
// been released by completed batches.  Queue order is kept (a request that
// does not fit blocks the ones behind it), so no request is starved.
//
// Results: the emit kernel writes counts and positions directly into pinned
// host memory mapped into the device's address space (on a Grace-Blackwell
// node, over the coherent chip-to-chip link), so a batch needs no
// device-to-host copy: once its completion event has fired the worker copies
// each request's positions into the request's own host buffer and publishes
// it to hc_server_poll.
//
// Plain mode (comparison): each request is preprocessed on the host and runs
// as one plain search launch (scan and emit kernels of hc_search_async), the
// requests of one assembly still sharing one stream and one completion event.
// In the batched mode the same single-search launches serve a batch's lone
// request and, in batches of at most 16, the requests with m = q (the dense
// single-search kernel, one q-gram per window), unless batch_only is set.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "hc_batch_internal.h"

namespace hc {
namespace {

constexpr uint32_t kServerMagic = 0x48435356u;  // "HCSV"
constexpr size_t kAlign = 256;
constexpr size_t kSoloDenseMax = 16;  // batches up to this size route m = q requests to single searches
constexpr size_t kSoloMax = 3;        // batches up to this size run every request as a single search

size_t align_up(size_t v, size_t a = kAlign) { return (v + a - 1) / a * a; }

uint64_t now_ns() {
  return static_cast<uint64_t>(std::chrono::duration_cast<std::chrono::nanoseconds>(
                                   std::chrono::steady_clock::now().time_since_epoch())
                                   .count());
}

struct Text {
  const uint8_t* y = nullptr;  // device
  uint64_t n = 0;
  double sigma = 0;
  bool owned = false;
};

struct Req {
  uint64_t id = 0;
  uint32_t text = 0;
  const uint8_t* y = nullptr;
  uint64_t n = 0;
  std::vector<uint8_t> x;
  QueryParams p;
  uint64_t cap = 0;
  // shared-memory layout and admitted device bytes (an estimate from its
  // one-query plan; the batch it joins is planned again at launch)
  BatchLayout lay{};
  uint64_t dev_bytes = 0;
  // outcome
  uint64_t submit_ns = 0, start_ns = 0, done_ns = 0;
  uint64_t batch = 0;
  uint32_t batch_size = 0;
  int status = HC_OK;
  uint64_t count = 0;
  std::vector<uint64_t> pos;
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  bool busy = false;
  std::vector<Req*> reqs;
  std::vector<size_t> pos_off;  // per request: first entry of its positions in the result arena
  uint8_t* stage = nullptr;     // pinned host staging of the batched launch tables
  size_t stage_cap = 0;
  uint8_t* stage_plain = nullptr;  // ... and of the single-search filters (a separate
  size_t stage_plain_cap = 0;      // buffer: both copies may be in flight at once)
  uint8_t* res = nullptr;       // mapped pinned host memory: counts, then positions
  uint64_t* res_dev = nullptr;  // its device address
  size_t res_cap = 0;           // bytes
  unsigned int* status = nullptr;  // pinned copy of the device status word after the batch
  std::vector<void*> retired;      // outgrown pinned buffers (freed with the server)
  uint64_t admitted = 0;
  uint64_t batch = 0;
};

struct ServerStats {
  uint64_t submitted = 0, completed = 0, batches = 0, rejected = 0, admission_waits = 0;
  uint64_t max_batch = 0, peak_inflight_bytes = 0;
};

}  // namespace

struct Server {
  uint32_t magic = kServerMagic;
  int dev = 0;
  hc_server_config cfg{};
  const Tuner* tuner = nullptr;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Text> texts;
  uint64_t text_bytes = 0;
  std::deque<Req*> pending;
  uint64_t pending_text = 0;                // text bytes of the queued requests
  std::unordered_map<uint64_t, Req*> done;  // completed, not yet released
  std::deque<uint64_t> done_queue;          // completed, not yet polled
  std::vector<Slot> slots;
  uint64_t next_id = 1, inflight_bytes = 0, next_batch = 1, blocked_id = 0;
  bool stop = false;
  int fatal = HC_OK;
  ServerStats st;
  std::thread worker;

  uint64_t request_limit() const { return cfg.mem_limit > text_bytes ? cfg.mem_limit - text_bytes : 0; }
  void run();
  std::vector<Req*> take_batch();
  int launch(Slot& s, std::vector<Req*>& b);
  int launch_batched(Slot& s, const std::vector<size_t>& which);
  int launch_plain(Slot& s, const std::vector<size_t>& which);
  void finish(Slot& s, cudaError_t q);
  void fail(std::vector<Req*>& b, int status);
};

namespace {

Server* as_server(const hc_server* s) {
  auto* p = reinterpret_cast<Server*>(const_cast<hc_server*>(s));
  return (p != nullptr && p->magic == kServerMagic) ? p : nullptr;
}

bool layout_fits(const BatchLayout& lay, size_t smem_optin) {
  const size_t f = (lay.f_bytes + 15u) & ~15u;
  const size_t smem = f + lay.x_bytes + size_t(kSlots) * kThreads * 4 + size_t(kWarps) * lay.ring_bytes;
  return smem + 2048 <= smem_optin;
}

BatchLayout layout_max(const BatchLayout& a, const BatchLayout& b) {
  return {std::max(a.f_bytes, b.f_bytes), std::max(a.x_bytes, b.x_bytes), std::max(a.ring_bytes, b.ring_bytes)};
}

// Grows a pinned host buffer to at least `need` bytes (by half again, in
// 64 KiB units).  The old buffer is not freed here: cudaFreeHost waits for
// the whole device, which would stall every request in flight; it goes to
// `retired`, freed when the server is destroyed (growth by half keeps the
// retired buffers below twice the final size).
template <typename T>
int grow_pinned(T** p, size_t* cap, size_t need, unsigned flags, const char* what,
                std::vector<void*>* retired) {
  if (need <= *cap && *p != nullptr) return HC_OK;
  if (*p != nullptr) retired->push_back(*p);
  *p = nullptr;
  *cap = 0;
  const size_t n = align_up(std::max<size_t>(need + need / 2, 1 << 16), 1 << 16);
  void* v = nullptr;
  cudaError_t e = cudaHostAlloc(&v, n, flags);
  if (e != cudaSuccess) return cuda_error(e, what);
  *p = static_cast<T*>(v);
  *cap = n;
  return HC_OK;
}

}  // namespace

// Text bytes the next batch may take: max_batch_bytes while the queue is
// short, so that a request that arrives behind a batch waits for little text;
// an equal share of the queued text per stream once more than max_inflight
// batches of that size wait, so that a backlog drains in few large batches
// (a request in a backlog waits for the text ahead of it whatever the cut).
static uint64_t batch_text_bound(uint64_t max_batch_bytes, uint64_t queued_text, int streams) {
  return std::max<uint64_t>(max_batch_bytes, queued_text / static_cast<uint64_t>(std::max(streams, 1)));
}

// Takes the next batch from the queue (lock held): queue order, at most
// max_batch requests and batch_text_bound bytes of text (a lone larger
// request still forms a batch), admitted memory within the limit, the
// combined shared-memory layout within one CTA.
std::vector<Req*> Server::take_batch() {
  std::vector<Req*> b;
  BatchLayout lay{};
  const size_t optin = device_info(dev).smem_optin;
  const uint64_t bound = batch_text_bound(cfg.max_batch_bytes, pending_text, cfg.max_inflight);
  uint64_t text_bytes = 0;  // of the batch
  while (!pending.empty() && b.size() < static_cast<size_t>(cfg.max_batch)) {
    Req* r = pending.front();
    if (!b.empty() && text_bytes + r->n > bound) break;
    if (r->dev_bytes > request_limit()) {  // can never be admitted
      pending.pop_front();
      pending_text -= r->n;
      r->status = HC_ERR_ADMISSION;
      r->done_ns = now_ns();
      done[r->id] = r;
      done_queue.push_back(r->id);
      st.rejected++;
      st.completed++;
      cv_done.notify_all();
      continue;
    }
    if (inflight_bytes + r->dev_bytes > request_limit()) {
      if (r->id != blocked_id) st.admission_waits++;  // requests that had to wait for memory
      blocked_id = r->id;
      break;
    }
    const BatchLayout nl = layout_max(lay, r->lay);
    if (!b.empty() && !layout_fits(nl, optin)) break;
    lay = nl;
    b.push_back(r);
    text_bytes += r->n;
    inflight_bytes += r->dev_bytes;
    pending.pop_front();
    pending_text -= r->n;
  }
  st.peak_inflight_bytes = std::max(st.peak_inflight_bytes, inflight_bytes);
  return b;
}

void Server::fail(std::vector<Req*>& b, int status) {
  const uint64_t t = now_ns();
  std::lock_guard<std::mutex> lock(mu);
  for (Req* r : b) {
    r->status = status;
    r->done_ns = t;
    inflight_bytes -= r->dev_bytes;
    done[r->id] = r;
    done_queue.push_back(r->id);
    st.completed++;
  }
  cv_done.notify_all();
}

// Device block of one batch (stream-ordered, from the library's pool):
// [counter | args | tiles | emit tiles | patterns | filters | workspace].
int Server::launch(Slot& s, std::vector<Req*>& b) {
  const size_t nq = b.size();
  // result arena: counts, then each request's positions
  s.pos_off.assign(nq, 0);
  size_t entries = nq;
  for (size_t i = 0; i < nq; ++i) {
    s.pos_off[i] = entries;
    entries += b[i]->cap;
  }
  int rc = grow_pinned(&s.res, &s.res_cap, entries * 8, cudaHostAllocMapped | cudaHostAllocPortable,
                       "cudaHostAlloc(server results)", &s.retired);
  if (rc == HC_OK) {
    void* d = nullptr;
    cudaError_t e = cudaHostGetDevicePointer(&d, s.res, 0);
    if (e != cudaSuccess) rc = cuda_error(e, "cudaHostGetDevicePointer(server results)");
    s.res_dev = static_cast<uint64_t*>(d);
  }
  if (rc != HC_OK) return rc;
  // routing: a batch of at most kSoloMax requests runs the single-search
  // kernels (at low load the batched kernels' table setup and three launches
  // only add latency); in a batch of at most kSoloDenseMax, m = q requests
  // (one q-gram per window: the dense single-search kernel) run the
  // single-search kernels, and so does a batch's lone request; the rest run
  // the batched kernels.  In a large batch (a backlog) the per-launch host
  // cost of the single searches would cost more than the dense kernel saves.
  std::vector<size_t> solo, batched;
  const bool route_dense = !cfg.batch_only && nq <= kSoloDenseMax;
  const bool all_solo = !cfg.batch_only && nq <= kSoloMax;
  for (size_t i = 0; i < nq; ++i) {
    const bool dense = b[i]->x.size() == static_cast<size_t>(b[i]->p.q);
    if (cfg.plain || all_solo || (route_dense && dense)) solo.push_back(i);
    else batched.push_back(i);
  }
  if (!cfg.batch_only && batched.size() == 1) {
    solo.push_back(batched[0]);
    batched.clear();
  }
  if (!batched.empty()) rc = launch_batched(s, batched);
  if (rc == HC_OK && !solo.empty()) rc = launch_plain(s, solo);
  cudaError_t e;
  if (rc == HC_OK) {
    e = cudaMemcpyAsync(s.status, status_word(), sizeof(unsigned int), cudaMemcpyDeviceToHost, s.stream);
    if (e != cudaSuccess) rc = cuda_error(e, "cudaMemcpyAsync(server status)");
  }
  if (rc != HC_OK) return rc;
  e = cudaEventRecord(s.done, s.stream);
  if (e != cudaSuccess) return cuda_error(e, "cudaEventRecord(server)");
  return HC_OK;
}

// The batched kernels over requests `which` of the slot (indices into its
// requests and result arena).
int Server::launch_batched(Slot& s, const std::vector<size_t>& which) {
  const size_t nq = which.size();
  int rc = HC_OK;
  cudaError_t e;
  // plan first (patterns at placeholder addresses, patched below), then
  // one device block sized from the plan:
  // [counter | args | tiles | emit tiles | patterns | filters | workspace]
  static const uint64_t placeholder[2] = {0, 0};
  BatchPlan plan;
  plan.args.reserve(nq);
  unsigned long long total_text = 0;
  for (size_t w : which) total_text += s.reqs[w]->n;
  const unsigned long long rec_bytes = record_bytes_for(total_text, dev);
  std::vector<size_t> xoff(nq);
  size_t xbytes = 0;
  for (size_t i = 0; i < nq && rc == HC_OK; ++i) {
    Req* r = s.reqs[which[i]];
    hc_batch_query Q{};
    Q.x_dev = reinterpret_cast<const uint8_t*>(placeholder);
    Q.m = r->x.size();
    Q.y_dev = r->y;
    Q.n = r->n;
    Q.q = r->p.q;
    Q.alpha = r->p.alpha;
    Q.pos_dev = r->cap ? reinterpret_cast<uint64_t*>(s.res_dev + s.pos_off[which[i]]) : nullptr;
    Q.cap = r->cap;
    Q.count_dev = reinterpret_cast<uint64_t*>(s.res_dev + which[i]);
    Q.lane_bytes = r->p.lane_bytes;
    Q.mode = r->p.mode;
    rc = plan_add_query(plan, Q, i, r->p, rec_bytes, "hc_server");
    xoff[i] = xbytes;
    xbytes += align_up(r->x.size(), 16);
  }
  if (rc == HC_OK) rc = plan_finish(plan, dev, "hc_server");
  if (rc == HC_OK) rc = batch_grids(plan, dev);
  if (rc != HC_OK) return rc;
  const size_t o_args = kAlign;
  const size_t o_tiles = o_args + align_up(nq * sizeof(SearchArgs));
  const size_t o_etiles = o_tiles + align_up(plan.tiles.size() * sizeof(BatchTile));
  const size_t o_x = o_etiles + align_up(plan.etiles.size() * sizeof(EmitTile));
  const size_t table_end = o_x + align_up(xbytes);
  const size_t o_f = table_end;
  const size_t o_ws = o_f + align_up(plan.filter_words * 4);
  const size_t total = o_ws + align_up(plan.ws_bytes);
  rc = grow_pinned(&s.stage, &s.stage_cap, table_end, cudaHostAllocPortable, "cudaHostAlloc(server staging)", &s.retired);
  if (rc != HC_OK) return rc;
  void* blk = nullptr;
  e = cudaMallocFromPoolAsync(&blk, total, device_pool(dev), s.stream);
  if (e != cudaSuccess) return cuda_error(e, "cudaMallocFromPoolAsync(server batch)");
  uint8_t* d = static_cast<uint8_t*>(blk);
  plan_bind(plan, reinterpret_cast<uint32_t*>(d + o_f), d + o_ws);
  for (size_t i = 0; i < nq; ++i) {
    std::memcpy(s.stage + o_x + xoff[i], s.reqs[which[i]]->x.data(), s.reqs[which[i]]->x.size());
    plan.args[i].x = d + o_x + xoff[i];
  }
  std::memcpy(s.stage + o_args, plan.args.data(), nq * sizeof(SearchArgs));
  if (!plan.tiles.empty())
    std::memcpy(s.stage + o_tiles, plan.tiles.data(), plan.tiles.size() * sizeof(BatchTile));
  if (!plan.etiles.empty())
    std::memcpy(s.stage + o_etiles, plan.etiles.data(), plan.etiles.size() * sizeof(EmitTile));
  e = cudaMemcpyAsync(d + o_args, s.stage + o_args, table_end - o_args, cudaMemcpyHostToDevice, s.stream);
  if (e != cudaSuccess) rc = cuda_error(e, "cudaMemcpyAsync(server tables)");
  if (rc == HC_OK) {
    const BatchLaunch L = make_launch(plan, reinterpret_cast<const SearchArgs*>(d + o_args),
                                      reinterpret_cast<const BatchTile*>(d + o_tiles),
                                      reinterpret_cast<const EmitTile*>(d + o_etiles),
                                      reinterpret_cast<unsigned long long*>(d));  // kAlign bytes of counters
    rc = launch_batch(L, s.stream);
  }
  cudaFreeAsync(blk, s.stream);  // after the kernels, in stream order
  return rc;
}

// Plain mode: per request a host-built filter (hc_preprocess), uploaded with
// the others in one copy, and one plain search launch with its own
// stream-ordered workspace.
int Server::launch_plain(Slot& s, const std::vector<size_t>& which) {
  const size_t nq = which.size();
  std::vector<hc_filter*> fs(nq, nullptr);
  size_t off = 0;
  int rc = HC_OK;
  std::vector<size_t> offs(nq);
  for (size_t i = 0; i < nq && rc == HC_OK; ++i) {
    Req* r = s.reqs[which[i]];
    rc = hc_preprocess(r->x.data(), r->x.size(), r->p.q, r->p.alpha, &fs[i]);
    if (rc != HC_OK) break;
    const Filter* f = as_filter(fs[i]);
    offs[i] = off;
    off += align_up(f->F.size() * 4 + r->x.size(), 16);
  }
  if (rc == HC_OK)
    rc = grow_pinned(&s.stage_plain, &s.stage_plain_cap, off, cudaHostAllocPortable, "cudaHostAlloc(server staging)", &s.retired);
  void* fx = nullptr;
  if (rc == HC_OK) {
    cudaError_t e = cudaMallocFromPoolAsync(&fx, std::max<size_t>(off, 16), device_pool(dev), s.stream);
    if (e != cudaSuccess) rc = cuda_error(e, "cudaMallocFromPoolAsync(server plain filters)");
  }
  if (rc == HC_OK) {
    for (size_t i = 0; i < nq; ++i) {
      const Filter* f = as_filter(fs[i]);
      std::memcpy(s.stage_plain + offs[i], f->F.data(), f->F.size() * 4);
      std::memcpy(s.stage_plain + offs[i] + f->F.size() * 4, f->x.data(), f->x.size());
    }
    cudaError_t e = cudaMemcpyAsync(fx, s.stage_plain, off, cudaMemcpyHostToDevice, s.stream);
    if (e != cudaSuccess) rc = cuda_error(e, "cudaMemcpyAsync(server plain filters)");
  }
  for (size_t i = 0; i < nq && rc == HC_OK; ++i) {
    Req* r = s.reqs[which[i]];
    const Filter* f = as_filter(fs[i]);
    uint64_t* count = reinterpret_cast<uint64_t*>(s.res_dev + which[i]);
    uint64_t* pos = r->cap ? reinterpret_cast<uint64_t*>(s.res_dev + s.pos_off[which[i]]) : nullptr;
    if (r->n < r->x.size()) {
      cudaError_t e = cudaMemsetAsync(count, 0, sizeof(uint64_t), s.stream);
      if (e != cudaSuccess) rc = cuda_error(e, "cudaMemsetAsync(server count)");
      continue;
    }
    SearchPlan sp;
    hc_search_opts o{};
    o.struct_size = sizeof o;
    rc = plan_search(f, r->n, r->cap, &o, dev, &sp);
    if (rc != HC_OK) break;
    void* ws = nullptr;
    cudaError_t e = cudaMallocFromPoolAsync(&ws, std::max<size_t>(sp.ws_bytes, 16), device_pool(dev), s.stream);
    if (e != cudaSuccess) {
      rc = cuda_error(e, "cudaMallocFromPoolAsync(server plain workspace)");
      break;
    }
    const uint8_t* base = static_cast<const uint8_t*>(fx) + offs[i];
    rc = launch_planned_filter_ptrs(f, sp, reinterpret_cast<const uint32_t*>(base), base + f->F.size() * 4, r->y,
                                    r->n, pos, r->cap, count, ws, s.stream);
    cudaFreeAsync(ws, s.stream);
  }
  if (fx != nullptr) cudaFreeAsync(fx, s.stream);
  for (hc_filter* f : fs) hc_filter_free(f);
  return rc;
}

void Server::finish(Slot& s, cudaError_t q) {
  const uint64_t t = now_ns();
  int bad = HC_OK;
  if (q != cudaSuccess) {
    bad = cuda_error(q, "hc_server batch");
  } else if (*s.status != 0u) {
    bad = HC_ERR_TIMEOUT;  // a bounded device wait gave up: results of this batch are void
    unsigned int* sw = status_word();
    if (sw != nullptr) cudaMemsetAsync(sw, 0, sizeof(unsigned int), s.stream);
  }
  const uint64_t* counts = reinterpret_cast<const uint64_t*>(s.res);
  for (size_t i = 0; i < s.reqs.size(); ++i) {
    Req* r = s.reqs[i];
    r->done_ns = t;
    if (bad != HC_OK) {
      r->status = bad;
      continue;
    }
    r->count = counts[i];
    const uint64_t np = std::min<uint64_t>(r->count, r->cap);
    const uint64_t* src = reinterpret_cast<const uint64_t*>(s.res) + s.pos_off[i];
    r->pos.assign(src, src + np);
    r->status = r->count > r->cap ? HC_ERR_CAPACITY : HC_OK;
  }
  std::lock_guard<std::mutex> lock(mu);
  inflight_bytes -= s.admitted;
  for (Req* r : s.reqs) {
    done[r->id] = r;
    done_queue.push_back(r->id);
    st.completed++;
  }
  s.reqs.clear();
  s.admitted = 0;
  s.busy = false;
  if (q != cudaSuccess && fatal == HC_OK) fatal = HC_ERR_CUDA;
  cv_done.notify_all();
}

void Server::run() {
  cudaSetDevice(dev);
  std::unique_lock<std::mutex> lk(mu);
  while (true) {
    bool progress = false;
    for (Slot& s : slots) {
      if (!s.busy) continue;
      lk.unlock();
      const cudaError_t q = cudaEventQuery(s.done);
      if (q != cudaErrorNotReady) {
        finish(s, q);
        progress = true;
      }
      lk.lock();
    }
    bool any_busy = false;
    Slot* free_slot = nullptr;
    for (Slot& s : slots) {
      if (s.busy) any_busy = true;
      else if (free_slot == nullptr) free_slot = &s;
    }
    if (stop && !any_busy) break;  // queued requests are cancelled below
    if (free_slot != nullptr && !pending.empty() && fatal == HC_OK && !stop) {
      std::vector<Req*> b = take_batch();
      if (!b.empty()) {
        Slot& s = *free_slot;
        s.busy = true;
        s.reqs = b;
        s.batch = next_batch++;
        s.admitted = 0;
        for (Req* r : b) s.admitted += r->dev_bytes;
        st.batches++;
        st.max_batch = std::max<uint64_t>(st.max_batch, b.size());
        lk.unlock();
        const uint64_t t = now_ns();
        for (Req* r : b) {
          r->start_ns = t;
          r->batch = s.batch;
          r->batch_size = static_cast<uint32_t>(b.size());
        }
        const int rc = launch(s, b);
        if (rc != HC_OK) {
          // nothing of this batch is in flight beyond what the stream already
          // holds: wait for it, then report the error on its requests
          cudaStreamSynchronize(s.stream);
          s.reqs.clear();
          s.admitted = 0;
          fail(b, rc);
          lk.lock();
          s.busy = false;
          if (rc == HC_ERR_CUDA && fatal == HC_OK) fatal = rc;
        } else {
          lk.lock();
        }
        progress = true;
      }
    }
    if (!progress) {
      if (any_busy) {
        lk.unlock();
        std::this_thread::yield();
        lk.lock();
      } else {
        cv_work.wait_for(lk, std::chrono::milliseconds(50));
      }
    }
  }
  // cancelled requests (destroy with a queue, or after a CUDA error)
  for (Req* r : pending) {
    r->status = HC_ERR_STATE;
    r->done_ns = now_ns();
    done[r->id] = r;
    done_queue.push_back(r->id);
  }
  pending.clear();
  pending_text = 0;
  cv_done.notify_all();
}

}  // namespace hc

using namespace hc;

namespace {

void destroy_server(Server* s) {
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != s->dev) cudaSetDevice(s->dev);
  for (Slot& sl : s->slots) {
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.stream) cudaStreamDestroy(sl.stream);
    if (sl.stage) cudaFreeHost(sl.stage);
    if (sl.stage_plain) cudaFreeHost(sl.stage_plain);
    if (sl.res) cudaFreeHost(sl.res);
    if (sl.status) cudaFreeHost(sl.status);
    for (void* v : sl.retired) cudaFreeHost(v);
  }
  for (Text& t : s->texts)
    if (t.owned) cudaFree(const_cast<uint8_t*>(t.y));
  for (auto& kv : s->done) delete kv.second;
  if (cur != s->dev) cudaSetDevice(cur);
  s->magic = 0;
  delete s;
}

}  // namespace

extern "C" {

int hc_server_create(const hc_server_config* cfg_in, const hc_tuner* tuner, hc_server** out) {
  clear_error();
  if (out == nullptr) return set_error(HC_ERR_ARG, "hc_server_create: out is NULL");
  *out = nullptr;
  hc_server_config cfg{};
  cfg.struct_size = sizeof cfg;
  if (cfg_in != nullptr) {
    if (cfg_in->struct_size != sizeof(hc_server_config))
      return set_error(HC_ERR_ARG, "hc_server_create: config struct_size mismatch");
    cfg = *cfg_in;
  }
  if (cfg.mem_limit == 0) cfg.mem_limit = uint64_t(32) << 30;
  if (cfg.max_inflight == 0) cfg.max_inflight = 3;
  if (cfg.max_batch == 0) cfg.max_batch = 1024;
  if (cfg.default_cap == 0) cfg.default_cap = 4096;
  if (cfg.max_batch_bytes == 0) cfg.max_batch_bytes = uint64_t(64) << 20;
  if (cfg.max_inflight < 1 || cfg.max_inflight > 16 || cfg.max_batch < 1 || cfg.max_batch > (1 << 20) ||
      cfg.default_cap > (uint64_t(1) << 32))
    return set_error(HC_ERR_ARG, "hc_server_create: max_inflight in [1, 16], max_batch in [1, 2^20], default_cap <= 2^32");
  const Tuner* t = nullptr;
  if (tuner != nullptr && (t = as_tuner(tuner)) == nullptr)
    return set_error(HC_ERR_ARG, "hc_server_create: invalid tuner");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
  Server* s = new (std::nothrow) Server();
  if (s == nullptr) return set_error(HC_ERR_NOMEM, "hc_server_create: out of host memory");
  s->dev = dev;
  s->cfg = cfg;
  s->tuner = t;
  s->slots.resize(cfg.max_inflight);
  for (Slot& sl : s->slots) {
    e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void**>(&sl.status), sizeof(unsigned int), cudaHostAllocPortable);
    if (e != cudaSuccess) break;
    // pinned buffers sized up front for a full batch of requests with the
    // default capacity (at most 64 MiB of results), the launch tables of a
    // full batch and 16 single-search filters of 2^13 words, so that they
    // rarely grow while requests are served
    const size_t res0 = std::min<size_t>((size_t(cfg.max_batch) * (cfg.default_cap + 1)) * 8, size_t(64) << 20);
    int rc0 = grow_pinned(&sl.res, &sl.res_cap, res0, cudaHostAllocMapped | cudaHostAllocPortable,
                          "cudaHostAlloc(server results)", &sl.retired);
    if (rc0 == HC_OK)
      rc0 = grow_pinned(&sl.stage, &sl.stage_cap, size_t(cfg.max_batch) * 1024, cudaHostAllocPortable,
                        "cudaHostAlloc(server staging)", &sl.retired);
    if (rc0 == HC_OK)
      rc0 = grow_pinned(&sl.stage_plain, &sl.stage_plain_cap, size_t(16) * ((size_t(1) << 13) * 4 + 4096),
                        cudaHostAllocPortable, "cudaHostAlloc(server staging)", &sl.retired);
    if (rc0 != HC_OK) {
      e = cudaErrorMemoryAllocation;
      break;
    }
  }
  if (e != cudaSuccess || status_word() == nullptr) {
    const int rc = e != cudaSuccess ? cuda_error(e, "hc_server_create") : set_error(HC_ERR_CUDA, "device status word unavailable");
    destroy_server(s);
    return rc;
  }
  s->worker = std::thread([s] { s->run(); });
  *out = reinterpret_cast<hc_server*>(s);
  return HC_OK;
}

int hc_server_add_text(hc_server* sp, const uint8_t* y, uint64_t n, int on_device, int sigma, uint32_t* text_id) {
  clear_error();
  Server* s = as_server(sp);
  if (s == nullptr || text_id == nullptr || (y == nullptr && n > 0) || sigma < 0)
    return set_error(HC_ERR_ARG, "hc_server_add_text: invalid argument");
  {
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->text_bytes + n > s->cfg.mem_limit)
      return set_error(HC_ERR_ADMISSION, "hc_server_add_text: resident texts would exceed the memory limit");
  }
  Text t;
  t.n = n;
  t.y = y;
  if (!on_device && n > 0) {
    uint8_t* d = nullptr;
    cudaError_t e = cudaMalloc(&d, n);
    if (e != cudaSuccess) return cuda_error(e, "cudaMalloc(server text)");
    e = cudaMemcpy(d, y, n, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaFree(d);
      return cuda_error(e, "cudaMemcpy(server text)");
    }
    t.y = d;
    t.owned = true;
  }
  t.sigma = sigma;
  if (sigma == 0 && n > 0) {
    std::vector<double> est;
    const uint8_t* yy = t.y;
    uint64_t nn = n;
    int rc = estimate_sigma(&yy, &nn, 1, &est, nullptr);
    if (rc != HC_OK) {
      if (t.owned) cudaFree(const_cast<uint8_t*>(t.y));
      return rc;
    }
    t.sigma = est[0];
  }
  std::lock_guard<std::mutex> lock(s->mu);
  if (s->text_bytes + n > s->cfg.mem_limit) {
    if (t.owned) cudaFree(const_cast<uint8_t*>(t.y));
    return set_error(HC_ERR_ADMISSION, "hc_server_add_text: resident texts would exceed the memory limit");
  }
  s->texts.push_back(t);
  s->text_bytes += n;
  *text_id = static_cast<uint32_t>(s->texts.size() - 1);
  return HC_OK;
}

int hc_server_text_info(const hc_server* sp, uint32_t text_id, uint64_t* n, double* sigma) {
  Server* s = as_server(sp);
  if (s == nullptr) return set_error(HC_ERR_ARG, "hc_server_text_info: invalid server");
  std::lock_guard<std::mutex> lock(s->mu);
  if (text_id >= s->texts.size()) return set_error(HC_ERR_ARG, "hc_server_text_info: unknown text");
  if (n) *n = s->texts[text_id].n;
  if (sigma) *sigma = s->texts[text_id].sigma;
  return HC_OK;
}

}  // extern "C"

namespace {

// Validates and sizes a request (a one-query plan with placeholder device
// addresses: plans read no device memory).
int make_request(Server* s, const hc_server_request& q, uint64_t submit_ns, Req** out) {
  Text t;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    if (q.text >= s->texts.size()) return set_error(HC_ERR_ARG, "hc_server_submit: unknown text");
    t = s->texts[q.text];
  }
  if (q.x == nullptr || q.m < 1 || q.m > 65536)
    return set_error(HC_ERR_ARG, "hc_server_submit: need a host pattern of 1 to 65536 bytes");
  if (q.cap > (uint64_t(1) << 32)) return set_error(HC_ERR_ARG, "hc_server_submit: cap above 2^32");
  Req* r = new (std::nothrow) Req();
  if (r == nullptr) return set_error(HC_ERR_NOMEM, "hc_server_submit: out of host memory");
  r->text = q.text;
  r->y = t.y;
  r->n = t.n;
  r->x.assign(q.x, q.x + q.m);
  // positions kept: at most one per window start (bounds the result arena)
  const uint64_t nwin = t.n >= q.m ? t.n - q.m + 1 : 0;
  r->cap = std::min<uint64_t>(q.cap ? q.cap : s->cfg.default_cap, nwin);
  if (q.q == 0) {
    // q and alpha from the tuner; launch options automatic, as in a batch
    const QueryParams tp = tuner_lookup(s->tuner, t.sigma, q.m);
    r->p.q = tp.q;
    r->p.alpha = tp.alpha;
  } else {
    r->p.q = q.q;
    r->p.alpha = q.alpha;
  }
  if (q.lane_bytes > 0) r->p.lane_bytes = q.lane_bytes;
  if (q.mode != HC_MODE_AUTO) r->p.mode = q.mode;
  // one-query plan at placeholder addresses (16-byte aligned, never dereferenced)
  static const uint64_t placeholder[2] = {0, 0};
  hc_batch_query Q{};
  Q.x_dev = reinterpret_cast<const uint8_t*>(placeholder);
  Q.m = q.m;
  Q.y_dev = t.y ? t.y : reinterpret_cast<const uint8_t*>(placeholder);
  Q.n = t.n;
  Q.q = r->p.q;
  Q.alpha = r->p.alpha;
  Q.pos_dev = const_cast<uint64_t*>(placeholder);
  Q.cap = r->cap;
  Q.count_dev = const_cast<uint64_t*>(placeholder);
  BatchPlan plan;
  // sized as a batch of its own (the finest records it can be given)
  int rc = plan_add_query(plan, Q, 0, r->p, record_bytes_for(t.n, s->dev), "hc_server_submit");
  if (rc == HC_OK) rc = plan_finish(plan, s->dev, "hc_server_submit");
  if (rc != HC_OK) {
    delete r;
    return rc;
  }
  r->lay = plan.lay;
  r->dev_bytes = align_up(sizeof(SearchArgs)) + align_up(plan.tiles.size() * sizeof(BatchTile)) +
                 align_up(plan.etiles.size() * sizeof(EmitTile)) + align_up(q.m, 16) +
                 align_up(plan.filter_words * 4) + align_up(plan.ws_bytes);
  r->submit_ns = submit_ns;
  *out = r;
  return HC_OK;
}

void enqueue(Server* s, Req* r, uint64_t* id) {
  {
    std::lock_guard<std::mutex> lock(s->mu);
    r->id = s->next_id++;
    s->pending.push_back(r);
    s->pending_text += r->n;
    s->st.submitted++;
    *id = r->id;
  }
  s->cv_work.notify_one();
}

}  // namespace

extern "C" {

int hc_server_submit(hc_server* sp, const hc_server_request* q, uint64_t* id) {
  clear_error();
  Server* s = as_server(sp);
  if (s == nullptr || q == nullptr || id == nullptr) return set_error(HC_ERR_ARG, "hc_server_submit: invalid argument");
  {
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->fatal != HC_OK) return set_error(HC_ERR_STATE, "hc_server_submit: server stopped after a CUDA error");
  }
  Req* r = nullptr;
  int rc = make_request(s, *q, now_ns(), &r);
  if (rc != HC_OK) return rc;
  enqueue(s, r, id);
  return HC_OK;
}

int hc_server_replay(hc_server* sp, const hc_server_request* qs, size_t nreq, const uint64_t* arrival_ns,
                     uint64_t* ids) {
  clear_error();
  Server* s = as_server(sp);
  if (s == nullptr || (nreq > 0 && (qs == nullptr || arrival_ns == nullptr || ids == nullptr)))
    return set_error(HC_ERR_ARG, "hc_server_replay: invalid argument");
  // requests are validated and sized before the clock starts
  std::vector<Req*> rs(nreq, nullptr);
  for (size_t i = 0; i < nreq; ++i) {
    int rc = make_request(s, qs[i], 0, &rs[i]);
    if (rc != HC_OK) {
      for (Req* r : rs) delete r;
      return rc;
    }
    if (i > 0 && arrival_ns[i] < arrival_ns[i - 1]) {
      for (Req* r : rs) delete r;
      return set_error(HC_ERR_ARG, "hc_server_replay: arrival times must not decrease");
    }
  }
  const uint64_t t0 = now_ns();
  for (size_t i = 0; i < nreq; ++i) {
    const uint64_t due = t0 + arrival_ns[i];
    uint64_t t = now_ns();
    while (t < due) {
      if (due - t > 200000) std::this_thread::sleep_for(std::chrono::nanoseconds(due - t - 100000));
      else std::this_thread::yield();
      t = now_ns();
    }
    rs[i]->submit_ns = due;  // latency counts from the scheduled arrival
    enqueue(s, rs[i], &ids[i]);
  }
  return HC_OK;
}

int hc_server_poll(hc_server* sp, hc_server_result* out, size_t max, size_t* got, int64_t wait_us) {
  clear_error();
  Server* s = as_server(sp);
  if (s == nullptr || got == nullptr || (out == nullptr && max > 0))
    return set_error(HC_ERR_ARG, "hc_server_poll: invalid argument");
  *got = 0;
  std::unique_lock<std::mutex> lk(s->mu);
  if (s->done_queue.empty() && wait_us != 0) {
    auto ready = [s] { return !s->done_queue.empty(); };
    if (wait_us < 0) s->cv_done.wait(lk, ready);
    else s->cv_done.wait_for(lk, std::chrono::microseconds(wait_us), ready);
  }
  while (*got < max && !s->done_queue.empty()) {
    const uint64_t id = s->done_queue.front();
    s->done_queue.pop_front();
    const Req* r = s->done.at(id);
    hc_server_result& o = out[(*got)++];
    o = hc_server_result{};
    o.id = r->id;
    o.status = r->status;
    o.text = r->text;
    o.q = r->p.q;
    o.alpha = r->p.alpha;
    o.count = r->count;
    o.npos = r->pos.size();
    o.pos = r->pos.data();
    o.submit_ns = r->submit_ns;
    o.start_ns = r->start_ns;
    o.done_ns = r->done_ns;
    o.batch = r->batch;
    o.batch_size = r->batch_size;
  }
  return HC_OK;
}

int hc_server_release(hc_server* sp, uint64_t id) {
  Server* s = as_server(sp);
  if (s == nullptr) return set_error(HC_ERR_ARG, "hc_server_release: invalid server");
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->done.find(id);
  if (it == s->done.end()) return set_error(HC_ERR_ARG, "hc_server_release: unknown or unfinished request");
  for (uint64_t qid : s->done_queue)
    if (qid == id) return set_error(HC_ERR_STATE, "hc_server_release: request not yet polled");
  delete it->second;
  s->done.erase(it);
  return HC_OK;
}

int hc_server_drain(hc_server* sp, int64_t timeout_ms) {
  clear_error();
  Server* s = as_server(sp);
  if (s == nullptr) return set_error(HC_ERR_ARG, "hc_server_drain: invalid server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto idle = [s] {
    if (!s->pending.empty()) return false;
    for (const Slot& sl : s->slots)
      if (sl.busy) return false;
    return true;
  };
  if (timeout_ms < 0) s->cv_done.wait(lk, idle);
  else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), idle))
    return set_error(HC_ERR_TIMEOUT, "hc_server_drain: requests still pending");
  return s->fatal;
}

int hc_server_get_stats(const hc_server* sp, hc_server_stats* out) {
  Server* s = as_server(sp);
  if (s == nullptr || out == nullptr) return set_error(HC_ERR_ARG, "hc_server_get_stats: invalid argument");
  std::lock_guard<std::mutex> lock(s->mu);
  *out = hc_server_stats{};
  out->submitted = s->st.submitted;
  out->completed = s->st.completed;
  out->batches = s->st.batches;
  out->rejected = s->st.rejected;
  out->admission_waits = s->st.admission_waits;
  out->max_batch = s->st.max_batch;
  out->pending = s->pending.size();
  out->inflight_bytes = s->inflight_bytes;
  out->peak_inflight_bytes = s->st.peak_inflight_bytes;
  out->text_bytes = s->text_bytes;
  out->mem_limit = s->cfg.mem_limit;
  return HC_OK;
}

void hc_server_destroy(hc_server* sp) {
  Server* s = as_server(sp);
  if (s == nullptr) return;
  destroy_server(s);
}

}  // extern "C"
