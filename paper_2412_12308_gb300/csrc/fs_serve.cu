// fs_serve.cu -- the serving loop: continuous batching of solve and advance
// requests on one device.
//
// A host thread owns the request queue.  Whenever one of its `slots` (each
// with its own CUDA stream) is free, it forms the next batch from the queue
// in arrival order: a request is admitted when its workspace, plus the
// spectrum it asks to keep, fits the HBM budget next to everything already
// in flight or kept; follow-up (advance) requests wait until the spectrum of
// their parent request is on the device.  A batch is one persistent launch
// (the batch executor); several batches run concurrently on their streams,
// so requests arriving while others are on the GPU start as soon as a slot
// and memory free up.  Kept spectra live in the budgeted device arena until
// their expected follow-ups complete.  Latency = enqueue -> observed
// completion, per request.
#include <algorithm>
#include <chrono>
#include <cstdlib>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "fs_batch.h"

namespace fs {
namespace {

using clk = std::chrono::steady_clock;

size_t al256(size_t b) { return (b + 255) / 256 * 256; }

// First-fit allocator over one device buffer (host-side bookkeeping).
struct DevArena {
  char *base = nullptr;
  size_t cap = 0;
  std::map<size_t, size_t> free_;  // offset -> bytes
  cudaError_t init(size_t bytes) {
    cap = al256(bytes);
    cudaError_t e = cudaMalloc((void **)&base, cap);
    if (e == cudaSuccess) free_[0] = cap;
    return e;
  }
  long long alloc(size_t bytes) {
    bytes = al256(bytes ? bytes : 256);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      const size_t off = it->first, rem = it->second - bytes;
      free_.erase(it);
      if (rem) free_[off + bytes] = rem;
      return (long long)off;
    }
    return -1;
  }
  void release(size_t off, size_t bytes) {
    bytes = al256(bytes ? bytes : 256);
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  void destroy() {
    cudaFree(base);
    base = nullptr;
    cap = 0;
    free_.clear();
  }
};

struct Req {
  uint64_t ticket = 0;
  fs_request r{};
  clk::time_point arrival;
  size_t ws = 0;       // workspace bytes in a batch arena
  size_t keep = 0;     // bytes of the spectrum kept for follow-ups
  size_t reserve = 0;  // workspace reserved for the follow-ups (keep requests)
};

struct Kept {
  fs_state_s st{};
  long long off = -1;
  size_t bytes = 0;
  size_t reserve_each = 0;  // workspace reserved per expected follow-up
  bool ready = false;
  int remaining = 0;  // follow-ups still expected
};

struct Flight {
  cudaEvent_t ev = nullptr;
  int slot = 0;
  bool large = false;  // a batch of grids run as standalone passes
  long long ws_off = -1;
  size_t ws_bytes = 0;
  std::vector<Req> reqs;
};

struct Server {
  std::mutex mu;
  std::condition_variable cv, done_cv;
  std::deque<Req> queue;
  std::unordered_map<uint64_t, Kept> kept;
  // follow-ups a keep request may still receive (ticket -> keep minus the
  // follow-ups enqueued so far); an entry leaves the map at zero
  std::unordered_map<uint64_t, int> follow_left;
  std::deque<uint64_t> done_q;
  std::unordered_map<uint64_t, double> lat_us;
  std::deque<uint64_t> lat_order;
  std::vector<cudaStream_t> streams;
  std::vector<char> busy;
  std::vector<Flight> flights;
  DevArena arena;
  size_t budget = 0, used = 0, peak_used = 0;
  int max_batch = 64, device = 0;
  bool stopping = false;
  std::thread th;
  uint64_t next_ticket = 1;
  size_t queue_cap = 1u << 20;
  long long direct_min_points = 2048LL * 2048LL;  // grids this large run as standalone passes
  // statistics
  uint64_t n_batches = 0, n_done = 0, max_inflight = 0, overlap_batches = 0, n_failed = 0;
  fs_status last_error = FS_OK;
};

Server *g_srv = nullptr;
std::mutex g_srv_mu;

size_t spec_bytes_of(const fs_request &r) {
  fs_plan p = r.plan ? r.plan : (r.state ? r.state->plan : nullptr);
  return p ? p->spec_bytes : 0;
}

// Grids of at least direct_min_points run as standalone pass kernels inside
// their batch; a follow-up takes its parent's grid (its plan is filled in at
// enqueue).
bool is_large(const Server *S, const Req &q) {
  return S->direct_min_points > 0 && q.r.plan &&
         (long long)q.r.plan->nx * q.r.plan->ny >= S->direct_min_points;
}

void harvest_locked(Server *S) {
  for (size_t i = 0; i < S->flights.size();) {
    Flight &f = S->flights[i];
    const cudaError_t q = cudaEventQuery(f.ev);
    if (q == cudaErrorNotReady) {
      ++i;
      continue;
    }
    if (q != cudaSuccess) S->last_error = FS_ERR_CUDA;
    const auto now = clk::now();
    for (Req &rq : f.reqs) {
      const double us = std::chrono::duration<double, std::micro>(now - rq.arrival).count();
      S->lat_us[rq.ticket] = us;
      S->lat_order.push_back(rq.ticket);
      while (S->lat_order.size() > (1u << 20)) {
        S->lat_us.erase(S->lat_order.front());
        S->lat_order.pop_front();
      }
      S->done_q.push_back(rq.ticket);
      ++S->n_done;
      if (rq.keep) {
        auto it = S->kept.find(rq.ticket);
        if (it != S->kept.end()) it->second.ready = true;
      }
      if (rq.r.parent) {
        auto it = S->kept.find(rq.r.parent);
        if (it != S->kept.end() && --it->second.remaining <= 0) {
          S->arena.release((size_t)it->second.off, it->second.bytes);
          S->used -= it->second.bytes;
          S->kept.erase(it);
        }
      }
    }
    if (f.ws_off >= 0) {
      S->arena.release((size_t)f.ws_off, f.ws_bytes);
      S->used -= f.ws_bytes;
    }
    S->busy[f.slot] = 0;
    cudaEventDestroy(f.ev);
    S->flights.erase(S->flights.begin() + i);
  }
  if (!S->done_q.empty()) S->done_cv.notify_all();
}

// Is request `ticket` still queued or in flight (a parent whose spectrum is
// not kept yet)?
bool parent_pending_locked(const Server *S, uint64_t ticket) {
  for (const Req &w : S->queue)
    if (w.ticket == ticket) return true;
  for (const Flight &f : S->flights)
    for (const Req &w : f.reqs)
      if (w.ticket == ticket) return true;
  return false;
}

// Form and launch one batch on a free slot; returns true if one was launched.
bool launch_one_locked(Server *S) {
  int slot = -1;
  for (size_t i = 0; i < S->busy.size(); ++i)
    if (!S->busy[i]) {
      slot = (int)i;
      break;
    }
  if (slot < 0 || S->queue.empty()) return false;
  // A batch holds either grids that run as standalone passes (large) or grids
  // that share the persistent launch (small), never both, so small requests
  // do not wait on their stream behind a large grid's passes; large batches
  // take at most all slots but one, so one slot always serves small ones.
  int large_in_flight = 0;
  for (const Flight &f : S->flights) large_in_flight += f.large ? 1 : 0;
  const bool allow_large = large_in_flight < (int)S->streams.size() - 1;
  int cls = -1;  // class of this batch: decided by its first request
  std::vector<Req> take;
  std::vector<fs_request> reqs;
  std::vector<void *> keeps;
  size_t ws = 0;
  bool blocked = false;  // an earlier request did not fit: only follow-ups (which free memory) pass it
  for (auto it = S->queue.begin(); it != S->queue.end() && (int)take.size() < S->max_batch;) {
    Req &q = *it;
    const int qc = is_large(S, q) ? 1 : 0;
    if ((qc == 1 && !allow_large) || (cls >= 0 && qc != cls)) {
      ++it;
      continue;
    }
    if (blocked && !q.r.parent) {
      ++it;
      continue;
    }
    size_t credit = 0;  // a follow-up spends the workspace its parent reserved
    if (q.r.parent) {
      auto k = S->kept.find(q.r.parent);
      if (k == S->kept.end() && !parent_pending_locked(S, q.r.parent)) {
        // the parent's spectrum is gone (it was released after its declared
        // follow-ups): this request can never run, so finish it with an error
        // instead of leaving it in the queue (fs_serve_stop waits for an empty
        // queue)
        S->done_q.push_back(q.ticket);
        S->lat_us[q.ticket] = -1.0;
        S->lat_order.push_back(q.ticket);
        ++S->n_done;
        ++S->n_failed;
        S->last_error = FS_ERR_ARG;
        it = S->queue.erase(it);
        S->done_cv.notify_all();
        continue;
      }
      if (k == S->kept.end() || !k->second.ready) {
        ++it;  // its spectrum is not on the device yet
        continue;
      }
      q.r.state = &k->second.st;
      credit = k->second.reserve_each;
    }
    if (S->used + al256(ws) + al256(q.ws) + q.keep + q.reserve > S->budget + credit) {
      blocked = true;  // admission in arrival order
      ++it;
      continue;
    }
    S->used -= credit;
    long long koff = -1;
    if (q.keep) {
      koff = S->arena.alloc(q.keep);
      if (koff < 0) {
        blocked = true;
        ++it;
        continue;
      }
      Kept k;
      k.st.plan = q.r.plan;
      k.st.su = S->arena.base + koff;
      k.st.sv = nullptr;
      k.st.has_v = false;
      k.off = koff;
      k.bytes = q.keep;
      k.remaining = q.r.keep;
      k.reserve_each = q.r.keep > 0 ? q.reserve / q.r.keep : 0;
      S->kept[q.ticket] = k;
      S->used += q.keep + q.reserve;
    }
    ws += al256(q.ws);
    cls = qc;
    reqs.push_back(q.r);
    keeps.push_back(q.keep ? (void *)(S->arena.base + koff) : nullptr);
    take.push_back(q);
    it = S->queue.erase(it);
  }
  if (take.empty()) return false;
  Flight f;
  f.slot = slot;
  f.large = cls == 1;
  if (ws) {
    f.ws_off = S->arena.alloc(ws);
    if (f.ws_off < 0) {
      // fragmentation: put the requests back (front, original order)
      for (auto rit = take.rbegin(); rit != take.rend(); ++rit) {
        if (rit->keep) {
          auto k = S->kept.find(rit->ticket);
          S->arena.release((size_t)k->second.off, k->second.bytes);
          S->used -= k->second.bytes + rit->reserve;
          S->kept.erase(k);
        }
        if (rit->r.parent) {
          auto k = S->kept.find(rit->r.parent);
          if (k != S->kept.end()) S->used += k->second.reserve_each;
          rit->r.state = nullptr;
        }
        S->queue.push_front(*rit);
      }
      return false;
    }
    f.ws_bytes = ws;
    S->used += ws;
  }
  S->peak_used = std::max(S->peak_used, S->used);
  uint64_t bt = 0;
  fs_status st = batch_submit_internal(reqs.data(), (int)reqs.size(), keeps.data(), &bt, S->streams[slot],
                                       ws ? S->arena.base + f.ws_off : nullptr, ws, S->direct_min_points);
  cudaError_t e = cudaEventCreateWithFlags(&f.ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(f.ev, S->streams[slot]);
  if (st != FS_OK || e != cudaSuccess) S->last_error = st != FS_OK ? st : FS_ERR_CUDA;
  f.reqs = std::move(take);
  S->busy[slot] = 1;
  S->flights.push_back(std::move(f));
  ++S->n_batches;
  if (S->flights.size() >= 2) ++S->overlap_batches;
  S->max_inflight = std::max<uint64_t>(S->max_inflight, S->flights.size());
  return true;
}

void server_loop(Server *S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    harvest_locked(S);
    while (launch_one_locked(S)) {
    }
    if (S->stopping && S->queue.empty() && S->flights.empty()) break;
    if (S->flights.empty()) {
      S->cv.wait_for(lk, std::chrono::milliseconds(20));
    } else {
      lk.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds(5));
      lk.lock();
    }
  }
}

}  // namespace
}  // namespace fs

using namespace fs;

extern "C" fs_status fs_serve_start(size_t hbm_budget_bytes, int slots, int max_batch) {
  std::lock_guard<std::mutex> g(g_srv_mu);
  if (g_srv) return set_error(FS_ERR_BUSY, "fs_serve_start: already running");
  if (slots < 2 || max_batch < 1 || hbm_budget_bytes < (1u << 20))
    return set_error(FS_ERR_ARG, "fs_serve_start: need slots >= 2, max_batch >= 1, budget >= 1 MiB");
  Server *S = new Server();
  S->budget = al256(hbm_budget_bytes);
  S->max_batch = max_batch;
  if (const char *v = getenv("FS_SERVE_DIRECT_MIN")) S->direct_min_points = atoll(v);
  cudaError_t e = cudaGetDevice(&S->device);
  if (e == cudaSuccess) e = S->arena.init(S->budget);
  for (int i = 0; e == cudaSuccess && i < slots; ++i) {
    cudaStream_t s;
    e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) S->streams.push_back(s);
  }
  if (e != cudaSuccess) {
    for (auto s : S->streams) cudaStreamDestroy(s);
    S->arena.destroy();
    delete S;
    return cuda_error(e, "fs_serve_start");
  }
  S->busy.assign(S->streams.size(), 0);
  S->th = std::thread(server_loop, S);
  g_srv = S;
  return FS_OK;
}

static fs_status enqueue_locked(Server *S, const fs_request *req, clk::time_point arrival, uint64_t *ticket_out) {
  const fs_request &r = *req;
  Req q;
  q.r = r;
  q.arrival = arrival;
  const bool adv = r.op == FS_OP_DIFFUSION_ADVANCE || r.op == FS_OP_WAVE_ADVANCE;
  auto left = S->follow_left.end();
  if (adv && r.parent) {
    // at most `keep` follow-ups per kept spectrum: the spectrum (and the
    // workspace its parent reserved) is released after that many complete
    left = S->follow_left.find(r.parent);
    if (left == S->follow_left.end() || left->second <= 0)
      return set_error(FS_ERR_ARG,
                       "fs_serve_enqueue: parent spectrum is not kept, or all its declared follow-ups were enqueued");
    auto k = S->kept.find(r.parent);
    fs_plan p = k != S->kept.end() ? k->second.st.plan : nullptr;
    if (!p)
      for (auto &w : S->queue)
        if (w.ticket == r.parent) p = w.r.plan;
    if (!p)
      for (auto &f : S->flights)
        for (auto &w : f.reqs)
          if (w.ticket == r.parent) p = w.r.plan;
    if (!p) return set_error(FS_ERR_ARG, "fs_serve_enqueue: parent spectrum is not kept");
    q.r.plan = p;
    fs_state_s probe{};
    probe.plan = p;
    q.r.state = &probe;  // for the workspace estimate only
    const fs_status st = request_workspace(q.r, &q.ws);
    q.r.state = nullptr;
    if (st != FS_OK) return st;
  } else {
    if (r.keep && r.op != FS_OP_DIFFUSION && !(r.op == FS_OP_WAVE && !r.in_v))
      return set_error(FS_ERR_ARG, "fs_serve_enqueue: only diffusion / zero-velocity wave solves keep spectra");
    fs_status st = request_workspace(r, &q.ws);
    if (st != FS_OK) return st;
    if (r.keep) {
      q.keep = al256(spec_bytes_of(r));
      // workspace of one follow-up advance on this grid, reserved up front so
      // follow-ups (which free the kept spectrum) can always be admitted
      fs_request f{};
      f.op = r.op == FS_OP_DIFFUSION ? FS_OP_DIFFUSION_ADVANCE : FS_OP_WAVE_ADVANCE;
      fs_state_s probe{};
      probe.plan = r.plan;
      f.state = &probe;
      f.out_u = r.out_u;
      f.c = 1.0;
      size_t fws = 0;
      st = request_workspace(f, &fws);
      if (st != FS_OK) return st;
      q.reserve = al256(fws) * (size_t)r.keep;
    }
  }
  if (al256(q.ws) + q.keep + q.reserve > S->budget)
    return set_error(FS_ERR_BUDGET, "fs_serve_enqueue: request exceeds the budget");
  if (S->queue.size() >= S->queue_cap) return set_error(FS_ERR_BUSY, "fs_serve_enqueue: queue full");
  q.ticket = S->next_ticket++;
  if (left != S->follow_left.end() && --left->second <= 0) S->follow_left.erase(left);
  if (q.keep && r.keep > 0) S->follow_left[q.ticket] = r.keep;
  S->queue.push_back(q);
  if (ticket_out) *ticket_out = q.ticket;
  S->cv.notify_one();
  return FS_OK;
}

extern "C" fs_status fs_serve_enqueue(const fs_request *req, uint64_t *ticket_out) {
  if (!req) return set_error(FS_ERR_ARG, "fs_serve_enqueue: NULL request");
  Server *S = g_srv;
  if (!S) return set_error(FS_ERR_ARG, "fs_serve_enqueue: server not started");
  std::lock_guard<std::mutex> lk(S->mu);
  return enqueue_locked(S, req, clk::now(), ticket_out);
}

extern "C" fs_status fs_serve_replay(const fs_request *reqs, const double *arrival_s, int n, uint64_t *tickets_out) {
  Server *S = g_srv;
  if (!S) return set_error(FS_ERR_ARG, "fs_serve_replay: server not started");
  if (!reqs || !arrival_s || n < 0) return set_error(FS_ERR_ARG, "fs_serve_replay: NULL argument");
  std::vector<uint64_t> tk(n, 0);
  const auto t0 = clk::now();
  for (int i = 0; i < n; ++i) {
    const auto due = t0 + std::chrono::duration_cast<clk::duration>(std::chrono::duration<double>(arrival_s[i]));
    for (;;) {
      const auto now = clk::now();
      if (now >= due) break;
      if (due - now > std::chrono::microseconds(300)) std::this_thread::sleep_for(due - now - std::chrono::microseconds(200));
      else std::this_thread::yield();
    }
    fs_request r = reqs[i];
    if (r.parent) {
      const uint64_t pi = r.parent - 1;  // parent given as (index + 1) in this replay
      if (pi >= (uint64_t)i) return set_error(FS_ERR_ARG, "fs_serve_replay: parent must come earlier");
      r.parent = tk[pi];
    }
    std::lock_guard<std::mutex> lk(S->mu);
    fs_status st = enqueue_locked(S, &r, clk::now(), &tk[i]);
    if (st != FS_OK) return st;
  }
  if (tickets_out) memcpy(tickets_out, tk.data(), n * sizeof(uint64_t));
  return FS_OK;
}

extern "C" fs_status fs_serve_poll(uint64_t *done_tickets, int cap, int *n_done, int timeout_us) {
  if (n_done) *n_done = 0;
  Server *S = g_srv;
  if (!S) return set_error(FS_ERR_ARG, "fs_serve_poll: server not started");
  std::unique_lock<std::mutex> lk(S->mu);
  if (S->done_q.empty() && timeout_us != 0) {
    if (timeout_us < 0) S->done_cv.wait(lk, [&] { return !S->done_q.empty(); });
    else S->done_cv.wait_for(lk, std::chrono::microseconds(timeout_us), [&] { return !S->done_q.empty(); });
  }
  int k = 0;
  while (k < cap && !S->done_q.empty()) {
    if (done_tickets) done_tickets[k] = S->done_q.front();
    S->done_q.pop_front();
    ++k;
  }
  if (n_done) *n_done = k;
  if (S->last_error != FS_OK) {
    const fs_status st = S->last_error;
    S->last_error = FS_OK;
    return set_error(st, "fs_serve_poll: a batch failed");
  }
  return (k == 0 && timeout_us != 0) ? set_error(FS_ERR_TIMEOUT, "fs_serve_poll: timed out") : FS_OK;
}

extern "C" fs_status fs_serve_latency(uint64_t ticket, double *latency_us) {
  Server *S = g_srv;
  if (!S || !latency_us) return set_error(FS_ERR_ARG, "fs_serve_latency: server not started / NULL");
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->lat_us.find(ticket);
  if (it == S->lat_us.end()) return set_error(FS_ERR_ARG, "fs_serve_latency: ticket not finished");
  *latency_us = it->second;
  return FS_OK;
}

extern "C" fs_status fs_serve_stats(uint64_t *out, int cap) {
  Server *S = g_srv;
  if (!S || !out) return set_error(FS_ERR_ARG, "fs_serve_stats: server not started / NULL");
  std::lock_guard<std::mutex> lk(S->mu);
  const uint64_t v[] = {S->n_batches, S->n_done, S->max_inflight, S->overlap_batches, S->peak_used, S->used,
                        S->queue.size(), S->kept.size(), S->n_failed};
  for (int i = 0; i < cap && i < (int)(sizeof v / sizeof v[0]); ++i) out[i] = v[i];
  return FS_OK;
}

extern "C" fs_status fs_serve_stop(void) {
  Server *S;
  {
    std::lock_guard<std::mutex> g(g_srv_mu);
    S = g_srv;
    if (!S) return FS_OK;
    g_srv = nullptr;
  }
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stopping = true;
    S->cv.notify_all();
  }
  S->th.join();
  for (auto s : S->streams) {
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }
  S->arena.destroy();
  delete S;
  return FS_OK;
}
