// Request loop over cached plans (hankel_server_* in include/hankel.h).
//
// One dispatcher thread owns every plan, stream and staging buffer. submit() only appends to
// the request table and the queue under the lock; the dispatcher
//  1. retires finished batches (event query), copies results to the callers' host arrays and
//     records each request's latency;
//  2. fills idle streams: it takes the oldest queued request whose plan has an idle execution
//     context (or may get one more: up to contexts_per_plan, while the device memory allows),
//     gathers the queued requests of the same plan (FIFO, up to max_batch vectors), builds the
//     plan if it is not cached (evicting idle plans, least recently used first, while the device
//     memory held exceeds the cap), packs the coefficients into the stream's pinned buffer and
//     issues copy-in, batched execution on that context and copy-out on the stream (or replays
//     them from a captured CUDA graph). So a request for a plan whose batch is on the GPU is
//     admitted as soon as a stream and a context are free, and its work overlaps the other's.
#include <cuda_runtime_api.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <tuple>
#include <vector>

#include "hankel.h"

namespace hk {
bool alloc_fault();  // api.cpp: hankel_debug_fail_allocs
}

namespace {

typedef std::chrono::steady_clock Clock;
typedef std::tuple<int, int, int64_t, double> Key;        // task, nu, N, eps
typedef std::tuple<int, int, int64_t, double, int> PKey;  // Key and the plan class (0: small batches)

PKey plan_key(const Key& k, int cls) { return PKey(std::get<0>(k), std::get<1>(k), std::get<2>(k), std::get<3>(k), cls); }

constexpr size_t kDefaultCap = size_t(120) << 30;
constexpr size_t kPlanWorkspace = size_t(1) << 30;

struct Request {
  Key key;
  const double* c;
  double* f;
  int nrhs;
  bool c_pinned = false, f_pinned = false;  // page-locked host arrays: copied without staging
  Clock::time_point t_submit, t_done;
  int status = HANKEL_OK;
  bool done = false;
};

struct PlanEntry {
  hankel_plan_t plan = nullptr;
  size_t bytes = 0;
  size_t ctx_bytes = 0;         // device bytes of one more execution context
  std::vector<char> ctx_busy;   // per execution context: a batch is in flight on it
  int ctx_limit = 1 << 30;      // contexts the memory cap allowed at the last failed attempt to add one
  int64_t runs = 0;
  uint64_t last_used = 0;
  std::map<std::tuple<int, int, int>, cudaGraphExec_t> graphs;  // (stream slot, context, nrhs) -> graph
  std::map<std::tuple<int, int, int>, int> seen;                 // keys run once, uncaptured
  bool any_busy() const {
    for (char b : ctx_busy)
      if (b) return true;
    return false;
  }
  int idle_ctx() const {
    for (size_t i = 0; i < ctx_busy.size(); ++i)
      if (!ctx_busy[i]) return (int)i;
    return -1;
  }
};

// A request as the dispatcher carries it through a batch (copied under the lock).
struct Item {
  int64_t ticket;
  const double* c;
  double* f;
  int nrhs;
  bool c_pinned, f_pinned;
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  double* c_pin = nullptr;
  double* f_pin = nullptr;
  double* c_dev = nullptr;
  double* f_dev = nullptr;
  size_t cap = 0;      // doubles in each device buffer
  size_t pin_cap = 0;  // doubles in each staging buffer (allocated only for pageable requests)
  bool busy = false;
  std::vector<Item> items;
  PKey key;
  int ctx = 0;  // the plan's execution context the batch runs on
  int64_t N = 0;
};

}  // namespace

struct hankel_server_s {
  hankel_server_options opt;
  int device = 0;
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request> reqs;   // indexed by ticket
  std::deque<int64_t> queue;  // tickets waiting for dispatch
  int64_t outstanding = 0;    // submitted but not completed
  bool stop = false;
  hankel_server_stats stats{};
  // dispatcher-owned
  std::map<PKey, PlanEntry> plans;
  std::vector<Slot> slots;
  uint64_t tick = 0;
  size_t plan_bytes = 0, slot_bytes = 0;
};

namespace {

// The class of plan a batch of nrhs vectors runs on: 0 (built for small_batch vectors) when it
// has at most that many and the option is on, else 1 (built for max_batch).
int plan_class(const hankel_server_s* s, int nrhs) { return s->opt.small_batch > 0 && nrhs <= s->opt.small_batch ? 0 : 1; }

void drop_slot_graphs(hankel_server_s* s, int slot) {
  for (auto& kv : s->plans) {
    for (auto it = kv.second.graphs.begin(); it != kv.second.graphs.end();) {
      if (std::get<0>(it->first) == slot) {
        cudaGraphExecDestroy(it->second);
        it = kv.second.graphs.erase(it);
      } else {
        ++it;
      }
    }
  }
}

void free_slot_buffers(Slot& sl) {
  if (sl.c_pin) cudaFreeHost(sl.c_pin);
  if (sl.f_pin) cudaFreeHost(sl.f_pin);
  if (sl.c_dev) cudaFree(sl.c_dev);
  if (sl.f_dev) cudaFree(sl.f_dev);
  sl.c_pin = sl.f_pin = sl.c_dev = sl.f_dev = nullptr;
  sl.cap = sl.pin_cap = 0;
}

// Device buffers of slot i for need doubles each (growing drops the slot's graphs, which hold
// the buffers' addresses) and, with staging, page-locked staging buffers of the same size.
// The slot is idle, so nothing in flight uses the buffers being replaced.
int ensure_slot_capacity(hankel_server_s* s, int i, size_t need, bool staging) {
  Slot& sl = s->slots[i];
  const size_t cap = std::max(need, size_t(1) << 16);
  if (sl.cap < need) {
    drop_slot_graphs(s, i);
    s->slot_bytes -= 2 * sl.cap * sizeof(double);
    if (sl.c_dev) cudaFree(sl.c_dev);
    if (sl.f_dev) cudaFree(sl.f_dev);
    sl.c_dev = sl.f_dev = nullptr;
    sl.cap = 0;
    if (hk::alloc_fault() || cudaMalloc((void**)&sl.c_dev, cap * sizeof(double)) != cudaSuccess ||
        hk::alloc_fault() || cudaMalloc((void**)&sl.f_dev, cap * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      free_slot_buffers(sl);
      return HANKEL_ENOMEM;
    }
    sl.cap = cap;
    s->slot_bytes += 2 * cap * sizeof(double);
  }
  if (staging && sl.pin_cap < need) {
    if (sl.c_pin) cudaFreeHost(sl.c_pin);
    if (sl.f_pin) cudaFreeHost(sl.f_pin);
    sl.c_pin = sl.f_pin = nullptr;
    sl.pin_cap = 0;
    if (hk::alloc_fault() || cudaMallocHost((void**)&sl.c_pin, cap * sizeof(double)) != cudaSuccess ||
        hk::alloc_fault() || cudaMallocHost((void**)&sl.f_pin, cap * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      s->slot_bytes -= 2 * sl.cap * sizeof(double);
      drop_slot_graphs(s, i);
      free_slot_buffers(sl);
      return HANKEL_ENOMEM;
    }
    sl.pin_cap = cap;
  }
  return HANKEL_OK;
}

void destroy_plan(hankel_server_s* s, PlanEntry& pe) {
  for (auto& g : pe.graphs) cudaGraphExecDestroy(g.second);
  pe.graphs.clear();
  hankel_destroy(pe.plan);
  s->plan_bytes -= pe.bytes;
  pe.plan = nullptr;
  for (auto& kv : s->plans) kv.second.ctx_limit = 1 << 30;  // memory was freed: contexts may be added again
}

// Cached plan for key, built on a miss; idle plans are evicted (LRU) while over the cap.
int get_plan(hankel_server_s* s, const PKey& key, PlanEntry** out) {
  auto it = s->plans.find(key);
  if (it == s->plans.end()) {
    hankel_options o;
    hankel_options_default(&o, std::get<0>(key), std::get<1>(key), std::get<2>(key), std::get<3>(key));
    o.max_nrhs = std::get<4>(key) == 0 ? s->opt.small_batch : s->opt.max_batch;
    o.precision = s->opt.precision;
    o.workspace_limit = kPlanWorkspace;
    hankel_plan_t p = nullptr;
    int st = hankel_plan_ex(&p, &o);
    if (st != HANKEL_OK) return st;
    hankel_info info;
    hankel_plan_info(p, &info);
    PlanEntry pe;
    pe.plan = p;
    pe.bytes = info.device_bytes;
    pe.ctx_bytes = info.context_bytes;
    pe.ctx_busy.assign((size_t)info.contexts, 0);
    s->plan_bytes += pe.bytes;
    it = s->plans.emplace(key, pe).first;
    std::lock_guard<std::mutex> lk(s->mu);
    s->stats.plans_built++;
  }
  it->second.last_used = ++s->tick;
  const size_t cap = s->opt.memory_cap;
  while (s->plan_bytes + s->slot_bytes > cap) {
    auto victim = s->plans.end();
    for (auto jt = s->plans.begin(); jt != s->plans.end(); ++jt)
      if (jt != it && !jt->second.any_busy() &&
          (victim == s->plans.end() || jt->second.last_used < victim->second.last_used))
        victim = jt;
    if (victim == s->plans.end()) break;  // only busy plans left: admit and let them retire
    destroy_plan(s, victim->second);
    s->plans.erase(victim);
    std::lock_guard<std::mutex> lk(s->mu);
    s->stats.plans_evicted++;
  }
  *out = &it->second;
  return HANKEL_OK;
}

// An idle execution context of pe: an existing one, or a new one while the plan has fewer than
// contexts_per_plan and the device memory cap allows it (idle plans are evicted to make room).
// Returns -1 when every context is busy and no other can be made now.
int take_context(hankel_server_s* s, const PKey& key, PlanEntry& pe) {
  int k = pe.idle_ctx();
  if (k >= 0) return k;
  if ((int)pe.ctx_busy.size() >= std::min(s->opt.contexts_per_plan, pe.ctx_limit)) return -1;
  while (s->plan_bytes + s->slot_bytes + pe.ctx_bytes > s->opt.memory_cap) {
    auto victim = s->plans.end();
    for (auto jt = s->plans.begin(); jt != s->plans.end(); ++jt)
      if (jt->first != key && !jt->second.any_busy() &&
          (victim == s->plans.end() || jt->second.last_used < victim->second.last_used))
        victim = jt;
    if (victim == s->plans.end()) {
      pe.ctx_limit = (int)pe.ctx_busy.size();
      return -1;
    }
    destroy_plan(s, victim->second);
    s->plans.erase(victim);
    std::lock_guard<std::mutex> lk(s->mu);
    s->stats.plans_evicted++;
  }
  int idx = -1;
  const int st = hankel_plan_add_context(pe.plan, &idx);
  hankel_info info;
  hankel_plan_info(pe.plan, &info);  // a failed attempt may still hold some of its memory
  s->plan_bytes += info.device_bytes - pe.bytes;
  pe.bytes = info.device_bytes;
  if (st != HANKEL_OK) {
    pe.ctx_limit = (int)pe.ctx_busy.size();  // until memory is freed by an eviction
    return -1;
  }
  pe.ctx_busy.resize((size_t)info.contexts, 0);
  std::lock_guard<std::mutex> lk(s->mu);
  s->stats.contexts_added++;
  return idx;
}

// Issue copy-in, execution and copy-out of a packed batch on slot i. Page-locked request
// arrays are copied straight to and from the slot's device buffers; the others go through the
// slot's staging buffers (filled by dispatch, emptied by retire). With graphs, the execution
// alone is captured once per (slot, context, batch size), at the key's second use, and replayed
// between the copies: a key that occurs once (a batch size that comes up rarely) runs uncaptured
// and pays no instantiation.
int launch_batch(hankel_server_s* s, int i, PlanEntry& pe, int ctx, int64_t N, int nrhs,
                 const std::vector<Item>& batch) {
  Slot& sl = s->slots[i];
  size_t off = 0;
  for (const Item& it : batch) {
    const size_t n = (size_t)N * it.nrhs;
    const double* src = it.c_pinned ? it.c : sl.c_pin + off;
    if (cudaMemcpyAsync(sl.c_dev + off, src, n * sizeof(double), cudaMemcpyHostToDevice, sl.stream) != cudaSuccess)
      return HANKEL_ECUDA;
    off += n;
  }
  auto exec = [&]() { return hankel_exec_batched_ctx(pe.plan, ctx, sl.c_dev, N, sl.f_dev, N, nrhs, sl.stream); };
  int st = HANKEL_OK;
  const auto key = std::make_tuple(i, ctx, nrhs);
  auto git = pe.graphs.find(key);
  if (!s->opt.use_graphs || pe.runs == 0 || (git == pe.graphs.end() && pe.seen[key]++ == 0)) {
    st = exec();  // the plan's first run configures kernels; a key's first run goes uncaptured
  } else {
    if (git == pe.graphs.end()) {
      cudaGraph_t g = nullptr;
      if (cudaStreamBeginCapture(sl.stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return HANKEL_ECUDA;
      st = exec();
      cudaError_t e = cudaStreamEndCapture(sl.stream, &g);
      if (st != HANKEL_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return st != HANKEL_OK ? st : HANKEL_ECUDA;
      }
      cudaGraphExec_t ge = nullptr;
      e = cudaGraphInstantiate(&ge, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return HANKEL_ECUDA;
      git = pe.graphs.emplace(key, ge).first;
      std::lock_guard<std::mutex> lk(s->mu);
      s->stats.graphs_captured++;
    }
    if (cudaGraphLaunch(git->second, sl.stream) != cudaSuccess) st = HANKEL_ECUDA;
  }
  if (st != HANKEL_OK) return st;
  off = 0;
  for (const Item& it : batch) {
    const size_t n = (size_t)N * it.nrhs;
    double* dst = it.f_pinned ? it.f : sl.f_pin + off;
    if (cudaMemcpyAsync(dst, sl.f_dev + off, n * sizeof(double), cudaMemcpyDeviceToHost, sl.stream) != cudaSuccess)
      return HANKEL_ECUDA;
    off += n;
  }
  return HANKEL_OK;
}

void finish(hankel_server_s* s, const std::vector<Item>& items, int status) {
  std::lock_guard<std::mutex> lk(s->mu);
  const auto now = Clock::now();
  for (const Item& it : items) {
    Request& r = s->reqs[it.ticket];
    r.done = true;
    r.status = status;
    r.t_done = now;
    s->outstanding--;
    if (status == HANKEL_OK) {
      s->stats.completed++;
      s->stats.coefficients += (double)std::get<2>(r.key) * r.nrhs;
    } else {
      s->stats.failed++;
    }
  }
  s->cv_done.notify_all();
}

// Retire finished batches. Returns true if any finished.
bool retire(hankel_server_s* s) {
  bool any = false;
  for (size_t i = 0; i < s->slots.size(); ++i) {
    Slot& sl = s->slots[i];
    if (!sl.busy) continue;
    cudaError_t q = cudaEventQuery(sl.done);
    if (q == cudaErrorNotReady) continue;
    int status = q == cudaSuccess ? HANKEL_OK : HANKEL_ECUDA;
    if (status == HANKEL_OK) {
      size_t off = 0;
      for (const Item& it : sl.items) {
        if (!it.f_pinned) memcpy(it.f, sl.f_pin + off, (size_t)sl.N * it.nrhs * sizeof(double));
        off += (size_t)sl.N * it.nrhs;
      }
    }
    auto pit = s->plans.find(sl.key);
    if (pit != s->plans.end() && sl.ctx < (int)pit->second.ctx_busy.size()) pit->second.ctx_busy[sl.ctx] = 0;
    finish(s, sl.items, status);
    sl.items.clear();
    sl.busy = false;
    any = true;
  }
  return any;
}

// Fill one idle slot. Returns true if a batch was dispatched.
bool dispatch(hankel_server_s* s, int i) {
  std::vector<Item> batch;
  Key key;
  int nrhs = 0;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    // a plan is busy when every context it has or may still get carries a batch
    auto busy = [&](const PKey& k) {
      auto it = s->plans.find(k);
      return it != s->plans.end() && it->second.idle_ctx() < 0 &&
             (int)it->second.ctx_busy.size() >= std::min(s->opt.contexts_per_plan, it->second.ctx_limit);
    };
    // the oldest queued request whose plan is idle and whose batch is ready: full, packing off,
    // no request of the plan arrived within the batch window (a burst of submissions stays one
    // batch), or its oldest request has waited ten windows. The plan is the one of the class the
    // batch would take (its vectors so far; the batch formed below settles it)
    const Clock::time_point now = Clock::now();
    const auto window = std::chrono::microseconds(std::max(0, s->opt.batch_window_us));
    std::vector<Key> seen;
    auto q = s->queue.begin();
    for (; q != s->queue.end(); ++q) {
      const Request& r0 = s->reqs[*q];
      if (std::find(seen.begin(), seen.end(), r0.key) != seen.end()) continue;
      seen.push_back(r0.key);
      int queued = 0;
      Clock::time_point newest = r0.t_submit;
      for (int64_t t : s->queue)
        if (s->reqs[t].key == r0.key) {
          queued += s->reqs[t].nrhs;
          newest = std::max(newest, s->reqs[t].t_submit);
        }
      if (!s->opt.pack_requests) queued = r0.nrhs;
      if (busy(plan_key(r0.key, plan_class(s, std::min(queued, s->opt.max_batch))))) continue;
      if (!s->opt.pack_requests) break;
      if (queued >= s->opt.max_batch || now - newest >= window || now - r0.t_submit >= 10 * window) break;
    }
    if (q == s->queue.end()) return false;
    key = s->reqs[*q].key;
    for (auto it = s->queue.begin(); it != s->queue.end();) {
      const Request& r = s->reqs[*it];
      if (r.key == key && nrhs + r.nrhs <= s->opt.max_batch && (s->opt.pack_requests || batch.empty())) {
        nrhs += r.nrhs;
        batch.push_back(Item{*it, r.c, r.f, r.nrhs, r.c_pinned, r.f_pinned});
        it = s->queue.erase(it);
      } else {
        ++it;
      }
    }
  }
  const PKey pkey = plan_key(key, plan_class(s, nrhs));
  PlanEntry* pe = nullptr;
  int st = get_plan(s, pkey, &pe);
  const int64_t N = std::get<2>(key);
  bool staging = false;
  for (const Item& it : batch) staging = staging || !it.c_pinned || !it.f_pinned;
  int ctx = -1;
  if (st == HANKEL_OK) {
    ctx = take_context(s, pkey, *pe);
    if (ctx < 0) {
      // no context can be had now (memory): put the batch back at the front of the queue; it
      // is dispatched once a batch of this plan retires
      std::lock_guard<std::mutex> lk(s->mu);
      for (auto it = batch.rbegin(); it != batch.rend(); ++it) s->queue.push_front(it->ticket);
      return false;
    }
  }
  if (st == HANKEL_OK) st = ensure_slot_capacity(s, i, (size_t)N * nrhs, staging);
  if (st != HANKEL_OK) {
    finish(s, batch, st);
    return true;
  }
  Slot& sl = s->slots[i];
  size_t off = 0;
  for (const Item& it : batch) {
    if (!it.c_pinned) memcpy(sl.c_pin + off, it.c, (size_t)N * it.nrhs * sizeof(double));
    off += (size_t)N * it.nrhs;
  }
  st = launch_batch(s, i, *pe, ctx, N, nrhs, batch);
  if (st == HANKEL_OK && cudaEventRecord(sl.done, sl.stream) != cudaSuccess) st = HANKEL_ECUDA;
  if (st != HANKEL_OK) {
    cudaStreamSynchronize(sl.stream);
    cudaGetLastError();
    finish(s, batch, st);
    return true;
  }
  pe->ctx_busy[ctx] = 1;
  pe->runs++;
  sl.busy = true;
  sl.items = batch;
  sl.key = pkey;
  sl.ctx = ctx;
  sl.N = N;
  std::lock_guard<std::mutex> lk(s->mu);
  s->stats.batches++;
  s->stats.vectors += nrhs;
  return true;
}

void run(hankel_server_s* s) {
  cudaSetDevice(s->device);
  for (;;) {
    bool progressed = retire(s);
    for (size_t i = 0; i < s->slots.size(); ++i)
      if (!s->slots[i].busy && dispatch(s, (int)i)) progressed = true;
    bool inflight = false;
    for (const Slot& sl : s->slots) inflight |= sl.busy;
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->stop && s->queue.empty() && !inflight) break;
    if (progressed) continue;
    if (inflight || !s->queue.empty()) {
      // batches are running, or queued requests wait for their batch window: look again
      // shortly, or sooner if work arrives
      s->cv_work.wait_for(lk, std::chrono::microseconds(20));
    } else {
      s->cv_work.wait(lk, [&] { return s->stop || !s->queue.empty(); });
    }
  }
}

}  // namespace

extern "C" {

int hankel_server_options_default(hankel_server_options* o) {
  if (!o) return HANKEL_EINVAL;
  memset(o, 0, sizeof(*o));
  o->memory_cap = kDefaultCap;
  o->streams = 4;
  o->max_batch = 64;
  o->use_graphs = 0;
  o->precision = HANKEL_PREC_AUTO;
  o->pack_requests = 1;
  o->batch_window_us = 200;
  o->contexts_per_plan = 2;
  o->small_batch = 0;
  return HANKEL_OK;
}

int hankel_server_create(hankel_server_t* out, const hankel_server_options* o) {
  if (!out) return HANKEL_EINVAL;
  *out = nullptr;
  hankel_server_options opt;
  hankel_server_options_default(&opt);
  if (o) opt = *o;
  if (opt.memory_cap == 0) opt.memory_cap = kDefaultCap;
  if (opt.streams < 1 || opt.streams > 16 || opt.max_batch < 1 || opt.batch_window_us < 0) return HANKEL_EINVAL;
  if (opt.contexts_per_plan < 1 || opt.contexts_per_plan > 8) return HANKEL_EINVAL;
  if (opt.small_batch < 0 || opt.small_batch >= opt.max_batch) opt.small_batch = 0;  // one plan per key
  if (opt.precision != HANKEL_PREC_AUTO && opt.precision != HANKEL_PREC_FP64 && opt.precision != HANKEL_PREC_MIXED)
    return HANKEL_EINVAL;
  hankel_server_s* s = new hankel_server_s();
  s->opt = opt;
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    return HANKEL_ECUDA;
  }
  s->slots.resize(opt.streams);
  for (Slot& sl : s->slots) {
    if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      for (Slot& t : s->slots) {
        if (t.stream) cudaStreamDestroy(t.stream);
        if (t.done) cudaEventDestroy(t.done);
      }
      delete s;
      return HANKEL_ECUDA;
    }
  }
  s->worker = std::thread(run, s);
  *out = s;
  return HANKEL_OK;
}

int hankel_server_submit(hankel_server_t s, int task, int nu, int64_t N, double eps, const double* c, double* f,
                         int nrhs, int64_t* ticket) {
  if (!s || !c || !f || !ticket || nrhs < 1 || nrhs > s->opt.max_batch || N < 2) return HANKEL_EINVAL;
  hankel_options o;
  hankel_options_default(&o, task, nu, N, eps);
  o.precision = s->opt.precision;
  hankel_info info;
  int st = hankel_params(&o, &info);  // reject bad parameters now, without a GPU round trip
  if (st != HANKEL_OK) return st;
  // page-locked arrays (allocated with cudaMallocHost or registered) skip the staging copies
  auto pinned = [](const void* q) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, q) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    return a.type == cudaMemoryTypeHost;
  };
  const bool cp = pinned(c), fp = pinned(f);
  std::lock_guard<std::mutex> lk(s->mu);
  Request r;
  r.key = Key(task, nu, N, eps);
  r.c = c;
  r.f = f;
  r.nrhs = nrhs;
  r.c_pinned = cp;
  r.f_pinned = fp;
  r.t_submit = Clock::now();
  s->reqs.push_back(r);
  *ticket = (int64_t)s->reqs.size() - 1;
  s->queue.push_back(*ticket);
  s->outstanding++;
  s->stats.submitted++;
  s->cv_work.notify_one();
  return HANKEL_OK;
}

int hankel_server_wait(hankel_server_t s, int64_t ticket, int* status, double* latency_ms) {
  if (!s) return HANKEL_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  if (ticket < 0 || ticket >= (int64_t)s->reqs.size()) return HANKEL_EINVAL;
  s->cv_done.wait(lk, [&] { return s->reqs[ticket].done; });
  const Request& r = s->reqs[ticket];
  if (status) *status = r.status;
  if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r.t_done - r.t_submit).count();
  return HANKEL_OK;
}

int hankel_server_cancel(hankel_server_t s, int64_t ticket, int* cancelled) {
  if (!s) return HANKEL_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (ticket < 0 || ticket >= (int64_t)s->reqs.size()) return HANKEL_EINVAL;
  if (cancelled) *cancelled = 0;
  auto it = std::find(s->queue.begin(), s->queue.end(), ticket);
  if (it == s->queue.end()) return HANKEL_OK;  // in a batch already, or done
  s->queue.erase(it);
  Request& r = s->reqs[ticket];
  r.done = true;
  r.status = HANKEL_ECANCELED;
  r.t_done = Clock::now();
  s->outstanding--;
  s->stats.failed++;
  s->stats.cancelled++;
  if (cancelled) *cancelled = 1;
  s->cv_done.notify_all();
  return HANKEL_OK;
}

int hankel_server_drain(hankel_server_t s) {
  if (!s) return HANKEL_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  s->cv_done.wait(lk, [&] { return s->outstanding == 0; });
  return HANKEL_OK;
}

int hankel_server_get_stats(hankel_server_t s, hankel_server_stats* out) {
  if (!s || !out) return HANKEL_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->stats;
  out->device_bytes = s->plan_bytes + s->slot_bytes;
  return HANKEL_OK;
}

int hankel_server_destroy(hankel_server_t s) {
  if (!s) return HANKEL_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv_work.notify_all();
  }
  s->worker.join();
  cudaSetDevice(s->device);
  for (auto& kv : s->plans) destroy_plan(s, kv.second);
  s->plans.clear();
  for (Slot& sl : s->slots) {
    cudaStreamSynchronize(sl.stream);
    free_slot_buffers(sl);
    cudaStreamDestroy(sl.stream);
    cudaEventDestroy(sl.done);
  }
  delete s;
  return HANKEL_OK;
}

}  // extern "C"
