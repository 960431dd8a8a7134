// Continuous-batching request loop (see include/gq_server.h for the contract).
//
// One native worker thread owns the lanes and the resident warm-start cache:
//   retire   a lane whose completion event has fired: copy every request's
//            solution from the lane's pinned staging to the caller's buffers,
//            release its cache pins and keys, mark the tickets done;
//   admit    while a lane is free and requests wait: take them in arrival
//            order (skipping those whose key is still being solved), plan the
//            micro-batch with the batch planner, halve it until it fits the
//            lane's device and pinned partitions, copy each distinct stage
//            data block from the request sources into the lane's staging;
//   launch   on the lane's stream: one host-to-device copy of inputs and copy
//            descriptors, a gather of resident iterates into the warm QPs'
//            solution slots, the IPM solve, a scatter of the keyed solutions
//            into the cache, one device-to-host copy of the solution block,
//            and the completion event.
// Lanes run concurrently, so micro-batches admitted while others are on the
// GPU overlap with them.
#include <cuda_runtime.h>
#include <time.h>

#include <algorithm>
#include <cmath>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "../../include/gq_server.h"
#include "gq_batch.h"

static_assert(sizeof(gq_server_cfg) == 16 + 8 + sizeof(gq_ipm_arg) + 8, "gq_server_cfg layout");
static_assert(sizeof(gq_request) == 64, "gq_request layout");
static_assert(sizeof(gq_ticket_info) == 32 + sizeof(gq_stats), "gq_ticket_info layout");
static_assert(sizeof(gq_server_report) == 15 * 8, "gq_server_report layout");

namespace {

int64_t now_ns() {
  timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return (int64_t)ts.tv_sec * 1000000000LL + ts.tv_nsec;
}

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// One contiguous copy of `len` doubles (offsets in doubles).
struct CopyOp {
  int64_t src, dst, len;
};

// Copies op ranges src[op.src..] -> dst[op.dst..]; one block per op.
__global__ void copy_ranges_kernel(const CopyOp* __restrict__ ops, int nops, const double* __restrict__ src,
                                   double* __restrict__ dst) {
  for (int o = blockIdx.x; o < nops; o += gridDim.x) {
    const CopyOp op = ops[o];
    for (int64_t i = threadIdx.x; i < op.len; i += blockDim.x) dst[op.dst + i] = src[op.src + i];
  }
}

struct Req {
  gq_request r;
  int64_t ticket;
  int64_t t_arr;
  int32_t attempt;  // 1 after a warm start that did not converge was re-queued cold
  int32_t cls;      // size class (power of class_ratio of the cost estimate)
};

struct Ticket {
  gq_ticket_info info;
};

// A resident iterate [y | pi | lam | t] of one key in the device cache.
struct Entry {
  int64_t id;
  int64_t off, len;  // doubles
  int64_t nvt, neqt, nside;
  uint64_t key;
  int pins;
  bool live;
};

struct Lane {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  char* dev = nullptr;
  size_t dev_bytes = 0;
  char* pin = nullptr;
  size_t pin_bytes = 0;
  std::vector<unsigned char> handle;  // batch handle memory
  gq_batch* b = nullptr;
  std::vector<Req> reqs;
  std::vector<int> warm_used;
  std::vector<int64_t> pinned_ids;
  int64_t t_admit = 0;
  int launch_code = GQ_OK;
  bool busy = false;
};

}  // namespace

struct gq_server {
  gq_server_cfg cfg;
  char* dev_arena;
  size_t dev_bytes;
  double* cache;  // device, cache_len doubles
  int64_t cache_len;

  std::vector<Lane> lanes;

  // shared with submitters (under mu)
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::list<Req> pending;
  std::vector<Ticket> tickets;
  int64_t outstanding = 0;
  bool stop = false;
  bool broken = false;
  gq_server_report rep;

  // worker-private
  struct {
    int64_t warm_hits = 0, warm_misses = 0, cache_entries = 0, cache_evictions = 0, cache_skips = 0;
  } wc;  // cache counters, copied into rep under mu by the worker
  std::deque<Entry> ring;
  int64_t ring_next_id = 0;
  int64_t head = 0;
  std::unordered_map<uint64_t, int64_t> where;  // key -> entry id
  std::unordered_set<uint64_t> busy_keys;
  std::thread worker;
};

namespace {

using gq::set_error;

// ---------------------------------------------------------------------------
// resident cache: a ring of variable-size entries in allocation order
// ---------------------------------------------------------------------------
Entry* entry_by_id(gq_server* s, int64_t id) {
  if (s->ring.empty()) return nullptr;
  const int64_t first = s->ring.front().id;
  if (id < first || id >= first + (int64_t)s->ring.size()) return nullptr;
  return &s->ring[(size_t)(id - first)];
}

// Evicts the oldest entry; false if it is pinned by a lane in flight.
bool evict_front(gq_server* s) {
  Entry& e = s->ring.front();
  if (e.pins > 0) return false;
  if (e.live) {
    auto it = s->where.find(e.key);
    if (it != s->where.end() && it->second == e.id) s->where.erase(it);
    s->wc.cache_evictions++;
    s->wc.cache_entries--;
  }
  s->ring.pop_front();
  return true;
}

// Allocates len doubles; returns the entry id or -1 (too large, or the space
// it needs still belongs to an entry a lane in flight reads or writes).
int64_t cache_alloc(gq_server* s, int64_t len, uint64_t key, int64_t nvt, int64_t neqt, int64_t nside) {
  if (len <= 0 || len > s->cache_len) return -1;
  int64_t start = s->head;
  if (start + len > s->cache_len) {
    // wrap: everything still stored beyond the head is the oldest lap
    while (!s->ring.empty() && s->ring.front().off >= s->head) {
      if (!evict_front(s)) return -1;
    }
    start = 0;
  }
  while (!s->ring.empty()) {
    const Entry& f = s->ring.front();
    const bool overlap = f.off < start + len && start < f.off + f.len;
    if (!overlap) break;
    if (!evict_front(s)) return -1;
  }
  Entry e;
  e.id = s->ring_next_id++;
  e.off = start;
  e.len = len;
  e.nvt = nvt;
  e.neqt = neqt;
  e.nside = nside;
  e.key = key;
  e.pins = 0;
  e.live = true;
  s->ring.push_back(e);
  s->head = start + len;
  s->wc.cache_entries++;
  return e.id;
}

// ---------------------------------------------------------------------------
// micro-batch planning
// ---------------------------------------------------------------------------
struct Plan {
  std::vector<int> dims;
  std::vector<int> slots;
  std::vector<int> ns;
};

void plan_dims(const std::vector<Req>& reqs, size_t count, Plan* p) {
  p->dims.clear();
  p->slots.clear();
  p->ns.clear();
  // stages that read the same source block share one block in the lane
  std::unordered_map<const void*, int> ids;
  ids.reserve(count * 4);
  for (size_t j = 0; j < count; ++j) {
    const gq_batch* src = reqs[j].r.src;
    const gq::QpDesc& q = src->qp[reqs[j].r.src_qp];
    p->dims.push_back(q.N);
    for (int n = 0; n <= q.N; ++n) {
      const gq::StageDesc& st = src->st[q.stage0 + n];
      p->dims.push_back(st.nx);
      p->dims.push_back(st.nu);
      p->dims.push_back(st.nbx);
      p->dims.push_back(st.nbu);
      p->dims.push_back(st.ng);
      p->ns.push_back(st.ns);
      const void* blk = static_cast<const char*>(src->host_in) + src->L.data + 8 * (int64_t)st.data;
      auto it = ids.find(blk);
      if (it == ids.end()) it = ids.emplace(blk, (int)ids.size()).first;
      p->slots.push_back(it->second);
    }
  }
}

struct Fit {
  size_t in_bytes, ops_bytes, sol_bytes, ws_bytes;
};

// Builds the lane batch for the first `count` requests; returns GQ_OK and the
// byte sizes, or an error code.
int build_batch(gq_server* s, Lane& L, const std::vector<Req>& reqs, size_t count, Plan* p, Fit* f) {
  plan_dims(reqs, count, p);
  const size_t need = gq_batch_memsize((int)count, p->dims.data(), p->dims.size(), p->slots.data());
  if (need == 0) return GQ_ERR_DIMS;
  if (L.handle.size() < need + 64) L.handle.resize(need + 64);
  unsigned char* base = L.handle.data();
  unsigned char* mem = base + ((64 - (reinterpret_cast<uintptr_t>(base) % 64)) % 64);
  gq_batch* b = nullptr;
  int rc = gq_batch_create_soft((int)count, p->dims.data(), p->dims.size(), p->slots.data(), p->ns.data(), mem,
                                need, &b);
  if (rc) return rc;
  L.b = b;
  f->in_bytes = align256(b->sizes.in_bytes);
  f->ops_bytes = align256(sizeof(CopyOp) * 8 * count);
  f->sol_bytes = align256(b->sizes.sol_bytes);
  f->ws_bytes = align256(b->sizes.ws_bytes);
  (void)s;
  return GQ_OK;
}

bool fits(const Lane& L, const Fit& f) {
  return f.in_bytes + f.ops_bytes + f.sol_bytes + f.ws_bytes <= L.dev_bytes &&
         f.in_bytes + f.ops_bytes + f.sol_bytes <= L.pin_bytes;
}

void complete_ticket(gq_server* s, const Req& r, int code, const gq_stats* st, int warm_used, int bsize,
                     int64_t t_admit, int64_t t_done) {
  Ticket& t = s->tickets[(size_t)r.ticket];
  t.info.code = code;
  t.info.warm_used = warm_used;
  t.info.batch_size = bsize;
  t.info.latency_ns = t_done - r.t_arr;
  t.info.wait_ns = t_admit > 0 ? t_admit - r.t_arr : 0;
  if (st) t.info.stats = *st;
  t.info.done = 1;
  s->outstanding--;
  if (code == GQ_OK)
    s->rep.completed++;
  else if (code == GQ_ERR_SIZE)
    s->rep.rejected++;
  else
    s->rep.failed++;
}

// ---------------------------------------------------------------------------
// retire
// ---------------------------------------------------------------------------
void retire(gq_server* s, Lane& L) {
  const gq_batch* b = L.b;
  const size_t in_ops = align256(b->sizes.in_bytes) + align256(sizeof(CopyOp) * 8 * L.reqs.size());
  const char* sol = L.pin + in_ops;
  const int64_t t_done_base = now_ns();
  // outputs first, outside the lock (caller buffers are private per ticket)
  for (size_t j = 0; j < L.reqs.size() && L.launch_code == GQ_OK; ++j) {
    const gq_request& r = L.reqs[j].r;
    const gq::QpDesc& q = b->qp[j];
    const double* Y = reinterpret_cast<const double*>(sol + b->L.y) + q.var0;
    const double* P = reinterpret_cast<const double*>(sol + b->L.pi) + q.eq0;
    const double* La = reinterpret_cast<const double*>(sol + b->L.lam) + q.side0;
    const double* T = reinterpret_cast<const double*>(sol + b->L.t) + q.side0;
    if (r.y) std::memcpy(r.y, Y, 8 * (size_t)q.nvt);
    if (r.pi) std::memcpy(r.pi, P, 8 * (size_t)q.neqt);
    if (r.lam) std::memcpy(r.lam, La, 8 * (size_t)q.nsidet);
    if (r.t) std::memcpy(r.t, T, 8 * (size_t)q.nsidet);
  }
  for (int64_t id : L.pinned_ids) {
    Entry* e = entry_by_id(s, id);
    if (e) e->pins--;
  }
  L.pinned_ids.clear();
  const int64_t t_done = std::max(t_done_base, now_ns());
  // a warm start that did not converge is solved once more from a cold start
  // (its resident iterate is dropped); it keeps its arrival time
  std::vector<Req> retry;
  if (L.launch_code == GQ_OK) {
    for (size_t j = 0; j < L.reqs.size(); ++j) {
      const gq_stats* st = reinterpret_cast<const gq_stats*>(sol + b->L.stats) + j;
      if (L.warm_used[j] && st->status != GQ_STATUS_CONVERGED && L.reqs[j].attempt == 0) {
        Req r = L.reqs[j];
        r.attempt = 1;
        r.r.warm = 0;
        retry.push_back(r);
        auto it = s->where.find(r.r.key);
        if (it != s->where.end()) {
          Entry* e = entry_by_id(s, it->second);
          if (e && e->live) {
            e->live = false;
            s->wc.cache_entries--;
          }
          s->where.erase(it);
        }
      }
    }
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    size_t k = 0;
    for (size_t j = 0; j < L.reqs.size(); ++j) {
      if (L.reqs[j].r.key) s->busy_keys.erase(L.reqs[j].r.key);
      if (k < retry.size() && retry[k].ticket == L.reqs[j].ticket) {
        ++k;
        continue;
      }
      const gq_stats* st =
          L.launch_code == GQ_OK ? reinterpret_cast<const gq_stats*>(sol + b->L.stats) + j : nullptr;
      complete_ticket(s, L.reqs[j], L.launch_code, st, L.warm_used[j], (int)L.reqs.size(), L.t_admit, t_done);
    }
    for (size_t j = retry.size(); j-- > 0;) s->pending.push_front(retry[j]);
    s->rep.cold_retries += (int64_t)retry.size();
  }
  s->cv_done.notify_all();
  L.reqs.clear();
  L.warm_used.clear();
  L.busy = false;
}

// ---------------------------------------------------------------------------
// admit + launch
// ---------------------------------------------------------------------------
// Takes up to max_batch eligible requests off the queue (arrival order, keys
// not in flight, no key twice).  Returns false if none is eligible.
bool take(gq_server* s, std::vector<Req>* out, bool force) {
  std::lock_guard<std::mutex> lk(s->mu);
  out->clear();
  if (s->pending.empty()) return false;
  std::unordered_set<uint64_t> chosen;
  std::vector<std::list<Req>::iterator> its;
  bool have_cls = false;
  int cls = 0;
  for (auto it = s->pending.begin(); it != s->pending.end() && (int)its.size() < s->cfg.max_batch; ++it) {
    const uint64_t k = it->r.key;
    if (k && (s->busy_keys.count(k) || chosen.count(k))) {
      s->rep.deferrals++;
      continue;
    }
    // the oldest eligible request sets the micro-batch's size class
    if (!have_cls) {
      have_cls = true;
      cls = it->cls;
    } else if (it->cls != cls) {
      continue;
    }
    if (k) chosen.insert(k);
    its.push_back(it);
  }
  if (its.empty()) return false;
  if (!force && (int)its.size() < s->cfg.max_batch && s->cfg.max_wait_us > 0) {
    const int64_t waited = now_ns() - its.front()->t_arr;
    if (waited < (int64_t)s->cfg.max_wait_us * 1000) return false;
  }
  for (auto& it : its) {
    out->push_back(*it);
    if (it->r.key) s->busy_keys.insert(it->r.key);
    s->pending.erase(it);
  }
  return true;
}

// Puts requests [from, end) back at the queue front in their order.
void give_back(gq_server* s, const std::vector<Req>& reqs, size_t from) {
  std::lock_guard<std::mutex> lk(s->mu);
  for (size_t j = reqs.size(); j-- > from;) {
    s->pending.push_front(reqs[j]);
    if (reqs[j].r.key) s->busy_keys.erase(reqs[j].r.key);
  }
}

constexpr int kRejected = 1;

// Admits reqs (or a prefix of them) into lane L and enqueues its device work.
// Returns GQ_OK (launched; reqs holds the admitted prefix), kRejected (reqs[0]
// was completed as too large, the rest went back to the queue) or a negative
// error code (nothing launched; reqs must be retired with that code).
int launch_lane(gq_server* s, Lane& L, std::vector<Req>& reqs) {
  Plan plan;
  Fit fit;
  size_t count = reqs.size();
  int rc = GQ_OK;
  for (;;) {
    rc = build_batch(s, L, reqs, count, &plan, &fit);
    if (rc == GQ_OK && fits(L, fit)) break;
    if (count == 1) {
      // a single QP that does not fit a lane partition is rejected; the
      // other requests go back to the queue front
      const int64_t t = now_ns();
      give_back(s, reqs, 1);
      {
        std::lock_guard<std::mutex> lk(s->mu);
        complete_ticket(s, reqs[0], rc == GQ_OK ? GQ_ERR_SIZE : rc, nullptr, 0, 1, t, t);
        if (reqs[0].r.key) s->busy_keys.erase(reqs[0].r.key);
      }
      s->cv_done.notify_all();
      return kRejected;
    }
    count = (count + 1) / 2;
  }
  if (count < reqs.size()) {
    give_back(s, reqs, count);
    reqs.resize(count);
  }
  gq_batch* b = L.b;
  char* pin_in = L.pin;
  CopyOp* ops = reinterpret_cast<CopyOp*>(L.pin + fit.in_bytes);
  char* pin_sol = L.pin + fit.in_bytes + fit.ops_bytes;
  char* dev_in = L.dev;
  char* dev_ops = L.dev + fit.in_bytes;
  char* dev_sol = dev_ops + fit.ops_bytes;
  char* dev_ws = dev_sol + fit.sol_bytes;
  rc = gq_batch_attach(b, pin_in, pin_sol, dev_in, dev_sol, dev_ws);
  if (rc) return rc;

  // stage data blocks (each distinct block once)
  std::vector<char> copied(b->n_slots > 0 ? (size_t)b->n_slots : 1, 0);
  char* dst_data = pin_in + b->L.data;
  int64_t si = 0;
  for (size_t j = 0; j < count; ++j) {
    const gq_batch* src = reqs[j].r.src;
    const gq::QpDesc& q = src->qp[reqs[j].r.src_qp];
    const char* src_data = static_cast<const char*>(src->host_in) + src->L.data;
    for (int n = 0; n <= q.N; ++n, ++si) {
      const int slot = plan.slots[(size_t)si];
      if (copied[(size_t)slot]) continue;
      copied[(size_t)slot] = 1;
      const gq::StageDesc& ss = src->st[q.stage0 + n];
      const gq::StageDesc& ds = b->st[b->qp[j].stage0 + n];
      const gq::StageData lay = gq::stage_data_layout(ss);
      std::memcpy(dst_data + 8 * ds.data, src_data + 8 * ss.data, 8 * (size_t)lay.size);
    }
  }

  // warm starts from resident iterates; cache slots for the new solutions
  int ngather = 0, nscatter = 0;
  std::vector<CopyOp> scatter;
  L.warm_used.assign(count, 0);
  gq::QpDesc* hq = reinterpret_cast<gq::QpDesc*>(pin_in + b->L.qpdesc);
  const int64_t oy = b->L.y / 8, opi = b->L.pi / 8, olam = b->L.lam / 8, ot = b->L.t / 8;
  for (size_t j = 0; j < count; ++j) {
    const gq_request& r = reqs[j].r;
    const gq::QpDesc& q = b->qp[j];
    int level = 0;
    if (r.key && s->cache_len > 0) {
      auto it = s->where.find(r.key);
      Entry* e = it == s->where.end() ? nullptr : entry_by_id(s, it->second);
      if (r.warm) {
        if (e && e->live && e->nvt == q.nvt && e->neqt == q.neqt && e->nside == q.nsidet) {
          level = 2;
          ops[ngather++] = CopyOp{e->off, oy + q.var0, q.nvt};
          ops[ngather++] = CopyOp{e->off + q.nvt, opi + q.eq0, q.neqt};
          ops[ngather++] = CopyOp{e->off + q.nvt + q.neqt, olam + q.side0, q.nsidet};
          ops[ngather++] = CopyOp{e->off + q.nvt + q.neqt + q.nsidet, ot + q.side0, q.nsidet};
          e->pins++;
          L.pinned_ids.push_back(e->id);
          s->wc.warm_hits++;
        } else {
          s->wc.warm_misses++;
        }
      }
      if (e && e->live) {
        // superseded by this request's solution
        e->live = false;
        s->where.erase(r.key);
        s->wc.cache_entries--;
      }
      const int64_t len = q.nvt + q.neqt + 2 * (int64_t)q.nsidet;
      const int64_t id = cache_alloc(s, len, r.key, q.nvt, q.neqt, q.nsidet);
      if (id >= 0) {
        Entry* ne = entry_by_id(s, id);
        ne->pins++;
        L.pinned_ids.push_back(id);
        s->where[r.key] = id;
        scatter.push_back(CopyOp{oy + q.var0, ne->off, q.nvt});
        scatter.push_back(CopyOp{opi + q.eq0, ne->off + q.nvt, q.neqt});
        scatter.push_back(CopyOp{olam + q.side0, ne->off + q.nvt + q.neqt, q.nsidet});
        scatter.push_back(CopyOp{ot + q.side0, ne->off + q.nvt + q.neqt + q.nsidet, q.nsidet});
      } else {
        s->wc.cache_skips++;
      }
    } else if (r.warm) {
      s->wc.warm_misses++;
    }
    hq[j].warm = level + 1;  // explicit per-QP level (cold = 0)
    b->qp[j].warm = level + 1;
    L.warm_used[j] = level > 0;
  }
  nscatter = (int)scatter.size();
  std::memcpy(ops + ngather, scatter.data(), sizeof(CopyOp) * (size_t)nscatter);

  // device work on the lane stream
  cudaError_t e = cudaMemcpyAsync(dev_in, pin_in, fit.in_bytes + fit.ops_bytes, cudaMemcpyHostToDevice, L.stream);
  if (e == cudaSuccess && ngather > 0) {
    copy_ranges_kernel<<<std::min(ngather, 1024), 128, 0, L.stream>>>(
        reinterpret_cast<const CopyOp*>(dev_ops), ngather, s->cache, reinterpret_cast<double*>(dev_sol));
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return set_error(GQ_ERR_CUDA, "server upload: %s", cudaGetErrorString(e));
  rc = gq_solve(b, &s->cfg.arg, L.stream);
  if (rc) return rc;
  if (nscatter > 0) {
    copy_ranges_kernel<<<std::min(nscatter, 1024), 128, 0, L.stream>>>(
        reinterpret_cast<const CopyOp*>(dev_ops) + ngather, nscatter, reinterpret_cast<const double*>(dev_sol),
        s->cache);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(pin_sol, dev_sol, b->sizes.sol_bytes, cudaMemcpyDeviceToHost, L.stream);
  if (e == cudaSuccess) e = cudaEventRecord(L.done, L.stream);
  if (e != cudaSuccess) return set_error(GQ_ERR_CUDA, "server launch: %s", cudaGetErrorString(e));
  return GQ_OK;
}

void fail_all_pending(gq_server* s, int code) {
  // under mu
  const int64_t t = now_ns();
  while (!s->pending.empty()) {
    Req r = s->pending.front();
    s->pending.pop_front();
    complete_ticket(s, r, code, nullptr, 0, 0, 0, t);
  }
}

void worker_main(gq_server* s) {
  cudaSetDevice(s->cfg.device);
  std::vector<Req> reqs;
  for (;;) {
    bool worked = false;
    int busy = 0;
    for (Lane& L : s->lanes) {
      if (!L.busy) continue;
      const cudaError_t q = cudaEventQuery(L.done);
      if (q == cudaSuccess) {
        retire(s, L);
        worked = true;
      } else if (q != cudaErrorNotReady) {
        L.launch_code = set_error(GQ_ERR_CUDA, "server lane: %s", cudaGetErrorString(q));
        {
          std::lock_guard<std::mutex> lk(s->mu);
          s->broken = true;
        }
        retire(s, L);
        worked = true;
      } else {
        ++busy;
      }
    }
    bool stopping, broken;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      stopping = s->stop;
      broken = s->broken;
      if (broken) fail_all_pending(s, GQ_ERR_CUDA);
      if (busy > s->rep.max_lanes_busy) s->rep.max_lanes_busy = busy;
      s->rep.warm_hits = s->wc.warm_hits;
      s->rep.warm_misses = s->wc.warm_misses;
      s->rep.cache_entries = s->wc.cache_entries;
      s->rep.cache_evictions = s->wc.cache_evictions;
      s->rep.cache_skips = s->wc.cache_skips;
    }
    if (!broken) {
      for (Lane& L : s->lanes) {
        if (L.busy) continue;
        if (!take(s, &reqs, stopping)) break;
        L.t_admit = now_ns();
        L.launch_code = GQ_OK;
        const int rc = launch_lane(s, L, reqs);
        worked = true;
        if (rc == kRejected) continue;
        if (rc != GQ_OK) {
          // nothing (or not all) of the device work was enqueued: wait for
          // what was, then report the error for this micro-batch
          cudaStreamSynchronize(L.stream);
          L.launch_code = rc;
          L.reqs = reqs;
          L.warm_used.assign(reqs.size(), 0);
          retire(s, L);
          continue;
        }
        L.reqs = reqs;
        L.busy = true;
        ++busy;
        std::lock_guard<std::mutex> lk(s->mu);
        s->rep.batches++;
        s->rep.batched_qps += (int64_t)reqs.size();
      }
    }
    if (stopping) {
      bool any = false;
      for (Lane& L : s->lanes) any |= L.busy;
      std::lock_guard<std::mutex> lk(s->mu);
      if (!any && (s->pending.empty() || broken)) break;
    }
    if (!worked) {
      std::unique_lock<std::mutex> lk(s->mu);
      if (busy > 0)
        s->cv_work.wait_for(lk, std::chrono::microseconds(10));
      else if (s->pending.empty() && !s->stop)
        s->cv_work.wait_for(lk, std::chrono::milliseconds(2));
      else
        s->cv_work.wait_for(lk, std::chrono::microseconds(20));
    }
  }
}

}  // namespace

extern "C" {

int gq_server_cfg_default(gq_server_cfg* cfg) {
  if (cfg == nullptr) return set_error(GQ_ERR_ARG, "cfg is NULL");
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->lanes = 4;
  cfg->max_batch = 256;
  cfg->max_wait_us = 0;
  cfg->device = 0;
  cfg->cache_bytes = 0;
  cfg->class_ratio = 4.0;
  return gq_ipm_arg_default(&cfg->arg, GQ_MODE_SPEED, GQ_PREC_MIXED);
}

int gq_server_create(const gq_server_cfg* cfg, void* dev_arena, size_t dev_bytes, void* pinned, size_t pinned_bytes,
                     gq_server** out) {
  if (out == nullptr) return set_error(GQ_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (cfg == nullptr || dev_arena == nullptr || pinned == nullptr)
    return set_error(GQ_ERR_ARG, "cfg, dev_arena and pinned must be non-NULL");
  if (cfg->lanes < 1 || cfg->lanes > 64) return set_error(GQ_ERR_ARG, "lanes must be in 1..64");
  if (cfg->max_batch < 1) return set_error(GQ_ERR_ARG, "max_batch must be >= 1");
  if (cfg->max_wait_us < 0) return set_error(GQ_ERR_ARG, "max_wait_us must be >= 0");
  if (reinterpret_cast<uintptr_t>(dev_arena) % 256) return set_error(GQ_ERR_ARG, "dev_arena must be 256-byte aligned");
  if (reinterpret_cast<uintptr_t>(pinned) % 16) return set_error(GQ_ERR_ARG, "pinned must be 16-byte aligned");
  if (cfg->arg.warm_start < 0 || cfg->arg.warm_start > 2) return set_error(GQ_ERR_ARG, "arg.warm_start out of range");
  const size_t cache = align256(cfg->cache_bytes);
  if (dev_bytes <= cache + 256u * (size_t)cfg->lanes)
    return set_error(GQ_ERR_SIZE, "device arena %zu bytes leaves nothing for %d lanes after a %zu-byte cache",
                     dev_bytes, cfg->lanes, cache);
  if (pinned_bytes < 256u * (size_t)cfg->lanes) return set_error(GQ_ERR_SIZE, "pinned arena too small");

  gq_server* s = new (std::nothrow) gq_server();
  if (s == nullptr) return set_error(GQ_ERR_SIZE, "out of host memory");
  s->cfg = *cfg;
  s->dev_arena = static_cast<char*>(dev_arena);
  s->dev_bytes = dev_bytes;
  s->cache = reinterpret_cast<double*>(dev_arena);
  s->cache_len = (int64_t)(cfg->cache_bytes / 8);
  std::memset(&s->rep, 0, sizeof(s->rep));
  const size_t lane_dev = ((dev_bytes - cache) / (size_t)cfg->lanes) & ~size_t(255);
  const size_t lane_pin = (pinned_bytes / (size_t)cfg->lanes) & ~size_t(255);
  s->lanes.resize((size_t)cfg->lanes);
  int prev = 0;
  cudaGetDevice(&prev);
  cudaError_t e = cudaSetDevice(cfg->device);
  for (int i = 0; i < cfg->lanes && e == cudaSuccess; ++i) {
    Lane& L = s->lanes[(size_t)i];
    L.dev = s->dev_arena + cache + lane_dev * (size_t)i;
    L.dev_bytes = lane_dev;
    L.pin = static_cast<char*>(pinned) + lane_pin * (size_t)i;
    L.pin_bytes = lane_pin;
    e = cudaStreamCreateWithFlags(&L.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming);
  }
  cudaSetDevice(prev);
  if (e != cudaSuccess) {
    for (Lane& L : s->lanes) {
      if (L.done) cudaEventDestroy(L.done);
      if (L.stream) cudaStreamDestroy(L.stream);
    }
    delete s;
    return set_error(GQ_ERR_CUDA, "server streams: %s", cudaGetErrorString(e));
  }
  s->worker = std::thread(worker_main, s);
  *out = s;
  return GQ_OK;
}

int gq_server_submit(gq_server* s, const gq_request* req, int64_t* ticket) {
  if (s == nullptr || req == nullptr || ticket == nullptr) return set_error(GQ_ERR_ARG, "NULL argument");
  const gq_batch* src = req->src;
  if (src == nullptr || src->host_in == nullptr)
    return set_error(GQ_ERR_ARG, "request source must be a batch with host_in attached");
  if (req->src_qp < 0 || req->src_qp >= src->nqp) return set_error(GQ_ERR_ARG, "src_qp out of range");
  Req r;
  r.r = *req;
  r.t_arr = req->t_arrival_ns > 0 ? req->t_arrival_ns : now_ns();
  r.attempt = 0;
  r.cls = 0;
  if (s->cfg.class_ratio > 1.0) {
    const double c = src->qp[req->src_qp].cost;
    r.cls = (int32_t)std::floor(std::log(c > 1.0 ? c : 1.0) / std::log(s->cfg.class_ratio));
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->broken || s->stop) return set_error(GQ_ERR_STATE, "server stopped");
    r.ticket = (int64_t)s->tickets.size();
    Ticket t;
    std::memset(&t, 0, sizeof(t));
    s->tickets.push_back(t);
    s->pending.push_back(r);
    s->outstanding++;
    s->rep.submitted++;
    if ((int64_t)s->pending.size() > s->rep.max_queue) s->rep.max_queue = (int64_t)s->pending.size();
    *ticket = r.ticket;
  }
  s->cv_work.notify_one();
  return GQ_OK;
}

int gq_server_poll(gq_server* s, int64_t ticket, gq_ticket_info* info) {
  if (s == nullptr || info == nullptr) return set_error(GQ_ERR_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  if (ticket < 0 || ticket >= (int64_t)s->tickets.size()) return set_error(GQ_ERR_ARG, "unknown ticket");
  *info = s->tickets[(size_t)ticket].info;
  return GQ_OK;
}

int gq_server_drain(gq_server* s, int64_t timeout_ns) {
  if (s == nullptr || timeout_ns <= 0) return set_error(GQ_ERR_ARG, "NULL server or non-positive timeout");
  std::unique_lock<std::mutex> lk(s->mu);
  const auto until = std::chrono::steady_clock::now() + std::chrono::nanoseconds(timeout_ns);
  while (s->outstanding > 0) {
    if (s->cv_done.wait_until(lk, until) == std::cv_status::timeout && s->outstanding > 0)
      return set_error(GQ_ERR_STATE, "drain timed out with %lld requests outstanding", (long long)s->outstanding);
  }
  if (s->broken) return set_error(GQ_ERR_STATE, "server stopped after a CUDA error");
  return GQ_OK;
}

int gq_server_report_get(gq_server* s, gq_server_report* out) {
  if (s == nullptr || out == nullptr) return set_error(GQ_ERR_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->rep;
  return GQ_OK;
}

int gq_server_destroy(gq_server* s) {
  if (s == nullptr) return set_error(GQ_ERR_ARG, "server is NULL");
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    fail_all_pending(s, GQ_ERR_STATE);
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(s->cfg.device);
  for (Lane& L : s->lanes) {
    if (L.stream) cudaStreamSynchronize(L.stream);
    if (L.done) cudaEventDestroy(L.done);
    if (L.stream) cudaStreamDestroy(L.stream);
  }
  cudaSetDevice(prev);
  delete s;
  return GQ_OK;
}

}  // extern "C"
