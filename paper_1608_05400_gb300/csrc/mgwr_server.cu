// Serving runtime: a request queue in front of the solver.  Requests of any
// shape (d, n, M) and any (T, alpha, precision) are submitted from any host
// thread and admitted while their device-memory footprint fits the budget and
// a slot is free.  A slot's worker thread prepares the request's handle (from
// a pool of idle handles of the same shape and precision, re-parameterised in
// place by mgwr_set_problem, else a new one) and copies its data in; the
// request then joins the server's group (mgwr_group_*), where one batcher
// thread advances every admitted solve together: each iteration of all of them
// is one CUDA graph launch whose branches run concurrently on the device.
// Requests join and leave between iterations, so one that arrives while others
// are on the GPU starts at the next iteration (continuous batching at
// iteration granularity).  Each solve runs exactly the launches it runs alone,
// so its result does not depend on what else runs.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <cstdlib>
#include <deque>
#include <map>
#include <list>
#include <memory>
#include <mutex>
#include <tuple>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/mgwr.h"

namespace {

using Clock = std::chrono::steady_clock;

// Pinned (page-locked) host buffers for the requests' right-hand sides and
// results: they move between host and device at the copy engines' rate (about
// 200 GB/s each way on GB300) instead of through the driver's staging of
// pageable memory (about 25 GB/s).  Pinning pages is slow, so released buffers
// are kept, up to kKeep bytes, and handed out again to requests that fit.
class PinnedPool {
 public:
  static constexpr size_t kKeep = size_t(32) << 30;
  ~PinnedPool() {
    for (auto& kv : free_) cudaFreeHost(kv.second);
  }
  // A buffer of at least `count` doubles (its capacity in *cap), or nullptr
  // when no page-locked memory can be had.
  double* get(size_t count, size_t* cap) {
    {
      std::lock_guard<std::mutex> lk(mu_);
      auto it = free_.lower_bound(count);
      if (it != free_.end() && it->first <= 2 * count + (size_t(1) << 20)) {
        double* p = it->second;
        *cap = it->first;
        kept_ -= it->first * sizeof(double);
        free_.erase(it);
        return p;
      }
    }
    void* p = nullptr;
    const auto t0 = std::chrono::steady_clock::now();
    if (cudaMallocHost(&p, count * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    {
      std::lock_guard<std::mutex> lk(mu_);
      pin_s_ += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      pinned_++;
    }
    *cap = count;
    return static_cast<double*>(p);
  }
  // seconds spent page-locking new buffers, and how many
  void stats(double* pin_s, long long* pinned) {
    std::lock_guard<std::mutex> lk(mu_);
    *pin_s = pin_s_;
    *pinned = pinned_;
  }
  void put(double* p, size_t cap) {
    {
      std::lock_guard<std::mutex> lk(mu_);
      if (kept_ + cap * sizeof(double) <= kKeep) {
        kept_ += cap * sizeof(double);
        free_.emplace(cap, p);
        return;
      }
    }
    cudaFreeHost(p);
  }

 private:
  std::mutex mu_;
  std::multimap<size_t, double*> free_;
  size_t kept_ = 0;
  double pin_s_ = 0.0;
  long long pinned_ = 0;
};

// `count` doubles of host memory: pinned from the pool when it has some, else
// ordinary (pageable) memory.
class HostBuf {
 public:
  HostBuf() = default;
  HostBuf(const HostBuf&) = delete;
  HostBuf& operator=(const HostBuf&) = delete;
  ~HostBuf() { release(); }
  bool alloc(PinnedPool* pool, size_t count) {
    release();
    size_t cap = 0;
    p_ = pool->get(count, &cap);
    if (p_ != nullptr) {
      pool_ = pool;
      cap_ = cap;
    } else {
      p_ = static_cast<double*>(std::malloc(count * sizeof(double)));
      if (p_ == nullptr) return false;
    }
    n_ = count;
    return true;
  }
  // takes over a pool buffer of capacity cap holding count values
  void adopt(PinnedPool* pool, double* p, size_t cap, size_t count) {
    release();
    p_ = p;
    pool_ = pool;
    cap_ = cap;
    n_ = count;
  }
  double* data() const { return p_; }
  size_t size() const { return n_; }
  bool empty() const { return n_ == 0; }
  void reset() { release(); }

 private:
  void release() {
    if (p_ == nullptr) return;
    if (pool_ != nullptr)
      pool_->put(p_, cap_);
    else
      std::free(p_);
    p_ = nullptr;
    pool_ = nullptr;
    n_ = cap_ = 0;
  }
  double* p_ = nullptr;
  PinnedPool* pool_ = nullptr;
  size_t n_ = 0, cap_ = 0;
};

struct Ticket {
  uint64_t id = 0;
  mgwr_request rq{};
  HostBuf f, u;
  std::vector<double> g;
  size_t footprint = 0;
  size_t N = 0;
  int state = 0;  // 0 queued, 1 running, 2 done
  mgwr_t h = nullptr;   // its handle while it runs
  bool solved = false;  // the group has finished its solve (status in res)
  int skipped = 0;
  Clock::time_point t_submit, t_admit, t_done;
  mgwr_result res{};
  PinnedPool* pool = nullptr;  // where the result buffer comes from
};

bool pow2(long long x) { return x > 0 && (x & (x - 1)) == 0; }

}  // namespace

// Idle handles kept for later requests of the same shape and precision.
struct IdleHandle {
  std::tuple<int, int, int, int> key;  // d, n, M, resolved precision
  mgwr_t h;
  size_t bytes;
};

struct mgwr_server {
  PinnedPool pool;  // declared first: outlives the tickets that hold its buffers
  size_t budget = 0, in_use = 0, peak = 0;
  int slots = 1, max_queue = 1 << 20, device = 0;
  int policy = MGWR_POLICY_FIFO;
  std::mutex mu;
  std::condition_variable cv_work, cv_done, cv_batch, cv_solved;
  std::deque<Ticket*> queue;
  std::unordered_map<uint64_t, std::unique_ptr<Ticket>> tickets;
  std::vector<std::thread> workers;
  bool stop = false;
  bool stop_batcher = false;  // set once every worker has left
  uint64_t next_id = 1;
  long long completed = 0, admitted = 0;
  // the groups admitted solves run in, one per size class (space-time unknowns
  // below 2^22, below 2^26, larger), each advanced by its own batcher thread, so
  // that small solves do not wait for the iterations of large ones; and the
  // requests about to join each
  static constexpr int kClasses = 3;
  mgwr_group_t group[kClasses] = {};
  std::vector<Ticket*> joining[kClasses];
  std::thread batchers[kClasses];
  // idle handles, most recently used first; their bytes count in in_use
  std::list<IdleHandle> idle;
  size_t idle_bytes = 0;
  long long reused = 0;
  // each group's counters, copied by its batcher after every step
  long long launches[kClasses] = {}, iterations[kClasses] = {};
  long long launches_seen[kClasses] = {}, iterations_seen[kClasses] = {};  // of the current group
  int most[kClasses] = {};
  // pool buffers handed to callers (mgwr_server_buffer) and their capacities
  std::unordered_map<double*, size_t> lent;
  // host seconds: right-hand sides copied by mgwr_submit, handles prepared and
  // data uploaded by the slots, results downloaded
  double submit_copy_s = 0.0, prepare_s = 0.0, finish_s = 0.0;
};

namespace {

// Queue position that may start now.  FIFO: the oldest request that fits the
// free memory.  SMALLEST: the request with the fewest space-time unknowns
// that fits (ties: the oldest).  Either way a request that was passed over
// this many times blocks the others until it fits (no starvation of large
// requests), and every request older than the one taken counts as passed over.
constexpr int kMaxSkips = 64;

Ticket* pick(mgwr_server* s) {
  const size_t free_bytes = s->budget - s->in_use;
  auto chosen = s->queue.end();
  for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
    Ticket* t = *it;
    if (t->skipped >= kMaxSkips) {  // starving: it goes next, or nothing does
      if (t->footprint <= free_bytes) chosen = it;
      break;
    }
    if (t->footprint > free_bytes) continue;
    if (chosen == s->queue.end()) {
      chosen = it;
      if (s->policy == MGWR_POLICY_FIFO) break;
    } else if (t->N * (size_t)t->rq.M < (*chosen)->N * (size_t)(*chosen)->rq.M) {
      chosen = it;
    }
  }
  if (chosen == s->queue.end()) return nullptr;
  for (auto jt = s->queue.begin(); jt != chosen; ++jt) (*jt)->skipped++;
  Ticket* t = *chosen;
  s->queue.erase(chosen);
  return t;
}

constexpr size_t kMaxIdle = 32;  // idle handles kept at most (and within the budget)

std::tuple<int, int, int, int> shape_key(const mgwr_request& q) {
  int prec = q.precision;
  mgwr_auto_precision(q.d, q.n, q.M, q.precision, &prec);
  return std::make_tuple(q.d, q.n, q.M, prec);
}

// Destroys idle handles (least recently used first) until `need` more bytes fit
// the budget or none is left; called with the lock held, destroys outside it.
std::vector<mgwr_t> evict_for(mgwr_server* s, size_t need) {
  std::vector<mgwr_t> out;
  while (!s->idle.empty() && (s->in_use + need > s->budget || s->idle.size() > kMaxIdle)) {
    out.push_back(s->idle.back().h);
    s->in_use -= s->idle.back().bytes;
    s->idle_bytes -= s->idle.back().bytes;
    s->idle.pop_back();
  }
  return out;
}

// Size class of a request by its space-time unknowns n^d M.
int size_class(const Ticket* t) {
  const double u = (double)t->N * t->rq.M;
  return u < (double)(1 << 22) ? 0 : u < (double)(1 << 26) ? 1 : 2;
}

// The request's handle: an idle one of its shape and precision, set up in
// place for its (T, alpha) (nothing to redo when those match too), else a new
// one; then its settings and data.
int prepare(mgwr_server* s, Ticket* t) {
  const mgwr_request& q = t->rq;
  mgwr_t h = nullptr;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (auto it = s->idle.begin(); it != s->idle.end(); ++it) {
      if (it->key != shape_key(q)) continue;
      h = it->h;
      // its bytes now belong to the request: the request's footprint was added on
      // admission, so the idle share goes
      s->in_use -= it->bytes;
      s->idle_bytes -= it->bytes;
      s->idle.erase(it);
      s->reused++;
      break;
    }
  }
  int st = MGWR_OK;
  if (h != nullptr) {
    st = mgwr_set_problem(h, &q.T, &q.alpha);
  } else {
    st = mgwr_create(q.d, q.n, q.M, q.T, q.alpha, &h);
    if (st == MGWR_OK && q.precision != MGWR_FP64) st = mgwr_set_precision(h, q.precision);
  }
  if (st == MGWR_OK) st = mgwr_set_order(h, q.order);
  if (st == MGWR_OK) st = mgwr_set_rhs(h, t->f.data(), t->g.empty() ? nullptr : t->g.data());
  if (st != MGWR_OK && h != nullptr) {
    mgwr_destroy(h);
    h = nullptr;
  }
  t->h = h;
  return st;
}

// After the solve: the result copied out, the handle kept idle (or destroyed).
int finish(mgwr_server* s, Ticket* t, int st) {
  const mgwr_request& q = t->rq;
  if (st == MGWR_OK || st == MGWR_E_NOCONV) {
    const int st2 = t->u.alloc(t->pool, t->N * q.M) ? mgwr_get_solution(t->h, t->u.data())
                                                    : MGWR_E_NOMEM;
    if (st2 != MGWR_OK) st = st2;
  }
  std::vector<mgwr_t> drop;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->in_use -= t->footprint;
    if (st == MGWR_OK || st == MGWR_E_NOCONV) {
      s->idle.push_front({shape_key(q), t->h, t->footprint});
      s->in_use += t->footprint;
      s->idle_bytes += t->footprint;
      drop = evict_for(s, 0);
    } else {
      drop.push_back(t->h);
    }
    t->h = nullptr;
  }
  for (mgwr_t h : drop) mgwr_destroy(h);
  return st;
}

void worker(mgwr_server* s) {
  cudaSetDevice(s->device);
  for (;;) {
    Ticket* t = nullptr;
    std::vector<mgwr_t> drop;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait(lk, [&] {
        if (s->stop) return true;
        t = pick(s);
        if (t == nullptr && !s->idle.empty() && !s->queue.empty()) {
          // idle handles may be what keeps the oldest request out
          drop = evict_for(s, s->queue.front()->footprint);
          t = pick(s);
        }
        return t != nullptr;
      });
      if (t == nullptr) return;  // stopping
      s->in_use += t->footprint;
      if (s->in_use > s->peak) s->peak = s->in_use;
      t->state = 1;
      t->t_admit = Clock::now();
      s->admitted++;
    }
    for (mgwr_t h : drop) mgwr_destroy(h);
    const auto tp = Clock::now();
    int st = prepare(s, t);
    t->f.reset();  // uploaded (mgwr_set_rhs waits for its copy): back to the pool
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->prepare_s += std::chrono::duration<double>(Clock::now() - tp).count();
    }
    if (st == MGWR_OK) {
      // the batcher adds it to the group at the next iteration boundary
      std::unique_lock<std::mutex> lk(s->mu);
      s->joining[size_class(t)].push_back(t);
      s->cv_batch.notify_all();
      s->cv_solved.wait(lk, [&] { return t->solved; });
      st = t->res.status;
    }
    if (t->h != nullptr) {
      const auto tf = Clock::now();
      st = finish(s, t, st);
      std::lock_guard<std::mutex> lk(s->mu);
      s->finish_s += std::chrono::duration<double>(Clock::now() - tf).count();
    } else {
      std::lock_guard<std::mutex> lk(s->mu);
      s->in_use -= t->footprint;
    }
    {
      std::lock_guard<std::mutex> lk(s->mu);
      t->t_done = Clock::now();
      t->res.status = st;
      t->res.queue_s = std::chrono::duration<double>(t->t_admit - t->t_submit).count();
      t->res.latency_s = std::chrono::duration<double>(t->t_done - t->t_submit).count();
      t->state = 2;
      s->completed++;
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();
  }
}

// The batcher of size class `cls`: admits prepared requests into its group
// between iterations and advances all of them, one graph launch per iteration.
void batcher(mgwr_server* s, int cls) {
  cudaSetDevice(s->device);
  std::unordered_map<mgwr_t, Ticket*> members;
  mgwr_group_t& group = s->group[cls];
  for (;;) {
    std::vector<Ticket*> join;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_batch.wait(lk, [&] {
        return s->stop_batcher || !s->joining[cls].empty() || !members.empty();
      });
      if (s->stop_batcher && members.empty() && s->joining[cls].empty()) return;
      join.swap(s->joining[cls]);
    }
    std::vector<Ticket*> failed;
    for (Ticket* t : join) {
      const mgwr_request& q = t->rq;
      const int st = mgwr_group_add(group, t->h, q.cycle, q.nu1, q.nu2, q.tol, q.max_cycles);
      if (st == MGWR_OK) {
        members[t->h] = t;
      } else {
        t->res.status = st;
        failed.push_back(t);
      }
    }
    int left = 0;
    const int gst = members.empty() ? MGWR_OK : mgwr_group_step(group, &left);
    std::vector<Ticket*> done = failed;
    mgwr_t h = nullptr;
    int code = 0;
    mgwr_stats st{};
    while (mgwr_group_collect(group, &h, &code, &st) == MGWR_OK) {
      auto it = members.find(h);
      if (it == members.end()) continue;
      it->second->res.status = code;
      it->second->res.stats = st;
      done.push_back(it->second);
      members.erase(it);
    }
    if (gst != MGWR_OK) {  // the group itself failed: every member fails with it
      mgwr_group_destroy(group);
      group = nullptr;
      mgwr_group_create(&group);
      {
        std::lock_guard<std::mutex> lk(s->mu);
        s->launches_seen[cls] = s->iterations_seen[cls] = 0;
      }
      for (auto& kv : members) {
        kv.second->res.status = gst;
        done.push_back(kv.second);
      }
      members.clear();
    }
    long long launches = 0, iters = 0;
    int most = 0;
    if (group != nullptr) mgwr_group_info(group, &launches, &iters, &most);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->launches[cls] += launches - s->launches_seen[cls];
      s->iterations[cls] += iters - s->iterations_seen[cls];
      s->launches_seen[cls] = launches;
      s->iterations_seen[cls] = iters;
      s->most[cls] = std::max(s->most[cls], most);
      for (Ticket* t : done) t->solved = true;
    }
    if (!done.empty()) s->cv_solved.notify_all();
  }
}

int check_request(const mgwr_request* q) {
  if (q == nullptr || q->f == nullptr) return MGWR_E_INVAL;
  if (q->d != 1 && q->d != 2) return MGWR_E_INVAL;
  if (q->n < 1 || !pow2((long long)q->n + 1)) return MGWR_E_INVAL;
  if ((q->d == 1 && q->n > 32767) || (q->d == 2 && q->n > 4095)) return MGWR_E_INVAL;
  if (!pow2(q->M) || q->M < 4 || q->M > (1 << 20)) return MGWR_E_INVAL;
  if (!(q->T > 0.0) || !(q->alpha > 0.0) || !(q->alpha <= 1.0)) return MGWR_E_INVAL;
  if (q->precision != MGWR_FP64 && q->precision != MGWR_MIXED && q->precision != MGWR_MIXED_DD &&
      q->precision != MGWR_DD && q->precision != MGWR_AUTO)
    return MGWR_E_INVAL;
  if (q->cycle != 1 && q->cycle != 2) return MGWR_E_INVAL;
  if (q->nu1 < 0 || q->nu2 < 0 || q->nu1 + q->nu2 == 0 || q->nu1 > 16 || q->nu2 > 16)
    return MGWR_E_INVAL;
  if (!(q->tol >= 0.0) || q->max_cycles < 1) return MGWR_E_INVAL;
  return MGWR_OK;
}

// Queues a checked request.  Without `lent`, f is copied into a pool buffer;
// with it, that buffer (from mgwr_server_buffer, holding f) is taken over
// without a copy, on success only: on any error the caller still holds it.
int submit_ticket(mgwr_server* s, const mgwr_request* rq, double* lent, uint64_t* ticket) {
  size_t fp = 0;
  if (mgwr_footprint(rq->d, rq->n, rq->M, 1, rq->precision, &fp) != MGWR_OK) return MGWR_E_INVAL;
  if (fp > s->budget) return MGWR_E_TOOBIG;
  auto t = std::unique_ptr<Ticket>(new (std::nothrow) Ticket);
  if (!t) return MGWR_E_NOMEM;
  t->rq = *rq;
  t->N = rq->d == 1 ? (size_t)rq->n : (size_t)rq->n * rq->n;
  const size_t count = t->N * rq->M;
  try {
    if (lent == nullptr) {
      if (!t->f.alloc(&s->pool, count)) return MGWR_E_NOMEM;
      const auto t0 = Clock::now();
      std::memcpy(t->f.data(), rq->f, count * sizeof(double));
      std::lock_guard<std::mutex> lk(s->mu);
      s->submit_copy_s += std::chrono::duration<double>(Clock::now() - t0).count();
    }
    t->pool = &s->pool;
    if (rq->g != nullptr) t->g.assign(rq->g, rq->g + t->N);
  } catch (const std::bad_alloc&) {
    return MGWR_E_NOMEM;
  }
  t->rq.f = nullptr;
  t->rq.g = nullptr;
  t->footprint = fp;
  t->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return MGWR_E_STATE;
    if ((int)s->queue.size() >= s->max_queue) return MGWR_E_AGAIN;
    if (lent != nullptr) {
      auto it = s->lent.find(lent);
      if (it == s->lent.end() || it->second < count) return MGWR_E_INVAL;
      t->f.adopt(&s->pool, lent, it->second, count);
      s->lent.erase(it);
    }
    t->id = s->next_id++;
    *ticket = t->id;
    s->queue.push_back(t.get());
    s->tickets.emplace(t->id, std::move(t));
  }
  s->cv_work.notify_one();
  return MGWR_OK;
}

}  // namespace

extern "C" {

int mgwr_server_create(size_t hbm_budget, int max_slots, mgwr_server_t* out) {
  if (out == nullptr) return MGWR_E_INVAL;
  *out = nullptr;
  if (hbm_budget == 0 || max_slots < 1 || max_slots > 64) return MGWR_E_INVAL;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || count < 1) {
    cudaGetLastError();
    return MGWR_E_CUDA;
  }
  mgwr_server_t s = new (std::nothrow) mgwr_server;
  if (s == nullptr) return MGWR_E_NOMEM;
  s->budget = hbm_budget;
  s->slots = max_slots;
  cudaGetDevice(&s->device);
  for (int c = 0; c < mgwr_server::kClasses; ++c) {
    if (mgwr_group_create(&s->group[c]) != MGWR_OK) {
      for (int k = 0; k < c; ++k) mgwr_group_destroy(s->group[k]);
      delete s;
      return MGWR_E_CUDA;
    }
  }
  for (int i = 0; i < max_slots; ++i) s->workers.emplace_back(worker, s);
  for (int c = 0; c < mgwr_server::kClasses; ++c) s->batchers[c] = std::thread(batcher, s, c);
  *out = s;
  return MGWR_OK;
}

int mgwr_server_set_policy(mgwr_server_t s, int policy) {
  if (s == nullptr) return MGWR_E_INVAL;
  if (policy != MGWR_POLICY_FIFO && policy != MGWR_POLICY_SMALLEST) return MGWR_E_INVAL;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->policy = policy;
  }
  s->cv_work.notify_all();
  return MGWR_OK;
}

int mgwr_server_destroy(mgwr_server_t s) {
  if (s == nullptr) return MGWR_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->queue.clear();
  }
  s->cv_work.notify_all();
  for (auto& w : s->workers) w.join();  // each finishes its running request first
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop_batcher = true;
  }
  s->cv_batch.notify_all();
  for (auto& b : s->batchers) b.join();
  for (auto& i : s->idle) mgwr_destroy(i.h);
  for (auto& g : s->group) mgwr_group_destroy(g);
  for (auto& kv : s->lent) s->pool.put(kv.first, kv.second);  // freed with the pool
  delete s;
  return MGWR_OK;
}

int mgwr_submit(mgwr_server_t s, const mgwr_request* rq, uint64_t* ticket) {
  if (s == nullptr || ticket == nullptr) return MGWR_E_INVAL;
  const int st = check_request(rq);
  if (st != MGWR_OK) return st;
  return submit_ticket(s, rq, nullptr, ticket);
}

int mgwr_server_buffer(mgwr_server_t s, size_t count, double** buf) {
  if (s == nullptr || buf == nullptr || count == 0) return MGWR_E_INVAL;
  *buf = nullptr;
  size_t cap = 0;
  double* p = s->pool.get(count, &cap);
  if (p == nullptr) return MGWR_E_NOMEM;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    try {
      s->lent.emplace(p, cap);
    } catch (const std::bad_alloc&) {
      s->pool.put(p, cap);
      return MGWR_E_NOMEM;
    }
  }
  *buf = p;
  return MGWR_OK;
}

int mgwr_submit_buffer(mgwr_server_t s, const mgwr_request* rq, double* buf, uint64_t* ticket) {
  if (s == nullptr || ticket == nullptr || rq == nullptr || buf == nullptr) return MGWR_E_INVAL;
  mgwr_request q = *rq;
  q.f = buf;
  const int st = check_request(&q);
  if (st != MGWR_OK) return st;
  return submit_ticket(s, &q, buf, ticket);
}

int mgwr_server_release(mgwr_server_t s, double* buf) {
  if (s == nullptr || buf == nullptr) return MGWR_E_INVAL;
  size_t cap = 0;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->lent.find(buf);
    if (it == s->lent.end()) return MGWR_E_INVAL;
    cap = it->second;
    s->lent.erase(it);
  }
  s->pool.put(buf, cap);
  return MGWR_OK;
}

int mgwr_poll(mgwr_server_t s, uint64_t ticket, int timeout_us, double* u_out, mgwr_result* res) {
  if (s == nullptr) return MGWR_E_INVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->tickets.find(ticket);
  if (it == s->tickets.end()) return MGWR_E_INVAL;
  Ticket* t = it->second.get();
  if (t->state != 2) {
    if (timeout_us <= 0) return MGWR_E_AGAIN;
    const bool done = s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us),
                                          [&] { return t->state == 2; });
    if (!done) return MGWR_E_TIMEOUT;
  }
  if (res != nullptr) *res = t->res;
  if (u_out != nullptr && !t->u.empty()) std::memcpy(u_out, t->u.data(), t->u.size() * sizeof(double));
  s->tickets.erase(it);
  return MGWR_OK;
}

int mgwr_server_stats(mgwr_server_t s, mgwr_server_info* info) {
  if (s == nullptr || info == nullptr) return MGWR_E_INVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  info->queued = (long long)s->queue.size();
  info->completed = s->completed;
  info->admitted = s->admitted;
  info->in_use_bytes = s->in_use;
  info->peak_bytes = s->peak;
  info->budget_bytes = s->budget;
  info->slots = s->slots;
  info->reused_handles = s->reused;
  info->submit_copy_s = s->submit_copy_s;
  info->prepare_s = s->prepare_s;
  info->finish_s = s->finish_s;
  s->pool.stats(&info->pin_s, &info->pinned_buffers);
  info->group_launches = 0;
  info->member_iterations = 0;
  info->max_group_members = 0;
  for (int c = 0; c < mgwr_server::kClasses; ++c) {
    info->group_launches += s->launches[c];
    info->member_iterations += s->iterations[c];
    info->max_group_members = std::max(info->max_group_members, s->most[c]);
  }
  return MGWR_OK;
}

}  // extern "C"
