// Serving loop over the FLR solver: slots, admission by device-memory
// footprint, concurrent solves on separate streams (see include/flr.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/flr.h"
#include "flr_internal.h"

namespace {

constexpr double kBackfill = 2.0;   // seconds a waiting solve may be overtaken

struct Job {
  uint64_t id;
  flr_request r;
  int64_t footprint;
  double t_submit;
};

struct Done {
  flr_result res;
  std::vector<double> beta;
};

}  // namespace

struct flr_server {
  struct Resident {             // a slot's handle kept between requests with one data_id
    uint64_t id = 0;
    flr_t h = nullptr;
    int64_t footprint = 0;
  };
  flr_server_opts o{};
  int device = 0;
  int sm_count = 0;
  std::vector<std::thread> workers;
  std::vector<cudaStream_t> streams;
  std::vector<Resident> resident;   // per slot; its footprint stays in in_use
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Job> queue;
  std::unordered_map<uint64_t, Done> done;
  std::unordered_map<uint64_t, bool> pending;   // submitted, not yet finished
  int64_t in_use = 0;
  // thread blocks of the device the server's cooperative solves may hold at once
  // (slots x grid_per_slot <= #SMs, one block per SM).  Solves take them in
  // arrival order; while the oldest waiting solve cannot run, a later one that
  // fits in the free blocks may go first, for at most kBackfill seconds of the
  // oldest one's wait (so it is never starved).
  struct Waiter { uint64_t ticket; int need; double since; };
  int blocks_free = 0, blocks_total = 0;
  uint64_t ticket_next = 0;
  std::deque<Waiter> waiting;
  std::condition_variable cv_blocks;
  uint64_t next_id = 1;
  bool stopping = false;
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  void worker(int slot);
};

namespace {

size_t esz(int dt) { return dt == FLR_F64 ? 8 : dt == FLR_F32 ? 4 : (dt == FLR_BF16 || dt == FLR_F16) ? 2 : 0; }

long long graph_edges(const flr_graph& E, long long p) {
  if (E.kind == FLR_E_CHAIN) return p - 1;
  if (E.kind == FLR_E_LATTICE) return E.q1 * (E.q2 - 1) + (E.q1 - 1) * E.q2;
  return E.m;
}

}  // namespace

extern "C" int64_t flr_footprint(int64_t n, int64_t p, int64_t m, int32_t dtype, int32_t mem) {
  const size_t es = esz(dtype);
  if (es == 0 || n < 1 || p < 1) return -1;
  const int64_t vec = 16 / (int64_t)es;
  const int64_t ldn = (n + vec - 1) / vec * vec;
  int64_t b = p * ldn * (int64_t)es;                 // column-major copy of X
  if (mem == FLR_MEM_HOST) b += n * p * (int64_t)es; // staging during flr_create
  b += 8 * n + 16 * ldn;                             // y, u buffers
  b += 8 * p * (15 + 2 * 13);                        // FP64 vectors and PCR multipliers
  b += (8 + 4 + 8) * 2 * std::max<int64_t>(m, 1) + 8 * (p + 1);   // CSR
  b += 64 * 1024;                                    // partials, control
  return b;
}

void flr_server::worker(int slot) {
  cudaSetDevice(device);
  Resident& res = resident[slot];
  while (true) {
    Job job;
    bool hit = false;
    flr_t drop = nullptr;    // a resident handle to release outside the lock
    {
      std::unique_lock<std::mutex> lk(mu);
      // the job this slot would run: one on its resident handle first, else the
      // oldest whose footprint fits once the slot drops its resident handle
      auto choose = [&](bool& is_hit) -> std::deque<Job>::iterator {
        if (res.h)
          for (auto it = queue.begin(); it != queue.end(); ++it)
            if (it->r.data_id != 0 && it->r.data_id == res.id) { is_hit = true; return it; }
        is_hit = false;
        const int64_t freed = res.h ? res.footprint : 0;
        for (auto it = queue.begin(); it != queue.end(); ++it)
          if (in_use - freed + it->footprint <= o.hbm_budget) return it;
        return queue.end();
      };
      while (true) {
        if (stopping && queue.empty()) {
          if (res.h) { in_use -= res.footprint; drop = res.h; res = Resident{}; }
          lk.unlock();
          if (drop) flr_destroy(drop);
          return;
        }
        bool h_ = false;
        auto it = queue.empty() ? queue.end() : choose(h_);
        if (it != queue.end()) {
          job = *it;
          queue.erase(it);
          hit = h_;
          if (!hit) {
            if (res.h) { in_use -= res.footprint; drop = res.h; res = Resident{}; }
            in_use += job.footprint;
          }
          break;
        }
        // queued work that fits nowhere while this slot holds a resident handle:
        // release it so memory frees up
        if (!queue.empty() && res.h) {
          in_use -= res.footprint;
          drop = res.h;
          res = Resident{};
          lk.unlock();
          flr_destroy(drop);
          drop = nullptr;
          cv_work.notify_all();
          lk.lock();
          continue;
        }
        cv_work.wait(lk);
      }
    }
    if (drop) flr_destroy(drop);
    const int64_t held = hit ? res.footprint : job.footprint;   // bytes counted for this handle
    Done d;
    d.res = flr_result{};
    d.res.slot = slot;
    d.res.t_submit = job.t_submit;
    d.res.t_start = now();
    d.res.footprint = job.footprint;
    d.res.reused = hit ? 1 : 0;
    d.beta.assign((size_t)job.r.p, 0.0);
    const flr_request& r = job.r;
    flr_t h = hit ? res.h : nullptr;
    flr_status st = FLR_OK;
    if (!hit) st = flr_create(r.X, r.dtype, r.n, r.p, r.ldx, r.y, &r.E, r.mem, streams[slot], &h);
    if (st == FLR_OK) {
      flr_opts op;
      flr_default_opts(&op);
      if (r.use_opts) op = r.opts;
      // the solve kernel's own sizing rule, capped at the slot's share of the SMs;
      // a problem whose slabs need more blocks than that (their vectors must fit
      // in shared memory) takes more of the server's blocks, waiting for them
      const long long per_block = r.dtype == FLR_F64 ? 8192 : 65536;
      long long g = op.grid > 0 ? op.grid : (r.n * r.p + per_block - 1) / per_block;
      g = std::max<long long>(1, std::min<long long>(g, o.grid_per_slot));
      const int gmin = flr_min_grid(h);
      if (gmin > g) g = gmin;
      op.grid = (int32_t)g;
      // blocks held: a solve wider than the server's whole share runs alone
      const int need = (int)std::min<long long>(g, blocks_total);
      {
        std::unique_lock<std::mutex> lk(mu);
        const uint64_t t = ticket_next++;
        waiting.push_back(Waiter{t, need, now()});
        auto can_go = [&] {
          if (blocks_free < need) return false;
          const Waiter& head = waiting.front();
          if (head.ticket == t) return true;
          return head.need > blocks_free && now() - head.since < kBackfill;
        };
        // timed waits: the backfill window closes without a notification
        while (!can_go()) cv_blocks.wait_for(lk, std::chrono::milliseconds(50));
        blocks_free -= need;
        for (auto it = waiting.begin(); it != waiting.end(); ++it)
          if (it->ticket == t) { waiting.erase(it); break; }
      }
      cv_blocks.notify_all();
      st = gmin < 0 ? FLR_ENOTIMPL
                    : flr_solve(h, r.lambda1, r.lambda2, r.eps, r.tol, &op, nullptr, d.beta.data(),
                                FLR_MEM_HOST, &d.res.stats);
      {
        std::lock_guard<std::mutex> lk(mu);
        blocks_free += need;
      }
      cv_blocks.notify_all();
      unsigned long long t0 = 0, t1 = 0;
      flr_kernel_span(h, &t0, &t1);
      d.res.dev_t0_ns = t0;
      d.res.dev_t1_ns = t1;
    }
    d.res.status = st;
    d.res.t_end = now();
    // keep the handle for the next request with this data_id, else release it
    const bool keep = h && r.data_id != 0 && st != FLR_ECUDA && st != FLR_ETIMEOUT;
    if (h && !keep) flr_destroy(h);
    {
      std::lock_guard<std::mutex> lk(mu);
      if (keep) {
        if (!hit) res = Resident{r.data_id, h, held};
      } else {
        if (hit) res = Resident{};
        in_use -= held;
      }
      done[job.id] = std::move(d);
      pending.erase(job.id);
    }
    cv_done.notify_all();
    cv_work.notify_all();
  }
}

extern "C" flr_status flr_server_create(const flr_server_opts* opts, flr_server_t* out) {
  if (!out) return FLR_EINVAL;
  *out = nullptr;
  flr_server* s = new (std::nothrow) flr_server();
  if (!s) return FLR_ENOMEM;
  if (cudaGetDevice(&s->device) != cudaSuccess) { (void)cudaGetLastError(); delete s; return FLR_ECUDA; }
  cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, s->device);
  if (opts) s->o = *opts;
  if (s->o.slots <= 0) s->o.slots = 4;
  if (s->o.grid_per_slot <= 0) s->o.grid_per_slot = std::max(1, s->sm_count / s->o.slots);
  if (s->o.hbm_budget <= 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) { (void)cudaGetLastError(); delete s; return FLR_ECUDA; }
    s->o.hbm_budget = (int64_t)(fr / 4 * 3);
  }
  if ((long long)s->o.slots * s->o.grid_per_slot > s->sm_count) {
    delete s;   // cooperative solves must all fit on the device at once
    return FLR_EINVAL;
  }
  s->blocks_total = s->blocks_free = s->o.slots * s->o.grid_per_slot;
  for (int i = 0; i < s->o.slots; ++i) {
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      (void)cudaGetLastError();
      for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
      delete s;
      return FLR_ECUDA;
    }
    s->streams.push_back(st);
  }
  s->resident.assign((size_t)s->o.slots, flr_server::Resident{});
  for (int i = 0; i < s->o.slots; ++i) s->workers.emplace_back(&flr_server::worker, s, i);
  *out = s;
  return FLR_OK;
}

extern "C" flr_status flr_server_submit(flr_server_t s, const flr_request* r, uint64_t* id) {
  if (!s || !r || !id) return FLR_EINVAL;
  if (!r->X || !r->y || r->n < 1 || r->p < 1 || r->ldx < r->p || esz(r->dtype) == 0) return FLR_EINVAL;
  if (r->mem != FLR_MEM_HOST && r->mem != FLR_MEM_DEVICE) return FLR_EINVAL;
  if (!(r->lambda1 >= 0.0) || !(r->lambda2 >= 0.0) || !(r->eps > 0.0) || !(r->tol > 0.0)) return FLR_EINVAL;
  if (r->E.kind != FLR_E_CHAIN && r->E.kind != FLR_E_LATTICE && r->E.kind != FLR_E_EDGES) return FLR_EINVAL;
  const int64_t fp = flr_footprint(r->n, r->p, graph_edges(r->E, r->p), r->dtype, r->mem);
  if (fp < 0) return FLR_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stopping) return FLR_EINVAL;
  if (fp > s->o.hbm_budget) return FLR_ENOMEM;
  Job j{s->next_id++, *r, fp, s->now()};
  s->pending[j.id] = true;
  s->queue.push_back(j);
  *id = j.id;
  s->cv_work.notify_one();
  return FLR_OK;
}

extern "C" flr_status flr_server_poll(flr_server_t s, uint64_t id, int32_t* is_done) {
  if (!s || !is_done) return FLR_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->done.count(id)) { *is_done = 1; return FLR_OK; }
  if (s->pending.count(id)) { *is_done = 0; return FLR_OK; }
  return FLR_EINVAL;
}

extern "C" flr_status flr_server_wait(flr_server_t s, uint64_t id, double* beta_out, flr_result* res) {
  if (!s) return FLR_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  if (!s->done.count(id) && !s->pending.count(id)) return FLR_EINVAL;
  s->cv_done.wait(lk, [&] { return s->done.count(id) > 0; });
  Done d = std::move(s->done[id]);
  s->done.erase(id);
  lk.unlock();
  if (beta_out) std::memcpy(beta_out, d.beta.data(), sizeof(double) * d.beta.size());
  if (res) *res = d.res;
  return (flr_status)d.res.status;
}

extern "C" flr_status flr_server_destroy(flr_server_t s) {
  if (!s) return FLR_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stopping = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
  delete s;
  return FLR_OK;
}
