// serve.cu -- continuous-batching request loop over device-resident Markov chains.
//
// A server holds one context per "class" (lattice + Hamiltonian + network + parameters),
// each with a pool of walker slots whose state (configuration, Phi^-1, projector, cached
// features) stays in HBM between requests. Chains are opened (walkers loaded into free
// slots), then serve requests -- local energies, local energies followed by one Woodbury
// commit per walker, or log|psi| -- until closed.
//
// Scheduling: one host thread. Requests that arrive while a class's previous batch is on
// the GPU wait in that class's queue; when the batch completes, everything queued for the
// class (at most one request per chain) is launched as the next batch over the union of
// the chains' slots. Each class has its own CUDA stream, so batches of different classes
// overlap on the device. Admission: a chain is admitted when its class has enough free
// slots and the resident footprint of all open chains plus its own stays within the
// server's HBM budget; otherwise it waits (or fails with SCALE_EBUDGET when it could
// never fit). Every wait on the host is bounded (scale_server_poll's timeout); no kernel
// waits on the host.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "scale_internal.cuh"

using namespace scale;

namespace {

using Clock = std::chrono::steady_clock;

struct Ticket {
  int64_t id = 0;
  int32_t op = 0, cls = 0;
  int64_t chain = -1;
  int32_t n = 0;                    // walkers
  std::vector<int8_t> occ;          // OPEN
  std::vector<int32_t> moves;       // STEP [n][4]
  double* out_host = nullptr;       // ELOC / STEP / LOGPSI results [n]
  bool done = false;
  scale_status status = SCALE_OK;
  double latency_us = 0.0;
  Clock::time_point t_submit;
};

struct Chain {
  int32_t cls;
  std::vector<int32_t> slots;
  bool ready = false;   // loaded
  bool busy = false;    // a request of this chain is in flight
  size_t bytes = 0;
};

struct Batch {
  std::vector<Ticket*> reqs;
  cudaEvent_t done_ev = nullptr;
  bool active = false;
};

struct ClassState {
  scale_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  std::vector<int32_t> free_slots;
  size_t per_walker = 0;
  // pinned host staging and device buffers, one slot-indexed entry per walker slot
  int32_t* list_host = nullptr;
  int32_t* list_dev = nullptr;
  int32_t* moves_host = nullptr;
  int32_t* moves_dev = nullptr;
  int8_t* occ_dev = nullptr;
  double* out_dev = nullptr;
  double* out_host = nullptr;
  int32_t* sign_dev = nullptr;
  int32_t* sign_host = nullptr;
  int32_t* open_list_dev = nullptr;
  std::deque<Ticket*> queue;   // requests of ready chains
  std::vector<std::pair<Ticket*, cudaEvent_t>> opening;  // loads in flight
  Batch batch;
};

}  // namespace

struct scale_server {
  std::vector<ClassState> cls;
  size_t budget = 0, resident = 0, resident_max = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::thread worker;
  bool stop = false;
  int64_t next_id = 1;
  std::map<int64_t, Ticket*> tickets;
  std::map<int64_t, Chain> chains;
  std::deque<Ticket*> admit;   // OPEN requests waiting for admission
  std::deque<Ticket*> incoming;
  std::string err;
  int64_t n_batches = 0, n_requests = 0;
};

namespace {

scale_status launch_batch(scale_server* s, int ci) {
  ClassState& C = s->cls[ci];
  Batch& bt = C.batch;
  // gather slots of every request in the batch
  int n = 0;
  const int P = C.ctx->B_max;
  for (int q = 0; q < P; ++q) C.moves_host[4 * q] = -1;
  bool any_step = false, any_eloc = false, any_logpsi = false;
  for (Ticket* t : bt.reqs) {
    Chain& ch = s->chains[t->chain];
    for (int w = 0; w < t->n; ++w) {
      const int slot = ch.slots[w];
      C.list_host[n++] = slot;
      if (t->op == SCALE_SRV_STEP)
        std::memcpy(&C.moves_host[4 * slot], &t->moves[4 * w], 16);
    }
    any_step |= t->op == SCALE_SRV_STEP;
    any_eloc |= t->op == SCALE_SRV_ELOC || t->op == SCALE_SRV_STEP;
    any_logpsi |= t->op == SCALE_SRV_LOGPSI;
  }
  cudaStream_t st = C.stream;
  if (cudaMemcpyAsync(C.list_dev, C.list_host, sizeof(int32_t) * n, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return SCALE_ECUDA;
  if (any_eloc && launch_eloc_lowrank_list(C.ctx, C.list_dev, n, C.out_dev) != cudaSuccess) return SCALE_ECUDA;
  if (any_logpsi && launch_logpsi_list(C.ctx, C.list_dev, n, C.out_dev + P, C.sign_dev) != cudaSuccess)
    return SCALE_ECUDA;
  if (cudaMemcpyAsync(C.out_host, C.out_dev, sizeof(double) * 2 * P, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return SCALE_ECUDA;
  if (any_logpsi &&
      cudaMemcpyAsync(C.sign_host, C.sign_dev, sizeof(int32_t) * P, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return SCALE_ECUDA;
  if (any_step) {
    if (cudaMemcpyAsync(C.moves_dev, C.moves_host, sizeof(int32_t) * 4 * P, cudaMemcpyHostToDevice, st) !=
        cudaSuccess)
      return SCALE_ECUDA;
    if (launch_commit(C.ctx, C.moves_dev) != cudaSuccess) return SCALE_ECUDA;
    if (refresh_samples(C.ctx, false) != cudaSuccess) return SCALE_ECUDA;
  }
  if (cudaEventRecord(bt.done_ev, st) != cudaSuccess) return SCALE_ECUDA;
  bt.active = true;
  s->n_batches++;
  return SCALE_OK;
}

void finish_batch(scale_server* s, int ci) {
  ClassState& C = s->cls[ci];
  const int P = C.ctx->B_max;
  const auto now = Clock::now();
  for (Ticket* t : C.batch.reqs) {
    Chain& ch = s->chains[t->chain];
    for (int w = 0; w < t->n; ++w) {
      const int slot = ch.slots[w];
      if (t->op == SCALE_SRV_LOGPSI)
        t->out_host[w] = C.sign_host[slot] == 0 ? -INFINITY : C.out_host[P + slot];
      else if (t->out_host)
        t->out_host[w] = C.out_host[slot];
    }
    ch.busy = false;
    t->done = true;
    t->latency_us = std::chrono::duration<double, std::micro>(now - t->t_submit).count();
  }
  C.batch.reqs.clear();
  C.batch.active = false;
}

// OPEN: load the chain's walkers into free slots on the class stream. The chain is usable
// at once (later batches of the class are ordered behind the load on the same stream);
// the OPEN ticket completes when the load's event has fired.
scale_status do_open(scale_server* s, Ticket* t, bool* admitted) {
  ClassState& C = s->cls[t->cls];
  *admitted = false;
  const size_t bytes = C.per_walker * (size_t)t->n;
  if ((int)C.free_slots.size() < t->n || (s->budget && s->resident + bytes > s->budget)) return SCALE_OK;
  Chain ch;
  ch.cls = t->cls;
  ch.bytes = bytes;
  for (int w = 0; w < t->n; ++w) {
    ch.slots.push_back(C.free_slots.back());
    C.free_slots.pop_back();
  }
  cudaStream_t st = C.stream;
  // pageable sources: the copies are staged before cudaMemcpyAsync returns
  bool ok = cudaMemcpyAsync(C.open_list_dev, ch.slots.data(), sizeof(int32_t) * t->n, cudaMemcpyHostToDevice, st) ==
            cudaSuccess;
  ok = ok && cudaMemcpyAsync(C.occ_dev, t->occ.data(), t->occ.size(), cudaMemcpyHostToDevice, st) == cudaSuccess;
  ok = ok && launch_load_list(C.ctx, C.occ_dev, C.open_list_dev, t->n) == cudaSuccess;
  cudaEvent_t ev = nullptr;
  ok = ok && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess;
  ok = ok && cudaEventRecord(ev, st) == cudaSuccess;
  if (!ok) {
    if (ev) cudaEventDestroy(ev);
    for (int sl : ch.slots) C.free_slots.push_back(sl);
    return SCALE_ECUDA;
  }
  ch.ready = true;
  s->resident += bytes;
  s->resident_max = std::max(s->resident_max, s->resident);
  s->chains[t->id] = ch;
  t->chain = t->id;
  C.opening.push_back({t, ev});
  *admitted = true;
  return SCALE_OK;
}

void worker_loop(scale_server* s) {
  std::unique_lock<std::mutex> lk(s->mu);
  while (!s->stop) {
    // route new requests
    while (!s->incoming.empty()) {
      Ticket* t = s->incoming.front();
      s->incoming.pop_front();
      if (t->op == SCALE_SRV_OPEN) {
        s->admit.push_back(t);
      } else {
        s->cls[t->cls].queue.push_back(t);  // CLOSE too: it follows the chain's requests
      }
    }
    // free closed chains that are idle
    for (auto it = s->chains.begin(); it != s->chains.end();) {
      Chain& ch = it->second;
      if (!ch.ready && !ch.busy) {
        ClassState& C = s->cls[ch.cls];
        bool queued = false;
        for (Ticket* q : C.queue) queued |= q->chain == it->first;
        if (!queued) {
          for (int sl : ch.slots) C.free_slots.push_back(sl);
          s->resident -= ch.bytes;
          it = s->chains.erase(it);
          continue;
        }
      }
      ++it;
    }
    // admissions in arrival order
    for (auto it = s->admit.begin(); it != s->admit.end();) {
      bool admitted = false;
      const scale_status st = do_open(s, *it, &admitted);
      if (st != SCALE_OK) {
        (*it)->status = st;
        (*it)->done = true;
        it = s->admit.erase(it);
      } else if (admitted) {
        it = s->admit.erase(it);
      } else {
        ++it;
      }
    }
    // completions and new batches
    for (size_t ci = 0; ci < s->cls.size(); ++ci) {
      ClassState& C = s->cls[ci];
      for (auto it = C.opening.begin(); it != C.opening.end();) {
        if (cudaEventQuery(it->second) == cudaSuccess) {
          it->first->done = true;
          it->first->latency_us =
              std::chrono::duration<double, std::micro>(Clock::now() - it->first->t_submit).count();
          cudaEventDestroy(it->second);
          it = C.opening.erase(it);
        } else {
          ++it;
        }
      }
      if (C.batch.active && cudaEventQuery(C.batch.done_ev) == cudaSuccess) finish_batch(s, (int)ci);
      if (!C.batch.active && !C.queue.empty()) {
        // FIFO per chain: a request joins the batch when its chain is idle and has no
        // earlier request left waiting; CLOSE marks the chain closed once it is reached.
        std::deque<Ticket*> rest;
        std::vector<int64_t> held;  // chains with a request left in `rest`
        auto is_held = [&](int64_t id) { return std::find(held.begin(), held.end(), id) != held.end(); };
        for (Ticket* t : C.queue) {
          auto it = s->chains.find(t->chain);
          if (it == s->chains.end()) {
            auto op = s->tickets.find(t->chain);
            if (op != s->tickets.end() && op->second->op == SCALE_SRV_OPEN && !op->second->done &&
                op->second->status == SCALE_OK) {
              rest.push_back(t);  // the chain is still waiting for admission
              held.push_back(t->chain);
              continue;
            }
            t->status = SCALE_EINVAL;
            t->done = true;
            continue;
          }
          Chain& ch = it->second;
          if (ch.busy || is_held(t->chain)) {
            rest.push_back(t);  // one request per chain per batch, in order
            held.push_back(t->chain);
            continue;
          }
          if (t->op == SCALE_SRV_CLOSE) {
            ch.ready = false;  // freed below once idle
            t->done = true;
            t->latency_us = std::chrono::duration<double, std::micro>(Clock::now() - t->t_submit).count();
            continue;
          }
          ch.busy = true;
          C.batch.reqs.push_back(t);
        }
        C.queue.swap(rest);
        if (!C.batch.reqs.empty()) {
          const scale_status st = launch_batch(s, (int)ci);
          if (st != SCALE_OK) {
            for (Ticket* t : C.batch.reqs) {
              t->status = st;
              t->done = true;
              s->chains[t->chain].busy = false;
            }
            C.batch.reqs.clear();
          }
        }
      }
    }
    s->cv_done.notify_all();
    bool inflight = false;
    for (auto& C : s->cls) inflight |= C.batch.active || !C.opening.empty();
    if (inflight)
      s->cv_work.wait_for(lk, std::chrono::microseconds(20));
    else
      s->cv_work.wait_for(lk, std::chrono::milliseconds(2),
                          [&] { return s->stop || !s->incoming.empty() || !s->admit.empty(); });
  }
}

template <typename P>
bool alloc_pinned(P** p, size_t bytes) {
  return cudaMallocHost((void**)p, std::max<size_t>(bytes, 16)) == cudaSuccess;
}

}  // namespace

extern "C" {

scale_status scale_server_create(const scale_server_cfg* cfg, scale_server** out) {
  if (!cfg || !out || cfg->n_classes < 1) return SCALE_EINVAL;
  *out = nullptr;
  scale_server* s = new scale_server();
  s->budget = cfg->hbm_budget_bytes;
  s->cls.resize(cfg->n_classes);
  for (int i = 0; i < cfg->n_classes; ++i) {
    ClassState& C = s->cls[i];
    const int slots = cfg->slots[i];
    scale_status st = SCALE_OK;
    if (cudaStreamCreateWithFlags(&C.stream, cudaStreamNonBlocking) != cudaSuccess) st = SCALE_ECUDA;
    if (st == SCALE_OK) st = scale_create(&cfg->sys[i], &cfg->arch[i], slots, 0, C.stream, &C.ctx);
    if (st == SCALE_OK) st = scale_set_params(C.ctx, cfg->params[i], cfg->M0[i]);
    if (st == SCALE_OK && !C.ctx->lowrank_ok) st = SCALE_EUNSUPPORTED;
    if (st != SCALE_OK) {
      scale_server_destroy(s);
      return st;
    }
    C.per_walker = scale_footprint_bytes(&cfg->sys[i], &cfg->arch[i], slots) / slots;
    const int N = C.ctx->N;
    bool ok = alloc_pinned(&C.list_host, sizeof(int32_t) * slots) && alloc_pinned(&C.moves_host, 16 * (size_t)slots) &&
              alloc_pinned(&C.out_host, 16 * (size_t)slots) &&
              alloc_pinned(&C.sign_host, 4 * (size_t)slots);
    ok = ok && cudaMalloc(&C.list_dev, sizeof(int32_t) * slots) == cudaSuccess &&
         cudaMalloc(&C.moves_dev, 16 * (size_t)slots) == cudaSuccess &&
         cudaMalloc(&C.occ_dev, (size_t)slots * N) == cudaSuccess &&
         cudaMalloc(&C.out_dev, 16 * (size_t)slots) == cudaSuccess &&
         cudaMalloc(&C.sign_dev, 4 * (size_t)slots) == cudaSuccess &&
         cudaMalloc(&C.open_list_dev, sizeof(int32_t) * slots) == cudaSuccess &&
         cudaEventCreateWithFlags(&C.batch.done_ev, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
      scale_server_destroy(s);
      return SCALE_ENOMEM;
    }
    // every slot starts empty: flagged so that whole-pool kernels skip it
    C.ctx->B = slots;
    std::vector<int32_t> st_init(slots, SCALE_SAMPLE_BAD_COUNT);
    cudaMemcpy(C.ctx->status, st_init.data(), sizeof(int32_t) * slots, cudaMemcpyHostToDevice);
    for (int q = slots - 1; q >= 0; --q) C.free_slots.push_back(q);
  }
  s->worker = std::thread(worker_loop, s);
  *out = s;
  return SCALE_OK;
}

scale_status scale_server_submit(scale_server* s, const scale_request* rq, uint64_t* ticket) {
  if (!s || !rq || !ticket) return SCALE_EINVAL;
  Ticket* t = new Ticket();
  t->op = rq->op;
  t->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (rq->op == SCALE_SRV_OPEN) {
      if (rq->cls < 0 || rq->cls >= (int)s->cls.size() || rq->n_walkers < 1 || !rq->occ_host) {
        delete t;
        return SCALE_EINVAL;
      }
      ClassState& C = s->cls[rq->cls];
      const size_t bytes = C.per_walker * (size_t)rq->n_walkers;
      if (rq->n_walkers > C.ctx->B_max || (s->budget && bytes > s->budget)) {
        delete t;
        return SCALE_EBUDGET;  // could never be admitted
      }
      t->cls = rq->cls;
      t->n = rq->n_walkers;
      t->occ.assign(rq->occ_host, rq->occ_host + (size_t)rq->n_walkers * C.ctx->N);
    } else {
      auto it = s->chains.find((int64_t)rq->chain);
      auto pend = s->tickets.find((int64_t)rq->chain);
      const bool pending_open = pend != s->tickets.end() && pend->second->op == SCALE_SRV_OPEN;
      const bool known = it != s->chains.end() || pending_open;
      if (!known || (rq->op != SCALE_SRV_CLOSE && rq->op != SCALE_SRV_ELOC && rq->op != SCALE_SRV_STEP &&
                     rq->op != SCALE_SRV_LOGPSI)) {
        delete t;
        return SCALE_EINVAL;
      }
      t->chain = (int64_t)rq->chain;
      if (it != s->chains.end()) {
        t->cls = it->second.cls;
        t->n = (int32_t)it->second.slots.size();
      } else {
        t->cls = pend->second->cls;
        t->n = pend->second->n;
      }
      t->out_host = rq->out_host;
      if (rq->op == SCALE_SRV_STEP) {
        if (!rq->moves_host) {
          delete t;
          return SCALE_EINVAL;
        }
        t->moves.assign(rq->moves_host, rq->moves_host + 4 * (size_t)t->n);
      }
    }
    t->id = s->next_id++;
    s->tickets[t->id] = t;
    s->incoming.push_back(t);
    s->n_requests++;
  }
  s->cv_work.notify_one();
  *ticket = (uint64_t)t->id;
  return SCALE_OK;
}

scale_status scale_server_poll(scale_server* s, uint64_t ticket, scale_result* out, int32_t timeout_us) {
  if (!s) return SCALE_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->tickets.find((int64_t)ticket);
  if (it == s->tickets.end()) return SCALE_EINVAL;
  Ticket* t = it->second;
  if (!t->done) {
    s->cv_done.wait_for(lk, std::chrono::microseconds(std::max(0, timeout_us)), [&] { return t->done; });
    if (!t->done) return SCALE_ETIMEOUT;
  }
  if (out) {
    out->status = t->status;
    out->latency_us = t->latency_us;
    out->chain = (uint64_t)(t->op == SCALE_SRV_OPEN ? t->id : t->chain);
  }
  s->tickets.erase(it);
  delete t;
  return SCALE_OK;
}

scale_status scale_server_cancel(scale_server* s, uint64_t ticket) {
  if (!s) return SCALE_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->tickets.find((int64_t)ticket);
  if (it == s->tickets.end() || it->second->done) return SCALE_EINVAL;
  Ticket* t = it->second;
  auto drop = [&](std::deque<Ticket*>& q) {
    auto f = std::find(q.begin(), q.end(), t);
    if (f == q.end()) return false;
    q.erase(f);
    return true;
  };
  // queued for routing, for admission, or in its class's queue; a request already in a
  // batch is in none of them
  bool found = drop(s->incoming) || drop(s->admit);
  for (size_t ci = 0; !found && ci < s->cls.size(); ++ci) found = drop(s->cls[ci].queue);
  if (!found) return SCALE_EINVAL;
  t->status = SCALE_ECANCELED;
  t->done = true;
  t->latency_us = std::chrono::duration<double, std::micro>(Clock::now() - t->t_submit).count();
  s->cv_done.notify_all();
  return SCALE_OK;
}

scale_status scale_server_stats(scale_server* s, scale_server_stats_t* out) {
  if (!s || !out) return SCALE_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  out->resident_bytes = s->resident;
  out->resident_max_bytes = s->resident_max;
  out->budget_bytes = s->budget;
  out->n_batches = s->n_batches;
  out->n_requests = s->n_requests;
  out->open_chains = (int64_t)s->chains.size();
  return SCALE_OK;
}

void scale_server_destroy(scale_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (auto& C : s->cls) {
    if (C.stream) cudaStreamSynchronize(C.stream);
    if (C.ctx) scale_destroy(C.ctx);
    cudaFreeHost(C.list_host);
    cudaFreeHost(C.moves_host);
    cudaFreeHost(C.out_host);
    cudaFreeHost(C.sign_host);
    cudaFree(C.list_dev);
    cudaFree(C.moves_dev);
    cudaFree(C.occ_dev);
    cudaFree(C.out_dev);
    cudaFree(C.sign_dev);
    cudaFree(C.open_list_dev);
    for (auto& o : C.opening) cudaEventDestroy(o.second);
    if (C.batch.done_ev) cudaEventDestroy(C.batch.done_ev);
    if (C.stream) cudaStreamDestroy(C.stream);
  }
  for (auto& kv : s->tickets) delete kv.second;
  delete s;
}

}  // extern "C"
