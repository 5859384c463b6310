// Serving loop: many MERA optimisations on one GPU.
//
// Requests (a Hamiltonian, a starting point, a stopping rule) are queued in
// arrival order.  A request is admitted when its device footprint
// (mera_footprint_bytes) fits in the memory budget next to the requests that
// are already running; it then gets its own mera_t on its own CUDA stream,
// so its tensors, Krylov warm starts and L-BFGS history stay on the device
// until it finishes.  Worker threads take turns over the running requests,
// one L-BFGS (or CG) iteration at a time, so the kernels of different
// requests overlap on the GPU while each request's host-side control (line
// search, Krylov scalars) waits only for its own stream.
//
// Requests with the same network configuration (binary, real, unsliced)
// form a cohort: their energy/gradient evaluations meet at a rendezvous, and
// the evaluations waiting there run together (eval_group: one batched
// tensor-core launch per contraction for all of them, the Krylov solves in
// lockstep) on the cohort's stream.  An evaluation waits for the cohort's
// other stepping requests at most a short gathering window.  A request's
// arithmetic does not depend on what else is running (every kernel has a
// fixed reduction order and a batched product computes each member as it
// would alone), so its result is the same alone and in the mix.
#include "ctx.h"

#include <chrono>
#include <cstdio>
#include <string>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>

namespace {

using clk = std::chrono::steady_clock;

// Same-configuration problems evaluated together (see the file comment).
struct Cohort {
  std::mutex mu;
  std::condition_variable cv;
  int stepping = 0;  // its requests inside an iteration step
  int refs = 0;      // its requests with a live problem
  struct Pend {
    mera_ctx* c = nullptr;
    const double* W = nullptr;
    mera::Eval* E = nullptr;
    bool done = false;
    int nb = 0;
    std::exception_ptr err;
  };
  std::vector<Pend*> pending;
  clk::time_point first;  // arrival of the oldest pending evaluation
  bool driving = false;
  cudaStream_t s = nullptr;
  mera::DevBuf ws, flag;
  mera::Exec ex;
  size_t bytes = 0;
  ~Cohort() {
    if (s) cudaStreamDestroy(s);
  }
};

// How long an evaluation waits for the cohort's other stepping requests.
constexpr auto kGather = std::chrono::microseconds(1500);

void cohort_eval(void* co, mera_ctx& c, const double* W, mera::Eval& E) {
  Cohort& h = *static_cast<Cohort*>(co);
  MERA_CUDA(cudaStreamSynchronize(c.s));  // the member's own stream has produced W
  Cohort::Pend p;
  p.c = &c;
  p.W = W;
  p.E = &E;
  std::unique_lock<std::mutex> lk(h.mu);
  if (h.pending.empty()) h.first = clk::now();
  h.pending.push_back(&p);
  h.cv.notify_all();
  constexpr int MAXB = mera::tc::TcEpilogue::MAXB;
  while (!p.done) {
    const int np = (int)h.pending.size();
    const bool ready = np >= h.stepping || np >= MAXB || clk::now() - h.first > kGather;
    if (!h.driving && np > 0 && ready) {
      h.driving = true;
      const int nb = std::min(np, MAXB);
      std::vector<Cohort::Pend*> batch(h.pending.begin(), h.pending.begin() + nb);
      h.pending.erase(h.pending.begin(), h.pending.begin() + nb);
      if (!h.pending.empty()) h.first = clk::now();
      lk.unlock();
      mera_ctx* cs[MAXB];
      const double* Ws[MAXB];
      mera::Eval* Es[MAXB];
      std::exception_ptr errs[MAXB];
      for (int k = 0; k < nb; ++k) {
        cs[k] = batch[k]->c;
        Ws[k] = batch[k]->W;
        Es[k] = batch[k]->E;
      }
      try {
        mera::eval_group(cs, Ws, Es, nb, true, h.ex, h.s, errs);
        MERA_CUDA(cudaStreamSynchronize(h.s));  // results complete before the members go on
      } catch (...) {
        for (int k = 0; k < nb; ++k) errs[k] = std::current_exception();
      }
      lk.lock();
      for (int k = 0; k < nb; ++k) {
        batch[k]->err = errs[k];
        batch[k]->nb = nb;
        batch[k]->done = true;
      }
      h.driving = false;
      h.cv.notify_all();
    } else {
      h.cv.wait_for(lk, std::chrono::microseconds(100));
    }
  }
  lk.unlock();
  if (p.nb > 1) ++c.evals_batched;
  if (p.err) std::rethrow_exception(p.err);
}

// Requests that may share a cohort: the same network configuration, binary,
// real, without slicing of the chi^9 chain (the fields that decide the
// plans, the arithmetic and the workspace).
std::string cohort_key(const mera_config& c) {
  return std::to_string(c.d_b) + "/" + std::to_string(c.chi) + "/" + std::to_string(c.n_trans) + "/" +
         std::to_string(c.prec) + "/" + std::to_string(c.w_stiefel) + "/" + std::to_string(c.precond) + "/" +
         std::to_string(c.krylov_dim) + "/" + std::to_string(c.recompute_env) + "/" + std::to_string(c.b_chunk);
}
bool cohort_eligible(const mera_config& cfg, const mera_ctx& m) {
  if (cfg.network != MERA_BINARY || cfg.dtype != MERA_F64 || cfg.z2 || !mera::grouped_eval(m)) return false;
  for (const auto& ly : m.layers)
    for (int sd = 0; sd < 2; ++sd)
      if (!ly.net[sd] || ly.net[sd]->sliced()) return false;
  return true;
}

struct Request {
  int64_t id = 0;
  mera_config cfg{};
  std::vector<char> h3;
  std::vector<std::vector<char>> tensors;
  double gtol = 1e-6;
  int maxiter = 100;
  int method = 0;
  size_t bytes = 0;
  // run state
  mera_t m = nullptr;
  cudaStream_t stream = nullptr;
  Cohort* cohort = nullptr;
  int batched = 0;  // evaluations run together with other requests
  int state = 0;  // 0 queued, 1 running, 2 done, 3 failed
  bool busy = false;
  int iters = 0, n_evals = 0, error = 0, deferred = 0;
  std::string message;
  double energy = 0.0, gnorm = 0.0;
  clk::time_point t_submit, t_admit, t_done;
};

}  // namespace

struct mera_server {
  size_t budget = 0;
  size_t in_use = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<int64_t> queue;                          // waiting, arrival order
  std::map<int64_t, std::unique_ptr<Request>> reqs;   // all requests
  std::vector<int64_t> running;
  size_t rr = 0;
  int64_t next_id = 1;
  bool stop = false;
  int device = 0;
  std::vector<std::thread> workers;
  int64_t done = 0, failed = 0, submitted = 0;
  std::map<std::string, std::unique_ptr<Cohort>> cohorts;
  // a request whose creation ran out of device memory while others ran went
  // back to the head of the queue; nothing is admitted until one of those
  // finishes (done + failed passes this mark); -1: no such wait
  int64_t defer_mark = -1;
  clk::time_point t0 = clk::now();
};

namespace {

// Leave the request's cohort (caller holds mu); the last one frees it.
void leave_cohort(mera_server* sv, Request& r) {
  if (!r.cohort) return;
  Cohort* h = r.cohort;
  r.cohort = nullptr;
  if (--h->refs > 0) return;
  for (auto it = sv->cohorts.begin(); it != sv->cohorts.end(); ++it)
    if (it->second.get() == h) {
      sv->in_use -= h->bytes;
      sv->cohorts.erase(it);
      break;
    }
}

// Join (or found) the cohort of the request's configuration (caller holds
// mu).  The cohort's workspace holds the planes of as many members as a
// batched product takes; without the memory the request runs alone.
void join_cohort(mera_server* sv, Request& r) {
  if (!cohort_eligible(r.cfg, *r.m)) return;
  const std::string key = cohort_key(r.cfg);
  auto it = sv->cohorts.find(key);
  if (it == sv->cohorts.end()) {
    auto h = std::make_unique<Cohort>();
    try {
      constexpr int MAXB = mera::tc::TcEpilogue::MAXB;
      h->ex = r.m->ex;
      h->ex.keep[0] = h->ex.keep[1] = nullptr;
      h->ex.keep_bytes[0] = h->ex.keep_bytes[1] = 0;
      if (r.m->ex.prec != MERA_PREC_FP64) {
        h->ws.alloc((size_t)MAXB * r.m->ex.ws_bytes);
        h->flag.alloc(sizeof(int));
        MERA_CUDA(cudaMemset(h->flag.p, 0, sizeof(int)));
        h->ex.ws = h->ws.p;
        h->ex.ws_bytes = h->ws.bytes;
        h->ex.err = h->flag.as<int>();
      }
      MERA_CUDA(cudaStreamCreateWithFlags(&h->s, cudaStreamNonBlocking));
      h->bytes = h->ws.bytes + h->flag.bytes;
    } catch (...) {
      return;  // no memory for a cohort: this request evaluates alone
    }
    sv->in_use += h->bytes;
    it = sv->cohorts.emplace(key, std::move(h)).first;
  }
  Cohort* h = it->second.get();
  ++h->refs;
  r.cohort = h;
  r.m->cohort = h;
  r.m->cohort_eval = &cohort_eval;
}

void finish(mera_server* sv, Request& r, int err) {
  r.state = err ? 3 : 2;
  r.error = err;
  r.t_done = clk::now();
  leave_cohort(sv, r);
  if (r.m) mera_destroy(r.m);
  r.m = nullptr;
  if (r.stream) cudaStreamDestroy(r.stream);
  r.stream = nullptr;
  r.h3.clear();
  r.tensors.clear();
  sv->in_use -= r.bytes;
  if (err) sv->failed++; else sv->done++;
}

// Admit queued requests in arrival order while they fit (caller holds mu).
void admit_locked(mera_server* sv) {
  if (sv->defer_mark >= 0) {
    if (sv->done + sv->failed <= sv->defer_mark && !sv->running.empty()) return;
    sv->defer_mark = -1;
  }
  while (!sv->queue.empty()) {
    Request& r = *sv->reqs[sv->queue.front()];
    if (sv->in_use + r.bytes > sv->budget && !sv->running.empty()) break;  // wait for memory
    sv->queue.pop_front();
    sv->in_use += r.bytes;
    r.state = 1;
    r.t_admit = clk::now();
    sv->running.push_back(r.id);
  }
}

void worker(mera_server* sv) {
  cudaSetDevice(sv->device);
  std::unique_lock<std::mutex> lk(sv->mu);
  while (true) {
    if (sv->stop) return;  // destroy: leave running requests to the destructor
    admit_locked(sv);
    // pick the next running request that no other worker is stepping
    Request* pick = nullptr;
    for (size_t k = 0; k < sv->running.size(); ++k) {
      Request& r = *sv->reqs[sv->running[(sv->rr + k) % sv->running.size()]];
      if (!r.busy) {
        pick = &r;
        sv->rr = (sv->rr + k + 1) % std::max<size_t>(1, sv->running.size());
        break;
      }
    }
    if (!pick) {
      sv->cv.wait_for(lk, std::chrono::milliseconds(20));
      continue;
    }
    Request& r = *pick;
    r.busy = true;
    // fields a worker may touch without the lock while busy is set: m and
    // stream (no other thread uses them then); everything mera_server_poll
    // reads is written only with the lock held
    const int iters0 = r.iters;
    const double gtol = r.gtol;
    const int maxiter = r.maxiter, method = r.method;
    lk.unlock();
    int err = 0;
    bool finished = false, stepped = false;
    mera_iter_info info{};
    std::string message;
    if (!r.m) {
      // first turn: build the problem on its own stream and load its point
      err = cudaStreamCreateWithFlags(&r.stream, cudaStreamNonBlocking) == cudaSuccess ? 0 : MERA_ERR_CUDA;
      if (!err) err = mera_create(&r.cfg, r.h3.data(), r.stream, &r.m);
      if (!err) {
        std::vector<const void*> ptrs;
        for (auto& t : r.tensors) ptrs.push_back(t.data());
        err = mera_set_tensors(r.m, ptrs.data());
      }
      if (!err) {
        std::lock_guard<std::mutex> g(sv->mu);
        join_cohort(sv, r);
      }
    }
    if (!err) {
      Cohort* h = r.cohort;
      if (h) {
        std::lock_guard<std::mutex> g(h->mu);
        ++h->stepping;
      }
      err = method == 1 ? mera_cg_step(r.m, &info) : mera_lbfgs_step(r.m, &info);
      if (h) {
        std::lock_guard<std::mutex> g(h->mu);
        --h->stepping;
        h->cv.notify_all();  // an evaluation waiting for this request's next one need not
      }
      if (!err) {
        stepped = true;
        finished = info.gnorm < gtol || iters0 + 1 >= maxiter;
      }
    }
    if (err) message = r.m ? mera_last_error(r.m) : "creation failed";
    lk.lock();
    if (err == MERA_ERR_OOM && !r.m && sv->running.size() > 1) {
      // the memory the footprint promised is not there (another user, a
      // bounded allocator): wait for a running request to finish, then retry
      if (r.stream) cudaStreamDestroy(r.stream);
      r.stream = nullptr;
      for (size_t k = 0; k < sv->running.size(); ++k)
        if (sv->running[k] == r.id) {
          sv->running.erase(sv->running.begin() + k);
          break;
        }
      sv->in_use -= r.bytes;
      r.state = 0;
      r.busy = false;
      sv->queue.push_front(r.id);
      sv->defer_mark = sv->done + sv->failed;
      r.deferred++;
      continue;
    }
    if (stepped) {
      r.iters = iters0 + 1;
      r.n_evals += info.n_evals;
      r.energy = info.energy;
      r.gnorm = info.gnorm;
      r.batched = (int)r.m->evals_batched;
    }
    if (err) r.message = message;
    r.busy = false;
    if (err || finished) {
      for (size_t k = 0; k < sv->running.size(); ++k)
        if (sv->running[k] == r.id) {
          sv->running.erase(sv->running.begin() + k);
          break;
        }
      finish(sv, r, err);
      sv->cv.notify_all();
    }
  }
}

}  // namespace

extern "C" {

int mera_server_create(size_t mem_budget_bytes, int n_workers, mera_server_t* out) {
  if (!out || n_workers < 1 || mem_budget_bytes == 0) return MERA_ERR_ARG;
  auto* sv = new (std::nothrow) mera_server();
  if (!sv) return MERA_ERR_OOM;
  sv->budget = mem_budget_bytes;
  cudaGetDevice(&sv->device);
  for (int i = 0; i < n_workers; ++i) sv->workers.emplace_back(worker, sv);
  *out = sv;
  return MERA_OK;
}

int mera_server_submit(mera_server_t sv, const mera_config* cfg, const void* h3, const void* const* tensors,
                       int method, double gtol, int maxiter, int64_t* id) {
  if (!sv || !cfg || !h3 || !tensors || !id || maxiter < 1) return MERA_ERR_ARG;
  if (cfg->network == MERA_MPS) return MERA_ERR_UNSUPPORTED;  // the request stream holds MERA problems
  auto r = std::make_unique<Request>();
  r->cfg = *cfg;
  r->bytes = mera_footprint_bytes(cfg);
  if (r->bytes == 0) return MERA_ERR_ARG;
  if (r->bytes > sv->budget) return MERA_ERR_OOM;
  const bool tern = cfg->network == MERA_TERNARY;
  // operator order: three (binary) or two (ternary) sites
  const int64_t n3 = tern ? (int64_t)cfg->d_b * cfg->d_b : (int64_t)cfg->d_b * cfg->d_b * cfg->d_b;
  const size_t es = sizeof(double) * (cfg->dtype == MERA_C128 ? 2 : 1);
  r->h3.assign(static_cast<const char*>(h3), static_cast<const char*>(h3) + es * n3 * n3);
  std::vector<int64_t> dims{cfg->d_b};
  for (int l = 0; l < cfg->n_trans; ++l) {
    const int64_t d = dims.back();
    dims.push_back(std::min<int64_t>(cfg->chi, tern ? d * d * d : d * d));
  }
  for (int l = 0; l <= cfg->n_trans; ++l) {
    const int64_t cf = dims[l], cc = l < cfg->n_trans ? dims[l + 1] : dims[l];
    const int64_t sz[2] = {cf * cf * cf * cf, (tern ? cf * cf * cf : cf * cf) * cc};
    for (int k = 0; k < 2; ++k) {
      const char* p = static_cast<const char*>(tensors[2 * l + k]);
      if (!p) return MERA_ERR_ARG;
      r->tensors.emplace_back(p, p + es * sz[k]);
    }
  }
  r->gtol = gtol;
  r->maxiter = maxiter;
  r->method = method;
  r->t_submit = clk::now();
  std::lock_guard<std::mutex> lk(sv->mu);
  r->id = sv->next_id++;
  *id = r->id;
  sv->queue.push_back(r->id);
  sv->reqs.emplace(r->id, std::move(r));
  sv->submitted++;
  sv->cv.notify_all();
  return MERA_OK;
}

int mera_server_poll(mera_server_t sv, int64_t id, mera_request_status* st) {
  if (!sv || !st) return MERA_ERR_ARG;
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(id);
  if (it == sv->reqs.end()) return MERA_ERR_ARG;
  const Request& r = *it->second;
  auto sec = [&](clk::time_point t) { return std::chrono::duration<double>(t - sv->t0).count(); };
  st->state = r.state;
  st->error = r.error;
  st->iters = r.iters;
  st->n_evals = r.n_evals;
  st->energy = r.energy;
  st->gnorm = r.gnorm;
  st->t_submit = sec(r.t_submit);
  st->t_admit = r.state >= 1 ? sec(r.t_admit) : -1.0;
  st->t_done = r.state >= 2 ? sec(r.t_done) : -1.0;
  st->bytes = r.bytes;
  std::snprintf(st->message, sizeof(st->message), "%s", r.message.c_str());
  st->deferred = r.deferred;
  st->batched_evals = r.batched;
  return MERA_OK;
}

int mera_server_wait(mera_server_t sv, double timeout_s) {
  if (!sv) return MERA_ERR_ARG;
  std::unique_lock<std::mutex> lk(sv->mu);
  const auto until = clk::now() + std::chrono::duration<double>(timeout_s);
  while (sv->done + sv->failed < sv->submitted) {
    if (sv->cv.wait_until(lk, until) == std::cv_status::timeout) return MERA_ERR_NOCONV;
  }
  return MERA_OK;
}

int mera_server_destroy(mera_server_t sv) {
  if (!sv) return MERA_ERR_ARG;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
    // queued requests that never started are dropped
    sv->queue.clear();
    sv->cv.notify_all();
  }
  for (auto& t : sv->workers) t.join();
  for (auto& kv : sv->reqs)
    if (kv.second->m) finish(sv, *kv.second, MERA_ERR_ARG);
  delete sv;
  return MERA_OK;
}

}  // extern "C"
