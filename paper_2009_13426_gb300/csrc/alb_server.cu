// Serving loop (include/alb.h, alb_server_* / alb_submit / alb_poll): a
// worker thread admits queued requests within a device-memory budget and
// advances every resident flow in chunks of batched steps.
//
// Chunk schedule: resident flows are ranked by remaining work, least first,
// and taken until the chunk's node budget is reached. The selected flows of a
// precision are ordered by remaining steps, longest first, and their work
// items laid out in that order, so the flows that still step at chunk step s
// are a prefix of the table; step s launches that prefix with buffer parity
// s & 1. After the chunk each flow's current buffer has flipped once per step
// it took.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "alb_batcher.h"

using namespace alb;

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t id = 0;
  alb_config cfg{};
  int nsteps = 0;
  std::vector<double> fields;  // 4 n, copied at submit (empty: use fill)
  alb_fill_fn fill = nullptr;
  void* user = nullptr;
  int keep = 0;
  int state = ALB_QUEUED;
  int status = ALB_OK;
  size_t bytes = 0;
  double t_submit = 0, t_admit = 0, t_done = 0;
  alb_handle* h = nullptr;
  int remaining = 0;
  uint64_t steps_done = 0;
  std::vector<double> result;  // 4 n if keep
  alb_stats stats{};
  size_t n() const { return (size_t)cfg.nx * cfg.ny; }
};

}  // namespace

struct alb_server {
  alb_server_config cfg{};
  int device = 0;
  cudaStream_t stream = nullptr;        // chunks of steps (worker thread)
  cudaStream_t admit_stream = nullptr;  // initial states (admission thread)
  GroupPlan* plan[2] = {nullptr, nullptr};  // by precision: 0 FP64 plain, 1 FP32 form
  int* d_counter = nullptr;
  bool tuned[2] = {false, false};
  Clock::time_point t0;
  std::thread worker, admitter;

  std::mutex mu;                  // guards everything below
  std::condition_variable cv;     // submissions, admissions, completions, stop
  bool stop = false;
  uint64_t next_id = 1;
  std::vector<Request*> queue;    // submitted, not yet admitted
  std::vector<Request*> ready;    // initialised, not yet taken by the worker
  std::unordered_map<uint64_t, Request*> live;  // not yet collected by alb_poll
  size_t budget = 0, resident = 0;  // device bytes of admitted flows
  double resident_nodes = 0.0;
  uint64_t running = 0;             // admitted and not finished
  alb_server_stats st{};
  // time of one node update per precision (0 FP64 plain, 1 FP32 form), ms;
  // starting guesses, then measured on every chunk
  double ms_per_update[2] = {1.5e-5, 2.0e-6};

  // worker-only
  std::vector<Request*> active;
  std::vector<cudaEvent_t> ev;    // two per (step, group) of a chunk
  std::vector<int> ev_group;

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

// Publish the outcome. After this call alb_poll may free r at any time: the
// worker must not touch r again.
void finish(alb_server* s, Request* r, int state, int status, bool was_running) {
  std::lock_guard<std::mutex> lk(s->mu);
  r->state = state;
  r->status = status;
  r->t_done = s->now();
  s->resident -= r->bytes;
  s->resident_nodes -= (double)r->n();
  if (was_running) s->running -= 1;
  if (state == ALB_DONE) s->st.completed += 1;
  else s->st.failed += 1;
  s->cv.notify_all();
}

// Admission (admission thread): create the flow, produce its fields and
// Grad-initialise it on the admission stream, then hand it to the worker.
void start(alb_server* s, Request* r) {
  alb_config c = r->cfg;
  c.stream = s->admit_stream;
  alb_handle* h = nullptr;
  int rc = alb_create(&c, &h);
  if (rc != ALB_OK) {
    finish(s, r, ALB_FAILED, rc, false);
    return;
  }
  h->owner = s;
  const size_t n = r->n();
  try {
    if (r->fields.empty()) {
      r->fields.resize(4 * n);
      double* f = r->fields.data();
      if (!r->fill || r->fill(r->user, f, f + n, f + 2 * n, f + 3 * n) != 0) rc = ALB_EINVAL;
    }
  } catch (const std::bad_alloc&) {
    rc = ALB_ENOMEM;
  }
  if (rc == ALB_OK) {
    const double* f = r->fields.data();
    rc = alb_init(h, f, f + n, f + 2 * n, f + 3 * n, ALB_HOST);
  }
  std::vector<double>().swap(r->fields);
  if (rc != ALB_OK) {
    handle_destroy(h);
    finish(s, r, ALB_FAILED, rc, false);
    return;
  }
  // from now on the flow works on the worker's stream (alb_init has
  // synchronised the admission stream)
  h->stream = s->stream;
  r->h = h;
  r->remaining = r->nsteps;
  std::lock_guard<std::mutex> lk(s->mu);
  r->state = ALB_RUNNING;
  r->t_admit = s->now();
  s->running += 1;
  s->st.admitted += 1;
  s->ready.push_back(r);
  s->cv.notify_all();
}

// A flow that took all its steps: counters, moments to host, free the device.
void complete(alb_server* s, Request* r) {
  int status = alb_stats_get(r->h, &r->stats);
  if (status == ALB_OK && (r->stats.newton_failures || r->stats.reconstruction_failures))
    status = ALB_ENEWTON;
  if (r->keep) {
    const size_t n = r->n();
    try {
      r->result.resize(4 * n);
      double* f = r->result.data();
      const int rc = alb_moments(r->h, f, f + n, f + 2 * n, f + 3 * n, ALB_HOST);
      if (rc != ALB_OK) status = rc;
    } catch (const std::bad_alloc&) {
      status = ALB_ENOMEM;
    }
  }
  handle_destroy(r->h);
  r->h = nullptr;
  finish(s, r, status == ALB_OK || status == ALB_ENEWTON ? ALB_DONE : ALB_FAILED, status, true);
}

// One chunk of batched steps: the selected flows (least remaining work
// first, up to batch_nodes nodes) step min(k, their remaining) times. Returns
// false on a CUDA error (every active request then fails).
bool run_chunk(alb_server* s) {
  auto& act = s->active;
  double cost[2];
  {
    std::lock_guard<std::mutex> lk(s->mu);
    cost[0] = s->ms_per_update[0];
    cost[1] = s->ms_per_update[1];
  }
  auto prec = [](const Request* r) { return r->cfg.precision == ALB_FP32_FORM ? 1 : 0; };
  auto work = [&](const Request* r) {
    return (double)r->n() * (double)r->remaining * cost[prec(r)];
  };
  std::stable_sort(act.begin(), act.end(),
                   [&](const Request* a, const Request* b) { return work(a) < work(b); });
  size_t nsel = 0;
  double nodes = 0.0;
  while (nsel < act.size() &&
         (nsel == 0 || s->cfg.batch_nodes <= 0 || nodes < (double)s->cfg.batch_nodes))
    nodes += (double)act[nsel++]->n();
  std::vector<Request*> sel(act.begin(), act.begin() + nsel);
  // within the chunk, the flows that still step form a prefix of each group
  std::stable_sort(sel.begin(), sel.end(),
                   [](const Request* a, const Request* b) { return a->remaining > b->remaining; });
  std::vector<FlowDev*> grp[2];
  std::vector<int> rem[2];
  double step_ms = 0.0;
  for (Request* r : sel) {
    grp[prec(r)].push_back(&r->h->dev);
    rem[prec(r)].push_back(r->remaining);
    step_ms += (double)r->n() * cost[prec(r)];
  }
  int k = (int)(s->cfg.chunk_ms / step_ms + 0.5);
  k = std::max(1, std::min(k, s->cfg.max_chunk));
  k = std::min(k, sel.front()->remaining);
  cudaError_t e = cudaSuccess;
  for (int g = 0; g < 2 && e == cudaSuccess; ++g) {
    e = s->plan[g]->set_flows(grp[g], s->stream);
    if (e == cudaSuccess && s->cfg.tune && !s->tuned[g] && !grp[g].empty()) {
      tune_group(s->plan[g], s->stream, s->d_counter + g, 2);
      s->tuned[g] = true;
    }
  }
  const auto t = Clock::now();
  double updates[2] = {0.0, 0.0};
  int nev = 0;
  for (int st = 0; st < k && e == cudaSuccess; ++st) {
    for (int g = 0; g < 2 && e == cudaSuccess; ++g) {
      // flows with more than st steps left form a prefix of the group
      const int nf = (int)(std::upper_bound(rem[g].begin(), rem[g].end(), st,
                                            [](int v, int r) { return v >= r; }) -
                           rem[g].begin());
      if (nf == 0) continue;
      for (int f = 0; f < nf; ++f) updates[g] += (double)grp[g][f]->n;
      e = cudaEventRecord(s->ev[nev], s->stream);
      if (e == cudaSuccess)
        e = s->plan[g]->launch(st & 1, s->plan[g]->items_before(nf), s->d_counter + g, s->stream);
      if (e == cudaSuccess) e = cudaEventRecord(s->ev[nev + 1], s->stream);
      s->ev_group[nev / 2] = g;
      nev += 2;
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  const double ms = std::chrono::duration<double, std::milli>(Clock::now() - t).count();
  if (e != cudaSuccess) {
    cudaGetLastError();
    for (Request* r : act) {
      handle_destroy(r->h);
      r->h = nullptr;
      finish(s, r, ALB_FAILED, ALB_ECUDA, true);
    }
    act.clear();
    return false;
  }
  // measured time of a node update per precision (smoothed)
  double gms[2] = {0.0, 0.0};
  for (int j = 0; j < nev; j += 2) {
    float m = 0.0f;
    if (cudaEventElapsedTime(&m, s->ev[j], s->ev[j + 1]) == cudaSuccess) gms[s->ev_group[j / 2]] += m;
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (int g = 0; g < 2; ++g)
      if (updates[g] > 0.0 && gms[g] > 0.0)
        s->ms_per_update[g] = 0.5 * s->ms_per_update[g] + 0.5 * gms[g] / updates[g];
    s->st.chunks += 1;
    s->st.steps += (uint64_t)k;
    s->st.node_updates += (uint64_t)(updates[0] + updates[1]);
    s->st.busy_seconds += ms * 1e-3;
  }
  std::vector<Request*> still(act.begin() + nsel, act.end());
  for (Request* r : sel) {
    const int d = std::min(k, r->remaining);
    r->remaining -= d;
    r->steps_done += (uint64_t)d;
    r->h->steps += (uint64_t)d;
    if (d & 1) r->h->dev.cur ^= 1;
    if (r->remaining == 0) complete(s, r);
    else still.push_back(r);
  }
  act.swap(still);
  return true;
}

// Queued request to admit next, or null: least estimated work first, among
// those that fit the device-memory budget, while the resident flows hold
// fewer than twice batch_nodes nodes (and fewer than max_flows flows).
// Called with s->mu held.
Request* pick_admission(alb_server* s) {
  if (s->queue.empty()) return nullptr;
  if (s->cfg.batch_nodes > 0 && s->resident_nodes >= 2.0 * (double)s->cfg.batch_nodes)
    return nullptr;
  if (s->cfg.max_flows > 0 && s->running >= (uint64_t)s->cfg.max_flows) return nullptr;
  size_t best = s->queue.size();
  double wbest = 0.0;
  for (size_t j = 0; j < s->queue.size(); ++j) {
    const Request* r = s->queue[j];
    if (s->resident + r->bytes > s->budget) continue;
    const double w = (double)r->n() * (double)r->nsteps *
                     s->ms_per_update[r->cfg.precision == ALB_FP32_FORM ? 1 : 0];
    if (best == s->queue.size() || w < wbest) {
      best = j;
      wbest = w;
    }
  }
  if (best == s->queue.size()) return nullptr;
  Request* r = s->queue[best];
  s->queue.erase(s->queue.begin() + best);
  return r;
}

void admitter_main(alb_server* s) {
  cudaSetDevice(s->device);
  for (;;) {
    Request* r = nullptr;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      for (;;) {
        if (s->stop) return;
        if ((r = pick_admission(s)) != nullptr) break;
        s->cv.wait_for(lk, std::chrono::milliseconds(20));
      }
      s->resident += r->bytes;
      s->resident_nodes += (double)r->n();
    }
    start(s, r);
  }
}

void worker_main(alb_server* s) {
  cudaSetDevice(s->device);
  for (;;) {
    std::vector<Request*> fresh;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      for (;;) {
        if (s->stop) return;
        if (!s->ready.empty() || !s->active.empty()) break;
        s->cv.wait_for(lk, std::chrono::milliseconds(20));
      }
      fresh.swap(s->ready);
    }
    for (Request* r : fresh) {
      if (r->remaining == 0) complete(s, r);
      else s->active.push_back(r);
    }
    if (!s->active.empty()) run_chunk(s);
  }
}

}  // namespace

extern "C" {

int alb_server_config_default(alb_server_config* c) {
  if (!c) return set_error(ALB_EINVAL, "alb_server_config_default: null pointer");
  c->hbm_fraction = 0.8;
  c->chunk_ms = 100.0;
  c->max_chunk = 256;
  c->max_flows = 0;
  c->batch_nodes = 1LL << 22;
  c->tune = 0;
  return ALB_OK;
}

int alb_server_destroy(alb_server* s) {
  if (!s) return ALB_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv.notify_all();
  }
  if (s->worker.joinable()) s->worker.join();
  if (s->admitter.joinable()) s->admitter.join();
  if (s->stream) cudaStreamSynchronize(s->stream);
  for (auto* list : {&s->active, &s->ready})
    for (Request* r : *list) {
      if (r->h) handle_destroy(r->h);
      r->h = nullptr;
    }
  for (auto& kv : s->live) delete kv.second;
  delete s->plan[0];
  delete s->plan[1];
  cudaFree(s->d_counter);
  for (cudaEvent_t ev : s->ev)
    if (ev) cudaEventDestroy(ev);
  if (s->stream) cudaStreamDestroy(s->stream);
  if (s->admit_stream) cudaStreamDestroy(s->admit_stream);
  delete s;
  return ALB_OK;
}

int alb_server_create(const alb_server_config* c, alb_server** out) {
  if (!out) return set_error(ALB_EINVAL, "alb_server_create: null output");
  *out = nullptr;
  alb_server_config cfg;
  alb_server_config_default(&cfg);
  if (c) cfg = *c;
  if (!(cfg.hbm_fraction > 0.0 && cfg.hbm_fraction <= 1.0) || !(cfg.chunk_ms > 0.0) ||
      cfg.max_chunk < 1 || cfg.max_chunk > 4096 || cfg.max_flows < 0 || cfg.batch_nodes < 0)
    return set_error(ALB_EINVAL, "alb_server_create: bad configuration");
  alb_server* s = new (std::nothrow) alb_server();
  if (!s) return set_error(ALB_ENOMEM, "alb_server_create: host allocation failed");
  s->cfg = cfg;
  s->t0 = Clock::now();
  size_t free_b = 0, total_b = 0;
  cudaError_t e = cudaGetDevice(&s->device);
  if (e == cudaSuccess) e = cudaMemGetInfo(&free_b, &total_b);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->admit_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMalloc((void**)&s->d_counter, 2 * sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(s->d_counter, 0, 2 * sizeof(int));
  s->ev.assign(4 * (size_t)cfg.max_chunk, nullptr);
  s->ev_group.assign(2 * (size_t)cfg.max_chunk, 0);
  for (size_t j = 0; j < s->ev.size() && e == cudaSuccess; ++j) e = cudaEventCreate(&s->ev[j]);
  if (e != cudaSuccess) {
    alb_server_destroy(s);
    return cuda_error(e, "alb_server_create");
  }
  const size_t reserve = (size_t)1 << 30;
  s->budget = std::min((size_t)(cfg.hbm_fraction * (double)total_b),
                       free_b > reserve ? free_b - reserve : 0);
  s->st.budget_bytes = s->budget;
  for (int g = 0; g < 2; ++g) {
    const int prec = g == 1 ? ALB_FP32_FORM : ALB_FP64_PLAIN;
    s->plan[g] = new (std::nothrow) GroupPlan(prec);
    if (!s->plan[g] || s->plan[g]->set_tuning(default_tuning(prec), s->stream) != cudaSuccess) {
      alb_server_destroy(s);
      return set_error(ALB_ECUDA, "alb_server_create: batch plan");
    }
  }
  try {
    s->worker = std::thread(worker_main, s);
    s->admitter = std::thread(admitter_main, s);
  } catch (...) {
    alb_server_destroy(s);
    return set_error(ALB_ENOMEM, "alb_server_create: worker thread");
  }
  *out = s;
  return ALB_OK;
}

int alb_submit(alb_server* s, const alb_request* r, uint64_t* id) {
  if (!s || !r || !id) return set_error(ALB_EINVAL, "alb_submit: null pointer");
  int rc = config_check(&r->cfg);
  if (rc != ALB_OK) return rc;
  if (r->cfg.stencil != ALB_D2Q21)
    return set_error(ALB_EUNSUPPORTED, "alb_submit: the server runs D2Q21 flows only");
  if (r->nsteps < 0) return set_error(ALB_EINVAL, "alb_submit: nsteps < 0");
  const bool copy = r->rho || r->rhoux || r->rhouy || r->rhoE;
  if (copy && !(r->rho && r->rhoux && r->rhouy && r->rhoE))
    return set_error(ALB_EINVAL, "alb_submit: give all four fields or none");
  if (!copy && !r->fill) return set_error(ALB_EINVAL, "alb_submit: no fields and no fill");
  Request* q = new (std::nothrow) Request();
  if (!q) return set_error(ALB_ENOMEM, "alb_submit: host allocation failed");
  q->cfg = r->cfg;
  q->cfg.stream = nullptr;
  q->nsteps = r->nsteps;
  q->fill = r->fill;
  q->user = r->user;
  q->keep = r->keep_result ? 1 : 0;
  q->bytes = flow_device_bytes(&q->cfg);
  if (q->bytes > s->budget) {
    delete q;
    return set_error(ALB_ENOMEM, "alb_submit: the flow needs more device memory than the budget");
  }
  if (copy) {
    const size_t n = q->n();
    try {
      q->fields.resize(4 * n);
    } catch (const std::bad_alloc&) {
      delete q;
      return set_error(ALB_ENOMEM, "alb_submit: host allocation failed");
    }
    memcpy(q->fields.data(), r->rho, n * sizeof(double));
    memcpy(q->fields.data() + n, r->rhoux, n * sizeof(double));
    memcpy(q->fields.data() + 2 * n, r->rhouy, n * sizeof(double));
    memcpy(q->fields.data() + 3 * n, r->rhoE, n * sizeof(double));
  }
  std::lock_guard<std::mutex> lk(s->mu);
  q->id = s->next_id++;
  q->t_submit = s->now();
  s->queue.push_back(q);
  s->live[q->id] = q;
  s->st.submitted += 1;
  *id = q->id;
  s->cv.notify_all();
  return ALB_OK;
}

int alb_poll(alb_server* s, uint64_t id, int* state, alb_result* res) {
  if (!s || !state) return set_error(ALB_EINVAL, "alb_poll: null pointer");
  Request* q = nullptr;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->live.find(id);
    if (it == s->live.end()) return set_error(ALB_ENOTFOUND, "alb_poll: unknown request %llu",
                                              (unsigned long long)id);
    q = it->second;
    *state = q->state;
    if (q->state != ALB_DONE && q->state != ALB_FAILED) return ALB_OK;
    s->live.erase(it);
  }
  if (res) {
    const size_t n = q->n();
    if (q->keep && q->result.size() == 4 * n) {
      double* outs[4] = {res->rho, res->rhoux, res->rhouy, res->rhoE};
      for (int j = 0; j < 4; ++j)
        if (outs[j]) memcpy(outs[j], q->result.data() + j * n, n * sizeof(double));
    }
    res->status = q->status;
    res->steps = q->steps_done;
    res->stats = q->stats;
    res->t_submit = q->t_submit;
    res->t_admit = q->t_admit;
    res->t_done = q->t_done;
  }
  delete q;
  return ALB_OK;
}

int alb_server_drain(alb_server* s, int timeout_ms) {
  if (!s) return set_error(ALB_EINVAL, "alb_server_drain: null server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto idle = [s] {
    return s->queue.empty() && s->ready.empty() && s->running == 0 && s->resident == 0;
  };
  if (timeout_ms < 0) {
    s->cv.wait(lk, idle);
  } else if (!s->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), idle)) {
    return set_error(ALB_ETIMEDOUT, "alb_server_drain: still busy after %d ms", timeout_ms);
  }
  return ALB_OK;
}

int alb_server_stats_get(alb_server* s, alb_server_stats* out) {
  if (!s || !out) return set_error(ALB_EINVAL, "alb_server_stats_get: null pointer");
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->st;
  out->queued = s->queue.size();
  out->running = s->running;
  out->resident_bytes = s->resident;
  out->budget_bytes = s->budget;
  out->elapsed_seconds = s->now();
  out->ns_per_update[0] = s->ms_per_update[0] * 1e6;
  out->ns_per_update[1] = s->ms_per_update[1] * 1e6;
  return ALB_OK;
}

}  // extern "C"
