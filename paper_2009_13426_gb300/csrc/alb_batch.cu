// Batched flows (include/alb.h, alb_batch_*): many independent flows of
// uneven size advanced by one persistent launch per step and precision, two
// steps captured as a CUDA graph, launch shape chosen by an autotuner.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "alb_batcher.h"

using namespace alb;

namespace alb {

// ------------------------------------------------------------------ variants

int batch_variant_count(int precision) {
  return precision == ALB_FP32_FORM ? batch_variant_count_f32() : batch_variant_count_f64();
}

BatchVariant batch_variant(int precision, int v) {
  return precision == ALB_FP32_FORM ? batch_variant_f32(v) : batch_variant_f64(v);
}

static int batch_occupancy(int precision, int v) {
  return precision == ALB_FP32_FORM ? batch_occupancy_f32(v) : batch_occupancy_f64(v);
}

static cudaError_t launch_variant(int precision, int v, const void* args, const int* cur,
                                  const WorkItem* items, int nitems, int parity, int* counter,
                                  int grid, cudaStream_t s) {
  return precision == ALB_FP32_FORM
             ? launch_batch_step_f32(v, args, cur, items, nitems, parity, counter, grid, s)
             : launch_batch_step_f64(v, args, cur, items, nitems, parity, counter, grid, s);
}

const char* check_tuning(int precision, const Tuning& t) {
  if (t.variant < 0 || t.variant >= batch_variant_count(precision)) return "unknown variant";
  const int block = batch_variant(precision, t.variant).block;
  for (int c = 0; c < 3; ++c) {
    const int w = t.tile_w[c];
    if (w < 8 || w > block || (w & (w - 1))) return "tile_w must be a power of two in [8, block]";
  }
  if (t.dynamic != 0 && t.dynamic != 1) return "dynamic must be 0 or 1";
  if (t.blocks_per_sm < 0) return "blocks_per_sm must be >= 0";
  return nullptr;
}

__global__ void flip_kernel(int* cur, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) cur[i] ^= 1;
}

cudaError_t launch_flip(int* cur, int n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  flip_kernel<<<(n + 255) / 256, 256, 0, s>>>(cur, n);
  return cudaGetLastError();
}

// ----------------------------------------------------------------- GroupPlan

GroupPlan::~GroupPlan() {
  cudaFree(d_args_);
  cudaFree(d_cur_);
  cudaFree(d_items_);
}

cudaError_t GroupPlan::reserve(void** p, size_t* cap, size_t bytes) {
  if (bytes <= *cap) return cudaSuccess;
  const size_t want = std::max(bytes, *cap * 2);
  cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  const cudaError_t e = cudaMalloc(p, want);
  if (e == cudaSuccess) *cap = want;
  return e;
}

cudaError_t GroupPlan::set_flows(const std::vector<FlowDev*>& flows, cudaStream_t s) {
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  flows_ = flows;
  const int n = nflows();
  if (n == 0) {
    ends_.clear();
    ntable_ = 0;
    return cudaSuccess;
  }
  const size_t asz = precision_ == ALB_FP32_FORM ? sizeof(StepArgs<float>) : sizeof(StepArgs<double>);
  std::vector<unsigned char> host(asz * 2 * n);
  for (int f = 0; f < n; ++f)
    for (int b = 0; b < 2; ++b) {
      unsigned char* dst = host.data() + asz * (2 * (size_t)f + b);
      if (precision_ == ALB_FP32_FORM) {
        const StepArgs<float> a = step_args<float>(*flows_[f], b);
        memcpy(dst, &a, asz);
      } else {
        const StepArgs<double> a = step_args<double>(*flows_[f], b);
        memcpy(dst, &a, asz);
      }
    }
  if ((e = reserve(&d_args_, &args_cap_, host.size())) != cudaSuccess) return e;
  if ((e = cudaMemcpy(d_args_, host.data(), host.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
    return e;
  if ((e = reserve((void**)&d_cur_, &cur_cap_, sizeof(int) * n)) != cudaSuccess) return e;
  if ((e = upload_cur(s)) != cudaSuccess) return e;
  return set_tuning(tuning_, s);
}

cudaError_t GroupPlan::upload_cur(cudaStream_t s) {
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess || flows_.empty()) return e;
  std::vector<int> cur(flows_.size());
  for (size_t f = 0; f < flows_.size(); ++f) cur[f] = flows_[f]->cur;
  return cudaMemcpy(d_cur_, cur.data(), sizeof(int) * cur.size(), cudaMemcpyHostToDevice);
}

cudaError_t GroupPlan::build_items(cudaStream_t s, int only_class) {
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  const int block = batch_variant(precision_, tuning_.variant).block;
  std::vector<WorkItem> items;
  if (only_class < 0) ends_.assign(flows_.size(), 0);
  for (size_t f = 0; f < flows_.size(); ++f) {
    const Params& p = flows_[f]->prm;
    const int c = size_class(p.nx);
    if (only_class < 0 || c == only_class) {
      const int tw = std::min(tuning_.tile_w[c], block);
      int lg = 0;
      while ((1 << lg) < tw) ++lg;
      const int th = block >> lg;
      for (int y0 = 0; y0 < p.ny; y0 += th)
        for (int x0 = 0; x0 < p.nx; x0 += (1 << lg)) items.push_back(WorkItem{(int)f, x0, y0, lg});
    }
    if (only_class < 0) ends_[f] = (int)items.size();
  }
  ntable_ = (int)items.size();
  if (items.empty()) return cudaSuccess;
  if ((e = reserve((void**)&d_items_, &items_cap_, sizeof(WorkItem) * items.size())) != cudaSuccess)
    return e;
  return cudaMemcpy(d_items_, items.data(), sizeof(WorkItem) * items.size(),
                    cudaMemcpyHostToDevice);
}

cudaError_t GroupPlan::set_tuning(const Tuning& t, cudaStream_t s) {
  tuning_ = t;
  const int occ = batch_occupancy(precision_, t.variant);
  if (occ <= 0) return cudaErrorInvalidConfiguration;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int per_sm = t.blocks_per_sm > 0 ? std::min(t.blocks_per_sm, occ) : occ;
  grid_ = per_sm * sms;
  return build_items(s, -1);
}

cudaError_t GroupPlan::restrict_to_class(int c, cudaStream_t s) { return build_items(s, c); }

cudaError_t GroupPlan::launch(int parity, int nitems, int* counter, cudaStream_t s) const {
  if (nitems <= 0) return cudaSuccess;
  if (nitems > ntable_) return cudaErrorInvalidValue;  // never read past the table
  if (tuning_.dynamic) {
    const cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
  }
  const int grid = std::max(1, std::min(grid_, nitems));
  return launch_variant(precision_, tuning_.variant, d_args_, d_cur_, d_items_, nitems, parity,
                        tuning_.dynamic ? counter : nullptr, grid, s);
}

cudaError_t GroupPlan::flip(cudaStream_t s) const { return launch_flip(d_cur_, nflows(), s); }

#define ALB_CUDA(call, what)                                \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_error(e_, what);     \
  } while (0)

// Default launch shape of a precision: variant 0, tiles no wider than it.
Tuning default_tuning(int precision) {
  Tuning t;
  const int block = batch_variant(precision, 0).block;
  for (int c = 0; c < 3; ++c) t.tile_w[c] = std::min(t.tile_w[c], block);
  return t;
}

// Mean time of one step of the plan's current table, without changing any
// flow's state: every launch reads the current buffers (parity 0) and writes
// the other ones, and the flows' counters are saved and restored around it.
static int time_plan(cudaStream_t stream, GroupPlan* p, int nitems, int trials, unsigned long long* saved,
              int* counter, float* ms) {
  const auto& fl = p->flows();
  for (size_t f = 0; f < fl.size(); ++f)
    ALB_CUDA(cudaMemcpyAsync(saved + CTR_COUNT * f, fl[f]->ctr,
                             CTR_COUNT * sizeof(unsigned long long), cudaMemcpyDeviceToDevice,
                             stream), "alb_batch_tune: save counters");
  cudaEvent_t e0, e1;
  ALB_CUDA(cudaEventCreate(&e0), "alb_batch_tune: event");
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return set_error(ALB_ECUDA, "alb_batch_tune: event");
  }
  cudaError_t e = p->launch(0, nitems, counter, stream);  // warm-up
  if (e == cudaSuccess) e = cudaEventRecord(e0, stream);
  for (int t = 0; t < trials && e == cudaSuccess; ++t) e = p->launch(0, nitems, counter, stream);
  if (e == cudaSuccess) e = cudaEventRecord(e1, stream);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_error(e, "alb_batch_tune: timed launch");
  *ms /= (float)trials;
  for (size_t f = 0; f < fl.size(); ++f)
    ALB_CUDA(cudaMemcpyAsync(fl[f]->ctr, saved + CTR_COUNT * f,
                             CTR_COUNT * sizeof(unsigned long long), cudaMemcpyDeviceToDevice,
                             stream), "alb_batch_tune: restore counters");
  ALB_CUDA(cudaStreamSynchronize(stream), "alb_batch_tune: synchronise");
  return ALB_OK;
}

static int try_tuning(cudaStream_t stream, GroupPlan* p, const Tuning& t, int only_class, int trials,
               unsigned long long* saved, int* counter, float* ms) {
  ALB_CUDA(p->set_tuning(t, stream), "alb_batch_tune: tuning");
  if (only_class >= 0)
    ALB_CUDA(p->restrict_to_class(only_class, stream), "alb_batch_tune: class table");
  return time_plan(stream, p, p->table_items(), trials, saved, counter, ms);
}


// Coordinate search of one precision's launch shape: the kernel variant
// (tiles as wide as the block), then the tile width of each size class
// present (timing only that class's items), then static against dynamic work
// distribution. The plan ends with the best shape found (the default one
// after an error) and a full item table.
int tune_group(GroupPlan* p, cudaStream_t stream, int* counter, int trials) {
  unsigned long long* saved = nullptr;
  cudaError_t e = cudaMalloc((void**)&saved, (size_t)std::max(1, p->nflows()) * CTR_COUNT *
                                                 sizeof(unsigned long long));
  if (e != cudaSuccess) return cuda_error(e, "alb_batch_tune: scratch");
  int rc = ALB_OK;
  const int prec = p->precision();
  bool present[3] = {false, false, false};
  for (FlowDev* f : p->flows()) present[size_class(f->prm.nx)] = true;
  Tuning best = p->tuning();
  float best_ms = 0.0f;
  // 1. kernel variant, tiles as wide as the block
  for (int v = 0; v < batch_variant_count(prec) && rc == ALB_OK; ++v) {
    Tuning t = best;
    t.variant = v;
    const int block = batch_variant(prec, v).block;
    for (int c = 0; c < 3; ++c) t.tile_w[c] = std::min(128, block);
    float ms = 0.0f;
    rc = try_tuning(stream, p, t, -1, trials, saved, counter, &ms);
    if (rc == ALB_OK && (v == 0 || ms < best_ms)) {
      best = t;
      best_ms = ms;
    }
  }
  // 2. tile width per size class
  const int block = batch_variant(prec, best.variant).block;
  for (int c = 0; c < 3 && rc == ALB_OK; ++c) {
    if (!present[c]) continue;
    float cbest = -1.0f;
    int wbest = best.tile_w[c];
    for (int w = 8; w <= block && rc == ALB_OK; w *= 2) {
      Tuning t = best;
      t.tile_w[c] = w;
      float ms = 0.0f;
      rc = try_tuning(stream, p, t, c, trials, saved, counter, &ms);
      if (rc == ALB_OK && (cbest < 0.0f || ms < cbest)) {
        cbest = ms;
        wbest = w;
      }
    }
    best.tile_w[c] = wbest;
  }
  // 3. work distribution
  float ms_d[2] = {0.0f, 0.0f};
  for (int d = 0; d < 2 && rc == ALB_OK; ++d) {
    Tuning t = best;
    t.dynamic = d;
    rc = try_tuning(stream, p, t, -1, trials, saved, counter, &ms_d[d]);
  }
  if (rc == ALB_OK) best.dynamic = ms_d[1] < ms_d[0] ? 1 : 0;
  if (p->set_tuning(rc == ALB_OK ? best : default_tuning(prec), stream) != cudaSuccess &&
      rc == ALB_OK)
    rc = set_error(ALB_ECUDA, "alb_batch_tune: final tuning");
  cudaFree(saved);
  return rc;
}

}  // namespace alb

// ----------------------------------------------------------------- the batch

struct alb_batch {
  std::vector<alb_handle*> flows;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  GroupPlan* plan[2] = {nullptr, nullptr};  // by precision
  std::vector<int> cur_seen;                // FlowDev::cur as last uploaded
  int* d_counter = nullptr;                 // one work counter per precision
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool dirty = true;
};

namespace {

void drop_graph(alb_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  b->dirty = true;
}

// One step of every flow: flow f reads its buffer cur[f] ^ parity.
cudaError_t step_all(alb_batch* b, int parity) {
  for (int g = 0; g < 2; ++g) {
    const GroupPlan* p = b->plan[g];
    if (!p || p->nflows() == 0) continue;
    const cudaError_t e = p->launch(parity, p->nitems(), b->d_counter + g, b->stream);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int build_graph(alb_batch* b) {
  drop_graph(b);
  ALB_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal),
           "alb_batch: begin capture");
  cudaError_t e = step_all(b, 0);
  if (e == cudaSuccess) e = step_all(b, 1);
  cudaGraph_t g = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return cuda_error(e != cudaSuccess ? e : e2, "alb_batch: capture of two steps");
  }
  b->graph = g;
  ALB_CUDA(cudaGraphInstantiate(&b->exec, g, 0), "alb_batch: graph instantiate");
  b->dirty = false;
  return ALB_OK;
}

// Bring the device copy of each flow's current buffer up to date (a flow may
// have been stepped or re-initialised through its own handle).
int sync_cur(alb_batch* b) {
  bool changed = false;
  for (size_t f = 0; f < b->flows.size(); ++f)
    if (b->flows[f]->dev.cur != b->cur_seen[f]) changed = true;
  if (!changed) return ALB_OK;
  for (int g = 0; g < 2; ++g)
    if (b->plan[g] && b->plan[g]->nflows())
      ALB_CUDA(b->plan[g]->upload_cur(b->stream), "alb_batch: current buffers");
  for (size_t f = 0; f < b->flows.size(); ++f) b->cur_seen[f] = b->flows[f]->dev.cur;
  return ALB_OK;
}

int to_tuning(const alb_batch_tuning* in, Tuning* out) {
  out->variant = in->variant;
  for (int c = 0; c < 3; ++c) out->tile_w[c] = in->tile_w[c];
  out->dynamic = in->dynamic;
  out->blocks_per_sm = in->blocks_per_sm;
  return ALB_OK;
}

void from_tuning(const Tuning& in, alb_batch_tuning* out) {
  out->variant = in.variant;
  for (int c = 0; c < 3; ++c) out->tile_w[c] = in.tile_w[c];
  out->dynamic = in.dynamic;
  out->blocks_per_sm = in.blocks_per_sm;
}

}  // namespace

extern "C" {

int alb_batch_variants(int precision, int* count, int* block, int* min_blocks) {
  if (precision != ALB_FP32_FORM && precision != ALB_FP64_PLAIN)
    return set_error(ALB_EINVAL, "alb_batch_variants: unknown precision %d", precision);
  const int n = batch_variant_count(precision);
  if (count) *count = n;
  for (int v = 0; v < n; ++v) {
    if (block) block[v] = batch_variant(precision, v).block;
    if (min_blocks) min_blocks[v] = batch_variant(precision, v).min_blocks;
  }
  return ALB_OK;
}

int alb_batch_destroy(alb_batch* b) {
  if (!b) return ALB_OK;
  if (b->stream) cudaStreamSynchronize(b->stream);
  drop_graph(b);
  delete b->plan[0];
  delete b->plan[1];
  cudaFree(b->d_counter);
  for (alb_handle* h : b->flows) handle_destroy(h);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
  return ALB_OK;
}

int alb_batch_create(const alb_config* cfgs, int nflows, void* stream, alb_batch** out) {
  if (!out) return set_error(ALB_EINVAL, "alb_batch_create: null output");
  *out = nullptr;
  if (!cfgs || nflows < 1) return set_error(ALB_EINVAL, "alb_batch_create: need >= 1 flow");
  alb_batch* b = new (std::nothrow) alb_batch();
  if (!b) return set_error(ALB_ENOMEM, "alb_batch_create: host allocation failed");
  if (stream) {
    b->stream = (cudaStream_t)stream;
  } else {
    const cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete b;
      return cuda_error(e, "alb_batch_create: stream");
    }
    b->own_stream = true;
  }
  std::vector<FlowDev*> groups[2];
  for (int i = 0; i < nflows; ++i) {
    alb_config c = cfgs[i];
    c.stream = b->stream;
    if (c.stencil != ALB_D2Q21) {
      alb_batch_destroy(b);
      return set_error(ALB_EUNSUPPORTED, "alb_batch_create: flow %d: batches run D2Q21 only", i);
    }
    alb_handle* h = nullptr;
    const int rc = alb_create(&c, &h);
    if (rc != ALB_OK) {
      alb_batch_destroy(b);
      return rc;
    }
    h->owner = b;
    b->flows.push_back(h);
    groups[c.precision == ALB_FP32_FORM ? 1 : 0].push_back(&h->dev);
  }
  b->cur_seen.assign(nflows, 0);
  cudaError_t e = cudaMalloc((void**)&b->d_counter, 2 * sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(b->d_counter, 0, 2 * sizeof(int));
  for (int g = 0; g < 2 && e == cudaSuccess; ++g) {
    const int precision = g == 1 ? ALB_FP32_FORM : ALB_FP64_PLAIN;
    b->plan[g] = new (std::nothrow) GroupPlan(precision);
    if (!b->plan[g]) {
      alb_batch_destroy(b);
      return set_error(ALB_ENOMEM, "alb_batch_create: host allocation failed");
    }
    e = b->plan[g]->set_tuning(default_tuning(precision), b->stream);
    if (e == cudaSuccess) e = b->plan[g]->set_flows(groups[g], b->stream);
  }
  if (e != cudaSuccess) {
    alb_batch_destroy(b);
    return cuda_error(e, "alb_batch_create");
  }
  *out = b;
  return ALB_OK;
}

int alb_batch_flow(alb_batch* b, int i, alb_handle** out) {
  if (!b || !out) return set_error(ALB_EINVAL, "alb_batch_flow: null pointer");
  if (i < 0 || i >= (int)b->flows.size())
    return set_error(ALB_EINVAL, "alb_batch_flow: index %d out of range", i);
  *out = b->flows[i];
  return ALB_OK;
}

int alb_batch_step(alb_batch* b, int nsteps) {
  if (!b) return set_error(ALB_EINVAL, "alb_batch_step: null batch");
  if (nsteps < 0) return set_error(ALB_EINVAL, "alb_batch_step: nsteps < 0");
  for (alb_handle* h : b->flows)
    if (!h->initialised) return set_error(ALB_EINVAL, "alb_batch_step: a flow is not initialised");
  if (nsteps == 0) return ALB_OK;
  int rc = sync_cur(b);
  if (rc) return rc;
  if (nsteps >= 2 && b->dirty && (rc = build_graph(b)) != ALB_OK) return rc;
  for (int k = 0; k < nsteps / 2; ++k)
    ALB_CUDA(cudaGraphLaunch(b->exec, b->stream), "alb_batch_step: graph launch");
  if (nsteps & 1) {
    ALB_CUDA(step_all(b, 0), "alb_batch_step: step");
    for (int g = 0; g < 2; ++g)
      if (b->plan[g]->nflows()) ALB_CUDA(b->plan[g]->flip(b->stream), "alb_batch_step: flip");
    for (size_t f = 0; f < b->flows.size(); ++f) {
      b->flows[f]->dev.cur ^= 1;
      b->cur_seen[f] = b->flows[f]->dev.cur;
    }
  }
  for (alb_handle* h : b->flows) h->steps += (uint64_t)nsteps;
  return ALB_OK;
}

int alb_batch_sync(alb_batch* b, int timeout_ms) {
  if (!b) return set_error(ALB_EINVAL, "alb_batch_sync: null batch");
  int first = ALB_OK;
  for (alb_handle* h : b->flows) {
    const int rc = alb_sync(h, timeout_ms);
    if (rc == ALB_ETIMEDOUT || rc == ALB_ECUDA) return rc;
    if (rc != ALB_OK && first == ALB_OK) first = rc;
  }
  return first;
}

int alb_batch_get_tuning(alb_batch* b, int precision, alb_batch_tuning* t) {
  if (!b || !t) return set_error(ALB_EINVAL, "alb_batch_get_tuning: null pointer");
  if (precision != ALB_FP32_FORM && precision != ALB_FP64_PLAIN)
    return set_error(ALB_EINVAL, "alb_batch_get_tuning: unknown precision");
  from_tuning(b->plan[precision == ALB_FP32_FORM ? 1 : 0]->tuning(), t);
  return ALB_OK;
}

int alb_batch_set_tuning(alb_batch* b, int precision, const alb_batch_tuning* t) {
  if (!b || !t) return set_error(ALB_EINVAL, "alb_batch_set_tuning: null pointer");
  if (precision != ALB_FP32_FORM && precision != ALB_FP64_PLAIN)
    return set_error(ALB_EINVAL, "alb_batch_set_tuning: unknown precision");
  Tuning tt;
  to_tuning(t, &tt);
  if (const char* why = check_tuning(precision, tt))
    return set_error(ALB_EINVAL, "alb_batch_set_tuning: %s", why);
  ALB_CUDA(b->plan[precision == ALB_FP32_FORM ? 1 : 0]->set_tuning(tt, b->stream),
           "alb_batch_set_tuning");
  drop_graph(b);
  return ALB_OK;
}

// Coordinate search, per precision: the kernel variant (tiles as wide as
// possible), then the tile width of each size class present (timing only
// that class's items), then static against dynamic work distribution.
int alb_batch_tune(alb_batch* b, int trials) {
  if (!b) return set_error(ALB_EINVAL, "alb_batch_tune: null batch");
  if (trials < 1) return set_error(ALB_EINVAL, "alb_batch_tune: trials must be >= 1");
  for (alb_handle* h : b->flows)
    if (!h->initialised) return set_error(ALB_EINVAL, "alb_batch_tune: a flow is not initialised");
  int rc = sync_cur(b);
  if (rc) return rc;
  drop_graph(b);
  for (int g = 0; g < 2 && rc == ALB_OK; ++g)
    if (b->plan[g]->nflows()) rc = tune_group(b->plan[g], b->stream, b->d_counter + g, trials);
  return rc;
}
}  // extern "C"
