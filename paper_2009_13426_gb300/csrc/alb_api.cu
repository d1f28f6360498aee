// C ABI of the single-flow path (include/alb.h): configuration checks, device
// allocation, stream handling, host/device staging, error reporting.
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <thread>

#include "alb_internal.h"

using namespace alb;

namespace {

thread_local char g_err[512] = "";

int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(ALB_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define ALB_CUDA(call, what)                      \
  do {                                            \
    cudaError_t e_ = (call);                      \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

}  // namespace

namespace alb {

int set_error(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

int cuda_error(cudaError_t e, const char* what) { return cuda_fail(e, what); }

int handle_destroy(alb_handle* h) {
  if (!h) return ALB_OK;
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (int b = 0; b < 2; ++b) {
    cudaFree(h->dev.pop[b]);
    cudaFree(h->dev.mom[b]);
    cudaFree(h->dev.lat[b]);
    cudaFree(h->dev.nxt[b]);
    cudaFree(h->dev.lam[b]);
  }
  cudaFree(h->dev.ctr);
  cudaFree(h->staging);
  cudaFree(h->tot_partials);
  cudaFree(h->tot_out);
  cudaFreeHost(h->ctr_host);
  cudaFreeHost(h->tot_host);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
  return ALB_OK;
}

}  // namespace alb

extern "C" {

const char* alb_last_error(void) { return g_err; }

int alb_velocities(int* xi_x, int* xi_y) {
  if (!xi_x || !xi_y) return fail(ALB_EINVAL, "alb_velocities: null pointer");
  for (int i = 0; i < Q; ++i) {
    xi_x[i] = XI_X(i);
    xi_y[i] = XI_Y(i);
  }
  return ALB_OK;
}

int alb_stencil_velocities(int stencil, int* xi_x, int* xi_y) {
  if (!xi_x || !xi_y) return fail(ALB_EINVAL, "alb_stencil_velocities: null pointer");
  if (stencil == ALB_D2Q21) return alb_velocities(xi_x, xi_y);
  if (stencil != ALB_D2Q49) return fail(ALB_EUNSUPPORTED, "unknown stencil %d", stencil);
  for (int i = 0; i < 49; ++i) {
    xi_x[i] = i % 7 - 3;
    xi_y[i] = i / 7 - 3;
  }
  return ALB_OK;
}

int alb_config_default(alb_config* c) {
  if (!c) return fail(ALB_EINVAL, "alb_config_default: null pointer");
  memset(c, 0, sizeof(*c));
  c->nx = 64;
  c->ny = 64;
  c->stencil = ALB_D2Q21;
  c->u_max = 2;
  c->nu = 1e-3;
  c->gamma = 1.4;
  c->n0 = 0.5;
  c->precision = ALB_FP64_PLAIN;
  c->bc_x = ALB_PERIODIC;
  c->bc_y = ALB_PERIODIC;
  c->sensor = 0;
  c->sensor_eps[0] = 0.01;
  c->sensor_eps[1] = 0.1;
  c->sensor_eps[2] = 1.0;
  c->sensor_alpha[0] = 1.05;
  c->sensor_alpha[1] = 1.35;
  c->sensor_alpha[2] = 1.6;
  c->newton_tol = 1e-12;
  c->newton_maxit = 50;
  c->newton_start = ALB_START_AUTO;
  c->shift_overlap = 0.0;
  c->shift_rule = ALB_RULE_HISTORY;
  c->moments = 8;
  c->prandtl = 1.0;
  c->stream = nullptr;
  return ALB_OK;
}

// Whether the solves of this configuration start from the stored multipliers.
static bool uses_previous_start(const alb_config* c) {
  return c->newton_start == ALB_START_PREVIOUS ||
         (c->newton_start == ALB_START_AUTO && c->precision == ALB_FP32_FORM);
}

static int check_config(const alb_config* c) {
  if (!c) return fail(ALB_EINVAL, "null config");
  if (c->stencil != ALB_D2Q21 && c->stencil != ALB_D2Q49)
    return fail(ALB_EUNSUPPORTED, "stencil must be ALB_D2Q21 or ALB_D2Q49");
  if (c->nx < 1 || c->ny < 1) return fail(ALB_EINVAL, "grid %d x %d is empty", c->nx, c->ny);
  if ((long long)c->nx * c->ny > (1LL << 31)) return fail(ALB_EINVAL, "grid too large");
  if (c->ny > 65535) return fail(ALB_EINVAL, "ny must be <= 65535");
  if (c->u_max < 0 || c->u_max > 3) return fail(ALB_EINVAL, "u_max must be in [0, 3]");
  if (!(c->nu >= 0.0)) return fail(ALB_EINVAL, "nu must be >= 0");
  if (!(c->gamma > 1.0)) return fail(ALB_EINVAL, "gamma must be > 1");
  if (!(c->n0 > 0.0 && c->n0 < 1.0)) return fail(ALB_EINVAL, "n0 must be in (0, 1)");
  if (c->precision != ALB_FP64_PLAIN && c->precision != ALB_FP32_FORM)
    return fail(ALB_EINVAL, "unknown precision %d", c->precision);
  if ((c->bc_x != ALB_PERIODIC && c->bc_x != ALB_ZERO_GRADIENT) ||
      (c->bc_y != ALB_PERIODIC && c->bc_y != ALB_ZERO_GRADIENT))
    return fail(ALB_EINVAL, "unknown boundary kind");
  if (c->sensor && !(c->sensor_eps[0] > 0.0 && c->sensor_eps[0] < c->sensor_eps[1] &&
                     c->sensor_eps[1] < c->sensor_eps[2]))
    return fail(ALB_EINVAL, "sensor_eps must be positive and increasing");
  if (!(c->newton_tol > 0.0) || c->newton_maxit < 1)
    return fail(ALB_EINVAL, "newton_tol must be > 0 and newton_maxit >= 1");
  if (c->newton_start != ALB_START_AUTO && c->newton_start != ALB_START_MAXWELLIAN &&
      c->newton_start != ALB_START_PREVIOUS)
    return fail(ALB_EINVAL, "unknown newton_start %d", c->newton_start);
  if (!(c->shift_overlap >= 0.0 && c->shift_overlap <= 1.0))
    return fail(ALB_EINVAL, "shift_overlap must be in [0, 1]");
  if (c->shift_rule != ALB_RULE_HISTORY && c->shift_rule != ALB_RULE_NEIGHBOURS)
    return fail(ALB_EINVAL, "unknown shift_rule %d", c->shift_rule);
  if (c->stencil == ALB_D2Q21 && c->moments != 8 && c->moments != 4)
    return fail(ALB_EINVAL, "moments must be 8 or 4 on D2Q21");
  if (c->stencil == ALB_D2Q49) {
    if (c->moments != 13) return fail(ALB_EINVAL, "moments must be 13 on D2Q49");
    if (c->precision != ALB_FP64_PLAIN)
      return fail(ALB_EUNSUPPORTED, "D2Q49 runs in ALB_FP64_PLAIN only");
    if (c->newton_start == ALB_START_PREVIOUS)
      return fail(ALB_EUNSUPPORTED, "D2Q49 solves start from the Maxwellian");
  }
  if (!(c->prandtl > 0.0 && c->prandtl < 1e300)) return fail(ALB_EINVAL, "prandtl must be > 0");
  return ALB_OK;
}

int alb_destroy(alb_handle* h) {
  if (!h) return ALB_OK;
  if (h->owner) return fail(ALB_EINVAL, "alb_destroy: the handle belongs to a batch or server");
  return handle_destroy(h);
}

int alb_create(const alb_config* cfg, alb_handle** out) {
  if (!out) return fail(ALB_EINVAL, "alb_create: null output");
  *out = nullptr;
  int rc = check_config(cfg);
  if (rc) return rc;
  alb_handle* h = new (std::nothrow) alb_handle();
  if (!h) return fail(ALB_ENOMEM, "host allocation failed");
  h->cfg = *cfg;
  FlowDev& d = h->dev;
  Params& p = d.prm;
  p.nx = cfg->nx;
  p.ny = cfg->ny;
  p.umax = cfg->u_max;
  p.bcx = cfg->bc_x;
  p.bcy = cfg->bc_y;
  p.sensor = cfg->sensor;
  p.maxit = cfg->newton_maxit;
  p.warm = uses_previous_start(cfg) ? 1 : 0;
  p.overlap = cfg->shift_overlap;
  p.rule = cfg->shift_rule;
  p.moments = cfg->moments;
  p.nu = cfg->nu;
  p.gamma = cfg->gamma;
  p.n0 = cfg->n0;
  p.tol = cfg->newton_tol;
  p.cv = 1.0 / (cfg->gamma - 1.0);
  p.cp = cfg->gamma * p.cv;
  p.half_gm1 = 0.5 * (cfg->gamma - 1.0);
  p.shakhov = cfg->prandtl != 1.0 ? 1 : 0;
  p.prandtl = cfg->prandtl;
  for (int j = 0; j < 3; ++j) {
    p.seps[j] = cfg->sensor_eps[j];
    p.salpha[j] = cfg->sensor_alpha[j];
  }
  p.skx[0] = log10(cfg->sensor_eps[0]);
  p.skx[1] = log10(cfg->sensor_eps[1]);
  p.skx[2] = log10(cfg->sensor_eps[2]);
  p.skx[3] = p.skx[2] + 1.0;
  p.sky[0] = 1.0;
  p.sky[1] = cfg->sensor_alpha[0];
  p.sky[2] = cfg->sensor_alpha[1];
  p.sky[3] = cfg->sensor_alpha[2];
  for (int t = 0; t < 6; ++t) p.thr[t] = (double)(t - cfg->u_max + 1) - cfg->n0;
  for (int j = 0; j < 7; ++j) {
    p.wlo[j] = ((double)(j - 3) - cfg->n0) - cfg->shift_overlap;
    p.whi[j] = ((double)(j - 2) - cfg->n0) + cfg->shift_overlap;
  }
  d.precision = cfg->precision;
  d.q = cfg->stencil == ALB_D2Q49 ? 49 : Q;
  d.nplanes = 2 * d.q;
  d.n = (size_t)cfg->nx * cfg->ny;
  d.ps = (d.n + 63) / 64 * 64;
  d.cur = 0;
  const size_t es = d.precision == ALB_FP64_PLAIN ? sizeof(double) : sizeof(float);
  if (cfg->stream) {
    h->stream = (cudaStream_t)cfg->stream;
    h->own_stream = false;
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete h;
      return cuda_fail(e, "cudaStreamCreate");
    }
    h->own_stream = true;
  }
#define ALLOC(ptr, bytes)                                              \
  do {                                                                 \
    cudaError_t e_ = cudaMalloc((void**)&(ptr), (bytes));              \
    if (e_ != cudaSuccess) {                                           \
      handle_destroy(h);                                               \
      cudaGetLastError();                                              \
      return fail(ALB_ENOMEM, "cudaMalloc of %zu bytes failed: %s", (size_t)(bytes), \
                  cudaGetErrorString(e_));                             \
    }                                                                  \
  } while (0)
  for (int b = 0; b < 2; ++b) {
    ALLOC(d.pop[b], (size_t)d.nplanes * d.ps * es);
    ALLOC(d.mom[b], 4 * d.ps * es);
    ALLOC(d.lat[b], d.ps);
    ALLOC(d.nxt[b], d.ps);
    if (p.warm) ALLOC(d.lam[b], NM * d.ps * es);
  }
  ALLOC(d.ctr, CTR_COUNT * sizeof(unsigned long long));
  ALLOC(h->staging, 4 * d.n * sizeof(double));
  ALLOC(h->tot_partials, (size_t)(totals_blocks((long long)d.n) + 1) * 4 * sizeof(double));
  ALLOC(h->tot_out, 4 * sizeof(double));
#undef ALLOC
  if (cudaMallocHost((void**)&h->ctr_host, CTR_COUNT * sizeof(unsigned long long)) != cudaSuccess ||
      cudaMallocHost((void**)&h->tot_host, 4 * sizeof(double)) != cudaSuccess) {
    handle_destroy(h);
    return fail(ALB_ENOMEM, "pinned host allocation failed");
  }
  *out = h;
  return ALB_OK;
}

int alb_init(alb_handle* h, const double* rho, const double* rhoux, const double* rhouy,
             const double* rhoE, int where) {
  if (!h || !rho || !rhoux || !rhouy || !rhoE) return fail(ALB_EINVAL, "alb_init: null pointer");
  const size_t n = h->dev.n;
  const double *r = rho, *a = rhoux, *b = rhouy, *e = rhoE;
  ALB_CUDA(cudaMemsetAsync(h->dev.ctr, 0, CTR_COUNT * sizeof(unsigned long long), h->stream),
           "alb_init: counter reset");
  if (where == ALB_HOST) {
    double* s = h->staging;
    ALB_CUDA(cudaMemcpyAsync(s, rho, n * sizeof(double), cudaMemcpyHostToDevice, h->stream), "H2D");
    ALB_CUDA(cudaMemcpyAsync(s + n, rhoux, n * sizeof(double), cudaMemcpyHostToDevice, h->stream),
             "H2D");
    ALB_CUDA(cudaMemcpyAsync(s + 2 * n, rhouy, n * sizeof(double), cudaMemcpyHostToDevice,
                             h->stream), "H2D");
    ALB_CUDA(cudaMemcpyAsync(s + 3 * n, rhoE, n * sizeof(double), cudaMemcpyHostToDevice,
                             h->stream), "H2D");
    r = s; a = s + n; b = s + 2 * n; e = s + 3 * n;
  } else if (where != ALB_DEVICE) {
    return fail(ALB_EINVAL, "alb_init: where must be ALB_HOST or ALB_DEVICE");
  }
  h->dev.cur = 0;
  ALB_CUDA(launch_init(h->dev, r, a, b, e, h->stream), "alb_init: init kernel");
  ALB_CUDA(cudaMemcpyAsync(h->ctr_host, h->dev.ctr, CTR_COUNT * sizeof(unsigned long long),
                           cudaMemcpyDeviceToHost, h->stream), "alb_init: counters");
  ALB_CUDA(cudaStreamSynchronize(h->stream), "alb_init: synchronise");
  h->steps = 0;
  h->initialised = true;
  if (h->ctr_host[CTR_UNREALIZABLE])
    return fail(ALB_EUNREALIZABLE, "alb_init: %llu nodes with rho <= 0 or T <= 0",
                h->ctr_host[CTR_UNREALIZABLE]);
  if (h->ctr_host[CTR_NEWTON_FAIL])
    return fail(ALB_ENEWTON, "alb_init: %llu nodes without a converged equilibrium",
                h->ctr_host[CTR_NEWTON_FAIL]);
  return ALB_OK;
}

int alb_step(alb_handle* h, int nsteps) {
  if (!h) return fail(ALB_EINVAL, "alb_step: null handle");
  if (!h->initialised) return fail(ALB_EINVAL, "alb_step: call alb_init first");
  if (nsteps < 0) return fail(ALB_EINVAL, "alb_step: nsteps < 0");
  for (int s = 0; s < nsteps; ++s)
    ALB_CUDA(launch_step(h->dev, h->stream), "alb_step: step kernel");
  h->steps += (uint64_t)nsteps;
  return ALB_OK;
}

int alb_sync(alb_handle* h, int timeout_ms) {
  if (!h) return fail(ALB_EINVAL, "alb_sync: null handle");
  ALB_CUDA(cudaMemcpyAsync(h->ctr_host, h->dev.ctr, CTR_COUNT * sizeof(unsigned long long),
                           cudaMemcpyDeviceToHost, h->stream), "alb_sync: counters");
  if (timeout_ms < 0) {
    ALB_CUDA(cudaStreamSynchronize(h->stream), "alb_sync");
  } else {
    auto t0 = std::chrono::steady_clock::now();
    for (;;) {
      cudaError_t e = cudaStreamQuery(h->stream);
      if (e == cudaSuccess) break;
      if (e != cudaErrorNotReady) return cuda_fail(e, "alb_sync");
      auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(
                    std::chrono::steady_clock::now() - t0).count();
      if (ms >= timeout_ms) return fail(ALB_ETIMEDOUT, "alb_sync: still running after %d ms", timeout_ms);
      std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
  }
  if (h->ctr_host[CTR_NEWTON_FAIL] || h->ctr_host[CTR_REC_FAIL])
    return fail(ALB_ENEWTON, "%llu node equilibria and %llu rebuilds failed",
                h->ctr_host[CTR_NEWTON_FAIL], h->ctr_host[CTR_REC_FAIL]);
  return ALB_OK;
}

int alb_moments(alb_handle* h, double* rho, double* rhoux, double* rhouy, double* rhoE,
                int where) {
  if (!h || !rho || !rhoux || !rhouy || !rhoE) return fail(ALB_EINVAL, "alb_moments: null pointer");
  if (!h->initialised) return fail(ALB_EINVAL, "alb_moments: call alb_init first");
  const size_t n = h->dev.n;
  if (where == ALB_DEVICE) {
    ALB_CUDA(launch_export_moments(h->dev, rho, rhoux, rhouy, rhoE, h->stream), "alb_moments");
    return ALB_OK;
  }
  if (where != ALB_HOST) return fail(ALB_EINVAL, "alb_moments: bad where");
  double* s = h->staging;
  ALB_CUDA(launch_export_moments(h->dev, s, s + n, s + 2 * n, s + 3 * n, h->stream), "alb_moments");
  double* outs[4] = {rho, rhoux, rhouy, rhoE};
  for (int j = 0; j < 4; ++j)
    ALB_CUDA(cudaMemcpyAsync(outs[j], s + j * n, n * sizeof(double), cudaMemcpyDeviceToHost,
                             h->stream), "alb_moments: D2H");
  ALB_CUDA(cudaStreamSynchronize(h->stream), "alb_moments: synchronise");
  return ALB_OK;
}

int alb_shifts(alb_handle* h, signed char* ux, signed char* uy, int where) {
  if (!h || !ux || !uy) return fail(ALB_EINVAL, "alb_shifts: null pointer");
  if (!h->initialised) return fail(ALB_EINVAL, "alb_shifts: call alb_init first");
  const size_t n = h->dev.n;
  if (where == ALB_DEVICE) {
    ALB_CUDA(launch_export_shifts(h->dev, ux, uy, h->stream), "alb_shifts");
    return ALB_OK;
  }
  if (where != ALB_HOST) return fail(ALB_EINVAL, "alb_shifts: bad where");
  signed char* s = (signed char*)h->staging;
  ALB_CUDA(launch_export_shifts(h->dev, s, s + n, h->stream), "alb_shifts");
  ALB_CUDA(cudaMemcpyAsync(ux, s, n, cudaMemcpyDeviceToHost, h->stream), "alb_shifts: D2H");
  ALB_CUDA(cudaMemcpyAsync(uy, s + n, n, cudaMemcpyDeviceToHost, h->stream), "alb_shifts: D2H");
  ALB_CUDA(cudaStreamSynchronize(h->stream), "alb_shifts: synchronise");
  return ALB_OK;
}

int alb_next_shifts(alb_handle* h, signed char* ux, signed char* uy, int where) {
  if (!h || !ux || !uy) return fail(ALB_EINVAL, "alb_next_shifts: null pointer");
  if (!h->initialised) return fail(ALB_EINVAL, "alb_next_shifts: call alb_init first");
  const size_t n = h->dev.n;
  if (where == ALB_DEVICE) {
    ALB_CUDA(launch_export_shifts(h->dev, ux, uy, h->stream, true), "alb_next_shifts");
    return ALB_OK;
  }
  if (where != ALB_HOST) return fail(ALB_EINVAL, "alb_next_shifts: bad where");
  signed char* s = (signed char*)h->staging;
  ALB_CUDA(launch_export_shifts(h->dev, s, s + n, h->stream, true), "alb_next_shifts");
  ALB_CUDA(cudaMemcpyAsync(ux, s, n, cudaMemcpyDeviceToHost, h->stream), "alb_next_shifts: D2H");
  ALB_CUDA(cudaMemcpyAsync(uy, s + n, n, cudaMemcpyDeviceToHost, h->stream),
           "alb_next_shifts: D2H");
  ALB_CUDA(cudaStreamSynchronize(h->stream), "alb_next_shifts: synchronise");
  return ALB_OK;
}

// Planes of the current buffer as FP64 planes: what = 0 populations (outs[0]
// receives planes 0..20, outs[1] planes 21..41), what = 1 moments (outs[j]
// receives plane j).
static int export_planes(alb_handle* h, int what, double* const* outs, int nout, int per_out,
                         int where, const char* name) {
  const size_t n = h->dev.n;
  if (where == ALB_DEVICE) {
    for (int j = 0; j < nout; ++j)
      ALB_CUDA(launch_export_planes(h->dev, what, j * per_out, per_out, outs[j], h->stream), name);
    return ALB_OK;
  }
  if (where != ALB_HOST) return fail(ALB_EINVAL, "%s: bad where", name);
  // through the staging buffer (4 planes of n doubles at a time)
  double* st = h->staging;
  for (int j = 0; j < nout; ++j)
    for (int p = 0; p < per_out; p += 4) {
      const int np = per_out - p < 4 ? per_out - p : 4;
      ALB_CUDA(launch_export_planes(h->dev, what, j * per_out + p, np, st, h->stream), name);
      ALB_CUDA(cudaMemcpyAsync(outs[j] + (size_t)p * n, st, (size_t)np * n * sizeof(double),
                               cudaMemcpyDeviceToHost, h->stream), name);
      ALB_CUDA(cudaStreamSynchronize(h->stream), name);
    }
  return ALB_OK;
}

int alb_populations(alb_handle* h, double* f, double* g, int where) {
  if (!h || !f || !g) return fail(ALB_EINVAL, "alb_populations: null pointer");
  if (!h->initialised) return fail(ALB_EINVAL, "alb_populations: call alb_init first");
  double* outs[2] = {f, g};
  return export_planes(h, 0, outs, 2, h->dev.q, where, "alb_populations");
}

int alb_primitives(alb_handle* h, double* rho, double* ux, double* uy, double* T, int where) {
  if (!h || !rho || !ux || !uy || !T) return fail(ALB_EINVAL, "alb_primitives: null pointer");
  if (!h->initialised) return fail(ALB_EINVAL, "alb_primitives: call alb_init first");
  double* outs[4] = {rho, ux, uy, T};
  return export_planes(h, 1, outs, 4, 1, where, "alb_primitives");
}

// ------------------------------------------------------------- checkpoints

struct CheckpointHeader {
  char magic[8];          // "ALBCKPT1"
  int32_t nx, ny, precision, warm;
  int32_t u_max, bc_x, bc_y, q;  // q: velocities per node (0 read as 21)
  uint64_t ps, steps;
};

struct Piece {
  void* dev;
  size_t bytes;
};

static int checkpoint_pieces(alb_handle* h, Piece* out) {
  const FlowDev& d = h->dev;
  const size_t es = d.precision == ALB_FP64_PLAIN ? sizeof(double) : sizeof(float);
  const int b = d.cur;
  int k = 0;
  out[k++] = {d.pop[b], (size_t)d.nplanes * d.ps * es};
  out[k++] = {d.mom[b], 4 * d.ps * es};
  out[k++] = {d.lat[b], d.ps};
  out[k++] = {d.nxt[b], d.ps};
  if (d.prm.warm) out[k++] = {d.lam[b], NM * d.ps * es};
  out[k++] = {d.ctr, CTR_COUNT * sizeof(unsigned long long)};
  return k;
}

int alb_checkpoint_size(alb_handle* h, size_t* bytes) {
  if (!h || !bytes) return fail(ALB_EINVAL, "alb_checkpoint_size: null pointer");
  Piece pc[6];
  const int k = checkpoint_pieces(h, pc);
  size_t total = sizeof(CheckpointHeader);
  for (int j = 0; j < k; ++j) total += pc[j].bytes;
  *bytes = total;
  return ALB_OK;
}

int alb_checkpoint_save(alb_handle* h, void* buf) {
  if (!h || !buf) return fail(ALB_EINVAL, "alb_checkpoint_save: null pointer");
  if (!h->initialised) return fail(ALB_EINVAL, "alb_checkpoint_save: call alb_init first");
  CheckpointHeader hd;
  memset(&hd, 0, sizeof(hd));
  memcpy(hd.magic, "ALBCKPT1", 8);
  hd.nx = h->cfg.nx;
  hd.ny = h->cfg.ny;
  hd.precision = h->dev.precision;
  hd.warm = h->dev.prm.warm;
  hd.u_max = h->cfg.u_max;
  hd.bc_x = h->cfg.bc_x;
  hd.bc_y = h->cfg.bc_y;
  hd.q = h->dev.q;
  hd.ps = h->dev.ps;
  hd.steps = h->steps;
  unsigned char* p = (unsigned char*)buf;
  memcpy(p, &hd, sizeof(hd));
  p += sizeof(hd);
  Piece pc[6];
  const int k = checkpoint_pieces(h, pc);
  for (int j = 0; j < k; ++j) {
    ALB_CUDA(cudaMemcpyAsync(p, pc[j].dev, pc[j].bytes, cudaMemcpyDeviceToHost, h->stream),
             "alb_checkpoint_save: D2H");
    p += pc[j].bytes;
  }
  ALB_CUDA(cudaStreamSynchronize(h->stream), "alb_checkpoint_save: synchronise");
  return ALB_OK;
}

int alb_checkpoint_load(alb_handle* h, const void* buf) {
  if (!h || !buf) return fail(ALB_EINVAL, "alb_checkpoint_load: null pointer");
  CheckpointHeader hd;
  memcpy(&hd, buf, sizeof(hd));
  if (memcmp(hd.magic, "ALBCKPT1", 8) != 0)
    return fail(ALB_EINVAL, "alb_checkpoint_load: not a checkpoint of this library");
  if (hd.nx != h->cfg.nx || hd.ny != h->cfg.ny || hd.precision != h->dev.precision ||
      hd.warm != h->dev.prm.warm || hd.u_max != h->cfg.u_max || hd.bc_x != h->cfg.bc_x ||
      hd.bc_y != h->cfg.bc_y || hd.ps != h->dev.ps || (hd.q ? hd.q : Q) != h->dev.q)
    return fail(ALB_EINVAL, "alb_checkpoint_load: checkpoint of another configuration");
  ALB_CUDA(cudaStreamSynchronize(h->stream), "alb_checkpoint_load: synchronise");
  const unsigned char* p = (const unsigned char*)buf + sizeof(hd);
  Piece pc[6];
  const int k = checkpoint_pieces(h, pc);
  for (int j = 0; j < k; ++j) {
    ALB_CUDA(cudaMemcpyAsync(pc[j].dev, p, pc[j].bytes, cudaMemcpyHostToDevice, h->stream),
             "alb_checkpoint_load: H2D");
    p += pc[j].bytes;
  }
  ALB_CUDA(cudaStreamSynchronize(h->stream), "alb_checkpoint_load: synchronise");
  h->steps = hd.steps;
  h->initialised = true;
  return ALB_OK;
}

int alb_totals(alb_handle* h, double* out) {
  if (!h || !out) return fail(ALB_EINVAL, "alb_totals: null pointer");
  if (!h->initialised) return fail(ALB_EINVAL, "alb_totals: call alb_init first");
  ALB_CUDA(launch_totals(h->dev, h->tot_partials, h->tot_out, h->stream), "alb_totals");
  ALB_CUDA(cudaMemcpyAsync(h->tot_host, h->tot_out, 4 * sizeof(double), cudaMemcpyDeviceToHost,
                           h->stream), "alb_totals: D2H");
  ALB_CUDA(cudaStreamSynchronize(h->stream), "alb_totals: synchronise");
  for (int j = 0; j < 4; ++j) out[j] = h->tot_host[j];
  return ALB_OK;
}

// For callers that cannot allocate device memory: the totals of caller-owned
// conserved fields, with the partial sums in a static device array. The first
// call on a device looks the array's address up (with that device current);
// make that first call before any stream capture. Calls that overlap on the
// GPU share the array and race.
int alb_totals_noalloc(const double* rho, const double* rhoux, const double* rhouy,
                       const double* rhoE, long long n, double* out, void* stream) {
  if (n < 0 || !out || (n > 0 && (!rho || !rhoux || !rhouy || !rhoE)))
    return fail(ALB_EINVAL, "alb_totals_noalloc: bad arguments");
  if (n > noalloc_max_nodes())
    return fail(ALB_EINVAL,
                "alb_totals_noalloc: n = %lld exceeds the %lld nodes its static scratch holds",
                n, noalloc_max_nodes());
  ALB_CUDA(launch_totals_noalloc(rho, rhoux, rhouy, rhoE, n, out, (cudaStream_t)stream),
           "alb_totals_noalloc");
  return ALB_OK;
}

int alb_stats_get(alb_handle* h, alb_stats* out) {
  if (!h || !out) return fail(ALB_EINVAL, "alb_stats_get: null pointer");
  ALB_CUDA(cudaMemcpyAsync(h->ctr_host, h->dev.ctr, CTR_COUNT * sizeof(unsigned long long),
                           cudaMemcpyDeviceToHost, h->stream), "alb_stats_get");
  ALB_CUDA(cudaStreamSynchronize(h->stream), "alb_stats_get: synchronise");
  out->steps = h->steps;
  out->node_updates = h->steps * (uint64_t)h->dev.n;
  out->newton_iterations = h->ctr_host[CTR_NEWTON_ITERS];
  out->newton_failures = h->ctr_host[CTR_NEWTON_FAIL];
  out->reconstructions = h->ctr_host[CTR_REC];
  out->reconstruction_failures = h->ctr_host[CTR_REC_FAIL];
  out->newton_calls = h->ctr_host[CTR_NEWTON_CALLS];
  out->fp64_evaluations = h->ctr_host[CTR_FP64_EVALS];
  out->fp32_iterations = h->ctr_host[CTR_FP32_ITERS];
  out->fp64_updates = h->ctr_host[CTR_FP64_UPDATES];
  return ALB_OK;
}

int alb_equilibrium(const double* rho, const double* ubx, const double* uby, const double* T,
                    int n, double tol, int maxit, int precision, double* feq, double* lambda,
                    int* iters, int* status, void* stream) {
  if (n < 0 || (n > 0 && (!rho || !ubx || !uby || !T || !feq)))
    return fail(ALB_EINVAL, "alb_equilibrium: bad arguments");
  if (!(tol > 0.0) || maxit < 1) return fail(ALB_EINVAL, "alb_equilibrium: bad tolerance");
  if (precision != ALB_FP64_PLAIN && precision != ALB_FP32_FORM)
    return fail(ALB_EINVAL, "alb_equilibrium: unknown precision %d", precision);
  ALB_CUDA(launch_equilibrium(rho, ubx, uby, T, n, tol, maxit, precision, feq, lambda, iters,
                              status, (cudaStream_t)stream), "alb_equilibrium");
  return ALB_OK;
}

int alb_equilibrium13(const double* rho, const double* ubx, const double* uby, const double* T,
                      int n, double tol, int maxit, double* feq, double* lambda, int* iters,
                      int* status, void* stream) {
  if (n < 0 || (n > 0 && (!rho || !ubx || !uby || !T || !feq || !lambda || !iters || !status)))
    return fail(ALB_EINVAL, "alb_equilibrium13: bad arguments");
  if (!(tol > 0.0) || maxit < 1) return fail(ALB_EINVAL, "alb_equilibrium13: bad tolerance");
  ALB_CUDA(launch_equilibrium13(rho, ubx, uby, T, n, tol, maxit, feq, lambda, iters, status,
                                (cudaStream_t)stream), "alb_equilibrium13");
  return ALB_OK;
}

int alb_exp_neg_refine(const double* s, int n, double* out, void* stream) {
  if (n < 0 || (n > 0 && (!s || !out)))
    return fail(ALB_EINVAL, "alb_exp_neg_refine: bad arguments");
  ALB_CUDA(launch_exp_neg(s, n, out, (cudaStream_t)stream, true), "alb_exp_neg_refine");
  return ALB_OK;
}

int alb_exp_neg(const double* s, int n, double* out, void* stream) {
  if (n < 0 || (n > 0 && (!s || !out))) return fail(ALB_EINVAL, "alb_exp_neg: bad arguments");
  ALB_CUDA(launch_exp_neg(s, n, out, (cudaStream_t)stream), "alb_exp_neg");
  return ALB_OK;
}

int alb_select_shift(const double* rho, const double* rhou, int n, double n0, int u_max,
                     signed char* out, void* stream) {
  if (n < 0 || (n > 0 && (!rho || !rhou || !out)))
    return fail(ALB_EINVAL, "alb_select_shift: bad arguments");
  if (u_max < 0 || u_max > 3 || !(n0 > 0.0 && n0 < 1.0))
    return fail(ALB_EINVAL, "alb_select_shift: bad u_max or n0");
  ALB_CUDA(launch_select(rho, rhou, n, n0, u_max, out, (cudaStream_t)stream), "alb_select_shift");
  return ALB_OK;
}

}  // extern "C"

namespace alb {

int config_check(const alb_config* c) { return check_config(c); }

// Device bytes alb_create allocates for a flow (the same sizes as there).
size_t flow_device_bytes(const alb_config* c) {
  const size_t n = (size_t)c->nx * c->ny, ps = (n + 63) / 64 * 64;
  const size_t es = c->precision == ALB_FP64_PLAIN ? sizeof(double) : sizeof(float);
  const size_t np = c->stencil == ALB_D2Q49 ? 98 : NPLANES;
  size_t b = 2 * (np * ps * es + 4 * ps * es + 2 * ps);
  if (uses_previous_start(c)) b += 2 * NM * ps * es;
  b += CTR_COUNT * sizeof(unsigned long long) + 4 * n * sizeof(double) +
       (size_t)(totals_blocks((long long)n) + 1) * 4 * sizeof(double) + 4 * sizeof(double);
  return b;
}

}  // namespace alb
