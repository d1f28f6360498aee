// Host-side internals shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/alb.h"
#include "alb_device.cuh"

namespace alb {

// Device counters, one 64-bit slot each. Newton counts cover node and
// rebuild equilibria; they feed the arithmetic roofline of the step.
enum Counter {
  CTR_NEWTON_ITERS = 0,   // FP64 Newton steps (Jacobian + Cholesky + solve)
  CTR_NEWTON_FAIL = 1,    // node equilibria that failed
  CTR_REC = 2,            // rebuilt pulls
  CTR_REC_FAIL = 3,       // rebuilds that fell back
  CTR_UNREALIZABLE = 4,   // initial nodes with rho <= 0 or T <= 0
  CTR_NEWTON_CALLS = 5,   // equilibrium solves (node + rebuild)
  CTR_FP64_EVALS = 6,     // FP64 evaluations of the 21 exponentials
  CTR_FP32_ITERS = 7,     // FP32 Newton steps
  CTR_FP64_UPDATES = 8,   // multiplicative FP64 updates of the 21 populations
  CTR_COUNT = 9
};

// Device state of one flow: double-buffered population, lattice and moment
// planes. Plane p of buffer b starts at pop[b] + p * ps (elements).
struct FlowDev {
  Params prm;
  int precision;     // 0 FP64 plain, 1 FP32 form
  int q;             // velocities: 21 (D2Q21) or 49 (D2Q49 reference solver)
  int nplanes;       // population planes, 2 q
  size_t n;          // nx * ny
  size_t ps;         // plane stride in elements (n rounded up to 64)
  void* pop[2];      // nplanes planes of double or float
  void* mom[2];      // 4 planes (rho, ux, uy, T) of double or float
  uint8_t* lat[2];   // lattice code of the stored populations
  uint8_t* nxt[2];   // lattice code selected for the next pull
  void* lam[2];      // 8 planes of multipliers in the population precision (warm start)
  unsigned long long* ctr;
  int cur;           // buffer holding the current state
};

// Arguments of one step of one flow: read buffer `in`, write buffer in ^ 1.
template <typename P>
struct StepArgs {
  const P* pop_in;
  P* pop_out;
  const P* mom_in;
  P* mom_out;
  const uint8_t* lat_in;
  const uint8_t* nxt_in;
  uint8_t* lat_out;
  uint8_t* nxt_out;
  const P* lam_in;  // multipliers of the previous step (8 planes)
  P* lam_out;
  size_t ps;
  Params prm;
  unsigned long long* ctr;
};

template <typename P>
inline StepArgs<P> step_args(const FlowDev& f, int in) {
  const int out = in ^ 1;
  return StepArgs<P>{(const P*)f.pop[in], (P*)f.pop[out], (const P*)f.mom[in], (P*)f.mom[out],
                     f.lat[in], f.nxt[in], f.lat[out], f.nxt[out], (const P*)f.lam[in],
                     (P*)f.lam[out],
                     f.ps, f.prm, f.ctr};
}

// Global totals (alb_totals.cu): one block per chunk of TOT_CHUNK nodes writes
// 4 partial sums; a single block adds them in order.
constexpr int TOT_THREADS = 256;
constexpr long long TOT_CHUNK = 65536;
int totals_blocks(long long n);
cudaError_t launch_totals(const FlowDev& f, double* partials, double* out, cudaStream_t s);
// Same reduction over caller-owned conserved fields, with its partial sums in
// a file-scope device array (no allocation); n <= noalloc_max_nodes().
long long noalloc_max_nodes();
cudaError_t launch_totals_noalloc(const double* rho, const double* rhoux, const double* rhouy,
                                  const double* rhoE, long long n, double* out, cudaStream_t s);

// Kernel launchers (alb_kernels.cu). All enqueue on `s` and return the launch error.
cudaError_t launch_init(FlowDev& f, const double* rho, const double* rhoux, const double* rhouy,
                        const double* rhoE, cudaStream_t s);
cudaError_t launch_step(FlowDev& f, cudaStream_t s);
cudaError_t launch_export_moments(const FlowDev& f, double* rho, double* rhoux, double* rhouy,
                                  double* rhoE, cudaStream_t s);
cudaError_t launch_export_shifts(const FlowDev& f, signed char* ux, signed char* uy,
                                 cudaStream_t s, bool next = false);
// Planes [p0, p0 + np) of the current population (what = 0) or moment
// (what = 1) buffer as FP64 planes of n values.
cudaError_t launch_export_planes(const FlowDev& f, int what, int p0, int np, double* dst,
                                 cudaStream_t s);
cudaError_t launch_equilibrium(const double* rho, const double* ubx, const double* uby,
                               const double* T, int n, double tol, int maxit, int precision,
                               double* feq, double* lambda, int* iters, int* status,
                               cudaStream_t s);
cudaError_t launch_exp_neg(const double* x, int n, double* out, cudaStream_t s,
                           bool refine = false);
// D2Q49 reference solver (alb_q49.cu), FP64 only.
cudaError_t launch_init_q49(FlowDev& f, const double* rho, const double* rhoux,
                            const double* rhouy, const double* rhoE, cudaStream_t s);
cudaError_t launch_step_q49(FlowDev& f, cudaStream_t s);
cudaError_t launch_equilibrium13(const double* rho, const double* ubx, const double* uby,
                                 const double* T, int n, double tol, int maxit, double* feq,
                                 double* lambda, int* iters, int* status, cudaStream_t s);
cudaError_t launch_select(const double* rho, const double* rhou, int n, double n0, int umax,
                          signed char* out, cudaStream_t s);

// Batched step (alb_batch_f32.cu, alb_batch_f64.cu). A work item is a tile of
// 2^tw_log2 x (block >> tw_log2) nodes of flow `flow` with origin (x0, y0).
struct WorkItem {
  int flow, x0, y0, tw_log2;
};
// Compiled variants of the batched kernel per precision.
struct BatchVariant {
  int block, min_blocks;
};
int batch_variant_count(int precision);
BatchVariant batch_variant(int precision, int v);
cudaError_t launch_flip(int* cur, int n, cudaStream_t s);

// Error reporting of the C ABI (alb_api.cu): sets the thread's message and
// returns code.
int set_error(int code, const char* fmt, ...);
int cuda_error(cudaError_t e, const char* what);

}  // namespace alb

// State behind an alb_handle (alb_api.cu). A handle that belongs to a batch or
// a server (owner != null) is destroyed with its owner.
struct alb_handle {
  alb_config cfg;
  alb::FlowDev dev;
  cudaStream_t stream;
  bool own_stream;
  double* staging;        // 4 * n doubles for host transfers
  double* tot_partials;   // 4 doubles per chunk of the totals reduction
  double* tot_out;        // 4 doubles, device result of the totals reduction
  unsigned long long* ctr_host;
  double* tot_host;       // pinned copy of tot_out
  uint64_t steps;
  bool initialised;
  const void* owner;
};

namespace alb {
// Frees a handle whatever its owner (alb_api.cu).
int handle_destroy(alb_handle* h);
// Validation of alb_create (ALB_OK or an error code with the message set).
int config_check(const alb_config* c);
// Device bytes alb_create allocates for a flow of this configuration.
size_t flow_device_bytes(const alb_config* c);
}  // namespace alb
