// Host-side internals shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

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
  CTR_COUNT = 8
};

// Device state of one flow: double-buffered population, lattice and moment
// planes. Plane p of buffer b starts at pop[b] + p * ps (elements).
struct FlowDev {
  Params prm;
  int precision;     // 0 FP64 plain, 1 FP32 form
  size_t n;          // nx * ny
  size_t ps;         // plane stride in elements (n rounded up to 64)
  void* pop[2];      // 42 planes of double or float
  void* mom[2];      // 4 planes (rho, ux, uy, T) of double or float
  uint8_t* lat[2];   // lattice code of the stored populations
  uint8_t* nxt[2];   // lattice code selected for the next pull
  float* lam[2];     // FP32 form: 8 planes of multipliers (warm start); else null
  unsigned long long* ctr;
  int cur;           // buffer holding the current state
};

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
                                 cudaStream_t s);
cudaError_t launch_equilibrium(const double* rho, const double* ubx, const double* uby,
                               const double* T, int n, double tol, int maxit, int precision,
                               double* feq, double* lambda, int* iters, int* status,
                               cudaStream_t s);
cudaError_t launch_exp_neg(const double* x, int n, double* out, cudaStream_t s);
cudaError_t launch_select(const double* rho, const double* rhou, int n, double n0, int umax,
                          signed char* out, cudaStream_t s);

}  // namespace alb
