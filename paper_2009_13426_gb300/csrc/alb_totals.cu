// Global totals of the conserved moments (mass, momentum, total energy).
//
// Deterministic two-pass reduction: the grid is cut into fixed chunks of
// TOT_CHUNK nodes, one block per chunk; every block writes its four partial
// sums to a scratch array, and one block then adds the partials in index
// order. The result depends only on n, never on the launch configuration.

#include "alb_internal.h"

namespace alb {

// Conserved moments of node k from the primitive planes (rho, ux, uy, T).
template <typename P>
struct MomentPlanes {
  const P* mom;
  size_t ps;
  double cv;
  __device__ __forceinline__ void get(size_t k, double v[4]) const {
    const double r = (double)mom[k], ux = (double)mom[ps + k], uy = (double)mom[2 * ps + k],
                 T = (double)mom[3 * ps + k];
    v[0] = r;
    v[1] = r * ux;
    v[2] = r * uy;
    v[3] = 0.5 * r * (ux * ux + uy * uy) + r * cv * T;
  }
};

// Four conserved fields given by the caller as separate double arrays.
struct ConservedFields {
  const double *rho, *rhoux, *rhouy, *rhoE;
  __device__ __forceinline__ void get(size_t k, double v[4]) const {
    v[0] = rho[k];
    v[1] = rhoux[k];
    v[2] = rhouy[k];
    v[3] = rhoE[k];
  }
};

template <typename Src>
__global__ void __launch_bounds__(TOT_THREADS) totals_partial_kernel(Src src, long long n,
                                                                     double* partials) {
  __shared__ double sh[4][TOT_THREADS];
  const long long base = (long long)blockIdx.x * TOT_CHUNK;
  const long long end = base + TOT_CHUNK < n ? base + TOT_CHUNK : n;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (long long k = base + threadIdx.x; k < end; k += TOT_THREADS) {
    double v[4];
    src.get((size_t)k, v);
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[j] += v[j];
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) sh[j][threadIdx.x] = acc[j];
  __syncthreads();
  for (int s = TOT_THREADS / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s)
#pragma unroll
      for (int j = 0; j < 4; ++j) sh[j][threadIdx.x] += sh[j][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x < 4) partials[(size_t)blockIdx.x * 4 + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void __launch_bounds__(TOT_THREADS) totals_final_kernel(const double* partials,
                                                                   int nblocks, double* out) {
  __shared__ double sh[4][TOT_THREADS];
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < nblocks; b += TOT_THREADS)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[j] += partials[(size_t)b * 4 + j];
#pragma unroll
  for (int j = 0; j < 4; ++j) sh[j][threadIdx.x] = acc[j];
  __syncthreads();
  for (int s = TOT_THREADS / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s)
#pragma unroll
      for (int j = 0; j < 4; ++j) sh[j][threadIdx.x] += sh[j][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x < 4) out[threadIdx.x] = sh[threadIdx.x][0];
}

int totals_blocks(long long n) { return (int)((n + TOT_CHUNK - 1) / TOT_CHUNK); }

template <typename Src>
static cudaError_t launch_totals_src(const Src& src, long long n, double* partials, double* out,
                                     cudaStream_t s) {
  const int nb = totals_blocks(n);
  if (nb > 0) totals_partial_kernel<Src><<<nb, TOT_THREADS, 0, s>>>(src, n, partials);
  totals_final_kernel<<<1, TOT_THREADS, 0, s>>>(partials, nb, out);
  return cudaGetLastError();
}

cudaError_t launch_totals(const FlowDev& f, double* partials, double* out, cudaStream_t s) {
  if (f.precision == 0)
    return launch_totals_src(MomentPlanes<double>{(const double*)f.mom[f.cur], f.ps, f.prm.cv},
                             (long long)f.n, partials, out, s);
  return launch_totals_src(MomentPlanes<float>{(const float*)f.mom[f.cur], f.ps, f.prm.cv},
                           (long long)f.n, partials, out, s);
}

// ---------------------------------------------------------------------------
// Allocation-free totals for callers that cannot allocate device memory.
//
// The partial sums live in a file-scope device array instead of memory from
// cudaMalloc. Every GPU that loads this library holds the array until the
// process exits. In host code the array's name is only a host-side stand-in
// for the symbol, so its device address is looked up with cudaGetSymbolAddress
// (on the current device) and passed to the kernels. The lookup is repeated on
// every call: it is a host-side query, and an address kept from an earlier
// call would point at unmapped memory after a device reset reloads the module.

constexpr int NOALLOC_MAX_CHUNKS = 4096;  // up to 4096 * 65536 = 268,435,456 nodes

static __device__ __align__(256) double g_noalloc_partials[NOALLOC_MAX_CHUNKS * 4];

long long noalloc_max_nodes() { return (long long)NOALLOC_MAX_CHUNKS * TOT_CHUNK; }

// Device address of the scratch array on the current device.
static cudaError_t noalloc_scratch(double** out) {
  double* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress((void**)&p, g_noalloc_partials);
  if (e != cudaSuccess) return e;
  *out = p;
  return cudaSuccess;
}

cudaError_t launch_totals_noalloc(const double* rho, const double* rhoux, const double* rhouy,
                                  const double* rhoE, long long n, double* out, cudaStream_t s) {
  double* partials = nullptr;
  cudaError_t e = noalloc_scratch(&partials);
  if (e != cudaSuccess) return e;
  // Every partial the final pass reads is written by the partial pass of the
  // same call, so nothing left by an earlier call is ever read.
  return launch_totals_src(ConservedFields{rho, rhoux, rhouy, rhoE}, n, partials, out, s);
}

}  // namespace alb
