// Batched step kernels of the FP64 plain path: the compiled (block, minimum
// resident blocks) variants the autotuner chooses from.
#include "alb_batch_kernel.cuh"
#include "alb_batcher.h"

namespace alb {

namespace {
using K0 = BatchKernel<double, 128, 1>;
using K1 = BatchKernel<double, 64, 2>;
constexpr BatchVariant kF64[] = {{128, 1}, {64, 2}};
}  // namespace

int batch_variant_count_f64() { return (int)(sizeof(kF64) / sizeof(kF64[0])); }
BatchVariant batch_variant_f64(int v) { return kF64[v]; }

int batch_occupancy_f64(int v) {
  switch (v) {
    case 0: return K0::occupancy();
    case 1: return K1::occupancy();
  }
  return 0;
}

cudaError_t launch_batch_step_f64(int v, const void* args, const int* cur, const WorkItem* items,
                                  int nitems, int parity, int* counter, int grid, cudaStream_t s) {
  switch (v) {
    case 0: return K0::launch(args, cur, items, nitems, parity, counter, grid, s);
    case 1: return K1::launch(args, cur, items, nitems, parity, counter, grid, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace alb
