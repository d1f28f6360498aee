// Batched step kernels of the FP32 form: the compiled (block, minimum
// resident blocks) variants the autotuner chooses from.
#include "alb_batch_kernel.cuh"
#include "alb_batcher.h"

namespace alb {

namespace {
using K0 = BatchKernel<float, 128, 4>;
using K1 = BatchKernel<float, 64, 8>;
using K2 = BatchKernel<float, 256, 2>;
using K3 = BatchKernel<float, 128, 3>;
constexpr BatchVariant kF32[] = {{128, 4}, {64, 8}, {256, 2}, {128, 3}};
}  // namespace

int batch_variant_count_f32() { return (int)(sizeof(kF32) / sizeof(kF32[0])); }
BatchVariant batch_variant_f32(int v) { return kF32[v]; }

int batch_occupancy_f32(int v) {
  switch (v) {
    case 0: return K0::occupancy();
    case 1: return K1::occupancy();
    case 2: return K2::occupancy();
    case 3: return K3::occupancy();
  }
  return 0;
}

cudaError_t launch_batch_step_f32(int v, const void* args, const int* cur, const WorkItem* items,
                                  int nitems, int parity, int* counter, int grid, cudaStream_t s) {
  switch (v) {
    case 0: return K0::launch(args, cur, items, nitems, parity, counter, grid, s);
    case 1: return K1::launch(args, cur, items, nitems, parity, counter, grid, s);
    case 2: return K2::launch(args, cur, items, nitems, parity, counter, grid, s);
    case 3: return K3::launch(args, cur, items, nitems, parity, counter, grid, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace alb
