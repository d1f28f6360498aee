// Batched step kernel: one launch advances every flow of a batch by one time
// step. The tile update is the single-flow kernel's (tile_step), so the
// result of a node depends only on its flow's state, never on the batch, the
// tile shape or the block size.
//
// The grid is persistent (resident blocks x SMs). A block takes work items,
// each a tile of one flow (2^tw_log2 nodes along x by block >> tw_log2 rows),
// either from an atomic counter or by a fixed stride. When an item belongs to
// another flow (or buffer) than the block's previous one, the block copies
// that flow's step arguments into shared memory; then each thread updates
// one node.
#pragma once

#include "alb_step.cuh"

namespace alb {

template <typename P, int B, int MINB>
__global__ void __launch_bounds__(B, MINB)
    batch_step_kernel(const StepArgs<P>* __restrict__ args, const int* __restrict__ cur,
                      const WorkItem* __restrict__ items, int nitems, int parity, int* counter) {
  static_assert(sizeof(StepArgs<P>) % 8 == 0, "step arguments copy as 8-byte words");
  static_assert(sizeof(StepArgs<P>) / 8 <= B, "one word per thread");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double s_tab[EXPT_N];
  __shared__ __align__(16) unsigned long long s_args[sizeof(StepArgs<P>) / 8];
  __shared__ int s_item;
  __shared__ RebuildQueue<B> s_rq;
  load_exptab(s_tab);  // includes a barrier
  const StepArgs<P>& a = *reinterpret_cast<const StepArgs<P>*>(s_args);
  const Columns<P, B> cl(smem_raw);
  int it = blockIdx.x;
  int loaded = -1;  // (flow, buffer) whose arguments s_args holds
  for (;;) {
    __syncthreads();  // the previous item's readers of s_args / s_item are done
    if (counter) {
      if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
      __syncthreads();
      it = s_item;
    }
    if (it >= nitems) break;
    const WorkItem w = items[it];
    // Items are laid out flow by flow, so consecutive items of a block mostly
    // belong to one flow: copy its arguments only when the flow or buffer
    // changes (the same decision in every thread of the block).
    const int want = 2 * w.flow + (cur[w.flow] ^ parity);
    if (want != loaded) {
      if (threadIdx.x < sizeof(StepArgs<P>) / 8) {
        const unsigned long long* src =
            reinterpret_cast<const unsigned long long*>(args + want);
        s_args[threadIdx.x] = src[threadIdx.x];
      }
      __syncthreads();
      loaded = want;
    }
    NodeCount nc;
    tile_step<P, B>(a, w.x0, w.y0, w.tw_log2, cl, s_tab, s_rq, nc);
    flush_counts(a.ctr, nc);
    if (!counter) it += gridDim.x;
  }
}

// Launch helpers of one variant. occupancy() also opts the kernel in to its
// dynamic shared memory; the host calls it before any launch (and before any
// stream capture), so launch() itself makes no attribute call.
template <typename P, int B, int MINB>
struct BatchKernel {
  static constexpr size_t smem() { return smem_bytes<P, B>(); }
  static int occupancy() {
    auto k = batch_step_kernel<P, B, MINB>;
    // static shared memory counts against the default 48 KB too: always declare
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem()) !=
        cudaSuccess)
      return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, B, smem()) != cudaSuccess) return 0;
    return nb;
  }
  static cudaError_t launch(const void* args, const int* cur, const WorkItem* items, int nitems,
                            int parity, int* counter, int grid, cudaStream_t s) {
    batch_step_kernel<P, B, MINB><<<grid, B, smem(), s>>>((const StepArgs<P>*)args, cur, items,
                                                          nitems, parity, counter);
    return cudaGetLastError();
  }
};

}  // namespace alb
