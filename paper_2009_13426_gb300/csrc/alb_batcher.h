// Work plan of a batched step (host side), shared by alb_batch and the
// serving loop: the flows of one precision, their step arguments for both
// buffer parities, their current buffer and the table of work items.
#pragma once

#include <vector>

#include "alb_internal.h"

namespace alb {

// Launch shape of one precision (the C ABI's alb_batch_tuning).
struct Tuning {
  int variant = 0;
  int tile_w[3] = {64, 128, 128};  // flows with nx < 128, nx < 512, larger
  int dynamic = 1;
  int blocks_per_sm = 0;           // 0: occupancy maximum
};

inline int size_class(int nx) { return nx < 128 ? 0 : nx < 512 ? 1 : 2; }

class GroupPlan {
 public:
  explicit GroupPlan(int precision) : precision_(precision) {}
  ~GroupPlan();
  GroupPlan(const GroupPlan&) = delete;
  GroupPlan& operator=(const GroupPlan&) = delete;

  int precision() const { return precision_; }
  int nflows() const { return (int)flows_.size(); }
  int nitems() const { return ends_.empty() ? 0 : ends_.back(); }
  const Tuning& tuning() const { return tuning_; }
  int grid() const { return grid_; }

  // Replace the flows (pointers are not owned and must outlive the plan).
  // Items are laid out flow by flow in the given order, so the flows that
  // take part in step s of a chunk must come first (see items_before).
  // Uploads arguments, current buffers and items; synchronises `s`.
  cudaError_t set_flows(const std::vector<FlowDev*>& flows, cudaStream_t s);
  // Change the launch shape (rebuilds the items); synchronises `s`.
  cudaError_t set_tuning(const Tuning& t, cudaStream_t s);
  // Upload the flows' current buffer (FlowDev::cur) after a host-side change.
  cudaError_t upload_cur(cudaStream_t s);
  // Items of the first nf flows.
  int items_before(int nf) const { return nf <= 0 ? 0 : ends_[nf - 1]; }
  // Replace the table by the items of the flows of size class c only (a
  // scratch table for tuning; set_tuning restores the full one).
  cudaError_t restrict_to_class(int c, cudaStream_t s);
  // Items in the device table.
  int table_items() const { return ntable_; }

  // One step of the first nitems items with parity p (flow f reads buffer
  // cur[f] ^ p). counter: a device int of this plan, zeroed before the launch
  // when the tuning is dynamic.
  cudaError_t launch(int parity, int nitems, int* counter, cudaStream_t s) const;
  // Flip every flow's current buffer on the device (after an odd step).
  cudaError_t flip(cudaStream_t s) const;

  const std::vector<FlowDev*>& flows() const { return flows_; }

 private:
  cudaError_t build_items(cudaStream_t s, int only_class);
  cudaError_t reserve(void** p, size_t* cap, size_t bytes);

  int precision_;
  std::vector<FlowDev*> flows_;
  std::vector<int> ends_;  // cumulative item counts per flow
  Tuning tuning_;
  int grid_ = 0;
  int ntable_ = 0;         // items in the device table
  void* d_args_ = nullptr;
  size_t args_cap_ = 0;
  int* d_cur_ = nullptr;
  size_t cur_cap_ = 0;
  WorkItem* d_items_ = nullptr;
  size_t items_cap_ = 0;
};

// Variants and launchers per precision (alb_batch_f32.cu / alb_batch_f64.cu).
int batch_variant_count_f32();
BatchVariant batch_variant_f32(int v);
int batch_occupancy_f32(int v);
cudaError_t launch_batch_step_f32(int v, const void* args, const int* cur, const WorkItem* items,
                                  int nitems, int parity, int* counter, int grid, cudaStream_t s);
int batch_variant_count_f64();
BatchVariant batch_variant_f64(int v);
int batch_occupancy_f64(int v);
cudaError_t launch_batch_step_f64(int v, const void* args, const int* cur, const WorkItem* items,
                                  int nitems, int parity, int* counter, int grid, cudaStream_t s);

// Check a tuning against the compiled variants; returns a message or null.
const char* check_tuning(int precision, const Tuning& t);
// Default launch shape of a precision: variant 0, tiles no wider than it.
Tuning default_tuning(int precision);
// Autotune the plan's launch shape on its flows' current state (alb_batch_tune).
int tune_group(GroupPlan* p, cudaStream_t stream, int* counter, int trials);

}  // namespace alb
