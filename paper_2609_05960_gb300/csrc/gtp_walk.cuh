// The fused power walk and its adjoint: launch interface.
#pragma once

#include "gtp_internal.cuh"

namespace gtp {

// Device-side plan scratch of one run (all windows of the run).
struct PlanBufs {
  int4* dtask;                  // dense segments: {window, gate, segment index in gate, 0}
  Seed* dseed;                  // seed of each dense segment
  int2* slist;                  // sparse gates {window, gate}, sorted by event count (descending)
  unsigned long long* counters; // see plan_counter_slots()
  int64_t* runs;                // dense segments whose seed needs the fix-up pass
  int64_t dcap, scap;           // capacities of dtask/dseed/runs and of slist
};

// counters[0] = dense segments, [1] = sparse gates, [2] = unresolved seeds,
// [3, 3 + dmin] = sparse histogram by event count, then the bucket cursors.
inline int plan_counter_slots(int dense_min) { return 3 + 2 * (dense_min + 1); }

struct WalkArgs {
  const WinDesc* wins;      // device array of n_win descriptors
  int n_win;
  int rpt;                  // records per lane of a dense segment: 4, 8 or 16
  int dense_min;            // gates with more events than this are cut into segments
  int block;                // threads per CTA: 128 or 256
  int grid;                 // persistent CTAs (0 = one wave at full occupancy)
  int n_sm;
  DevError* err;
  double* cell_acc;         // adjoint: [2 * n_cells] FP64 sums (d_escale, d_lscale)
  PlanBufs plan;
  int64_t n_gates;
};

bool walk_rpt_supported(int rpt);
// Classify gates, build the dense segment list and the sorted sparse list,
// and seed the dense segments (no host synchronisation).
cudaError_t launch_plan(const NetView& N, const LibView& L, const WalkArgs& A, cudaStream_t st);
cudaError_t launch_walk(const LibView& L, const NetView& N, const WalkArgs& A, bool backward, cudaStream_t st);

}  // namespace gtp
