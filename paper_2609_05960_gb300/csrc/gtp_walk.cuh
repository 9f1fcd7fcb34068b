// The fused power walk and its adjoint: launch interface.
#pragma once

#include "gtp_internal.cuh"

namespace gtp {

struct WalkArgs {
  const WinDesc* wins;      // device array of n_win descriptors
  const int64_t* seg_base;  // device [n_win + 1]: first global segment of each window
  int n_win;
  int64_t n_seg_total;
  int64_t seg_len;          // 32 * rpt
  int rpt;                  // records per lane: 4, 8 or 16
  int block;                // threads per CTA: 128 or 256
  int grid;                 // persistent CTAs (0 = one wave at full occupancy)
  int n_sm;
  DevError* err;
  double* cell_acc;         // adjoint: [2 * n_cells] FP64 sums (d_escale, d_lscale)
};

bool walk_rpt_supported(int rpt);
// Segment gates, seeds and seed fix-up (runs: n_seg_total + 1 int64 scratch).
cudaError_t launch_seeds(const NetView& N, const LibView& L, const WalkArgs& A, int64_t* runs, cudaStream_t st);
cudaError_t launch_walk(const LibView& L, const NetView& N, const WalkArgs& A, bool backward, cudaStream_t st);
size_t walk_smem_bytes(const LibView& L, int rpt, int block, int n_win, bool backward);

}  // namespace gtp
