// Segmented warp walk: plan and launcher.
#pragma once

#include "gtp_internal.cuh"

namespace gtp {

struct SegPlan {
  int rpt;          // records per thread (K)
  int block;        // threads per CTA
  int grid;         // persistent CTAs
  int64_t seg_len;  // records per warp segment = 32 * K
  int64_t n_seg;    // segments covering the window's records
};

bool seg_rpt_supported(int rpt);
SegPlan make_seg_plan(int rpt, int block, int ctas_per_sm, int n_sm, int64_t n_events);

// Enqueue the seed prepass and the seed fix-up.  `runs` holds n_seg + 1 int64.
cudaError_t launch_seeds(const LibView& L, const NetView& N, const WindowView& W, const SegPlan& P, Seed* seeds,
                         int64_t* runs, cudaStream_t st);
// Enqueue the walk (seeds must be ready on the stream).
cudaError_t launch_walk(const LibView& L, const NetView& N, const WindowView& W, const Outputs& O, const SegPlan& P,
                        const Seed* seeds, cudaStream_t st);

}  // namespace gtp
