// The fused walk with clock-cycle glitch detection (Sec. 2.4.1), compiled
// apart from the plain walk so that the two build in parallel.
#include "gtp_walk_body.cuh"

namespace gtp {

cudaError_t launch_walk_glitch(const LibView& L, const NetView& N, const WalkArgs& A, bool backward, cudaStream_t st) {
  return launch_walk_gl<true>(L, N, A, backward, st);
}

}  // namespace gtp
