// The fused forward walk that also keeps the power components' bins apart
// (leakage, internal, switching and glitch energy, Sec. 2.2), compiled apart
// from the plain walk so that the two build in parallel.
#include "gtp_walk_body.cuh"

namespace gtp {

cudaError_t launch_walk_components(const LibView& L, const NetView& N, const WalkArgs& A, cudaStream_t st) {
  if (N.clock_ps > 0) return launch_walk_cmp<true>(L, N, A, st);
  return launch_walk_cmp<false>(L, N, A, st);
}

}  // namespace gtp
