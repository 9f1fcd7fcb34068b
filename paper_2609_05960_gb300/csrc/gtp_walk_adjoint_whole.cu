// The adjoint walk for runs in which no gate is split into pieces (see
// gtp_walk_whole.cu), built apart to compile in parallel.
#include "gtp_walk_body.cuh"

namespace gtp {

cudaError_t launch_walk_adjoint_whole(const LibView& L, const NetView& N, const WalkArgs& A, cudaStream_t st) {
  return launch_walk_whole<true, false>(L, N, A, st);
}

}  // namespace gtp
