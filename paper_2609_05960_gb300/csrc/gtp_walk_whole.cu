// The plain forward walk for runs in which no gate is split into pieces (no
// gate has more events than the run's piece length): every work item is a
// whole gate, so the piece bookkeeping compiles away.  Built apart so that it
// compiles in parallel with the other walks.
#include "gtp_walk_body.cuh"

namespace gtp {

cudaError_t launch_walk_plain_whole(const LibView& L, const NetView& N, const WalkArgs& A, cudaStream_t st) {
  return launch_walk_whole<false, false>(L, N, A, st);
}

}  // namespace gtp
