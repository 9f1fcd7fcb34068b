// The adjoint walk with the sparse threads' gate tables staged in shared
// memory (two CTAs an SM) instead of read in place (three CTAs), for small
// windows.  Staged tables cost occupancy but spare each event an L1 miss;
// the walk takes them below about 200,000 events per SM (adjoint recipe,
// backward walk ms in place / staged: 5M events 0.255 / 0.145, 10M 0.287 /
// 0.158, 20M 0.298 / 0.224, 40M 0.329 / 0.370, 100M 0.712 / 0.793).
// Built apart: the table placement and the register budget are
// compile-time choices of the walk body.
#define GTP_BWD_TAB_L1 0
#define GTP_WALK_MINB_BWD 2
#include "gtp_walk_body.cuh"

namespace gtp {

cudaError_t launch_walk_adjoint_staged(const LibView& L, const NetView& N, const WalkArgs& A, cudaStream_t st) {
  if (A.whole) return launch_walk_whole<true, false>(L, N, A, st);
  switch (A.rpt) {
    case 4: return launch_walk_k<4, true, false, false>(L, N, A, st);
    case 16: return launch_walk_k<16, true, false, false>(L, N, A, st);
    default: return launch_walk_k<8, true, false, false>(L, N, A, st);
  }
}

}  // namespace gtp
