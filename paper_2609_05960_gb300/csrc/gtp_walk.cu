// Work-list planning (the preparation pass and the scatter) and the walk
// launcher; the walk itself is in gtp_walk_body.cuh.
#include <algorithm>
#include <cstdio>

#include "gtp_walk_body.cuh"

namespace gtp {

namespace {

constexpr int kBigBuckets = 32;
constexpr int kSparseBase = kBigBuckets + kWarps;

// ------------------------------------------------------------------ plan
// Work-list bucket of a gate with c > 0 events (lower buckets first):
//   big    (c > kWarps * seg_len):        0..31 by decreasing floor(log2 c)
//   medium (dense_min < c, <= 8 segments): 32..39 by decreasing segment count
//   sparse (c <= dense_min):              40..40+dense_min-1 by decreasing c
//   tiled  (see is_tiled; walked by the time-sliced walk, gtp_tiled.cu):
//          the 32 buckets after the sparse ones, by decreasing floor(log2 c)
__device__ __forceinline__ int work_bucket(int64_t c, int dmin, int64_t seg_len, bool tiled, bool piece = false) {
  if (tiled) return kSparseBase + dmin + 31 - min(31, 63 - __clzll((unsigned long long)c));
  if (piece || c > kWarps * seg_len)  // the pieces of a split gate are always big items
    return kBigBuckets - 1 - min(kBigBuckets - 1, 63 - __clzll((unsigned long long)c));
  if (c <= dmin) return kSparseBase + dmin - (int)c;
  return kSparseBase - (int)((c + seg_len - 1) / seg_len);
}

__host__ __device__ constexpr int n_buckets(int dmin) { return kSparseBase + dmin + 32; }

// Plan counters: [0] big, [1] medium, [2] sparse gates; [3] the walk's work
// counter; [4] blocks of the preparation pass that have finished; [5] tiled
// gates, [6] the tiled walk's work counter, [7] its chunks; then the
// work-list histogram [nb] and the bucket cursors [nb].
constexpr int kCntDone = 4;
constexpr int kCntHist = kPlanCntHist;

// Block-wide exclusive scan of one value per thread (blockDim.x a multiple of
// 32); returns the thread's exclusive prefix and writes the block total.
__device__ unsigned long long block_excl_scan_u64(unsigned long long v, unsigned long long* total) {
  __shared__ unsigned long long warp_tot[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned long long inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long u = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += u;
  }
  if (lane == 31) warp_tot[w] = inc;
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    const unsigned long long x = lane < nw ? warp_tot[lane] : 0ull;
    unsigned long long xi = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long u = __shfl_up_sync(0xffffffffu, xi, o);
      if (lane >= o) xi += u;
    }
    if (lane < nw) warp_tot[lane] = xi - x;
    if (lane == nw - 1) *total = xi;
  }
  __syncthreads();
  const unsigned long long r = inc - v + warp_tot[w];
  __syncthreads();
  return r;
}

// Bucket starts (exclusive scan of the histogram in bucket order) and the
// three list sizes; run by one whole block once every histogram update has
// landed.
__device__ void plan_bucket_starts(int nb, PlanBufs P) {
  const unsigned long long* hist = P.counters + kCntHist;
  unsigned long long* cursor = P.counters + kCntHist + nb;
  __shared__ unsigned long long starts[3], tot;
  const int tiled_base = nb - 32;
  const int per = (nb + (int)blockDim.x - 1) / (int)blockDim.x;
  const int b0 = min(nb, (int)threadIdx.x * per), b1 = min(nb, b0 + per);
  unsigned long long sum = 0ull;
  for (int b = b0; b < b1; ++b) sum += __ldcg(hist + b);
  unsigned long long pre = block_excl_scan_u64(sum, &tot);
  for (int b = b0; b < b1; ++b) {
    if (b == kBigBuckets) starts[0] = pre;
    if (b == kSparseBase) starts[1] = pre;
    if (b == tiled_base) starts[2] = pre;
    cursor[b] = pre;
    pre += __ldcg(hist + b);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    P.counters[0] = starts[0];
    P.counters[1] = starts[1] - starts[0];
    P.counters[2] = starts[2] - starts[1];
    P.counters[kPlanCntTiled] = tot - starts[2];
  }
}

// One pass over (window, gate), launched on a grid of (blocks, windows):
//   GATE  clear the window's bins and do the gate pass: L0 = sum over gates
//         of P_leak(cell, initial state) * lscale into the window's l0, and a
//         gate without events leaks at its initial state over the whole
//         window (with PLAN the walk writes the results of the other gates;
//         without it every gate's results are initialised here);
//   PLAN  histogram of work buckets (block-aggregated); the block that
//         finishes last turns it into bucket starts.
template <bool GATE, bool PLAN>
__global__ void __launch_bounds__(256) k_prepare(LibView L, NetView N, const WinDesc* __restrict__ wins,
                                                 DevError* err, int64_t seg_len, int dmin, PlanBufs P,
                                                 int64_t tmin, int64_t piece_len) {
  extern __shared__ unsigned int sh[];  // PLAN: [nb] bucket counts of this block
  __shared__ double red[32];
  __shared__ bool s_last;
  const int nb = n_buckets(dmin);
  const WinDesc& W = wins[blockIdx.y];
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  if (PLAN) {
    for (int b = threadIdx.x; b < nb; b += blockDim.x) sh[b] = 0u;
    __syncthreads();
  }
  if (GATE && !W.keep_bins) {  // bins are 8-byte pairs in a 256-byte aligned buffer: two per 16-byte store
    float4* b4 = reinterpret_cast<float4*>(W.bins);
    const int64_t n4 = (int64_t)W.n_bins >> 1;
    for (int64_t i = tid; i < n4; i += stride) b4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (tid == 0 && (W.n_bins & 1)) W.bins[W.n_bins - 1] = make_float2(0.f, 0.f);
    if (W.cbins)
      for (int64_t i = tid; i < W.n_bins; i += stride) W.cbins[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (W.tbins)
      for (int64_t i = tid; i < W.n_bins; i += stride) W.tbins[i] = make_double2(0.0, 0.0);
  }
  double p0 = 0.0;
  // kP gates a thread per round, their loads issued together (a window of a batched run has a few blocks
  // for many gates, so one gate at a time left each thread waiting on one load chain after another)
  constexpr int kP = 4;
  for (int64_t g0 = W.g0 + tid; g0 < W.g1; g0 += (int64_t)kP * stride) {
    int64_t c[kP];
    int32_t cl[kP];
    uint32_t s0[kP];
#pragma unroll
    for (int j = 0; j < kP; ++j) {
      const int64_t g = g0 + (int64_t)j * stride;
      const bool ok = g < W.g1;
      c[j] = ok ? W.offsets[g + 1] - W.offsets[g] : 0;
      cl[j] = ok && (GATE || tmin > 0) ? N.cell[g] : 0;
      s0[j] = ok && GATE ? (uint32_t)W.init[g] : 0u;
    }
    float p4 = 0.f;  // the round's initial leakage powers (FP32 for at most kP terms, then one FP64 add)
#pragma unroll
    for (int j = 0; j < kP; ++j) {
      const int64_t g = g0 + (int64_t)j * stride;
      if (g >= W.g1) break;
      const bool tiled = PLAN && tmin > 0 && is_tiled(c[j], tmin, (uint32_t)L.cells[cl[j]].n_in);
      if (GATE) {
        const CellInfo ci = L.cells[cl[j]];
        uint32_t s = s0[j];
        if (s >> (ci.n_in + 1)) {
          report_error(err, GTP_ERANGE, -1 - g);
          s &= (2u << ci.n_in) - 1u;
        }
        const float Pl = L.leak[ci.leak_base + s] * L.lscale[cl[j]];
        p4 += Pl;
        const bool split = PLAN && !tiled && gate_items(c[j], piece_len) > 1;
        if (!PLAN || c[j] == 0 || tiled || split) {  // the tiled walk and the pieces of a split gate add into its sums
          W.e_leak[g] = c[j] == 0 ? (double)Pl * (double)W.window_ps * 1e-6 : 0.0;
          W.e_int[g] = 0.0;
          W.e_sw[g] = 0.0;
          if (W.e_gl) W.e_gl[g] = 0.0;
          W.final_state[g] = (uint8_t)s;
        }
      }
      if (PLAN && c[j] > 0) {
        const int64_t items = tiled ? 1 : gate_items(c[j], piece_len);
        atomicAdd(&sh[work_bucket(items > 1 ? piece_len : c[j], dmin, seg_len, tiled, items > 1)],
                  (unsigned int)items);
      }
    }
    if (GATE) p0 += (double)p4;
  }
  if (GATE) {
    for (int o = 16; o > 0; o >>= 1) p0 += __shfl_down_sync(0xffffffffu, p0, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = p0;
    __syncthreads();
    if (threadIdx.x < 32) {
      double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (threadIdx.x == 0) atomicAdd(W.l0, v);
    }
  }
  if (PLAN) {
    __syncthreads();
    unsigned long long* hist = P.counters + kCntHist;
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
      if (sh[b]) atomicAdd(hist + b, (unsigned long long)sh[b]);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0)
      s_last = atomicAdd(P.counters + kCntDone, 1ull) == (unsigned long long)gridDim.x * gridDim.y - 1ull;
    __syncthreads();
    if (s_last) {
      __threadfence();
      plan_bucket_starts(nb, P);
    }
  }
}

// Each block round places kScatterPer gates per thread, so the bucket
// cursors see one atomic per bucket per 256 * kScatterPer gates.
#ifndef GTP_SCATTER_PER
#define GTP_SCATTER_PER 8
#endif
constexpr int kScatterPer = GTP_SCATTER_PER;

__global__ void k_plan_scatter(const WinDesc* __restrict__ wins, int64_t seg_len, int dmin, PlanBufs P,
                               const int32_t* __restrict__ gcell, const CellInfo* __restrict__ cells, int64_t tmin,
                               int64_t piece_len) {
  extern __shared__ unsigned long long sbase[];  // [0, nb): block bases; then [0, nb) local counts (32-bit)
  const int nb = n_buckets(dmin);
  unsigned int* sh = reinterpret_cast<unsigned int*>(sbase + nb);
  const WinDesc& W = wins[blockIdx.y];
  unsigned long long* cursor = P.counters + kCntHist + nb;
  const int64_t round = (int64_t)blockDim.x * kScatterPer;
  for (int64_t base = W.g0 + (int64_t)blockIdx.x * round; base < W.g1;
       base += (int64_t)gridDim.x * round) {  // block-uniform: the loop holds barriers
    for (int b = threadIdx.x; b < nb; b += blockDim.x) sh[b] = 0u;
    __syncthreads();
    int bk[kScatterPer];
    unsigned int local[kScatterPer], items[kScatterPer];
#pragma unroll
    for (int j = 0; j < kScatterPer; ++j) {
      const int64_t g = base + (int64_t)j * blockDim.x + threadIdx.x;
      const int64_t c = g < W.g1 ? W.offsets[g + 1] - W.offsets[g] : 0;
      const bool tiled = c > 0 && tmin > 0 && is_tiled(c, tmin, (uint32_t)cells[gcell[g]].n_in);
      items[j] = (unsigned int)(tiled ? 1 : gate_items(c, piece_len));
      bk[j] = c > 0 ? work_bucket(items[j] > 1 ? piece_len : c, dmin, seg_len, tiled, items[j] > 1) : -1;
      local[j] = bk[j] >= 0 ? atomicAdd(&sh[bk[j]], items[j]) : 0u;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nb; k += blockDim.x)
      if (sh[k]) sbase[k] = atomicAdd(cursor + k, (unsigned long long)sh[k]);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kScatterPer; ++j)
      if (bk[j] >= 0)
        for (unsigned int p = 0; p < items[j]; ++p)  // a split gate: one entry per piece
          P.glist[(int64_t)sbase[bk[j]] + local[j] + p] =
              make_int2((int)(blockIdx.y | (p << kPieceShift)), (int)(base + (int64_t)j * blockDim.x + threadIdx.x));
    __syncthreads();
  }
}

}  // namespace

bool walk_rpt_supported(int rpt) { return rpt == 4 || rpt == 8 || rpt == 16; }

int plan_counter_slots(int dense_min) { return kCntHist + 2 * n_buckets(dense_min); }

namespace {

// About 1024 blocks in all (at least 4 per window): every block ends with a
// few same-address atomics (bucket counts, cursors, the done counter, L0),
// so many windows of small blocks would serialise on them.
#ifndef GTP_PREP_BLOCKS
#define GTP_PREP_BLOCKS 512  // preparation blocks in all (measured on Large: 25 us at 512, 32 us at 1024, 38 us at 2048)
#endif
dim3 prepare_grid(const WalkArgs& A) {
  int64_t blocks = (A.n_gates + 255) / 256;
  const int64_t cap = std::max<int64_t>(4, GTP_PREP_BLOCKS / std::max(A.n_win, 1));
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  return dim3((unsigned)blocks, (unsigned)A.n_win);
}

template <bool GATE>
cudaError_t launch_prepare_plan(const LibView& L, const NetView& N, const WalkArgs& A, cudaStream_t st) {
  const int dmin = A.dense_min;
  cudaError_t e = cudaMemsetAsync(A.plan.counters, 0, sizeof(unsigned long long) * plan_counter_slots(dmin), st);
  if (e != cudaSuccess) return e;
  k_prepare<GATE, true><<<prepare_grid(A), 256, sizeof(unsigned int) * (size_t)n_buckets(dmin), st>>>(
      L, N, A.wins, A.err, 32ll * A.rpt, dmin, A.plan, GATE ? A.tile_min : 0, A.piece_len);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_prepare(const LibView& L, const NetView& N, const WalkArgs& A, bool plan, cudaStream_t st) {
  if (plan) return launch_prepare_plan<true>(L, N, A, st);
  k_prepare<true, false><<<prepare_grid(A), 256, 0, st>>>(L, N, A.wins, A.err, 32ll * A.rpt, A.dense_min, A.plan, 0,
                                                          0);
  return cudaGetLastError();
}

cudaError_t launch_plan_scatter(const LibView& L, const NetView& N, const WalkArgs& A, cudaStream_t st) {
  const int dmin = A.dense_min;
  const size_t nb = (size_t)n_buckets(dmin);
  const size_t scatter_smem = nb * (sizeof(unsigned long long) + sizeof(unsigned int));
  cudaError_t e = cudaFuncSetAttribute(k_plan_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)scatter_smem);
  if (e != cudaSuccess) return e;
  dim3 grid = prepare_grid(A);
  grid.x = (unsigned)std::max<int64_t>(1, std::min<int64_t>(grid.x, (A.n_gates + 256 * kScatterPer - 1) / (256 * kScatterPer)));
  k_plan_scatter<<<grid, 256, scatter_smem, st>>>(A.wins, 32ll * A.rpt, dmin, A.plan, N.cell, L.cells, A.tile_min,
                                                  A.piece_len);
  return cudaGetLastError();
}

cudaError_t launch_plan(const NetView& N, const LibView& L, const WalkArgs& A, cudaStream_t st) {
  WalkArgs B = A;
  B.tile_min = 0;  // the whole list for the walk (the adjoint has no tiled form)
  cudaError_t e = launch_prepare_plan<false>(L, N, B, st);
  if (e != cudaSuccess) return e;
  return launch_plan_scatter(L, N, B, st);
}

cudaError_t launch_walk(const LibView& L, const NetView& N, const WalkArgs& A, bool backward, cudaStream_t st) {
  if (!backward && A.comp) return launch_walk_components(L, N, A, st);
  if (N.clock_ps > 0) {
    if (!backward && A.whole) return launch_walk_glitch_whole(L, N, A, st);
    return launch_walk_glitch(L, N, A, backward, st);
  }
  if (backward && A.staged) return launch_walk_adjoint_staged(L, N, A, st);
  if (A.whole) return backward ? launch_walk_adjoint_whole(L, N, A, st) : launch_walk_plain_whole(L, N, A, st);
  return launch_walk_gl<false>(L, N, A, backward, st);
}

}  // namespace gtp
