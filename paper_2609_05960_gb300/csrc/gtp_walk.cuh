// The fused power walk and its adjoint: launch interface.
#pragma once

#include "gtp_internal.cuh"

namespace gtp {

constexpr int kWalkThreads = 256;  // threads of a walk CTA

// Per-gate energy tables (built by launch_gate_prep): for a gate whose cell
// has at most kGateTabMaxIn inputs, entry (pin << n_in) | s holds the
// energy of an event on `pin` when the input-pin state before it is s (the
// pin's own bit being its old value): the internal energy (fJ, bilinear NLDM
// value times escale) for an input pin, 0.5 * C * Vdd^2 for the output pin
// (pin n_in).  The adjoint table holds the unscaled energies in
// [0, kGateTab) (output slots 0) and their load derivatives in
// [kGateTab, 2 * kGateTab) (output slots 0.5 * Vdd^2).
constexpr int kGateTab = 32;
constexpr int kGateTabMaxIn = 3;

// Device-side plan scratch of one run (all windows of the run).
struct PlanBufs {
  int2* glist;                  // gates with events {window, gate}: big, then medium, then sparse
  unsigned long long* counters; // see plan_counter_slots()
  int64_t gcap;                 // capacity of glist (windows x gates)
};

// counters[0] = big gates, [1] = medium gates, [2] = sparse gates, [3] = work
// items handed out so far (the walk's work counter), [4] = blocks of the
// preparation pass that finished, [5] = tiled gates, [6] = the tiled walk's
// work counter, [7] = the tiled walk's chunks, then the work-list histogram
// and its bucket cursors.  The work list holds big, medium, sparse, then
// tiled gates.
constexpr int kPlanCntTiled = 5;
constexpr int kPlanCntTiledWork = 6;
constexpr int kPlanCntChunks = 7;
constexpr int kPlanCntHist = 8;
int plan_counter_slots(int dense_min);

// Gates walked by the time-sliced walk (gtp_tiled.cu) instead of the
// persistent walk: at least tmin events (tmin > 0), fewer than 2^31 (the walk
// keeps run offsets within a gate in 32 bits) and a cell with a per-gate
// energy table.
__host__ __device__ inline bool is_tiled(int64_t c, int64_t tmin, uint32_t n_in) {
  return tmin > 0 && c >= tmin && c < (1ll << 31) && n_in <= (uint32_t)kGateTabMaxIn;
}

struct WalkArgs {
  const WinDesc* wins;      // device array of n_win descriptors
  int n_win;
  int rpt;                  // records per lane of a dense segment: 4, 8 or 16
  int dense_min;            // gates with more events than this are cut into segments
  int grid;                 // persistent CTAs (0 = one wave at full occupancy)
  int n_sm;
  DevError* err;
  double* cell_acc;         // adjoint: [2 * n_cells] FP64 sums (d_escale, d_lscale)
  const float* gtab;        // forward gate tables [G][kGateTab]
  const float* gtab_bwd;    // adjoint gate tables [G][2 * kGateTab] (adjoint runs only)
  PlanBufs plan;
  int64_t n_gates;
  bool comp;                // forward: also accumulate every window's component bins (WinDesc::cbins)
  int64_t tile_min;         // single-window plain forward runs: gates with this many events or more go
                            // to the time-sliced walk (0: none)
  int32_t* chunks;          // tiled walk: chunk starts in the tiled list (capacity tile_chunk_cap(n_gates))
  int64_t piece_len;        // gates with more events are split into pieces of this many (0: none); a
                            // multiple of kPieceUnit
  bool whole;               // no gate of the run has more than piece_len events, so the walk compiled without
                            // pieces is launched (forward and adjoint runs)
  bool staged;              // adjoint without glitch detection: the build with the sparse threads' gate tables
                            // staged in shared memory (small windows)
};

// Work-list entries are {window | piece << kPieceShift, gate}.
constexpr int kPieceShift = 10;
constexpr int kWindowMask = (1 << kPieceShift) - 1;
// Pieces are multiples of the longest chunk a big gate is walked in (8 warps x 32 lanes x 16 records).
constexpr int64_t kPieceUnit = 4096;
// Work items of a gate with c events: its pieces, or 1.
__host__ __device__ inline int64_t gate_items(int64_t c, int64_t piece_len) {
  return (piece_len > 0 && c > piece_len) ? (c + piece_len - 1) / piece_len : 1;
}

bool walk_rpt_supported(int rpt);
// Forward preparation in one launch over (window, gate): clear the windows'
// bins, the gate pass (L0 into each window's l0; results of gates without
// events), and with `plan` the work-list histogram and bucket starts.
cudaError_t launch_prepare(const LibView& L, const NetView& N, const WalkArgs& A, bool plan, cudaStream_t st);
// Scatter of the (window, gate) pairs with events into the work list: big
// gates (largest first), medium gates, sparse gates, tiled gates.  Follows
// launch_prepare with plan, or launch_plan's histogram.
cudaError_t launch_plan_scatter(const LibView& L, const NetView& N, const WalkArgs& A, cudaStream_t st);

// The time-sliced walk of the tiled gates (gtp_tiled.cu): chunking of the
// tiled list (one block), then the persistent walk over (chunk, slice) items.
// Single window (A.wins[0]), plain forward walk only.
int64_t tile_chunk_cap(int64_t n_gates);
// Whether the library's leakage table fits the tiled walk's shared memory.
bool tiled_fits(const LibView& L);
cudaError_t launch_tiled(const LibView& L, const NetView& N, const WalkArgs& A, int32_t n_bins, cudaStream_t st);
// The whole work list without the gate pass (the adjoint): histogram, bucket
// starts and scatter (no host synchronisation).
cudaError_t launch_plan(const NetView& N, const LibView& L, const WalkArgs& A, cudaStream_t st);
cudaError_t launch_walk(const LibView& L, const NetView& N, const WalkArgs& A, bool backward, cudaStream_t st);
// The walk with glitch detection (N.clock_ps > 0), in its own translation unit.
cudaError_t launch_walk_glitch(const LibView& L, const NetView& N, const WalkArgs& A, bool backward, cudaStream_t st);
// The forward walk (with or without glitch detection) that also accumulates
// each window's component bins (WinDesc::cbins), in its own translation unit.
cudaError_t launch_walk_components(const LibView& L, const NetView& N, const WalkArgs& A, cudaStream_t st);
// The forward walk (plain or with glitch detection) and the adjoint walk
// compiled for runs without split gates (A.whole).
cudaError_t launch_walk_plain_whole(const LibView& L, const NetView& N, const WalkArgs& A, cudaStream_t st);
cudaError_t launch_walk_glitch_whole(const LibView& L, const NetView& N, const WalkArgs& A, cudaStream_t st);
cudaError_t launch_walk_adjoint_whole(const LibView& L, const NetView& N, const WalkArgs& A, cudaStream_t st);
cudaError_t launch_walk_adjoint_staged(const LibView& L, const NetView& N, const WalkArgs& A, cudaStream_t st);
// The gates' event descriptors and energy tables in one pass (null outputs
// are skipped).
cudaError_t launch_gate_prep(const LibView& L, const NetView& N, uint4* desc, float* gtab, float* gtab_bwd,
                             cudaStream_t st);

}  // namespace gtp
