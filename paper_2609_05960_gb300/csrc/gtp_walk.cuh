// The fused power walk and its adjoint: launch interface.
#pragma once

#include "gtp_internal.cuh"

namespace gtp {

constexpr int kWalkThreads = 256;  // threads of a walk CTA

// Per-gate energy tables (built by launch_gate_tables): for a gate whose cell
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
// preparation pass that finished, then the work-list histogram and its bucket
// cursors.
int plan_counter_slots(int dense_min);

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
};

bool walk_rpt_supported(int rpt);
// Forward preparation in one launch over (window, gate): clear the windows'
// bins, the gate pass (L0 into each window's l0; results of gates without
// events), and with `plan` the work-list histogram and bucket starts.
cudaError_t launch_prepare(const LibView& L, const NetView& N, const WalkArgs& A, bool plan, cudaStream_t st);
// Scatter of the (window, gate) pairs with events into the work list: big
// gates (largest first), medium gates, sparse gates.  Follows launch_prepare
// with plan, or launch_plan's histogram.
cudaError_t launch_plan_scatter(const NetView& N, const WalkArgs& A, cudaStream_t st);
// The whole work list without the gate pass (the adjoint): histogram, bucket
// starts and scatter (no host synchronisation).
cudaError_t launch_plan(const NetView& N, const LibView& L, const WalkArgs& A, cudaStream_t st);
cudaError_t launch_walk(const LibView& L, const NetView& N, const WalkArgs& A, bool backward, cudaStream_t st);
// The walk with glitch detection (N.clock_ps > 0), in its own translation unit.
cudaError_t launch_walk_glitch(const LibView& L, const NetView& N, const WalkArgs& A, bool backward, cudaStream_t st);
// The forward walk (with or without glitch detection) that also accumulates
// each window's component bins (WinDesc::cbins), in its own translation unit.
cudaError_t launch_walk_components(const LibView& L, const NetView& N, const WalkArgs& A, cudaStream_t st);
cudaError_t launch_gate_tables(const LibView& L, const NetView& N, float* gtab, float* gtab_bwd, cudaStream_t st);

}  // namespace gtp
