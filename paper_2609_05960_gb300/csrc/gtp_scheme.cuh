// The paper's own GPU schemes, restated as sm_103a kernels for the ablation
// against the engine's walk: Naive-D (one event per thread, Sec. 2.4.1),
// Naive-L (one window of n_cyc bins per thread and gate, Sec. 2.4.2), the
// state-pattern traversal they start from (Sec. 3.1) and its
// replacement by state-indexed lookup (SIPL, Sec. 4.1), event-density-aware
// per-gate partitioning (Sec. 4.2), and the fused kernel (Sec. 4.3,
// Algorithm 1) with the two-phase per-gate reduction (Sec. 4.4).
//
// They work on the paper's input form, one time-ordered event stream per
// (gate, pin), built once per window from the engine's per-gate records.
// The waveform bin plays the part of the paper's clock cycle (the paper sets
// the waveform interval to the cycle); the clock of glitch detection is the
// engine's (NetView::clock_ps).
#pragma once

#include "gtp_internal.cuh"

namespace gtp {

constexpr int kSchemeTpb = 128;  // threads per block (the paper's setting)
constexpr int kStreamSlots = 8;  // pin streams per gate (pins 0-7)

// Per-pin event streams of one window.  Stream (g, p) is
// ev[off[g * 9 + p], off[g * 9 + p + 1]); an event is t | value << 31; the
// streams of gate g fill the gate's own record range [offsets[g],
// offsets[g+1]) in pin order.  slot[i] = g * 8 + p names the stream of event i.
struct PinStreams {
  int64_t* off;    // [G][9]
  uint32_t* ev;    // [E]
  uint32_t* slot;  // [E]
};

// Device state of one scheme run.
struct SchemeArgs {
  const WinDesc* win;        // the window's descriptor (device)
  PinStreams ps;
  const uint16_t* pat_int;   // state pattern of each table (its side-input state), for the traversal
  const uint16_t* pat_leak;  // state pattern of each leakage entry (its full state)
  double* ebins;             // [n_bins] energy per bin, fJ (FP64 atomics)
  double* R;                 // [G][kSchemeTpb][4] per-gate reduction rows {leak, int, sw, gl} fJ
  // density-aware partitioning (host-planned): the gate of each block, the
  // gate's first block and its window length in bins
  const int32_t* blk_gate;
  const int64_t* blk_first;
  const int32_t* ncyc;
  int64_t n_blocks;
  int32_t ncyc_fix;          // the fixed window length of Naive-L (bins)
  int32_t n_gates_i;
};

enum SchemeId { kSchemeNaive = 0, kSchemeSipl = 1, kSchemeDensity = 2, kSchemeFused = 3 };

// Per-pin streams from the window's records, checking the trace as the walk
// does (a malformed gate reports its first bad record into err and leaves its
// streams empty).
cudaError_t launch_pin_streams(const LibView& L, const NetView& N, const WinDesc* win, PinStreams ps, DevError* err,
                               cudaStream_t st);
// The kernels of one scheme (ebins and R must be zero; R is left zero, the
// per-gate results, final states and the waveform written).
cudaError_t launch_scheme(int scheme, const LibView& L, const NetView& N, const SchemeArgs& A, int64_t n_events,
                          int32_t n_bins, cudaStream_t st);

}  // namespace gtp
