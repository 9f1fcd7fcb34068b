// Internal definitions shared by the engine's translation units.
//
// Device data layout (per context):
//   library   tab[n_tables * ns * nl] (fJ, unscaled), leak[n_leak] (nW,
//             unscaled), cells[n_cells] = {first table, first leakage entry,
//             n_in}, table_cell[n_tables], leak_cell[n_leak] (owning cell of
//             each table / leakage entry, for scaling), escale/lscale[n_cells]
//   netlist   cell[G] int32, load[G] float, slew[G][stride][2] float, and the
//             event descriptors derived from them once per netlist:
//             desc[G][2*(stride+1)] (16 B each, see NetView)
//   window    offsets[G+1] int64, records[E] 8 B {int32 t, uint32 meta},
//             init[G] uint8, per-gate outputs (FP64 energies, uint8 final
//             state), and the bin
//             accumulators float2[n_bins] = {dynamic + in-bin leakage energy
//             (fJ), leakage-power step (nW)}
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/gtpower.h"

namespace gtp {

constexpr int kMaxAxis = GTP_MAX_AXIS;
constexpr int kMaxPins = GTP_MAX_PINS;

struct CellInfo {
  int32_t tab_base;   // index of the cell's first table
  int32_t leak_base;  // index of the cell's first leakage entry
  int32_t n_in;       // input pins
  int32_t pad;
};

// Everything a kernel needs to evaluate energies.  Passed by value.
struct LibView {
  const float* tab;          // unscaled tables
  const float* leak;         // unscaled leakage
  const CellInfo* cells;
  const uint8_t* table_cell; // cell of each table
  const uint8_t* leak_cell;  // cell of each leakage entry
  const float* escale;
  const float* lscale;
  int32_t n_cells;
  int32_t n_tables;
  int32_t n_leak;
  int32_t ns, nl, tsize;     // axis lengths, ns*nl
  float half_v2;             // 0.5 * Vdd^2
  float slew_axis[kMaxAxis];
  float load_axis[kMaxAxis];
  float slew_rw[kMaxAxis];   // 1 / (axis[i+1] - axis[i])
  float load_rw[kMaxAxis];
};

// Event descriptor of one (gate, pin, edge), 16 bytes, built once per
// netlist / load update, before the next run (k_gate_prep):
//   input pin:  x = slew fraction, y = load fraction, w = 1 / load-segment width
//   output pin: w = 0.5 * C * Vdd^2 (the switching energy)
//   z = table element offset without the side bits (bits 0-15; for the
//       output pin the cell's first table) | cell << 16 | output << 24 |
//       load segment << 25
struct NetView {
  const int32_t* cell;
  const float* load;
  const float* slew;         // [G][stride][2]
  const uint4* desc;         // [G][dstride] event descriptors
  int64_t n_gates;
  int32_t stride;            // slew stride (input pins per gate)
  int32_t dstride;           // descriptors per gate = 2 * (stride + 1)
  // glitch detection (Sec. 2.4.1): clock period in ps (0: off), its
  // division constants (see bin_of), and the output pins' {fall, rise}
  // transition times [G][2]
  int32_t clock_ps;
  uint32_t clock_magic, clock_shift;
  const float* out_slew;
};

// Pattern cells: cells given by state patterns, up to 32 pins (Sec. 4.1's
// fallback for wide cells).  A cell's internal patterns are stored per pin,
// in list order within the pin (the first match of the pin's list is the
// first match of the whole list: the other pins' patterns never match).
struct PatCell {
  int32_t n_in;      // input pins; the output pin is pin n_in
  int32_t ipo;       // first of the cell's n_in + 1 entries of PatLib::ipo
  int32_t lp0, lp1;  // leakage patterns [lp0, lp1) of PatLib::lp
  int32_t dtab;      // default table of (pin, edge): dtab + 2 * pin + edge
  float leak_def;    // default leakage, nW
  int64_t iidx;      // state-indexed table ids [n_in][2][2^(n_in-1)] at PatLib::iidx + iidx, or -1: traversal
  int64_t lidx;      // state-indexed leakage [2^(n_in+1)] at PatLib::lidx + lidx, or -1: traversal
};

struct PatLib {
  const PatCell* cells;
  const uint4* ip;           // {care, val, edge (0xFFFFFFFF: either), table}
  const int32_t* ipo;        // per cell, n_in + 1 offsets into ip (pin p: [ipo[p], ipo[p + 1]))
  const uint4* lp;           // {care, val, power (float bits, nW), 0}
  const float* tab;          // [n_tab][ns * nl] fJ: the patterns' tables, then the defaults
  const int32_t* iidx;       // state-indexed table ids of the indexed cells
  const float* lidx;         // state-indexed leakage of the indexed cells
  int32_t n_cells;
  int32_t ns, nl, tsize;
  float half_v2;             // 0.5 * Vdd^2
  float slew_axis[kMaxAxis];
  float load_axis[kMaxAxis];
};

struct PatNet {
  const int32_t* cell;       // [Gp]
  const float* load;         // [Gp] fF
  const float* slew;         // [Gp][stride][2] input transition times, ps
  const float* oslew;        // [Gp][2] output {fall, rise} transition times, ps
  const uint2* desc;         // [Gp][stride][2] per (gate, input pin, edge): {table element of the lower slew
                             //   and load knots, slew fraction (float bits)}, located once per netlist
  int64_t n_gates;
  int32_t stride;
};

// First failure seen by a kernel: code and record index.
struct DevError {
  int32_t code;
  int32_t pad;
  int64_t index;
};

// One stimulus window as the kernels see it (single, batched and adjoint
// runs all use an array of these in device memory).
struct WinDesc {
  const int64_t* offsets;    // [G+1]
  const uint2* rec;          // [E]
  const uint8_t* init;       // [G]
  double* e_leak;            // [G]
  double* e_int;             // [G]
  double* e_sw;              // [G]
  double* e_gl;              // [G] glitch energy, or null without glitch detection
  uint8_t* final_state;      // [G]
  float2* bins;              // [n_bins] accumulators
  double2* tbins;            // [n_bins] {energy fJ, leakage step nW} of the time-sliced walk (FP64), or null
  float4* cbins;             // [n_bins] component accumulators, or null (no per-component waveform):
                             //   cpack 0: {internal, switching, glitch fJ, leakage in-bin corrections fJ},
                             //            beside the bins as usual (runs with glitch detection)
                             //   cpack 1: {internal, switching fJ, leakage in-bin corrections fJ,
                             //            leakage step nW}, the bins unused (runs without)
  double* cwave;             // [4][n_bins] component waveforms (W): leakage, internal, switching, glitch, or null
  double* l0;                // sum over gates of P_leak(initial state), nW
  double* tiles;             // merge scratch
  double* wave;              // [n_bins] output waveform (W), or null
  const float2* grad;        // adjoint: [n_bins] {dL/dE_b, G(b * bin_ps)}
  float* dC;                 // adjoint: [G]
  int64_t n_events;
  int64_t tile_base;         // first global merge tile of this window
  int64_t g0, g1;            // the gates this descriptor covers: [g0, g1) (all gates, but for a streamed chunk)
  int32_t n_tiles;
  int32_t window_ps;
  int32_t bin_ps;
  uint32_t bin_magic;        // see bin_of()
  uint32_t bin_shift;
  int32_t n_bins;
  float g_total;             // adjoint: G(window_ps)
  int32_t keep_bins;         // the preparation pass leaves the bins as they are (a streamed run's later chunks)
  int32_t cpack;             // layout of cbins (see there)
  // the window's pattern gates (p_n_items == 0: none), walked into tbins
  const int64_t* p_off;      // [Gp + 1]
  const uint2* p_rec;        // [Ep] {t, pin | value << 8}
  const uint32_t* p_init;    // [Gp]
  const int2* p_items;       // [p_n_items] {gate, piece}: the gate's records from piece * kPatPiece on
  const int64_t* p_first;    // [Gp + 1] first item of each gate
  uint32_t* p_mask;          // [p_n_items] XOR of the pin bits of each item's records
  double* p_e_leak;          // [Gp]
  double* p_e_int;
  double* p_e_sw;
  double* p_e_gl;
  uint32_t* p_final;         // [Gp]
  float* p_dC;               // adjoint: [Gp] dL/dC of the pattern gates
  int64_t p_n_items;
};

// ------------------------------------------------------------------ device helpers
__device__ __forceinline__ void report_error(DevError* err, int code, int64_t index) {
  if (atomicCAS(&err->code, 0, code) == 0) err->index = index;
}

// Side-input bits: input pins other than `pin`, compacted in pin order.
__device__ __forceinline__ uint32_t side_bits(uint32_t S, uint32_t pin, uint32_t n_in) {
  uint32_t in_mask = (1u << n_in) - 1u;
  uint32_t low = S & ((1u << pin) - 1u);
  uint32_t high = (S >> 1) & ~((1u << pin) - 1u);
  return (low | high) & (in_mask >> 1);
}

// floor(t / bin_ps) for 0 <= t < 2^31: the multiply-high estimate is q or
// q - 1 (magic = min(floor(2^(32+s) / d), 2^32 - 1), s = floor(log2 d)), and
// one correction step makes it exact.  bin_magic() builds the two constants
// on the host; every path that bins events uses this one definition.
inline void bin_magic(int32_t d, uint32_t* magic, uint32_t* shift) {
  uint32_t s = 0;
  while ((2ull << s) <= (uint64_t)d) ++s;  // s = floor(log2 d)
  unsigned __int128 m = (((unsigned __int128)1) << (32 + s)) / (uint64_t)d;
  if (m > 0xFFFFFFFFull) m = 0xFFFFFFFFull;
  *magic = (uint32_t)m;
  *shift = s;
}

__device__ __forceinline__ uint32_t bin_of(uint32_t t, uint32_t magic, uint32_t shift, uint32_t bin_ps) {
  uint32_t b = __umulhi(t, magic) >> shift;
  return b + (((b + 1u) * bin_ps <= t) ? 1u : 0u);
}

// Glitch scaling ratio (Eq. 2) of an event `width` ps
// after the previous event on its pin, for the pin's rise + fall transition
// time sum: min(1, (2 * width / sum)^2); a pin without transition time
// (sum <= 0) swings fully.
__device__ __forceinline__ float glitch_ratio(uint32_t width, float sum) {
  if (!(sum > 0.f)) return 1.f;
  const float x = 2.f * (float)width / sum;
  return fminf(1.f, x * x);
}

// The same ratio from a pin's precomputed inv = 2 / (rise + fall), or -1 for
// a pin without transition time: min(1, (width * inv)^2).
__device__ __forceinline__ float glitch_inv(float sum) { return sum > 0.f ? 2.f / sum : -1.f; }
__device__ __forceinline__ float glitch_ratio_inv(uint32_t width, float inv) {
  if (inv < 0.f) return 1.f;
  const float x = (float)width * inv;
  return fminf(1.f, x * x);
}

// Start of the clock cycle holding t (glitch detection).
__device__ __forceinline__ uint32_t cycle_start(uint32_t t, int32_t clock_ps, uint32_t magic, uint32_t shift) {
  return bin_of(t, magic, shift, (uint32_t)clock_ps) * (uint32_t)clock_ps;
}

// Fire-and-forget vector add of {energy, leakage step} into one bin.
__device__ __forceinline__ void red_bin(float2* bins, uint32_t b, float e, float dp) {
  float2* p = bins + b;
  asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(e), "f"(dp) : "memory");
}

// The same for a bin's component accumulators (one 16-byte reduction).
__device__ __forceinline__ void red_cbin(float4* cbins, uint32_t b, float ei, float es, float eg, float lc) {
  float4* p = cbins + b;
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(ei), "f"(es), "f"(eg), "f"(lc)
               : "memory");
}

// Kahan-compensated FP32 accumulator.
struct Kahan {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    float y = x - c;
    float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// Shared-memory copy of the library: [axes 4 x kMaxAxis][tab][leak][cells][escale].
struct SmemLib {
  const float* axes;  // slew axis, load axis, slew 1/width, load 1/width
  const float* tab;
  const float* leak;
  const CellInfo* cells;
  const float* escale;
};

__host__ __device__ inline size_t smem_lib_bytes(const LibView& L) {
  size_t b = sizeof(float) * 4 * kMaxAxis + (size_t)L.n_tables * L.tsize * 4 + (size_t)((L.n_leak + 3) & ~3) * 4 +
             (size_t)L.n_cells * (sizeof(CellInfo) + sizeof(float));
  return (b + 15) & ~(size_t)15;
}

// Stage the library into dynamic shared memory.  With `scaled`, tables and
// leakage are multiplied by the per-cell scales (forward); without, they are
// copied unscaled (adjoint).  All threads participate; ends with a barrier.
__device__ __forceinline__ SmemLib stage_library(const LibView& L, unsigned char* smem, bool scaled) {
  float* axes = reinterpret_cast<float*>(smem);
  float* tab = axes + 4 * kMaxAxis;
  float* leak = tab + (size_t)L.n_tables * L.tsize;
  CellInfo* cells = reinterpret_cast<CellInfo*>(leak + ((L.n_leak + 3) & ~3));
  float* esc = reinterpret_cast<float*>(cells + L.n_cells);
  int nt = L.n_tables * L.tsize;
  for (int k = threadIdx.x; k < nt; k += blockDim.x)
    tab[k] = scaled ? L.tab[k] * L.escale[L.table_cell[k / L.tsize]] : L.tab[k];
  for (int k = threadIdx.x; k < L.n_leak; k += blockDim.x)
    leak[k] = scaled ? L.leak[k] * L.lscale[L.leak_cell[k]] : L.leak[k];
  for (int k = threadIdx.x; k < L.n_cells; k += blockDim.x) {
    cells[k] = L.cells[k];
    esc[k] = L.escale[k];
  }
  if (threadIdx.x < kMaxAxis) {
    axes[threadIdx.x] = L.slew_axis[threadIdx.x];
    axes[kMaxAxis + threadIdx.x] = L.load_axis[threadIdx.x];
    axes[2 * kMaxAxis + threadIdx.x] = L.slew_rw[threadIdx.x];
    axes[3 * kMaxAxis + threadIdx.x] = L.load_rw[threadIdx.x];
  }
  __syncthreads();
  return SmemLib{axes, tab, leak, cells, esc};
}

// ------------------------------------------------------------------ launchers (host)
cudaError_t launch_gate_pass_bwd(const LibView& L, const NetView& N, const WinDesc* wins, double* cell_acc,
                                 cudaStream_t st);
cudaError_t launch_walk_per_gate(const LibView& L, const NetView& N, const WinDesc* wins, int n_win,
                                 DevError* err, cudaStream_t st);
cudaError_t launch_merge(const WinDesc* wins, const int64_t* tile_base, int n_win, int64_t n_tiles_total,
                         cudaStream_t st);
// Adjoint input: grad[b] = {dL/dP_b * 1e-3 / bin_ps, G(b * bin_ps)}, and G(T).
cudaError_t launch_grad_prep(const WinDesc* wins, const float* dLdP, float2* grad, double* tiles, int n_tiles,
                             int n_bins, int bin_ps, float* g_total, cudaStream_t st);
cudaError_t launch_cells_out(const double* acc, int n_cells, float* d_escale, float* d_lscale, cudaStream_t st);
// Design-level sums of the per-gate energies and the waveform's peak:
// scratch[0..3] = sum of e_leak, e_int, e_sw, e_gl (fJ; e_gl may be null),
// scratch[4] = the peak bin's ordered key, scratch[5] = its first index (as
// unsigned 64-bit; all ones without a waveform).
cudaError_t launch_design_power(const double* e_leak, const double* e_int, const double* e_sw, const double* e_gl,
                                int64_t G, const double* wave, int64_t n_bins, double* scratch, cudaStream_t st);
// Exact first malformed record of the given windows (see k_validate): *first
// = ((window << 40 | record) << 3) | -code, or ~0 if every record is valid.
cudaError_t launch_validate(const LibView& L, const NetView& N, const WinDesc* wins, int n_win,
                            unsigned long long* first, cudaStream_t st);
// The same check of one descriptor's gates, run only if `err` already holds
// an error (a device-side test, so it can be enqueued unconditionally);
// *first must have been set to ~0 beforehand.
cudaError_t launch_validate_if(const LibView& L, const NetView& N, const WinDesc* win, const DevError* err,
                               int64_t n_gates, unsigned long long* first, cudaStream_t st);
int merge_tiles(int n_bins);
// Pattern gates: a gate's records are cut into items of kPatPiece records
// (each item extended to the end of the timestamp group it ends in).
#ifndef GTP_PAT_PIECE
#define GTP_PAT_PIECE 512
#endif
constexpr int64_t kPatPiece = GTP_PAT_PIECE;
// Pattern records {t, pin | value << 8} from the ABI's arrays (device).
cudaError_t launch_pattern_pack(const int32_t* t, const uint8_t* pin, const uint8_t* value, int64_t n, uint2* out,
                                cudaStream_t st);
// State-indexed arrays of pattern cell c (its iidx / lidx offsets set) into
// iidx / lidx, the arrays PatLib::iidx / lidx point to.
cudaError_t launch_pattern_index(const PatLib& P, int32_t c, int32_t n_in, int32_t* iidx, float* lidx,
                                 cudaStream_t st);
// The pattern gates of the windows: initial leakage, items' pin masks, and
// the walk into each window's bins (backward: dL/dC of each pattern gate
// into p_dC from the windows' gradient tables); errors as the smallest key
// ((window << 40 | record) << 3) | -code in *bad (see launch_validate).
cudaError_t launch_pattern_walk(const PatLib& P, const PatNet& Q, const WinDesc* wins, int n_win,
                                int64_t max_items, int32_t clock_ps, unsigned long long* bad, cudaStream_t st,
                                bool backward = false);
// The reduction-rate probe: n_red reductions of `width` (2 or 4) floats into
// hashed places of slots[n_slots] (16 B a slot).
cudaError_t launch_red_probe(float4* slots, uint32_t n_slots, int width, int64_t n_red, int n_sm, cudaStream_t st);
// The bin reductions of n records alone, one 8-byte reduction per distinct
// bin of 8 consecutive records, into slots[window_ps / bin_ps] (16 B each).
cudaError_t launch_red_replay(const uint2* rec, int64_t n, int32_t window_ps, int32_t bin_ps, float4* slots, int n_sm,
                              cudaStream_t st);
// Unpack records [r0, r0 + n) of the packed transfer form into out[0, n):
// `anchors` holds the anchors of blocks r0 / 32 .. (r0 + n - 1) / 32, `words`
// the n words (16-byte aligned).
cudaError_t launch_unpack(const uint32_t* anchors, const uint32_t* words, int64_t r0, int64_t n, uint2* out,
                          cudaStream_t st);

}  // namespace gtp
