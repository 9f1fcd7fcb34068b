// Internal definitions shared by the engine's translation units.
//
// Device data layout (per context):
//   library   tab[n_tab_floats] (fJ, unscaled), leak[n_leak] (nW, unscaled),
//             cell_info[n_cells] = {tab_base (first table of the cell),
//             leak_base, n_in}, table_cell[n_tables], leak_cell[n_leak]
//             (owning cell of each table / leakage entry, for scaling),
//             escale[n_cells], lscale[n_cells]
//   netlist   cell[G] int32, load[G] float, slew[G][stride][2] float
//   window    offsets[G+1] int64, records[E] (8 B: int32 t, uint32 meta),
//             init[G] uint8, segment seeds, per-gate outputs (FP64 energies,
//             uint8 final state), bin accumulators float2[n_bins] =
//             {dynamic + in-bin leakage energy (fJ), leakage-power step (nW)}
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

struct NetView {
  const int32_t* cell;
  const float* load;
  const float* slew;         // [G][stride][2]
  int64_t n_gates;
  int32_t stride;
};

// First failure seen by a kernel: code and record index.
struct DevError {
  int32_t code;
  int32_t pad;
  int64_t index;
};

// Per-segment seed for the segmented walk (16 bytes).
struct Seed {
  int32_t gate;      // gate holding the segment's first record
  int32_t t_prev;    // time of the group before the first record's group (0 at gate start)
  uint8_t x;         // state just before the first record
  uint8_t p;         // state before the first record's timestamp group
  uint8_t flags;     // kSeed* bits
  uint8_t pad0;
  int32_t pad1;
};
constexpr uint8_t kSeedGateStart = 1;   // first record starts its gate
constexpr uint8_t kSeedGroupHead = 2;   // first record starts its timestamp group
constexpr uint8_t kSeedUnresolved = 4;  // x / p still partial (keep masks pending)

struct WindowView {
  const int64_t* offsets;    // [G+1]
  const uint2* rec;          // [E] {t, meta}
  const uint8_t* init;       // [G]
  int64_t n_events;
  int32_t window_ps;
};

struct Outputs {
  double* e_leak;            // [G]
  double* e_int;             // [G]
  double* e_sw;              // [G]
  uint8_t* final_state;      // [G]
  float2* bins;              // [n_bins]
  double* l0;                // [1] sum over gates of P_leak(init) (nW)
  DevError* err;
  int32_t bin_ps;
  uint32_t bin_magic;        // t / bin_ps == __umulhi(t, magic) >> shift for t < 2^31
  uint32_t bin_shift;
  int32_t n_bins;
};

// ------------------------------------------------------------------ device helpers
__device__ __forceinline__ void report_error(DevError* err, int code, int64_t index) {
  if (atomicCAS(&err->code, 0, code) == 0) err->index = index;
}

__device__ __forceinline__ int segment_of(const float* axis, int n, float x) {
  int i = 0;
#pragma unroll
  for (int k = 1; k < kMaxAxis - 1; ++k)
    if (k < n - 1) i += (x >= axis[k]) ? 1 : 0;
  return i;
}

// Side-input bits: input pins other than `pin`, compacted in pin order.
__device__ __forceinline__ uint32_t side_bits(uint32_t S, uint32_t pin, uint32_t n_in) {
  uint32_t in_mask = (1u << n_in) - 1u;
  uint32_t low = S & ((1u << pin) - 1u);
  uint32_t high = (S >> 1) & ~((1u << pin) - 1u);
  return (low | high) & (in_mask >> 1);
}

// Shared-memory copy of the (scaled) library.  Layout in dynamic smem:
// [axes: 4 x kMaxAxis floats][tab: n_tab_floats][leak: n_leak][cells].
struct SmemLib {
  const float* axes;  // slew axis, load axis, slew 1/width, load 1/width
  const float* tab;
  const float* leak;
  const CellInfo* cells;
};

// Bilinear NLDM interpolation of one table at (slew, load); the located
// segment is clamped to the axis so that outside points extrapolate linearly.
__device__ __forceinline__ float bilinear(const LibView& L, const SmemLib& sl, const float* table, float slew,
                                          float load) {
  const float* sa = sl.axes;
  const float* la = sl.axes + kMaxAxis;
  int i = segment_of(sa, L.ns, slew);
  int j = segment_of(la, L.nl, load);
  float fs = (slew - sa[i]) * sa[2 * kMaxAxis + i];
  float fl = (load - la[j]) * la[2 * kMaxAxis + j];
  const float* r0 = table + i * L.nl + j;
  const float* r1 = r0 + L.nl;
  float a = fmaf(fl, r0[1] - r0[0], r0[0]);
  float b = fmaf(fl, r1[1] - r1[0], r1[0]);
  return fmaf(fs, b - a, a);
}

// floor(t / bin_ps) for 0 <= t < 2^31: the multiply-high estimate is q or
// q - 1 (magic = min(floor(2^(32+s) / d), 2^32 - 1), s = floor(log2 d)), and
// one correction step makes it exact.
__device__ __forceinline__ uint32_t bin_of(const Outputs& O, uint32_t t) {
  uint32_t b = __umulhi(t, O.bin_magic) >> O.bin_shift;
  return b + (((b + 1u) * (uint32_t)O.bin_ps <= t) ? 1u : 0u);
}

// Fire-and-forget vector add of {energy, leakage step} into one bin.
__device__ __forceinline__ void red_bin(float2* bins, uint32_t b, float e, float dp) {
  float2* p = bins + b;
  asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(e), "f"(dp) : "memory");
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

size_t smem_lib_bytes(const LibView& L);

// Stage the library into dynamic shared memory, applying the per-cell
// scales; all threads of the block participate; ends with __syncthreads().
__device__ __forceinline__ SmemLib stage_library(const LibView& L, unsigned char* smem) {
  float* axes = reinterpret_cast<float*>(smem);
  float* tab = axes + 4 * kMaxAxis;
  float* leak = tab + (size_t)L.n_tables * L.tsize;
  CellInfo* cells = reinterpret_cast<CellInfo*>(leak + ((L.n_leak + 3) & ~3));
  int nt = L.n_tables * L.tsize;
  for (int k = threadIdx.x; k < nt; k += blockDim.x) tab[k] = L.tab[k] * L.escale[L.table_cell[k / L.tsize]];
  for (int k = threadIdx.x; k < L.n_leak; k += blockDim.x) leak[k] = L.leak[k] * L.lscale[L.leak_cell[k]];
  for (int k = threadIdx.x; k < L.n_cells; k += blockDim.x) cells[k] = L.cells[k];
  if (threadIdx.x < kMaxAxis) {
    axes[threadIdx.x] = L.slew_axis[threadIdx.x];
    axes[kMaxAxis + threadIdx.x] = L.load_axis[threadIdx.x];
    axes[2 * kMaxAxis + threadIdx.x] = L.slew_rw[threadIdx.x];
    axes[3 * kMaxAxis + threadIdx.x] = L.load_rw[threadIdx.x];
  }
  __syncthreads();
  return SmemLib{axes, tab, leak, cells};
}

// ------------------------------------------------------------------ launchers (host)
// Each returns cudaError_t of the launch.
cudaError_t launch_gate_pass(const LibView& L, const NetView& N, const WindowView& W, const Outputs& O,
                             cudaStream_t st);
cudaError_t launch_walk_per_gate(const LibView& L, const NetView& N, const WindowView& W, const Outputs& O,
                                 int block, cudaStream_t st);
cudaError_t launch_merge(const Outputs& O, double* waveform_w, double* tile_sums, int n_tiles, cudaStream_t st);
int merge_tiles(int n_bins);

}  // namespace gtp
