// The paper's GPU schemes as comparator kernels (see gtp_scheme.cuh).  They
// compute what the engine's walk computes (the same readings: pre-group state
// for lookups, switching energy on every output-pin event, glitch detection
// per pin and clock cycle), accumulate in FP64 with atomics as the paper
// does, and are written for clarity of the scheme, not for speed.
#include "gtp_scheme.cuh"

namespace gtp {

namespace {

constexpr uint32_t kNone = 0xFFFFFFFFu;

__device__ __forceinline__ uint32_t ev_time(uint32_t x) { return x & 0x7FFFFFFFu; }
__device__ __forceinline__ uint32_t ev_val(uint32_t x) { return x >> 31; }

// First index in [lo, hi) of a stream whose time is >= t (hi if none).
__device__ __forceinline__ int64_t first_at_or_after(const uint32_t* __restrict__ ev, int64_t lo, int64_t hi,
                                                     uint32_t t) {
  while (lo < hi) {
    const int64_t mid = lo + ((hi - lo) >> 1);
    if (ev_time(ev[mid]) < t) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ int axis_segment(const float* axis, int n, float x) {
  int i = 0;
  while (i < n - 2 && x >= axis[i + 1]) ++i;
  return i;
}

// Bilinear NLDM value of one ns x nl table (slew-major) at (slew s, load C),
// located by the lower knot and extrapolated linearly outside the axes.
__device__ float lut_energy(const LibView& L, const float* __restrict__ tab, float s, float C) {
  const int i = axis_segment(L.slew_axis, L.ns, s), j = axis_segment(L.load_axis, L.nl, C);
  const float fs = (s - L.slew_axis[i]) * L.slew_rw[i];
  const float fl = (C - L.load_axis[j]) * L.load_rw[j];
  const float* p = tab + i * L.nl + j;
  const float a0 = __ldg(p), a1 = __ldg(p + 1), b0 = __ldg(p + L.nl), b1 = __ldg(p + L.nl + 1);
  const float lo = fmaf(fl, a1 - a0, a0), hi = fmaf(fl, b1 - b0, b0);
  return fmaf(fs, hi - lo, lo);
}

// Internal-power table of (cell, pin, edge) at side-input state `side`.
// SIPL (Sec. 4.1) indexes it; without SIPL the group's state patterns are
// scanned, pin by pin, until one matches (Sec. 3.1: O(n_pin *
// n_sd) per lookup).
template <bool SIPL>
__device__ int64_t int_table(const SchemeArgs& A, const CellInfo& ci, uint32_t pin, uint32_t edge, uint32_t side) {
  const int64_t base = (int64_t)ci.tab_base + ((int64_t)(pin * 2u + edge) << (ci.n_in - 1));
  if (SIPL) return base + side;
  const int n_side = ci.n_in - 1;
  const int64_t n_sd = 1ll << n_side;
  for (int64_t k = 0; k < n_sd; ++k) {
    const uint32_t pat = A.pat_int[base + k];
    bool match = true;
    for (int q = 0; q < n_side; ++q) match = match && ((pat >> q) & 1u) == ((side >> q) & 1u);
    if (match) return base + k;
  }
  return base;  // a complete pattern set always matches
}

// Leakage power (nW, scaled) of the cell at full state S, by SIPL or by the
// traversal of the cell's leakage state patterns.
template <bool SIPL>
__device__ float leak_power(const LibView& L, const SchemeArgs& A, const CellInfo& ci, uint32_t S, float lsc) {
  if (SIPL) return __ldg(L.leak + ci.leak_base + S) * lsc;
  const int n_pins = ci.n_in + 1;
  const int n_sd = 1 << n_pins;
  for (int k = 0; k < n_sd; ++k) {
    const uint32_t pat = A.pat_leak[ci.leak_base + k];
    bool match = true;
    for (int q = 0; q < n_pins; ++q) match = match && ((pat >> q) & 1u) == ((S >> q) & 1u);
    if (match) return __ldg(L.leak + ci.leak_base + k) * lsc;
  }
  return 0.f;
}

// Dynamic energy (fJ) of an event on `pin` with new value `val` at the
// pre-group state S: internal energy for an input pin, 0.5 C Vdd^2 for the
// output pin.
template <bool SIPL>
__device__ float event_energy(const LibView& L, const NetView& N, const SchemeArgs& A, const CellInfo& ci,
                              uint32_t cell, int64_t g, uint32_t pin, uint32_t val, uint32_t S, float C) {
  if (pin >= (uint32_t)ci.n_in) return L.half_v2 * C;
  const int64_t ti = int_table<SIPL>(A, ci, pin, val, side_bits(S, pin, (uint32_t)ci.n_in));
  const float s = __ldg(N.slew + ((size_t)g * N.stride + pin) * 2 + val);
  return lut_energy(L, L.tab + ti * L.tsize, s, C) * __ldg(L.escale + cell);
}

// Rise + fall transition time of a pin (glitch scaling ratio).
__device__ __forceinline__ float slew_sum(const NetView& N, const CellInfo& ci, int64_t g, uint32_t pin) {
  const float* s = pin < (uint32_t)ci.n_in ? N.slew + ((size_t)g * N.stride + pin) * 2 : N.out_slew + 2 * g;
  return __ldg(s) + __ldg(s + 1);
}

// Leakage power P (nW) held over [a, b) into every bin it overlaps, one
// atomic per bin (the cycle-side work of Sec. 2.4.2); returns the energy (fJ).
__device__ double leak_into_bins(double* ebins, float P, uint32_t a, uint32_t b, uint32_t bin_ps) {
  double tot = 0.0;
  uint32_t k = a / bin_ps;
  for (uint32_t lo = a; lo < b; ++k) {
    const uint32_t end = min((k + 1u) * bin_ps, b);
    const double e = (double)P * (double)(end - lo) * 1e-6;
    atomicAdd(ebins + k, e);
    tot += e;
    lo = end;
  }
  return tot;
}

__device__ __forceinline__ double* row_of(const SchemeArgs& A, int64_t g) {
  return A.R + ((size_t)g * kSchemeTpb + threadIdx.x) * 4;
}

// ------------------------------------------------------------------ input form
__global__ void k_pin_streams(LibView L, NetView N, const WinDesc* __restrict__ wins, PinStreams ps, DevError* err) {
  const WinDesc& W = wins[0];
  const int32_t T = W.window_ps;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < N.n_gates;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = W.offsets[g], b = W.offsets[g + 1];
    const uint32_t n_pins = (uint32_t)L.cells[N.cell[g]].n_in + 1u;
    int64_t cnt[kStreamSlots];
    for (int p = 0; p < kStreamSlots; ++p) cnt[p] = 0;
    uint32_t S = W.init[g];
    bool bad = false;
    if (S >> n_pins) {
      report_error(err, GTP_ERANGE, -1 - g);
      bad = true;
    }
    int32_t tp = 0;
    for (int64_t i = a; i < b && !bad; ++i) {
      const uint2 r = W.rec[i];
      const int32_t t = (int32_t)r.x;
      const uint32_t pin = r.y & 0xFu, val = (r.y >> 4) & 1u;
      int code = 0;
      if (t < 0 || t >= T || (r.y >> 5) != 0u || pin >= n_pins) code = GTP_ERANGE;
      else if (t < tp) code = GTP_EORDER;
      else if (((S >> pin) & 1u) == val) code = GTP_ENOTOGGLE;
      if (code) {
        report_error(err, code, i);
        bad = true;
        break;
      }
      S ^= 1u << pin;
      tp = t;
      ++cnt[pin];
    }
    int64_t o = a, cur[kStreamSlots];
    for (int p = 0; p <= kStreamSlots; ++p) {
      ps.off[g * 9 + p] = o;
      if (p < kStreamSlots) {
        cur[p] = o;
        if (!bad) o += cnt[p];
      }
    }
    if (bad) continue;
    for (int64_t i = a; i < b; ++i) {
      const uint2 r = W.rec[i];
      const uint32_t pin = r.y & 0xFu;
      const int64_t k = cur[pin]++;
      ps.ev[k] = r.x | (((r.y >> 4) & 1u) << 31);
      ps.slot[k] = (uint32_t)g * kStreamSlots + pin;
    }
  }
}

// ------------------------------------------------------------------ Naive-D
// One thread per event (Sec. 2.4.1): reconstruct the gate state before the
// event by a binary search in each pin's stream, look up and interpolate the
// energy, detect a glitch from the previous event of the pin's stream, add
// the energy to its bin and to the gate's reduction row.
template <bool SIPL>
__global__ void __launch_bounds__(kSchemeTpb) k_naive_d(LibView L, NetView N, SchemeArgs A, int64_t n_events) {
  const WinDesc& W = *A.win;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_events) return;
  const uint32_t slot = A.ps.slot[i];
  const int64_t g = slot / kStreamSlots;
  const uint32_t pin = slot % kStreamSlots;
  const uint32_t x = A.ps.ev[i];
  const uint32_t t = ev_time(x), val = ev_val(x);
  const uint32_t cell = (uint32_t)N.cell[g];
  const CellInfo ci = L.cells[cell];
  const int64_t* off = A.ps.off + g * 9;
  uint32_t S = 0u;
  if (pin < (uint32_t)ci.n_in) {
    const uint32_t init = W.init[g];
    for (int q = 0; q <= ci.n_in; ++q) {
      const int64_t lo = off[q];
      const int64_t k = first_at_or_after(A.ps.ev, lo, off[q + 1], t);
      S |= (k > lo ? ev_val(A.ps.ev[k - 1]) : (init >> q) & 1u) << q;
    }
  }
  float E = event_energy<SIPL>(L, N, A, ci, cell, g, pin, val, S, N.load[g]);
  int kind = pin < (uint32_t)ci.n_in ? 1 : 2;
  if (N.clock_ps > 0 && i > off[pin]) {
    const uint32_t tp = ev_time(A.ps.ev[i - 1]);
    if (tp >= cycle_start(t, N.clock_ps, N.clock_magic, N.clock_shift)) {
      E *= glitch_ratio(t - tp, slew_sum(N, ci, g, pin));
      kind = 3;
    }
  }
  atomicAdd(A.ebins + bin_of(t, W.bin_magic, W.bin_shift, (uint32_t)W.bin_ps), (double)E);
  atomicAdd(row_of(A, g) + kind, (double)E);
}

// ------------------------------------------------------------------ per-thread windows
// State of gate g at t0 (each pin's last event before t0) and each pin's
// stream range inside [t0, t1).
struct WindowCursor {
  int64_t cur[kStreamSlots], end[kStreamSlots];
  uint32_t last[kStreamSlots];  // each pin's last event time before t0 (kNone: none)
  uint32_t S;
};

__device__ __forceinline__ void open_window(const SchemeArgs& A, const WinDesc& W, int64_t g, int n_pins,
                                            uint32_t t0, uint32_t t1, WindowCursor& c) {
  const int64_t* off = A.ps.off + g * 9;
  const uint32_t init = W.init[g];
  c.S = 0u;
  for (int q = 0; q < n_pins; ++q) {
    const int64_t lo = off[q], hi = off[q + 1];
    c.cur[q] = first_at_or_after(A.ps.ev, lo, hi, t0);
    c.end[q] = first_at_or_after(A.ps.ev, c.cur[q], hi, t1);
    const bool before = c.cur[q] > lo;
    c.S |= (before ? ev_val(A.ps.ev[c.cur[q] - 1]) : (init >> q) & 1u) << q;
    c.last[q] = before ? ev_time(A.ps.ev[c.cur[q] - 1]) : kNone;
  }
}

// Earliest unprocessed event time of the window (k-way merge), kNone at its end.
__device__ __forceinline__ uint32_t next_time(const SchemeArgs& A, const WindowCursor& c, int n_pins) {
  uint32_t tc = kNone;
  for (int q = 0; q < n_pins; ++q)
    if (c.cur[q] < c.end[q]) tc = min(tc, ev_time(A.ps.ev[c.cur[q]]));
  return tc;
}

// Apply the events at tc to the state and advance past them.
__device__ __forceinline__ void apply_group(const SchemeArgs& A, WindowCursor& c, int n_pins, uint32_t tc) {
  for (int q = 0; q < n_pins; ++q)
    while (c.cur[q] < c.end[q] && ev_time(A.ps.ev[c.cur[q]]) == tc) {
      c.S = (c.S & ~(1u << q)) | (ev_val(A.ps.ev[c.cur[q]]) << q);
      ++c.cur[q];
    }
}

// Naive-L's work for one gate and window [t0, t1) (Sec. 2.4.2): leakage of
// every inter-event interval into the bins it overlaps.
template <bool SIPL>
__device__ void leak_window(const LibView& L, const NetView& N, const SchemeArgs& A, const WinDesc& W, int64_t g,
                            uint32_t t0, uint32_t t1) {
  const uint32_t cell = (uint32_t)N.cell[g];
  const CellInfo ci = L.cells[cell];
  const int n_pins = ci.n_in + 1;
  const float lsc = __ldg(L.lscale + cell);
  const uint32_t bin_ps = (uint32_t)W.bin_ps;
  WindowCursor c;
  open_window(A, W, g, n_pins, t0, t1, c);
  float P = leak_power<SIPL>(L, A, ci, c.S, lsc);
  uint32_t tp = t0;
  double El = 0.0;
  for (uint32_t tc = next_time(A, c, n_pins); tc != kNone; tc = next_time(A, c, n_pins)) {
    El += leak_into_bins(A.ebins, P, tp, tc, bin_ps);
    apply_group(A, c, n_pins, tc);
    P = leak_power<SIPL>(L, A, ci, c.S, lsc);
    tp = tc;
  }
  El += leak_into_bins(A.ebins, P, tp, t1, bin_ps);
  if (t1 == (uint32_t)W.window_ps) W.final_state[g] = (uint8_t)c.S;
  atomicAdd(row_of(A, g), El);
}

// The fused kernel's work for one gate and window [t0, t1) (Algorithm 1):
// the state and each pin's previous event time are set up once, then each
// timestamp of the merged streams adds the leakage since the previous one,
// the dynamic energy of its events at the pre-group state (glitches scaled),
// and updates the state.
__device__ void fused_window(const LibView& L, const NetView& N, const SchemeArgs& A, const WinDesc& W, int64_t g,
                             uint32_t t0, uint32_t t1) {
  const uint32_t cell = (uint32_t)N.cell[g];
  const CellInfo ci = L.cells[cell];
  const int n_pins = ci.n_in + 1;
  const float lsc = __ldg(L.lscale + cell);
  const float C = N.load[g];
  const uint32_t bin_ps = (uint32_t)W.bin_ps;
  WindowCursor c;
  open_window(A, W, g, n_pins, t0, t1, c);
  float P = leak_power<true>(L, A, ci, c.S, lsc);
  uint32_t tp = t0;
  double sum[4] = {0.0, 0.0, 0.0, 0.0};
  for (uint32_t tc = next_time(A, c, n_pins); tc != kNone; tc = next_time(A, c, n_pins)) {
    sum[0] += leak_into_bins(A.ebins, P, tp, tc, bin_ps);
    const uint32_t bin = bin_of(tc, W.bin_magic, W.bin_shift, bin_ps);
    const uint32_t cyc = N.clock_ps > 0 ? cycle_start(tc, N.clock_ps, N.clock_magic, N.clock_shift) : 0u;
    for (int q = 0; q < n_pins; ++q) {
      for (int64_t k = c.cur[q]; k < c.end[q]; ++k) {
        const uint32_t x = A.ps.ev[k];
        if (ev_time(x) != tc) break;
        float E = event_energy<true>(L, N, A, ci, cell, g, (uint32_t)q, ev_val(x), c.S, C);
        int kind = q < ci.n_in ? 1 : 2;
        if (N.clock_ps > 0) {
          if (c.last[q] != kNone && c.last[q] >= cyc) {
            E *= glitch_ratio(tc - c.last[q], slew_sum(N, ci, g, (uint32_t)q));
            kind = 3;
          }
          c.last[q] = tc;
        }
        atomicAdd(A.ebins + bin, (double)E);
        sum[kind] += E;
      }
    }
    apply_group(A, c, n_pins, tc);
    P = leak_power<true>(L, A, ci, c.S, lsc);
    tp = tc;
  }
  sum[0] += leak_into_bins(A.ebins, P, tp, t1, bin_ps);
  if (t1 == (uint32_t)W.window_ps) W.final_state[g] = (uint8_t)c.S;
  double* row = row_of(A, g);
  for (int k = 0; k < 4; ++k)
    if (sum[k] != 0.0) atomicAdd(row + k, sum[k]);
}

// Naive-L: one thread per gate and window of ncyc_fix bins (Sec. 2.4.2).
template <bool SIPL>
__global__ void __launch_bounds__(kSchemeTpb) k_naive_l(LibView L, NetView N, SchemeArgs A, int64_t thr_per_gate,
                                                         int64_t total) {
  const WinDesc& W = *A.win;
  const int64_t span = (int64_t)A.ncyc_fix * W.bin_ps;
  for (int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; id < total; id += (int64_t)gridDim.x * blockDim.x) {
    const int64_t g = id / thr_per_gate, tau = id % thr_per_gate;
    const int64_t t0 = tau * span;
    const int64_t t1 = t0 + span < W.window_ps ? t0 + span : W.window_ps;
    leak_window<SIPL>(L, N, A, W, g, (uint32_t)t0, (uint32_t)t1);
  }
}

// Event-density-aware partitioning (Sec. 4.2): the blocks of gate g cover
// its windows of ncyc[g] bins, thread tau taking window tau.  FUSED: the
// fused kernel (Algorithm 1); otherwise Naive-L's leakage work.
template <bool FUSED>
__global__ void __launch_bounds__(kSchemeTpb) k_density(LibView L, NetView N, SchemeArgs A) {
  const WinDesc& W = *A.win;
  const int64_t b = blockIdx.x;
  const int32_t g = A.blk_gate[b];
  const int64_t tau = (b - A.blk_first[g]) * kSchemeTpb + threadIdx.x;
  const int64_t ncyc = A.ncyc[g];
  if (tau * ncyc >= (int64_t)W.n_bins) return;
  const int64_t span = ncyc * W.bin_ps;
  const int64_t t0 = tau * span;
  const int64_t t1 = t0 + span < W.window_ps ? t0 + span : W.window_ps;
  if (FUSED) fused_window(L, N, A, W, g, (uint32_t)t0, (uint32_t)t1);
  else leak_window<true>(L, N, A, W, g, (uint32_t)t0, (uint32_t)t1);
}

// Second phase of the reduction (Sec. 4.4): each gate's rows summed serially
// into its results; the rows are cleared for the next run.
__global__ void k_reduce_rows(SchemeArgs A, int64_t n_gates) {
  const WinDesc& W = *A.win;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n_gates; g += (int64_t)gridDim.x * blockDim.x) {
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    double* rows = A.R + (size_t)g * kSchemeTpb * 4;
    for (int r = 0; r < kSchemeTpb; ++r)
      for (int k = 0; k < 4; ++k) {
        s[k] += rows[r * 4 + k];
        rows[r * 4 + k] = 0.0;
      }
    W.e_leak[g] = s[0];
    W.e_int[g] = s[1];
    W.e_sw[g] = s[2];
    if (W.e_gl) W.e_gl[g] = s[3];
  }
}

__global__ void k_scheme_wave(SchemeArgs A) {
  const WinDesc& W = *A.win;
  const double to_w = 1e-3 / (double)W.bin_ps;
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < W.n_bins; b += (int64_t)gridDim.x * blockDim.x)
    if (W.wave) W.wave[b] = A.ebins[b] * to_w;
}

}  // namespace

cudaError_t launch_pin_streams(const LibView& L, const NetView& N, const WinDesc* win, PinStreams ps, DevError* err,
                               cudaStream_t st) {
  int64_t blocks = (N.n_gates + 127) / 128;
  if (blocks > 65536) blocks = 65536;
  k_pin_streams<<<(unsigned)(blocks < 1 ? 1 : blocks), 128, 0, st>>>(L, N, win, ps, err);
  return cudaGetLastError();
}

cudaError_t launch_scheme(int scheme, const LibView& L, const NetView& N, const SchemeArgs& A, int64_t n_events,
                          int32_t n_bins, cudaStream_t st) {
  const int64_t G = N.n_gates;
  if (scheme == kSchemeFused || scheme == kSchemeDensity) {
    if (A.n_blocks > 0x7FFFFFFFll) return cudaErrorInvalidConfiguration;
  }
  if (scheme == kSchemeFused) {
    if (A.n_blocks > 0) k_density<true><<<(unsigned)A.n_blocks, kSchemeTpb, 0, st>>>(L, N, A);
  } else {
    if (n_events > 0) {
      const int64_t blocks = (n_events + kSchemeTpb - 1) / kSchemeTpb;
      if (blocks > 0x7FFFFFFFll) return cudaErrorInvalidConfiguration;
      if (scheme == kSchemeNaive) k_naive_d<false><<<(unsigned)blocks, kSchemeTpb, 0, st>>>(L, N, A, n_events);
      else k_naive_d<true><<<(unsigned)blocks, kSchemeTpb, 0, st>>>(L, N, A, n_events);
    }
    if (scheme == kSchemeDensity) {
      if (A.n_blocks > 0) k_density<false><<<(unsigned)A.n_blocks, kSchemeTpb, 0, st>>>(L, N, A);
    } else {
      const int64_t thr = (n_bins + A.ncyc_fix - 1) / A.ncyc_fix;
      const int64_t total = G * thr;
      int64_t blocks = (total + kSchemeTpb - 1) / kSchemeTpb;
      if (blocks > (1ll << 30)) blocks = 1ll << 30;
      if (blocks > 0) {
        if (scheme == kSchemeNaive) k_naive_l<false><<<(unsigned)blocks, kSchemeTpb, 0, st>>>(L, N, A, thr, total);
        else k_naive_l<true><<<(unsigned)blocks, kSchemeTpb, 0, st>>>(L, N, A, thr, total);
      }
    }
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int64_t rb = (G + 255) / 256;
  if (rb > 65536) rb = 65536;
  k_reduce_rows<<<(unsigned)(rb < 1 ? 1 : rb), 256, 0, st>>>(A, G);
  int64_t wb = ((int64_t)n_bins + 255) / 256;
  if (wb > 65536) wb = 65536;
  k_scheme_wave<<<(unsigned)(wb < 1 ? 1 : wb), 256, 0, st>>>(A);
  return cudaGetLastError();
}

}  // namespace gtp
