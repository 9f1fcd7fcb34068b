// Interpolation coordinates, gate pass, one-thread-per-gate walk, the FP64
// bin merge, and the adjoint's gradient prefix.
//
// Leakage in the waveform uses a step representation: the design's leakage
// power is a step function of time, L(t) = L0 + sum_k dP_k [t >= t_k], where
// L0 = sum over gates of P_leak(initial state) and dP_k is the change of one
// gate's leakage power at the end of its timestamp group k.  A step at t_k
// in bin b contributes dP_k * ((b+1)*bin_ps - t_k) to bin b (added to the bin's
// energy accumulator) and dP_k * bin_ps to every later bin (recorded in the
// bin's step accumulator and applied by an exclusive FP64 prefix sum).  This
// gives the same per-bin leakage energy as splitting every inter-event
// interval over the bins it overlaps (Sec. 2.4.2), without touching the bins
// in between.
#include <cstdio>

#include "gtp_walk.cuh"

namespace gtp {

namespace {

__device__ __forceinline__ int segment_of(const float* axis, int n, float x) {
  int i = 0;
  while (i < n - 2 && x >= axis[i + 1]) ++i;
  return i;
}

// Window of a global index given ascending bases (n_win + 1 entries).
__device__ __forceinline__ int window_of(const int64_t* base, int n_win, int64_t x) {
  int lo = 0, hi = n_win - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (base[mid] <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}

}  // namespace

// ------------------------------------------------------------------ lookup points and per-gate energy tables
// The NLDM lookup point of every (gate, input pin, edge) is static: its slew
// segment and fraction and the gate's load segment and fraction are located
// once per netlist, load or scale change (with the table element and the
// switching energy) into the gate's event descriptors, instead of once per
// event.  Descriptor (pin p, edge e) of gate g is desc[g * dstride + 2p + e];
// pins from the cell's output on hold the switching energy 0.5 * C * Vdd^2
// (Eq. 1).
//
// For each gate whose cell has at most kGateTabMaxIn inputs, the same pass
// evaluates every (input pin, edge, side state) lookup at the gate's slews
// and load, i.e. the bilinear NLDM value of Sec. 2.2.1 on the state-indexed
// table of Sec. 4.1, and the switching energy of its output.  Entry
// (pin << n_in) | s, with s the input-pin state before the event: the pin's
// own bit in s is its old value (so the edge is its complement) and the other
// bits are the side state; the output pin is pin n_in.  Forward table:
// energies times escale, output slots 0.5 * C * Vdd^2.  Adjoint table:
// unscaled energies (output slots 0), then their load derivatives (the slope
// of the located load segment; output slots 0.5 * Vdd^2).
//
// A warp takes four consecutive gates at a time.  First its lanes compute
// the four gates' descriptors, one (gate, pin, edge) a lane (the descriptors
// of consecutive gates are consecutive, so the writes coalesce), from the
// gates' cells, loads and slews (loaded together; cell data in shared memory)
// into a shared-memory copy; then, gate by gate, lane k of the table reads
// its entry's descriptor there and interpolates.  Every gate costs one round
// of independent loads.  Null outputs are not written.
__device__ __forceinline__ int segment_bsearch(const float* axis, int n, float x) {
  // the last knot i in [0, n - 2] with axis[i] <= x (0 below the axis): the loop of segment_of, branch-free
  int i = 0;
#pragma unroll
  for (int step = 8; step > 0; step >>= 1)
    if (i + step <= n - 2 && x >= axis[i + step]) i += step;
  return i;
}

__global__ void __launch_bounds__(256, 4) k_gate_prep(LibView L, NetView N, uint4* __restrict__ desc,
                                                   float* __restrict__ gtab, float* __restrict__ gbwd) {
  constexpr int kG = 4;
  constexpr int kMaxDesc = 2 * (GTP_MAX_PINS + 1);
  __shared__ float ax[4 * kMaxAxis];
  __shared__ CellInfo cells[256];  // cell indices are bytes in the library's tables
  __shared__ float esc[256];
  __shared__ uint4 sdesc[8][kG * kMaxDesc];  // per warp: its four gates' descriptors
  __shared__ int32_t scell[8][kG];
  for (int i = threadIdx.x; i < kMaxAxis; i += blockDim.x) {
    ax[i] = L.slew_axis[i];
    ax[kMaxAxis + i] = L.load_axis[i];
    ax[2 * kMaxAxis + i] = L.slew_rw[i];
    ax[3 * kMaxAxis + i] = L.load_rw[i];
  }
  for (int i = threadIdx.x; i < L.n_cells && i < 256; i += blockDim.x) {
    cells[i] = L.cells[i];
    esc[i] = L.escale[i];
  }
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31u, wib = threadIdx.x >> 5;
  uint4* const sd = sdesc[wib];
  const int ds = N.dstride;
  const int n_items = kG * ds;
  const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t g0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * kG; g0 < N.n_gates;
       g0 += n_warps * kG) {
    // descriptors of gates g0 .. g0 + 3: item i is gate i / ds, (pin, edge) i % ds
    for (int i = (int)lane; i < n_items; i += 32) {
      const int k = (i >= ds) + (i >= 2 * ds) + (i >= 3 * ds);
      const int idx = i - k * ds, p = idx >> 1, e = idx & 1;
      const int64_t g = g0 + k;
      if (g >= N.n_gates) continue;
      const int32_t c = __ldg(N.cell + g);
      const float C = __ldg(N.load + g);
      const float sl = p < N.stride ? __ldg(N.slew + (size_t)g * N.stride * 2 + idx) : 0.f;
      if (idx == 0) scell[wib][k] = c;
      const CellInfo ci = cells[c];
      const int n_in = ci.n_in;
      const int j = segment_bsearch(ax + kMaxAxis, L.nl, C);
      const float fl = (C - ax[kMaxAxis + j]) * ax[3 * kMaxAxis + j];
      const uint32_t hi_bits = ((uint32_t)c << 16) | ((uint32_t)j << 25);
      uint4 d;
      if (p < n_in) {
        const int si = segment_bsearch(ax, L.ns, sl);
        const uint32_t tab = (uint32_t)(ci.tab_base + ((p * 2 + e) << (n_in - 1))) * (uint32_t)L.tsize +
                             (uint32_t)(si * L.nl + j);
        d = make_uint4(__float_as_uint((sl - ax[si]) * ax[2 * kMaxAxis + si]), __float_as_uint(fl), tab | hi_bits,
                       __float_as_uint(ax[3 * kMaxAxis + j]));
      } else {  // output pin (and any pin past it): switching energy
        d = make_uint4(0u, 0u, ((uint32_t)ci.tab_base * (uint32_t)L.tsize) | hi_bits | (1u << 24),
                       __float_as_uint(L.half_v2 * C));
      }
      sd[i] = d;
      if (desc) desc[(size_t)g0 * ds + i] = d;
    }
    if (!gtab && !gbwd) continue;
    __syncwarp();
#pragma unroll
    for (int k = 0; k < kG; ++k) {
      const int64_t g = g0 + k;
      if (g >= N.n_gates) break;
      const int32_t c = scell[wib][k];
      const uint32_t n_in = (uint32_t)cells[c].n_in;
      if (n_in > (uint32_t)kGateTabMaxIn || lane >= ((n_in + 1u) << n_in)) continue;
      const uint32_t pin = lane >> n_in, s = lane & ((1u << n_in) - 1u);
      const uint32_t val = pin < n_in ? (((s >> pin) & 1u) ^ 1u) : 0u;  // own bit: the value before the edge
      const uint4 q = sd[k * ds + (int)(pin * 2u + val)];                 // pin <= n_in <= stride
      float eu, ed, ef;
      if (pin < n_in) {
        const float* tp = L.tab + (q.z & 0xFFFFu) + side_bits(s, pin, n_in) * (uint32_t)L.tsize;
        const float a0 = __ldg(tp), a1 = __ldg(tp + 1), b0 = __ldg(tp + L.nl), b1 = __ldg(tp + L.nl + 1);
        const float fl = __uint_as_float(q.y), fs = __uint_as_float(q.x);
        const float lo = fmaf(fl, a1 - a0, a0), hi = fmaf(fl, b1 - b0, b0);
        eu = fmaf(fs, hi - lo, lo);
        ed = fmaf(fs, (b1 - b0) - (a1 - a0), a1 - a0) * __uint_as_float(q.w);
        ef = eu * esc[c];
      } else {
        eu = 0.f;
        ed = L.half_v2;
        ef = __uint_as_float(q.w);  // the output pin's descriptor: 0.5 * C * Vdd^2
      }
      if (gtab) gtab[(size_t)g * kGateTab + lane] = ef;
      if (gbwd) {
        gbwd[(size_t)g * 2 * kGateTab + lane] = eu;
        gbwd[(size_t)g * 2 * kGateTab + kGateTab + lane] = ed;
      }
    }
    __syncwarp();  // the next gates' descriptors overwrite this copy
  }
}

cudaError_t launch_gate_prep(const LibView& L, const NetView& N, uint4* desc, float* gtab, float* gtab_bwd,
                             cudaStream_t st) {
  if (L.n_cells > 256 || N.dstride > 2 * (GTP_MAX_PINS + 1)) return cudaErrorInvalidValue;
  int64_t blocks = (N.n_gates + 31) / 32;  // 8 warps of 4 gates a block
  if (blocks > 16384) blocks = 16384;
  k_gate_prep<<<(unsigned)(blocks < 1 ? 1 : blocks), 256, 0, st>>>(L, N, desc, gtab, gtab_bwd);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ gate pass (adjoint)
// Adjoint of the gate pass: a gate without events leaks at its initial state
// over the whole window, so d L / d lscale[c] gains P0(init) * G(T) * 1e-6.
__global__ void k_gate_pass_bwd(LibView L, NetView N, const WinDesc* __restrict__ wins, double* __restrict__ cell_acc) {
  const WinDesc& W = wins[0];
  extern __shared__ double acc[];
  for (int c = threadIdx.x; c < L.n_cells; c += blockDim.x) acc[c] = 0.0;
  __syncthreads();
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < N.n_gates;
       g += (int64_t)gridDim.x * blockDim.x) {
    if (W.offsets[g + 1] != W.offsets[g]) continue;
    const int32_t c = N.cell[g];
    const CellInfo ci = L.cells[c];
    const uint32_t s0 = W.init[g] & ((2u << ci.n_in) - 1u);
    atomicAdd(acc + c, (double)L.leak[ci.leak_base + s0]);
  }
  __syncthreads();
  const double gT = (double)W.g_total * 1e-6;
  for (int c = threadIdx.x; c < L.n_cells; c += blockDim.x)
    if (acc[c] != 0.0) atomicAdd(cell_acc + L.n_cells + c, acc[c] * gT);
}

cudaError_t launch_gate_pass_bwd(const LibView& L, const NetView& N, const WinDesc* wins, double* cell_acc,
                                 cudaStream_t st) {
  int64_t blocks = (N.n_gates + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  k_gate_pass_bwd<<<(unsigned)(blocks < 1 ? 1 : blocks), 256, sizeof(double) * L.n_cells, st>>>(L, N, wins, cell_acc);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ one thread per gate
// The plain walk of Algorithm 1, one (window, gate) per thread: timestamp
// groups with lookups at the pre-group state, the state update after the
// group, leakage held between groups.  Kahan-compensated FP32 per-gate sums.
// With a clock, glitch detection as in the fused walk.  A simple
// cross-check of the segmented walk; it is not tuned.
__global__ void k_walk_per_gate(LibView L, NetView N, const WinDesc* __restrict__ wins, DevError* err) {
  extern __shared__ __align__(16) unsigned char smem[];
  const SmemLib sl = stage_library(L, smem, true);
  const WinDesc& W = wins[blockIdx.y];
  const float T = (float)W.window_ps;
  for (int64_t g = W.g0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < W.g1;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = W.offsets[g], b = W.offsets[g + 1];
    if (a == b) continue;
    const CellInfo ci = sl.cells[N.cell[g]];
    const uint32_t n_in = (uint32_t)ci.n_in, n_pins = n_in + 1;
    const float* leak = sl.leak + ci.leak_base;
    const uint4* dsc = N.desc + (size_t)g * N.dstride;
    uint32_t st = W.init[g] & ((2u << n_in) - 1u);
    float P = leak[st];
    int32_t t_prev = 0;
    Kahan El, Ei, Es, Eg;
    float4* const cb = W.cbins;
    uint32_t last[8];  // glitch detection: each pin's previous event time
    for (int p = 0; p < 8; ++p) last[p] = 0xFFFFFFFFu;
    bool bad = false;
    int64_t i = a;
    while (i < b) {
      const int32_t t = (int32_t)W.rec[i].x;
      if (t < 0 || t >= W.window_ps) { report_error(err, GTP_ERANGE, i); bad = true; break; }
      if (t < t_prev) { report_error(err, GTP_EORDER, i); bad = true; break; }
      El.add(P * (float)(t - t_prev) * 1e-6f);
      const uint32_t bin = bin_of((uint32_t)t, W.bin_magic, W.bin_shift, (uint32_t)W.bin_ps);
      uint32_t s_next = st;
      float e_bin = 0.f, c_int = 0.f, c_sw = 0.f, c_gl = 0.f;
      int64_t j = i;
      for (; j < b; ++j) {
        const uint2 r = W.rec[j];
        if ((int32_t)r.x != t) break;
        const uint32_t pin = r.y & 0xFu, val = (r.y >> 4) & 1u;
        if ((r.y >> 5) != 0u || pin >= n_pins) { report_error(err, GTP_ERANGE, j); bad = true; break; }
        if (((s_next >> pin) & 1u) == val) { report_error(err, GTP_ENOTOGGLE, j); bad = true; break; }
        s_next ^= 1u << pin;
        float E;
        const uint4 d = dsc[pin * 2 + val];
        if (pin < n_in) {
          const uint32_t side = side_bits(st, pin, n_in);
          const float* p = sl.tab + (d.z & 0xFFFFu) + side * (uint32_t)L.tsize;
          const float fl = __uint_as_float(d.y);
          const float lo = fmaf(fl, p[1] - p[0], p[0]);
          const float hi = fmaf(fl, p[L.nl + 1] - p[L.nl], p[L.nl]);
          E = fmaf(__uint_as_float(d.x), hi - lo, lo);
        } else {
          E = __uint_as_float(d.w);
        }
        bool glitch = false;
        if (N.clock_ps > 0) {  // Sec. 2.4.1: an earlier event on this pin in the same clock cycle
          const uint32_t tp = last[pin];
          last[pin] = (uint32_t)t;
          if (tp != 0xFFFFFFFFu && tp >= cycle_start((uint32_t)t, N.clock_ps, N.clock_magic, N.clock_shift)) {
            const float* sw = pin < n_in ? N.slew + ((size_t)g * N.stride + pin) * 2 : N.out_slew + 2 * g;
            E *= glitch_ratio((uint32_t)t - tp, sw[0] + sw[1]);
            glitch = true;
          }
        }
        if (glitch) {
          Eg.add(E);
          c_gl += E;
        } else if (pin < n_in) {
          Ei.add(E);
          c_int += E;
        } else {
          Es.add(E);
          c_sw += E;
        }
        e_bin += E;
      }
      if (bad) break;
      const float P_new = leak[s_next];
      const float dP = P_new - P;
      const float frac = (float)((int32_t)(bin + 1u) * W.bin_ps - t);
      if (cb && W.cpack) {
        red_cbin(cb, bin, c_int, c_sw, dP * frac * 1e-6f, dP);
      } else {
        red_bin(W.bins, bin, e_bin + dP * frac * 1e-6f, dP);
        if (cb) red_cbin(cb, bin, c_int, c_sw, c_gl, dP * frac * 1e-6f);
      }
      st = s_next;
      P = P_new;
      t_prev = t;
      i = j;
    }
    if (bad) continue;
    El.add(P * (T - (float)t_prev) * 1e-6f);
    W.e_leak[g] = El.value();
    W.e_int[g] = Ei.value();
    W.e_sw[g] = Es.value();
    if (W.e_gl) W.e_gl[g] = Eg.value();
    W.final_state[g] = (uint8_t)st;
  }
}

cudaError_t launch_walk_per_gate(const LibView& L, const NetView& N, const WinDesc* wins, int n_win,
                                 DevError* err, cudaStream_t st) {
  const size_t smem = smem_lib_bytes(L);
  cudaError_t e = cudaFuncSetAttribute(k_walk_per_gate, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int64_t blocks = (N.n_gates + 127) / 128;
  if (blocks > 4096) blocks = 4096;
  dim3 grid((unsigned)(blocks < 1 ? 1 : blocks), (unsigned)n_win);
  k_walk_per_gate<<<grid, 128, smem, st>>>(L, N, wins, err);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ reduction-rate probe
// n_red fire-and-forget float reductions of W floats (2: the walk's {energy,
// step} bin update; 4: the component runs' update) into places of an
// n_slots array picked by an integer mix of the reduction's number: the rate
// the L2 sustains for the walk's bin updates.
__device__ __forceinline__ uint32_t probe_mix(uint32_t x) {
  x = (x ^ 61u) ^ (x >> 16);
  x *= 9u;
  x ^= x >> 4;
  x *= 0x27d4eb2du;
  return x ^ (x >> 15);
}

template <int W>
static __global__ void k_red_probe(float4* __restrict__ slots, uint32_t n_slots, int64_t n_red) {
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n_red; r += nth) {
    const uint32_t i = probe_mix((uint32_t)r) % n_slots;
    if (W == 2)
      asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(reinterpret_cast<float2*>(slots) + i), "f"(1.f),
                   "f"(0.5f)
                   : "memory");
    else
      red_cbin(slots, i, 1.f, 0.5f, 0.25f, 0.125f);
  }
}

cudaError_t launch_red_probe(float4* slots, uint32_t n_slots, int width, int64_t n_red, int n_sm, cudaStream_t st) {
  const unsigned grid = (unsigned)(n_sm > 0 ? n_sm * 8 : 1024);
  if (width == 4) k_red_probe<4><<<grid, 256, 0, st>>>(slots, n_slots, n_red);
  else k_red_probe<2><<<grid, 256, 0, st>>>(slots, n_slots, n_red);
  return cudaGetLastError();
}

// The bin reductions of a window's own records, without the rest of the
// walk: lane l of a warp takes 8 consecutive records and issues one 8-byte
// reduction per distinct bin among them (the walk's dense-segment pattern),
// into 8-byte bins laid out as the walk's (`slots` holds at least the
// window's bin count of 16-byte slots).  Records out of the window are
// skipped.
static __global__ void k_red_replay(const uint2* __restrict__ rec, int64_t n, uint32_t T, uint32_t bin_ps,
                                    uint32_t magic, uint32_t shift, float4* __restrict__ slots) {
  constexpr int kPer = 8;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q * kPer < n; q += nth) {
    const int64_t r0 = q * kPer;
    uint32_t pb = 0xFFFFFFFFu;
    float pe = 0.f;
    for (int k = 0; k < kPer && r0 + k < n; ++k) {
      const uint32_t t = rec[r0 + k].x;
      if (t >= T) continue;
      const uint32_t b = bin_of(t, magic, shift, bin_ps);
      if (b != pb) {
        if (pb != 0xFFFFFFFFu) red_bin(reinterpret_cast<float2*>(slots), pb, pe, 0.5f);
        pb = b;
        pe = 0.f;
      }
      pe += 1.f;
    }
    if (pb != 0xFFFFFFFFu) red_bin(reinterpret_cast<float2*>(slots), pb, pe, 0.5f);
  }
}

cudaError_t launch_red_replay(const uint2* rec, int64_t n, int32_t window_ps, int32_t bin_ps, float4* slots, int n_sm,
                              cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  uint32_t magic, shift;
  bin_magic(bin_ps, &magic, &shift);
  const unsigned grid = (unsigned)(n_sm > 0 ? n_sm * 8 : 1024);
  k_red_replay<<<grid, 256, 0, st>>>(rec, n, (uint32_t)window_ps, (uint32_t)bin_ps, magic, shift, slots);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ packed transfer form
// Four records a thread: one 16-byte load of words, two 16-byte stores of
// records; t = anchor of the record's block + the word's high 27 bits.
static __global__ void k_unpack(const uint32_t* __restrict__ anchors, const uint32_t* __restrict__ words, int64_t r0,
                         int64_t n, uint2* __restrict__ out) {
  const int64_t a0 = r0 >> 5;
  const int64_t n4 = n >> 2;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n4; q += (int64_t)gridDim.x * blockDim.x) {
    const uint4 w = reinterpret_cast<const uint4*>(words)[q];
    const int64_t r = r0 + 4 * q;
    const uint32_t wv[4] = {w.x, w.y, w.z, w.w};
    uint32_t t[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) t[k] = __ldg(anchors + (((r + k) >> 5) - a0)) + (wv[k] >> 5);
    uint4* o = reinterpret_cast<uint4*>(out + 4 * q);
    o[0] = make_uint4(t[0], wv[0] & 31u, t[1], wv[1] & 31u);
    o[1] = make_uint4(t[2], wv[2] & 31u, t[3], wv[3] & 31u);
  }
  if (blockIdx.x == 0 && threadIdx.x < (n & 3)) {
    const int64_t i = 4 * n4 + threadIdx.x;
    const uint32_t wv = words[i];
    out[i] = make_uint2(anchors[((r0 + i) >> 5) - a0] + (wv >> 5), wv & 31u);
  }
}

cudaError_t launch_unpack(const uint32_t* anchors, const uint32_t* words, int64_t r0, int64_t n, uint2* out,
                          cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int64_t blocks = ((n >> 2) + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  k_unpack<<<(unsigned)(blocks < 1 ? 1 : blocks), 256, 0, st>>>(anchors, words, r0, n, out);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ merge
// out[b] = (E[b] + bin_ps * 1e-6 * (L0 + sum_{b' < b} dP[b'])) * 1e-3 / bin_ps   (W)
constexpr int kMergeThreads = 256;
constexpr int kMergePer = 8;
constexpr int kMergeTile = kMergeThreads * kMergePer;

int merge_tiles(int n_bins) { return (n_bins + kMergeTile - 1) / kMergeTile; }

namespace {

__device__ __forceinline__ double warp_incl_scan(double v) {
  const int lane = threadIdx.x & 31;
  for (int o = 1; o < 32; o <<= 1) {
    const double u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  return v;
}

// Block-wide exclusive scan of one double per thread; returns the exclusive
// prefix and writes the block total.
__device__ double block_excl_scan(double v, double* total) {
  __shared__ double warp_tot[32];
  const double inc = warp_incl_scan(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 31) warp_tot[w] = inc;
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    const double x = lane < nw ? warp_tot[lane] : 0.0;
    const double xi = warp_incl_scan(x);
    if (lane < nw) warp_tot[lane] = xi - x;
    if (lane == nw - 1) *total = xi;
  }
  __syncthreads();
  const double r = inc - v + warp_tot[w];
  __syncthreads();
  return r;
}

// Block-wide sum of one double per thread (valid in thread 0).
__device__ double block_sum(double v) {
  __shared__ double warp_tot[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) warp_tot[w] = v;
  __syncthreads();
  v = 0.0;
  if (w == 0) {
    v = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  }
  return v;
}

// Leakage-step sum of each merge tile.  A thread adds its kMergePer steps in
// FP32 (a handful of terms of the same bins' FP32 accumulators) and the block
// sums the threads' partials in FP64, so the long prefix is FP64 throughout.
__global__ void k_tile_sums(const WinDesc* __restrict__ wins, const int64_t* __restrict__ tile_base, int n_win) {
  const int64_t gt = blockIdx.x;
  const int w = window_of(tile_base, n_win, gt);
  const WinDesc& W = wins[w];
  const int tile = (int)(gt - W.tile_base);
  if (tile >= W.n_tiles) return;
  const int base = tile * kMergeTile + threadIdx.x * kMergePer;
  float s = 0.f;
  double st = 0.0;  // the time-sliced walk's FP64 steps
#pragma unroll
  for (int k = 0; k < kMergePer; ++k)
    if (base + k < W.n_bins) {
      s += W.cpack ? W.cbins[base + k].w : W.bins[base + k].y;
      if (W.tbins) st += W.tbins[base + k].y;
    }
  const double tot = block_sum((double)s + st);
  if (threadIdx.x == 0) W.tiles[tile] = tot;
}

// Exclusive scan of one window's tile sums in place (one block per window).
__global__ void k_scan_tiles(const WinDesc* __restrict__ wins) {
  const WinDesc& W = wins[blockIdx.x];
  __shared__ double tot;
  double carry = 0.0;
  for (int base = 0; base < W.n_tiles; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const double v = i < W.n_tiles ? W.tiles[i] : 0.0;
    const double ex = block_excl_scan(v, &tot);
    if (i < W.n_tiles) W.tiles[i] = carry + ex;
    carry += tot;
    __syncthreads();
  }
}

// Waveform of each merge tile: the leakage power entering a thread's first
// bin is the FP64 prefix (L0, the earlier tiles, the block's earlier
// threads); the thread's own bins add, in FP32, their energy and the steps
// of its earlier bins (a few terms) to that FP64 base.
__global__ void k_finalize(const WinDesc* __restrict__ wins, const int64_t* __restrict__ tile_base, int n_win) {
  const int64_t gt = blockIdx.x;
  const int w = window_of(tile_base, n_win, gt);
  const WinDesc& W = wins[w];
  const int tile = (int)(gt - W.tile_base);
  if (tile >= W.n_tiles) return;
  const int base = tile * kMergeTile + threadIdx.x * kMergePer;
  float2 v[kMergePer];
  float s = 0.f;
  double st = 0.0;
#pragma unroll
  for (int k = 0; k < kMergePer; ++k) {
    if (W.cpack) {  // {internal, switching, correction, step}: the bin's energy is the first three
      const float4 c = base + k < W.n_bins ? W.cbins[base + k] : make_float4(0.f, 0.f, 0.f, 0.f);
      v[k] = make_float2(c.x + c.y + c.z, c.w);
    } else {
      v[k] = base + k < W.n_bins ? W.bins[base + k] : make_float2(0.f, 0.f);
    }
    s += v[k].y;
    if (W.tbins && base + k < W.n_bins) st += W.tbins[base + k].y;
  }
  __shared__ double tot;
  const double pre = block_excl_scan((double)s + st, &tot) + W.tiles[tile] + *W.l0;
  // W per bin: E (fJ) * 1e-3 / bin_ps + P (nW) * 1e-9
  const float to_w = (float)(1e-3 / (double)W.bin_ps);
  const double p0 = pre * 1e-9;
  if (W.wave) {
    float dp = 0.f;
    if (W.tbins) {  // plus the time-sliced walk's FP64 energies and steps
      const double to_wd = 1e-3 / (double)W.bin_ps;
      double dpt = 0.0;
#pragma unroll
      for (int k = 0; k < kMergePer; ++k) {
        if (base + k < W.n_bins) {
          const double2 t = W.tbins[base + k];
          W.wave[base + k] = (double)fmaf(v[k].x, to_w, dp * 1e-9f) + p0 + (t.x * to_wd + dpt * 1e-9);
          dpt += t.y;
        }
        dp += v[k].y;
      }
    } else {
#pragma unroll
      for (int k = 0; k < kMergePer; ++k) {
        if (base + k < W.n_bins) W.wave[base + k] = (double)fmaf(v[k].x, to_w, dp * 1e-9f) + p0;
        dp += v[k].y;
      }
    }
  }
  if (W.cwave) {  // components: the leakage is the step prefix plus its in-bin corrections
    const int64_t nb = W.n_bins;
    float dp = 0.f;
#pragma unroll
    for (int k = 0; k < kMergePer; ++k) {
      if (base + k < W.n_bins) {
        const float4 c = W.cbins[base + k];
        const float corr = W.cpack ? c.z : c.w, gl = W.cpack ? 0.f : c.z;
        W.cwave[base + k] = (double)fmaf(corr, to_w, dp * 1e-9f) + p0;
        W.cwave[nb + base + k] = (double)(c.x * to_w);
        W.cwave[2 * nb + base + k] = (double)(c.y * to_w);
        W.cwave[3 * nb + base + k] = (double)(gl * to_w);
      }
      dp += v[k].y;
    }
  }
}

// ------------------------------------------------------------------ adjoint gradient prefix
// grad[b] = {g_b, G(b * bin_ps)} with g_b = dL/dP_b * 1e-3 / bin_ps = dL/dE_b
// and G(t) = integral of g over [0, t) (g piecewise constant per bin), the
// weight a leakage interval [t0, t1) receives: G(t1) - G(t0).
__global__ void k_grad_tiles(const float* __restrict__ dLdP, int n_bins, int bin_ps, double* __restrict__ tiles) {
  const int base = blockIdx.x * kMergeTile + threadIdx.x * kMergePer;
  const double f = 1e-3;  // dE_b -> dP_b is 1e-3 / bin_ps; times bin_ps for the integral
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kMergePer; ++k)
    if (base + k < n_bins) s += (double)dLdP[base + k] * f;
  __shared__ double tot;
  block_excl_scan(s, &tot);
  if (threadIdx.x == 0) tiles[blockIdx.x] = tot;
  (void)bin_ps;
}

__global__ void k_grad_scan(double* tiles, int n_tiles, float* g_total) {
  __shared__ double tot;
  double carry = 0.0;
  for (int base = 0; base < n_tiles; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const double v = i < n_tiles ? tiles[i] : 0.0;
    const double ex = block_excl_scan(v, &tot);
    if (i < n_tiles) tiles[i] = carry + ex;
    carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) *g_total = (float)carry;
}

__global__ void k_grad_finalize(const float* __restrict__ dLdP, int n_bins, int bin_ps,
                                const double* __restrict__ tiles, float2* __restrict__ grad) {
  const int base = blockIdx.x * kMergeTile + threadIdx.x * kMergePer;
  double v[kMergePer];
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kMergePer; ++k) {
    v[k] = base + k < n_bins ? (double)dLdP[base + k] * 1e-3 : 0.0;  // g_b * bin_ps
    s += v[k];
  }
  __shared__ double tot;
  double pre = block_excl_scan(s, &tot) + tiles[blockIdx.x];
  const double inv = 1.0 / (double)bin_ps;
#pragma unroll
  for (int k = 0; k < kMergePer; ++k) {
    if (base + k < n_bins) grad[base + k] = make_float2((float)(v[k] * inv), (float)pre);
    pre += v[k];
  }
}

// Zero every window's bin accumulators, one tile per block.
__global__ void k_cells_out(const double* __restrict__ acc, int n_cells, float* d_escale, float* d_lscale) {
  const int c = threadIdx.x + blockIdx.x * blockDim.x;
  if (c < n_cells) {
    if (d_escale) d_escale[c] = (float)acc[c];
    if (d_lscale) d_lscale[c] = (float)acc[n_cells + c];
  }
}

}  // namespace

// ------------------------------------------------------------------ exact trace check
// Run after a walk flagged a malformed trace.  Per (window, gate), the
// events in record order against the input rules of Algorithm 1, in the
// order the oracle applies them: the time in [0, T), not below the previous
// event's, no reserved meta bits and a pin of the cell, and an event that
// toggles its pin.  The smallest failing (window, record) wins, so the
// reported error does not depend on the order in which threads ran:
// key = ((window << 40 | record) << 3) | -code.
__global__ void k_validate(LibView L, NetView N, const WinDesc* __restrict__ wins, const DevError* gate,
                           unsigned long long* first) {
  if (gate && gate->code == 0) return;
  const WinDesc& W = wins[blockIdx.y];
  const int32_t T = W.window_ps;
  for (int64_t g = W.g0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < W.g1;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = W.offsets[g], b = W.offsets[g + 1];
    if (a == b) continue;
    const uint32_t n_pins = (uint32_t)L.cells[N.cell[g]].n_in + 1u;
    uint32_t S = (uint32_t)W.init[g] & ((1u << n_pins) - 1u);
    int32_t tp = 0;
    for (int64_t i = a; i < b; ++i) {
      const uint2 r = W.rec[i];
      const int32_t t = (int32_t)r.x;
      const uint32_t pin = r.y & 0xFu, val = (r.y >> 4) & 1u;
      int code = 0;
      if (t < 0 || t >= T) code = GTP_ERANGE;
      else if (t < tp) code = GTP_EORDER;
      else if ((r.y >> 5) != 0u || pin >= n_pins) code = GTP_ERANGE;
      else if (((S >> pin) & 1u) == val) code = GTP_ENOTOGGLE;
      if (code != 0) {
        const unsigned long long key =
            ((((unsigned long long)blockIdx.y << 40) | (unsigned long long)i) << 3) | (unsigned long long)(-code);
        atomicMin(first, key);
        break;
      }
      S ^= 1u << pin;
      tp = t;
    }
  }
}

cudaError_t launch_validate(const LibView& L, const NetView& N, const WinDesc* wins, int n_win,
                            unsigned long long* first, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(first, 0xFF, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  int64_t blocks = (N.n_gates + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  k_validate<<<dim3((unsigned)(blocks < 1 ? 1 : blocks), (unsigned)n_win), 256, 0, st>>>(L, N, wins, nullptr, first);
  return cudaGetLastError();
}

cudaError_t launch_validate_if(const LibView& L, const NetView& N, const WinDesc* win, const DevError* err,
                               int64_t n_gates, unsigned long long* first, cudaStream_t st) {
  int64_t blocks = (n_gates + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  k_validate<<<(unsigned)(blocks < 1 ? 1 : blocks), 256, 0, st>>>(L, N, win, err, first);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ design-level power
// Key of a double that orders like the value (for an integer atomic max).
__device__ __forceinline__ unsigned long long ordered_key(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

// Sums of the per-gate energies (FP64; e_gl may be null) into sums[0..3] and
// the largest waveform bin's key into *maxkey.
__global__ void k_design_sums(const double* __restrict__ e_leak, const double* __restrict__ e_int,
                              const double* __restrict__ e_sw, const double* __restrict__ e_gl, int64_t G,
                              const double* __restrict__ wave, int64_t n_bins, double* sums,
                              unsigned long long* maxkey) {
  double a[4] = {0.0, 0.0, 0.0, 0.0};
  unsigned long long mk = 0ull;
  const int64_t n = G > n_bins ? G : n_bins;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (i < G) {
      a[0] += e_leak[i];
      a[1] += e_int[i];
      a[2] += e_sw[i];
      if (e_gl) a[3] += e_gl[i];
    }
    if (wave && i < n_bins) mk = max(mk, ordered_key(wave[i]));
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    double v = a[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(sums + k, v);
  }
  for (int o = 16; o > 0; o >>= 1) mk = max(mk, __shfl_down_sync(0xffffffffu, mk, o));
  if ((threadIdx.x & 31) == 0 && wave) atomicMax(maxkey, mk);
}

// The first bin holding the largest value.
__global__ void k_peak_index(const double* __restrict__ wave, int64_t n_bins, const unsigned long long* maxkey,
                             unsigned long long* idx) {
  const unsigned long long mk = *maxkey;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_bins; i += (int64_t)gridDim.x * blockDim.x)
    if (ordered_key(wave[i]) == mk) atomicMin(idx, (unsigned long long)i);
}

cudaError_t launch_design_power(const double* e_leak, const double* e_int, const double* e_sw, const double* e_gl,
                                int64_t G, const double* wave, int64_t n_bins, double* scratch, cudaStream_t st) {
  // scratch: [0..3] sums, [4] max key, [5] peak index
  cudaError_t e = cudaMemsetAsync(scratch, 0, 5 * sizeof(double), st);
  if (e != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(scratch + 5, 0xFF, sizeof(double), st)) != cudaSuccess) return e;
  const int64_t n = G > n_bins ? G : n_bins;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  unsigned long long* keys = reinterpret_cast<unsigned long long*>(scratch + 4);
  k_design_sums<<<(unsigned)(blocks < 1 ? 1 : blocks), 256, 0, st>>>(e_leak, e_int, e_sw, e_gl, G, wave, n_bins,
                                                                      scratch, keys);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (wave && n_bins > 0) {
    int64_t b2 = (n_bins + 255) / 256;
    if (b2 > 1024) b2 = 1024;
    k_peak_index<<<(unsigned)b2, 256, 0, st>>>(wave, n_bins, keys, keys + 1);
  }
  return cudaGetLastError();
}

cudaError_t launch_cells_out(const double* acc, int n_cells, float* d_escale, float* d_lscale, cudaStream_t st) {
  k_cells_out<<<(n_cells + 255) / 256, 256, 0, st>>>(acc, n_cells, d_escale, d_lscale);
  return cudaGetLastError();
}

cudaError_t launch_merge(const WinDesc* wins, const int64_t* tile_base, int n_win, int64_t n_tiles_total,
                         cudaStream_t st) {
  if (n_tiles_total <= 0) return cudaSuccess;
  k_tile_sums<<<(unsigned)n_tiles_total, kMergeThreads, 0, st>>>(wins, tile_base, n_win);
  k_scan_tiles<<<(unsigned)n_win, 1024, 0, st>>>(wins);
  k_finalize<<<(unsigned)n_tiles_total, kMergeThreads, 0, st>>>(wins, tile_base, n_win);
  return cudaGetLastError();
}

cudaError_t launch_grad_prep(const WinDesc* wins, const float* dLdP, float2* grad, double* tiles, int n_tiles,
                             int n_bins, int bin_ps, float* g_total, cudaStream_t st) {
  (void)wins;
  if (n_tiles <= 0) return cudaSuccess;
  k_grad_tiles<<<n_tiles, kMergeThreads, 0, st>>>(dLdP, n_bins, bin_ps, tiles);
  k_grad_scan<<<1, 1024, 0, st>>>(tiles, n_tiles, g_total);
  k_grad_finalize<<<n_tiles, kMergeThreads, 0, st>>>(dLdP, n_bins, bin_ps, tiles, grad);
  return cudaGetLastError();
}

}  // namespace gtp
