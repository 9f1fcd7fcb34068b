// gtp_run_power_noalloc: the single-window power walk for callers that
// cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is unavailable or forbidden,
// such as a host callback or a plugin inside another framework's memory pool
// (which owns every device byte), or a caller that must not trigger the
// implicit synchronisation and fragmentation of cudaMalloc/cudaFree between
// its own launches.  Such callers already hold every input and output in
// device memory; what the walk adds is scratch: the per-bin accumulators,
// the merge's tile sums, the leakage base L0, the error word and a small
// header with the cell map.  Here that scratch is one file-scope device array
// of fixed size, which every GPU that loads this library holds until the
// process exits.
//
// The kernel is a variant of the one-thread-per-gate walk: it locates the
// NLDM point of every event from the slew and load arrays directly (the
// context-based engine reads precomputed per-netlist descriptors instead,
// which would need G * 2 * (pins + 1) * 16 bytes of scratch), and it folds the
// gate pass (empty gates, L0, initial-state checks) and the CSR checks into
// the same kernel.  The bin merge is the engine's.
#include <mutex>

#include "gtp_internal.cuh"

namespace gtp {
namespace {

constexpr int kNaMaxCells = 256;
constexpr int kNaMaxDevices = 64;
constexpr int kNaThreads = 128;

// Header of the scratch array, written from the host at every call.
struct NaHeader {
  DevError err;                   // first failure of this call
  double l0;                      // sum over gates of P_leak(initial state), nW
  double pad;
  int64_t tile_base[2];           // {0, n_tiles}: the merge's window bases
  float axes[4 * kMaxAxis];       // slew axis, load axis, their 1 / segment widths
  CellInfo cells[kNaMaxCells];
  WinDesc win;                    // the merge's view of this window
};

constexpr size_t kNaHeaderBytes = 8192;
static_assert(sizeof(NaHeader) <= kNaHeaderBytes, "scratch header too large");
constexpr size_t kNaTileBytes = sizeof(double) * ((GTP_NOALLOC_MAX_BINS + 2047) / 2048);
constexpr size_t kNaBinsOffset = kNaHeaderBytes + ((kNaTileBytes + 255) & ~(size_t)255);
constexpr size_t kNaScratchBytes = kNaBinsOffset + sizeof(float2) * (size_t)GTP_NOALLOC_MAX_BINS;

// The scratch.  In host code this name is only a handle for the runtime;
// kernels receive the device address that cudaGetSymbolAddress returns.
static __device__ __align__(256) unsigned char gtp_noalloc_scratch[kNaScratchBytes];

// Device address of the scratch on each device, set once per device.
std::mutex g_na_mutex;
void* g_na_ptr[kNaMaxDevices] = {};

struct NaArgs {
  const NaHeader* hdr;
  DevError* err;
  double* l0;
  float2* bins;
  const float* tab;        // caller's tables (fJ)
  const float* leak;       // caller's leakage (nW)
  const int32_t* cell;
  const float* load;
  const float* slew;       // [G][stride][2]
  const int64_t* offsets;  // [G+1]
  const uint2* rec;        // [E]
  const uint8_t* init;     // [G]
  double* e_leak;          // [G] or null
  double* e_int;           // [G] or null
  double* e_sw;            // [G] or null
  uint8_t* final_state;    // [G] or null
  int64_t n_gates;
  int64_t n_events;
  int32_t stride;
  int32_t n_cells;
  int32_t ns, nl, tsize;
  int32_t window_ps;
  int32_t bin_ps;
  uint32_t bin_magic, bin_shift;
  float half_v2;
};

__device__ __forceinline__ int na_segment(const float* axis, int n, float x) {
  int i = 0;
  while (i < n - 2 && x >= axis[i + 1]) ++i;
  return i;
}

// One thread per gate (Algorithm 1 on one gate): timestamp groups looked up
// at the pre-group state, the state updated after the group, leakage held
// between groups (Sec. 2.4.2), bilinear internal energy (Sec. 2.2.1) and
// 0.5 * C * Vdd^2 per output toggle (Sec. 2.4.1).  Bins receive the same
// {energy, leakage step} pairs as the engine's walks.
__global__ void __launch_bounds__(kNaThreads) k_noalloc_walk(NaArgs a) {
  __shared__ float ax[4 * kMaxAxis];
  __shared__ CellInfo cells[kNaMaxCells];
  __shared__ double red[kNaThreads / 32];
  for (int k = threadIdx.x; k < 4 * kMaxAxis; k += blockDim.x) ax[k] = a.hdr->axes[k];
  for (int k = threadIdx.x; k < a.n_cells; k += blockDim.x) cells[k] = a.hdr->cells[k];
  __syncthreads();
  const float* sax = ax;
  const float* lax = ax + kMaxAxis;
  const float* srw = ax + 2 * kMaxAxis;
  const float* lrw = ax + 3 * kMaxAxis;
  const float T = (float)a.window_ps;
  double p0 = 0.0;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < a.n_gates;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t lo = a.offsets[g], hi = a.offsets[g + 1];
    if (lo < 0 || hi < lo || hi > a.n_events || (g == 0 && lo != 0) || (g == a.n_gates - 1 && hi != a.n_events)) {
      report_error(a.err, GTP_EINVAL, g);
      continue;
    }
    const int32_t c = a.cell[g];
    if (c < 0 || c >= a.n_cells) {
      report_error(a.err, GTP_EINVAL, g);
      continue;
    }
    const CellInfo ci = cells[c];
    const uint32_t n_in = (uint32_t)ci.n_in, n_pins = n_in + 1;
    const float* leak = a.leak + ci.leak_base;
    uint32_t st = a.init[g];
    if (st >> n_pins) {
      report_error(a.err, GTP_ERANGE, -1 - g);
      st &= (2u << n_in) - 1u;
    }
    float P = leak[st];
    p0 += (double)P;
    if (lo == hi) {
      if (a.e_leak) a.e_leak[g] = (double)P * (double)a.window_ps * 1e-6;
      if (a.e_int) a.e_int[g] = 0.0;
      if (a.e_sw) a.e_sw[g] = 0.0;
      if (a.final_state) a.final_state[g] = (uint8_t)st;
      continue;
    }
    const float C = a.load[g];
    const int j = na_segment(lax, a.nl, C);
    const float fl = (C - lax[j]) * lrw[j];
    const float e_switch = a.half_v2 * C;
    int32_t t_prev = 0;
    Kahan El, Ei, Es;
    bool bad = false;
    int64_t i = lo;
    while (i < hi) {
      const int32_t t = (int32_t)a.rec[i].x;
      if (t < 0 || t >= a.window_ps) { report_error(a.err, GTP_ERANGE, i); bad = true; break; }
      if (t < t_prev) { report_error(a.err, GTP_EORDER, i); bad = true; break; }
      El.add(P * (float)(t - t_prev) * 1e-6f);
      const uint32_t bin = bin_of((uint32_t)t, a.bin_magic, a.bin_shift, (uint32_t)a.bin_ps);
      uint32_t s_next = st;
      float e_bin = 0.f;
      int64_t k = i;
      for (; k < hi; ++k) {
        const uint2 r = a.rec[k];
        if ((int32_t)r.x != t) break;
        const uint32_t pin = r.y & 0xFu, val = (r.y >> 4) & 1u;
        if ((r.y >> 5) != 0u || pin >= n_pins) { report_error(a.err, GTP_ERANGE, k); bad = true; break; }
        if (((s_next >> pin) & 1u) == val) { report_error(a.err, GTP_ENOTOGGLE, k); bad = true; break; }
        s_next ^= 1u << pin;
        float E;
        if (pin < n_in) {
          const float s = a.slew[((size_t)g * a.stride + pin) * 2 + val];
          const int is = na_segment(sax, a.ns, s);
          const float fs = (s - sax[is]) * srw[is];
          const uint32_t table = (uint32_t)ci.tab_base + ((pin * 2u + val) << (n_in - 1)) + side_bits(st, pin, n_in);
          const float* p = a.tab + (size_t)table * a.tsize + is * a.nl + j;
          const float e_lo = fmaf(fl, p[1] - p[0], p[0]);
          const float e_hi = fmaf(fl, p[a.nl + 1] - p[a.nl], p[a.nl]);
          E = fmaf(fs, e_hi - e_lo, e_lo);
          Ei.add(E);
        } else {
          E = e_switch;
          Es.add(E);
        }
        e_bin += E;
      }
      if (bad) break;
      const float P_new = leak[s_next];
      const float dP = P_new - P;
      const float frac = (float)((int32_t)(bin + 1u) * a.bin_ps - t);
      red_bin(a.bins, bin, e_bin + dP * frac * 1e-6f, dP);
      st = s_next;
      P = P_new;
      t_prev = t;
      i = k;
    }
    if (bad) continue;
    El.add(P * (T - (float)t_prev) * 1e-6f);
    if (a.e_leak) a.e_leak[g] = El.value();
    if (a.e_int) a.e_int[g] = Ei.value();
    if (a.e_sw) a.e_sw[g] = Es.value();
    if (a.final_state) a.final_state[g] = (uint8_t)st;
  }
  for (int o = 16; o > 0; o >>= 1) p0 += __shfl_down_sync(0xffffffffu, p0, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = p0;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int w = 0; w < kNaThreads / 32; ++w) v += red[w];
    if (v != 0.0) atomicAdd(a.l0, v);
  }
}

// Device address of the scratch on the current device (set-up on first use).
int na_scratch(unsigned char** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return GTP_ECUDA;
  if (dev < 0 || dev >= kNaMaxDevices) return GTP_EINVAL;
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_ptr[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, gtp_noalloc_scratch) != cudaSuccess || ptr == nullptr) return GTP_ECUDA;
    g_na_ptr[dev] = ptr;
  }
  *out = static_cast<unsigned char*>(g_na_ptr[dev]);
  return GTP_OK;
}

}  // namespace
}  // namespace gtp

using namespace gtp;

extern "C" int gtp_run_power_noalloc(void* cuda_stream, int32_t n_cells, const int32_t* n_in, float vdd,
                                     int32_t n_slew, const float* slew_axis, int32_t n_load, const float* load_axis,
                                     const float* e_int, int64_t n_e_int, const float* p_leak, int64_t n_p_leak,
                                     int64_t n_gates, const int32_t* cell, const float* load_ff, const float* slew_ps,
                                     int32_t slew_stride, int64_t window_ps, int64_t n_events,
                                     const int64_t* gate_offsets, const gtp_event* events, const uint8_t* init_state,
                                     int32_t bin_ps, double* waveform_w, double* e_leak, double* e_int_out,
                                     double* e_sw, uint8_t* final_state) {
  // ---- host-side checks (nothing is enqueued before they pass)
  if (n_cells <= 0 || n_cells > kNaMaxCells || !n_in || !slew_axis || !load_axis || !e_int || !p_leak)
    return GTP_EINVAL;
  if (n_slew < 2 || n_slew > GTP_MAX_AXIS || n_load < 2 || n_load > GTP_MAX_AXIS) return GTP_ERANGE;
  for (int i = 0; i + 1 < n_slew; ++i)
    if (!(slew_axis[i + 1] > slew_axis[i])) return GTP_EINVAL;
  for (int i = 0; i + 1 < n_load; ++i)
    if (!(load_axis[i + 1] > load_axis[i])) return GTP_EINVAL;
  if (n_gates <= 0 || n_gates >= (1ll << 31) || !cell || !load_ff || !slew_ps || !gate_offsets || !init_state)
    return GTP_EINVAL;
  if (n_events < 0 || (n_events > 0 && !events)) return GTP_EINVAL;
  if (window_ps <= 0 || window_ps >= (1ll << 31) || bin_ps <= 0 || window_ps % bin_ps != 0) return GTP_ERANGE;
  const int64_t n_bins = window_ps / bin_ps;
  if (n_bins > GTP_NOALLOC_MAX_BINS) return GTP_ERANGE;
  if ((reinterpret_cast<uintptr_t>(events) & 7u) != 0) return GTP_EINVAL;

  NaHeader h{};
  int64_t n_tables = 0, n_leak = 0;
  int max_in = 0;
  for (int c = 0; c < n_cells; ++c) {
    if (n_in[c] < 1 || n_in[c] > GTP_MAX_PINS - 1) return GTP_ERANGE;
    h.cells[c].tab_base = (int32_t)n_tables;
    h.cells[c].leak_base = (int32_t)n_leak;
    h.cells[c].n_in = n_in[c];
    n_tables += (int64_t)n_in[c] * (2ll << (n_in[c] - 1));
    n_leak += 2ll << n_in[c];
    if (n_in[c] > max_in) max_in = n_in[c];
  }
  const int64_t tsize = (int64_t)n_slew * n_load;
  if (n_e_int != n_tables * tsize || n_e_int >= (1ll << 31) || n_p_leak != n_leak) return GTP_EINVAL;
  if (slew_stride < max_in || slew_stride > GTP_MAX_PINS) return GTP_EINVAL;
  for (int i = 0; i < GTP_MAX_AXIS; ++i) {
    h.axes[i] = i < n_slew ? slew_axis[i] : 0.f;
    h.axes[kMaxAxis + i] = i < n_load ? load_axis[i] : 0.f;
    h.axes[2 * kMaxAxis + i] = i + 1 < n_slew ? 1.0f / (slew_axis[i + 1] - slew_axis[i]) : 0.f;
    h.axes[3 * kMaxAxis + i] = i + 1 < n_load ? 1.0f / (load_axis[i + 1] - load_axis[i]) : 0.f;
  }

  // ---- the call ends by waiting for its stream, which a capturing stream
  // does not allow: refuse before anything is enqueued
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return GTP_ECUDA;
  if (cs != cudaStreamCaptureStatusNone) return GTP_EINVAL;

  // ---- scratch of this device
  unsigned char* base = nullptr;
  const int rc = na_scratch(&base);
  if (rc != GTP_OK) return rc;
  NaHeader* d_hdr = reinterpret_cast<NaHeader*>(base);
  double* d_tiles = reinterpret_cast<double*>(base + kNaHeaderBytes);
  float2* d_bins = reinterpret_cast<float2*>(base + kNaBinsOffset);

  const int n_tiles = merge_tiles((int)n_bins);
  if (sizeof(double) * (size_t)n_tiles > kNaTileBytes) return GTP_ERANGE;
  h.tile_base[0] = 0;
  h.tile_base[1] = n_tiles;
  WinDesc& w = h.win;
  w.bins = d_bins;
  w.l0 = &d_hdr->l0;
  w.tiles = d_tiles;
  w.wave = waveform_w;
  w.n_tiles = n_tiles;
  w.tile_base = 0;
  w.window_ps = (int32_t)window_ps;
  w.bin_ps = bin_ps;
  bin_magic(bin_ps, &w.bin_magic, &w.bin_shift);
  w.n_bins = (int32_t)n_bins;

  NaArgs a{};
  a.hdr = d_hdr;
  a.err = &d_hdr->err;
  a.l0 = &d_hdr->l0;
  a.bins = d_bins;
  a.tab = e_int;
  a.leak = p_leak;
  a.cell = cell;
  a.load = load_ff;
  a.slew = slew_ps;
  a.offsets = gate_offsets;
  a.rec = reinterpret_cast<const uint2*>(events);
  a.init = init_state;
  a.e_leak = e_leak;
  a.e_int = e_int_out;
  a.e_sw = e_sw;
  a.final_state = final_state;
  a.n_gates = n_gates;
  a.n_events = n_events;
  a.stride = slew_stride;
  a.n_cells = n_cells;
  a.ns = n_slew;
  a.nl = n_load;
  a.tsize = (int32_t)tsize;
  a.window_ps = (int32_t)window_ps;
  a.bin_ps = bin_ps;
  a.bin_magic = w.bin_magic;
  a.bin_shift = w.bin_shift;
  a.half_v2 = 0.5f * vdd * vdd;

  // ---- enqueue: header (error word and L0 start at zero), cleared bins,
  // the walk, the merge; then read the error word back.
  if (cudaMemcpyAsync(d_hdr, &h, sizeof(NaHeader), cudaMemcpyHostToDevice, st) != cudaSuccess) return GTP_ECUDA;
  if (cudaMemsetAsync(d_bins, 0, sizeof(float2) * (size_t)n_bins, st) != cudaSuccess) return GTP_ECUDA;
  int64_t blocks = (n_gates + kNaThreads - 1) / kNaThreads;
  if (blocks > 4096) blocks = 4096;
  k_noalloc_walk<<<(unsigned)blocks, kNaThreads, 0, st>>>(a);
  if (cudaGetLastError() != cudaSuccess) return GTP_ECUDA;
  if (waveform_w && launch_merge(&d_hdr->win, d_hdr->tile_base, 1, n_tiles, st) != cudaSuccess) return GTP_ECUDA;
  DevError e{};
  if (cudaMemcpyAsync(&e, &d_hdr->err, sizeof(DevError), cudaMemcpyDeviceToHost, st) != cudaSuccess) return GTP_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return GTP_ECUDA;
  return e.code;
}
