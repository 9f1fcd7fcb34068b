// Host engine behind the C ABI of include/gtpower.h: device buffers, input
// validation, launch plans (window descriptor tables), CUDA-graph replay of
// batched runs, the adjoint, phase timing and the autotuner.  All device work
// goes to the context's stream; results are synchronised only where the ABI
// says so.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "gtp_internal.cuh"
#include "gtp_scheme.cuh"
#include "gtp_walk.cuh"

using namespace gtp;

namespace {

constexpr int kMaxWindows = 1024;
constexpr size_t kStatusBytes = sizeof(DevError) + 16;  // DevError, then a 64-bit count
// Default bin bytes (8 a bin) of the windows one walk launch reduces into
// at most, unless a single window has more: well inside the 129 MB L2,
// beside the records streaming through it.
constexpr int64_t kGroupBinBytes = 96ll << 20;

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  // Grow-only (re)allocation; contents are not preserved.
  cudaError_t reserve(size_t n) {
    if (n <= bytes && p) return cudaSuccess;
    release();
    cudaError_t e = cudaMalloc(&p, n ? n : 16);
    if (e == cudaSuccess) bytes = n ? n : 16;
    return e;
  }
  template <class T>
  T* as() const { return static_cast<T*>(p); }
};

struct Window {
  bool loaded = false;
  int64_t window_ps = 0;
  int64_t n_events = 0;
  DevBuf offsets, records, init;
  const uint2* borrowed = nullptr;
  DevBuf e_leak, e_int, e_sw, e_gl, final_state, bins, tiles, wave;
  DevBuf tbins;  // the time-sliced walk's FP64 bins
  DevBuf cbins, cwave;  // per-component runs: component accumulators and the host-bound waveforms
  // the paper's schemes: per-pin event streams (built once per load) and the
  // density-aware block plan (per bin count and partitioning parameters)
  DevBuf ps_off, ps_ev, ps_slot, blk_gate, blk_first, ncyc;
  bool ps_ok = false;
  int64_t dplan_key[3] = {-1, -1, -1};
  int64_t n_blocks = 0;
  bool has_result = false;
  bool glitch_result = false;  // the last run detected glitches (e_gl holds them)
  bool streamed = false;       // filled by a streamed run: results only, no resident records
  int32_t last_bin_ps = 0;
  // pattern gates: records {t, pin | value << 8}, initial states, items, and per-gate results
  unsigned long long max_count = 0;  // the busiest gate's events (set by gtp_load_events)
  bool pat_loaded = false;
  int64_t pat_n_events = 0, pat_n_items = 0;
  std::vector<int64_t> pat_h_off;
  DevBuf pat_off, pat_rec, pat_init, pat_items, pat_first, pat_mask, pat_e_leak, pat_e_int, pat_e_sw, pat_e_gl,
      pat_final, pat_dC;
  bool pat_grad = false;  // pat_dC holds the pattern gates' dL/dC of the last backward run
  void release_patterns() {
    for (DevBuf* b : {&pat_off, &pat_rec, &pat_init, &pat_items, &pat_first, &pat_mask, &pat_e_leak, &pat_e_int,
                      &pat_e_sw, &pat_e_gl, &pat_final, &pat_dC})
      b->release();
    pat_h_off.clear();
    pat_loaded = false;
    pat_grad = false;
    pat_n_events = pat_n_items = 0;
  }
  const uint2* rec() const { return borrowed ? borrowed : records.as<uint2>(); }
  void release() {
    for (DevBuf* b : {&offsets, &records, &init, &e_leak, &e_int, &e_sw, &e_gl, &final_state, &bins, &tbins, &tiles, &wave,
                      &cbins, &cwave, &ps_off, &ps_ev, &ps_slot, &blk_gate, &blk_first, &ncyc})
      b->release();
    release_patterns();
    borrowed = nullptr;
    loaded = false;
    has_result = false;
    ps_ok = false;
    dplan_key[0] = -1;
  }
};

struct GraphKey {
  std::vector<int32_t> windows;
  int32_t bin_ps;
  int64_t rpt, ctas, kernel, dmin, tmin, piece, plan_gen;
  int64_t n_tiles;  // launch sizes baked into the graph
  bool any_events;  // whether the walk was captured
  int timing;       // the phase-timing level the graph was captured with
  std::vector<int32_t> groups;  // first window of each window group
  int64_t pat_items;            // pattern walk launch size (-1: no pattern gates)
  bool whole;                   // the walk without pieces
  bool operator<(const GraphKey& o) const {
    return std::tie(windows, bin_ps, rpt, ctas, kernel, dmin, tmin, piece, plan_gen, n_tiles, any_events, timing,
                    groups, pat_items, whole) < std::tie(o.windows, o.bin_ps, o.rpt, o.ctas, o.kernel, o.dmin,
                                                         o.tmin, o.piece, o.plan_gen, o.n_tiles, o.any_events,
                                                         o.timing, o.groups, o.pat_items, o.whole);
  }
};

}  // namespace

struct gtp_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  int n_sm = 0;
  // library
  bool lib_loaded = false;
  std::vector<int32_t> n_in;
  int max_in = 0;
  DevBuf tab, leak, cells, table_cell, leak_cell, escale, lscale;
  LibView L{};
  // netlist
  bool net_loaded = false;
  DevBuf cell, load, slew, desc;
  NetView N{};
  // per-gate energy tables (forward: scaled; adjoint: unscaled + load derivative), rebuilt when stale
  DevBuf gtab, gtab_bwd;
  bool gtab_ok = false, gtab_bwd_ok = false;
  bool desc_ok = false;  // the event descriptors match the netlist and loads
  std::map<int, Window> windows;
  // launch plan: device descriptor table and its pinned host staging copy
  DevBuf plan;  // WinDesc[kMaxWindows] | tile_base[kMaxWindows+1] | l0[kMaxWindows+1]
  unsigned char* h_plan = nullptr;
  // device-side work plan: dense segments, their seeds, sorted sparse gates, counters
  DevBuf glist, counters;
  DevBuf chunks;         // the tiled walk's chunk starts
  int64_t gcap = 0;
  int64_t plan_gen = 0;  // bumped whenever a plan buffer moves (captured graphs hold its pointers)
  DevBuf cell_acc, grad, gtiles, dC_scratch;
  DevBuf counts;  // per-gate event counts for host outputs of gtp_gate_energy
  DevBuf d_err;
  DevBuf first_bad;  // trace check result (see launch_validate)
  DevBuf out_slew;   // glitch detection: [n_gates][2] output {fall, rise} transition times
  DevBuf dp_scratch; // design-level power: sums, peak key and index
  // the paper's schemes: state patterns of the library's tables and leakage
  // entries, FP64 bins, per-gate reduction rows, timing events
  DevBuf pat_int, pat_leak, sch_ebins, sch_R;
  DevBuf probe;  // reduction-rate probe scratch
  bool pat_ok = false;
  cudaEvent_t sch_ev[2] = {};
  int64_t p_evt_tgt = 8, p_thr_floor = 512, p_ncyc_fix = 1;
  // streamed runs: two chunk buffers, a copy stream and its events
  DevBuf chunk_buf[2];
  DevBuf pk_buf[2];  // packed transfer form of a chunk: words, then the anchors of its blocks
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_copied[2] = {}, ev_walked[2] = {};
  DevError* h_err = nullptr;
  std::map<GraphKey, cudaGraphExec_t> graphs;
  cudaStream_t capture_stream = nullptr;
  // parameters
  int64_t p_kernel = 0;
  int64_t p_rpt = 8;
  int64_t p_ctas_per_sm = 0;
  int64_t p_dense_min = -1;  // -1: chosen per run (see dense_min_auto)
  int64_t run_dense_min = 0; // the run being planned (0 before the first)
  int64_t p_bwd_staged = -1; // adjoint gate tables: 1 staged, 0 in place, -1 by the window's events per SM
  int64_t p_tile_min = 0;  // gates with this many events or more take the time-sliced walk (0: none)
  int64_t p_piece_len = -1;   // gates with more events are split into pieces (0: never, -1: chosen per run)
  int64_t run_piece_len = 0;  // the piece length of the run being planned
  bool run_whole = false;     // no gate of the run being planned is split into pieces
  std::vector<std::pair<int, int>> run_groups;  // the run's window groups [first, end), walked one after another
  int64_t p_group_bytes = kGroupBinBytes;       // bin bytes of a window group at most
  // pattern cells (state patterns, up to 32 pins) and pattern gates
  bool pat_cells_ok = false, pat_net_ok = false, pat_index_ok = false;
  std::vector<PatCell> h_pat_cells;
  DevBuf pc_cells, pc_ip, pc_ipo, pc_lp, pc_tab, pc_iidx, pc_lidx;
  PatLib P{};
  DevBuf pn_cell, pn_load, pn_slew, pn_oslew, pn_desc;
  PatNet Q{};
  int64_t p_sipl_max_pins = 16;  // pattern cells with at most this many pins get state-indexed arrays
  int64_t pat_index_bytes = 0;
  int32_t pat_indexed = 0;
  DevBuf pat_bad;  // smallest error key of the pattern walk
  int64_t run_pat_items = -1;  // the run's pattern walk launch size (-1: none)
  // phase timing (CUDA events on the context stream) and launch counting: 0 off, 1 every phase, 2 the walk only
  int timing = 0;
  cudaEvent_t ev[14] = {};
  // gate pass, plan, walk (all walks), merge; the tiled and pattern walks; the descriptor and gate-table pass
  int64_t t_ns[7] = {0, 0, 0, 0, 0, 0, 0};
  bool prep_marked = false;  // the run rebuilt descriptors and gate tables under timing level 1
  // streamed runs under timing level 1: start, first copy, last copy done, end
  cudaEvent_t ev_sx[4] = {};
  int64_t t_sx[3] = {0, 0, 0};  // setup (to the first copy), copies, tail (last copy to the end)
  int64_t n_timed = 0;
  int64_t launches = 0;
};

namespace {

size_t plan_bytes() { return sizeof(WinDesc) * kMaxWindows + 2 * sizeof(int64_t) * (kMaxWindows + 1); }
WinDesc* plan_wins(void* base) { return static_cast<WinDesc*>(base); }
int64_t* plan_tile_base(void* base) {
  return reinterpret_cast<int64_t*>(static_cast<unsigned char*>(base) + sizeof(WinDesc) * kMaxWindows);
}
double* plan_l0(void* base) { return reinterpret_cast<double*>(plan_tile_base(base) + (kMaxWindows + 1)); }

int fail(gtp_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

int cuda_fail(gtp_ctx* c, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) return fail(c, GTP_ENOMEM, m);
  return fail(c, GTP_ECUDA, m);
}

#define CU(call, where)                                      \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, where); \
  } while (0)

#define RC(call)                 \
  do {                           \
    int r_ = (call);             \
    if (r_ != GTP_OK) return r_; \
  } while (0)

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

cudaMemcpyKind kind_in(int flags) { return (flags & GTP_DEVICE) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice; }
cudaMemcpyKind kind_out(int flags) { return (flags & GTP_DEVICE) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost; }

const char* code_name(int code) {
  switch (code) {
    case GTP_EORDER: return "timestamps decrease within a gate";
    case GTP_ERANGE: return "value out of range (time, pin, reserved bits or initial state)";
    case GTP_ENOTOGGLE: return "event does not toggle its pin";
    case GTP_ETIMEOUT: return "bounded device wait expired";
    case GTP_EDEVICE: return "kernel reported an internal inconsistency";
    default: return "error";
  }
}

int check_device_error(gtp_ctx* ctx, const char* what) {
  CU(cudaMemcpyAsync(ctx->h_err, ctx->d_err.p, sizeof(DevError), cudaMemcpyDeviceToHost, ctx->stream), "read status");
  CU(cudaStreamSynchronize(ctx->stream), what);
  if (ctx->h_err->code != 0) {
    char buf[256];
    const long long idx = (long long)ctx->h_err->index;
    if (idx >= 0)
      snprintf(buf, sizeof buf, "%s: %s at record %lld", what, code_name(ctx->h_err->code), idx);
    else
      snprintf(buf, sizeof buf, "%s: %s at gate %lld", what, code_name(ctx->h_err->code), -1 - idx);
    return fail(ctx, ctx->h_err->code, buf);
  }
  return GTP_OK;
}

// Status of a walk over the n_win planned windows (window slots ids[]).  The
// walk flags a malformed trace without classifying it exactly; the exact
// first bad record (smallest window, then record) is found by the trace
// check before the error is reported, so the code and index match the
// oracle's and do not depend on thread timing.
int check_walk_error(gtp_ctx* ctx, int n_win, const int32_t* ids, const char* what) {
  CU(cudaMemcpyAsync(ctx->h_err, ctx->d_err.p, sizeof(DevError), cudaMemcpyDeviceToHost, ctx->stream), "read status");
  CU(cudaStreamSynchronize(ctx->stream), what);
  if (ctx->h_err->code == 0) return GTP_OK;
  if (ctx->h_err->index < 0 || n_win <= 0) return check_device_error(ctx, what);
  CU(ctx->first_bad.reserve(sizeof(unsigned long long)), "alloc trace check");
  CU(launch_validate(ctx->L, ctx->N, plan_wins(ctx->plan.p), n_win, ctx->first_bad.as<unsigned long long>(),
                     ctx->stream), "trace check");
  unsigned long long key = ~0ull;
  CU(cudaMemcpyAsync(&key, ctx->first_bad.p, sizeof key, cudaMemcpyDeviceToHost, ctx->stream), "read trace check");
  CU(cudaStreamSynchronize(ctx->stream), what);
  if (key == ~0ull) return check_device_error(ctx, what);
  const int code = -(int)(key & 7ull);
  const long long rec = (long long)((key >> 3) & ((1ull << 40) - 1ull));
  const int w = (int)(key >> 43);
  char buf[256];
  if (n_win > 1)
    snprintf(buf, sizeof buf, "%s: %s at record %lld of window %d", what, code_name(code), rec, ids[w]);
  else
    snprintf(buf, sizeof buf, "%s: %s at record %lld", what, code_name(code), rec);
  ctx->h_err->code = code;
  ctx->h_err->index = rec;
  return fail(ctx, code, buf);
}

Window* get_window(gtp_ctx* ctx, int32_t w) {
  auto it = ctx->windows.find(w);
  if (it == ctx->windows.end() || !it->second.loaded) return nullptr;
  return &it->second;
}

int64_t seg_len_of(const gtp_ctx* ctx) { return 32 * ctx->p_rpt; }

// Gates with more events than dense_min are walked by warps, the others one
// per thread.  A thread walks its gate's events one after another, so a
// sparse item (256 gates of similar count) lasts about dense_min event
// latencies: a large dense_min pays off only when there is enough work to
// hide the longest items.  Forward walk ms on the large recipe scaled from
// 10M to 200M events (dense_min 256 / 384 / 512 / 768): 10M 0.164 / 0.227 /
// 0.276 / 0.371, 20M 0.182 / 0.244 / 0.310 / 0.421, 40M 0.300 / 0.296 /
// 0.309 / 0.449, 70M 0.475 / 0.468 / 0.469 / 0.477, 100M 0.638 / 0.628 /
// 0.628 / 0.629, 200M 1.204 / 1.185 / 1.181 / 1.178.  The adjoint, whose
// sparse threads wait on a gradient load per event, stays at 256 (large:
// 1.408 ms at 256, 1.449 at 512).  With glitch detection the dense segments
// cost more (per-pin prefixes), so more gates go to threads: glitch walk ms
// (dense_min 256 / 384 / 512 / 768 / 1024) 20M 0.298 / 0.294 / 0.294 /
// 0.337 / 0.430, 40M 0.499 / 0.488 / 0.486 / 0.483 / 0.479, 100M 1.036 /
// 1.010 / 0.999 / 0.987 / 0.980, 200M 1.959 / 1.903 / 1.878 / 1.850 / 1.833.
// The adjoint (without glitch detection) stages its sparse threads' gate
// tables below this many events per SM.
constexpr int64_t kBwdStagedBelow = 200000;

int dense_min_auto(int64_t events_per_sm, bool backward, bool glitch) {
  if (backward) return 256;
  if (glitch) return events_per_sm < 200000 ? 384 : 1024;
  if (events_per_sm < 260000) return 256;
  return events_per_sm < 600000 ? 384 : 512;
}

// Fill the descriptor table of a run in the pinned staging buffer, reserving
// the windows' device buffers.  The upload is enqueued by upload_plan().
int build_plan(gtp_ctx* ctx, const std::vector<Window*>& ws, int32_t bin_ps, const std::vector<double*>& waves,
               bool backward, int64_t* n_seg_total, int64_t* n_tiles_total,
               const std::vector<double*>* cwaves = nullptr, bool tiled = false) {
  const int n = (int)ws.size();
  if (n <= 0 || n > kMaxWindows) return fail(ctx, GTP_EINVAL, "between 1 and 1024 windows per run");
  WinDesc* hw = plan_wins(ctx->h_plan);
  int64_t* ht = plan_tile_base(ctx->h_plan);
  double* dl0 = plan_l0(ctx->plan.p);
  const int64_t G = ctx->N.n_gates;
  const int64_t seg_len = seg_len_of(ctx);
  int64_t sb = 0, tb = 0;
  for (int i = 0; i < n; ++i) {
    Window& W = *ws[i];
    if (bin_ps <= 0 || W.window_ps % bin_ps != 0)
      return fail(ctx, GTP_ERANGE, "window_ps must be a multiple of bin_ps > 0");
    const int64_t nb = W.window_ps / bin_ps;
    const int64_t n_seg = W.n_events / seg_len + G + 1;  // bound on the dense segments of this window (reported)
    const int nt = merge_tiles((int)nb);
    CU(W.e_leak.reserve(sizeof(double) * G), "alloc e_leak");
    CU(W.e_int.reserve(sizeof(double) * G), "alloc e_int");
    CU(W.e_sw.reserve(sizeof(double) * G), "alloc e_sw");
    if (ctx->N.clock_ps > 0) CU(W.e_gl.reserve(sizeof(double) * G), "alloc e_gl");
    CU(W.final_state.reserve((size_t)G), "alloc final_state");
    CU(W.bins.reserve(sizeof(float2) * nb), "alloc bins");
    CU(W.tiles.reserve(sizeof(double) * (size_t)nt), "alloc tiles");
    WinDesc d{};
    d.offsets = W.offsets.as<int64_t>();
    d.rec = W.rec();
    d.init = W.init.as<uint8_t>();
    d.e_leak = W.e_leak.as<double>();
    d.e_int = W.e_int.as<double>();
    d.e_sw = W.e_sw.as<double>();
    d.e_gl = ctx->N.clock_ps > 0 ? W.e_gl.as<double>() : nullptr;
    d.final_state = W.final_state.as<uint8_t>();
    d.bins = W.bins.as<float2>();
    d.tbins = nullptr;
    const bool pat = W.pat_loaded && ctx->pat_net_ok;
    if (tiled) {
      CU(W.tbins.reserve(sizeof(double2) * nb), "alloc FP64 bins");
      d.tbins = W.tbins.as<double2>();
    }
    d.p_n_items = 0;
    d.p_off = nullptr;
    d.p_dC = nullptr;
    if (pat) {
      d.p_off = W.pat_off.as<int64_t>();
      d.p_rec = W.pat_rec.as<uint2>();
      d.p_init = W.pat_init.as<uint32_t>();
      d.p_items = W.pat_items.as<int2>();
      d.p_first = W.pat_first.as<int64_t>();
      d.p_mask = W.pat_mask.as<uint32_t>();
      d.p_e_leak = W.pat_e_leak.as<double>();
      d.p_e_int = W.pat_e_int.as<double>();
      d.p_e_sw = W.pat_e_sw.as<double>();
      d.p_e_gl = W.pat_e_gl.as<double>();
      d.p_final = W.pat_final.as<uint32_t>();
      d.p_n_items = W.pat_n_items;
      d.p_dC = nullptr;
      if (backward) {
        CU(W.pat_dC.reserve(sizeof(float) * (size_t)std::max<int64_t>(ctx->Q.n_gates, 1)), "alloc pattern gradients");
        d.p_dC = W.pat_dC.as<float>();
      }
    }
    d.cbins = nullptr;
    d.cwave = nullptr;
    if (cwaves && (*cwaves)[i]) {
      CU(W.cbins.reserve(sizeof(float4) * nb), "alloc component bins");
      d.cbins = W.cbins.as<float4>();
      d.cwave = (*cwaves)[i];
      d.cpack = ctx->N.clock_ps > 0 ? 0 : 1;
    }
    d.l0 = dl0 + i;
    d.tiles = W.tiles.as<double>();
    d.wave = waves.empty() ? nullptr : waves[i];
    d.grad = backward ? ctx->grad.as<float2>() : nullptr;
    d.dC = nullptr;
    d.n_events = W.n_events;
    d.tile_base = tb;
    d.g0 = 0;
    d.g1 = G;
    d.keep_bins = 0;
    d.n_tiles = nt;
    d.window_ps = (int32_t)W.window_ps;
    d.bin_ps = bin_ps;
    bin_magic(bin_ps, &d.bin_magic, &d.bin_shift);
    d.n_bins = (int32_t)nb;
    hw[i] = d;
    ht[i] = tb;
    sb += n_seg;
    tb += nt;
  }
  ht[n] = tb;
  // window groups: consecutive windows whose bins (8 B each) together stay within p_group_bytes are walked in one
  // launch; a larger set is walked group after group, so that the bins the walk reduces into stay in L2
  ctx->run_groups.clear();
  int64_t e_total = 0;
  {
    int a = 0;
    int64_t bytes = 0, ev = 0;
    for (int i = 0; i < n; ++i) {
      const int64_t b = (int64_t)sizeof(float2) * hw[i].n_bins;
      if (i > a && bytes + b > ctx->p_group_bytes) {
        ctx->run_groups.emplace_back(a, i);
        e_total = std::max(e_total, ev);
        a = i;
        bytes = 0;
        ev = 0;
      }
      bytes += b;
      ev += ws[i]->n_events;
    }
    ctx->run_groups.emplace_back(a, n);
    e_total = std::max(e_total, ev);
  }
  // pieces: a gate with more than piece_len events is walked as several big items, so that no single gate
  // of a skewed trace walks longer than about a sixth of an SM's even share of its group's walk
  int64_t pl = ctx->p_piece_len;
  if (pl < 0) pl = std::max<int64_t>(65536, e_total / (6 * std::max(ctx->n_sm, 1)));
  if (pl > 0) pl = (pl + kPieceUnit - 1) / kPieceUnit * kPieceUnit;
  int64_t e_all = 0;
  for (Window* w : ws) e_all += w->n_events;
  if (pl > 0 && e_all / pl >= (int64_t)1 << 20) pl = (e_all >> 20) / kPieceUnit * kPieceUnit + kPieceUnit;
  ctx->run_piece_len = pl;
  ctx->run_dense_min = ctx->p_dense_min > 0 ? ctx->p_dense_min
                                            : dense_min_auto(e_total / std::max(ctx->n_sm, 1), backward,
                                                             ctx->N.clock_ps > 0);
  ctx->run_whole = true;
  for (Window* w : ws)
    if (pl > 0 && (w->streamed || (int64_t)w->max_count > pl)) ctx->run_whole = false;
  const int64_t cap = (int64_t)n * G + (pl > 0 ? e_all / pl + n : 0);
  if (cap > ctx->gcap) {
    CU(ctx->glist.reserve(sizeof(int2) * (size_t)cap), "alloc work list");
    ctx->gcap = cap;
    ++ctx->plan_gen;
  }
  if (!ctx->counters.p) {
    CU(ctx->counters.reserve(sizeof(unsigned long long) * plan_counter_slots(4096)), "alloc plan counters");
    ++ctx->plan_gen;
  }
  *n_seg_total = sb;
  *n_tiles_total = tb;
  return GTP_OK;
}

int upload_plan(gtp_ctx* ctx, int n, cudaStream_t st) {
  CU(cudaMemcpyAsync(ctx->plan.p, ctx->h_plan, sizeof(WinDesc) * n, cudaMemcpyHostToDevice, st), "upload plan");
  CU(cudaMemcpyAsync(plan_tile_base(ctx->plan.p), plan_tile_base(ctx->h_plan), sizeof(int64_t) * (kMaxWindows + 1),
                     cudaMemcpyHostToDevice, st), "upload plan bases");
  return GTP_OK;
}

WalkArgs walk_args(gtp_ctx* ctx, int n) {
  WalkArgs A{};
  A.wins = plan_wins(ctx->plan.p);
  A.n_win = n;
  A.rpt = (int)ctx->p_rpt;
  A.dense_min = (int)ctx->run_dense_min;  // set by build_plan
  A.grid = ctx->p_ctas_per_sm > 0 ? (int)(ctx->p_ctas_per_sm * ctx->n_sm) : 0;
  A.n_sm = ctx->n_sm;
  A.err = ctx->d_err.as<DevError>();
  A.cell_acc = ctx->cell_acc.as<double>();
  A.gtab = ctx->gtab.as<float>();
  A.gtab_bwd = ctx->gtab_bwd.as<float>();
  A.plan.glist = ctx->glist.as<int2>();
  A.plan.counters = ctx->counters.as<unsigned long long>();
  A.plan.gcap = ctx->gcap;
  A.n_gates = ctx->N.n_gates;
  A.tile_min = 0;
  A.chunks = ctx->chunks.as<int32_t>();
  A.piece_len = ctx->run_piece_len;
  A.whole = false;
  return A;
}

// Phase boundary i (0..7); on a capturing stream the record becomes an
// event-record node of the graph and is re-recorded at every replay.
void mark(gtp_ctx* ctx, int i, cudaStream_t st) {
  if (!ctx->timing || (ctx->timing == 2 && i != 4 && i != 5)) return;  // marks 12, 13: the preparation pass
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(st, &cs);
  cudaEventRecordWithFlags(ctx->ev[i], st, cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : 0u);
}

void collect_timing(gtp_ctx* ctx) {
  if (!ctx->timing) return;
  for (int k = 0; k < (ctx->run_pat_items >= 0 ? 6 : 5); ++k) {
    if (ctx->timing == 2 && k != 2) continue;  // only the walk's pair was recorded
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ctx->ev[2 * k], ctx->ev[2 * k + 1]) == cudaSuccess)
      ctx->t_ns[k] += (int64_t)(ms * 1e6);
  }
  if (ctx->prep_marked) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ctx->ev[12], ctx->ev[13]) == cudaSuccess) ctx->t_ns[6] += (int64_t)(ms * 1e6);
    ctx->prep_marked = false;
  }
  ctx->n_timed += 1;
}

// Whether a forward run takes the time-sliced walk for its busiest gates:
// one window, no per-component bins, no glitch detection, the fused walk, a
// library whose leakage table fits, and the chunk buffer in place.
bool tiling_on(const gtp_ctx* ctx, int n, bool comp) {
  return n == 1 && !comp && ctx->N.clock_ps == 0 && ctx->p_kernel != 1 && ctx->p_tile_min > 0 &&
         tiled_fits(ctx->L) && ctx->chunks.p != nullptr;
}

// Enqueue the forward pass of the planned windows (no synchronisation).
int enqueue_forward(gtp_ctx* ctx, int n, int64_t n_seg_total, int64_t n_tiles_total, bool any_events,
                    cudaStream_t st, bool comp = false) {
  const WinDesc* dw = plan_wins(ctx->plan.p);
  const int64_t* tile_base = plan_tile_base(ctx->plan.p);
  RC(upload_plan(ctx, n, st));
  CU(cudaMemsetAsync(plan_l0(ctx->plan.p), 0, sizeof(double) * n, st), "zero l0");
  WalkArgs A = walk_args(ctx, n);
  A.comp = comp;
  A.whole = ctx->run_whole;
  const bool fused = any_events && ctx->p_kernel != 1;
  const bool tiled = fused && tiling_on(ctx, n, comp);
  if (tiled) A.tile_min = ctx->p_tile_min;
  // the fused walk takes the window groups one after another (a later group's preparation and plan are timed
  // as walk time); the per-gate walk and runs without events take all windows at once
  const std::vector<std::pair<int, int>> all{{0, n}};
  const auto& groups = fused ? ctx->run_groups : all;
  for (size_t k = 0; k < groups.size(); ++k) {
    WalkArgs Ag = A;
    Ag.wins = A.wins + groups[k].first;
    Ag.n_win = groups[k].second - groups[k].first;
    if (k == 0) mark(ctx, 0, st);
    CU(launch_prepare(ctx->L, ctx->N, Ag, fused, st), "prepare");
    ctx->launches += 1;
    if (k == 0) {
      mark(ctx, 1, st);
      mark(ctx, 2, st);
    }
    if (any_events) {
      if (!fused) {
        mark(ctx, 3, st);
        mark(ctx, 4, st);
        CU(launch_walk_per_gate(ctx->L, ctx->N, dw, n, ctx->d_err.as<DevError>(), st), "walk (per gate)");
        ctx->launches += 1;
      } else {
        CU(launch_plan_scatter(ctx->L, ctx->N, Ag, st), "plan");
        if (k == 0) {
          mark(ctx, 3, st);
          mark(ctx, 4, st);
          mark(ctx, 8, st);
        }
        if (tiled) {
          CU(launch_tiled(ctx->L, ctx->N, Ag, plan_wins(ctx->h_plan)[0].n_bins, st), "tiled walk");
          ctx->launches += 2;
        }
        if (k == 0) mark(ctx, 9, st);
        CU(launch_walk(ctx->L, ctx->N, Ag, false, st), "walk");
        ctx->launches += 2;
      }
    } else {
      mark(ctx, 3, st);
      mark(ctx, 4, st);
    }
  }
  if (ctx->run_pat_items >= 0) {  // the pattern gates, into the windows' FP64 bins and L0 (timed as walk)
    CU(cudaMemsetAsync(ctx->pat_bad.p, 0xFF, sizeof(unsigned long long), st), "reset pattern status");
    mark(ctx, 10, st);
    CU(launch_pattern_walk(ctx->P, ctx->Q, dw, n, ctx->run_pat_items, ctx->N.clock_ps,
                           ctx->pat_bad.as<unsigned long long>(), st), "pattern walk");
    mark(ctx, 11, st);
    ctx->launches += ctx->run_pat_items > 0 ? 3 : 1;
  }
  mark(ctx, 5, st);
  mark(ctx, 6, st);
  CU(launch_merge(dw, tile_base, n, n_tiles_total, st), "merge");
  ctx->launches += 3;
  mark(ctx, 7, st);
  return GTP_OK;
}

// The event descriptors of a new netlist or load are built with the gate
// tables, at the next run (ensure_gate_tables).
int ensure_netlist_coords(gtp_ctx* ctx) {
  const int64_t G = ctx->N.n_gates;
  ctx->N.dstride = 2 * (ctx->N.stride + 1);
  CU(ctx->desc.reserve(sizeof(uint4) * ctx->N.dstride * G), "alloc event descriptors");
  ctx->N.desc = ctx->desc.as<uint4>();
  ctx->desc_ok = false;
  ctx->gtab_ok = false;
  ctx->gtab_bwd_ok = false;
  return GTP_OK;
}

// Event descriptors and per-gate energy tables for the walk (forward: scaled
// energies; adjoint: unscaled energies and load derivatives), rebuilt in one
// pass after a netlist, load, scale or library change.  Every run calls this
// before its first launch that reads them.
int ensure_gate_tables(gtp_ctx* ctx, bool backward) {
  const int64_t G = ctx->N.n_gates;
  const bool need_d = !ctx->desc_ok, need_f = !ctx->gtab_ok, need_b = backward && !ctx->gtab_bwd_ok;
  if (!need_d && !need_f && !need_b) return GTP_OK;
  if (need_f) CU(ctx->gtab.reserve(sizeof(float) * kGateTab * (size_t)G), "alloc gate tables");
  if (need_b) CU(ctx->gtab_bwd.reserve(sizeof(float) * 2 * kGateTab * (size_t)G), "alloc adjoint gate tables");
  mark(ctx, 12, ctx->stream);
  CU(launch_gate_prep(ctx->L, ctx->N, need_d ? ctx->desc.as<uint4>() : nullptr, need_f ? ctx->gtab.as<float>() : nullptr,
                      need_b ? ctx->gtab_bwd.as<float>() : nullptr, ctx->stream), "gate tables");
  mark(ctx, 13, ctx->stream);
  ctx->prep_marked = ctx->timing == 1;
  ctx->launches += 1;
  ctx->desc_ok = true;
  ctx->gtab_ok |= need_f;
  ctx->gtab_bwd_ok |= need_b;
  return GTP_OK;
}

void drop_graphs(gtp_ctx* ctx) {
  for (auto& kv : ctx->graphs) cudaGraphExecDestroy(kv.second);
  ctx->graphs.clear();
}

__global__ void k_check_cells(const int32_t* cell, int64_t n, int32_t n_cells, DevError* err) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    if (cell[g] < 0 || cell[g] >= n_cells) report_error(err, GTP_ERANGE, -1 - g);
}

// Offsets checked (from 0 to n_events, never decreasing), and the busiest
// gate's event count into *max_count.  With device inputs the same pass
// copies the offsets (src -> dst) and the initial states (init_src ->
// init_dst) into the window's buffers, so a load is one launch and one
// readback; with host inputs they were copied before (src == dst, no init).
__global__ void k_load_offsets(const int64_t* src, int64_t* dst, const uint8_t* init_src, uint8_t* init_dst,
                               int64_t n_gates, int64_t n_events, DevError* err, unsigned long long* max_count) {
  int64_t mx = 0;
  const bool copy = src != dst;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n_gates;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o0 = src[g], o1 = src[g + 1];
    const int64_t c = o1 - o0;
    if (c < 0) report_error(err, GTP_EINVAL, -1 - g);
    mx = c > mx ? c : mx;
    if (copy) dst[g] = o0;
    if (init_dst) init_dst[g] = init_src[g];
  }
  for (int o = 16; o > 0; o >>= 1) {
    const int64_t y = __shfl_xor_sync(0xFFFFFFFFu, mx, o);
    mx = y > mx ? y : mx;
  }
  __shared__ int64_t wmax[32];  // one atomic a block
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mx = wmax[w] > mx ? wmax[w] : mx;
    if (mx > 0) atomicMax(max_count, (unsigned long long)mx);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const int64_t last = src[n_gates];
    if (copy) dst[n_gates] = last;
    if (src[0] != 0 || last != n_events) report_error(err, GTP_EINVAL, -1);
  }
}

// Per-gate results of a run into device outputs in one pass (null outputs
// are skipped): energies and final states copied, counts from the offsets.
__global__ void k_gate_out(const double* el, const double* ei, const double* es, const uint8_t* fs,
                           const int64_t* off, int64_t n, double* o_el, double* o_ei, double* o_es, int64_t* o_cnt,
                           uint8_t* o_fs) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    if (o_el) o_el[g] = el[g];
    if (o_ei) o_ei[g] = ei[g];
    if (o_es) o_es[g] = es[g];
    if (o_cnt) o_cnt[g] = off[g + 1] - off[g];
    if (o_fs) o_fs[g] = fs[g];
  }
}

// State-indexed arrays of the pattern cells with at most p_sipl_max_pins
// pins (and at most GTP_MAX_INDEXED_PINS), built on the device from their
// patterns; the others are walked by traversal.
int ensure_pattern_index(gtp_ctx* ctx) {
  if (ctx->pat_index_ok) return GTP_OK;
  int64_t ni = 0, nl = 0;
  int32_t n_idx = 0;
  for (PatCell& c : ctx->h_pat_cells) {
    const int pins = c.n_in + 1;
    if (pins <= ctx->p_sipl_max_pins && pins <= GTP_MAX_INDEXED_PINS) {
      c.iidx = ni;
      c.lidx = nl;
      ni += (int64_t)c.n_in << c.n_in;  // n_in pins x 2 edges x 2^(n_in - 1) side states
      nl += 2ll << c.n_in;
      ++n_idx;
    } else {
      c.iidx = c.lidx = -1;
    }
  }
  drop_graphs(ctx);
  CU(cudaStreamSynchronize(ctx->stream), "pattern index");
  if (ni > 0) {
    CU(ctx->pc_iidx.reserve(sizeof(int32_t) * (size_t)ni), "alloc pattern index");
    CU(ctx->pc_lidx.reserve(sizeof(float) * (size_t)nl), "alloc pattern index");
  }
  CU(cudaMemcpyAsync(ctx->pc_cells.p, ctx->h_pat_cells.data(), sizeof(PatCell) * ctx->h_pat_cells.size(),
                     cudaMemcpyHostToDevice, ctx->stream), "copy pattern cells");
  ctx->P.iidx = ctx->pc_iidx.as<int32_t>();
  ctx->P.lidx = ctx->pc_lidx.as<float>();
  for (size_t c = 0; c < ctx->h_pat_cells.size(); ++c)
    if (ctx->h_pat_cells[c].iidx >= 0) {
      CU(launch_pattern_index(ctx->P, (int32_t)c, ctx->h_pat_cells[c].n_in, ctx->pc_iidx.as<int32_t>(),
                              ctx->pc_lidx.as<float>(), ctx->stream), "pattern index");
      ctx->launches += 1;
    }
  CU(cudaStreamSynchronize(ctx->stream), "pattern index");
  ctx->pat_index_bytes = 4 * (ni + nl);
  ctx->pat_indexed = n_idx;
  ctx->pat_index_ok = true;
  return GTP_OK;
}

// Status of the pattern walk of a run over windows ids[0, n_win): its
// smallest error key (see launch_pattern_walk), or GTP_OK.
int check_pattern_error(gtp_ctx* ctx, int n_win, const int32_t* ids, const char* what) {
  unsigned long long key = ~0ull;
  CU(cudaMemcpyAsync(&key, ctx->pat_bad.p, sizeof key, cudaMemcpyDeviceToHost, ctx->stream), "read pattern status");
  CU(cudaStreamSynchronize(ctx->stream), what);
  if (key == ~0ull) return GTP_OK;
  const int code = -(int)(key & 7ull);
  const long long rec = (long long)((key >> 3) & ((1ull << 40) - 1ull));
  const int w = (int)(key >> 43);
  char buf[256];
  if (n_win > 1)
    snprintf(buf, sizeof buf, "%s: %s at pattern record %lld of window %d", what, code_name(code), rec, ids[w]);
  else
    snprintf(buf, sizeof buf, "%s: %s at pattern record %lld", what, code_name(code), rec);
  ctx->h_err->code = code;
  ctx->h_err->index = rec;
  return fail(ctx, code, buf);
}

// Forward run of a window list; waveforms per window (device or host).
int run_forward(gtp_ctx* ctx, const int32_t* windows, int n, int32_t bin_ps, double* const* waveforms, int flags,
                bool use_graph, double* const* components = nullptr) {
  if (!ctx->net_loaded) return fail(ctx, GTP_EINVAL, "run_power: load the library, netlist and events first");
  std::vector<Window*> ws(n);
  bool any_events = false;
  for (int i = 0; i < n; ++i) {
    ws[i] = get_window(ctx, windows[i]);
    if (!ws[i] || ws[i]->streamed) return fail(ctx, GTP_EINVAL, "run_power: window not loaded");
    for (int j = 0; j < i; ++j)
      if (windows[j] == windows[i]) return fail(ctx, GTP_EINVAL, "run_power: a window is listed twice");
    any_events |= ws[i]->n_events > 0;
  }
  if (bin_ps <= 0) return fail(ctx, GTP_ERANGE, "window_ps must be a multiple of bin_ps > 0");
  // pattern gates of the windows: the launch size of their walk (-1: none)
  ctx->run_pat_items = -1;
  if (ctx->pat_net_ok)
    for (Window* w : ws)
      if (w->pat_loaded) ctx->run_pat_items = std::max(ctx->run_pat_items, w->pat_n_items);
  if (ctx->run_pat_items >= 0) {
    RC(ensure_pattern_index(ctx));
    CU(ctx->pat_bad.reserve(sizeof(unsigned long long)), "alloc pattern status");
  }
  std::vector<double*> waves(n, nullptr);
  for (int i = 0; i < n; ++i) {
    if (!waveforms || !waveforms[i]) continue;
    if (flags & GTP_DEVICE) {
      waves[i] = waveforms[i];
    } else {
      CU(ws[i]->wave.reserve(sizeof(double) * (size_t)(ws[i]->window_ps / bin_ps)), "alloc waveform");
      waves[i] = ws[i]->wave.as<double>();
    }
  }
  std::vector<double*> cwaves(n, nullptr);
  if (components) {
    use_graph = false;
    for (int i = 0; i < n; ++i) {
      if (!components[i]) continue;
      if (flags & GTP_DEVICE) {
        cwaves[i] = components[i];
      } else {
        CU(ws[i]->cwave.reserve(4 * sizeof(double) * (size_t)(ws[i]->window_ps / bin_ps)), "alloc components");
        cwaves[i] = ws[i]->cwave.as<double>();
      }
    }
  }
  int64_t n_seg_total = 0, n_tiles_total = 0;
  RC(ensure_gate_tables(ctx, false));
  const bool want_tiled = n == 1 && !components && ctx->N.clock_ps == 0 && ctx->p_kernel != 1 &&
                          ctx->p_tile_min > 0 && tiled_fits(ctx->L) && any_events;
  if (want_tiled) {  // the tiled walk's chunk list (allocated here, never under capture)
    const size_t need = sizeof(int32_t) * (size_t)(tile_chunk_cap(ctx->N.n_gates) + 2);
    if (ctx->chunks.bytes < need) {
      CU(ctx->chunks.reserve(need), "alloc tile chunks");
      ++ctx->plan_gen;
    }
  }
  RC(build_plan(ctx, ws, bin_ps, waves, false, &n_seg_total, &n_tiles_total, components ? &cwaves : nullptr,
                want_tiled && tiling_on(ctx, n, false)));
  CU(cudaMemsetAsync(ctx->d_err.p, 0, sizeof(DevError), ctx->stream), "zero status");
  if (use_graph) {
    GraphKey key{std::vector<int32_t>(windows, windows + n), bin_ps, ctx->p_rpt,
                       ctx->p_ctas_per_sm, ctx->p_kernel, ctx->run_dense_min, ctx->p_tile_min, ctx->run_piece_len,
                       ctx->plan_gen,
                       n_tiles_total, any_events, ctx->timing, {}, ctx->run_pat_items, ctx->run_whole};
    for (const auto& gr : ctx->run_groups) key.groups.push_back(gr.first);
    auto it = ctx->graphs.find(key);
    if (it == ctx->graphs.end()) {
      if (!ctx->capture_stream) CU(cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking), "stream");
      const int64_t launches0 = ctx->launches;
      CU(cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
      const int rc = enqueue_forward(ctx, n, n_seg_total, n_tiles_total, any_events, ctx->capture_stream);
      cudaGraph_t graph = nullptr;
      cudaError_t ce = cudaStreamEndCapture(ctx->capture_stream, &graph);
      if (rc != GTP_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
      }
      CU(ce, "end capture");
      cudaGraphExec_t exec = nullptr;
      ce = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      CU(ce, "instantiate graph");
      it = ctx->graphs.emplace(key, exec).first;
      ctx->launches = launches0;
    }
    // the graph's first node uploads the descriptor table from the staging buffer
    CU(cudaGraphLaunch(it->second, ctx->stream), "graph launch");
    const int64_t ng = (int64_t)ctx->run_groups.size();
    ctx->launches += any_events ? (ctx->p_kernel == 1 ? 5 : 3 * ng + 3 + (tiling_on(ctx, n, false) ? 2 : 0)) : 4;
    if (ctx->run_pat_items >= 0) ctx->launches += ctx->run_pat_items > 0 ? 3 : 1;
  } else {
    RC(enqueue_forward(ctx, n, n_seg_total, n_tiles_total, any_events, ctx->stream, components != nullptr));
  }
  if (waveforms && !(flags & GTP_DEVICE)) {
    for (int i = 0; i < n; ++i)
      if (waveforms[i])
        CU(cudaMemcpyAsync(waveforms[i], waves[i], sizeof(double) * (size_t)(ws[i]->window_ps / bin_ps),
                           cudaMemcpyDeviceToHost, ctx->stream), "copy waveform");
  }
  if (components && !(flags & GTP_DEVICE)) {
    for (int i = 0; i < n; ++i)
      if (components[i])
        CU(cudaMemcpyAsync(components[i], cwaves[i], 4 * sizeof(double) * (size_t)(ws[i]->window_ps / bin_ps),
                           cudaMemcpyDeviceToHost, ctx->stream), "copy components");
  }
  int rc = check_walk_error(ctx, n, windows, "run_power");
  if (rc == GTP_OK && ctx->run_pat_items >= 0) rc = check_pattern_error(ctx, n, windows, "run_power");
  collect_timing(ctx);
  for (Window* w : ws) {
    w->has_result = (rc == GTP_OK);
    w->glitch_result = ctx->N.clock_ps > 0;
    w->last_bin_ps = bin_ps;
  }
  return rc;
}

// State patterns of the library for the schemes' traversal: each table's
// side-input state and each leakage entry's full state, in the library's
// order (the same order SIPL indexes).
int ensure_patterns(gtp_ctx* ctx) {
  if (ctx->pat_ok) return GTP_OK;
  std::vector<uint16_t> pi, pl;
  for (int32_t n : ctx->n_in) {
    for (int pin = 0; pin < n; ++pin)
      for (int e = 0; e < 2; ++e)
        for (int s = 0; s < (1 << (n - 1)); ++s) pi.push_back((uint16_t)s);
    for (int s = 0; s < (2 << n); ++s) pl.push_back((uint16_t)s);
  }
  CU(ctx->pat_int.reserve(sizeof(uint16_t) * pi.size()), "alloc patterns");
  CU(ctx->pat_leak.reserve(sizeof(uint16_t) * pl.size()), "alloc patterns");
  CU(cudaMemcpyAsync(ctx->pat_int.p, pi.data(), sizeof(uint16_t) * pi.size(), cudaMemcpyHostToDevice, ctx->stream),
     "copy patterns");
  CU(cudaMemcpyAsync(ctx->pat_leak.p, pl.data(), sizeof(uint16_t) * pl.size(), cudaMemcpyHostToDevice, ctx->stream),
     "copy patterns");
  CU(cudaStreamSynchronize(ctx->stream), "copy patterns");
  ctx->pat_ok = true;
  return GTP_OK;
}

// Event-density-aware partitioning of a window (Sec. 4.2), planned on the
// host: rho_g = N_evt(g) / N_cyc, rho_floor = n_evt_tgt / ceil(N_cyc /
// N_thr_floor), n_cyc(g) = round(n_evt_tgt / (rho_g + rho_floor)) clamped to
// [1, N_cyc], ceil(N_cyc / n_cyc(g)) threads in blocks of 128 per gate.
int plan_density(gtp_ctx* ctx, Window* W, int64_t n_bins) {
  const int64_t key[3] = {n_bins, ctx->p_evt_tgt, ctx->p_thr_floor};
  if (W->dplan_key[0] == key[0] && W->dplan_key[1] == key[1] && W->dplan_key[2] == key[2]) return GTP_OK;
  const int64_t G = ctx->N.n_gates;
  std::vector<int64_t> off((size_t)G + 1);
  CU(cudaMemcpyAsync(off.data(), W->offsets.p, sizeof(int64_t) * (G + 1), cudaMemcpyDeviceToHost, ctx->stream),
     "read offsets");
  CU(cudaStreamSynchronize(ctx->stream), "read offsets");
  const double tgt = (double)ctx->p_evt_tgt;
  const int64_t n_cyc_floor = (n_bins + ctx->p_thr_floor - 1) / ctx->p_thr_floor;
  const double rho_floor = tgt / (double)n_cyc_floor;
  std::vector<int32_t> ncyc((size_t)G);
  std::vector<int64_t> first((size_t)G);
  int64_t B = 0;
  for (int64_t g = 0; g < G; ++g) {
    const double rho = (double)(off[g + 1] - off[g]) / (double)n_bins;
    int64_t n = std::llround(tgt / (rho + rho_floor));
    n = std::min<int64_t>(std::max<int64_t>(n, 1), n_bins);
    const int64_t thr = (n_bins + n - 1) / n;
    ncyc[g] = (int32_t)n;
    first[g] = B;
    B += (thr + kSchemeTpb - 1) / kSchemeTpb;
  }
  if (B > 0x7FFFFFFFll) return fail(ctx, GTP_ERANGE, "run_power_scheme: more than 2^31 blocks");
  std::vector<int32_t> bg((size_t)B);
  for (int64_t g = 0; g < G; ++g) {
    const int64_t e = g + 1 < G ? first[g + 1] : B;
    for (int64_t b = first[g]; b < e; ++b) bg[b] = (int32_t)g;
  }
  CU(W->blk_gate.reserve(sizeof(int32_t) * (size_t)B), "alloc block plan");
  CU(W->blk_first.reserve(sizeof(int64_t) * (size_t)G), "alloc block plan");
  CU(W->ncyc.reserve(sizeof(int32_t) * (size_t)G), "alloc block plan");
  CU(cudaMemcpyAsync(W->blk_gate.p, bg.data(), sizeof(int32_t) * (size_t)B, cudaMemcpyHostToDevice, ctx->stream),
     "copy block plan");
  CU(cudaMemcpyAsync(W->blk_first.p, first.data(), sizeof(int64_t) * (size_t)G, cudaMemcpyHostToDevice, ctx->stream),
     "copy block plan");
  CU(cudaMemcpyAsync(W->ncyc.p, ncyc.data(), sizeof(int32_t) * (size_t)G, cudaMemcpyHostToDevice, ctx->stream),
     "copy block plan");
  CU(cudaStreamSynchronize(ctx->stream), "copy block plan");
  W->n_blocks = B;
  for (int i = 0; i < 3; ++i) W->dplan_key[i] = key[i];
  return GTP_OK;
}

}  // namespace

// =================================================================== C ABI
extern "C" {

int gtp_create(gtp_ctx** out, int device, void* cuda_stream) {
  if (!out) return GTP_EINVAL;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return GTP_ECUDA;
  gtp_ctx* ctx = new (std::nothrow) gtp_ctx();
  if (!ctx) return GTP_ENOMEM;
  ctx->device = device;
  ctx->stream = (cudaStream_t)cuda_stream;
  DeviceGuard dg(device);
  cudaDeviceGetAttribute(&ctx->n_sm, cudaDevAttrMultiProcessorCount, device);
  // status word: the first error, then the busiest gate's event count of the last load_events
  if (ctx->d_err.reserve(kStatusBytes) != cudaSuccess || ctx->plan.reserve(plan_bytes()) != cudaSuccess ||
      cudaMallocHost(&ctx->h_err, kStatusBytes) != cudaSuccess ||
      cudaMallocHost(&ctx->h_plan, plan_bytes()) != cudaSuccess) {
    ctx->d_err.release();
    ctx->plan.release();
    if (ctx->h_err) cudaFreeHost(ctx->h_err);
    delete ctx;
    return GTP_ENOMEM;
  }
  memset(ctx->h_plan, 0, plan_bytes());
  cudaMemset(ctx->d_err.p, 0, kStatusBytes);
  *out = ctx;
  return GTP_OK;
}

void gtp_destroy(gtp_ctx* ctx) {
  if (!ctx) return;
  DeviceGuard dg(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  cudaDeviceSynchronize();
  drop_graphs(ctx);
  if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
  if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
  for (int i = 0; i < 2; ++i) {
    if (ctx->ev_copied[i]) cudaEventDestroy(ctx->ev_copied[i]);
    if (ctx->ev_walked[i]) cudaEventDestroy(ctx->ev_walked[i]);
    ctx->chunk_buf[i].release();
    ctx->pk_buf[i].release();
  }
  for (auto& kv : ctx->windows) kv.second.release();
  for (DevBuf* b : {&ctx->tab, &ctx->leak, &ctx->cells, &ctx->table_cell, &ctx->leak_cell, &ctx->escale, &ctx->lscale,
                    &ctx->cell, &ctx->load, &ctx->slew, &ctx->desc, &ctx->plan, &ctx->glist, &ctx->gtab, &ctx->gtab_bwd,
                    &ctx->counters, &ctx->first_bad, &ctx->out_slew, &ctx->dp_scratch,
                    &ctx->cell_acc, &ctx->grad, &ctx->gtiles, &ctx->dC_scratch, &ctx->d_err, &ctx->pat_int,
                    &ctx->pat_leak, &ctx->sch_ebins, &ctx->sch_R, &ctx->probe, &ctx->chunks, &ctx->pc_cells,
                    &ctx->pc_ip, &ctx->pc_ipo, &ctx->pc_lp, &ctx->pc_tab, &ctx->pc_iidx, &ctx->pc_lidx,
                    &ctx->pn_cell, &ctx->pn_load, &ctx->pn_slew, &ctx->pn_oslew, &ctx->pn_desc, &ctx->pat_bad})
    b->release();
  for (auto& e : ctx->sch_ev)
    if (e) cudaEventDestroy(e);
  if (ctx->h_err) cudaFreeHost(ctx->h_err);
  if (ctx->h_plan) cudaFreeHost(ctx->h_plan);
  for (auto& e : ctx->ev)
    if (e) cudaEventDestroy(e);
  for (auto& e : ctx->ev_sx)
    if (e) cudaEventDestroy(e);
  delete ctx;
}

int gtp_set_stream(gtp_ctx* ctx, void* cuda_stream) {
  if (!ctx) return GTP_EINVAL;
  ctx->stream = (cudaStream_t)cuda_stream;
  return GTP_OK;
}

const char* gtp_last_error(const gtp_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int gtp_load_library(gtp_ctx* ctx, int32_t n_cells, const int32_t* n_in, float vdd, int32_t n_slew,
                     const float* slew_axis, int32_t n_load, const float* load_axis, const float* e_int,
                     int64_t n_e_int, const float* p_leak, int64_t n_p_leak) {
  if (!ctx) return GTP_EINVAL;
  if (n_cells <= 0 || n_cells > 256 || !n_in || !slew_axis || !load_axis || !e_int || !p_leak)
    return fail(ctx, GTP_EINVAL, "load_library: null array or n_cells not in [1, 256]");
  if (n_slew < 2 || n_slew > GTP_MAX_AXIS || n_load < 2 || n_load > GTP_MAX_AXIS)
    return fail(ctx, GTP_ERANGE, "load_library: axes need 2..16 points");
  for (int i = 0; i + 1 < n_slew; ++i)
    if (!(slew_axis[i + 1] > slew_axis[i])) return fail(ctx, GTP_EINVAL, "load_library: slew axis not increasing");
  for (int i = 0; i + 1 < n_load; ++i)
    if (!(load_axis[i + 1] > load_axis[i])) return fail(ctx, GTP_EINVAL, "load_library: load axis not increasing");
  int64_t n_tables = 0, n_leak = 0;
  int max_in = 0;
  std::vector<CellInfo> ci(n_cells);
  for (int c = 0; c < n_cells; ++c) {
    if (n_in[c] < 1 || n_in[c] > GTP_MAX_PINS - 1) return fail(ctx, GTP_ERANGE, "load_library: n_in must be 1..7");
    ci[c].tab_base = (int32_t)n_tables;
    ci[c].leak_base = (int32_t)n_leak;
    ci[c].n_in = n_in[c];
    ci[c].pad = 0;
    n_tables += (int64_t)n_in[c] * (2ll << (n_in[c] - 1));
    n_leak += 2ll << n_in[c];
    if (n_in[c] > max_in) max_in = n_in[c];
  }
  const int64_t tsize = (int64_t)n_slew * n_load;
  if (n_e_int != n_tables * tsize) return fail(ctx, GTP_EINVAL, "load_library: e_int size does not match the cells");
  if (n_p_leak != n_leak) return fail(ctx, GTP_EINVAL, "load_library: p_leak size does not match the cells");
  LibView L{};
  L.n_cells = n_cells;
  L.n_tables = (int32_t)n_tables;
  L.n_leak = (int32_t)n_leak;
  L.ns = n_slew;
  L.nl = n_load;
  L.tsize = (int32_t)tsize;
  if (smem_lib_bytes(L) > GTP_MAX_TABLE_BYTES || n_tables * tsize > 65535)
    return fail(ctx, GTP_ERANGE, "load_library: tables exceed the shared-memory budget");
  DeviceGuard dg(ctx->device);
  std::vector<uint8_t> tcell(n_tables), lcell(n_leak);
  for (int c = 0; c < n_cells; ++c) {
    const int64_t nt = (int64_t)n_in[c] * (2ll << (n_in[c] - 1));
    for (int64_t k = 0; k < nt; ++k) tcell[ci[c].tab_base + k] = (uint8_t)c;
    for (int64_t k = 0; k < (2ll << n_in[c]); ++k) lcell[ci[c].leak_base + k] = (uint8_t)c;
  }
  std::vector<float> ones(n_cells, 1.0f);
  CU(cudaStreamSynchronize(ctx->stream), "load_library");
  drop_graphs(ctx);
  CU(ctx->tab.reserve(sizeof(float) * n_e_int), "alloc tables");
  CU(ctx->leak.reserve(sizeof(float) * n_leak), "alloc leakage");
  CU(ctx->cells.reserve(sizeof(CellInfo) * n_cells), "alloc cells");
  CU(ctx->table_cell.reserve(n_tables), "alloc table_cell");
  CU(ctx->leak_cell.reserve(n_leak), "alloc leak_cell");
  CU(ctx->escale.reserve(sizeof(float) * n_cells), "alloc escale");
  CU(ctx->lscale.reserve(sizeof(float) * n_cells), "alloc lscale");
  CU(ctx->cell_acc.reserve(sizeof(double) * 2 * n_cells), "alloc cell_acc");
  CU(cudaMemcpy(ctx->tab.p, e_int, sizeof(float) * n_e_int, cudaMemcpyHostToDevice), "copy tables");
  CU(cudaMemcpy(ctx->leak.p, p_leak, sizeof(float) * n_leak, cudaMemcpyHostToDevice), "copy leakage");
  CU(cudaMemcpy(ctx->cells.p, ci.data(), sizeof(CellInfo) * n_cells, cudaMemcpyHostToDevice), "copy cells");
  CU(cudaMemcpy(ctx->table_cell.p, tcell.data(), n_tables, cudaMemcpyHostToDevice), "copy table_cell");
  CU(cudaMemcpy(ctx->leak_cell.p, lcell.data(), n_leak, cudaMemcpyHostToDevice), "copy leak_cell");
  CU(cudaMemcpy(ctx->escale.p, ones.data(), sizeof(float) * n_cells, cudaMemcpyHostToDevice), "copy escale");
  CU(cudaMemcpy(ctx->lscale.p, ones.data(), sizeof(float) * n_cells, cudaMemcpyHostToDevice), "copy lscale");
  L.tab = ctx->tab.as<float>();
  L.leak = ctx->leak.as<float>();
  L.cells = ctx->cells.as<CellInfo>();
  L.table_cell = ctx->table_cell.as<uint8_t>();
  L.leak_cell = ctx->leak_cell.as<uint8_t>();
  L.escale = ctx->escale.as<float>();
  L.lscale = ctx->lscale.as<float>();
  L.half_v2 = 0.5f * vdd * vdd;
  for (int i = 0; i < GTP_MAX_AXIS; ++i) {
    L.slew_axis[i] = i < n_slew ? slew_axis[i] : 0.f;
    L.load_axis[i] = i < n_load ? load_axis[i] : 0.f;
    L.slew_rw[i] = i + 1 < n_slew ? 1.0f / (slew_axis[i + 1] - slew_axis[i]) : 0.f;
    L.load_rw[i] = i + 1 < n_load ? 1.0f / (load_axis[i + 1] - load_axis[i]) : 0.f;
  }
  ctx->L = L;
  ctx->n_in.assign(n_in, n_in + n_cells);
  ctx->max_in = max_in;
  ctx->lib_loaded = true;
  ctx->pat_ok = false;
  for (auto& kv : ctx->windows) kv.second.ps_ok = false;
  ctx->desc_ok = false;
  ctx->gtab_ok = false;
  ctx->gtab_bwd_ok = false;
  ctx->net_loaded = false;
  for (auto& kv : ctx->windows) kv.second.release();
  ctx->windows.clear();
  return GTP_OK;
}

int gtp_set_scales(gtp_ctx* ctx, const float* escale, const float* lscale) {
  if (!ctx) return GTP_EINVAL;
  if (!ctx->lib_loaded) return fail(ctx, GTP_EINVAL, "set_scales: no library loaded");
  DeviceGuard dg(ctx->device);
  std::vector<float> ones(ctx->L.n_cells, 1.0f);
  CU(cudaMemcpyAsync(ctx->escale.p, escale ? escale : ones.data(), sizeof(float) * ctx->L.n_cells,
                     cudaMemcpyHostToDevice, ctx->stream), "copy escale");
  CU(cudaMemcpyAsync(ctx->lscale.p, lscale ? lscale : ones.data(), sizeof(float) * ctx->L.n_cells,
                     cudaMemcpyHostToDevice, ctx->stream), "copy lscale");
  CU(cudaStreamSynchronize(ctx->stream), "set_scales");
  ctx->gtab_ok = false;
  return GTP_OK;
}

int gtp_load_netlist(gtp_ctx* ctx, int64_t n_gates, const int32_t* cell, const float* load_ff,
                     const float* slew_ps, int32_t slew_stride, int flags) {
  if (!ctx) return GTP_EINVAL;
  if (!ctx->lib_loaded) return fail(ctx, GTP_EINVAL, "load_netlist: load the library first");
  if (n_gates <= 0 || n_gates >= (1ll << 31) || !cell || !load_ff || !slew_ps)
    return fail(ctx, GTP_EINVAL, "load_netlist: need 1 <= n_gates < 2^31 and non-null arrays");
  if (slew_stride < ctx->max_in || slew_stride > GTP_MAX_PINS)
    return fail(ctx, GTP_EINVAL, "load_netlist: slew_stride must cover the widest cell (and be <= 8)");
  DeviceGuard dg(ctx->device);
  CU(cudaStreamSynchronize(ctx->stream), "load_netlist");
  drop_graphs(ctx);
  const cudaMemcpyKind k = kind_in(flags);
  CU(ctx->cell.reserve(sizeof(int32_t) * n_gates), "alloc cell");
  CU(ctx->load.reserve(sizeof(float) * n_gates), "alloc load");
  CU(ctx->slew.reserve(sizeof(float) * 2 * slew_stride * n_gates), "alloc slew");
  CU(cudaMemcpyAsync(ctx->cell.p, cell, sizeof(int32_t) * n_gates, k, ctx->stream), "copy cell");
  CU(cudaMemcpyAsync(ctx->load.p, load_ff, sizeof(float) * n_gates, k, ctx->stream), "copy load");
  CU(cudaMemcpyAsync(ctx->slew.p, slew_ps, sizeof(float) * 2 * slew_stride * n_gates, k, ctx->stream), "copy slew");
  CU(cudaMemsetAsync(ctx->d_err.p, 0, sizeof(DevError), ctx->stream), "zero status");
  k_check_cells<<<1024, 256, 0, ctx->stream>>>(ctx->cell.as<int32_t>(), n_gates, ctx->L.n_cells,
                                                ctx->d_err.as<DevError>());
  CU(cudaGetLastError(), "check cells");
  ctx->launches += 1;
  const int rc = check_device_error(ctx, "load_netlist");
  if (rc != GTP_OK) return fail(ctx, GTP_ERANGE, "load_netlist: cell index out of range");
  ctx->N.cell = ctx->cell.as<int32_t>();
  ctx->N.load = ctx->load.as<float>();
  ctx->N.slew = ctx->slew.as<float>();
  ctx->N.n_gates = n_gates;
  ctx->N.stride = slew_stride;
  ctx->N.clock_ps = 0;  // glitch detection is set per netlist
  ctx->N.out_slew = nullptr;
  RC(ensure_netlist_coords(ctx));
  CU(cudaStreamSynchronize(ctx->stream), "load_netlist");
  ctx->net_loaded = true;
  for (auto& kv : ctx->windows) {
    kv.second.ps_ok = false;
    kv.second.dplan_key[0] = -1;
  }
  for (auto& kv : ctx->windows) kv.second.release();
  ctx->windows.clear();
  return GTP_OK;
}

int gtp_set_glitch(gtp_ctx* ctx, int64_t clock_ps, const float* out_slew_ps, int flags) {
  if (!ctx) return GTP_EINVAL;
  if (!ctx->net_loaded) return fail(ctx, GTP_EINVAL, "set_glitch: load the netlist first");
  if (clock_ps < 0 || clock_ps >= (1ll << 31)) return fail(ctx, GTP_ERANGE, "set_glitch: clock_ps must be in [0, 2^31)");
  if (clock_ps > 0 && !out_slew_ps) return fail(ctx, GTP_EINVAL, "set_glitch: out_slew_ps is null");
  DeviceGuard dg(ctx->device);
  CU(cudaStreamSynchronize(ctx->stream), "set_glitch");
  drop_graphs(ctx);
  if (clock_ps == 0) {
    ctx->N.clock_ps = 0;
    ctx->N.out_slew = nullptr;
    return GTP_OK;
  }
  const int64_t G = ctx->N.n_gates;
  CU(ctx->out_slew.reserve(sizeof(float) * 2 * (size_t)G), "alloc out_slew");
  CU(cudaMemcpyAsync(ctx->out_slew.p, out_slew_ps, sizeof(float) * 2 * (size_t)G, kind_in(flags), ctx->stream),
     "copy out_slew");
  CU(cudaStreamSynchronize(ctx->stream), "set_glitch");
  ctx->N.out_slew = ctx->out_slew.as<float>();
  ctx->N.clock_ps = (int32_t)clock_ps;
  bin_magic((int32_t)clock_ps, &ctx->N.clock_magic, &ctx->N.clock_shift);
  return GTP_OK;
}

int gtp_design_power(gtp_ctx* ctx, int32_t window, const double* waveform_w, int flags, double* out) {
  if (!ctx) return GTP_EINVAL;
  Window* W = get_window(ctx, window);
  if (!W || !W->has_result) return fail(ctx, GTP_EINVAL, "design_power: no result for this window");
  if (!out) return fail(ctx, GTP_EINVAL, "design_power: null output");
  DeviceGuard dg(ctx->device);
  const int64_t G = ctx->N.n_gates;
  const int64_t nb = W->last_bin_ps > 0 ? W->window_ps / W->last_bin_ps : 0;
  const double* wave = nullptr;
  if (waveform_w && nb > 0) {
    if (flags & GTP_DEVICE) {
      wave = waveform_w;
    } else {
      CU(W->wave.reserve(sizeof(double) * (size_t)nb), "alloc waveform");
      CU(cudaMemcpyAsync(W->wave.p, waveform_w, sizeof(double) * (size_t)nb, cudaMemcpyHostToDevice, ctx->stream),
         "copy waveform");
      wave = W->wave.as<double>();
    }
  }
  CU(ctx->dp_scratch.reserve(6 * sizeof(double)), "alloc design power");
  CU(launch_design_power(W->e_leak.as<double>(), W->e_int.as<double>(), W->e_sw.as<double>(),
                         W->glitch_result ? W->e_gl.as<double>() : nullptr, G, wave, nb,
                         ctx->dp_scratch.as<double>(), ctx->stream), "design power");
  ctx->launches += wave ? 2 : 1;
  double h[6];
  CU(cudaMemcpyAsync(h, ctx->dp_scratch.p, sizeof h, cudaMemcpyDeviceToHost, ctx->stream), "read design power");
  CU(cudaStreamSynchronize(ctx->stream), "design_power");
  if (W->pat_loaded && ctx->pat_net_ok) {  // the pattern gates' energies, added in gate order
    const int64_t Gp = ctx->Q.n_gates;
    std::vector<double> e((size_t)Gp);
    DevBuf* src[4] = {&W->pat_e_leak, &W->pat_e_int, &W->pat_e_sw, &W->pat_e_gl};
    for (int k = 0; k < 4; ++k) {
      CU(cudaMemcpyAsync(e.data(), src[k]->p, sizeof(double) * (size_t)Gp, cudaMemcpyDeviceToHost, ctx->stream),
         "read pattern energies");
      CU(cudaStreamSynchronize(ctx->stream), "design_power");
      for (double x : e) h[k] += x;
    }
  }
  const double to_w = 1e-3 / (double)W->window_ps;  // fJ over the window in ps -> W
  for (int k = 0; k < 4; ++k) out[k] = h[k] * to_w;
  out[4] = out[0] + out[1] + out[2] + out[3];
  unsigned long long idx;
  memcpy(&idx, h + 5, sizeof idx);
  if (wave && idx < (unsigned long long)nb) {
    CU(cudaMemcpyAsync(out + 5, wave + idx, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream), "read peak");
    CU(cudaStreamSynchronize(ctx->stream), "design_power");
    out[6] = (double)idx;
  } else {
    out[5] = 0.0;
    out[6] = -1.0;
  }
  return GTP_OK;
}

int gtp_gate_glitch(gtp_ctx* ctx, int32_t window, double* e_gl, int flags) {
  if (!ctx) return GTP_EINVAL;
  Window* W = get_window(ctx, window);
  if (!W || !W->has_result) return fail(ctx, GTP_EINVAL, "gate_glitch: no result for this window");
  if (!e_gl) return fail(ctx, GTP_EINVAL, "gate_glitch: null output");
  DeviceGuard dg(ctx->device);
  const size_t bytes = sizeof(double) * (size_t)ctx->N.n_gates;
  if (W->glitch_result) {
    CU(cudaMemcpyAsync(e_gl, W->e_gl.p, bytes, kind_out(flags), ctx->stream), "copy e_gl");
  } else if (flags & GTP_DEVICE) {
    CU(cudaMemsetAsync(e_gl, 0, bytes, ctx->stream), "zero e_gl");
  } else {
    memset(e_gl, 0, bytes);
  }
  CU(cudaStreamSynchronize(ctx->stream), "gate_glitch");
  return GTP_OK;
}

int gtp_set_load(gtp_ctx* ctx, const float* load_ff, int flags) {
  if (!ctx) return GTP_EINVAL;
  if (!ctx->net_loaded || !load_ff) return fail(ctx, GTP_EINVAL, "set_load: no netlist or null array");
  DeviceGuard dg(ctx->device);
  CU(cudaMemcpyAsync(ctx->load.p, load_ff, sizeof(float) * ctx->N.n_gates, kind_in(flags), ctx->stream), "copy load");
  RC(ensure_netlist_coords(ctx));
  CU(cudaStreamSynchronize(ctx->stream), "set_load");
  return GTP_OK;
}

int gtp_load_events(gtp_ctx* ctx, int32_t window, int64_t window_ps, int64_t n_events, const int64_t* gate_offsets,
                    const gtp_event* events, const uint8_t* init_state, int flags) {
  if (!ctx) return GTP_EINVAL;
  if (!ctx->net_loaded) return fail(ctx, GTP_EINVAL, "load_events: load the netlist first");
  if (window < 0 || window >= kMaxWindows) return fail(ctx, GTP_EINVAL, "load_events: window slot must be 0..1023");
  if (window_ps <= 0 || window_ps >= (1ll << 31))
    return fail(ctx, GTP_ERANGE, "load_events: window_ps must be in (0, 2^31)");
  if (n_events < 0 || !gate_offsets || !init_state || (n_events > 0 && !events))
    return fail(ctx, GTP_EINVAL, "load_events: null array or negative n_events");
  const bool borrow = (flags & GTP_BORROW) != 0;
  if (borrow && !(flags & GTP_DEVICE)) return fail(ctx, GTP_EINVAL, "load_events: GTP_BORROW needs GTP_DEVICE");
  if (borrow && (((uintptr_t)events) & 15))
    return fail(ctx, GTP_EINVAL, "load_events: borrowed events must be 16-byte aligned");
  const bool packed = (flags & GTP_PACKED) != 0;
  if (packed && borrow) return fail(ctx, GTP_EINVAL, "load_events: packed events cannot be borrowed");
  DeviceGuard dg(ctx->device);
  const int64_t G = ctx->N.n_gates;
  Window& W = ctx->windows[window];
  // buffers are kept and grown as needed, so reloading a slot does not reallocate; its pattern events go
  if (W.pat_loaded) {
    CU(cudaStreamSynchronize(ctx->stream), "load_events");
    W.release_patterns();
  }
  W.loaded = false;
  W.has_result = false;
  W.streamed = false;
  W.borrowed = nullptr;
  W.ps_ok = false;
  W.dplan_key[0] = -1;
  const cudaMemcpyKind k = kind_in(flags);
  CU(W.offsets.reserve(sizeof(int64_t) * (G + 1)), "alloc offsets");
  CU(W.init.reserve((size_t)G), "alloc init");
  const bool dev_in = (flags & GTP_DEVICE) != 0;  // device offsets and states are copied by the check pass
  if (!dev_in) {
    CU(cudaMemcpyAsync(W.offsets.p, gate_offsets, sizeof(int64_t) * (G + 1), k, ctx->stream), "copy offsets");
    CU(cudaMemcpyAsync(W.init.p, init_state, (size_t)G, k, ctx->stream), "copy init");
  }
  if (borrow) {
    W.borrowed = reinterpret_cast<const uint2*>(events);
  } else if (packed) {
    // the packed transfer form: words and anchors into an aligned staging buffer, then unpacked
    const int64_t nb = (n_events + 31) / 32, nw = (n_events + 3) & ~(int64_t)3;
    CU(W.records.reserve(sizeof(uint2) * (size_t)(n_events + 2)), "alloc records");
    CU(cudaMemsetAsync(W.records.as<uint2>() + n_events, 0, 2 * sizeof(uint2), ctx->stream), "zero padding");
    if (n_events > 0) {
      CU(ctx->pk_buf[0].reserve(sizeof(uint32_t) * (size_t)(nw + nb)), "alloc packed buffer");
      const uint32_t* src = reinterpret_cast<const uint32_t*>(events);
      uint32_t* pk = ctx->pk_buf[0].as<uint32_t>();
      CU(cudaMemcpyAsync(pk, src + nb, sizeof(uint32_t) * (size_t)n_events, k, ctx->stream), "copy packed words");
      CU(cudaMemcpyAsync(pk + nw, src, sizeof(uint32_t) * (size_t)nb, k, ctx->stream), "copy packed anchors");
      CU(launch_unpack(pk + nw, pk, 0, n_events, W.records.as<uint2>(), ctx->stream), "unpack");
      ctx->launches += 1;
    }
  } else {
    // padded by two records so that 16-byte vector loads stay in bounds
    const size_t bytes = sizeof(uint2) * (size_t)(n_events + 2);
    CU(W.records.reserve(bytes), "alloc records");
    CU(cudaMemsetAsync(W.records.as<uint2>() + n_events, 0, 2 * sizeof(uint2), ctx->stream), "zero padding");
    if (n_events > 0)
      CU(cudaMemcpyAsync(W.records.p, events, sizeof(uint2) * (size_t)n_events, k, ctx->stream), "copy records");
  }
  CU(cudaMemsetAsync(ctx->d_err.p, 0, kStatusBytes, ctx->stream), "zero status");
  unsigned long long* max_count =
      reinterpret_cast<unsigned long long*>(static_cast<unsigned char*>(ctx->d_err.p) + sizeof(DevError));
  k_load_offsets<<<1024, 256, 0, ctx->stream>>>(dev_in ? gate_offsets : W.offsets.as<int64_t>(), W.offsets.as<int64_t>(),
                                                dev_in ? init_state : nullptr, dev_in ? W.init.as<uint8_t>() : nullptr,
                                                G, n_events, ctx->d_err.as<DevError>(), max_count);
  CU(cudaGetLastError(), "check offsets");
  ctx->launches += 1;
  CU(cudaMemcpyAsync(ctx->h_err, ctx->d_err.p, sizeof(DevError) + sizeof(unsigned long long),
                     cudaMemcpyDeviceToHost, ctx->stream), "read status");
  CU(cudaStreamSynchronize(ctx->stream), "load_events");
  if (ctx->h_err->code != 0)
    return fail(ctx, GTP_EINVAL, "load_events: offsets must start at 0, end at n_events and not decrease");
  memcpy(&W.max_count, reinterpret_cast<unsigned char*>(ctx->h_err) + sizeof(DevError), sizeof(W.max_count));
  W.window_ps = window_ps;
  W.n_events = n_events;
  W.loaded = true;
  return GTP_OK;
}

int gtp_run_power(gtp_ctx* ctx, int32_t window, int32_t bin_ps, double* waveform_w, int flags) {
  if (!ctx) return GTP_EINVAL;
  if ((flags & GTP_GRAPH) && !(flags & GTP_DEVICE))
    return fail(ctx, GTP_EINVAL, "run_power: graph replay needs a device waveform");
  DeviceGuard dg(ctx->device);
  double* const waves[1] = {waveform_w};
  return run_forward(ctx, &window, 1, bin_ps, waves, flags, (flags & GTP_GRAPH) != 0);
}

int gtp_run_power_components(gtp_ctx* ctx, int32_t window, int32_t bin_ps, double* waveform_w,
                             double* components_w, int flags) {
  if (!ctx) return GTP_EINVAL;
  if (!components_w) return fail(ctx, GTP_EINVAL, "run_power_components: components_w is required");
  if (flags & GTP_GRAPH) return fail(ctx, GTP_EINVAL, "run_power_components: no graph replay");
  DeviceGuard dg(ctx->device);
  double* const waves[1] = {waveform_w};
  double* const comps[1] = {components_w};
  return run_forward(ctx, &window, 1, bin_ps, waves, flags, false, comps);
}

int gtp_run_power_scheme(gtp_ctx* ctx, int32_t window, int32_t bin_ps, int32_t scheme, double* waveform_w,
                         int flags, float* kernel_ms) {
  if (!ctx) return GTP_EINVAL;
  if (scheme < kSchemeNaive || scheme > kSchemeFused) return fail(ctx, GTP_EINVAL, "run_power_scheme: unknown scheme");
  if (flags & GTP_GRAPH) return fail(ctx, GTP_EINVAL, "run_power_scheme: no graph replay");
  if (!ctx->net_loaded) return fail(ctx, GTP_EINVAL, "run_power_scheme: load the library, netlist and events first");
  DeviceGuard dg(ctx->device);
  Window* W = get_window(ctx, window);
  if (!W || W->streamed) return fail(ctx, GTP_EINVAL, "run_power_scheme: window not loaded");
  if (W->pat_loaded && ctx->pat_net_ok)
    return fail(ctx, GTP_EINVAL,
                "run_power_scheme: windows with pattern gates are walked by gtp_run_power, gtp_run_power_batched "
                "and gtp_run_power_components only");
  if (bin_ps <= 0 || W->window_ps % bin_ps != 0) return fail(ctx, GTP_ERANGE, "window_ps must be a multiple of bin_ps > 0");
  const int64_t nb = W->window_ps / bin_ps;
  const int64_t G = ctx->N.n_gates;
  double* wave = nullptr;
  if (waveform_w) {
    if (flags & GTP_DEVICE) {
      wave = waveform_w;
    } else {
      CU(W->wave.reserve(sizeof(double) * (size_t)nb), "alloc waveform");
      wave = W->wave.as<double>();
    }
  }
  int64_t n_seg_total = 0, n_tiles_total = 0;
  RC(build_plan(ctx, std::vector<Window*>{W}, bin_ps, std::vector<double*>{wave}, false, &n_seg_total,
                &n_tiles_total));
  RC(upload_plan(ctx, 1, ctx->stream));
  CU(cudaMemsetAsync(ctx->d_err.p, 0, sizeof(DevError), ctx->stream), "zero status");
  const WinDesc* dw = plan_wins(ctx->plan.p);
  if (!W->ps_ok) {  // the paper's input form: one event stream per (gate, pin), checked as the walk checks
    CU(W->ps_off.reserve(sizeof(int64_t) * 9 * (size_t)G), "alloc pin streams");
    CU(W->ps_ev.reserve(sizeof(uint32_t) * (size_t)W->n_events), "alloc pin streams");
    CU(W->ps_slot.reserve(sizeof(uint32_t) * (size_t)W->n_events), "alloc pin streams");
    CU(launch_pin_streams(ctx->L, ctx->N, dw,
                          PinStreams{W->ps_off.as<int64_t>(), W->ps_ev.as<uint32_t>(), W->ps_slot.as<uint32_t>()},
                          ctx->d_err.as<DevError>(), ctx->stream), "pin streams");
    RC(check_walk_error(ctx, 1, &window, "run_power_scheme"));
    W->ps_ok = true;
  }
  RC(ensure_patterns(ctx));
  if (scheme >= kSchemeDensity) RC(plan_density(ctx, W, nb));
  CU(ctx->sch_ebins.reserve(sizeof(double) * (size_t)nb), "alloc scheme bins");
  const size_t r_bytes = sizeof(double) * 4 * kSchemeTpb * (size_t)G;
  if (ctx->sch_R.bytes < r_bytes) {  // rows start at zero and the reduction leaves them at zero
    CU(ctx->sch_R.reserve(r_bytes), "alloc reduction rows");
    CU(cudaMemsetAsync(ctx->sch_R.p, 0, r_bytes, ctx->stream), "zero reduction rows");
  }
  if (!ctx->sch_ev[0])
    for (auto& e : ctx->sch_ev) CU(cudaEventCreate(&e), "event create");
  SchemeArgs A{};
  A.win = dw;
  A.ps = PinStreams{W->ps_off.as<int64_t>(), W->ps_ev.as<uint32_t>(), W->ps_slot.as<uint32_t>()};
  A.pat_int = ctx->pat_int.as<uint16_t>();
  A.pat_leak = ctx->pat_leak.as<uint16_t>();
  A.ebins = ctx->sch_ebins.as<double>();
  A.R = ctx->sch_R.as<double>();
  A.blk_gate = W->blk_gate.as<int32_t>();
  A.blk_first = W->blk_first.as<int64_t>();
  A.ncyc = W->ncyc.as<int32_t>();
  A.n_blocks = scheme >= kSchemeDensity ? W->n_blocks : 0;
  A.ncyc_fix = (int32_t)std::min<int64_t>(ctx->p_ncyc_fix, nb);
  CU(cudaEventRecord(ctx->sch_ev[0], ctx->stream), "event record");
  CU(cudaMemsetAsync(A.ebins, 0, sizeof(double) * (size_t)nb, ctx->stream), "zero scheme bins");
  CU(launch_scheme(scheme, ctx->L, ctx->N, A, W->n_events, (int32_t)nb, ctx->stream), "scheme kernels");
  CU(cudaEventRecord(ctx->sch_ev[1], ctx->stream), "event record");
  ctx->launches += 4;
  if (waveform_w && !(flags & GTP_DEVICE))
    CU(cudaMemcpyAsync(waveform_w, wave, sizeof(double) * (size_t)nb, cudaMemcpyDeviceToHost, ctx->stream),
       "copy waveform");
  RC(check_walk_error(ctx, 1, &window, "run_power_scheme"));
  float ms = 0.f;
  CU(cudaEventElapsedTime(&ms, ctx->sch_ev[0], ctx->sch_ev[1]), "event time");
  if (kernel_ms) *kernel_ms = ms;
  W->has_result = true;
  W->glitch_result = ctx->N.clock_ps > 0;
  W->last_bin_ps = bin_ps;
  return GTP_OK;
}

int gtp_run_power_batched(gtp_ctx* ctx, int32_t n_windows, const int32_t* windows, int32_t bin_ps,
                          double* const* waveforms, int flags) {
  if (!ctx) return GTP_EINVAL;
  if (n_windows <= 0 || n_windows > kMaxWindows || !windows || !waveforms)
    return fail(ctx, GTP_EINVAL, "run_power_batched: bad arguments");
  if ((flags & GTP_GRAPH) && !(flags & GTP_DEVICE))
    return fail(ctx, GTP_EINVAL, "run_power_batched: graph replay needs device waveforms");
  DeviceGuard dg(ctx->device);
  return run_forward(ctx, windows, n_windows, bin_ps, waveforms, flags, (flags & GTP_GRAPH) != 0);
}

int gtp_pack_events(int64_t n_events, const gtp_event* events, uint32_t* packed) {
  if (n_events < 0 || (n_events > 0 && (!events || !packed))) return GTP_EINVAL;
  const int64_t nb = (n_events + 31) / 32;
  uint32_t* word = packed + nb;
  for (int64_t b = 0; b < nb; ++b) {
    const int64_t i0 = 32 * b, i1 = std::min<int64_t>(i0 + 32, n_events);
    int32_t lo = events[i0].t_ps, hi = lo;
    for (int64_t i = i0; i < i1; ++i) {
      if (events[i].t_ps < 0 || (events[i].meta >> 5) != 0u) return GTP_ERANGE;
      lo = std::min(lo, events[i].t_ps);
      hi = std::max(hi, events[i].t_ps);
    }
    if ((int64_t)hi - lo >= (1ll << 27)) return GTP_ERANGE;
    packed[b] = (uint32_t)lo;
    for (int64_t i = i0; i < i1; ++i) word[i] = ((uint32_t)(events[i].t_ps - lo) << 5) | events[i].meta;
  }
  return GTP_OK;
}

int gtp_run_power_streamed(gtp_ctx* ctx, int32_t window, int64_t window_ps, int64_t n_events,
                           const int64_t* gate_offsets, const gtp_event* events, const uint8_t* init_state,
                           int32_t bin_ps, double* waveform_w, int32_t n_chunks, int flags) {
  if (!ctx) return GTP_EINVAL;
  if (!ctx->net_loaded) return fail(ctx, GTP_EINVAL, "run_power_streamed: load the netlist first");
  if (window < 0 || window >= kMaxWindows) return fail(ctx, GTP_EINVAL, "run_power_streamed: window slot 0..1023");
  if (window_ps <= 0 || window_ps >= (1ll << 31))
    return fail(ctx, GTP_ERANGE, "run_power_streamed: window_ps must be in (0, 2^31)");
  if (bin_ps <= 0 || window_ps % bin_ps != 0)
    return fail(ctx, GTP_ERANGE, "run_power_streamed: window_ps must be a multiple of bin_ps > 0");
  if (n_events < 0 || !gate_offsets || !init_state || (n_events > 0 && !events))
    return fail(ctx, GTP_EINVAL, "run_power_streamed: null array or negative n_events");
  if (n_chunks < 1 || n_chunks > kMaxWindows) return fail(ctx, GTP_EINVAL, "run_power_streamed: n_chunks 1..1024");
  const int64_t G = ctx->N.n_gates;
  // The offsets decide which host bytes are copied and which records the
  // kernels read: each chunk's offsets are checked (in [0, n_events], not
  // decreasing) on the host before its copy is enqueued, while earlier chunks
  // are copied and walked.
  if (gate_offsets[0] != 0 || gate_offsets[G] != n_events)
    return fail(ctx, GTP_EINVAL, "run_power_streamed: offsets must start at 0 and end at n_events");
  DeviceGuard dg(ctx->device);
  const cudaStream_t st = ctx->stream;
  if (!ctx->copy_stream) {
    CU(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking), "copy stream");
    for (int i = 0; i < 2; ++i) {
      CU(cudaEventCreateWithFlags(&ctx->ev_copied[i], cudaEventDisableTiming), "event");
      CU(cudaEventCreateWithFlags(&ctx->ev_walked[i], cudaEventDisableTiming), "event");
    }
  }
  // chunks: gate ranges by record count, the first at half and the last at a
  // quarter of the others (with three or more chunks): only the first chunk's
  // host checks and copy, and the last chunk's walk, stay outside the overlap
  std::vector<double> cum(n_chunks + 1, 0.0);
  for (int c = 0; c < n_chunks; ++c)
    cum[c + 1] = cum[c] + (n_chunks < 3 ? 1.0 : c == 0 ? 0.5 : c == n_chunks - 1 ? 0.25 : 1.0);
  std::vector<int64_t> gb(n_chunks + 1);
  gb[0] = 0;
  gb[n_chunks] = G;
  for (int c = 1; c < n_chunks; ++c) {
    const int64_t target = (int64_t)((double)n_events * (cum[c] / cum[n_chunks]));
    gb[c] = std::lower_bound(gate_offsets, gate_offsets + G + 1, target) - gate_offsets;
    if (gb[c] < gb[c - 1]) gb[c] = gb[c - 1];
    if (gb[c] > G) gb[c] = G;
  }
  auto clamped = [&](int64_t g) { return std::min(std::max(gate_offsets[g], (int64_t)0), n_events); };
  int64_t max_chunk = 0;
  for (int c = 0; c < n_chunks; ++c) max_chunk = std::max(max_chunk, clamped(gb[c + 1]) - clamped(gb[c]));
  for (int i = 0; i < 2; ++i)
    CU(ctx->chunk_buf[i].reserve(sizeof(uint2) * (size_t)(max_chunk + 2)), "alloc chunk buffer");
  const bool packed = (flags & GTP_PACKED) != 0;
  const int64_t pk_words = (max_chunk + 3) & ~(int64_t)3;  // the anchors start 16-byte aligned
  if (packed)
    for (int i = 0; i < 2; ++i)
      CU(ctx->pk_buf[i].reserve(sizeof(uint32_t) * (size_t)(pk_words + max_chunk / 32 + 2)), "alloc packed buffer");
  // the window: offsets and initial states on the device, records only chunk by chunk
  CU(cudaStreamSynchronize(st), "run_power_streamed");
  if (ctx->timing == 1 && ctx->ev_sx[0]) cudaEventRecord(ctx->ev_sx[0], st);
  Window& W = ctx->windows[window];
  W.loaded = false;
  W.has_result = false;
  W.streamed = false;
  W.borrowed = nullptr;
  W.ps_ok = false;
  W.dplan_key[0] = -1;
  CU(W.offsets.reserve(sizeof(int64_t) * (G + 1)), "alloc offsets");
  CU(W.init.reserve((size_t)G), "alloc init");
  CU(cudaMemcpyAsync(W.offsets.p, gate_offsets, sizeof(int64_t) * (G + 1), cudaMemcpyHostToDevice, st), "copy offsets");
  CU(cudaMemcpyAsync(W.init.p, init_state, (size_t)G, cudaMemcpyHostToDevice, st), "copy init");
  W.window_ps = window_ps;
  W.n_events = n_events;
  W.loaded = true;
  W.streamed = true;  // its records never become resident: other runs need them loaded again
  double* wave = nullptr;
  if (waveform_w) {
    if (flags & GTP_DEVICE) {
      wave = waveform_w;
    } else {
      CU(W.wave.reserve(sizeof(double) * (size_t)(window_ps / bin_ps)), "alloc waveform");
      wave = W.wave.as<double>();
    }
  }
  RC(ensure_gate_tables(ctx, false));
  int64_t n_seg_total = 0, n_tiles_total = 0;
  std::vector<Window*> ws{&W};
  RC(build_plan(ctx, ws, bin_ps, std::vector<double*>{wave}, false, &n_seg_total, &n_tiles_total));
  // each chunk is walked by its own launch: the split between warps and threads follows the chunk's size
  if (ctx->p_dense_min <= 0)
    ctx->run_dense_min = dense_min_auto(max_chunk / std::max(ctx->n_sm, 1), false, ctx->N.clock_ps > 0);
  // one descriptor per chunk: the window's, with the chunk's gates and a record base that puts the
  // chunk buffer at the chunk's first record index (only that chunk's records are ever read)
  WinDesc* hw = plan_wins(ctx->h_plan);
  for (int c = 0; c < n_chunks; ++c) {
    hw[c] = hw[0];
    hw[c].g0 = gb[c];
    hw[c].g1 = gb[c + 1];
    hw[c].keep_bins = c > 0;
    hw[c].rec = ctx->chunk_buf[c & 1].as<uint2>() - gate_offsets[gb[c]];
  }
  RC(upload_plan(ctx, n_chunks, st));
  CU(cudaMemsetAsync(plan_l0(ctx->plan.p), 0, sizeof(double), st), "zero l0");
  CU(cudaMemsetAsync(ctx->d_err.p, 0, sizeof(DevError), st), "zero status");
  CU(ctx->first_bad.reserve(sizeof(unsigned long long)), "alloc trace check");
  CU(cudaMemsetAsync(ctx->first_bad.p, 0xFF, sizeof(unsigned long long), st), "clear trace check");
  // the copy stream starts after the uploads above
  CU(cudaEventRecord(ctx->ev_walked[0], st), "event");
  CU(cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_walked[0], 0), "wait");
  const bool sx = ctx->timing == 1 && ctx->ev_sx[0];
  const uint2* host_rec = reinterpret_cast<const uint2*>(events);
  const uint32_t* host_anchor = reinterpret_cast<const uint32_t*>(events);
  const uint32_t* host_word = host_anchor + (n_events + 31) / 32;
  for (int c = 0; c < n_chunks; ++c) {
    const int b = c & 1;
    bool ok = gate_offsets[gb[c]] >= 0 && gate_offsets[gb[c + 1]] <= n_events;
    int bad = 0;  // branch-free, so that the compiler vectorises the scan
    for (int64_t g = gb[c]; g < gb[c + 1]; ++g) bad |= gate_offsets[g + 1] < gate_offsets[g];
    ok = ok && !bad;
    if (!ok) {
      cudaStreamSynchronize(ctx->copy_stream);
      cudaStreamSynchronize(st);
      return fail(ctx, GTP_EINVAL, "run_power_streamed: offsets must not decrease and must stay in [0, n_events]");
    }
    const int64_t r0 = gate_offsets[gb[c]], nr = gate_offsets[gb[c + 1]] - r0;
    if (c >= 2) CU(cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_walked[b], 0), "wait walk");
    if (sx && c == 0) cudaEventRecord(ctx->ev_sx[1], ctx->copy_stream);
    uint32_t* pk_word = ctx->pk_buf[b].as<uint32_t>();
    uint32_t* pk_anchor = pk_word + pk_words;
    if (nr > 0 && !packed)
      CU(cudaMemcpyAsync(ctx->chunk_buf[b].p, host_rec + r0, sizeof(uint2) * (size_t)nr, cudaMemcpyHostToDevice,
                         ctx->copy_stream), "copy chunk");
    if (nr > 0 && packed) {
      const int64_t a0 = r0 >> 5, a1 = (r0 + nr - 1) >> 5;
      CU(cudaMemcpyAsync(pk_word, host_word + r0, sizeof(uint32_t) * (size_t)nr, cudaMemcpyHostToDevice,
                         ctx->copy_stream), "copy chunk");
      CU(cudaMemcpyAsync(pk_anchor, host_anchor + a0, sizeof(uint32_t) * (size_t)(a1 - a0 + 1),
                         cudaMemcpyHostToDevice, ctx->copy_stream), "copy chunk anchors");
    }
    if (sx && c == n_chunks - 1) cudaEventRecord(ctx->ev_sx[2], ctx->copy_stream);
    CU(cudaEventRecord(ctx->ev_copied[b], ctx->copy_stream), "event");
    CU(cudaStreamWaitEvent(st, ctx->ev_copied[b], 0), "wait copy");
    if (nr > 0 && packed) {
      CU(launch_unpack(pk_anchor, pk_word, r0, nr, ctx->chunk_buf[b].as<uint2>(), st), "unpack");
      ctx->launches += 1;
    }
    WalkArgs A = walk_args(ctx, 1);
    A.wins = plan_wins(ctx->plan.p) + c;
    A.n_gates = std::max<int64_t>(gb[c + 1] - gb[c], 1);
    if (ctx->p_kernel == 1) {
      CU(launch_prepare(ctx->L, ctx->N, A, false, st), "prepare");
      if (nr > 0) CU(launch_walk_per_gate(ctx->L, ctx->N, A.wins, 1, ctx->d_err.as<DevError>(), st), "walk");
    } else {
      CU(launch_prepare(ctx->L, ctx->N, A, true, st), "prepare");
      CU(launch_plan_scatter(ctx->L, ctx->N, A, st), "plan");
      CU(launch_walk(ctx->L, ctx->N, A, false, st), "walk");
    }
    // locate a bad record while this chunk is still on the device (a no-op unless one was flagged)
    CU(launch_validate_if(ctx->L, ctx->N, A.wins, ctx->d_err.as<DevError>(), A.n_gates,
                          ctx->first_bad.as<unsigned long long>(), st), "trace check");
    CU(cudaEventRecord(ctx->ev_walked[b], st), "event");
    ctx->launches += ctx->p_kernel == 1 ? 3 : 4;
  }
  CU(launch_merge(plan_wins(ctx->plan.p), plan_tile_base(ctx->plan.p), 1, n_tiles_total, st), "merge");
  ctx->launches += 3;
  if (waveform_w && !(flags & GTP_DEVICE))
    CU(cudaMemcpyAsync(waveform_w, wave, sizeof(double) * (size_t)(window_ps / bin_ps), cudaMemcpyDeviceToHost, st),
       "copy waveform");
  CU(cudaMemcpyAsync(ctx->h_err, ctx->d_err.p, sizeof(DevError), cudaMemcpyDeviceToHost, st), "read status");
  unsigned long long key = ~0ull;
  CU(cudaMemcpyAsync(&key, ctx->first_bad.p, sizeof key, cudaMemcpyDeviceToHost, st), "read trace check");
  if (sx) cudaEventRecord(ctx->ev_sx[3], st);
  CU(cudaStreamSynchronize(st), "run_power_streamed");
  if (sx) {
    for (int k = 0; k < 3; ++k) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, ctx->ev_sx[k], ctx->ev_sx[k + 1]) == cudaSuccess) ctx->t_sx[k] += (int64_t)(ms * 1e6);
    }
    ctx->n_timed += 1;
  }
  int rc = GTP_OK;
  if (ctx->h_err->code != 0) {
    if (key != ~0ull) {
      const int code = -(int)(key & 7ull);
      const long long rec = (long long)((key >> 3) & ((1ull << 40) - 1ull));
      char buf[200];
      snprintf(buf, sizeof buf, "run_power_streamed: %s at record %lld", code_name(code), rec);
      rc = fail(ctx, code, buf);
    } else {
      rc = check_device_error(ctx, "run_power_streamed");
    }
  }
  W.has_result = rc == GTP_OK;
  W.glitch_result = ctx->N.clock_ps > 0;
  W.last_bin_ps = bin_ps;
  return rc;
}

int gtp_gate_energy(gtp_ctx* ctx, int32_t window, double* e_leak, double* e_int, double* e_sw, int64_t* n_events,
                    uint8_t* final_state, int flags) {
  if (!ctx) return GTP_EINVAL;
  Window* W = get_window(ctx, window);
  if (!W || !W->has_result) return fail(ctx, GTP_EINVAL, "gate_energy: no result for this window");
  DeviceGuard dg(ctx->device);
  const int64_t G = ctx->N.n_gates;
  if (flags & GTP_DEVICE) {  // device outputs: one pass, stream-ordered on the context's stream
    if (e_leak || e_int || e_sw || n_events || final_state) {
      k_gate_out<<<1024, 256, 0, ctx->stream>>>(W->e_leak.as<double>(), W->e_int.as<double>(), W->e_sw.as<double>(),
                                                W->final_state.as<uint8_t>(), W->offsets.as<int64_t>(), G, e_leak,
                                                e_int, e_sw, n_events, final_state);
      CU(cudaGetLastError(), "gate outputs");
      ctx->launches += 1;
    }
    return GTP_OK;
  }
  const cudaMemcpyKind k = kind_out(flags);
  if (e_leak) CU(cudaMemcpyAsync(e_leak, W->e_leak.p, sizeof(double) * G, k, ctx->stream), "copy e_leak");
  if (e_int) CU(cudaMemcpyAsync(e_int, W->e_int.p, sizeof(double) * G, k, ctx->stream), "copy e_int");
  if (e_sw) CU(cudaMemcpyAsync(e_sw, W->e_sw.p, sizeof(double) * G, k, ctx->stream), "copy e_sw");
  if (final_state) CU(cudaMemcpyAsync(final_state, W->final_state.p, (size_t)G, k, ctx->stream), "copy final_state");
  if (n_events) {  // counts from the offsets on the device, then one copy into the caller's array
    CU(ctx->counts.reserve(sizeof(int64_t) * (size_t)std::max<int64_t>(G, 1)), "alloc counts");
    k_gate_out<<<1024, 256, 0, ctx->stream>>>(nullptr, nullptr, nullptr, nullptr, W->offsets.as<int64_t>(), G,
                                              nullptr, nullptr, nullptr, ctx->counts.as<int64_t>(), nullptr);
    CU(cudaGetLastError(), "counts");
    ctx->launches += 1;
    CU(cudaMemcpyAsync(n_events, ctx->counts.p, sizeof(int64_t) * G, k, ctx->stream), "copy counts");
  }
  // host outputs are complete on return
  CU(cudaStreamSynchronize(ctx->stream), "gate_energy");
  return GTP_OK;
}

int gtp_run_power_backward(gtp_ctx* ctx, int32_t window, int32_t bin_ps, const float* dL_dP, float* dC,
                           float* d_escale, float* d_lscale) {
  if (!ctx) return GTP_EINVAL;
  Window* W = get_window(ctx, window);
  if (!W || W->streamed) return fail(ctx, GTP_EINVAL, "run_power_backward: window not loaded");
  // the window's pattern gates are walked too: their dL/dC is read with gtp_pattern_gate_gradient
  ctx->run_pat_items = (W->pat_loaded && ctx->pat_net_ok) ? W->pat_n_items : -1;
  W->pat_grad = false;
  if (!dL_dP) return fail(ctx, GTP_EINVAL, "run_power_backward: dL_dP is required");
  if (bin_ps <= 0 || W->window_ps % bin_ps != 0)
    return fail(ctx, GTP_ERANGE, "window_ps must be a multiple of bin_ps > 0");
  DeviceGuard dg(ctx->device);
  const int64_t nb = W->window_ps / bin_ps;
  const int nt = merge_tiles((int)nb);
  const int64_t G = ctx->N.n_gates;
  if (ctx->run_pat_items >= 0) {
    RC(ensure_pattern_index(ctx));
    CU(ctx->pat_bad.reserve(sizeof(unsigned long long)), "alloc pattern status");
  }
  CU(ctx->grad.reserve(sizeof(float2) * nb), "alloc grad");
  CU(ctx->gtiles.reserve(sizeof(double) * nt), "alloc grad tiles");
  float* dc = dC;
  if (!dc) {
    CU(ctx->dC_scratch.reserve(sizeof(float) * G), "alloc dC");
    dc = ctx->dC_scratch.as<float>();
  }
  std::vector<Window*> ws{W};
  std::vector<double*> waves;
  int64_t n_seg_total = 0, n_tiles_total = 0;
  RC(ensure_gate_tables(ctx, true));
  RC(build_plan(ctx, ws, bin_ps, waves, true, &n_seg_total, &n_tiles_total));
  plan_wins(ctx->h_plan)[0].dC = dc;
  cudaStream_t st = ctx->stream;
  CU(cudaMemsetAsync(ctx->d_err.p, 0, sizeof(DevError), st), "zero status");
  RC(upload_plan(ctx, 1, st));
  CU(cudaMemsetAsync(dc, 0, sizeof(float) * G, st), "zero dC");
  CU(cudaMemsetAsync(ctx->cell_acc.p, 0, sizeof(double) * 2 * ctx->L.n_cells, st), "zero cell sums");
  // phases as in a forward run: gradient prefix and gate pass, plan, walk, cell outputs
  mark(ctx, 0, st);
  CU(launch_grad_prep(plan_wins(ctx->plan.p), dL_dP, ctx->grad.as<float2>(), ctx->gtiles.as<double>(), nt, (int)nb,
                      bin_ps, &plan_wins(ctx->plan.p)[0].g_total, st), "gradient prefix");
  CU(launch_gate_pass_bwd(ctx->L, ctx->N, plan_wins(ctx->plan.p), ctx->cell_acc.as<double>(), st), "gate pass");
  mark(ctx, 1, st);
  ctx->launches += 4;
  mark(ctx, 2, st);
  WalkArgs A = walk_args(ctx, 1);
  A.whole = ctx->run_whole;
  // small windows: the build with staged gate tables (see gtp_walk_adjoint_staged.cu)
  A.staged = ctx->p_bwd_staged != 0 &&
             (ctx->p_bwd_staged > 0 || W->n_events / std::max(ctx->n_sm, 1) < kBwdStagedBelow);
  if (W->n_events > 0) CU(launch_plan(ctx->N, ctx->L, A, st), "plan");
  mark(ctx, 3, st);
  mark(ctx, 4, st);
  mark(ctx, 8, st);
  mark(ctx, 9, st);
  if (W->n_events > 0) {
    CU(launch_walk(ctx->L, ctx->N, A, true, st), "adjoint walk");
    ctx->launches += 4;
  }
  if (ctx->run_pat_items >= 0) {  // the pattern gates' dL/dC (timed as walk)
    CU(cudaMemsetAsync(ctx->pat_bad.p, 0xFF, sizeof(unsigned long long), st), "reset pattern status");
    mark(ctx, 10, st);
    CU(launch_pattern_walk(ctx->P, ctx->Q, plan_wins(ctx->plan.p), 1, ctx->run_pat_items, ctx->N.clock_ps,
                           ctx->pat_bad.as<unsigned long long>(), st, true), "pattern adjoint walk");
    mark(ctx, 11, st);
    ctx->launches += ctx->run_pat_items > 0 ? 3 : 1;
  }
  mark(ctx, 5, st);
  mark(ctx, 6, st);
  if (d_escale || d_lscale) {
    CU(launch_cells_out(ctx->cell_acc.as<double>(), ctx->L.n_cells, d_escale, d_lscale, st), "cell gradients");
    ctx->launches += 1;
  }
  mark(ctx, 7, st);
  int rc = check_walk_error(ctx, W->n_events > 0 ? 1 : 0, &window, "run_power_backward");
  if (rc == GTP_OK && ctx->run_pat_items >= 0) rc = check_pattern_error(ctx, 1, &window, "run_power_backward");
  W->pat_grad = rc == GTP_OK && ctx->run_pat_items >= 0;
  collect_timing(ctx);
  return rc;
}

int gtp_autotune(gtp_ctx* ctx, int32_t n_windows, const int32_t* windows, int32_t bin_ps, int32_t iters,
                 double* best_ms) {
  if (!ctx) return GTP_EINVAL;
  if (n_windows <= 0 || n_windows > kMaxWindows || !windows) return fail(ctx, GTP_EINVAL, "autotune: bad arguments");
  DeviceGuard dg(ctx->device);
  if (iters <= 0) iters = 3;
  const int64_t keep_kernel = ctx->p_kernel;
  const int keep_timing = ctx->timing;
  ctx->p_kernel = 0;
  ctx->timing = 0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CU(cudaEventCreate(&e0), "event");
  CU(cudaEventCreate(&e1), "event");
  double best = 1e300;
  int64_t br = ctx->p_rpt, bc = ctx->p_dense_min;
  std::vector<double*> none(n_windows, nullptr);
  const int rpts[] = {4, 8, 16};
  const int dmins[] = {64, 256, 512, 1024};
  int rc = GTP_OK;
  ctx->p_ctas_per_sm = 0;
  for (int r : rpts) {
    {
      for (int c : dmins) {
        ctx->p_rpt = r;
        ctx->p_dense_min = c;
        rc = run_forward(ctx, windows, n_windows, bin_ps, none.data(), GTP_DEVICE, false);  // warm-up
        if (rc != GTP_OK) break;
        cudaEventRecord(e0, ctx->stream);
        for (int it = 0; it < iters && rc == GTP_OK; ++it)
          rc = run_forward(ctx, windows, n_windows, bin_ps, none.data(), GTP_DEVICE, false);
        cudaEventRecord(e1, ctx->stream);
        cudaEventSynchronize(e1);
        if (rc != GTP_OK) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms / iters < best) {
          best = ms / iters;
          br = r;
          bc = c;
        }
      }
      if (rc != GTP_OK) break;
    }
    if (rc != GTP_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->p_rpt = br;
  ctx->p_dense_min = bc;
  ctx->p_kernel = keep_kernel;
  ctx->timing = keep_timing;
  if (best_ms) *best_ms = best;
  return rc;
}

int gtp_measure_reductions(gtp_ctx* ctx, int32_t n_slots, int32_t width, int64_t n_red, double* per_s) {
  if (!ctx) return GTP_EINVAL;
  if (n_slots <= 0 || (width != 2 && width != 4) || n_red <= 0 || !per_s)
    return fail(ctx, GTP_EINVAL, "measure_reductions: n_slots > 0, width 2 or 4, n_red > 0 and an output");
  DeviceGuard dg(ctx->device);
  CU(ctx->probe.reserve(sizeof(float4) * (size_t)n_slots), "alloc probe");
  CU(cudaMemsetAsync(ctx->probe.p, 0, sizeof(float4) * (size_t)n_slots, ctx->stream), "zero probe");
  // both events are created before any early return and destroyed on every path below
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float4* slots = ctx->probe.as<float4>();
  if (e == cudaSuccess) e = launch_red_probe(slots, (uint32_t)n_slots, width, n_red, ctx->n_sm, ctx->stream);  // warm-up
  if (e == cudaSuccess) e = cudaEventRecord(e0, ctx->stream);
  if (e == cudaSuccess) e = launch_red_probe(slots, (uint32_t)n_slots, width, n_red, ctx->n_sm, ctx->stream);
  if (e == cudaSuccess) e = cudaEventRecord(e1, ctx->stream);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  CU(e, "measure_reductions");
  ctx->launches += 2;
  *per_s = ms > 0.f ? (double)n_red / (ms * 1e-3) : 0.0;
  return GTP_OK;
}

int gtp_measure_replay(gtp_ctx* ctx, int32_t window, int32_t bin_ps, double* ms) {
  if (!ctx) return GTP_EINVAL;
  Window* W = get_window(ctx, window);
  if (!W || W->streamed || !ms || bin_ps <= 0 || W->window_ps % bin_ps != 0)
    return fail(ctx, GTP_EINVAL, "measure_replay: a loaded window, bin_ps dividing its window_ps and an output");
  DeviceGuard dg(ctx->device);
  const int64_t nb = W->window_ps / bin_ps;
  CU(ctx->probe.reserve(sizeof(float4) * (size_t)nb), "alloc probe");
  CU(cudaMemsetAsync(ctx->probe.p, 0, sizeof(float4) * (size_t)nb, ctx->stream), "zero probe");
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float4* slots = ctx->probe.as<float4>();
  const uint2* rec = W->rec();
  if (e == cudaSuccess)  // warm-up
    e = launch_red_replay(rec, W->n_events, (int32_t)W->window_ps, bin_ps, slots, ctx->n_sm, ctx->stream);
  if (e == cudaSuccess) e = cudaEventRecord(e0, ctx->stream);
  if (e == cudaSuccess)
    e = launch_red_replay(rec, W->n_events, (int32_t)W->window_ps, bin_ps, slots, ctx->n_sm, ctx->stream);
  if (e == cudaSuccess) e = cudaEventRecord(e1, ctx->stream);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  CU(e, "measure_replay");
  ctx->launches += 2;
  *ms = (double)t;
  return GTP_OK;
}

int gtp_load_pattern_cells(gtp_ctx* ctx, int32_t n_cells, const int32_t* n_in, float vdd, int32_t n_slew,
                           const float* slew_axis, int32_t n_load, const float* load_axis, const int32_t* int_offsets,
                           const int32_t* int_pin, const int32_t* int_edge, const uint32_t* int_care,
                           const uint32_t* int_val, const float* int_tab, const float* int_default,
                           const int32_t* leak_offsets, const uint32_t* leak_care, const uint32_t* leak_val,
                           const float* leak_pw, const float* leak_default) {
  if (!ctx) return GTP_EINVAL;
  if (n_cells <= 0 || n_cells > (1 << 20) || !n_in || !slew_axis || !load_axis || !int_offsets || !int_default ||
      !leak_offsets || !leak_default)
    return fail(ctx, GTP_EINVAL, "load_pattern_cells: need 1 <= n_cells <= 2^20 and non-null arrays");
  if (n_slew < 2 || n_slew > GTP_MAX_AXIS || n_load < 2 || n_load > GTP_MAX_AXIS)
    return fail(ctx, GTP_ERANGE, "load_pattern_cells: axis lengths must be 2..16");
  for (int i = 0; i + 1 < n_slew; ++i)
    if (!(slew_axis[i] < slew_axis[i + 1])) return fail(ctx, GTP_EINVAL, "load_pattern_cells: slew axis not increasing");
  for (int i = 0; i + 1 < n_load; ++i)
    if (!(load_axis[i] < load_axis[i + 1])) return fail(ctx, GTP_EINVAL, "load_pattern_cells: load axis not increasing");
  if (int_offsets[0] != 0 || leak_offsets[0] != 0)
    return fail(ctx, GTP_EINVAL, "load_pattern_cells: offsets must start at 0");
  int64_t n_def = 0;
  for (int32_t c = 0; c < n_cells; ++c) {
    if (n_in[c] < 1 || n_in[c] > GTP_MAX_PATTERN_PINS - 1)
      return fail(ctx, GTP_ERANGE, "load_pattern_cells: n_in must be 1..31");
    if (int_offsets[c + 1] < int_offsets[c] || leak_offsets[c + 1] < leak_offsets[c])
      return fail(ctx, GTP_EINVAL, "load_pattern_cells: offsets must not decrease");
    n_def += 2ll * n_in[c];
  }
  const int64_t n_int = int_offsets[n_cells], n_lp = leak_offsets[n_cells];
  if (n_int > 0 && (!int_pin || !int_edge || !int_care || !int_val || !int_tab))
    return fail(ctx, GTP_EINVAL, "load_pattern_cells: null internal pattern arrays");
  if (n_lp > 0 && (!leak_care || !leak_val || !leak_pw))
    return fail(ctx, GTP_EINVAL, "load_pattern_cells: null leakage pattern arrays");
  if (n_int + n_def >= (1ll << 31)) return fail(ctx, GTP_ERANGE, "load_pattern_cells: too many tables");
  const size_t T = (size_t)n_slew * n_load;
  std::vector<uint4> ip;
  std::vector<int32_t> ipo;
  std::vector<uint4> lp((size_t)n_lp);
  std::vector<PatCell> cells((size_t)n_cells);
  int64_t d0 = n_int;
  for (int32_t c = 0; c < n_cells; ++c) {
    const uint32_t n = (uint32_t)n_in[c];
    const uint32_t inputs = (1u << n) - 1u;
    const uint32_t all = n >= 31 ? 0xFFFFFFFFu : (2u << n) - 1u;
    for (int32_t k = int_offsets[c]; k < int_offsets[c + 1]; ++k) {
      const int32_t p = int_pin[k];
      if (p < 0 || p >= (int32_t)n || int_edge[k] < -1 || int_edge[k] > 1)
        return fail(ctx, GTP_EINVAL, "load_pattern_cells: internal pattern " + std::to_string(k) + ": bad pin or edge");
      if ((int_care[k] & ~(inputs & ~(1u << p))) || (int_val[k] & ~int_care[k]))
        return fail(ctx, GTP_EINVAL, "load_pattern_cells: internal pattern " + std::to_string(k) +
                                         ": care must hold only other input pins, val only cared pins");
    }
    for (int32_t k = leak_offsets[c]; k < leak_offsets[c + 1]; ++k) {
      if ((leak_care[k] & ~all) || (leak_val[k] & ~leak_care[k]))
        return fail(ctx, GTP_EINVAL, "load_pattern_cells: leakage pattern " + std::to_string(k) +
                                         ": care must hold only the cell's pins, val only cared pins");
      uint32_t bits;
      memcpy(&bits, leak_pw + k, 4);
      lp[(size_t)k] = make_uint4(leak_care[k], leak_val[k], bits, 0u);
    }
    PatCell& pc = cells[(size_t)c];
    pc.n_in = (int32_t)n;
    pc.ipo = (int32_t)ipo.size();
    for (uint32_t p = 0; p < n; ++p) {  // each pin's patterns, in list order
      ipo.push_back((int32_t)ip.size());
      for (int32_t k = int_offsets[c]; k < int_offsets[c + 1]; ++k)
        if (int_pin[k] == (int32_t)p)
          ip.push_back(make_uint4(int_care[k], int_val[k], (uint32_t)int_edge[k], (uint32_t)k));
    }
    ipo.push_back((int32_t)ip.size());
    pc.lp0 = leak_offsets[c];
    pc.lp1 = leak_offsets[c + 1];
    pc.dtab = (int32_t)d0;
    d0 += 2ll * n;
    pc.leak_def = leak_default[c];
    pc.iidx = pc.lidx = -1;
  }
  DeviceGuard dg(ctx->device);
  CU(cudaStreamSynchronize(ctx->stream), "load_pattern_cells");
  drop_graphs(ctx);
  for (auto& kv : ctx->windows) kv.second.release_patterns();
  ctx->pat_cells_ok = ctx->pat_net_ok = ctx->pat_index_ok = false;
  CU(ctx->pc_cells.reserve(sizeof(PatCell) * cells.size()), "alloc pattern cells");
  CU(ctx->pc_ip.reserve(sizeof(uint4) * std::max<size_t>(ip.size(), 1)), "alloc patterns");
  CU(ctx->pc_ipo.reserve(sizeof(int32_t) * ipo.size()), "alloc patterns");
  CU(ctx->pc_lp.reserve(sizeof(uint4) * std::max<size_t>(lp.size(), 1)), "alloc patterns");
  CU(ctx->pc_tab.reserve(sizeof(float) * T * (size_t)(n_int + n_def)), "alloc pattern tables");
  CU(cudaMemcpy(ctx->pc_cells.p, cells.data(), sizeof(PatCell) * cells.size(), cudaMemcpyHostToDevice), "copy cells");
  if (!ip.empty()) CU(cudaMemcpy(ctx->pc_ip.p, ip.data(), sizeof(uint4) * ip.size(), cudaMemcpyHostToDevice), "copy");
  CU(cudaMemcpy(ctx->pc_ipo.p, ipo.data(), sizeof(int32_t) * ipo.size(), cudaMemcpyHostToDevice), "copy patterns");
  if (!lp.empty()) CU(cudaMemcpy(ctx->pc_lp.p, lp.data(), sizeof(uint4) * lp.size(), cudaMemcpyHostToDevice), "copy");
  if (n_int > 0)
    CU(cudaMemcpy(ctx->pc_tab.p, int_tab, sizeof(float) * T * (size_t)n_int, cudaMemcpyHostToDevice), "copy tables");
  CU(cudaMemcpy(ctx->pc_tab.as<float>() + T * (size_t)n_int, int_default, sizeof(float) * T * (size_t)n_def,
                cudaMemcpyHostToDevice), "copy default tables");
  ctx->h_pat_cells = cells;
  PatLib& P = ctx->P;
  P = PatLib{};
  P.cells = ctx->pc_cells.as<PatCell>();
  P.ip = ctx->pc_ip.as<uint4>();
  P.ipo = ctx->pc_ipo.as<int32_t>();
  P.lp = ctx->pc_lp.as<uint4>();
  P.tab = ctx->pc_tab.as<float>();
  P.n_cells = n_cells;
  P.ns = n_slew;
  P.nl = n_load;
  P.tsize = (int32_t)T;
  P.half_v2 = 0.5f * vdd * vdd;
  for (int i = 0; i < kMaxAxis; ++i) {
    P.slew_axis[i] = slew_axis[std::min(i, n_slew - 1)];
    P.load_axis[i] = load_axis[std::min(i, n_load - 1)];
  }
  ctx->pat_cells_ok = true;
  return GTP_OK;
}

int gtp_load_pattern_netlist(gtp_ctx* ctx, int64_t n_gates, const int32_t* cell, const float* load_ff,
                             const float* slew_ps, int32_t slew_stride, const float* out_slew_ps) {
  if (!ctx) return GTP_EINVAL;
  if (!ctx->pat_cells_ok) return fail(ctx, GTP_EINVAL, "load_pattern_netlist: load the pattern cells first");
  if (n_gates <= 0 || n_gates >= (1ll << 31) || !cell || !load_ff || !slew_ps)
    return fail(ctx, GTP_EINVAL, "load_pattern_netlist: need 1 <= n_gates < 2^31 and non-null arrays");
  int32_t widest = 0;
  for (int64_t g = 0; g < n_gates; ++g) {
    if (cell[g] < 0 || cell[g] >= ctx->P.n_cells)
      return fail(ctx, GTP_ERANGE, "load_pattern_netlist: cell index out of range at gate " + std::to_string(g));
    widest = std::max(widest, ctx->h_pat_cells[(size_t)cell[g]].n_in);
  }
  if (slew_stride < widest || slew_stride > GTP_MAX_PATTERN_PINS)
    return fail(ctx, GTP_EINVAL, "load_pattern_netlist: slew_stride must cover the widest cell (and be <= 32)");
  DeviceGuard dg(ctx->device);
  CU(cudaStreamSynchronize(ctx->stream), "load_pattern_netlist");
  drop_graphs(ctx);
  for (auto& kv : ctx->windows) kv.second.release_patterns();
  ctx->pat_net_ok = false;
  const size_t n = (size_t)n_gates;
  CU(ctx->pn_cell.reserve(sizeof(int32_t) * n), "alloc pattern netlist");
  CU(ctx->pn_load.reserve(sizeof(float) * n), "alloc pattern netlist");
  CU(ctx->pn_slew.reserve(sizeof(float) * 2 * (size_t)slew_stride * n), "alloc pattern netlist");
  CU(ctx->pn_oslew.reserve(sizeof(float) * 2 * n), "alloc pattern netlist");
  CU(cudaMemcpy(ctx->pn_cell.p, cell, sizeof(int32_t) * n, cudaMemcpyHostToDevice), "copy pattern netlist");
  CU(cudaMemcpy(ctx->pn_load.p, load_ff, sizeof(float) * n, cudaMemcpyHostToDevice), "copy pattern netlist");
  CU(cudaMemcpy(ctx->pn_slew.p, slew_ps, sizeof(float) * 2 * (size_t)slew_stride * n, cudaMemcpyHostToDevice),
     "copy pattern netlist");
  if (out_slew_ps)
    CU(cudaMemcpy(ctx->pn_oslew.p, out_slew_ps, sizeof(float) * 2 * n, cudaMemcpyHostToDevice), "copy out slews");
  else
    CU(cudaMemset(ctx->pn_oslew.p, 0, sizeof(float) * 2 * n), "zero out slews");
  // the interpolation point of every (gate, input pin, edge): lower knots (segments clamped to the edge ones,
  // so points outside the axes extrapolate) and the slew fraction; the load fraction is found per walk item
  {
    const PatLib& P = ctx->P;
    auto seg = [](const float* ax, int na, float x) {
      int i = 0;
      while (i < na - 2 && x >= ax[i + 1]) ++i;
      return i;
    };
    std::vector<uint2> desc(n * (size_t)slew_stride * 2, make_uint2(0u, 0u));
    for (int64_t g = 0; g < n_gates; ++g) {
      const int j = seg(P.load_axis, P.nl, load_ff[g]);
      const int n_in = ctx->h_pat_cells[(size_t)cell[g]].n_in;
      for (int p = 0; p < n_in; ++p)
        for (int e = 0; e < 2; ++e) {
          const float sl = slew_ps[((size_t)g * slew_stride + p) * 2 + e];
          const int i = seg(P.slew_axis, P.ns, sl);
          const float fs = (sl - P.slew_axis[i]) / (P.slew_axis[i + 1] - P.slew_axis[i]);
          uint32_t fb;
          memcpy(&fb, &fs, 4);
          desc[((size_t)g * slew_stride + p) * 2 + e] = make_uint2((uint32_t)(i * P.nl + j), fb);
        }
    }
    CU(ctx->pn_desc.reserve(sizeof(uint2) * desc.size()), "alloc pattern descriptors");
    CU(cudaMemcpy(ctx->pn_desc.p, desc.data(), sizeof(uint2) * desc.size(), cudaMemcpyHostToDevice),
       "copy pattern descriptors");
  }
  ctx->Q = PatNet{ctx->pn_cell.as<int32_t>(), ctx->pn_load.as<float>(), ctx->pn_slew.as<float>(),
                  ctx->pn_oslew.as<float>(), ctx->pn_desc.as<uint2>(), n_gates, slew_stride};
  ctx->pat_net_ok = true;
  return GTP_OK;
}

int gtp_load_pattern_events(gtp_ctx* ctx, int32_t window, int64_t n_events, const int64_t* gate_offsets,
                            const int32_t* t_ps, const uint8_t* pin, const uint8_t* value,
                            const uint32_t* init_state, int flags) {
  if (!ctx) return GTP_EINVAL;
  if (!ctx->pat_net_ok) return fail(ctx, GTP_EINVAL, "load_pattern_events: load the pattern netlist first");
  Window* W = get_window(ctx, window);
  if (!W || W->streamed) return fail(ctx, GTP_EINVAL, "load_pattern_events: load the window's events first");
  if (n_events < 0 || n_events >= (1ll << 40) || !gate_offsets || !init_state ||
      (n_events > 0 && (!t_ps || !pin || !value)))
    return fail(ctx, GTP_EINVAL, "load_pattern_events: need 0 <= n_events < 2^40 and non-null arrays");
  DeviceGuard dg(ctx->device);
  const int64_t G = ctx->Q.n_gates;
  const bool dev = (flags & GTP_DEVICE) != 0;
  CU(cudaStreamSynchronize(ctx->stream), "load_pattern_events");
  drop_graphs(ctx);
  W->release_patterns();
  W->has_result = false;
  std::vector<int64_t> off((size_t)G + 1);
  std::vector<uint32_t> init((size_t)G);
  CU(cudaMemcpy(off.data(), gate_offsets, sizeof(int64_t) * (G + 1), dev ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost),
     "read pattern offsets");
  CU(cudaMemcpy(init.data(), init_state, sizeof(uint32_t) * G, dev ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost),
     "read initial states");
  if (off[0] != 0 || off[(size_t)G] != n_events)
    return fail(ctx, GTP_EINVAL, "load_pattern_events: offsets must run from 0 to n_events");
  std::vector<int2> items;
  std::vector<int64_t> first((size_t)G + 1);
  std::vector<int32_t> cell((size_t)G);
  CU(cudaMemcpy(cell.data(), ctx->pn_cell.p, sizeof(int32_t) * G, cudaMemcpyDeviceToHost), "read pattern cells");
  for (int64_t g = 0; g < G; ++g) {
    if (off[(size_t)g + 1] < off[(size_t)g])
      return fail(ctx, GTP_EINVAL, "load_pattern_events: offsets decrease at gate " + std::to_string(g));
    const int n_in = ctx->h_pat_cells[(size_t)cell[(size_t)g]].n_in;
    if (n_in < 31 && (init[(size_t)g] >> (n_in + 1)))
      return fail(ctx, GTP_ERANGE, "load_pattern_events: initial state has bits past the pins at gate " +
                                       std::to_string(g));
    first[(size_t)g] = (int64_t)items.size();
    const int64_t n = off[(size_t)g + 1] - off[(size_t)g];
    for (int64_t k = 0; k * kPatPiece < n; ++k) items.push_back(make_int2((int)g, (int)k));
  }
  first[(size_t)G] = (int64_t)items.size();
  const size_t ni = std::max<size_t>(items.size(), 1);
  CU(W->pat_off.reserve(sizeof(int64_t) * (G + 1)), "alloc pattern events");
  CU(W->pat_rec.reserve(sizeof(uint2) * (size_t)std::max<int64_t>(n_events, 1)), "alloc pattern events");
  CU(W->pat_init.reserve(sizeof(uint32_t) * G), "alloc pattern events");
  CU(W->pat_items.reserve(sizeof(int2) * ni), "alloc pattern items");
  CU(W->pat_first.reserve(sizeof(int64_t) * (G + 1)), "alloc pattern items");
  CU(W->pat_mask.reserve(sizeof(uint32_t) * ni), "alloc pattern items");
  for (DevBuf* b : {&W->pat_e_leak, &W->pat_e_int, &W->pat_e_sw, &W->pat_e_gl})
    CU(b->reserve(sizeof(double) * G), "alloc pattern results");
  CU(W->pat_final.reserve(sizeof(uint32_t) * G), "alloc pattern results");
  CU(cudaMemcpy(W->pat_off.p, off.data(), sizeof(int64_t) * (G + 1), cudaMemcpyHostToDevice), "copy offsets");
  CU(cudaMemcpy(W->pat_init.p, init.data(), sizeof(uint32_t) * G, cudaMemcpyHostToDevice), "copy initial states");
  if (!items.empty())
    CU(cudaMemcpy(W->pat_items.p, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice), "copy items");
  CU(cudaMemcpy(W->pat_first.p, first.data(), sizeof(int64_t) * (G + 1), cudaMemcpyHostToDevice), "copy items");
  if (n_events > 0) {
    if (dev) {
      CU(launch_pattern_pack(t_ps, pin, value, n_events, W->pat_rec.as<uint2>(), ctx->stream), "pack records");
      ctx->launches += 1;
      CU(cudaStreamSynchronize(ctx->stream), "pack records");
    } else {
      std::vector<uint2> rec((size_t)n_events);
      for (int64_t i = 0; i < n_events; ++i)
        rec[(size_t)i] = make_uint2((uint32_t)t_ps[i], (uint32_t)pin[i] | (value[i] > 1 ? 0x200u : (uint32_t)value[i] << 8));
      CU(cudaMemcpy(W->pat_rec.p, rec.data(), sizeof(uint2) * (size_t)n_events, cudaMemcpyHostToDevice), "copy records");
    }
  }
  W->pat_h_off = std::move(off);
  W->pat_n_events = n_events;
  W->pat_n_items = (int64_t)items.size();
  W->pat_loaded = true;
  return GTP_OK;
}

int gtp_pattern_gate_energy(gtp_ctx* ctx, int32_t window, double* e_leak, double* e_int, double* e_sw, double* e_gl,
                            int64_t* n_events, uint32_t* final_state, int flags) {
  if (!ctx) return GTP_EINVAL;
  Window* W = get_window(ctx, window);
  if (!W || !W->has_result || !W->pat_loaded || !ctx->pat_net_ok)
    return fail(ctx, GTP_EINVAL, "pattern_gate_energy: no pattern gate result for this window");
  DeviceGuard dg(ctx->device);
  const size_t G = (size_t)ctx->Q.n_gates;
  const cudaMemcpyKind k = kind_out(flags);
  if (e_leak) CU(cudaMemcpyAsync(e_leak, W->pat_e_leak.p, sizeof(double) * G, k, ctx->stream), "copy e_leak");
  if (e_int) CU(cudaMemcpyAsync(e_int, W->pat_e_int.p, sizeof(double) * G, k, ctx->stream), "copy e_int");
  if (e_sw) CU(cudaMemcpyAsync(e_sw, W->pat_e_sw.p, sizeof(double) * G, k, ctx->stream), "copy e_sw");
  if (e_gl) CU(cudaMemcpyAsync(e_gl, W->pat_e_gl.p, sizeof(double) * G, k, ctx->stream), "copy e_gl");
  if (final_state)
    CU(cudaMemcpyAsync(final_state, W->pat_final.p, sizeof(uint32_t) * G, k, ctx->stream), "copy final state");
  std::vector<int64_t> cnt;
  if (n_events) {
    cnt.resize(G);
    for (size_t g = 0; g < G; ++g) cnt[g] = W->pat_h_off[g + 1] - W->pat_h_off[g];
    CU(cudaMemcpyAsync(n_events, cnt.data(), sizeof(int64_t) * G,
                       (flags & GTP_DEVICE) ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost, ctx->stream),
       "copy counts");
  }
  CU(cudaStreamSynchronize(ctx->stream), "pattern_gate_energy");
  return GTP_OK;
}

int gtp_pattern_gate_gradient(gtp_ctx* ctx, int32_t window, float* dC, int flags) {
  if (!ctx) return GTP_EINVAL;
  Window* W = get_window(ctx, window);
  if (!W || !W->pat_grad || !W->pat_loaded || !ctx->pat_net_ok || !dC)
    return fail(ctx, GTP_EINVAL, "pattern_gate_gradient: no pattern gate gradient for this window");
  DeviceGuard dg(ctx->device);
  CU(cudaMemcpyAsync(dC, W->pat_dC.p, sizeof(float) * (size_t)ctx->Q.n_gates, kind_out(flags), ctx->stream),
     "copy pattern gradients");
  CU(cudaStreamSynchronize(ctx->stream), "pattern_gate_gradient");
  return GTP_OK;
}

int gtp_set_param(gtp_ctx* ctx, const char* key, int64_t value) {
  if (!ctx || !key) return GTP_EINVAL;
  const std::string k(key);
  if (k == "kernel") {
    if (value > 1) return fail(ctx, GTP_ERANGE, "kernel must be 0 or 1");
    ctx->p_kernel = value < 0 ? 0 : value;
  } else if (k == "records_per_thread") {
    if (value >= 0 && !walk_rpt_supported((int)value))
      return fail(ctx, GTP_ERANGE, "records_per_thread must be 4, 8 or 16");
    ctx->p_rpt = value < 0 ? 8 : value;
  } else if (k == "ctas_per_sm") {
    if (value > 32) return fail(ctx, GTP_ERANGE, "ctas_per_sm must be <= 32");
    ctx->p_ctas_per_sm = value < 0 ? 0 : value;
  } else if (k == "bwd_staged") {
    if (value > 1) return fail(ctx, GTP_ERANGE, "bwd_staged must be -1, 0 or 1");
    ctx->p_bwd_staged = value < 0 ? -1 : value;
  } else if (k == "dense_min") {
    if (value == 0 || value > 4096) return fail(ctx, GTP_ERANGE, "dense_min must be 1..4096");
    ctx->p_dense_min = value < 0 ? -1 : value;
  } else if (k == "piece_len") {
    ctx->p_piece_len = value < 0 ? -1 : value;
  } else if (k == "sipl_max_pins") {
    if (value > GTP_MAX_INDEXED_PINS) return fail(ctx, GTP_ERANGE, "sipl_max_pins must be <= 24");
    const int64_t v = value < 0 ? 16 : value;
    if (v != ctx->p_sipl_max_pins) ctx->pat_index_ok = false;
    ctx->p_sipl_max_pins = v;
  } else if (k == "group_bin_bytes") {
    ctx->p_group_bytes = value < 0 ? kGroupBinBytes : value;
  } else if (k == "tile_min") {
    if (value > (1ll << 31)) return fail(ctx, GTP_ERANGE, "tile_min must be 0..2^31");
    ctx->p_tile_min = value < 0 ? 0 : value;
  } else if (k == "scheme_evt_tgt") {
    if (value == 0 || value > (1 << 20)) return fail(ctx, GTP_ERANGE, "scheme_evt_tgt must be 1..2^20");
    ctx->p_evt_tgt = value < 0 ? 8 : value;
  } else if (k == "scheme_thr_floor") {
    if (value == 0 || value > (1 << 20)) return fail(ctx, GTP_ERANGE, "scheme_thr_floor must be 1..2^20");
    ctx->p_thr_floor = value < 0 ? 512 : value;
  } else if (k == "scheme_ncyc_fix") {
    if (value == 0 || value > (1 << 30)) return fail(ctx, GTP_ERANGE, "scheme_ncyc_fix must be 1..2^30");
    ctx->p_ncyc_fix = value < 0 ? 1 : value;
  } else if (k == "timing") {
    // 1: time the phases of every following run with CUDA events; 2: the walk only (two events a run, so
    // the timing barely adds to a step); any value resets the totals
    DeviceGuard dg(ctx->device);
    if (value > 0 && !ctx->ev[0]) {
      for (auto& e : ctx->ev) CU(cudaEventCreate(&e), "event create");
      for (auto& e : ctx->ev_sx) CU(cudaEventCreate(&e), "event create");
    }
    if (value > 2) return fail(ctx, GTP_ERANGE, "timing must be 0, 1 or 2");
    ctx->timing = value > 0 ? (int)value : 0;
    for (auto& t : ctx->t_ns) t = 0;
    for (auto& t : ctx->t_sx) t = 0;
    ctx->prep_marked = false;
    ctx->n_timed = 0;
    ctx->launches = 0;
  } else {
    return fail(ctx, GTP_EINVAL, "unknown parameter " + k);
  }
  return GTP_OK;
}

int64_t gtp_get_param(const gtp_ctx* ctx, const char* key) {
  if (!ctx || !key) return -1;
  const std::string k(key);
  if (k == "kernel") return ctx->p_kernel;
  if (k == "records_per_thread") return ctx->p_rpt;
  if (k == "ctas_per_sm") return ctx->p_ctas_per_sm;
  if (k == "bwd_staged") return ctx->p_bwd_staged;
  if (k == "dense_min") return ctx->p_dense_min > 0 ? ctx->p_dense_min : (ctx->run_dense_min > 0 ? ctx->run_dense_min : 256);
  if (k == "tile_min") return ctx->p_tile_min;
  if (k == "piece_len") return ctx->p_piece_len;
  if (k == "run_piece_len") return ctx->run_piece_len;
  if (k == "run_whole") return ctx->run_whole ? 1 : 0;
  if (k == "group_bin_bytes") return ctx->p_group_bytes;
  if (k == "sipl_max_pins") return ctx->p_sipl_max_pins;
  if (k == "pattern_indexed_cells") return ctx->pat_index_ok ? ctx->pat_indexed : -1;
  if (k == "pattern_index_bytes") return ctx->pat_index_ok ? ctx->pat_index_bytes : -1;
  if (k == "run_groups") return (int64_t)ctx->run_groups.size();
  if (k == "t_tiled_ns") return ctx->t_ns[4];
  if (k == "t_pattern_ns") return ctx->t_ns[5];
  if (k == "t_prep_ns") return ctx->t_ns[6];
  if (k == "t_stream_setup_ns") return ctx->t_sx[0];
  if (k == "t_stream_copy_ns") return ctx->t_sx[1];
  if (k == "t_stream_tail_ns") return ctx->t_sx[2];
  if (k == "scheme_evt_tgt") return ctx->p_evt_tgt;
  if (k == "scheme_thr_floor") return ctx->p_thr_floor;
  if (k == "scheme_ncyc_fix") return ctx->p_ncyc_fix;
  if (k == "n_sm") return ctx->n_sm;
  if (k == "timing") return ctx->timing;
  if (k == "t_gate_pass_ns") return ctx->t_ns[0];
  if (k == "t_plan_ns") return ctx->t_ns[1];
  if (k == "t_walk_ns") return ctx->t_ns[2];
  if (k == "t_merge_ns") return ctx->t_ns[3];
  if (k == "n_timed") return ctx->n_timed;
  if (k == "launches") return ctx->launches;
  return -1;
}

}  // extern "C"
