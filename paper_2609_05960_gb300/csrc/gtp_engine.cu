// Host engine behind the C ABI of include/gtpower.h: device buffers, input
// validation, plans and launches.  All device work goes to the context's
// stream; results are synchronised only where the ABI says so.
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "gtp_internal.cuh"
#include "gtp_segwalk.cuh"

using namespace gtp;

namespace {

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
  // per-gate results and scratch
  DevBuf e_leak, e_int, e_sw, final_state;
  DevBuf bins, tiles, l0, wave;
  DevBuf seeds, runs;
  bool has_result = false;
  int32_t last_bin_ps = 0;
  const uint2* rec() const { return borrowed ? borrowed : records.as<uint2>(); }
  void release() {
    for (DevBuf* b : {&offsets, &records, &init, &e_leak, &e_int, &e_sw, &final_state, &bins, &tiles, &l0,
                      &wave, &seeds, &runs})
      b->release();
    borrowed = nullptr;
    loaded = false;
    has_result = false;
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
  DevBuf cell, load, slew;
  NetView N{};
  std::map<int, Window> windows;
  DevBuf d_err;
  DevError* h_err = nullptr;
  // parameters
  int64_t p_kernel = 0;
  int64_t p_rpt = 8;
  int64_t p_block = 256;
  int64_t p_ctas_per_sm = 0;
  // phase timing (CUDA events on the context stream) and launch counting
  bool timing = false;
  cudaEvent_t ev[8] = {};
  int64_t t_ns[4] = {0, 0, 0, 0};  // gate pass, seeds, walk, merge
  int64_t n_timed = 0;
  int64_t launches = 0;
};

namespace {

int fail(gtp_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

int cuda_fail(gtp_ctx* c, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) return fail(c, GTP_ENOMEM, m);
  return fail(c, GTP_ECUDA, m);
}

#define CU(call, where)                           \
  do {                                            \
    cudaError_t e_ = (call);                      \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, where); \
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

void bin_magic(int32_t d, uint32_t* magic, uint32_t* shift) {
  uint32_t s = 0;
  while ((2ull << s) <= (uint64_t)d) ++s;  // s = floor(log2 d)
  unsigned __int128 m = (((unsigned __int128)1) << (32 + s)) / (uint64_t)d;
  if (m > 0xFFFFFFFFull) m = 0xFFFFFFFFull;
  *magic = (uint32_t)m;
  *shift = s;
}

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
    long long idx = (long long)ctx->h_err->index;
    if (idx >= 0)
      snprintf(buf, sizeof buf, "%s: %s at record %lld", what, code_name(ctx->h_err->code), idx);
    else
      snprintf(buf, sizeof buf, "%s: %s at gate %lld", what, code_name(ctx->h_err->code), -1 - idx);
    return fail(ctx, ctx->h_err->code, buf);
  }
  return GTP_OK;
}

Window* get_window(gtp_ctx* ctx, int32_t w) {
  auto it = ctx->windows.find(w);
  if (it == ctx->windows.end() || !it->second.loaded) return nullptr;
  return &it->second;
}

int prepare_outputs(gtp_ctx* ctx, Window& W, int32_t bin_ps, Outputs* O) {
  if (bin_ps <= 0 || W.window_ps % bin_ps != 0) return fail(ctx, GTP_ERANGE, "window_ps must be a multiple of bin_ps > 0");
  int64_t nb = W.window_ps / bin_ps;
  int64_t G = ctx->N.n_gates;
  CU(W.e_leak.reserve(sizeof(double) * G), "alloc e_leak");
  CU(W.e_int.reserve(sizeof(double) * G), "alloc e_int");
  CU(W.e_sw.reserve(sizeof(double) * G), "alloc e_sw");
  CU(W.final_state.reserve((size_t)G), "alloc final_state");
  CU(W.bins.reserve(sizeof(float2) * nb), "alloc bins");
  CU(W.tiles.reserve(sizeof(double) * (size_t)merge_tiles((int)nb)), "alloc tiles");
  CU(W.l0.reserve(sizeof(double)), "alloc l0");
  Outputs o{};
  o.e_leak = W.e_leak.as<double>();
  o.e_int = W.e_int.as<double>();
  o.e_sw = W.e_sw.as<double>();
  o.final_state = W.final_state.as<uint8_t>();
  o.bins = W.bins.as<float2>();
  o.l0 = W.l0.as<double>();
  o.err = ctx->d_err.as<DevError>();
  o.bin_ps = bin_ps;
  bin_magic(bin_ps, &o.bin_magic, &o.bin_shift);
  o.n_bins = (int32_t)nb;
  *O = o;
  return GTP_OK;
}

WindowView view_of(const gtp_ctx* ctx, const Window& W) {
  WindowView v{};
  v.offsets = W.offsets.as<int64_t>();
  v.rec = W.rec();
  v.init = W.init.as<uint8_t>();
  v.n_events = W.n_events;
  v.window_ps = (int32_t)W.window_ps;
  (void)ctx;
  return v;
}

void mark(gtp_ctx* ctx, int i) {
  if (ctx->timing) cudaEventRecord(ctx->ev[i], ctx->stream);
}

// Accumulate the phase times of the last enqueue_forward (stream synchronised).
void collect_timing(gtp_ctx* ctx) {
  if (!ctx->timing) return;
  for (int k = 0; k < 4; ++k) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ctx->ev[2 * k], ctx->ev[2 * k + 1]) == cudaSuccess)
      ctx->t_ns[k] += (int64_t)(ms * 1e6);
  }
  ctx->n_timed += 1;
}

// Enqueue one window's forward pass (no synchronisation).
int enqueue_forward(gtp_ctx* ctx, Window& W, const Outputs& O, double* wave_dev) {
  cudaStream_t st = ctx->stream;
  WindowView V = view_of(ctx, W);
  CU(cudaMemsetAsync(O.bins, 0, sizeof(float2) * (size_t)O.n_bins, st), "zero bins");
  CU(cudaMemsetAsync(O.l0, 0, sizeof(double), st), "zero l0");
  mark(ctx, 0);
  CU(launch_gate_pass(ctx->L, ctx->N, V, O, st), "gate pass");
  ctx->launches += 1;
  mark(ctx, 1);
  mark(ctx, 2);
  if (W.n_events > 0) {
    if (ctx->p_kernel == 1) {
      mark(ctx, 3);
      mark(ctx, 4);
      CU(launch_walk_per_gate(ctx->L, ctx->N, V, O, 128, st), "walk (per gate)");
      ctx->launches += 1;
    } else {
      SegPlan P = make_seg_plan((int)ctx->p_rpt, (int)ctx->p_block, (int)ctx->p_ctas_per_sm, ctx->n_sm, W.n_events);
      CU(W.seeds.reserve(sizeof(Seed) * (size_t)P.n_seg), "alloc seeds");
      CU(W.runs.reserve(sizeof(int64_t) * (size_t)(P.n_seg + 1)), "alloc runs");
      CU(launch_seeds(ctx->L, ctx->N, V, P, W.seeds.as<Seed>(), W.runs.as<int64_t>(), st), "seeds");
      mark(ctx, 3);
      mark(ctx, 4);
      CU(launch_walk(ctx->L, ctx->N, V, O, P, W.seeds.as<Seed>(), st), "walk (segmented)");
      ctx->launches += 3;
    }
  } else {
    mark(ctx, 3);
    mark(ctx, 4);
  }
  mark(ctx, 5);
  mark(ctx, 6);
  if (wave_dev) {
    CU(launch_merge(O, wave_dev, W.tiles.as<double>(), merge_tiles(O.n_bins), st), "merge");
    ctx->launches += 3;
  }
  mark(ctx, 7);
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
  if (ctx->d_err.reserve(sizeof(DevError)) != cudaSuccess ||
      cudaMallocHost(&ctx->h_err, sizeof(DevError)) != cudaSuccess) {
    ctx->d_err.release();
    delete ctx;
    return GTP_ENOMEM;
  }
  cudaMemset(ctx->d_err.p, 0, sizeof(DevError));
  *out = ctx;
  return GTP_OK;
}

void gtp_destroy(gtp_ctx* ctx) {
  if (!ctx) return;
  DeviceGuard dg(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  for (auto& kv : ctx->windows) kv.second.release();
  for (DevBuf* b : {&ctx->tab, &ctx->leak, &ctx->cells, &ctx->table_cell, &ctx->leak_cell, &ctx->escale,
                    &ctx->lscale, &ctx->cell, &ctx->load, &ctx->slew, &ctx->d_err})
    b->release();
  if (ctx->h_err) cudaFreeHost(ctx->h_err);
  for (auto& e : ctx->ev)
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
  int64_t tsize = (int64_t)n_slew * n_load;
  if (n_e_int != n_tables * tsize) return fail(ctx, GTP_EINVAL, "load_library: e_int size does not match the cells");
  if (n_p_leak != n_leak) return fail(ctx, GTP_EINVAL, "load_library: p_leak size does not match the cells");
  LibView L{};
  L.n_cells = n_cells;
  L.n_tables = (int32_t)n_tables;
  L.n_leak = (int32_t)n_leak;
  L.ns = n_slew;
  L.nl = n_load;
  L.tsize = (int32_t)tsize;
  if (smem_lib_bytes(L) > GTP_MAX_TABLE_BYTES)
    return fail(ctx, GTP_ERANGE, "load_library: tables exceed the shared-memory budget");
  DeviceGuard dg(ctx->device);
  std::vector<uint8_t> tcell(n_tables), lcell(n_leak);
  for (int c = 0; c < n_cells; ++c) {
    int64_t nt = (int64_t)n_in[c] * (2ll << (n_in[c] - 1));
    for (int64_t k = 0; k < nt; ++k) tcell[ci[c].tab_base + k] = (uint8_t)c;
    for (int64_t k = 0; k < (2ll << n_in[c]); ++k) lcell[ci[c].leak_base + k] = (uint8_t)c;
  }
  std::vector<float> ones(n_cells, 1.0f);
  CU(ctx->tab.reserve(sizeof(float) * n_e_int), "alloc tables");
  CU(ctx->leak.reserve(sizeof(float) * n_leak), "alloc leakage");
  CU(ctx->cells.reserve(sizeof(CellInfo) * n_cells), "alloc cells");
  CU(ctx->table_cell.reserve(n_tables), "alloc table_cell");
  CU(ctx->leak_cell.reserve(n_leak), "alloc leak_cell");
  CU(ctx->escale.reserve(sizeof(float) * n_cells), "alloc escale");
  CU(ctx->lscale.reserve(sizeof(float) * n_cells), "alloc lscale");
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
  return GTP_OK;
}

namespace {
__global__ void k_check_cells(const int32_t* cell, int64_t n, int32_t n_cells, DevError* err) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    if (cell[g] < 0 || cell[g] >= n_cells) report_error(err, GTP_ERANGE, -1 - g);
}

__global__ void k_check_offsets(const int64_t* off, int64_t n_gates, int64_t n_events, DevError* err) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n_gates;
       g += (int64_t)gridDim.x * blockDim.x) {
    if (off[g + 1] < off[g]) report_error(err, GTP_EINVAL, -1 - g);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && (off[0] != 0 || off[n_gates] != n_events))
    report_error(err, GTP_EINVAL, -1);
}
}  // namespace

int gtp_load_netlist(gtp_ctx* ctx, int64_t n_gates, const int32_t* cell, const float* load_ff,
                     const float* slew_ps, int32_t slew_stride, int flags) {
  if (!ctx) return GTP_EINVAL;
  if (!ctx->lib_loaded) return fail(ctx, GTP_EINVAL, "load_netlist: load the library first");
  if (n_gates <= 0 || n_gates >= (1ll << 31) || !cell || !load_ff || !slew_ps)
    return fail(ctx, GTP_EINVAL, "load_netlist: need 1 <= n_gates < 2^31 and non-null arrays");
  if (slew_stride < ctx->max_in) return fail(ctx, GTP_EINVAL, "load_netlist: slew_stride < max input pins");
  DeviceGuard dg(ctx->device);
  cudaMemcpyKind k = kind_in(flags);
  CU(ctx->cell.reserve(sizeof(int32_t) * n_gates), "alloc cell");
  CU(ctx->load.reserve(sizeof(float) * n_gates), "alloc load");
  CU(ctx->slew.reserve(sizeof(float) * 2 * slew_stride * n_gates), "alloc slew");
  CU(cudaMemcpyAsync(ctx->cell.p, cell, sizeof(int32_t) * n_gates, k, ctx->stream), "copy cell");
  CU(cudaMemcpyAsync(ctx->load.p, load_ff, sizeof(float) * n_gates, k, ctx->stream), "copy load");
  CU(cudaMemcpyAsync(ctx->slew.p, slew_ps, sizeof(float) * 2 * slew_stride * n_gates, k, ctx->stream), "copy slew");
  CU(cudaMemsetAsync(ctx->d_err.p, 0, sizeof(DevError), ctx->stream), "zero status");
  k_check_cells<<<1024, 256, 0, ctx->stream>>>(ctx->cell.as<int32_t>(), n_gates, ctx->L.n_cells, ctx->d_err.as<DevError>());
  CU(cudaGetLastError(), "check cells");
  int rc = check_device_error(ctx, "load_netlist");
  if (rc != GTP_OK) return fail(ctx, GTP_ERANGE, "load_netlist: cell index out of range");
  ctx->N.cell = ctx->cell.as<int32_t>();
  ctx->N.load = ctx->load.as<float>();
  ctx->N.slew = ctx->slew.as<float>();
  ctx->N.n_gates = n_gates;
  ctx->N.stride = slew_stride;
  ctx->net_loaded = true;
  for (auto& kv : ctx->windows) kv.second.release();
  ctx->windows.clear();
  return GTP_OK;
}

int gtp_set_load(gtp_ctx* ctx, const float* load_ff, int flags) {
  if (!ctx) return GTP_EINVAL;
  if (!ctx->net_loaded || !load_ff) return fail(ctx, GTP_EINVAL, "set_load: no netlist or null array");
  DeviceGuard dg(ctx->device);
  CU(cudaMemcpyAsync(ctx->load.p, load_ff, sizeof(float) * ctx->N.n_gates, kind_in(flags), ctx->stream), "copy load");
  CU(cudaStreamSynchronize(ctx->stream), "set_load");
  return GTP_OK;
}

int gtp_load_events(gtp_ctx* ctx, int32_t window, int64_t window_ps, int64_t n_events, const int64_t* gate_offsets,
                    const gtp_event* events, const uint8_t* init_state, int flags) {
  if (!ctx) return GTP_EINVAL;
  if (!ctx->net_loaded) return fail(ctx, GTP_EINVAL, "load_events: load the netlist first");
  if (window < 0 || window >= 1024) return fail(ctx, GTP_EINVAL, "load_events: window slot must be 0..1023");
  if (window_ps <= 0 || window_ps >= (1ll << 31)) return fail(ctx, GTP_ERANGE, "load_events: window_ps must be in (0, 2^31)");
  if (n_events < 0 || !gate_offsets || !init_state || (n_events > 0 && !events))
    return fail(ctx, GTP_EINVAL, "load_events: null array or negative n_events");
  bool borrow = (flags & GTP_BORROW) != 0;
  if (borrow && !(flags & GTP_DEVICE)) return fail(ctx, GTP_EINVAL, "load_events: GTP_BORROW needs GTP_DEVICE");
  if (borrow && (((uintptr_t)events) & 15)) return fail(ctx, GTP_EINVAL, "load_events: borrowed events must be 16-byte aligned");
  DeviceGuard dg(ctx->device);
  int64_t G = ctx->N.n_gates;
  Window& W = ctx->windows[window];
  // buffers are kept and grown as needed, so reloading a slot does not reallocate
  W.loaded = false;
  W.has_result = false;
  W.borrowed = nullptr;
  cudaMemcpyKind k = kind_in(flags);
  CU(W.offsets.reserve(sizeof(int64_t) * (G + 1)), "alloc offsets");
  CU(W.init.reserve((size_t)G), "alloc init");
  CU(cudaMemcpyAsync(W.offsets.p, gate_offsets, sizeof(int64_t) * (G + 1), k, ctx->stream), "copy offsets");
  CU(cudaMemcpyAsync(W.init.p, init_state, (size_t)G, k, ctx->stream), "copy init");
  if (borrow) {
    W.borrowed = reinterpret_cast<const uint2*>(events);
  } else {
    // pad to an even number of records so 16-byte vector loads stay in bounds
    size_t bytes = sizeof(uint2) * (size_t)(n_events + 2);
    CU(W.records.reserve(bytes), "alloc records");
    CU(cudaMemsetAsync(W.records.as<uint2>() + n_events, 0, 2 * sizeof(uint2), ctx->stream), "zero padding");
    if (n_events > 0)
      CU(cudaMemcpyAsync(W.records.p, events, sizeof(uint2) * (size_t)n_events, k, ctx->stream), "copy records");
  }
  CU(cudaMemsetAsync(ctx->d_err.p, 0, sizeof(DevError), ctx->stream), "zero status");
  k_check_offsets<<<1024, 256, 0, ctx->stream>>>(W.offsets.as<int64_t>(), G, n_events, ctx->d_err.as<DevError>());
  CU(cudaGetLastError(), "check offsets");
  ctx->launches += 1;
  int rc = check_device_error(ctx, "load_events");
  if (rc != GTP_OK) return fail(ctx, GTP_EINVAL, "load_events: offsets must start at 0, end at n_events and not decrease");
  W.window_ps = window_ps;
  W.n_events = n_events;
  W.loaded = true;
  return GTP_OK;
}

int gtp_run_power(gtp_ctx* ctx, int32_t window, int32_t bin_ps, double* waveform_w, int flags) {
  if (!ctx) return GTP_EINVAL;
  Window* W = get_window(ctx, window);
  if (!W) return fail(ctx, GTP_EINVAL, "run_power: window not loaded");
  DeviceGuard dg(ctx->device);
  Outputs O;
  int rc = prepare_outputs(ctx, *W, bin_ps, &O);
  if (rc) return rc;
  double* wave = nullptr;
  if (waveform_w) {
    if (flags & GTP_DEVICE) {
      wave = waveform_w;
    } else {
      CU(W->wave.reserve(sizeof(double) * (size_t)O.n_bins), "alloc waveform");
      wave = W->wave.as<double>();
    }
  }
  CU(cudaMemsetAsync(ctx->d_err.p, 0, sizeof(DevError), ctx->stream), "zero status");
  rc = enqueue_forward(ctx, *W, O, wave);
  if (rc) return rc;
  if (waveform_w && !(flags & GTP_DEVICE))
    CU(cudaMemcpyAsync(waveform_w, wave, sizeof(double) * (size_t)O.n_bins, cudaMemcpyDeviceToHost, ctx->stream),
       "copy waveform");
  rc = check_device_error(ctx, "run_power");
  collect_timing(ctx);
  W->has_result = (rc == GTP_OK);
  W->last_bin_ps = bin_ps;
  return rc;
}

namespace {
__global__ void k_counts(const int64_t* off, int64_t n, int64_t* out) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    out[g] = off[g + 1] - off[g];
}
}  // namespace

int gtp_gate_energy(gtp_ctx* ctx, int32_t window, double* e_leak, double* e_int, double* e_sw, int64_t* n_events,
                    uint8_t* final_state, int flags) {
  if (!ctx) return GTP_EINVAL;
  Window* W = get_window(ctx, window);
  if (!W || !W->has_result) return fail(ctx, GTP_EINVAL, "gate_energy: no result for this window");
  DeviceGuard dg(ctx->device);
  int64_t G = ctx->N.n_gates;
  cudaMemcpyKind k = kind_out(flags);
  if (e_leak) CU(cudaMemcpyAsync(e_leak, W->e_leak.p, sizeof(double) * G, k, ctx->stream), "copy e_leak");
  if (e_int) CU(cudaMemcpyAsync(e_int, W->e_int.p, sizeof(double) * G, k, ctx->stream), "copy e_int");
  if (e_sw) CU(cudaMemcpyAsync(e_sw, W->e_sw.p, sizeof(double) * G, k, ctx->stream), "copy e_sw");
  if (final_state) CU(cudaMemcpyAsync(final_state, W->final_state.p, (size_t)G, k, ctx->stream), "copy final_state");
  if (n_events) {
    if (flags & GTP_DEVICE) {
      k_counts<<<1024, 256, 0, ctx->stream>>>(W->offsets.as<int64_t>(), G, n_events);
      CU(cudaGetLastError(), "counts");
      ctx->launches += 1;
    } else {
      std::vector<int64_t> off(G + 1);
      CU(cudaMemcpyAsync(off.data(), W->offsets.p, sizeof(int64_t) * (G + 1), cudaMemcpyDeviceToHost, ctx->stream),
         "copy offsets");
      CU(cudaStreamSynchronize(ctx->stream), "gate_energy");
      for (int64_t g = 0; g < G; ++g) n_events[g] = off[g + 1] - off[g];
    }
  }
  CU(cudaStreamSynchronize(ctx->stream), "gate_energy");
  return GTP_OK;
}

int gtp_run_power_batched(gtp_ctx* ctx, int32_t n_windows, const int32_t* windows, int32_t bin_ps,
                          double* const* waveforms, int flags) {
  if (!ctx) return GTP_EINVAL;
  if (n_windows <= 0 || !windows || !waveforms) return fail(ctx, GTP_EINVAL, "run_power_batched: bad arguments");
  DeviceGuard dg(ctx->device);
  std::vector<Window*> ws(n_windows);
  std::vector<Outputs> os(n_windows);
  for (int i = 0; i < n_windows; ++i) {
    ws[i] = get_window(ctx, windows[i]);
    if (!ws[i]) return fail(ctx, GTP_EINVAL, "run_power_batched: window not loaded");
    int rc = prepare_outputs(ctx, *ws[i], bin_ps, &os[i]);
    if (rc) return rc;
  }
  CU(cudaMemsetAsync(ctx->d_err.p, 0, sizeof(DevError), ctx->stream), "zero status");
  for (int i = 0; i < n_windows; ++i) {
    double* wave = nullptr;
    if (waveforms[i]) {
      if (flags & GTP_DEVICE) {
        wave = waveforms[i];
      } else {
        CU(ws[i]->wave.reserve(sizeof(double) * (size_t)os[i].n_bins), "alloc waveform");
        wave = ws[i]->wave.as<double>();
      }
    }
    int rc = enqueue_forward(ctx, *ws[i], os[i], wave);
    if (rc) return rc;
    if (waveforms[i] && !(flags & GTP_DEVICE))
      CU(cudaMemcpyAsync(waveforms[i], wave, sizeof(double) * (size_t)os[i].n_bins, cudaMemcpyDeviceToHost,
                         ctx->stream), "copy waveform");
  }
  int rc = check_device_error(ctx, "run_power_batched");
  for (int i = 0; i < n_windows; ++i) {
    ws[i]->has_result = (rc == GTP_OK);
    ws[i]->last_bin_ps = bin_ps;
  }
  return rc;
}

int gtp_run_power_backward(gtp_ctx* ctx, int32_t window, int32_t bin_ps, const float* dL_dP, float* dC,
                           float* d_escale, float* d_lscale) {
  if (!ctx) return GTP_EINVAL;
  (void)window; (void)bin_ps; (void)dL_dP; (void)dC; (void)d_escale; (void)d_lscale;
  return fail(ctx, GTP_EINVAL, "run_power_backward: not available in this build");
}

int gtp_set_param(gtp_ctx* ctx, const char* key, int64_t value) {
  if (!ctx || !key) return GTP_EINVAL;
  std::string k(key);
  if (k == "kernel") {
    if (value > 1) return fail(ctx, GTP_ERANGE, "kernel must be 0 or 1");
    ctx->p_kernel = value < 0 ? 0 : value;
  } else if (k == "records_per_thread") {
    if (value >= 0 && !seg_rpt_supported((int)value)) return fail(ctx, GTP_ERANGE, "records_per_thread must be 4, 8 or 16");
    ctx->p_rpt = value < 0 ? 8 : value;
  } else if (k == "block_threads") {
    if (value >= 0 && value != 128 && value != 256)
      return fail(ctx, GTP_ERANGE, "block_threads must be 128 or 256");
    ctx->p_block = value < 0 ? 256 : value;
  } else if (k == "ctas_per_sm") {
    if (value > 32) return fail(ctx, GTP_ERANGE, "ctas_per_sm must be <= 32");
    ctx->p_ctas_per_sm = value < 0 ? 0 : value;
  } else if (k == "timing") {
    // 1: time the phases of every following run with CUDA events; any value resets the totals
    DeviceGuard dg(ctx->device);
    if (value > 0 && !ctx->ev[0])
      for (auto& e : ctx->ev) CU(cudaEventCreate(&e), "event create");
    ctx->timing = value > 0;
    for (auto& t : ctx->t_ns) t = 0;
    ctx->n_timed = 0;
    ctx->launches = 0;
  } else {
    return fail(ctx, GTP_EINVAL, "unknown parameter " + k);
  }
  return GTP_OK;
}

int64_t gtp_get_param(const gtp_ctx* ctx, const char* key) {
  if (!ctx || !key) return -1;
  std::string k(key);
  if (k == "kernel") return ctx->p_kernel;
  if (k == "records_per_thread") return ctx->p_rpt;
  if (k == "block_threads") return ctx->p_block;
  if (k == "ctas_per_sm") return ctx->p_ctas_per_sm;
  if (k == "n_sm") return ctx->n_sm;
  if (k == "timing") return ctx->timing ? 1 : 0;
  if (k == "t_gate_pass_ns") return ctx->t_ns[0];
  if (k == "t_seeds_ns") return ctx->t_ns[1];
  if (k == "t_walk_ns") return ctx->t_ns[2];
  if (k == "t_merge_ns") return ctx->t_ns[3];
  if (k == "n_timed") return ctx->n_timed;
  if (k == "launches") return ctx->launches;
  return -1;
}

}  // extern "C"
