// Gates whose cells are given by state patterns (up to 32 pins): the paper's
// fallback for cells too wide for state-indexed arrays (Sec. 4.1), and the
// state-indexed arrays themselves for pattern cells under the pin threshold.
//
// Lookups.  A cell under the threshold has its arrays built here on the
// device: every entry (pin, edge, side-input state) scans the pin's patterns
// and keeps the first that covers it, the same item the paper's don't-care
// enumeration puts there (Sec. 4.1); leakage likewise over all 2^pins states.
// A cell above the threshold scans its patterns at every lookup, the
// paper's traversal fallback.  Internal patterns are stored per pin (a pin's
// list keeps the original order), so a scan only visits the event pin's
// patterns.
//
// The walk.  A gate's records are cut into items of kPatPiece records, each
// extended to the end of its last timestamp group, so no group spans two
// items.  One warp walks one item, 32 records at a time: a warp XOR scan of
// the records' pin bits gives each record's state (every event toggles its
// pin, so the state after a record is the initial state XOR the pin bits of
// every earlier record); the state before a record's timestamp group is the
// state before the group's first record (Algorithm 1: lookups of a group use
// the state held before it, the state changes after the whole group).  An
// item starts from the initial state XOR the pin bits of the gate's earlier
// items (k_pat_masks).  Leakage: at the end of each group the gate's power
// changes to that of the state after the group, which holds until the next
// group or the window's end (Eq. 4); the per-gate sum takes each such
// interval, and the bins take the change in the merge's step form (Sec.
// 2.4.2): dP * ((b + 1) * bin_ps - t) into the group's bin b and dP into its
// step accumulator; the initial power goes into the window's L0.  Per-event
// arithmetic is FP32 (the FP64 pipe of this GPU is slow): one {energy, step}
// reduction per distinct bin of the 32 records into the window's bin
// accumulators (in a component run, each record's internal, switching,
// glitch and leakage-correction parts into the component accumulators, as
// the fused walk lays them out), per-gate sums in FP32 within an item and
// FP64 across items.
// Glitch detection (Sec. 2.4.1, Eq. 2) keeps each pin's last event time in
// shared memory; an item first looks back over the earlier records of its
// first clock cycle.
#include "gtp_internal.cuh"

namespace gtp {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kPatWarps = 4;

__device__ __forceinline__ uint64_t pat_key(int w, int64_t r, int code) {
  return (((uint64_t)w << 40 | (uint64_t)r) << 3) | (uint64_t)(-code);
}

// Table id of an event on input `pin` with new value `edge` at input state S.
__device__ __forceinline__ int32_t pat_table(const PatLib& P, const PatCell& c, uint32_t pin, uint32_t edge,
                                             uint32_t S) {
  S &= (1u << c.n_in) - 1u;  // n_in <= 31
  if (c.iidx >= 0) {
    const uint32_t side = (S & ((1u << pin) - 1u)) | ((S >> (pin + 1)) << pin);
    return __ldg(P.iidx + c.iidx + ((int64_t)(pin * 2 + edge) << (c.n_in - 1)) + side);
  }
  const int32_t a = __ldg(P.ipo + c.ipo + pin), b = __ldg(P.ipo + c.ipo + pin + 1);
  for (int32_t k = a; k < b; ++k) {
    const uint4 q = __ldg(P.ip + k);
    if ((q.z == 0xFFFFFFFFu || q.z == edge) && (S & q.x) == q.y) return (int32_t)q.w;
  }
  return c.dtab + 2 * (int32_t)pin + (int32_t)edge;
}

// Leakage power (nW) of full state S by traversal.
__device__ __forceinline__ float pat_leak_scan(const PatLib& P, const PatCell& c, uint32_t S) {
  for (int32_t k = c.lp0; k < c.lp1; ++k) {
    const uint4 q = __ldg(P.lp + k);
    if ((S & q.x) == q.y) return __uint_as_float(q.z);
  }
  return c.leak_def;
}

__device__ __forceinline__ float pat_leak(const PatLib& P, const PatCell& c, uint32_t S) {
  return c.lidx >= 0 ? __ldg(P.lidx + c.lidx + S) : pat_leak_scan(P, c, S);
}

// ------------------------------------------------------------------ state-indexed arrays
// Cell c's arrays: table ids into iidx_all + its iidx, leakage into
// lidx_all + its lidx (the PatLib's arrays, written here only).
__global__ void k_pat_index(PatLib P, int32_t c, int32_t* __restrict__ iidx_all, float* __restrict__ lidx_all) {
  const PatCell cell = P.cells[c];
  const int n_in = cell.n_in;
  const int64_t n_side = 1ll << (n_in - 1);
  const int64_t n_int = (int64_t)n_in * 2 * n_side;
  const int64_t n_leak = 2ll << n_in;
  int32_t* iidx = iidx_all + cell.iidx;
  float* lidx = lidx_all + cell.lidx;
  PatCell scan = cell;
  scan.iidx = -1;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_int + n_leak;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (e < n_int) {
      const uint32_t pin = (uint32_t)(e / (2 * n_side));
      const uint32_t edge = (uint32_t)((e / n_side) & 1);
      const uint32_t side = (uint32_t)(e % n_side);
      const uint32_t S = (side & ((1u << pin) - 1u)) | ((side >> pin) << (pin + 1));  // pin's own bit 0
      iidx[e] = pat_table(P, scan, pin, edge, S);
    } else {
      lidx[e - n_int] = pat_leak_scan(P, cell, (uint32_t)(e - n_int));
    }
  }
}

// ------------------------------------------------------------------ items
// First record at or after x that starts a timestamp group (x itself if
// x == a), or b.  Warp-cooperative; all lanes return the same value.
__device__ __forceinline__ int64_t group_start(const uint2* __restrict__ rec, int64_t a, int64_t b, int64_t x,
                                               int lane) {
  if (x <= a) return a;
  for (int64_t base = x; base < b; base += 32) {
    const int64_t r = base + lane;
    const bool hit = r >= b || __ldg(&rec[r].x) != __ldg(&rec[r - 1].x);
    const unsigned m = __ballot_sync(kFull, hit);
    if (m) return min(b, base + __ffs(m) - 1);
  }
  return b;
}

// Records [s, e) of item `piece` of the gate with records [a, b).
__device__ __forceinline__ void item_bounds(const uint2* __restrict__ rec, int64_t a, int64_t b, int32_t piece,
                                            int lane, int64_t* s, int64_t* e) {
  const int64_t s0 = a + (int64_t)piece * kPatPiece;
  const int64_t e0 = min(s0 + kPatPiece, b);
  *s = group_start(rec, a, b, s0, lane);
  *e = e0 >= b ? b : group_start(rec, a, b, e0, lane);
}

__device__ __forceinline__ uint32_t warp_xor(uint32_t v) {
  for (int o = 16; o > 0; o >>= 1) v ^= __shfl_xor_sync(kFull, v, o);
  return v;
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// Per window and pattern gate: outputs initialised (the initial state's
// leakage over the whole window; the walk adds each change of it), and the
// initial leakage powers added into the window's L0.  In the adjoint only
// dL/dC is initialised (leakage does not depend on the load).
template <bool BWD>
__global__ void __launch_bounds__(256) k_pat_prepare(PatLib P, PatNet Q, const WinDesc* __restrict__ wins) {
  __shared__ double red[8];
  const WinDesc& W = wins[blockIdx.y];
  if (BWD) {
    if (W.p_off)
      for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < Q.n_gates;
           g += (int64_t)gridDim.x * blockDim.x)
        W.p_dC[g] = 0.f;
    return;
  }
  double p0 = 0.0;
  if (W.p_n_items > 0 || W.p_off) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < Q.n_gates;
         g += (int64_t)gridDim.x * blockDim.x) {
      const PatCell c = P.cells[Q.cell[g]];
      const uint32_t s0 = W.p_init[g];
      const float Pl = pat_leak(P, c, s0);
      p0 += (double)Pl;
      // the initial state's leakage until the first group (the walk adds each later interval)
      const int64_t a = W.p_off[g];
      const uint32_t t1 = a < W.p_off[g + 1] ? min(W.p_rec[a].x, (uint32_t)W.window_ps) : (uint32_t)W.window_ps;
      W.p_e_leak[g] = (double)Pl * (double)t1 * 1e-6;
      W.p_e_int[g] = 0.0;
      W.p_e_sw[g] = 0.0;
      W.p_e_gl[g] = 0.0;
      W.p_final[g] = s0;
    }
  }
  p0 = warp_sum(p0);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = p0;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) v += red[k];
    if (v != 0.0) atomicAdd(W.l0, v);
  }
}

// Per item: the XOR of its records' pin bits.
__global__ void __launch_bounds__(kPatWarps * 32) k_pat_masks(const WinDesc* __restrict__ wins) {
  const WinDesc& W = wins[blockIdx.y];
  const int lane = threadIdx.x & 31;
  const int64_t it = (int64_t)blockIdx.x * kPatWarps + (threadIdx.x >> 5);
  if (it >= W.p_n_items) return;
  const int2 item = W.p_items[it];
  const int64_t a = W.p_off[item.x], b = W.p_off[item.x + 1];
  int64_t s, e;
  item_bounds(W.p_rec, a, b, item.y, lane, &s, &e);
  uint32_t m = 0u;
  for (int64_t r = s + lane; r < e; r += 32) {
    const uint32_t pin = __ldg(&W.p_rec[r].y) & 0xFFu;
    m ^= pin < 32u ? 1u << pin : 0u;
  }
  m = warp_xor(m);
  if (lane == 0) W.p_mask[it] = m;
}

// ------------------------------------------------------------------ the walk
// The adjoint (BWD) walks the same records with the same states, checks and
// glitch detection, and sums dL/dC = sum over events of g_b(event) * dE/dC:
// the slope in load of the event's bilinear interpolation (Sec. 2.2) or
// 0.5 * Vdd^2 for the output pin (Eq. 1), times a glitch event's ratio
// (Eq. 2); leakage does not depend on the load.
template <bool GL, bool BWD>
__global__ void __launch_bounds__(kPatWarps * 32) k_pat_walk(PatLib P, PatNet Q, const WinDesc* __restrict__ wins,
                                                             int32_t clk, unsigned long long* bad) {
  __shared__ float ax[2][kMaxAxis];
  __shared__ int32_t last_t[kPatWarps][32];  // glitch detection: each pin's last event time (-1: none in reach)
  if (threadIdx.x < kMaxAxis) {
    ax[0][threadIdx.x] = P.slew_axis[threadIdx.x];
    ax[1][threadIdx.x] = P.load_axis[threadIdx.x];
  }
  __syncthreads();
  const WinDesc& W = wins[blockIdx.y];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t it = (int64_t)blockIdx.x * kPatWarps + warp;
  if (it >= W.p_n_items) return;
  const int2 item = W.p_items[it];
  const int64_t g = item.x;
  const int64_t ga = W.p_off[g], gb = W.p_off[g + 1];
  int64_t s, e;
  item_bounds(W.p_rec, ga, gb, item.y, lane, &s, &e);
  if (s >= e) return;
  const PatCell c = P.cells[Q.cell[g]];
  const uint32_t n_in = (uint32_t)c.n_in;
  const uint32_t T = (uint32_t)W.window_ps, bin_ps = (uint32_t)W.bin_ps;
  const float C = Q.load[g];
  int j = 0;
  while (j < P.nl - 2 && C >= ax[1][j + 1]) ++j;
  const float lrw = 1.f / (ax[1][j + 1] - ax[1][j]);
  const float fl = (C - ax[1][j]) * lrw;
  const float esw = P.half_v2 * C;
  const float* slew = Q.slew + (int64_t)g * Q.stride * 2;
  // entry state: the initial state XOR the pin bits of the gate's earlier items (kept to the cell's pins:
  // a malformed earlier record, reported by its own item, may have set others)
  const uint32_t full = n_in >= 31u ? 0xFFFFFFFFu : (2u << n_in) - 1u;
  uint32_t S = 0u;
  for (int64_t k = W.p_first[g] + lane; k < it; k += 32) S ^= W.p_mask[k];
  S = (warp_xor(S) ^ W.p_init[g]) & full;
  uint32_t Sg = S;               // state before the timestamp group in progress
  float Pc = pat_leak(P, c, S);  // its leakage power
  uint32_t t_last = s > ga ? __ldg(&W.p_rec[s - 1].x) : 0u;
  if (GL) {
    // each pin's last event time before the item within the item's first clock cycle
    last_t[warp][lane] = -1;
    __syncwarp();
    const uint32_t c0 = __ldg(&W.p_rec[s].x) / (uint32_t)clk * (uint32_t)clk;
    for (int64_t base = s - 1; base >= ga; base -= 32) {
      const int64_t r = base - lane;
      const uint2 q = r >= ga ? W.p_rec[r] : make_uint2(0u, 0xFFu);
      const bool in = r >= ga && q.x >= c0 && q.x < T;
      const uint32_t pin = q.y & 0xFFu;
      const unsigned peers = __match_any_sync(kFull, in && pin < 32u ? pin : 64u + (uint32_t)lane);
      // the newest record of each pin in this chunk is its lowest lane
      if (in && pin < 32u && (peers & ((1u << lane) - 1u)) == 0u && last_t[warp][pin] < 0)
        last_t[warp][pin] = (int32_t)q.x;
      __syncwarp();
      if (__ballot_sync(kFull, !in)) break;
    }
  }
  float ei = 0.f, es = 0.f, eg = 0.f, el = 0.f;  // FP32 within the item (at most 16 terms a lane)
  float dc = 0.f;                                // adjoint: this lane's share of dL/dC
  // records are read 32 at a time, the next 32 loaded while these are walked; every lane reads its record
  // while it lies inside the gate, so the time after the item's last record comes from the lane after it
  constexpr uint2 kNone = {0xFFFFFFFFu, 0u};
  uint2 qc = s + lane < gb ? W.p_rec[s + lane] : kNone;
  for (int64_t base = s; base < e; base += 32) {
    const int64_t r = base + lane;
    const bool valid = r < e;
    const uint2 qn = (r + 32 < gb && (base + 32 < e || lane == 0)) ? W.p_rec[r + 32] : kNone;
    const uint2 q = valid ? qc : make_uint2(0u, 0u);
    const uint32_t t = q.x, pin = q.y & 0xFFu, v = (q.y >> 8) & 1u;
    const int last_lane = (int)min((int64_t)31, e - 1 - base);
    uint32_t tn = __shfl_down_sync(kFull, qc.x, 1);
    const uint32_t tn31 = __shfl_sync(kFull, qn.x, 0);
    if (lane == 31) tn = tn31;
    if (r + 1 >= gb) tn = 0xFFFFFFFFu;
    qc = qn;
    uint32_t tp = __shfl_up_sync(kFull, t, 1);
    if (lane == 0) tp = t_last;
    const bool head = valid && (r == s || t != tp);
    const bool tail = valid && tn != t;
    int code = 0;
    if (valid) {
      if (t >= T) code = GTP_ERANGE;
      else if (r > ga && t < tp) code = GTP_EORDER;
      else if (pin > n_in || (q.y >> 9) != 0u) code = GTP_ERANGE;
    }
    const uint32_t m = (valid && code == 0) ? 1u << pin : 0u;
    uint32_t X = m;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, X, o);
      if (lane >= o) X ^= y;
    }
    const uint32_t Xi = X ^ S;   // state after this record
    const uint32_t Xe = Xi ^ m;  // state before it
    if (valid && code == 0 && ((Xe >> pin) & 1u) == v) code = GTP_ENOTOGGLE;
    if (code) atomicMin(bad, pat_key(blockIdx.y, r, code));
    const unsigned hb = __ballot_sync(kFull, head) & (kFull >> (31 - lane));
    const uint32_t Xh = __shfl_sync(kFull, Xe, hb ? 31 - __clz(hb) : 0);
    const uint32_t Spre = hb ? Xh : Sg;  // state before this record's group
    float E = 0.f;
    int kind = 0;  // 1 internal, 2 switching, 3 glitch
    float sum_slew = 0.f;
    if (valid && code == 0) {
      if (pin < n_in) {
        const int32_t tb = pat_table(P, c, pin, v, Spre);
        const uint2 dd = __ldg(Q.desc + ((int64_t)g * Q.stride + pin) * 2 + v);  // {knots' element, slew fraction}
        const float fs = __uint_as_float(dd.y);
        const float* tp4 = P.tab + (int64_t)tb * P.tsize + dd.x;
        const float t00 = __ldg(tp4), t01 = __ldg(tp4 + 1), t10 = __ldg(tp4 + P.nl), t11 = __ldg(tp4 + P.nl + 1);
        if (BWD) E = ((1.f - fs) * (t01 - t00) + fs * (t11 - t10)) * lrw;  // dE/dC on the located load segment
        else E = (1.f - fs) * ((1.f - fl) * t00 + fl * t01) + fs * ((1.f - fl) * t10 + fl * t11);
        kind = 1;
        if (GL) sum_slew = slew[pin * 2] + slew[pin * 2 + 1];
      } else {
        E = BWD ? P.half_v2 : esw;
        kind = 2;
        if (GL) sum_slew = Q.oslew[2 * g] + Q.oslew[2 * g + 1];
      }
    }
    if (GL) {
      const bool pv = valid && code == 0;
      const unsigned peers = __match_any_sync(kFull, pv ? pin : 64u + (uint32_t)lane);
      const unsigned lower = peers & ((1u << lane) - 1u);
      const uint32_t tq = __shfl_sync(kFull, t, lower ? 31 - __clz(lower) : lane);
      const int32_t prev = lower ? (int32_t)tq : (pv ? last_t[warp][pin] : -1);
      if (pv && prev >= 0 && (uint32_t)prev / (uint32_t)clk == t / (uint32_t)clk) {
        E *= glitch_ratio(t - (uint32_t)prev, sum_slew);
        kind = 3;
      }
      __syncwarp();
      if (pv && (lane == 31 || (peers >> (lane + 1)) == 0u)) last_t[warp][pin] = (int32_t)t;
      __syncwarp();
    }
    if (BWD) {
      if (kind != 0) dc += __ldcg(&W.grad[bin_of(t, W.bin_magic, W.bin_shift, bin_ps)].x) * E;
      const uint32_t Sg_n = tail ? Xi : Spre;
      Sg = __shfl_sync(kFull, Sg_n, last_lane);
      t_last = __shfl_sync(kFull, t, last_lane);
      S = __shfl_sync(kFull, Xi, 31);
      continue;
    }
    if (kind == 1) ei += E;
    else if (kind == 2) es += E;
    else if (kind == 3) eg += E;
    // leakage: at the end of each group the power changes to that of the state after it, which holds until
    // the next group (or the window's end); the bins take the change in step form
    const float Ppost = (tail && code == 0) ? pat_leak(P, c, Xi) : 0.f;
    const unsigned tl = __ballot_sync(kFull, tail) & ((1u << lane) - 1u);
    const float Pt = __shfl_sync(kFull, Ppost, tl ? 31 - __clz(tl) : 0);
    const float Pbefore = tl ? Pt : Pc;
    const float dP = (tail && code == 0) ? Ppost - Pbefore : 0.f;
    if (tail && code == 0) el += Ppost * (float)((tn < T ? tn : T) - t);
    // bin updates: one {energy, step} reduction per distinct bin of the 32 records
    uint32_t b = 0xFFFFFFFFu;
    float x = 0.f, y = 0.f, corr = 0.f;
    if (valid && code == 0) {
      b = bin_of(t, W.bin_magic, W.bin_shift, bin_ps);
      corr = dP * (float)((b + 1u) * bin_ps - t) * 1e-6f;  // the step's share of this bin
      x = E + corr;
      y = dP;
    }
    if (W.cbins) {  // a component run: every record's components, laid out as the fused walk's (WinDesc::cbins)
      if (b != 0xFFFFFFFFu) {
        const float ki = kind == 1 ? E : 0.f, ks = kind == 2 ? E : 0.f, kg = kind == 3 ? E : 0.f;
        if (W.cpack) {
          red_cbin(W.cbins, b, ki, ks, corr, y);
        } else {
          red_bin(W.bins, b, x, y);
          red_cbin(W.cbins, b, ki, ks, kg, corr);
        }
      }
    } else {
      const uint32_t bprev = __shfl_up_sync(kFull, b, 1);
      if (__any_sync(kFull, lane > 0 && b != 0xFFFFFFFFu && bprev == b)) {  // lanes share a bin: sum them first
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const float xo = __shfl_down_sync(kFull, x, o);
          const float yo = __shfl_down_sync(kFull, y, o);
          const uint32_t bo = __shfl_down_sync(kFull, b, o);
          if (lane + o < 32 && bo == b) {
            x += xo;
            y += yo;
          }
        }
      }
      if (b != 0xFFFFFFFFu && (lane == 0 || bprev != b)) red_bin(W.bins, b, x, y);
    }
    // carries into the next 32 records
    const uint32_t Sg_n = tail ? Xi : Spre;
    const float Pc_n = tail ? Ppost : Pbefore;
    Sg = __shfl_sync(kFull, Sg_n, last_lane);
    Pc = __shfl_sync(kFull, Pc_n, last_lane);
    t_last = __shfl_sync(kFull, t, last_lane);
    S = __shfl_sync(kFull, Xi, 31);
  }
  if (BWD) {
    const double d = warp_sum((double)dc);
    if (lane == 0 && d != 0.0) atomicAdd(W.p_dC + g, (float)d);
    return;
  }
  const double di = warp_sum((double)ei), ds = warp_sum((double)es), dg = warp_sum((double)eg),
               dl = warp_sum((double)el) * 1e-6;
  if (lane == 0) {
    if (di != 0.0) atomicAdd(W.p_e_int + g, di);
    if (ds != 0.0) atomicAdd(W.p_e_sw + g, ds);
    if (dg != 0.0) atomicAdd(W.p_e_gl + g, dg);
    if (dl != 0.0) atomicAdd(W.p_e_leak + g, dl);
    if (e == gb) W.p_final[g] = S;
  }
}

// Records {t, pin | value << 8} from the three arrays of the ABI; a value
// other than 0 or 1 sets bit 9 (rejected by the walk).
__global__ void k_pat_pack(const int32_t* __restrict__ t, const uint8_t* __restrict__ pin,
                           const uint8_t* __restrict__ value, int64_t n, uint2* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t v = value[i];
    out[i] = make_uint2((uint32_t)t[i], (uint32_t)pin[i] | (v > 1u ? 0x200u : v << 8));
  }
}

}  // namespace

cudaError_t launch_pattern_pack(const int32_t* t, const uint8_t* pin, const uint8_t* value, int64_t n, uint2* out,
                                cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  k_pat_pack<<<(unsigned)blocks, 256, 0, st>>>(t, pin, value, n, out);
  return cudaGetLastError();
}

cudaError_t launch_pattern_index(const PatLib& P, int32_t c, int32_t n_in, int32_t* iidx, float* lidx,
                                 cudaStream_t st) {
  const int64_t n = (int64_t)n_in * (1ll << n_in) + (2ll << n_in);
  int64_t blocks = (n + 255) / 256;
  if (blocks > 8192) blocks = 8192;
  k_pat_index<<<(unsigned)blocks, 256, 0, st>>>(P, c, iidx, lidx);
  return cudaGetLastError();
}

cudaError_t launch_pattern_walk(const PatLib& P, const PatNet& Q, const WinDesc* wins, int n_win, int64_t max_items,
                                int32_t clock_ps, unsigned long long* bad, cudaStream_t st, bool backward) {
  if (n_win <= 0) return cudaSuccess;
  int64_t pb = (Q.n_gates + 255) / 256;
  pb = pb < 1 ? 1 : (pb > 256 ? 256 : pb);
  if (backward) k_pat_prepare<true><<<dim3((unsigned)pb, (unsigned)n_win), 256, 0, st>>>(P, Q, wins);
  else k_pat_prepare<false><<<dim3((unsigned)pb, (unsigned)n_win), 256, 0, st>>>(P, Q, wins);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || max_items <= 0) return e;
  const dim3 grid((unsigned)((max_items + kPatWarps - 1) / kPatWarps), (unsigned)n_win);
  k_pat_masks<<<grid, kPatWarps * 32, 0, st>>>(wins);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const dim3 blk(kPatWarps * 32);
  if (backward) {
    if (clock_ps > 0) k_pat_walk<true, true><<<grid, blk, 0, st>>>(P, Q, wins, clock_ps, bad);
    else k_pat_walk<false, true><<<grid, blk, 0, st>>>(P, Q, wins, clock_ps, bad);
  } else {
    if (clock_ps > 0) k_pat_walk<true, false><<<grid, blk, 0, st>>>(P, Q, wins, clock_ps, bad);
    else k_pat_walk<false, false><<<grid, blk, 0, st>>>(P, Q, wins, clock_ps, bad);
  }
  return cudaGetLastError();
}

}  // namespace gtp
