// The time-sliced walk of the busiest gates, with the waveform bins privatised
// in shared memory.
//
// Waveform accumulation (Sec. 2.4.1, Sec. 2.4.2, Sec. 4.3) adds every event's
// energy into the bin that holds its time.  Done straight into L2, that costs
// one reduction per event, and L2 sustains about 200 G reductions a second,
// well below what HBM delivers in records.  Events of different gates only
// meet in a bin if they are walked close together in time, so this walk cuts
// the window into slices of kSliceBins bins and hands out work items
// (chunk of gates, slice): one CTA walks every event of its chunk's gates
// that falls in its slice, adds the energies into the slice's bins in shared
// memory, and at the end adds the whole slice into the window's FP64 bins of
// this walk in L2 with bulk reductions (cp.reduce.async.bulk: one L2
// operation per 32 bytes, i.e. per 2 bins, instead of one per event).
//
// Shared-memory accumulation is exact integer arithmetic: a bin holds two
// signed 32-bit words (energy in units of 2^-24 fJ, leakage step in units of
// 2^-22 nW), updated by 32-bit integer atomics (the fast shared atomic on this
// GPU).  The thread whose add overflows a word sees it in the returned old
// value and adds the lost 2^32 units to the bin's FP64 sum in L2 instead, so
// every per-slice sum is exact and independent of the order of the adds.  The
// slices meet in those FP64 sums (WinDesc::tbins, the cross-block merge), and
// the waveform merge adds them to the other walks' FP32 bins in FP64.
//
// A gate's events in a slice are a contiguous run of its records, found by
// a search for the slice's first and last times (a first guess from the
// gate's mean event rate, then an exponential and a binary search).  The gate
// state entering the run is the state after every earlier event: each pin's
// value is the value written by the last event on that pin (events are
// toggles that carry the new value, Sec. 2.1), found by scanning backwards
// from the run's start; pins without an earlier event keep their initial
// value.  Inside a run, state tracking, lookups and leakage follow the
// persistent walk exactly (XOR transfer words, Algorithm 1's timestamp
// groups, the leakage step representation).  A lane whose records hold no
// tie takes a shorter path (each event is then the head and the tail of its
// own group); each run's energies come from a 256-entry table indexed by the
// input state before the event's group and the record's pin and value.
// Slice boundaries are time boundaries, so no timestamp group is ever split
// between two runs.
//
// Every record of every tiled gate is screened as in the persistent walk
// (time within the run's slice, pin and reserved bits, non-decreasing times,
// toggles); a run whose end search lands before its start means the gate's
// times are not ordered.  Any failure flags the trace; the host then locates
// the first bad record exactly.
#include <algorithm>

#include "gtp_walk_body.cuh"

namespace gtp {
namespace {

constexpr int kTThreads = 512;
constexpr int kTWarps = kTThreads / 32;
constexpr int kTK = 8;                   // records per lane of a segment
constexpr int kTSeg = 32 * kTK;
constexpr int kSliceBins = 16384;        // bins of one slice
constexpr int kChunkMaxGates = 512;      // gates of one chunk
constexpr int kTLeakMax = 512;           // leakage entries staged per CTA
constexpr int kT4 = 64;                  // a warp's event table: (state << 2) | pin
constexpr int kFlushBins = 4096;         // bins converted to FP64 per bulk reduction (64 KB)
constexpr float kEScale = 16777216.f;    // energy words: units of 2^-24 fJ
constexpr float kSScale = 4194304.f;     // leakage-step words: units of 2^-22 nW
constexpr float kQMax = 2.1e9f;          // a larger quantised term goes to L2 directly (FP64)
constexpr int kTargetItems = 4;          // work items wanted per CTA (sets the chunk size)
constexpr uint32_t kVStart = 1u << 30;   // visit flags: the run starts at the gate's first record,
constexpr uint32_t kVEnd = 1u << 31;     //   the run ends at the gate's last record

// Shared memory of a tiled CTA.
constexpr size_t kTBinsBytes = sizeof(int2) * kSliceBins;
constexpr size_t kTRecBytes = sizeof(uint2) * kTWarps * 2 * kTSeg;
constexpr size_t kTHaloBytes = sizeof(uint2) * kTWarps * 4;
constexpr size_t kTT2Bytes = sizeof(float4) * kTWarps * kT4 + sizeof(float) * kTWarps * kGateTab;
constexpr size_t kTLeakBytes = sizeof(float) * kTLeakMax;
constexpr size_t kTVisitBytes = (sizeof(int64_t) + 3 * sizeof(int32_t) + 1) * kChunkMaxGates;
constexpr size_t kTSmem = kTBinsBytes + kTRecBytes + kTHaloBytes + kTT2Bytes + kTLeakBytes + kTVisitBytes;
static_assert(kTSmem <= 227 * 1024, "tiled walk shared memory");

struct TSmem {
  int2* bins;     // [kSliceBins] {energy word, step word}, signed
  uint2* rec;     // this warp's [2][kTSeg] staged records
  uint2* halo;    // this warp's [2][2]: the records just before and just after a segment
  float4* t4;     // this warp's [kT4] table of a toggle of pin p at gate state s, entry (s << 2) | p:
                  //   {energy, leakage after, leakage change * 1e-6, leakage change in step units (int bits)}
  float* gt;      // this warp's copy of the gate's energy table [kGateTab] (timestamp groups with ties)
  float* leak;    // [n_leak] leakage per state, times lscale
  int64_t* vr0;   // [kChunkMaxGates] the chunk's runs in this slice: first record
  int32_t* vn;    //   records in the run
  int32_t* vg;    //   gate
  uint32_t* vinf; //   n_in | leak_base << 4 | kVStart | kVEnd
  uint8_t* vs;    //   state entering the run
};

// One run (a visit) as its warp walks it.
struct TV {
  int64_t r0;
  int32_t n, g;
  uint32_t inf, entry;
};

// The slice of the current work item.
struct TSlice {
  const uint2* rec;
  double2* gbins;         // the window's FP64 bins of this walk (WinDesc::tbins)
  uint32_t T, bin_ps, magic, shift, tau0, tau1, b0, nb;
};

struct TSeg {
  int64_t s0;
  int n_rem, nk;
  uint32_t t_before, t_after;
  bool fh, bad, fast;
  uint32_t ex;
};

// First index in [lo, hi) whose time is >= tau (hi if none), for records
// sorted by time: an exponential search around a guess from the gate's mean
// rate, then a binary search.  On unsorted records it still ends, at some
// index in [lo, hi].
__device__ int64_t lower_bound_time(const uint2* __restrict__ rec, int64_t lo, int64_t hi, uint32_t tau,
                                    uint32_t T) {
  if (lo >= hi) return lo;
  int64_t g = lo + (int64_t)(((uint64_t)(hi - lo) * (uint64_t)tau) / (uint64_t)T);
  g = g < lo ? lo : (g >= hi ? hi - 1 : g);
  int64_t a, b;  // the answer lies in (a, b]
  if (__ldg(&rec[g].x) < tau) {
    a = g;
    b = g + 1;
    int64_t step = 1;
    while (b < hi && __ldg(&rec[b].x) < tau) {
      a = b;
      step <<= 1;
      b = g + step < hi ? g + step : hi;
    }
  } else {
    b = g;
    a = g - 1;
    int64_t step = 1;
    while (a >= lo && __ldg(&rec[a].x) >= tau) {
      b = a;
      step <<= 1;
      a = g - step >= lo ? g - step : lo - 1;
    }
  }
  while (b - a > 1) {
    const int64_t m = a + (b - a) / 2;
    if (__ldg(&rec[m].x) < tau) a = m;
    else b = m;
  }
  return b;
}

// State after records [ga, c): for each pin, the value written by the last
// earlier event on it (a pin with none keeps its bit of `init`).  Reads
// backwards in batches of 8 independent loads.
__device__ uint32_t state_before(const uint2* __restrict__ rec, int64_t ga, int64_t c, uint32_t n_in,
                                 uint32_t init) {
  uint32_t need = (2u << n_in) - 1u, st = 0u;
  int64_t i = c;
  while (need && i > ga) {
    const int nb = i - ga < 8 ? (int)(i - ga) : 8;
    uint32_t m[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) m[k] = k < nb ? __ldg(&rec[i - 1 - k].y) : 0xFFu;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const uint32_t p = m[k] & 0xFu;
      if (k < nb && p <= n_in) {
        const uint32_t bit = 1u << p;
        if (need & bit) {
          st |= ((m[k] >> 4) & 1u) << p;
          need &= ~bit;
        }
      }
    }
    i -= nb;
  }
  return st | (init & need);
}

__device__ __forceinline__ TV load_visit(const TSmem& sm, int i) {
  TV v;
  v.r0 = sm.vr0[i];
  v.n = sm.vn[i];
  v.g = sm.vg[i];
  v.inf = sm.vinf[i];
  v.entry = sm.vs[i];
  return v;
}

// The warp's tables for a visit.  sm.gt holds the gate's 32-entry energy
// table (lane l brought entry l in `gt`), entry (pin << n_in) | s indexed by
// the input pins' state with the pin's own bit at its old value.  sm.t4 holds,
// for a toggle of pin p in gate state s (a valid event: its new value is the
// complement of bit p of s), entry (s << 2) | p: the event's energy, the
// leakage power after it, the leakage change times 1e-6 and the change in
// step-word units.  Returns false if a leakage change is too large for a
// step word (the visit then takes the general path).
__device__ __forceinline__ bool build_t4(const TSmem& sm, float gt, uint32_t n_in, const float* leak, int lane) {
  sm.gt[lane] = gt;
  const uint32_t inmask = (1u << n_in) - 1u;
  bool ok = true;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const uint32_t e = (uint32_t)lane + 32u * h;
    const uint32_t st = e >> 2, pin = e & 3u;
    const bool valid = pin <= n_in && st < (2u << n_in);
    const float E = __shfl_sync(kFull, gt, (int)(((pin << n_in) | (st & inmask)) & 31u));
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (valid) {
      const float P0 = leak[st], P1 = leak[st ^ (1u << pin)];
      const float dp = P1 - P0;
      const float x = dp * kSScale;
      ok = ok && fabsf(x) < kQMax;
      v = make_float4(E, P1, dp * 1e-6f, __int_as_float(fabsf(x) < kQMax ? __float2int_rn(x) : 0));
    }
    sm.t4[e] = v;
  }
  __syncwarp();
  return __all_sync(kFull, ok);
}

// Copy segment s of visit v into `buf`, with the record before it (if the
// gate has one) and the record after it (if the gate has one) into `halo`.
// One commit group (empty when s is past the run).
__device__ __forceinline__ void t_issue(const TSlice& sl, const TV& v, int s, uint2* buf, uint2* halo, int lane) {
  constexpr uint32_t M = kTK / 2 - 1;
  if (s * kTSeg < v.n) {
    const int64_t s0 = v.r0 + (int64_t)s * kTSeg;
    const int n_rem = min(kTSeg, v.n - s * kTSeg);
    const uint32_t sb = smem_addr(buf);
    const uint32_t c0 = 8u * (row_base<kTK>(lane / kTK) ^ (uint32_t)(lane % kTK));
    const uint2* src = sl.rec + s0 + lane;
#pragma unroll
    for (int m = 0; m < kTK; ++m) {
      const uint32_t cm = 8u * ((((uint32_t)(2 * m)) & M) << 1);
      if (m * 32 + lane < n_rem) cp_async8(sb + 256u * m + (c0 ^ cm), src + m * 32);
    }
    if (lane == 0 && (s > 0 || !(v.inf & kVStart))) cp_async8(smem_addr(halo), sl.rec + s0 - 1);
    if (lane == 31 && (s * kTSeg + n_rem < v.n || !(v.inf & kVEnd))) cp_async8(smem_addr(halo + 1), sl.rec + s0 + n_rem);
  }
  cp_async_commit();
}

// First pass over a staged segment: the lane's transfer word, the warp scan
// of transfers, the screen, and whether the lane's events are free of ties
// (every event is then both the head and the tail of its timestamp group).
__device__ __forceinline__ uint32_t t_front(const TSlice& sl, const TV& v, int s, const uint2* buf, const uint2* halo,
                                            TSeg& q, int lane) {
  q.s0 = v.r0 + (int64_t)s * kTSeg;
  q.n_rem = min(kTSeg, v.n - s * kTSeg);
  const int j0 = lane * kTK;
  q.nk = max(0, min(kTK, q.n_rem - j0));
  q.fh = s == 0 && (v.inf & kVStart) && lane == 0;
  q.ex = 0u;
  const bool has_before = s > 0 || !(v.inf & kVStart);
  const bool has_after = s * kTSeg + q.n_rem < v.n || !(v.inf & kVEnd);
  const uint32_t seg_before = has_before ? halo[0].x : 0u;
  const uint32_t seg_after = has_after ? halo[1].x : 0xFFFFFFFFu;
  const uint32_t t_prev_lane = buf[row_base<kTK>(max(lane - 1, 0)) ^ (uint32_t)(kTK - 1)].x;
  const uint32_t t_next_lane = buf[row_base<kTK>(min(lane + 1, 31))].x;
  q.t_before = lane == 0 ? seg_before : t_prev_lane;
  q.t_after = j0 + kTK < q.n_rem ? t_next_lane : seg_after;
  const uint32_t rb = row_base<kTK>(lane);
  const uint4* b4 = reinterpret_cast<const uint4*>(buf);
  uint32_t X = 0u, Y = 0u, H = 0u, tmax = 0u, tmin = 0xFFFFFFFFu, mmax = 0u, tl = 0u;
  int32_t step_min = 0, step_strict = 1;
  uint32_t tp = q.t_before;
#pragma unroll
  for (int k = 0; k < kTK; k += 2) {
    const uint4 w = b4[(rb ^ (uint32_t)k) >> 1];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (k + h < q.nk) {
        const uint32_t t = h ? w.z : w.x, m = h ? w.w : w.y;
        const bool forced = k + h == 0 && q.fh;
        const bool head = t != tp || forced;
        Y = head ? X : Y;
        H = head ? kXH : H;
        X ^= (1u << (m & 0xFu)) & 0xFFu;
        tmax = max(tmax, t);
        tmin = min(tmin, t);
        mmax = max(mmax, m & ~0x10u);
        const int32_t d = (int32_t)(t - tp);
        step_min = min(step_min, d);
        step_strict = forced ? step_strict : min(step_strict, d);
        tp = t;
        tl = t;
      }
    }
  }
  // a time outside the run's slice (the slice ends at or before the window
  // end), a pin or reserved bit out of range, or a decrease
  q.bad = tmax >= sl.tau1 || tmin < sl.tau0 || mmax > (v.inf & 0xFu) || step_min < 0;
  q.fast = step_strict > 0 && (q.nk == 0 || q.t_after > tl);
  uint32_t w = X | (Y << 8) | H;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t a = __shfl_up_sync(kFull, w, o);
    if (lane >= o) w = xcompose(a, w);
  }
  q.ex = __shfl_up_sync(kFull, w, 1);
  if (lane == 0) q.ex = 0u;
  return __shfl_sync(kFull, w, 31);
}

__device__ __forceinline__ void red_f64(double* p, double v) {
  asm volatile("red.global.add.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}

// Add v, in units of 1 / scale, to a signed shared word.  The thread whose
// add overflows the word sees it (the operands' sign against the result's)
// and adds the lost 2^32 units to the bin's FP64 sum in L2 (gaddr, exact)
// instead; a term too large to quantise goes there whole.
__device__ __forceinline__ void acc_word(int* w, float v, float scale, double* gaddr) {
  const float x = v * scale;
  if (fabsf(x) < kQMax) {
    const int q = __float2int_rn(x);
    const int old = atomicAdd(w, q);
    const int now = (int)((unsigned)old + (unsigned)q);
    if (((old ^ now) & (q ^ now)) < 0) red_f64(gaddr, q > 0 ? 4294967296.0 / scale : -4294967296.0 / scale);
  } else {
    red_f64(gaddr, (double)v);
  }
}

// acc_word for a term already in word units (q).
__device__ __forceinline__ void acc_int(int* w, int q, float scale, double* gaddr) {
  const int old = atomicAdd(w, q);
  const int now = (int)((unsigned)old + (unsigned)q);
  if (((old ^ now) & (q ^ now)) < 0) red_f64(gaddr, q > 0 ? 4294967296.0 / scale : -4294967296.0 / scale);
}

// v * 2^-sh as a double, built with integer operations (the FP64 pipe is
// narrow on this GPU); exact for every 32-bit v.
__device__ __forceinline__ double i2d_scaled(int v, int sh) {
  if (v == 0) return 0.0;
  const unsigned long long sign = v < 0 ? 1ull << 63 : 0ull;
  const uint32_t a = v < 0 ? 0u - (uint32_t)v : (uint32_t)v;
  const int lz = __clz(a);
  const unsigned long long frac = ((unsigned long long)a << (lz + 21)) & ((1ull << 52) - 1ull);
  const unsigned long long ex = (unsigned long long)(1023 + 31 - lz - sh);
  return __longlong_as_double((long long)(sign | (ex << 52) | frac));
}

struct TSums {
  float leak, dyn, sw;  // leakage (nW*ps), internal energy (fJ), output events (switching energy = count * Esw)
};

// Replay of a screened segment into the slice's shared bins.
__device__ __forceinline__ TSums t_back(const TSlice& sl, const TSmem& sm, const TV& v, const WinDesc& W,
                                        const uint2* buf, const TSeg& q, uint32_t seg_in, bool fast_ok, DevError* err,
                                        int lane) {
  TSums out{0.f, 0.f, 0.f};
  if (__any_sync(kFull, q.bad)) {
    if (q.bad) report_error(err, GTP_ERANGE, q.s0 + lane * kTK);
    return out;
  }
  const uint32_t n_in = v.inf & 0xFu;
  const uint32_t pmask = (2u << n_in) - 1u, inmask = (1u << n_in) - 1u;
  const float* leak = sm.leak + ((v.inf >> 4) & 0x3FFFFFu);
  const uint32_t li = xcompose(seg_in, q.ex);
  uint32_t st = li & pmask;
  uint32_t spre = (li >> 8) & pmask;
  float Pcur = leak[st];
  float v0 = 0.f, vd = 0.f, vw = 0.f;
  uint32_t tog = 1u;
  uint32_t tp = q.t_before;
  const uint32_t rb = row_base<kTK>(lane);
  bool lb_bad = false;
  if (q.fast && fast_ok) {  // no ties: every event is the head and the tail of its own group
#pragma unroll
    for (int k = 0; k < kTK; ++k) {
      if (k < q.nk) {
        const uint2 rc = buf[rb ^ (uint32_t)k];
        const uint32_t t = rc.x, m = rc.y;
        const uint32_t pin = m & 3u;  // tiled gates have at most 4 pins (screened)
        tog &= (st >> pin) ^ (m >> 4);
        const float4 T4 = sm.t4[(st << 2) | pin];
        st ^= 1u << pin;
        v0 = fmaf(Pcur, (float)(int32_t)(t - tp), v0);
        Pcur = T4.y;
        uint32_t bn = __umulhi(t, sl.magic) >> sl.shift;
        uint32_t bend = (bn + 1u) * sl.bin_ps;
        if (bend <= t) {
          ++bn;
          bend += sl.bin_ps;
        }
        vd += pin < n_in ? T4.x : 0.f;
        vw += pin == n_in ? 1.f : 0.f;
        const uint32_t lb = bn - sl.b0;
        if (lb < sl.nb) {
          acc_word(&sm.bins[lb].x, fmaf(T4.z, (float)(int32_t)(bend - t), T4.x), kEScale, &sl.gbins[bn].x);
          acc_int(&sm.bins[lb].y, __float_as_int(T4.w), kSScale, &sl.gbins[bn].y);
        } else {
          lb_bad = true;
        }
        tp = t;
      }
    }
  } else {  // timestamp groups (Algorithm 1): lookups at the state before the group
    float Pg = leak[spre];
#pragma unroll
    for (int k = 0; k < kTK; ++k) {
      if (k < q.nk) {
        const uint2 rc = buf[rb ^ (uint32_t)k];
        const uint32_t t = rc.x, m = rc.y;
        const uint32_t tn = k + 1 < q.nk ? buf[rb ^ (uint32_t)(k + 1)].x : q.t_after;
        const uint32_t pin = m & 0xFu;
        const bool head = t != tp || (k == 0 && q.fh);
        v0 = head ? fmaf(Pcur, (float)(int32_t)(t - tp), v0) : v0;
        spre = head ? st : spre;
        Pg = head ? Pcur : Pg;
        const uint32_t bitp = 1u << pin;
        const uint32_t own = ((m >> 4) - 1u) & bitp & inmask;
        const float E = sm.gt[((pin << n_in) | (spre & inmask & ~bitp) | own) & 31u];
        tog &= (st >> pin) ^ (m >> 4);
        st = (st ^ bitp) & pmask;
        const bool tail = tn != t;
        const float Pn = tail ? leak[st] : Pcur;
        const float dp = tail ? Pn - Pg : 0.f;
        uint32_t bn = __umulhi(t, sl.magic) >> sl.shift;
        uint32_t bend = (bn + 1u) * sl.bin_ps;
        if (bend <= t) {
          ++bn;
          bend += sl.bin_ps;
        }
        vd += pin < n_in ? E : 0.f;
        vw += pin == n_in ? 1.f : 0.f;
        const uint32_t lb = bn - sl.b0;
        if (lb < sl.nb) {
          acc_word(&sm.bins[lb].x, fmaf(dp, (float)(int32_t)(bend - t) * 1e-6f, E), kEScale, &sl.gbins[bn].x);
          if (dp != 0.f) acc_word(&sm.bins[lb].y, dp, kSScale, &sl.gbins[bn].y);
        } else {
          lb_bad = true;
        }
        Pcur = Pn;
        tp = t;
      }
    }
  }
  if (lb_bad) report_error(err, GTP_ERANGE, q.s0 + lane * kTK);  // cannot happen after the screen
  if (!(tog & 1u)) report_error(err, GTP_ENOTOGGLE, q.s0 + lane * kTK);
  // the gate's last record: leakage to the window end and the final state
  if (q.nk > 0 && (v.inf & kVEnd) && q.s0 + lane * kTK + q.nk == v.r0 + v.n) {
    v0 = fmaf(Pcur, (float)(int32_t)(sl.T - tp), v0);
    W.final_state[v.g] = (uint8_t)st;
  }
  out.leak = v0;
  out.dyn = vd;
  out.sw = vw;
  return out;
}

// Exclusive scan of one value per thread over the block (blockDim.x a
// multiple of 32); *total receives the block's sum.  Ends with a barrier.
__device__ unsigned long long t_block_scan(unsigned long long v, unsigned long long* total) {
  __shared__ unsigned long long wt[32];
  const int l = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  unsigned long long inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long u = __shfl_up_sync(kFull, inc, o);
    if (l >= o) inc += u;
  }
  if (l == 31) wt[w] = inc;
  __syncthreads();
  if (w == 0) {
    const unsigned long long x = l < nw ? wt[l] : 0ull;
    unsigned long long xi = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long u = __shfl_up_sync(kFull, xi, o);
      if (l >= o) xi += u;
    }
    if (l < nw) wt[l] = xi - x;
    if (l == nw - 1) *total = xi;
  }
  __syncthreads();
  const unsigned long long r = inc - v + wt[w];
  __syncthreads();
  return r;
}

// Chunk starts of the tiled list (one block of 1024 threads).  With P_i the
// events of the tiled gates before gate i, gate i starts a chunk if it is the
// first, if floor(P_i / target) > floor(P_(i-1) / target) (the running count
// crossed a multiple of the target), or at every kChunkMaxGates-th gate, so
// that no chunk holds more gates than the visit list.  chunks[0 .. n] with
// chunks[n] = the tiled gate count; n goes to counters[kPlanCntChunks].
__global__ void __launch_bounds__(1024) k_tile_chunks(const WinDesc* __restrict__ wins, PlanBufs P, int32_t* chunks,
                                                      int64_t target_chunks) {
  const WinDesc& W = wins[0];
  const int64_t base = (int64_t)(P.counters[0] + P.counters[1] + P.counters[2]);
  const int64_t n = (int64_t)P.counters[kPlanCntTiled];
  __shared__ unsigned long long cnt[1024];
  __shared__ unsigned long long s_tot, s_starts, s_all, carry_ev, last_c;
  __shared__ long long carry_chunks;
  unsigned long long mine = 0ull;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const int64_t g = P.glist[base + i].y;
    mine += (unsigned long long)(W.offsets[g + 1] - W.offsets[g]);
  }
  t_block_scan(mine, &s_all);
  if (threadIdx.x == 0) {
    carry_ev = 0ull;
    carry_chunks = 0;
    last_c = 0ull;
  }
  __syncthreads();
  const unsigned long long tc = (unsigned long long)(target_chunks > 0 ? target_chunks : 1);
  unsigned long long tgt = (s_all + tc - 1ull) / tc;
  if (tgt == 0ull) tgt = 1ull;
  for (int64_t base_i = 0; base_i < n; base_i += blockDim.x) {
    const int64_t i = base_i + threadIdx.x;
    unsigned long long c = 0ull;
    if (i < n) {
      const int64_t g = P.glist[base + i].y;
      c = (unsigned long long)(W.offsets[g + 1] - W.offsets[g]);
    }
    cnt[threadIdx.x] = c;
    const unsigned long long pi = t_block_scan(c, &s_tot) + carry_ev;  // P_i
    const unsigned long long prev_c = threadIdx.x == 0 ? last_c : cnt[threadIdx.x - 1];
    const bool start = i < n && (i == 0 || (i % kChunkMaxGates) == 0 || pi / tgt != (pi - prev_c) / tgt);
    const unsigned long long k = t_block_scan(start ? 1ull : 0ull, &s_starts);
    if (start) chunks[carry_chunks + (long long)k] = (int32_t)i;
    __syncthreads();
    if (threadIdx.x == 0) {
      carry_ev += s_tot;
      carry_chunks += (long long)s_starts;
      last_c = cnt[blockDim.x - 1];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    chunks[carry_chunks] = (int32_t)n;
    P.counters[kPlanCntChunks] = (unsigned long long)carry_chunks;
  }
}

__global__ void __launch_bounds__(kTThreads, 1) k_tiled(LibView L, NetView N, WalkArgs A, int32_t n_slices) {
  extern __shared__ __align__(16) unsigned char tsmem[];
  __shared__ unsigned long long s_item;
  __shared__ int s_next, s_any;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  TSmem sm;
  unsigned char* p = tsmem;
  sm.bins = reinterpret_cast<int2*>(p);
  p += kTBinsBytes;
  uint2* rec_all = reinterpret_cast<uint2*>(p);
  sm.rec = rec_all + (size_t)wib * 2 * kTSeg;
  p += kTRecBytes;
  sm.halo = reinterpret_cast<uint2*>(p) + (size_t)wib * 4;
  p += kTHaloBytes;
  sm.t4 = reinterpret_cast<float4*>(p) + (size_t)wib * kT4;
  sm.gt = reinterpret_cast<float*>(reinterpret_cast<float4*>(p) + (size_t)kTWarps * kT4) + (size_t)wib * kGateTab;
  p += kTT2Bytes;
  sm.leak = reinterpret_cast<float*>(p);
  p += kTLeakBytes;
  sm.vr0 = reinterpret_cast<int64_t*>(p);
  sm.vn = reinterpret_cast<int32_t*>(sm.vr0 + kChunkMaxGates);
  sm.vg = sm.vn + kChunkMaxGates;
  sm.vinf = reinterpret_cast<uint32_t*>(sm.vg + kChunkMaxGates);
  sm.vs = reinterpret_cast<uint8_t*>(sm.vinf + kChunkMaxGates);

  const WinDesc& W = A.wins[0];
  const PlanBufs& P = A.plan;
  DevError* err = A.err;
  for (int k = threadIdx.x; k < L.n_leak; k += kTThreads) sm.leak[k] = L.leak[k] * L.lscale[L.leak_cell[k]];
  for (int i = threadIdx.x; i < kSliceBins; i += kTThreads) sm.bins[i] = make_int2(0, 0);
  const int64_t tbase = (int64_t)(P.counters[0] + P.counters[1] + P.counters[2]);
  const int64_t n_chunks = (int64_t)P.counters[kPlanCntChunks];
  const int64_t n_items = n_chunks * n_slices;
  TSlice sl;
  sl.rec = W.rec;
  sl.gbins = W.tbins;
  sl.T = (uint32_t)W.window_ps;
  sl.bin_ps = (uint32_t)W.bin_ps;
  sl.magic = W.bin_magic;
  sl.shift = W.bin_shift;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) {
      s_item = atomicAdd(P.counters + kPlanCntTiledWork, 1ull);
      s_next = 0;
      s_any = 0;
    }
    __syncthreads();
    const int64_t item = (int64_t)s_item;
    if (item >= n_items) break;
    const int64_t j = item / n_chunks, c = item % n_chunks;
    const int32_t cs = A.chunks[c], ng = A.chunks[c + 1] - cs;
    sl.b0 = (uint32_t)(j * kSliceBins);
    sl.nb = (uint32_t)min((int64_t)kSliceBins, (int64_t)W.n_bins - sl.b0);
    sl.tau0 = sl.b0 * sl.bin_ps;
    sl.tau1 = j == n_slices - 1 ? sl.T : (sl.b0 + sl.nb) * sl.bin_ps;
    // ---- the chunk's runs in this slice, and each run's entering state
    for (int i = threadIdx.x; i < ng; i += kTThreads) {
      const int64_t g = P.glist[tbase + cs + i].y;
      const int64_t ga = W.offsets[g], ge = W.offsets[g + 1];
      const CellInfo ci = L.cells[N.cell[g]];
      const uint32_t n_in = (uint32_t)ci.n_in;
      int64_t c0 = j == 0 ? ga : lower_bound_time(W.rec, ga, ge, sl.tau0, sl.T);
      int64_t c1 = j == n_slices - 1 ? ge : lower_bound_time(W.rec, ga, ge, sl.tau1, sl.T);
      if (c1 < c0) {  // only on unordered times
        report_error(err, GTP_EORDER, c1);
        c1 = c0;
      }
      const uint32_t init = (uint32_t)W.init[g] & ((2u << n_in) - 1u);
      const uint32_t st = (c1 > c0 && c0 > ga) ? state_before(W.rec, ga, c0, n_in, init) : init;
      sm.vr0[i] = c0;
      sm.vn[i] = (int32_t)(c1 - c0);
      sm.vg[i] = (int32_t)g;
      sm.vinf[i] = n_in | ((uint32_t)ci.leak_base << 4) | (c0 == ga ? kVStart : 0u) | (c1 == ge ? kVEnd : 0u);
      sm.vs[i] = (uint8_t)st;
    }
    __syncthreads();
    // ---- the runs: each warp takes runs from the chunk's list, and the first
    // segment of its next run is copied while it walks the last one of the
    // current run
    auto grab = [&]() -> int {
      int i = 0;
      for (;;) {
        if (lane == 0) i = atomicAdd(&s_next, 1);
        i = __shfl_sync(kFull, i, 0);
        if (i >= ng) return -1;
        if (sm.vn[i] > 0) return i;
      }
    };
    int cur = grab();
    TV vc{}, vn{};
    float gt_next = 0.f, gt_cur = 0.f;
    bool fast_ok = false;
    if (cur >= 0) {
      vc = load_visit(sm, cur);
      if (lane == 0) s_any = 1;
      gt_cur = __ldg(A.gtab + (size_t)vc.g * kGateTab + lane);
      fast_ok = build_t4(sm, gt_cur, vc.inf & 0xFu, sm.leak + ((vc.inf >> 4) & 0x3FFFFFu), lane);
      t_issue(sl, vc, 0, sm.rec, sm.halo, lane);
    }
    int s = 0, kb = 0;
    uint32_t carry = kXAbs | kXH | vc.entry | (vc.entry << 8);
    float f0 = 0.f, f1 = 0.f, f2 = 0.f;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    int nf = 0;
    while (cur >= 0) {
      const int nseg = (vc.n + kTSeg - 1) / kTSeg;
      int nxt = cur, s_n = s + 1;
      if (s_n >= nseg) {
        nxt = grab();
        s_n = 0;
        if (nxt >= 0) {
          vn = load_visit(sm, nxt);
          gt_next = __ldg(A.gtab + (size_t)vn.g * kGateTab + lane);
        }
      }
      const int nb = (kb + 1) & 1;
      if (nxt >= 0) t_issue(sl, nxt == cur ? vc : vn, s_n, sm.rec + nb * kTSeg, sm.halo + nb * 2, lane);
      else cp_async_commit();
      cp_async_wait_1();
      __syncwarp();
      const uint2* buf = sm.rec + (kb & 1) * kTSeg;
      TSeg q;
      const uint32_t tx = t_front(sl, vc, s, buf, sm.halo + (kb & 1) * 2, q, lane);
      const TSums o = t_back(sl, sm, vc, W, buf, q, carry, fast_ok, err, lane);
      carry = xcompose(carry, tx);
      f0 += o.leak;
      f1 += o.dyn;
      f2 += o.sw;
      if (++nf == 8) {  // into FP64 every 64 events a lane
        a0 += (double)warp_sum(f0);
        a1 += (double)warp_sum(f1);
        a2 += (double)warp_sum(f2);
        f0 = f1 = f2 = 0.f;
        nf = 0;
      }
      __syncwarp();
      if (s_n == 0) {  // the run is done: its gate's sums, then the next run
        a0 += (double)warp_sum(f0);
        a1 += (double)warp_sum(f1);
        a2 += (double)warp_sum(f2);
        const uint32_t vin = vc.inf & 0xFu;
        const float esw = __shfl_sync(kFull, gt_cur, (int)((vin << vin) & 31u));  // the output pin's energy
        if (lane == 0) {
          atomicAdd(W.e_leak + vc.g, a0 * 1e-6);
          atomicAdd(W.e_int + vc.g, a1);
          atomicAdd(W.e_sw + vc.g, a2 * (double)esw);
        }
        f0 = f1 = f2 = 0.f;
        a0 = a1 = a2 = 0.0;
        nf = 0;
        cur = nxt;
        if (cur >= 0) {
          vc = vn;
          gt_cur = gt_next;
          fast_ok = build_t4(sm, gt_cur, vc.inf & 0xFu, sm.leak + ((vc.inf >> 4) & 0x3FFFFFu), lane);
          carry = kXAbs | kXH | vc.entry | (vc.entry << 8);
        }
      }
      s = s_n;
      ++kb;
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    // ---- the slice's exact sums into the window's FP64 bins: bulk
    // reductions of kFlushBins bins at a time, converted into the (now idle)
    // record staging area
    if (s_any) {
      double2* fb = reinterpret_cast<double2*>(rec_all);
      for (uint32_t f0 = 0; f0 < sl.nb; f0 += kFlushBins) {
        const uint32_t nf = min((uint32_t)kFlushBins, sl.nb - f0);
        for (uint32_t i = threadIdx.x; i < nf; i += kTThreads) {
          const int2 w = sm.bins[f0 + i];
          fb[i] = make_double2(i2d_scaled(w.x, 24), i2d_scaled(w.y, 22));
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0) {
          asm volatile(
              "cp.reduce.async.bulk.global.shared::cta.bulk_group.add.f64 [%0], [%1], %2;" ::"l"(W.tbins + sl.b0 + f0),
              "r"(smem_addr(fb)), "r"(nf * 16u)
              : "memory");
          asm volatile("cp.async.bulk.commit_group;" ::: "memory");
          asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
        }
        __syncthreads();
      }
      for (int i = threadIdx.x; i < kSliceBins; i += kTThreads) sm.bins[i] = make_int2(0, 0);
    }
  }
}

}  // namespace

int64_t tile_chunk_cap(int64_t n_gates) { return n_gates / kChunkMaxGates + (int64_t)kTargetItems * 1024 + 4; }

bool tiled_fits(const LibView& L) { return L.n_leak <= kTLeakMax; }

cudaError_t launch_tiled(const LibView& L, const NetView& N, const WalkArgs& A, int32_t n_bins, cudaStream_t st) {
  const int32_t n_slices = (n_bins + kSliceBins - 1) / kSliceBins;
  const int64_t target_chunks =
      std::max<int64_t>(1, ((int64_t)kTargetItems * A.n_sm + n_slices - 1) / n_slices);
  k_tile_chunks<<<1, 1024, 0, st>>>(A.wins, A.plan, A.chunks, target_chunks);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_tiled, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTSmem);
  if (e != cudaSuccess) return e;
  k_tiled<<<A.n_sm, kTThreads, kTSmem, st>>>(L, N, A, n_slices);
  return cudaGetLastError();
}

}  // namespace gtp
