// The fused power walk (forward) and its adjoint, over one or many windows:
// device code and the launch template, included by the translation units
// that instantiate the walk (gtp_walk.cu, gtp_walk_glitch.cu).
//
// Gates are split by event density (the paper's event-density-aware
// partitioning, Sec. 4.2, re-cast for one GB300), and every gate is owned by
// exactly one warp or one CTA, so no walk waits on another CTA:
//   * sparse gates (at most `dense_min` events) are packed one per lane: a
//     warp takes 32 gates with equal event counts and each lane walks its
//     gate's events sequentially;
//   * medium gates (up to 8 segments of 32*K events) belong to one warp,
//     which walks their segments in order, K consecutive events per lane;
//   * big gates belong to one CTA of 8 warps, which walks them in chunks of
//     8 consecutive segments, one per warp.
// A counting sort on the device orders the work list big gates first
// (largest first), then medium, then sparse, so persistent CTAs that take
// work from a shared counter finish together.
//
// State tracking inside a segment.  Every valid event toggles its pin, so a
// run of events acts on the gate state by XOR; Algorithm 1 looks energies up
// at the state before the event's timestamp group, so a run is summarised by
// a transfer word (see xcompose): the XOR of its toggles, whether it holds a
// group head, and the XOR of its toggles before its last head.  Transfers
// compose associatively: each lane folds its K events, a warp shuffle scan
// composes the lanes, and the state entering a segment is the composition of
// the gate's earlier segments (carried by the warp, or exchanged through
// shared memory across the 8 warps of a chunk).  An event that does not
// toggle is reported (GTP_ENOTOGGLE).
//
// Energies (Sec. 2.2, Algorithm 1): for cells with at most kTabMaxIn inputs
// the owning warp tabulates the gate's energy per (pin, edge, input state)
// once per gate (bilinear NLDM value of the state-indexed table for an input
// pin, 0.5*C*Vdd^2 for the output pin), so an event's energy is one
// shared-memory load; wider cells interpolate per event.
//
// Forward outputs: one vector reduction {energy, leakage step} per distinct
// bin of a lane's consecutive events (leakage step representation, see
// gtp_kernels.cu); per-gate sums in FP32 per lane and segment, FP64 across
// segments, one plain store per gate.
//
// Adjoint: the same walks gather g_b = dL/dE_b of each event's bin instead of
// scattering energy, and accumulate dL/dC per gate and dL/d(escale),
// dL/d(lscale) per cell.
#pragma once

#include "gtp_walk.cuh"

namespace gtp {

namespace {

constexpr uint32_t kFull = 0xffffffffu;
constexpr int kWarps = kWalkThreads / 32;  // warps of a walk CTA (a big gate's chunk is kWarps segments)

// ------------------------------------------------------------------ shared per-event math
// The adjoint's gradient entry {g_b, G_b} of an event's bin, loaded through
// L2 only: these scattered 8-byte loads would otherwise take L1 lines from
// the sparse threads' gate tables, which the adjoint reads in place (Large:
// adjoint walk 1.416 ms against 1.466 ms through L1; the 100M-event adjoint
// workload 0.718 against 0.734 ms).
__device__ __forceinline__ float2 ld_grad(const float2* p) { return __ldcg(p); }

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// ------------------------------------------------------------------ dense gates
// Transfer word of a run of events:
//   bits 0-7   X: XOR of the run's toggled pin bits
//   bits 8-15  Y: XOR of the toggles before the run's last group head
//   bit 16     H: the run holds a group head (Y is 0 without one)
//   bit 17     A: absolute: X is the state after the run and Y the state
//              before its last group (the state entering the run is folded in)
// Applying a transfer to (state S, pre-group state P) gives
// (S ^ X, H ? S ^ Y : P); xcompose(a, b) is "a, then b".
constexpr uint32_t kXH = 1u << 16;
constexpr uint32_t kXAbs = 1u << 17;
constexpr int kTabMaxIn = 4;                                     // wider cells interpolate per event
constexpr int kTabEntries = (kTabMaxIn + 1) << (kTabMaxIn + 1);  // energies by (pin, edge, input state)
constexpr int kLeakEntries = 2 << kTabMaxIn;

__device__ __forceinline__ uint32_t xcompose(uint32_t a, uint32_t b) {
  if (b & kXAbs) return b;
  if (b & kXH) return (b ^ ((a & 0xFFu) * 0x101u)) | (a & kXAbs);
  return a ^ b;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void cp_async8(uint32_t dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// Staging layout of a warp's segment: lane `row` owns K consecutive records,
// and record k of that row sits at word
//   pos(row, k) = row * K + ((((k >> 1) ^ sw) << 1) | (k & 1)),
//   sw = (row >> s) & (K/2 - 1),  s = 0, 1, 2 for K = 16, 8, 4:
// the row's 16-byte pairs are XOR-permuted so that both the transposing
// 8-byte copies and the lanes' 16-byte reads are free of bank conflicts.

// Per-warp shared memory of the dense walk.
struct DenseSmem {
  uint2* rec;      // [2][32 * K] staged records (double buffer)
  float* etab;     // [kTabEntries] energy at ((pin * 2 + val) << n_in) | input state; adjoint: unscaled
  float* dtab;     // adjoint: [kTabEntries] escale * dE/dC
  float* leak;     // [kLeakEntries] leakage per state (forward: scaled)
  uint2* halo;     // [2][2] per staging buffer: the records just before and just after the segment
  float* ginv;     // glitch detection: [8] per pin 2 / (rise + fall transition time), -1 for none
  uint32_t* gprev; // glitch detection: [8][32] per pin and lane, the pin's previous event time + 1 (0: none)
  uint32_t* gown;  // glitch detection: [8][32] per pin and lane, the lane's last time + 1 on the pin in the segment
  uint32_t* gtot;  // glitch detection: [8] per pin, the last time + 1 before the warp's segment (big gates)
  uint32_t* gcarry;// glitch detection: [8] per pin, the gate's last event time + 1 before the segment
  double* wacc;    // adjoint: [2 * n_cells] per-warp cell sums
};

// One gate as its owning warp sees it.
struct DGate {
  const WinDesc* W;
  const uint2* rec;
  int64_t g, ga, n;          // gate, first record, events (of the piece, for a gate split into pieces)
  bool starts, ends, split;  // the piece starts / ends the gate; the gate is split into pieces
  const uint4* dsc;          // the gate's event descriptors
  const float* gleak;        // the cell's leakage entries (unscaled)
  uint32_t cell, n_in, pmask, inmask, init;
  float esc, lsc;            // energy scale; leakage scale (1 in the adjoint)
  uint32_t T, bin_ps, magic, shift;
};

// A work-list entry {window | piece << kPieceShift, gate}: a gate of more
// than piece_len events (piece_len > 0) is split into pieces of piece_len
// events (a multiple of the longest chunk, so only a gate's last piece can
// end in a partial segment), each its own big item.  PC = false compiles a
// walk for runs in which no gate is split: every item is a whole gate.
template <bool BWD, bool GL, bool PC>
__device__ __forceinline__ DGate dense_gate(const LibView& L, const NetView& N, const WinDesc* __restrict__ wins,
                                            int2 wg, int64_t piece_len) {
  DGate d;
  d.W = wins + (wg.x & kWindowMask);
  d.rec = d.W->rec;
  d.g = wg.y;
  const int64_t gs = d.W->offsets[d.g], ge = d.W->offsets[d.g + 1];
  if (!PC) piece_len = 0;
  d.split = piece_len > 0 && ge - gs > piece_len;
  if (d.split) {
    d.ga = gs + (int64_t)((uint32_t)wg.x >> kPieceShift) * piece_len;
    d.n = min(piece_len, ge - d.ga);
  } else {
    d.ga = gs;
    d.n = ge - gs;
  }
  d.starts = d.ga == gs;
  d.ends = d.ga + d.n == ge;
  d.cell = (uint32_t)N.cell[d.g];
  const CellInfo ci = L.cells[d.cell];
  d.n_in = (uint32_t)ci.n_in;
  d.pmask = (2u << d.n_in) - 1u;
  d.inmask = (1u << d.n_in) - 1u;
  d.init = (uint32_t)d.W->init[d.g] & d.pmask;
  d.esc = L.escale[d.cell];
  d.lsc = BWD ? 1.f : L.lscale[d.cell];
  d.dsc = N.desc + (size_t)d.g * N.dstride;
  d.gleak = L.leak + ci.leak_base;
  d.T = (uint32_t)d.W->window_ps;
  d.bin_ps = (uint32_t)d.W->bin_ps;
  d.magic = d.W->bin_magic;
  d.shift = d.W->bin_shift;
  (void)GL;
  return d;
}

// The gate's energy table and leakage row in the warp's shared memory (TAB:
// cells of at most kTabMaxIn inputs) and, for glitch detection, each pin's
// inverse transition time (any cell: at most 8 pins).
template <bool BWD, bool TAB, bool GL>
__device__ __forceinline__ void build_tables(const LibView& L, const NetView& N, const DGate& d, const DenseSmem& sm,
                                             int lane) {
  if (GL && lane <= (int)d.n_in) {
    const float* sl = lane < (int)d.n_in ? N.slew + ((size_t)d.g * N.stride + lane) * 2 : N.out_slew + 2 * d.g;
    sm.ginv[lane] = glitch_inv(__ldg(sl) + __ldg(sl + 1));
  }
  if (!TAB) return;
  const int ne = (int)((d.n_in + 1u) << (d.n_in + 1u));
  for (int e = lane; e < ne; e += 32) {
    const uint32_t pv = (uint32_t)e >> d.n_in, s = (uint32_t)e & d.inmask;
    const uint32_t pin = pv >> 1;
    const uint4 q = __ldg(d.dsc + pv);
    float E, dE;
    if (pin < d.n_in) {
      const float* p = L.tab + (q.z & 0xFFFFu) + side_bits(s, pin, d.n_in) * (uint32_t)L.tsize;
      const float a0 = __ldg(p), a1 = __ldg(p + 1), b0 = __ldg(p + L.nl), b1 = __ldg(p + L.nl + 1);
      const float fl = __uint_as_float(q.y), fs = __uint_as_float(q.x);
      const float lo = fmaf(fl, a1 - a0, a0), hi = fmaf(fl, b1 - b0, b0);
      const float eu = fmaf(fs, hi - lo, lo);
      E = BWD ? eu : eu * d.esc;
      dE = d.esc * (fmaf(fs, (b1 - b0) - (a1 - a0), a1 - a0) * __uint_as_float(q.w));
    } else {
      E = BWD ? 0.f : __uint_as_float(q.w);
      dE = L.half_v2;
    }
    sm.etab[e] = E;
    if (BWD) sm.dtab[e] = dE;
  }
  for (int s = lane; s < (int)(2u << d.n_in); s += 32) sm.leak[s] = __ldg(d.gleak + s) * d.lsc;
}

// Word offset of record 0 of lane `row` in a staging buffer: record k of
// that row sits at row_base ^ k (pos(row, k) == pos(row, 0) ^ k, because the
// swizzle only permutes aligned pairs within the row).
template <int K>
__device__ __forceinline__ uint32_t row_base(int row) {
  constexpr int kShift = K == 16 ? 0 : (K == 8 ? 1 : 2);
  return (uint32_t)(row * K) ^ ((((uint32_t)row >> kShift) & (uint32_t)(K / 2 - 1)) << 1);
}

// Start the copy of segment `s` of the gate into staging buffer `buf`, with
// its neighbouring records (the gate's record before the segment, if any, and
// the one after it, if any) into `halo` (one commit group, possibly empty).
// Lane l copies records m * 32 + l; their swizzled positions are
// 32 * m + (c0 ^ (((2 * m) & (K/2 - 1)) << 1)) with c0 = pos(l / K, l % K).
template <int K>
__device__ __forceinline__ void issue_segment(const DGate& d, int64_t s, uint2* buf, uint2* halo, int lane) {
  constexpr int SEG = 32 * K;
  constexpr uint32_t M = K / 2 - 1;
  if (s * SEG < d.n) {
    const int64_t s0 = d.ga + s * SEG;
    const int n_rem = (int)min((int64_t)SEG, d.n - s * SEG);
    const uint32_t sb = smem_addr(buf);
    const uint32_t c0 = 8u * (row_base<K>(lane / K) ^ (uint32_t)(lane % K));  // bytes
    const uint2* src = d.rec + s0 + lane;
#pragma unroll
    for (int m = 0; m < K; ++m) {
      const uint32_t cm = 8u * ((((uint32_t)(2 * m)) & M) << 1);
      if (m * 32 + lane < n_rem) cp_async8(sb + 256u * m + (c0 ^ cm), src + m * 32);
    }
    if (lane == 0 && (s > 0 || !d.starts)) cp_async8(smem_addr(halo), d.rec + s0 - 1);
    if (lane == 31 && (s * SEG + SEG < d.n || (!d.ends && n_rem == SEG))) cp_async8(smem_addr(halo + 1), d.rec + s0 + SEG);
  }
  cp_async_commit();
}

// One staged segment with its first pass done.
struct Seg {
  int64_t s0;
  int n_rem, nk;             // events in the segment; this lane's events
  uint32_t t_before;         // time of the event before the lane's first (0 at the gate start)
  uint32_t t_after;          // time of the event after the lane's last (~0 at the gate end)
  bool fh, last_seg;         // the lane's first event starts the gate; the segment ends it
  bool bad;                  // one of the lane's records fails a check (located by the host's trace check)
  uint32_t ex;               // transfer of the segment's events before this lane
};

// Pass 1 of segment s of the gate, staged in `buf` with its neighbours in
// `halo` (the copy must have landed): the lane's transfer, the warp scan of
// transfers, and a cheap screen of the records (the largest time and pin,
// the smallest step between times).  Returns the segment's transfer
// (identity past the gate's end).  FULL: the segment holds 32 * K events.
template <int K, bool FULL>
__device__ __forceinline__ uint32_t seg_front(const DGate& d, int64_t s, const uint2* buf, const uint2* halo, Seg& q,
                                              int lane) {
  constexpr int SEG = 32 * K;
  q.s0 = d.ga + s * SEG;
  q.n_rem = FULL ? SEG : (int)max((int64_t)0, min((int64_t)SEG, d.n - s * SEG));
  const int j0 = lane * K;
  q.nk = FULL ? K : max(0, min(K, q.n_rem - j0));
  q.last_seg = s * SEG + SEG >= d.n && d.ends;  // the segment ends the gate
  q.fh = s == 0 && lane == 0 && d.starts;
  q.bad = false;
  q.ex = 0u;
  if (!FULL && q.n_rem == 0) return 0u;
  const uint32_t seg_before = (s > 0 || !d.starts) ? halo[0].x : 0u;
  const uint32_t seg_after = q.last_seg ? 0xFFFFFFFFu : halo[1].x;  // (a piece's end reads the next piece's first)
  const uint32_t t_prev_lane = buf[row_base<K>(max(lane - 1, 0)) ^ (uint32_t)(K - 1)].x;  // garbage where unused
  const uint32_t t_next_lane = buf[row_base<K>(min(lane + 1, 31))].x;
  q.t_before = lane == 0 ? seg_before : t_prev_lane;
  q.t_after = (FULL ? lane < 31 : j0 + K < q.n_rem) ? t_next_lane : seg_after;

  const uint32_t rb = row_base<K>(lane);
  const uint4* b4 = reinterpret_cast<const uint4*>(buf);
  uint32_t X = 0u, Y = 0u, H = 0u, tmax = 0u, mmax = 0u;
  int32_t step_min = 0;
  uint32_t tp = q.t_before;
#pragma unroll
  for (int k = 0; k < K; k += 2) {
    const uint4 v = b4[(rb ^ (uint32_t)k) >> 1];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (FULL || k + h < q.nk) {
        const uint32_t t = h ? v.z : v.x, m = h ? v.w : v.y;
        const bool head = t != tp || (k + h == 0 && q.fh);
        Y = head ? X : Y;
        H = head ? kXH : H;
        X ^= (1u << (m & 0xFu)) & 0xFFu;
        tmax = max(tmax, t);
        mmax = max(mmax, m & ~0x10u);
        step_min = min(step_min, (int32_t)(t - tp));
        tp = t;
      }
    }
  }
  // any time at or past the window end or past 2^31, any pin or reserved bit
  // out of range, or any decrease (exactly: see seg_check_bits)
  q.bad = tmax >= d.T || mmax > d.n_in || step_min < 0;
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

// Fire-and-forget {energy, leakage step} reduction into bin b when p holds
// (predicated, no branch).
__device__ __forceinline__ void red_bin_if(bool p, float2* bins, uint32_t b, float e, float dp) {
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %3, 0;\n\t@q red.global.add.v2.f32 [%0], {%1, %2};\n\t}" ::"l"(bins + b),
      "f"(e), "f"(dp), "r"((uint32_t)p)
      : "memory");
}

// The same for the bin's component accumulators {internal, switching,
// glitch, leakage in-bin correction}.
__device__ __forceinline__ void red_cbin_if(bool p, float4* cbins, uint32_t b, float ei, float es, float eg,
                                            float lc) {
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %5, 0;\n\t@q red.global.add.v4.f32 [%0], {%1, %2, %3, %4};\n\t}" ::"l"(
          cbins + b),
      "f"(ei), "f"(es), "f"(eg), "f"(lc), "r"((uint32_t)p)
      : "memory");
}

// Bin of t (as bin_of) and the end of that bin in ps.
__device__ __forceinline__ uint32_t bin_end_of(uint32_t t, const DGate& d, uint32_t& end) {
  uint32_t b = __umulhi(t, d.magic) >> d.shift;
  end = (b + 1u) * d.bin_ps;
  const bool up = end <= t;
  b += up ? 1u : 0u;
  end += up ? d.bin_ps : 0u;
  return b;
}

// Per-lane sums of one segment (forward: leakage nW*ps, internal fJ,
// switching fJ, glitch fJ; adjoint: dC, d_escale, d_lscale * 1e6, unused).
struct SegSums {
  float v0, v1, v2, v3;
};

// Glitch detection, per staged segment: each pin's previous event time (+1;
// 0: none) as the lane's first event on that pin sees it (times do not
// decrease along a gate).  Each lane writes its records' times into its
// column of gown (by pin; its last one stays) and notes which pins its
// records hold; per pin, one ballot gives the nearest earlier lane with an
// event on the pin, whose time the lane takes, else before[pin] (the gate's
// last time on the pin before the segment; 0 with before == nullptr, when the
// caller folds it in afterwards).  Returns, in lane p <= n_in, the segment's
// last time on pin p, else before[p] (0).
template <int K, bool FULL>
__device__ __forceinline__ uint32_t gl_segment_prev(const DGate& d, const uint2* buf, const Seg& q, uint32_t* gprev,
                                                    uint32_t* gown, const uint32_t* before, int lane) {
  const uint32_t rb = row_base<K>(lane);
  uint32_t pm = 0u;
#pragma unroll
  for (int k = 0; k < K; ++k)
    if (FULL || k < q.nk) {
      const uint2 r = buf[rb ^ (uint32_t)k];
      const uint32_t pin = min(r.y & 0xFu, 7u);  // a bad pin is screened out before the replay
      gown[pin * 32 + lane] = r.x + 1u;
      pm |= 1u << pin;
    }
  __syncwarp();
  const unsigned lt = (1u << lane) - 1u;
  uint32_t tot = 0u;
#pragma unroll
  for (uint32_t p = 0; p < 8u; ++p) {  // unrolled so that the pins' ballots and loads overlap
    if (p > d.n_in) break;
    const unsigned m = __ballot_sync(kFull, (pm >> p) & 1u);
    const unsigned lo = m & lt;
    const uint32_t b = before ? before[p] : 0u;
    gprev[p * 32 + lane] = lo ? gown[p * 32 + 31 - __clz(lo)] : b;
    if (lane == (int)p) tot = m ? gown[p * 32 + 31 - __clz(m)] : b;
  }
  return tot;
}

template <int K, bool BWD, bool TAB, bool FULL, bool GL, bool CMP>
__device__ __forceinline__ SegSums seg_back(const LibView& L, const NetView& N, const DGate& d, const DenseSmem& sm,
                                            const uint2* buf,
                                            const Seg& q, uint32_t seg_in, DevError* err, int lane) {
  SegSums out{0.f, 0.f, 0.f, 0.f};
  if (!FULL && q.n_rem == 0) return out;
  // A record out of range or out of order: flag the trace (the host then
  // locates the first bad record exactly) and skip the replay, whose bins
  // and table entries would not be safe to index.
  if (__any_sync(kFull, q.bad)) {
    if (q.bad) report_error(err, GTP_ERANGE, q.s0 + lane * K);
    return out;
  }
  const uint32_t li = xcompose(seg_in, q.ex);
  uint32_t st = li & d.pmask;            // state before the lane's first event
  uint32_t spre = (li >> 8) & d.pmask;   // state before the group in progress
  float Pcur, Pg;                        // leakage after the last group; before the current one
  if (TAB) {
    Pcur = sm.leak[st];
    Pg = sm.leak[spre];
  } else {
    Pcur = __ldg(d.gleak + st) * d.lsc;
    Pg = __ldg(d.gleak + spre) * d.lsc;
  }
  float v0 = 0.f, v1 = 0.f, v2 = 0.f, v3 = 0.f;
  float Gcur = 0.f;
  if (BWD && q.t_before < d.T && !q.fh) {
    const uint32_t bb = bin_of(q.t_before, d.magic, d.shift, d.bin_ps);
    const float2 gv = ld_grad(d.W->grad + bb);
    Gcur = gv.y + gv.x * (float)(q.t_before - bb * d.bin_ps);
  }
  const uint32_t rb = row_base<K>(lane);
  uint2 r = buf[rb];                       // the lane's next record
  uint32_t pb = bin_of(r.x, d.magic, d.shift, d.bin_ps);  // pending bin (garbage for a lane without events)
  float pe = 0.f, pdp = 0.f;
  float pi = 0.f, ps = 0.f, pg = 0.f, pc = 0.f;  // CMP: the pending bin's components
  uint32_t tog = 1u;                       // bit 0 clears on an event that does not toggle its pin
  uint32_t tp = q.t_before;
  auto event = [&](int k, uint32_t t, uint32_t m, uint32_t tn) {
    if (!FULL && k >= q.nk) return;
    const uint32_t pin = m & 0xFu, val = (m >> 4) & 1u;
    const bool head = t != tp || (k == 0 && q.fh);
    uint32_t bend;
    const uint32_t bn = bin_end_of(t, d, bend);
    float Gt = 0.f, gE = 0.f;
    if (BWD) {
      const float2 gv = ld_grad(d.W->grad + bn);
      gE = gv.x;
      Gt = gv.y + gv.x * (float)(t - (bend - d.bin_ps));
      v2 = head ? fmaf(Pcur, Gt - Gcur, v2) : v2;
      Gcur = head ? Gt : Gcur;
    } else {
      v0 = head ? fmaf(Pcur, (float)(int32_t)(t - tp), v0) : v0;
    }
    spre = head ? st : spre;
    Pg = head ? Pcur : Pg;
    tog &= (st >> pin) ^ val;
    st = (st ^ (1u << pin)) & d.pmask;
    const bool is_out = pin >= d.n_in;
    float E, dE = 0.f;
    if (TAB) {
      const uint32_t idx = ((pin * 2u + val) << d.n_in) | (spre & d.inmask);
      E = sm.etab[idx];
      if (BWD) dE = sm.dtab[idx];
    } else {
      const uint4 dq = __ldg(d.dsc + min(pin, d.n_in) * 2u + val);
      if (is_out) {
        E = BWD ? 0.f : __uint_as_float(dq.w);
        dE = L.half_v2;
      } else {
        const float* p = L.tab + (dq.z & 0xFFFFu) + side_bits(spre, pin, d.n_in) * (uint32_t)L.tsize;
        const float a0 = __ldg(p), a1 = __ldg(p + 1), b0 = __ldg(p + L.nl), b1 = __ldg(p + L.nl + 1);
        const float fl = __uint_as_float(dq.y), fs = __uint_as_float(dq.x);
        const float lo = fmaf(fl, a1 - a0, a0), hi = fmaf(fl, b1 - b0, b0);
        const float eu = fmaf(fs, hi - lo, lo);
        E = BWD ? eu : eu * d.esc;
        dE = d.esc * (fmaf(fs, (b1 - b0) - (a1 - a0), a1 - a0) * __uint_as_float(dq.w));
      }
    }
    bool glitch = false;
    if (GL) {  // Sec. 2.4.1: an earlier event on this pin in the same clock cycle
      const uint32_t pv = sm.gprev[pin * 32 + lane];
      sm.gprev[pin * 32 + lane] = t + 1u;
      if (pv != 0u && pv - 1u >= cycle_start(t, N.clock_ps, N.clock_magic, N.clock_shift)) {
        const float r = glitch_ratio_inv(t - (pv - 1u), sm.ginv[pin]);
        E *= r;
        dE *= r;
        glitch = true;
      }
    }
    const bool tail = tn != t;
    float Pn = Pcur;
    if (tail) Pn = TAB ? sm.leak[st] : __ldg(d.gleak + st) * d.lsc;
    if (BWD) {
      v0 = fmaf(gE, dE, v0);
      v1 = fmaf(gE, E, v1);
    } else {
      const float Eg = GL && glitch ? E : 0.f;
      const float Er = E - Eg;
      const float Eo = is_out ? Er : 0.f;
      v2 += Eo;
      v1 += Er - Eo;
      if (GL) v3 += Eg;
      const float dp = tail ? Pn - Pg : 0.f;
      const float add = dp * (float)(int32_t)(bend - t) * 1e-6f;
      const bool nb = bn != pb;
      if (CMP && !GL) {  // components without glitches: one {internal, switching, correction, step} reduction
        red_cbin_if(nb, d.W->cbins, pb, pi, ps, pc, pdp);
      } else {
        red_bin_if(nb, d.W->bins, pb, pe, pdp);
        if (CMP) red_cbin_if(nb, d.W->cbins, pb, pi, ps, pg, pc);
      }
      if (CMP) {
        pi = (nb ? 0.f : pi) + (Er - Eo);
        ps = (nb ? 0.f : ps) + Eo;
        pg = (nb ? 0.f : pg) + Eg;
        pc = (nb ? 0.f : pc) + add;
      }
      pe = (nb ? 0.f : pe) + (E + add);
      pdp = (nb ? 0.f : pdp) + dp;
      pb = bn;
    }
    Pcur = Pn;
    tp = t;
  };
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const uint32_t t = r.x, m = r.y;
    if (k + 1 < K) r = buf[rb ^ (uint32_t)(k + 1)];
    event(k, t, m, (k + 1 < K && (FULL || k + 1 < q.nk)) ? r.x : q.t_after);
  }
  if (!BWD && (FULL || q.nk > 0)) {
    if (CMP && !GL) {
      red_cbin(d.W->cbins, pb, pi, ps, pc, pdp);
    } else {
      red_bin(d.W->bins, pb, pe, pdp);
      if (CMP) red_cbin(d.W->cbins, pb, pi, ps, pg, pc);
    }
  }
  if (!(tog & 1u)) report_error(err, GTP_ENOTOGGLE, q.s0 + lane * K);  // located exactly by the host
  // gate end: leakage to the window end and the final state
  if (q.last_seg && q.nk > 0 && lane * K + q.nk == q.n_rem) {
    if (BWD) {
      v2 += Pcur * (d.W->g_total - Gcur);
    } else {
      v0 += Pcur * (float)(int32_t)(d.T - tp);
      d.W->final_state[d.g] = (uint8_t)st;
    }
  }
  out.v0 = v0;
  out.v1 = v1;
  out.v2 = v2;
  out.v3 = v3;
  return out;
}

// Per-gate sums of a warp: each lane adds its segment sums in FP32 for up to
// F segments (at most 64 events a lane), then the warp folds them into FP64
// (valid in lane 0 after flush()).  GB300 issues FP64 at a small fraction of
// the FP32 rate, so the FP64 work is kept to one fold per F segments.
template <int K>
struct GateAcc {
  static constexpr int F = 64 / K;
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  float f0 = 0.f, f1 = 0.f, f2 = 0.f, f3 = 0.f;
  int n = 0;
  __device__ __forceinline__ void flush(bool gl) {
    const float v0 = warp_sum(f0), v1 = warp_sum(f1), v2 = warp_sum(f2);
    a0 += (double)v0;
    a1 += (double)v1;
    a2 += (double)v2;
    if (gl) a3 += (double)warp_sum(f3);
    f0 = f1 = f2 = f3 = 0.f;
    n = 0;
  }
  __device__ __forceinline__ void add(const SegSums& s, bool gl) {
    f0 += s.v0;
    f1 += s.v1;
    f2 += s.v2;
    f3 += s.v3;
    if (++n == F) flush(gl);
  }
};

// Per-gate results from the gate's totals.
// (The pieces of a split gate add their totals: its outputs start at zero.)
template <bool BWD, bool GL>
__device__ __forceinline__ void store_gate(const LibView& L, const DGate& d, const DenseSmem& sm, double a0,
                                           double a1, double a2, double a3) {
  if (BWD) {
    if (d.split) atomicAdd(d.W->dC + d.g, (float)a0);
    else d.W->dC[d.g] = (float)a0;
    sm.wacc[d.cell] += a1;
    sm.wacc[L.n_cells + d.cell] += a2 * 1e-6;
  } else if (d.split) {
    atomicAdd(d.W->e_leak + d.g, a0 * 1e-6);
    atomicAdd(d.W->e_int + d.g, a1);
    atomicAdd(d.W->e_sw + d.g, a2);
    if (GL) atomicAdd(d.W->e_gl + d.g, a3);
  } else {
    d.W->e_leak[d.g] = a0 * 1e-6;
    d.W->e_int[d.g] = a1;
    d.W->e_sw[d.g] = a2;
    if (GL) d.W->e_gl[d.g] = a3;
  }
}

// The transfer word entering a piece that does not start its gate: the
// state after every earlier record and the state before the timestamp group
// the piece starts in (these differ only if that group began in the earlier
// piece).  Each pin's value is the value written by the last earlier event
// on it (events carry their new value, Sec. 2.1); a pin without one keeps its
// initial value.  The warp reads 32 earlier records at a time, newest in
// lane 0.  With glitch detection, gcarry[p] receives the time + 1 of pin p's
// last earlier event (0: none).
template <bool GL>
__device__ __forceinline__ uint32_t piece_entry(const DGate& d, const DenseSmem& sm, int lane) {
  const uint32_t t0 = d.rec[d.ga].x;
  const int64_t gs = d.W->offsets[d.g];
  uint32_t needS = d.pmask, needP = d.pmask, S = 0u, Sp = 0u, last = 0u;
  for (int64_t i = d.ga; (needS | needP) && i > gs; i -= 32) {
    const int64_t j = i - 1 - lane;
    const bool ok = j >= gs;
    const uint2 r = ok ? d.rec[j] : make_uint2(0xFFFFFFFFu, 0xFu);
    const uint32_t pin = r.y & 0xFu, val = (r.y >> 4) & 1u;
    for (uint32_t p = 0; p <= d.n_in; ++p) {
      const uint32_t bit = 1u << p;
      const unsigned bs = __ballot_sync(kFull, ok && pin == p);
      const unsigned bp = __ballot_sync(kFull, ok && pin == p && r.x < t0);
      if ((needS & bit) && bs) {
        const int src = __ffs(bs) - 1;
        S |= __shfl_sync(kFull, val, src) << p;
        const uint32_t tl = __shfl_sync(kFull, r.x, src);
        if (GL && lane == (int)p) last = tl + 1u;
        needS &= ~bit;
      }
      if ((needP & bit) && bp) {
        Sp |= __shfl_sync(kFull, val, __ffs(bp) - 1) << p;
        needP &= ~bit;
      }
    }
  }
  S |= d.init & needS;
  Sp |= d.init & needP;
  if (GL && lane <= (int)d.n_in) sm.gcarry[lane] = last;
  return kXAbs | kXH | S | (Sp << 8);
}

// A medium gate, walked by one warp segment by segment.
template <int K, bool BWD, bool TAB, bool GL, bool CMP>
__device__ __forceinline__ void medium_gate(const LibView& L, const NetView& N, const DGate& d, const DenseSmem& sm,
                                            DevError* err,
                                            int lane) {
  constexpr int SEG = 32 * K;
  const int64_t nseg = (d.n + SEG - 1) / SEG;
  __syncwarp();
  issue_segment<K>(d, 0, sm.rec, sm.halo, lane);
  if (TAB || GL) build_tables<BWD, TAB, GL>(L, N, d, sm, lane);
  if (GL && lane <= (int)d.n_in) sm.gcarry[lane] = 0u;
  uint32_t carry = kXAbs | kXH | d.init | (d.init << 8);
  if (!d.starts) {  // a later piece of a split gate (pieces are big items; kept correct here too)
    __syncwarp();
    carry = piece_entry<GL>(d, sm, lane);
  }
  GateAcc<K> acc;
  Seg q;
  for (int64_t s = 0; s < nseg; ++s) {
    const uint2* cur = sm.rec + (s & 1) * SEG;
    issue_segment<K>(d, s + 1, sm.rec + ((s + 1) & 1) * SEG, sm.halo + ((s + 1) & 1) * 2, lane);
    cp_async_wait_1();
    __syncwarp();
    const uint2* halo = sm.halo + (s & 1) * 2;
    const bool full = (s + 1) * SEG <= d.n;
    const uint32_t tx = full ? seg_front<K, true>(d, s, cur, halo, q, lane) : seg_front<K, false>(d, s, cur, halo, q, lane);
    if (GL) {  // previous event times per pin: this segment's earlier lanes, else the gate's earlier segments
      const uint32_t tot = full ? gl_segment_prev<K, true>(d, cur, q, sm.gprev, sm.gown, sm.gcarry, lane)
                                : gl_segment_prev<K, false>(d, cur, q, sm.gprev, sm.gown, sm.gcarry, lane);
      __syncwarp();
      if (lane <= (int)d.n_in) sm.gcarry[lane] = tot;
    }
    if (full) {
      acc.add(seg_back<K, BWD, TAB, true, GL, CMP>(L, N, d, sm, cur, q, carry, err, lane), GL);
    } else {
      acc.add(seg_back<K, BWD, TAB, false, GL, CMP>(L, N, d, sm, cur, q, carry, err, lane), GL);
    }
    carry = xcompose(carry, tx);
    __syncwarp();
  }
  acc.flush(GL);
  if (lane == 0) store_gate<BWD, GL>(L, d, sm, acc.a0, acc.a1, acc.a2, acc.a3);
}

// A big gate, walked by the CTA's 8 warps in chunks of 8 consecutive
// segments; the state entering each segment is the carry into the chunk
// composed with the transfers of the chunk's earlier segments.
template <int K, bool BWD, bool TAB, bool GL, bool CMP>
__device__ __forceinline__ void big_gate(const LibView& L, const NetView& N, const DGate& d, const DenseSmem& sm,
                                         DevError* err,
                                         uint32_t (*xfer)[kWarps], uint32_t (*gx)[kWarps][8], double (*red)[4],
                                         int wib, int lane) {
  constexpr int SEG = 32 * K;
  const int64_t nchunk = (d.n + (int64_t)kWarps * SEG - 1) / ((int64_t)kWarps * SEG);
  __syncwarp();
  issue_segment<K>(d, wib, sm.rec, sm.halo, lane);
  if (TAB || GL) build_tables<BWD, TAB, GL>(L, N, d, sm, lane);
  if (GL && lane <= (int)d.n_in) sm.gcarry[lane] = 0u;
  uint32_t carry = kXAbs | kXH | d.init | (d.init << 8);
  if (!d.starts) {  // a later piece of a split gate: every warp reads the state it starts from
    __syncwarp();
    carry = piece_entry<GL>(d, sm, lane);
  }
  GateAcc<K> acc;
  Seg q;
  for (int64_t c = 0; c < nchunk; ++c) {
    const int64_t s = c * kWarps + wib;
    const uint2* cur = sm.rec + (c & 1) * SEG;
    issue_segment<K>(d, s + kWarps, sm.rec + ((c + 1) & 1) * SEG, sm.halo + ((c + 1) & 1) * 2, lane);
    cp_async_wait_1();
    __syncwarp();
    const uint2* halo = sm.halo + (c & 1) * 2;
    const bool full = (s + 1) * SEG <= d.n;
    const uint32_t tx = full ? seg_front<K, true>(d, s, cur, halo, q, lane) : seg_front<K, false>(d, s, cur, halo, q, lane);
    if (GL) {  // this segment's own earlier lanes; the segment's last time per pin for the other warps
      const uint32_t tot = full ? gl_segment_prev<K, true>(d, cur, q, sm.gprev, sm.gown, nullptr, lane)
                                : gl_segment_prev<K, false>(d, cur, q, sm.gprev, sm.gown, nullptr, lane);
      if (lane <= (int)d.n_in) gx[c & 1][wib][lane] = tot;
    }
    if (lane == 0) xfer[c & 1][wib] = tx;
    __syncthreads();
    if (GL) {  // fold in the chunk's earlier segments (other warps) and the earlier chunks: lane p for pin p
      if (lane <= (int)d.n_in) {
        uint32_t before = sm.gcarry[lane], all = before;
#pragma unroll
        for (int v = 0; v < kWarps; ++v) {
          const uint32_t m = gx[c & 1][v][lane];
          if (v < wib) before = max(before, m);
          all = max(all, m);
        }
        sm.gtot[lane] = before;
        sm.gcarry[lane] = all;
      }
      __syncwarp();
#pragma unroll
      for (uint32_t p = 0; p < 8u; ++p) {
        if (p > d.n_in) break;
        sm.gprev[p * 32 + lane] = max(sm.gprev[p * 32 + lane], sm.gtot[p]);
      }
    }
    uint32_t seg_in = carry;
#pragma unroll
    for (int v = 0; v < kWarps; ++v) {
      const uint32_t x = xfer[c & 1][v];
      if (v == wib) seg_in = carry;
      carry = xcompose(carry, x);
    }
    acc.add(full ? seg_back<K, BWD, TAB, true, GL, CMP>(L, N, d, sm, cur, q, seg_in, err, lane)
                 : seg_back<K, BWD, TAB, false, GL, CMP>(L, N, d, sm, cur, q, seg_in, err, lane), GL);
    __syncwarp();
  }
  acc.flush(GL);
  if (lane == 0) {
    red[wib][0] = acc.a0;
    red[wib][1] = acc.a1;
    red[wib][2] = acc.a2;
    red[wib][3] = acc.a3;
  }
  __syncthreads();
  if (wib == 0 && lane == 0) {
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    for (int v = 0; v < kWarps; ++v) {
      a0 += red[v][0];
      a1 += red[v][1];
      a2 += red[v][2];
      a3 += red[v][3];
    }
    store_gate<BWD, GL>(L, d, sm, a0, a1, a2, a3);
  }
}

// ------------------------------------------------------------------ sparse gates, one per thread
#ifndef GTP_BWD_TAB_L1
#define GTP_BWD_TAB_L1 1
#endif
// The adjoint's sparse threads read their gate tables in place (through L1)
// instead of staging them in shared memory (64 KB a CTA), so that three
// adjoint CTAs fit an SM (Large: 1.49 ms against 1.68 ms staged at two).
constexpr bool kBwdTabL1 = GTP_BWD_TAB_L1 != 0;
#ifndef GTP_FWD_TAB_L1
#define GTP_FWD_TAB_L1 0
#endif
constexpr bool kFwdTabL1 = GTP_FWD_TAB_L1 != 0;  // the same for the forward walk
template <bool BWD>
constexpr bool kTabL1 = BWD ? kBwdTabL1 : kFwdTabL1;
// Stride between a sparse thread's gate-table entries: its shared-memory
// column, or the table in place.
template <bool BWD>
constexpr int kTabStride = kTabL1<BWD> ? 1 : kWalkThreads;
constexpr int kChunk = 4;                  // events a thread walks per staged round
constexpr int kStage = kChunk + 1;         // records staged per round: its events and the one after them
constexpr int kRounds = 2;                 // rounds in flight (a power of two)
constexpr uint32_t kNoTime = 0xFFFFFFFFu;  // past every valid timestamp

// Copy records [u, u + kStage) of a gate (base rec_g, n records) into one
// staging slot of this thread's column (stride kWalkThreads); records at or
// past n are zero-filled without reading.  One commit group.
__device__ __forceinline__ void stage_round(const uint2* __restrict__ rec_g, uint32_t u, uint32_t n, uint2* slot) {
#pragma unroll
  for (int k = 0; k < kStage; ++k) {
    const bool v = u + k < n;
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(smem_addr(slot + k * kWalkThreads)),
                 "l"(v ? rec_g + u + k : rec_g), "r"(v ? 8 : 0)
                 : "memory");
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

// Per-thread sums, FP32 over a few rounds, then folded into FP64.
struct Sums {
  float f0 = 0.f, f1 = 0.f, f2 = 0.f, f3 = 0.f;
  double d0 = 0.0, d1 = 0.0, d2 = 0.0, d3 = 0.0;
  __device__ __forceinline__ void fold(bool gl) {
    d0 += (double)f0;
    d1 += (double)f1;
    d2 += (double)f2;
    if (gl) d3 += (double)f3;
    f0 = f1 = f2 = f3 = 0.f;
  }
};

__device__ __forceinline__ int bad_event_code(uint32_t t, uint32_t m, uint32_t T, uint32_t n_in, bool order_bad) {
  if (t >= T || (m & ~0x10u) > n_in) return GTP_ERANGE;
  return order_bad ? GTP_EORDER : GTP_ENOTOGGLE;
}

struct WalkOut {
  double v0, v1, v2;  // forward: leakage (nW*ps), internal, switching; adjoint: dC, d_escale, d_lscale * 1e6
  double v3;          // forward with glitch detection: glitch energy
};

// Walk of one sparse gate by one thread (Algorithm 1 in event order): n > 0
// events from rec_g, initial state st.  `tabl` is this thread's column of the
// CTA's staged gate tables (stride kWalkThreads), `col` its staging column
// (kRounds slots of kStage records, stride kWalkThreads), `sleak` the CTA's
// leakage table (forward: scaled).  The records are staged kRounds rounds
// ahead, each round with the record after it so that the last event of a
// round sees the next timestamp without another load.  Forward: each distinct
// bin of consecutive events gets one reduction {energy, leakage step} into L2.
//
// Glitch detection (GL): `last` is this thread's column (stride
// kWalkThreads) of each pin's previous event time, followed by a column of
// each pin's inverse transition time (8 * kWalkThreads further on).
template <bool BWD, bool GL, bool CMP>
__device__ __forceinline__ WalkOut walk_gate(const LibView& L, const NetView& N, const WinDesc& W, const float* tabl,
                                             uint2* col, const float* sleak, DevError* err, int64_t g,
                                             const uint2* __restrict__ rec_g, uint32_t n, uint32_t st,
                                             uint32_t* last) {
#pragma unroll
  for (int r = 0; r < kRounds; ++r) stage_round(rec_g, (uint32_t)(r * kChunk), n, col + r * kStage * kWalkThreads);
  const uint32_t cell = (uint32_t)N.cell[g];
  const CellInfo ci = L.cells[cell];
  const uint32_t n_in = (uint32_t)ci.n_in;
  const uint32_t pmask = (2u << n_in) - 1u, inmask = (1u << n_in) - 1u;
  const float* leak = sleak + ci.leak_base;
  const float esc = L.escale[cell];
  const bool tab = n_in <= (uint32_t)kGateTabMaxIn;
  const uint4* __restrict__ dsc = N.desc + (size_t)g * N.dstride;
  const uint32_t T = (uint32_t)W.window_ps, bin_ps = (uint32_t)W.bin_ps, magic = W.bin_magic,
                 shift = W.bin_shift;

  st &= pmask;
  float Pcur = leak[st];  // leakage after the last group
  float Pg = Pcur;        // leakage before the current group
  uint32_t spre = st;     // state before the current group
  Sums acc;
  float* ginv = reinterpret_cast<float*>(last + 8 * kWalkThreads);
  if (GL)
    for (uint32_t p = 0; p <= n_in; ++p) {
      last[p * kWalkThreads] = kNoTime;
      const float* sl = p < n_in ? N.slew + ((size_t)g * N.stride + p) * 2 : N.out_slew + 2 * g;
      ginv[p * kWalkThreads] = glitch_inv(__ldg(sl) + __ldg(sl + 1));
    }
  float Gcur = 0.f;       // adjoint: G at the last group (G(0) = 0)
  uint32_t tp = 0u;
  uint32_t pb = kNoTime;
  float pe = 0.f, pdp = 0.f;
  float pi = 0.f, ps = 0.f, pg = 0.f, pc = 0.f;  // CMP: the pending bin's components
  bool live = true, bad = false, first = true;
  uint32_t u = 0u;  // first event of the current round
  int slot = 0, n_done = 0;
  while (live) {
    asm volatile("cp.async.wait_group %0;" ::"n"(kRounds - 1) : "memory");
    uint2* buf = col + slot * kStage * kWalkThreads;
    uint32_t rt[kStage], rm[kChunk];
#pragma unroll
    for (int k = 0; k < kStage; ++k) {
      const uint2 r = buf[k * kWalkThreads];
      rt[k] = u + k < n ? r.x : kNoTime;
      if (k < kChunk) rm[k] = r.y;
    }
#pragma unroll
    for (int k = 0; k < kChunk; ++k) {
      if (!live) continue;
      if (u + k >= n) {  // the gate's end
        live = false;
        continue;
      }
      const uint32_t t = rt[k], m = rm[k];
      const uint32_t t_next = rt[k + 1];
      const uint32_t pin = m & 0xFu, val = (m >> 4) & 1u;
      const bool order_bad = (int32_t)t < (int32_t)tp;
      if (t >= T || (m & ~0x10u) > n_in || order_bad || ((st >> pin) & 1u) == val) {
        report_error(err, bad_event_code(t, m, T, n_in, order_bad), (rec_g - W.rec) + u + k);
        live = false;
        bad = true;
        continue;
      }
      const bool head = first || t != tp;
      first = false;
      const uint32_t bn = bin_of(t, magic, shift, bin_ps);
      float gE = 0.f, Gt = 0.f;
      if (BWD) {
        const float2 gv = ld_grad(W.grad + bn);
        gE = gv.x;
        Gt = gv.y + gv.x * (float)(t - bn * bin_ps);
        if (head) acc.f2 += Pcur * (Gt - Gcur);
        Gcur = head ? Gt : Gcur;
      } else {
        if (head) acc.f0 += Pcur * (float)(int32_t)(t - tp);
      }
      Pg = head ? Pcur : Pg;
      spre = head ? st : spre;
      const uint32_t bitp = 1u << pin;
      st ^= bitp;
      const bool is_out = pin == n_in;
      float E, dE = 0.f;
      if (tab) {
        // entry (pin, input state with the pin's own bit = its value before the edge)
        const uint32_t own = (val - 1u) & bitp & inmask;
        const uint32_t idx = (pin << n_in) | (spre & inmask & ~bitp) | own;
        if (kTabL1<BWD>) {  // the table in place: read-only loads
          E = __ldg(tabl + idx);
          if (BWD) dE = __ldg(tabl + kGateTab + idx) * (is_out ? 1.f : esc);
        } else {
          E = tabl[idx * kTabStride<BWD>];
          if (BWD) dE = tabl[(kGateTab + idx) * kTabStride<BWD>] * (is_out ? 1.f : esc);
        }
      } else if (is_out) {
        E = BWD ? 0.f : __uint_as_float(__ldg(dsc + 2u * n_in).w);
        dE = L.half_v2;
      } else {
        const uint4 d = __ldg(dsc + pin * 2u + val);
        const float* p = L.tab + (d.z & 0xFFFFu) + side_bits(spre, pin, n_in) * (uint32_t)L.tsize;
        const float a0 = __ldg(p), a1 = __ldg(p + 1), b0 = __ldg(p + L.nl), b1 = __ldg(p + L.nl + 1);
        const float fl = __uint_as_float(d.y), fs = __uint_as_float(d.x);
        const float lo = fmaf(fl, a1 - a0, a0), hi = fmaf(fl, b1 - b0, b0);
        const float eu = fmaf(fs, hi - lo, lo);
        E = BWD ? eu : eu * esc;
        dE = esc * (fmaf(fs, (b1 - b0) - (a1 - a0), a1 - a0) * __uint_as_float(d.w));
      }
      bool glitch = false;
      if (GL) {  // Sec. 2.4.1: an earlier event on this pin in the same clock cycle
        const uint32_t t_prev = last[pin * kWalkThreads];
        last[pin * kWalkThreads] = t;
        if (t_prev != kNoTime && t_prev >= cycle_start(t, N.clock_ps, N.clock_magic, N.clock_shift)) {
          const float r = glitch_ratio_inv(t - t_prev, ginv[pin * kWalkThreads]);
          E *= r;
          dE *= r;
          glitch = true;
        }
      }
      const bool tail = t_next != t;
      const float Pn = leak[st];
      if (BWD) {
        acc.f0 += gE * dE;
        acc.f1 += gE * E;
      } else {
        if (GL && glitch) acc.f3 += E; else if (is_out) acc.f2 += E; else acc.f1 += E;
        const float dp = tail ? Pn - Pg : 0.f;
        const float add = dp * (float)(int32_t)((bn + 1u) * bin_ps - t) * 1e-6f;
        if (bn != pb) {
          if (pb != kNoTime) {
            if (CMP && !GL) {
              red_cbin(W.cbins, pb, pi, ps, pc, pdp);
            } else {
              red_bin(W.bins, pb, pe, pdp);
              if (CMP) red_cbin(W.cbins, pb, pi, ps, pg, pc);
            }
          }
          pb = bn;
          pe = 0.f;
          pdp = 0.f;
          pi = ps = pg = pc = 0.f;
        }
        pe += E + add;
        pdp += dp;
        if (CMP) {
          if (GL && glitch) pg += E; else if (is_out) ps += E; else pi += E;
          pc += add;
        }
      }
      Pcur = tail ? Pn : Pcur;
      tp = t;
    }
    if (!live) break;
    // refill the slot just walked with the round kRounds ahead
    stage_round(rec_g, u + kRounds * kChunk, n, buf);
    u += kChunk;
    slot = (slot + 1) & (kRounds - 1);
    if (++n_done == 16) {
      acc.fold(GL);
      n_done = 0;
    }
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  if (!BWD && pb != kNoTime) {
    if (CMP && !GL) {
      red_cbin(W.cbins, pb, pi, ps, pc, pdp);
    } else {
      red_bin(W.bins, pb, pe, pdp);
      if (CMP) red_cbin(W.cbins, pb, pi, ps, pg, pc);
    }
  }
  // the gate's end: leakage to the window end, and the final state
  if (!bad) {
    if (BWD) {
      acc.f2 += Pcur * (W.g_total - Gcur);
    } else {
      acc.f0 += Pcur * (float)(int32_t)(T - tp);
      W.final_state[g] = (uint8_t)st;
    }
  }
  acc.fold(GL);
  return WalkOut{acc.d0, acc.d1, acc.d2, acc.d3};
}

// This thread's gate table into its column of the CTA's staged tables.
template <bool BWD>
__device__ __forceinline__ void stage_gate_table(const float* __restrict__ gt, int64_t g, float* stab, uint32_t n_in) {
  constexpr int kN = BWD ? 2 * kGateTab : kGateTab;
  const float4* src = reinterpret_cast<const float4*>(gt + (size_t)g * kN);
  // only the cell's entries: 4, 12 or 32 for 1, 2 or 3 inputs (the forward table; the adjoint's two halves whole)
  const int nq = BWD ? kN / 4 : (int)((((n_in + 1u) << n_in) + 3u) >> 2);
#pragma unroll
  for (int q = 0; q < kN / 4; ++q) {
    if (q >= nq) break;
    const float4 v = __ldg(src + q);
    stab[(4 * q + 0) * kWalkThreads] = v.x;
    stab[(4 * q + 1) * kWalkThreads] = v.y;
    stab[(4 * q + 2) * kWalkThreads] = v.z;
    stab[(4 * q + 3) * kWalkThreads] = v.w;
  }
}

// Shared memory of a walk CTA: a union of the dense items' per-warp areas
// (staged records and their neighbours, energy table, leakage row) and the sparse items' area
// (per-thread gate tables, per-thread staged records, the leakage table),
// then, for the adjoint, the per-warp cell sums.
// With glitch detection the dense area adds each warp's per-pin transition
// times and the sparse area each thread's per-pin previous event times.
__host__ __device__ inline size_t dense_area(int K, bool bwd, bool gl) {
  return (size_t)kWarps * (2 * 32 * K * sizeof(uint2) + (bwd ? 2 : 1) * kTabEntries * sizeof(float) +
                           kLeakEntries * sizeof(float) + 4 * sizeof(uint2) +
                           (gl ? 8 * sizeof(float) + (2 * 8 * 32 + 16) * sizeof(uint32_t) : 0));
}
__host__ __device__ inline size_t sparse_area(int n_leak, bool bwd, bool gl) {
  return (size_t)(bwd ? (kBwdTabL1 ? 0 : 2) : (kFwdTabL1 ? 0 : 1)) * kGateTab * kWalkThreads * sizeof(float) +
         (size_t)kRounds * kStage * kWalkThreads * sizeof(uint2) + (gl ? (size_t)16 * kWalkThreads * sizeof(uint32_t) : 0) +
         (((size_t)n_leak * sizeof(float) + 15) & ~(size_t)15);
}
__host__ __device__ inline size_t union_area(int K, int n_leak, bool bwd, bool gl) {
  const size_t d = dense_area(K, bwd, gl), sp = sparse_area(n_leak, bwd, gl);
  return d > sp ? d : sp;
}

// Persistent CTAs of 8 warps take work items from the shared counter: one big
// gate per item (all 8 warps), 8 medium gates per item (one per warp), then
// 256 sparse gates per item (one per thread).  The forward walk with 4 or 8
// records per lane fits three CTAs per SM (80 registers), and so does the
// adjoint with its gate tables read in place (a few bytes spilled).  With 16
// records per lane or glitch detection the walk would spill at 80: these
// are given the registers of two CTAs (measured on the large workload: 16
// records per lane at two CTAs 1.18 ms, at three 1.38 ms; glitch detection
// at two 2.11 ms, at three 2.19 ms).
#ifndef GTP_WALK_MINB
#define GTP_WALK_MINB 3  // resident CTAs an SM the forward walk is compiled for (registers: 80)
#endif
#ifndef GTP_WALK_MINB_GL
#define GTP_WALK_MINB_GL 2  // resident CTAs an SM the glitch walk is compiled for (registers: 128)
#endif
#ifndef GTP_WALK_MINB_BWD
#define GTP_WALK_MINB_BWD 3  // the same for the adjoint walk (80 registers, a few bytes spilled)
#endif
template <int K, bool BWD, bool GL, bool CMP, bool PC>
__global__ void __launch_bounds__(kWalkThreads,
                                  K == 16 ? 2 : (GL ? GTP_WALK_MINB_GL : (BWD ? GTP_WALK_MINB_BWD : GTP_WALK_MINB)))
    k_walk(LibView L, NetView N, WalkArgs A) {
  constexpr int SEG = 32 * K;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ uint32_t xfer[2][kWarps];
  __shared__ double red[kWarps][4];
  __shared__ uint32_t gx[GL ? 2 : 1][kWarps][8];  // glitch detection: each warp's segment-last time per pin
  __shared__ unsigned long long s_item;
  const int wib = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const PlanBufs& P = A.plan;
  const WinDesc* __restrict__ wins = A.wins;
  DevError* err = A.err;
  // dense view of the union area
  unsigned char* sp = smem;
  DenseSmem sm;
  sm.rec = reinterpret_cast<uint2*>(sp) + (size_t)wib * 2 * SEG;
  sp += (size_t)kWarps * 2 * SEG * sizeof(uint2);
  sm.etab = reinterpret_cast<float*>(sp) + (size_t)wib * kTabEntries;
  sp += (size_t)kWarps * kTabEntries * sizeof(float);
  sm.dtab = reinterpret_cast<float*>(sp) + (size_t)wib * kTabEntries;
  if (BWD) sp += (size_t)kWarps * kTabEntries * sizeof(float);
  sm.leak = reinterpret_cast<float*>(sp) + (size_t)wib * kLeakEntries;
  sp += (size_t)kWarps * kLeakEntries * sizeof(float);
  sm.halo = reinterpret_cast<uint2*>(sp) + (size_t)wib * 4;
  sp += (size_t)kWarps * 4 * sizeof(uint2);
  sm.ginv = reinterpret_cast<float*>(sp) + (size_t)wib * 8;
  sp += (size_t)kWarps * 8 * sizeof(float);
  sm.gprev = reinterpret_cast<uint32_t*>(sp) + (size_t)wib * (2 * 8 * 32 + 16);
  sm.gown = sm.gprev + 8 * 32;
  sm.gtot = sm.gown + 8 * 32;
  sm.gcarry = sm.gtot + 8;
  // sparse view of the union area
  float* stab = reinterpret_cast<float*>(smem);
  uint2* sstg = reinterpret_cast<uint2*>(stab + (BWD ? (kBwdTabL1 ? 0 : 2) : (kFwdTabL1 ? 0 : 1)) * kGateTab * kWalkThreads);
  uint32_t* slast = reinterpret_cast<uint32_t*>(sstg + kRounds * kStage * kWalkThreads);
  float* sleak = reinterpret_cast<float*>(slast + (GL ? 16 * kWalkThreads : 0));
  // adjoint cell sums, after the union
  sm.wacc = reinterpret_cast<double*>(smem + union_area(K, L.n_leak, BWD, GL)) + (size_t)wib * 2 * L.n_cells;
  if (BWD)
    for (int c = lane; c < 2 * L.n_cells; c += 32) sm.wacc[c] = 0.0;

  const int64_t n_big = (int64_t)P.counters[0];
  const int64_t n_med = (int64_t)P.counters[1];
  const int64_t n_sparse = (int64_t)P.counters[2];
  const int64_t n_dense_items = n_big + (n_med + kWarps - 1) / kWarps;
  const int64_t n_sparse_items = (n_sparse + kWalkThreads - 1) / kWalkThreads;
  const int64_t n_items = n_dense_items + n_sparse_items;
  const float* gt = BWD ? A.gtab_bwd : A.gtab;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = atomicAdd(P.counters + 3, 1ull);
    __syncthreads();
    const int64_t pos = (int64_t)s_item;
    if (pos >= n_items) break;
    // Dense and sparse items are handed out evenly interleaved (each list
    // keeps its order), so L2-reduction-bound dense work and latency-bound
    // sparse work share the SMs for the whole launch.
    const int64_t dense_before = pos * n_dense_items / n_items;
    const bool is_dense = (pos + 1) * n_dense_items / n_items > dense_before;
    const int64_t item = is_dense ? dense_before : n_dense_items + (pos - dense_before);
    if (item < n_big) {
      const DGate d = dense_gate<BWD, GL, PC>(L, N, wins, P.glist[item], A.piece_len);
      if (d.n_in <= (uint32_t)kTabMaxIn) big_gate<K, BWD, true, GL, CMP>(L, N, d, sm, err, xfer, gx, red, wib, lane);
      else big_gate<K, BWD, false, GL, CMP>(L, N, d, sm, err, xfer, gx, red, wib, lane);
    } else if (item < n_dense_items) {
      const int64_t i = (item - n_big) * kWarps + wib;
      if (i < n_med) {
        const DGate d = dense_gate<BWD, GL, PC>(L, N, wins, P.glist[n_big + i], A.piece_len);
        if (d.n_in <= (uint32_t)kTabMaxIn) medium_gate<K, BWD, true, GL, CMP>(L, N, d, sm, err, lane);
        else medium_gate<K, BWD, false, GL, CMP>(L, N, d, sm, err, lane);
      }
    } else {
      // ---- 256 sparse gates, one per thread
      for (int k = threadIdx.x; k < L.n_leak; k += kWalkThreads)
        sleak[k] = BWD ? L.leak[k] : L.leak[k] * L.lscale[L.leak_cell[k]];
      __syncthreads();
      const int64_t i = (item - n_dense_items) * kWalkThreads + threadIdx.x;
      if (i < n_sparse) {
        const int2 wg = P.glist[n_big + n_med + i];
        const WinDesc& W = wins[wg.x & kWindowMask];
        const int64_t g = wg.y;
        const int64_t ga = W.offsets[g], ge = W.offsets[g + 1];
        const float* my_tab = stab + threadIdx.x;
        if (kTabL1<BWD>)
          my_tab = gt + (size_t)g * (BWD ? 2 : 1) * kGateTab;  // read in place, through L1
        else if (const uint32_t nin = (uint32_t)L.cells[N.cell[g]].n_in; nin <= (uint32_t)kGateTabMaxIn)
          stage_gate_table<BWD>(gt, g, stab + threadIdx.x, nin);
        const WalkOut o = walk_gate<BWD, GL, CMP>(L, N, W, my_tab, sstg + threadIdx.x, sleak, err, g, W.rec + ga,
                                             (uint32_t)(ge - ga), (uint32_t)W.init[g], slast + threadIdx.x);
        if (BWD) {
          W.dC[g] = (float)o.v0;
          const uint32_t cell = (uint32_t)N.cell[g];
          atomicAdd(sm.wacc + cell, o.v1);
          atomicAdd(sm.wacc + L.n_cells + cell, o.v2 * 1e-6);
        } else {
          W.e_leak[g] = o.v0 * 1e-6;
          W.e_int[g] = o.v1;
          W.e_sw[g] = o.v2;
          if (GL) W.e_gl[g] = o.v3;
        }
      }
    }
  }
  if (BWD) {
    __syncwarp();
    for (int c = lane; c < 2 * L.n_cells; c += 32)
      if (sm.wacc[c] != 0.0) atomicAdd(A.cell_acc + c, sm.wacc[c]);
  }
}

// ------------------------------------------------------------------ launchers
template <int K, bool BWD, bool GL, bool CMP, bool PC = true>
cudaError_t launch_walk_k(const LibView& L, const NetView& N, const WalkArgs& A, cudaStream_t st) {
  const size_t smem =
      union_area(K, L.n_leak, BWD, GL) + (BWD ? (size_t)kWarps * 2 * L.n_cells * sizeof(double) : 0);
  cudaError_t e =
      cudaFuncSetAttribute(k_walk<K, BWD, GL, CMP, PC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int grid = A.grid;
  if (grid <= 0) {
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_walk<K, BWD, GL, CMP, PC>, kWalkThreads, smem);
    if (e != cudaSuccess) return e;
    grid = (per_sm > 0 ? per_sm : 1) * A.n_sm;
  }
  k_walk<K, BWD, GL, CMP, PC><<<grid, kWalkThreads, smem, st>>>(L, N, A);
  return cudaGetLastError();
}

// The walk of a run with no gate split into pieces (BWD: the adjoint).
template <bool BWD, bool GL>
cudaError_t launch_walk_whole(const LibView& L, const NetView& N, const WalkArgs& A, cudaStream_t st) {
  switch (A.rpt) {
    case 4: return launch_walk_k<4, BWD, GL, false, false>(L, N, A, st);
    case 16: return launch_walk_k<16, BWD, GL, false, false>(L, N, A, st);
    default: return launch_walk_k<8, BWD, GL, false, false>(L, N, A, st);
  }
}

// The walk of one glitch setting: GL = whether glitch detection is on.
template <bool GL>
cudaError_t launch_walk_gl(const LibView& L, const NetView& N, const WalkArgs& A, bool backward, cudaStream_t st) {
  if (backward) {
    switch (A.rpt) {
      case 4: return launch_walk_k<4, true, GL, false>(L, N, A, st);
      case 16: return launch_walk_k<16, true, GL, false>(L, N, A, st);
      default: return launch_walk_k<8, true, GL, false>(L, N, A, st);
    }
  }
  switch (A.rpt) {
    case 4: return launch_walk_k<4, false, GL, false>(L, N, A, st);
    case 16: return launch_walk_k<16, false, GL, false>(L, N, A, st);
    default: return launch_walk_k<8, false, GL, false>(L, N, A, st);
  }
}

// The forward walk that also accumulates the per-component bins.
template <bool GL>
cudaError_t launch_walk_cmp(const LibView& L, const NetView& N, const WalkArgs& A, cudaStream_t st) {
  switch (A.rpt) {
    case 4: return launch_walk_k<4, false, GL, true>(L, N, A, st);
    case 16: return launch_walk_k<16, false, GL, true>(L, N, A, st);
    default: return launch_walk_k<8, false, GL, true>(L, N, A, st);
  }
}

}  // namespace

}  // namespace gtp
