// The fused power walk (forward) and its adjoint, over one or many windows.
//
// Gates are split by event density (the paper's event-density-aware
// partitioning, Sec. 4.2, re-cast for one GB300):
//   * sparse gates (at most `dense_min` events) are packed one per lane: a
//     warp takes 32 gates with equal event counts (a counting sort by count
//     builds that order on the device) and each lane walks its gate's events
//     sequentially, so a gate start and end are just the loop bounds;
//   * dense gates are cut into time segments of 32*K events, one warp per
//     segment and K consecutive events per lane; every segment lies inside
//     one gate.
//
// State tracking in a dense segment.  Every event sets one pin to a value, so
// a run of events acts on the gate state as an affine bit map
// S -> (S & keep) | set.  Maps compose associatively: each lane folds its K
// events into a map, a warp shuffle scan composes the lane maps, and the
// segment's incoming state comes from its seed.  Lookups use the state before
// the event's timestamp group (Algorithm 1), so the scan carries a second map:
// the state before the lane's last group.
//
// Seeds.  A dense segment's seed is the state just before its first event,
// read from the events just before it: scanning backwards, the last event of
// each pin fixes that pin's bit; pins without an event since the gate start
// keep their initial bit.  A bounded scan that leaves a pin open (a pin idle
// for a long stretch of a very long gate) hands the segment to a sequential
// fix-up that walks forward from the previous segment's seed, chain by chain,
// so the total fix-up cost stays linear.
//
// Energies (Sec. 2.2, Algorithm 1): each event's 16-byte descriptor (see
// NetView) holds its table element (without the side bits) and its
// interpolation weights; the internal energy is the bilinear value of the
// state-indexed table selected by the side bits of the pre-group state; an
// output event carries 0.5*C*Vdd^2.  Tables live in shared memory.
//
// Forward outputs: one vector reduction {energy, leakage step} per distinct
// bin of a lane's consecutive events (leakage step representation, see
// gtp_kernels.cu); per-gate sums in FP32 per lane, then FP64 (a plain store
// for a sparse gate, one warp reduction and FP64 atomic add per dense
// segment).
//
// Adjoint: the same walks gather g_b = dL/dE_b of each event's bin instead of
// scattering energy, and accumulate dL/dC per gate and dL/d(escale),
// dL/d(lscale) per cell.
#include <cstdio>

#include "gtp_walk.cuh"

namespace gtp {

namespace {

constexpr uint32_t kFull = 0xffffffffu;
constexpr int kSeedScanSegments = 4;  // backward seed scan bound, in segments
constexpr int KS = 8;                 // events staged per lane and chunk in the sparse walk

// ------------------------------------------------------------------ plan
// Per (window, gate): dense gates get consecutive slots in the segment list;
// sparse gates are counted per event count.  Block-aggregated atomics.
__global__ void k_plan_classify(const WinDesc* __restrict__ wins, int64_t G, int64_t seg_len, int dmin, PlanBufs P) {
  extern __shared__ unsigned int sh[];  // [0, dmin]: sparse counts; [dmin+1]: dense slots; [dmin+2]: dense base
  const WinDesc& W = wins[blockIdx.y];
  unsigned long long* hist = P.counters + 3;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < G; base += (int64_t)gridDim.x * blockDim.x) {
    for (int b = threadIdx.x; b <= dmin + 2; b += blockDim.x) sh[b] = 0u;
    __syncthreads();
    const int64_t g = base + threadIdx.x;
    const int64_t c = g < G ? W.offsets[g + 1] - W.offsets[g] : 0;
    unsigned int nseg = 0u, local = 0u;
    if (c > dmin) {
      nseg = (unsigned int)((c + seg_len - 1) / seg_len);
      local = atomicAdd(&sh[dmin + 1], nseg);
    } else if (c > 0) {
      atomicAdd(&sh[c], 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0 && sh[dmin + 1])
      sh[dmin + 2] = (unsigned int)atomicAdd(P.counters, (unsigned long long)sh[dmin + 1]);
    for (int b = 1 + threadIdx.x; b <= dmin; b += blockDim.x)
      if (sh[b]) atomicAdd(hist + b, (unsigned long long)sh[b]);
    __syncthreads();
    if (nseg) {
      const int64_t slot = (int64_t)sh[dmin + 2] + local;
      for (unsigned int k = 0; k < nseg; ++k) P.dtask[slot + k] = make_int4((int)blockIdx.y, (int)g, (int)k, 0);
    }
    __syncthreads();
  }
}

// Bucket starts for the sparse list, largest event count first.
__global__ void k_plan_scan(int dmin, PlanBufs P) {
  if (threadIdx.x != 0) return;
  unsigned long long* hist = P.counters + 3;
  unsigned long long* cursor = hist + dmin + 1;
  unsigned long long acc = 0;
  for (int c = dmin; c >= 1; --c) {
    cursor[c] = acc;
    acc += hist[c];
  }
  P.counters[1] = acc;
}

__global__ void k_plan_scatter(const WinDesc* __restrict__ wins, int64_t G, int dmin, PlanBufs P) {
  extern __shared__ unsigned int sh[];  // [0, dmin]: local counts; [dmin+1, 2*dmin+1]: block bases
  const WinDesc& W = wins[blockIdx.y];
  unsigned long long* cursor = P.counters + 3 + dmin + 1;
  unsigned int* sbase = sh + dmin + 1;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < G; base += (int64_t)gridDim.x * blockDim.x) {
    for (int b = threadIdx.x; b <= dmin; b += blockDim.x) sh[b] = 0u;
    __syncthreads();
    const int64_t g = base + threadIdx.x;
    const int64_t c = g < G ? W.offsets[g + 1] - W.offsets[g] : 0;
    unsigned int local = 0u;
    const bool sparse = c > 0 && c <= dmin;
    if (sparse) local = atomicAdd(&sh[c], 1u);
    __syncthreads();
    for (int b = 1 + threadIdx.x; b <= dmin; b += blockDim.x)
      if (sh[b]) sbase[b] = (unsigned int)atomicAdd(cursor + b, (unsigned long long)sh[b]);
    __syncthreads();
    if (sparse) P.slist[(int64_t)sbase[c] + local] = make_int2((int)blockIdx.y, (int)g);
    __syncthreads();
  }
}

// One thread per dense segment: the state just before its first event (x),
// the state before that event's timestamp group (p), and the time of the
// group before it.
__global__ void k_dseed(LibView L, NetView N, const WinDesc* __restrict__ wins, int64_t seg_len, PlanBufs P) {
  const int64_t n_task = (int64_t)P.counters[0];
  const int64_t limit = seg_len * kSeedScanSegments;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n_task; t += (int64_t)gridDim.x * blockDim.x) {
    const int4 dt = P.dtask[t];
    const WinDesc& W = wins[dt.x];
    const int64_t g = dt.y;
    const int64_t gs = W.offsets[g];
    const int64_t s0 = gs + (int64_t)dt.z * seg_len;
    const uint32_t init = W.init[g];
    const uint32_t full = (2u << L.cells[N.cell[g]].n_in) - 1u;
    Seed sd;
    sd.gate = (int32_t)g;
    sd.pad0 = 0;
    sd.pad1 = 0;
    if (dt.z == 0) {
      sd.t_prev = 0;
      sd.x = (uint8_t)(init & full);
      sd.p = (uint8_t)(init & full);
      sd.flags = kSeedGateStart | kSeedGroupHead;
      P.dseed[t] = sd;
      continue;
    }
    const uint2* rec = W.rec;
    const uint32_t t0 = rec[s0].x;
    int64_t h = s0;
    while (h > gs && s0 - h < limit && rec[h - 1].x == t0) --h;
    const bool head_found = h == gs || rec[h - 1].x != t0;
    uint32_t xres = 0, xval = 0, pres = 0, pval = 0;
    int64_t j = s0 - 1;
    if (head_found) {
      while (j >= gs && ((xres & pres) & full) != full && s0 - 1 - j < limit) {
        const uint32_t meta = rec[j].y;
        const uint32_t bit = (1u << (meta & 0xFu)) & 0xFFu;
        const uint32_t v = (meta & 0x10u) ? bit : 0u;
        if (!(xres & bit)) {
          xres |= bit;
          xval |= v;
        }
        if (j < h && !(pres & bit)) {
          pres |= bit;
          pval |= v;
        }
        --j;
      }
      if (j < gs) {  // reached the gate start: untouched pins keep their initial value
        xval |= init & ~xres;
        pval |= init & ~pres;
        xres = pres = full;
      }
    }
    const bool unresolved = !head_found || (xres & full) != full || (pres & full) != full;
    sd.t_prev = (head_found && h > gs) ? (int32_t)rec[h - 1].x : 0;
    sd.x = (uint8_t)(xval & full);
    sd.p = (uint8_t)(pval & full);
    sd.flags = (uint8_t)((head_found && h == s0 ? kSeedGroupHead : 0) | (unresolved ? kSeedUnresolved : 0));
    P.dseed[t] = sd;
    if (unresolved) {
      const int64_t k = (int64_t)atomicAdd(P.counters + 2, 1ull);
      P.runs[k] = t;
    }
  }
}

// Resolve seeds left partial by k_dseed: the head of each chain of
// unresolved segments of a gate walks forward from the previous segment's
// resolved seed (segments of one gate have consecutive slots).  The
// unresolved flag stays set, since other threads read it to find chain heads.
__global__ void k_dseed_fix(const WinDesc* __restrict__ wins, int64_t seg_len, PlanBufs P) {
  const int64_t n = (int64_t)P.counters[2];
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = P.runs[u];
    if (P.dseed[t - 1].flags & kSeedUnresolved) continue;  // not the head of its chain (t - 1: same gate)
    const int4 dt = P.dtask[t];
    const WinDesc& W = wins[dt.x];
    const int64_t g = dt.y;
    const int64_t gs = W.offsets[g], ge = W.offsets[g + 1];
    const Seed an = P.dseed[t - 1];
    const int64_t a = gs + (int64_t)(dt.z - 1) * seg_len;
    uint32_t X = an.x, Pg = an.p;
    int32_t tp = an.t_prev;
    int32_t tcur = (int32_t)W.rec[a].x;
    int64_t tk = t;
    for (int64_t i = a; i < ge; ++i) {
      const int32_t ti = (int32_t)W.rec[i].x;
      const bool head = ti != tcur;
      if (i > a && (i - gs) % seg_len == 0) {
        if (!(P.dseed[tk].flags & kSeedUnresolved)) break;
        Seed r;
        r.gate = (int32_t)g;
        r.x = (uint8_t)X;
        r.p = (uint8_t)(head ? X : Pg);
        r.t_prev = head ? tcur : tp;
        r.flags = (uint8_t)((head ? kSeedGroupHead : 0) | kSeedUnresolved);
        r.pad0 = 0;
        r.pad1 = 0;
        P.dseed[tk] = r;
        ++tk;
      }
      if (head) {
        tp = tcur;
        tcur = ti;
        Pg = X;
      }
      const uint32_t meta = W.rec[i].y;
      const uint32_t bit = (1u << (meta & 0xFu)) & 0xFFu;
      X = (X & ~bit) | ((meta & 0x10u) ? bit : 0u);
    }
  }
}

// ------------------------------------------------------------------ shared per-event math
struct EventOut {
  float e_in;  // internal energy from the table (meaningful for input events)
  float da, db;
};

__device__ __forceinline__ EventOut table_energy(const SmemLib& sl, const uint4& d, uint32_t spre, uint32_t pin,
                                                 uint32_t n_in, int tsize, int nl) {
  const uint32_t side = side_bits(spre, min(pin, n_in), n_in);
  const float* p = sl.tab + (d.z & 0xFFFFu) + side * (uint32_t)tsize;
  const float a0 = p[0], a1 = p[1], b0 = p[nl], b1 = p[nl + 1];
  EventOut o;
  o.da = a1 - a0;
  o.db = b1 - b0;
  const float lo = fmaf(__uint_as_float(d.y), o.da, a0);
  const float hi = fmaf(__uint_as_float(d.y), o.db, b0);
  o.e_in = fmaf(__uint_as_float(d.x), hi - lo, lo);
  return o;
}

__device__ __forceinline__ int bad_code(bool t_bad, bool o_bad, bool p_bad) {
  return t_bad ? GTP_ERANGE : (o_bad ? GTP_EORDER : (p_bad ? GTP_ERANGE : GTP_ENOTOGGLE));
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// ------------------------------------------------------------------ dense segments
template <int K, bool BWD>
__global__ void __launch_bounds__(256) k_dense(LibView L, NetView N, const WinDesc* __restrict__ wins, PlanBufs P,
                                               DevError* err, double* __restrict__ cell_acc) {
  constexpr int SEG = 32 * K;
  extern __shared__ __align__(16) unsigned char smem[];
  const SmemLib sl = stage_library(L, smem, !BWD);
  unsigned char* sp = smem + smem_lib_bytes(L);
  const int n_wib = blockDim.x >> 5;
  const int wib = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int dstride = N.dstride;
  uint4* dblk = reinterpret_cast<uint4*>(sp) + (size_t)wib * dstride;  // the gate's event descriptors
  sp += (size_t)n_wib * dstride * sizeof(uint4);
  uint2* rec_s = reinterpret_cast<uint2*>(sp) + (size_t)wib * SEG;     // [k][lane]
  sp += (size_t)n_wib * SEG * sizeof(uint2);
  double* wacc = reinterpret_cast<double*>(sp) + (size_t)wib * 2 * L.n_cells;  // adjoint: per-warp cell sums
  if (BWD)
    for (int c = lane; c < 2 * L.n_cells; c += 32) wacc[c] = 0.0;
  __syncthreads();

  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t n_task = (int64_t)P.counters[0];
  const int tsize = L.tsize, nl = L.nl;
  const uint32_t dmax = (uint32_t)(dstride / 2 - 1);

  for (int64_t tk = warp; tk < n_task; tk += n_warps) {
    const int4 dt = P.dtask[tk];
    const WinDesc* Wp = wins + dt.x;
    const int64_t g = dt.y;
    const int64_t* __restrict__ off = Wp->offsets;
    const uint2* __restrict__ rec = Wp->rec;
    const int64_t ga = off[g], ge = off[g + 1];
    const int64_t s0 = ga + (int64_t)dt.z * SEG;
    const int n_rem = (int)min((int64_t)SEG, ge - s0);
    const bool last_seg = s0 + n_rem == ge;
    const bool first_seg = dt.z == 0;
    const int32_t T = Wp->window_ps;
    const uint32_t bin_ps = (uint32_t)Wp->bin_ps, magic = Wp->bin_magic, shift = Wp->bin_shift;
    const int j0 = lane * K;
    const bool active = j0 < n_rem;

    __syncwarp();
#pragma unroll
    for (int m = 0; m < K; ++m) {
      const int r = m * 32 + lane;
      if (r < n_rem) rec_s[(r % K) * 32 + r / K] = __ldcs(rec + s0 + r);
    }
    if (lane < dstride) dblk[lane] = __ldg(N.desc + (size_t)g * dstride + lane);
    const Seed sd = P.dseed[tk];
    uint32_t t_next = 0u;  // first event after the segment, for the group-tail test
    if (lane == 31 && !last_seg) t_next = rec[s0 + n_rem].x;
    const uint32_t cell = (uint32_t)N.cell[g];
    const CellInfo ci = sl.cells[cell];
    const uint32_t n_in = (uint32_t)ci.n_in;
    const uint32_t pmask = (2u << n_in) - 1u;
    const float* leak = sl.leak + ci.leak_base;
    __syncwarp();
    uint32_t t_before;
    if (lane > 0) t_before = rec_s[(K - 1) * 32 + lane - 1].x;
    else t_before = (sd.flags & kSeedGroupHead) ? (uint32_t)sd.t_prev : rec_s[0].x;

    // ---- pass 1: group heads, range checks, the lane's state maps
    uint32_t gh_mask = 0u;
    uint32_t xk = 0xFFu, xs = 0u, pk = 0xFFu, ps = 0u, pm = 0u;
    {
      uint32_t tp = t_before;
#pragma unroll 1
      for (int k = 0; k < K; ++k) {
        const int j = j0 + k;
        if (j >= n_rem) break;
        const uint2 r = rec_s[k * 32 + lane];
        const bool gate_first = first_seg && j == 0;
        const bool is_gh = gate_first || r.x != tp;
        const bool t_bad = r.x >= (uint32_t)T;
        const bool o_bad = !gate_first && (int32_t)r.x < (int32_t)tp;
        const bool p_bad = (r.y >> 5) != 0u || (r.y & 0xFu) > n_in;
        if (t_bad || o_bad || p_bad) report_error(err, bad_code(t_bad, o_bad, p_bad), s0 + j);
        if (is_gh) {
          pk = xk;
          ps = xs;
          pm = 1u;
        }
        const uint32_t bit = (1u << (r.y & 0xFu)) & 0xFFu;
        xk &= ~bit;
        xs = (xs & ~bit) | ((r.y & 0x10u) ? bit : 0u);
        gh_mask |= (is_gh ? 1u : 0u) << k;
        tp = r.x;
      }
    }

    // ---- warp scan of lane maps: (X map, P map, P mode)
    uint32_t wa = (xk & 0xFFu) | ((xs & 0xFFu) << 8) | ((pk & 0xFFu) << 16) | ((ps & 0xFFu) << 24);
    uint32_t wb = pm;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t oa = __shfl_up_sync(kFull, wa, o);
      const uint32_t ob = __shfl_up_sync(kFull, wb, o);
      if (lane >= o) {
        const uint32_t Axk = oa & 0xFFu, Axs = (oa >> 8) & 0xFFu, Apk = (oa >> 16) & 0xFFu, Aps = oa >> 24;
        const uint32_t Bxk = wa & 0xFFu, Bxs = (wa >> 8) & 0xFFu, Bpk = (wa >> 16) & 0xFFu, Bps = wa >> 24;
        const uint32_t nxk = Axk & Bxk, nxs = (Axs & Bxk) | Bxs;
        uint32_t npk, nps, npm;
        if (wb) {
          npk = Axk & Bpk;
          nps = (Axs & Bpk) | Bps;
          npm = 1u;
        } else {
          npk = Apk;
          nps = Aps;
          npm = ob;
        }
        wa = nxk | (nxs << 8) | (npk << 16) | (nps << 24);
        wb = npm;
      }
    }
    uint32_t ea = __shfl_up_sync(kFull, wa, 1), eb = __shfl_up_sync(kFull, wb, 1);
    if (lane == 0) {
      ea = 0xFFu;
      eb = 0u;
    }
    uint32_t st = (((uint32_t)sd.x & (ea & 0xFFu)) | ((ea >> 8) & 0xFFu)) & pmask;
    uint32_t spre = (eb ? (((uint32_t)sd.x & ((ea >> 16) & 0xFFu)) | (ea >> 24)) : (uint32_t)sd.p) & pmask;

    // ---- pass 2: replay
    float v0 = 0.f, v1 = 0.f, v2 = 0.f;  // forward: e_leak, e_int, e_sw; adjoint: dC, d_escale, d_lscale
    uint32_t pb = 0xFFFFFFFFu;
    float pe = 0.f, pdp = 0.f;
    float Gcur = 0.f;  // adjoint: G(time of the current group)
    if (BWD && active && !(first_seg && lane == 0)) {
      const uint32_t tb = t_before;
      if (tb < (uint32_t)T) {
        const uint32_t bb = bin_of(tb, magic, shift, bin_ps);
        const float2 gv = Wp->grad[bb];
        Gcur = gv.y + gv.x * (float)(tb - bb * bin_ps);
      }
    }
    uint32_t tp = t_before;
#pragma unroll 1
    for (int k = 0; k < K; ++k) {
      const int j = j0 + k;
      if (j >= n_rem) break;
      const uint2 r = rec_s[k * 32 + lane];
      const uint32_t t = r.x, pin = r.y & 0xFu, val = (r.y >> 4) & 1u;
      const bool is_gh = (gh_mask >> k) & 1u;
      if (is_gh) spre = st;
      if (((st >> pin) & 1u) == val && pin <= n_in) report_error(err, GTP_ENOTOGGLE, s0 + j);
      const bool ok = t < (uint32_t)T;
      const uint32_t bn = ok ? bin_of(t, magic, shift, bin_ps) : 0u;
      const uint4 d = dblk[min(pin, dmax) * 2u + val];
      const bool is_out = (d.z >> 24) & 1u;
      const EventOut eo = table_energy(sl, d, spre, pin, n_in, tsize, nl);
      if (pin <= n_in) st = ((st & ~(1u << pin)) | (val << pin)) & pmask;
      const bool seg_last = j + 1 == n_rem;
      const bool gate_end = seg_last && last_seg;
      bool tail;
      if (seg_last) tail = gate_end || t_next != t;
      else if (k + 1 < K) tail = rec_s[(k + 1) * 32 + lane].x != t;
      else tail = rec_s[lane + 1].x != t;
      if (BWD) {
        float gE = 0.f, Gt = 0.f;
        if (ok) {
          const float2 gv = Wp->grad[bn];
          gE = gv.x;
          Gt = gv.y + gv.x * (float)(t - bn * bin_ps);
        }
        if (is_gh) {
          v2 += leak[spre] * (Gt - Gcur) * 1e-6f;
          Gcur = Gt;
        }
        if (is_out) {
          v0 += gE * L.half_v2;
        } else {
          v0 += gE * sl.escale[cell] * (fmaf(__uint_as_float(d.x), eo.db - eo.da, eo.da) * __uint_as_float(d.w));
          v1 += gE * eo.e_in;
        }
        if (gate_end) v2 += leak[st] * (Wp->g_total - Gt) * 1e-6f;
      } else {
        if (is_gh) v0 += leak[spre] * (float)((int32_t)t - (int32_t)tp) * 1e-6f;
        const float e = is_out ? __uint_as_float(d.w) : eo.e_in;
        if (is_out) v2 += e; else v1 += e;
        float dp = 0.f, add = 0.f;
        if (tail) {
          dp = leak[st] - leak[spre];
          add = dp * (float)((int32_t)((bn + 1u) * bin_ps) - (int32_t)t) * 1e-6f;
        }
        if (ok) {
          if (bn != pb) {
            if (pb != 0xFFFFFFFFu) red_bin(Wp->bins, pb, pe, pdp);
            pb = bn;
            pe = 0.f;
            pdp = 0.f;
          }
          pe += e + add;
          pdp += dp;
        }
        if (gate_end) {
          v0 += leak[st] * (float)(T - (int32_t)t) * 1e-6f;
          Wp->final_state[g] = (uint8_t)st;
        }
      }
      tp = t;
    }
    if (!BWD && pb != 0xFFFFFFFFu) red_bin(Wp->bins, pb, pe, pdp);
    // ---- per-gate sums: one warp reduction and one atomic add per segment
    v0 = warp_sum(v0);
    v1 = warp_sum(v1);
    v2 = warp_sum(v2);
    if (lane == 0) {
      if (BWD) {
        atomicAdd(Wp->dC + g, v0);
        wacc[cell] += (double)v1;
        wacc[L.n_cells + cell] += (double)v2;
      } else {
        atomicAdd(Wp->e_leak + g, (double)v0);
        atomicAdd(Wp->e_int + g, (double)v1);
        atomicAdd(Wp->e_sw + g, (double)v2);
      }
    }
  }
  if (BWD) {
    __syncwarp();
    for (int c = lane; c < 2 * L.n_cells; c += 32)
      if (wacc[c] != 0.0) atomicAdd(cell_acc + c, wacc[c]);
  }
}

// ------------------------------------------------------------------ sparse gates, one per lane
template <bool BWD>
__global__ void __launch_bounds__(256) k_sparse(LibView L, NetView N, const WinDesc* __restrict__ wins, PlanBufs P,
                                                DevError* err, double* __restrict__ cell_acc) {
  extern __shared__ __align__(16) unsigned char smem[];
  const SmemLib sl = stage_library(L, smem, !BWD);
  unsigned char* sp = smem + smem_lib_bytes(L);
  const int n_wib = blockDim.x >> 5;
  const int wib = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int dstride = N.dstride;
  uint4* dblk = reinterpret_cast<uint4*>(sp) + (size_t)wib * dstride * 32;  // [entry][lane]
  sp += (size_t)n_wib * dstride * 32 * sizeof(uint4);
  uint2* stage = reinterpret_cast<uint2*>(sp) + (size_t)wib * KS * 32;      // [k][lane]
  sp += (size_t)n_wib * KS * 32 * sizeof(uint2);
  double* wacc64 = reinterpret_cast<double*>(sp) + (size_t)wib * 2 * L.n_cells;  // adjoint: per-warp cell sums
  sp += (size_t)n_wib * 2 * L.n_cells * sizeof(double);
  float* wacc = reinterpret_cast<float*>(sp) + (size_t)wib * 2 * L.n_cells;
  if (BWD)
    for (int c = lane; c < 2 * L.n_cells; c += 32) {
      wacc[c] = 0.f;
      wacc64[c] = 0.0;
    }
  __syncthreads();

  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t n_sparse = (int64_t)P.counters[1];
  const int64_t n_task = (n_sparse + 31) / 32;
  const int tsize = L.tsize, nl = L.nl;
  const uint32_t dmax = (uint32_t)(dstride / 2 - 1);

  for (int64_t tk = warp; tk < n_task; tk += n_warps) {
    const int64_t idx = tk * 32 + lane;
    const bool valid = idx < n_sparse;
    const int2 wg = valid ? P.slist[idx] : make_int2(0, 0);
    const WinDesc* Wp = wins + wg.x;
    const int64_t g = wg.y;
    const uint2* rec = Wp->rec;
    const int64_t a = valid ? Wp->offsets[g] : 0;
    const int n = valid ? (int)(Wp->offsets[g + 1] - a) : 0;
    const uint32_t cell = valid ? (uint32_t)N.cell[g] : 0u;
    const CellInfo ci = sl.cells[cell];
    const uint32_t n_in = (uint32_t)ci.n_in;
    const uint32_t pmask = (2u << n_in) - 1u;
    const float* leak = sl.leak + ci.leak_base;
    const int32_t T = Wp->window_ps;
    const uint32_t bin_ps = (uint32_t)Wp->bin_ps, magic = Wp->bin_magic, shift = Wp->bin_shift;
    __syncwarp();
    for (int e = 0; e < dstride; ++e)
      dblk[e * 32 + lane] = valid ? __ldg(N.desc + (size_t)g * dstride + e) : make_uint4(0u, 0u, 0u, 0u);
    uint32_t st = valid ? (uint32_t)Wp->init[g] & pmask : 0u;
    uint32_t spre = st;
    uint32_t tp = 0u;
    int n_max = n;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) n_max = max(n_max, __shfl_xor_sync(kFull, n_max, o));
    float v0 = 0.f, v1 = 0.f, v2 = 0.f;
    float Gcur = 0.f, Gt = 0.f;
    uint32_t pb = 0xFFFFFFFFu;
    float pe = 0.f, pdp = 0.f;
    const uint64_t rec_addr = reinterpret_cast<uint64_t>(rec + a);
    for (int c0 = 0; c0 < n_max; c0 += KS) {
      // stage KS events of each of the 32 gates: 8 lanes copy one gate's 64-byte run
      __syncwarp();
#pragma unroll
      for (int m = 0; m < KS; ++m) {
        const int q = m * 32 + lane;
        const int gi = q / KS, kk = q % KS;
        const uint64_t ra = __shfl_sync(kFull, rec_addr, gi);
        const int ngi = __shfl_sync(kFull, n, gi);
        uint2 rr = make_uint2(0u, 0u);
        if (c0 + kk < ngi) rr = __ldcs(reinterpret_cast<const uint2*>(ra) + c0 + kk);
        stage[kk * 32 + gi] = rr;
      }
      uint32_t t_look = 0u;  // first event of the next chunk
      if (c0 + KS < n) t_look = rec[a + c0 + KS].x;
      __syncwarp();
#pragma unroll 1
      for (int kk = 0; kk < KS; ++kk) {
        const int j = c0 + kk;
        if (j >= n) break;
        const uint2 r = stage[kk * 32 + lane];
        const uint32_t t = r.x, pin = r.y & 0xFu, val = (r.y >> 4) & 1u;
        const bool is_gh = j == 0 || t != tp;
        const bool t_bad = t >= (uint32_t)T;
        const bool o_bad = j > 0 && (int32_t)t < (int32_t)tp;
        const bool p_bad = (r.y >> 5) != 0u || pin > n_in;
        const bool g_bad = !p_bad && ((st >> pin) & 1u) == val;
        if (t_bad || o_bad || p_bad || g_bad) report_error(err, bad_code(t_bad, o_bad, p_bad), a + j);
        const bool ok = !t_bad;
        if (is_gh) spre = st;
        const uint32_t bn = ok ? bin_of(t, magic, shift, bin_ps) : 0u;
        const uint4 d = dblk[(min(pin, dmax) * 2u + val) * 32 + lane];
        const bool is_out = (d.z >> 24) & 1u;
        const EventOut eo = table_energy(sl, d, spre, pin, n_in, tsize, nl);
        if (pin <= n_in) st = ((st & ~(1u << pin)) | (val << pin)) & pmask;
        const bool gate_end = j + 1 == n;
        const uint32_t t_nx = kk + 1 < KS ? stage[(kk + 1) * 32 + lane].x : t_look;
        const bool tail = gate_end || t_nx != t;
        if (BWD) {
          float gE = 0.f;
          Gt = 0.f;
          if (ok) {
            const float2 gv = Wp->grad[bn];
            gE = gv.x;
            Gt = gv.y + gv.x * (float)(t - bn * bin_ps);
          }
          if (is_gh) {
            v2 += leak[spre] * (Gt - Gcur) * 1e-6f;
            Gcur = Gt;
          }
          if (is_out) {
            v0 += gE * L.half_v2;
          } else {
            v0 += gE * sl.escale[cell] * (fmaf(__uint_as_float(d.x), eo.db - eo.da, eo.da) * __uint_as_float(d.w));
            v1 += gE * eo.e_in;
          }
          if (gate_end) v2 += leak[st] * (Wp->g_total - Gt) * 1e-6f;
        } else {
          if (is_gh) v0 += leak[spre] * (float)((int32_t)t - (int32_t)tp) * 1e-6f;
          const float e = is_out ? __uint_as_float(d.w) : eo.e_in;
          if (is_out) v2 += e; else v1 += e;
          float dp = 0.f, add = 0.f;
          if (tail) {
            dp = leak[st] - leak[spre];
            add = dp * (float)((int32_t)((bn + 1u) * bin_ps) - (int32_t)t) * 1e-6f;
          }
          if (ok) {
            if (bn != pb) {
              if (pb != 0xFFFFFFFFu) red_bin(Wp->bins, pb, pe, pdp);
              pb = bn;
              pe = 0.f;
              pdp = 0.f;
            }
            pe += e + add;
            pdp += dp;
          }
          if (gate_end) v0 += leak[st] * (float)(T - (int32_t)t) * 1e-6f;
        }
        tp = t;
      }
    }
    if (BWD) {
      if (valid) {
        Wp->dC[g] = v0;
        atomicAdd(wacc + cell, v1);
        atomicAdd(wacc + L.n_cells + cell, v2);
      }
      __syncwarp();
      for (int c = lane; c < 2 * L.n_cells; c += 32) {
        wacc64[c] += (double)wacc[c];
        wacc[c] = 0.f;
      }
    } else if (valid) {
      if (pb != 0xFFFFFFFFu) red_bin(Wp->bins, pb, pe, pdp);
      Wp->e_leak[g] = (double)v0;
      Wp->e_int[g] = (double)v1;
      Wp->e_sw[g] = (double)v2;
      Wp->final_state[g] = (uint8_t)st;
    }
  }
  if (BWD) {
    __syncwarp();
    for (int c = lane; c < 2 * L.n_cells; c += 32)
      if (wacc64[c] != 0.0) atomicAdd(cell_acc + c, wacc64[c]);
  }
}

// ------------------------------------------------------------------ launchers
size_t dense_smem(const LibView& L, const NetView& N, int K, int block, bool bwd) {
  const size_t w = (size_t)(block / 32);
  size_t b = smem_lib_bytes(L) + w * N.dstride * sizeof(uint4) + w * 32 * K * sizeof(uint2);
  if (bwd) b += w * 2 * L.n_cells * sizeof(double);
  return b;
}

size_t sparse_smem(const LibView& L, const NetView& N, int block, bool bwd) {
  const size_t w = (size_t)(block / 32);
  size_t b = smem_lib_bytes(L) + w * N.dstride * 32 * sizeof(uint4) + w * KS * 32 * sizeof(uint2);
  if (bwd) b += w * 2 * L.n_cells * (sizeof(float) + sizeof(double));
  return b;
}

template <class Kern>
cudaError_t launch_persistent(Kern kern, size_t smem, const WalkArgs& A, const LibView& L, const NetView& N,
                              cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int grid = A.grid;
  if (grid <= 0) {
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, A.block, smem);
    if (e != cudaSuccess) return e;
    grid = (per_sm > 0 ? per_sm : 1) * A.n_sm;
  }
  kern<<<grid, A.block, smem, st>>>(L, N, A.wins, A.plan, A.err, A.cell_acc);
  return cudaGetLastError();
}

template <int K, bool BWD>
cudaError_t launch_dense_k(const LibView& L, const NetView& N, const WalkArgs& A, cudaStream_t st) {
  return launch_persistent(k_dense<K, BWD>, dense_smem(L, N, K, A.block, BWD), A, L, N, st);
}

}  // namespace

bool walk_rpt_supported(int rpt) { return rpt == 4 || rpt == 8 || rpt == 16; }

cudaError_t launch_plan(const NetView& N, const LibView& L, const WalkArgs& A, cudaStream_t st) {
  const int64_t seg_len = 32ll * A.rpt;
  const int dmin = A.dense_min;
  cudaError_t e = cudaMemsetAsync(A.plan.counters, 0, sizeof(unsigned long long) * plan_counter_slots(dmin), st);
  if (e != cudaSuccess) return e;
  int64_t blocks = (A.n_gates + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  if (blocks < 1) blocks = 1;
  const dim3 grid((unsigned)blocks, (unsigned)A.n_win);
  k_plan_classify<<<grid, 256, sizeof(unsigned int) * (dmin + 3), st>>>(A.wins, A.n_gates, seg_len, dmin, A.plan);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_plan_scan<<<1, 32, 0, st>>>(dmin, A.plan);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_plan_scatter<<<grid, 256, sizeof(unsigned int) * 2 * (dmin + 1), st>>>(A.wins, A.n_gates, dmin, A.plan);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_dseed<<<(unsigned)(4 * A.n_sm), 128, 0, st>>>(L, N, A.wins, seg_len, A.plan);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_dseed_fix<<<64, 128, 0, st>>>(A.wins, seg_len, A.plan);
  return cudaGetLastError();
}

cudaError_t launch_walk(const LibView& L, const NetView& N, const WalkArgs& A, bool backward, cudaStream_t st) {
  cudaError_t e;
  if (backward) {
    switch (A.rpt) {
      case 4: e = launch_dense_k<4, true>(L, N, A, st); break;
      case 16: e = launch_dense_k<16, true>(L, N, A, st); break;
      default: e = launch_dense_k<8, true>(L, N, A, st); break;
    }
    if (e != cudaSuccess) return e;
    return launch_persistent(k_sparse<true>, sparse_smem(L, N, A.block, true), A, L, N, st);
  }
  switch (A.rpt) {
    case 4: e = launch_dense_k<4, false>(L, N, A, st); break;
    case 16: e = launch_dense_k<16, false>(L, N, A, st); break;
    default: e = launch_dense_k<8, false>(L, N, A, st); break;
  }
  if (e != cudaSuccess) return e;
  return launch_persistent(k_sparse<false>, sparse_smem(L, N, A.block, false), A, L, N, st);
}

}  // namespace gtp
