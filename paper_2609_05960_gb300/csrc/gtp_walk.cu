// The fused power walk (forward) and its adjoint, over one or many windows.
//
// The records of all gates form one flat, gate-major array per window (CSR by
// gate, time-ordered within a gate).  It is cut into equal segments of 32*K
// records; each warp of a persistent grid takes one segment at a time (from
// one global list covering every window of the launch), and each lane owns K
// consecutive records.  Work is balanced whatever the per-gate event skew: a
// sparse gate is walked inside one lane, a dense gate is cut into time slices
// across lanes and warps (the paper's per-gate temporal partitioning,
// Sec. 4.2, with equal event counts per slice instead of equal cycle counts).
//
// State tracking.  Every event sets one pin to a value, so the effect of a
// run of events on the gate state is an affine bit map S -> (S & keep) | set.
// Maps compose associatively, so the state before any record is a prefix
// composition: each lane folds its K records into a map (a gate start resets
// the map to the constant initial state), the warp scans lane maps with
// shuffles, and the segment's first state comes from a seed.  Lookups use the
// state before the record's timestamp group (Algorithm 1), so the scan also
// carries a second map: the state before the lane's last group.
//
// Seeds.  A segment's seed is the state just before its first record, read
// from the events just before it: scanning backwards, the last event of each
// pin fixes that pin's bit; pins with no event since the gate start keep their
// initial bit.  One thread per segment scans backwards, usually resolving
// every pin within a few records.  A bounded scan that has not resolved every
// pin (a pin idle for a long time inside a very long gate) leaves the seed to
// a sequential fix-up that walks forward from the previous segment's seed, so
// the total fix-up cost stays linear in the trace.
//
// Energies (Sec. 2.2, Algorithm 1): internal energy of an input-pin event from
// the state-indexed table of (cell, pin, edge, side bits of the pre-group
// state), bilinear at the gate's precomputed (slew, load) coordinates;
// 0.5*C*Vdd^2 for an output event.  Tables live in shared memory.
//
// Forward outputs: per bin one vector reduction {energy, leakage step} per
// distinct bin of a lane's consecutive records (leakage step representation,
// see gtp_kernels.cu); per gate FP32 sums within a warp segment (lane
// sequential, then a segmented warp scan) and FP64 across segments (atomic
// adds only for gates that cross a segment boundary).
//
// Adjoint (gradient of a loss of the waveform): the same walk gathers
// g_b = dL/dE_b of each event's bin instead of scattering energy, and
// accumulates dL/dC per gate and dL/d(escale), dL/d(lscale) per cell.
#include <cstdio>

#include "gtp_walk.cuh"

namespace gtp {

namespace {

constexpr uint32_t kFull = 0xffffffffu;
constexpr int kSeedScanSegments = 4;  // backward seed scan bound, in segments

__device__ __forceinline__ int window_of(const int64_t* base, int n_win, int64_t x) {
  int lo = 0, hi = n_win - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (base[mid] <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// ------------------------------------------------------------------ seeds
// Gate of each segment's first record: a gate owning records [a, b) owns the
// segments starting in that range.  Gate-parallel, no per-segment search.
__global__ void k_seg_gates(NetView N, const WinDesc* __restrict__ wins, int64_t seg_len) {
  const WinDesc& W = wins[blockIdx.y];
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < N.n_gates;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = W.offsets[g], b = W.offsets[g + 1];
    if (a == b) continue;
    for (int64_t s = (a + seg_len - 1) / seg_len; s * seg_len < b; ++s) W.seeds[s].gate = (int32_t)g;
  }
}

// One thread per segment: the state just before the segment's first record
// (x), the state before that record's timestamp group (p), and the time of
// the group before it.
__global__ void k_seed(LibView L, NetView N, const WinDesc* __restrict__ wins, const int64_t* __restrict__ seg_base,
                       int n_win, int64_t n_seg_total, int64_t seg_len, int64_t* __restrict__ runs) {
  const int64_t limit = seg_len * kSeedScanSegments;
  for (int64_t sg = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; sg < n_seg_total;
       sg += (int64_t)gridDim.x * blockDim.x) {
    const int w = window_of(seg_base, n_win, sg);
    const WinDesc& W = wins[w];
    const int64_t s = sg - W.seg_base;
    const int64_t s0 = s * seg_len;
    const int64_t g = W.seeds[s].gate;
    const int64_t gs = W.offsets[g];
    const uint32_t init = W.init[g];
    Seed sd;
    sd.gate = (int32_t)g;
    sd.pad0 = 0;
    sd.pad1 = 0;
    if (s0 == gs) {
      sd.t_prev = 0;
      sd.x = (uint8_t)init;
      sd.p = (uint8_t)init;
      sd.flags = kSeedGateStart | kSeedGroupHead;
      W.seeds[s] = sd;
      continue;
    }
    const uint2* rec = W.rec;
    const uint32_t t0 = rec[s0].x;
    int64_t h = s0;
    while (h > gs && s0 - h < limit && rec[h - 1].x == t0) --h;
    const bool head_found = h == gs || rec[h - 1].x != t0;
    const uint32_t full = (2u << L.cells[N.cell[g]].n_in) - 1u;
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
    W.seeds[s] = sd;
    if (unresolved) {
      const int64_t k = (int64_t)atomicAdd(reinterpret_cast<unsigned long long*>(runs), 1ull);
      runs[1 + k] = sg;
    }
  }
}

// Resolve seeds left partial by k_seed: the head of each chain of unresolved
// segments walks forward from the previous segment's (resolved) seed.  The
// unresolved flag stays set, since other threads read it to find chain heads.
__global__ void k_seed_fix(const WinDesc* __restrict__ wins, const int64_t* __restrict__ seg_base, int n_win,
                           int64_t seg_len, const int64_t* __restrict__ runs) {
  const int64_t n = runs[0];
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
    const int64_t sg = runs[1 + u];
    const int w = window_of(seg_base, n_win, sg);
    const WinDesc& W = wins[w];
    const int64_t s = sg - W.seg_base;
    if (s <= 0 || (W.seeds[s - 1].flags & kSeedUnresolved)) continue;  // not the head of its chain
    const Seed an = W.seeds[s - 1];
    const int64_t g = an.gate;
    const int64_t ge = W.offsets[g + 1];
    const int64_t a = (s - 1) * seg_len;
    uint32_t X = an.x, Pg = an.p;
    int32_t tp = an.t_prev;
    int32_t tcur = (int32_t)W.rec[a].x;
    for (int64_t i = a; i < ge; ++i) {
      const int32_t ti = (int32_t)W.rec[i].x;
      const bool head = ti != tcur;
      if (i > a && i % seg_len == 0) {
        const int64_t s2 = i / seg_len;
        if (!(W.seeds[s2].flags & kSeedUnresolved)) break;
        Seed r;
        r.gate = (int32_t)g;
        r.x = (uint8_t)X;
        r.p = (uint8_t)(head ? X : Pg);
        r.t_prev = head ? tcur : tp;
        r.flags = (uint8_t)((head ? kSeedGroupHead : 0) | kSeedUnresolved);
        r.pad0 = 0;
        r.pad1 = 0;
        W.seeds[s2] = r;
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

// ------------------------------------------------------------------ the walk
template <int K, bool BWD>
__global__ void __launch_bounds__(256) k_walk(LibView L, NetView N, const WinDesc* __restrict__ wins,
                                              const int64_t* __restrict__ seg_base_g, int n_win,
                                              int64_t n_seg_total, DevError* err, double* __restrict__ cell_acc) {
  constexpr int SEG = 32 * K;
  constexpr int NV = BWD ? 1 : 3;  // per-gate values reduced across lanes
  extern __shared__ __align__(16) unsigned char smem[];
  const SmemLib sl = stage_library(L, smem, !BWD);
  unsigned char* sp = smem + smem_lib_bytes(L);
  int64_t* sbase = reinterpret_cast<int64_t*>(sp);
  sp += ((size_t)(n_win + 1) * 8 + 15) & ~(size_t)15;
  for (int k = threadIdx.x; k <= n_win; k += blockDim.x) sbase[k] = seg_base_g[k];
  const int n_wib = blockDim.x >> 5;
  const int wib = threadIdx.x >> 5;
  // per-warp staging, all [k][lane]: event descriptors, records, gate ids
  uint4* dsc_s = reinterpret_cast<uint4*>(sp) + (size_t)wib * SEG;
  sp += (size_t)n_wib * SEG * sizeof(uint4);
  uint2* rec_s = reinterpret_cast<uint2*>(sp) + (size_t)wib * SEG;
  sp += (size_t)n_wib * SEG * sizeof(uint2);
  int* gid_s = reinterpret_cast<int*>(sp) + (size_t)wib * SEG;
  sp += (size_t)n_wib * SEG * sizeof(int);
  float* wacc = nullptr;     // adjoint: per warp 2*n_cells FP32 (escale, lscale)
  double* wacc64 = nullptr;  // adjoint: per warp 2*n_cells FP64
  const int nc2 = 2 * L.n_cells;
  if (BWD) {
    wacc64 = reinterpret_cast<double*>(sp) + (size_t)wib * nc2;
    sp += (size_t)n_wib * nc2 * sizeof(double);
    wacc = reinterpret_cast<float*>(sp) + (size_t)wib * nc2;
    for (int c = threadIdx.x & 31; c < nc2; c += 32) {
      wacc[c] = 0.f;
      wacc64[c] = 0.0;
    }
  }
  __syncthreads();

  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t G = N.n_gates;
  const int tsize = L.tsize;
  const int nl = L.nl;
  const int dstride = N.dstride;
  const uint4* __restrict__ desc = N.desc;

  for (int64_t sgl = warp; sgl < n_seg_total; sgl += n_warps) {
    const int w = window_of(sbase, n_win, sgl);
    const WinDesc* Wp = wins + w;
    const uint2* __restrict__ rec = Wp->rec;
    const int64_t* __restrict__ off = Wp->offsets;
    const uint8_t* __restrict__ init = Wp->init;
    const int64_t n_ev = Wp->n_events;
    const int64_t s = sgl - Wp->seg_base;
    const int64_t n_seg = Wp->n_seg;
    const int32_t T = Wp->window_ps;
    const uint32_t bin_ps = (uint32_t)Wp->bin_ps, magic = Wp->bin_magic, shift = Wp->bin_shift;
    const int64_t s0 = s * SEG;
    const int n_rem = (int)min((int64_t)SEG, n_ev - s0);  // records in this segment
    const int j0 = lane * K;                                // first segment-local record of the lane
    const bool active = j0 < n_rem;

    // ---- stage the segment's records, transposed [k][lane], with 16-byte loads
    __syncwarp();
#pragma unroll
    for (int j = 0; j < K / 2; ++j) {
      const int r = 2 * (j * 32 + lane);
      uint2 a = make_uint2(0u, 0u), b = make_uint2(0u, 0u);
      if (r + 1 < n_rem) {
        const uint4 v = __ldcs(reinterpret_cast<const uint4*>(rec + s0 + r));
        a = make_uint2(v.x, v.y);
        b = make_uint2(v.z, v.w);
      } else if (r < n_rem) {
        a = rec[s0 + r];
      }
      rec_s[(r % K) * 32 + r / K] = a;
      rec_s[((r + 1) % K) * 32 + (r + 1) / K] = b;
    }
    const Seed sd = Wp->seeds[s];
    const bool has_next = s + 1 < n_seg;
    const int64_t g_lo = sd.gate;
    int64_t g_hi = G - 1;
    bool next_is_gs = false;
    if (has_next) {
      const Seed sn = Wp->seeds[s + 1];
      g_hi = sn.gate;
      next_is_gs = (sn.flags & kSeedGateStart) != 0;
    }
    uint32_t t_next_seg = 0u;  // first record after the segment, for the last lane's group-tail test
    if (lane == 31 && n_rem == SEG && s0 + SEG < n_ev) t_next_seg = rec[s0 + SEG].x;

    // ---- gate starts inside the segment, from one coalesced pass over its
    // CSR offsets: gid[k][lane] = the gate whose first record is (lane, k)
#pragma unroll
    for (int k = 0; k < K; ++k) gid_s[k * 32 + lane] = -1;
    __syncwarp();
    for (int64_t jg = g_lo + lane; jg <= g_hi; jg += 32) {
      const int64_t b = off[jg];
      if (b >= s0 && b < s0 + n_rem) {
        const int r = (int)(b - s0);
        atomicMax(&gid_s[(r % K) * 32 + r / K], (int)jg);  // empty gates share a start: the last one owns it
      }
    }
    __syncwarp();
    int lmax = -1;
#pragma unroll
    for (int k = 0; k < K; ++k) lmax = max(lmax, gid_s[k * 32 + lane]);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(kFull, lmax, o);
      if (lane >= o) lmax = max(lmax, u);
    }
    int g_before = __shfl_up_sync(kFull, lmax, 1);
    if (lane == 0) g_before = -1;
    const int g0 = (int)max((int64_t)g_before, g_lo);
    uint32_t t_before;
    if (lane > 0) t_before = rec_s[(K - 1) * 32 + lane - 1].x;
    else t_before = (sd.flags & kSeedGroupHead) ? (uint32_t)sd.t_prev : rec_s[0].x;

    // ---- pass 1: flags, per-record gate ids, the lane's state maps
    uint32_t gs_mask = 0u, gh_mask = 0u;
    uint32_t xk = 0xFFu, xs = 0u, pk = 0xFFu, ps = 0u, pm = 0u;
    {
      uint32_t tp = t_before;
      int gg = g0;
#pragma unroll 1
      for (int k = 0; k < K; ++k) {
        if (j0 + k >= n_rem) break;
        const uint2 r = rec_s[k * 32 + lane];
        const int gm = gid_s[k * 32 + lane];
        const bool is_gs = gm >= 0;
        const bool is_gh = is_gs || r.x != tp;
        if (is_gs) {
          gg = gm;
          xk = 0u;
          xs = init[gm];
        }
        gid_s[k * 32 + lane] = gg;
        if (is_gh) {
          pk = xk;
          ps = xs;
          pm = 1u;
        }
        const uint32_t bit = (1u << (r.y & 0xFu)) & 0xFFu;
        xk &= ~bit;
        xs = (xs & ~bit) | ((r.y & 0x10u) ? bit : 0u);
        gs_mask |= (is_gs ? 1u : 0u) << k;
        gh_mask |= (is_gh ? 1u : 0u) << k;
        tp = r.x;
      }
    }

    __syncwarp();  // pass 2 reads the next lane's gate ids

    // ---- gather every record's event descriptor in one burst of independent loads
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (j0 + k < n_rem) {
        const uint2 r = rec_s[k * 32 + lane];
        const uint32_t pin = min(r.y & 0xFu, (uint32_t)(dstride / 2 - 1));
        dsc_s[k * 32 + lane] = __ldg(desc + (size_t)gid_s[k * 32 + lane] * dstride + pin * 2u + ((r.y >> 4) & 1u));
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
    const uint32_t x_in = ((uint32_t)sd.x & (ea & 0xFFu)) | ((ea >> 8) & 0xFFu);
    const uint32_t p_in = eb ? (((uint32_t)sd.x & ((ea >> 16) & 0xFFu)) | (ea >> 24)) : (uint32_t)sd.p;

    // ---- pass 2: replay with energies (forward) or gradients (adjoint)
    float v0 = 0.f, v1 = 0.f, v2 = 0.f;  // forward: e_leak, e_int, e_sw; adjoint: dC, d_escale, d_lscale
    bool run_here = false, last_closed = false, has_head = false;
    float h0 = 0.f, h1 = 0.f, h2 = 0.f;
    int head_gate = 0;
    uint32_t st = x_in, spre = p_in;
    uint32_t pb = 0xFFFFFFFFu;
    float pe = 0.f, pdp = 0.f;
    int gg = g0;
    uint32_t cell = 0u;
    float Gcur = 0.f;  // adjoint: G(time of the current group)
    if (BWD && active && !(gs_mask & 1u)) {
      const uint32_t tb = t_before;
      if ((int32_t)tb >= 0 && (int32_t)tb < T) {
        const uint32_t bb = bin_of(tb, magic, shift, bin_ps);
        const float2 gv = Wp->grad[bb];
        Gcur = gv.y + gv.x * (float)(tb - bb * bin_ps);
      }
    }
    uint32_t tp = t_before;
#pragma unroll 1
    for (int k = 0; k < K; ++k) {
      const int jl = j0 + k;
      if (jl >= n_rem) break;
      const uint2 r = rec_s[k * 32 + lane];
      const uint4 d = dsc_s[k * 32 + lane];
      const bool is_gs = (gs_mask >> k) & 1u;
      const bool is_gh = (gh_mask >> k) & 1u;
      if (is_gs) {
        gg = gid_s[k * 32 + lane];
        st = init[gg];
        v0 = v1 = v2 = 0.f;
        run_here = true;
        Gcur = 0.f;
      }
      cell = (d.z >> 16) & 0xFFu;
      const CellInfo ci = sl.cells[cell];
      const uint32_t n_in = (uint32_t)ci.n_in;
      const uint32_t pmask = (2u << n_in) - 1u;
      const float* leak = sl.leak + ci.leak_base;
      const uint32_t t = r.x, meta = r.y;
      const uint32_t pin = meta & 0xFu, val = (meta >> 4) & 1u;
      const bool t_bad = (int32_t)t < 0 || (int32_t)t >= T;
      const bool o_bad = !is_gs && (int32_t)t < (int32_t)tp;
      const bool p_bad = (meta >> 5) != 0u || pin > n_in;
      const bool g_bad = !p_bad && ((st >> pin) & 1u) == val;
      const bool ok = !(t_bad || o_bad || p_bad || g_bad);
      if (!ok)
        report_error(err, t_bad ? GTP_ERANGE : (o_bad ? GTP_EORDER : (p_bad ? GTP_ERANGE : GTP_ENOTOGGLE)), s0 + jl);
      const uint32_t bn = ok ? bin_of(t, magic, shift, bin_ps) : 0u;
      float gE = 0.f, Gt = 0.f;
      if (BWD && ok) {
        const float2 gv = Wp->grad[bn];
        gE = gv.x;
        Gt = gv.y + gv.x * (float)(t - bn * bin_ps);
      }
      if (is_gh) {
        spre = st & pmask;
        if (ok) {
          if (BWD) {
            v2 += leak[spre] * (Gt - Gcur) * 1e-6f;
            Gcur = Gt;
          } else {
            v0 += leak[spre] * (float)((int32_t)t - (is_gs ? 0 : (int32_t)tp)) * 1e-6f;
          }
        }
      }
      // internal energy: the descriptor holds the table element of this (gate, pin, edge)
      // without the side bits; output events point at a valid table and take d.w instead
      const bool is_out = (d.z >> 24) & 1u;
      const uint32_t side = side_bits(spre & pmask, min(pin, n_in), n_in);
      const float* p = sl.tab + (d.z & 0xFFFFu) + side * (uint32_t)tsize;
      const float a0 = p[0], a1 = p[1], b0 = p[nl], b1 = p[nl + 1];
      const float da = a1 - a0, db = b1 - b0;
      const float lo = fmaf(__uint_as_float(d.y), da, a0);
      const float hi = fmaf(__uint_as_float(d.y), db, b0);
      const float e_in = fmaf(__uint_as_float(d.x), hi - lo, lo);
      float e = 0.f;
      if (BWD) {
        if (ok) {
          if (is_out) {
            v0 += gE * L.half_v2;
          } else {
            const float dB = fmaf(__uint_as_float(d.x), db - da, da) * __uint_as_float(d.w);
            v0 += gE * sl.escale[cell] * dB;
            v1 += gE * e_in;
          }
        }
      } else if (ok) {
        e = is_out ? __uint_as_float(d.w) : e_in;
        if (is_out) v2 += e; else v1 += e;
      }
      if (pin <= n_in) st = (st & ~(1u << pin)) | (val << pin);
      st &= pmask;
      // last record of its gate / of its timestamp group (from shared memory)
      bool gate_end, tail;
      if (s0 + jl + 1 >= n_ev) {  // last record of the window
        gate_end = tail = true;
      } else if (jl + 1 >= n_rem) {  // last record of the segment
        gate_end = next_is_gs;
        tail = gate_end || t_next_seg != t;
      } else if (k + 1 < K) {
        gate_end = ((gs_mask >> (k + 1)) & 1u) != 0u;
        tail = gate_end || rec_s[(k + 1) * 32 + lane].x != t;
      } else {  // the next record is the next lane's first
        gate_end = gid_s[lane + 1] != gg;
        tail = gate_end || rec_s[lane + 1].x != t;
      }
      if (!BWD && ok) {
        float add = 0.f, dp = 0.f;
        if (tail) {
          dp = leak[st] - leak[spre & pmask];
          add = dp * (float)((int32_t)((bn + 1u) * bin_ps) - (int32_t)t) * 1e-6f;
        }
        if (bn != pb) {
          if (pb != 0xFFFFFFFFu) red_bin(Wp->bins, pb, pe, pdp);
          pb = bn;
          pe = 0.f;
          pdp = 0.f;
        }
        pe += e + add;
        pdp += dp;
      }
      last_closed = gate_end;
      if (gate_end) {
        if (BWD) {
          v2 += leak[st] * (Wp->g_total - Gt) * 1e-6f;
          atomicAdd(wacc + cell, v1);
          atomicAdd(wacc + L.n_cells + cell, v2);
          if (run_here) {
            Wp->dC[gg] = v0;
          } else {
            has_head = true;
            head_gate = gg;
            h0 = v0;
          }
        } else {
          v0 += leak[st] * (float)(T - (int32_t)t) * 1e-6f;
          Wp->final_state[gg] = (uint8_t)st;
          if (run_here) {
            Wp->e_leak[gg] = (double)v0;
            Wp->e_int[gg] = (double)v1;
            Wp->e_sw[gg] = (double)v2;
          } else {
            has_head = true;
            head_gate = gg;
            h0 = v0;
            h1 = v1;
            h2 = v2;
          }
        }
        v0 = v1 = v2 = 0.f;
        run_here = false;
      }
      tp = t;
    }
    if (!BWD && pb != 0xFFFFFFFFu) red_bin(Wp->bins, pb, pe, pdp);

    // ---- per-gate sums of runs that cross lanes: segmented warp scan
    const bool open = active && !last_closed;
    if (BWD && open) {
      atomicAdd(wacc + cell, v1);
      atomicAdd(wacc + L.n_cells + cell, v2);
    }
    float c0 = open ? v0 : 0.f, c1 = open ? v1 : 0.f, c2 = open ? v2 : 0.f;
    uint32_t cf = (!open || run_here) ? 1u : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const float u0 = __shfl_up_sync(kFull, c0, o);
      const float u1 = NV > 1 ? __shfl_up_sync(kFull, c1, o) : 0.f;
      const float u2 = NV > 1 ? __shfl_up_sync(kFull, c2, o) : 0.f;
      const uint32_t uf = __shfl_up_sync(kFull, cf, o);
      if (lane >= o && !cf) {
        c0 += u0;
        c1 += u1;
        c2 += u2;
        cf = uf;
      }
    }
    const float q0 = __shfl_up_sync(kFull, c0, 1);
    const float q1 = NV > 1 ? __shfl_up_sync(kFull, c1, 1) : 0.f;
    const float q2 = NV > 1 ? __shfl_up_sync(kFull, c2, 1) : 0.f;
    const uint32_t qf = __shfl_up_sync(kFull, cf, 1);
    if (has_head) {
      const bool in_seg = lane > 0 && qf;
      if (BWD) {
        const float t0v = h0 + (lane > 0 ? q0 : 0.f);
        if (in_seg) Wp->dC[head_gate] = t0v;
        else atomicAdd(Wp->dC + head_gate, t0v);
      } else {
        const double a0 = (double)h0 + (lane > 0 ? (double)q0 : 0.0);
        const double a1 = (double)h1 + (lane > 0 ? (double)q1 : 0.0);
        const double a2 = (double)h2 + (lane > 0 ? (double)q2 : 0.0);
        if (in_seg) {
          Wp->e_leak[head_gate] = a0;
          Wp->e_int[head_gate] = a1;
          Wp->e_sw[head_gate] = a2;
        } else {
          atomicAdd(Wp->e_leak + head_gate, a0);
          atomicAdd(Wp->e_int + head_gate, a1);
          atomicAdd(Wp->e_sw + head_gate, a2);
        }
      }
    }
    if (lane == 31 && open) {
      if (BWD) {
        atomicAdd(Wp->dC + gg, c0);
      } else {
        atomicAdd(Wp->e_leak + gg, (double)c0);
        atomicAdd(Wp->e_int + gg, (double)c1);
        atomicAdd(Wp->e_sw + gg, (double)c2);
      }
    }
    if (BWD) {  // fold the warp's FP32 per-cell sums into its FP64 ones
      __syncwarp();
      for (int c = lane; c < nc2; c += 32) {
        wacc64[c] += (double)wacc[c];
        wacc[c] = 0.f;
      }
      __syncwarp();
    }
  }
  if (BWD) {
    __syncwarp();
    for (int c = lane; c < nc2; c += 32)
      if (wacc64[c] != 0.0) atomicAdd(cell_acc + c, wacc64[c]);
  }
}

template <int K, bool BWD>
size_t walk_smem(const LibView& L, int block, int n_win) {
  size_t b = smem_lib_bytes(L) + (((size_t)(n_win + 1) * 8 + 15) & ~(size_t)15) +
             (size_t)(block / 32) * 32 * K * (sizeof(uint4) + sizeof(uint2) + sizeof(int));
  if (BWD) b += (size_t)(block / 32) * 2 * L.n_cells * (sizeof(double) + sizeof(float));
  return b;
}

template <int K, bool BWD>
cudaError_t launch_k(const LibView& L, const NetView& N, const WalkArgs& A, cudaStream_t st) {
  const size_t smem = walk_smem<K, BWD>(L, A.block, A.n_win);
  cudaError_t e = cudaFuncSetAttribute(k_walk<K, BWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int grid = A.grid;
  if (grid <= 0) {
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_walk<K, BWD>, A.block, smem);
    if (e != cudaSuccess) return e;
    grid = (per_sm > 0 ? per_sm : 1) * A.n_sm;
  }
  const int64_t max_grid = (A.n_seg_total * 32 + A.block - 1) / A.block;
  if (grid > max_grid) grid = (int)max_grid;
  if (grid < 1) grid = 1;
  k_walk<K, BWD><<<grid, A.block, smem, st>>>(L, N, A.wins, A.seg_base, A.n_win, A.n_seg_total, A.err,
                                               A.cell_acc);
  return cudaGetLastError();
}

}  // namespace

bool walk_rpt_supported(int rpt) { return rpt == 4 || rpt == 8 || rpt == 16; }

cudaError_t launch_seeds(const NetView& N, const LibView& L, const WalkArgs& A, int64_t* runs, cudaStream_t st) {
  if (A.n_seg_total <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(runs, 0, sizeof(int64_t), st);
  if (e != cudaSuccess) return e;
  int64_t blocks = (N.n_gates + 255) / 256;
  if (blocks > 2048) blocks = 2048;
  k_seg_gates<<<dim3((unsigned)(blocks < 1 ? 1 : blocks), (unsigned)A.n_win), 256, 0, st>>>(N, A.wins, A.seg_len);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  blocks = (A.n_seg_total + 127) / 128;
  if (blocks > 16384) blocks = 16384;
  k_seed<<<(unsigned)blocks, 128, 0, st>>>(L, N, A.wins, A.seg_base, A.n_win, A.n_seg_total, A.seg_len, runs);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_seed_fix<<<64, 128, 0, st>>>(A.wins, A.seg_base, A.n_win, A.seg_len, runs);
  return cudaGetLastError();
}

cudaError_t launch_walk(const LibView& L, const NetView& N, const WalkArgs& A, bool backward, cudaStream_t st) {
  if (A.n_seg_total <= 0) return cudaSuccess;
  if (backward) {
    switch (A.rpt) {
      case 4: return launch_k<4, true>(L, N, A, st);
      case 16: return launch_k<16, true>(L, N, A, st);
      default: return launch_k<8, true>(L, N, A, st);
    }
  }
  switch (A.rpt) {
    case 4: return launch_k<4, false>(L, N, A, st);
    case 16: return launch_k<16, false>(L, N, A, st);
    default: return launch_k<8, false>(L, N, A, st);
  }
}

size_t walk_smem_bytes(const LibView& L, int rpt, int block, int n_win, bool backward) {
  switch (rpt) {
    case 4: return backward ? walk_smem<4, true>(L, block, n_win) : walk_smem<4, false>(L, block, n_win);
    case 16: return backward ? walk_smem<16, true>(L, block, n_win) : walk_smem<16, false>(L, block, n_win);
    default: return backward ? walk_smem<8, true>(L, block, n_win) : walk_smem<8, false>(L, block, n_win);
  }
}

}  // namespace gtp
