// Segmented warp walk (the fused power kernel).
//
// The records of all gates form one flat, gate-major array (CSR by gate,
// time-ordered within a gate).  It is cut into equal segments of 32*K
// records; each warp owns one segment at a time (persistent grid), and each
// lane owns K consecutive records.  This balances work perfectly whatever the
// per-gate event skew: a sparse gate is walked inside one lane, a dense gate
// is cut into time slices across lanes and warps (the paper's per-gate
// temporal partitioning, Sec. 4.2, with equal event counts per slice instead
// of equal cycle counts).
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
// initial bit.  One warp per segment scans 32 records per step with ballots,
// usually resolving every pin in the first step.  A bounded scan that has not
// resolved every pin (a pin idle for a long time inside a very long gate)
// leaves the seed for a sequential fix-up pass that walks forward from the
// previous segment's seed, so the total fix-up cost stays linear.
//
// Energies (Sec. 2.2, Algorithm 1): internal energy of an input-pin event by
// the state-indexed table of (cell, pin, edge, side bits of the pre-group
// state), bilinear in (slew, load), scaled; 0.5*C*Vdd^2 for an output event.
// The library (scaled tables and leakage) is staged in shared memory.
//
// Leakage uses the step representation described in gtp_kernels.cu; per gate
// the leakage energy is the sum over groups of P(pre-group state) * (t - t of
// the previous group) plus P(final state) * (T - t_last).
//
// Bins are updated with one vector reduction {energy, leakage step} per
// distinct bin of a lane's consecutive records.  Per-gate sums are FP32 within
// a warp segment (lane-sequential, then a segmented warp scan) and FP64 across
// segments (atomic adds only for gates that cross a segment boundary).
#include <cstdio>

#include "gtp_segwalk.cuh"

namespace gtp {

namespace {

constexpr uint32_t kFull = 0xffffffffu;
constexpr int kSeedScanSegments = 4;  // backward seed scan bound, in segments

__device__ __forceinline__ int64_t gate_of(const int64_t* __restrict__ off, int64_t lo, int64_t hi, int64_t i) {
  // largest g in [lo, hi] with off[g] <= i (requires off[lo] <= i)
  while (lo < hi) {
    int64_t mid = (lo + hi + 1) >> 1;
    if (off[mid] <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// ------------------------------------------------------------------ seeds
__global__ void k_seed(LibView L, NetView N, WindowView W, int64_t seg_len, int64_t n_seg, Seed* __restrict__ seeds,
                       int64_t* __restrict__ runs) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t limit = seg_len * kSeedScanSegments;
  for (int64_t s = warp; s < n_seg; s += n_warps) {
    const int64_t s0 = s * seg_len;
    const int64_t g = gate_of(W.offsets, 0, N.n_gates - 1, s0);
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
      if (lane == 0) seeds[s] = sd;
      continue;
    }
    const int32_t t0 = (int32_t)W.rec[s0].x;
    // head of the timestamp group holding record s0
    int64_t h = s0;
    bool head_found = false;
    while (s0 - h < limit) {
      const int64_t q = h - 1 - lane;
      const bool eq = q >= gs && (int32_t)W.rec[q].x == t0;
      const uint32_t m = __ballot_sync(kFull, eq);
      const int run = (m == kFull) ? 32 : (__ffs(~m) - 1);
      h -= run;
      if (run < 32) {
        head_found = true;
        break;
      }
    }
    const uint32_t n_pins = (uint32_t)L.cells[N.cell[g]].n_in + 1u;
    const uint32_t full = (1u << n_pins) - 1u;
    uint32_t xres = 0, xval = 0, pres = 0, pval = 0;
    bool reached_start = false;
    if (head_found) {
      for (int64_t pos = s0 - 1;; pos -= 32) {
        if (pos < gs) {
          reached_start = true;
          break;
        }
        if ((xres & pres) == full || s0 - 1 - pos >= limit) break;
        const int64_t q = pos - lane;
        const bool valid = q >= gs;
        const uint32_t meta = valid ? W.rec[q].y : 0u;
        const uint32_t pin = meta & 0xFu, val = (meta >> 4) & 1u;
        for (uint32_t p = 0; p < n_pins; ++p) {
          const uint32_t mx = __ballot_sync(kFull, valid && pin == p);
          const uint32_t mp = __ballot_sync(kFull, valid && pin == p && q < h);
          if (mx && !((xres >> p) & 1u)) {
            const uint32_t v = __shfl_sync(kFull, val, __ffs(mx) - 1);
            xval |= v << p;
            xres |= 1u << p;
          }
          if (mp && !((pres >> p) & 1u)) {
            const uint32_t v = __shfl_sync(kFull, val, __ffs(mp) - 1);
            pval |= v << p;
            pres |= 1u << p;
          }
        }
      }
    }
    if (reached_start) {
      xval |= init & ~xres;
      pval |= init & ~pres;
      xres = pres = full;
    }
    const bool unresolved = !head_found || xres != full || pres != full;
    sd.t_prev = (head_found && h > gs) ? (int32_t)W.rec[h - 1].x : 0;
    sd.x = (uint8_t)xval;
    sd.p = (uint8_t)pval;
    sd.flags = (uint8_t)((head_found && h == s0 ? kSeedGroupHead : 0) | (unresolved ? kSeedUnresolved : 0));
    if (lane == 0) {
      seeds[s] = sd;
      if (unresolved) {
        const int64_t k = (int64_t)atomicAdd(reinterpret_cast<unsigned long long*>(runs), 1ull);
        runs[1 + k] = s;
      }
    }
  }
}

// Resolve seeds left partial by k_seed: the head of each chain of unresolved
// segments walks forward from the previous segment's (resolved) seed.
__global__ void k_seed_fix(WindowView W, int64_t seg_len, Seed* __restrict__ seeds, const int64_t* __restrict__ runs) {
  const int64_t n = runs[0];
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = runs[1 + u];
    if (s <= 0 || (seeds[s - 1].flags & kSeedUnresolved)) continue;  // not the head of its chain
    const Seed an = seeds[s - 1];
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
        if (!(seeds[s2].flags & kSeedUnresolved)) break;
        Seed r;
        r.gate = (int32_t)g;
        r.x = (uint8_t)X;
        r.p = (uint8_t)(head ? X : Pg);
        r.t_prev = head ? tcur : tp;
        // the unresolved bit stays set: other threads test it to find chain heads
        r.flags = (uint8_t)((head ? kSeedGroupHead : 0) | kSeedUnresolved);
        r.pad0 = 0;
        r.pad1 = 0;
        seeds[s2] = r;
      }
      if (head) {
        tp = tcur;
        tcur = ti;
        Pg = X;
      }
      const uint32_t meta = W.rec[i].y;
      const uint32_t pin = meta & 0xFu, val = (meta >> 4) & 1u;
      if (pin < 8u) X = (X & ~(1u << pin)) | (val << pin);
    }
  }
}

// ------------------------------------------------------------------ the walk
template <int K>
__global__ void __launch_bounds__(256) k_segwalk(LibView L, NetView N, WindowView W, Outputs O,
                                                 const Seed* __restrict__ seeds, int64_t n_seg) {
  extern __shared__ __align__(16) unsigned char smem[];
  const SmemLib sl = stage_library(L, smem);
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  constexpr int64_t SEG = 32 * K;
  const int64_t n_ev = W.n_events;
  const int64_t* __restrict__ off = W.offsets;
  const int32_t T = W.window_ps;

  for (int64_t s = warp; s < n_seg; s += n_warps) {
    const int64_t s0 = s * SEG;
    const int64_t i0 = s0 + (int64_t)lane * K;
    const bool active = i0 < n_ev;

    // ---- load K records (16-byte vector loads, evict-first)
    uint32_t tt[K], mm[K];
#pragma unroll
    for (int k = 0; k < K; k += 2) {
      const int64_t i = i0 + k;
      if (i + 1 < n_ev) {
        const uint4 v = __ldcs(reinterpret_cast<const uint4*>(W.rec + i));
        tt[k] = v.x;
        mm[k] = v.y;
        tt[k + 1] = v.z;
        mm[k + 1] = v.w;
      } else if (i < n_ev) {
        const uint2 v = W.rec[i];
        tt[k] = v.x;
        mm[k] = v.y;
        tt[k + 1] = 0u;
        mm[k + 1] = 0u;
      } else {
        tt[k] = tt[k + 1] = 0u;
        mm[k] = mm[k + 1] = 0u;
      }
    }

    const Seed sd = seeds[s];
    const int64_t g_hi = (s + 1 < n_seg) ? (int64_t)seeds[s + 1].gate : N.n_gates - 1;
    const int64_t g0 = active ? gate_of(off, sd.gate, g_hi, i0) : g_hi;
    const int64_t gstart0 = off[g0], gend0 = off[g0 + 1];

    // time of the record before my first one
    uint32_t t_before = __shfl_up_sync(kFull, tt[K - 1], 1);
    if (lane == 0) t_before = (sd.flags & kSeedGroupHead) ? (uint32_t)sd.t_prev : tt[0];

    // ---- pass 1: gate-start / group-head flags and the lane's state maps
    uint32_t gs_mask = 0u, gh_mask = 0u;
    uint32_t xk = 0xFFu, xs = 0u, pk = 0xFFu, ps = 0u, pm = 0u;
    {
      int64_t gg = g0, a = gstart0, b = gend0;
      uint32_t tp = t_before;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int64_t i = i0 + k;
        if (i < n_ev) {
          while (i >= b) {
            ++gg;
            a = b;
            b = off[gg + 1];
          }
          const bool is_gs = (i == a);
          const bool is_gh = is_gs || tt[k] != tp;
          if (is_gs) {
            xk = 0u;
            xs = W.init[gg];
          }
          if (is_gh) {
            pk = xk;
            ps = xs;
            pm = 1u;
          }
          const uint32_t pin = mm[k] & 0xFu, val = (mm[k] >> 4) & 1u;
          const uint32_t bit = (pin < 8u) ? (1u << pin) : 0u;
          xk &= ~bit;
          xs = (xs & ~bit) | (val ? bit : 0u);
          gs_mask |= (is_gs ? 1u : 0u) << k;
          gh_mask |= (is_gh ? 1u : 0u) << k;
        }
        tp = tt[k];
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
    const uint32_t next_gh = __shfl_down_sync(kFull, gh_mask & 1u, 1);

    // ---- pass 2: replay with energies, leakage and bins
    float el = 0.f, ei = 0.f, es = 0.f;
    bool run_here = false;       // current run began at a gate start in this lane
    bool last_closed = false;    // last processed record ended its gate
    bool has_head = false;       // first run continued from before and ended its gate here
    float h0 = 0.f, h1 = 0.f, h2 = 0.f;
    int64_t head_gate = 0;
    uint32_t st = x_in, spre = p_in;
    uint32_t pb = 0xFFFFFFFFu;
    float pe = 0.f, pdp = 0.f;
    int64_t gg = g0, b = gend0;
    int64_t loaded = -1;
    CellInfo ci{};
    const float* leak = sl.leak;
    const float* tabs = sl.tab;
    const float* slew = nullptr;
    float C = 0.f;
    uint32_t pmask = 0u;  // valid state bits of the current cell: leakage indices stay in its table
    uint32_t tp = t_before;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int64_t i = i0 + k;
      if (i < n_ev) {
        const bool is_gs = (gs_mask >> k) & 1u;
        const bool is_gh = (gh_mask >> k) & 1u;
        if (is_gs) {
          while (i >= b) {
            ++gg;
            b = off[gg + 1];
          }
          st = W.init[gg];
          el = ei = es = 0.f;
          run_here = true;
        }
        if (gg != loaded) {
          loaded = gg;
          ci = sl.cells[N.cell[gg]];
          leak = sl.leak + ci.leak_base;
          tabs = sl.tab + (size_t)ci.tab_base * L.tsize;
          slew = N.slew + (size_t)gg * N.stride * 2;
          C = N.load[gg];
          pmask = (2u << ci.n_in) - 1u;
        }
        const uint32_t n_in = (uint32_t)ci.n_in;
        const uint32_t t = tt[k], meta = mm[k];
        const uint32_t pin = meta & 0xFu, val = (meta >> 4) & 1u;
        bool ok = true;
        if ((int32_t)t < 0 || (int32_t)t >= T) {
          report_error(O.err, GTP_ERANGE, i);
          ok = false;
        } else if (!is_gs && (int32_t)t < (int32_t)tp) {
          report_error(O.err, GTP_EORDER, i);
          ok = false;
        }
        if ((meta >> 5) != 0u || pin > n_in) {
          report_error(O.err, GTP_ERANGE, i);
          ok = false;
        } else if (((st >> pin) & 1u) == val) {
          report_error(O.err, GTP_ENOTOGGLE, i);
          ok = false;
        }
        if (is_gh) {
          spre = st & pmask;
          if (ok) el += leak[spre] * (float)((int32_t)t - (is_gs ? 0 : (int32_t)tp)) * 1e-6f;
        }
        float e = 0.f;
        if (ok) {
          if (pin < n_in) {
            const uint32_t side = side_bits(spre & pmask, pin, n_in);
            const float* tb = tabs + (size_t)(((pin * 2u + val) << (n_in - 1u)) + side) * L.tsize;
            e = bilinear(L, sl, tb, slew[pin * 2u + val], C);
            ei += e;
          } else {
            e = L.half_v2 * C;
            es += e;
          }
        }
        if (pin <= n_in) st = (st & ~(1u << pin)) | (val << pin);
        st &= pmask;
        bool tail;
        if (i + 1 >= n_ev || i + 1 >= b) tail = true;
        else if (k + 1 < K) tail = (gh_mask >> (k + 1)) & 1u;
        else if (lane < 31) tail = next_gh != 0u;
        else tail = (int32_t)W.rec[i + 1].x != (int32_t)t;
        if (ok) {
          const uint32_t bn = bin_of(O, t);
          float add = 0.f, dp = 0.f;
          if (tail) {
            dp = leak[st] - leak[spre & pmask];
            add = dp * (float)((int32_t)(bn + 1u) * O.bin_ps - (int32_t)t) * 1e-6f;
          }
          if (bn != pb) {
            if (pb != 0xFFFFFFFFu) red_bin(O.bins, pb, pe, pdp);
            pb = bn;
            pe = 0.f;
            pdp = 0.f;
          }
          pe += e + add;
          pdp += dp;
        }
        last_closed = (i + 1 == b);
        if (last_closed) {
          el += leak[st] * (float)(T - (int32_t)t) * 1e-6f;
          O.final_state[gg] = (uint8_t)st;
          if (run_here) {
            O.e_leak[gg] = (double)el;
            O.e_int[gg] = (double)ei;
            O.e_sw[gg] = (double)es;
          } else {
            has_head = true;
            head_gate = gg;
            h0 = el;
            h1 = ei;
            h2 = es;
          }
          el = ei = es = 0.f;
          run_here = false;
        }
        tp = t;
      }
    }
    if (pb != 0xFFFFFFFFu) red_bin(O.bins, pb, pe, pdp);

    // ---- per-gate sums of runs that cross lanes: segmented warp scan
    const bool open = active && !last_closed;
    float c0 = open ? el : 0.f, c1 = open ? ei : 0.f, c2 = open ? es : 0.f;
    uint32_t cf = (!open || run_here) ? 1u : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const float u0 = __shfl_up_sync(kFull, c0, o);
      const float u1 = __shfl_up_sync(kFull, c1, o);
      const float u2 = __shfl_up_sync(kFull, c2, o);
      const uint32_t uf = __shfl_up_sync(kFull, cf, o);
      if (lane >= o && !cf) {
        c0 += u0;
        c1 += u1;
        c2 += u2;
        cf = uf;
      }
    }
    const float q0 = __shfl_up_sync(kFull, c0, 1);
    const float q1 = __shfl_up_sync(kFull, c1, 1);
    const float q2 = __shfl_up_sync(kFull, c2, 1);
    const uint32_t qf = __shfl_up_sync(kFull, cf, 1);
    if (has_head) {
      const bool in_seg = lane > 0 && qf;
      const double v0 = (double)h0 + (lane > 0 ? (double)q0 : 0.0);
      const double v1 = (double)h1 + (lane > 0 ? (double)q1 : 0.0);
      const double v2 = (double)h2 + (lane > 0 ? (double)q2 : 0.0);
      if (in_seg) {
        O.e_leak[head_gate] = v0;
        O.e_int[head_gate] = v1;
        O.e_sw[head_gate] = v2;
      } else {
        atomicAdd(O.e_leak + head_gate, v0);
        atomicAdd(O.e_int + head_gate, v1);
        atomicAdd(O.e_sw + head_gate, v2);
      }
    }
    if (lane == 31 && open) {
      atomicAdd(O.e_leak + gg, (double)c0);
      atomicAdd(O.e_int + gg, (double)c1);
      atomicAdd(O.e_sw + gg, (double)c2);
    }
  }
}

template <int K>
cudaError_t launch_k(const LibView& L, const NetView& N, const WindowView& W, const Outputs& O, const SegPlan& P,
                     const Seed* seeds, cudaStream_t st) {
  const size_t smem = smem_lib_bytes(L);
  cudaError_t e = cudaFuncSetAttribute(k_segwalk<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int grid = P.grid;
  if (grid <= 0) {
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_segwalk<K>, P.block, smem);
    if (e != cudaSuccess) return e;
    int dev = 0, n_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    grid = (per_sm > 0 ? per_sm : 1) * n_sm;
  }
  const int64_t warps_needed = P.n_seg;
  const int64_t max_grid = (warps_needed * 32 + P.block - 1) / P.block;
  if (grid > max_grid) grid = (int)max_grid;
  if (grid < 1) grid = 1;
  k_segwalk<K><<<grid, P.block, smem, st>>>(L, N, W, O, seeds, P.n_seg);
  return cudaGetLastError();
}

}  // namespace

bool seg_rpt_supported(int rpt) { return rpt == 4 || rpt == 8 || rpt == 16; }

SegPlan make_seg_plan(int rpt, int block, int ctas_per_sm, int n_sm, int64_t n_events) {
  SegPlan P{};
  P.rpt = seg_rpt_supported(rpt) ? rpt : 8;
  P.block = (block == 128 || block == 256) ? block : 256;
  P.grid = ctas_per_sm > 0 ? ctas_per_sm * n_sm : 0;
  P.seg_len = 32ll * P.rpt;
  P.n_seg = (n_events + P.seg_len - 1) / P.seg_len;
  return P;
}

cudaError_t launch_seeds(const LibView& L, const NetView& N, const WindowView& W, const SegPlan& P, Seed* seeds,
                         int64_t* runs, cudaStream_t st) {
  if (P.n_seg <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(runs, 0, sizeof(int64_t), st);
  if (e != cudaSuccess) return e;
  {
    const int block = 256;
    int64_t blocks = (P.n_seg * 32 + block - 1) / block;
    if (blocks > 8192) blocks = 8192;
    k_seed<<<(unsigned)blocks, block, 0, st>>>(L, N, W, P.seg_len, P.n_seg, seeds, runs);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  k_seed_fix<<<64, 128, 0, st>>>(W, P.seg_len, seeds, runs);
  return cudaGetLastError();
}

cudaError_t launch_walk(const LibView& L, const NetView& N, const WindowView& W, const Outputs& O, const SegPlan& P,
                        const Seed* seeds, cudaStream_t st) {
  if (P.n_seg <= 0) return cudaSuccess;
  switch (P.rpt) {
    case 4: return launch_k<4>(L, N, W, O, P, seeds, st);
    case 16: return launch_k<16>(L, N, W, O, P, seeds, st);
    default: return launch_k<8>(L, N, W, O, P, seeds, st);
  }
}

}  // namespace gtp
