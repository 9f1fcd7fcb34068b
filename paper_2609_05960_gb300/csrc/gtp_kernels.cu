// Gate pass, one-thread-per-gate walk, and the FP64 bin merge.
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

#include "gtp_internal.cuh"

namespace gtp {

// ------------------------------------------------------------------ gate pass
// Per gate: zero the energy accumulators, resolve gates without events
// (leakage at the initial state over the whole window), and reduce
// L0 = sum_g P_leak(cell_g, init_g) * lscale into O.l0.
__global__ void k_gate_pass(LibView L, NetView N, WindowView W, Outputs O, int64_t* counts) {
  double p0 = 0.0;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < N.n_gates;
       g += (int64_t)gridDim.x * blockDim.x) {
    int32_t c = N.cell[g];
    CellInfo ci = L.cells[c];
    uint32_t s0 = W.init[g];
    if (s0 >> (ci.n_in + 1)) {
      report_error(O.err, GTP_ERANGE, -1 - g);
      s0 &= (2u << ci.n_in) - 1u;
    }
    float P = L.leak[ci.leak_base + s0] * L.lscale[c];
    p0 += (double)P;
    int64_t cnt = W.offsets[g + 1] - W.offsets[g];
    if (counts) counts[g] = cnt;
    O.e_leak[g] = cnt == 0 ? (double)P * (double)W.window_ps * 1e-6 : 0.0;
    O.e_int[g] = 0.0;
    O.e_sw[g] = 0.0;
    O.final_state[g] = (uint8_t)s0;
  }
  // block reduction of p0
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) p0 += __shfl_down_sync(0xffffffffu, p0, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = p0;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) atomicAdd(O.l0, v);
  }
}

cudaError_t launch_gate_pass(const LibView& L, const NetView& N, const WindowView& W, const Outputs& O,
                             cudaStream_t st) {
  (void)0;
  int block = 256;
  int64_t blocks = (N.n_gates + block - 1) / block;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  k_gate_pass<<<(unsigned)blocks, block, 0, st>>>(L, N, W, O, nullptr);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ one thread per gate
// The plain walk of Algorithm 1, one gate per thread: timestamp groups with
// lookups at the pre-group state, the state update after the group, leakage
// held between groups.  Per-gate energies use Kahan-compensated FP32 sums.
__global__ void k_walk_per_gate(LibView L, NetView N, WindowView W, Outputs O) {
  extern __shared__ __align__(16) unsigned char smem[];
  SmemLib sl = stage_library(L, smem);
  const float T = (float)W.window_ps;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < N.n_gates;
       g += (int64_t)gridDim.x * blockDim.x) {
    int64_t a = W.offsets[g], b = W.offsets[g + 1];
    if (a == b) continue;
    int32_t c = N.cell[g];
    CellInfo ci = sl.cells[c];
    uint32_t n_in = (uint32_t)ci.n_in, n_pins = n_in + 1;
    const float* leak = sl.leak + ci.leak_base;
    const float* tabs = sl.tab + (size_t)ci.tab_base * L.tsize;
    uint32_t n_side = 1u << (n_in - 1);
    float C = N.load[g];
    const float* slew = N.slew + (size_t)g * N.stride * 2;
    uint32_t st = W.init[g] & ((2u << n_in) - 1u);
    float P = leak[st];
    int32_t t_prev = 0;
    Kahan El, Ei, Es;
    bool bad = false;
    int64_t i = a;
    while (i < b) {
      uint2 r0 = W.rec[i];
      int32_t t = (int32_t)r0.x;
      if (t < 0 || t >= W.window_ps) { report_error(O.err, GTP_ERANGE, i); bad = true; break; }
      if (t < t_prev) { report_error(O.err, GTP_EORDER, i); bad = true; break; }
      El.add(P * (float)(t - t_prev) * 1e-6f);
      uint32_t bin = bin_of(O, (uint32_t)t);
      uint32_t s_next = st;
      float e_bin = 0.f;
      int64_t j = i;
      for (; j < b; ++j) {
        uint2 r = W.rec[j];
        if ((int32_t)r.x != t) break;
        uint32_t pin = r.y & 0xFu, val = (r.y >> 4) & 1u;
        if ((r.y >> 5) != 0u || pin >= n_pins) { report_error(O.err, GTP_ERANGE, j); bad = true; break; }
        if (((s_next >> pin) & 1u) == val) { report_error(O.err, GTP_ENOTOGGLE, j); bad = true; break; }
        s_next ^= 1u << pin;
        float E;
        if (pin < n_in) {
          uint32_t side = side_bits(st, pin, n_in);
          const float* tb = tabs + (size_t)(((pin * 2u + val) * n_side) + side) * L.tsize;
          E = bilinear(L, sl, tb, slew[pin * 2 + val], C);
          Ei.add(E);
        } else {
          E = L.half_v2 * C;
          Es.add(E);
        }
        e_bin += E;
      }
      if (bad) break;
      float P_new = leak[s_next];
      float dP = P_new - P;
      float frac = (float)((int32_t)(bin + 1u) * O.bin_ps - t);
      red_bin(O.bins, bin, e_bin + dP * frac * 1e-6f, dP);
      st = s_next;
      P = P_new;
      t_prev = t;
      i = j;
    }
    if (bad) continue;
    El.add(P * (T - (float)t_prev) * 1e-6f);
    O.e_leak[g] = El.value();
    O.e_int[g] = Ei.value();
    O.e_sw[g] = Es.value();
    O.final_state[g] = (uint8_t)st;
  }
}

cudaError_t launch_walk_per_gate(const LibView& L, const NetView& N, const WindowView& W, const Outputs& O,
                                 int block, cudaStream_t st) {
  size_t smem = smem_lib_bytes(L);
  cudaError_t e = cudaFuncSetAttribute(k_walk_per_gate, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int64_t blocks = (N.n_gates + block - 1) / block;
  if (blocks > 65535) blocks = 65535;
  if (blocks < 1) blocks = 1;
  k_walk_per_gate<<<(unsigned)blocks, block, smem, st>>>(L, N, W, O);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ merge
// out[b] = (E[b] + bin_ps * 1e-6 * (L0 + sum_{b' < b} dP[b'])) * 1e-3 / bin_ps   (W)
constexpr int kMergeThreads = 256;
constexpr int kMergePer = 8;
constexpr int kMergeTile = kMergeThreads * kMergePer;

int merge_tiles(int n_bins) { return (n_bins + kMergeTile - 1) / kMergeTile; }

__device__ __forceinline__ double warp_incl_scan(double v) {
  int lane = threadIdx.x & 31;
  for (int o = 1; o < 32; o <<= 1) {
    double u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  return v;
}

// Block-wide exclusive scan of one double per thread; returns the exclusive
// prefix and writes the block total.
__device__ double block_excl_scan(double v, double* total) {
  __shared__ double warp_tot[32];
  double inc = warp_incl_scan(v);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 31) warp_tot[w] = inc;
  __syncthreads();
  if (w == 0) {
    int nw = blockDim.x >> 5;
    double x = lane < nw ? warp_tot[lane] : 0.0;
    double xi = warp_incl_scan(x);
    if (lane < nw) warp_tot[lane] = xi - x;
    if (lane == nw - 1) *total = xi;
  }
  __syncthreads();
  double r = inc - v + warp_tot[w];
  __syncthreads();
  return r;
}

__global__ void k_tile_sums(const float2* __restrict__ bins, int n_bins, double* __restrict__ tile_sums) {
  int tile = blockIdx.x;
  int base = tile * kMergeTile + threadIdx.x * kMergePer;
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kMergePer; ++k)
    if (base + k < n_bins) s += (double)bins[base + k].y;
  __shared__ double tot;
  block_excl_scan(s, &tot);
  if (threadIdx.x == 0) tile_sums[tile] = tot;
}

// Exclusive scan of tile sums in place (one block, sequential over chunks).
__global__ void k_scan_tiles(double* tile_sums, int n_tiles) {
  __shared__ double tot;
  double carry = 0.0;
  for (int base = 0; base < n_tiles; base += blockDim.x) {
    int i = base + threadIdx.x;
    double v = i < n_tiles ? tile_sums[i] : 0.0;
    double ex = block_excl_scan(v, &tot);
    if (i < n_tiles) tile_sums[i] = carry + ex;
    carry += tot;
    __syncthreads();
  }
}

__global__ void k_finalize(const float2* __restrict__ bins, int n_bins, const double* __restrict__ tile_pre,
                           const double* __restrict__ l0, int bin_ps, double* __restrict__ out) {
  int tile = blockIdx.x;
  int base = tile * kMergeTile + threadIdx.x * kMergePer;
  float2 v[kMergePer];
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kMergePer; ++k) {
    v[k] = base + k < n_bins ? bins[base + k] : make_float2(0.f, 0.f);
    s += (double)v[k].y;
  }
  __shared__ double tot;
  double pre = block_excl_scan(s, &tot) + tile_pre[tile] + *l0;
  const double dt = (double)bin_ps;
  const double to_w = 1e-3 / dt;
#pragma unroll
  for (int k = 0; k < kMergePer; ++k) {
    if (base + k < n_bins) out[base + k] = ((double)v[k].x + pre * dt * 1e-6) * to_w;
    pre += (double)v[k].y;
  }
}

cudaError_t launch_merge(const Outputs& O, double* waveform_w, double* tile_sums, int n_tiles, cudaStream_t st) {
  if (O.n_bins <= 0) return cudaSuccess;
  k_tile_sums<<<n_tiles, kMergeThreads, 0, st>>>(O.bins, O.n_bins, tile_sums);
  k_scan_tiles<<<1, 1024, 0, st>>>(tile_sums, n_tiles);
  k_finalize<<<n_tiles, kMergeThreads, 0, st>>>(O.bins, O.n_bins, tile_sums, O.l0, O.bin_ps, waveform_w);
  return cudaGetLastError();
}

size_t smem_lib_bytes(const LibView& L) {
  size_t b = sizeof(float) * 4 * kMaxAxis + (size_t)L.n_tables * L.tsize * 4 + (size_t)((L.n_leak + 3) & ~3) * 4 + (size_t)L.n_cells * sizeof(CellInfo);
  return (b + 15) & ~(size_t)15;
}

}  // namespace gtp
