// GPU copy of the counter-based event generator in synth.c (same integer-only
// definition, same bits).  Used to materialise large synthetic traces
// directly in device memory.  It generates inputs only and holds none of the
// power arithmetic.
//
// Work is split into chunks of consecutive events of one gate.  Pass 1 writes
// timestamps and pins and the XOR of the chunk's pin toggles; the caller turns
// those into each chunk's starting state (an exclusive XOR scan per gate);
// pass 2 fills in the values (value = NOT current pin value).
#include <cstdint>
#include <cuda_runtime.h>

namespace {

__device__ __forceinline__ uint64_t mix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

__device__ __forceinline__ uint64_t key(uint64_t seed, uint64_t stream, uint64_t a, uint64_t b) {
  return mix64(mix64(mix64(seed ^ (stream << 56)) ^ a) ^ b);
}

constexpr uint64_t kStreamEvent = 1ull;

__device__ __forceinline__ int64_t base_time(uint64_t h, int64_t k, int64_t n, int64_t T) {
  uint64_t lo = ((uint64_t)k * (uint64_t)T) / (uint64_t)n;
  uint64_t hi = ((uint64_t)(k + 1) * (uint64_t)T) / (uint64_t)n;
  return (int64_t)(lo + (((h >> 32) * (hi - lo)) >> 32));
}

__device__ __forceinline__ bool is_tie(uint64_t h, int64_t k, uint32_t tie24) {
  return k > 0 && ((h >> 8) & 0xFFFFFFull) < (uint64_t)tie24;
}

// Timestamp of event j of gate g, following tie chains back to their start.
__device__ int64_t time_of(uint64_t seed, int64_t g, int64_t j, int64_t n, int64_t T, uint32_t tie24) {
  int64_t m = j;
  uint64_t h = key(seed, kStreamEvent, (uint64_t)g, (uint64_t)m);
  while (is_tie(h, m, tie24)) {
    --m;
    h = key(seed, kStreamEvent, (uint64_t)g, (uint64_t)m);
  }
  return base_time(h, m, n, T);
}

__global__ void gen_pass1(uint64_t seed, int64_t n_chunks, const int64_t* __restrict__ cg,
                          const int64_t* __restrict__ ck0, const int64_t* __restrict__ ck1,
                          const int64_t* __restrict__ offsets, const uint8_t* __restrict__ n_pins,
                          int64_t T, uint32_t tie24, uint32_t* __restrict__ rec,
                          uint8_t* __restrict__ chunk_mask) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_chunks) return;
  int64_t g = cg[c], k0 = ck0[c], k1 = ck1[c];
  int64_t base = offsets[g];
  int64_t n = offsets[g + 1] - base;
  uint32_t np_ = n_pins[g];
  int64_t t_prev = (k0 > 0) ? time_of(seed, g, k0 - 1, n, T, tie24) : 0;
  uint32_t mask = 0;
  for (int64_t k = k0; k < k1; ++k) {
    uint64_t h = key(seed, kStreamEvent, (uint64_t)g, (uint64_t)k);
    int64_t t = base_time(h, k, n, T);
    if (is_tie(h, k, tie24)) t = t_prev;
    uint32_t pin = (uint32_t)(((h & 0xFFFFull) * np_) >> 16);
    mask ^= (1u << pin);
    rec[2 * (base + k)] = (uint32_t)t;
    rec[2 * (base + k) + 1] = pin;
    t_prev = t;
  }
  chunk_mask[c] = (uint8_t)mask;
}

__global__ void gen_pass2(int64_t n_chunks, const int64_t* __restrict__ cg,
                          const int64_t* __restrict__ ck0, const int64_t* __restrict__ ck1,
                          const int64_t* __restrict__ offsets, const uint8_t* __restrict__ chunk_state,
                          uint32_t* __restrict__ rec) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_chunks) return;
  int64_t g = cg[c], k0 = ck0[c], k1 = ck1[c];
  int64_t base = offsets[g];
  uint32_t S = chunk_state[c];
  for (int64_t k = k0; k < k1; ++k) {
    uint32_t pin = rec[2 * (base + k) + 1] & 0xFu;
    uint32_t value = ((S >> pin) & 1u) ^ 1u;
    S ^= (1u << pin);
    rec[2 * (base + k) + 1] = pin | (value << 4);
  }
}

}  // namespace

extern "C" int synth_gpu_pass1(uint64_t seed, int64_t n_chunks, const int64_t* cg, const int64_t* ck0,
                               const int64_t* ck1, const int64_t* offsets, const uint8_t* n_pins,
                               int64_t window_ps, uint32_t tie24, uint32_t* records,
                               uint8_t* chunk_mask, void* stream) {
  if (n_chunks <= 0) return 0;
  int threads = 128;
  int64_t blocks = (n_chunks + threads - 1) / threads;
  gen_pass1<<<(unsigned)blocks, threads, 0, (cudaStream_t)stream>>>(
      seed, n_chunks, cg, ck0, ck1, offsets, n_pins, window_ps, tie24, records, chunk_mask);
  return (int)cudaGetLastError();
}

extern "C" int synth_gpu_pass2(int64_t n_chunks, const int64_t* cg, const int64_t* ck0, const int64_t* ck1,
                               const int64_t* offsets, const uint8_t* chunk_state, uint32_t* records,
                               void* stream) {
  if (n_chunks <= 0) return 0;
  int threads = 128;
  int64_t blocks = (n_chunks + threads - 1) / threads;
  gen_pass2<<<(unsigned)blocks, threads, 0, (cudaStream_t)stream>>>(n_chunks, cg, ck0, ck1, offsets,
                                                                     chunk_state, records);
  return (int)cudaGetLastError();
}
