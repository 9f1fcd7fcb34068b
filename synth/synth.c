/*
 * Seeded synthetic inputs for the gate-level power walk: a counter-based
 * generator of per-gate event streams.
 *
 * This file generates INPUTS only (library tables, netlist parameters and
 * event traces are drawn elsewhere in numpy; the event streams are drawn
 * here).  It holds none of the power arithmetic.  The GPU copy in
 * synth_gpu.cu implements the same integer-only definition and must produce
 * the same bits; both follow the definition below.
 *
 * Definition (all arithmetic on unsigned 64-bit integers, wrapping):
 *   mix(x)        = SplitMix64 finaliser of (x + 0x9E3779B97F4A7C15)
 *   key(s,st,a,b) = mix(mix(mix(s ^ (st << 56)) ^ a) ^ b)
 * For gate g with n events over a window of T ps, event k (0 <= k < n):
 *   h   = key(seed, STREAM_EVENT, g, k)
 *   lo  = floor(k*T/n), hi = floor((k+1)*T/n)
 *   t_k = lo + (((h >> 32) * (hi - lo)) >> 32)                (so lo <= t_k < hi, or t_k = lo if hi == lo)
 *   tie: if k > 0 and ((h >> 8) & 0xFFFFFF) < tie24 then t_k = t_{k-1}
 *   pin = ((h & 0xFFFF) * n_pins) >> 16
 *   value = NOT(current value of pin); the pin's bit in the running state flips.
 * Records are two 32-bit words {t_ps, meta} with meta = pin | value << 4.
 * The initial state of gate g is key(seed, STREAM_INIT, g, 0) masked to its pins.
 */
#include <stdint.h>
#include <stddef.h>
#include <pthread.h>

#define STREAM_EVENT 1ull
#define STREAM_INIT 2ull

static inline uint64_t mix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

uint64_t synth_key(uint64_t seed, uint64_t stream, uint64_t a, uint64_t b) {
  return mix64(mix64(mix64(seed ^ (stream << 56)) ^ a) ^ b);
}

/* Vectorised key for numpy callers: out[i] = key(seed, stream, a0 + i, b). */
void synth_keys(uint64_t seed, uint64_t stream, uint64_t a0, uint64_t b, int64_t n, uint64_t* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = synth_key(seed, stream, a0 + (uint64_t)i, b);
}

void synth_init_state(uint64_t seed, int64_t n_gates, const uint8_t* n_pins, uint8_t* init_out) {
  for (int64_t g = 0; g < n_gates; ++g) {
    uint64_t h = synth_key(seed, STREAM_INIT, (uint64_t)g, 0);
    init_out[g] = (uint8_t)(h & ((1u << n_pins[g]) - 1u));
  }
}

static void gen_gate(uint64_t seed, int64_t g, int64_t n, int64_t T, uint32_t np_, uint8_t init,
                     uint32_t tie24, uint32_t* rec) {
  uint32_t S = init;
  int64_t t_prev = 0;
  for (int64_t k = 0; k < n; ++k) {
    uint64_t h = synth_key(seed, STREAM_EVENT, (uint64_t)g, (uint64_t)k);
    uint64_t lo = ((uint64_t)k * (uint64_t)T) / (uint64_t)n;
    uint64_t hi = ((uint64_t)(k + 1) * (uint64_t)T) / (uint64_t)n;
    int64_t t = (int64_t)(lo + (((h >> 32) * (hi - lo)) >> 32));
    if (k > 0 && ((h >> 8) & 0xFFFFFFull) < (uint64_t)tie24) t = t_prev;
    uint32_t pin = (uint32_t)(((h & 0xFFFFull) * np_) >> 16);
    uint32_t value = ((S >> pin) & 1u) ^ 1u;
    S ^= (1u << pin);
    rec[2 * k] = (uint32_t)t;
    rec[2 * k + 1] = pin | (value << 4);
    t_prev = t;
  }
}

typedef struct {
  uint64_t seed;
  int64_t g0, g1;
  const int64_t* offsets;
  const uint8_t* n_pins;
  const uint8_t* init;
  int64_t T;
  uint32_t tie24;
  uint32_t* records;
} job_t;

static void* run_job(void* p) {
  job_t* j = (job_t*)p;
  for (int64_t g = j->g0; g < j->g1; ++g) {
    int64_t a = j->offsets[g], b = j->offsets[g + 1];
    gen_gate(j->seed, g, b - a, j->T, j->n_pins[g], j->init[g], j->tie24, j->records + 2 * a);
  }
  return NULL;
}

/* Generate the records of gates [0, n_gates) into records[2*offsets[0] ...].
 * Gates are split over n_threads host threads by event count. */
int synth_events(uint64_t seed, int64_t n_gates, const int64_t* offsets, const uint8_t* n_pins,
                 const uint8_t* init, int64_t window_ps, uint32_t tie24, uint32_t* records,
                 int n_threads) {
  if (n_threads < 1) n_threads = 1;
  if (n_threads > 256) n_threads = 256;
  job_t jobs[256];
  pthread_t th[256];
  int64_t total = offsets[n_gates] - offsets[0];
  int64_t g = 0;
  int used = 0;
  for (int i = 0; i < n_threads && g < n_gates; ++i) {
    int64_t target = offsets[0] + (total * (i + 1)) / n_threads;
    int64_t g1 = g;
    while (g1 < n_gates && (offsets[g1 + 1] <= target || g1 == g)) ++g1;
    if (i == n_threads - 1) g1 = n_gates;
    jobs[i] = (job_t){seed, g, g1, offsets, n_pins, init, window_ps, tie24, records};
    g = g1;
    used = i + 1;
  }
  for (int i = 1; i < used; ++i) pthread_create(&th[i], NULL, run_job, &jobs[i]);
  if (used > 0) run_job(&jobs[0]);
  for (int i = 1; i < used; ++i) pthread_join(th[i], NULL);
  return 0;
}

/* Generate the records of a list of gates into a compact buffer: the records
 * of gate gates[i] land at out[2*out_offsets[i] ...]. Used to regenerate the
 * streams of sampled gates without materialising a whole trace. */
int synth_events_subset(uint64_t seed, int64_t n_sel, const int64_t* gates, const int64_t* counts,
                        const uint8_t* n_pins, const uint8_t* init, int64_t window_ps,
                        uint32_t tie24, const int64_t* out_offsets, uint32_t* out) {
  for (int64_t i = 0; i < n_sel; ++i)
    gen_gate(seed, gates[i], counts[i], window_ps, n_pins[i], init[i], tie24, out + 2 * out_offsets[i]);
  return 0;
}
