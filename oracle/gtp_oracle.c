/*
 * FP64 reference oracle for gate-level time-based power analysis.
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, single-threaded CPU
 * statement of what the GPU engine computes.  Only the test suite, the smoke
 * check and the benchmark's CPU baseline call it; the GPU engine never does.
 * It shares no code with the engine.
 *
 * What it computes (paper section / equation in brackets):
 *   * An event is (value, timestamp) on one pin of one gate; the gate state is
 *     the vector of all pin values, changed by each event [Sec. 2.1].
 *   * Events of a gate are processed in time order; all events sharing one
 *     timestamp form a group.  Lookups for every event of the group use the
 *     state held before the group; the state is updated after the whole group
 *     [Algorithm 1, the timestamp loop].
 *   * Internal energy of an input-pin event: the state-dependent NLDM table
 *     selected by (cell, pin, edge, side-input bits of the pre-group state),
 *     interpolated bilinearly at (input slew, output load), times the cell's
 *     energy scale [Sec. 2.2; Sec. 4.1 state-indexed lookup].
 *   * Switching energy of an output-pin event: 0.5*C*Vdd^2 per output toggle
 *     [Eq. 1, read as half of c*v^2 per toggle].
 *   * Leakage: the state-dependent leakage power holds between events; the
 *     energy of an interval is P*dt [Eq. 4], and each interval
 *     is split over the time bins it overlaps in proportion to the overlap
 *     [Sec. 2.4.2, waveform accumulation].
 *   * Dynamic energy goes to the bin containing the event time.
 *   * Glitches (optional, with a clock period T_clk): an event on a pin that
 *     already had an event earlier in the same clock cycle floor(t / T_clk)
 *     is a glitch event [Sec. 2.4.1, clock-cycle glitch detection;
 *     Algorithm 1, GlitchDetectUpdate].  Its dynamic energy is scaled by
 *     r_gl = min(1, (2 * pulse_width / (rSlew + fSlew))^2) [Eq. 2], with
 *     pulse_width the time since that pin's previous
 *     event and rSlew, fSlew the pin's rise and fall transition times; the
 *     scaled energy is glitch energy (not internal or switching energy) and
 *     goes to the event's bin.
 * Units: ps, fF, V, fJ, nW.  E[fJ] = P[nW] * dt[ps] * 1e-6; 0.5*C[fF]*V^2 = fJ.
 *
 * Parity status: the walk and the adjoint are pinned by closed forms, a
 * per-picosecond brute-force simulator, library interpolation and invariants
 * (tests/test_oracle_*.py); glitch detection by a hand-worked trace, closed
 * forms, the brute-force simulator's per-cycle pin counters and central
 * differences (tests/test_oracle_glitch.py).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_EINVAL (-1)
#define OR_EORDER (-2)
#define OR_ERANGE (-3)
#define OR_ENOTOGGLE (-4)

typedef struct {
  int32_t n_cells;
  const int32_t* n_in;      /* [n_cells] input pins; output pin index = n_in */
  double vdd;               /* V */
  int32_t n_slew;
  const float* slew_axis;   /* [n_slew] ps, increasing */
  int32_t n_load;
  const float* load_axis;   /* [n_load] fF, increasing */
  const float* e_int;       /* flat tables, fJ */
  const float* p_leak;      /* flat leakage, nW */
  const double* escale;     /* [n_cells] */
  const double* lscale;     /* [n_cells] */
} oracle_lib;

typedef struct {
  int64_t n_gates;
  const int32_t* cell;      /* [n_gates] */
  const double* load_ff;    /* [n_gates] */
  const float* slew_ps;     /* [n_gates][slew_stride][2] */
  int32_t slew_stride;
} oracle_net;

typedef struct {
  int64_t clock_ps;         /* > 0: clock period for glitch detection */
  const float* out_slew_ps; /* [n_gates][2] output-pin {fall, rise} transition times */
} oracle_glitch;

typedef struct {
  int64_t window_ps;
  const int64_t* offsets;   /* [n_gates + 1] */
  const uint32_t* records;  /* [n_events][2] = {t_ps, meta} */
  const uint8_t* init_state;/* [n_gates] */
} oracle_trace;

/* ---------------------------------------------------------------- lookup */

/* Segment of an interpolation axis: the lower knot index i with
 * axis[i] <= x < axis[i+1], clamped to [0, n-2] so that points outside the
 * axis extrapolate linearly from the edge segment. */
static int32_t segment_of(const float* axis, int32_t n, double x) {
  int32_t i = 0;
  while (i < n - 2 && x >= (double)axis[i + 1]) ++i;
  return i;
}

/* Bilinear interpolation of one n_slew x n_load table (slew-major). */
double oracle_bilinear(int32_t n_slew, const float* slew_axis, int32_t n_load, const float* load_axis,
                       const float* table, double slew, double load) {
  int32_t i = segment_of(slew_axis, n_slew, slew);
  int32_t j = segment_of(load_axis, n_load, load);
  double fs = (slew - slew_axis[i]) / ((double)slew_axis[i + 1] - slew_axis[i]);
  double fl = (load - load_axis[j]) / ((double)load_axis[j + 1] - load_axis[j]);
  double t00 = table[i * n_load + j], t01 = table[i * n_load + j + 1];
  double t10 = table[(i + 1) * n_load + j], t11 = table[(i + 1) * n_load + j + 1];
  return (1.0 - fs) * (1.0 - fl) * t00 + (1.0 - fs) * fl * t01 + fs * (1.0 - fl) * t10 + fs * fl * t11;
}

/* Partial derivative of the bilinear interpolant with respect to the load,
 * on the located load segment (right derivative at a knot). */
double oracle_bilinear_dload(int32_t n_slew, const float* slew_axis, int32_t n_load, const float* load_axis,
                             const float* table, double slew, double load) {
  int32_t i = segment_of(slew_axis, n_slew, slew);
  int32_t j = segment_of(load_axis, n_load, load);
  double fs = (slew - slew_axis[i]) / ((double)slew_axis[i + 1] - slew_axis[i]);
  double w = (double)load_axis[j + 1] - load_axis[j];
  double t00 = table[i * n_load + j], t01 = table[i * n_load + j + 1];
  double t10 = table[(i + 1) * n_load + j], t11 = table[(i + 1) * n_load + j + 1];
  return ((1.0 - fs) * (t01 - t00) + fs * (t11 - t10)) / w;
}

/* Side-input state: the input-pin bits of S other than `pin`, compacted in
 * pin order (state-indexed lookup, Sec. 4.1). */
static uint32_t side_bits(uint32_t S, int32_t pin, int32_t n_in) {
  uint32_t side = 0;
  int32_t pos = 0;
  for (int32_t p = 0; p < n_in; ++p) {
    if (p == pin) continue;
    side |= ((S >> p) & 1u) << pos;
    ++pos;
  }
  return side;
}

/* Start of cell c's tables (in tables) and of its leakage entries. */
static void cell_bases(const oracle_lib* L, int64_t* tab_base, int64_t* leak_base) {
  int64_t t = 0, l = 0;
  for (int32_t c = 0; c < L->n_cells; ++c) {
    tab_base[c] = t;
    leak_base[c] = l;
    t += (int64_t)L->n_in[c] * 2 * (1ll << (L->n_in[c] - 1));
    l += 1ll << (L->n_in[c] + 1);
  }
}

static const float* table_for(const oracle_lib* L, const int64_t* tab_base, int32_t c, int32_t pin,
                              int32_t edge, uint32_t side) {
  int64_t n_side = 1ll << (L->n_in[c] - 1);
  int64_t idx = tab_base[c] + ((int64_t)(pin * 2 + edge) * n_side + side);
  return L->e_int + idx * (int64_t)L->n_slew * L->n_load;
}

/* ---------------------------------------------------------------- binning */

typedef struct {
  int64_t bin_ps;
  int64_t n_bins;
  double* out;              /* all bins, or the sampled bins */
  int64_t n_sample;         /* 0 = all bins */
  const int64_t* sample;    /* sorted bin indices */
  double* diff;             /* range mode only: [n_bins + 1] differences of the
                               whole-bin leakage shares (see bin_add_interval) */
} binner;

static int64_t first_sample_at_or_after(const binner* B, int64_t b) {
  int64_t lo = 0, hi = B->n_sample;
  while (lo < hi) {
    int64_t mid = (lo + hi) / 2;
    if (B->sample[mid] < b) lo = mid + 1; else hi = mid;
  }
  return lo;
}

static void bin_add(const binner* B, int64_t t, double e) {
  if (!B->out) return;
  int64_t b = t / B->bin_ps;
  if (B->n_sample == 0) { B->out[b] += e; return; }
  int64_t k = first_sample_at_or_after(B, b);
  if (k < B->n_sample && B->sample[k] == b) B->out[k] += e;
}

/* Leakage of power P (nW) over [a, b) ps, split over the overlapped bins
 * [Sec. 2.4.2]: each bin receives P times its overlap with the interval.
 *
 * Range mode (B->diff set, all bins): the same split, with the bins the
 * interval covers whole (every bin strictly between the first and the last
 * one) receiving their equal share P * bin_ps through a difference array,
 * diff[k0 + 1] += share, diff[k1] -= share, which range_flush() turns into
 * the per-bin amounts with one running sum.  Only the order of the FP64
 * additions differs from the plain split; this mode exists so that the
 * oracle can check full-size waveforms, where the plain split costs
 * gates x bins additions. */
static void bin_add_interval(const binner* B, double P, int64_t a, int64_t b) {
  if (!B->out || b <= a) return;
  int64_t k0 = a / B->bin_ps, k1 = (b - 1) / B->bin_ps;
  if (B->diff && B->n_sample == 0) {
    if (k0 == k1) {
      B->out[k0] += P * (double)(b - a) * 1e-6;
      return;
    }
    B->out[k0] += P * (double)((k0 + 1) * B->bin_ps - a) * 1e-6;
    B->out[k1] += P * (double)(b - k1 * B->bin_ps) * 1e-6;
    if (k1 > k0 + 1) {
      double share = P * (double)B->bin_ps * 1e-6;
      B->diff[k0 + 1] += share;
      B->diff[k1] -= share;
    }
    return;
  }
  if (B->n_sample == 0) {
    for (int64_t k = k0; k <= k1; ++k) {
      int64_t lo = a > k * B->bin_ps ? a : k * B->bin_ps;
      int64_t hi = b < (k + 1) * B->bin_ps ? b : (k + 1) * B->bin_ps;
      B->out[k] += P * (double)(hi - lo) * 1e-6;
    }
    return;
  }
  for (int64_t s = first_sample_at_or_after(B, k0); s < B->n_sample && B->sample[s] <= k1; ++s) {
    int64_t k = B->sample[s];
    int64_t lo = a > k * B->bin_ps ? a : k * B->bin_ps;
    int64_t hi = b < (k + 1) * B->bin_ps ? b : (k + 1) * B->bin_ps;
    B->out[s] += P * (double)(hi - lo) * 1e-6;
  }
}

/* Range mode: add the whole-bin leakage shares recorded in B->diff to the
 * bins (a running sum of the differences) and clear the differences. */
static void range_flush(const binner* B) {
  if (!B->diff || !B->out) return;
  double run = 0.0;
  for (int64_t k = 0; k < B->n_bins; ++k) {
    run += B->diff[k];
    B->out[k] += run;
    B->diff[k] = 0.0;
  }
  B->diff[B->n_bins] = 0.0;
}

/* ---------------------------------------------------------------- the walk */

/*
 * Walk every selected gate.  gates == NULL selects all; otherwise gates[i]
 * (i < n_sel) names gate indices and the per-gate outputs are written at
 * position i.  bins: all n_bins bins (sample == NULL) or the n_sample sorted
 * bins in `sample`; NULL skips the waveform.  Per-gate outputs may be NULL.
 * On a malformed trace returns a negative code and the offending record
 * index in *bad_record.
 * comp_bins (optional) receives the same bins split by component, as four
 * consecutive rows of the bins' length: leakage, internal, switching and
 * glitch energy (Sec. 2.2: the power components; their sum is `bins`).
 */
/* Glitch scaling ratio of an event pulse_width ps after the previous event on
 * its pin, for rise + fall transition time sum_slew ps [Eq. 2]; a pin without transition time (sum <= 0) swings fully: ratio 1. */
static double glitch_ratio(double pulse_width, double sum_slew) {
  if (sum_slew <= 0.0) return 1.0;
  double x = 2.0 * pulse_width / sum_slew;
  double r = x * x;
  return r < 1.0 ? r : 1.0;
}

static int walk_impl(const oracle_lib* L, const oracle_net* N, const oracle_trace* T, int64_t bin_ps,
                     int64_t n_sel, const int64_t* gates,
                     double* bins, int64_t n_sample, const int64_t* sample,
                     double* e_leak, double* e_int, double* e_sw, int64_t* n_events, uint8_t* final_state,
                     int64_t* bad_record, const oracle_glitch* GL, double* e_gl, double* comp_bins,
                     int leak_range) {
  if (bin_ps <= 0 || T->window_ps <= 0 || T->window_ps % bin_ps != 0) return OR_EINVAL;
  int64_t n_bins_all = T->window_ps / bin_ps;
  int ranged = leak_range && n_sample == 0;
  int64_t* tab_base = (int64_t*)malloc(sizeof(int64_t) * (size_t)L->n_cells);
  int64_t* leak_base = (int64_t*)malloc(sizeof(int64_t) * (size_t)L->n_cells);
  double* diff = ranged ? (double*)calloc((size_t)(n_bins_all + 1), sizeof(double)) : NULL;
  double* cdiff = ranged && comp_bins ? (double*)calloc((size_t)(n_bins_all + 1), sizeof(double)) : NULL;
  cell_bases(L, tab_base, leak_base);
  binner B = {bin_ps, n_bins_all, bins, n_sample, sample, diff};
  int64_t n_out = n_sample ? n_sample : n_bins_all;
  binner BC[4]; /* leakage, internal, switching, glitch */
  for (int k = 0; k < 4; ++k) {
    binner x = {bin_ps, n_bins_all, comp_bins ? comp_bins + k * n_out : NULL, n_sample, sample,
                k == 0 ? cdiff : NULL};
    BC[k] = x;
  }
  int64_t count = gates ? n_sel : N->n_gates;
  int rc = OR_OK;
  double half_v2 = 0.5 * L->vdd * L->vdd;
  for (int64_t gi = 0; gi < count && rc == OR_OK; ++gi) {
    int64_t g = gates ? gates[gi] : gi;
    int32_t c = N->cell[g];
    int32_t n_in = L->n_in[c];
    int32_t n_pins = n_in + 1;
    double C = N->load_ff[g];
    double ls = L->lscale[c], es = L->escale[c];
    const float* leak = L->p_leak + leak_base[c];
    uint32_t S = T->init_state[g];
    int64_t t_prev = 0;
    double El = 0.0, Ei = 0.0, Es = 0.0, Eg = 0.0;
    int64_t last_t[16];  /* each pin's previous event time, -1 before its first */
    for (int p = 0; p < 16; ++p) last_t[p] = -1;
    int64_t a = T->offsets[g], b = T->offsets[g + 1];
    int64_t i = a;
    while (i < b) {
      int64_t t = (int32_t)T->records[2 * i];
      int64_t j = i;
      while (j < b && (int32_t)T->records[2 * j] == t) ++j;
      if (t < 0 || t >= T->window_ps) { rc = OR_ERANGE; *bad_record = i; break; }
      if (t < t_prev) { rc = OR_EORDER; *bad_record = i; break; }
      /* leakage held since the previous group, at the pre-group state */
      double P = (double)leak[S] * ls;
      El += P * (double)(t - t_prev) * 1e-6;
      bin_add_interval(&B, P, t_prev, t);
      bin_add_interval(&BC[0], P, t_prev, t);
      /* dynamic energy of each event in the group, at the pre-group state */
      uint32_t S_next = S;
      for (int64_t e = i; e < j; ++e) {
        uint32_t meta = T->records[2 * e + 1];
        int32_t pin = (int32_t)(meta & 0xFu);
        int32_t value = (int32_t)((meta >> 4) & 1u);
        if ((meta >> 5) != 0 || pin >= n_pins) { rc = OR_ERANGE; *bad_record = e; break; }
        if ((int32_t)((S_next >> pin) & 1u) == value) { rc = OR_ENOTOGGLE; *bad_record = e; break; }
        S_next ^= 1u << pin;
        double E, sum_slew;
        if (pin < n_in) {
          const float* tab = table_for(L, tab_base, c, pin, value, side_bits(S, pin, n_in));
          const float* sl = N->slew_ps + ((int64_t)g * N->slew_stride + pin) * 2;
          E = es * oracle_bilinear(L->n_slew, L->slew_axis, L->n_load, L->load_axis, tab, sl[value], C);
          sum_slew = (double)sl[0] + (double)sl[1];
        } else {
          E = half_v2 * C;
          sum_slew = GL ? (double)GL->out_slew_ps[2 * g] + (double)GL->out_slew_ps[2 * g + 1] : 0.0;
        }
        if (GL && GL->clock_ps > 0 && last_t[pin] >= 0 && last_t[pin] / GL->clock_ps == t / GL->clock_ps) {
          E *= glitch_ratio((double)(t - last_t[pin]), sum_slew);
          Eg += E;
          bin_add(&BC[3], t, E);
        } else if (pin < n_in) {
          Ei += E;
          bin_add(&BC[1], t, E);
        } else {
          Es += E;
          bin_add(&BC[2], t, E);
        }
        last_t[pin] = t;
        bin_add(&B, t, E);
      }
      if (rc != OR_OK) break;
      S = S_next;
      t_prev = t;
      i = j;
    }
    if (rc != OR_OK) break;
    double P = (double)leak[S] * ls;
    El += P * (double)(T->window_ps - t_prev) * 1e-6;
    bin_add_interval(&B, P, t_prev, T->window_ps);
    bin_add_interval(&BC[0], P, t_prev, T->window_ps);
    if (e_leak) e_leak[gi] = El;
    if (e_int) e_int[gi] = Ei;
    if (e_sw) e_sw[gi] = Es;
    if (e_gl) e_gl[gi] = Eg;
    if (n_events) n_events[gi] = b - a;
    if (final_state) final_state[gi] = (uint8_t)S;
  }
  range_flush(&B);
  range_flush(&BC[0]);
  free(diff);
  free(cdiff);
  free(tab_base);
  free(leak_base);
  return rc;
}

int oracle_walk(const oracle_lib* L, const oracle_net* N, const oracle_trace* T, int64_t bin_ps,
                int64_t n_sel, const int64_t* gates,
                double* bins, int64_t n_sample, const int64_t* sample,
                double* e_leak, double* e_int, double* e_sw, int64_t* n_events, uint8_t* final_state,
                int64_t* bad_record, const oracle_glitch* GL, double* e_gl, double* comp_bins) {
  return walk_impl(L, N, T, bin_ps, n_sel, gates, bins, n_sample, sample, e_leak, e_int, e_sw, n_events,
                   final_state, bad_record, GL, e_gl, comp_bins, 0);
}

/* oracle_walk with the range-mode leakage split (see bin_add_interval): the
 * same bins up to the order of FP64 additions, in time proportional to
 * events + bins instead of gates x bins.  For full-size waveforms. */
int oracle_walk_range(const oracle_lib* L, const oracle_net* N, const oracle_trace* T, int64_t bin_ps,
                      int64_t n_sel, const int64_t* gates, double* bins,
                      double* e_leak, double* e_int, double* e_sw, int64_t* n_events, uint8_t* final_state,
                      int64_t* bad_record, const oracle_glitch* GL, double* e_gl, double* comp_bins) {
  return walk_impl(L, N, T, bin_ps, n_sel, gates, bins, 0, NULL, e_leak, e_int, e_sw, n_events, final_state,
                   bad_record, GL, e_gl, comp_bins, 1);
}

/* ---------------------------------------------------------------- adjoint */

/*
 * Gradient of a loss L(P) of the power waveform P_b = E_b * 1e-3 / bin_ps
 * (W), given dLdP[b], with respect to each gate's load C (dC), each cell's
 * energy scale (d_escale) and leakage scale (d_lscale).  FP64, by the chain
 * rule through the same definition as oracle_walk.  With `gates`, only the
 * listed gates are walked: dC[i] belongs to gates[i] and the cell gradients
 * hold those gates' contributions only.
 *   dE_int/dC = escale * d(bilinear)/d(load)   (located load segment)
 *   dE_sw/dC  = 0.5 * Vdd^2
 *   dE_int/d escale = bilinear value;  leakage energy is linear in lscale.
 * With glitch detection (GL), a glitch event's derivatives carry its ratio
 * r_gl, which depends on times and transition times only.
 */
int oracle_adjoint(const oracle_lib* L, const oracle_net* N, const oracle_trace* T, int64_t bin_ps,
                   const double* dLdP, int64_t n_sel, const int64_t* gates,
                   double* dC, double* d_escale, double* d_lscale, const oracle_glitch* GL) {
  if (bin_ps <= 0 || T->window_ps <= 0 || T->window_ps % bin_ps != 0) return OR_EINVAL;
  int64_t* tab_base = (int64_t*)malloc(sizeof(int64_t) * (size_t)L->n_cells);
  int64_t* leak_base = (int64_t*)malloc(sizeof(int64_t) * (size_t)L->n_cells);
  cell_bases(L, tab_base, leak_base);
  double per_fj = 1e-3 / (double)bin_ps;     /* dP_b / dE_b */
  double half_v2 = 0.5 * L->vdd * L->vdd;
  for (int32_t c = 0; c < L->n_cells; ++c) { d_escale[c] = 0.0; d_lscale[c] = 0.0; }
  int64_t count = gates ? n_sel : N->n_gates;
  for (int64_t gi = 0; gi < count; ++gi) {
    int64_t g = gates ? gates[gi] : gi;
    int32_t c = N->cell[g];
    int32_t n_in = L->n_in[c];
    double C = N->load_ff[g];
    double es = L->escale[c];
    const float* leak = L->p_leak + leak_base[c];
    uint32_t S = T->init_state[g];
    int64_t t_prev = 0;
    double gC = 0.0;
    int64_t last_t[16];
    for (int p = 0; p < 16; ++p) last_t[p] = -1;
    int64_t a = T->offsets[g], b = T->offsets[g + 1];
    int64_t i = a;
    for (;;) {
      int64_t t = (i < b) ? (int32_t)T->records[2 * i] : T->window_ps;
      /* leakage interval [t_prev, t) at state S: dL/dlscale += P0 * sum_b dL/dE_b * overlap */
      double P0 = leak[S];
      if (t > t_prev) {
        int64_t k0 = t_prev / bin_ps, k1 = (t - 1) / bin_ps;
        for (int64_t k = k0; k <= k1; ++k) {
          int64_t lo = t_prev > k * bin_ps ? t_prev : k * bin_ps;
          int64_t hi = t < (k + 1) * bin_ps ? t : (k + 1) * bin_ps;
          d_lscale[c] += P0 * (double)(hi - lo) * 1e-6 * dLdP[k] * per_fj;
        }
      }
      if (i >= b) break;
      int64_t j = i;
      while (j < b && (int32_t)T->records[2 * j] == t) ++j;
      double gb = dLdP[t / bin_ps] * per_fj;
      uint32_t S_next = S;
      for (int64_t e = i; e < j; ++e) {
        uint32_t meta = T->records[2 * e + 1];
        int32_t pin = (int32_t)(meta & 0xFu);
        int32_t value = (int32_t)((meta >> 4) & 1u);
        S_next ^= 1u << pin;
        double r = 1.0;
        if (GL && GL->clock_ps > 0 && last_t[pin] >= 0 && last_t[pin] / GL->clock_ps == t / GL->clock_ps) {
          double sum_slew = pin < n_in ? (double)N->slew_ps[((int64_t)g * N->slew_stride + pin) * 2] +
                                             (double)N->slew_ps[((int64_t)g * N->slew_stride + pin) * 2 + 1]
                                       : (double)GL->out_slew_ps[2 * g] + (double)GL->out_slew_ps[2 * g + 1];
          r = glitch_ratio((double)(t - last_t[pin]), sum_slew);
        }
        last_t[pin] = t;
        if (pin < n_in) {
          const float* tab = table_for(L, tab_base, c, pin, value, side_bits(S, pin, n_in));
          double slew = N->slew_ps[((int64_t)g * N->slew_stride + pin) * 2 + value];
          double B0 = oracle_bilinear(L->n_slew, L->slew_axis, L->n_load, L->load_axis, tab, slew, C);
          double dB = oracle_bilinear_dload(L->n_slew, L->slew_axis, L->n_load, L->load_axis, tab, slew, C);
          gC += gb * r * es * dB;
          d_escale[c] += gb * r * B0;
        } else {
          gC += gb * r * half_v2;
        }
      }
      S = S_next;
      t_prev = t;
      i = j;
    }
    dC[gi] = gC;
  }
  free(tab_base);
  free(leak_base);
  return OR_OK;
}
