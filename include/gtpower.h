/*
 * gtpower.h - C ABI of the GB300 engine for gate-level time-based power
 * analysis (event-driven power walk of arxiv 2609.05960, "GPU-Accelerated
 * Gate-Level Time-Based Power Analysis via Event-Density-Aware Partitioning
 * and Kernel Fusion").
 *
 * The engine walks each gate's time-ordered events, tracks the gate state,
 * looks up state-dependent internal energy (bilinear NLDM interpolation),
 * adds output switching energy and state-dependent leakage between events,
 * and accumulates everything into a per-time-bin power waveform and per-gate
 * energies.
 *
 * Conventions for every entry point:
 *   - Return value: GTP_OK (0) or a negative GTP_E* code; gtp_last_error()
 *     returns a message for the last failure on that context.  No C++
 *     exception crosses this boundary.
 *   - Units: time in ps (int32 timestamps), load in fF, slew in ps, supply in
 *     V, energy in fJ, leakage power in nW, waveform power in W.
 *   - Ownership: input arrays are copied unless GTP_BORROW is given; the
 *     caller may free them on return.  Outputs go into caller buffers on the
 *     host (GTP_HOST) or the device (GTP_DEVICE) as flagged.
 *   - Streams: all device work is enqueued on the context's stream.  Calls
 *     that return results or validation status synchronise that stream.
 *   - A context is bound to one device and is not thread-safe.
 */
#ifndef GTPOWER_H
#define GTPOWER_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define GTP_OK 0
#define GTP_EINVAL (-1)     /* bad argument (NULL, size, flag, call order) */
#define GTP_EORDER (-2)     /* timestamps decrease within a gate */
#define GTP_ERANGE (-3)     /* t outside [0, window_ps), pin >= pins of the cell,
                               reserved meta bits set, window_ps % bin_ps != 0,
                               or a size beyond an engine limit */
#define GTP_ENOTOGGLE (-4)  /* an event sets a pin to the value it already has */
#define GTP_ENOMEM (-5)     /* device or host allocation failed */
#define GTP_ECUDA (-6)      /* a CUDA runtime call failed */
#define GTP_ETIMEOUT (-7)   /* a bounded device wait expired; reserved: no
                               kernel of this engine waits on another block,
                               so no call returns it at present */
#define GTP_EDEVICE (-8)    /* a kernel reported an internal inconsistency */

/* ---- memory-space flags ---------------------------------------------- */
#define GTP_HOST 0          /* pointer is host memory */
#define GTP_DEVICE 1        /* pointer is device memory of the context's device */
#define GTP_BORROW 2        /* gtp_load_events only, with GTP_DEVICE: use the
                               caller's event buffer in place (no copy); it must
                               stay valid and unchanged while the window is used
                               and be 16-byte aligned */
#define GTP_GRAPH 4         /* gtp_run_power and gtp_run_power_batched, with
                               GTP_DEVICE: capture the run in a CUDA graph on
                               its first call and replay it on later calls with
                               the same window list, bin size, window sizes,
                               tuning and phase-timing setting */
#define GTP_PACKED 8        /* gtp_load_events (not with GTP_BORROW) and
                               gtp_run_power_streamed: `events` holds the
                               packed transfer form of gtp_pack_events */

/* Limits of this engine: at most 7 input pins per cell (8 pins, so the gate
 * state fits in one byte), at most 16 points per interpolation axis, and
 * library tables that fit in one SM's shared memory (GTP_MAX_TABLE_BYTES). */
#define GTP_MAX_PINS 8
#define GTP_MAX_AXIS 16
#define GTP_MAX_TABLE_BYTES (160 * 1024)

/* One event record, 8 bytes.  An event is a (value, timestamp) pair on one
 * pin: the pin switches to `value` at t_ps (Sec. 2.1).
 *   t_ps: timestamp in ps, 0 <= t_ps < window_ps
 *   meta: bits [0,4) gate-local pin (inputs 0..n_in-1, output = n_in),
 *         bit 4 the new value, bits [5,32) reserved and must be 0. */
typedef struct gtp_event {
  int32_t t_ps;
  uint32_t meta;
} gtp_event;

/*
 * Packed transfer form of n_events records, for runs bound by the host link
 * (gtp_run_power_streamed with GTP_PACKED): 4.125 bytes a record instead of
 * 8.  Records are taken in blocks of 32 (the last block may be shorter);
 * each block has one uint32 anchor, the smallest t_ps in the block, and each
 * record one uint32 word, (t_ps - anchor) << 5 | meta.  Layout: packed[0 ..
 * nb) the anchors, nb = (n_events + 31) / 32, then packed[nb .. nb +
 * n_events) the words.  Host only (no context, no GPU).  Returns GTP_ERANGE
 * if a record has t_ps < 0 or reserved meta bits set, or if a block spans
 * 2^27 ps or more (any window up to 134 us fits), GTP_EINVAL for null arrays.
 */
int gtp_pack_events(int64_t n_events, const gtp_event* events, uint32_t* packed);

typedef struct gtp_ctx gtp_ctx;

/* Create a context on CUDA device `device`, enqueueing on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  *out receives the
 * context, or NULL on failure. */
int gtp_create(gtp_ctx** out, int device, void* cuda_stream);

/* Free every device buffer the context owns, then the context. */
void gtp_destroy(gtp_ctx* ctx);

/* Change the stream later calls enqueue on. */
int gtp_set_stream(gtp_ctx* ctx, void* cuda_stream);

/* Message describing the last failure on ctx ("" if none).  Valid until the
 * next call on ctx. */
const char* gtp_last_error(const gtp_ctx* ctx);

/*
 * Load the cell library (host arrays).  Internal power is state dependent
 * (Sec. 2.2): each (cell, input pin, edge, side-input state) has its own
 * NLDM table, and the state is binary-encoded into a table index in pin
 * order (state-indexed lookup, Sec. 4.1).
 *   n_in[c]      input pins of cell c (1..7); the output pin is pin n_in[c]
 *   vdd          supply voltage (V)
 *   slew_axis    n_slew increasing input-slew knots (ps)
 *   load_axis    n_load increasing output-load knots (fF)
 *   e_int        n_e_int floats: cell-major; cell c holds n_in[c] pins x 2
 *                edges (0 fall, 1 rise) x 2^(n_in[c]-1) side states (the
 *                other input pins' bits, compacted in pin order) x
 *                n_slew x n_load (slew-major) internal energies in fJ
 *   p_leak       n_p_leak floats: cell-major; cell c holds 2^(n_in[c]+1)
 *                leakage powers in nW indexed by the full pin state
 *                (bit p = value of pin p, output included)
 * Errors: GTP_EINVAL on inconsistent sizes, GTP_ERANGE beyond the limits.
 * Loading a library invalidates loaded netlists and windows.
 */
int gtp_load_library(gtp_ctx* ctx, int32_t n_cells, const int32_t* n_in, float vdd,
                     int32_t n_slew, const float* slew_axis, int32_t n_load, const float* load_axis,
                     const float* e_int, int64_t n_e_int, const float* p_leak, int64_t n_p_leak);

/*
 * State-indexed lookup construction from Liberty-style state patterns
 * [Sec. 4.1], for one cell; host only (no context, no GPU).  Writes the
 * cell's part of gtp_load_library's e_int and p_leak arrays.
 *   Internal power: n_int_pat patterns.  Pattern k applies to input pin
 *     int_pin[k] (0..n_in-1) and edge int_edge[k] (0 fall, 1 rise, -1 both);
 *     its condition fixes the pins in int_care[k] (bit q = pin q; only other
 *     input pins) to the values in int_val[k] (a subset of int_care[k]) and
 *     leaves the rest don't-care; its table is int_tab[k * n_slew * n_load ..]
 *     (slew-major, fJ).  int_default[(pin * 2 + edge) * n_slew * n_load ..]
 *     is the table of a (pin, edge, side state) no pattern covers.
 *   Leakage: n_leak_pat patterns over all pins, output (bit n_in) included:
 *     leak_care[k], leak_val[k], power leak_pw[k] (nW); leak_default for the
 *     states none covers.
 *   Each pattern's don't-care pins are enumerated; an entry takes the item of
 *   the first pattern in list order that covers it (overlapping conditions
 *   resolve as a scan of the list in order would).
 *   e_int  out: n_in * 2 * 2^(n_in-1) * n_slew * n_load floats (the layout of
 *               gtp_load_library's e_int for this cell)
 *   p_leak out: 2^(n_in+1) floats
 * Returns GTP_ERANGE for n_in outside 1..GTP_MAX_PINS-1 or axes outside
 * 2..GTP_MAX_AXIS, GTP_EINVAL for a null array, a pin or edge out of range,
 * a condition on a pin it may not name, or values outside the care mask.
 */
int gtp_sipl_expand(int32_t n_in, int32_t n_slew, int32_t n_load, int32_t n_int_pat, const int32_t* int_pin,
                    const int32_t* int_edge, const uint32_t* int_care, const uint32_t* int_val, const float* int_tab,
                    const float* int_default, int32_t n_leak_pat, const uint32_t* leak_care, const uint32_t* leak_val,
                    const float* leak_pw, float leak_default, float* e_int, float* p_leak);

/* ------------------------------------------------------------------------
 * Pattern gates: gates whose cells are given by Liberty-style state patterns,
 * up to GTP_MAX_PATTERN_PINS pins (inputs and one output), such as the wide
 * cells and macros (SRAMs) the state-indexed library above cannot hold
 * [Sec. 4.1: state-indexed lookup for gates of at most 16 pins, direct
 * traversal of the state patterns for wider ones].  A pattern cell with at
 * most "sipl_max_pins" pins (gtp_set_param; default 16, the paper's
 * threshold; at most GTP_MAX_INDEXED_PINS) is walked through state-indexed
 * arrays the engine builds on the device from its patterns at the first run
 * after a change (each entry takes the first pattern covering it, as the
 * paper's don't-care enumeration fills it); a wider one scans its patterns
 * at every lookup.  Both give the same power items, so the threshold changes
 * speed and memory (4 * (n_in * 2^n_in + 2^(n_in+1)) bytes for a cell of
 * n_in inputs), never results.  The pattern gates of a window are walked
 * with its ordinary gates by gtp_run_power and gtp_run_power_batched, by the
 * same definition (Algorithm 1: groups of equal timestamps, lookups at the
 * pre-group state; Sec. 2.2, Eq. 1, Eq. 4, Sec. 2.4.2; glitch detection of
 * Sec. 2.4.1 and Eq. 2 when gtp_set_glitch is on, with the transition times
 * given here), and add into the same waveform (and, in
 * gtp_run_power_components, into the component waveforms);
 * gtp_design_power includes them.  gtp_run_power_backward walks them too
 * (their dL/dC through gtp_pattern_gate_gradient; pattern cells have no
 * energy or leakage scales).  gtp_run_power_scheme returns GTP_EINVAL for a
 * window with pattern gates.
 * ------------------------------------------------------------------------ */
#define GTP_MAX_PATTERN_PINS 32
#define GTP_MAX_INDEXED_PINS 24

/*
 * Load the pattern cells [Sec. 4.1: Liberty state patterns over a fixed pin
 * order] (host arrays; replaces earlier ones and drops the
 * pattern netlist and every window's pattern events).
 *   n_in[c]      input pins of cell c, 1..31; pin n_in[c] is its output
 *   vdd, axes    supply (V) and the table axes, as in gtp_load_library
 *   int_offsets  [n_cells + 1] from 0: cell c's internal patterns are
 *                k in [int_offsets[c], int_offsets[c + 1]), in list order
 *   int_pin[k], int_edge[k] (0 fall, 1 rise, -1 both), int_care[k],
 *   int_val[k]   as in gtp_sipl_expand (care: other input pins only)
 *   int_tab      [n_int][n_slew][n_load] fJ, pattern k's table
 *   int_default  per cell, [n_in[c]][2][n_slew][n_load] fJ, cell-major: the
 *                table of an event no pattern of its (pin, edge) matches
 *   leak_offsets [n_cells + 1]; leak_care/val[k] over all the cell's pins,
 *                leak_pw[k] nW; leak_default[c] nW
 * Errors: GTP_ERANGE for n_in or axis lengths out of range, GTP_EINVAL for
 * null arrays, decreasing offsets or a pattern naming a pin it may not.
 */
int gtp_load_pattern_cells(gtp_ctx* ctx, int32_t n_cells, const int32_t* n_in, float vdd, int32_t n_slew,
                           const float* slew_axis, int32_t n_load, const float* load_axis,
                           const int32_t* int_offsets, const int32_t* int_pin, const int32_t* int_edge,
                           const uint32_t* int_care, const uint32_t* int_val, const float* int_tab,
                           const float* int_default, const int32_t* leak_offsets, const uint32_t* leak_care,
                           const uint32_t* leak_val, const float* leak_pw, const float* leak_default);

/*
 * Load the pattern gates [Sec. 2.2: per-gate load and transition times;
 * Sec. 2.4.1 for the output transition times] (host arrays; drops every
 * window's pattern events):
 * cell[g] (a pattern cell), load_ff[g] (fF), slew_ps[g][slew_stride][2]
 * input {fall, rise} transition times (ps; slew_stride >= the widest cell's
 * inputs, <= 32), out_slew_ps[g][2] output {fall, rise} transition times for
 * glitch detection (NULL: none, an output glitch swings fully).  The
 * ordinary netlist (gtp_load_netlist) must be loaded for runs; loading it
 * again drops the windows and their pattern events.
 * Errors: GTP_EINVAL (no pattern cells, null arrays, stride), GTP_ERANGE
 * (cell index).
 */
int gtp_load_pattern_netlist(gtp_ctx* ctx, int64_t n_gates, const int32_t* cell, const float* load_ff,
                             const float* slew_ps, int32_t slew_stride, const float* out_slew_ps);

/*
 * Load a window's pattern-gate events [Sec. 2.1: an event is a pin's new
 * value at a time] (the window must be loaded by
 * gtp_load_events first, which fixes its window_ps; loading it again drops
 * them).  Arrays are host memory, or device memory with GTP_DEVICE; they are
 * copied.  gate_offsets[n_gates + 1] (CSR over the pattern gates, from 0 to
 * n_events); per event t_ps (non-decreasing within a gate), pin (< the
 * gate's pin count) and value (the pin's new value, 0 or 1, which must
 * differ from its current value); init_state[g] the gate's initial state
 * (bit q = pin q; no bits past its pins).  Times, pins and values are checked
 * by the run, which reports the first malformed record as gtp_run_power does
 * ("at pattern record N").
 * Errors: GTP_EINVAL (no pattern netlist, window not loaded, offsets),
 * GTP_ERANGE (initial state).
 */
int gtp_load_pattern_events(gtp_ctx* ctx, int32_t window, int64_t n_events, const int64_t* gate_offsets,
                            const int32_t* t_ps, const uint8_t* pin, const uint8_t* value,
                            const uint32_t* init_state, int flags);

/*
 * Per-pattern-gate results of the window's last run [Sec. 2.2 components;
 * Eq. 3 sums them]: energies in fJ (FP64;
 * e_gl is zero without glitch detection), event counts and final states
 * (uint32: up to 32 pins).  NULL outputs are skipped; outputs are host
 * memory, or device memory with GTP_DEVICE.
 * Errors: GTP_EINVAL when the window has no pattern-gate result.
 */
int gtp_pattern_gate_energy(gtp_ctx* ctx, int32_t window, double* e_leak, double* e_int, double* e_sw, double* e_gl,
                            int64_t* n_events, uint32_t* final_state, int flags);

/*
 * dL/dC of the pattern gates from the window's last gtp_run_power_backward
 * [the chain rule through Sec. 2.2's bilinear lookup in load and Eq. 1, a
 * glitch event's derivative carrying its ratio of Eq. 2; leakage does not
 * depend on the load]: dC[n_pattern_gates] float32, in the units of dL_dP
 * per fF, host memory or device memory with GTP_DEVICE.
 * Errors: GTP_EINVAL when the window has no pattern-gate gradient (no
 * backward run since its pattern events were loaded) or dC is NULL.
 */
int gtp_pattern_gate_gradient(gtp_ctx* ctx, int32_t window, float* dC, int flags);

/*
 * Per-cell multipliers on internal energy and on leakage power (host arrays
 * of n_cells; NULL leaves that scale at 1).  The paper has no counterpart:
 * they are parameters of this engine's adjoint (gtp_run_power_backward).  An
 * internal energy of cell c (the bilinear NLDM value of Sec. 2.2 / 2.4.1) is
 * multiplied by escale[c]; a leakage power of cell c (the state-indexed
 * value of Eq. 4) by lscale[c]; switching energy (Eq. 1) is not scaled.
 * Errors: GTP_EINVAL without a library.
 */
int gtp_set_scales(gtp_ctx* ctx, const float* escale, const float* lscale);

/*
 * Load the netlist: per gate its cell, output load C (fF; the total load of
 * the switching-energy equation, Sec. 2.4.1) and input slews (ps) per
 * (input pin, edge), as static timing provides them (Sec. 2.3).
 *   cell      [n_gates] int32 in [0, n_cells)
 *   load_ff   [n_gates] float
 *   slew_ps   [n_gates][slew_stride][2] float, slew_stride >= max n_in
 * flags: GTP_HOST or GTP_DEVICE for all three arrays.  Connectivity is not
 * needed by the walk.  Invalidates loaded windows.
 */
int gtp_load_netlist(gtp_ctx* ctx, int64_t n_gates, const int32_t* cell, const float* load_ff,
                     const float* slew_ps, int32_t slew_stride, int flags);

/* Replace every gate's output load (fF) without reloading the netlist
 * (e.g. inside an optimisation loop driven by the adjoint).  The load is the
 * c of the switching energy (Eq. 1) and the load coordinate of the NLDM
 * interpolation (Sec. 2.4.1).  flags: GTP_HOST or GTP_DEVICE. */
int gtp_set_load(gtp_ctx* ctx, const float* load_ff, int flags);

/*
 * Clock-cycle glitch detection [Sec. 2.4.1, Eq. 2,
 * Algorithm 1 GlitchDetectUpdate] for the following runs (forward, batched
 * and adjoint).  With clock_ps > 0, an event on a pin that already had an
 * event earlier in the same clock cycle floor(t / clock_ps) (t in window
 * time, so windows start on cycle boundaries) is a glitch event: its dynamic
 * energy is scaled by r = min(1, (2 w / (rise + fall))^2), w the time since
 * that pin's previous event and rise, fall the pin's transition times (input
 * pins: the netlist's slews; the output pin: out_slew_ps), and it counts as
 * glitch energy (gtp_gate_glitch) instead of internal or switching energy.
 * The waveform receives the scaled energy.  clock_ps = 0 turns detection off
 * (the default; also after gtp_load_netlist).
 *   out_slew_ps [n_gates][2] float {fall, rise} ps, copied; may be NULL when
 *               clock_ps == 0.  flags: GTP_HOST or GTP_DEVICE.
 * Errors: GTP_EINVAL without a netlist or with a NULL array, GTP_ERANGE for
 * clock_ps outside [0, 2^31).  gtp_run_power_noalloc does not detect
 * glitches.
 */
int gtp_set_glitch(gtp_ctx* ctx, int64_t clock_ps, const float* out_slew_ps, int flags);

/* Per-gate glitch energy (fJ, FP64; the E_gl of Eq. 2 summed per gate,
 * Sec. 4.3) of the last run of `window`: zeros if that run did not detect
 * glitches.  flags: GTP_HOST or GTP_DEVICE. */
int gtp_gate_glitch(gtp_ctx* ctx, int32_t window, double* e_gl, int flags);

/*
 * Design-level power of the last run of `window` [Eq. 3,
 * Sec. 2.4.1; peak power, Sec. 5], into out[7] (host, FP64):
 *   out[0..3]  leakage, internal, switching and glitch power in W: the
 *              per-gate energies summed over the design, over window_ps
 *              (the paper divides by the end of its analysis, here the
 *              window's end);
 *   out[4]     their total;
 *   out[5]     the peak bin power of waveform_w (W), out[6] its first bin
 *              index; 0 and -1 when waveform_w is NULL.
 * waveform_w [n_bins of that run]: the waveform the run wrote, or NULL;
 * flags: GTP_HOST or GTP_DEVICE for it.
 */
int gtp_design_power(gtp_ctx* ctx, int32_t window, const double* waveform_w, int flags, double* out);

/*
 * Load one stimulus window's events as slot `window` (0 <= window < 1024;
 * reloading a slot replaces it).  An event is a (value, timestamp) pair on
 * one pin (Sec. 2.1); the paper keeps one stream per pin and merges them on
 * the fly (Sec. 2.4.2, Algorithm 1), while here each gate's events arrive
 * already merged into one time-ordered stream.
 *   window_ps     length of the analysis window, > 0, < 2^31
 *   n_events      number of records (may be 0)
 *   gate_offsets  [n_gates+1] int64 CSR offsets: gate g's records are
 *                 events[gate_offsets[g] .. gate_offsets[g+1]), time-ordered
 *                 (ties allowed: events sharing a timestamp form one group)
 *   events        [n_events] records
 *   init_state    [n_gates] state of every gate at t = 0 (bit p = pin p)
 * flags: GTP_HOST, GTP_DEVICE, or GTP_DEVICE|GTP_BORROW (events only);
 * GTP_PACKED: `events` is the packed transfer form (gtp_pack_events) of the
 * n_events records, unpacked on the device.
 * The CSR structure is checked here (GTP_EINVAL); timestamps, pins and
 * toggles are checked by the walk and reported by gtp_run_power.
 */
int gtp_load_events(gtp_ctx* ctx, int32_t window, int64_t window_ps, int64_t n_events,
                    const int64_t* gate_offsets, const gtp_event* events, const uint8_t* init_state,
                    int flags);

/*
 * Run the power walk of one window with bins of bin_ps ps
 * (n_bins = window_ps / bin_ps; window_ps % bin_ps must be 0).  This is the
 * fused computation of Sec. 4.3 (Algorithm 1) over every gate: per
 * timestamp group the lookups use the state before the group and the state
 * is updated after it; internal energy is the state-indexed NLDM value
 * (Sec. 2.2, Sec. 4.1) interpolated at (slew, load); switching energy is
 * 0.5*C*Vdd^2 per output toggle (Eq. 1, one half per edge); leakage power
 * of the current state holds between groups (Eq. 4) and is split over the
 * bins each interval overlaps in proportion to the overlap (Sec. 2.4.2);
 * dynamic energy goes to the bin holding the event (Sec. 2.4.1).  The bin
 * plays the part of the paper's clock cycle.
 * Writes waveform_w[n_bins] (FP64, W): the mean power of each bin, i.e. the
 * energy of all events in the bin (dynamic energy goes to the bin holding the
 * event time; a time on a bin boundary belongs to the later bin) plus the
 * leakage energy overlapping the bin, divided by bin_ps.  Per-gate results are
 * kept for gtp_gate_energy.  Synchronous; returns GTP_EORDER / GTP_ERANGE /
 * GTP_ENOTOGGLE if the trace is malformed (results are then undefined).
 * waveform_w may be NULL to compute per-gate results only.
 * flags: GTP_HOST or GTP_DEVICE for waveform_w, optionally | GTP_GRAPH
 * (device waveform only).
 */
int gtp_run_power(gtp_ctx* ctx, int32_t window, int32_t bin_ps, double* waveform_w, int flags);

/*
 * gtp_run_power that also returns the waveform of each power component
 * [Sec. 2.2: leakage, internal, switching and glitch power; Sec. 2.4.1 for
 * the glitch component, which is zero unless gtp_set_glitch set a clock].
 *   components_w [4][n_bins] (FP64, W), component-major: row 0 leakage, row 1
 *     internal (input-pin events that are not glitches), row 2 switching
 *     (output-pin events that are not glitches), row 3 glitch energy.  Each
 *     bin is that component's energy in the bin divided by bin_ps; the four
 *     rows add up to waveform_w up to FP32 rounding.  Required.
 *   waveform_w [n_bins] or NULL: the total, as gtp_run_power writes it.
 * The walk keeps 16-byte accumulators per bin: without glitch detection it
 * costs about what gtp_run_power costs; with it, one more reduction per bin
 * update.  Per-gate results are kept as for gtp_run_power.  flags: GTP_HOST or GTP_DEVICE for
 * both outputs; GTP_GRAPH is rejected (GTP_EINVAL).  Errors as gtp_run_power.
 */
int gtp_run_power_components(gtp_ctx* ctx, int32_t window, int32_t bin_ps, double* waveform_w,
                             double* components_w, int flags);

/*
 * The paper's own GPU schemes, for comparison with gtp_run_power on the same
 * window (they compute the same waveform and per-gate results):
 *   GTP_SCHEME_NAIVE    Naive-D (one thread per event, the gate state rebuilt
 *                       by binary searches in each pin's event stream,
 *                       Sec. 2.4.1) and Naive-L (one thread per gate and
 *                       window of scheme_ncyc_fix bins, leakage added to every
 *                       overlapped bin, Sec. 2.4.2), with state-dependent
 *                       energies found by traversing the state patterns
 *                       (Sec. 3.1);
 *   GTP_SCHEME_SIPL     the same with state-indexed lookup (Sec. 4.1);
 *   GTP_SCHEME_DENSITY  and Naive-L's windows sized per gate by event density
 *                       (Sec. 4.2: scheme_evt_tgt events a thread, parallelism
 *                       floor scheme_thr_floor);
 *   GTP_SCHEME_FUSED    one fused kernel over the density-aware windows
 *                       (Sec. 4.3, Algorithm 1) and the two-phase per-gate
 *                       reduction (Sec. 4.4).
 * The waveform bin plays the part of the paper's clock cycle; glitch
 * detection follows gtp_set_glitch.  Bins and per-gate sums are FP64
 * atomics.  The first call on a window builds its per-pin event streams
 * (checking the trace as gtp_run_power does) and, for the density-aware
 * schemes, the block plan; later calls reuse them.  *kernel_ms (may be NULL)
 * receives the device time of the scheme's kernels alone (CUDA events).
 * Per-gate results are kept for gtp_gate_energy.  flags: GTP_HOST or
 * GTP_DEVICE for waveform_w (may be NULL); GTP_GRAPH is rejected.  Device
 * memory: 8 B per event, 72 B per gate of streams, 4 KB per gate of reduction
 * rows, 8 B per bin.
 */
#define GTP_SCHEME_NAIVE 0
#define GTP_SCHEME_SIPL 1
#define GTP_SCHEME_DENSITY 2
#define GTP_SCHEME_FUSED 3
int gtp_run_power_scheme(gtp_ctx* ctx, int32_t window, int32_t bin_ps, int32_t scheme, double* waveform_w,
                         int flags, float* kernel_ms);

/*
 * One window run straight from host memory, in chunks [Sec. 5, event
 * chunking with the packing and copy of the next chunk overlapping the
 * kernel]: the window's records are copied to the GPU in n_chunks gate-range
 * chunks, through two device buffers of the largest chunk's size, and the
 * walk of each chunk overlaps the copy of the next.  Chunks hold about equal
 * numbers of records, except that with three or more chunks the first holds
 * half and the last a quarter of the others' share (the first copy and the
 * last walk are the parts that cannot overlap).  A trace larger than the device memory runs this way.  Results
 * equal gtp_load_events + gtp_run_power on the same inputs; the per-gate
 * results are kept for gtp_gate_energy / gtp_gate_glitch, but the records
 * are not: the window must be loaded again for any other run.
 *   gate_offsets [n_gates+1], events [n_events] and init_state [n_gates]
 *   are host memory (events pinned for the copies to overlap), as for
 *   gtp_load_events; waveform_w [n_bins] as for gtp_run_power.
 *   n_chunks: 1..1024.  flags: GTP_HOST or GTP_DEVICE for waveform_w,
 *   optionally | GTP_PACKED: `events` is then the packed transfer form of
 *   gtp_pack_events (cast to const gtp_event*), of which each chunk's
 *   anchors and words are copied and unpacked on the device; record indices
 *   in errors are those of the unpacked records.
 * Synchronous.  Errors as gtp_load_events and gtp_run_power (offsets are
 * checked on the host before any copy).
 */
int gtp_run_power_streamed(gtp_ctx* ctx, int32_t window, int64_t window_ps, int64_t n_events,
                           const int64_t* gate_offsets, const gtp_event* events, const uint8_t* init_state,
                           int32_t bin_ps, double* waveform_w, int32_t n_chunks, int flags);

/*
 * Per-gate results of the last gtp_run_power / batched run of `window`:
 * leakage, internal and switching energy (fJ, FP64), event count and the
 * state after the last event.  These are the per-gate power results the
 * paper reduces per gate (Sec. 4.4, the R^(g) buffers; reported per gate,
 * Sec. 5) kept as energies (divide by the window for power, Eq. 3).  Any
 * pointer may be NULL.  Errors: GTP_EINVAL if the window has no result.
 * flags: GTP_HOST or GTP_DEVICE for all outputs.  Host outputs are complete
 * on return; device outputs are written in order on the context's stream
 * (no host synchronisation).
 */
int gtp_gate_energy(gtp_ctx* ctx, int32_t window, double* e_leak, double* e_int, double* e_sw,
                    int64_t* n_events, uint8_t* final_state, int flags);

/*
 * The paper has no batched form: this is gtp_run_power (Sec. 4.3,
 * Algorithm 1) for many stimulus windows of one netlist at once.
 * Run n_windows (<= 1024) distinct loaded windows over the same netlist: one
 * gate-pass launch, one seed pass and one persistent walk launch whose warps
 * take segments from a single list covering every window, and one merge
 * (windows[i] names the slot; waveforms[i] receives window i's waveform,
 * same layout as gtp_run_power; a NULL entry skips that waveform).
 * flags: GTP_HOST or GTP_DEVICE for the waveform buffers (the pointer array
 * itself is host memory), optionally | GTP_GRAPH (device buffers only).
 */
int gtp_run_power_batched(gtp_ctx* ctx, int32_t n_windows, const int32_t* windows, int32_t bin_ps,
                          double* const* waveforms, int flags);

/*
 * The paper has no adjoint; this differentiates gtp_run_power's waveform,
 * whose energies are the bilinear internal energy (Sec. 2.2, Sec. 2.4.1),
 * 0.5*C*Vdd^2 switching energy (Eq. 1) and leakage P*dt (Eq. 4) split over
 * the bins (Sec. 2.4.2).
 * Adjoint of gtp_run_power for one window: given dL_dP[n_bins] (device,
 * FP32, the gradient of a scalar loss with respect to each bin's power in W),
 * write the gradients with respect to every gate's load (dC[n_gates]) and
 * every cell's energy and leakage scale (d_escale[n_cells],
 * d_lscale[n_cells]), all FP32 device buffers; any output may be NULL.
 * The internal-energy derivative in the load is the slope of the located
 * load segment of the bilinear table (right derivative on a knot);
 * d(0.5*C*Vdd^2)/dC = 0.5*Vdd^2; leakage energy is linear in lscale and
 * internal energy in escale.  Uses the context's current scales and loads.
 * A window with pattern gates also gets their dL/dC, read with
 * gtp_pattern_gate_gradient.  Synchronous; reports malformed traces (of
 * either kind of gate) like gtp_run_power.
 */
int gtp_run_power_backward(gtp_ctx* ctx, int32_t window, int32_t bin_ps, const float* dL_dP, float* dC,
                           float* d_escale, float* d_lscale);

/*
 * The counterpart of the paper's parameter study of its density-aware
 * partitioning (Sec. 4.2, Eqs. 7-13: the target events per thread and the
 * parallelism floor; Sec. 6.4) for this engine's partitioning parameters.
 * Autotuner: time the walk of the given windows for every candidate
 * (records per lane 4/8/16 = segment length 128/256/512 events, dense_min
 * 64/256/512/1024), `iters` timed runs each, keep the fastest as the context's
 * parameters and report its time per run (ms) in *best_ms.  Runs the windows
 * repeatedly; their per-gate results are those of the last run.
 */
int gtp_autotune(gtp_ctx* ctx, int32_t n_windows, const int32_t* windows, int32_t bin_ps, int32_t iters,
                 double* best_ms);

/*
 * The GPU's rate for the walk's bin updates, measured: n_red
 * fire-and-forget float reductions of `width` floats (2: the 8-byte
 * {energy, leakage step} update of a bin; 4: the 16-byte update of the
 * component runs) into places of an array of n_slots entries (use the bin
 * count) picked by an integer hash, timed with CUDA events after one
 * warm-up launch.  *per_s receives reductions per second.  The array is
 * context scratch of 16 B a slot.  Errors: GTP_EINVAL for bad arguments.
 */
int gtp_measure_reductions(gtp_ctx* ctx, int32_t n_slots, int32_t width, int64_t n_red, double* per_s);

/*
 * The bin reductions of a loaded window's own records, alone: each thread
 * takes 8 consecutive records and issues one 8-byte reduction per distinct
 * bin among them (the pattern of the walk's dense segments), into context
 * scratch laid out as the walk's 8-byte bins; records outside the window
 * are skipped.  Timed with CUDA events after one warm-up launch; *ms
 * receives the time of one pass.  It is the walk's own reduction stream
 * without the walk, a floor for it on this GPU.  Errors: GTP_EINVAL.
 */
int gtp_measure_replay(gtp_ctx* ctx, int32_t window, int32_t bin_ps, double* ms);

/* Engine tuning knobs; value < 0 restores the default.  Keys:
 * "records_per_thread" (4, 8, 16; events per lane of a dense segment),
 * "ctas_per_sm" (0 = full occupancy), "bwd_staged" (the adjoint's sparse
 * threads stage their gate tables in shared memory: 1 always, 0 never, -1 =
 * below 200,000 events per SM, the default; runs without glitch detection),
 * "dense_min" (gates with more events are cut into segments and
 * walked by warps, the others one per thread; 1..4096; by default chosen
 * per run: 256 in the adjoint and in forward runs of fewer than 260,000
 * events per SM (in the busiest window group, or streamed chunk), 384 up to
 * 600,000, 512 above; with glitch detection 384 below 200,000 and 1024
 * above; gtp_get_param "dense_min" reports the value set, else the last
 * run's),
 * "piece_len" (a gate with more events than this is walked as several
 * work items of piece_len events, each starting from the state its earlier
 * records leave, so that one very busy gate cannot hold up a run; -1 = chosen
 * per run: at least 65,536 and about a sixth of an SM's even share of the
 * run's events, the default; 0 = never; other values round up to a multiple
 * of 4,096; gtp_get_param "run_piece_len" and "run_whole" (1: no gate of
 * the last run was split) report the last run's choice),
 * "sipl_max_pins" (pattern cells with at most this many pins are walked
 * through state-indexed arrays, wider ones by pattern traversal; 0..24,
 * default 16; gtp_get_param "pattern_indexed_cells" and
 * "pattern_index_bytes" report the arrays built at the last run, -1 before),
 * "group_bin_bytes" (a forward run over several windows walks them in
 * groups of consecutive windows whose bins, 8 B each, add up to at most
 * this many bytes (a window with more is a group of its own), one group after
 * another, so that the bins a walk reduces into stay in L2; default 96 MiB;
 * gtp_get_param "run_groups" returns the last run's group count),
 * "tile_min" (single-window runs without glitch detection or component
 * waveforms: gates with at least this many events, and at most 3 inputs,
 * take the time-sliced walk, which keeps each 16,384-bin slice of the
 * waveform in shared memory as exact integer sums and merges slices in FP64;
 * 0 = off, the default),
 * "kernel" (0 = density-split walk,
 * 1 = one thread per gate, a plain cross-check), "scheme_evt_tgt" (8),
 * "scheme_thr_floor" (512) and "scheme_ncyc_fix" (1) for gtp_run_power_scheme,
 * "timing" (1 = time the
 * phases of later runs with CUDA events; read back with gtp_get_param keys
 * "t_gate_pass_ns" (the preparation launch: bins cleared, gate pass and
 * work-list histogram), "t_plan_ns" (work-list scatter), "t_walk_ns",
 * "t_merge_ns", "t_pattern_ns" (the pattern gates' walk, also inside
 * "t_walk_ns"), "t_prep_ns" (the pass that rebuilds the event descriptors
 * and per-gate energy tables after a netlist, load or scale change, at the
 * start of the next run), "t_stream_setup_ns", "t_stream_copy_ns",
 * "t_stream_tail_ns" (a streamed run's time before its first copy, from the
 * first copy's start to the last copy's end, and after that), "n_timed",
 * and "launches" = kernels launched since timing
 * was last set; 2 = "t_walk_ns" only, two events a run instead of twelve,
 * so that timing a step barely lengthens it; 0 = off). */
int gtp_set_param(gtp_ctx* ctx, const char* key, int64_t value);
int64_t gtp_get_param(const gtp_ctx* ctx, const char* key);

/* Largest window (in bins) gtp_run_power_noalloc accepts. */
#define GTP_NOALLOC_MAX_BINS (1 << 19)

/*
 * gtp_run_power_noalloc - one window's power walk that allocates nothing.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot call cudaMalloc, such as code inside another framework's device
 * memory pool (which owns every device byte), a host callback, or a caller
 * that must not pay cudaMalloc/cudaFree's implicit synchronisation between
 * its own launches.  It needs no context: inputs and outputs are the
 * caller's, and the walk's scratch (bin accumulators, merge tile sums, L0,
 * error word, cell map) lives in one fixed file-scope device array of about
 * 4.2 MB (header 8 KB, tile sums 2 KB, GTP_NOALLOC_MAX_BINS x 8 bytes of bin
 * accumulators), which every GPU that loads this library holds until the
 * process exits.
 *
 * Runs on the calling thread's current device, enqueues on cuda_stream (a
 * cudaStream_t of that device; NULL = the legacy default stream) and
 * synchronises it before returning (it reads the kernel's status word back).
 * The first call on a device looks up the scratch array's device address
 * (cudaGetSymbolAddress) and keeps it for later calls; make that first call
 * outside any stream capture.  Because every call waits for its stream, no
 * call may be made while that stream is being captured: such a call returns
 * GTP_EINVAL and enqueues nothing.  Calls no cudaMalloc, cudaFree or other
 * allocating routine.
 *
 * Every call on a device shares the one scratch array and starts by clearing
 * what must begin at zero (bins, L0, error word).  Calls whose GPU work
 * overlaps (other host threads, other streams) race on the scratch and give
 * undefined results: serialise them.
 *
 * Arguments, with the meaning, layout and units of gtp_load_library,
 * gtp_load_netlist, gtp_load_events and gtp_run_power:
 *   host memory:   n_in[n_cells] (n_cells <= 256), slew_axis[n_slew],
 *                  load_axis[n_load]
 *   device memory: e_int[n_e_int], p_leak[n_p_leak], cell[n_gates],
 *                  load_ff[n_gates], slew_ps[n_gates][slew_stride][2],
 *                  gate_offsets[n_gates+1], events[n_events] (8-byte
 *                  aligned), init_state[n_gates]; outputs waveform_w[n_bins]
 *                  (W), e_leak/e_int_out/e_sw[n_gates] (fJ, FP64) and
 *                  final_state[n_gates], each of which may be NULL.
 * Per-cell energy and leakage scales are 1.  n_bins = window_ps / bin_ps.
 * Errors: GTP_ERANGE for n_bins > GTP_NOALLOC_MAX_BINS or the limits of
 * gtp_load_library (checked before any work is enqueued), GTP_EINVAL for bad
 * sizes or pointers and for a malformed CSR or cell index (found by the
 * kernel), GTP_EORDER / GTP_ERANGE / GTP_ENOTOGGLE for a malformed trace as
 * in gtp_run_power (outputs are then undefined), GTP_ECUDA if a CUDA call
 * fails.  There is no message string.
 */
int gtp_run_power_noalloc(void* cuda_stream, int32_t n_cells, const int32_t* n_in, float vdd, int32_t n_slew,
                          const float* slew_axis, int32_t n_load, const float* load_axis, const float* e_int,
                          int64_t n_e_int, const float* p_leak, int64_t n_p_leak, int64_t n_gates,
                          const int32_t* cell, const float* load_ff, const float* slew_ps, int32_t slew_stride,
                          int64_t window_ps, int64_t n_events, const int64_t* gate_offsets,
                          const gtp_event* events, const uint8_t* init_state, int32_t bin_ps, double* waveform_w,
                          double* e_leak, double* e_int_out, double* e_sw, uint8_t* final_state);

#ifdef __cplusplus
}
#endif

#endif /* GTPOWER_H */
