"""The FP64 oracle over a whole seeded workload, on every host core.

TEST INFRASTRUCTURE ONLY: used by ``tests/`` and by ``bench.py`` to state
each result's error against the oracle.  The GPU engine never imports it.

The walk is additive over gates (each gate's energies go to its own per-gate
outputs and add into the shared bins), so the gates are split into ranges of
about equal event counts, one task per host process.  Each process rebuilds
the library, netlist and per-gate event counts from the workload's seeds,
regenerates its gates' records with the counter-based generator (the same
bits the GPU generator writes), and runs ``oracle.walk`` with the range-mode
leakage split on sub-ranges of gates, adding the bins in FP64.  The parent
adds the processes' bins in FP64 in gate order.  Nothing here does any of the
method's arithmetic; that is all in ``gtp_oracle.c``.
"""
from __future__ import annotations

import dataclasses
import multiprocessing as mp
import os
from typing import Optional

import numpy as np

_STATE = {}


@dataclasses.dataclass(frozen=True)
class Workload:
    """A seeded workload: the library, netlist and per-gate Zipf counts of a
    synth.Config, a window, and optional glitch detection with output
    transition times drawn uniform in out_slew_range from
    numpy.random.default_rng(out_slew_seed) as an [n_gates, 2] float32 array."""
    n_gates: int
    n_events: int
    zipf_s: float
    cap: Optional[int]
    window_ps: int
    seed_lib: int
    seed_net: int
    seed_ev: int
    tie_p: float = 0.0
    clock_ps: int = 0
    out_slew_seed: int = 7
    out_slew_range: tuple = (10.0, 200.0)

    @staticmethod
    def of(cfg, seed_ev: Optional[int] = None, clock_ps: int = 0, **kw) -> "Workload":
        return Workload(cfg.n_gates, cfg.n_events, cfg.zipf_s, cfg.cap, cfg.window_ps, cfg.seed_lib, cfg.seed_net,
                        cfg.seed_ev if seed_ev is None else seed_ev, cfg.tie_p, clock_ps, **kw)


def _build(wl: Workload):
    import synth
    lib = synth.make_library(wl.seed_lib)
    net = synth.make_netlist(lib, wl.n_gates, wl.seed_net)
    counts = synth.zipf_counts(wl.n_gates, wl.n_events, wl.zipf_s, wl.cap, wl.seed_ev)
    trace = synth.make_trace(net, counts, wl.window_ps, wl.seed_ev, wl.tie_p, materialise=False)
    out_slew = None
    if wl.clock_ps > 0:
        out_slew = np.random.default_rng(wl.out_slew_seed).uniform(
            wl.out_slew_range[0], wl.out_slew_range[1], (wl.n_gates, 2)).astype(np.float32)
    return lib, net, counts, trace, out_slew


def _inputs(wl: Workload):
    """The workload's inputs in this worker, built once (the last one kept)."""
    cache = _STATE.setdefault("cache", {})
    if wl not in cache:
        while len(cache) >= 1:
            cache.pop(next(iter(cache)))
        cache[wl] = _build(wl)
    return cache[wl]


def _task(job):
    """Gates [g0, g1) of a workload, in sub-ranges of about `chunk` events."""
    import oracle
    import synth
    wl, g0, g1, bin_ps, chunk, escale, lscale, components = job
    lib, net, counts, trace, out_slew = _inputs(wl)
    n_bins = wl.window_ps // bin_ps
    bins = np.zeros(n_bins, np.float64)
    comp = np.zeros((4, n_bins), np.float64) if components else None
    n = g1 - g0
    per = {k: np.zeros(n, np.float64) for k in ("e_leak", "e_int", "e_sw", "e_gl")}
    per["n_events"] = np.zeros(n, np.int64)
    per["final_state"] = np.zeros(n, np.uint8)
    cum = np.concatenate([[0], np.cumsum(counts[g0:g1])])
    a = 0
    while a < n:
        b = int(np.searchsorted(cum, cum[a] + chunk, side="right")) - 1
        b = min(max(b, a + 1), n)
        gates = np.arange(g0 + a, g0 + b, dtype=np.int64)
        off, rec = synth.gate_records(net, trace, gates)
        sub_net = synth.Netlist(net.cell[gates], net.load_ff[gates], np.ascontiguousarray(net.slew_ps[gates]),
                                net.n_pins[gates], net.level[gates], net.fanin[gates])
        sub_tr = synth.Trace(trace.window_ps, off, rec, trace.init_state[gates], trace.seed, trace.tie24)
        glitch = (wl.clock_ps, out_slew[gates]) if out_slew is not None else None
        r = oracle.walk(lib, sub_net, sub_tr, bin_ps, escale=escale, lscale=lscale, glitch=glitch,
                        components=components, leak_range=True)
        bins += r["bins"]
        if comp is not None:
            comp += r["comp_bins"]
        for k in per:
            per[k][a:b] = r[k]
        a = b
    return g0, bins, comp, per


def walk(wl: Workload, bin_ps: int, n_proc: Optional[int] = None, escale=None, lscale=None,
         components: bool = False) -> dict:
    """The oracle's full result for a workload: ``bins`` (fJ, every bin),
    the per-gate outputs of every gate, and ``comp_bins`` with components.
    Runs on n_proc spawned processes (default: every host core)."""
    with Pool(n_proc) as p:
        return p.walk(wl, bin_ps, escale=escale, lscale=lscale, components=components)


class Pool:
    """Spawned worker processes that walk workloads for the parent; each
    worker builds a workload's inputs from its seeds the first time it sees
    it.  Start it before the parent uses the GPU, or use it from a process
    that never does: the workers are spawned, not forked."""

    def __init__(self, n_proc: Optional[int] = None):
        import oracle
        oracle.build()  # once here, not concurrently in the workers
        self.n = max(1, n_proc or os.cpu_count() or 1)
        self.pool = mp.get_context("spawn").Pool(self.n)

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def close(self):
        if self.pool is not None:
            self.pool.close()
            self.pool.join()
            self.pool = None

    def walk(self, wl: Workload, bin_ps: int, escale=None, lscale=None, components: bool = False) -> dict:
        import synth
        counts = synth.zipf_counts(wl.n_gates, wl.n_events, wl.zipf_s, wl.cap, wl.seed_ev)
        n_bins = wl.window_ps // bin_ps
        # about 4 tasks a process, split by events plus a gate's fixed cost
        n_tasks = 4 * self.n
        weight = np.cumsum(counts + 8)
        cuts = np.searchsorted(weight, np.linspace(0, weight[-1], n_tasks + 1)[1:-1])
        edges = np.unique(np.concatenate([[0], cuts, [wl.n_gates]]))
        chunk = max(4_000_000, 2 * n_bins)
        es = None if escale is None else np.asarray(escale, np.float64)
        ls = None if lscale is None else np.asarray(lscale, np.float64)
        jobs = [(wl, int(a), int(b), int(bin_ps), chunk, es, ls, components) for a, b in zip(edges[:-1], edges[1:])]
        out = {k: np.zeros(wl.n_gates, np.float64) for k in ("e_leak", "e_int", "e_sw", "e_gl")}
        out["n_events"] = np.zeros(wl.n_gates, np.int64)
        out["final_state"] = np.zeros(wl.n_gates, np.uint8)
        bins = np.zeros(n_bins, np.float64)
        comp = np.zeros((4, n_bins), np.float64) if components else None
        for g0, b, c, per in self.pool.imap(_task, jobs):
            bins += b
            if comp is not None:
                comp += c
            n = len(per["n_events"])
            for k in out:
                out[k][g0:g0 + n] = per[k]
        out["bins"] = bins
        if comp is not None:
            out["comp_bins"] = comp
        return out


def bin_errors(got_w: np.ndarray, ref_bins_fj: np.ndarray, bin_ps: int) -> dict:
    """Relative error of a waveform in W against oracle bins in fJ: the
    largest and the mean over bins, and the bin holding the largest."""
    import oracle
    want = oracle.waveform_w(ref_bins_fj, bin_ps)
    den = np.abs(want)
    rel = np.abs(np.asarray(got_w, np.float64) - want) / np.where(den > 0, den, 1.0)
    return {"max_rel_bin_err": float(rel.max()) if rel.size else 0.0,
            "mean_rel_bin_err": float(rel.mean()) if rel.size else 0.0,
            "worst_bin": int(rel.argmax()) if rel.size else -1, "bins": int(rel.size)}


def gate_errors(got: dict, ref: dict, keys=("e_leak", "e_int", "e_sw")) -> dict:
    """Per-gate results against the oracle's: mismatched event counts and
    final states (must be 0), and the largest relative error of each energy
    (1e-9 fJ absolute floor for exact zeros)."""
    out = {"count_mismatches": int(np.sum(np.asarray(got["n_events"]) != ref["n_events"])),
           "state_mismatches": int(np.sum(np.asarray(got["final_state"]) != ref["final_state"]))}
    for k in keys:
        g = np.asarray(got[k], np.float64)
        err = np.abs(g - ref[k]) / np.maximum(np.abs(ref[k]), 1e-9 / 1e-5)
        out[f"max_rel_{k}_err"] = float(err.max()) if err.size else 0.0
    return out
