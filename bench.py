"""Benchmark of the GB300 power-walk engine.

One step = one pass of the whole hot path over one stimulus window with its
inputs resident in HBM: gtp_load_events (device records used in place, CSR
check), gtp_run_power (replayed as a CUDA graph: the preparation pass that
clears the bins, does the gate pass and counts the work list, the work-list
scatter, the fused walk, and the merge into the waveform) and gtp_gate_energy
(per-gate results to device buffers).

Default workload: 1M gates, 200M events (1.6 GB of 8-byte records), Zipf 1.2
per-gate counts capped at 1e5, 10 us window, 10 ps bins (1M bins).  The
records (1.6 GB) are larger than L2 (129 MB), so no L2 flush is needed
between steps.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle on a bounded sample of the same workload instead.

Multi-GPU (torchrun): every rank runs its own stimulus window (seeded per
rank) on its own GPU, with no collective on the data path (weak scaling);
the only collectives are the barrier and the max-over-ranks of the timings.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "events/sec and % of HBM roofline; batched and adjoint vs plain kernel"
# DRAM bytes (read + write) of one walk launch (k_walk<8,0,0,0,0>, the build without pieces) on the full large workload with
# the default plan, from one ncu capture of dram__bytes_read.sum + dram__bytes_write.sum (one
# pass); reported as roofline.traffic for that workload and plan only, and to be captured again
# whenever the walk changes
WALK_TRAFFIC = {("large", 8, 512): 2_020_504_064 + 82_823_168}
UNIT = "events/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--config", default="large")
    p.add_argument("--e2e-steps", type=int, default=10)
    p.add_argument("--cpu-seconds", type=float, default=12.0, help="CPU-baseline sample budget")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-clocks", action="store_true")
    p.add_argument("--no-extras", action="store_true",
                   help="skip the glitch, components, batched, adjoint, load-change and stress measurements")
    p.add_argument("--no-oracle-check", action="store_true",
                   help="skip the FP64 oracle over every bin and gate of each measured workload")
    p.add_argument("--no-stress", action="store_true", help="skip the stress workload (10M gates, 2B events)")
    p.add_argument("--no-patterns", action="store_true", help="skip the pattern-gate threshold sweep")
    p.add_argument("--events", type=int, default=0,
                   help="scale the configuration to this many events (same gates and distribution; "
                        "for profiling a smaller case)")
    p.add_argument("--sweep", default="", choices=["", "contention", "streamed", "schemes", "adjoint", "glitch", "tiled",
                                                    "patterns", "prep"],
                   help="contention: uniform high activity (1, 2, 4, 8 events per gate per 1k bins); "
                        "streamed: the large window streamed from pinned host memory in 1-32 chunks, "
                        "against a plain copy of its records; schemes: the paper's GPU schemes (naive, "
                        "state-indexed lookup, density-aware partitioning, fused kernel) against this "
                        "engine's walk; adjoint: the adjoint workload's forward and backward alone (--events "
                        "scales it); glitch: the large workload's plain walk, then with glitch detection (--events "
                        "scales it); tiled: the large workload with the time-sliced walk at tile_min 0, 32768, "
                        "8192, 2048; patterns: the pattern-gate pin-threshold study alone; prep: the pass "
                        "that rebuilds event descriptors and gate tables after a load change, on the large "
                        "netlist; instead of the default run, one JSON line per case")
    return p.parse_args()


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if ws > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        backend = "nccl"
        try:
            import torch
            if not torch.cuda.is_available():
                backend = "gloo"
            else:
                torch.cuda.set_device(local)
        except Exception:
            backend = "gloo"
        dist.init_process_group(backend)
        pg = dist
    return ws, rank, local, pg


def max_over_ranks(pg, x: float) -> float:
    if pg is None:
        return x
    import torch
    dev = torch.device("cuda", torch.cuda.current_device()) if torch.cuda.is_available() else torch.device("cpu")
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def barrier(pg):
    if pg is not None:
        pg.barrier()


def config_of(args, cfg_name):
    import dataclasses
    import synth
    cfg = synth.CONFIGS[cfg_name]
    if args.events:
        cfg = dataclasses.replace(cfg, n_events=int(args.events), name=f"{cfg.name} ({args.events:,} events)")
    return cfg


def workload_desc(cfg, n_bins, n_events=0):
    cap = f", cap {cfg.cap:g}" if cfg.cap else ""
    return (f"{cfg.name}: {cfg.n_gates:,} gates, {n_events or cfg.n_events:,} events, Zipf {cfg.zipf_s}{cap}, "
            f"{cfg.window_ps / 1e6:g} us window, {cfg.bin_ps} ps bins ({n_bins:,} bins)")


def algorithmic_bytes(n_events, n_gates_active, n_gates, n_bins):
    """Bytes the walk must move: 8 per record read; per gate with events the
    cell id, load, 6 slews, CSR offset and initial state read (41 B) and three
    FP64 energies plus the final state written (25 B); 8 per bin (the
    {energy, leakage step} accumulator pair)."""
    return 8 * n_events + 66 * n_gates_active + 8 * n_bins


# ------------------------------------------------------------------ clocks
class ClockSampler:
    def __init__(self, gpu_index: int, enabled: bool):
        self.enabled = enabled
        self.proc = None
        self.path = None
        self.gpu = gpu_index

    def __enter__(self):
        if not self.enabled:
            return self
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.25)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.enabled or self.path is None:
            return None
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), float(parts[2]), parts[3:]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for n, v in zip(names, r[3][1:]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "power_w_max": max(r[2] for r in rows), "reasons": sorted(reasons), "samples": len(rows)}


# ------------------------------------------------------------------ CPU oracle sample
def oracle_sample(lib, net, counts, cfg, seed_ev, budget_s, rng_seed=0):
    """Time the FP64 oracle on randomly chosen gates of the workload (their
    events regenerated on the host) until ``budget_s`` seconds of CPU work."""
    import oracle
    import synth

    rng = np.random.default_rng(rng_seed)
    order = rng.permutation(cfg.n_gates)
    trace = synth.make_trace(net, counts, cfg.window_ps, seed_ev, cfg.tie_p, materialise=False)
    done_ev, done_g, spent = 0, 0, 0.0
    pos = 0
    chunk = 16
    while spent < budget_s and pos < len(order):
        gates = np.sort(order[pos:pos + chunk])
        pos += chunk
        off, rec = synth.gate_records(net, trace, gates)
        sub_net = synth.Netlist(net.cell[gates], net.load_ff[gates], np.ascontiguousarray(net.slew_ps[gates]),
                                net.n_pins[gates], net.level[gates], net.fanin[gates])
        sub_tr = synth.Trace(cfg.window_ps, off, rec, trace.init_state[gates], trace.seed, trace.tie24)
        t0 = time.perf_counter()
        oracle.walk(lib, sub_net, sub_tr, cfg.bin_ps)
        spent += time.perf_counter() - t0
        done_ev += int(off[-1])
        done_g += len(gates)
    return done_ev, done_g, spent


# The same sample on every host core: a pool of spawned processes (no fork
# after the GPU is in use), each building the workload once from its seeds and
# timing the oracle on its own random gates.
_POOL_STATE = {}


def _pool_init(cfg_name, events, seed_ev):
    import dataclasses

    import synth
    cfg = synth.CONFIGS[cfg_name]
    if events:
        cfg = dataclasses.replace(cfg, n_events=int(events))
    lib = synth.make_library(cfg.seed_lib)
    net = synth.make_netlist(lib, cfg.n_gates, cfg.seed_net)
    counts = synth.zipf_counts(cfg.n_gates, cfg.n_events, cfg.zipf_s, cfg.cap, cfg.seed_ev)
    _POOL_STATE.update(cfg=cfg, lib=lib, net=net, counts=counts, seed_ev=seed_ev)


def _pool_sample(job):
    budget_s, rng_seed = job
    st = _POOL_STATE
    return oracle_sample(st["lib"], st["net"], st["counts"], st["cfg"], st["seed_ev"], budget_s, rng_seed)


class OraclePool:
    """The oracle sample on n host processes at once; sample() returns
    (events, gates, aggregate events/s, seconds of CPU work per process)."""

    def __init__(self, cfg_name, events, seed_ev, n=None):
        import multiprocessing as mp

        import oracle
        oracle.build()  # once here, not concurrently in every worker
        self.n = n or os.cpu_count() or 1
        self.pool = mp.get_context("spawn").Pool(self.n, initializer=_pool_init,
                                                 initargs=(cfg_name, events, seed_ev))

    def sample(self, budget_s, seed_base=0):
        res = self.pool.map(_pool_sample, [(budget_s, 1000 * seed_base + w) for w in range(self.n)])
        ev = sum(r[0] for r in res)
        g = sum(r[1] for r in res)
        rate = sum(r[0] / r[2] for r in res if r[2] > 0)
        return ev, g, rate, max(r[2] for r in res)

    def close(self):
        self.pool.close()
        self.pool.join()


def run_reference(args, cfg_name):
    import synth
    ws, rank, local, pg = dist_init()
    if rank != 0:
        return
    cfg = config_of(args, cfg_name)
    lib = synth.make_library(cfg.seed_lib)
    net = synth.make_netlist(lib, cfg.n_gates, cfg.seed_net)
    counts = synth.zipf_counts(cfg.n_gates, cfg.n_events, cfg.zipf_s, cfg.cap, cfg.seed_ev)
    n_bins = cfg.window_ps // cfg.bin_ps
    total = args.steps + args.warmup
    per_step = max(0.05, min(args.cpu_seconds, 150.0 / max(total, 1)))
    ev_tot, g_tot, t_tot, rates = 0, 0, 0.0, []
    pool = OraclePool(cfg_name, args.events, cfg.seed_ev)
    try:
        for i in range(total):
            ev, g, rate, t = pool.sample(per_step, seed_base=i)
            if i >= args.warmup:
                ev_tot, g_tot, t_tot = ev_tot + ev, g_tot + g, t_tot + t
                rates.append(rate)
    finally:
        pool.close()
    value = statistics.mean(rates) if rates else 0.0
    sample = (f"FP64 oracle on {pool.n} host processes at once (one thread each), on {g_tot:,} randomly chosen "
              f"gates ({ev_tot:,} events, all {n_bins:,} bins) over {args.steps} steps of ~{per_step:.2f} s "
              f"of CPU work per process")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * t_tot / max(args.steps, 1), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": workload_desc(cfg, n_bins), "gates": cfg.n_gates, "events": cfg.n_events,
                      "bins": n_bins},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.n, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ------------------------------------------------------------------ our engine
def run_ours(args, cfg_name):
    import torch

    import synth
    from paper_2609_05960_gb300 import Engine, gtpower

    ws, rank, local, pg = dist_init()
    # the FP64 oracle on every host core, for each measured result's error (spawned workers)
    opool = None
    if rank == 0 and not args.no_oracle_check:
        from oracle import fullsize
        opool = fullsize.Pool()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    cfg = config_of(args, cfg_name)
    seed_ev = cfg.seed_ev + 1000 * rank
    lib = synth.make_library(cfg.seed_lib)
    net = synth.make_netlist(lib, cfg.n_gates, cfg.seed_net)
    counts = synth.zipf_counts(cfg.n_gates, cfg.n_events, cfg.zipf_s, cfg.cap, seed_ev)
    trace, rec = synth.make_trace_gpu(net, counts, cfg.window_ps, seed_ev, cfg.tie_p, device=dev)
    n_ev = trace.n_events
    n_bins = cfg.window_ps // cfg.bin_ps
    G = cfg.n_gates
    n_active = int((counts > 0).sum())

    eng = Engine(local)
    eng.load_library(lib)
    eng.load_netlist(net)
    ctx = eng.ctx
    off_d = torch.from_numpy(trace.offsets).to(dev)
    init_d = torch.from_numpy(trace.init_state).to(dev)
    wave = torch.empty(n_bins, dtype=torch.float64, device=dev)
    g_leak = torch.empty(G, dtype=torch.float64, device=dev)
    g_int = torch.empty_like(g_leak)
    g_sw = torch.empty_like(g_leak)
    g_cnt = torch.empty(G, dtype=torch.int64, device=dev)
    g_fin = torch.empty(G, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        gtpower.gtp_load_events(ctx, 0, cfg.window_ps, off_d, rec, init_d, borrow=True)
        gtpower.gtp_run_power(ctx, 0, cfg.bin_ps, wave, graph=True)
        gtpower.gtp_gate_energy(ctx, 0, g_leak, g_int, g_sw, g_cnt, g_fin)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    # the timed region records two CUDA events a run around the walk (timing level 2), in the run's graph
    eng.set_param("timing", 2)
    step()  # the graph of this timing level, captured before the timed region
    torch.cuda.synchronize(dev)
    eng.set_param("timing", 2)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local, not args.no_clocks) as clk:
        barrier(pg)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier(pg)
    ms = e0.elapsed_time(e1)
    clocks = clk.summary()
    n_timed = max(eng.get_param("n_timed"), 1)
    walk_s = eng.get_param("t_walk_ns") * 1e-9 / n_timed
    launches = eng.get_param("launches")
    # the other phases from a second pass with every phase's events (twelve a run, which lengthen a step)
    eng.set_param("timing", 1)
    for _ in range(min(args.steps, 50)):
        step()
    torch.cuda.synchronize(dev)
    n_ph = max(eng.get_param("n_timed"), 1)
    plan_s = eng.get_param("t_plan_ns") * 1e-9 / n_ph
    merge_s = eng.get_param("t_merge_ns") * 1e-9 / n_ph
    gate_s = eng.get_param("t_gate_pass_ns") * 1e-9 / n_ph
    eng.set_param("timing", 0)
    ms_max = max_over_ranks(pg, ms)
    value = ws * args.steps * n_ev / (ms_max * 1e-3)

    import json as _json
    peaks = {}
    pk_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk_path):
        peaks = _json.load(open(pk_path))
    peak = peaks.get("hbm_gbs")
    peak_src = "measured" if peak else "fallback"
    peak = peak or 6800.0
    alg = algorithmic_bytes(n_ev, n_active, G, n_bins)
    # a reference rate for the walk's bin updates: 8-byte reductions into as many hashed slots as bins
    red_peak = gtpower.gtp_measure_reductions(ctx, n_bins, 2)
    # and the window's own reduction stream alone (its records' bins, 8 records a thread), a floor for the walk
    replay_ms = gtpower.gtp_measure_replay(ctx, 0, cfg.bin_ps)
    achieved = alg / walk_s / 1e9 if walk_s > 0 else 0.0
    oracle_err = None
    if opool is not None:  # every bin and every gate of this run against the FP64 oracle
        from oracle import fullsize
        ref = opool.walk(fullsize.Workload.of(cfg, seed_ev=seed_ev), cfg.bin_ps)
        got = {"e_leak": g_leak.cpu().numpy(), "e_int": g_int.cpu().numpy(), "e_sw": g_sw.cpu().numpy(),
               "n_events": g_cnt.cpu().numpy(), "final_state": g_fin.cpu().numpy()}
        oracle_err = {**fullsize.bin_errors(wave.cpu().numpy(), ref["bins"], cfg.bin_ps),
                      **fullsize.gate_errors(got, ref)}
        del ref

    # ---- end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        rec_h = torch.empty((n_ev, 2), dtype=torch.int32, pin_memory=True)
        rec_h.copy_(rec)
        off_h = torch.from_numpy(trace.offsets).pin_memory()
        init_h = torch.from_numpy(trace.init_state).pin_memory()
        wave_h = torch.empty(n_bins, dtype=torch.float64, pin_memory=True)
        outs_h = [torch.empty(G, dtype=torch.float64, pin_memory=True) for _ in range(3)]
        cnt_h = torch.empty(G, dtype=torch.int64, pin_memory=True)
        fin_h = torch.empty(G, dtype=torch.uint8, pin_memory=True)

        # the packed transfer form (4.125 B a record), written once like the trace itself
        pk_h = torch.empty(gtpower.packed_words(n_ev), dtype=torch.int32, pin_memory=True)
        gtpower.gtp_pack_events(rec_h.numpy(), out=pk_h)

        def e2e_step(packed):
            # records streamed from pinned host memory in 8 chunks, copies overlapping the walk
            if packed:
                gtpower.gtp_run_power_streamed(ctx, 1, cfg.window_ps, off_h, pk_h, init_h, cfg.bin_ps, wave_h, 8,
                                               n_events=n_ev, packed=True)
            else:
                gtpower.gtp_run_power_streamed(ctx, 1, cfg.window_ps, off_h, rec_h, init_h, cfg.bin_ps, wave_h, 8)
            gtpower.gtp_gate_energy(ctx, 1, outs_h[0], outs_h[1], outs_h[2], cnt_h, fin_h)

        def time_e2e(packed, trials=5):
            # the host link and host memory are shared with the machine's other jobs: the median of a few
            # trials of e2e_steps steps each keeps a transient slowdown out of the figure
            e2e_step(packed)
            torch.cuda.synchronize(dev)
            times = []
            for _ in range(trials):
                barrier(pg)
                t0 = time.perf_counter()
                for _ in range(args.e2e_steps):
                    e2e_step(packed)
                torch.cuda.synchronize(dev)
                times.append(max_over_ranks(pg, time.perf_counter() - t0))
            return statistics.median(times)

        d2h = n_bins * 8 + G * (8 * 3 + 8 + 1)
        t_e2e8 = time_e2e(False)
        h2d8 = rec_h.numel() * 4 + off_h.numel() * 8 + init_h.numel()
        t_e2e = time_e2e(True)
        h2d = pk_h.numel() * 4 + off_h.numel() * 8 + init_h.numel()
        e2e = {"value": ws * args.e2e_steps * n_ev / t_e2e8, "unit": UNIT, "h2d_bytes_per_step": int(h2d8),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": 1e3 * t_e2e8 / args.e2e_steps,
               "input": "the ABI's 8-byte records from pinned host memory, streamed in 8 chunks "
                        "(gtp_run_power_streamed), then per-gate results to host memory (gtp_gate_energy)",
               "timing": f"median of 5 trials of {args.e2e_steps} steps, host clock around CUDA-synchronised steps",
               "packed": {"value": ws * args.e2e_steps * n_ev / t_e2e, "h2d_bytes_per_step": int(h2d),
                          "ms_per_step": 1e3 * t_e2e / args.e2e_steps,
                          "input": "the packed transfer form (gtp_pack_events, 4.125 B a record), streamed in 8 "
                                   "chunks; the packing runs once before the timed region, like writing the trace"}}
        del rec_h, pk_h

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        pool = OraclePool(cfg_name, args.events, seed_ev)
        try:
            ev, g, rate, t = pool.sample(args.cpu_seconds)
        finally:
            pool.close()
        cpu = {"value": rate, "unit": UNIT, "cores": pool.n, "kind": "oracle", "per_core_value": rate / pool.n,
               "sample": f"FP64 oracle on {pool.n} host processes at once (one thread each), on {g:,} randomly "
                         f"chosen gates of this workload ({ev:,} events, all {n_bins:,} bins), {t:.1f} s of CPU "
                         f"work per process"}

    extras = {}
    if rank == 0 and not args.no_extras and cfg_name == "large" and not args.events:
        xs = max(3, min(args.steps // 10, 10))
        wl_large = None
        if opool is not None:
            from oracle import fullsize
            wl_large = fullsize.Workload.of(cfg, seed_ev=seed_ev)
        extras["load_change"] = measure_load_change(eng, dev, cfg, wave, n_ev, ms_max / args.steps, xs, lib, net)
        extras["glitch"] = measure_glitch(eng, dev, cfg, wave, walk_s * 1e3, n_ev, xs, opool, wl_large)
        extras["components"] = measure_components(eng, dev, cfg, walk_s * 1e3, n_ev, xs, opool, wl_large)
        if not args.no_patterns:
            extras["patterns"] = measure_patterns(eng, dev, cfg, wave, n_ev, xs)
        del rec
        torch.cuda.empty_cache()
        extras["batched"] = measure_batched(eng, dev, xs, peak, value, opool)
        extras["adjoint"] = measure_adjoint(eng, dev, xs, peak=peak, opool=opool)
        if not args.no_stress:
            extras["stress"] = measure_stress(eng, dev, xs, peak, opool)
    if opool is not None:
        opool.close()

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_desc(cfg, n_bins), "gates": G, "events": n_ev, "bins": n_bins,
                       "records_bytes": 8 * n_ev, "l2_flush": "none: inputs (records) larger than L2",
                       "kernel": "density-split walk (dense gates in per-gate segments, sparse gates one per thread), one launch",
                       "run_power": "CUDA-graph replay (phase events recorded inside the graph)",
                       "records_per_thread": eng.get_param("records_per_thread"),
                       "dense_min": eng.get_param("dense_min")},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "kernel": "k_walk",
                         "traffic": None if args.events else WALK_TRAFFIC.get(
                             (cfg.name, eng.get_param("records_per_thread"), eng.get_param("dense_min"))),
                         "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one walk launch of "
                                           "this kernel on this workload and plan",
                         "peak_kind": "burst copy bandwidth (the walk is timed alone, per launch)",
                         "algorithmic_bytes": alg, "walk_ms": walk_s * 1e3, "peak_source": peak_src,
                         "frac_of_nominal_8tbs": achieved / 8000.0,
                         "l2_reductions": {"achieved_per_s": n_ev / walk_s if walk_s > 0 else 0.0,
                                           "reference_rate_per_s": red_peak,
                                           "ratio": (n_ev / walk_s) / red_peak if walk_s > 0 and red_peak > 0
                                           else 0.0,
                                           "replay_ms": replay_ms,
                                           "walk_over_replay": walk_s * 1e3 / replay_ms if replay_ms > 0 else None,
                                           "note": "about one bin reduction per event; the reference rate is "
                                                   "gtp_measure_reductions (8-byte reductions spread by a hash "
                                                   "over as many slots as bins, in this run), not a roofline: "
                                                   "the walk's own updates are local in time; replay_ms is "
                                                   "gtp_measure_replay, the window's own records' bin reductions "
                                                   "alone (reading the records, one reduction per distinct bin of "
                                                   "8 consecutive records), a floor for the walk"}},
            "oracle_error": oracle_err,
            "phases_ms": {"prepare": gate_s * 1e3, "scatter": plan_s * 1e3, "walk": walk_s * 1e3,
                          "merge": merge_s * 1e3,
                          "how": "walk: CUDA events around the walk in the timed region's graph; the others "
                                 "from a second pass of up to 50 steps with events around every phase"},
            "e2e": e2e,
            "cpu_baseline": cpu,
            "gpu_launches": int(launches),
            "clocks": clocks,
        }
        out.update(extras)
        print(json.dumps(out), flush=True)
    eng.close()


# ------------------------------------------------------------------ batched and adjoint forms
def _events_per_s(fn, steps, dev):
    import torch
    fn()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        fn()
    e1.record()
    torch.cuda.synchronize(dev)
    return e0.elapsed_time(e1) / steps  # ms


def roofline(alg_bytes, walk_ms, peak):
    """HBM roofline of a walk: its algorithmic bytes over its measured time."""
    ach = alg_bytes / (walk_ms * 1e-3) / 1e9 if walk_ms > 0 else 0.0
    return {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak if peak else None,
            "algorithmic_bytes": int(alg_bytes), "walk_ms": walk_ms}


def _timed_walk(eng, fn, steps, dev):
    """(ms per call, walk-phase ms per call) of fn, with the engine's
    walk-only timing on (two CUDA events a run)."""
    eng.set_param("timing", 2)
    ms = _events_per_s(fn, steps, dev)
    n_t = max(eng.get_param("n_timed"), 1)
    walk_ms = eng.get_param("t_walk_ns") * 1e-6 / n_t
    eng.set_param("timing", 0)
    return ms, walk_ms


def _gate_results(eng, w, glitch=False):
    ge = eng.gate_energy(w, device=False)
    if glitch:
        ge["e_gl"] = eng.gate_glitch(w, device=False)
    return ge


def _oracle_errors(opool, wl, bin_ps, wave, ge, keys=("e_leak", "e_int", "e_sw")):
    from oracle import fullsize
    ref = opool.walk(wl, bin_ps)
    w = wave.cpu().numpy() if hasattr(wave, "cpu") else np.asarray(wave)
    return {**fullsize.bin_errors(w, ref["bins"], bin_ps), **fullsize.gate_errors(ge, ref, keys)}


def measure_load_change(eng, dev, cfg, wave, n_ev, step_ms, steps, lib, net):
    """The step of an optimisation loop over the large window (slot 0): a new
    load per gate (gtp_set_load, which rebuilds the interpolation
    coordinates and the per-gate energy tables) and then the run."""
    import torch

    from paper_2609_05960_gb300 import gtpower

    base = torch.from_numpy(np.ascontiguousarray(net.load_ff, dtype=np.float32)).to(dev)
    k = [0]

    def step():
        k[0] += 1
        gtpower.gtp_set_load(eng.ctx, base * (1.0 + 1e-3 * (k[0] & 1)))
        gtpower.gtp_run_power(eng.ctx, 0, cfg.bin_ps, wave, graph=True)

    for _ in range(3):
        step()
    torch.cuda.synchronize(dev)
    ms = _events_per_s(step, steps, dev)
    # the preparation pass alone (CUDA events around its launch, timing level 1, a separate pass)
    eng.set_param("timing", 1)
    for _ in range(10):
        step()
    torch.cuda.synchronize(dev)
    prep_ms = eng.get_param("t_prep_ns") * 1e-6 / max(eng.get_param("n_timed"), 1)
    eng.set_param("timing", 0)
    gtpower.gtp_set_load(eng.ctx, base)
    alg = gate_prep_bytes(lib, net)
    return {"ms_per_step": ms, "value": n_ev / (ms * 1e-3), "unit": UNIT,
            "over_plain_step": ms / step_ms if step_ms > 0 else None,
            "what": "gtp_set_load (new load per gate) + gtp_run_power, whose first launch rebuilds the event "
                    "descriptors and per-gate energy tables (k_gate_prep), as in an optimisation loop",
            "gate_prep": {"ms": prep_ms, "algorithmic_bytes": alg,
                          "roofline": roofline(alg, prep_ms, peak_gbs()) if prep_ms > 0 else None,
                          "bytes": "per gate: cell 4 + load 4 + slews 8 x stride read; descriptors 16 x "
                                   "2 (stride + 1) and the cell's (n_in + 1) 2^n_in table entries x 4 written"}}


def gate_prep_bytes(lib, net):
    """Algorithmic bytes of one preparation pass over the netlist."""
    stride = net.slew_stride
    n_in = np.asarray(lib.n_in)[np.asarray(net.cell)]
    entries = np.where(n_in <= 3, (n_in + 1) << n_in, 0)
    G = len(n_in)
    return int(G * (8 + 8 * stride + 16 * 2 * (stride + 1)) + 4 * int(entries.sum()))


def peak_gbs():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        return json.load(open(path)).get("hbm_gbs") or 6800.0
    return 6800.0


def measure_batched(eng, dev, steps, peak, plain_value, opool=None):
    """64 windows of uneven length over a 200k-gate netlist: autotuned plan,
    one persistent launch per run, replayed from a CUDA graph.  Reported with
    its walk's roofline, against the plain large window's rate (one window of
    200M events), against the same windows run one at a time, and each
    window's error against the oracle."""
    import torch

    import synth
    from paper_2609_05960_gb300 import gtpower

    lib = synth.make_library(1)
    net = synth.make_netlist(lib, synth.BATCHED_GATES, 2)
    eng.load_library(lib)
    eng.load_netlist(net)
    wins = synth.batched_windows()
    keep, total, alg, specs = [], 0, 0, []
    for w, spec in enumerate(wins):
        counts = synth.zipf_counts(synth.BATCHED_GATES, spec["n_events"], 1.2, 100_000, spec["seed"])
        tr, rec = synth.make_trace_gpu(net, counts, spec["window_ps"], spec["seed"], device=dev)
        off = torch.from_numpy(tr.offsets).to(dev)
        init = torch.from_numpy(tr.init_state).to(dev)
        eng.load_events(w, window_ps=spec["window_ps"], offsets=off, records=rec, init_state=init, borrow=True)
        keep.append((rec, off, init))
        total += tr.n_events
        alg += algorithmic_bytes(tr.n_events, int((counts > 0).sum()), synth.BATCHED_GATES, spec["window_ps"] // 10)
        specs.append((spec, int(counts.sum())))
    ids = list(range(len(wins)))
    tuned_ms = eng.autotune(ids, 10, iters=2)
    plan = {k: eng.get_param(k) for k in ("records_per_thread", "ctas_per_sm", "dense_min")}
    outs = [torch.empty(s["window_ps"] // 10, dtype=torch.float64, device=dev) for s in wins]
    run = lambda: gtpower.gtp_run_power_batched(eng.ctx, ids, 10, outs, graph=True)
    run()
    ms_b, walk_ms = _timed_walk(eng, run, steps, dev)
    ref = [o.clone() for o in outs]
    ms_p = _events_per_s(lambda: [gtpower.gtp_run_power(eng.ctx, w, 10, outs[w]) for w in ids], steps, dev)
    diff = max(float(((o - r).abs() / r.abs()).max()) for o, r in zip(outs, ref))
    err = None
    if opool is not None:
        from oracle import fullsize
        worst = {}
        for w, (spec, n) in enumerate(specs):
            wl = fullsize.Workload(synth.BATCHED_GATES, spec["n_events"], 1.2, 100_000, spec["window_ps"], 1, 2,
                                   spec["seed"])
            e = _oracle_errors(opool, wl, 10, ref[w], _gate_results(eng, w))
            for k, v in e.items():
                if k.startswith("max_rel") or k.endswith("mismatches"):
                    worst[k] = max(worst.get(k, 0), v)
            worst["mean_rel_bin_err"] = worst.get("mean_rel_bin_err", 0.0) + e["mean_rel_bin_err"] * e["bins"]
            worst["bins"] = worst.get("bins", 0) + e["bins"]
        worst["mean_rel_bin_err"] /= max(worst["bins"], 1)
        err = worst
    del keep
    value = total / (ms_b * 1e-3)
    return {"workload": f"{len(wins)} windows over {synth.BATCHED_GATES:,} gates, {total:,} events, "
                        f"1k-100k bins of 10 ps", "events": total, "ms_per_run": ms_b,
            "value": value, "unit": UNIT, "roofline": roofline(alg, walk_ms, peak),
            "vs_one_plain_window": value / plain_value if plain_value else None,
            "one_plain_window": "the large window (200M events in one window) timed above",
            "separate_runs_ms": ms_p, "speedup_vs_separate_runs": ms_p / ms_b,
            "max_rel_diff_vs_separate_runs": diff, "oracle_error": err, "autotuned_plan": plan,
            "autotune_best_ms": tuned_ms, "graph": True}


# pattern gates beside the large window: cells of 5 to 21 pins given by state patterns
PATTERN_GATES = 2_000
PATTERN_EVENTS = 6_000_000
PATTERN_WEIGHTS = [0.0, 0.25, 0.2, 0.2, 0.15, 0.1, 0.05, 0.05]  # over synth.patterns.PATTERN_CELLS (4-pin AOI3P: none)


def measure_patterns(eng, dev, cfg, wave, n_ev, steps):
    """The large window (slot 0) plus 2,000 gates of wide cells given by
    state patterns (0.2 % of the gates) carrying 6M events (3 %), and the
    state-indexed threshold swept in the spirit of the paper's pin-threshold
    study (Sec. 6.4.1: thresholds 4 to 32): per threshold, the share of gates
    and events that take the traversal fallback, the pattern walk's time,
    the run's time against the plain window, and the index memory.  Every
    threshold gives the same per-gate results; sampled pattern gates are
    checked against the oracle (oracle/patterns.py)."""
    import torch

    from oracle import patterns as opat
    from paper_2609_05960_gb300 import gtpower
    from synth import patterns as spat

    plib = spat.make_pattern_library(cfg.seed_lib)
    pnet = spat.make_pattern_netlist(plib, PATTERN_GATES, seed=cfg.seed_net, weights=PATTERN_WEIGHTS)
    counts = synth_zipf(PATTERN_GATES, PATTERN_EVENTS, 1.2, 100_000, cfg.seed_ev + 100)
    ptr = spat.make_pattern_trace(pnet, counts, cfg.window_ps, cfg.seed_ev + 100, tie_p=0.02, clock_pin_share=0.3)
    run = lambda: gtpower.gtp_run_power(eng.ctx, 0, cfg.bin_ps, wave, graph=True)
    for _ in range(3):
        run()
    torch.cuda.synchronize(dev)
    # the plain run with the same phase events as the rows below; the median of three trials
    eng.set_param("timing", 1)
    plain_run_ms = statistics.median(_events_per_s(run, steps, dev) for _ in range(3))
    eng.set_param("timing", 0)
    eng.load_pattern_cells(plib)
    eng.load_pattern_netlist(pnet)
    eng.load_pattern_events(0, ptr)
    pins = (plib.n_in + 1)[pnet.cell]
    G_all = eng.n_gates + PATTERN_GATES
    E_all = n_ev + PATTERN_EVENTS
    # oracle sample: a few gates of every cell, about 150k events
    rng = np.random.default_rng(11)
    sample = []
    for c in range(plib.n_cells):
        idx = np.flatnonzero(pnet.cell == c)
        idx = idx[counts[idx] <= 40_000]
        sample += list(rng.choice(idx, size=min(8, len(idx)), replace=False)) if len(idx) else []
    sample = np.sort(np.array(sample, np.int64))
    ref = opat.walk(plib, pnet, ptr, cfg.bin_ps, gates=sample)
    rows, first = [], None
    for thr in (0, 4, 8, 12, 16, 20, 24):
        eng.set_param("sipl_max_pins", thr)
        for _ in range(3):
            run()
        torch.cuda.synchronize(dev)
        eng.set_param("timing", 1)
        ms = _events_per_s(run, steps, dev)
        n_t = max(eng.get_param("n_timed"), 1)
        pat_ms = eng.get_param("t_pattern_ns") * 1e-6 / n_t
        eng.set_param("timing", 0)
        pe = eng.pattern_gate_energy(0)
        err = {k: float(np.max(np.abs(pe[k][sample] - ref[k]) / np.maximum(np.abs(ref[k]), 1e-4)))
               for k in ("e_leak", "e_int", "e_sw")}
        err["count_mismatches"] = int(np.sum(pe["n_events"][sample] != ref["n_events"]))
        err["state_mismatches"] = int(np.sum(pe["final_state"][sample] != ref["final_state"]))
        if first is None:
            first = pe
        fb = pins > thr
        rows.append({"sipl_max_pins": thr, "fallback_gates": int(fb.sum()),
                     "fallback_gate_share": float(fb.sum()) / G_all,
                     "fallback_event_share": float(counts[fb].sum()) / E_all,
                     "pattern_walk_ms": pat_ms, "pattern_events_per_s": PATTERN_EVENTS / (pat_ms * 1e-3),
                     "ms_per_run": ms, "over_plain_run": ms / plain_run_ms,
                     "indexed_cells": eng.get_param("pattern_indexed_cells"),
                     "index_bytes": eng.get_param("pattern_index_bytes"),
                     "max_rel_diff_vs_threshold_0": float(max(
                         np.max(np.abs(pe[k] - first[k]) / np.maximum(np.abs(first[k]), 1e-4))
                         for k in ("e_leak", "e_int", "e_sw"))),
                     "oracle_error_sampled_gates": err})
    eng.set_param("sipl_max_pins", -1)
    return {"workload": f"the large window plus {PATTERN_GATES:,} pattern gates (cells of 5-21 pins: "
                        f"5 25%, 6 20%, 9 20%, 12 15%, 16 10%, 20 5%, 21 5%) carrying {PATTERN_EVENTS:,} events "
                        f"(Zipf 1.2, cap 1e5, clock pin 30%, ties 2%)",
            "oracle_sample": f"{len(sample)} pattern gates, {int(counts[sample].sum()):,} events, per-gate results",
            "plain_run_ms": plain_run_ms,
            "sweep": rows}


def synth_zipf(n, total, s, cap, seed):
    import synth
    return synth.zipf_counts(n, total, s, cap, seed)


def measure_glitch(eng, dev, cfg, wave, walk_plain_ms, n_ev, steps, opool=None, wl=None):
    """The same window (still loaded in slot 0) with clock-cycle glitch
    detection at a 1 GHz clock (output transition times 10-200 ps, seeded):
    run time, walk time against the plain walk, the glitch share of the
    dynamic energy, and the error against the oracle."""
    import dataclasses

    import torch

    from paper_2609_05960_gb300 import gtpower

    clock_ps = 1000
    rng = np.random.default_rng(7)
    out_slew = rng.uniform(10.0, 200.0, (eng.n_gates, 2)).astype(np.float32)
    eng.set_glitch(clock_ps, out_slew)
    run = lambda: gtpower.gtp_run_power(eng.ctx, 0, cfg.bin_ps, wave, graph=True)
    for _ in range(3):
        run()
    torch.cuda.synchronize(dev)
    ms, walk_ms = _timed_walk(eng, run, steps, dev)
    ge = _gate_results(eng, 0, glitch=True)
    dyn = float(ge["e_int"].sum() + ge["e_sw"].sum() + ge["e_gl"].sum())
    err = None
    if opool is not None and wl is not None:
        err = _oracle_errors(opool, dataclasses.replace(wl, clock_ps=clock_ps), cfg.bin_ps, wave, ge,
                             ("e_leak", "e_int", "e_sw", "e_gl"))
    eng.set_glitch(0)
    return {"clock_ps": clock_ps, "ms_per_run": ms, "value": n_ev / (ms * 1e-3), "unit": UNIT, "walk_ms": walk_ms,
            "walk_over_plain": walk_ms / walk_plain_ms,
            "glitch_share_of_dynamic_energy": float(ge["e_gl"].sum()) / dyn if dyn > 0 else 0.0,
            "out_slew": "uniform 10-200 ps per gate and edge, seed 7", "oracle_error": err}


def measure_components(eng, dev, cfg, walk_plain_ms, n_ev, steps, opool=None, wl=None):
    """The same window (slot 0) with the per-component waveforms (leakage,
    internal, switching, glitch rows, on the device) as well as the total:
    run time, walk time against the plain walk, and each row's error against
    the oracle's component bins."""
    import torch

    from paper_2609_05960_gb300 import gtpower

    nb = cfg.window_ps // cfg.bin_ps
    comp = torch.empty((4, nb), dtype=torch.float64, device=dev)
    total = torch.empty(nb, dtype=torch.float64, device=dev)
    run = lambda: gtpower.gtp_run_power_components(eng.ctx, 0, cfg.bin_ps, comp, total)
    for _ in range(3):
        run()
    torch.cuda.synchronize(dev)
    ms, walk_ms = _timed_walk(eng, run, steps, dev)
    rel = float(((comp.sum(0) - total).abs() / total.abs()).max())
    err = None
    if opool is not None and wl is not None:
        from oracle import fullsize
        ref = opool.walk(wl, cfg.bin_ps, components=True)
        c = comp.cpu().numpy()
        err = {"total": fullsize.bin_errors(total.cpu().numpy(), ref["bins"], cfg.bin_ps)}
        for i, name in enumerate(("leakage", "internal", "switching")):
            err[name] = fullsize.bin_errors(c[i], ref["comp_bins"][i], cfg.bin_ps)
        err["glitch_max_abs_w"] = float(np.abs(c[3]).max())
    return {"ms_per_run": ms, "value": n_ev / (ms * 1e-3), "unit": UNIT, "walk_ms": walk_ms,
            "walk_over_plain": walk_ms / walk_plain_ms, "max_rel_sum_of_components_vs_total": rel,
            "oracle_error": err}


def adjoint_bytes(n_events, n_active, n_gates, n_bins):
    """Bytes the adjoint walk must move: 8 per record; per gate with events
    the cell id, load, 6 slews, CSR offset and initial state (41 B); the
    per-bin gradient table read once (8 B a bin: dL/dE and its prefix G); dC
    written (4 B a gate)."""
    return 8 * n_events + 41 * n_active + 8 * n_bins + 4 * n_gates


def measure_adjoint(eng, dev, steps, n_events=0, peak=None, opool=None, cfg_name="adjoint"):
    """500k gates, 100M events (or n_events), 5 us, 10 ps bins: the adjoint
    walk (gradients of sum P^2 + tau*LSE(P/tau)) against the forward walk on
    the same window, both with their rooflines; the forward waveform and
    per-gate results against the oracle in full, the load gradients of
    sampled gates against the oracle's adjoint."""
    import dataclasses

    import torch

    import oracle
    import synth
    from paper_2609_05960_gb300 import gtpower, peak_loss

    cfg = synth.CONFIGS[cfg_name]
    if n_events:
        cfg = dataclasses.replace(cfg, n_events=n_events)
    lib = synth.make_library(cfg.seed_lib)
    net = synth.make_netlist(lib, cfg.n_gates, cfg.seed_net)
    eng.load_library(lib)
    eng.load_netlist(net)
    counts = synth.zipf_counts(cfg.n_gates, cfg.n_events, cfg.zipf_s, cfg.cap, cfg.seed_ev)
    tr, rec = synth.make_trace_gpu(net, counts, cfg.window_ps, cfg.seed_ev, device=dev)
    off = torch.from_numpy(tr.offsets).to(dev)
    init = torch.from_numpy(tr.init_state).to(dev)
    eng.load_events(0, window_ps=cfg.window_ps, offsets=off, records=rec, init_state=init, borrow=True)
    nb = cfg.window_ps // cfg.bin_ps
    wave = torch.empty(nb, dtype=torch.float64, device=dev)
    gtpower.gtp_run_power(eng.ctx, 0, cfg.bin_ps, wave)
    P = wave.clone().requires_grad_(True)
    peak_loss(P).backward()
    g = P.grad.to(torch.float32).contiguous()
    kw = dict(dtype=torch.float32, device=dev)
    dC, de, dl = torch.empty(cfg.n_gates, **kw), torch.empty(lib.n_cells, **kw), torch.empty(lib.n_cells, **kw)
    ms_f, walk_f = _timed_walk(eng, lambda: gtpower.gtp_run_power(eng.ctx, 0, cfg.bin_ps, wave), steps, dev)
    ms_b, walk_b = _timed_walk(eng, lambda: gtpower.gtp_run_power_backward(eng.ctx, 0, cfg.bin_ps, g, dC, de, dl),
                               steps, dev)
    n = tr.n_events
    act = int((counts > 0).sum())
    out = {"workload": workload_desc(cfg, nb, n), "events": n, "ms_per_backward": ms_b, "value": n / (ms_b * 1e-3),
           "unit": UNIT, "forward_ms": ms_f, "forward_value": n / (ms_f * 1e-3), "backward_over_forward": ms_b / ms_f,
           "walk_backward_ms": walk_b, "walk_forward_ms": walk_f, "walk_backward_over_forward": walk_b / walk_f,
           "loss": "sum P^2 + tau*logsumexp(P/tau), P in mW, tau = 0.01*mean(P)"}
    if peak:
        out["roofline_backward"] = roofline(adjoint_bytes(n, act, cfg.n_gates, nb), walk_b, peak)
        out["roofline_forward"] = roofline(algorithmic_bytes(n, act, cfg.n_gates, nb), walk_f, peak)
    if opool is not None:
        from oracle import fullsize
        out["oracle_error_forward"] = _oracle_errors(opool, fullsize.Workload.of(cfg), cfg.bin_ps, wave,
                                                     _gate_results(eng, 0))
        rng = np.random.default_rng(0)
        gates = np.unique(np.concatenate([np.argsort(-counts, kind="stable")[:8],
                                          rng.choice(cfg.n_gates, 400, replace=False)]))
        off_s, rec_s = synth.gate_records(net, tr, gates)
        sub_net = synth.Netlist(net.cell[gates], net.load_ff[gates], np.ascontiguousarray(net.slew_ps[gates]),
                                net.n_pins[gates], net.level[gates], net.fanin[gates])
        sub_tr = synth.Trace(tr.window_ps, off_s, rec_s, tr.init_state[gates], tr.seed, tr.tie24)
        rC, _, _ = oracle.adjoint(lib, sub_net, sub_tr, cfg.bin_ps, g.cpu().numpy().astype(np.float64))
        got = dC.cpu().numpy()[gates]
        scale = float(np.abs(rC).max())
        out["oracle_error_dC"] = {"gates": int(len(gates)),
                                  "max_abs_err_over_max": float(np.abs(got - rC).max() / scale) if scale else 0.0,
                                  "bar": "|dC - oracle| <= 1e-4 |oracle| + 1e-5 max|oracle|",
                                  "within_bar": bool(np.all(np.abs(got - rC) <= 1e-4 * np.abs(rC) + 1e-5 * scale))}
    del rec, off, init
    return out


def measure_stress(eng, dev, steps, peak, opool=None):
    """The stress workload (10M gates, 2B events, 16 GB of records, Zipf 1.5,
    100 us in 10M bins of 10 ps) in its three forms on one GPU: the plain
    run, the batched run of four windows of 500M events each, and the adjoint
    (gradients of sum P^2 + tau*LSE(P/tau)); each with events/s, its walk's
    roofline and its error against the oracle over every bin and gate."""
    import dataclasses

    import torch

    import synth
    from paper_2609_05960_gb300 import gtpower, peak_loss

    cfg = synth.CONFIGS["stress"]
    lib = synth.make_library(cfg.seed_lib)
    net = synth.make_netlist(lib, cfg.n_gates, cfg.seed_net)
    eng.load_library(lib)
    eng.load_netlist(net)
    for k in ("records_per_thread", "ctas_per_sm", "dense_min"):
        eng.set_param(k, -1)
    nb = cfg.window_ps // cfg.bin_ps
    counts = synth.zipf_counts(cfg.n_gates, cfg.n_events, cfg.zipf_s, cfg.cap, cfg.seed_ev)
    tr, rec = synth.make_trace_gpu(net, counts, cfg.window_ps, cfg.seed_ev, device=dev)
    off = torch.from_numpy(tr.offsets).to(dev)
    init = torch.from_numpy(tr.init_state).to(dev)
    eng.load_events(0, window_ps=cfg.window_ps, offsets=off, records=rec, init_state=init, borrow=True)
    wave = torch.empty(nb, dtype=torch.float64, device=dev)
    run = lambda: gtpower.gtp_run_power(eng.ctx, 0, cfg.bin_ps, wave, graph=True)
    for _ in range(3):
        run()
    torch.cuda.synchronize(dev)
    ms, walk = _timed_walk(eng, run, steps, dev)
    n = tr.n_events
    act = int((counts > 0).sum())
    plain = {"workload": workload_desc(cfg, nb, n), "events": n, "ms_per_run": ms, "value": n / (ms * 1e-3),
             "unit": UNIT, "roofline": roofline(algorithmic_bytes(n, act, cfg.n_gates, nb), walk, peak)}
    from oracle import fullsize
    if opool is not None:
        plain["oracle_error"] = _oracle_errors(opool, fullsize.Workload.of(cfg), cfg.bin_ps, wave,
                                               _gate_results(eng, 0))
    # adjoint form on the same window
    P = wave.clone().requires_grad_(True)
    peak_loss(P).backward()
    g = P.grad.to(torch.float32).contiguous()
    kw = dict(dtype=torch.float32, device=dev)
    dC, de, dl = torch.empty(cfg.n_gates, **kw), torch.empty(lib.n_cells, **kw), torch.empty(lib.n_cells, **kw)
    ms_b, walk_b = _timed_walk(eng, lambda: gtpower.gtp_run_power_backward(eng.ctx, 0, cfg.bin_ps, g, dC, de, dl),
                               steps, dev)
    adj = {"events": n, "ms_per_backward": ms_b, "value": n / (ms_b * 1e-3), "unit": UNIT,
           "backward_over_forward": ms_b / ms, "walk_backward_over_forward": walk_b / walk,
           "roofline": roofline(adjoint_bytes(n, act, cfg.n_gates, nb), walk_b, peak)}
    del rec, off, init, P, g, dC
    torch.cuda.empty_cache()
    # batched form: four windows of 500M events
    keep, wls, alg, total = [], [], 0, 0
    for w in range(4):
        c4 = dataclasses.replace(cfg, n_events=cfg.n_events // 4, seed_ev=cfg.seed_ev + 10 * (w + 1))
        cnt = synth.zipf_counts(c4.n_gates, c4.n_events, c4.zipf_s, c4.cap, c4.seed_ev)
        t4, r4 = synth.make_trace_gpu(net, cnt, c4.window_ps, c4.seed_ev, device=dev)
        o4 = torch.from_numpy(t4.offsets).to(dev)
        i4 = torch.from_numpy(t4.init_state).to(dev)
        eng.load_events(w, window_ps=c4.window_ps, offsets=o4, records=r4, init_state=i4, borrow=True)
        keep.append((r4, o4, i4))
        wls.append(fullsize.Workload.of(c4))
        alg += algorithmic_bytes(t4.n_events, int((cnt > 0).sum()), c4.n_gates, nb)
        total += t4.n_events
    outs = [torch.empty(nb, dtype=torch.float64, device=dev) for _ in range(4)]
    runb = lambda: gtpower.gtp_run_power_batched(eng.ctx, [0, 1, 2, 3], cfg.bin_ps, outs, graph=True)
    runb()
    ms4, walk4 = _timed_walk(eng, runb, steps, dev)
    bat = {"windows": 4, "events": total, "ms_per_run": ms4, "value": total / (ms4 * 1e-3), "unit": UNIT,
           "roofline": roofline(alg, walk4, peak), "vs_plain": (total / ms4) / (n / ms)}
    if opool is not None:
        errs = [_oracle_errors(opool, wls[w], cfg.bin_ps, outs[w], _gate_results(eng, w)) for w in range(4)]
        bat["oracle_error"] = {k: max(e[k] for e in errs) for k in errs[0] if k.startswith("max_rel")
                               or k.endswith("mismatches")}
        bat["oracle_error"]["bins"] = sum(e["bins"] for e in errs)
    del keep, outs
    torch.cuda.empty_cache()
    return {"plain": plain, "adjoint": adj, "batched": bat}


def run_contention_sweep(args):
    """Bin-update contention: every gate equally active, 1, 2, 4 and 8 events
    per gate per 1k bins, over 250k gates and 1M bins of 10 ps (up to 2B
    events, 2,000 events per bin).  Each density runs with the autotuned
    plan; one JSON line each, timed like the main bench (CUDA events around
    graph-replayed gtp_run_power calls, phase timing for the walk)."""
    import torch

    import synth
    from paper_2609_05960_gb300 import Engine, gtpower

    dev = torch.device("cuda", 0)
    G, window_ps, bin_ps = 250_000, 10_000_000, 10
    n_bins = window_ps // bin_ps
    lib = synth.make_library(1)
    net = synth.make_netlist(lib, G, 2)
    eng = Engine(0)
    eng.load_library(lib)
    eng.load_netlist(net)
    wave = torch.empty(n_bins, dtype=torch.float64, device=dev)
    for k in (1, 2, 4, 8):
        counts = np.full(G, k * n_bins // 1000, np.int64)
        tr, rec = synth.make_trace_gpu(net, counts, window_ps, 40 + k, device=dev)
        off = torch.from_numpy(tr.offsets).to(dev)
        init = torch.from_numpy(tr.init_state).to(dev)
        eng.load_events(0, window_ps=window_ps, offsets=off, records=rec, init_state=init, borrow=True)
        for key in ("records_per_thread", "ctas_per_sm", "dense_min"):
            eng.set_param(key, -1)
        best = gtpower.gtp_autotune(eng.ctx, [0], bin_ps, 3)
        run = lambda: gtpower.gtp_run_power(eng.ctx, 0, bin_ps, wave, graph=True)
        for _ in range(max(args.warmup, 3)):
            run()
        torch.cuda.synchronize(dev)
        eng.set_param("timing", 1)
        steps = max(3, min(args.steps, 20))
        ms = _events_per_s(run, steps, dev)
        n_t = max(eng.get_param("n_timed"), 1)
        walk_ms = eng.get_param("t_walk_ns") * 1e-6 / n_t
        eng.set_param("timing", 0)
        n = int(tr.n_events)
        print(json.dumps({
            "sweep": "contention", "events_per_gate_per_1k_bins": k, "gates": G, "bins": n_bins,
            "events": n, "events_per_bin": n / n_bins, "ms_per_run": ms, "value": n / (ms * 1e-3), "unit": UNIT,
            "walk_ms": walk_ms, "walk_events_per_s": n / (walk_ms * 1e-3),
            "autotuned_plan": {key: eng.get_param(key) for key in ("records_per_thread", "dense_min")},
            "autotune_best_ms": best, "data": "synthetic"}), flush=True)
        del rec, off, init
        torch.cuda.empty_cache()
    eng.close()


def run_streamed_sweep(args):
    """gtp_run_power_streamed on the large window from pinned host memory,
    for 1 to 32 chunks, next to a plain host-to-device copy of the same
    records (the floor of any run that starts from host memory)."""
    import torch

    import synth
    from paper_2609_05960_gb300 import Engine, gtpower

    dev = torch.device("cuda", 0)
    cfg = synth.CONFIGS["large"]
    lib = synth.make_library(cfg.seed_lib)
    net = synth.make_netlist(lib, cfg.n_gates, cfg.seed_net)
    counts = synth.zipf_counts(cfg.n_gates, cfg.n_events, cfg.zipf_s, cfg.cap, cfg.seed_ev)
    tr, rec = synth.make_trace_gpu(net, counts, cfg.window_ps, cfg.seed_ev, device=dev)
    eng = Engine(0)
    eng.load_library(lib)
    eng.load_netlist(net)
    rec_h = torch.empty(rec.shape, dtype=torch.int32, pin_memory=True)
    rec_h.copy_(rec)
    off_h = torch.from_numpy(tr.offsets).pin_memory()
    init_h = torch.from_numpy(tr.init_state).pin_memory()
    wave_h = torch.empty(cfg.window_ps // cfg.bin_ps, dtype=torch.float64, pin_memory=True)
    steps = max(3, min(args.steps, 10))
    ms_copy = _events_per_s(lambda: rec.copy_(rec_h, non_blocking=True), steps, dev)
    del rec
    torch.cuda.empty_cache()
    n = int(tr.n_events)
    print(json.dumps({"sweep": "streamed", "case": "plain host-to-device copy of the records",
                      "bytes": n * 8, "ms": ms_copy, "gb_per_s": n * 8 / (ms_copy * 1e6)}), flush=True)
    for nc in (1, 2, 4, 8, 16, 32):
        run = lambda: gtpower.gtp_run_power_streamed(eng.ctx, 0, cfg.window_ps, off_h, rec_h, init_h, cfg.bin_ps,
                                                     wave_h, nc)
        ms = _events_per_s(run, steps, dev)
        print(json.dumps({"sweep": "streamed", "case": f"gtp_run_power_streamed, {nc} chunks", "n_chunks": nc,
                          "events": n, "ms": ms, "value": n / (ms * 1e-3), "unit": UNIT,
                          "over_plain_copy": ms / ms_copy}), flush=True)
    # the packed transfer form: 4.125 B a record over the host link, unpacked on the device
    pk_h = torch.empty(gtpower.packed_words(n), dtype=torch.int32, pin_memory=True)
    gtpower.gtp_pack_events(rec_h.numpy(), out=pk_h)
    pk_d = torch.empty_like(pk_h, device=dev)
    ms_pcopy = _events_per_s(lambda: pk_d.copy_(pk_h, non_blocking=True), steps, dev)
    del pk_d
    print(json.dumps({"sweep": "streamed", "case": "plain host-to-device copy of the packed records",
                      "bytes": pk_h.numel() * 4, "ms": ms_pcopy, "gb_per_s": pk_h.numel() * 4 / (ms_pcopy * 1e6)}),
          flush=True)
    for nc in (2, 4, 8, 16):
        run = lambda: gtpower.gtp_run_power_streamed(eng.ctx, 0, cfg.window_ps, off_h, pk_h, init_h, cfg.bin_ps,
                                                     wave_h, nc, n_events=n, packed=True)
        ms = _events_per_s(run, steps, dev)
        print(json.dumps({"sweep": "streamed", "case": f"gtp_run_power_streamed, packed, {nc} chunks",
                          "n_chunks": nc, "events": n, "ms": ms, "value": n / (ms * 1e-3), "unit": UNIT,
                          "over_plain_copy_of_packed": ms / ms_pcopy}), flush=True)
    eng.close()


def run_schemes_sweep(args):
    """The paper's own schemes (gtp_run_power_scheme: Naive-D + Naive-L with
    state-pattern traversal, + state-indexed lookup, + event-density-aware
    partitioning, the fused kernel) against this engine's gtp_run_power on
    the same window: the tiny workload, a mid-sized one (200k gates, 20M
    events, 10k bins of 100 ps) and, for the fused kernel alone, the large
    one.  Scheme times are the device time of their kernels (CUDA events
    inside the call, median of the steps); the engine's is the CUDA-event
    time of graph-replayed runs (preparation, walk and merge)."""
    import torch

    import synth
    from paper_2609_05960_gb300 import Engine, gtpower

    dev = torch.device("cuda", 0)
    steps = max(3, min(args.steps, 10))
    cases = [("tiny", synth.CONFIGS["tiny"], None, ["naive", "sipl", "density", "fused"]),
             ("mid: 200,000 gates, 20,000,000 events, Zipf 1.2, cap 100000, 1 us window, 100 ps bins (10,000 bins)",
              None, (200_000, 20_000_000, 1_000_000, 100), ["naive", "sipl", "density", "fused"]),
             ("large", synth.CONFIGS["large"], None, ["fused"])]
    eng = Engine(0)
    for name, cfg, shape, schemes in cases:
        lib = synth.make_library(1)
        if cfg is not None:
            G, n_ev, window_ps, bin_ps = cfg.n_gates, cfg.n_events, cfg.window_ps, cfg.bin_ps
            net = synth.make_netlist(lib, G, cfg.seed_net)
            counts = synth.zipf_counts(G, n_ev, cfg.zipf_s, cfg.cap, cfg.seed_ev)
            seed = cfg.seed_ev
        else:
            G, n_ev, window_ps, bin_ps = shape
            net = synth.make_netlist(lib, G, 2)
            counts = synth.zipf_counts(G, n_ev, 1.2, 100_000, 5)
            seed = 5
        tr, rec = synth.make_trace_gpu(net, counts, window_ps, seed, device=dev)
        off = torch.from_numpy(tr.offsets).to(dev)
        init = torch.from_numpy(tr.init_state).to(dev)
        eng.load_library(lib)
        eng.load_netlist(net)
        eng.load_events(0, window_ps=window_ps, offsets=off, records=rec, init_state=init, borrow=True)
        for key in ("records_per_thread", "ctas_per_sm", "dense_min"):
            eng.set_param(key, -1)
        nb = window_ps // bin_ps
        wave = torch.empty(nb, dtype=torch.float64, device=dev)
        run = lambda: gtpower.gtp_run_power(eng.ctx, 0, bin_ps, wave, graph=True)
        for _ in range(3):
            run()
        ms_engine = _events_per_s(run, steps, dev)
        ref = wave.clone()
        n = int(tr.n_events)
        line = {"sweep": "schemes", "workload": name, "gates": G, "events": n, "bins": nb,
                "engine_ms": ms_engine, "engine_value": n / (ms_engine * 1e-3), "unit": UNIT, "schemes": {}}
        for sc in schemes:
            gtpower.gtp_run_power_scheme(eng.ctx, 0, bin_ps, sc, wave)  # builds the pin streams and block plan
            reps = 1 if name == "large" else steps
            ms = sorted(gtpower.gtp_run_power_scheme(eng.ctx, 0, bin_ps, sc, wave) for _ in range(reps))[reps // 2]
            rel = float(((wave - ref).abs() / ref.abs()).max())
            line["schemes"][sc] = {"kernel_ms": ms, "over_engine": ms / ms_engine, "max_rel_diff_vs_engine": rel}
        if "naive" in line["schemes"]:
            for sc in line["schemes"].values():
                sc["over_naive"] = sc["kernel_ms"] / line["schemes"]["naive"]["kernel_ms"]
        line["partitioning"] = {k: eng.get_param(k) for k in ("scheme_evt_tgt", "scheme_thr_floor", "scheme_ncyc_fix")}
        print(json.dumps(line), flush=True)
        del rec, off, init, wave, ref
        torch.cuda.empty_cache()
    eng.close()


def run_adjoint_sweep(args):
    """The adjoint measurement alone (as in the default run's extras)."""
    import torch

    from paper_2609_05960_gb300 import Engine

    dev = torch.device("cuda", 0)
    eng = Engine(0)
    out = measure_adjoint(eng, dev, max(1, min(args.steps, 20)), args.events)
    print(json.dumps({"sweep": "adjoint", **out}), flush=True)
    eng.close()


def run_glitch_sweep(args):
    """The large workload (scaled by --events): the plain walk, then the same
    window with glitch detection (as in the default run's extras)."""
    import torch

    import synth
    from paper_2609_05960_gb300 import Engine, gtpower

    dev = torch.device("cuda", 0)
    cfg = config_of(args, "large")
    lib = synth.make_library(cfg.seed_lib)
    net = synth.make_netlist(lib, cfg.n_gates, cfg.seed_net)
    counts = synth.zipf_counts(cfg.n_gates, cfg.n_events, cfg.zipf_s, cfg.cap, cfg.seed_ev)
    tr, rec = synth.make_trace_gpu(net, counts, cfg.window_ps, cfg.seed_ev, cfg.tie_p, device=dev)
    eng = Engine(0)
    eng.load_library(lib)
    eng.load_netlist(net)
    eng.load_events(0, window_ps=cfg.window_ps, offsets=torch.from_numpy(tr.offsets).to(dev), records=rec,
                    init_state=torch.from_numpy(tr.init_state).to(dev), borrow=True)
    nb = cfg.window_ps // cfg.bin_ps
    wave = torch.empty(nb, dtype=torch.float64, device=dev)
    steps = max(1, min(args.steps, 20))
    run = lambda: gtpower.gtp_run_power(eng.ctx, 0, cfg.bin_ps, wave, graph=True)
    for _ in range(3):
        run()
    torch.cuda.synchronize(dev)
    eng.set_param("timing", 1)
    _events_per_s(run, steps, dev)
    walk_ms = eng.get_param("t_walk_ns") * 1e-6 / max(eng.get_param("n_timed"), 1)
    eng.set_param("timing", 0)
    n = int(tr.n_events)
    out = measure_glitch(eng, dev, cfg, wave, walk_ms, n, steps)
    print(json.dumps({"sweep": "glitch", "workload": workload_desc(cfg, nb), "events": n, "plain_walk_ms": walk_ms,
                      **out}), flush=True)
    eng.close()


def _large_engine(args):
    """(engine, device, config, waveform tensor, events) with the large
    workload (scaled by --events) loaded in window 0 from device records."""
    import torch

    import synth
    from paper_2609_05960_gb300 import Engine

    dev = torch.device("cuda", 0)
    cfg = config_of(args, "large")
    lib = synth.make_library(cfg.seed_lib)
    net = synth.make_netlist(lib, cfg.n_gates, cfg.seed_net)
    counts = synth.zipf_counts(cfg.n_gates, cfg.n_events, cfg.zipf_s, cfg.cap, cfg.seed_ev)
    tr, rec = synth.make_trace_gpu(net, counts, cfg.window_ps, cfg.seed_ev, cfg.tie_p, device=dev)
    eng = Engine(0)
    eng.load_library(lib)
    eng.load_netlist(net)
    eng.load_events(0, window_ps=cfg.window_ps, offsets=torch.from_numpy(tr.offsets).to(dev), records=rec,
                    init_state=torch.from_numpy(tr.init_state).to(dev), borrow=True)
    eng._keep = rec
    wave = torch.empty(cfg.window_ps // cfg.bin_ps, dtype=torch.float64, device=dev)
    return eng, dev, cfg, wave, int(tr.n_events)


def run_tiled_sweep(args):
    """The time-sliced walk (tile_min) on the large workload: walk time and
    the tiled part's time per threshold (0 = off, the default)."""
    import torch

    from paper_2609_05960_gb300 import gtpower

    eng, dev, cfg, wave, n = _large_engine(args)
    steps = max(1, min(args.steps, 20))
    run = lambda: gtpower.gtp_run_power(eng.ctx, 0, cfg.bin_ps, wave, graph=True)
    for tmin in (0, 32768, 8192, 2048):
        eng.set_param("tile_min", tmin)
        for _ in range(3):
            run()
        torch.cuda.synchronize(dev)
        eng.set_param("timing", 1)
        ms = _events_per_s(run, steps, dev)
        k = max(eng.get_param("n_timed"), 1)
        print(json.dumps({"sweep": "tiled", "tile_min": tmin, "ms_per_run": ms,
                          "walk_ms": eng.get_param("t_walk_ns") * 1e-6 / k,
                          "tiled_ms": eng.get_param("t_tiled_ns") * 1e-6 / k if tmin else 0.0, "events": n}),
              flush=True)
        eng.set_param("timing", 0)
    eng.close()


def run_patterns_sweep(args):
    """The pattern-gate threshold study alone (bench extra `patterns`)."""
    eng, dev, cfg, wave, n = _large_engine(args)
    out = measure_patterns(eng, dev, cfg, wave, n, max(3, min(args.steps, 10)))
    print(json.dumps({"sweep": "patterns", **out}), flush=True)
    eng.close()


def run_prep_sweep(args):
    """The descriptor and gate-table pass alone: the large netlist (1M gates)
    with a small window (--events, default 100k), its loads changed before
    every run; one JSON line with the pass's time and roofline."""
    import torch

    import synth
    from paper_2609_05960_gb300 import Engine, gtpower

    dev = torch.device("cuda", 0)
    cfg = config_of(args, "large")
    n_ev = int(args.events) if args.events else 100_000
    lib = synth.make_library(cfg.seed_lib)
    net = synth.make_netlist(lib, cfg.n_gates, cfg.seed_net)
    counts = synth.zipf_counts(cfg.n_gates, n_ev, cfg.zipf_s, cfg.cap, cfg.seed_ev)
    tr, rec = synth.make_trace_gpu(net, counts, cfg.window_ps, cfg.seed_ev, cfg.tie_p, device=dev)
    eng = Engine(0)
    eng.load_library(lib)
    eng.load_netlist(net)
    eng.load_events(0, window_ps=cfg.window_ps, offsets=torch.from_numpy(tr.offsets).to(dev), records=rec,
                    init_state=torch.from_numpy(tr.init_state).to(dev), borrow=True)
    wave = torch.empty(cfg.window_ps // cfg.bin_ps, dtype=torch.float64, device=dev)
    base = torch.from_numpy(np.ascontiguousarray(net.load_ff, dtype=np.float32)).to(dev)
    loads = [base, base * 1.001]
    steps = max(3, min(args.steps, 50))
    for i in range(args.warmup + steps):
        if i == args.warmup:
            torch.cuda.synchronize(dev)
            eng.set_param("timing", 1)
        gtpower.gtp_set_load(eng.ctx, loads[i & 1])
        gtpower.gtp_run_power(eng.ctx, 0, cfg.bin_ps, wave)
    torch.cuda.synchronize(dev)
    prep_ms = eng.get_param("t_prep_ns") * 1e-6 / max(eng.get_param("n_timed"), 1)
    eng.set_param("timing", 0)
    alg = gate_prep_bytes(lib, net)
    print(json.dumps({"sweep": "prep", "gates": cfg.n_gates, "events": n_ev, "steps": steps, "prep_ms": prep_ms,
                      "algorithmic_bytes": alg, "roofline": roofline(alg, prep_ms, peak_gbs())}), flush=True)
    eng.close()


def main():
    args = parse()
    if args.sweep == "prep":
        run_prep_sweep(args)
        return
    if args.sweep == "tiled":
        run_tiled_sweep(args)
        return
    if args.sweep == "patterns":
        run_patterns_sweep(args)
        return
    if args.sweep == "glitch":
        run_glitch_sweep(args)
        return
    if args.sweep == "adjoint":
        run_adjoint_sweep(args)
        return
    if args.sweep == "schemes":
        run_schemes_sweep(args)
        return
    if args.sweep == "contention":
        run_contention_sweep(args)
        return
    if args.sweep == "streamed":
        run_streamed_sweep(args)
        return
    if args.impl == "reference":
        run_reference(args, args.config)
    else:
        run_ours(args, args.config)


if __name__ == "__main__":
    main()
