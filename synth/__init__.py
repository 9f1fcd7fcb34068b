"""Seeded synthetic inputs for gate-level time-based power analysis.

This module generates the inputs that the GPU engine and the CPU oracle both
consume: a 12-cell standard-cell power library, a random-DAG netlist with
per-gate load capacitance and input slews, and per-gate event traces whose
per-gate counts follow a Zipf law.  It holds none of the power arithmetic
(no interpolation, no energy, no leakage, no binning): only random draws.

The paper's designs (Chipyard SoCs synthesised in a commercial 28 nm node) and
its activity files are not available; these seeded recipes stand in for them,
with event-count skew shaped like the per-gate percentile figure of Section 3.2
(highly skewed, a few gates carrying most events).

Event traces are drawn by a counter-based integer generator (``synth.c``;
the same definition runs on the GPU in ``synth_gpu.cu``), so any gate's
stream can be regenerated on its own and both sides produce identical bits.

Data layouts (shared by every consumer):
  * library tables ``e_int``: cell-major; cell c holds ``n_in[c]`` input pins,
    each with 2 edges (0 = fall, 1 = rise), each with ``2**(n_in[c]-1)``
    side-input states, each a ``n_slew x n_load`` table (slew-major) in fJ.
  * ``p_leak``: cell-major; cell c holds ``2**(n_in[c]+1)`` entries in nW indexed
    by the full pin state (bit p = value of pin p; the output pin is pin n_in).
  * records: ``uint32[n_events, 2]`` = {t_ps (int32 >= 0), meta}, with
    meta bits [0:4) = gate-local pin, bit 4 = new value, bits [5:32) = 0.
    Records are grouped by gate (CSR ``offsets``), time-ordered within a gate.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import subprocess
from typing import Dict, List, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libsynth.so")
_GPU_LIB_PATH = os.path.join(_HERE, "libsynth_gpu.so")

# (name, number of input pins); the output pin follows the inputs.
CELLS = [
    ("INV", 1), ("BUF", 1), ("NAND2", 2), ("NAND3", 3), ("NOR2", 2), ("NOR3", 3),
    ("AND2", 2), ("OR2", 2), ("XOR2", 2), ("AOI21", 3), ("OAI21", 3), ("MUX2", 3),
]
SLEW_AXIS_PS = [5.0, 10.0, 20.0, 40.0, 80.0, 160.0, 320.0]
LOAD_AXIS_FF = [0.25, 0.5, 1.0, 2.0, 4.0, 8.0, 16.0]
VDD = 0.8

STREAM_TABLE = 10
STREAM_LEAK = 11
STREAM_CELL = 12
STREAM_LOAD = 13
STREAM_SLEW = 14
STREAM_PERM = 15
STREAM_FANIN = 16


# --------------------------------------------------------------------------- build
def build(force: bool = False) -> None:
    """Compile the host generator (gcc).  The GPU generator is compiled by
    ``build_gpu``."""
    src = os.path.join(_HERE, "synth.c")
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(src):
        subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-std=c11", "-o", _LIB_PATH + ".tmp",
                               src, "-lpthread"])
        os.replace(_LIB_PATH + ".tmp", _LIB_PATH)


def build_gpu_cmd() -> List[str]:
    src = os.path.join(_HERE, "synth_gpu.cu")
    return ["nvcc", "-O3", "-shared", "-Xcompiler", "-fPIC", "-gencode", "arch=compute_103a,code=sm_103a",
            "-o", _GPU_LIB_PATH + ".tmp", src]


def build_gpu(force: bool = False) -> None:
    src = os.path.join(_HERE, "synth_gpu.cu")
    if force or not os.path.exists(_GPU_LIB_PATH) or os.path.getmtime(_GPU_LIB_PATH) < os.path.getmtime(src):
        subprocess.check_call(build_gpu_cmd())
        os.replace(_GPU_LIB_PATH + ".tmp", _GPU_LIB_PATH)


_lib = None
_gpu_lib = None


def _clib():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        lib.synth_key.restype = ctypes.c_uint64
        lib.synth_key.argtypes = [ctypes.c_uint64] * 4
        lib.synth_keys.restype = None
        lib.synth_keys.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                   ctypes.c_int64, ctypes.c_void_p]
        lib.synth_init_state.restype = None
        lib.synth_init_state.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
        lib.synth_events.restype = ctypes.c_int
        lib.synth_events.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint32, ctypes.c_void_p,
                                     ctypes.c_int]
        lib.synth_events_subset.restype = ctypes.c_int
        lib.synth_events_subset.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_int64, ctypes.c_uint32, ctypes.c_void_p,
                                            ctypes.c_void_p]
        _lib = lib
    return _lib


def _glib():
    global _gpu_lib
    if _gpu_lib is None:
        if not os.path.exists(_GPU_LIB_PATH):
            raise RuntimeError("synth GPU generator not built: run __graft_entry__.build()")
        lib = ctypes.CDLL(_GPU_LIB_PATH)
        lib.synth_gpu_pass1.restype = ctypes.c_int
        lib.synth_gpu_pass1.argtypes = [ctypes.c_uint64, ctypes.c_int64] + [ctypes.c_void_p] * 5 + [
            ctypes.c_int64, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        lib.synth_gpu_pass2.restype = ctypes.c_int
        lib.synth_gpu_pass2.argtypes = [ctypes.c_int64] + [ctypes.c_void_p] * 7
        _gpu_lib = lib
    return _gpu_lib


def _ptr(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


# --------------------------------------------------------------------------- draws
def keys(seed: int, stream: int, n: int, b: int = 0, a0: int = 0) -> np.ndarray:
    """key(seed, stream, a0 + i, b) for i < n, as uint64."""
    out = np.empty(n, dtype=np.uint64)
    if n:
        _clib().synth_keys(seed, stream, a0, b, n, _ptr(out))
    return out


def uniform(seed: int, stream: int, n: int, b: int = 0) -> np.ndarray:
    """U[0,1) doubles from the top 53 bits of the keys (exact conversion)."""
    return (keys(seed, stream, n, b) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


# --------------------------------------------------------------------------- library
@dataclasses.dataclass
class Library:
    names: List[str]
    n_in: np.ndarray          # int32[n_cells]
    vdd: float
    slew_axis: np.ndarray     # float32[n_slew], ps
    load_axis: np.ndarray     # float32[n_load], fF
    e_int: np.ndarray         # float32 flat, fJ (layout in the module docstring)
    p_leak: np.ndarray        # float32 flat, nW

    @property
    def n_cells(self) -> int:
        return len(self.n_in)

    @property
    def max_in(self) -> int:
        return int(self.n_in.max())


def make_library(seed: int = 1, cells=CELLS, e_range=(0.5, 5.0), leak_range=(1.0, 50.0),
                 vdd: float = VDD) -> Library:
    """Tables i.i.d. U[0.5, 5] fJ, leakage i.i.d. U[1, 50] nW per (cell, state)."""
    n_in = np.array([k for _, k in cells], dtype=np.int32)
    ns, nl = len(SLEW_AXIS_PS), len(LOAD_AXIS_FF)
    n_tab = int(sum(k * (2 ** k) for k in n_in))  # n_in * 2 edges * 2**(n_in-1) side states
    n_leak = int(sum(2 ** (k + 1) for k in n_in))
    u = uniform(seed, STREAM_TABLE, n_tab * ns * nl)
    e_int = (e_range[0] + (e_range[1] - e_range[0]) * u).astype(np.float32)
    u = uniform(seed, STREAM_LEAK, n_leak)
    p_leak = (leak_range[0] + (leak_range[1] - leak_range[0]) * u).astype(np.float32)
    return Library([n for n, _ in cells], n_in, float(np.float32(vdd)),
                   np.array(SLEW_AXIS_PS, np.float32), np.array(LOAD_AXIS_FF, np.float32), e_int, p_leak)


# --------------------------------------------------------------------------- netlist
@dataclasses.dataclass
class Netlist:
    cell: np.ndarray          # int32[n_gates]
    load_ff: np.ndarray       # float32[n_gates]
    slew_ps: np.ndarray       # float32[n_gates, slew_stride, 2]  (edge 0 = fall, 1 = rise)
    n_pins: np.ndarray        # uint8[n_gates] = n_in(cell) + 1
    level: np.ndarray         # int32[n_gates], DAG level (connectivity is not used by the walk)
    fanin: np.ndarray         # int64[n_gates, slew_stride], -1 = primary input / unused

    @property
    def n_gates(self) -> int:
        return len(self.cell)

    @property
    def slew_stride(self) -> int:
        return self.slew_ps.shape[1]


def make_netlist(lib: Library, n_gates: int, seed: int = 2, depth: int = 20,
                 load_median_ff: float = 2.0, load_sigma: float = 0.5,
                 slew_range=(10.0, 200.0)) -> Netlist:
    """Random DAG of the given depth; cell uniform over the library;
    C ~ lognormal(ln median, sigma); slews U[10, 200] ps per (gate, input, edge)."""
    G = int(n_gates)
    stride = lib.max_in
    cell = (keys(seed, STREAM_CELL, G) % np.uint64(lib.n_cells)).astype(np.int32)
    u1 = uniform(seed, STREAM_LOAD, G, b=0)
    u2 = uniform(seed, STREAM_LOAD, G, b=1)
    z = np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)
    load = np.exp(math.log(load_median_ff) + load_sigma * z).astype(np.float32)
    us = uniform(seed, STREAM_SLEW, G * stride * 2).reshape(G, stride, 2)
    slew = (slew_range[0] + (slew_range[1] - slew_range[0]) * us).astype(np.float32)
    n_in_g = lib.n_in[cell]
    for p in range(stride):
        slew[n_in_g <= p, p, :] = 0.0
    n_pins = (n_in_g + 1).astype(np.uint8)
    level = (np.arange(G, dtype=np.int64) * depth // max(G, 1)).astype(np.int32)
    first_of_level = np.searchsorted(level, np.arange(depth + 1), side="left")
    lim = first_of_level[level]
    fk = keys(seed, STREAM_FANIN, G * stride).reshape(G, stride)
    fanin = np.where(lim[:, None] > 0, (fk % np.maximum(lim, 1)[:, None].astype(np.uint64)).astype(np.int64), -1)
    fanin[np.arange(stride)[None, :] >= n_in_g[:, None]] = -1
    return Netlist(cell, load, slew, n_pins, level, fanin)


# --------------------------------------------------------------------------- event counts
def zipf_counts(n_gates: int, total: int, s: float, cap: Optional[int], seed: int) -> np.ndarray:
    """Per-gate event counts: Zipf(s) over a seeded random rank permutation,
    capped at ``cap`` with iterative water-filling, made integer by largest
    remainder so that the counts sum to ``total`` exactly."""
    G = int(n_gates)
    order = np.argsort(keys(seed, STREAM_PERM, G), kind="stable")
    rank = np.empty(G, dtype=np.float64)
    rank[order] = np.arange(1, G + 1, dtype=np.float64)
    w = rank ** (-float(s))
    target = total * w / w.sum()
    if cap is not None:
        if cap * G < total:
            raise ValueError("cap too small for the total")
        capped = np.zeros(G, dtype=bool)
        for _ in range(200):
            over = (target > cap) & ~capped
            if not over.any():
                break
            capped |= over
            free = ~capped
            remaining = total - cap * capped.sum()
            target = np.where(capped, float(cap), remaining * w / w[free].sum())
    base = np.floor(target).astype(np.int64)
    if cap is not None:
        base = np.minimum(base, cap)
    rem = int(total - base.sum())
    if rem:
        frac = target - base
        if cap is not None:
            frac = np.where(base >= cap, -1.0, frac)
        pick = np.argsort(-frac, kind="stable")[:rem]
        base[pick] += 1
    return base


def offsets_from_counts(counts: np.ndarray) -> np.ndarray:
    off = np.zeros(len(counts) + 1, dtype=np.int64)
    np.cumsum(counts, out=off[1:])
    return off


# --------------------------------------------------------------------------- traces
@dataclasses.dataclass
class Trace:
    window_ps: int
    offsets: np.ndarray       # int64[n_gates + 1]
    records: Optional[np.ndarray]  # uint32[n_events, 2] (None when generated on the GPU only)
    init_state: np.ndarray    # uint8[n_gates]
    seed: int
    tie24: int

    @property
    def n_events(self) -> int:
        return int(self.offsets[-1])


def tie_threshold(tie_p: float) -> int:
    return int(round(tie_p * (1 << 24)))


def init_states(net: Netlist, seed: int) -> np.ndarray:
    out = np.empty(net.n_gates, dtype=np.uint8)
    np_ = np.ascontiguousarray(net.n_pins)
    if net.n_gates:
        _clib().synth_init_state(seed, net.n_gates, _ptr(np_), _ptr(out))
    return out


def make_trace(net: Netlist, counts: np.ndarray, window_ps: int, seed: int, tie_p: float = 0.0,
               n_threads: Optional[int] = None, materialise: bool = True) -> Trace:
    offsets = offsets_from_counts(np.asarray(counts, dtype=np.int64))
    init = init_states(net, seed)
    tie24 = tie_threshold(tie_p)
    rec = None
    if materialise:
        rec = np.empty((int(offsets[-1]), 2), dtype=np.uint32)
        if n_threads is None:
            n_threads = min(os.cpu_count() or 1, 32)
        np_ = np.ascontiguousarray(net.n_pins)
        if rec.size:
            _clib().synth_events(seed, net.n_gates, _ptr(offsets), _ptr(np_), _ptr(init), int(window_ps),
                                 tie24, _ptr(rec), int(n_threads))
    return Trace(int(window_ps), offsets, rec, init, seed, tie24)


def gate_records(net: Netlist, trace: Trace, gates: np.ndarray):
    """Regenerate the records of the selected gates only.  Returns
    (offsets_sel[int64, len+1], records_sel[uint32, n, 2])."""
    gates = np.ascontiguousarray(np.asarray(gates, dtype=np.int64))
    counts = (trace.offsets[gates + 1] - trace.offsets[gates]).astype(np.int64)
    off = offsets_from_counts(counts)
    rec = np.empty((int(off[-1]), 2), dtype=np.uint32)
    np_ = np.ascontiguousarray(net.n_pins[gates])
    init = np.ascontiguousarray(trace.init_state[gates])
    if len(gates):
        _clib().synth_events_subset(trace.seed, len(gates), _ptr(gates), _ptr(counts), _ptr(np_), _ptr(init),
                                    trace.window_ps, trace.tie24, _ptr(off), _ptr(rec))
    return off, rec


def make_trace_gpu(net: Netlist, counts: np.ndarray, window_ps: int, seed: int, tie_p: float = 0.0,
                   device="cuda", chunk: int = 1024):
    """Materialise the records in device memory with the GPU copy of the
    generator.  Returns (Trace with records=None, torch uint32 tensor [n, 2])."""
    import torch

    trace = make_trace(net, counts, window_ps, seed, tie_p, materialise=False)
    counts = np.asarray(counts, dtype=np.int64)
    nchunk = (counts + chunk - 1) // chunk
    cg = np.repeat(np.arange(len(counts), dtype=np.int64), nchunk)
    first = offsets_from_counts(nchunk)
    local = np.arange(len(cg), dtype=np.int64) - first[cg]
    ck0 = local * chunk
    ck1 = np.minimum(ck0 + chunk, counts[cg])
    dev = torch.device(device)
    t_cg = torch.from_numpy(cg).to(dev)
    t_k0 = torch.from_numpy(ck0).to(dev)
    t_k1 = torch.from_numpy(ck1).to(dev)
    t_off = torch.from_numpy(trace.offsets).to(dev)
    t_np = torch.from_numpy(np.ascontiguousarray(net.n_pins)).to(dev)
    n_ev = trace.n_events
    rec = torch.empty((max(n_ev, 1), 2), dtype=torch.int32, device=dev)
    masks = torch.empty(max(len(cg), 1), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    lib = _glib()
    rc = lib.synth_gpu_pass1(seed, len(cg), t_cg.data_ptr(), t_k0.data_ptr(), t_k1.data_ptr(), t_off.data_ptr(),
                             t_np.data_ptr(), trace.window_ps, trace.tie24, rec.data_ptr(), masks.data_ptr(),
                             stream)
    if rc:
        raise RuntimeError(f"synth_gpu_pass1 failed: CUDA error {rc}")
    # starting state of each chunk = init XOR (pin toggles of the gate's earlier chunks)
    m = masks[: len(cg)].cpu().numpy()
    cum = np.bitwise_xor.accumulate(m) if len(m) else m
    before = np.zeros_like(m)
    if len(m):
        before[1:] = cum[:-1]
    gate_first = first[cg]
    gate_before = np.where(gate_first > 0, cum[np.maximum(gate_first - 1, 0)], 0).astype(np.uint8)
    state = (trace.init_state[cg] ^ before ^ gate_before).astype(np.uint8)
    t_state = torch.from_numpy(state).to(dev)
    rc = lib.synth_gpu_pass2(len(cg), t_cg.data_ptr(), t_k0.data_ptr(), t_k1.data_ptr(), t_off.data_ptr(),
                             t_state.data_ptr(), rec.data_ptr(), stream)
    if rc:
        raise RuntimeError(f"synth_gpu_pass2 failed: CUDA error {rc}")
    return trace, rec[:n_ev]


# --------------------------------------------------------------------------- configs
@dataclasses.dataclass
class Config:
    name: str
    n_gates: int
    n_events: int
    zipf_s: float
    cap: Optional[int]
    window_ps: int
    bin_ps: int
    seed_lib: int = 1
    seed_net: int = 2
    seed_ev: int = 3
    tie_p: float = 0.0


CONFIGS: Dict[str, Config] = {
    # 2,000 gates, 200k events, Zipf 1.1, 1 us window, 100 ps bins (10k bins)
    "tiny": Config("tiny", 2_000, 200_000, 1.1, None, 1_000_000, 100, seed_ev=3),
    # 1M gates, 200M events, Zipf 1.2 capped at 1e5, 10 us, 10 ps bins (1M bins)
    "large": Config("large", 1_000_000, 200_000_000, 1.2, 100_000, 10_000_000, 10, seed_ev=4),
    # 500k gates, 100M events, 5 us, 10 ps bins
    "adjoint": Config("adjoint", 500_000, 100_000_000, 1.2, 100_000, 5_000_000, 10, seed_ev=6),
    # 10M gates, 2B events, Zipf 1.5 capped at 1e7, 100 us, 10 ps bins (10M bins)
    "stress": Config("stress", 10_000_000, 2_000_000_000, 1.5, 10_000_000, 100_000_000, 10, seed_ev=7),
}

BATCHED_GATES = 200_000
BATCHED_WINDOWS = 64


def batched_windows(n_windows: int = BATCHED_WINDOWS, seed: int = 5, bins_range=(1_000, 100_000),
                    events_range=(1_000_000, 20_000_000), bin_ps: int = 10):
    """Window list for the batched workload: bins and events per window
    log-uniform and independent; window w uses event seed ``seed + w``."""
    u1 = uniform(seed, 20, n_windows)
    u2 = uniform(seed, 21, n_windows)
    bins = np.floor(np.exp(np.log(bins_range[0]) + u1 * (np.log(bins_range[1]) - np.log(bins_range[0]))))
    evs = np.floor(np.exp(np.log(events_range[0]) + u2 * (np.log(events_range[1]) - np.log(events_range[0]))))
    return [dict(window_ps=int(b) * bin_ps, n_events=int(e), seed=seed + w, bin_ps=bin_ps)
            for w, (b, e) in enumerate(zip(bins, evs))]


def scaled(cfg: Config, gates: int, events: int, **kw) -> Config:
    """Same recipe at another size (used for small parity cases)."""
    return dataclasses.replace(cfg, n_gates=gates, n_events=events, **kw)


def make_inputs(cfg: Config, materialise: bool = True):
    lib = make_library(cfg.seed_lib)
    net = make_netlist(lib, cfg.n_gates, cfg.seed_net)
    counts = zipf_counts(cfg.n_gates, cfg.n_events, cfg.zipf_s, cfg.cap, cfg.seed_ev)
    trace = make_trace(net, counts, cfg.window_ps, cfg.seed_ev, cfg.tie_p, materialise=materialise)
    return lib, net, trace
