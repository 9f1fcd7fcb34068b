"""Python binding of the C ABI in ``include/gtpower.h`` (ctypes).

Argument marshalling only: every step of the power walk runs in the CUDA
library ``libgtpower.so``.  Functions carry the C names; ``Engine`` bundles
them for convenience.  PyTorch provides device memory and streams.  If the
library is missing the binding raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Dict, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgtpower.so")

GTP_OK, GTP_EINVAL, GTP_EORDER, GTP_ERANGE, GTP_ENOTOGGLE = 0, -1, -2, -3, -4
GTP_ENOMEM, GTP_ECUDA, GTP_ETIMEOUT, GTP_EDEVICE = -5, -6, -7, -8
GTP_HOST, GTP_DEVICE, GTP_BORROW, GTP_GRAPH, GTP_PACKED = 0, 1, 2, 4, 8
GTP_NOALLOC_MAX_BINS = 1 << 19
GTP_MAX_PINS = 8
GTP_MAX_PATTERN_PINS = 32
GTP_MAX_INDEXED_PINS = 24

CODE_NAMES = {GTP_EINVAL: "EINVAL", GTP_EORDER: "EORDER", GTP_ERANGE: "ERANGE", GTP_ENOTOGGLE: "ENOTOGGLE",
              GTP_ENOMEM: "ENOMEM", GTP_ECUDA: "ECUDA", GTP_ETIMEOUT: "ETIMEOUT", GTP_EDEVICE: "EDEVICE"}

# every entry point the header declares
ABI_SYMBOLS = ["gtp_create", "gtp_destroy", "gtp_set_stream", "gtp_last_error", "gtp_load_library",
               "gtp_set_scales", "gtp_load_netlist", "gtp_set_load", "gtp_load_events", "gtp_run_power",
               "gtp_gate_energy", "gtp_run_power_batched", "gtp_run_power_backward", "gtp_autotune",
               "gtp_set_param", "gtp_get_param", "gtp_run_power_noalloc", "gtp_set_glitch", "gtp_gate_glitch",
               "gtp_run_power_streamed", "gtp_design_power", "gtp_run_power_components",
               "gtp_run_power_scheme", "gtp_sipl_expand",
               "gtp_pack_events", "gtp_measure_reductions", "gtp_load_pattern_cells", "gtp_load_pattern_netlist",
               "gtp_load_pattern_events", "gtp_pattern_gate_energy", "gtp_pattern_gate_gradient", "gtp_measure_replay"]


class GtpError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{CODE_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None


def load(path: str = LIB_PATH):
    """Load libgtpower.so and declare the ABI signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() (no CPU fallback exists)")
    L = ctypes.CDLL(path)
    P, I32, I64, F = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float
    sig = {
        "gtp_create": ([ctypes.POINTER(P), ctypes.c_int, P], ctypes.c_int),
        "gtp_destroy": ([P], None),
        "gtp_set_stream": ([P, P], ctypes.c_int),
        "gtp_last_error": ([P], ctypes.c_char_p),
        "gtp_load_library": ([P, I32, P, F, I32, P, I32, P, P, I64, P, I64], ctypes.c_int),
        "gtp_set_scales": ([P, P, P], ctypes.c_int),
        "gtp_load_netlist": ([P, I64, P, P, P, I32, ctypes.c_int], ctypes.c_int),
        "gtp_set_load": ([P, P, ctypes.c_int], ctypes.c_int),
        "gtp_set_glitch": ([P, I64, P, ctypes.c_int], ctypes.c_int),
        "gtp_gate_glitch": ([P, I32, P, ctypes.c_int], ctypes.c_int),
        "gtp_design_power": ([P, I32, P, ctypes.c_int, P], ctypes.c_int),
        "gtp_run_power_streamed": ([P, I32, I64, I64, P, P, P, I32, P, I32, ctypes.c_int], ctypes.c_int),
        "gtp_load_events": ([P, I32, I64, I64, P, P, P, ctypes.c_int], ctypes.c_int),
        "gtp_run_power": ([P, I32, I32, P, ctypes.c_int], ctypes.c_int),
        "gtp_run_power_components": ([P, I32, I32, P, P, ctypes.c_int], ctypes.c_int),
        "gtp_pack_events": ([I64, P, P], ctypes.c_int),
        "gtp_measure_reductions": ([P, I32, I32, I64, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
        "gtp_measure_replay": ([P, I32, I32, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
        "gtp_sipl_expand": ([I32, I32, I32, I32, P, P, P, P, P, P, I32, P, P, P, F, P, P], ctypes.c_int),
        "gtp_run_power_scheme": ([P, I32, I32, I32, P, ctypes.c_int, ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
        "gtp_gate_energy": ([P, I32, P, P, P, P, P, ctypes.c_int], ctypes.c_int),
        "gtp_run_power_batched": ([P, I32, P, I32, P, ctypes.c_int], ctypes.c_int),
        "gtp_run_power_backward": ([P, I32, I32, P, P, P, P], ctypes.c_int),
        "gtp_autotune": ([P, I32, P, I32, I32, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
        "gtp_set_param": ([P, ctypes.c_char_p, I64], ctypes.c_int),
        "gtp_get_param": ([P, ctypes.c_char_p], I64),
        "gtp_load_pattern_cells": ([P, I32, P, F, I32, P, I32, P] + [P] * 12, ctypes.c_int),
        "gtp_load_pattern_netlist": ([P, I64, P, P, P, I32, P], ctypes.c_int),
        "gtp_load_pattern_events": ([P, I32, I64, P, P, P, P, P, ctypes.c_int], ctypes.c_int),
        "gtp_pattern_gate_energy": ([P, I32, P, P, P, P, P, P, ctypes.c_int], ctypes.c_int),
        "gtp_pattern_gate_gradient": ([P, I32, P, ctypes.c_int], ctypes.c_int),
        "gtp_run_power_noalloc": ([P, I32, P, F, I32, P, I32, P, P, I64, P, I64, I64, P, P, P, I32, I64, I64, P, P, P,
                                   I32, P, P, P, P, P], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


# ------------------------------------------------------------------ marshalling helpers
def _ptr_flags(a, dtype):
    """(pointer, flags, keepalive) for a numpy array or torch tensor."""
    if a is None:
        return None, GTP_HOST, None
    try:
        import torch
        if isinstance(a, torch.Tensor):
            want = {np.float32: torch.float32, np.float64: torch.float64, np.int32: torch.int32,
                    np.int64: torch.int64, np.uint8: torch.uint8, np.uint32: torch.int32}[dtype]
            if a.dtype != want or not a.is_contiguous():
                raise TypeError(f"tensor must be contiguous {want}, got {a.dtype}")
            return a.data_ptr(), (GTP_DEVICE if a.is_cuda else GTP_HOST), a
    except ImportError:
        pass
    arr = np.ascontiguousarray(np.asarray(a), dtype=dtype)
    return arr.ctypes.data, GTP_HOST, arr


def _check(ctx, rc: int):
    if rc != GTP_OK:
        msg = gtp_last_error(ctx) if ctx else ""
        raise GtpError(rc, msg)


# ------------------------------------------------------------------ ABI-named functions
def gtp_create(device: int = 0, stream: Optional[int] = None):
    h = ctypes.c_void_p()
    rc = load().gtp_create(ctypes.byref(h), int(device), stream)
    if rc != GTP_OK:
        raise GtpError(rc, f"gtp_create failed on device {device}")
    return h


def gtp_destroy(ctx) -> None:
    load().gtp_destroy(ctx)


def gtp_set_stream(ctx, stream: Optional[int]) -> None:
    _check(ctx, load().gtp_set_stream(ctx, stream))


def gtp_last_error(ctx) -> str:
    r = load().gtp_last_error(ctx)
    return r.decode() if r else ""


def gtp_load_library(ctx, n_in, vdd, slew_axis, load_axis, e_int, p_leak) -> None:
    ni = np.ascontiguousarray(n_in, np.int32)
    sa = np.ascontiguousarray(slew_axis, np.float32)
    la = np.ascontiguousarray(load_axis, np.float32)
    ei = np.ascontiguousarray(e_int, np.float32)
    pl = np.ascontiguousarray(p_leak, np.float32)
    _check(ctx, load().gtp_load_library(ctx, len(ni), ni.ctypes.data, float(vdd), len(sa), sa.ctypes.data, len(la),
                                        la.ctypes.data, ei.ctypes.data, ei.size, pl.ctypes.data, pl.size))


def gtp_set_scales(ctx, escale=None, lscale=None) -> None:
    e = None if escale is None else np.ascontiguousarray(escale, np.float32)
    l = None if lscale is None else np.ascontiguousarray(lscale, np.float32)
    _check(ctx, load().gtp_set_scales(ctx, None if e is None else e.ctypes.data, None if l is None else l.ctypes.data))


def gtp_load_netlist(ctx, cell, load_ff, slew_ps) -> None:
    pc, fc, kc = _ptr_flags(cell, np.int32)
    pl, fl, kl = _ptr_flags(load_ff, np.float32)
    ps, fs, ks = _ptr_flags(slew_ps, np.float32)
    if not (fc == fl == fs):
        raise ValueError("netlist arrays must all be host or all be device")
    n = len(cell)
    stride = int(slew_ps.shape[1]) if len(slew_ps.shape) == 3 else int(np.asarray(slew_ps).size // (2 * n))
    _check(ctx, load().gtp_load_netlist(ctx, n, pc, pl, ps, stride, fc))


def gtp_set_load(ctx, load_ff) -> None:
    p, f, k = _ptr_flags(load_ff, np.float32)
    _check(ctx, load().gtp_set_load(ctx, p, f))


def gtp_set_glitch(ctx, clock_ps: int, out_slew=None) -> None:
    """Glitch detection with a clock of clock_ps (0: off); out_slew[n_gates][2]
    {fall, rise} output transition times in ps (float32)."""
    p, f, k = _ptr_flags(out_slew, np.float32)
    _check(ctx, load().gtp_set_glitch(ctx, int(clock_ps), p, f))


def gtp_measure_reductions(ctx, n_slots: int, width: int = 2, n_red: int = 160_000_000) -> float:
    """Bin-update reductions per second the GPU sustains (see the header)."""
    out = ctypes.c_double(0.0)
    _check(ctx, load().gtp_measure_reductions(ctx, int(n_slots), int(width), int(n_red), ctypes.byref(out)))
    return float(out.value)


def gtp_measure_replay(ctx, window: int, bin_ps: int) -> float:
    """Time (ms) of the window's own bin reductions alone (see the header)."""
    out = ctypes.c_double(0.0)
    _check(ctx, load().gtp_measure_replay(ctx, int(window), int(bin_ps), ctypes.byref(out)))
    return float(out.value)


def packed_words(n_events: int) -> int:
    """Length (uint32 words) of the packed transfer form of n_events records."""
    return (int(n_events) + 31) // 32 + int(n_events)


def gtp_pack_events(events, out=None):
    """Packed transfer form (uint32, packed_words(n) long) of [n][2] records;
    `out` may be a preallocated (e.g. pinned) uint32/int32 array or tensor."""
    rec = np.ascontiguousarray(np.asarray(events).view(np.uint32).reshape(-1, 2))
    n = rec.shape[0]
    if out is None:
        out = np.empty(packed_words(n), np.uint32)
    po, fo, ko = _ptr_flags(out, np.uint32)
    if fo != GTP_HOST or (out.shape[0] if hasattr(out, "shape") else len(out)) < packed_words(n):
        raise ValueError("out must be a host array of packed_words(n) words")
    rc = load().gtp_pack_events(int(n), rec.ctypes.data if n else None, po if n else None)
    if rc != GTP_OK:
        raise GtpError(rc, "pack_events: a negative time, reserved bits, or a block spanning 2^27 ps")
    return out


def gtp_run_power_streamed(ctx, window: int, window_ps: int, gate_offsets, events, init_state, bin_ps: int,
                           waveform=None, n_chunks: int = 8, n_events=None, packed: bool = False) -> None:
    """Run a window from host arrays in n_chunks overlapped chunks (events
    pinned for overlap); the waveform may be host or device.  packed: events
    is the packed transfer form of n_events records (gtp_pack_events)."""
    po, fo, ko = _ptr_flags(gate_offsets, np.int64)
    pe, fe, ke = _ptr_flags(events, np.uint32)
    pi, fi, ki = _ptr_flags(init_state, np.uint8)
    if GTP_DEVICE in (fo, fe, fi):
        raise ValueError("run_power_streamed takes host inputs")
    pw, fw, kw = _ptr_flags(waveform, np.float64)
    if packed:
        n = int(n_events) if n_events is not None else int(gate_offsets[-1])
        size = events.shape[0] if hasattr(events, "shape") else len(events)
        if size < packed_words(n):
            raise ValueError("packed events shorter than packed_words(n_events)")
    else:
        n = 0 if events is None else (events.shape[0] if hasattr(events, "shape") else len(events))
    _check(ctx, load().gtp_run_power_streamed(ctx, int(window), int(window_ps), int(n), po, pe, pi, int(bin_ps), pw,
                                              int(n_chunks), fw | (GTP_PACKED if packed else 0)))


def gtp_design_power(ctx, window: int, waveform=None) -> dict:
    """Design-level power of the window's last run (W): averages of each
    component over the window, their total, and the waveform's peak."""
    pw, fw, kw = _ptr_flags(waveform, np.float64)
    out = np.zeros(7)
    _check(ctx, load().gtp_design_power(ctx, int(window), pw, fw, out.ctypes.data))
    return dict(p_leak=out[0], p_int=out[1], p_sw=out[2], p_gl=out[3], p_total=out[4], p_peak=out[5],
                peak_bin=int(out[6]))


def gtp_gate_glitch(ctx, window: int, e_gl) -> None:
    p, f, k = _ptr_flags(e_gl, np.float64)
    _check(ctx, load().gtp_gate_glitch(ctx, int(window), p, f))


def gtp_load_events(ctx, window: int, window_ps: int, gate_offsets, events, init_state, borrow: bool = False,
                    packed: bool = False) -> None:
    """packed: events is the packed transfer form (gtp_pack_events) of
    gate_offsets[-1] records."""
    po, fo, ko = _ptr_flags(gate_offsets, np.int64)
    pe, fe, ke = _ptr_flags(events, np.uint32)
    pi, fi, ki = _ptr_flags(init_state, np.uint8)
    if not (fo == fe == fi):
        raise ValueError("event arrays must all be host or all be device")
    if packed:
        n_events = int(gate_offsets[-1])
        if (events.shape[0] if hasattr(events, "shape") else len(events)) < packed_words(n_events):
            raise ValueError("packed events shorter than packed_words(n_events)")
    else:
        n_events = int(events.shape[0]) if events is not None else 0
    flags = fo | (GTP_BORROW if borrow else 0) | (GTP_PACKED if packed else 0)
    _check(ctx, load().gtp_load_events(ctx, int(window), int(window_ps), n_events, po, pe, pi, flags))


def gtp_run_power(ctx, window: int, bin_ps: int, waveform=None, graph: bool = False) -> None:
    p, f, k = _ptr_flags(waveform, np.float64)
    _check(ctx, load().gtp_run_power(ctx, int(window), int(bin_ps), p, f | (GTP_GRAPH if graph else 0)))


def gtp_run_power_components(ctx, window: int, bin_ps: int, components, waveform=None) -> None:
    pc, fc, kc = _ptr_flags(components, np.float64)
    pw, fw, kw = _ptr_flags(waveform, np.float64)
    if pw is not None and fw != fc:
        raise ValueError("components and waveform must both be host or both be device")
    _check(ctx, load().gtp_run_power_components(ctx, int(window), int(bin_ps), pw, pc, fc))


def gtp_sipl_expand(n_in: int, n_slew: int, n_load: int, int_patterns, int_default, leak_patterns,
                    leak_default: float):
    """One cell's state-indexed arrays (e_int, p_leak) from Liberty-style
    patterns: int_patterns = [(pin, edge or -1, care, val, table)];
    int_default = [n_in][2] tables (or scalars); leak_patterns =
    [(care, val, nW)].  Tables are n_slew x n_load (or scalars)."""
    shape = (n_slew, n_load)
    ip = np.array([p[0] for p in int_patterns], np.int32)
    ie = np.array([p[1] for p in int_patterns], np.int32)
    ic = np.array([p[2] for p in int_patterns], np.uint32)
    iv = np.array([p[3] for p in int_patterns], np.uint32)
    it = np.array([np.broadcast_to(np.asarray(p[4], np.float32), shape) for p in int_patterns], np.float32)
    dflt = np.asarray(int_default, np.float32)
    if 1 <= n_in < 8 and dflt.shape[:2] != (n_in, 2):
        raise ValueError("int_default must hold [n_in][2] tables")
    dflt = np.ascontiguousarray(np.broadcast_to(dflt.reshape(dflt.shape + (1, 1)) if dflt.ndim == 2 else dflt,
                                                dflt.shape[:2] + shape), np.float32)
    lc = np.array([p[0] for p in leak_patterns], np.uint32)
    lv = np.array([p[1] for p in leak_patterns], np.uint32)
    lp = np.array([p[2] for p in leak_patterns], np.float32)
    ok = 1 <= n_in < 8
    e_int = np.empty(n_in * 2 * (1 << (n_in - 1)) * n_slew * n_load if ok else 1, np.float32)
    p_leak = np.empty(2 << n_in if ok else 1, np.float32)
    ptr = lambda a: a.ctypes.data if a.size else None
    rc = load().gtp_sipl_expand(int(n_in), int(n_slew), int(n_load), len(ip), ptr(ip), ptr(ie), ptr(ic), ptr(iv),
                                ptr(it), dflt.ctypes.data, len(lc), ptr(lc), ptr(lv), ptr(lp), float(leak_default),
                                e_int.ctypes.data, p_leak.ctypes.data)
    if rc != GTP_OK:
        raise GtpError(rc, "sipl_expand: bad pattern list")
    return e_int, p_leak


def gtp_load_pattern_cells(ctx, plib) -> None:
    """Pattern cells from a synth.patterns.PatternLibrary-shaped object."""
    ns, nl = len(plib.slew_axis), len(plib.load_axis)
    a = dict(n_in=np.ascontiguousarray(plib.n_in, np.int32), sa=np.ascontiguousarray(plib.slew_axis, np.float32),
             la=np.ascontiguousarray(plib.load_axis, np.float32),
             io=np.ascontiguousarray(plib.int_offsets, np.int32), ip=np.ascontiguousarray(plib.int_pin, np.int32),
             ie=np.ascontiguousarray(plib.int_edge, np.int32), ic=np.ascontiguousarray(plib.int_care, np.uint32),
             iv=np.ascontiguousarray(plib.int_val, np.uint32),
             it=np.ascontiguousarray(np.asarray(plib.int_tab, np.float32).reshape(-1, ns * nl)),
             idf=np.ascontiguousarray(np.asarray(plib.int_default, np.float32).reshape(-1)),
             lo=np.ascontiguousarray(plib.leak_offsets, np.int32), lc=np.ascontiguousarray(plib.leak_care, np.uint32),
             lv=np.ascontiguousarray(plib.leak_val, np.uint32), lp=np.ascontiguousarray(plib.leak_pw, np.float32),
             ld=np.ascontiguousarray(plib.leak_default, np.float32))
    ptr = lambda x: x.ctypes.data if x.size else None
    _check(ctx, load().gtp_load_pattern_cells(
        ctx, len(a["n_in"]), ptr(a["n_in"]), float(plib.vdd), ns, ptr(a["sa"]), nl, ptr(a["la"]), ptr(a["io"]),
        ptr(a["ip"]), ptr(a["ie"]), ptr(a["ic"]), ptr(a["iv"]), ptr(a["it"]), ptr(a["idf"]), ptr(a["lo"]),
        ptr(a["lc"]), ptr(a["lv"]), ptr(a["lp"]), ptr(a["ld"])))


def gtp_load_pattern_netlist(ctx, pnet) -> None:
    """Pattern gates from a synth.patterns.PatternNetlist-shaped object."""
    cell = np.ascontiguousarray(pnet.cell, np.int32)
    load_ff = np.ascontiguousarray(pnet.load_ff, np.float32)
    slew = np.ascontiguousarray(pnet.slew_ps, np.float32)
    oslew = None if getattr(pnet, "out_slew_ps", None) is None else np.ascontiguousarray(pnet.out_slew_ps, np.float32)
    _check(ctx, load().gtp_load_pattern_netlist(ctx, len(cell), cell.ctypes.data, load_ff.ctypes.data,
                                                slew.ctypes.data, int(slew.shape[1]),
                                                None if oslew is None else oslew.ctypes.data))


def gtp_load_pattern_events(ctx, window: int, gate_offsets, t_ps, pin, value, init_state) -> None:
    """A window's pattern-gate events (host arrays or CUDA tensors, all alike)."""
    po, fo, ko = _ptr_flags(gate_offsets, np.int64)
    pt, ft, kt = _ptr_flags(t_ps, np.int32)
    pp, fp, kp = _ptr_flags(pin, np.uint8)
    pv, fv, kv = _ptr_flags(value, np.uint8)
    pi, fi, ki = _ptr_flags(init_state, np.uint32)
    if len({fo, ft, fp, fv, fi}) > 1:
        raise ValueError("pattern event arrays must all be host or all be device")
    n = int(t_ps.shape[0]) if hasattr(t_ps, "shape") else len(t_ps)
    _check(ctx, load().gtp_load_pattern_events(ctx, int(window), n, po, pt if n else None, pp if n else None,
                                               pv if n else None, pi, fo))


def gtp_pattern_gate_energy(ctx, window: int, e_leak=None, e_int=None, e_sw=None, e_gl=None, n_events=None,
                            final_state=None) -> None:
    args = [_ptr_flags(e_leak, np.float64), _ptr_flags(e_int, np.float64), _ptr_flags(e_sw, np.float64),
            _ptr_flags(e_gl, np.float64), _ptr_flags(n_events, np.int64), _ptr_flags(final_state, np.uint32)]
    flags = {a[1] for a in args if a[0] is not None}
    if len(flags) > 1:
        raise ValueError("outputs must all be host or all be device")
    f = flags.pop() if flags else GTP_HOST
    _check(ctx, load().gtp_pattern_gate_energy(ctx, int(window), *[a[0] for a in args], f))


def gtp_pattern_gate_gradient(ctx, window: int, dC) -> None:
    p, f, k = _ptr_flags(dC, np.float32)
    _check(ctx, load().gtp_pattern_gate_gradient(ctx, int(window), p, f))


SCHEMES = {"naive": 0, "sipl": 1, "density": 2, "fused": 3}


def gtp_run_power_scheme(ctx, window: int, bin_ps: int, scheme, waveform=None) -> float:
    """One run of one of the paper's schemes; returns the device time (ms)
    of its kernels."""
    s = SCHEMES[scheme] if isinstance(scheme, str) else int(scheme)
    p, f, k = _ptr_flags(waveform, np.float64)
    ms = ctypes.c_float(0.0)
    _check(ctx, load().gtp_run_power_scheme(ctx, int(window), int(bin_ps), s, p, f, ctypes.byref(ms)))
    return float(ms.value)


def gtp_gate_energy(ctx, window: int, e_leak=None, e_int=None, e_sw=None, n_events=None, final_state=None) -> None:
    args = [_ptr_flags(e_leak, np.float64), _ptr_flags(e_int, np.float64), _ptr_flags(e_sw, np.float64),
            _ptr_flags(n_events, np.int64), _ptr_flags(final_state, np.uint8)]
    flags = {a[1] for a in args if a[0] is not None}
    if len(flags) > 1:
        raise ValueError("outputs must all be host or all be device")
    f = flags.pop() if flags else GTP_HOST
    _check(ctx, load().gtp_gate_energy(ctx, int(window), *[a[0] for a in args], f))


def gtp_run_power_batched(ctx, windows: Sequence[int], bin_ps: int, waveforms: Sequence, graph: bool = False) -> None:
    w = np.ascontiguousarray(windows, np.int32)
    ptrs = [_ptr_flags(x, np.float64) for x in waveforms]
    flags = {p[1] for p in ptrs if p[0] is not None}
    if len(flags) > 1:
        raise ValueError("waveforms must all be host or all be device")
    f = (flags.pop() if flags else GTP_HOST) | (GTP_GRAPH if graph else 0)
    arr = (ctypes.c_void_p * len(ptrs))(*[p[0] for p in ptrs])
    _check(ctx, load().gtp_run_power_batched(ctx, len(w), w.ctypes.data, int(bin_ps), ctypes.cast(arr, ctypes.c_void_p), f))


def gtp_autotune(ctx, windows: Sequence[int], bin_ps: int, iters: int = 3) -> float:
    w = np.ascontiguousarray(windows, np.int32)
    best = ctypes.c_double(0.0)
    _check(ctx, load().gtp_autotune(ctx, len(w), w.ctypes.data, int(bin_ps), int(iters), ctypes.byref(best)))
    return best.value


def gtp_run_power_backward(ctx, window: int, bin_ps: int, dL_dP, dC=None, d_escale=None, d_lscale=None) -> None:
    ptr = lambda t: None if t is None else t.data_ptr()  # device tensors
    _check(ctx, load().gtp_run_power_backward(ctx, int(window), int(bin_ps), ptr(dL_dP), ptr(dC), ptr(d_escale),
                                              ptr(d_lscale)))


def gtp_set_param(ctx, key: str, value: int) -> None:
    _check(ctx, load().gtp_set_param(ctx, key.encode(), int(value)))


def gtp_get_param(ctx, key: str) -> int:
    return int(load().gtp_get_param(ctx, key.encode()))


def _noalloc_validate(n_in, e_int, p_leak, cell, load_ff, slew_ps, window_ps, gate_offsets, events, init_state,
                      bin_ps, slew_axis_len, load_axis_len, outputs, require_cuda: bool = True):
    """Every check gtp_run_power_noalloc's arguments need before the call.
    The C side cannot see the length of a device array, so a short output or
    input here would become an out-of-bounds device access there; the device
    of every tensor must also be the one the call runs on.  Returns
    (n_gates, slew_stride, device).  Raises TypeError or ValueError."""
    import torch
    ni = np.ascontiguousarray(n_in, np.int32)
    want = [("e_int", e_int, torch.float32), ("p_leak", p_leak, torch.float32), ("cell", cell, torch.int32),
            ("load_ff", load_ff, torch.float32), ("slew_ps", slew_ps, torch.float32),
            ("gate_offsets", gate_offsets, torch.int64), ("events", events, torch.int32),
            ("init_state", init_state, torch.uint8)]
    want += [(k, v, torch.uint8 if k == "final_state" else torch.float64) for k, v in outputs.items()]
    device = None
    for name, t, dt in want:
        if t is None:
            if name in outputs:
                continue
            raise TypeError(f"gtp_run_power_noalloc: {name} is required")
        if not isinstance(t, torch.Tensor) or t.dtype != dt or not t.is_contiguous():
            raise TypeError(f"gtp_run_power_noalloc: {name} must be a contiguous {dt} tensor")
        if require_cuda and not t.is_cuda:
            raise TypeError(f"gtp_run_power_noalloc: {name} must be a CUDA tensor")
        if device is None:
            device = t.device
        elif t.device != device:
            raise ValueError(f"gtp_run_power_noalloc: {name} is on {t.device}, other arrays on {device}")
    if len(ni) == 0 or (ni < 1).any() or (ni >= GTP_MAX_PINS).any():
        raise ValueError("gtp_run_power_noalloc: n_in must hold 1..7 inputs per cell")
    tsize = int(slew_axis_len) * int(load_axis_len)
    n_tab = int(sum(int(k) * (2 << (int(k) - 1)) for k in ni))
    n_leak = int(sum(2 << int(k) for k in ni))
    if e_int.numel() != n_tab * tsize:
        raise ValueError(f"gtp_run_power_noalloc: e_int holds {e_int.numel()} floats, the library needs {n_tab * tsize}")
    if p_leak.numel() != n_leak:
        raise ValueError(f"gtp_run_power_noalloc: p_leak holds {p_leak.numel()} floats, the library needs {n_leak}")
    G = int(cell.numel())
    if G <= 0:
        raise ValueError("gtp_run_power_noalloc: no gates")
    for name, t in (("load_ff", load_ff), ("init_state", init_state)):
        if t.numel() != G:
            raise ValueError(f"gtp_run_power_noalloc: {name} has {t.numel()} entries for {G} gates")
    if gate_offsets.numel() != G + 1:
        raise ValueError(f"gtp_run_power_noalloc: gate_offsets has {gate_offsets.numel()} entries, needs {G + 1}")
    if slew_ps.dim() == 3:
        if slew_ps.shape[0] != G or slew_ps.shape[2] != 2:
            raise ValueError(f"gtp_run_power_noalloc: slew_ps is {tuple(slew_ps.shape)}, needs [{G}, stride, 2]")
        stride = int(slew_ps.shape[1])
    else:
        if slew_ps.numel() % (2 * G):
            raise ValueError("gtp_run_power_noalloc: slew_ps must hold n_gates * stride * 2 floats")
        stride = int(slew_ps.numel() // (2 * G))
    if stride < int(ni.max()):
        raise ValueError(f"gtp_run_power_noalloc: slew stride {stride} below the widest cell's {int(ni.max())} inputs")
    if events.dim() != 2 or events.shape[1] != 2:
        raise ValueError(f"gtp_run_power_noalloc: events must be [n_events, 2] int32, got {tuple(events.shape)}")
    if int(bin_ps) <= 0 or int(window_ps) <= 0 or int(window_ps) % int(bin_ps):
        raise ValueError("gtp_run_power_noalloc: window_ps must be a positive multiple of bin_ps > 0")
    n_bins = int(window_ps) // int(bin_ps)
    wf = outputs.get("waveform")
    if wf is not None and wf.numel() != n_bins:
        raise ValueError(f"gtp_run_power_noalloc: waveform has {wf.numel()} entries for {n_bins} bins")
    for name in ("e_leak", "e_int_out", "e_sw", "final_state"):
        t = outputs.get(name)
        if t is not None and t.numel() != G:
            raise ValueError(f"gtp_run_power_noalloc: {name} has {t.numel()} entries for {G} gates")
    return G, stride, device


def gtp_run_power_noalloc(n_in, vdd, slew_axis, load_axis, e_int, p_leak, cell, load_ff, slew_ps, window_ps: int,
                          gate_offsets, events, init_state, bin_ps: int, waveform=None, e_leak=None, e_int_out=None,
                          e_sw=None, final_state=None, stream: Optional[int] = None) -> None:
    """The allocation-free single-window walk.  n_in and the axes are host
    arrays; every other array is a contiguous CUDA tensor, all on one device
    (slew_ps shaped [G, stride, 2], events [E, 2] int32); outputs may be None.
    Every length is checked here, and the call runs with the tensors' device
    current.  Raises TypeError / ValueError before the call, GtpError with the
    returned code after it."""
    import torch
    ni = np.ascontiguousarray(n_in, np.int32)
    sa = np.ascontiguousarray(slew_axis, np.float32)
    la = np.ascontiguousarray(load_axis, np.float32)
    outputs = dict(waveform=waveform, e_leak=e_leak, e_int_out=e_int_out, e_sw=e_sw, final_state=final_state)
    G, stride, device = _noalloc_validate(ni, e_int, p_leak, cell, load_ff, slew_ps, window_ps, gate_offsets, events,
                                          init_state, bin_ps, len(sa), len(la), outputs)
    ptr = lambda t: None if t is None else t.data_ptr()
    with torch.cuda.device(device):
        rc = load().gtp_run_power_noalloc(stream, len(ni), ni.ctypes.data, float(vdd), len(sa), sa.ctypes.data,
                                          len(la), la.ctypes.data, ptr(e_int), int(e_int.numel()), ptr(p_leak),
                                          int(p_leak.numel()), G, ptr(cell), ptr(load_ff), ptr(slew_ps), stride,
                                          int(window_ps), int(events.shape[0]), ptr(gate_offsets), ptr(events),
                                          ptr(init_state), int(bin_ps), ptr(waveform), ptr(e_leak), ptr(e_int_out),
                                          ptr(e_sw), ptr(final_state))
    if rc != GTP_OK:
        raise GtpError(rc, "gtp_run_power_noalloc failed")


# ------------------------------------------------------------------ convenience object
class Engine:
    """One context on one GPU, enqueueing on torch's current stream."""

    def __init__(self, device: int = 0, stream=None):
        import torch
        self.device = torch.device("cuda", device)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        self.ctx = gtp_create(device, stream.cuda_stream)
        self.n_gates = 0
        self.n_pattern_gates = 0
        self.n_cells = 0
        self.windows: Dict[int, dict] = {}

    def close(self):
        if self.ctx:
            gtp_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load_library(self, lib) -> None:
        gtp_load_library(self.ctx, lib.n_in, lib.vdd, lib.slew_axis, lib.load_axis, lib.e_int, lib.p_leak)
        self.n_cells = len(lib.n_in)

    def set_scales(self, escale=None, lscale=None) -> None:
        gtp_set_scales(self.ctx, escale, lscale)

    def load_netlist(self, net) -> None:
        gtp_load_netlist(self.ctx, net.cell, net.load_ff, net.slew_ps)
        self.n_gates = len(net.cell)

    def set_load(self, load_ff) -> None:
        gtp_set_load(self.ctx, load_ff)

    def set_glitch(self, clock_ps: int, out_slew=None) -> None:
        gtp_set_glitch(self.ctx, clock_ps, out_slew)

    def design_power(self, window: int, waveform=None) -> dict:
        return gtp_design_power(self.ctx, window, waveform)

    def gate_glitch(self, window: int, device: bool = True):
        """Per-gate glitch energy (fJ, float64) of the window's last run."""
        import torch
        out = (torch.empty(self.n_gates, dtype=torch.float64, device=self.device) if device
               else np.empty(self.n_gates))
        gtp_gate_glitch(self.ctx, window, out)
        return out

    def load_pattern_cells(self, plib) -> None:
        gtp_load_pattern_cells(self.ctx, plib)

    def load_pattern_netlist(self, pnet) -> None:
        gtp_load_pattern_netlist(self.ctx, pnet)
        self.n_pattern_gates = len(pnet.cell)

    def load_pattern_events(self, window: int, ptrace=None, *, offsets=None, t_ps=None, pin=None, value=None,
                            init_state=None) -> None:
        """A window's pattern-gate events from a synth.patterns.PatternTrace
        or explicit arrays (load the window's ordinary events first)."""
        if ptrace is not None:
            offsets, t_ps, pin, value, init_state = (ptrace.offsets, ptrace.t_ps, ptrace.pin, ptrace.value,
                                                     ptrace.init_state)
        gtp_load_pattern_events(self.ctx, window, offsets, t_ps, pin, value, init_state)

    def pattern_gate_energy(self, window: int, device: bool = False) -> Dict[str, object]:
        """Per-pattern-gate results of the window's last run (numpy, or CUDA
        tensors with device=True)."""
        n = self.n_pattern_gates
        if device:
            import torch
            out = {k: torch.empty(n, dtype=torch.float64, device=self.device) for k in ("e_leak", "e_int", "e_sw",
                                                                                        "e_gl")}
            out["n_events"] = torch.empty(n, dtype=torch.int64, device=self.device)
            out["final_state"] = torch.empty(n, dtype=torch.int32, device=self.device)
        else:
            out = {k: np.empty(n) for k in ("e_leak", "e_int", "e_sw", "e_gl")}
            out["n_events"] = np.empty(n, np.int64)
            out["final_state"] = np.empty(n, np.uint32)
        gtp_pattern_gate_energy(self.ctx, window, out["e_leak"], out["e_int"], out["e_sw"], out["e_gl"],
                                out["n_events"], out["final_state"])
        return out

    def pattern_gate_gradient(self, window: int, device: bool = False):
        """dL/dC of the pattern gates from the window's last backward run
        (numpy float32, or a CUDA tensor with device=True)."""
        n = self.n_pattern_gates
        if device:
            import torch
            out = torch.empty(n, dtype=torch.float32, device=self.device)
        else:
            out = np.empty(n, np.float32)
        gtp_pattern_gate_gradient(self.ctx, window, out)
        return out

    def load_events(self, window: int, trace=None, *, window_ps=None, offsets=None, records=None, init_state=None,
                    borrow: bool = False, packed=None) -> None:
        """Load a window from a trace or explicit arrays; `packed` (the
        gtp_pack_events form) replaces the records."""
        if trace is not None:
            window_ps, offsets, records, init_state = trace.window_ps, trace.offsets, trace.records, trace.init_state
        if packed is not None:
            gtp_load_events(self.ctx, window, window_ps, offsets, packed, init_state, packed=True)
        else:
            gtp_load_events(self.ctx, window, window_ps, offsets, records, init_state, borrow=borrow)
        self.windows[window] = dict(window_ps=int(window_ps))

    def run_power(self, window: int, bin_ps: int, out=None, graph: bool = False):
        """Waveform in W as a float64 CUDA tensor of window_ps / bin_ps bins
        (graph: capture the run in a CUDA graph once and replay it)."""
        import torch
        nb = self.windows[window]["window_ps"] // bin_ps
        if out is None:
            out = torch.empty(nb, dtype=torch.float64, device=self.device)
        gtp_run_power(self.ctx, window, bin_ps, out, graph=graph)
        return out

    def run_power_components(self, window: int, bin_ps: int, out=None, total=None):
        """Per-component waveforms in W, [4][window_ps / bin_ps] float64 rows
        leakage, internal, switching, glitch (a CUDA tensor unless `out` is a
        host array); `total`, if given, receives the total waveform."""
        import torch
        nb = self.windows[window]["window_ps"] // bin_ps
        if out is None:
            out = torch.empty((4, nb), dtype=torch.float64, device=self.device)
        gtp_run_power_components(self.ctx, window, bin_ps, out, total)
        return out

    def run_power_scheme(self, window: int, bin_ps: int, scheme, out=None):
        """Waveform (W, float64 CUDA tensor unless `out` is a host array) by
        one of the paper's schemes ("naive", "sipl", "density", "fused");
        returns (waveform, kernel ms)."""
        import torch
        nb = self.windows[window]["window_ps"] // bin_ps
        if out is None:
            out = torch.empty(nb, dtype=torch.float64, device=self.device)
        ms = gtp_run_power_scheme(self.ctx, window, bin_ps, scheme, out)
        return out, ms

    def run_power_streamed(self, window: int, trace=None, bin_ps: int = 10, out=None, n_chunks: int = 8, *,
                           window_ps=None, offsets=None, records=None, init_state=None, packed=None):
        """Waveform (float64; on the device unless `out` is a host array) of a
        window streamed from host arrays in n_chunks overlapped chunks;
        `packed` (the gtp_pack_events form) replaces the records."""
        import torch
        if trace is not None:  # explicit arrays take precedence (e.g. pinned records)
            window_ps = trace.window_ps if window_ps is None else window_ps
            offsets = trace.offsets if offsets is None else offsets
            records = trace.records if records is None else records
            init_state = trace.init_state if init_state is None else init_state
        if out is None:
            out = torch.empty(int(window_ps) // bin_ps, dtype=torch.float64, device=self.device)
        if packed is not None:
            gtp_run_power_streamed(self.ctx, window, window_ps, offsets, packed, init_state, bin_ps, out, n_chunks,
                                   n_events=int(np.asarray(offsets)[-1]), packed=True)
        else:
            gtp_run_power_streamed(self.ctx, window, window_ps, offsets, records, init_state, bin_ps, out, n_chunks)
        self.windows[window] = dict(window_ps=int(window_ps))
        return out

    def gate_energy(self, window: int, device: bool = True):
        import torch
        G = self.n_gates
        if device:
            kw = dict(device=self.device)
            r = dict(e_leak=torch.empty(G, dtype=torch.float64, **kw), e_int=torch.empty(G, dtype=torch.float64, **kw),
                     e_sw=torch.empty(G, dtype=torch.float64, **kw), n_events=torch.empty(G, dtype=torch.int64, **kw),
                     final_state=torch.empty(G, dtype=torch.uint8, **kw))
        else:
            r = dict(e_leak=np.empty(G), e_int=np.empty(G), e_sw=np.empty(G), n_events=np.empty(G, np.int64),
                     final_state=np.empty(G, np.uint8))
        gtp_gate_energy(self.ctx, window, r["e_leak"], r["e_int"], r["e_sw"], r["n_events"], r["final_state"])
        return r

    def run_power_batched(self, windows: Sequence[int], bin_ps: int, outs=None, graph: bool = False):
        import torch
        if outs is None:
            outs = [torch.empty(self.windows[w]["window_ps"] // bin_ps, dtype=torch.float64, device=self.device)
                    for w in windows]
        gtp_run_power_batched(self.ctx, windows, bin_ps, outs, graph=graph)
        return outs

    def run_power_backward(self, window: int, bin_ps: int, dL_dP):
        """Gradients (dC[n_gates], d_escale[n_cells], d_lscale[n_cells]) as
        float32 CUDA tensors, for dL/dP given per bin (float32 CUDA)."""
        import torch
        kw = dict(dtype=torch.float32, device=self.device)
        dC = torch.empty(self.n_gates, **kw)
        de = torch.empty(self.n_cells, **kw)
        dl = torch.empty(self.n_cells, **kw)
        gtp_run_power_backward(self.ctx, window, bin_ps, dL_dP.to(torch.float32).contiguous(), dC, de, dl)
        return dC, de, dl

    def autotune(self, windows: Sequence[int], bin_ps: int, iters: int = 3) -> float:
        return gtp_autotune(self.ctx, windows, bin_ps, iters)

    def set_param(self, key: str, value: int) -> None:
        gtp_set_param(self.ctx, key, value)

    def get_param(self, key: str) -> int:
        return gtp_get_param(self.ctx, key)
