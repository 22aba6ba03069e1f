"""Seeded synthetic feeds shared by the oracle and the GPU path (input generation only).

The feed model and its parameters are documented in ``feed.cpp``. ``workloads`` holds the
five workload definitions (stream counts, lengths, window lengths, feed parameters and the
excision settings they are run with).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "feed.cpp")
_LIB = os.path.join(_HERE, "libsynth.so")
_lock = threading.Lock()
_lib = None


class SynthParams(ctypes.Structure):
    _fields_ = [
        ("seed", ctypes.c_uint64),
        ("sigma", ctypes.c_double),
        ("burst_rate", ctypes.c_double),
        ("burst_len_max", ctypes.c_int32),
        ("bits", ctypes.c_int32),
        ("amp_lo", ctypes.c_double),
        ("amp_hi", ctypes.c_double),
        ("drift_amp", ctypes.c_double),
        ("drift_period", ctypes.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile libsynth.so next to its source (plain g++, no architecture flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-pthread",
                               "-ffp-contract=off", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.synth_fill.restype = ctypes.c_int
            lib.synth_fill.argtypes = [ctypes.c_void_p, ctypes.POINTER(SynthParams), ctypes.c_uint32,
                                       ctypes.c_int64, ctypes.c_int64, ctypes.c_int]
            _lib = lib
    return _lib


def params(seed, sigma, burst_rate, burst_len_max, bits=8, amp=(5.0, 15.0),
           drift_amp=0.0, drift_period=float(1 << 20)) -> SynthParams:
    return SynthParams(int(seed), float(sigma), float(burst_rate), int(burst_len_max), int(bits),
                       float(amp[0]), float(amp[1]), float(drift_amp), float(drift_period))


def fill(p: SynthParams, stream: int, n: int, i0: int = 0, out: np.ndarray | None = None,
         threads: int | None = None) -> np.ndarray:
    """Samples i0..i0+n-1 of stream ``stream`` as int8 (bits 8) or int16 (bits 12)."""
    dt = np.int8 if p.bits == 8 else np.int16
    if out is None:
        out = np.empty(n, dtype=dt)
    assert out.dtype == dt and out.size >= n and out.flags.c_contiguous
    nt = threads if threads is not None else (os.cpu_count() or 1)
    rc = _load().synth_fill(out.ctypes.data, ctypes.byref(p), int(stream), int(i0), int(n), int(nt))
    if rc != 0:
        raise ValueError("synth_fill rejected its arguments")
    return out
