"""CPU oracle for windowed median/MAD RFI excision (Section II-D, Eq. 1 and Eq. 2), its
Median-of-MAD variant (Eq. 3), and the improvement metric of Section III-A.

TEST INFRASTRUCTURE: only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline leg may import this package. The definition it computes, and every reading it takes
where the paper is silent, is stated in ``rfi_oracle.cpp``.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from .build import build

_lock = threading.Lock()
_lib = None

ZERO, CONST, CLIP, NOISE = 0, 1, 2, 3
STATUS_OK, STATUS_BAD_ARG, STATUS_SAMPLE_RANGE = 0, 1, 6


class OracleArgs(ctypes.Structure):
    _fields_ = [
        ("x", ctypes.c_void_p), ("z", ctypes.c_void_p), ("bits", ctypes.c_int32),
        ("len", ctypes.c_int64), ("W", ctypes.c_int32), ("abs0", ctypes.c_int64),
        ("n_sigma", ctypes.c_double), ("mode", ctypes.c_int32), ("const_value", ctypes.c_int32),
        ("seed", ctypes.c_uint64), ("stream_id", ctypes.c_uint32),
        ("mask", ctypes.c_void_p), ("counts", ctypes.c_void_p), ("median", ctypes.c_void_p),
        ("mad", ctypes.c_void_p), ("nthreads", ctypes.c_int32),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.oracle_excise.restype = ctypes.c_int
            L.oracle_excise.argtypes = [ctypes.POINTER(OracleArgs)]
            L.oracle_k_q16.restype = ctypes.c_int64
            L.oracle_k_q16.argtypes = [ctypes.c_double]
            L.oracle_philox4x32_10.restype = None
            L.oracle_philox4x32_10.argtypes = [ctypes.POINTER(ctypes.c_uint32)] * 3
            L.oracle_noise_value.restype = ctypes.c_int32
            L.oracle_noise_value.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64,
                                             ctypes.c_uint32, ctypes.c_int64, ctypes.c_int32]
            L.oracle_excise_mom.restype = ctypes.c_int
            L.oracle_excise_mom.argtypes = [ctypes.POINTER(OracleArgs), ctypes.c_int32, ctypes.c_void_p,
                                            ctypes.c_int64, ctypes.c_void_p]
            L.oracle_median_mad.restype = None
            L.oracle_median_mad.argtypes = [ctypes.c_void_p, ctypes.c_int64,
                                            ctypes.POINTER(ctypes.c_int32),
                                            ctypes.POINTER(ctypes.c_int32)]
            _lib = L
    return _lib


def k_q16(k: float) -> int:
    """k*1.4826 in Q16, rounded half up (the fixed-point form of Eq. 1's multiple)."""
    return int(lib().oracle_k_q16(float(k)))


def philox4x32_10(ctr, key):
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().oracle_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def noise_value(M: int, D: int, seed: int, stream_id: int, idx: int, bits: int = 8) -> int:
    return int(lib().oracle_noise_value(M, D, seed, stream_id, idx, bits))


def median_mad(x) -> tuple[int, int]:
    """Lower median M and lower-median MAD D of one window of integers."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.int32))
    M, D = ctypes.c_int32(), ctypes.c_int32()
    lib().oracle_median_mad(a.ctypes.data, a.size, ctypes.byref(M), ctypes.byref(D))
    return M.value, D.value


def excise_mom(x: np.ndarray, W: int, k: float, mode: int, k_mom: int, const: int = 0, seed: int = 0,
               stream_id: int = 0, abs0: int = 0, bits: int | None = None, threads: int = 1,
               history=None, want=("z", "mask", "counts", "median", "mad", "mom")):
    """Median-of-MAD excision (Eq. 3) of one stream or slice; ``history`` is the MADs of the
    windows just before the slice (oldest first, at most k_mom - 1). Returns excise()'s dict
    plus ``mom``, the dispersion each window used."""
    x = np.ascontiguousarray(x)
    if bits is None:
        bits = 8 if x.dtype == np.int8 else 12
    assert x.dtype == (np.int8 if bits == 8 else np.int16)
    n = x.size
    nw = -(-n // W) if (n > 0 and W > 0) else 0
    res = {"z": np.empty_like(x)}
    res["mask"] = np.zeros(mask_words(W, nw), np.uint32) if "mask" in want else None
    for key, dt in (("counts", np.uint32), ("median", np.int32), ("mad", np.int32), ("mom", np.int32)):
        res[key] = np.zeros(nw, dt) if key in want else None
    hist = np.ascontiguousarray(history if history is not None else np.zeros(0), dtype=np.int32)

    def p(a):
        return None if a is None else a.ctypes.data

    args = OracleArgs(x.ctypes.data, res["z"].ctypes.data, bits, n, W, abs0, float(k), mode, const,
                      seed, stream_id, p(res["mask"]), p(res["counts"]), p(res["median"]),
                      p(res["mad"]), max(1, int(threads)))
    res["status"] = int(lib().oracle_excise_mom(ctypes.byref(args), int(k_mom),
                                                p(hist) if hist.size else None, int(hist.size),
                                                p(res["mom"])))
    return res


def window_power(x: np.ndarray, W: int) -> np.ndarray:
    """Detected power of each data window: the sum of x_i^2 over its samples (int64), the
    per-window point of the power series the improvement metric is computed on."""
    x = np.ascontiguousarray(x).astype(np.int64)
    nw = -(-x.size // W)
    p = np.zeros(nw, np.int64)
    for w in range(nw):
        seg = x[w * W:(w + 1) * W]
        p[w] = int(np.dot(seg, seg))
    return p


def mean_to_rms(power: np.ndarray, windows_per_point: int = 1, points_per_block: int = 64) -> float:
    """Average mean-to-RMS ratio of a detected-power series (Section III-A): the per-window
    powers are summed into points of windows_per_point windows; the points are cut into blocks
    of points_per_block; each block gives mean / RMS deviation about its mean; the blocks'
    ratios are averaged. Blocks of zero RMS deviation are left out; a partial block is dropped."""
    p = np.asarray(power, dtype=np.float64)
    npt = p.size // windows_per_point
    pts = p[:npt * windows_per_point].reshape(npt, windows_per_point).sum(axis=1)
    nb = npt // points_per_block
    ratios = []
    for b in range(nb):
        blk = pts[b * points_per_block:(b + 1) * points_per_block]
        mean = blk.sum() / blk.size
        rms = np.sqrt(((blk - mean) ** 2).sum() / blk.size)
        if rms > 0:
            ratios.append(mean / rms)
    return float(np.mean(ratios)) if ratios else float("nan")


def improvement_db(power_unfiltered, power_filtered, windows_per_point: int = 1, points_per_block: int = 64):
    """The improvement metric of Section III-A from the per-window detected power of the
    unfiltered and the filtered signal: 10 log10 of the ratio of their average mean-to-RMS
    ratios, taken as S_F / S_U so that a positive value is an improvement. Returns
    (dB, S_U, S_F)."""
    su = mean_to_rms(power_unfiltered, windows_per_point, points_per_block)
    sf = mean_to_rms(power_filtered, windows_per_point, points_per_block)
    return 10.0 * np.log10(sf / su), su, sf


def mask_words(W: int, n_windows: int) -> int:
    return n_windows * ((W + 31) // 32)


def excise(x: np.ndarray, W: int, k: float, mode: int, const: int = 0, seed: int = 0,
           stream_id: int = 0, abs0: int = 0, bits: int | None = None, threads: int = 1,
           out: np.ndarray | None = None, want=("z", "mask", "counts", "median", "mad")):
    """Excise one stream (or a window-aligned slice of one). Returns a dict of numpy arrays
    plus ``status`` (0 ok, 1 bad argument, 6 12-bit sample out of range)."""
    x = np.ascontiguousarray(x)
    if bits is None:
        bits = 8 if x.dtype == np.int8 else 12
    assert x.dtype == (np.int8 if bits == 8 else np.int16)
    n = x.size
    nw = -(-n // W) if (n > 0 and W > 0) else 0
    res = {}
    z = out if out is not None else np.empty_like(x)
    res["z"] = z
    res["mask"] = np.zeros(mask_words(W, nw), np.uint32) if "mask" in want else None
    res["counts"] = np.zeros(nw, np.uint32) if "counts" in want else None
    res["median"] = np.zeros(nw, np.int32) if "median" in want else None
    res["mad"] = np.zeros(nw, np.int32) if "mad" in want else None

    def p(a):
        return None if a is None else a.ctypes.data

    args = OracleArgs(x.ctypes.data, z.ctypes.data, bits, n, W, abs0, float(k), mode, const,
                      seed, stream_id, p(res["mask"]), p(res["counts"]), p(res["median"]),
                      p(res["mad"]), max(1, int(threads)))
    res["status"] = int(lib().oracle_excise(ctypes.byref(args)))
    return res
