"""The five synthetic workloads (stream shapes, feed parameters, excision settings).

All draws that shape a workload (per-stream burst rates, lengths and window lengths) come
from ``numpy.random.default_rng(<workload seed>)``, which is reproducible on every platform.

1. ``single``   1 stream x 2^20 int8, sigma 16, bursts rate 1e-3, length U{1..64},
                amplitude U[5,15] sigma; window 4096, k 3, zero replacement.
2. ``gwb60``    60 streams (30 antennas x 2 polarisations) x 2^26 int8, same model with a
                per-stream burst rate log-uniform in [1e-4, 1e-2]; window 16384,
                k in {3, 5} x {zero, constant 1, clip, noise (seed 7)}.
3. ``uneven60`` 60 int8 streams, lengths floor(2^U[22,27]), windows 2^U{10..16};
                k 3, noise replacement (seed 7).
4. ``twelve60`` 60 streams x 2^25 12-bit samples (int16 container), sigma 120, bursts rate
                5e-3, length U{1..256}, amplitude U[4,30] sigma, drift 50 LSB sinusoid of
                period 2^20 samples; window 8192, k 3.5, noise replacement (seed 7).
5. ``serve60``  the serving workload: 60 int8 streams shaped like ``gwb60``, window 16384,
                k 3, noise replacement (seed 7).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import params

ZERO, CONST, CLIP, NOISE = 0, 1, 2, 3
MODE_NAMES = {ZERO: "zero", CONST: "const", CLIP: "clip", NOISE: "noise"}


@dataclass
class Stream:
    index: int      # stream number: feed stream key and replacement-noise stream id
    length: int     # samples
    window: int     # window length W
    feed: object    # synth.SynthParams


@dataclass
class Variant:
    k: float
    mode: int
    const: int = 0
    seed: int = 0

    @property
    def name(self) -> str:
        return "k%g-%s" % (self.k, MODE_NAMES[self.mode])


@dataclass
class Workload:
    name: str
    bits: int
    streams: list = field(default_factory=list)
    variants: list = field(default_factory=list)

    @property
    def total_samples(self) -> int:
        return sum(s.length for s in self.streams)

    @property
    def total_windows(self) -> int:
        return sum(-(-s.length // s.window) for s in self.streams)


def _gwb_rates(n, seed):
    rng = np.random.default_rng(seed)
    return [float(10.0 ** (-4.0 + 2.0 * u)) for u in rng.uniform(size=n)]


def single(length=1 << 20, window=4096) -> Workload:
    f = params(seed=1, sigma=16.0, burst_rate=1e-3, burst_len_max=64, bits=8, amp=(5.0, 15.0))
    return Workload("single", 8, [Stream(0, length, window, f)], [Variant(3.0, ZERO, 0, 0)])


def gwb60(length=1 << 26, window=16384, nstreams=60) -> Workload:
    rates = _gwb_rates(60, 2)
    streams = [Stream(s, length, window,
                      params(seed=2, sigma=16.0, burst_rate=rates[s], burst_len_max=64, bits=8,
                             amp=(5.0, 15.0)))
               for s in range(nstreams)]
    variants = [Variant(k, m, 1 if m == CONST else 0, 7 if m == NOISE else 0)
                for k in (3.0, 5.0) for m in (ZERO, CONST, CLIP, NOISE)]
    return Workload("gwb60", 8, streams, variants)


def uneven60(nstreams=60, len_log2=(22.0, 27.0), win_log2=(10, 16)) -> Workload:
    rng = np.random.default_rng(3)
    lens = [int(math.floor(2.0 ** u)) for u in rng.uniform(len_log2[0], len_log2[1], size=60)]
    wins = [1 << int(e) for e in rng.integers(win_log2[0], win_log2[1] + 1, size=60)]
    rates = _gwb_rates(60, 3)
    streams = [Stream(s, lens[s], wins[s],
                      params(seed=3, sigma=16.0, burst_rate=rates[s], burst_len_max=64, bits=8,
                             amp=(5.0, 15.0)))
               for s in range(nstreams)]
    return Workload("uneven60", 8, streams, [Variant(3.0, NOISE, 0, 7)])


def twelve60(length=1 << 25, window=8192, nstreams=60) -> Workload:
    streams = [Stream(s, length, window,
                      params(seed=4, sigma=120.0, burst_rate=5e-3, burst_len_max=256, bits=12,
                             amp=(4.0, 30.0), drift_amp=50.0, drift_period=float(1 << 20)))
               for s in range(nstreams)]
    return Workload("twelve60", 12, streams, [Variant(3.5, NOISE, 0, 7)])


def serve60(window=16384, nstreams=60) -> Workload:
    rates = _gwb_rates(60, 5)
    streams = [Stream(s, 0, window,
                      params(seed=5, sigma=16.0, burst_rate=rates[s], burst_len_max=64, bits=8,
                             amp=(5.0, 15.0)))
               for s in range(nstreams)]
    return Workload("serve60", 8, streams, [Variant(3.0, NOISE, 0, 7)])
