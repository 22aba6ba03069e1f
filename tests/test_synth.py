"""The synthetic feed: determinism, chunk consistency and its stated statistics."""
import numpy as np

import synth
from synth import workloads


def test_chunks_equal_whole_stream():
    p = synth.params(seed=9, sigma=16.0, burst_rate=1e-2, burst_len_max=64, bits=8)
    whole = synth.fill(p, 4, 300_000, threads=4)
    for i0, n in [(0, 1), (1, 17), (12345, 70000), (299_990, 10), (65536 - 3, 65536 + 7)]:
        assert (synth.fill(p, 4, n, i0=i0, threads=3) == whole[i0:i0 + n]).all()
    assert (synth.fill(p, 4, 300_000, threads=1) == whole).all()
    assert not (synth.fill(p, 5, 1000) == whole[:1000]).all()


def test_clean_noise_statistics():
    p = synth.params(seed=10, sigma=16.0, burst_rate=0.0, burst_len_max=1, bits=8)
    x = synth.fill(p, 0, 1 << 20).astype(float)
    assert abs(x.mean()) < 0.1
    # variance of a rounded Gaussian: sigma^2 + 1/12 (Sheppard)
    assert abs(x.var() / (16.0 ** 2 + 1 / 12) - 1) < 0.01


def test_burst_coverage_and_twelve_bit_range():
    lam, L = 5e-3, 256
    p = synth.params(seed=11, sigma=120.0, burst_rate=lam, burst_len_max=L, bits=12,
                     amp=(4.0, 30.0), drift_amp=50.0)
    x = synth.fill(p, 1, 1 << 20)
    assert x.dtype == np.int16 and x.min() >= -2048 and x.max() <= 2047
    # burst starts are a Bernoulli(lam) process: coverage 1 - (1-lam)^E[L] for E[L] = (L+1)/2
    clean = synth.params(seed=11, sigma=120.0, burst_rate=0.0, burst_len_max=L, bits=12,
                         drift_amp=50.0)
    y = synth.fill(clean, 1, 1 << 20)
    cov = (x != y).mean()
    expect = 1 - (1 - lam) ** ((L + 1) / 2)
    assert abs(cov - expect) < 0.05


def test_workload_shapes():
    w2 = workloads.gwb60()
    assert len(w2.streams) == 60 and w2.total_samples == 60 << 26 and len(w2.variants) == 8
    rates = [s.feed.burst_rate for s in w2.streams]
    assert 1e-4 <= min(rates) and max(rates) <= 1e-2
    w3 = workloads.uneven60()
    assert all((1 << 22) <= s.length < (1 << 27) for s in w3.streams)
    assert {s.window for s in w3.streams} <= {1 << e for e in range(10, 17)}
    w4 = workloads.twelve60()
    assert w4.bits == 12 and w4.total_windows == 60 * (1 << 25) // 8192
    assert workloads.single().total_windows == 256
