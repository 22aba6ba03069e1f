"""Seeded random sweep: the GPU path against the oracle, bit for bit, over random combinations of
sample width, window lengths (1 to 70000, any residue mod 16 and 32), stream lengths (ragged
tails), k, replacement mode, constant, noise seed, stream ids and plan form (batched, CUDA
graph, digital noise as a second kernel, per-stream). Each case is small enough for the oracle
to finish in well under a second; the draw is fixed by the case index."""
import numpy as np
import pytest

import synth

from .parity import assert_same, gpu_run, oracle_run

pytestmark = pytest.mark.gpu

FORMS = [0, 0x4, 0x40, 0x40 | 0x4, 0x1]


def _case(i):
    rng = np.random.default_rng(1000 + i)
    bits = int(rng.choice([8, 12]))
    S = int(rng.integers(1, 5))
    wins, lens = [], []
    for _ in range(S):
        W = int(rng.choice([int(rng.integers(1, 64)), int(rng.integers(64, 5000)), 4096, 16384,
                            int(rng.integers(5000, 70000))]))
        W = min(W, 65536)
        nw = int(rng.integers(1, max(2, 300000 // W)))
        n = max(1, nw * W - int(rng.integers(0, W)))
        wins.append(W)
        lens.append(n)
    k = float(rng.choice([1.5, 2.0, 3.0, 3.5, 5.0, float(rng.uniform(0.5, 8.0))]))
    mode = int(rng.integers(0, 4))
    lo, hi = (-128, 127) if bits == 8 else (-2048, 2047)
    const = int(rng.integers(lo - 50, hi + 50))  # saturated by the plan
    seed = int(rng.integers(0, 2 ** 63))
    sids = [int(v) for v in rng.integers(0, 2 ** 32, size=S)]
    flags = int(FORMS[i % len(FORMS)])
    sigma = float(rng.uniform(2.0, 30.0)) if bits == 8 else float(rng.uniform(20.0, 300.0))
    p = synth.params(seed=int(rng.integers(0, 1 << 30)), sigma=sigma, burst_rate=float(rng.uniform(1e-4, 2e-2)),
                     burst_len_max=int(rng.integers(1, 300)), bits=bits)
    xs = [synth.fill(p, s, n) for s, n in enumerate(lens)]
    return bits, wins, lens, k, mode, const, seed, sids, flags, xs


@pytest.mark.parametrize("i", range(40))
def test_random_case(cuda, rfi, i):
    bits, wins, lens, k, mode, const, seed, sids, flags, xs = _case(i)
    got, st, totals, _ = gpu_run(rfi, xs, wins, bits, k, mode, const, seed, flags=flags, stream_ids=sids)
    assert st == 0
    ref = oracle_run(xs, wins, bits, k, mode, const, seed, sids)
    assert_same(got, ref, "case %d: bits %d W %s mode %d k %g flags %#x" % (i, bits, wins, mode, k, flags))
    assert totals.flagged == sum(int(r["counts"].sum()) for r in ref)
    assert totals.windows == sum(-(-n // w) for n, w in zip(lens, wins))


def _mom_case(i):
    rng = np.random.default_rng(5000 + i)
    bits = int(rng.choice([8, 12]))
    S = int(rng.integers(1, 4))
    wins = [int(rng.choice([256, 512, 1000, 1024, 2048, 4096, int(rng.integers(16, 3000))])) for _ in range(S)]
    lens = [max(1, int(rng.integers(1, 200)) * W - int(rng.integers(0, W))) for W in wins]
    kmom = int(rng.choice([2, 3, 7, 64, 300, 5000]))
    k = float(rng.choice([2.0, 3.0, 3.5, 5.0]))
    mode = int(rng.integers(0, 4))
    flags = int([0, 0x4, 0x40, 0x44][i % 4])
    sigma = 16.0 if bits == 8 else 120.0
    p = synth.params(seed=int(rng.integers(0, 1 << 30)), sigma=sigma, burst_rate=float(rng.uniform(1e-4, 5e-3)),
                     burst_len_max=int(rng.integers(16, 5000)), bits=bits)
    xs = [synth.fill(p, s, n) for s, n in enumerate(lens)]
    return bits, wins, k, mode, kmom, flags, xs


@pytest.mark.parametrize("i", range(16))
def test_random_mom_case(cuda, rfi, i):
    import oracle
    from .test_mom_gpu import _check, _gpu
    bits, wins, k, mode, kmom, flags, xs = _mom_case(i)
    sids = [7 * s + 1 for s in range(len(xs))]
    st, totals, got = _gpu(rfi, xs, wins, bits, k, mode, kmom, const=3, seed=1234 + i, flags=flags, sids=sids)
    assert st == rfi.RFI_OK and totals.device_status == rfi.RFI_OK
    flagged = 0
    for s, x in enumerate(xs):
        ref = oracle.excise_mom(x, wins[s], k, mode, kmom, const=3, seed=1234 + i, stream_id=sids[s], bits=bits,
                                threads=8)
        _check(got[s], ref, "case %d stream %d (W %d, kmom %d, mode %d, flags %#x)" % (i, s, wins[s], kmom, mode, flags))
        flagged += int(ref["counts"].sum())
    assert totals.flagged == flagged


@pytest.mark.parametrize("i", range(12))
def test_random_digital_copy_case(cuda, rfi, i):
    from .test_copies_gpu import _check, _run, _streams
    rng = np.random.default_rng(7000 + i)
    bits = int(rng.choice([8, 12]))
    S = int(rng.integers(1, 4))
    wins = [int(rng.choice([16, 100, 1024, 4096, 16384, int(rng.integers(1, 20000))])) for _ in range(S)]
    lens = [max(1, int(rng.integers(1, 30)) * W - int(rng.integers(0, W))) for W in wins]
    nvar = int(rng.integers(1, 9))
    variants = [(float(rng.choice([2.0, 3.0, 3.5, 5.0, float(rng.uniform(1.0, 6.0))])), int(rng.integers(0, 4)),
                 int(rng.integers(-200, 200)), int(rng.integers(0, 2 ** 63))) for _ in range(nvar)]
    xs = _streams(bits, lens, 70 + i)
    st, totals, res, meds, mads = _run(rfi, xs, wins, bits, variants, flags=int([0, 0x4][i % 2]))
    assert st == rfi.RFI_OK
    assert totals.flagged == _check(xs, wins, bits, variants, res, meds, mads)


@pytest.mark.parametrize("i", range(12))
def test_random_output_format_case(cuda, rfi, i):
    from .test_format_gpu import _check, _run, _streams
    rng = np.random.default_rng(9000 + i)
    bits = int(rng.choice([8, 12]))
    fmt = rfi.RFI_OUT_F16 if bits == 12 or i % 2 else rfi.RFI_OUT_BF16
    S = int(rng.integers(1, 4))
    wins = [int(rng.choice([7, 64, 1000, 4096, 16384, 65536, int(rng.integers(1, 30000))])) for _ in range(S)]
    lens = [max(1, int(rng.integers(1, 20)) * W - int(rng.integers(0, W))) for W in wins]
    k = float(rng.choice([2.0, 3.0, 3.5, 5.0]))
    mode = int(rng.integers(0, 4))
    xs = _streams(bits, lens, 90 + i)
    res = _run(rfi, xs, wins, bits, k, mode, fmt, flags=int([0, 0x4, 0x20][i % 3]), offset=2 * int(rng.integers(0, 4)))
    _check(xs, wins, bits, k, mode, res)


@pytest.mark.parametrize("i", range(10))
def test_random_power_case(cuda, rfi, i):
    import oracle
    from .test_power_gpu import _run, _streams
    rng = np.random.default_rng(11000 + i)
    bits = int(rng.choice([8, 12]))
    S = int(rng.integers(1, 4))
    wins = [int(rng.choice([1, 33, 512, 4096, 16384, 65536, int(rng.integers(1, 30000))])) for _ in range(S)]
    lens = [max(1, int(rng.integers(1, 20)) * W - int(rng.integers(0, W))) for W in wins]
    mode = int(rng.integers(0, 4))
    k = float(rng.choice([2.0, 3.0, 5.0]))
    flags = rfi.RFI_PLAN_POWER | int([0, 0x4, 0x20][i % 3])
    xs = _streams(bits, lens, 110 + i)
    z, m, pw = _run(rfi, xs, wins, bits, mode, flags, seed=70 + i, k=k)
    for s, x in enumerate(xs):
        ref = oracle.excise(x, wins[s], k, mode, const=2, seed=70 + i, stream_id=s, bits=bits, threads=8)
        assert np.array_equal(z[s], ref["z"]), "case %d stream %d samples" % (i, s)
        assert np.array_equal(pw[s][0::2], oracle.window_power(x, wins[s])), "case %d stream %d input power" % (i, s)
        assert np.array_equal(pw[s][1::2], oracle.window_power(ref["z"], wins[s])), "case %d stream %d output" % (i, s)
