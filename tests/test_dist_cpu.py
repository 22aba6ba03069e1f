"""The multi-GPU layout on CPU: two gloo ranks, each with its own antenna set (weak scaling).

Each rank excises its own streams with the CPU oracle; the ranks share nothing but the
benchmark's reductions. The test checks that the shards are disjoint, that their union is the
single-process workload, and that the sum / max reductions give the whole-job totals and the
slowest rank's time.
"""
import multiprocessing as mp
import os
import socket

import numpy as np

import oracle
import synth

FEED = dict(seed=31, sigma=16.0, burst_rate=3e-3, burst_len_max=64, bits=8)
N = 40000


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _excise(sid):
    x = synth.fill(synth.params(**FEED), sid, N)
    r = oracle.excise(x, 4096, 3.0, oracle.NOISE, seed=7, stream_id=sid)
    return int(r["counts"].sum()), x.size, int(np.bitwise_xor.reduce(r["z"].view(np.uint8)))


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    from paper_1710_08576_gb300 import dist as rdist
    g = rdist.Group("gloo")
    ids = rdist.stream_ids(g.rank, 2)
    flagged = n = 0
    digest = []
    for sid in ids:
        f, k, d = _excise(sid)
        flagged += f
        n += k
        digest.append(d)
    out = dict(rank=g.rank, ids=ids, flagged=g.sum(flagged), samples=g.sum(n), tmax=g.max(1.0 + g.rank),
               thr=rdist.throughput(n, 1.0 + g.rank, g), digest=digest)
    g.barrier()
    g.close()
    q.put(out)


def test_two_rank_weak_scaling_layout():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=240) for _ in procs], key=lambda d: d["rank"])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ids0, ids1 = res[0]["ids"], res[1]["ids"]
    assert not set(ids0) & set(ids1)
    single = [_excise(sid) for sid in ids0 + ids1]
    assert res[0]["flagged"] == res[1]["flagged"] == sum(f for f, _, _ in single)
    assert res[0]["samples"] == 4 * N
    assert res[0]["tmax"] == res[1]["tmax"] == 2.0
    assert res[0]["thr"] == 4 * N / 2.0
    assert res[0]["digest"] + res[1]["digest"] == [d for _, _, d in single]
