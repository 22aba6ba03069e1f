"""Serving loop (rfi_server_*) against the oracle: chunked real-time streams and backfill
requests, continuously batched into persistent-kernel passes.

Every output is checked bit for bit against the oracle run offline on the whole stream (or the
whole request), so the tests pin that chunking, ring wrap-around, batching with other streams
and requests, and checkpoint/resume change nothing in what Section II-D computes: windows stay
aligned to absolute sample 0 and the digital noise stays keyed by (stream id, absolute index).
"""
import time

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

K = 3.0
SEED = 0x5EED
CONST = -3


def _params(bits, seed):
    if bits == 8:
        return synth.params(seed=seed, sigma=16.0, burst_rate=5e-3, burst_len_max=64, bits=8)
    return synth.params(seed=seed, sigma=120.0, burst_rate=5e-3, burst_len_max=256, bits=12,
                        amp=(4.0, 30.0), drift_amp=50.0)


def _oracle(x, W, mode, sid, bits, abs0=0):
    r = oracle.excise(x, W, K, mode, const=CONST, seed=SEED, stream_id=sid, abs0=abs0, bits=bits,
                      threads=8, want=("z", "mask", "counts"))
    assert r["status"] == 0
    return r


def _server(rfi, bits, windows, ring, mode, sids=None, starts=None, budget=256 << 20, max_requests=4,
            req_windows=0):
    return rfi.Server(bits, windows, ring, K, mode, CONST, SEED, budget, max_requests, req_windows,
                      stream_id=sids, stream_start=starts)


class Feed:
    """Pushes one stream in ragged chunks and reads its output back as it completes."""

    def __init__(self, srv, idx, x, W, start, rng, max_chunk):
        import torch
        self.srv, self.idx, self.W, self.start = srv, idx, W, start
        self.esz = x.itemsize
        self.dx = torch.from_numpy(x.view(np.uint8).copy()).cuda()
        self.n = x.size
        self.mw = (W + 31) // 32
        nwin = -(-self.n // W)
        self.out = torch.full((self.n * self.esz,), 0x5A, dtype=torch.uint8, device="cuda")
        self.mask = torch.full((nwin * self.mw,), -1, dtype=torch.int32, device="cuda")
        self.pushed = 0
        self.read = 0
        self.rng = rng
        self.max_chunk = max_chunk
        self.tickets = []
        self.flushed = False

    def push(self):
        from paper_1710_08576_gb300 import RFI_OK, RFI_ERR_BUSY
        if self.pushed >= self.n:
            if not self.flushed:
                self.srv.flush(self.idx)
                self.flushed = True
            return False
        m = int(min(self.n - self.pushed, self.rng.integers(1, self.max_chunk + 1)))
        ptr = self.dx.data_ptr() + self.pushed * self.esz
        st, t = self.srv.push(self.idx, ptr, m, on_device=True)
        if st == RFI_ERR_BUSY:
            return False
        assert st == RFI_OK, st
        self.tickets.append(t)
        self.pushed += m
        return True

    def drain_output(self, peek_first=False):
        from paper_1710_08576_gb300 import RFI_OK
        p, c, r = self.srv.position(self.idx)
        assert r == self.start + self.read
        n = c - r
        if n <= 0:
            return
        dst = self.out.data_ptr() + self.read * self.esz
        mdst = self.mask.data_ptr() + (self.read // self.W) * self.mw * 4
        if peek_first:
            assert self.srv.read(self.idx, r, n, dst, mdst, on_device=True, release=False) == RFI_OK
            assert self.srv.position(self.idx)[2] == r
        assert self.srv.read(self.idx, r, n, dst, mdst, on_device=True, release=True) == RFI_OK
        self.read += n

    def done(self):
        return self.flushed and self.read == self.n

    def result(self, bits):
        z = self.out.cpu().numpy().view(np.int8 if bits == 8 else np.int16)
        return z, self.mask.cpu().numpy().view(np.uint32)


def _run_feeds(srv, feeds, max_iters=200000):
    import torch
    torch.cuda.synchronize()  # device inputs are complete before the server's streams read them
    it = 0
    while not all(f.done() for f in feeds):
        it += 1
        assert it < max_iters, "serving loop made no progress"
        progressed = False
        for f in feeds:
            progressed |= f.push()
        srv.step()
        for i, f in enumerate(feeds):
            f.drain_output(peek_first=(i == 0 and it % 7 == 0))
        if not progressed:
            time.sleep(2e-4)


WIN8 = [1024, 4096, 2000]      # 2000 B windows are not 16-byte multiples: the per-window path
WIN12 = [1024, 2048, 1001]


@pytest.mark.parametrize("bits,mode", [(8, 0), (8, 1), (8, 2), (8, 3), (12, 2), (12, 3)])
def test_chunked_streams_match_offline(cuda, rfi, bits, mode):
    windows = WIN8 if bits == 8 else WIN12
    sids = [7, 1001, 42]
    lens = [37 * windows[0] + 517, 23 * windows[1], 41 * windows[2] + 1]
    p = _params(bits, 100 + mode)
    xs = [synth.fill(p, s, n) for s, n in enumerate(lens)]
    ring = 5 * max(windows)
    srv = _server(rfi, bits, windows, ring, mode, sids=sids)
    try:
        rng = np.random.default_rng(mode * 10 + bits)
        feeds = [Feed(srv, i, xs[i], windows[i], 0, rng, 2 * windows[i]) for i in range(3)]
        _run_feeds(srv, feeds)
        st = srv.stats()
        assert st.device_status == rfi.RFI_OK
        assert st.samples_done == sum(lens)
        assert st.chunks_done == sum(len(f.tickets) for f in feeds)
        assert st.passes >= 1 and st.chunk_latency_p50_us > 0
        assert st.chunk_latency_p99_us >= st.chunk_latency_p50_us
        total_flagged = 0
        for i, f in enumerate(feeds):
            z, m = f.result(bits)
            ref = _oracle(xs[i], windows[i], mode, sids[i], bits)
            assert np.array_equal(z, ref["z"]), "stream %d output" % i
            assert np.array_equal(m, ref["mask"]), "stream %d mask" % i
            total_flagged += int(ref["counts"].sum())
            for t in f.tickets:
                done, lat = srv.poll(t)
                assert done and lat >= 0
        assert st.flagged == total_flagged
    finally:
        srv.close()


def _request_bufs(x, W, on_device):
    import torch
    nwin = -(-x.size // W)
    mw = (W + 31) // 32
    if on_device:
        inp = torch.from_numpy(x.copy()).cuda()
        out = torch.full_like(inp, 9)
        mask = torch.full((nwin * mw,), -1, dtype=torch.int32, device="cuda")
        counts = torch.full((nwin,), -1, dtype=torch.int32, device="cuda")
    else:
        inp = x.copy()
        out = np.full_like(x, 9)
        mask = np.full(nwin * mw, 0xFFFFFFFF, np.uint32)
        counts = np.full(nwin, 0xFFFFFFFF, np.uint32)
    return inp, out, mask, counts


def _host(a):
    if hasattr(a, "cpu"):
        return a.cpu().numpy()
    return a


def _wait(srv, ticket, timeout=60.0):
    t0 = time.time()
    while True:
        srv.step()
        done, lat = srv.poll(ticket)
        if done:
            return lat
        assert time.time() - t0 < timeout, "request did not finish"
        time.sleep(2e-4)


@pytest.mark.parametrize("bits,mode", [(8, 3), (8, 2), (12, 3)])
def test_requests_alone_and_in_the_mix(cuda, rfi, bits, mode):
    """A backfill request gives the oracle's result whether it runs alone or batched with live
    streams and other requests, from device or from host memory."""
    import torch
    windows = WIN8 if bits == 8 else WIN12
    p = _params(bits, 7)
    xs = [synth.fill(p, s, 29 * windows[s] + 3) for s in range(3)]
    # requests: (window, length, stream id, abs0, on_device)
    W_req = 16384 if bits == 8 else 4096
    specs = [(W_req, 2500 * W_req + 77, 900, 64 * W_req, True),   # spans several passes
             (W_req, 3 * W_req, 901, 0, False),
             (512, 100 * 512 + 5, 902, 512 * 1000, True)]
    rx = [synth.fill(p, 50 + j, n, i0=a0) for j, (W, n, sid, a0, dev) in enumerate(specs)]
    refs = [_oracle(rx[j], W, mode, sid, bits, abs0=a0) for j, (W, n, sid, a0, dev) in enumerate(specs)]

    def submit_all(srv):
        bufs, tickets = [], []
        for j, (W, n, sid, a0, dev) in enumerate(specs):
            b = _request_bufs(rx[j], W, dev)
            torch.cuda.synchronize()
            st, t = srv.submit(b[0], b[1], W, sid, a0, mask=b[2], counts=b[3], on_device=dev)
            assert st == rfi.RFI_OK, st
            bufs.append(b)
            tickets.append(t)
        return bufs, tickets

    def check(bufs):
        for j, b in enumerate(bufs):
            assert np.array_equal(_host(b[1]), refs[j]["z"]), "request %d output" % j
            assert np.array_equal(_host(b[2]).view(np.uint32), refs[j]["mask"]), "request %d mask" % j
            assert np.array_equal(_host(b[3]).view(np.uint32), refs[j]["counts"]), "request %d counts" % j

    # alone (one at a time, no streams)
    for j in range(len(specs)):
        srv = _server(rfi, bits, [windows[0]], 4 * windows[0], mode, req_windows=700)
        try:
            W, n, sid, a0, dev = specs[j]
            b = _request_bufs(rx[j], W, dev)
            torch.cuda.synchronize()
            st, t = srv.submit(b[0], b[1], W, sid, a0, mask=b[2], counts=b[3], on_device=dev)
            assert st == rfi.RFI_OK
            lat = _wait(srv, t)
            assert lat > 0
            assert np.array_equal(_host(b[1]), refs[j]["z"])
            assert np.array_equal(_host(b[2]).view(np.uint32), refs[j]["mask"])
            assert np.array_equal(_host(b[3]).view(np.uint32), refs[j]["counts"])
        finally:
            srv.close()

    # in the mix: three live streams plus all requests at once
    srv = _server(rfi, bits, windows, 6 * max(windows), mode, sids=[3, 4, 5], req_windows=700)
    try:
        rng = np.random.default_rng(5)
        feeds = [Feed(srv, i, xs[i], windows[i], 0, rng, 3 * windows[i]) for i in range(3)]
        bufs, tickets = submit_all(srv)
        _run_feeds(srv, feeds)
        for t in tickets:
            _wait(srv, t)
        srv.drain()
        check(bufs)
        for i, f in enumerate(feeds):
            z, m = f.result(bits)
            ref = _oracle(xs[i], windows[i], mode, 3 + i, bits)
            assert np.array_equal(z, ref["z"]) and np.array_equal(m, ref["mask"])
        st = srv.stats()
        assert st.requests_done == len(specs)
        assert st.request_samples_done == sum(s[1] for s in specs)
        assert st.request_latency_p99_us >= st.request_latency_p50_us > 0
        assert st.device_status == rfi.RFI_OK
    finally:
        srv.close()


def test_admission_and_back_pressure(cuda, rfi):
    import torch
    W = 1024
    ring = 8 * W
    budget = 64 << 20
    srv = _server(rfi, 8, [W], ring, 0, budget=budget, max_requests=2)
    try:
        x = synth.fill(_params(8, 3), 0, 3 * ring)
        dx = torch.from_numpy(x).cuda()
        torch.cuda.synchronize()
        # ring: exactly full is accepted, one more sample is not
        assert srv.push(0, dx.data_ptr(), ring)[0] == rfi.RFI_OK
        assert srv.push(0, dx.data_ptr() + ring, 1)[0] == rfi.RFI_ERR_BUSY
        srv.drain()
        # processed but not read: still no room
        assert srv.push(0, dx.data_ptr() + ring, 1)[0] == rfi.RFI_ERR_BUSY
        out = torch.empty(ring, dtype=torch.int8, device="cuda")
        assert srv.read(0, 0, ring, out, on_device=True, release=True) == rfi.RFI_OK
        assert srv.push(0, dx.data_ptr() + ring, ring)[0] == rfi.RFI_OK
        ref = _oracle(x[:2 * ring], W, 0, 0, 8)
        assert np.array_equal(out.cpu().numpy(), ref["z"][:ring])
        # reads: outside [released, completed) or off a window boundary are rejected
        srv.drain()
        assert srv.read(0, 0, W, out, on_device=True, release=False) == rfi.RFI_ERR_INVALID_ARG
        assert srv.read(0, ring + 1, W, out, on_device=True, release=False) == rfi.RFI_ERR_INVALID_ARG
        assert srv.read(0, ring, W + 1, out, on_device=True, release=False) == rfi.RFI_ERR_INVALID_ARG
        assert srv.read(0, ring, 2 * ring, out, on_device=True, release=False) == rfi.RFI_ERR_INVALID_ARG
        assert srv.read(0, ring + W, W, out, on_device=True, release=True) == rfi.RFI_ERR_INVALID_ARG
        # requests: slots, then the arena
        big = np.zeros(budget, np.int8)  # its device copies can never fit in the arena
        o_big = np.empty_like(big)
        assert srv.submit(big, o_big, W, on_device=False)[0] == rfi.RFI_ERR_OOM
        half = np.zeros(int(budget * 0.35), np.int8)  # its two copies (in, out) take 70% of the arena
        o1, o2 = np.empty_like(half), np.empty_like(half)
        st1, t1 = srv.submit(half, o1, W, on_device=False)
        assert st1 == rfi.RFI_OK
        st2, _ = srv.submit(half, o2, W, on_device=False)
        assert st2 == rfi.RFI_ERR_BUSY  # fits the budget, but not next to the first one
        d_in = torch.zeros(4 * W, dtype=torch.int8, device="cuda")
        d_out = torch.empty_like(d_in)
        st3, t3 = srv.submit(d_in, d_out, W, on_device=True)
        assert st3 == rfi.RFI_OK
        assert srv.submit(d_in, d_out, W, on_device=True)[0] == rfi.RFI_ERR_BUSY  # both slots taken
        _wait(srv, t1)
        _wait(srv, t3)
        st2, t2 = srv.submit(half, o2, W, on_device=False)
        assert st2 == rfi.RFI_OK
        _wait(srv, t2)
        assert not o2.any() and not o1.any()
        assert srv.stats().arena_peak_bytes <= budget
    finally:
        srv.close()


@pytest.mark.parametrize("bits", [8, 12])
def test_checkpoint_resume_equals_uninterrupted(cuda, rfi, bits):
    """Stop a server at its completed position, start a new one there (stream_start), and the
    joined output equals one uninterrupted run; with digital noise this needs the absolute
    sample index to carry over."""
    windows = [2048, 1024] if bits == 8 else [1024, 1001]
    sids = [11, 12]
    lens = [60 * windows[0] + 100, 90 * windows[1]]
    p = _params(bits, 21)
    xs = [synth.fill(p, s, n) for s, n in enumerate(lens)]
    refs = [_oracle(xs[i], windows[i], 3, sids[i], bits) for i in range(2)]
    cut = [27 * windows[0] + 300, 41 * windows[1] + 5]  # pushed before the checkpoint
    rng = np.random.default_rng(1)
    srv = _server(rfi, bits, windows, 4 * max(windows), 3, sids=sids)
    try:
        feeds = [Feed(srv, i, xs[i][:cut[i]], windows[i], 0, rng, windows[i]) for i in range(2)]
        import torch
        torch.cuda.synchronize()
        while not all(f.pushed == f.n for f in feeds):
            for f in feeds:
                if f.pushed < f.n:
                    f.push()
            srv.step()
            for f in feeds:
                f.drain_output()
        srv.drain()
        for f in feeds:
            f.drain_output()
        pos = [srv.position(i) for i in range(2)]
        first = [f.result(bits) for f in feeds]
    finally:
        srv.close()
    resume = [c for (_, c, _) in pos]
    for i in range(2):
        assert resume[i] % windows[i] == 0 and resume[i] == cut[i] // windows[i] * windows[i]
    srv = _server(rfi, bits, windows, 4 * max(windows), 3, sids=sids, starts=resume)
    try:
        feeds = [Feed(srv, i, xs[i][resume[i]:], windows[i], resume[i], rng, windows[i]) for i in range(2)]
        _run_feeds(srv, feeds)
        for i in range(2):
            z0, m0 = first[i]
            z1, m1 = feeds[i].result(bits)
            mw = (windows[i] + 31) // 32
            nw0 = resume[i] // windows[i]
            z = np.concatenate([z0[:resume[i]], z1])
            m = np.concatenate([m0[:nw0 * mw], m1])
            assert np.array_equal(z, refs[i]["z"]), "stream %d" % i
            assert np.array_equal(m, refs[i]["mask"]), "stream %d mask" % i
    finally:
        srv.close()


def test_twelve_bit_range_error_is_reported(cuda, rfi):
    import torch
    W = 1024
    srv = _server(rfi, 12, [W], 4 * W, 0)
    try:
        x = synth.fill(_params(12, 2), 0, 2 * W)
        x[W + 17] = 3000  # outside the 12-bit range
        dx = torch.from_numpy(x).cuda()
        torch.cuda.synchronize()
        assert srv.push(0, dx, 2 * W)[0] == rfi.RFI_OK
        srv.drain()
        assert srv.stats().device_status == rfi.RFI_ERR_SAMPLE_RANGE
    finally:
        srv.close()


class _DevArray:
    """A raw device pointer seen as a tensor (zero-copy), through __cuda_array_interface__."""

    def __init__(self, ptr, n, typestr):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False),
                                         "version": 2}


def test_zero_copy_view_and_release(cuda, rfi):
    """A consumer reads the output in place through rfi_server_view and frees it with
    rfi_server_release; what it sees is the oracle's output, across the ring's wrap."""
    import torch
    W = 2048
    ring = 5 * W
    x = synth.fill(_params(8, 9), 0, 13 * W + 100)
    ref = _oracle(x, W, 3, 77, 8)
    srv = _server(rfi, 8, [W], ring, 3, sids=[77])
    try:
        dx = torch.from_numpy(x).cuda()
        torch.cuda.synchronize()
        got = np.zeros_like(x)
        got_mask = np.zeros_like(ref["mask"])
        pushed = consumed = 0
        mw = W // 32
        for _ in range(10000):
            if pushed < x.size:
                m = min(x.size - pushed, 3 * W // 2)
                st, _ = srv.push(0, dx.data_ptr() + pushed, m)
                if st == rfi.RFI_OK:
                    pushed += m
                    if pushed == x.size:
                        srv.flush(0)
            srv.step()
            st, optr, mptr, n = srv.view(0, consumed)
            assert st == rfi.RFI_OK
            if n > 0:
                assert (optr - srv.view(0, consumed)[1]) == 0
                got[consumed:consumed + n] = torch.as_tensor(_DevArray(optr, n, "|i1"), device="cuda").cpu().numpy()
                nwm = -(-n // W) * mw
                w0 = consumed // W
                got_mask[w0 * mw:w0 * mw + nwm] = torch.as_tensor(
                    _DevArray(mptr, nwm, "<i4"), device="cuda").cpu().numpy().view(np.uint32)
                assert srv.release(0, consumed + n + 1) == rfi.RFI_ERR_INVALID_ARG
                assert srv.release(0, consumed + n) == rfi.RFI_OK
                consumed += n
            if consumed == x.size:
                break
            time.sleep(1e-4)
        assert consumed == x.size
        assert np.array_equal(got, ref["z"]) and np.array_equal(got_mask, ref["mask"])
        # every chunk's latency record comes out once, then no ticket polls as done
        tickets, lats = srv.take_latencies()
        assert len(tickets) == srv.stats().chunks_done and all(v >= 0 for v in lats)
        assert srv.take_latencies() == ([], [])
        assert not srv.poll(tickets[0])[0]
        assert srv.stats().gpu_busy_seconds > 0
    finally:
        srv.close()
