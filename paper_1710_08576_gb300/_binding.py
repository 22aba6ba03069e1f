"""ctypes binding of librfi (include/rfi.h): argument marshalling only.

Every function named ``rfi_*`` here calls the C entry point of the same name. Buffers may be
given as integers (raw pointers), torch tensors (``data_ptr()``) or numpy arrays (host buffers
for ``rfi_excise_host``). All computation happens in the CUDA kernels of librfi.so; there is no
fallback: if the library cannot be loaded, importing this module fails.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

RFI_OK = 0
RFI_ERR_INVALID_ARG = 1
RFI_ERR_UNSUPPORTED = 2
RFI_ERR_ALIGNMENT = 3
RFI_ERR_OOM = 4
RFI_ERR_CUDA = 5
RFI_ERR_SAMPLE_RANGE = 6
RFI_ERR_TIMEOUT = 7
RFI_ERR_BUSY = 8

RFI_REPLACE_ZERO, RFI_REPLACE_CONST, RFI_REPLACE_CLIP, RFI_REPLACE_NOISE = 0, 1, 2, 3

RFI_PLAN_PER_STREAM = 0x1
RFI_PLAN_BATCHED = 0x2
RFI_PLAN_GRAPH = 0x4
RFI_PLAN_AUTOTUNE = 0x8
RFI_PLAN_POWER = 0x10
RFI_PLAN_NO_SPLIT = 0x20
RFI_PLAN_NOISE_PASS = 0x40
RFI_PLAN_WRITE_FLAGGED = 0x80
RFI_OUT_SAME, RFI_OUT_F16, RFI_OUT_BF16 = 0, 1, 2
RFI_MAX_COPIES = 8
RFI_PLAN_INJECT_TIMEOUT = 0x100
RFI_NOALLOC_MAX_STREAMS = 64
RFI_NOALLOC_MAX_TILES = 65536
RFI_NOALLOC_SCRATCH_BYTES = 256 + 96 * RFI_NOALLOC_MAX_STREAMS + 16 * RFI_NOALLOC_MAX_TILES


class RfiLaunchShape(ctypes.Structure):
    _fields_ = [("consumer_warps", ctypes.c_int32), ("stages", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("stage_bytes", ctypes.c_int32),
                ("dynamic_tiles", ctypes.c_int32), ("hist_copies", ctypes.c_int32),
                ("groups", ctypes.c_int32), ("warp_split", ctypes.c_int32)]


class RfiPlanDesc(ctypes.Structure):
    _fields_ = [("sample_bits", ctypes.c_int32), ("num_streams", ctypes.c_int32),
                ("stream_len", ctypes.POINTER(ctypes.c_int64)),
                ("window_len", ctypes.POINTER(ctypes.c_int32)),
                ("stream_id", ctypes.POINTER(ctypes.c_uint32)), ("k", ctypes.c_double),
                ("mode", ctypes.c_int32), ("const_value", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("flags", ctypes.c_uint32), ("shape", ctypes.POINTER(RfiLaunchShape)),
                ("mom_windows", ctypes.c_int32), ("out_format", ctypes.c_int32)]


class RfiVariant(ctypes.Structure):
    _fields_ = [("k", ctypes.c_double), ("mode", ctypes.c_int32), ("const_value", ctypes.c_int32),
                ("seed", ctypes.c_uint64)]


class RfiTotals(ctypes.Structure):
    _fields_ = [("windows", ctypes.c_uint64), ("flagged", ctypes.c_uint64),
                ("device_status", ctypes.c_int32)]


class RfiPlanInfo(ctypes.Structure):
    _fields_ = [("k_q16", ctypes.c_int64), ("total_windows", ctypes.c_uint64),
                ("total_samples", ctypes.c_uint64), ("workspace_bytes", ctypes.c_uint64),
                ("tiles", ctypes.c_int32), ("grid", ctypes.c_int32), ("shape", RfiLaunchShape),
                ("sm_count", ctypes.c_int32), ("kernels_per_call", ctypes.c_int32)]


class RfiServerDesc(ctypes.Structure):
    _fields_ = [("sample_bits", ctypes.c_int32), ("num_streams", ctypes.c_int32),
                ("window_len", ctypes.POINTER(ctypes.c_int32)),
                ("stream_id", ctypes.POINTER(ctypes.c_uint32)),
                ("stream_start", ctypes.POINTER(ctypes.c_int64)), ("ring_samples", ctypes.c_int64),
                ("k", ctypes.c_double), ("mode", ctypes.c_int32), ("const_value", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("memory_budget", ctypes.c_uint64),
                ("max_requests", ctypes.c_int32), ("request_windows_per_step", ctypes.c_int32)]


class RfiRequestDesc(ctypes.Structure):
    _fields_ = [("in_", ctypes.c_void_p), ("out", ctypes.c_void_p), ("mask", ctypes.c_void_p),
                ("counts", ctypes.c_void_p), ("len", ctypes.c_int64), ("window_len", ctypes.c_int32),
                ("stream_id", ctypes.c_uint32), ("abs0", ctypes.c_int64), ("on_device", ctypes.c_int32)]


class RfiServerStats(ctypes.Structure):
    _fields_ = [("passes", ctypes.c_uint64), ("chunks_done", ctypes.c_uint64),
                ("requests_done", ctypes.c_uint64), ("samples_done", ctypes.c_uint64),
                ("request_samples_done", ctypes.c_uint64), ("flagged", ctypes.c_uint64),
                ("chunk_latency_p50_us", ctypes.c_double), ("chunk_latency_p99_us", ctypes.c_double),
                ("chunk_latency_max_us", ctypes.c_double), ("request_latency_p50_us", ctypes.c_double),
                ("request_latency_p99_us", ctypes.c_double), ("wall_seconds", ctypes.c_double),
                ("arena_bytes", ctypes.c_uint64), ("arena_peak_bytes", ctypes.c_uint64),
                ("device_status", ctypes.c_int32), ("gpu_busy_seconds", ctypes.c_double)]


_P = ctypes.c_void_p
_PP = ctypes.POINTER(ctypes.c_void_p)
_I64P = ctypes.POINTER(ctypes.c_int64)


def _load():
    path = _build.LIB
    if _build.stale():
        try:
            path = _build.build()
        except Exception as e:  # no toolkit and no library: fail loudly
            if not os.path.exists(_build.LIB):
                raise ImportError("librfi.so is missing and could not be built: %s" % e) from e
    lib = ctypes.CDLL(path)
    sig = {
        "rfi_plan_create": (ctypes.c_int, [ctypes.POINTER(RfiPlanDesc), ctypes.POINTER(_P)]),
        "rfi_excise": (ctypes.c_int, [_P, _PP, _PP, _PP, _PP, _P]),
        "rfi_excise_host": (ctypes.c_int, [_P, _PP, _PP, _PP, _PP, _P]),
        "rfi_stats": (ctypes.c_int, [_P, _PP, _PP, ctypes.POINTER(RfiTotals), _P]),
        "rfi_stats_mom": (ctypes.c_int, [_P, _PP, _P]),
        "rfi_plan_create_copies": (ctypes.c_int, [ctypes.POINTER(RfiPlanDesc), ctypes.c_int32,
                                                  ctypes.POINTER(RfiVariant), ctypes.POINTER(_P)]),
        "rfi_excise_copies": (ctypes.c_int, [_P, _PP, _PP, _PP, _PP, _P]),
        "rfi_stats_power": (ctypes.c_int, [_P, _PP, _P]),
        "rfi_improvement_db": (ctypes.c_int, [ctypes.POINTER(ctypes.c_uint64), ctypes.c_int64, ctypes.c_int32,
                                              ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                              ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
        "rfi_plan_get_info": (ctypes.c_int, [_P, ctypes.POINTER(RfiPlanInfo)]),
        "rfi_excise_noalloc": (ctypes.c_int, [ctypes.POINTER(RfiPlanDesc), _PP, _PP, _PP, _PP, _PP, _PP,
                                              ctypes.POINTER(RfiTotals), _P]),
        "rfi_plan_destroy": (ctypes.c_int, [_P]),
        "rfi_server_create": (ctypes.c_int, [ctypes.POINTER(RfiServerDesc), ctypes.POINTER(_P)]),
        "rfi_server_push": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_int64, ctypes.c_int32,
                                           ctypes.POINTER(ctypes.c_uint64)]),
        "rfi_server_submit": (ctypes.c_int, [_P, ctypes.POINTER(RfiRequestDesc), ctypes.POINTER(ctypes.c_uint64)]),
        "rfi_server_step": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32)]),
        "rfi_server_poll": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int32),
                                           ctypes.POINTER(ctypes.c_double)]),
        "rfi_server_read": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, _P, _P,
                                           ctypes.c_int32, ctypes.c_int32]),
        "rfi_server_view": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int64, _PP,
                                           ctypes.POINTER(ctypes.POINTER(ctypes.c_uint32)), _I64P]),
        "rfi_server_release": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int64]),
        "rfi_server_take_latencies": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_uint64),
                                                     ctypes.POINTER(ctypes.c_double), ctypes.c_int64, _I64P]),
        "rfi_server_flush": (ctypes.c_int, [_P, ctypes.c_int32]),
        "rfi_server_position": (ctypes.c_int, [_P, ctypes.c_int32, _I64P, _I64P, _I64P]),
        "rfi_server_drain": (ctypes.c_int, [_P, ctypes.c_double]),
        "rfi_server_get_stats": (ctypes.c_int, [_P, ctypes.POINTER(RfiServerStats)]),
        "rfi_server_destroy": (ctypes.c_int, [_P]),
        "rfi_status_string": (ctypes.c_char_p, [ctypes.c_int]),
        "rfi_version": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


LIB = _load()
LIB_PATH = _build.LIB


def _ptr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return int(x.data_ptr())
    if hasattr(x, "ctypes"):
        return int(x.ctypes.data)
    raise TypeError("cannot take a pointer of %r" % type(x))


def _ptr_array(seq):
    if seq is None:
        return None
    arr = (ctypes.c_void_p * len(seq))(*[_ptr(x) or None for x in seq])
    return ctypes.cast(arr, _PP), arr


def _stream(stream) -> int:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return int(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return 0
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def make_desc(bits, stream_len, window_len, k, mode, const_value=0, seed=0, flags=0, stream_id=None,
              shape=None, mom_windows=0, out_format=0):
    n = len(stream_len)
    keep = []
    lens = (ctypes.c_int64 * n)(*[int(v) for v in stream_len])
    wins = (ctypes.c_int32 * n)(*[int(v) for v in window_len])
    keep += [lens, wins]
    sid = None
    if stream_id is not None:
        sid = (ctypes.c_uint32 * n)(*[int(v) for v in stream_id])
        keep.append(sid)
    shp = None
    if shape is not None:
        if not isinstance(shape, RfiLaunchShape):
            shape = RfiLaunchShape(**shape)
        shp = ctypes.pointer(shape)
        keep.append(shape)
    d = RfiPlanDesc(int(bits), n, lens, wins, sid, float(k), int(mode), int(const_value), int(seed),
                    int(flags), shp, int(mom_windows), int(out_format))
    d._keep = keep
    return d


# ---------------------------------------------------------------- C entry points
def rfi_plan_create(desc: RfiPlanDesc):
    h = ctypes.c_void_p()
    st = LIB.rfi_plan_create(ctypes.byref(desc), ctypes.byref(h))
    return st, h.value


def rfi_excise(plan, ins, outs, masks=None, counts=None, stream=None) -> int:
    a, b, c, d = _ptr_array(ins), _ptr_array(outs), _ptr_array(masks), _ptr_array(counts)
    return LIB.rfi_excise(plan, a[0] if a else None, b[0] if b else None, c[0] if c else None,
                          d[0] if d else None, _stream(stream))


def rfi_excise_host(plan, ins, outs, masks=None, counts=None, stream=None) -> int:
    a, b, c, d = _ptr_array(ins), _ptr_array(outs), _ptr_array(masks), _ptr_array(counts)
    return LIB.rfi_excise_host(plan, a[0] if a else None, b[0] if b else None, c[0] if c else None,
                               d[0] if d else None, _stream(stream))


def rfi_stats(plan, medians=None, mads=None, stream=None):
    t = RfiTotals()
    a, b = _ptr_array(medians), _ptr_array(mads)
    st = LIB.rfi_stats(plan, a[0] if a else None, b[0] if b else None, ctypes.byref(t), _stream(stream))
    return st, t


def rfi_excise_noalloc(desc, ins, outs, masks=None, counts=None, medians=None, mads=None, totals=True,
                       stream=None):
    """Allocation-free excision (see include/rfi.h). Returns (status, totals or None)."""
    arrs = [_ptr_array(x) for x in (ins, outs, masks, counts, medians, mads)]
    t = RfiTotals() if totals else None
    st = LIB.rfi_excise_noalloc(ctypes.byref(desc), *[a[0] if a else None for a in arrs],
                                ctypes.byref(t) if t is not None else None, _stream(stream))
    return st, t


def rfi_plan_get_info(plan):
    info = RfiPlanInfo()
    st = LIB.rfi_plan_get_info(plan, ctypes.byref(info))
    return st, info


def rfi_plan_destroy(plan) -> int:
    return LIB.rfi_plan_destroy(plan)


def rfi_status_string(status: int) -> str:
    return LIB.rfi_status_string(int(status)).decode()


def rfi_version() -> str:
    return LIB.rfi_version().decode()


def rfi_server_create(desc: RfiServerDesc):
    h = ctypes.c_void_p()
    st = LIB.rfi_server_create(ctypes.byref(desc), ctypes.byref(h))
    return st, h.value


def rfi_server_push(server, stream, samples, n, on_device=True):
    t = ctypes.c_uint64()
    st = LIB.rfi_server_push(server, int(stream), _ptr(samples), int(n), int(bool(on_device)), ctypes.byref(t))
    return st, t.value


def rfi_server_submit(server, req: RfiRequestDesc):
    t = ctypes.c_uint64()
    st = LIB.rfi_server_submit(server, ctypes.byref(req), ctypes.byref(t))
    return st, t.value


def rfi_server_step(server):
    launched = ctypes.c_int32()
    st = LIB.rfi_server_step(server, ctypes.byref(launched))
    return st, launched.value


def rfi_server_poll(server, ticket):
    done, lat = ctypes.c_int32(), ctypes.c_double()
    st = LIB.rfi_server_poll(server, int(ticket), ctypes.byref(done), ctypes.byref(lat))
    return st, bool(done.value), lat.value


def rfi_server_read(server, stream, start, n, dst, mask_dst=None, on_device=True, release=True):
    return LIB.rfi_server_read(server, int(stream), int(start), int(n), _ptr(dst), _ptr(mask_dst) or None,
                               int(bool(on_device)), int(bool(release)))


def rfi_server_view(server, stream, start):
    out, mask, n = ctypes.c_void_p(), ctypes.POINTER(ctypes.c_uint32)(), ctypes.c_int64()
    st = LIB.rfi_server_view(server, int(stream), int(start), ctypes.byref(out), ctypes.byref(mask),
                             ctypes.byref(n))
    mptr = ctypes.cast(mask, ctypes.c_void_p).value if mask else 0
    return st, out.value or 0, mptr or 0, n.value


def rfi_server_release(server, stream, upto):
    return LIB.rfi_server_release(server, int(stream), int(upto))


def rfi_server_take_latencies(server, cap=65536):
    t = (ctypes.c_uint64 * cap)()
    lat = (ctypes.c_double * cap)()
    n = ctypes.c_int64()
    st = LIB.rfi_server_take_latencies(server, t, lat, int(cap), ctypes.byref(n))
    return st, list(t[:n.value]), list(lat[:n.value])


def rfi_server_flush(server, stream):
    return LIB.rfi_server_flush(server, int(stream))


def rfi_server_position(server, stream):
    a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    st = LIB.rfi_server_position(server, int(stream), ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
    return st, a.value, b.value, c.value


def rfi_server_drain(server, timeout_seconds=60.0):
    return LIB.rfi_server_drain(server, float(timeout_seconds))


def rfi_server_get_stats(server):
    s = RfiServerStats()
    st = LIB.rfi_server_get_stats(server, ctypes.byref(s))
    return st, s


def rfi_server_destroy(server):
    return LIB.rfi_server_destroy(server)


def rfi_improvement_db(power, windows_per_point=1, points_per_block=64):
    """The improvement metric (Section III-A) of one stream's interleaved per-window power
    (a host numpy array of 2 * nwin uint64/int64). Returns (status, dB, S_U, S_F)."""
    import numpy as np
    p = np.ascontiguousarray(power).view(np.uint64)
    db, su, sf = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    st = LIB.rfi_improvement_db(p.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), p.size // 2,
                                int(windows_per_point), int(points_per_block), ctypes.byref(db),
                                ctypes.byref(su), ctypes.byref(sf))
    return st, db.value, su.value, sf.value


# ---------------------------------------------------------------- convenience wrapper
class RfiError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__("%s: %s (%d)" % (what, rfi_status_string(status), status))
        self.status = status


def check(status: int, what: str):
    if status != RFI_OK:
        raise RfiError(status, what)


class Plan:
    """Owns one rfi_plan_t. Buffers are torch tensors (or raw device pointers)."""

    def __init__(self, bits, stream_len, window_len, k, mode, const_value=0, seed=0, flags=0,
                 stream_id=None, shape=None, mom_windows=0, out_format=0):
        self.desc = make_desc(bits, stream_len, window_len, k, mode, const_value, seed, flags,
                              stream_id, shape, mom_windows, out_format)
        st, h = rfi_plan_create(self.desc)
        check(st, "rfi_plan_create")
        self.handle = h
        self.bits = bits
        self.stream_len = [int(v) for v in stream_len]
        self.window_len = [int(v) for v in window_len]

    @property
    def num_windows(self):
        return [-(-n // w) for n, w in zip(self.stream_len, self.window_len)]

    def mask_words(self, s):
        return self.num_windows[s] * ((self.window_len[s] + 31) // 32)

    def excise(self, ins, outs, masks=None, counts=None, stream=None):
        check(rfi_excise(self.handle, ins, outs, masks, counts, stream), "rfi_excise")

    def excise_host(self, ins, outs, masks=None, counts=None, stream=None):
        check(rfi_excise_host(self.handle, ins, outs, masks, counts, stream), "rfi_excise_host")

    def stats(self, medians=None, mads=None, stream=None):
        st, t = rfi_stats(self.handle, medians, mads, stream)
        return st, t

    def stats_power(self, powers, stream=None):
        """RFI_PLAN_POWER plans: copy {sum x^2, sum z^2} per window into the device arrays `powers`
        (2 * nwin uint64, or int64 tensors of that size)."""
        pa = _ptr_array(powers)
        check(LIB.rfi_stats_power(self.handle, pa[0], _stream(stream)), "rfi_stats_power")

    def stats_mom(self, moms, stream=None):
        """Median-of-MAD plans: copy each window's MoM (Eq. 3) into the device arrays `moms`."""
        pa = _ptr_array(moms)
        check(LIB.rfi_stats_mom(self.handle, pa[0], _stream(stream)), "rfi_stats_mom")

    def info(self) -> RfiPlanInfo:
        st, i = rfi_plan_get_info(self.handle)
        check(st, "rfi_plan_get_info")
        return i

    def close(self):
        if self.handle:
            rfi_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Server:
    """Owns one rfi_server_t (real-time rings + backfill requests, continuous batching)."""

    def __init__(self, bits, window_len, ring_samples, k, mode, const_value=0, seed=0,
                 memory_budget=1 << 30, max_requests=4, request_windows_per_step=0,
                 stream_id=None, stream_start=None):
        n = len(window_len)
        self._keep = [(ctypes.c_int32 * n)(*[int(v) for v in window_len])]
        sid = start = None
        if stream_id is not None:
            sid = (ctypes.c_uint32 * n)(*[int(v) for v in stream_id])
            self._keep.append(sid)
        if stream_start is not None:
            start = (ctypes.c_int64 * n)(*[int(v) for v in stream_start])
            self._keep.append(start)
        self.desc = RfiServerDesc(int(bits), n, self._keep[0], sid, start, int(ring_samples), float(k),
                                  int(mode), int(const_value), int(seed), int(memory_budget),
                                  int(max_requests), int(request_windows_per_step))
        st, h = rfi_server_create(self.desc)
        check(st, "rfi_server_create")
        self.handle = h
        self.bits = bits

    def push(self, stream, samples, n=None, on_device=True):
        n = samples.numel() if n is None else n
        return rfi_server_push(self.handle, stream, samples, n, on_device)

    def submit(self, inp, out, window_len, stream_id=0, abs0=0, mask=None, counts=None, on_device=True, n=None):
        if n is None:
            n = inp.numel() if hasattr(inp, "numel") else inp.size
        req = RfiRequestDesc(_ptr(inp), _ptr(out), _ptr(mask) or None, _ptr(counts) or None, int(n),
                             int(window_len), int(stream_id), int(abs0), int(bool(on_device)))
        return rfi_server_submit(self.handle, req)

    def step(self):
        st, launched = rfi_server_step(self.handle)
        check(st, "rfi_server_step")
        return launched

    def poll(self, ticket):
        st, done, lat = rfi_server_poll(self.handle, ticket)
        check(st, "rfi_server_poll")
        return done, lat

    def read(self, stream, start, n, dst, mask_dst=None, on_device=True, release=True):
        return rfi_server_read(self.handle, stream, start, n, dst, mask_dst, on_device, release)

    def flush(self, stream):
        check(rfi_server_flush(self.handle, stream), "rfi_server_flush")

    def view(self, stream, start):
        """(status, output device pointer, mask device pointer, samples readable there)."""
        return rfi_server_view(self.handle, stream, start)

    def release(self, stream, upto):
        return rfi_server_release(self.handle, stream, upto)

    def take_latencies(self, cap=65536):
        """All finished (ticket, latency us) records not yet taken, oldest first."""
        tickets, lats = [], []
        while True:
            st, t, l = rfi_server_take_latencies(self.handle, cap)
            check(st, "rfi_server_take_latencies")
            tickets += t
            lats += l
            if len(t) < cap:
                return tickets, lats

    def position(self, stream):
        st, p, c, r = rfi_server_position(self.handle, stream)
        check(st, "rfi_server_position")
        return p, c, r

    def drain(self, timeout_seconds=120.0):
        check(rfi_server_drain(self.handle, timeout_seconds), "rfi_server_drain")

    def stats(self):
        st, s = rfi_server_get_stats(self.handle)
        check(st, "rfi_server_get_stats")
        return s

    def close(self):
        if self.handle:
            rfi_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class CopiesPlan(Plan):
    """A digital-copy plan (rfi_plan_create_copies): one pass, several (k, mode, const, seed)
    variants; outputs are given per variant (lists of per-stream buffers)."""

    def __init__(self, bits, stream_len, window_len, variants, flags=0, stream_id=None, shape=None):
        self.desc = make_desc(bits, stream_len, window_len, 3.0, 0, 0, 0, flags, stream_id, shape)
        n = len(variants)
        self._vars = (RfiVariant * n)(*[RfiVariant(float(v[0]), int(v[1]), int(v[2]), int(v[3])) for v in variants])
        h = ctypes.c_void_p()
        check(LIB.rfi_plan_create_copies(ctypes.byref(self.desc), n, self._vars, ctypes.byref(h)),
              "rfi_plan_create_copies")
        self.handle = h.value
        self.bits = bits
        self.stream_len = [int(v) for v in stream_len]
        self.window_len = [int(v) for v in window_len]
        self.nvariants = n

    def excise(self, ins, outs, masks=None, counts=None, stream=None):
        """outs / masks / counts: one list of per-stream buffers per variant (None entries allowed)."""
        flat = lambda per_var: None if per_var is None else [b for lst in per_var for b in lst]  # noqa: E731
        a, b, c, d = _ptr_array(ins), _ptr_array(flat(outs)), _ptr_array(flat(masks)), _ptr_array(flat(counts))
        check(LIB.rfi_excise_copies(self.handle, a[0], b[0], c[0] if c else None, d[0] if d else None,
                                    _stream(stream)), "rfi_excise_copies")
