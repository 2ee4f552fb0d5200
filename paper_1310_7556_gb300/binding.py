"""Thin ctypes binding of the hough C ABI (``include/hough.h``): argument marshalling only.

Every step of the path runs in the CUDA library.  There is no fallback: when the library is
missing, loading it raises.  Device buffers are passed as raw pointers (anything with a
``data_ptr()`` method, e.g. a CUDA torch tensor, or an integer), host buffers as numpy arrays,
and a stream as a ``cudaStream_t`` value (e.g. ``torch.cuda.current_stream().cuda_stream``).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HOST, DEVICE = 0, 1
OK, EINVAL, ENOMEM, ECUDA, ETRUNC, ECAPACITY, EBUSY, ETIMEDOUT, EDEVICE, ENOTREADY = \
    0, -1, -2, -3, -4, -5, -6, -7, -8, -9
MAX_LAYERS = 16

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libhough.so")
_lib = None
_lock = threading.Lock()


class HoughError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"hough error {code}: {msg}")
        self.code = code


class Geometry(ctypes.Structure):
    _fields_ = [("n_layers", ctypes.c_int32), ("reserved", ctypes.c_int32), ("b_tesla", ctypes.c_double)]


class Binning(ctypes.Structure):
    _fields_ = [("n_qpt", ctypes.c_int32), ("n_phi", ctypes.c_int32), ("threshold", ctypes.c_int32),
                ("n_cot", ctypes.c_int32), ("n_z0", ctypes.c_int32), ("accumulator", ctypes.c_int32),
                ("qpt_min", ctypes.c_double), ("qpt_max", ctypes.c_double),
                ("cot_min", ctypes.c_double), ("cot_max", ctypes.c_double),
                ("z0_min_cm", ctypes.c_double), ("z0_max_cm", ctypes.c_double),
                ("n_d0", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("d0_min_cm", ctypes.c_double), ("d0_max_cm", ctypes.c_double)]


class Limits(ctypes.Structure):
    _fields_ = [("max_hits", ctypes.c_int64), ("max_candidates", ctypes.c_int32),
                ("max_members", ctypes.c_int32)]


class BatchLimits(ctypes.Structure):
    _fields_ = [("max_events", ctypes.c_int32), ("max_candidates", ctypes.c_int32), ("max_hits", ctypes.c_int64),
                ("max_members", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("votes", ctypes.c_uint64), ("votes_by_layer", ctypes.c_uint64 * MAX_LAYERS),
                ("general_votes", ctypes.c_uint64), ("refined_votes", ctypes.c_uint64),
                ("stage2_votes", ctypes.c_uint64), ("n_hits", ctypes.c_int64),
                ("n_candidates", ctypes.c_int64), ("n_members", ctypes.c_int64),
                ("device_error", ctypes.c_uint32), ("uniform_layers", ctypes.c_uint32)]


class Timing(ctypes.Structure):
    _fields_ = [(n, ctypes.c_float) for n in ("stage_ms", "vote_ms", "peaks_ms", "stage2_ms", "gather_ms",
                                              "scatter_ms", "band_peaks_ms", "compact_ms", "member_ms", "large_ms",
                                              "clear_ms", "count_ms", "table_ms", "scan_ms", "sort_ms")]


TILING_FIELDS = ("tile_qpt", "tile_phi", "threads", "vote_mode", "band_rows", "gather_rows", "gather_cols",
                 "gather_threads")


class Tiling(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in TILING_FIELDS]


VOTE_GATHER, VOTE_SCATTER, VOTE_FUSED = 0, 1, 2
ACC_LAYERS, ACC_COUNTS = 0, 1   # hough_binning.accumulator: layer masks, saturating vote counts


class ServeConfig(ctypes.Structure):
    _fields_ = [("lanes", ctypes.c_int32), ("max_in_flight", ctypes.c_int32), ("max_batch_events", ctypes.c_int32),
                ("max_candidates", ctypes.c_int32), ("max_batch_hits", ctypes.c_int64),
                ("max_members", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("memory_budget", ctypes.c_int64), ("lane_timeout_us", ctypes.c_int64)]


class ServeResult(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_uint64), ("arrival_ns", ctypes.c_int64), ("submit_ns", ctypes.c_int64),
                ("launch_ns", ctypes.c_int64), ("done_ns", ctypes.c_int64), ("n_candidates", ctypes.c_int64),
                ("votes", ctypes.c_uint64), ("status", ctypes.c_int32), ("batch_events", ctypes.c_int32),
                ("device_error", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class ServeStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in (
        "submitted", "admitted", "rejected_busy", "rejected_invalid", "completed", "failed", "launches",
        "launched_events", "max_in_flight", "timeouts", "alloc_failures", "retired_lanes", "lanes", "in_flight",
        "pending_tickets", "device_bytes")]


class EventView(ctypes.Structure):
    _fields_ = [("r", ctypes.c_void_p), ("phi", ctypes.c_void_p), ("z", ctypes.c_void_p),
                ("layer", ctypes.c_void_p), ("n_hits", ctypes.c_int64)]


SERVE_FAULT_HOLD, SERVE_FAULT_STALL, SERVE_FAULT_ALLOC = 1, 2, 3


class TuneResult(ctypes.Structure):
    _fields_ = [("tiling", Tiling), ("ms", ctypes.c_float), ("default_ms", ctypes.c_float),
                ("tried", ctypes.c_int32), ("from_cache", ctypes.c_int32)]


CANDIDATE_DTYPE = np.dtype([("iq", np.uint32), ("jphi", np.uint32), ("mask", np.uint32),
                            ("n_members", np.uint32), ("icot", np.uint32), ("jz0", np.uint32),
                            ("mask2", np.uint32), ("flags", np.uint32)])
assert CANDIDATE_DTYPE.itemsize == 32

# Every entry point the header declares, with its ctypes signature.
_P = ctypes.c_void_p
_I32, _I64 = ctypes.c_int32, ctypes.c_int64
_SIGNATURES = {
    "hough_last_error": ([], ctypes.c_char_p),
    "hough_version": ([], ctypes.c_char_p),
    "hough_create": ([ctypes.POINTER(Geometry), ctypes.POINTER(Binning), ctypes.POINTER(Limits), ctypes.c_int,
                      ctypes.POINTER(_P)], ctypes.c_int),
    "hough_destroy": ([_P], None),
    "hough_vote": ([_P, _P, _P, _P, _P, _I64, ctypes.c_int, _P], ctypes.c_int),
    "hough_peaks": ([_P, _P], ctypes.c_int),
    "hough_stage2": ([_P, _P], ctypes.c_int),
    "hough_get_candidates": ([_P, _P, _I32, ctypes.POINTER(_I32), ctypes.c_int, _P], ctypes.c_int),
    "hough_get_accumulator": ([_P, _P, ctypes.c_int, _P], ctypes.c_int),
    "hough_get_members": ([_P, _P, _P, _I64, ctypes.c_int, _P], ctypes.c_int),
    "hough_get_stats": ([_P, ctypes.POINTER(Stats), _P], ctypes.c_int),
    "hough_process": ([_P, _P, _P, _P, _P, _I64, _P, _I32, ctypes.POINTER(_I32), ctypes.c_int, _P], ctypes.c_int),
    "hough_set_tiling": ([_P, ctypes.POINTER(Tiling)], ctypes.c_int),
    "hough_get_tiling": ([_P, ctypes.POINTER(Tiling)], ctypes.c_int),
    "hough_enable_timing": ([_P, ctypes.c_int], ctypes.c_int),
    "hough_get_timing": ([_P, ctypes.POINTER(Timing)], ctypes.c_int),
    "hough_kernel_launches": ([], ctypes.c_uint64),
    "hough_microbench_smem_or": ([ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_double)],
                                 ctypes.c_int),
    "hough_vote_static": ([ctypes.POINTER(Geometry), ctypes.POINTER(Binning), _P, _P, _P, _P, _I64, _P, _P, _P],
                          ctypes.c_int),
    "hough_batch_create": ([ctypes.POINTER(Geometry), ctypes.POINTER(Binning), ctypes.POINTER(BatchLimits),
                            ctypes.c_int, ctypes.POINTER(_P)], ctypes.c_int),
    "hough_batch_destroy": ([_P], None),
    "hough_batch_set_tiling": ([_P, ctypes.POINTER(Tiling)], ctypes.c_int),
    "hough_set_copy_wait": ([_P, ctypes.c_int], ctypes.c_int),
    "hough_batch_run": ([_P, _P, _P, _P, _P, _P, _I32, ctypes.c_int, _P], ctypes.c_int),
    "hough_batch_profile": ([_P, _P, _P, _P, _P, _P, _I32, ctypes.c_int, _P, ctypes.POINTER(Timing)], ctypes.c_int),
    "hough_batch_candidates": ([_P, _P, _I64, _P, ctypes.c_int, _P], ctypes.c_int),
    "hough_batch_stats": ([_P, _I32, ctypes.POINTER(Stats), _P], ctypes.c_int),
    "hough_batch_accumulator": ([_P, _I32, _P, ctypes.c_int, _P], ctypes.c_int),
    "hough_batch_autotune": ([_P, ctypes.POINTER(Geometry), ctypes.POINTER(Binning), _P, _P, _P, _P, _P, _I32,
                              ctypes.c_int, _I32, ctypes.c_char_p, ctypes.POINTER(TuneResult)], ctypes.c_int),
    "hough_tune_lookup": ([ctypes.c_char_p, ctypes.POINTER(Geometry), ctypes.POINTER(Binning), ctypes.c_int, _I32,
                           ctypes.POINTER(Tiling)], ctypes.c_int),
    "hough_serve_create": ([ctypes.POINTER(Geometry), ctypes.POINTER(Binning), ctypes.POINTER(ServeConfig),
                            ctypes.c_int, ctypes.POINTER(_P)], ctypes.c_int),
    "hough_serve_destroy": ([_P], None),
    "hough_serve_clock_ns": ([], ctypes.c_int64),
    "hough_serve_submit": ([_P, _P, _P, _P, _P, _I64, _I64, ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
    "hough_serve_poll": ([_P, ctypes.c_uint64, _P, _I64, ctypes.POINTER(ServeResult), _I64], ctypes.c_int),
    "hough_serve_drain": ([_P, _I64], ctypes.c_int),
    "hough_serve_get_stats": ([_P, ctypes.POINTER(ServeStats)], ctypes.c_int),
    "hough_serve_inject": ([_P, ctypes.c_int, ctypes.c_int], ctypes.c_int),
    "hough_serve_replay": ([_P, ctypes.POINTER(EventView), _I32, _P, _I64, _I32, ctypes.POINTER(ServeResult)],
                           ctypes.c_int),
}


def kernel_launches() -> int:
    return int(load().hough_kernel_launches())


def smem_or_throughput(device: int = 0, pattern: int = 0, ms: float = 50.0) -> float:
    """Measured shared-memory atomicOr lane-operations per second on the device."""
    out = ctypes.c_double(0.0)
    _check(load().hough_microbench_smem_or(device, pattern, ms, ctypes.byref(out)))
    return out.value


def vote_static(geometry, binning, r, phi, z, layer, n_hits, accumulator, device_error=None, stream=None):
    """hough_vote_static: the vote of one event into a caller-owned device accumulator, for callers
    that may not allocate device memory while running (device pointers only; see include/hough.h)."""
    g, b = make_geometry(geometry), make_binning(binning)
    _check(load().hough_vote_static(ctypes.byref(g), ctypes.byref(b), _ptr(r), _ptr(phi), _ptr(z), _ptr(layer),
                                    int(n_hits), _ptr(accumulator), _ptr(device_error), _stream(stream)))


def library_path() -> str:
    return _LIB_PATH


def load():
    """Open the CUDA library (raises when it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_LIB_PATH):
                raise RuntimeError(f"hough CUDA library missing at {_LIB_PATH}; build it with "
                                   "python -c 'import __graft_entry__ as g; g.build()'")
            lib = ctypes.CDLL(_LIB_PATH)
            for name, (args, res) in _SIGNATURES.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = res
            _lib = lib
    return _lib


def _check(rc: int, allow=()):
    if rc != OK and rc not in allow:
        raise HoughError(rc, load().hough_last_error().decode())
    return rc


def _ptr(x):
    """Raw address of a buffer: numpy array, object with data_ptr(), integer or None."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return int(x)


def _stream(s):
    if s is None:
        return None
    if hasattr(s, "cuda_stream"):
        return s.cuda_stream
    return int(s)


def make_geometry(geometry) -> Geometry:
    return Geometry(n_layers=geometry.n_layers, reserved=0, b_tesla=geometry.b_tesla)


def make_binning(binning) -> Binning:
    return Binning(n_qpt=binning.n_qpt, n_phi=binning.n_phi, threshold=binning.threshold,
                   n_cot=binning.n_cot, n_z0=binning.n_z0,
                   accumulator=int(getattr(binning, "accumulator", ACC_LAYERS)),
                   qpt_min=binning.qpt_min, qpt_max=binning.qpt_max,
                   cot_min=binning.cot_min, cot_max=binning.cot_max,
                   z0_min_cm=binning.z0_min, z0_max_cm=binning.z0_max,
                   n_d0=int(getattr(binning, "n_d0", 0)), reserved=0,
                   d0_min_cm=float(getattr(binning, "d0_min", -1.0)), d0_max_cm=float(getattr(binning, "d0_max", 1.0)))


def grid_rows(binning) -> int:
    """Rows of the accumulator: n_qpt, times n_d0 with a d0 axis (stacked rows m * n_qpt + i)."""
    return binning.n_qpt * max(int(getattr(binning, "n_d0", 0)), 1)


class HoughContext:
    """One hough_ctx: a GPU, a set of axes and the device buffers sized by the limits."""

    def __init__(self, geometry, binning, max_hits: int, max_candidates: int = 65536,
                 max_members: int = 1 << 22, device: int = 0):
        lib = load()
        self._lib = lib
        self.binning = binning
        self.geometry = geometry
        g, b = make_geometry(geometry), make_binning(binning)
        lim = Limits(max_hits=max_hits, max_candidates=max_candidates, max_members=max_members)
        h = _P()
        _check(lib.hough_create(ctypes.byref(g), ctypes.byref(b), ctypes.byref(lim), device, ctypes.byref(h)))
        self._h = h
        self.max_candidates = max_candidates

    def close(self):
        if getattr(self, "_h", None):
            self._lib.hough_destroy(self._h)
            self._h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- the path -----------------------------------------------------------------------------
    def vote(self, r, phi, z, layer, n_hits=None, where=HOST, stream=None):
        """hough_vote.  Host hits as numpy arrays, or pinned buffers (with data_ptr()) and n_hits."""
        if where == HOST and isinstance(r, np.ndarray):
            r, phi, z = (np.ascontiguousarray(a, dtype=np.float32) for a in (r, phi, z))
            layer = np.ascontiguousarray(layer, dtype=np.uint8)
            n_hits = r.shape[0]
        self._keep = (r, phi, z, layer)
        _check(self._lib.hough_vote(self._h, _ptr(r), _ptr(phi), _ptr(z), _ptr(layer), int(n_hits), where,
                                    _stream(stream)))

    def peaks(self, stream=None):
        _check(self._lib.hough_peaks(self._h, _stream(stream)))

    def stage2(self, stream=None):
        _check(self._lib.hough_stage2(self._h, _stream(stream)))

    def vote_event(self, event, stream=None):
        self.vote(event.r, event.phi, event.z, event.layer, stream=stream)

    # -- results ------------------------------------------------------------------------------
    def candidates(self, cap=None, stream=None) -> np.ndarray:
        cap = self.max_candidates if cap is None else cap
        out = np.zeros(max(cap, 1), dtype=CANDIDATE_DTYPE)
        n = _I32(0)
        _check(self._lib.hough_get_candidates(self._h, _ptr(out), cap, ctypes.byref(n), HOST, _stream(stream)))
        return out[: n.value].copy()

    def accumulator(self, stream=None) -> np.ndarray:
        out = np.zeros((grid_rows(self.binning), self.binning.n_phi), dtype=np.uint16)
        _check(self._lib.hough_get_accumulator(self._h, _ptr(out), HOST, _stream(stream)))
        return out

    def members(self, n_candidates: int, hit_cap: int = 1 << 22, stream=None, allow_truncated: bool = False):
        """(offsets, hit indices) of each candidate's members; with allow_truncated, lists cut by
        max_members or hit_cap (HOUGH_ETRUNC) are returned as they are."""
        offsets = np.zeros(n_candidates + 1, dtype=np.int64)
        hits = np.zeros(max(hit_cap, 1), dtype=np.int32)
        _check(self._lib.hough_get_members(self._h, _ptr(offsets), _ptr(hits), hit_cap, HOST, _stream(stream)),
               allow=(ETRUNC,) if allow_truncated else ())
        return offsets, hits[: offsets[-1]].copy()

    def stats(self, stream=None, allow_device_error=False) -> Stats:
        st = Stats()
        _check(self._lib.hough_get_stats(self._h, ctypes.byref(st), _stream(stream)),
               allow=(EDEVICE,) if allow_device_error else ())
        return st

    def process(self, r, phi, z, layer, n_hits=None, cap=None, out=None, stream=None) -> np.ndarray:
        """Whole path on host-resident hits (numpy arrays, or pinned buffers with data_ptr())."""
        cap = self.max_candidates if cap is None else cap
        if isinstance(r, np.ndarray):
            r, phi, z = (np.ascontiguousarray(a, dtype=np.float32) for a in (r, phi, z))
            layer = np.ascontiguousarray(layer, dtype=np.uint8)
            n_hits = r.shape[0]
        if out is None:
            out = np.zeros(max(cap, 1), dtype=CANDIDATE_DTYPE)
        n = _I32(0)
        _check(self._lib.hough_process(self._h, _ptr(r), _ptr(phi), _ptr(z), _ptr(layer), int(n_hits), _ptr(out),
                                       cap, ctypes.byref(n), HOST, _stream(stream)))
        return out[: n.value]

    # -- timing -------------------------------------------------------------------------------
    def enable_timing(self, on=True):
        _check(self._lib.hough_enable_timing(self._h, 1 if on else 0))

    def set_copy_wait(self, first_bound: int):
        """hough_set_copy_wait: < 0 makes the first bound of the vote's bulk-copy waits expire at once."""
        _check(self._lib.hough_set_copy_wait(self._h, int(first_bound)))

    def timing(self) -> dict:
        t = Timing()
        _check(self._lib.hough_get_timing(self._h, ctypes.byref(t)))
        return {n: getattr(t, n) for n, _ in Timing._fields_}

    # -- tiling -------------------------------------------------------------------------------
    def set_tiling(self, tile_qpt: int = None, tile_phi: int = None, threads: int = None,
                   vote_mode: int = None, band_rows: int = None, gather_rows: int = None,
                   gather_cols: int = None, gather_threads: int = None):
        """Change the kernel configuration; unspecified fields keep their current value."""
        new = self.get_tiling()
        for k, v in dict(tile_qpt=tile_qpt, tile_phi=tile_phi, threads=threads, vote_mode=vote_mode,
                         band_rows=band_rows, gather_rows=gather_rows, gather_cols=gather_cols,
                         gather_threads=gather_threads).items():
            if v is not None:
                new[k] = v
        t = Tiling(**new)
        _check(self._lib.hough_set_tiling(self._h, ctypes.byref(t)))

    def get_tiling(self) -> dict:
        t = Tiling()
        _check(self._lib.hough_get_tiling(self._h, ctypes.byref(t)))
        return {n: getattr(t, n) for n in TILING_FIELDS}


class HoughBatch:
    """One hough_batch: many events through the whole path per call, as a replayed CUDA graph."""

    def __init__(self, geometry, binning, max_events: int, max_hits: int, max_candidates: int = 1 << 17,
                 max_members: int = 1 << 21, device: int = 0):
        lib = load()
        self._lib = lib
        self.binning = binning
        g, b = make_geometry(geometry), make_binning(binning)
        self._geometry, self._binning = g, b
        lim = BatchLimits(max_events=max_events, max_candidates=max_candidates, max_hits=max_hits,
                          max_members=max_members, reserved=0)
        h = _P()
        _check(lib.hough_batch_create(ctypes.byref(g), ctypes.byref(b), ctypes.byref(lim), device, ctypes.byref(h)))
        self._h = h
        self.max_events, self.max_candidates = max_events, max_candidates
        self.n_events = 0

    def close(self):
        if getattr(self, "_h", None):
            self._lib.hough_batch_destroy(self._h)
            self._h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_tiling(self, tile_qpt=32, tile_phi=256, threads=256, vote_mode=VOTE_GATHER, band_rows=1,
                   gather_rows=0, gather_cols=0, gather_threads=0):
        t = Tiling(tile_qpt=tile_qpt, tile_phi=tile_phi, threads=threads, vote_mode=vote_mode, band_rows=band_rows,
                   gather_rows=gather_rows, gather_cols=gather_cols, gather_threads=gather_threads)
        _check(self._lib.hough_batch_set_tiling(self._h, ctypes.byref(t)))

    def run(self, r, phi, z, layer, hit_start, where=HOST, stream=None):
        """hit_start: int64 numpy array of n_events + 1 offsets (host)."""
        hit_start = np.ascontiguousarray(hit_start, dtype=np.int64)
        if where == HOST and isinstance(r, np.ndarray):
            r, phi, z = (np.ascontiguousarray(a, dtype=np.float32) for a in (r, phi, z))
            layer = np.ascontiguousarray(layer, dtype=np.uint8)
        self._keep = (r, phi, z, layer, hit_start)
        n_events = hit_start.shape[0] - 1
        _check(self._lib.hough_batch_run(self._h, _ptr(r), _ptr(phi), _ptr(z), _ptr(layer), _ptr(hit_start),
                                         n_events, where, _stream(stream)))
        self.n_events = n_events

    def profile(self, r, phi, z, layer, hit_start, where=HOST, stream=None) -> dict:
        """hough_batch_profile: the run with every step timed on the stream (synchronises)."""
        hit_start = np.ascontiguousarray(hit_start, dtype=np.int64)
        self._keep = (r, phi, z, layer, hit_start)
        n_events = hit_start.shape[0] - 1
        t = Timing()
        _check(self._lib.hough_batch_profile(self._h, _ptr(r), _ptr(phi), _ptr(z), _ptr(layer), _ptr(hit_start),
                                             n_events, where, _stream(stream), ctypes.byref(t)))
        self.n_events = n_events
        return {n: getattr(t, n) for n, _ in Timing._fields_}

    def run_events(self, events, stream=None):
        """Concatenate Event objects (host) and run them."""
        hs = np.zeros(len(events) + 1, dtype=np.int64)
        hs[1:] = np.cumsum([e.n_hits for e in events])
        cat = lambda name, dt: np.concatenate([getattr(e, name) for e in events]).astype(dt)
        self.run(cat("r", np.float32), cat("phi", np.float32), cat("z", np.float32), cat("layer", np.uint8), hs,
                 stream=stream)

    def autotune(self, r, phi, z, layer, hit_start, where=HOST, reps=3, cache_path=None) -> TuneResult:
        """hough_batch_autotune on these events; applies and returns the fastest configuration."""
        hit_start = np.ascontiguousarray(hit_start, dtype=np.int64)
        if where == HOST and isinstance(r, np.ndarray):
            r, phi, z = (np.ascontiguousarray(a, dtype=np.float32) for a in (r, phi, z))
            layer = np.ascontiguousarray(layer, dtype=np.uint8)
        res = TuneResult()
        path = cache_path.encode() if cache_path else None
        _check(self._lib.hough_batch_autotune(self._h, ctypes.byref(self._geometry), ctypes.byref(self._binning),
                                              _ptr(r), _ptr(phi), _ptr(z), _ptr(layer), _ptr(hit_start),
                                              hit_start.shape[0] - 1, where, reps, path, ctypes.byref(res)))
        self.n_events = 0
        return res

    def candidates(self, cap=None, stream=None):
        """(candidates of all events concatenated, offsets[n_events + 1])."""
        cap = self.max_events * self.max_candidates if cap is None else cap
        out = np.zeros(max(cap, 1), dtype=CANDIDATE_DTYPE)
        offs = np.zeros(self.n_events + 1, dtype=np.int64)
        _check(self._lib.hough_batch_candidates(self._h, _ptr(out), cap, _ptr(offs), HOST, _stream(stream)))
        return out[: offs[-1]].copy(), offs

    def stats(self, event, stream=None, allow_device_error=False) -> Stats:
        st = Stats()
        _check(self._lib.hough_batch_stats(self._h, event, ctypes.byref(st), _stream(stream)),
               allow=(EDEVICE,) if allow_device_error else ())
        return st

    def accumulator(self, event, stream=None) -> np.ndarray:
        out = np.zeros((grid_rows(self.binning), self.binning.n_phi), dtype=np.uint16)
        _check(self._lib.hough_batch_accumulator(self._h, event, _ptr(out), HOST, _stream(stream)))
        return out


def serve_clock_ns() -> int:
    """The server's clock (CLOCK_MONOTONIC nanoseconds, the clock of time.monotonic_ns)."""
    return int(load().hough_serve_clock_ns())


class HoughServer:
    """One hough_server: events submitted one by one, continuously batched onto the GPU by the
    library's dispatcher thread, results polled per ticket."""

    def __init__(self, geometry, binning, max_batch_events: int, max_batch_hits: int, lanes: int = 3,
                 max_in_flight: int = 0, max_candidates: int = 1 << 17, max_members: int = 1 << 21,
                 memory_budget: int = 0, lane_timeout_us: int = 0, device: int = 0):
        lib = load()
        self._lib = lib
        g, b = make_geometry(geometry), make_binning(binning)
        cfg = ServeConfig(lanes=lanes, max_in_flight=max_in_flight, max_batch_events=max_batch_events,
                          max_candidates=max_candidates, max_batch_hits=max_batch_hits, max_members=max_members,
                          reserved=0, memory_budget=memory_budget, lane_timeout_us=lane_timeout_us)
        h = _P()
        _check(lib.hough_serve_create(ctypes.byref(g), ctypes.byref(b), ctypes.byref(cfg), device, ctypes.byref(h)))
        self._h = h
        self.max_candidates = max_candidates

    def close(self):
        if getattr(self, "_h", None):
            self._lib.hough_serve_destroy(self._h)
            self._h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def submit(self, r, phi, z, layer, n_hits=None, arrival_ns: int = 0):
        """Ticket of the admitted event, or None when the server is busy (HOUGH_EBUSY).  Host arrays
        must be float32 / uint8 and contiguous."""
        n = r.shape[0] if n_hits is None else n_hits
        t = ctypes.c_uint64(0)
        rc = _check(self._lib.hough_serve_submit(self._h, _ptr(r), _ptr(phi), _ptr(z), _ptr(layer), int(n),
                                                 int(arrival_ns), ctypes.byref(t)), allow=(EBUSY,))
        return None if rc == EBUSY else int(t.value)

    def submit_event(self, event, arrival_ns: int = 0):
        return self.submit(event.r, event.phi, event.z, event.layer, event.n_hits, arrival_ns)

    def poll(self, ticket: int, timeout_us: int = 10_000_000, candidates: bool = True, allow=()):
        """(candidates or None, ServeResult) of a finished event; raises HoughError on timeout or an
        error status unless that status is in `allow` (the result is then still returned)."""
        res = ServeResult()
        if candidates:
            out = np.zeros(self.max_candidates, dtype=CANDIDATE_DTYPE)
            rc = self._lib.hough_serve_poll(self._h, ticket, _ptr(out), out.shape[0], ctypes.byref(res),
                                            int(timeout_us))
        else:
            out = None
            rc = self._lib.hough_serve_poll(self._h, ticket, None, 0, ctypes.byref(res), int(timeout_us))
        _check(rc, allow=allow)
        if rc == ETIMEDOUT and res.ticket == 0:
            return None, None
        return (out[: res.n_candidates].copy() if out is not None else None), res

    def drain(self, timeout_us: int = 60_000_000):
        _check(self._lib.hough_serve_drain(self._h, int(timeout_us)))

    def stats(self) -> ServeStats:
        st = ServeStats()
        _check(self._lib.hough_serve_get_stats(self._h, ctypes.byref(st)))
        return st

    def replay(self, pool, arrival_ns, threads: int = 4):
        """hough_serve_replay: offer arrival i = pool[i % len(pool)] (tuples of contiguous r, phi, z
        float32 and layer uint8 arrays) at arrival_ns[i]; returns the ServeResult array."""
        views = (EventView * len(pool))()
        for q, (r, phi, z, layer) in enumerate(pool):
            views[q] = EventView(_ptr(r), _ptr(phi), _ptr(z), _ptr(layer), int(r.shape[0]))
        arr = np.ascontiguousarray(arrival_ns, dtype=np.int64)
        res = (ServeResult * max(1, arr.shape[0]))()
        self._keep_pool = pool
        _check(self._lib.hough_serve_replay(self._h, views, len(pool), _ptr(arr), arr.shape[0], threads, res))
        return np.ctypeslib.as_array(res)[: arr.shape[0]].copy()

    def inject(self, fault: int, on: bool = True):
        _check(self._lib.hough_serve_inject(self._h, int(fault), int(bool(on))))


def tune_lookup(cache_path, geometry, binning, n_events, device=0):
    """The cached tiling (a dict) for these axes, device and batch size, or None."""
    g, b = make_geometry(geometry), make_binning(binning)
    t = Tiling()
    rc = _check(load().hough_tune_lookup(cache_path.encode(), ctypes.byref(g), ctypes.byref(b), device, n_events,
                                         ctypes.byref(t)), allow=(ENOTREADY,))
    return None if rc == ENOTREADY else {n: getattr(t, n) for n in TILING_FIELDS}
