"""FP64 CPU oracle of the Hough-transform track finder -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py`` may import this package.  The product path never does: it runs in
the CUDA library and fails loudly when that library is missing.

``hough_oracle.c`` holds the arithmetic (plain loops, IEEE double, no fused
multiply-add); this module compiles it with gcc and marshals numpy arrays.
It imports nothing from the CUDA package; the synthetic events it consumes
come from the shared, arithmetic-free generator module.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hough_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, ETRUNC = 0, -1, -2
ACC_LAYERS, ACC_COUNTS = 0, 1   # accumulator kinds: layer bit masks, saturating vote counts


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fused multiply-add, no fast math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c99",
                               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Binning(ctypes.Structure):
    _fields_ = [("n_layers", ctypes.c_int32), ("n_qpt", ctypes.c_int32), ("n_phi", ctypes.c_int32),
                ("threshold", ctypes.c_int32), ("n_cot", ctypes.c_int32), ("n_z0", ctypes.c_int32),
                ("accumulator", ctypes.c_int32), ("n_d0", ctypes.c_int32),
                ("b_tesla", ctypes.c_double), ("qpt_min", ctypes.c_double), ("qpt_max", ctypes.c_double),
                ("cot_min", ctypes.c_double), ("cot_max", ctypes.c_double),
                ("z0_min", ctypes.c_double), ("z0_max", ctypes.c_double),
                ("d0_min", ctypes.c_double), ("d0_max", ctypes.c_double)]

    @property
    def n_rows(self) -> int:
        """Rows of the stacked grid: d0 slices x q/pT rows."""
        return max(self.n_d0, 1) * self.n_qpt


FLAG_DTYPE = np.dtype([("hit", np.int64), ("row", np.int32), ("bin", np.int32), ("alt", np.int32),
                       ("layer", np.int32), ("kind", np.int32), ("cand", np.int32)], align=True)
CAND_DTYPE = np.dtype([("iq", np.int32), ("jphi", np.int32), ("mask", np.uint32), ("id0", np.int32)],
                      align=True)
STAGE2_DTYPE = np.dtype([("icot", np.int32), ("jz0", np.int32), ("mask2", np.uint32),
                         ("n_votes", np.int32)], align=True)
assert FLAG_DTYPE.itemsize == 32 and CAND_DTYPE.itemsize == 16 and STAGE2_DTYPE.itemsize == 16


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i64p = ctypes.POINTER(ctypes.c_int64)
            lib.oracle_vote.argtypes = [ctypes.POINTER(Binning), P, P, P, ctypes.c_int64, P, P, P,
                                        ctypes.c_int64, i64p]
            lib.oracle_peaks.argtypes = [ctypes.POINTER(Binning), P, P, ctypes.c_int64, i64p]
            lib.oracle_members.argtypes = [ctypes.POINTER(Binning), P, P, P, ctypes.c_int64, P,
                                           ctypes.c_int64, P, P, ctypes.c_int64, P, ctypes.c_int64, i64p]
            lib.oracle_stage2.argtypes = [ctypes.POINTER(Binning), P, P, P, ctypes.c_int64, P,
                                          ctypes.c_int64, P, P, P, P, ctypes.c_int64, i64p]
            for f in (lib.oracle_vote, lib.oracle_peaks, lib.oracle_members, lib.oracle_stage2):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def make_binning(geometry, binning) -> Binning:
    """The oracle's view of a (Geometry, Binning) pair from the event generator."""
    return Binning(n_layers=geometry.n_layers, n_qpt=binning.n_qpt, n_phi=binning.n_phi,
                   threshold=binning.threshold, n_cot=binning.n_cot, n_z0=binning.n_z0,
                   accumulator=int(getattr(binning, "accumulator", ACC_LAYERS)),
                   n_d0=int(getattr(binning, "n_d0", 0)),
                   b_tesla=geometry.b_tesla, qpt_min=binning.qpt_min, qpt_max=binning.qpt_max,
                   cot_min=binning.cot_min, cot_max=binning.cot_max,
                   z0_min=binning.z0_min, z0_max=binning.z0_max,
                   d0_min=float(getattr(binning, "d0_min", -1.0)), d0_max=float(getattr(binning, "d0_max", 1.0)))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _hits(event):
    r = np.ascontiguousarray(event.r, dtype=np.float32)
    phi = np.ascontiguousarray(event.phi, dtype=np.float32)
    z = np.ascontiguousarray(event.z, dtype=np.float32)
    layer = np.ascontiguousarray(event.layer, dtype=np.uint8)
    return r, phi, z, layer


def vote(b: Binning, event):
    """Stage-1 vote.  Returns (M uint16 [n_rows, n_phi], votes_by_layer uint64[16], flags).

    M holds layer masks or saturating vote counts, as ``b.accumulator`` says; its rows are the
    stacked rows m * n_qpt + i of the d0 slices (one slice without a d0 axis), as are the flags'."""
    lib = _load()
    r, phi, _, layer = _hits(event)
    M = np.zeros((b.n_rows, b.n_phi), dtype=np.uint16)
    votes = np.zeros(16, dtype=np.uint64)
    cap = 1 << 16
    while True:
        flags = np.zeros(cap, dtype=FLAG_DTYPE)
        nf = ctypes.c_int64(0)
        rc = lib.oracle_vote(ctypes.byref(b), _ptr(r), _ptr(phi), _ptr(layer), r.shape[0], _ptr(M),
                             _ptr(votes), _ptr(flags), cap, ctypes.byref(nf))
        if rc != OK:
            raise ValueError(f"oracle_vote failed: {rc}")
        if nf.value <= cap:
            return M, votes, flags[: nf.value].copy()
        cap = nf.value


def peaks(b: Binning, M: np.ndarray):
    """Local-maximum candidates in raster order (structured array iq, jphi, mask, id0)."""
    lib = _load()
    M = np.ascontiguousarray(M, dtype=np.uint16)
    cap = max(1024, M.size // 4 + 1)
    out = np.zeros(cap, dtype=CAND_DTYPE)
    n = ctypes.c_int64(0)
    rc = lib.oracle_peaks(ctypes.byref(b), _ptr(M), _ptr(out), cap, ctypes.byref(n))
    if rc != OK:
        raise ValueError(f"oracle_peaks failed: {rc}")
    return out[: n.value].copy()


def members(b: Binning, event, cands: np.ndarray):
    """Member hits of each candidate: (offsets int64[n_cand + 1], hits int64[], flags)."""
    lib = _load()
    r, phi, _, layer = _hits(event)
    cands = np.ascontiguousarray(cands, dtype=CAND_DTYPE)
    nc = cands.shape[0]
    offsets = np.zeros(nc + 1, dtype=np.int64)
    cap, fcap = max(1024, 64 * nc), 1 << 14
    while True:
        mem = np.zeros(cap, dtype=np.int64)
        flags = np.zeros(fcap, dtype=FLAG_DTYPE)
        nf = ctypes.c_int64(0)
        rc = lib.oracle_members(ctypes.byref(b), _ptr(r), _ptr(phi), _ptr(layer), r.shape[0],
                                _ptr(cands), nc, _ptr(offsets), _ptr(mem), cap, _ptr(flags), fcap,
                                ctypes.byref(nf))
        if rc == EINVAL:
            raise ValueError("oracle_members failed")
        if rc == ETRUNC or nf.value > fcap:
            cap = max(cap, int(offsets[-1]))
            fcap = max(fcap, nf.value)
            continue
        return offsets, mem[: offsets[-1]].copy(), flags[: nf.value].copy()


def stage2(b: Binning, event, cands: np.ndarray, offsets: np.ndarray, mem: np.ndarray):
    """Second-stage (cot theta, z0) vote per candidate: (results, flags)."""
    lib = _load()
    r, _, z, layer = _hits(event)
    cands = np.ascontiguousarray(cands, dtype=CAND_DTYPE)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    mem = np.ascontiguousarray(mem, dtype=np.int64)
    nc = cands.shape[0]
    out = np.zeros(max(nc, 1), dtype=STAGE2_DTYPE)
    fcap = 1 << 14
    while True:
        flags = np.zeros(fcap, dtype=FLAG_DTYPE)
        nf = ctypes.c_int64(0)
        rc = lib.oracle_stage2(ctypes.byref(b), _ptr(r), _ptr(z), _ptr(layer), r.shape[0], _ptr(cands),
                               nc, _ptr(offsets), _ptr(mem), _ptr(out), _ptr(flags), fcap,
                               ctypes.byref(nf))
        if rc != OK:
            raise ValueError(f"oracle_stage2 failed: {rc}")
        if nf.value <= fcap:
            return out[:nc].copy(), flags[: nf.value].copy()
        fcap = nf.value


def run(geometry, binning, event):
    """The whole path on one event: vote, peaks, membership, stage 2."""
    b = make_binning(geometry, binning)
    M, votes, vflags = vote(b, event)
    cands = peaks(b, M)
    offsets, mem, mflags = members(b, event, cands)
    s2, zflags = stage2(b, event, cands, offsets, mem)
    return dict(M=M, votes_by_layer=votes, vote_flags=vflags, candidates=cands, member_offsets=offsets,
                members=mem, member_flags=mflags, stage2=s2, stage2_flags=zflags)
