"""FP32 OpenMP CPU implementation of the track finder (hough_cpu.c): a context figure that the
benchmark times on the host cores beside the GPU path.  Neither the FP64 oracle the tests compare
against nor part of the CUDA path; nothing in the package imports it."""
import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "hough_cpu.c")
LIB = os.path.join(HERE, "libhough_cpu.so")
FIELDS = ("iq", "jphi", "mask", "n_members", "icot", "jz0", "mask2", "confirmed")


class Binning(ctypes.Structure):
    _fields_ = [("n_layers", ctypes.c_int32), ("n_qpt", ctypes.c_int32), ("n_phi", ctypes.c_int32),
                ("threshold", ctypes.c_int32), ("n_cot", ctypes.c_int32), ("n_z0", ctypes.c_int32),
                ("b_tesla", ctypes.c_float), ("qpt_min", ctypes.c_float), ("qpt_max", ctypes.c_float),
                ("cot_min", ctypes.c_float), ("cot_max", ctypes.c_float),
                ("z0_min", ctypes.c_float), ("z0_max", ctypes.c_float)]


def build(force: bool = False) -> str:
    """Compile the shared library in place (gcc with OpenMP, no host-specific flags)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O3", "-fopenmp", "-shared", "-fPIC", "-o", tmp, SRC, "-lm"], check=True)
        os.replace(tmp, LIB)
    return LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.hough_cpu_event.restype = ctypes.c_int64
        _lib.hough_cpu_event.argtypes = [ctypes.POINTER(Binning)] + [ctypes.c_void_p] * 4 + [
            ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
    return _lib


def make_binning(geometry, binning) -> Binning:
    return Binning(n_layers=geometry.n_layers, n_qpt=binning.n_qpt, n_phi=binning.n_phi,
                   threshold=binning.threshold, n_cot=binning.n_cot, n_z0=binning.n_z0,
                   b_tesla=geometry.b_tesla, qpt_min=binning.qpt_min, qpt_max=binning.qpt_max,
                   cot_min=binning.cot_min, cot_max=binning.cot_max, z0_min=binning.z0_min, z0_max=binning.z0_max)


def run_event(b: Binning, event, threads: int = 0, cap: int = 1 << 20, want_accumulator: bool = False):
    """The whole path on one event: (candidates as a dict of int arrays, accumulator or None)."""
    lib = _load()
    arr = [np.ascontiguousarray(a, dtype=t) for a, t in
           ((event.r, np.float32), (event.phi, np.float32), (event.z, np.float32), (event.layer, np.uint8))]
    out = np.zeros((cap, len(FIELDS)), dtype=np.int32)
    M = np.zeros((b.n_qpt, b.n_phi), dtype=np.uint16) if want_accumulator else None
    n = lib.hough_cpu_event(ctypes.byref(b), *[a.ctypes.data_as(ctypes.c_void_p) for a in arr], len(arr[0]),
                            int(threads), out.ctypes.data_as(ctypes.c_void_p), cap,
                            M.ctypes.data_as(ctypes.c_void_p) if M is not None else None)
    if n < 0:
        raise ValueError("hough_cpu_event rejected the event")
    kept = out[:min(n, cap)]
    return {f: kept[:, q].copy() for q, f in enumerate(FIELDS)}, M
