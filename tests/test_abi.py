"""The C-ABI library: it builds for sm_103a, loads without a GPU and exports every entry point
that include/hough.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hough.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hough_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1310_7556_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_path():
    names = _declared()
    for required in ("hough_create", "hough_vote", "hough_peaks", "hough_stage2", "hough_destroy",
                     "hough_get_candidates", "hough_get_accumulator", "hough_get_stats", "hough_process"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, f"declared but not exported: {missing}"


def test_binding_covers_every_declared_symbol(lib):
    from paper_1310_7556_gb300 import binding
    assert set(_declared()) <= set(binding._SIGNATURES), set(_declared()) - set(binding._SIGNATURES)


def test_struct_layouts_match_header(lib):
    from paper_1310_7556_gb300 import binding
    assert ctypes.sizeof(binding.Geometry) == 16
    assert ctypes.sizeof(binding.Binning) == 6 * 4 + 6 * 8 + 2 * 4 + 2 * 8
    assert ctypes.sizeof(binding.Limits) == 16
    assert binding.CANDIDATE_DTYPE.itemsize == 32
    assert ctypes.sizeof(binding.Tiling) == 32


def test_binding_constants_match_header():
    """Every integer #define of the header that the binding names (prefix HOUGH_ dropped) has the
    header's value; the vote modes, accumulators and status codes must all be named."""
    from paper_1310_7556_gb300 import binding
    text = open(HEADER).read()
    defines = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define\s+HOUGH_(\w+)\s+\(?(-?\d+)\)?", text)}
    for name in ("VOTE_GATHER", "VOTE_SCATTER", "VOTE_FUSED", "ACC_LAYERS", "ACC_COUNTS", "OK", "EINVAL",
                 "ENOTREADY", "EBUSY", "HOST", "DEVICE"):
        assert name in defines and hasattr(binding, name), name
    for name, value in defines.items():
        if hasattr(binding, name):
            assert getattr(binding, name) == value, name


def test_version_and_error_strings_without_gpu(lib):
    from paper_1310_7556_gb300 import binding
    L = binding.load()
    assert L.hough_version().decode().count(".") == 2
    assert isinstance(L.hough_last_error(), bytes)


def test_invalid_arguments_are_rejected_before_any_device_call(lib):
    """hough_create checks its arguments first: a bad binning is HOUGH_EINVAL even without a GPU."""
    from paper_1310_7556_gb300 import binding
    L = binding.load()
    g = binding.Geometry(n_layers=10, reserved=0, b_tesla=3.8)
    b = binding.Binning(n_qpt=128, n_phi=100, threshold=8, n_cot=64, n_z0=64, reserved=0,
                        qpt_min=-1, qpt_max=1, cot_min=-6, cot_max=6, z0_min_cm=-15, z0_max_cm=15)
    lim = binding.Limits(max_hits=10, max_candidates=10, max_members=10)
    h = ctypes.c_void_p()
    rc = L.hough_create(ctypes.byref(g), ctypes.byref(b), ctypes.byref(lim), 0, ctypes.byref(h))
    assert rc == binding.EINVAL and b"n_phi" in L.hough_last_error()
    b.n_phi = 256
    g.n_layers = 17
    assert L.hough_create(ctypes.byref(g), ctypes.byref(b), ctypes.byref(lim), 0, ctypes.byref(h)) == binding.EINVAL
    assert not h.value


def test_product_path_has_no_cpu_fallback():
    """The binding raises when the library is absent instead of computing anything on the CPU."""
    import importlib
    from paper_1310_7556_gb300 import binding
    saved = binding._LIB_PATH, binding._lib
    try:
        binding._LIB_PATH = os.path.join(ROOT, "does-not-exist.so")
        binding._lib = None
        with pytest.raises(RuntimeError):
            binding.load()
    finally:
        binding._LIB_PATH, binding._lib = saved
    src = open(binding.__file__).read()
    assert "import oracle" not in src and "from oracle" not in src
