"""The benchmark's host-side accounting (no GPU): the roofline arithmetic, the committed DRAM
traffic figures and their source digests, and the per-kernel table."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1310_7556_gb300 import eventgen as eg  # noqa: E402


def test_roofline_entry_arithmetic():
    e = bench.roofline_entry(2.0, 4e9, 1e10, smem_peak=1e13, hbm_peak=5000.0, peaks_kind="measured")
    assert e["bound"] == "smem_atomic"
    assert e["hbm"]["achieved_gbs"] == pytest.approx(2000.0)       # 4 GB in 2 ms
    assert e["hbm"]["frac"] == pytest.approx(0.4)
    assert e["smem_atomic"]["achieved_votes_per_s"] == pytest.approx(5e12)
    assert e["smem_atomic"]["frac"] == pytest.approx(0.5)
    h = bench.roofline_entry(1.0, 1e9, None, smem_peak=1e13, hbm_peak=5000.0, peaks_kind="measured")
    assert h["bound"] == "hbm" and "smem_atomic" not in h


def test_traffic_figures_follow_their_sources():
    """Every committed figure names a kernel the bench reports; the bench uses it exactly when its
    digest is that of the kernel's current sources (a kernel changed since its capture reports
    null traffic until it is captured again)."""
    path = os.path.join(ROOT, "profiles", "kernel_traffic.txt")
    lines = [ln.rstrip("\n").split("\t") for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert lines
    names = {n for n, _, _ in bench.PLAIN_KERNELS} | {n for n, _, _ in bench.BATCH_STEPS}
    src = {n: s for n, _, s in bench.PLAIN_KERNELS + bench.BATCH_STEPS}
    for kernel, workload, nbytes, digest in lines:
        assert kernel in names
        assert int(nbytes) > 0
        current = bench._sources_digest(src[kernel]) == digest
        assert bench.measured_traffic(kernel, workload, src[kernel]) == (float(nbytes) if current else None)
    assert bench.measured_traffic("confirm_kernel", "no_such_workload", "confirm_kernels.cu") is None


def test_kernel_table_leaves_out_kernels_that_did_not_run():
    w = eg.WORKLOADS["pileup_100k"]
    st = {"cells": w.binning.n_qpt * w.binning.n_phi, "events": 1, "candidates": 397, "general_votes": 0,
          "votes": 50067216, "members": 18425, "stage2_votes": 177107,
          "stage_ms": {k: 0.01 for _, k, _ in bench.PLAIN_KERNELS}}
    st["stage_ms"]["clear_ms"] = 0.0
    st["stage_ms"]["compact_ms"] = 0.0
    table = bench.kernel_table(w, 99794, st, 8.9e12, 6663.9, "measured")
    assert "clear_kernel" not in table and "compact_kernel" not in table
    assert table["confirm_kernel"]["smem_atomic"]["votes"] == 177107
    assert sum(e["share"] for e in table.values()) == pytest.approx(1.0, rel=1e-6)


def test_every_workload_named_on_the_command_line_exists():
    for name in bench.WORKLOAD_TEXT:
        assert name in eg.WORKLOADS


def _profile_commands():
    """Every ncu command line of the committed profile summaries (continuation lines joined)."""
    out = []
    pdir = os.path.join(ROOT, "profiles")
    for name in sorted(os.listdir(pdir)):
        text = open(os.path.join(pdir, name)).read().replace("\\\n", " ")
        for line in text.splitlines():
            k = line.find("ncu --")
            if k >= 0 and ("--metrics" in line or "--set" in line) and "python " in line[k:]:
                out.append((name, line[k:].strip()))
    assert out
    return out


def test_profile_recipes_keep_clocks_and_one_kernel_per_full_capture():
    """Each ncu command in profiles/ leaves the GPU clocks alone, and a capture that collects more
    than the launch time targets one kernel (-k) and at most three launches (-c)."""
    for name, cmd in _profile_commands():
        assert "--clock-control none" in cmd, (name, cmd)
        if "--set" in cmd or "dram__" in cmd or "smsp__" in cmd:
            assert " -k " in cmd, (name, cmd)
            c = cmd.split(" -c ")[1].split()[0]
            assert int(c) <= 3, (name, cmd)


def test_profile_recipes_run_committed_files_only():
    """The commands behind the profiles run bench.py with its own options, nothing from a working folder."""
    for name, cmd in _profile_commands():
        assert "_work" not in cmd, (name, cmd)
        for tok in cmd.split():
            if tok.endswith(".py"):
                assert os.path.exists(os.path.join(ROOT, tok)), (name, tok)
