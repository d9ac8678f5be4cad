"""Host-side logic of bench.py (CPU): the roofline numerator's algorithmic bytes, the
solve-only rate, the kernel-source hash that keys stored ncu captures, and the stored
traffic records themselves."""
import glob
import importlib.util
import json
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_algorithmic_bytes_counts(bench):
    N, F = 1000, 2970
    # one FP64 PCG iteration: p update 32N, A p with p.q 24N + 16F, updates with dots 56N
    assert bench.algorithmic_bytes(N, F, 1, 0, 0) == 112 * N + 16 * F
    # the same passes on 4-byte values
    assert bench.algorithmic_bytes(N, F, 1, 0, 1) == 56 * N + 12 * F
    # per step: assembly 40N + 16F and initial residual 48N + 16F
    assert bench.algorithmic_bytes(N, F, 0, 1, 0) == 88 * N + 32 * F
    assert bench.algorithmic_bytes(N, F, 7, 3, 0) == 7 * (112 * N + 16 * F) + 3 * (88 * N + 32 * F)


def test_solve_only_rate(bench):
    phases = {"p_update": 0.1, "amul_dot": 0.5, "update_dots": 0.4, "rows_initial_residual": 9.0}
    r = bench.solve_only(8_000_000, 500, 100, phases)  # 5 iterations per step over 1.0 ms per step
    assert r["iteration_passes_ms_per_step"] == pytest.approx(1.0)
    assert r["value"] == pytest.approx(8_000_000 * 5 / 1e-3)
    assert bench.solve_only(10, 1, 1, {"p_update": 0.0, "amul_dot": 0.0, "update_dots": 0.0})["value"] is None


def test_code_tokens_ignore_comments_and_layout(bench):
    a = "int f(int x) {  // one\n  return x + 1; /* two\n three */ }\n"
    b = "int f(int x) { return x + 1; }"
    assert bench._code_tokens(a) == bench._code_tokens(b)
    assert bench._code_tokens(a) != bench._code_tokens(b.replace("+ 1", "+ 2"))
    # a division survives, a trailing comment does not
    assert bench._code_tokens("a = b / c; // d") == "a = b / c;"


def test_kernel_hash_covers_each_family(bench):
    hashes = {fam: bench.kernel_hash(fam) for fam in bench.KERNEL_SOURCES}
    assert all(re.fullmatch(r"[0-9a-f]{16}", h) for h in hashes.values())
    assert len(set(hashes.values())) == len(hashes)  # the families' sources differ
    for fam, files in bench.KERNEL_SOURCES.items():
        for f in files:
            assert os.path.exists(os.path.join(ROOT, "paper_2507_18268_gb300", f)), (fam, f)


def test_traffic_records_are_consistent():
    recs = sorted(glob.glob(os.path.join(ROOT, "profiles", "traffic_*.json")))
    assert recs
    for p in recs:
        with open(p) as fh:
            d = json.load(fh)
        assert d["ratio"] == pytest.approx(d["dram_bytes"] / d["algorithmic_bytes"], rel=1e-3), p
        assert 0.9 < d["ratio"] < 2.0, p
        assert "--clock-control none" in d["command"] and d["command"].startswith("ncu "), p
        assert re.fullmatch(r"[0-9a-f]{16}", d["kernel_hash"]), p
