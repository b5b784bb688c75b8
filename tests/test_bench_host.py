"""Host-side logic of bench.py (CPU): latency statistics, the kernel-source hash that
ties the committed ncu figures to the kernels they were taken on, and those figures."""
import os

import numpy as np

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
MCAO_ALGORITHMIC_BYTES = 1_671_642_432     # one FP32 MVM launch with its fused finalisation


def test_stats_percentiles_jitter_and_deadline_misses():
    rng = np.random.default_rng(5)
    xs = list(rng.normal(35.0, 1.5, 1001)) + [2500.0, 3000.0]
    s = bench.stats(xs, period_us=2000.0)
    for q, key in ((50, "p50"), (99, "p99"), (99.9, "p999")):
        assert abs(s[key] - float(np.percentile(xs, q))) < 1e-9
    assert abs(s["jitter_rms"] - float(np.std(xs))) < 1e-9
    assert s["max"] == 3000.0 and s["n"] == len(xs) and s["deadline_misses"] == 2
    assert "deadline_misses" not in bench.stats(xs)


def test_kernel_source_hash_ignores_comments_and_whitespace_only():
    base = {"rtc_kernels.cu": "int f(int a) { return a + 1; }  // one\n/* two */",
            "rtc_internal.h": "struct S { int x; };"}
    h = bench.kernel_source_hash(base)
    reworded = {"rtc_kernels.cu": "// another comment\nint f(int a)\n{\n    return a + 1;   /* changed */\n}",
                "rtc_internal.h": "struct S {\n    int x;  // x\n};"}
    assert bench.kernel_source_hash(reworded) == h
    changed = dict(base, **{"rtc_kernels.cu": "int f(int a) { return a + 2; }"})
    assert bench.kernel_source_hash(changed) != h


def test_committed_mvm_profile_is_consistent():
    # The summary carries the hash and the DRAM bytes of one full MCAO launch; the bench
    # reports them only while the hash matches the source.  When it does, the traffic
    # must be the algorithmic bytes plus at most the 16-byte row padding (no re-reads).
    lines = open(os.path.join(ROOT, "profiles", "gemv_f32_mcao.md")).read().splitlines()
    fields = dict(l.split(":", 1) for l in lines if l.startswith(("kernel_source_sha256_16:",
                                                                  "dram_bytes_per_full_launch:")))
    assert len(fields["kernel_source_sha256_16"].strip()) == 16
    traffic = float(fields["dram_bytes_per_full_launch"])
    assert 1.0 <= traffic / MCAO_ALGORITHMIC_BYTES <= 1.01
    got = bench.profiled_traffic()
    if fields["kernel_source_sha256_16"].strip() == bench.kernel_source_hash():
        assert got == traffic
    else:
        assert got is None
