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


class FakeLoop:
    """Records the rounds run_host_path submits; get_commands sleeps a set time."""

    def __init__(self, wait_s=0.0):
        self.rounds, self.wait_s = [], wait_s

    @staticmethod
    def chunks(frame_id, items):
        return [type("Chunk", (), {"frame_id": frame_id, "item": it})() for it in items]

    def submit_chunks(self, arr):
        self.rounds.append([(c.frame_id, c.item[0], c.item[1], c.item[2]) for c in arr])

    def get_commands(self, timeout_us=-1):
        import time
        if self.wait_s:
            time.sleep(self.wait_s)
        return 0, None


class NoSampler:
    def mark(self, on):
        pass


def test_host_path_submits_one_round_per_call_and_times_from_the_arrival():
    # three cameras, two with three chunks and one with a single chunk: the rounds are
    # chunk c of every camera that has one, every frame id rewritten per frame
    frames = [[np.zeros((6, 4), np.int16), np.zeros((6, 4), np.int16), np.zeros((3, 4), np.int16)]] * 2
    plans = [[(0, 2), (2, 4), (4, 6)], [(0, 3), (3, 5), (5, 6)], [(0, 3)]]
    loop = FakeLoop(wait_s=0.002)
    arrival, slowest = [], {}
    lat, fid = bench.run_host_path(loop, frames, plans, 4, 1, NoSampler(), 10, paced=True, arrival=arrival,
                                   slowest=slowest, hz=200.0, readout_ms=1.0)
    assert fid == 15 and len(lat) == 4 and len(arrival) == 4
    assert len(loop.rounds) == 5 * 3
    for k in range(5):
        r0, r1, r2 = loop.rounds[3 * k:3 * k + 3]
        assert r0 == [(10 + k, 0, 0, 2), (10 + k, 1, 0, 3), (10 + k, 2, 0, 3)]
        assert r1 == [(10 + k, 0, 2, 4), (10 + k, 1, 3, 5)] and r2 == [(10 + k, 0, 4, 6), (10 + k, 1, 5, 6)]
    # the clock starts at the last round's arrival, before its call: at least the 2 ms wait
    assert all(a >= l >= 2000.0 for a, l in zip(arrival, lat))
    assert set(slowest) == {"frame", "latency_us", "submit_calls_us", "get_commands_wait_us"}
    assert slowest["latency_us"] == max(lat) and slowest["get_commands_wait_us"] >= 2000.0
