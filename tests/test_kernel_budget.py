"""Register and spill budgets of the hot kernels (CPU only: nvcc cross-compiles
for sm_103a here).  The measured bandwidths depend on occupancy: the float32
MVM runs 8 CTAs of 256 threads per SM only at <= 32 registers, the BF16 one 4
at <= 64.  A source change that raises them shows here before it shows as a
slower kernel on the GPU (a single-block float32 launch at 34 registers ran as
1.03 waves, and the POLC product took 51 instead of 41 us)."""
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_1903_01852_gb300", "csrc", "rtc_kernels.cu")

# mangled entry -> (what, register budget, spill budget in bytes)
BUDGET = {
    "_ZN3rtc11gemv_kernelILi0ELi4ELi1ELi4ELb0ELi1EEEvNS_8GemvArgsE": ("float32 MVM, 4 rows per warp", 32, 0),
    # one row per warp (single-block launches: the POLC product, a row chunk's block, and every
    # float32 launch too small for four rows per warp): held to 32 registers so that their ~1000
    # CTAs fit one wave (no spill with packed float32 sums; a few bytes allowed)
    "_ZN3rtc16gemv_kernel_1rowILi0ELi4ELi1ELb0EEEvNS_8GemvArgsE": ("float32 MVM, 1 row per warp", 32, 32),
    "_ZN3rtc11gemv_kernelILi1ELi2ELi4ELi4ELb0ELi1EEEvNS_8GemvArgsE": ("BF16 MVM", 64, 0),
    "_ZN3rtc11gemv_kernelILi2ELi1ELi4ELi4ELb0ELi1EEEvNS_8GemvArgsE": ("E4M3 MVM", 48, 0),
    # two column blocks per CTA (whole-frame BF16 / E4M3 launches), held to the one-block kernels' CTAs per SM
    "_ZN3rtc19gemv_kernel_groupedILi1ELi2ELi4ELi4ELb0ELi2EEEvNS_8GemvArgsE": ("BF16 MVM, two blocks per CTA", 64, 0),
    "_ZN3rtc19gemv_kernel_groupedILi2ELi1ELi4ELi4ELb0ELi2EEEvNS_8GemvArgsE": ("E4M3 MVM, two blocks per CTA", 48, 0),
    # the single-block E4M3 product without finalisation (POLC): two vectors per lane, two CTAs per SM
    "_ZN3rtc16gemv_kernel_deepILi2ELi2ELi4ELb0EEEvNS_8GemvArgsE": ("E4M3 POLC product", 128, 0),
    # a pre-enqueued chunk's MVM (its mailbox checked after the wait for the slopes); a chunk's
    # launches are small enough to take one row per warp
    "_ZN3rtc16gemv_kernel_1rowILi0ELi4ELi1ELb1EEEvNS_8GemvArgsE": ("float32 MVM, 1 row per warp, pre-enqueued",
                                                                  32, 32),
    "_ZN3rtc13slopes_kernelILb0ELb0EEEvNS_9SlopeArgsE": ("slope kernel", 64, 0),
    # pixels read over the CPU-GPU link: every pixel row of a thread and its calibration in flight at
    # once (launched for row chunks, a few dozen CTAs: one per SM is enough)
    "_ZN3rtc13slopes_kernelILb1ELb0EEEvNS_9SlopeArgsE": ("slope kernel, host pixels", 232, 0),
    # pre-enqueued chunks (launched behind the one-warp gate kernel)
    "_ZN3rtc13slopes_kernelILb0ELb1EEEvNS_9SlopeArgsE": ("slope kernel, pre-enqueued", 64, 0),
    "_ZN3rtc13slopes_kernelILb1ELb1EEEvNS_9SlopeArgsE": ("slope kernel, host pixels, pre-enqueued", 232, 0),
}


def ptxas_report():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    r = subprocess.run([nvcc, "-std=c++17", "-O3", "-gencode", "arch=compute_103a,code=sm_103a", "-Xptxas", "-v",
                        "-I", os.path.join(ROOT, "include"), "-c", SRC, "-o", os.devnull],
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    report, entry = {}, None
    for line in (r.stdout + r.stderr).splitlines():
        m = re.search(r"Compiling entry function '(\w+)'", line)
        if m:
            entry = m.group(1)
            continue
        m = re.search(r"(\d+) bytes spill stores, (\d+) bytes spill loads", line)
        if m and entry:
            report.setdefault(entry, {})["spill"] = int(m.group(1)) + int(m.group(2))
        m = re.search(r"Used (\d+) registers", line)
        if m and entry:
            report.setdefault(entry, {})["regs"] = int(m.group(1))
    return report


def test_hot_kernels_stay_within_their_register_budget_without_spills():
    rep = ptxas_report()
    for name, (what, budget, spill) in BUDGET.items():
        assert name in rep, f"{what}: entry {name} not compiled"
        assert rep[name]["regs"] <= budget, f"{what}: {rep[name]['regs']} registers > {budget}"
        assert rep[name].get("spill", 0) <= spill, f"{what}: {rep[name]['spill']} bytes of spill > {spill}"
    spilling = {k: v["spill"] for k, v in rep.items() if v.get("spill") and k not in BUDGET}
    assert not spilling, spilling
