"""A loop split by WFS on one GPU (paper_1903_01852_gb300.shard): shard loops
(RTC_FLAG_PARTIAL) write their partial reconstructions into a master's inputs,
the master applies the control law; against the FP64 oracle and the unsplit loop,
through the C ABI."""
import copy

import numpy as np
import pytest

from oracle import OracleLoop, quantize_rows
from paper_1903_01852_gb300 import shard, synth
from parity_util import TOL_F32, WAIT_US, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    return torch


def lgs_groups(cfg):
    """One shard per LGS (80x80 or 68x68 SH) and one for the NGS (2x2), as the paper's nodes."""
    big = [k for k, w in enumerate(cfg["wfs"]) if w["nsubx"] > 2]
    small = [k for k, w in enumerate(cfg["wfs"]) if w["nsubx"] <= 2]
    return [[k] for k in big] + ([small] if small else [])


def test_sharded_mcao_equals_the_oracle_and_the_unsplit_loop(rtc, torch_cuda):
    cfg = synth.make_config("mcao")
    frames = synth.draw_frames(cfg, 2, seed=401)
    ref = OracleLoop(cfg)
    with shard.ShardedLoop(cfg, lgs_groups(cfg)) as sl, rtc.Loop(cfg) as whole:
        assert len(sl.shards) == 7
        for k, f in enumerate(frames):
            sl.submit_frame(k + 1, f)
            fid, a = sl.get_commands(timeout_us=WAIT_US)
            whole.submit_frame(k + 1, f)
            _, b = whole.get_commands(timeout_us=WAIT_US)
            a_ref = ref.step(f)[1]
            assert fid == k + 1
            assert rel(a, a_ref) <= TOL_F32 and rel(a, b) <= TOL_F32
        assert all(lp.check_guards() == 0 for lp in sl.shards)


def test_one_shard_is_the_unsplit_loop_bit_for_bit(rtc, torch_cuda):
    # one shard holding every WFS: the master adds one partial (exactly) and applies
    # the same float32 operations as the loop's fused finalisation
    cfg = synth.make_config("elt_scao_sh", polc=True, with_ref=True)
    frames = synth.draw_frames(cfg, 3, seed=402)
    with shard.ShardedLoop(cfg, [[0]]) as sl, rtc.Loop(cfg) as whole:
        for k, f in enumerate(frames):
            sl.submit_frame(k + 1, f)
            whole.submit_frame(k + 1, f)
            assert np.array_equal(sl.get_commands(timeout_us=WAIT_US)[1], whole.get_commands(timeout_us=WAIT_US)[1])


@pytest.mark.parametrize("fmt", ["bf16", "e4m3"])
def test_sharded_quantised_ltao_row_chunks_and_graphs(rtc, torch_cuda, fmt):
    # shards keep the full rows' scales; chunked submission and graph mode give the same commands
    cfg = synth.make_config("ltao")
    q = copy.copy(cfg)
    codes, scale = quantize_rows(cfg["M"], fmt)
    pc, ps = quantize_rows(cfg["P"], fmt)
    q.update(M=codes, M_scale=scale, M_dtype=fmt, P=pc, P_scale=ps, P_dtype=fmt)
    frames = synth.draw_frames(q, 2, seed=403)
    plans = [synth.chunk_plan(w, 8 if w["nsubx"] > 2 else 1) for w in q["wfs"]]
    groups = [[0, 1, 2], [3, 4], [5, 6]]
    ref = OracleLoop(q)
    with shard.ShardedLoop(q, groups) as chunked, shard.ShardedLoop(q, groups, graphs=True) as graph:
        for k, f in enumerate(frames):
            chunked.submit_frame(k + 1, f, plans)
            graph.submit_frame(k + 1, f)
            a = chunked.get_commands(timeout_us=WAIT_US)[1]
            b = graph.get_commands(timeout_us=WAIT_US)[1]
            assert np.array_equal(a, b)
            assert rel(a, ref.step(f)[1]) <= TOL_F32


def test_master_inputs_copied_from_host_equal_the_shards_writes(rtc, torch_cuda):
    # the multi-node form: partials read back to the host and copied into another
    # master (rtc_master_set_input) give the same commands as the shards' own writes
    cfg = synth.make_config("scao_small", polc=True)
    frames = synth.draw_frames(cfg, 4, seed=404)
    rng = np.random.default_rng(5)
    wfs = [synth.sh_wfs(rng, 16, 8, 128, 128, 0.0, nblocks=2)]
    cfg2 = dict(cfg, wfs=cfg["wfs"] + wfs, ns=cfg["ns"] + 2 * synth.num_valid(wfs[0]),
                M=np.concatenate([cfg["M"], synth.control_matrix(rng, cfg["na"], 2 * synth.num_valid(wfs[0]))], 1))
    frames = [f + g for f, g in zip(frames, synth.draw_frames(dict(cfg, wfs=wfs), 4, seed=405))]
    _, master_cfg = shard.split(cfg2, [[0], [1]])
    with shard.ShardedLoop(cfg2, [[0], [1]]) as sl, rtc.Master(master_cfg, 2) as m2:
        for k, f in enumerate(frames):
            sl.submit_frame(k + 1, f)
            a = sl.get_commands(timeout_us=WAIT_US)[1]
            for j, y in enumerate(sl.partials()):
                m2.set_input(j, y)
            m2.step(k + 1)
            fid, b = m2.get_commands(timeout_us=WAIT_US)
            assert fid == k + 1 and np.array_equal(a, b)
        with pytest.raises(rtc.RtcError):
            m2.step(2)                                   # frame ids must increase
