"""The per-WFS split of a loop (paper_1903_01852_gb300.shard) on CPU: the shard
configurations' partial reconstructions add up to the whole loop's, and the
multi-process orchestration (partials gathered to rank 0 over torch.distributed,
two gloo ranks) gives the unsplit loop's commands.  The shards and the master are
the FP64 oracle here; the GPU tests run them on the library."""
import os
import socket

import numpy as np
import pytest

from oracle import OracleLoop, control_step, frame_slopes, mvm, quantize_rows, stored_matrix
from paper_1903_01852_gb300 import shard, synth


def small_loop(seed=7, fmt="f32"):
    rng = np.random.default_rng(seed)
    wfs = [synth.sh_wfs(rng, 6, 6, 40, 38, 0.2, nblocks=2),
           synth.pyramid_wfs(rng, 10, 26, 24, 0.0, nblocks=2),
           synth.sh_wfs(rng, 3, 8, 26, 25, 0.0, nblocks=1),
           synth.sh_wfs(rng, 2, 5, 10, 11, 0.0, nblocks=1)]
    ns = sum(2 * synth.num_valid(w) for w in wfs)
    na = 23
    cfg = dict(name="split", na=na, ns=ns, wfs=wfs, M=synth.control_matrix(rng, na, ns, sd=1e-2), M_scale=None,
               M_dtype="f32", P=synth.polc_matrix(rng, na), P_scale=None, P_dtype="f32", gain=0.4, leak=0.02,
               clip=None, a0=rng.normal(0, 0.05, na).astype(np.float32),
               ref_slopes=rng.normal(0, 0.1, ns).astype(np.float32))
    if fmt != "f32":
        codes, scale = quantize_rows(cfg["M"], fmt)
        cfg.update(M=codes, M_scale=scale, M_dtype=fmt)
    return cfg


GROUPS = [[0, 2], [1], [3]]


@pytest.mark.parametrize("fmt", ["f32", "bf16", "e4m3"])
def test_shard_partials_add_up_to_the_whole_reconstruction(fmt):
    cfg = small_loop(fmt=fmt)
    frames = synth.draw_frames(cfg, 2, seed=8)
    shards, master = shard.split(cfg, GROUPS)
    m_full = stored_matrix(cfg["M"], cfg["M_dtype"], cfg["M_scale"])
    cols = shard.wfs_columns(cfg)
    for f in frames:
        s_full = frame_slopes(cfg, f)
        total = np.zeros(cfg["na"])
        for g, sc in zip(GROUPS, shards):
            s = frame_slopes(sc, [f[k] for k in g])
            # a shard's slopes are the whole loop's slopes of its WFS, in its WFS order
            assert np.array_equal(s, np.concatenate([s_full[slice(*cols[k])] for k in g]))
            total += mvm(stored_matrix(sc["M"], sc["M_dtype"], sc["M_scale"]), s)
        np.testing.assert_allclose(total, mvm(m_full, s_full), rtol=0, atol=1e-12 * np.abs(m_full).sum())
    assert master["P"] is cfg["P"] and all(sc["P"] is None for sc in shards)
    assert sum(sc["ns"] for sc in shards) == cfg["ns"]


def test_split_rejects_groups_that_miss_or_repeat_a_wfs():
    cfg = small_loop()
    for bad in ([[0, 1], [2]], [[0, 1], [1, 2, 3]], [[0, 1, 2, 3, 4]]):
        with pytest.raises(ValueError):
            shard.split(cfg, bad)


class OracleShard:
    """A shard computed by the oracle: partial reconstruction of its WFS in float32."""

    def __init__(self, cfg):
        self.cfg = cfg
        self.m = stored_matrix(cfg["M"], cfg["M_dtype"], cfg["M_scale"])
        self.last = None

    def submit_frame(self, fid, frames):
        self.last = (fid, mvm(self.m, frame_slopes(self.cfg, frames)).astype(np.float32))

    def get_commands(self):
        return self.last


class OracleMaster:
    """The control law in float64 on the master's inputs (implicit POLC after the commands)."""

    def __init__(self, cfg, nshards):
        na = cfg["na"]
        self.cfg = cfg
        self.y = np.zeros((nshards, na))
        self.p = stored_matrix(cfg["P"], cfg["P_dtype"], cfg["P_scale"]) if cfg.get("P") is not None else None
        self.a = np.zeros(na) if cfg.get("a0") is None else np.asarray(cfg["a0"], np.float64)
        self.q = self.p @ self.a if self.p is not None else np.zeros(na)
        self.out = None

    def set_input(self, k, y):
        self.y[k] = y

    def step(self, fid):
        self.a = control_step(self.a, self.y.sum(axis=0), self.q, self.cfg["gain"], self.cfg["leak"],
                              self.cfg.get("clip"))
        if self.p is not None:
            self.q = self.p @ self.a
        self.out = (fid, self.a.copy())

    def get_commands(self):
        return self.out


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    sys.path.insert(0, os.path.join(root, "tests"))
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import test_shard_host as t
    cfg = t.small_loop()
    frames = synth.draw_frames(cfg, 4, seed=9)
    res = shard.run_rank(cfg, t.GROUPS, frames, rank, world, t.OracleShard, t.OracleMaster, dist)
    out[rank] = None if res is None else [a.tolist() for a in res]
    dist.barrier()
    dist.destroy_process_group()


def test_run_rank_two_gloo_ranks_give_the_unsplit_loop():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[1] is None and len(res[0]) == 4
    cfg = small_loop()
    ref = OracleLoop(cfg)
    for a, f in zip(res[0], synth.draw_frames(cfg, 4, seed=9)):
        a_ref = ref.step(f)[1]
        # the partials travel in float32: their rounding only
        assert np.max(np.abs(np.asarray(a) - a_ref)) <= 1e-6 * np.max(np.abs(a_ref))
