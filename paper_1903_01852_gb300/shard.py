"""A loop split by WFS: reconstruction shards and a master (Section 3).

The paper gives each WFS (or group of WFS) its own reconstruction node, which
turns that WFS's pixels into its share of the DM commands, the partial
reconstruction y_k = M[:, cols_k] s_k; a master adds the nodes' partials and
applies the control law (implicit POLC and the leaky integrator, Section 3.4).
Here a node is a loop created with RTC_FLAG_PARTIAL over the WFS of its group
(its columns of the control matrix, in their slope order; BF16 / E4M3 shards
keep the full matrix's row scales, so their codes are a plain column slice),
and the master is ``binding.Master``.

``ShardedLoop`` runs every shard and the master on one GPU: each shard's kernel
writes its partial straight into the master's input.  ``run_rank`` is the
multi-process form, one process per rank (one GPU each on a multi-GPU node):
rank r runs the shards r, r + world, ...; each frame the ranks' partials are
gathered to rank 0 in shard order over torch.distributed, and rank 0 steps the
master.  Both take the shards' and the master's constructors as arguments so
that the orchestration can run on other backends.
"""
from __future__ import annotations

import numpy as np

from . import synth


def wfs_columns(cfg):
    """[first, end) slope columns of each WFS, in configuration order."""
    offs = [0]
    for w in cfg["wfs"]:
        offs.append(offs[-1] + 2 * synth.num_valid(w))
    return [(offs[k], offs[k + 1]) for k in range(len(cfg["wfs"]))]


def split(cfg, groups):
    """The shard configurations (one per group of WFS indices) and the master's.

    A shard holds its WFS, their columns of M (codes and the full rows' scales
    for BF16 / E4M3), their reference slopes, and no POLC matrix.  The master
    holds na, P, gain, leak, clip and a0."""
    seen = sorted(k for g in groups for k in g)
    if seen != list(range(len(cfg["wfs"]))):
        raise ValueError("the groups must hold every WFS exactly once")
    cols = wfs_columns(cfg)
    shards = []
    for g in groups:
        idx = np.concatenate([np.arange(*cols[k]) for k in g]) if g else np.zeros(0, np.int64)
        ref = cfg.get("ref_slopes")
        shards.append(dict(
            name=f"{cfg.get('name', 'loop')}[{','.join(map(str, g))}]", na=cfg["na"], ns=int(idx.size),
            wfs=[cfg["wfs"][k] for k in g], M=np.ascontiguousarray(np.asarray(cfg["M"])[:, idx]),
            M_scale=cfg.get("M_scale"), M_dtype=cfg.get("M_dtype", "f32"), P=None, P_scale=None, P_dtype="f32",
            gain=cfg["gain"], leak=cfg["leak"], clip=None, a0=None,
            ref_slopes=None if ref is None else np.ascontiguousarray(np.asarray(ref)[idx])))
    master = dict(na=cfg["na"], wfs=[], P=cfg.get("P"), P_scale=cfg.get("P_scale"), P_dtype=cfg.get("P_dtype", "f32"),
                  gain=cfg["gain"], leak=cfg["leak"], clip=cfg.get("clip"), a0=cfg.get("a0"))
    return shards, master


class ShardedLoop:
    """Every shard and the master on one GPU; the shards write their partials
    into the master's inputs (rtc_set_partial_output)."""

    def __init__(self, cfg, groups, device=0, telemetry=False, graphs=False):
        from . import binding
        self.groups = [list(g) for g in groups]
        shard_cfgs, master_cfg = split(cfg, self.groups)
        self.master = binding.Master(master_cfg, len(self.groups), device)
        self.shards = []
        try:
            for k, c in enumerate(shard_cfgs):
                lp = binding.Loop(c, device=device, partial=True, telemetry=telemetry, graphs=graphs)
                self.shards.append(lp)
                binding.set_partial_output(lp, self.master.input(k))
        except Exception:
            self.close()
            raise
        self.graphs = graphs
        self.last_partials = []

    def submit_frame(self, frame_id, frames, plans=None, timeout_us=60_000_000):
        """One frame: each shard gets its WFS's pixels (row chunks per plans, or
        its graph buffers in graph mode); once every shard's partial is written,
        the master steps."""
        for g, lp in zip(self.groups, self.shards):
            sub = [frames[k] for k in g]
            if self.graphs:
                for b, f in zip(lp.next_frame_buffers(), sub):
                    b[:] = f
                lp.submit_graph(frame_id)
            else:
                lp.submit_frame(frame_id, sub, None if plans is None else [plans[k] for k in g])
        self.last_partials = []
        for lp in self.shards:
            got, y = lp.get_commands(timeout_us=timeout_us)
            if got != frame_id:
                raise RuntimeError(f"shard returned frame {got}, expected {frame_id}")
            self.last_partials.append(np.array(y, copy=True))
        self.master.step(frame_id)

    def get_commands(self, timeout_us=60_000_000):
        return self.master.get_commands(timeout_us=timeout_us)

    def partials(self):
        """The shards' partial reconstructions of the last frame (host copies), in shard order."""
        return list(self.last_partials)

    def close(self):
        for lp in self.shards:
            lp.close()
        self.shards = []
        self.master.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def run_rank(cfg, groups, frames, rank, world, make_shard, make_master, dist, device=None):
    """The multi-process split: rank r runs shards r, r + world, ... (make_shard(shard_cfg)
    returns an object with submit_frame(frame_id, frames) and get_commands() -> (id, y));
    each frame the partials are gathered to rank 0 (dist.gather of float32 tensors on
    `device`, None for CPU tensors), which loads them into the master (make_master(master_cfg,
    nshards) returns an object with set_input, step, get_commands) in shard order and steps
    it.  Returns rank 0's commands per frame (None on the other ranks)."""
    import torch
    shard_cfgs, master_cfg = split(cfg, groups)
    mine = list(range(rank, len(groups), world))
    shards = {k: make_shard(shard_cfgs[k]) for k in mine}
    master = make_master(master_cfg, len(groups)) if rank == 0 else None
    per_rank = [list(range(r, len(groups), world)) for r in range(world)]
    nmax = max(len(p) for p in per_rank)
    na = int(cfg["na"])
    out = [] if rank == 0 else None
    try:
        for fid, frame in enumerate(frames, start=1):
            for k in mine:
                shards[k].submit_frame(fid, [frame[w] for w in groups[k]])
            mat = np.zeros((nmax, na), np.float32)
            for i, k in enumerate(mine):
                got, y = shards[k].get_commands()
                if got != fid:
                    raise RuntimeError(f"shard {k} returned frame {got}, expected {fid}")
                mat[i] = y
            t = torch.from_numpy(mat)
            if device is not None:
                t = t.to(device)
            bufs = [torch.empty_like(t) for _ in range(world)] if rank == 0 else None
            dist.gather(t, gather_list=bufs, dst=0)
            if rank == 0:
                for r in range(world):
                    host = bufs[r].cpu().numpy()
                    for i, k in enumerate(per_rank[r]):
                        master.set_input(k, host[i])
                master.step(fid)
                out.append(master.get_commands()[1])
    finally:
        for s in shards.values():
            close = getattr(s, "close", None)
            if close:
                close()
        if master is not None and getattr(master, "close", None):
            master.close()
    return out
