"""Packet sharding over ranks (one process per GPU) and the one exchange the path has.

Step 1 is a sum over independent packets (Sec. 2.2), so ranks split the work by
packets with no collective on the data path: rank r runs its packets with Philox
stream ``base_stream + r`` (the counter-based generator makes every rank's packets
independent and reproducible).  Each rank's tallies are an estimate of the whole
model's tallies (every rank emits the full luminosity with its own packets), so a
combined image needs one exchange: the FP64 source and absorbed tallies averaged
over ranks, after which step 2 (linear in S) runs on any rank.

Throughput over ranks (weak scaling): events summed, time the maximum over ranks.
"""
from __future__ import annotations


def rank_run(run: dict, rank: int) -> dict:
    """The launch description of `rank`: its own Philox stream."""
    out = dict(run)
    out["stream"] = int(run.get("stream", 0)) + int(rank)
    return out


def combine_tallies(source, absorbed, dist=None):
    """Average the step-1 tallies over ranks in place (torch FP64 tensors; an
    all-reduce sum divided by the world size).  Without a process group: unchanged."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return source, absorbed
    w = float(dist.get_world_size())
    for t in (source, absorbed):
        if t is not None:
            dist.all_reduce(t, op=dist.ReduceOp.SUM)
            t.div_(w)
    return source, absorbed


def reduce_timing(ms: float, events: float, dist=None, device="cpu"):
    """(max over ranks of the timed milliseconds, sum over ranks of the events)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(ms), float(events)
    import torch

    t = torch.tensor([ms], dtype=torch.float64, device=device)
    e = torch.tensor([events], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(e, op=dist.ReduceOp.SUM)
    return float(t.item()), float(e.item())
