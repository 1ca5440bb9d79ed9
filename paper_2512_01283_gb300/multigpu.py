"""Packet sharding over ranks (one process per GPU) and the one exchange the path has.

Step 1 is a sum over independent packets (Sec. 2.2): ranks split the packet ids and
run them with the same Philox key, so the packets of all ranks together are exactly
the packets of a single run; no collective sits on the transport.  Each source's ids
are split into `world` consecutive shares, so every rank runs the same mix of sources.
A combined image needs one exchange: the FP64 source and absorbed tallies summed over
ranks, after which step 2 (linear in the tallies, Sec. 2.3) runs on the summed
tallies.  Summed tallies equal the single run's up to the order of the FP64 additions.
Step 2 is then split by camera (each camera's image depends only on the summed
tallies): rank r images cameras r, r + world, ..., and the images are gathered.

Throughput over ranks (weak scaling): events summed, time the maximum over ranks.
"""
from __future__ import annotations


def scaled_run(run: dict, world: int) -> dict:
    """The whole job of a weak-scaling run: every source with `world` times its packets
    (each rank then runs as many packets as `run` has)."""
    out = dict(run)
    out["sources"] = [dict(s, n_packets=int(s["n_packets"]) * int(world)) for s in run["sources"]]
    return out


def rank_ranges(run: dict, rank: int, world: int):
    """Packet-id ranges [begin, end) of `rank`: share `rank` of `world` consecutive
    shares of every source's ids (sources take consecutive ids); adjacent ranges are
    merged, so a single rank runs one range."""
    out = []
    start = 0
    for s in run["sources"]:
        n = int(s["n_packets"])
        b, e = start + n * rank // world, start + n * (rank + 1) // world
        if e > b:
            if out and out[-1][1] == b:
                out[-1] = (out[-1][0], e)
            else:
                out.append((b, e))
        start += n
    return out


def rank_launch(launch, run: dict, rank: int, world: int):
    """Run this rank's packets of `run` with `launch(run, accumulate)`: one launch per
    id range, the later ones adding to the tallies.  Returns the summed statistics of
    the additive fields."""
    total = {}
    for i, (b, e) in enumerate(rank_ranges(run, rank, world)):
        st = launch(dict(run, pid_begin=b, pid_end=e), 1 if i else 0)
        for k, v in st.items():
            if k == "status":  # MCRT_OK = 0, errors are negative
                total[k] = min(total.get(k, 0), v)
            elif k == "status_bits":
                total[k] = total.get(k, 0) | int(v)
            elif isinstance(v, (int, float)):
                total[k] = total.get(k, 0) + v
            else:
                total.setdefault(k, v)
    return total


def combine_tallies(source, absorbed, dist=None):
    """Sum the step-1 tallies over ranks in place (torch FP64 tensors; one all-reduce
    each).  Without a process group: unchanged."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return source, absorbed
    for t in (source, absorbed):
        if t is not None:
            dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return source, absorbed


def rank_cameras(n_cam: int, rank: int, world: int):
    """Cameras that `rank` images in step 2: rank, rank + world, ..."""
    return list(range(rank, n_cam, world))


def combine_images(images, dist=None):
    """Gather the images of all ranks in place (torch FP64 tensor [camera][4][ny][nx]
    holding this rank's cameras and zeros elsewhere; one sum all-reduce).  Without a
    process group: unchanged."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return images
    dist.all_reduce(images, op=dist.ReduceOp.SUM)
    return images


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
