"""Two ranks on the CPU (gloo): the packet sharding of the multi-GPU path and its one
exchange.  Each rank transports its share of every source's packet ids with the
oracle; after the all-reduce sum the tallies equal those of one run over all ids (to
the order of FP64 additions); step 2 split by camera and gathered gives the single
run's images; and the throughput reduction takes the slowest rank's time and all
events.  No GPU is used."""
import os

import numpy as np

from oracle import oracle as O
from paper_2512_01283_gb300 import multigpu as MG
from paper_2512_01283_gb300 import workloads as W


def _problem():
    model = W.disk(n=12)
    run = dict(W.disk_run(n_packets=1500, n_cam=2, npix=8), n_threads=1)
    return model, run


def _oracle_ranges(model, run, ranges):
    S = A = None
    events = 0.0
    for b, e in ranges:
        o = O.transport(model, dict(run, pid_begin=b, pid_end=e))
        S = o["S"] if S is None else S + o["S"]
        A = o["absorbed"] if A is None else A + o["absorbed"]
        events += o["stats"]["events"]
    return S, A, events


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    model, run = _problem()
    S, A, ev = _oracle_ranges(model, run, MG.rank_ranges(run, rank, world))
    S, A = torch.tensor(S, dtype=torch.float64), torch.tensor(A, dtype=torch.float64)
    MG.combine_tallies(S, A, dist)
    # step 2 split by camera, the images gathered
    n_cam, npix = len(run["cameras"]), run["cameras"][0]["npix"]
    imgs = torch.zeros((n_cam, 4, npix[1], npix[0]), dtype=torch.float64)
    for k in MG.rank_cameras(n_cam, rank, world):
        imgs[k] = torch.from_numpy(O.image(model, run, S.numpy(), k))
    MG.combine_images(imgs, dist)
    ms, ev_all = MG.reduce_timing(10.0 + rank, ev, dist)
    if rank == 0:
        q.put((S.numpy(), A.numpy(), ms, ev_all, imgs.numpy()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_sum_to_the_single_run():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29000 + os.getpid() % 2000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    S, A, ms, ev, imgs = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    model, run = _problem()
    o = O.transport(model, run)
    assert np.allclose(S, o["S"], rtol=1e-12, atol=1e-14 * np.abs(o["S"]).max())
    assert np.allclose(A, o["absorbed"], rtol=1e-12, atol=1e-14 * np.abs(o["absorbed"]).max())
    assert ms == 11.0
    assert ev == o["stats"]["events"]
    for k in range(len(run["cameras"])):
        ref = O.image(model, run, o["S"], k)
        assert np.allclose(imgs[k], ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())


def test_rank_cameras_cover_every_camera_once():
    for n_cam in (0, 1, 3, 8, 16):
        for world in (1, 2, 3, 4, 8):
            got = sorted(k for r in range(world) for k in MG.rank_cameras(n_cam, r, world))
            assert got == list(range(n_cam))
            assert max(len(MG.rank_cameras(n_cam, r, world)) for r in range(world)) <= -(-n_cam // world)


def test_rank_ranges_cover_every_source_once():
    run = {"sources": [{"n_packets": 10}, {"n_packets": 7}, {"n_packets": 0}, {"n_packets": 3}]}
    for world in (1, 2, 3, 4, 8):
        ids = []
        for r in range(world):
            rr = MG.rank_ranges(run, r, world)
            for b, e in rr:
                ids += list(range(b, e))
            # each rank gets its share of each source (within one packet)
            for lo, n in ((0, 10), (10, 7), (17, 3)):
                mine = sum(max(0, min(e, lo + n) - max(b, lo)) for b, e in rr)
                assert abs(mine - n / world) < 1.0
        assert sorted(ids) == list(range(20))
    assert MG.rank_ranges(run, 0, 1) == [(0, 20)]  # one rank: one launch


def test_rank_launch_accumulates_after_the_first_range():
    calls = []

    def fake(run, accumulate):
        calls.append((run["pid_begin"], run["pid_end"], accumulate))
        return {"events": run["pid_end"] - run["pid_begin"], "status": 0, "status_bits": 1 << len(calls)}

    run = {"sources": [{"n_packets": 100}, {"n_packets": 60}]}
    st = MG.rank_launch(fake, run, 1, 2)
    assert calls == [(50, 100, 0), (130, 160, 1)]
    assert st["events"] == 80 and st["status_bits"] == 6
    assert MG.scaled_run(run, 4)["sources"][1]["n_packets"] == 240
