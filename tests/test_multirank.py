"""Two ranks on the CPU (gloo): the packet sharding of the multi-GPU path and its one
exchange.  Each rank transports its own Philox stream with the oracle; the combined
tallies (all-reduce average) must equal the average of the two streams run in one
process, and the throughput reduction takes the slowest rank's time and all events.
No GPU is used."""
import os

import numpy as np

from oracle import oracle as O
from paper_2512_01283_gb300 import multigpu as MG
from paper_2512_01283_gb300 import workloads as W


def _problem():
    model = W.rayleigh_sphere(n=8)
    run = dict(W.rayleigh_sphere_run(n_packets=3000, npix=8), n_threads=1)
    return model, run


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    model, run = _problem()
    o = O.transport(model, MG.rank_run(run, rank))
    S = torch.tensor(o["S"], dtype=torch.float64)
    A = torch.tensor(o["absorbed"], dtype=torch.float64)
    MG.combine_tallies(S, A, dist)
    ms, ev = MG.reduce_timing(10.0 + rank, o["stats"]["events"], dist)
    if rank == 0:
        q.put((S.numpy(), A.numpy(), ms, ev))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_average_their_streams():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29000 + os.getpid() % 2000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    S, A, ms, ev = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    model, run = _problem()
    o0 = O.transport(model, MG.rank_run(run, 0))
    o1 = O.transport(model, MG.rank_run(run, 1))
    assert np.allclose(S, 0.5 * (o0["S"] + o1["S"]), rtol=1e-12, atol=1e-15 * np.abs(o0["S"]).max())
    assert np.allclose(A, 0.5 * (o0["absorbed"] + o1["absorbed"]), rtol=1e-12, atol=1e-15)
    assert ms == 11.0
    assert ev == o0["stats"]["events"] + o1["stats"]["events"]
    # the streams are different packets: the two runs differ
    assert not np.allclose(o0["S"], o1["S"])
