"""The multi-process side of bench.py on CPU (gloo, world size 2): the run is
replicas only (independent sensors per rank, no data-path collective), so
the host logic to cover is the rendezvous, the barrier around the timed
region, the MAX over ranks of the step time, and the reference arm, which
only rank 0 runs while the other ranks leave without work."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import argparse
    import torch.distributed as dist
    import bench
    r, local, w = bench.dist_init()
    assert (r, local, w) == (rank, rank, world) and dist.get_backend() == "gloo"
    bench.barrier(w)
    mx = bench.max_over_ranks(1.5 + rank, w)           # a per-rank step time
    out = {"rank": r, "max": mx}
    if rank == 1:
        # the reference arm: ranks other than 0 return at once, without the oracle
        args = argparse.Namespace(workload="c2", steps=1, warmup=0, gpus=world)
        out["ref_rc"] = bench.run_reference(args)
        out["oracle_imported"] = "oracle" in sys.modules
    bench.barrier(w)
    dist.destroy_process_group()
    q.put(out)


def test_two_ranks_on_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    res = sorted((q.get(timeout=10) for _ in procs), key=lambda d: d["rank"])
    assert [d["max"] for d in res] == [2.5, 2.5]
    assert res[1]["ref_rc"] == 0 and not res[1]["oracle_imported"]
