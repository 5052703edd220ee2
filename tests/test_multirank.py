"""The multi-rank path of bench.py on the CPU: two gloo ranks, as torchrun
launches them (one process per GPU on a GPU node).  The coded batches are
independent per rank (no data-path collective); the only exchange is the
max-over-ranks reduction of the timings, and the reference arm runs on
rank 0 alone."""
import contextlib
import io
import os
import socket

import pytest
import torch.multiprocessing as mp


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def rank_main(rank, world, port, results):
    import torch
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # per-rank timings: decode ms, encode ms, step ms, wall s
        mine = [1.0 + rank, 5.0 - rank, 2.5, 0.1 * (rank + 1)]
        dist.barrier()
        got = bench.max_over_ranks(mine, torch.device("cpu"), world)
        seeds = [None] * world
        dist.all_gather_object(seeds, bench.rank_seed("chunked", rank))
        out = io.StringIO()
        args = bench.parse_args(["--impl", "reference", "--steps", "1", "--warmup", "0"])
        rc = None
        if rank != 0:   # rank 0 would time the oracle: not needed to check the split
            with contextlib.redirect_stdout(out):
                rc = bench.reference_arm(args)
        results[rank] = dict(got=got, seeds=seeds, rc=rc, out=out.getvalue(),
                             value=bench.job_value(world, 1 << 30, got[0]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_timings_and_shard_batches():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        results = mgr.dict()
        mp.start_processes(rank_main, args=(2, free_port(), results), nprocs=2, join=True,
                           start_method="spawn")
        res = dict(results)
    assert set(res) == {0, 1}
    for r in (0, 1):
        assert res[r]["got"] == pytest.approx([2.0, 5.0, 2.5, 0.2])
    seeds = res[0]["seeds"]
    assert seeds == res[1]["seeds"] and len(set(seeds)) == 2   # independent batches
    assert res[1]["rc"] == 0 and res[1]["out"] == ""           # only rank 0 prints
    # whole-job value: both ranks' symbols over the slowest rank's decode time
    assert res[0]["value"] == pytest.approx(2 * (1 << 30) / 2.0e-3 / 1e9)
