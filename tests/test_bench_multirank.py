"""Multi-rank host logic of bench.py on CPU: two gloo ranks (world size 2, 127.0.0.1).

The replicas path has no data-path collective; what crosses ranks is the barrier around the
timed region and the maximum of the per-rank step time.  Each rank here reports a different
time and both must see the maximum; a rank that raises must not hang the other (its
barrier ends with the process-group timeout)."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q, fail_rank):
    import datetime

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=20))
    import bench
    try:
        bench.barrier(world)
        if rank == fail_rank:
            raise RuntimeError("rank failed between steps")
        v = bench.max_over_ranks(0.25 + rank, world)
        bench.barrier(world)
        q.put((rank, "ok", v))
    except Exception as e:  # noqa: BLE001 - reported to the parent
        q.put((rank, "err", type(e).__name__))
    finally:
        dist.destroy_process_group()


def _run(world, fail_rank=-1, timeout=120):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, world, port, q, fail_rank)) for r in range(world)]
    for p in ps:
        p.start()
    out = {}
    for _ in range(world):
        r, status, v = q.get(timeout=timeout)
        out[r] = (status, v)
    for p in ps:
        p.join(timeout=timeout)
        if p.is_alive():
            p.kill()
    return out


def test_max_over_ranks_two_gloo_ranks():
    out = _run(2)
    assert out[0] == ("ok", 1.25) and out[1] == ("ok", 1.25)


def test_failed_rank_does_not_hang_the_other():
    out = _run(2, fail_rank=1)
    assert out[1] == ("err", "RuntimeError")
    assert out[0][0] == "err"  # its collective ended with an error instead of hanging
