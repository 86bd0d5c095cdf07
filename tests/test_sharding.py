"""Host logic of the band-sharded solve on CPU (no GPU): the band assignment and the
all-reduce callback that the library calls on every operator output, across two gloo ranks
(world size 2, 127.0.0.1)."""
import ctypes
import os
import socket

import numpy as np

from paper_1710_00621_gb300 import sharding


def test_bands_of_one_grid_stay_together_and_load_is_balanced():
    # the multi-resolution bands: three per grid, costs ~ ring pairs x (L+1)^2
    keys = ["n256"] * 3 + ["n512"] * 3 + ["n1024"] * 3
    costs = [1.0] * 3 + [8.0] * 3 + [64.0] * 3
    for world in (1, 2, 3, 4):
        owned = sharding.assign_bands(keys, costs, world)
        assert sorted(nu for o in owned for nu in o) == list(range(9))      # each band once
        for o in owned:
            for key in set(keys[nu] for nu in o):
                assert all(nu in o for nu in range(9) if keys[nu] == key)   # groups intact
    owned = sharding.assign_bands(keys, costs, 2)
    loads = sorted(sum(costs[nu] for nu in o) for o in owned)
    assert loads == [3 * 1.0 + 3 * 8.0, 3 * 64.0]                           # largest group alone


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import datetime

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=20))
    try:
        v = np.arange(7, dtype=np.float64) * (rank + 1) + 0.5
        fn = sharding.make_allreduce(device=False)
        rc = fn(v.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), v.size, None, None)
        q.put((rank, rc, v.tolist()))
    except Exception as e:  # noqa: BLE001 - reported to the parent
        q.put((rank, -99, repr(e)))
    finally:
        dist.destroy_process_group()


def test_allreduce_callback_sums_the_vector_in_place_on_both_ranks():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = dict((r, (rc, v)) for r, rc, v in (q.get(timeout=120) for _ in range(2)))
    for p in ps:
        p.join(timeout=60)
        if p.is_alive():
            p.kill()
    want = (np.arange(7) * 3 + 1.0).tolist()
    assert out[0] == (0, want) and out[1] == (0, want)
