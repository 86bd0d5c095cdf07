"""Band sharding of the solve over several GPUs (one process and one model per GPU).

A is a sum over bands plus the prior (Eq. A) and M_PI a sum over the rows of U (Sec. 3.3),
so each rank owns a subset of the bands (cmbws_model_set_shard) and every apply of A and of
M_PI in PCG is the rank's partial terms plus one all-reduce of the stacked vector
(cmbws_cg_solve_sharded).  This module assigns bands to ranks and provides the all-reduce
callback over torch.distributed; all arithmetic runs in libcmbws.
"""
import ctypes

import numpy as np

from . import binding as B

ALLREDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_int64,
                                ctypes.c_void_p, ctypes.c_void_p)


def assign_bands(grid_keys, costs, world):
    """Owned-band lists, one per rank: bands that share a grid stay together (they are
    transformed in one launch), groups are placed largest first on the least-loaded rank.
    grid_keys[nu]: hashable grid identity of band nu; costs[nu]: relative SHT cost (e.g.
    ring pairs x (L+1)^2).  Ranks left without a group own no band."""
    groups = {}
    for nu, key in enumerate(grid_keys):
        groups.setdefault(key, []).append(nu)
    order = sorted(groups.values(), key=lambda g: -sum(costs[nu] for nu in g))
    load = [0.0] * world
    owned = [[] for _ in range(world)]
    for g in order:
        r = int(np.argmin(load))
        owned[r].extend(g)
        load[r] += sum(costs[nu] for nu in g)
    return [sorted(o) for o in owned]


class _DeviceView:
    """__cuda_array_interface__ of a device vector of n doubles (no copy)."""

    def __init__(self, ptr, n):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": "<f8",
                                         "data": (int(ptr), False), "version": 3, "strides": None}


def make_allreduce(group=None, device=True):
    """The ctypes all-reduce callback of cmbws_cg_solve_sharded: sums the vector over the ranks
    of `group` with torch.distributed on torch's current stream (the stream the binding hands
    the library).  With the gloo backend a device vector goes through a host copy.
    device=False treats the pointer as host memory (for host-side use of the callback).
    Keep the returned object alive for the duration of the solve."""
    import torch
    import torch.distributed as dist

    def cb(v, n, stream, ctx):
        try:
            addr = ctypes.cast(v, ctypes.c_void_p).value
            if device:
                t = torch.as_tensor(_DeviceView(addr, n), device="cuda")
            else:
                t = torch.from_numpy(np.ctypeslib.as_array(v, (int(n),)))
            if t.is_cuda and dist.get_backend(group) == "gloo":
                h = t.cpu()
                dist.all_reduce(h, group=group)
                t.copy_(h)
            else:
                dist.all_reduce(t, group=group)
            return 0
        except Exception:  # noqa: BLE001 - reported to the library as CMBWS_ERR_COMM
            return -1

    return ALLREDUCE_FN(cb)


def set_shard(model, owned, nobs, prior):
    """cmbws_model_set_shard with the list of owned band indices (None: no shard)."""
    B.cmbws_model_set_shard(model, None if owned is None else
                            [1 if nu in set(owned) else 0 for nu in range(nobs)], prior)


def cg_solve_sharded(model, b, x, group=None, **kw):
    """cmbws_cg_solve_sharded with the torch.distributed all-reduce of `group`."""
    fn = make_allreduce(group)
    return B.cmbws_cg_solve_sharded(model, b, x, fn, **kw)
