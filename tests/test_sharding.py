"""Velocity sharding on the CPU: the block split (through the footprint of each shard, which
needs no GPU), the option checks, and the torch.distributed all-reduce adapter over two gloo
ranks."""
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest

from paper_2310_18916_gb300 import gsis
from paper_2310_18916_gb300 import workloads as wl


def _f_bytes(p, shard=None):
    """VDF bytes of a (shard of a) solve: footprint with the VDF minus the footprint without it."""
    return gsis.footprint_bytes(p, "f32", shard)


@pytest.mark.parametrize("k", [2, 3, 5])
def test_shards_split_the_velocity_blocks(k):
    p = wl.cavity(n=16, nv=20, Kn=0.1)
    whole = _f_bytes(p)
    parts = [_f_bytes(p, (i, k)) for i in range(k)]
    # every shard keeps the per-cell data (c); the velocity-proportional part (v: the VDF, its
    # per-block partials and slot tables) is split: whole = c + v, sum(parts) = k c + v
    vdf_whole = (k * whole - sum(parts)) / (k - 1)
    per_cell = whole - vdf_whole
    vdf_parts = [q - per_cell for q in parts]
    assert vdf_whole > 0.9 * 4 * p.ncells * p.nvel  # the FP32 VDF dominates it
    assert sum(vdf_parts) == pytest.approx(vdf_whole, rel=1e-9)
    assert max(vdf_parts) - min(vdf_parts) <= 2 * vdf_whole / 8 / k + 1  # contiguous, near-even ranges


def test_shard_options_are_checked():
    p = wl.cavity(n=8, nv=8, Kn=0.1)
    with pytest.raises(gsis.GsisError):
        gsis.footprint_bytes(p, "f32", (2, 2))       # index out of range
    with pytest.raises(gsis.GsisError):
        gsis.footprint_bytes(p, "f32", (0, 1000))    # more shards than velocity blocks


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2310_18916_gb300 import sharding

    cb = sharding.dist_allreduce(on_host=True)
    a = np.arange(9, dtype=np.float64) * (rank + 1) + 0.25
    cb(a.ctypes.data, a.size, 0)
    q.put((rank, a.tolist()))
    dist.destroy_process_group()


def test_dist_allreduce_adapter_over_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    out = dict(q.get(timeout=120) for _ in procs)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    want = np.arange(9) * 3 + 0.5
    for r in (0, 1):
        np.testing.assert_array_equal(out[r], want)
