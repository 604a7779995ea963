"""A velocity-sharded GSIS solve across two processes on one GPU: each process owns half of
the velocity blocks and exchanges its partial sums through sharding.dist_allreduce, a
torch.distributed all-reduce (gloo) of CUDA tensors viewing the library's buffers, enqueued on
the library's stream.  Each process takes half of the SMs for its synthetic solve.  The shards'
states must be identical to each other and within 1e-11 of the unsharded solve."""
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
OPTS = dict(macro_steps=60, macro_tol=0.0, kinetic_presteps=2)
STEPS = 3


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    try:
        import torch
        import torch.distributed as dist

        from paper_2310_18916_gb300 import gsis, sharding
        from paper_2310_18916_gb300 import workloads as wl

        os.environ["MASTER_ADDR"] = "127.0.0.1"
        os.environ["MASTER_PORT"] = str(port)
        torch.cuda.set_device(0)
        dist.init_process_group("gloo", rank=rank, world_size=world)
        nsm = torch.cuda.get_device_properties(0).multi_processor_count
        p = wl.cavity(n=10, nv=12, Kn=0.1, lid=0.2)
        s = gsis.Solver(p, precision="f64", mode="gsis", shard=(rank, world), allreduce=sharding.dist_allreduce(),
                        macro_sms=nsm // world, **OPTS)
        hist = []
        for _ in range(STEPS):
            s.step()
            hist.append(s.W())
        s.close()
        dist.barrier()
        dist.destroy_process_group()
        q.put((rank, hist, None))
    except Exception as e:  # noqa: BLE001 - reported to the parent
        q.put((rank, None, repr(e)))


def test_two_process_velocity_shards_match_the_unsharded_solve():
    from gpu_common import scaled_close
    from paper_2310_18916_gb300 import gsis
    from paper_2310_18916_gb300 import workloads as wl

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    out = {}
    for _ in procs:
        r, hist, err = q.get(timeout=300)
        assert err is None, f"rank {r}: {err}"
        out[r] = hist
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    p = wl.cavity(n=10, nv=12, Kn=0.1, lid=0.2)
    ref = gsis.Solver(p, precision="f64", mode="gsis", **OPTS)
    for it in range(STEPS):
        ref.step()
        np.testing.assert_array_equal(out[1][it], out[0][it])
        scaled_close(out[0][it], ref.W(), 1e-11, f"two processes, step {it}")
    ref.close()
