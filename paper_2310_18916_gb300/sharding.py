"""Velocity sharding of one GSIS solve (the velocity decomposition of Section 4, Algorithm 3):
each shard holds a contiguous range of the velocity blocks for all cells, and per outer step the
library sum-all-reduces three partial sums through a callback: the wall re-emission densities,
the per-cell moments and kinetic flux sums, and the wall fluxes.  The synthetic solve and
everything after the exchanges are repeated identically on every shard.

Two callbacks:
  dist_allreduce(group): torch.distributed.all_reduce (NCCL across GPUs, or gloo) on a
      zero-copy view of the library's buffer, enqueued on the library's stream;
  LocalExchange(k): K logical shards of one solve in one process (one thread per shard, e.g. on
      one GPU), summed in fixed shard order, so the result does not depend on thread timing.
"""
from __future__ import annotations

import threading

import numpy as np


class _DeviceArray:
    """A raw FP64 device buffer exposed through the CUDA array interface (zero copy)."""

    def __init__(self, ptr, count):
        self.__cuda_array_interface__ = {"shape": (int(count),), "typestr": "<f8", "data": (int(ptr), False),
                                         "version": 3, "strides": None}


def device_view(ptr, count):
    """torch tensor viewing count FP64 values at device pointer ptr."""
    import torch

    return torch.as_tensor(_DeviceArray(ptr, count), device="cuda")


def host_view(ptr, count):
    """torch tensor viewing count FP64 values at host pointer ptr."""
    import ctypes

    import torch

    buf = (ctypes.c_double * int(count)).from_address(int(ptr))
    return torch.from_numpy(np.frombuffer(buf, dtype=np.float64))


def dist_allreduce(group=None, on_host=False):
    """Callback for Solver(..., shard=(rank, world), allreduce=...) across torch.distributed
    ranks.  on_host: the pointers are host memory (CPU ranks over gloo)."""
    import torch
    import torch.distributed as dist

    def cb(ptr, count, stream):
        if on_host:
            dist.all_reduce(host_view(ptr, count), op=dist.ReduceOp.SUM, group=group)
            return
        s = torch.cuda.ExternalStream(stream) if stream else torch.cuda.current_stream()
        with torch.cuda.stream(s):
            dist.all_reduce(device_view(ptr, count), op=dist.ReduceOp.SUM, group=group)

    return cb


class LocalExchange:
    """In-process sum-all-reduce for K shards driven by K threads: every shard's call copies its
    partial into a slot, waits for the others, and replaces its buffer by the slots' sum in
    shard order 0..K-1 (deterministic)."""

    def __init__(self, k, timeout=60.0):
        self.k = k
        self.barrier = threading.Barrier(k, timeout=timeout)
        self.slots = [None] * k

    def callback(self, shard):
        import torch

        def cb(ptr, count, stream):
            s = torch.cuda.ExternalStream(stream) if stream else torch.cuda.current_stream()
            view = device_view(ptr, count)
            with torch.cuda.stream(s):
                self.slots[shard] = view.clone()
            s.synchronize()
            self.barrier.wait()
            with torch.cuda.stream(s):
                tot = self.slots[0].clone()
                for j in range(1, self.k):
                    tot += self.slots[j]
                view.copy_(tot)
            s.synchronize()
            self.barrier.wait()  # nobody reuses the slots before everyone has summed

        return cb


def run_local_shards(problem, k, steps, precision="f64", **opts):
    """Solve problem with k logical velocity shards in one process (one thread and CUDA stream
    per shard) for the given outer steps; returns every shard's W after each step."""
    import torch

    from . import gsis

    ex = LocalExchange(k)
    streams = [torch.cuda.Stream() for _ in range(k)]
    # the shards' synthetic solves (cooperative kernels holding whole SMs) run at the same time
    nsm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    opts.setdefault("macro_sms", max(1, nsm // k))
    solvers, hist, errors = [None] * k, [[] for _ in range(k)], []

    def work(i):
        try:
            with torch.cuda.stream(streams[i]):
                solvers[i] = gsis.Solver(problem, precision=precision, shard=(i, k), allreduce=ex.callback(i), **opts)
                for _ in range(steps):
                    solvers[i].step()
                    hist[i].append(solvers[i].W())
        except Exception as e:  # noqa: BLE001 - re-raised in the caller
            errors.append(e)
            ex.barrier.abort()

    threads = [threading.Thread(target=work, args=(i,)) for i in range(k)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    for s in solvers:
        if s is not None:
            s.close()
    if errors:
        raise errors[0]
    return hist
