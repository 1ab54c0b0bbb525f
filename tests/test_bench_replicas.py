"""The host side of bench.py's replica mode (one independent square root per
rank under torchrun): rank 0's k* reaches every rank and the reported time
is the slowest rank's.  Two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp_


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        kstar = bench.share_kstar(dist, 2 if rank == 0 else None, torch.device("cpu"))
        ms = bench.slowest_rank_ms(dist, [3.25, 5.5][rank], torch.device("cpu"))
        out[rank] = (kstar, ms)
    finally:
        dist.destroy_process_group()


def test_replicas_share_kstar_and_report_slowest_rank():
    ctx = mp_.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        assert dict(out) == {0: (2, 5.5), 1: (2, 5.5)}


def test_chase_traffic_only_for_the_source_it_was_measured_on(monkeypatch):
    # the stored DRAM traffic of the chase kernel is reported for the qr.cu
    # it was captured with and dropped (null) as soon as the chase's source
    # differs by a byte
    import builtins

    import bench
    assert bench._chase_traffic() == bench.CHASE_TRAFFIC["bytes"]
    real_open = builtins.open

    class _Edited:
        def __init__(self, f):
            self._f = f

        def read(self):
            return self._f.read().replace("chase", "chasE", 1)

        def __enter__(self):
            return self

        def __exit__(self, *a):
            self._f.close()

    def fake_open(path, *a, **k):
        f = real_open(path, *a, **k)
        return _Edited(f) if str(path).endswith("qr.cu") else f

    monkeypatch.setattr(builtins, "open", fake_open)
    assert bench._chase_traffic() is None
