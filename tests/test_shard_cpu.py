"""The multi-GPU batch protocol on the CPU: the LPT partition of a batch over
ranks (sqrtm_batch_partition, host code in the library) and the sharded run
(each rank solves its share, statuses gathered on the host) with two gloo
ranks and a stand-in solver -- no GPU and no data-path collective."""
import itertools
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp_

mp = pytest.importorskip("paper_2607_12430_gb300")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not os.path.exists(mp.LIB_PATH):
        pytest.skip("library not built")
    mp.lib()


def _makespan(sizes, owner, parts):
    load = [0.0] * parts
    for n, o in zip(sizes, owner):
        load[o] += float(n) ** 3
    return max(load), load


def test_partition_covers_each_matrix_once_and_reports_loads():
    g = np.random.default_rng(5)
    sizes = [int(x) for x in g.integers(16, 257, 300)]
    for parts in (1, 2, 3, 8):
        owner, load = mp.batch_partition(sizes, parts)
        assert len(owner) == len(sizes) and all(0 <= o < parts for o in owner)
        _, mine = _makespan(sizes, owner, parts)
        assert np.allclose(load, mine)
        assert sum(load) == pytest.approx(sum(float(n) ** 3 for n in sizes))


def test_partition_within_lpt_bound_of_brute_force_optimum():
    # LPT's makespan is at most (4/3 - 1/(3p)) times the optimum; the optimum
    # by enumerating every assignment of a few matrices
    g = np.random.default_rng(7)
    for trial in range(20):
        sizes = [int(x) for x in g.integers(1, 40, 7)]
        parts = 2 + trial % 2
        owner, _ = mp.batch_partition(sizes, parts)
        got, _ = _makespan(sizes, owner, parts)
        best = min(_makespan(sizes, a, parts)[0] for a in itertools.product(range(parts), repeat=len(sizes)))
        assert got <= (4.0 / 3.0 - 1.0 / (3 * parts)) * best + 1e-9


def test_partition_is_largest_first_to_least_loaded():
    # the rule itself on a case where the order matters: 10^3 goes first to
    # part 0, 9^3 to part 1, 8^3 to part 1 (the lighter), then 7^3 to part 0
    owner, load = mp.batch_partition([7, 10, 8, 9], 2)
    assert owner == [0, 0, 1, 1]
    assert load == [7.0 ** 3 + 10.0 ** 3, 8.0 ** 3 + 9.0 ** 3]


def test_partition_arguments():
    with pytest.raises(mp.SqrtmError) as e:
        mp.batch_partition([4, 5], 0)
    assert e.value.code == -3
    with pytest.raises(mp.SqrtmError) as e:
        mp.batch_partition([4, -1], 2)
    assert e.value.code == -2
    owner, load = mp.batch_partition([], 3)
    assert owner == [] and load == [0.0, 0.0, 0.0]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _fake_status(i):
    return (7 * i) % 5


def _worker(rank, world, port, sizes, out):
    import paper_2607_12430_gb300 as m
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        def gather(obj):
            res = [None] * world
            dist.all_gather_object(res, obj)
            return res
        mine, full = m.sharded_run(sizes, rank, world, lambda idx: [_fake_status(i) for i in idx], gather)
        out[rank] = (mine, full)
    finally:
        dist.destroy_process_group()


def test_two_rank_sharded_run_gathers_every_status_in_order():
    sizes = [17, 256, 64, 200, 31, 128, 250, 16, 99, 180]
    ctx = mp_.get_context("spawn")
    with ctx.Manager() as man:
        out = man.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, sizes, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    owner, _ = mp.batch_partition(sizes, 2)
    expect = [_fake_status(i) for i in range(len(sizes))]
    for r in range(2):
        mine, full = res[r]
        assert mine == [i for i, o in enumerate(owner) if o == r]
        assert full == expect
    assert sorted(res[0][0] + res[1][0]) == list(range(len(sizes)))
