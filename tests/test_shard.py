"""Sharing one list out over ranks (paper_2602_02500_gb300/shard.py): the LPT
partition and the exchange of results, on CPU ranks (gloo, world size 2).
The per-rank compute is stood in for by the FP64 oracle on small matrices;
the library call it replaces is covered by the GPU parity tests."""
import os
import socket

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _shard():
    import importlib.util

    spec = importlib.util.spec_from_file_location(
        "shard", os.path.join(ROOT, "paper_2602_02500_gb300", "shard.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _bench():
    import importlib.util

    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    return b


def test_cost_is_algorithm1_flops():
    S = _shard()
    b = _bench()
    for r, c in [(2048, 2048), (2048, 5632), (5632, 2048), (128, 1024)]:
        h, w = min(r, c), max(r, c)
        assert S.ifnso_cost(r, c, 14) == b.flops_ifnso(h, w, 14) == 4 * h * h * w + 26 * h ** 3


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_lpt_partition_1b_list(world):
    S = _shard()
    b = _bench()
    shapes = b.workload_list(b.WORKLOADS["muon_1b"])
    costs = [S.ifnso_cost(r, c, 14) for _, r, c in shapes]
    parts = S.lpt_partition(costs, world)
    assert len(parts) == world
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(len(shapes)))  # every matrix exactly once
    assert all(p == sorted(p) for p in parts)
    loads = [sum(costs[i] for i in p) for p in parts]
    # list scheduling: no rank exceeds the mean load by more than one matrix
    assert max(loads) <= sum(loads) / world + max(costs)
    assert S.owner_table(parts)[parts[-1][0]] == world - 1
    assert S.lpt_partition(costs, world) == parts  # deterministic


def test_lpt_partition_small():
    S = _shard()
    # costs 7, 5, 4, 3, 3 on 2 ranks: 7 -> r0, 5 -> r1, 4 -> r1 (5 < 7),
    # 3 -> r0 (7 < 9), 3 -> r1 (9 < 10): loads 10 and 12
    parts = S.lpt_partition([7, 5, 4, 3, 3], 2)
    assert parts == [[0, 3], [1, 2, 4]]
    with pytest.raises(ValueError):
        S.lpt_partition([1], 0)


def test_pack_layout():
    S = _shard()
    # shares [0, 3] and [1, 2, 4] of matrices with 6, 4, 10, 2, 3 elements
    seg, offs = S.pack_layout([[0, 3], [1, 2, 4]], [6, 4, 10, 2, 3])
    assert seg == 17   # rank 1 packs 4 + 10 + 3
    assert offs == {0: (0, 0), 3: (0, 6), 1: (1, 0), 2: (1, 4), 4: (1, 14)}
    with pytest.raises(ValueError):
        S.pack_layout([[0], [2]], [1, 1, 1])


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _mats():
    """Mixed shapes, wide and tall, of different element counts (the shares'
    packed buffers differ in length)."""
    import synth

    return [synth.gaussian(40 + i, r, c)
            for i, (r, c) in enumerate([(16, 32), (32, 16), (24, 24), (8, 40), (20, 30), (36, 12), (9, 9)])]


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist

    from oracle import ifnso as O

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    S = _shard()
    mats = _mats()
    w = np.array([0.5, 0.4, 0.9, 1.0])
    parts = S.lpt_partition([S.ifnso_cost(*M.shape, 4) for M in mats], world)
    outs = [torch.zeros(M.shape, dtype=torch.float64) for M in mats]
    done = []

    def run_local(idx):
        for i in idx:
            outs[i].copy_(torch.from_numpy(O.ifnso_alg1(mats[i], w)))
            done.append(i)

    S.sharded_orthogonalize(run_local, outs, parts, rank, dist)
    ok = all(np.array_equal(outs[i].numpy(), O.ifnso_alg1(mats[i], w)) for i in range(len(mats)))
    q.put((rank, ok, sorted(done), parts[rank]))
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_exchange_two_gloo_ranks():
    pytest.importorskip("torch")
    import sys

    import torch.multiprocessing as mp

    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ok, done, mine in out:
        assert ok                      # every rank ends with every result
        assert done == sorted(mine)    # and computed only its own share
    assert sorted(out[0][2] + out[1][2]) == list(range(7))
