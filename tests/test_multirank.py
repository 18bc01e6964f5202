"""The N > 1 host logic of bench.py on CPU ranks (gloo, world size 2): every
rank owns an independent list (distinct seeds, same shapes), the job time is
the slowest rank's, and the whole-job rate counts every rank's matrices."""
import importlib.util
import os
import socket

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    return b


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b = _bench()
    ms = [120.0, 150.0][rank]
    m = b.max_over_ranks_of(dist, ms, torch.device("cpu"))
    shapes = b.workload_list(b.WORKLOADS["muon_1b"])
    q.put((rank, m, b.rank_seed0(rank), len(shapes)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

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
    assert [o[1] for o in out] == [150.0, 150.0]        # max over ranks
    assert out[0][2] != out[1][2]                      # independent lists
    assert out[0][3] == out[1][3] == 168
    b = _bench()
    # 2 ranks x 168 matrices x 10 steps in 1.5 s of the slowest rank
    assert abs(b.whole_job_rate(2, 168, 10, 1500.0) - 2240.0) < 1e-9
