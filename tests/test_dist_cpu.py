"""The multi-process path of the throughput harness on CPU (gloo, world size 2):
replicas report their own units and times; the job's units are the sum and its
time the maximum over ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    from paper_2603_24370_gb300 import dist as D
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert D.env_rank() == (rank, rank, world)
        D.barrier()
        units, sec = D.aggregate(100.0 * (rank + 1), 0.5 + rank)
        out.put((rank, units, sec))
    finally:
        dist.destroy_process_group()


def test_replica_aggregation_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for _, units, sec in res:
        assert units == 300.0 and sec == 1.5


def test_single_process_aggregate_is_identity():
    from paper_2603_24370_gb300 import dist as D
    assert D.aggregate(7.0, 2.0) == (7.0, 2.0)


def test_each_rank_sees_its_own_gpu(monkeypatch):
    from paper_2603_24370_gb300 import dist as D
    monkeypatch.setenv("CUDA_VISIBLE_DEVICES", "4,5,6,7")
    D.pin_visible_device(2, 4)
    assert os.environ["CUDA_VISIBLE_DEVICES"] == "6"
    monkeypatch.delenv("CUDA_VISIBLE_DEVICES")
    D.pin_visible_device(1, 2)
    assert os.environ["CUDA_VISIBLE_DEVICES"] == "1"
    monkeypatch.setenv("CUDA_VISIBLE_DEVICES", "3")
    D.pin_visible_device(0, 1)  # one process: untouched
    assert os.environ["CUDA_VISIBLE_DEVICES"] == "3"
