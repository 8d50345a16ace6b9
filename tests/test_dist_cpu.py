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


def _fake_solve(p, i):
    """Host-side stand-in for one relaxation: a deterministic record of the problem."""
    n = len(p.solitons)
    return {"index": i, "converged": (p.nx + n) % 3 != 0, "steps": 10 * p.nx + n, "arrests": n,
            "energy": 3.141592653589793 * n * p.params[0], "grad_max": 1e-7 * (1 + i % 5),
            "charge": float(n), "flux": 6.283185307179586 * n}


def _shard_worker(rank, world, port, out):
    import torch.distributed as dist
    from paper_2603_24370_gb300 import dist as D
    from paper_2603_24370_gb300 import inputs as I
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        probs = I.ah_batch(37, 20262)
        parts = D.shard([p.interior_sites for p in probs], world)
        mine = [_fake_solve(probs[i], i) for i in parts[rank]]
        full = D.gather_records(mine, len(probs))
        out.put((rank, parts, full))
    finally:
        dist.destroy_process_group()


def test_batch_shard_and_gather_over_two_gloo_ranks():
    """The work list splits into disjoint, covering, cost-balanced shares; each rank
    relaxes its share (a host stand-in here) and every rank ends with all records in
    problem order, each equal to the single-process result."""
    import torch.multiprocessing as mp
    from paper_2603_24370_gb300 import inputs as I
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    probs = I.ah_batch(37, 20262)
    expect = [_fake_solve(p, i) for i, p in enumerate(probs)]
    parts = res[0][1]
    assert res[1][1] == parts  # both ranks compute the same partition
    assert sorted(parts[0] + parts[1]) == list(range(len(probs)))
    cost = [p.interior_sites for p in probs]
    loads = [sum(cost[i] for i in part) for part in parts]
    assert abs(loads[0] - loads[1]) <= max(cost)
    for rank, _, full in res:
        assert [r["index"] for r in full] == list(range(len(probs)))
        for r, e in zip(full, expect):
            assert {k: r[k] for k in e} == e
            assert r["rank"] == (0 if r["index"] in parts[0] else 1)


def test_shard_partition_rules():
    from paper_2603_24370_gb300 import dist as D
    assert D.shard([5, 1, 4, 2, 3], 1) == [[0, 1, 2, 3, 4]]
    parts = D.shard([8, 1, 1, 1, 1, 1, 1, 1, 1], 2)
    assert parts == [[0], [1, 2, 3, 4, 5, 6, 7, 8]]
    assert D.shard([], 3) == [[], [], []]
    assert sorted(sum(D.shard(list(range(1, 50)), 4), [])) == list(range(49))
