"""Multi-GPU replicas (weak scaling) without a GPU: two gloo ranks on CPU
check that each rank steps its own realizations (different seeds, same grid
shapes) and that the job time is the maximum over ranks."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        out = {}
        for name in ("planewave", "batch"):
            specs = bench.workload_specs(name, rank, 10)
            out[name] = ([s.seed for s in specs], [tuple(s.shape) for s in specs])
        t = bench.rank_max(0.5 + rank, dist, device="cpu")
        q.put((rank, out, t))
    finally:
        dist.destroy_process_group()


def test_two_replicas_step_distinct_realizations_and_report_the_slowest():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in procs:
        rank, out, t = q.get(timeout=180)
        res[rank] = (out, t)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for name in ("planewave", "batch"):
        seeds0, shapes0 = res[0][0][name]
        seeds1, shapes1 = res[1][0][name]
        assert not set(seeds0) & set(seeds1)      # different realizations per rank
        if name == "planewave":
            assert shapes0 == shapes1               # same per-rank work (weak scaling)
    assert res[0][1] == res[1][1] == 1.5          # max over ranks
