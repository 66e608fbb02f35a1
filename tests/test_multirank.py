"""The N>1 host logic of bench.py on CPU: two gloo ranks, each with its own slide (weak scaling).
The whole-job duration is the slowest rank's and the whole-job pair count is the sum over ranks;
ranks draw different seeded workloads."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist          # noqa: E402
import torch.multiprocessing as mp        # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_1208_0277_gb300 import workload as W
    w = W.single_tile(seed=1 + rank, n=200)          # the seed bench.py gives rank `rank`
    import numpy as np
    import oracle as O
    pa, _ = O.candidate_pairs(O.polygon_areas(w.A.off, w.A.xy)[1], w.A.tile,
                              O.polygon_areas(w.B.off, w.B.xy)[1], w.B.tile)
    ms = 10.0 + 5.0 * rank
    out = bench.whole_job(ms, len(pa), dist, torch.device("cpu"))
    q.put((rank, len(pa), int(np.asarray(w.A.xy).sum()), out))
    dist.barrier()
    dist.destroy_process_group()


def test_weak_scaling_aggregation_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    pairs = [r[1] for r in res]
    assert res[0][2] != res[1][2]                      # different slides per rank
    for r in res:
        assert r[3] == (15.0, sum(pairs))              # slowest rank, all ranks' pairs


def test_whole_job_without_distributed():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.whole_job(3.5, 7, None, None) == (3.5, 7)
