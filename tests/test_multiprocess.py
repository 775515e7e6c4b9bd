"""The multi-GPU path is independent replicas: each rank processes its own
seeded measurements with no data-path collective, and the bench reports all
ranks' work over the slowest rank's time.  These CPU tests run that host
logic as two gloo ranks."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import synth
    r, w, loc = bench.dist_env()
    # each replica draws its own measurement (the bench's per-rank seeds)
    x = synth.single_sensor(n_samples=8192, n_dirs=4, seed_scene=1 + 1000 * r)["x"]
    t = 1.0 + 0.5 * rank  # per-rank elapsed seconds; rank 1 is the slowest
    t_max, t2_max = bench.max_over_ranks([t, 10.0 - rank])
    out.put((r, w, loc, t_max, t2_max, bench.replica_rate(20, w, t_max), int(np.abs(x).sum())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_replicas_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, l0, t0, u0, v0, x0), (r1, w1, l1, t1, u1, v1, x1) = res
    assert (r0, r1, w0, w1, l0, l1) == (0, 1, 2, 2, 0, 1)
    assert t0 == t1 == 1.5 and u0 == u1 == 10.0   # element-wise max over ranks
    assert v0 == v1 == pytest.approx(2 * 20 / 1.5)  # all ranks' units over the slowest time
    assert x0 != x1  # the replicas beamform different measurements


def test_single_process_is_unchanged():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([3.0, 4.0]) == [3.0, 4.0]
    assert bench.replica_rate(10, 1, 2.0) == 5.0
