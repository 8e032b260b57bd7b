"""The multi-rank path of bench.py on the CPU: two processes joined by a gloo
process group (the GPU runs use NCCL with the same calls).  Independent bond
updates shard with no data-path exchange: each rank draws its own batch, the
step time of the job is the slowest rank's, and the whole-job rate counts
every rank's items."""
import os
import queue
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank: int, world: int, port: int, out) -> None:
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist

    import bench
    from paper_2107_06635_gb300 import inputs as I

    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = [12.5, 20.0][rank]                    # rank 1 is the slower one
    ms = bench.reduce_max(local_ms, dist, "cpu")
    rate = bench.job_rate(world, 456, ms)
    Ta, _, _ = I.batch_items(bench.rank_seed(rank), 2, 2, 3, I.zz_gate(0.01))
    dist.barrier()
    out.put((rank, ms, rate, bench.rank_seed(rank), float(np.abs(Ta).sum())))
    dist.destroy_process_group()


def test_two_gloo_ranks_share_the_slowest_time_and_draw_disjoint_batches():
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = []
    try:
        for _ in procs:
            res.append(out.get(timeout=120))
    except queue.Empty:
        pytest.fail("a rank did not report within 120 s")
    finally:
        for p in procs:
            p.join(timeout=30)
            if p.is_alive():
                p.kill()
    res.sort()
    assert [r[0] for r in res] == [0, 1]
    for _, ms, rate, _, _ in res:
        assert ms == 20.0                                 # max over ranks
        assert rate == pytest.approx(2 * 456 / 0.020)     # whole-job bond updates/s
    assert res[0][3] != res[1][3] and res[0][4] != res[1][4]
    assert all(p.exitcode == 0 for p in procs)


def test_single_process_reduce_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(3.5) == 3.5
    assert bench.job_rate(1, 100, 50.0) == pytest.approx(2000.0)
    assert bench.rank_seed(0) == 5
