"""The N > 1 path of the benchmark: independent replicas on two CPU ranks
(gloo).  Each rank draws its own particles, nothing but the timing crosses
ranks, and the job time is the slowest rank's."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2602_23434_b300 import replicas as R  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, lr = R.env()
    seed = R.rank_seed(1236, r)
    # each replica's local time differs; the job takes the slowest
    t = R.max_over_ranks(1.5 + r, dist)
    rate = R.job_rate(1000, 10, w, t)
    dist.barrier()
    q.put((r, w, lr, seed, t, rate))
    dist.destroy_process_group()


def test_two_rank_replicas():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 for o in out)
    assert out[0][3] == 1236 and out[1][3] != out[0][3]          # own particles per rank
    assert all(o[4] == 2.5 for o in out)                          # slowest rank's time
    assert all(abs(o[5] - 1000 * 10 * 2 / 2.5) < 1e-9 for o in out)


def test_single_rank_is_identity():
    assert R.max_over_ranks(3.25) == 3.25
    assert R.rank_seed(7, 0) == 7
