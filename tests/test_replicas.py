"""Multi-GPU host logic on CPU: two gloo ranks (no GPU). Frames are disjoint across ranks and the
timed region's duration is the max over ranks."""
import os

import pytest

from paper_2504_05562_gb300 import replicas


def test_frames_disjoint_and_in_range():
    world, steps = 4, 300
    seen = set()
    for r in range(world):
        f = replicas.frames_for_rank(r, world, steps)
        assert len(f) == steps and all(0 <= x < 65536 for x in f)
        assert not (seen & set(f))
        seen |= set(f)
    with pytest.raises(ValueError):
        replicas.frames_for_rank(4, 4, 10)


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    replicas.barrier()
    m = replicas.max_over_ranks(10.0 + rank * 2.5)
    q.put((rank, m, replicas.frames_for_rank(rank, world, 3)))
    dist.destroy_process_group()


def test_max_over_two_gloo_ranks():
    import socket

    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [m for _, m, _ in res] == [12.5, 12.5]
    assert res[0][2] == [0, 1, 2] and res[1][2] == [3, 4, 5]
