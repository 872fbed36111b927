"""The multi-GPU bench path on CPU: two gloo ranks, disjoint frames, max/sum
reductions of timing and ray counts (no data-path collective)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    from paper_1903_03837_gb300 import replicas
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    frames = replicas.frames_for_rank(rank, world, 7, 240)
    t = replicas.reduce_max(1.5 + rank)
    n = replicas.reduce_sum(1000 * (rank + 1))
    dist.barrier()
    q.put((rank, frames, t, n))
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_frames_and_reduce_timing():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = dict((r, (f, t, n)) for r, f, t, n in (q.get(timeout=120) for _ in ps))
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert set(out[0][0]).isdisjoint(out[1][0])
    assert out[0][1] == out[1][1] == 2.5
    assert out[0][2] == out[1][2] == 3000.0


def test_single_process_reductions_are_identity():
    from paper_1903_03837_gb300 import replicas
    assert replicas.reduce_max(3.0) == 3.0
    assert replicas.frames_for_rank(0, 1, 3, 240) == [0, 1, 2]
    assert replicas.frames_for_rank(1, 2, 3, 4) == [3, 0, 1]
    with pytest.raises(ValueError):
        replicas.frames_for_rank(2, 2, 3, 240)
