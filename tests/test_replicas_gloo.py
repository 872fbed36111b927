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


# --------------------------------------------------------------------------
# Data-parallel fit: shards of the target views, one gradient all-reduce per
# step. A CPU stand-in for the light field (a fixed row-stochastic linear map per
# view, i.e. the same linear blend structure) lets gloo ranks run the same
# fit_step the GPU fit uses.
# --------------------------------------------------------------------------
class _LinearField:
    def __init__(self, mats, C):
        self.mats, self.C = mats, C          # view id -> [P_v, M*N] weights

    def render(self, views, idx=None):
        T = self.table.reshape(-1, self.C)
        return torch.cat([self.mats[v] @ T for v in views]), idx

    def render_backward(self, views, g, grad, idx=None):
        off = 0
        for v in views:
            P = self.mats[v].shape[0]
            grad.view(-1, self.C).add_(self.mats[v].t() @ g[off:off + P])
            off += P
        return grad


def _fit(rank, world, steps=6):
    from paper_1903_03837_gb300 import replicas, torch_api
    gen = torch.Generator().manual_seed(0)
    M, N, C, V, P = 6, 5, 3, 4, 7
    mats = []
    for _ in range(V):
        m = torch.rand((P, M * N), generator=gen, dtype=torch.float64)
        mats.append(m / m.sum(1, keepdim=True))
    truth = torch.rand((M, N, C), generator=gen, dtype=torch.float64)
    targets = [mats[v] @ truth.reshape(-1, C) for v in range(V)]
    mine = replicas.shard(list(range(V)), rank, world)
    table = torch.zeros((M, N, C), dtype=torch.float64, requires_grad=True)
    lf = _LinearField(mats, C)
    lf.table = table.detach()
    opt = torch.optim.Adam([table], lr=0.05)
    target = torch.cat([targets[v] for v in mine])
    table.grad = torch.zeros_like(table)
    for _ in range(steps):
        torch_api.fit_step(lf, table, opt, mine, target, None, V * P * C)
    return table.detach().clone()


def _fit_worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = _fit(rank, world)
    q.put((rank, t.numpy()))
    dist.barrier()
    dist.destroy_process_group()


def test_data_parallel_fit_matches_single_process():
    import numpy as np
    import torch.multiprocessing as mp
    single = _fit(0, 1).numpy()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_fit_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = dict(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert np.array_equal(out[0], out[1])                 # the replicas stay identical
    np.testing.assert_allclose(out[0], single, rtol=0, atol=1e-12)
    assert np.abs(single).max() > 0.1                    # the fit moved the table


def test_shard_covers_and_balances():
    from paper_1903_03837_gb300 import replicas
    items = list(range(11))
    parts = [replicas.shard(items, r, 3) for r in range(3)]
    assert sum(parts, []) == items
    assert max(map(len, parts)) - min(map(len, parts)) <= 1
    with pytest.raises(ValueError):
        replicas.shard(items, 3, 3)
