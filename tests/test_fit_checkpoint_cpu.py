"""Checkpoint / resume of a table fit: a fit stopped after k steps, saved and
restored into a fresh table and optimiser continues bit-identically (the same
fit_step the GPU fit uses, with a CPU stand-in for the light field)."""
import pytest

torch = pytest.importorskip("torch")


class _LinearField:
    def __init__(self, mats, C, table):
        self.mats, self.C, self.table = mats, C, table

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


def _problem():
    gen = torch.Generator().manual_seed(3)
    M, N, C, V, P = 5, 4, 3, 3, 6
    mats = []
    for _ in range(V):
        m = torch.rand((P, M * N), generator=gen, dtype=torch.float64)
        mats.append(m / m.sum(1, keepdim=True))
    truth = torch.rand((M, N, C), generator=gen, dtype=torch.float64)
    target = torch.cat([mats[v] @ truth.reshape(-1, C) for v in range(V)])
    return mats, target, (M, N, C), V * P * C


def _fresh(shape, mats):
    table = torch.zeros(shape, dtype=torch.float64, requires_grad=True)
    table.grad = torch.zeros_like(table)
    opt = torch.optim.Adam([table], lr=0.05)
    return table, opt, _LinearField(mats, shape[2], table.detach())


def test_resumed_fit_is_bit_identical(tmp_path):
    from paper_1903_03837_gb300 import torch_api
    mats, target, shape, gv = _problem()
    views = [0, 1, 2]
    table, opt, lf = _fresh(shape, mats)
    for _ in range(8):
        torch_api.fit_step(lf, table, opt, views, target, None, gv)
    straight = table.detach().clone()

    table, opt, lf = _fresh(shape, mats)
    for _ in range(5):
        torch_api.fit_step(lf, table, opt, views, target, None, gv)
    path = str(tmp_path / "fit.pt")
    torch_api.save_fit_state(path, table, opt, 5)
    table, opt, lf = _fresh(shape, mats)
    step = torch_api.load_fit_state(path, table, opt)
    assert step == 5
    for _ in range(8 - step):
        torch_api.fit_step(lf, table, opt, views, target, None, gv)
    assert torch.equal(table.detach(), straight)


def test_checkpoint_shape_mismatch_is_refused(tmp_path):
    from paper_1903_03837_gb300 import torch_api
    mats, target, shape, gv = _problem()
    table, opt, _ = _fresh(shape, mats)
    path = str(tmp_path / "fit.pt")
    torch_api.save_fit_state(path, table, opt, 0)
    other = torch.zeros((shape[0] + 1, shape[1], shape[2]), dtype=torch.float64, requires_grad=True)
    with pytest.raises(ValueError):
        torch_api.load_fit_state(path, other, torch.optim.Adam([other], lr=0.05))
