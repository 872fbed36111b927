"""lf_render_noalloc: the render entry point for callers that cannot allocate
device memory (a process whose memory is reserved by another runtime's pool,
or a frame-paced loop that must not call cudaMalloc/cudaFree because they
synchronise the device). It keeps the SF point caches and its status/queue
words in a fixed array inside the library instead of allocating them.

Checked here through the C ABI against the ordinary path (lf_create_table +
lf_render) on two calls in a row, with different tables, so the second call
must rebuild what the first left in the shared array; against the CPU oracle
with an upper-hemisphere table (5 neighbours and nearest sampling, which take
their own paths through the weights and the masking); with more than 64 views
(several launches in one call, re-arming the persistent grid's tile queue and
the exact pass's queue in between); and through lf_noalloc_sync_status, which
reads the array's device status word. This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

import lf_inputs
from paper_1903_03837_gb300 import lumipath as lp

ATOL = 1e-5


def _desc(M, N, Cc, dtype, upper=False, k_nearest=5):
    d = lp.lf_table_desc()
    d.radius = 1.0
    d.center[:] = [0.0, 0.0, 0.0]
    d.n_origins, d.n_directions, d.channels = M, N, Cc
    d.dtype = lp.DTYPES[dtype]
    d.flags = lp.LF_TABLE_UPPER_HEMISPHERE if upper else 0
    d.k_nearest = k_nearest
    return d


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def test_noalloc_rejects_more_points_than_its_array():
    d = _desc(270000, 9000, 4, "f32")
    views = lp.make_views([lf_inputs.look_at((2, 0, 0), (0, 0, 0), 8, 8)])
    s = lp.lib().lf_render_noalloc(C.byref(d), C.c_void_p(0x1000), None, views, 1, None,
                                   C.c_void_p(0x1000), None, None)
    assert s == lp.LF_ERR_INVALID_ARG
    msg = lp.lf_last_error()
    assert "exceeds the no-allocation scratch limit" in msg and "278528" in msg


@pytest.mark.gpu
def test_noalloc_matches_lf_render_on_two_calls_in_a_row():
    torch = _torch()
    from paper_1903_03837_gb300 import torch_api as api

    rng = np.random.default_rng(21)
    views = lf_inputs.pack_offsets([lf_inputs.look_at((2.0, -1.2, 0.6), (0, 0, 0), 96, 64),
                                    lf_inputs.look_at((0.1, 0.05, 2.3), (0, 0, 0), 40, 56),
                                    lf_inputs.look_at((-1.4, 1.4, -0.9), (0, 0, 0), 33, 21)])
    P = lf_inputs.total_pixels(views)
    cases = [
        # (M, N, C, storage, launch shape)
        (16384, 512, 4, "e4m3", lp.lf_launch(16, 16, 8, 1, 1, 0)),
        (3000, 700, 3, "f32", None),
    ]
    stream = torch.cuda.current_stream().cuda_stream
    for M, N, Cc, dtype, launch in cases:
        T = torch.from_numpy(rng.uniform(0, 2, (M, N, Cc)).astype(np.float32)).cuda()
        if dtype == "f32":
            tab, sc = T, None
        else:
            tab, sc = api.quantize_table(T, dtype)
        lf = api.LightField(tab, dtype, sc)
        if launch is not None:
            lf.set_launch(**launch.as_dict())
        want, want_idx = lf.render(views, with_idx=True)
        lf.sync_status()
        lf.close()

        out = torch.full((P, Cc), float("nan"), device="cuda")
        idx = torch.full((P, 10), -7, dtype=torch.int32, device="cuda")
        lp.lf_render_noalloc(_desc(M, N, Cc, dtype), tab.data_ptr(), sc.data_ptr() if sc is not None else None,
                             lp.make_views(views), len(views), launch, out.data_ptr(), idx.data_ptr(), stream)
        torch.cuda.synchronize()
        assert torch.equal(idx, want_idx)
        assert float((out - want).abs().max()) <= ATOL
        assert int((idx[:, 0] >= 0).sum()) > 1000


@pytest.mark.gpu
@pytest.mark.parametrize("k_nearest", [5, 1])
def test_noalloc_upper_hemisphere_against_the_oracle(k_nearest):
    """An upper-hemisphere table (rows i < M/2 stored) seen from above and from
    below: indices equal the oracle's, colours within 1e-5, and equal to
    lf_create_table + lf_render's."""
    torch = _torch()
    import oracle
    from paper_1903_03837_gb300 import torch_api as api

    M, N = 3001, 700
    rows = M // 2
    rng = np.random.default_rng(5 + k_nearest)
    T = rng.uniform(0, 1, (rows, N, 4)).astype(np.float32)
    views = lf_inputs.pack_offsets([lf_inputs.look_at((0.4, 0.3, 2.3), (0, 0, 0), 48, 40),
                                    lf_inputs.look_at((2.0, -0.9, -0.7), (0, 0, 0), 56, 32),
                                    lf_inputs.look_at((0.2, -0.3, -2.5), (0, 0, 0), 24, 24)])
    want_out, want_idx, hits = oracle.render_views(oracle.Scene(M, N, 4, "f32", T, K=k_nearest, upper=True), views)
    assert hits > 500
    P = lf_inputs.total_pixels(views)
    Td = torch.from_numpy(T).cuda()
    width = 2 if k_nearest == 1 else 10
    out = torch.full((P, 4), float("nan"), device="cuda")
    idx = torch.full((P, width), -7, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    lp.lf_render_noalloc(_desc(M, N, 4, "f32", upper=True, k_nearest=k_nearest), Td.data_ptr(), None,
                         lp.make_views(views), len(views), None, out.data_ptr(), idx.data_ptr(), stream)
    lp.lf_noalloc_sync_status(stream)
    got_out, got_idx = out.cpu().numpy(), idx.cpu().numpy()
    assert np.array_equal(got_idx, want_idx)
    assert float(np.abs(got_out - want_out).max()) <= ATOL

    lf = api.LightField(Td, "f32", n_origins=M, upper=True, k_nearest=k_nearest)
    ref_out, ref_idx = lf.render(views, with_idx=True)
    lf.sync_status()
    lf.close()
    assert torch.equal(idx, ref_idx)
    assert torch.equal(out, ref_out)


@pytest.mark.gpu
def test_noalloc_many_views_persistent():
    """70 views in one call (launches of 64 and 6 views) on the persistent grid:
    the same image and indices as lf_create_table + lf_render, bit for bit,
    and a clean status word."""
    torch = _torch()
    from paper_1903_03837_gb300 import torch_api as api

    rng = np.random.default_rng(70)
    M, N = 16384, 512
    T = torch.from_numpy(rng.uniform(0, 1, (M, N, 4)).astype(np.float32)).cuda()
    codes, sc = api.quantize_table(T, "f16")
    vs = []
    for k in range(70):
        d = rng.normal(size=3)
        d *= rng.uniform(1.6, 3.5) / np.linalg.norm(d)
        vs.append(lf_inputs.look_at(tuple(d), (0, 0, 0), int(rng.integers(8, 40)), int(rng.integers(8, 40))))
    views = lf_inputs.pack_offsets(vs)
    P = lf_inputs.total_pixels(views)
    launch = lp.lf_launch(16, 8, 8, 1, 1, 0)
    lf = api.LightField(codes, "f16", sc)
    lf.set_launch(**launch.as_dict())
    want, want_idx = lf.render(views, with_idx=True)
    lf.sync_status()
    lf.close()
    out = torch.full((P, 4), float("nan"), device="cuda")
    idx = torch.full((P, 10), -7, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        lp.lf_render_noalloc(_desc(M, N, 4, "f16"), codes.data_ptr(), sc.data_ptr(), lp.make_views(views),
                             len(views), launch, out.data_ptr(), idx.data_ptr(), stream)
        lp.lf_noalloc_sync_status(stream)
        assert torch.equal(idx, want_idx)
        assert torch.equal(out, want)
    assert int((idx[:, 0] >= 0).sum()) > 2000
