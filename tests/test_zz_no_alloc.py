"""lf_render_noalloc: the render entry point for callers that cannot allocate
device memory (a process whose memory is reserved by another runtime's pool,
or a frame-paced loop that must not call cudaMalloc/cudaFree because they
synchronise the device). It keeps the SF point caches and its status/queue
words in a fixed array inside the library instead of allocating them.

Checked here through the C ABI against the ordinary path (lf_create_table +
lf_render) on two calls in a row, with different tables, so the second call
must rebuild what the first left in the shared array. This file is collected
last on purpose."""
import ctypes as C

import numpy as np
import pytest

import lf_inputs
from paper_1903_03837_gb300 import lumipath as lp

ATOL = 1e-5


def _desc(M, N, Cc, dtype):
    d = lp.lf_table_desc()
    d.radius = 1.0
    d.center[:] = [0.0, 0.0, 0.0]
    d.n_origins, d.n_directions, d.channels = M, N, Cc
    d.dtype = lp.DTYPES[dtype]
    d.flags = 0
    d.k_nearest = 5
    return d


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
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
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
