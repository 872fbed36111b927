"""The debug build (-DLF_DEBUG_CHECKS), in place of a sanitizer: every index
the kernels dereference is checked against its bound and a failure would set a
status bit (never a trap). Renders, backwards, nine neighbours, an
upper-hemisphere table and the precompute run through it with no check firing
and with indices equal to the oracle's."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import os, sys
sys.path.insert(0, os.environ["LF_ROOT"])
import numpy as np, torch, lf_inputs, oracle
from paper_1903_03837_gb300 import lumipath as lp, torch_api as api
assert os.path.samefile(lp.lib()._name, os.environ["LUMIPATH_LIB"])
views = lf_inputs.pack_offsets([lf_inputs.look_at((2.4, 0.3, 0.4), (0, 0, 0), 80, 64),
                                lf_inputs.look_at((0.05, 0.02, 2.6), (0, 0, 0), 40, 40),
                                lf_inputs.look_at((0.1, -0.05, -3.0), (0, 0, 0), 32, 32)])
P = lf_inputs.total_pixels(views)
rng = np.random.default_rng(0)
for (M, N, K, upper) in [(1024, 256, 5, False), (100, 60, 5, False), (65536, 1024, 5, False),
                         (3001, 700, 5, True), (1024, 256, 9, False), (1024, 256, 1, False)]:
    rows = M // 2 if upper else M
    T = rng.uniform(0, 1, (rows, N, 4)).astype(np.float32)
    lf = api.LightField(torch.from_numpy(T).cuda(), "f32", n_origins=M, upper=upper, k_nearest=K)
    out, idx = lf.render(views, with_idx=True)
    g = torch.ones((P, 4), device="cuda")
    lf.render_backward(views, g)
    lf.render_backward(views, g, idx=idx)
    lf.sync_status()                      # raises if any check fired
    _, want_idx, _ = oracle.render_views(oracle.Scene(M, N, 4, "f32", T, K=K, upper=upper), views)
    assert np.array_equal(idx.cpu().numpy(), want_idx), (M, N, K, upper)
    lf.close()
vol = lf_inputs.draw_volume(1, B=5, spp=2, steps=8)
t = api.precompute_table(vol, 128, 64, 4)
torch.cuda.synchronize()
np.testing.assert_allclose(t.cpu().numpy(), oracle.volume_table(vol, 128, 64, 4), rtol=0, atol=1e-4)
print("debug-ok")
'''


def test_debug_build_runs_clean():
    from paper_1903_03837_gb300 import build as B
    lib = B.build(force=True, extra_flags=["-DLF_DEBUG_CHECKS"], out_dir=B.DEBUG_DIR)
    env = dict(os.environ, LUMIPATH_LIB=lib, LF_ROOT=ROOT)
    r = subprocess.run([sys.executable, "-c", SCRIPT], env=env, capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, (r.stdout[-2000:], r.stderr[-4000:])
    assert "debug-ok" in r.stdout
