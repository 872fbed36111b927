"""The C ABI used from a plain C program (tests/c_abi/abi_consumer.c) with
include/lumipath.h alone: its argument checks on the CPU, and on the GPU a
render whose indices and colours are checked against the oracle."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import lf_inputs
import oracle
from paper_1903_03837_gb300 import build as B
from paper_1903_03837_gb300 import lumipath as lp

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "c_abi", "abi_consumer.c")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


@pytest.fixture(scope="module")
def consumer(tmp_path_factory):
    if shutil.which("gcc") is None:
        pytest.skip("gcc is not installed")
    B.build()
    libdir = os.path.dirname(B.LIB)
    cudalib = os.path.join(CUDA, "lib64")
    exe = str(tmp_path_factory.mktemp("c_abi") / "abi_consumer")
    cmd = ["gcc", "-std=c11", "-O1", "-Wall", "-Werror", SRC, "-I", B.INCLUDE, "-I", os.path.join(CUDA, "include"),
           "-L", libdir, "-llumipath", "-L", cudalib, "-lcudart", f"-Wl,-rpath,{libdir}:{cudalib}", "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_c_program_sees_every_check(consumer):
    r = subprocess.run([consumer, "check"], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr


@pytest.mark.gpu
def test_c_program_renders_like_the_oracle(consumer, tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    views = lf_inputs.pack_offsets([lf_inputs.look_at((2.4, 0.3, 0.4), (0, 0, 0), 48, 40),
                                    lf_inputs.look_at((0.1, -0.2, -2.7), (0, 0, 0), 33, 21)])
    arr = lp.make_views(views)
    vpath, opath = tmp_path / "views.bin", tmp_path / "out.bin"
    vpath.write_bytes(bytes(arr)[:ctypes.sizeof(lp.lf_view) * len(views)])
    r = subprocess.run([consumer, "render", str(vpath), str(opath)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    P = lf_inputs.total_pixels(views)
    raw = opath.read_bytes()
    img = np.frombuffer(raw[:P * 16], np.float32).reshape(P, 4)
    idx = np.frombuffer(raw[P * 16:], np.int32).reshape(P, 10)
    M, N = 300, 100
    i, j, c = np.meshgrid(np.arange(M), np.arange(N), np.arange(4), indexing="ij")
    T = (((131 * i + 71 * j + 29 * c) % 1000) / 1000.0).astype(np.float32)
    want, want_idx, hits = oracle.render_views(oracle.Scene(M, N, 4, "f32", T), views)
    assert hits > 500
    np.testing.assert_array_equal(idx, want_idx)
    assert np.abs(img.astype(np.float64) - want).max() <= 1e-5
