"""The library's device generator (Philox4x32-10, xyl_philox) against cuRAND's
own Philox4x32-10 block function for 10^6 random (counter, key) pairs and
against the oracle's."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def env(tmp_path_factory):
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    from paper_1211_3991_gb300 import build
    build.build()
    from paper_1211_3991_gb300 import xyl
    xyl.load()
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    so = str(tmp_path_factory.mktemp("curand") / "libcurand_ref.so")
    subprocess.run([nvcc, "-gencode=arch=compute_103a,code=sm_103a", "-O2", "-shared", "-Xcompiler", "-fPIC",
                    "-cudart", "shared", "-o", so, os.path.join(HERE, "curand_philox_ref.cu")], check=True)
    ref = C.CDLL(so)
    ref.curand_philox_blocks.argtypes = [C.c_void_p, C.c_void_p, C.c_longlong, C.c_void_p]
    return torch, xyl, ref


def _device(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, np.uint32).view(np.int32)).cuda()


def _library(torch, xyl, ctr, key):
    out = torch.empty((len(ctr), 4), dtype=torch.int32, device="cuda")
    xyl.philox(_device(torch, ctr), _device(torch, key), out)
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint32)


def test_generator_equals_curand(env):
    torch, xyl, ref = env
    n = 1_000_000
    rng = np.random.default_rng(12)
    ctr = rng.integers(0, 2 ** 32, (n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, (n, 2), dtype=np.uint64).astype(np.uint32)
    ctr[:4] = [[0, 0, 0, 0], [0xFFFFFFFF] * 4, [1, 0, 0, 0], [0, 0, 0, 1]]
    key[:4] = [[0, 0], [0xFFFFFFFF] * 2, [0, 1], [1, 0]]
    got = _library(torch, xyl, ctr, key)
    c, k = _device(torch, ctr), _device(torch, key)
    want = torch.empty((n, 4), dtype=torch.int32, device="cuda")
    assert ref.curand_philox_blocks(C.c_void_p(c.data_ptr()), C.c_void_p(k.data_ptr()), n,
                                    C.c_void_p(want.data_ptr())) == 0
    assert np.array_equal(got, want.cpu().numpy().view(np.uint32))


def test_generator_equals_oracle(env, orc):
    torch, xyl, _ = env
    rng = np.random.default_rng(13)
    ctr = rng.integers(0, 2 ** 32, (2000, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, (2000, 2), dtype=np.uint64).astype(np.uint32)
    got = _library(torch, xyl, ctr, key)
    want = np.array([orc.philox(c, k) for c, k in zip(ctr, key)], np.uint32)
    assert np.array_equal(got, want)
