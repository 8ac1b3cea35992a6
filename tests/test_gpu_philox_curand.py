"""The oracle's Philox4x32-10 against cuRAND's (an independent implementation
of the same generator, run on the GPU): every word equal on random counters
and keys and on the counters the annealer uses (k >> 2, sweep, replica, tag).
The library's own generator is tied to the oracle's by the bit-exact parity of
every anneal."""
import ctypes as ct
import os
import subprocess
import tempfile

import numpy as np
import pytest

from conftest import has_gpu

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def curand_lib():
    if not has_gpu():
        pytest.skip("no CUDA device")
    out = os.path.join(tempfile.mkdtemp(), "philox_curand.so")
    cmd = ["nvcc", "-gencode=arch=compute_103a,code=sm_103a", "-shared", "-Xcompiler", "-fPIC", "-o", out,
           os.path.join(HERE, "philox_curand_probe.cu")]
    subprocess.run(cmd, check=True, capture_output=True)
    lib = ct.CDLL(out)
    lib.curand_philox_batch.argtypes = [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_int]
    lib.curand_philox_batch.restype = ct.c_int
    return lib


def test_oracle_philox_equals_curand(curand_lib, orc):
    rng = np.random.default_rng(17)
    n = 2000
    ctr = rng.integers(0, 2 ** 32, (n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, (n, 2), dtype=np.uint64).astype(np.uint32)
    # the annealer's own counters: (k >> 2, sweep, replica, 0x51505448) under seed keys
    for i in range(200):
        ctr[i] = [i * 7, i % 13, 1000 + i, 0x51505448]
        key[i] = [1 + i % 3, 0]
    ctr[200] = [0, 0, 0, 0]
    key[200] = [0, 0]
    ctr[201] = [0xFFFFFFFF] * 4
    key[201] = [0xFFFFFFFF] * 2
    out = np.zeros((n, 4), np.uint32)
    assert curand_lib.curand_philox_batch(ctr.ctypes.data, key.ctypes.data, out.ctypes.data, n) == 0
    for i in range(n):
        assert (orc.philox4x32_10(ctr[i], key[i]) == out[i]).all(), i
