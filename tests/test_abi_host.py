"""CPU-side checks of the C ABI: the library loads, exports every entry point
that include/qpath.h declares, and its host-only logic (the acceptance
threshold tables) is byte-equal to the oracle's."""
import os
import re

import numpy as np
import pytest

from paper_2608_25376_gb300 import build as qbuild
from paper_2608_25376_gb300 import qpath

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    qbuild.build()
    return qpath.lib()


def declared_functions():
    names = []
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if f.endswith(".h"):
            text = open(os.path.join(ROOT, "include", f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(qp_\w+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_binding_symbols():
    assert sorted(qpath.SYMBOLS) == declared_functions()


def test_library_exports_every_declared_symbol(L):
    for name in declared_functions():
        assert hasattr(L, name), name


def test_last_error_empty_and_bad_args_rejected_without_gpu(L):
    import ctypes as ct
    assert isinstance(qpath.qp_last_error(), str)
    out = ct.c_void_p()
    # NULL field is rejected before any CUDA call
    assert L.qp_build_qubo(None, 0, 1, 100, 0, ct.byref(out)) == qpath.QP_EINVAL
    assert "NULL" in qpath.qp_last_error()
    sc = qpath.schedule(10)
    assert L.qp_thresholds(ct.byref(sc), 10, None, 0, None) == qpath.QP_EINVAL


@pytest.mark.parametrize("n_sweeps,T0,T1", [(2000, 1e3, 1.0), (5000, 1e3, 1.0), (7, 3.5, 3.5), (1, 50.0, 1.0)])
def test_threshold_tables_byte_equal_to_oracle(L, orc, n_sweeps, T0, T1):
    sc = qpath.schedule(n_sweeps, T0, T1)
    sweeps = sorted(set([0, n_sweeps - 1, n_sweeps // 2, n_sweeps // 3, min(5, n_sweeps - 1)]))
    for s in sweeps:
        mine = qpath.qp_thresholds(sc, s)
        ref = orc.thresholds(orc.temperature(n_sweeps, T0, T1, s))
        assert mine.dtype == np.uint32 and ref.dtype == np.uint32
        assert mine.tobytes() == ref.tobytes(), s


def test_threshold_cap_error(L):
    import ctypes as ct
    sc = qpath.schedule(10, 100.0, 1.0)
    n = ct.c_int32()
    buf = np.zeros(4, np.uint32)
    st = L.qp_thresholds(ct.byref(sc), 0, buf.ctypes.data_as(ct.c_void_p), 4, ct.byref(n))
    assert st == qpath.QP_ERANGE and n.value > 4


def test_checked_build_compiles_and_exports_every_declared_symbol():
    """The checked build (device bounds checks compiled in) builds here and
    exposes the same ABI; it is run on the GPU by test_gpu_device_checks."""
    import ctypes as ct
    path = qbuild.build(checked=True)
    assert os.path.basename(path) == "libqpath_checked.so"
    lib = ct.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name
