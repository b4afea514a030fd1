"""The C-ABI library loads on a machine without a GPU and exports every symbol
that include/*.h declares (no compute calls are made here)."""
import ctypes
import os
import re

import paper_2507_14652_gb300 as hmc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            names += re.findall(r"^HMC_API[^(]*?\b(hmc_\w+)\s*\(", src, flags=re.M)
    return names


def test_library_exports_every_declared_symbol():
    if not os.path.exists(hmc.LIB_PATH):
        hmc.build()
    L = ctypes.CDLL(hmc.LIB_PATH)
    names = _declared()
    assert len(names) >= 13
    for n in names:
        assert hasattr(L, n), n
    assert sorted(names) == sorted(hmc.EXPORTS)


def test_last_error_is_callable_without_gpu():
    if not os.path.exists(hmc.LIB_PATH):
        hmc.build()
    assert hmc.lib().hmc_last_error() == b""


def test_training_arrays_keep_float32_only_when_all_are_float32():
    import numpy as np
    a32, b32 = np.zeros((3, 2), np.float32), np.zeros((3, 1), np.float32)
    (x, y), dt = hmc._training_arrays(a32, b32)
    assert dt == hmc.DATA_F32 and x.dtype == np.float32 and y.dtype == np.float32
    (x, y), dt = hmc._training_arrays(a32, np.zeros((3, 1)))
    assert dt == hmc.DATA_F64 and x.dtype == np.float64 and y.dtype == np.float64
    # the ctypes mirror of hmc_data ends with the dtype field, as include/hmc.h declares it
    assert hmc.Data._fields_[-1][0] == "dtype"
