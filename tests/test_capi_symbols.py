"""The C-ABI library loads on a machine without a GPU and exports every symbol
that include/*.h declares (no compute calls are made here)."""
import ctypes
import os
import re

import pytest

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


def test_batch_problem_tuples_are_checked_before_the_library_is_called():
    # a batch entry is an MLP 7-tuple or a ("deeponet", ...) 11-tuple; anything else is a
    # ValueError raised by the binding (no handle is created)
    import numpy as np
    if not os.path.exists(hmc.LIB_PATH):
        hmc.build()
    bad = ("transformer", [2, 4, 1], [2, 4, 1], np.zeros((3, 2)), np.zeros((2, 2)), np.zeros((3, 2)),
           np.zeros(21, np.uint8), np.zeros(21), 1.0, 0.1, True)
    with pytest.raises(ValueError, match="unknown problem kind"):
        hmc.BatchSampler([bad], 2, hmc.PREC_FP32)
