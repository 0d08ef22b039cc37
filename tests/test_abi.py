"""The C-ABI library without a GPU: it loads, exports every symbol that
include/prune.h declares, computes eq. (2) like the oracle, and rejects bad
descriptors before touching a device."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_1802_06625_b300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "prune.h")).read()
    return sorted(set(re.findall(r"PRUNE_API\s+[\w\s\*]+?\b(prune_\w+)\s*\(", txt)))


def test_library_builds_and_exports_every_declared_symbol():
    build.build()
    lib = _lib.lib()
    names = _declared()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(_lib.EXPORTS)


@pytest.mark.parametrize("r,Q,C", [(4, 1, 3), (1, 1, 3), (64, 0, 3), (3, 7, 2), (2, 8, 3), (5, 10, 1)])
def test_fifo_capacity_matches_oracle(r, Q, C):
    cap = ctypes.c_int64()
    assert _lib.lib().prune_fifo_capacity(r, Q, C, ctypes.byref(cap)) == _lib.PRUNE_OK
    assert cap.value == oracle.fifo_capacity(r, Q, C)


def test_fifo_capacity_rejects_bad_args():
    cap = ctypes.c_int64()
    assert _lib.lib().prune_fifo_capacity(0, 1, 3, ctypes.byref(cap)) == _lib.PRUNE_EINVAL
    assert _lib.lib().prune_fifo_capacity(1, -1, 3, ctypes.byref(cap)) == _lib.PRUNE_EINVAL
    assert _lib.lib().prune_fifo_capacity(1, 1, 0, ctypes.byref(cap)) == _lib.PRUNE_EINVAL


def _create(**kw):
    taps = np.ones(2 * kw.get("T", 4), np.float32)
    H = np.eye(kw.get("N", 4), dtype=np.complex64).view(np.float32)
    d = _lib.prune_graph_desc(F=kw.get("F", 4), B=kw.get("B", 64), T=kw.get("T", 4), N=kw.get("N", 4),
                              C=kw.get("C", 3), out_frames=0, tau=kw.get("tau", 1.0),
                              taps=taps.ctypes.data, H=H.ctypes.data, stream=None, device=-1)
    h = ctypes.c_void_p()
    st = _lib.lib().prune_graph_create(ctypes.byref(d), ctypes.byref(h))
    return st, h


@pytest.mark.parametrize("kw", [dict(F=0), dict(B=12), dict(B=4096), dict(B=40), dict(T=0), dict(T=300),
                                dict(B=64, T=70), dict(N=5), dict(N=256, B=256), dict(tau=float("nan")),
                                dict(C=-1)])
def test_create_rejects_bad_descriptors(kw):
    st, h = _create(**kw)
    assert st == _lib.PRUNE_EINVAL
    assert h.value is None
    assert _lib.lib().prune_last_error(None).decode()


def test_no_cpu_fallback():
    # A valid descriptor without a usable device fails with ECUDA instead of
    # computing anything on the CPU.
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    st, h = _create()
    assert st == _lib.PRUNE_ECUDA
    assert b"CUDA" in _lib.lib().prune_last_error(None) or b"device" in _lib.lib().prune_last_error(None)


def test_null_arguments():
    L = _lib.lib()
    assert L.prune_graph_create(None, None) == _lib.PRUNE_EINVAL
    assert L.prune_graph_destroy(None) == _lib.PRUNE_OK
    assert L.prune_push_frames(None, None, 1, 0) == _lib.PRUNE_EINVAL
    assert L.prune_run(None, 1, None, 0) == _lib.PRUNE_EINVAL
    assert L.prune_pull(None, None, 1, None, 0) == _lib.PRUNE_EINVAL
