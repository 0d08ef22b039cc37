"""PRUNE oracle: a plain, slow, sequential FP64 CPU model of the method.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import or
execute anything in this package.  It shares no code with the CUDA path (no
kernels, headers, helpers, tables or constants) and imports nothing from it.

Parts:
  * ``prune_oracle.c`` (loaded here through ctypes): the dataflow simulator of
    the canonical graph SRC -> FIR -> {DET, SEL}; DET -> {SEL, SINK} (control);
    SEL -> HX_b -> SINK for b < F, with blocking FIFOs sized by eq. (2), DRP
    rates set by eq. (1), FIR delay line carried as the initial token of a
    self-loop FIFO (Sec. III-D), FP64 arithmetic from FP32 inputs.
  * ``analysis.py``: the MoC-level checks of Sec. III-V (port/FIFO rate
    matching, control table, design rules 1-5, the DC-finding procedure, DPG
    validity, SDF consistency of every DC, eq. (2), and a brute-force deadlock
    and overflow search over all control sequences of tiny graphs).

Every function here is pinned by ``tests/test_oracle_*.py`` against values the
paper or the mathematics fix (impulse responses, direct convolution by numpy,
identity and permutation matrices, exact ties, the worked example of Fig. 6,
the DC example of Fig. 5, conservation invariants).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "prune_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")

FIFO_NAMES = ("f0", "f1", "f2", "f3", "f4", "f5", "f6", "f7")
ACTOR_NAMES = ("SRC", "FIR", "DET", "SEL", "HX", "SINK")

ORACLE_OK, ORACLE_EINVAL, ORACLE_ENOMEM, ORACLE_EDEADLOCK = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the C simulator with gcc (plain -O2, no fast-math) if needed."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(_LIB), exist_ok=True)
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fno-fast-math", "-ffp-contract=off",
                               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Graph(ctypes.Structure):
    _fields_ = [("F", ctypes.c_int32), ("B", ctypes.c_int32), ("T", ctypes.c_int32),
                ("N", ctypes.c_int32), ("C", ctypes.c_int32), ("tau", ctypes.c_float),
                ("taps", ctypes.c_void_p), ("H", ctypes.c_void_p)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        lib.oracle_run.argtypes = [ctypes.POINTER(_Graph), P, ctypes.c_int64, P, P, P, P, P, P, P, P]
        lib.oracle_run.restype = ctypes.c_int
        lib.oracle_fifo_capacity.argtypes = [ctypes.c_long] * 3
        lib.oracle_fifo_capacity.restype = ctypes.c_long
        lib.oracle_linear_fifo_replay.argtypes = [ctypes.c_long] * 5 + [P, P]
        lib.oracle_linear_fifo_replay.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class OracleResult:
    """Per-frame sink records and FIFO counters of one oracle run.

    c[k]       number of selected blocks of frame k (the DPG firing rate)
    idx[k]     ascending selected block indices of frame k (length c[k])
    y[k]       complex128 array [c[k], B]: compacted sink output of frame k
    energy     float64 [n_frames, F]: DET block energies
    stats      dict fifo -> (written, read, peak, final occupancy)
    fires      dict actor -> number of firings
    hist_out   complex128 [T-1]: delay token left in f1 after the run
    """
    c: np.ndarray
    idx: list
    y: list
    energy: np.ndarray
    stats: dict
    fires: dict
    hist_out: np.ndarray


def run(F, B, T, N, tau, taps, H, x, C=3, hist_in=None) -> OracleResult:
    """Fire the canonical graph over ``x`` ([n_frames, F, B] complex64).

    taps: complex [T];  H: complex [N, N] (row-major, out_row = H @ in_row);
    tau: float32 DET threshold;  C: buffering constant of eq. (2);
    hist_in: optional complex [T-1] initial delay token (default zeros).
    """
    lib = _load()
    x = np.ascontiguousarray(np.asarray(x, dtype=np.complex64).reshape(-1, F, B))
    n = x.shape[0]
    taps32 = np.ascontiguousarray(np.asarray(taps, dtype=np.complex64).reshape(T)).view(np.float32)
    H32 = np.ascontiguousarray(np.asarray(H, dtype=np.complex64).reshape(N, N)).view(np.float32)
    g = _Graph(F, B, T, N, C, np.float32(tau), taps32.ctypes.data, H32.ctypes.data)
    c = np.zeros(n, np.int32)
    idx = np.zeros((n, F), np.int32)
    y = np.zeros(max(n * F * B, 1) * 2, np.float64)
    energy = np.zeros((n, F), np.float64)
    stats = np.zeros((8, 4), np.int64)
    fires = np.zeros(6, np.int64)
    hin = None
    if hist_in is not None and T > 1:
        hin = np.ascontiguousarray(np.asarray(hist_in, np.complex128).reshape(T - 1)).view(np.float64)
    hout = np.zeros(max(T - 1, 1) * 2, np.float64)
    xs = x.view(np.float32)
    rc = lib.oracle_run(ctypes.byref(g), _ptr(xs), n, _ptr(c), _ptr(idx), _ptr(y), _ptr(energy),
                        _ptr(stats), _ptr(fires), _ptr(hin), _ptr(hout))
    if rc != ORACLE_OK:
        raise RuntimeError(f"oracle_run failed with code {rc}")
    yc = y.view(np.complex128)
    ys, off = [], 0
    for k in range(n):
        ys.append(yc[off:off + c[k] * B].reshape(c[k], B).copy())
        off += c[k] * B
    return OracleResult(
        c=c, idx=[idx[k, :c[k]].copy() for k in range(n)], y=ys, energy=energy,
        stats={FIFO_NAMES[i]: tuple(int(v) for v in stats[i]) for i in range(8)},
        fires={ACTOR_NAMES[i]: int(fires[i]) for i in range(6)},
        hist_out=hout.view(np.complex128)[:max(T - 1, 0)].copy())


def fifo_capacity(r: int, Q: int, C: int) -> int:
    """Eq. (2) in tokens (token size factored out)."""
    return int(_load().oracle_fifo_capacity(r, Q, C))


def linear_fifo_replay(r: int, Q: int, C: int, n_iter: int, cap_override: int = 0):
    """Replay the linear buffer with copy-back of Fig. 6; returns
    (error code, write window starts, read window starts)."""
    wp = np.zeros(max(n_iter, 1), np.int64)
    rp = np.zeros(max(n_iter, 1), np.int64)
    err = _load().oracle_linear_fifo_replay(r, Q, C, cap_override, n_iter, _ptr(wp), _ptr(rp))
    return int(err), wp[:n_iter].tolist(), rp[:n_iter].tolist()


def scatter(result: OracleResult, F: int, B: int) -> np.ndarray:
    """Host convenience: the compacted records expanded to [n_frames, F, B]
    with zeros for unselected blocks (inactive DCs produce nothing, itr = 0)."""
    n = len(result.c)
    out = np.zeros((n, F, B), np.complex128)
    for k in range(n):
        out[k, result.idx[k]] = result.y[k]
    return out
