"""Python view of the request loop (prune_server_*): argument marshalling
only.  Streams are admitted against the server's device-memory budget, their
frames are borrowed device tensors, and every step fires the next frames of
all ready streams in the library's batched kernels."""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import PruneError, check
from .graph import _c64_floats


class Server:
    def __init__(self, B, N, F_max, T_max, max_streams, hbm_budget, frames_per_step=1, ring=None,
                 max_inflight=2, auto_release=False, stream=None, device=None):
        if device is None:
            device = torch.cuda.current_device()
        ring = ring if ring is not None else max(2, 2 * frames_per_step)
        d = _lib.prune_server_desc(B=B, N=N, F_max=F_max, T_max=T_max, max_streams=max_streams,
                                   frames_per_step=frames_per_step, ring=ring, max_inflight=max_inflight,
                                   hbm_budget=int(hbm_budget),
                                   stream=stream.cuda_stream if stream is not None else None, device=device,
                                   flags=_lib.PRUNE_SERVER_AUTO_RELEASE if auto_release else 0)
        h = ctypes.c_void_p()
        check(_lib.lib().prune_server_create(ctypes.byref(d), ctypes.byref(h)))
        self.h = h
        self.B, self.N = B, N
        self._F = {}
        self._x = {}      # borrowed inputs kept alive until their stream closes

    def _check(self, st):
        return check(st, server=self.h)

    def close_server(self):
        if getattr(self, "h", None):
            _lib.lib().prune_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close_server()
        except Exception:
            pass

    def open(self, F, T, tau, taps, H):
        """Admit a stream; returns its id, or None when the server is full
        (no slot or no room in the budget: retry after a close)."""
        t = _c64_floats(taps).reshape(-1)
        h = _c64_floats(H).reshape(-1)
        d = _lib.prune_graph_desc(F=F, B=self.B, T=T, N=self.N, C=1, out_frames=1, tau=float(tau),
                                  taps=t.ctypes.data, H=h.ctypes.data, stream=None, device=-1, reserved=0,
                                  hbm_budget=0)
        sid = ctypes.c_int64()
        st = _lib.lib().prune_server_open(self.h, ctypes.byref(d), ctypes.byref(sid))
        if st == _lib.PRUNE_EAGAIN:
            return None
        self._check(st)
        self._F[sid.value] = F
        self._x[sid.value] = []
        return sid.value

    def submit(self, sid, x, n=None, period=None):
        """Queue frames: x is a CUDA complex64 tensor holding `period` frames
        of F*B samples; n frames are read cyclically (default n = period =
        all frames in x)."""
        F = self._F[sid]
        assert x.is_cuda and x.dtype == torch.complex64 and x.is_contiguous()
        have = x.numel() // (F * self.B)
        period = have if period is None else period
        n = period if n is None else n
        assert 1 <= period <= have
        self._x[sid].append(x)
        self._check(_lib.lib().prune_server_submit(self.h, sid, x.data_ptr(), n, period))

    def step(self):
        n = ctypes.c_int32()
        self._check(_lib.lib().prune_server_step(self.h, ctypes.byref(n)))
        return n.value

    def progress(self, sid):
        v = [ctypes.c_int64() for _ in range(4)]
        self._check(_lib.lib().prune_server_progress(self.h, sid, *[ctypes.byref(a) for a in v]))
        return tuple(a.value for a in v)   # queued, fired, done, pulled

    def poll(self, max_n=1024):
        ids = (ctypes.c_int64 * max_n)()
        ts = (ctypes.c_int64 * max_n)()
        n = ctypes.c_int32()
        self._check(_lib.lib().prune_server_poll(self.h, ids, ts, max_n, ctypes.byref(n)))
        return [(ids[i], ts[i]) for i in range(n.value)]

    def pull(self, sid, discard=False):
        """Oldest done frame: (frame, c, idx, y[c, B]) or None if none is
        waiting; with discard=True only the slot is freed (returns frame)."""
        F = self._F[sid]
        rec = _lib.prune_frame_out()
        if discard:
            st = _lib.lib().prune_server_pull(self.h, sid, ctypes.byref(rec), _lib.PRUNE_MEM_DISCARD)
            if st == _lib.PRUNE_EAGAIN:
                return None
            self._check(st)
            return rec.frame
        idx = np.zeros(F, np.int32)
        y = np.zeros((F, self.B), np.complex64)
        rec.idx = idx.ctypes.data
        rec.y = y.ctypes.data
        st = _lib.lib().prune_server_pull(self.h, sid, ctypes.byref(rec), _lib.PRUNE_MEM_HOST)
        if st == _lib.PRUNE_EAGAIN:
            return None
        self._check(st)
        return rec.frame, rec.c, idx[:rec.c].copy(), y[:rec.c].copy()

    def close(self, sid):
        self._check(_lib.lib().prune_server_close(self.h, sid))
        self._F.pop(sid, None)
        # inputs stay referenced until the stream's memory is reclaimed; the
        # library keeps no pointer to them after the last step completes
        self._retired = getattr(self, "_retired", [])
        self._retired.append(self._x.pop(sid, []))
        if len(self._retired) > 4096:
            self.sync()
            self._retired.clear()

    def sync(self):
        self._check(_lib.lib().prune_server_sync(self.h))

    def stats(self):
        used, budget = ctypes.c_uint64(), ctypes.c_uint64()
        nopen, steps = ctypes.c_int32(), ctypes.c_int64()
        self._check(_lib.lib().prune_server_stats(self.h, ctypes.byref(used), ctypes.byref(budget),
                                                  ctypes.byref(nopen), ctypes.byref(steps)))
        return {"hbm_used": used.value, "hbm_budget": budget.value, "open": nopen.value, "steps": steps.value}


__all__ = ["Server", "PruneError"]
