"""Python view of one PRUNE graph instance fired by libprune.so.

Argument marshalling only (torch supplies device memory and streams); the
actors fire in the library's CUDA kernels.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import check


def _c64_floats(a) -> np.ndarray:
    a = a.detach().cpu().numpy() if isinstance(a, torch.Tensor) else np.asarray(a)
    return np.ascontiguousarray(a.astype(np.complex64)).view(np.float32)


class Graph:
    """The canonical graph FIR -> DET -> {SEL, HX_b, SINK} with F blocks of B
    samples per frame, T taps, an N x N matrix H and threshold tau."""

    def __init__(self, F, B, T, N, tau, taps, H, C=3, out_frames=0, stream=None, device=None,
                 hbm_budget=0):
        self.F, self.B, self.T, self.N, self.C = F, B, T, N, C
        self.L = F * B
        self._taps = _c64_floats(taps).reshape(-1)
        self._H = _c64_floats(H).reshape(-1)
        if device is None:
            device = torch.cuda.current_device()
        self.device = device
        self.stream = stream
        d = _lib.prune_graph_desc(F=F, B=B, T=T, N=N, C=C, out_frames=out_frames, tau=float(tau),
                                  taps=self._taps.ctypes.data, H=self._H.ctypes.data,
                                  stream=stream.cuda_stream if stream is not None else None,
                                  device=device, reserved=0, hbm_budget=hbm_budget)
        h = ctypes.c_void_p()
        check(_lib.lib().prune_graph_create(ctypes.byref(d), ctypes.byref(h)))
        self.h = h
        self._borrowed = []   # keep borrowed frames alive until fired

    @classmethod
    def from_desc(cls, desc):
        """A graph made by prune_graph_create from a filled prune_graph_desc
        (e.g. the one prune_model_compile writes)."""
        g = cls.__new__(cls)
        g.F, g.B, g.T, g.N, g.C = desc.F, desc.B, desc.T, desc.N, desc.C
        g.L = desc.F * desc.B
        g.device = desc.device if desc.device >= 0 else torch.cuda.current_device()
        g.stream = None
        h = ctypes.c_void_p()
        check(_lib.lib().prune_graph_create(ctypes.byref(desc), ctypes.byref(h)))
        g.h = h
        g._borrowed = []
        return g

    def close(self):
        if getattr(self, "h", None):
            _lib.lib().prune_graph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- SRC
    def push(self, x, mem=None) -> None:
        """Push frames x [n, F, B] complex64 (torch CUDA tensor, torch CPU tensor
        or numpy array)."""
        if isinstance(x, np.ndarray):
            x = torch.from_numpy(np.ascontiguousarray(x.astype(np.complex64)))
        x = x.contiguous()
        n = x.shape[0] if x.dim() == 3 else 1
        if mem is None:
            mem = _lib.PRUNE_MEM_DEVICE if x.is_cuda else _lib.PRUNE_MEM_HOST
        if mem == _lib.PRUNE_MEM_DEVICE_BORROW:
            self._borrowed.append(x)
        check(_lib.lib().prune_push_frames(self.h, x.data_ptr(), n, mem), self.h)

    # -- all actors
    def run(self, max_frames=1 << 30, sync=False, actors=False, cuda_cores=False) -> int:
        n = ctypes.c_int32()
        flags = ((_lib.PRUNE_RUN_SYNC if sync else 0) | (_lib.PRUNE_RUN_ACTORS if actors else 0)
                 | (_lib.PRUNE_RUN_CUDA_CORES if cuda_cores else 0))
        check(_lib.lib().prune_run(self.h, max_frames, ctypes.byref(n), flags), self.h)
        if sync:
            self._borrowed.clear()
        return n.value

    def sync(self):
        check(_lib.lib().prune_sync(self.h), self.h)
        self._borrowed.clear()

    # -- SINK records
    def pull(self, max_frames=1 << 30):
        """Pop finished records: list of (frame, c, idx int32[c], y complex64[c, B])."""
        out = []
        while len(out) < max_frames:
            k = min(64, max_frames - len(out))
            idx = np.zeros((k, self.F), np.int32)
            y = np.zeros((k, self.F, self.B), np.complex64)
            recs = (_lib.prune_frame_out * k)()
            for i in range(k):
                recs[i].idx = idx[i].ctypes.data
                recs[i].y = y[i].ctypes.data
            n = ctypes.c_int32()
            st = _lib.lib().prune_pull(self.h, recs, k, ctypes.byref(n), _lib.PRUNE_MEM_HOST)
            if st == _lib.PRUNE_EAGAIN:
                break
            check(st, self.h)
            for i in range(n.value):
                c = recs[i].c
                out.append((recs[i].frame, c, idx[i, :c].copy(), y[i, :c].copy()))
            if n.value < k:
                break
        self._borrowed.clear()
        return out

    def discard(self, max_frames=1 << 30) -> int:
        n = ctypes.c_int32()
        st = _lib.lib().prune_pull(self.h, None, max_frames, ctypes.byref(n), _lib.PRUNE_MEM_DISCARD)
        if st == _lib.PRUNE_EAGAIN:
            return 0
        check(st, self.h)
        return n.value

    def fifo_stats(self):
        out = {}
        for f in range(_lib.PRUNE_NUM_FIFOS):
            w, r, p = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
            check(_lib.lib().prune_fifo_stats(self.h, f, ctypes.byref(w), ctypes.byref(r), ctypes.byref(p)), self.h)
            out[f"f{f}"] = (w.value, r.value, p.value)
        return out

    KIND_PUSH, KIND_FIR, KIND_DETSEL, KIND_HX_CUDA, KIND_HX_TC, KIND_LOOP, KIND_LOOP_TC = range(7)

    def profile(self, enable=True):
        check(_lib.lib().prune_profile(self.h, 1 if enable else 0), self.h)

    def kernel_times(self, kind, reset=True):
        """(summed device ms, launches) of one kernel kind since the last reset."""
        ms, n = ctypes.c_double(), ctypes.c_int64()
        check(_lib.lib().prune_kernel_times(self.h, kind, ctypes.byref(ms), ctypes.byref(n), 1 if reset else 0), self.h)
        return ms.value, n.value

    def capacity(self, fifo: int) -> int:
        c = ctypes.c_int64()
        check(_lib.lib().prune_fifo_capacity_of(self.h, fifo, ctypes.byref(c)), self.h)
        return c.value


# --------------------------------------------------------------- single actors

def _stream_ptr(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def fir_energy(x, taps, F, B, T, hist=None, want_y=True, stream=None):
    """x: CUDA complex64 [frames, F*B] -> (y or None, energy [frames, F], hist_out [T-1])."""
    x = x.contiguous()
    frames = x.shape[0]
    dev = x.device
    y = torch.empty_like(x) if want_y else None
    e = torch.empty(frames, F, dtype=torch.float32, device=dev)
    hout = torch.empty(max(T - 1, 1), dtype=torch.complex64, device=dev)
    taps = taps.to(dev, torch.complex64).contiguous()
    check(_lib.lib().prune_fir_energy(x.data_ptr(), hist.data_ptr() if hist is not None else None,
                                      taps.data_ptr(), F, B, T, frames,
                                      y.data_ptr() if y is not None else None, e.data_ptr(),
                                      hout.data_ptr(), _stream_ptr(stream)))
    return y, e, hout[:T - 1]


def det_sel(energy, tau, stream=None):
    energy = energy.contiguous()
    frames, F = energy.shape
    c = torch.zeros(frames, dtype=torch.int32, device=energy.device)
    idx = torch.full((frames, F), -1, dtype=torch.int32, device=energy.device)
    check(_lib.lib().prune_det_sel(energy.data_ptr(), F, frames, float(tau), c.data_ptr(), idx.data_ptr(),
                                   _stream_ptr(stream)))
    return c, idx


def hx(y, idx, c, H, F, B, N, stream=None):
    y = y.contiguous()
    frames = y.shape[0]
    out = torch.zeros_like(y)
    H = H.to(y.device, torch.complex64).contiguous()
    check(_lib.lib().prune_hx(y.data_ptr(), idx.contiguous().data_ptr(), c.contiguous().data_ptr(), F, B, N,
                              frames, H.data_ptr(), out.data_ptr(), _stream_ptr(stream)))
    return out


class Batch:
    """Many independent graph instances fired one frame each per step.
    ``instances``: list of dicts with F, T, tau, taps, H (common B, N)."""

    def __init__(self, B, N, instances, stream=None, device=None):
        self.B, self.N, self.n = B, N, len(instances)
        if device is None:
            device = torch.cuda.current_device()
        self._keep = []
        descs = (_lib.prune_graph_desc * self.n)()
        for i, inst in enumerate(instances):
            taps = _c64_floats(inst["taps"]).reshape(-1)
            H = _c64_floats(inst["H"]).reshape(-1)
            self._keep += [taps, H]
            descs[i] = _lib.prune_graph_desc(F=inst["F"], B=B, T=inst["T"], N=N, C=1, out_frames=1,
                                             tau=float(inst["tau"]), taps=taps.ctypes.data, H=H.ctypes.data,
                                             stream=stream.cuda_stream if (stream is not None and i == 0) else None,
                                             device=device, reserved=0, hbm_budget=0)
        h = ctypes.c_void_p()
        check(_lib.lib().prune_batch_create(descs, self.n, ctypes.byref(h)))
        self.h = h
        self.F = [inst["F"] for inst in instances]
        off, tot = ctypes.c_int64(), ctypes.c_int64()
        self.offsets = []
        for i in range(self.n):
            check(_lib.lib().prune_batch_offset(self.h, i, ctypes.byref(off), ctypes.byref(tot)), batch=self.h)
            self.offsets.append(off.value)
        self.total = tot.value

    def close(self):
        if getattr(self, "h", None):
            _lib.lib().prune_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def fire(self, x, graph=False):
        """x: CUDA complex64 tensor of self.total samples (instances back to back)."""
        assert x.is_cuda and x.numel() == self.total
        self._x = x
        check(_lib.lib().prune_batch_fire(self.h, x.data_ptr(), _lib.PRUNE_BATCH_GRAPH if graph else 0),
              batch=self.h)

    def sync(self):
        check(_lib.lib().prune_batch_sync(self.h), batch=self.h)

    @staticmethod
    def _tuning_dict(t):
        return {"fir_order": t.fir_order, "hx_chunk": t.hx_chunk, "hx_grid": t.hx_grid, "ms": t.ms}

    def autotune(self, x, reps=3):
        """Time every candidate launch shape on one step of x and keep the
        fastest; returns (best, all candidates) as dicts."""
        assert x.is_cuda and x.numel() == self.total
        best = _lib.prune_batch_tuning()
        allc = (_lib.prune_batch_tuning * 16)()
        n = ctypes.c_int32()
        check(_lib.lib().prune_batch_autotune(self.h, x.data_ptr(), reps, ctypes.byref(best), allc, 16,
                                              ctypes.byref(n)), batch=self.h)
        return self._tuning_dict(best), [self._tuning_dict(allc[i]) for i in range(n.value)]

    def set_tuning(self, fir_order=0, hx_chunk=0, hx_grid=0):
        t = _lib.prune_batch_tuning(fir_order=fir_order, hx_chunk=hx_chunk, hx_grid=hx_grid)
        check(_lib.lib().prune_batch_set_tuning(self.h, ctypes.byref(t)), batch=self.h)

    def tuning(self):
        t = _lib.prune_batch_tuning()
        check(_lib.lib().prune_batch_get_tuning(self.h, ctypes.byref(t)), batch=self.h)
        return self._tuning_dict(t)

    def pull(self, i):
        F = self.F[i]
        idx = np.zeros(F, np.int32)
        y = np.zeros((F, self.B), np.complex64)
        rec = _lib.prune_frame_out()
        rec.idx = idx.ctypes.data
        rec.y = y.ctypes.data
        check(_lib.lib().prune_batch_pull(self.h, i, ctypes.byref(rec), _lib.PRUNE_MEM_HOST), batch=self.h)
        return rec.frame, rec.c, idx[:rec.c].copy(), y[:rec.c].copy()
