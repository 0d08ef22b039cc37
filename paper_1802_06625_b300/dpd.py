"""Python view of the Dynamic Predistortion workload (prune_dpd_fire):
argument marshalling only; the branches fire in the library's kernels."""
from __future__ import annotations

import torch

from . import _lib
from ._lib import check
from .graph import _stream_ptr


def fire(x, masks, taps, period, hist=None, hist_out=None, y=None, stream=None):
    """x: CUDA complex64 [P * period]; masks: CUDA uint16-compatible [P]
    (bit k-1 = branch k fires); taps: complex64 [K, T]; hist: [K, T-1] tokens
    before the first period (None = zeros).  Returns (y, hist_out); hist_out
    may be hist itself (in-place token update)."""
    dev = x.device
    x = x.contiguous()
    P = x.numel() // period
    assert P * period == x.numel()
    taps = taps.to(dev, torch.complex64).contiguous()
    K, T = taps.shape
    m = masks.to(dev).to(torch.int32).to(torch.int16).contiguous()   # low 16 bits, as uint16
    if y is None:
        y = torch.empty_like(x)
    if hist_out is None and T > 1:
        hist_out = torch.empty(K, T - 1, dtype=torch.complex64, device=dev)
    ws = torch.empty(_lib.lib().prune_dpd_workspace_bytes(P, K), dtype=torch.uint8, device=dev)
    check(_lib.lib().prune_dpd_fire(x.data_ptr(), period, P, m.data_ptr(), K, T, taps.data_ptr(),
                                    hist.contiguous().data_ptr() if hist is not None else None,
                                    hist_out.data_ptr() if hist_out is not None else None, y.data_ptr(),
                                    ws.data_ptr(), ws.numel(), _stream_ptr(stream)))
    return y, hist_out
