"""Reverse-mode differentiation of the firing path over its control trace.

The decisions v[b] = E_b > tau (DET) are piecewise constant in the taps and
H, so the derivative of the sink output is taken with the control trace of
the forward firing (c, idx) held fixed: the DPG of every inactive block
fires zero times and passes no gradient, and for the active ones the output
is linear in H (HX_b, Sec. V) and, through the FIR, in the taps.  Both
adjoints run in the library's kernels (prune_hx_adjoint, prune_fir_adjoint);
this module marshals arguments and plugs them into torch.autograd.

Gradients follow torch's convention for a real loss of complex tensors,
grad = dL/dRe + i dL/dIm, which is also the kernels' convention.
"""
from __future__ import annotations

import torch

from . import _lib
from ._lib import check
from .graph import _stream_ptr, det_sel, fir_energy, hx


def hx_adjoint(y, idx, c, H, gout, F, B, N, gH=None, stream=None):
    """(gy, gH): gy [frames, F*B] holds H^H g_z on the selected blocks and
    zeros elsewhere; gH [N, N] = sum g_z w^H (accumulated into `gH` if
    given)."""
    y = y.contiguous()
    frames = y.shape[0]
    gy = torch.zeros_like(y)
    if gH is None:
        gH = torch.zeros(N, N, dtype=torch.complex64, device=y.device)
    H = H.to(y.device, torch.complex64).contiguous()
    gout = gout.to(torch.complex64).contiguous()
    check(_lib.lib().prune_hx_adjoint(y.data_ptr(), idx.contiguous().data_ptr(), c.contiguous().data_ptr(),
                                      F, B, N, frames, H.data_ptr(), gout.data_ptr(), gy.data_ptr(),
                                      gH.data_ptr(), _stream_ptr(stream)))
    return gy, gH


def fir_adjoint(x, gy, F, B, T, hist=None, gtaps=None, stream=None):
    """gtaps [T] += sum_n gy[n] conj(x[n-t]) over the frames as one stream."""
    x = x.contiguous()
    frames = x.shape[0]
    if gtaps is None:
        gtaps = torch.zeros(T, dtype=torch.complex64, device=x.device)
    gy = gy.contiguous()
    hist_p = hist.contiguous().data_ptr() if (hist is not None and T > 1) else None
    check(_lib.lib().prune_fir_adjoint(x.data_ptr(), hist_p, gy.data_ptr(), F, B, T, frames,
                                       gtaps.data_ptr(), _stream_ptr(stream)))
    return gtaps


class PruneFire(torch.autograd.Function):
    """out, c, idx = PruneFire.apply(taps, H, x, hist, F, B, T, N, tau, store)

    Forward fires FIR (with the delay token `hist`), DET, SEL and HX_b over
    the frames x [frames, F*B] and returns the compacted sink output (first
    c[k]*B samples of frame k valid, zeros after) with the control trace.
    Backward differentiates `out` w.r.t. taps and H over that trace.  With
    store=True the FIR output is kept from the forward pass (F*B*8 bytes per
    frame of HBM); with store=False only the inputs are kept and the FIR output
    is recomputed in the backward pass.
    """

    @staticmethod
    def forward(ctx, taps, H, x, hist, F, B, T, N, tau, store):
        y, e, _ = fir_energy(x, taps, F, B, T, hist=hist)
        c, idx = det_sel(e, tau)
        out = hx(y, idx, c, H, F, B, N)
        ctx.shape = (F, B, T, N)
        ctx.store = bool(store)
        ctx.mark_non_differentiable(c, idx)
        saved_y = y if store else None
        ctx.save_for_backward(taps, H, x, hist if hist is not None else torch.empty(0, device=x.device),
                              c, idx, saved_y if saved_y is not None else torch.empty(0, device=x.device))
        return out, c, idx

    @staticmethod
    def backward(ctx, gout, _gc, _gidx):
        taps, H, x, hist, c, idx, y = ctx.saved_tensors
        F, B, T, N = ctx.shape
        hist = hist if hist.numel() else None
        if not ctx.store:
            y, _, _ = fir_energy(x, taps, F, B, T, hist=hist)   # recompute the FIR output
        if gout is None:
            gout = torch.zeros_like(y)
        gy, gH = hx_adjoint(y, idx, c, H, gout, F, B, N)
        gt = fir_adjoint(x, gy, F, B, T, hist=hist)
        return (gt if ctx.needs_input_grad[0] else None, gH if ctx.needs_input_grad[1] else None,
                None, None, None, None, None, None, None, None)


def fire(taps, H, x, hist=None, *, F, B, T, N, tau, store=True):
    """Differentiable firing of `x` [frames, F*B] (complex64, CUDA): returns
    (out, c, idx) as PruneFire."""
    return PruneFire.apply(taps, H, x, hist, F, B, T, N, float(tau), store)


def scatter(out, c, idx, F, B):
    """Compacted sink output -> [frames, F, B] with the selected blocks at
    their places and zeros elsewhere (torch indexing, differentiable; the
    graph exists even when no block is selected)."""
    frames = out.shape[0]
    j = torch.arange(F, device=out.device)
    sel = j[None, :] < c[:, None].long()                       # slot j of frame k holds a block
    k, jj = sel.nonzero(as_tuple=True)
    src = k * F + jj
    dst = k * F + idx[k, jj].long()
    rows = out.reshape(frames * F, B)[src]
    scat = torch.zeros(frames * F, B, dtype=out.dtype, device=out.device).index_copy(0, dst, rows)
    return scat.view(frames, F, B)
