"""Oracle for the differentiation form (test infrastructure only).

With the control trace fixed (the decisions v[b] = E_b > tau are piecewise
constant in the parameters, so their derivative is zero almost everywhere),
the sink output of the canonical graph is linear in H and, through the FIR,
linear in the taps h.  For a real loss L of the scattered sink output and the
complex-gradient convention g = dL/dRe + i dL/dIm:

  HX_b (Sec. V, one DC per block):  z = H w  for every selected row w
      dL/dH = sum over selected rows of g_z w^H,   g_w = H^H g_z
  FIR:  y[n] = sum_t h[t] x[n-t]
      dL/dh[t] = sum_n g_y[n] conj(x[n-t]),  g_y = g_w on selected blocks, 0 elsewhere

This module computes the forward pass with a given trace in FP64 (numpy
convolution and einsum), the L2 loss against a target record, and the
gradient by the formulas above.  It is pinned by central finite differences
of `loss_fixed_trace` (exact up to roundoff, the loss being quadratic in
every single coordinate).
"""
from __future__ import annotations

import numpy as np


def fir_stream(x, taps, hist=None):
    """y[n] = sum_t h[t] x[n-t] over frames x [n, F, B] as one stream; the
    T-1 samples before frame 0 are `hist` (zeros if None)."""
    n, F, B = x.shape
    T = len(taps)
    s = x.reshape(-1).astype(np.complex128)
    pre = np.zeros(T - 1, np.complex128) if hist is None else np.asarray(hist, np.complex128)
    full = np.concatenate([pre, s])
    y = np.convolve(full, np.asarray(taps, np.complex128))[T - 1:T - 1 + s.size]
    return y.reshape(n, F, B)


def forward_fixed_trace(x, taps, H, idx, hist=None):
    """Scattered sink output [n, F, B] for the selected blocks idx[k] of each
    frame (zeros elsewhere): HX applied to the row-major (B/N, N) rows."""
    N = H.shape[0]
    y = fir_stream(x, taps, hist)
    n, F, B = y.shape
    out = np.zeros_like(y)
    Hc = np.asarray(H, np.complex128)
    for k in range(n):
        sel = np.asarray(idx[k], np.int64)
        if sel.size:
            X = y[k, sel].reshape(sel.size, B // N, N)
            out[k, sel] = np.einsum("ik,bjk->bji", Hc, X).reshape(sel.size, B)
    return out


def loss_fixed_trace(x, taps, H, idx, target, hist=None):
    """L = sum |S(out) - S(out*)|^2 over the scattered frames."""
    d = forward_fixed_trace(x, taps, H, idx, hist) - np.asarray(target, np.complex128)
    return float(np.sum(np.abs(d) ** 2))


def grad_fixed_trace(x, taps, H, idx, target, hist=None):
    """(L, dL/dtaps [T], dL/dH [N, N]) by the adjoint formulas."""
    N = H.shape[0]
    Hc = np.asarray(H, np.complex128)
    y = fir_stream(x, taps, hist)
    n, F, B = y.shape
    out = forward_fixed_trace(x, taps, H, idx, hist)
    d = out - np.asarray(target, np.complex128)
    L = float(np.sum(np.abs(d) ** 2))
    g_out = 2.0 * d                      # dL/dRe + i dL/dIm of the scattered output
    gH = np.zeros((N, N), np.complex128)
    gy = np.zeros_like(y)
    for k in range(n):
        sel = np.asarray(idx[k], np.int64)
        if not sel.size:
            continue
        G = g_out[k, sel].reshape(sel.size, B // N, N)   # rows of g_z
        W = y[k, sel].reshape(sel.size, B // N, N)       # rows of w
        gH += np.einsum("bji,bjk->ik", G, W.conj())
        gy[k, sel] = np.einsum("ik,bji->bjk", Hc.conj(), G).reshape(sel.size, B)
    T = len(taps)
    s = x.reshape(-1).astype(np.complex128)
    pre = np.zeros(T - 1, np.complex128) if hist is None else np.asarray(hist, np.complex128)
    full = np.concatenate([pre, s])
    g = gy.reshape(-1)
    gt = np.array([np.sum(g * full[T - 1 - t:T - 1 - t + s.size].conj()) for t in range(T)])
    return L, gt, gH


def central_difference(fun, z, i, step):
    """Central differences of real fun at complex parameter coordinate i:
    returns dL/dRe + i dL/dIm."""
    z1 = z.copy(); z1.flat[i] += step
    z2 = z.copy(); z2.flat[i] -= step
    dre = (fun(z1) - fun(z2)) / (2 * step)
    z1 = z.copy(); z1.flat[i] += 1j * step
    z2 = z.copy(); z2.flat[i] -= 1j * step
    dim = (fun(z1) - fun(z2)) / (2 * step)
    return dre + 1j * dim
