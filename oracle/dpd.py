"""Oracle for the Dynamic Predistortion graph (test infrastructure only).

Sec. VII-A2 describes DPD as ten parallel ten-tap complex FIR filters whose
active set a configuration actor picks from an external input once every
65536 samples (2 to 10 filters active); a polynomial actor feeds the
filters and an adder merges them.  The figure is missing from the source;
this oracle follows these readings:

  branch k = 1..K carries the memory-polynomial basis psi_k(x) = x |x|^(k-1);
  FIR_k filters psi_k with its own taps h_k[0..T) and its own delay token
  (the last T-1 samples of psi_k it consumed; T-1 zeros initially);
  in a period where branch k is inactive its DC does not fire (itr = 0, Sec.
  III-A), so its delay token stays as it was until it fires again;
  the adder sums the outputs of the active branches (zeros if none).

`run` fires the graph period by period, in order, in FP64 from the FP32
inputs (numpy convolution per branch and period)."""
from __future__ import annotations

import numpy as np


def psi(x, k):
    """Basis k >= 1 of the memory polynomial: x |x|^(k-1)."""
    x = np.asarray(x, np.complex128)
    return x * np.abs(x) ** (k - 1)


def run(x, masks, taps, period, hist=None):
    """x: complex [P * period]; masks: int [P], bit k-1 set = branch k active
    in that period; taps: complex [K, T]; hist: complex [K, T-1] initial
    delay tokens (zeros if None).  Returns (y complex128 [P * period],
    hist_out [K, T-1])."""
    x = np.asarray(x, np.complex128)
    taps = np.asarray(taps, np.complex128)
    K, T = taps.shape
    P = len(masks)
    assert x.size == P * period and period >= T - 1
    h = np.zeros((K, T - 1), np.complex128) if hist is None else np.array(hist, np.complex128).reshape(K, T - 1)
    y = np.zeros(P * period, np.complex128)
    for p in range(P):
        seg = x[p * period:(p + 1) * period]
        for k in range(K):
            if not (int(masks[p]) >> k) & 1:
                continue                                  # DC k does not fire this period
            u = psi(seg, k + 1)
            full = np.concatenate([h[k], u])
            y[p * period:(p + 1) * period] += np.convolve(full, taps[k])[T - 1:T - 1 + period]
            if T > 1:
                h[k] = full[full.size - (T - 1):]          # the delay token FIR_k produced
    return y, h
