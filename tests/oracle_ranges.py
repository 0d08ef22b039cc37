"""Oracle workers for the full-size control checks (test code only).

Frames of a stream depend on each other only through the delay token (the
last T-1 input samples of the frame before), so each frame can be fired by
the oracle on its own, fed the tail of the frame before it.  The caller
draws the frames with the seeded generator and sends each task its frame;
a worker only runs the FP64 oracle and returns the control (c, idx,
energies).  Used from a process pool started with the spawn method.
"""
import numpy as np

import oracle


def fire_frame(task):
    """task = (k, F, B, T, N, tau, taps, H, x [F, B] complex64, hist or None)
    -> (k, c, idx, energy)."""
    k, F, B, T, N, tau, taps, H, x, hist = task
    r = oracle.run(F, B, T, N, np.float32(tau), taps, H, np.asarray(x)[None], hist_in=hist)
    return int(k), int(r.c[0]), np.asarray(r.idx[0], np.int32), np.asarray(r.energy[0], np.float64)


def fire_instance(task):
    """task = (i, F, B, T, N, tau, taps, H, x [F, B] complex64): frame 0 of
    an instance with a zero delay token -> (i, c, idx, energy, y)."""
    i, F, B, T, N, tau, taps, H, x = task
    r = oracle.run(F, B, T, N, np.float32(tau), taps, H, np.asarray(x)[None])
    return (int(i), int(r.c[0]), np.asarray(r.idx[0], np.int32), np.asarray(r.energy[0], np.float64),
            np.asarray(r.y[0]))
