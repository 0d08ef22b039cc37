"""Oracle workers for the full-size control checks (test code only).

Frames of a stream depend on each other only through the delay token (the
last T-1 input samples of the frame before), so a range of frames can be
fired by the oracle on its own, fed the tail of the frame before the range.
Each worker regenerates its frames on the host from the seeded generator,
fires them through the FP64 oracle and returns the control of every frame:
(c, idx, energies).  Started from a process pool with the spawn method.
"""
import numpy as np
import torch

import oracle
from paper_1802_06625_b300 import synth


def plain_range(args):
    """Frames [a, b) of the plain-large workload -> [(k, c, idx, energy)]."""
    a, b = args
    torch.set_num_threads(1)
    w = synth.PLAIN_LARGE
    taps, H = w.taps().numpy(), w.H().numpy()
    prev = w.frame(a - 1).numpy().reshape(-1)[-(w.T - 1):] if a > 0 else None
    out = []
    for k in range(a, b):
        x = w.frame(k).numpy()
        r = oracle.run(w.F, w.B, w.T, w.N, np.float32(w.tau), taps, H, x[None], hist_in=prev)
        out.append((k, int(r.c[0]), np.asarray(r.idx[0], np.int32), np.asarray(r.energy[0], np.float64)))
        prev = x.reshape(-1)[-(w.T - 1):]
    return out


def batched_instances(ids):
    """Frame 0 of the listed instances of the batched workload (zero delay
    token) -> [(i, c, idx, energy, y)]."""
    torch.set_num_threads(1)
    b = synth.BATCHED
    out = []
    for i in ids:
        w = b.instance(i)
        r = oracle.run(w.F, w.B, w.T, w.N, np.float32(w.tau), w.taps().numpy(), w.H().numpy(),
                       w.frame(0).numpy()[None])
        out.append((i, int(r.c[0]), np.asarray(r.idx[0], np.int32), np.asarray(r.energy[0], np.float64),
                    np.asarray(r.y[0])))
    return out
