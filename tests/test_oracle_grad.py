"""The differentiation oracle pinned: its fixed-trace forward equals the C
dataflow simulator on the simulator's own trace, and its adjoint gradients
equal FP64 central finite differences (exact up to roundoff: the loss is
quadratic in every single coordinate)."""
import numpy as np

import oracle
from oracle import grad as OG


def _rc(rng, *shape, scale=1.0):
    return (scale * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2)).astype(np.complex64)


def _setup(seed=0, F=6, B=32, T=8, N=8, n=3):
    rng = np.random.default_rng(seed)
    x = _rc(rng, n, F, B)
    x[:, ::2] *= 4
    taps = _rc(rng, T, scale=1 / np.sqrt(T))
    H = _rc(rng, N, N, scale=1 / np.sqrt(N))
    return rng, x, taps, H


def test_fixed_trace_forward_equals_the_simulator():
    rng, x, taps, H = _setup(1)
    F, B, T, N = 6, 32, 8, 8
    r = oracle.run(F, B, T, N, 250.0, taps, H, x)
    assert 0 < sum(r.c) < 3 * F
    out = OG.forward_fixed_trace(x, taps.astype(np.complex128), H.astype(np.complex128), r.idx)
    assert np.allclose(out, oracle.scatter(r, F, B), atol=1e-12, rtol=0)
    hist = _rc(rng, T - 1).astype(np.complex128)
    r2 = oracle.run(F, B, T, N, 250.0, taps, H, x, hist_in=hist)
    out2 = OG.forward_fixed_trace(x, taps.astype(np.complex128), H.astype(np.complex128), r2.idx, hist=hist)
    assert np.allclose(out2, oracle.scatter(r2, F, B), atol=1e-12, rtol=0)


def test_adjoint_equals_central_differences():
    rng, x, taps, H = _setup(2)
    taps = taps.astype(np.complex128)
    H = H.astype(np.complex128)
    idx = [np.array([0, 2, 3]), np.array([], np.int64), np.array([1, 4, 5])]
    target = _rc(rng, 3, 6, 32).astype(np.complex128)
    hist = _rc(rng, 7).astype(np.complex128)
    L, gt, gH = OG.grad_fixed_trace(x, taps, H, idx, target, hist)
    assert L > 0
    ft = lambda z: OG.loss_fixed_trace(x, z, H, idx, target, hist)  # noqa: E731
    fH = lambda z: OG.loss_fixed_trace(x, taps, z, idx, target, hist)  # noqa: E731
    for t in range(len(taps)):
        fd = OG.central_difference(ft, taps, t, 1e-2)
        assert abs(fd - gt[t]) <= 1e-9 * max(1.0, abs(gt[t])), (t, fd, gt[t])
    for i in range(H.size):
        fd = OG.central_difference(fH, H, i, 1e-2)
        assert abs(fd - gH.flat[i]) <= 1e-9 * max(1.0, abs(gH.flat[i])), (i, fd, gH.flat[i])


def test_unselected_blocks_carry_no_gradient():
    rng, x, taps, H = _setup(3)
    taps = taps.astype(np.complex128)
    H = H.astype(np.complex128)
    idx = [np.array([], np.int64)] * 3
    L, gt, gH = OG.grad_fixed_trace(x, taps, H, idx, np.zeros((3, 6, 32)))
    assert L == 0 and np.all(gt == 0) and np.all(gH == 0)
