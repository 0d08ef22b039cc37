"""Differentiation form on the GPU: the adjoint kernels behind
torch.autograd against the FP64 oracle gradient (itself pinned to central
differences) and against central differences of the FP64 loss directly, over
the control trace recorded in the forward pass, with the FIR output stored or
recomputed."""
import numpy as np
import pytest
import torch

import oracle
from oracle import grad as OG
from parity import GUARD_REL
from paper_1802_06625_b300 import synth

pytestmark = pytest.mark.gpu

REL = 1e-3   # relative error bound of the FP32 gradients (norm-wise)


@pytest.fixture(scope="module")
def AD():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1802_06625_b300 import autodiff
    return autodiff


def _problem(w, frames, with_hist):
    x = w.frames_tensor(0, frames).numpy()                      # [n, F, B] complex64
    taps = w.taps().numpy()
    H = w.H().numpy()
    tt = synth.taps(synth.DIFF_TARGET_SEED, w.T).numpy()
    Ht = synth.hmat(synth.DIFF_TARGET_SEED, w.N).numpy()
    rng = np.random.default_rng(w.seed + 100)
    hist = ((rng.standard_normal(w.T - 1) + 1j * rng.standard_normal(w.T - 1)) / np.sqrt(2)).astype(np.complex64) \
        if with_hist else None
    tau = np.float32(w.tau)
    # the target graph's own sink output, fired by the oracle
    rt = oracle.run(w.F, w.B, w.T, w.N, tau, tt, Ht, x, hist_in=hist)
    target = oracle.scatter(rt, w.F, w.B)
    # the trace of the graph being trained, fired by the oracle
    r = oracle.run(w.F, w.B, w.T, w.N, tau, taps, H, x, hist_in=hist)
    e = np.asarray(r.energy, np.float64)
    assert np.all(np.abs(e - tau) > GUARD_REL * tau), "a block energy falls in the guard band"
    return x, taps, H, hist, target, r


def _gpu_grad(AD, w, x, taps, H, hist, target, store):
    dev = "cuda"
    t = torch.from_numpy(taps).to(dev).requires_grad_(True)
    h = torch.from_numpy(H).to(dev).requires_grad_(True)
    xt = torch.from_numpy(x.reshape(x.shape[0], -1)).to(dev)
    ht = torch.from_numpy(hist).to(dev) if hist is not None else None
    out, c, idx = AD.fire(t, h, xt, ht, F=w.F, B=w.B, T=w.T, N=w.N, tau=w.tau, store=store)
    scat = AD.scatter(out, c, idx, w.F, w.B)
    d = scat - torch.from_numpy(target.astype(np.complex64)).to(dev)
    loss = (d.real.square() + d.imag.square()).sum()
    loss.backward()
    torch.cuda.synchronize()
    return float(loss.detach()), t.grad.cpu().numpy(), h.grad.cpu().numpy(), c.cpu().numpy(), idx.cpu().numpy()


def _rel(a, b):
    return np.linalg.norm(np.asarray(a, np.complex128) - b) / np.linalg.norm(b)


@pytest.mark.parametrize("store", [True, False])
def test_gradient_matches_oracle_on_the_differentiation_workload(AD, store):
    w = synth.DIFF
    x, taps, H, hist, target, r = _problem(w, w.frames, with_hist=False)
    L, gt, gH, c, idx = _gpu_grad(AD, w, x, taps, H, None, target, store)
    # the control trace is integer work: bit-exact against the oracle
    assert np.array_equal(c, np.asarray(r.c))
    for k in range(w.frames):
        assert np.array_equal(idx[k, :c[k]], np.asarray(r.idx[k]))
    Lo, gto, gHo = OG.grad_fixed_trace(x, taps.astype(np.complex128), H.astype(np.complex128), r.idx, target)
    assert abs(L - Lo) <= REL * Lo
    assert _rel(gt, gto) <= REL, _rel(gt, gto)
    assert _rel(gH, gHo) <= REL, _rel(gH, gHo)


def test_store_and_recompute_agree(AD):
    w = synth.DIFF
    x, taps, H, hist, target, r = _problem(w, 20, with_hist=True)
    a = _gpu_grad(AD, w, x, taps, H, hist, target, True)
    b = _gpu_grad(AD, w, x, taps, H, hist, target, False)
    assert a[0] == b[0]
    # the recompute fires the same FIR kernel on the same inputs: same y, so
    # only the order of the FP32 atomic sums can differ
    assert _rel(a[1], b[1].astype(np.complex128)) <= 1e-5
    assert _rel(a[2], b[2].astype(np.complex128)) <= 1e-5


def test_gradient_matches_central_differences_with_delay_token(AD):
    # a small case with a nonzero delay token: GPU gradient against FP64
    # central differences of the loss (sampled coordinates) and against the
    # oracle gradient (all coordinates)
    w = synth.PlainWorkload("diff_small", F=8, B=64, T=17, N=16, frames=4, tau=4.0 * 64, seed=11, p=0.4)
    x, taps, H, hist, target, r = _problem(w, w.frames, with_hist=True)
    L, gt, gH, c, idx = _gpu_grad(AD, w, x, taps, H, hist, target, False)
    assert np.array_equal(c, np.asarray(r.c)) and 0 < c.sum() < w.F * w.frames
    t64, H64, h64 = taps.astype(np.complex128), H.astype(np.complex128), hist.astype(np.complex128)
    Lo, gto, gHo = OG.grad_fixed_trace(x, t64, H64, r.idx, target, h64)
    assert _rel(gt, gto) <= REL and _rel(gH, gHo) <= REL
    ft = lambda z: OG.loss_fixed_trace(x, z, H64, r.idx, target, h64)  # noqa: E731
    fH = lambda z: OG.loss_fixed_trace(x, t64, z, r.idx, target, h64)  # noqa: E731
    scale_t, scale_H = np.abs(gto).max(), np.abs(gHo).max()
    for i in (0, 1, 8, 16):
        fd = OG.central_difference(ft, t64, i, 1e-3)
        assert abs(gt[i] - fd) <= REL * scale_t, (i, gt[i], fd)
    for i in (0, 17, 100, 255):
        fd = OG.central_difference(fH, H64, i, 1e-3)
        assert abs(gH.flat[i] - fd) <= REL * scale_H, (i, gH.flat[i], fd)


def test_no_selected_block_gives_zero_gradient(AD):
    w = synth.PlainWorkload("diff_none", F=8, B=64, T=8, N=8, frames=3, tau=1e12, seed=12, p=0.0)
    x, taps, H, hist, target, r = _problem(w, w.frames, with_hist=False)
    L, gt, gH, c, idx = _gpu_grad(AD, w, x, taps, H, None, target, True)
    assert c.sum() == 0 and np.all(gt == 0) and np.all(gH == 0)


def test_adjoint_entry_points_reject_bad_shapes(AD):
    from paper_1802_06625_b300._lib import PruneError
    y = torch.zeros(1, 64, dtype=torch.complex64, device="cuda")
    c = torch.zeros(1, dtype=torch.int32, device="cuda")
    idx = torch.zeros(1, 8, dtype=torch.int32, device="cuda")
    with pytest.raises(PruneError):
        AD.hx_adjoint(y, idx, c, torch.zeros(7, 7, dtype=torch.complex64), y, 8, 8, 7)  # N does not divide B
    with pytest.raises(PruneError):
        AD.fir_adjoint(y, y, 8, 8, 10)                                                   # T - 1 > B
