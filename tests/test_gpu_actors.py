"""GPU parity of each actor through the C ABI against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from parity import TOL_REL, compare_frame, in_band
from paper_1802_06625_b300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1802_06625_b300 import graph
    return graph


def _rc(rng, *shape, scale=1.0):
    return (scale * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2)).astype(np.complex64)


def _oracle_fir(x, taps, hist=None):
    """FP64 direct convolution of the stream (numpy library primitive is the
    oracle's pinned FIR; here the oracle graph with H = I, tau = -1 gives it)."""
    n, F, B = x.shape
    r = oracle.run(F, B, len(taps), 1, -1.0, taps, np.eye(1, dtype=np.complex64), x, hist_in=hist)
    return oracle.scatter(r, F, B), r


@pytest.mark.parametrize("F,B,T,frames", [(4, 256, 16, 3), (3, 64, 5, 4), (1, 8, 1, 2), (2, 2048, 256, 2),
                                          (5, 1024, 64, 2), (7, 768, 33, 2), (33, 128, 128, 2), (1, 16, 17, 3)])
def test_fir_energy_matches_oracle(G, F, B, T, frames):
    rng = np.random.default_rng(F * 1000 + B + T)
    x = _rc(rng, frames, F, B)
    taps = _rc(rng, T, scale=1 / np.sqrt(T))
    hist = _rc(rng, max(T - 1, 1))[:T - 1]
    yo, r = _oracle_fir(x, taps, hist=hist.astype(np.complex128) if T > 1 else None)
    xd = torch.from_numpy(x.reshape(frames, F * B)).cuda()
    hd = torch.from_numpy(hist).cuda() if T > 1 else None
    y, e, hout = G.fir_energy(xd, torch.from_numpy(taps), F, B, T, hist=hd)
    torch.cuda.synchronize()
    y = y.cpu().numpy().reshape(frames, F, B).astype(np.complex128)
    rms = np.sqrt(np.mean(np.abs(yo) ** 2))
    assert np.max(np.abs(y - yo)) <= TOL_REL * rms
    eo = r.energy
    assert np.max(np.abs(e.cpu().numpy() - eo) / np.maximum(eo, 1e-30)) < 1e-5
    if T > 1:
        assert np.array_equal(hout.cpu().numpy(), x[-1].reshape(-1)[-(T - 1):])


def test_fir_impulse_gives_taps_exactly(G):
    F, B, T = 2, 64, 16
    rng = np.random.default_rng(0)
    taps = _rc(rng, T)
    x = np.zeros((2, F * B), np.complex64)
    x[0, 0] = 1.0
    x[1, F * B - 1] = 1.0      # rings into nothing: last sample of the stream
    y, e, _ = G.fir_energy(torch.from_numpy(x).cuda(), torch.from_numpy(taps), F, B, T)
    y = y.cpu().numpy()
    assert np.array_equal(y[0, :T], taps)         # h[t] * 1 + zeros, exact in FP32
    assert np.all(y[0, T:] == 0)


def test_fir_energies_only(G):
    rng = np.random.default_rng(3)
    F, B, T = 16, 256, 32
    x = _rc(rng, 2, F, B)
    taps = _rc(rng, T, scale=1 / np.sqrt(T))
    _, r = _oracle_fir(x, taps)
    y, e, _ = G.fir_energy(torch.from_numpy(x.reshape(2, -1)).cuda(), torch.from_numpy(taps), F, B, T, want_y=False)
    assert y is None
    assert np.allclose(e.cpu().numpy(), r.energy, rtol=1e-5)


@pytest.mark.parametrize("F", [1, 31, 32, 33, 1000, 1024, 1025, 4096, 5000])
def test_det_sel_compaction_is_exact(G, F):
    rng = np.random.default_rng(F)
    frames = 3
    e = rng.exponential(1.0, (frames, F)).astype(np.float32)
    tau = np.float32(1.0)
    c, idx = G.det_sel(torch.from_numpy(e).cuda(), float(tau))
    c, idx = c.cpu().numpy(), idx.cpu().numpy()
    for k in range(frames):
        want = np.nonzero(e[k] > tau)[0]    # same FP32 decision as the kernel
        assert c[k] == len(want)
        assert np.array_equal(idx[k, :c[k]], want)
        assert np.all(idx[k, c[k]:] == -1)   # untouched past c


def test_det_sel_extremes(G):
    e = np.array([[0.0, 1.0, 2.0, np.inf], [np.nan, 5.0, -1.0, 0.5]], np.float32)
    c, idx = G.det_sel(torch.from_numpy(e).cuda(), -np.inf)
    assert list(c.cpu().numpy()) == [4, 3]          # NaN never selected
    c, idx = G.det_sel(torch.from_numpy(e).cuda(), np.inf)
    assert list(c.cpu().numpy()) == [0, 0]
    c, idx = G.det_sel(torch.from_numpy(e).cuda(), 1.0)
    assert list(c.cpu().numpy()) == [2, 1] and list(idx.cpu().numpy()[0, :2]) == [2, 3]


def _oracle_hx(y, sel, H, F, B, N):
    """HX_b of the oracle on the given blocks: frames y [frames, F, B] fired
    through the oracle's graph with one unit tap (the FIR is the identity,
    T = 1) and tau between the energies of the chosen blocks and of the
    others (the others are scaled down by 1e-3 beforehand), so DET selects
    exactly `sel[k]`.  Returns the oracle's compacted outputs per frame."""
    frames = y.shape[0]
    x = y.copy()
    for k in range(frames):
        mask = np.ones(F, bool)
        mask[sel[k]] = False
        x[k, mask] *= np.float32(1e-3)
    tau = np.float32(1e-3 * B)       # selected blocks: E ~ B, the others: E ~ 1e-6 B
    r = oracle.run(F, B, 1, N, tau, np.ones(1, np.complex64), H, x.astype(np.complex64))
    for k in range(frames):
        assert np.array_equal(np.asarray(r.idx[k]), sel[k])
    return x, r


@pytest.mark.parametrize("N,B", [(1, 64), (2, 64), (4, 256), (8, 256), (16, 256), (32, 1024), (12, 96 * 8), (24, 768),
                                 (64, 64), (64, 256), (64, 512), (64, 2048)])
def test_hx_matches_oracle(G, N, B):
    rng = np.random.default_rng(N * 7 + B)
    F, frames = 9, 2
    y = _rc(rng, frames, F, B)
    H = _rc(rng, N, N, scale=1 / np.sqrt(N))
    sel = [np.sort(rng.choice(F, size=s, replace=False)) for s in (4, 0)]
    x, r = _oracle_hx(y, sel, H, F, B, N)
    c = np.array([len(s) for s in sel], np.int32)
    idx = np.full((frames, F), 0, np.int32)
    for k, s in enumerate(sel):
        idx[k, :len(s)] = s
    out = G.hx(torch.from_numpy(x.reshape(frames, -1)).cuda(), torch.from_numpy(idx).cuda(),
               torch.from_numpy(c).cuda(), torch.from_numpy(H), F, B, N).cpu().numpy().reshape(frames, F, B)
    for k in range(frames):
        want = np.asarray(r.y[k])
        got = out[k, :c[k]]
        if c[k]:
            rms = np.sqrt(np.mean(np.abs(want) ** 2))
            assert np.max(np.abs(got - want)) <= TOL_REL * rms
        assert np.all(out[k, c[k]:] == 0)   # nothing written for inactive DCs


@pytest.mark.parametrize("N", [16, 64])
def test_hx_cyclic_shift_is_a_permutation(G, N):
    B, F = 256, 4
    rng = np.random.default_rng(5)
    y = _rc(rng, 1, F, B)
    S = np.zeros((N, N), np.complex64)
    for i in range(N):
        S[i, (i + 1) % N] = 1.0
    c = np.array([F], np.int32)
    idx = np.arange(F, dtype=np.int32)[None]
    out = G.hx(torch.from_numpy(y.reshape(1, -1)).cuda(), torch.from_numpy(idx).cuda(), torch.from_numpy(c).cuda(),
               torch.from_numpy(S), F, B, N).cpu().numpy().reshape(F, B // N, N)
    want = np.roll(y.reshape(F, B // N, N), -1, axis=-1)
    if N < 64:
        assert np.array_equal(out, want)          # one FP32 product by 1.0: exact
    else:
        # three split-FP16 products: the dropped lo*lo term is below 2^-22 relative
        assert np.max(np.abs(out - want)) <= 2.0 ** -20 * np.max(np.abs(want))


def test_hx_tensor_core_many_tiles_and_frames(G):
    """N = 64 on tcgen05 with uneven c per frame: several 128-row tiles, a
    ragged last tile, c = 0 and c = F frames, against the oracle."""
    rng = np.random.default_rng(99)
    N, B, F, frames = 64, 256, 70, 4
    y = _rc(rng, frames, F, B, scale=4.0)
    H = _rc(rng, N, N, scale=1 / np.sqrt(N))
    sel = [np.sort(rng.choice(F, size=s, replace=False)) for s in (33, 0, F, 1)]
    x, r = _oracle_hx(y, sel, H, F, B, N)
    c = np.array([len(s) for s in sel], np.int32)
    idx = np.zeros((frames, F), np.int32)
    for k, s_ in enumerate(sel):
        idx[k, :len(s_)] = s_
    out = G.hx(torch.from_numpy(x.reshape(frames, -1)).cuda(), torch.from_numpy(idx).cuda(),
               torch.from_numpy(c).cuda(), torch.from_numpy(H), F, B, N).cpu().numpy().reshape(frames, F, B)
    for k in range(frames):
        want = np.asarray(r.y[k])
        if c[k]:
            rms = np.sqrt(np.mean(np.abs(want) ** 2))
            assert np.max(np.abs(out[k, :c[k]] - want)) <= TOL_REL * rms
        assert np.all(out[k, c[k]:] == 0)
