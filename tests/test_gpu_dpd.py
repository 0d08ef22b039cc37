"""DPD workload on the GPU against the FP64 oracle: uneven and empty active
sets, branches that sit out periods and resume from their stale delay
tokens, tokens handed over between calls (in place), the generic tap count,
and the 67 M-sample stream on sampled periods."""
import numpy as np
import pytest
import torch

from oracle import dpd as D
from parity import TOL_REL
from paper_1802_06625_b300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Dp():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1802_06625_b300 import dpd
    return dpd


def _close(y, ref, what):
    rms = float(np.sqrt(np.mean(np.abs(ref) ** 2)))
    err = float(np.max(np.abs(np.asarray(y, np.complex128) - ref)))
    assert err <= TOL_REL * rms, (what, err / rms)


def _case(seed, P, period, K, T):
    rng = np.random.default_rng(seed)
    x = ((rng.standard_normal(P * period) + 1j * rng.standard_normal(P * period)) * 0.35).astype(np.complex64)
    taps = ((rng.standard_normal((K, T)) + 1j * rng.standard_normal((K, T))) / np.sqrt(2 * K * T)).astype(np.complex64)
    hist = ((rng.standard_normal((K, T - 1)) + 1j * rng.standard_normal((K, T - 1))) * 0.3).astype(np.complex64)
    masks = rng.integers(0, 1 << K, P)
    masks[1] = 0                       # no branch fires
    masks[2] = (1 << K) - 1            # every branch fires
    if P > 4:
        masks[3] &= ~1                 # branch 1 sits out ...
        masks[4] |= 1                  # ... and resumes
    return x, taps, hist, masks


@pytest.mark.parametrize("K,T,period", [(10, 10, 4096), (3, 7, 2056), (16, 16, 16), (1, 1, 64), (16, 16, 4104)])
def test_dpd_matches_oracle(Dp, K, T, period):
    P = 7
    x, taps, hist, masks = _case(11 + K + T, P, period, K, T)
    yg, hg = Dp.fire(torch.from_numpy(x).cuda(), torch.from_numpy(masks), torch.from_numpy(taps), period,
                     hist=torch.from_numpy(hist).cuda() if T > 1 else None)
    torch.cuda.synchronize()
    y, h = D.run(x, masks, taps, period, hist if T > 1 else None)
    yg = yg.cpu().numpy()
    for p in range(P):
        seg = slice(p * period, (p + 1) * period)
        if masks[p] & ((1 << K) - 1):
            _close(yg[seg], y[seg], p)
        else:
            assert np.all(yg[seg] == 0)
    if T > 1:
        _close(hg.cpu().numpy(), h, "tokens")


def test_tokens_handed_over_in_place_between_calls(Dp):
    K, T, period, P = 10, 10, 4096, 8
    x, taps, hist, masks = _case(5, P, period, K, T)
    xt, tt = torch.from_numpy(x).cuda(), torch.from_numpy(taps)
    y_one, h_one = Dp.fire(xt, torch.from_numpy(masks), tt, period, hist=torch.from_numpy(hist).cuda())
    h = torch.from_numpy(hist).cuda()
    ya, _ = Dp.fire(xt[:3 * period], torch.from_numpy(masks[:3]), tt, period, hist=h, hist_out=h)
    yb, _ = Dp.fire(xt[3 * period:], torch.from_numpy(masks[3:]), tt, period, hist=h, hist_out=h)
    torch.cuda.synchronize()
    ref = y_one.cpu().numpy().astype(np.complex128)
    _close(torch.cat([ya, yb]).cpu().numpy(), ref, "split")
    _close(h.cpu().numpy(), h_one.cpu().numpy().astype(np.complex128), "tokens")


def test_dpd_stream_workload_sampled(Dp):
    # the 1024 x 65536 stream in one call; the oracle runs in chunks of
    # periods with its tokens handed over and is compared on sampled periods
    w = synth.DPD
    masks = w.masks()
    taps = w.taps()
    x = w.x(device="cuda")
    y, hout = Dp.fire(x, masks, taps, w.period)
    torch.cuda.synchronize()
    pick = {0, 1, 511, 1022, 1023}
    chunk, h = 64, None
    tn = taps.numpy()
    mn = masks.numpy()
    for c0 in range(0, w.periods, chunk):
        xc = w.x(c0, chunk).numpy()
        yc, h = D.run(xc, mn[c0:c0 + chunk], tn, w.period, h)
        for p in sorted(q for q in pick if c0 <= q < c0 + chunk):
            seg = slice((p - c0) * w.period, (p - c0 + 1) * w.period)
            _close(y[p * w.period:(p + 1) * w.period].cpu().numpy(), yc[seg], p)
    _close(hout.cpu().numpy(), h, "tokens")
