"""The allocation-free entry point prune_fire_frames_noalloc.

It exists for callers that cannot allocate device memory: real-time threads
that must not block in the device allocator, and deployments whose device
memory is budgeted and committed up front.  Its scratch is a fixed array
inside the library.  The GPU tests fire two calls in a row through the C ABI
and check each against the graph entry points (create / push / run / pull)
on the same frames and against the FP64 oracle, with the parity tolerance
used everywhere else; another case starts from a nonzero delay token and
drops the outgoing one.  The file is collected last, so that a run that
stops at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from parity import TOL_REL, compare_frame
from paper_1802_06625_b300 import _lib, synth


def _call(x, hist, taps, H, w, frames, tau, c, idx, y, hist_out, status):
    ptr = lambda t: None if t is None else t.data_ptr()  # noqa: E731
    return _lib.lib().prune_fire_frames_noalloc(
        ptr(x), ptr(hist), ptr(taps), ptr(H), w.F, w.B, w.T, w.N, frames, ctypes.c_float(tau),
        ptr(c), ptr(idx), ptr(y), ptr(hist_out), ptr(status), torch.cuda.current_stream().cuda_stream)


def _fire(xd, hin, td, Hd, w, n, hout, status):
    dev = xd.device
    c = torch.full((n,), -1, dtype=torch.int32, device=dev)
    idx = torch.full((n, w.F), -1, dtype=torch.int32, device=dev)
    y = torch.zeros(n, w.F * w.B, dtype=torch.complex64, device=dev)
    st = _call(xd, hin, td, Hd, w, n, w.tau, c, idx, y, hout, status)
    assert st == _lib.PRUNE_OK, _lib.lib().prune_last_error(None)
    torch.cuda.synchronize()
    assert status.cpu().tolist() == [0, 0, 0, 0], status
    return c.cpu().numpy(), idx.cpu().numpy(), y.cpu().numpy()


def _check_oracle(w, r, k, c, idx, y):
    """Frame k of a call (its c, idx row and y row) against oracle frame k."""
    got_y = y[:c * w.B].reshape(c, w.B)
    err, rms, _ = compare_frame(c, idx[:c], got_y, r.c[k], r.idx[k], r.y[k], r.energy[k], np.float32(w.tau), w.B)
    assert rms == 0 or err <= TOL_REL * rms, (k, err, rms)


def test_noalloc_rejects_requests_beyond_its_scratch():
    # Requests above the fixed scratch fail before any CUDA call (the fake,
    # aligned pointers below are never dereferenced).
    L = _lib.lib()
    fake = 4096
    st = L.prune_fire_frames_noalloc(fake, None, fake, fake, 64, 256, 16, 16, 257, ctypes.c_float(1.0),
                                     fake, fake, fake, None, fake, None)
    assert st == _lib.PRUNE_EINVAL
    assert b"scratch" in L.prune_last_error(None)
    # 33 frames of 4096 x 1024 samples: 33 x 2048 tiles > 65536 look-back words
    st = L.prune_fire_frames_noalloc(fake, None, fake, fake, 4096, 1024, 64, 32, 33, ctypes.c_float(1.0),
                                     fake, fake, fake, None, fake, None)
    assert st == _lib.PRUNE_EINVAL
    assert b"scratch" in L.prune_last_error(None)
    # the tensor-core N is not fired by the fused loop
    st = L.prune_fire_frames_noalloc(fake, None, fake, fake, 4, 256, 16, 64, 1, ctypes.c_float(1.0),
                                     fake, fake, fake, None, fake, None)
    assert st == _lib.PRUNE_EINVAL


NOALLOC_CASES = [synth.PLAIN_SMALL,                                        # N = 16, T = 16
                 synth.PlainWorkload("na32", F=64, B=1024, T=64, N=32, frames=6, tau=4096.0, seed=31, p=0.35)]


@pytest.mark.gpu
@pytest.mark.parametrize("w", NOALLOC_CASES, ids=lambda w: f"N{w.N}_T{w.T}")
def test_noalloc_matches_graph_entry_points_and_oracle_on_two_calls_in_a_row(w):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1802_06625_b300.graph import Graph
    n1, n2 = 3, 3
    x = w.frames_tensor(0, n1 + n2)
    taps, H = w.taps(), w.H()

    # the existing entry points on the same frames
    g = Graph(w.F, w.B, w.T, w.N, w.tau, taps, H, C=3, out_frames=n1 + n2)
    g.push(x[:n1].cuda())
    g.run()
    g.push(x[n1:].cuda())
    g.run()
    ref = g.pull()
    g.close()
    assert len(ref) == n1 + n2
    # the oracle on the whole stream (zero delay token before frame 0)
    r = oracle.run(w.F, w.B, w.T, w.N, np.float32(w.tau), taps.numpy(), H.numpy(), x.numpy())

    dev = torch.device("cuda")
    xd = x.reshape(n1 + n2, w.F * w.B).to(dev)
    td, Hd = taps.to(dev), H.to(dev)
    h1 = torch.zeros(w.T - 1, dtype=torch.complex64, device=dev)
    h2 = torch.zeros(w.T - 1, dtype=torch.complex64, device=dev)
    status = torch.full((4,), 7, dtype=torch.int32, device=dev)
    # the second call starts from the first call's (nonzero) delay token
    for call, (k0, n, hin, hout) in enumerate(((0, n1, None, h1), (n1, n2, h1, h2))):
        c, idx, y = _fire(xd[k0:k0 + n], hin, td, Hd, w, n, hout, status)
        for i in range(n):
            frame, rc, ridx, ry = ref[k0 + i]
            assert frame == k0 + i
            assert c[i] == rc, (call, i, c[i], rc)
            assert np.array_equal(idx[i, :rc], ridx)
            got = y[i, :rc * w.B].reshape(rc, w.B).astype(np.complex128)
            want = ry.astype(np.complex128)
            rms = np.sqrt(np.mean(np.abs(want) ** 2))
            assert np.max(np.abs(got - want)) <= TOL_REL * rms
            _check_oracle(w, r, k0 + i, int(c[i]), idx[i], y[i])
    # the delay token after the second call: the last T-1 input samples
    assert np.array_equal(h2.cpu().numpy(), x[-1].reshape(-1)[-(w.T - 1):].numpy())


@pytest.mark.gpu
@pytest.mark.parametrize("w", NOALLOC_CASES, ids=lambda w: f"N{w.N}_T{w.T}")
def test_noalloc_from_a_nonzero_delay_token_against_the_oracle(w):
    # A seeded nonzero delay token before frame 0 (the oracle's hist_in), and
    # no outgoing token kept (hist_out = NULL with T > 1).
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    n = 4
    x = w.frames_tensor(0, n)
    taps, H = w.taps(), w.H()
    rng = np.random.default_rng(w.seed + 77)
    hist = (3.0 * (rng.standard_normal(w.T - 1) + 1j * rng.standard_normal(w.T - 1))).astype(np.complex64)
    r = oracle.run(w.F, w.B, w.T, w.N, np.float32(w.tau), taps.numpy(), H.numpy(), x.numpy(), hist_in=hist)
    dev = torch.device("cuda")
    status = torch.full((4,), 7, dtype=torch.int32, device=dev)
    c, idx, y = _fire(x.reshape(n, -1).to(dev), torch.from_numpy(hist).to(dev), taps.to(dev), H.to(dev), w, n,
                      None, status)
    for k in range(n):
        _check_oracle(w, r, k, int(c[k]), idx[k], y[k])
