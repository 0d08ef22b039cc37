"""The allocation-free entry point prune_fire_frames_noalloc.

It exists for callers that cannot allocate device memory: code that
enqueues work while a CUDA graph is being captured, real-time threads that
must not block in the allocator, deployments with a fixed device-memory
budget.  Its scratch is a fixed array inside the library.  The GPU test
fires two calls in a row through the C ABI and checks each against the
graph entry points (create / push / run / pull) on the same frames, with the
parity tolerance used everywhere else.  The file is collected last, so that
a run that stops at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

from parity import TOL_REL
from paper_1802_06625_b300 import _lib, synth


def _call(x, hist, taps, H, w, frames, tau, c, idx, y, hist_out, status):
    ptr = lambda t: None if t is None else t.data_ptr()  # noqa: E731
    return _lib.lib().prune_fire_frames_noalloc(
        ptr(x), ptr(hist), ptr(taps), ptr(H), w.F, w.B, w.T, w.N, frames, ctypes.c_float(tau),
        ptr(c), ptr(idx), ptr(y), ptr(hist_out), ptr(status), torch.cuda.current_stream().cuda_stream)


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


@pytest.mark.gpu
def test_noalloc_matches_graph_entry_points_on_two_calls_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1802_06625_b300.graph import Graph
    w = synth.PLAIN_SMALL
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

    dev = torch.device("cuda")
    xd = x.reshape(n1 + n2, w.F * w.B).to(dev)
    td, Hd = taps.to(dev), H.to(dev)
    h1 = torch.zeros(w.T - 1, dtype=torch.complex64, device=dev)
    h2 = torch.zeros(w.T - 1, dtype=torch.complex64, device=dev)
    status = torch.full((4,), 7, dtype=torch.int32, device=dev)
    for call, (k0, n, hin, hout) in enumerate(((0, n1, None, h1), (n1, n2, h1, h2))):
        c = torch.full((n,), -1, dtype=torch.int32, device=dev)
        idx = torch.full((n, w.F), -1, dtype=torch.int32, device=dev)
        y = torch.zeros(n, w.F * w.B, dtype=torch.complex64, device=dev)
        st = _call(xd[k0:k0 + n], hin, td, Hd, w, n, w.tau, c, idx, y, hout, status)
        assert st == _lib.PRUNE_OK, _lib.lib().prune_last_error(None)
        torch.cuda.synchronize()
        assert status.cpu().tolist() == [0, 0, 0, 0], status
        c, idx, y = c.cpu().numpy(), idx.cpu().numpy(), y.cpu().numpy()
        for i in range(n):
            frame, rc, ridx, ry = ref[k0 + i]
            assert frame == k0 + i
            assert c[i] == rc, (call, i, c[i], rc)
            assert np.array_equal(idx[i, :rc], ridx)
            got = y[i, :rc * w.B].reshape(rc, w.B).astype(np.complex128)
            want = ry.astype(np.complex128)
            rms = np.sqrt(np.mean(np.abs(want) ** 2))
            assert np.max(np.abs(got - want)) <= TOL_REL * rms
    # the delay token after the second call: the last T-1 input samples
    assert np.array_equal(h2.cpu().numpy(), x[-1].reshape(-1)[-(w.T - 1):].numpy())
