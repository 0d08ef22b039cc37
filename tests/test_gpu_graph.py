"""The whole graph through the C ABI against the oracle: plain workloads,
ragged and degenerate shapes, FIFO counters, and host-side error paths."""
import numpy as np
import pytest
import torch

import oracle
from parity import TOL_REL, compare_frame
from paper_1802_06625_b300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1802_06625_b300 import graph
    return graph


PATHS = ("fused", "cuda_cores", "actors")


def run_graph(G, w, x, actors=False, C=None, out_frames=0, mem=None, chunk=None, path=None):
    """Push, fire and pull all frames of x [n, F, B]; returns records, stats.
    path: "fused" (tensor-core loop where the shape allows it, else the
    CUDA-core loop), "cuda_cores" (fused loop on CUDA cores) or "actors"."""
    if path is not None:
        actors = path == "actors"
    cuda_cores = path == "cuda_cores"
    C = C or w.C
    g = G.Graph(w.F, w.B, w.T, w.N, w.tau, w.taps(), w.H(), C=C, out_frames=out_frames)
    n = x.shape[0]
    recs = []
    k = 0
    xd = x if mem is None else x
    while k < n:
        m = min(chunk or C, n - k)
        g.push(xd[k:k + m], mem=mem)
        assert g.run(actors=actors, cuda_cores=cuda_cores) == m
        recs += g.pull()
        k += m
    stats = g.fifo_stats()
    caps = [g.capacity(f) for f in range(8)]
    g.close()
    return recs, stats, caps


def check_against_oracle(w, x_np, recs, stats=None, caps=None):
    r = oracle.run(w.F, w.B, w.T, w.N, np.float32(w.tau), w.taps().numpy(), w.H().numpy(), x_np, C=w.C)
    assert len(recs) == len(r.c)
    worst, bands = 0.0, 0
    for k, (frame, c, idx, y) in enumerate(recs):
        assert frame == k
        err, rms, nb = compare_frame(c, idx, y, r.c[k], r.idx[k], r.y[k], r.energy[k], np.float32(w.tau), w.B)
        if rms > 0:
            worst = max(worst, err / rms)
        bands += nb
    assert worst <= TOL_REL, worst
    if stats is not None:
        for f in range(8):
            w_, rd, peak = stats[f"f{f}"]
            ow, ordd = r.stats[f"f{f}"][:2]
            if bands == 0:
                assert (w_, rd) == (ow, ordd), (f, (w_, rd), (ow, ordd))
            assert peak <= caps[f]
    return r, worst, bands


@pytest.mark.parametrize("path", PATHS)
def test_plain_small_workload_100_frames(G, path):
    w = synth.PLAIN_SMALL
    x = w.frames_tensor(0, w.frames)
    recs, stats, caps = run_graph(G, w, x.cuda(), path=path)
    r, worst, bands = check_against_oracle(w, x.numpy(), recs, stats, caps)
    assert bands == 0
    assert np.all(r.c == 16)


@pytest.mark.parametrize("F,B,T,N,C,frames", [(3, 64, 5, 4, 3, 7), (1, 8, 1, 1, 1, 5), (5, 2048, 256, 32, 2, 3),
                                              (9, 768, 64, 12, 3, 4), (2, 256, 32, 16, 4, 9),
                                              (40, 256, 9, 8, 3, 5), (37, 256, 128, 64, 3, 3),
                                              (5, 512, 32, 64, 2, 4)])
def test_ragged_and_degenerate_shapes(G, F, B, T, N, C, frames):
    w = synth.PlainWorkload("t", F=F, B=B, T=T, N=N, frames=frames, tau=4.0 * B, seed=F + B + T, p=0.4, C=C)
    x = w.frames_tensor(0, frames)
    for path in PATHS:
        recs, stats, caps = run_graph(G, w, x.cuda(), C=C, path=path)
        check_against_oracle(w, x.numpy(), recs, stats, caps)


# Shapes of the tensor-core firing loop (N = 32, B | 4096): 1 to 5 tap
# shifts, B from 32 to 2048, ragged last tiles, single-frame runs.
@pytest.mark.parametrize("F,B,T,N,C,frames", [(64, 256, 64, 32, 3, 4), (5, 1024, 64, 32, 3, 5),
                                              (9, 512, 128, 32, 2, 3), (3, 2048, 1, 32, 3, 4),
                                              (130, 32, 33, 32, 3, 3), (37, 128, 17, 32, 4, 6),
                                              (7, 1024, 129, 32, 1, 3), (300, 256, 64, 32, 3, 3),
                                              (70, 64, 48, 32, 3, 3),
                                              # T = 65 is the warp-specialised loop's last T (3 shifts),
                                              # T = 66 the tile-pipeline loop's first (4 shifts)
                                              (24, 1024, 65, 32, 3, 4), (24, 1024, 66, 32, 3, 4)])
@pytest.mark.parametrize("path", PATHS)
def test_tensor_core_loop_shapes(G, F, B, T, N, C, frames, path):
    w = synth.PlainWorkload("t", F=F, B=B, T=T, N=N, frames=frames, tau=4.0 * B, seed=F * 7 + B + T, p=0.45, C=C)
    x = w.frames_tensor(0, frames)
    recs, stats, caps = run_graph(G, w, x.cuda(), C=C, path=path)
    check_against_oracle(w, x.numpy(), recs, stats, caps)


def test_paths_agree_on_control_and_within_tolerance(G):
    w = synth.PlainWorkload("t", F=512, B=1024, T=64, N=32, frames=6, tau=4096.0, seed=21, p=None)
    x = w.frames_tensor(0, 6).cuda()
    out = {path: run_graph(G, w, x, path=path)[0] for path in PATHS}
    for a, b in zip(out["fused"], out["cuda_cores"]):
        assert a[1] == b[1] and np.array_equal(a[2], b[2])
        rms = np.sqrt(np.mean(np.abs(b[3].astype(np.complex128)) ** 2))
        assert np.max(np.abs(a[3].astype(np.complex128) - b[3])) <= 2 * TOL_REL * rms


def test_tau_extremes_all_and_none(G):
    base = synth.PLAIN_SMALL
    x = base.frames_tensor(0, 4)
    for tau, want in ((-1.0, base.F), (float("inf"), 0)):
        w = synth.PlainWorkload("t", F=base.F, B=base.B, T=base.T, N=base.N, frames=4, tau=tau, seed=base.seed)
        recs, stats, _ = run_graph(G, w, x.cuda())
        assert [c for _, c, _, _ in recs] == [want] * 4
        assert stats["f6"][0] == 4 * want and stats["f5"][1] == 4   # SINK fires even at c = 0
        check_against_oracle(w, x.numpy(), recs)


def test_host_push_borrow_and_pull_kinds(G):
    w = synth.PLAIN_SMALL
    x = w.frames_tensor(0, 6)
    ref, _, _ = run_graph(G, w, x.cuda())
    host, _, _ = run_graph(G, w, x, mem=None)                          # host tensor -> H2D copy
    borrow, _, _ = run_graph(G, w, x.cuda(), mem=2)                    # borrowed in place
    for a, b in ((ref, host), (ref, borrow)):
        for (fa, ca, ia, ya), (fb, cb, ib, yb) in zip(a, b):
            assert fa == fb and ca == cb and np.array_equal(ia, ib) and np.array_equal(ya, yb)


def test_deterministic_runs(G):
    w = synth.PLAIN_SMALL
    x = w.frames_tensor(0, 5).cuda()
    a, _, _ = run_graph(G, w, x)
    b, _, _ = run_graph(G, w, x)
    for ra, rb in zip(a, b):
        assert ra[1] == rb[1] and np.array_equal(ra[2], rb[2]) and np.array_equal(ra[3], rb[3])


def test_history_carries_across_runs_and_chunking(G):
    w = synth.PlainWorkload("t", F=6, B=128, T=48, N=8, frames=10, tau=512.0, seed=11, p=0.5, C=4)
    x = w.frames_tensor(0, 10)
    one, _, _ = run_graph(G, w, x.cuda(), chunk=4)
    two, _, _ = run_graph(G, w, x.cuda(), chunk=1)
    for ra, rb in zip(one, two):
        assert ra[1] == rb[1] and np.array_equal(ra[2], rb[2])
        assert np.max(np.abs(ra[3] - rb[3])) <= 1e-6 * max(1.0, np.max(np.abs(ra[3])))
    check_against_oracle(w, x.numpy(), one)


def test_blocking_rules_on_the_host(G):
    from paper_1802_06625_b300 import _lib
    w = synth.PLAIN_SMALL
    g = G.Graph(w.F, w.B, w.T, w.N, w.tau, w.taps(), w.H(), C=2, out_frames=3)
    x = w.frames_tensor(0, 4).cuda()
    assert g.pull() == []                                   # nothing fired: EAGAIN -> empty
    g.push(x[:2])
    with pytest.raises(_lib.PruneError) as ei:
        g.push(x[2:3])                                      # f0 holds C = 2 frames
    assert ei.value.status == _lib.PRUNE_EAGAIN
    assert g.run() == 2
    g.push(x[2:4])
    assert g.run() == 1                                     # result ring holds 3 frames
    assert len(g.pull()) == 3
    assert g.run() == 1
    assert len(g.pull()) == 1
    assert g.run() == 0
    g.close()


def test_budget_is_enforced(G):
    from paper_1802_06625_b300 import _lib
    w = synth.PLAIN_SMALL
    with pytest.raises(_lib.PruneError) as ei:
        G.Graph(w.F, w.B, w.T, w.N, w.tau, w.taps(), w.H(), hbm_budget=1 << 16)
    assert ei.value.status == _lib.PRUNE_ENOMEM


def test_device_firing_rule_wait_gives_up_cleanly(G, monkeypatch):
    """The fused loop waits on f0's device counter for a frame that is never
    pushed; the bounded wait gives up, the status reaches the host as
    ETIMEOUT, the graph is poisoned and the CUDA context stays usable."""
    import ctypes
    from paper_1802_06625_b300 import _lib
    monkeypatch.setenv("PRUNE_TIMEOUT_MS", "200")
    w = synth.PLAIN_SMALL
    g = G.Graph(w.F, w.B, w.T, w.N, w.tau, w.taps(), w.H(), C=3)
    n = ctypes.c_int32()
    st = _lib.lib().prune_run(g.h, 1, ctypes.byref(n), _lib.PRUNE_RUN_DEVICE_RULE | _lib.PRUNE_RUN_SYNC)
    assert n.value == 1
    assert st == _lib.PRUNE_ETIMEOUT, _lib.lib().prune_last_error(g.h)
    assert b"bounded wait" in _lib.lib().prune_last_error(g.h)
    with pytest.raises(_lib.PruneError) as ei:
        g.push(w.frames_tensor(0, 1).cuda())
    assert ei.value.status == _lib.PRUNE_ETIMEOUT
    g.close()
    # the context still works
    a = torch.ones(1024, device="cuda")
    assert float((a * 2).sum()) == 2048.0
    # a fresh graph fires normally
    x = w.frames_tensor(0, 3)
    recs, stats, caps = run_graph(G, w, x.cuda())
    check_against_oracle(w, x.numpy(), recs, stats, caps)


def test_device_firing_rule_with_frames_present(G):
    """With the frames already pushed, the device-side rule passes at once."""
    import ctypes
    from paper_1802_06625_b300 import _lib
    w = synth.PLAIN_SMALL
    x = w.frames_tensor(0, 3)
    g = G.Graph(w.F, w.B, w.T, w.N, w.tau, w.taps(), w.H(), C=3)
    g.push(x.cuda())
    n = ctypes.c_int32()
    _lib.check(_lib.lib().prune_run(g.h, 3, ctypes.byref(n), _lib.PRUNE_RUN_DEVICE_RULE | _lib.PRUNE_RUN_SYNC), g.h)
    assert n.value == 3
    recs = g.pull()
    g.close()
    check_against_oracle(w, x.numpy(), recs)


@pytest.mark.parametrize("path", PATHS)
def test_pull_overlapping_later_pushes_and_runs(G, path):
    # Chunk k is pushed and fired before chunk k-1 is pulled: a pull copies
    # out (on the graph's pull stream) after the run that fired its records
    # while later pushes and runs are queued; the result ring (5 slots)
    # wraps inside pulls.
    w = synth.PlainWorkload("t", F=64, B=256, T=16, N=16, frames=13, tau=1024.0, seed=91, p=0.3, C=6)
    x = w.frames_tensor(0, 13)
    g = G.Graph(w.F, w.B, w.T, w.N, w.tau, w.taps(), w.H(), C=6, out_frames=5)
    recs, prev = [], None
    for k in range(0, 13, 2):
        m = min(2, 13 - k)
        g.push(x[k:k + m])
        assert g.run(actors=path == "actors", cuda_cores=path == "cuda_cores") == m
        if prev is not None:
            got = g.pull(prev)
            assert len(got) == prev
            recs += got
        prev = m
    recs += g.pull(prev)
    g.close()
    check_against_oracle(w, x.numpy(), recs)


def test_plain_large_shape_in_bench_runs_sampled(G):
    """The plain-large graph (F = 4096, B = 1024, T = 64, N = 32: the
    warp-specialised tensor-core loop) fired as the bench fires it: frames
    pushed by reference in runs of C = 336.  Two runs (340 frames); sampled
    frames on both sides of the run boundary against the oracle, each fed
    the frame before it for its delay token."""
    from paper_1802_06625_b300 import _lib

    w = synth.PLAIN_LARGE
    C, n = 336, 340
    dev = torch.device("cuda", 0)
    x = torch.empty(n, w.F, w.B, dtype=torch.complex64, device=dev)
    for k in range(n):
        x[k] = w.frame(k, device=dev)
    g = G.Graph(w.F, w.B, w.T, w.N, w.tau, w.taps(), w.H(), C=C, out_frames=n, device=0)
    for k in range(0, n, C):
        m = min(C, n - k)
        g.push(x[k:k + m], mem=_lib.PRUNE_MEM_DEVICE_BORROW)
        assert g.run() == m
    g.sync()
    sample = [0, 1, 197, 335, 336, 339]
    got, j = {}, 0
    for s in sample:
        if s > j:
            assert g.discard(s - j) == s - j
        (got[s],) = g.pull(1)
        j = s + 1
    g.close()
    del x
    for s in sample:
        xs = torch.stack([w.frame(k) for k in range(max(0, s - 1), s + 1)]).numpy()
        r = oracle.run(w.F, w.B, w.T, w.N, np.float32(w.tau), w.taps().numpy(), w.H().numpy(), xs)
        frame, c, idx, y = got[s]
        assert frame == s
        err, rms, nb = compare_frame(c, idx, y, r.c[-1], r.idx[-1], r.y[-1], r.energy[-1], np.float32(w.tau), w.B)
        assert rms > 0 and err <= TOL_REL * rms, (s, err / rms, nb)


def test_plain_large_host_frames_in_chunks_sampled(G):
    """The end-to-end path at the plain-large shape: pinned host frames
    pushed in chunks of 8 and fired, each chunk's records pulled to host
    after the next chunk was pushed and fired (the bench's e2e pattern).
    The records equal those of the same frames pushed by reference, and
    sampled frames (both sides of a chunk boundary) match the oracle."""
    from paper_1802_06625_b300 import _lib

    w = synth.PLAIN_LARGE
    E, ch = 24, 8
    xh = torch.empty(E, w.F, w.B, dtype=torch.complex64).pin_memory()
    for k in range(E):
        xh[k] = w.frame(k, device="cuda").cpu()
    g = G.Graph(w.F, w.B, w.T, w.N, w.tau, w.taps(), w.H(), C=336, out_frames=336, device=0)
    recs = []
    for k in range(0, E, ch):
        g.push(xh[k:k + ch])
        assert g.run() == ch
        if k > 0:
            recs += g.pull(ch)
    recs += g.pull(ch)
    g.close()
    assert [r[0] for r in recs] == list(range(E))
    xd = xh.cuda()
    g = G.Graph(w.F, w.B, w.T, w.N, w.tau, w.taps(), w.H(), C=336, out_frames=336, device=0)
    g.push(xd, mem=_lib.PRUNE_MEM_DEVICE_BORROW)
    assert g.run(sync=True) == E
    ref = g.pull(E)
    g.close()
    for (fa, ca, ia, ya), (fb, cb, ib, yb) in zip(recs, ref):
        assert fa == fb and ca == cb and np.array_equal(ia, ib) and np.array_equal(ya, yb), fa
    for s in (0, 7, 8, 23):
        xs = xh[max(0, s - 1):s + 1].numpy()
        r = oracle.run(w.F, w.B, w.T, w.N, np.float32(w.tau), w.taps().numpy(), w.H().numpy(), xs)
        frame, c, idx, y = recs[s]
        err, rms, nb = compare_frame(c, idx, y, r.c[-1], r.idx[-1], r.y[-1], r.energy[-1], np.float32(w.tau), w.B)
        assert rms > 0 and err <= TOL_REL * rms, (s, err / rms, nb)


def test_staging_and_fir_rings_are_allocated_only_when_needed(G):
    # F = 4096, B = 1024, C = 16: each C-frame ring is 16 x 32 MiB = 512 MiB.
    # The fused graph fed by borrowed pushes needs only its result ring (and
    # small state); the staging ring comes with the first copied push, the
    # FIR output ring with the first actor-path run, each against the budget.
    from paper_1802_06625_b300 import _lib

    w = synth.PlainWorkload("lazy", F=4096, B=1024, T=64, N=32, frames=2, tau=4096.0, seed=8, p=0.3)
    x = w.frames_tensor(0, 2).cuda()
    ring = 16 * w.F * w.B * 8
    g = G.Graph(w.F, w.B, w.T, w.N, w.tau, w.taps(), w.H(), C=16, out_frames=16,
                hbm_budget=ring + (64 << 20))
    g.push(x[:1], mem=_lib.PRUNE_MEM_DEVICE_BORROW)
    assert g.run(sync=True) == 1
    with pytest.raises(_lib.PruneError) as e:
        g.push(x[1:])                                   # a copied push: the staging ring does not fit
    assert e.value.status == _lib.PRUNE_ENOMEM
    g.push(x[1:], mem=_lib.PRUNE_MEM_DEVICE_BORROW)     # nothing changed: borrowed pushes still work
    with pytest.raises(_lib.PruneError) as e:
        g.run(actors=True)                              # the actor path's FIR ring does not fit either
    assert e.value.status == _lib.PRUNE_ENOMEM
    assert g.run(sync=True) == 1
    assert [r[0] for r in g.pull()] == [0, 1]
    g.close()
    # with room for one more ring, the copied push succeeds
    g = G.Graph(w.F, w.B, w.T, w.N, w.tau, w.taps(), w.H(), C=16, out_frames=16,
                hbm_budget=2 * ring + (64 << 20))
    g.push(x)
    assert g.run(sync=True) == 2
    g.close()


@pytest.mark.parametrize("T,kind", [(64, "ws"), (100, "pipes")])
def test_ring_slots_wrap_inside_runs(G, T, kind):
    # C = 5 look-back/frame slots and a 7-frame record ring, fired 3 frames
    # per run for 15 frames: runs start at frame slots 0, 3, 1, 4, 2 and
    # record slots 0, 3, 6, 2, 5, so both rings wrap inside runs; every
    # frame against the oracle on the whole stream.
    w = synth.PlainWorkload("wrap", F=40, B=256, T=T, N=32, frames=15, tau=1024.0, seed=T + 5, p=0.4, C=5)
    x = w.frames_tensor(0, 15)
    g = G.Graph(w.F, w.B, w.T, w.N, w.tau, w.taps(), w.H(), C=5, out_frames=7)
    g.profile(True)
    xd = x.cuda()
    recs = []
    for k in range(0, 15, 3):
        g.push(xd[k:k + 3])
        assert g.run(sync=True) == 3
        recs += g.pull()
    assert g.kernel_times(g.KIND_LOOP_TC)[1] == 5, "the tensor-core loop did not fire every run"
    g.close()
    check_against_oracle(w, x.numpy(), recs)
