"""Batched firing of many independent instances against the oracle: uneven
F, T and tau, the delay token carried across steps, HX on tensor cores
(N = 64) and on CUDA cores (N = 16), and CUDA-graph replay."""
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


def _instances(B, N, seed, n):
    specs = [(16, 8), (37, 32), (5, 128), (64, 1), (130, 32), (3, 8), (200, 128), (1, 32), (90, 17), (12, 64)]
    out = []
    for i in range(n):
        F, T = specs[i % len(specs)]
        w = synth.PlainWorkload(f"b{i}", F=F, B=B, T=T, N=N, frames=3, tau=float((2 + i % 6) * B),
                                seed=seed * 1000 + i, p=0.1 + 0.08 * (i % 10))
        out.append(w)
    return out


def _run(G, B, N, ws, steps, graph):
    insts = [{"F": w.F, "T": w.T, "tau": w.tau, "taps": w.taps(), "H": w.H()} for w in ws]
    bt = G.Batch(B, N, insts)
    frames = [[w.frame(k) for w in ws] for k in range(steps)]
    recs = []
    for k in range(steps):
        x = torch.cat([f.reshape(-1) for f in frames[k]]).cuda()
        bt.fire(x, graph=graph)
        bt.sync()
        recs.append([bt.pull(i) for i in range(len(ws))])
    bt.close()
    return frames, recs


@pytest.mark.parametrize("N", [64, 16])
@pytest.mark.parametrize("graph", [False, True])
def test_batch_matches_oracle_over_steps(G, N, graph):
    B = 256
    ws = _instances(B, N, seed=5 + N, n=10)
    steps = 3
    frames, recs = _run(G, B, N, ws, steps, graph)
    for i, w in enumerate(ws):
        x = np.stack([frames[k][i].numpy() for k in range(steps)])
        r = oracle.run(w.F, B, w.T, N, np.float32(w.tau), w.taps().numpy(), w.H().numpy(), x)
        for k in range(steps):
            frame, c, idx, y = recs[k][i]
            assert frame == k
            err, rms, nb = compare_frame(c, idx, y, r.c[k], r.idx[k], r.y[k], r.energy[k], np.float32(w.tau), B)
            if rms > 0:
                assert err <= TOL_REL * rms, (i, k, err / rms)


def test_batch_equals_single_graphs(G):
    # Each instance alone: as a batch of one it runs the same kernels on the
    # same data, so the records are bit-identical; as a single graph (actor
    # path, FIR on CUDA cores) the control matches outside the guard band and
    # the samples agree within the parity tolerance.
    B, N = 256, 64
    ws = _instances(B, N, seed=99, n=6)
    frames, recs = _run(G, B, N, ws, 2, graph=True)
    for i, w in enumerate(ws):
        _, alone = _run(G, B, N, [w], 2, graph=True)
        g = G.Graph(w.F, B, w.T, N, w.tau, w.taps(), w.H(), C=3, out_frames=2)
        g.push(torch.stack([frames[k][i] for k in range(2)]).cuda())
        g.run(actors=True)
        single = g.pull()
        g.close()
        x = np.stack([frames[k][i].numpy() for k in range(2)])
        r = oracle.run(w.F, B, w.T, N, np.float32(w.tau), w.taps().numpy(), w.H().numpy(), x)
        for k in range(2):
            assert alone[k][0][1] == recs[k][i][1]
            assert np.array_equal(alone[k][0][2], recs[k][i][2])
            assert np.array_equal(alone[k][0][3], recs[k][i][3])
            _, c, idx, y = recs[k][i]
            cs = single[k][1]
            err, rms, nb = compare_frame(c, idx, y, cs, np.asarray(single[k][2])[:cs], single[k][3], r.energy[k],
                                         np.float32(w.tau), B)
            if rms > 0:
                assert err <= TOL_REL * rms, (i, k, err / rms)


def test_batched_workload_shapes_fire(G):
    # the 512-instance workload's shapes, one step, control checked against
    # the oracle on a sample of instances
    b = synth.BATCHED
    ws = [b.instance(i) for i in range(b.instances)]
    insts = [{"F": w.F, "T": w.T, "tau": w.tau, "taps": w.taps(), "H": w.H()} for w in ws]
    bt = G.Batch(b.B, b.N, insts)
    x_host = torch.cat([w.frame(0).reshape(-1) for w in ws])   # generated on the CPU
    x = x_host.cuda()
    bt.fire(x, graph=True)
    bt.sync()
    for i in (0, 1, 100, 257, 511):
        w = ws[i]
        frame, c, idx, y = bt.pull(i)
        xi = x_host[bt.offsets[i]:bt.offsets[i] + w.F * w.B].numpy().reshape(1, w.F, w.B)
        r = oracle.run(w.F, w.B, w.T, w.N, np.float32(w.tau), w.taps().numpy(), w.H().numpy(), xi)
        err, rms, nb = compare_frame(c, idx, y, r.c[0], r.idx[0], r.y[0], r.energy[0], np.float32(w.tau), w.B)
        if rms > 0:
            assert err <= TOL_REL * rms
    bt.close()


@pytest.mark.parametrize("N", [64, 16])
def test_every_launch_shape_gives_identical_results_and_autotune_keeps_state(G, N):
    # the launch shape changes only which CTA fires which tile: results are
    # bit-identical; autotuning fires the step repeatedly at the same parity,
    # so the instances' delay tokens and step count are untouched
    B = 256
    ws = _instances(B, N, seed=41 + N, n=7)
    insts = [{"F": w.F, "T": w.T, "tau": w.tau, "taps": w.taps(), "H": w.H()} for w in ws]
    frames = [[w.frame(k) for w in ws] for k in range(2)]
    xs = [torch.cat([f.reshape(-1) for f in frames[k]]).cuda() for k in range(2)]
    ref = G.Batch(B, N, insts)
    recs_ref = []
    for k in range(2):
        ref.fire(xs[k])
        ref.sync()
        recs_ref.append([ref.pull(i) for i in range(len(ws))])
    ref.close()
    shapes = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (1, 3, 0), (0, 0, 1), (1, 0, 7)]
    for fo, ch, gr in shapes:
        bt = G.Batch(B, N, insts)
        bt.set_tuning(fir_order=fo, hx_chunk=ch, hx_grid=gr)
        assert bt.tuning()["hx_chunk"] == ch
        for k in range(2):
            bt.fire(xs[k], graph=(k == 1))
            bt.sync()
            for i in range(len(ws)):
                a, r = bt.pull(i), recs_ref[k][i]
                assert a[0] == r[0] and a[1] == r[1]
                assert np.array_equal(a[2], r[2]) and np.array_equal(a[3], r[3]), (fo, ch, gr, k, i)
        bt.close()
    at = G.Batch(B, N, insts)
    best, allc = at.autotune(xs[0], reps=2)
    assert len(allc) == 8 and all(c["ms"] > 0 for c in allc)
    assert best["ms"] == min(c["ms"] for c in allc) and at.tuning()["ms"] == best["ms"]
    for k in range(2):
        at.fire(xs[k], graph=True)
        at.sync()
        for i in range(len(ws)):
            a, r = at.pull(i), recs_ref[k][i]
            assert a[0] == r[0] and np.array_equal(a[2], r[2]) and np.array_equal(a[3], r[3])
    at.close()


# The tensor-core batched FIR (B | 4096, T <= 129) on other block sizes: B = 64
# (one HX row per block, T up to 65) and B = 2048 (two blocks per tile, five
# tap shifts at T = 129), ragged last tiles, against the oracle over steps.
@pytest.mark.parametrize("B,specs", [(64, [(3, 65), (70, 64), (1, 1), (40, 33), (129, 9)]),
                                     (2048, [(5, 129), (2, 65), (7, 8), (1, 2)])])
def test_tensor_core_batch_fir_block_sizes(G, B, specs):
    N = 64
    ws = [synth.PlainWorkload(f"s{i}", F=F, B=B, T=T, N=N, frames=3, tau=float((2 + i % 5) * B),
                              seed=700 + B + i, p=0.3 + 0.1 * i) for i, (F, T) in enumerate(specs)]
    steps = 3
    frames, recs = _run(G, B, N, ws, steps, graph=False)
    for i, w in enumerate(ws):
        x = np.stack([frames[k][i].numpy() for k in range(steps)])
        r = oracle.run(w.F, B, w.T, N, np.float32(w.tau), w.taps().numpy(), w.H().numpy(), x)
        for k in range(steps):
            frame, c, idx, y = recs[k][i]
            err, rms, nb = compare_frame(c, idx, y, r.c[k], r.idx[k], r.y[k], r.energy[k], np.float32(w.tau), B)
            if rms > 0:
                assert err <= TOL_REL * rms, (B, i, k, err / rms)


def test_batch_fir_on_tensor_and_cuda_cores_agree(G, monkeypatch):
    # the same instances with the FIR on tensor cores (default) and on CUDA
    # cores (PRUNE_BATCH_FIR=cuda_cores): control equal outside the guard
    # band, samples within the parity tolerance, both against the oracle
    B, N = 256, 64
    ws = _instances(B, N, seed=77, n=8)
    frames, recs_tc = _run(G, B, N, ws, 2, graph=True)
    monkeypatch.setenv("PRUNE_BATCH_FIR", "cuda_cores")
    _, recs_cc = _run(G, B, N, ws, 2, graph=True)
    for i, w in enumerate(ws):
        x = np.stack([frames[k][i].numpy() for k in range(2)])
        r = oracle.run(w.F, B, w.T, N, np.float32(w.tau), w.taps().numpy(), w.H().numpy(), x)
        for k in range(2):
            _, c, idx, y = recs_tc[k][i]
            _, cc, idxc, yc = recs_cc[k][i]
            err, rms, nb = compare_frame(c, idx, y, cc, np.asarray(idxc)[:cc], yc, r.energy[k], np.float32(w.tau), B)
            if rms > 0:
                assert err <= TOL_REL * rms, (i, k, err / rms)
            err, rms, nb = compare_frame(cc, idxc, yc, r.c[k], r.idx[k], r.y[k], r.energy[k], np.float32(w.tau), B)
            if rms > 0:
                assert err <= TOL_REL * rms, (i, k, err / rms)
