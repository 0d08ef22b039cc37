"""Signal level: the tensor-core paths (split FP16 with power-of-two scaling
of every operand) against the oracle when inputs, taps and H are scaled far
from unit size.  Scaling the input by a and the taps by b scales every FIR
output by a b and every energy by (a b)^2, so tau is scaled by (a b)^2 and
the decisions stay those of the unscaled workload up to FP32 rounding of the
scaled inputs; each case must meet the same bars as at unit scale: control
bit-exact outside the guard band, samples within 1e-4 of the oracle RMS.

Paths covered: the warp-specialised fused loop (N = 32, T <= 65), the
tile-pipeline fused loop (N = 32, 65 < T <= 129), the actor path with HX on
tensor cores (N = 64), the batched tensor-core FIR and HX (N = 64), and the
request loop (which fires through the batched kernels)."""
import numpy as np
import pytest
import torch

import oracle
from parity import TOL_REL, compare_frame
from paper_1802_06625_b300 import synth

pytestmark = pytest.mark.gpu

# (input scale, tap scale, H scale)
SCALES = [(1e-6, 1.0, 1.0), (1e-4, 1.0, 1.0), (1.0, 1.0, 1.0), (1e3, 1.0, 1.0), (3e4, 1.0, 1.0),
          (1.0, 1e-4, 1.0), (1e-4, 1e-4, 1e3), (3e4, 1e4, 1e-3)]


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1802_06625_b300 import graph
    return graph


def _scaled(w, x, a, b, hs):
    """Scaled FP32 copies of the frames, taps and H, and tau scaled by (a b)^2."""
    xs = (x.to(torch.complex128) * a).to(torch.complex64)
    taps = (w.taps().to(torch.complex128) * b).to(torch.complex64)
    H = (w.H().to(torch.complex128) * hs).to(torch.complex64)
    tau = np.float32(w.tau * (a * b) ** 2)
    return xs, taps, H, tau


def _check(F, B, T, N, tau, taps, H, xs, recs):
    r = oracle.run(F, B, T, N, tau, taps.numpy(), H.numpy(), xs.numpy())
    assert len(recs) == len(r.c)
    worst = 0.0
    for k, (frame, c, idx, y) in enumerate(recs):
        assert frame == k
        err, rms, _ = compare_frame(c, idx, y, r.c[k], r.idx[k], r.y[k], r.energy[k], tau, B)
        if rms > 0:
            worst = max(worst, err / rms)
    assert worst <= TOL_REL, worst
    return r


# (F, B, T, N, kernel kind the default path must launch)
GRAPH_CASES = [(64, 1024, 64, 32, "loop_tc"),    # warp-specialised fused loop
               (16, 1024, 100, 32, "loop_tc"),   # tile-pipeline fused loop (T > 65)
               (37, 256, 33, 64, "hx_tc")]       # actor path, HX on tensor cores


@pytest.mark.parametrize("a,b,hs", SCALES)
@pytest.mark.parametrize("F,B,T,N,kind", GRAPH_CASES)
def test_graph_tensor_core_paths_across_levels(G, F, B, T, N, kind, a, b, hs):
    w = synth.PlainWorkload("lvl", F=F, B=B, T=T, N=N, frames=3, tau=4.0 * B, seed=F + T + N, p=0.4, C=3)
    x = w.frames_tensor(0, 3)
    xs, taps, H, tau = _scaled(w, x, a, b, hs)
    g = G.Graph(F, B, T, N, float(tau), taps, H, C=3, out_frames=3)
    g.profile(True)
    g.push(xs.cuda())
    assert g.run(sync=True) == 3
    recs = g.pull()
    k = g.KIND_LOOP_TC if kind == "loop_tc" else g.KIND_HX_TC
    assert g.kernel_times(k)[1] > 0, "the tensor-core path did not run"
    g.close()
    _check(F, B, T, N, tau, taps, H, xs, recs)


def test_power_of_two_levels_scale_outputs_exactly(G):
    # Inputs scaled by 2^-24 and by 2^32 both fall outside the window
    # [2^0, 2^15) that the split takes unscaled; the tile exponent is a
    # multiple of 8 fixed by the tile's largest component alone, so both
    # runs split the same scaled tiles (-24 and 32 are congruent mod 8) and
    # the outputs differ by exactly 2^56, bit for bit, with equal decisions.
    w = synth.PlainWorkload("p2", F=64, B=1024, T=64, N=32, frames=2, tau=4096.0, seed=3, p=0.4)
    x = w.frames_tensor(0, 2)
    out = {}
    for k in (-24, 32):
        g = G.Graph(w.F, w.B, w.T, w.N, w.tau * 4.0 ** k, w.taps(), w.H(), C=3, out_frames=2)
        g.push((x * 2.0 ** k).cuda())
        g.run(sync=True)
        out[k] = g.pull()
        g.close()
    for (f0, c0, i0, y0), (f1, c1, i1, y1) in zip(out[-24], out[32]):
        assert c0 == c1 and np.array_equal(i0, i1)
        assert np.array_equal(y0.astype(np.complex128) * 2.0 ** 56, y1.astype(np.complex128))


def test_scaled_tiles_do_not_depend_on_scheduling(G):
    # Out-of-window inputs (level 1e-4): the exponent of each tile is
    # predicted from the tile its converter fired before, which depends on
    # the order tiles are claimed in; the exponent it is fired with does
    # not, so repeated runs are bit-identical.
    w = synth.PlainWorkload("det", F=512, B=1024, T=64, N=32, frames=6, tau=4096.0 * 1e-8, seed=12, p=None)
    x = (w.frames_tensor(0, 6).to(torch.complex128) * 1e-4).to(torch.complex64).cuda()
    runs = []
    for _ in range(3):
        g = G.Graph(w.F, w.B, w.T, w.N, w.tau, w.taps(), w.H(), C=6, out_frames=6)
        g.push(x)
        g.run(sync=True)
        runs.append(g.pull())
        g.close()
    for r in runs[1:]:
        for (f0, c0, i0, y0), (f1, c1, i1, y1) in zip(runs[0], r):
            assert c0 == c1 and np.array_equal(i0, i1) and np.array_equal(y0, y1)


@pytest.mark.parametrize("a,b,hs", SCALES)
def test_batched_tensor_core_paths_across_levels(G, a, b, hs):
    B, N = 256, 64
    specs = [(16, 8), (37, 32), (40, 128), (9, 32), (70, 128)]
    ws, insts, xs_all, pars = [], [], [], []
    for i, (F, T) in enumerate(specs):
        w = synth.PlainWorkload(f"bl{i}", F=F, B=B, T=T, N=N, frames=2, tau=float((3 + i % 4) * B),
                                seed=500 + i, p=0.2 + 0.15 * i)
        x = w.frames_tensor(0, 2)
        xs, taps, H, tau = _scaled(w, x, a, b, hs)
        ws.append(w)
        xs_all.append(xs)
        pars.append((taps, H, tau))
        insts.append({"F": F, "T": T, "tau": float(tau), "taps": taps, "H": H})
    bt = G.Batch(B, N, insts)
    recs = [[] for _ in ws]
    for k in range(2):
        bt.fire(torch.cat([xs[k].reshape(-1) for xs in xs_all]).cuda(), graph=k == 1)
        bt.sync()
        for i in range(len(ws)):
            frame, c, idx, y = bt.pull(i)
            recs[i].append((k, c, np.asarray(idx)[:c], np.asarray(y)[:c]))
    bt.close()
    for i, w in enumerate(ws):
        taps, H, tau = pars[i]
        _check(w.F, B, w.T, N, tau, taps, H, xs_all[i], recs[i])


@pytest.mark.parametrize("a,b,hs", [(1e-6, 1.0, 1.0), (3e4, 1.0, 1.0), (1e-4, 1e-4, 1e3)])
def test_request_loop_across_levels(a, b, hs):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1802_06625_b300 import serve
    B, N = 256, 64
    srv = serve.Server(B, N, F_max=128, T_max=129, max_streams=4, hbm_budget=256 << 20, frames_per_step=2, ring=4)
    cases = []
    for i, (F, T) in enumerate([(20, 32), (33, 129), (8, 8)]):
        w = synth.PlainWorkload(f"sl{i}", F=F, B=B, T=T, N=N, frames=3, tau=float((2 + i) * B), seed=900 + i,
                                p=0.3 + 0.2 * i)
        x = w.frames_tensor(0, 3)
        xs, taps, H, tau = _scaled(w, x, a, b, hs)
        sid = srv.open(F, T, float(tau), taps, H)
        xd = xs.reshape(3, -1).cuda()
        srv.submit(sid, xd)
        cases.append((w, sid, xs, xd, taps, H, tau))
    res = {sid: [] for _, sid, *_ in cases}
    for _ in range(50):
        srv.step()
        srv.sync()
        for _, sid, *_ in cases:
            while (r := srv.pull(sid)) is not None:
                res[sid].append(r)
        if all(len(res[sid]) == 3 for _, sid, *_ in cases):
            break
    for w, sid, xs, xd, taps, H, tau in cases:
        srv.close(sid)
        _check(w.F, B, w.T, N, tau, taps, H, xs, res[sid])
    srv.close_server()
