"""Request loop on the GPU: streams that arrive while others are being fired
join at the next step; every stream's results in the mix equal its results
alone (bit for bit: the same kernels on the same per-stream data) and the
oracle's (exact control, FP32 tolerance); admission by the device-memory
budget; result-FIFO backpressure; the delay token carried across requests."""
import numpy as np
import pytest
import torch

import oracle
from parity import TOL_REL, compare_frame
from paper_1802_06625_b300 import synth

pytestmark = pytest.mark.gpu

SPECS = [(16, 32), (37, 8), (5, 129), (64, 1), (130, 32), (3, 17), (90, 64)]  # (F, T)


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1802_06625_b300 import serve
    return serve


def _workloads(B, N, seed):
    out = []
    for i, (F, T) in enumerate(SPECS):
        n = 3 + (i * 2) % 5
        out.append(synth.PlainWorkload(f"s{i}", F=F, B=B, T=T, N=N, frames=n, tau=float((2 + i % 5) * B),
                                       seed=seed * 100 + i, p=0.15 + 0.1 * (i % 6)))
    return out


def _server(S, B, N, fps, ring, budget=256 << 20, max_streams=8, auto=False):
    return S.Server(B, N, F_max=256, T_max=129, max_streams=max_streams, hbm_budget=budget, frames_per_step=fps,
                    ring=ring, auto_release=auto)


def _drain(srv, sids, results):
    for i, sid in sids.items():
        while True:
            r = srv.pull(sid)
            if r is None:
                break
            results[i].append(r)


def _run_mix(S, ws, B, N):
    """Streams arrive in three waves while earlier ones are in flight; the
    frames of a stream come in two requests."""
    srv = _server(S, B, N, fps=2, ring=4)
    xs = [w.frames_tensor(0, w.frames).reshape(w.frames, -1).cuda() for w in ws]
    results = {i: [] for i in range(len(ws))}
    sids = {}
    waves = [[0, 1, 2], [3, 4], [5, 6]]
    for wave in waves:
        for i in wave:
            w = ws[i]
            sid = srv.open(w.F, w.T, w.tau, w.taps(), w.H())
            assert sid is not None
            sids[i] = sid
            srv.submit(sid, xs[i][:w.frames // 2])               # first request
        for _ in range(2):
            srv.step()
            _drain(srv, sids, results)
        for i in wave:
            srv.submit(sids[i], xs[i][ws[i].frames // 2:])       # second request
    for _ in range(200):
        n = srv.step()
        _drain(srv, sids, results)
        if n == 0:
            srv.sync()
            _drain(srv, sids, results)
            if all(len(results[i]) == ws[i].frames for i in sids):
                break
    for i in sids:
        srv.close(sids[i])
    srv.close_server()
    return xs, results


def _run_alone(S, w, x, B, N):
    srv = _server(S, B, N, fps=1, ring=2)
    sid = srv.open(w.F, w.T, w.tau, w.taps(), w.H())
    srv.submit(sid, x)
    res = []
    for _ in range(4 * w.frames + 4):
        srv.step()
        srv.sync()
        while (r := srv.pull(sid)) is not None:
            res.append(r)
        if len(res) == w.frames:
            break
    srv.close(sid)
    srv.close_server()
    return res


@pytest.mark.parametrize("N", [64, 16])
def test_mix_equals_alone_and_oracle(S, N):
    B = 256
    ws = _workloads(B, N, seed=7 + N)
    xs, mix = _run_mix(S, ws, B, N)
    for i, w in enumerate(ws):
        assert [r[0] for r in mix[i]] == list(range(w.frames)), (i, [r[0] for r in mix[i]])
        alone = _run_alone(S, w, xs[i], B, N)
        assert len(alone) == w.frames
        for a, m in zip(alone, mix[i]):
            assert a[0] == m[0] and a[1] == m[1]
            assert np.array_equal(a[2], m[2]) and np.array_equal(a[3], m[3]), (i, a[0])
        r = oracle.run(w.F, B, w.T, N, np.float32(w.tau), w.taps().numpy(), w.H().numpy(),
                       xs[i].cpu().numpy().reshape(w.frames, w.F, B))
        for k in range(w.frames):
            _, c, idx, y = mix[i][k]
            err, rms, nb = compare_frame(c, idx, y, r.c[k], r.idx[k], r.y[k], r.energy[k], np.float32(w.tau), B)
            if rms > 0:
                assert err <= TOL_REL * rms, (i, k, err / rms)


def test_admission_by_budget(S):
    B, N = 256, 64
    w = synth.PlainWorkload("adm", F=64, B=B, T=32, N=N, frames=2, tau=4.0 * B, seed=31, p=0.25)
    probe = _server(S, B, N, fps=1, ring=2, budget=64 << 20)
    sid = probe.open(w.F, w.T, w.tau, w.taps(), w.H())
    per_stream = probe.stats()["hbm_used"]
    probe.close(sid)
    probe.close_server()
    srv = _server(S, B, N, fps=1, ring=2, budget=2 * per_stream + per_stream // 2)
    a = srv.open(w.F, w.T, w.tau, w.taps(), w.H())
    b = srv.open(w.F, w.T, w.tau, w.taps(), w.H())
    assert a is not None and b is not None
    assert srv.open(w.F, w.T, w.tau, w.taps(), w.H()) is None          # over the budget
    x = w.frames_tensor(0, 2).reshape(2, -1).cuda()
    srv.submit(a, x)
    srv.step()
    srv.close(a)
    srv.sync()                                                        # a's last step done: memory back
    c = srv.open(w.F, w.T, w.tau, w.taps(), w.H())
    assert c is not None and srv.stats()["open"] == 2
    slots = _server(S, B, N, fps=1, ring=2, max_streams=1)
    assert slots.open(w.F, w.T, w.tau, w.taps(), w.H()) is not None
    assert slots.open(w.F, w.T, w.tau, w.taps(), w.H()) is None       # no slot
    slots.close_server()
    srv.close_server()


def test_backpressure_and_auto_release(S):
    B, N = 256, 16
    w = synth.PlainWorkload("bp", F=8, B=B, T=8, N=N, frames=5, tau=4.0 * B, seed=32, p=0.3)
    x = w.frames_tensor(0, 5).reshape(5, -1).cuda()
    srv = _server(S, B, N, fps=1, ring=2)
    sid = srv.open(w.F, w.T, w.tau, w.taps(), w.H())
    srv.submit(sid, x)
    fired = [srv.step() for _ in range(4)]
    srv.sync()
    assert fired == [1, 1, 0, 0] and srv.progress(sid) == (3, 2, 2, 0)   # result FIFO full
    assert srv.pull(sid)[0] == 0
    assert srv.step() == 1
    srv.close_server()
    auto = _server(S, B, N, fps=2, ring=2, auto=True)
    sid = auto.open(w.F, w.T, w.tau, w.taps(), w.H())
    auto.submit(sid, x)
    for _ in range(10):
        auto.step()
        auto.sync()
    assert auto.progress(sid) == (0, 5, 5, 5)
    assert [i for i, _ in auto.poll()] == [sid]                      # idle reported once
    assert auto.poll() == []
    auto.close_server()


def test_delay_token_across_requests_and_periodic_input(S):
    # frames queued as a periodic segment (period 2) fire like the same frames
    # laid out one after another; the delay token crosses requests
    B, N = 256, 64
    w = synth.PlainWorkload("per", F=12, B=B, T=64, N=N, frames=5, tau=3.0 * B, seed=33, p=0.4)
    two = w.frames_tensor(0, 2).reshape(2, -1).cuda()
    laid = torch.cat([two, two, two[:1]]).contiguous()
    srv = _server(S, B, N, fps=3, ring=6)
    a = srv.open(w.F, w.T, w.tau, w.taps(), w.H())
    b = srv.open(w.F, w.T, w.tau, w.taps(), w.H())
    srv.submit(a, two, n=5, period=2)
    srv.submit(b, laid[:1])
    srv.submit(b, laid[1:4])
    srv.submit(b, laid[4:])
    for _ in range(8):
        srv.step()
        srv.sync()
    ra = [srv.pull(a) for _ in range(5)]
    rb = [srv.pull(b) for _ in range(5)]
    for p, q in zip(ra, rb):
        assert p[0] == q[0] and p[1] == q[1] and np.array_equal(p[2], q[2]) and np.array_equal(p[3], q[3])
    r = oracle.run(w.F, B, w.T, N, np.float32(w.tau), w.taps().numpy(), w.H().numpy(),
                   laid.cpu().numpy().reshape(5, w.F, B))
    for k in range(5):
        err, rms, nb = compare_frame(ra[k][1], ra[k][2], ra[k][3], r.c[k], r.idx[k], r.y[k], r.energy[k],
                                     np.float32(w.tau), B)
        if rms > 0:
            assert err <= TOL_REL * rms
    srv.close_server()


def test_serving_workload_sampled_streams(S):
    """The serving workload's 256 streams (B = 512, T = 32, N = 64, F up to
    2048, 10 to 10^4 frames each, inputs read cyclically from the device
    pool) through a server configured as the bench's (256 slots, 40 GB
    budget, 16 frames per step, result rings of 32, two steps in flight),
    admitted in arrival order as room frees up.  Every record is pulled;
    the first, second and last frames of four streams are checked against
    the oracle, each fed the frame before it for its delay token."""
    sw = synth.SERVING
    specs = [sw.stream(i) for i in range(sw.streams)]
    fps = 16
    pool = sw.pool_tensor(device="cuda")
    srv = S.Server(sw.B, sw.N, F_max=sw.F_hi, T_max=sw.T, max_streams=256, hbm_budget=40 << 30,
                   frames_per_step=fps, ring=2 * fps, max_inflight=2, device=0)
    watch = [i for i in range(sw.streams) if specs[i]["frames"] <= 600][:4]
    want = {i: {0, 1, specs[i]["frames"] - 1} for i in watch}
    kept = {i: {} for i in watch}
    pulled = [0] * sw.streams
    nxt, sid_of = 0, {}
    while nxt < sw.streams or sid_of:
        while nxt < sw.streams:  # admission in arrival order
            sp = specs[nxt]
            sid = srv.open(sp["F"], sw.T, sp["tau"], sw.taps(nxt).numpy(), sw.H(nxt).numpy())
            if sid is None:
                break
            L = sp["F"] * sw.B
            srv.submit(sid, pool[sp["offset"]:sp["offset"] + sp["period"] * L], n=sp["frames"], period=sp["period"])
            sid_of[sid] = nxt
            nxt += 1
        n = srv.step()
        moved = 0
        for sid, i in list(sid_of.items()):
            while pulled[i] < specs[i]["frames"]:
                k = pulled[i]
                if i in want and k in want[i]:
                    r = srv.pull(sid)
                    if r is None:
                        break
                    kept[i][k] = r
                elif srv.pull(sid, discard=True) is None:
                    break
                pulled[i] += 1
                moved += 1
            if pulled[i] == specs[i]["frames"]:
                srv.close(sid)
                del sid_of[sid]
        if n == 0 and moved == 0:
            srv.sync()
    srv.sync()
    srv.close_server()
    poolh = pool.cpu()
    for i in watch:
        sp = specs[i]
        L = sp["F"] * sw.B

        def frame(k):  # the stream's frame k: pool frames read cyclically
            o = sp["offset"] + (k % sp["period"]) * L
            return poolh[o:o + L].reshape(sp["F"], sw.B)

        for k in sorted(want[i]):
            xs = torch.stack([frame(j) for j in range(max(0, k - 1), k + 1)]).numpy()
            r = oracle.run(sp["F"], sw.B, sw.T, sw.N, np.float32(sp["tau"]), sw.taps(i).numpy(), sw.H(i).numpy(), xs)
            fr, c, idx, y = kept[i][k]
            assert fr == k
            err, rms, nb = compare_frame(c, idx, y, r.c[-1], r.idx[-1], r.y[-1], r.energy[-1],
                                         np.float32(sp["tau"]), sw.B)
            if rms > 0:
                assert err <= TOL_REL * rms, (i, k, err / rms, nb)
