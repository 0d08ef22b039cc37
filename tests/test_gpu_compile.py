"""Graphs described through the front end (prune_model_*), compiled by
prune_model_compile into the runtime form that fires them, and fired: the
canonical graph through prune_graph_create with the compiled descriptor, the
DPD graph through prune_dpd_fire with the compiled K, T and period; each
against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from oracle import analysis as A
from oracle import dpd as D
from parity import TOL_REL, compare_frame
from paper_1802_06625_b300 import synth

from test_model_frontend import to_model

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1802_06625_b300 import graph
    return graph


@pytest.mark.parametrize("w", [synth.PLAIN_SMALL,
                               synth.PlainWorkload("cmp32", F=48, B=1024, T=64, N=32, frames=4, tau=4096.0,
                                                   seed=17, p=0.4),
                               synth.PlainWorkload("cmp64", F=20, B=256, T=33, N=64, frames=3, tau=1024.0,
                                                   seed=18, p=0.3)],
                         ids=lambda w: f"F{w.F}_B{w.B}_T{w.T}_N{w.N}")
def test_compiled_canonical_model_fires_like_the_oracle(G, w):
    m = to_model(A.canonical_graph(w.F))
    n = min(w.frames, 6)
    r = m.compile(B=w.B, T=w.T, N=w.N, C=3, tau=w.tau, taps=w.taps().numpy(), H=w.H().numpy(), out_frames=n)
    assert r["form"] == "canonical" and r["units"] == w.F
    g = G.Graph.from_desc(r["desc"])
    x = w.frames_tensor(0, n)
    xd = x.cuda()
    for k in range(0, n, 3):              # f0 holds C = 3 frames
        g.push(xd[k:k + 3])
        assert g.run(sync=True) == min(3, n - k)
    recs = g.pull()
    # the runtime FIFOs got the capacities eq. (2) gives the model's FIFOs
    caps = {role: cap for role, cap in zip(r["roles"], r["capacities"])}
    for role in (0, 2, 3):        # rate F, no delay: F * C tokens
        assert g.capacity(role) == caps[role] == w.F * 3
    g.close()
    ref = oracle.run(w.F, w.B, w.T, w.N, np.float32(w.tau), w.taps().numpy(), w.H().numpy(), x.numpy())
    for k, (frame, c, idx, y) in enumerate(recs):
        assert frame == k
        err, rms, _ = compare_frame(c, idx, y, ref.c[k], ref.idx[k], ref.y[k], ref.energy[k], np.float32(w.tau), w.B)
        assert rms == 0 or err <= TOL_REL * rms, (k, err / rms)


def test_compiled_dpd_model_fires_like_the_oracle():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1802_06625_b300 import dpd
    K, T, period, P = 10, 10, 4096, 12
    m = to_model(A.dpd_graph(K))
    r = m.compile(B=period, T=T, C=3)
    assert r["form"] == "dpd" and (r["K"], r["T"], r["period"]) == (K, T, period)
    rng = np.random.default_rng(5)
    x = ((rng.standard_normal(P * period) + 1j * rng.standard_normal(P * period)) * 0.35).astype(np.complex64)
    taps = ((rng.standard_normal((K, T)) + 1j * rng.standard_normal((K, T))) / np.sqrt(2 * K * T)).astype(np.complex64)
    masks = rng.integers(0, 1 << K, P)
    y, _ = dpd.fire(torch.from_numpy(x).cuda(), torch.from_numpy(masks).cuda(), torch.from_numpy(taps),
                    int(r["period"]))
    ref = D.run(x, masks, taps, period)
    ref = np.asarray(ref[0] if isinstance(ref, tuple) else ref)
    got = y.cpu().numpy().astype(np.complex128)
    rms = float(np.sqrt(np.mean(np.abs(ref) ** 2)))
    assert float(np.max(np.abs(got - ref))) <= TOL_REL * rms
