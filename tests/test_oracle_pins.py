"""The oracle pinned against values the paper and the mathematics fix.

Each test is chosen so that a plausible slip in the oracle fails it: a dropped
cross term or a conjugated tap (impulse response with complex taps, numpy
convolution), a lost delay token or an off-by-one in the history (impulse
across a frame boundary), a transposed H or a column-major reshape (cyclic
shift), a mean instead of a sum or a non-strict threshold (exact energies and
ties), miscounted tokens (conservation), and eq. (2) (the worked example of
Fig. 6 and the linear buffer replay).
"""
import os

import numpy as np
import pytest

import oracle


def _rand_c(rng, *shape, scale=1.0):
    return (scale * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2)).astype(np.complex64)


def _fir_only(F, B, T, taps, x, tau=-1.0, C=3, hist_in=None):
    """Graph with H = I and tau below every energy: every block is selected and
    the sink output equals the FIR output."""
    N = 1
    return oracle.run(F, B, T, N, tau, taps, np.eye(N, dtype=np.complex64), x, C=C, hist_in=hist_in)


def test_fir_impulse_response_is_taps():
    # Sec. III-D delays + FIR definition: x = delta[n] gives y[n] = h[n].
    rng = np.random.default_rng(0)
    F, B, T = 4, 8, 5
    taps = _rand_c(rng, T)
    x = np.zeros((2, F, B), np.complex64)
    x[0, 0, 0] = 1.0
    r = _fir_only(F, B, T, taps, x)
    y = oracle.scatter(r, F, B).reshape(-1)
    expect = np.zeros_like(y)
    expect[:T] = taps
    assert np.array_equal(y, expect.astype(np.complex128))


def test_fir_impulse_across_frame_boundary_uses_delay_token():
    # The last sample of frame 0 must ring into frame 1 through the f1 token.
    rng = np.random.default_rng(1)
    F, B, T = 2, 4, 6
    taps = _rand_c(rng, T)
    x = np.zeros((3, F, B), np.complex64)
    x[0, -1, -1] = 2.0 - 1.0j
    r = _fir_only(F, B, T, taps, x)
    y = oracle.scatter(r, F, B).reshape(3, F * B)
    L = F * B
    stream = y.reshape(-1)
    expect = np.zeros(3 * L, np.complex128)
    for t in range(T):
        expect[L - 1 + t] = (2.0 - 1.0j) * complex(taps[t])
    assert np.allclose(stream, expect, rtol=0, atol=1e-12)
    assert np.abs(stream[L:L + T - 1]).min() > 0  # carried into frame 1


def test_fir_matches_numpy_convolution_over_many_frames():
    rng = np.random.default_rng(2)
    F, B, T, n = 3, 16, 7, 5
    taps = _rand_c(rng, T)
    x = _rand_c(rng, n, F, B)
    r = _fir_only(F, B, T, taps, x)
    y = oracle.scatter(r, F, B).reshape(-1)
    ref = np.convolve(x.reshape(-1).astype(np.complex128), taps.astype(np.complex128))[: n * F * B]
    assert np.allclose(y, ref, rtol=0, atol=1e-12)


def test_fir_history_in_and_out():
    # Splitting a stream in two runs with the delay token handed over gives the
    # same output as one run.
    rng = np.random.default_rng(3)
    F, B, T = 2, 8, 9
    taps = _rand_c(rng, T)
    x = _rand_c(rng, 6, F, B)
    whole = oracle.scatter(_fir_only(F, B, T, taps, x), F, B)
    r1 = _fir_only(F, B, T, taps, x[:2])
    r2 = _fir_only(F, B, T, taps, x[2:], hist_in=r1.hist_out)
    split = np.concatenate([oracle.scatter(r1, F, B), oracle.scatter(r2, F, B)])
    assert np.allclose(whole, split, rtol=0, atol=1e-12)
    assert np.allclose(r1.hist_out, x[1].reshape(-1)[-(T - 1):].astype(np.complex128), atol=0)


def test_hx_identity_and_cyclic_shift_fix_the_reshape():
    # HX_b: X = reshape(block, (B/N, N)) row-major, out[jN+i] = sum_k H[i][k] X[j][k].
    rng = np.random.default_rng(4)
    F, B, T, N = 3, 12, 1, 4
    x = _rand_c(rng, 2, F, B)
    taps = np.array([1.0], np.complex64)
    ident = oracle.run(F, B, T, N, -1.0, taps, np.eye(N, dtype=np.complex64), x)
    assert np.array_equal(oracle.scatter(ident, F, B), x.astype(np.complex128))
    shift = np.zeros((N, N), np.complex64)
    for i in range(N):
        shift[i, (i + 1) % N] = 1.0
    rs = oracle.run(F, B, T, N, -1.0, taps, shift, x)
    got = oracle.scatter(rs, F, B).reshape(2, F, B // N, N)
    xr = x.reshape(2, F, B // N, N).astype(np.complex128)
    assert np.array_equal(got, np.roll(xr, -1, axis=-1))
    # a general H against numpy's matmul on the row-major reshape
    H = _rand_c(rng, N, N)
    rg = oracle.run(F, B, T, N, -1.0, taps, H, x)
    ref = np.einsum("ik,fbjk->fbji", H.astype(np.complex128), xr)
    assert np.allclose(oracle.scatter(rg, F, B).reshape(ref.shape), ref, atol=1e-12)


def test_det_energy_is_block_sum_and_threshold_is_strict():
    # E_b = sum over the block of |y|^2 ; v[b] = E_b > tau (strict).
    F, B, T, N = 4, 8, 1, 2
    taps = np.array([1.0], np.complex64)
    x = np.zeros((1, F, B), np.complex64)
    x[0, 0, :] = 1.0            # E = 8
    x[0, 1, :] = 1.0 + 1.0j     # E = 16
    x[0, 2, :3] = 2.0           # E = 12
    x[0, 3, :] = 0.5j           # E = 2
    r = oracle.run(F, B, T, N, 12.0, taps, np.eye(N, dtype=np.complex64), x)
    assert np.array_equal(r.energy[0], [8.0, 16.0, 12.0, 2.0])
    assert list(r.idx[0]) == [1] and r.c[0] == 1          # 12 is not > 12
    r = oracle.run(F, B, T, N, 7.999, taps, np.eye(N, dtype=np.complex64), x)
    assert list(r.idx[0]) == [0, 1, 2] and r.c[0] == 3    # ascending order


def test_tau_extremes():
    rng = np.random.default_rng(5)
    F, B, T, N = 5, 8, 3, 4
    taps, H = _rand_c(rng, T), _rand_c(rng, N, N)
    x = _rand_c(rng, 3, F, B)
    r = oracle.run(F, B, T, N, -1.0, taps, H, x)
    assert list(r.c) == [F] * 3 and all(list(i) == list(range(F)) for i in r.idx)
    r = oracle.run(F, B, T, N, np.inf, taps, H, x)
    assert list(r.c) == [0] * 3 and r.fires["SINK"] == 3   # the sink still fires
    assert r.stats["f6"][0] == 0 and r.fires["HX"] == 0


def test_token_conservation_and_rates():
    rng = np.random.default_rng(6)
    F, B, T, N, n = 6, 8, 4, 2, 7
    taps, H = _rand_c(rng, T, scale=0.5), _rand_c(rng, N, N)
    x = _rand_c(rng, n, F, B)
    x[:, ::2] *= 4
    r = oracle.run(F, B, T, N, 40.0, taps, H, x)
    C = int(np.sum(r.c))
    assert 0 < C < n * F
    s = r.stats
    assert s["f0"][:2] == (n * F, n * F)
    assert s["f1"][:2] == (n, n) and s["f1"][3] == 1          # delay token stays
    assert s["f2"][:2] == (n * F, n * F) and s["f3"][:2] == (n * F, n * F)
    assert s["f4"][:2] == (n, n) and s["f5"][:2] == (n, n)
    assert s["f6"][:2] == (C, C) and s["f7"][:2] == (C, C)   # DPG fires at rate c
    for name, (w, rd, peak, occ) in s.items():
        delay = 1 if name == "f1" else 0
        assert occ == delay + w - rd == delay                    # returns to delays
        cap_tok = oracle.fifo_capacity(F if name in ("f0", "f2", "f3") else 1, delay, 3)
        assert peak <= cap_tok
    assert r.fires == {"SRC": n, "FIR": n, "DET": n, "SEL": n, "HX": C, "SINK": n}


def test_buffering_constant_does_not_change_results():
    rng = np.random.default_rng(7)
    F, B, T, N = 3, 8, 5, 4
    taps, H = _rand_c(rng, T), _rand_c(rng, N, N)
    x = _rand_c(rng, 4, F, B)
    x[:, 1] *= 4
    ref = oracle.run(F, B, T, N, 20.0, taps, H, x, C=3)
    for C in (1, 2, 5):
        r = oracle.run(F, B, T, N, 20.0, taps, H, x, C=C)
        assert np.array_equal(r.c, ref.c)
        assert all(np.array_equal(a, b) for a, b in zip(r.y, ref.y))


def _golden(name):
    out = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", name)) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                k, *v = line.split()
                out.setdefault(k, []).append(v)
    return out


def test_eq2_worked_example_fig6():
    # r = 4, Q = 1, C = 3: 13 slots; D in slot 0, first write 1..4, first read
    # 0..3, third write ends at slot 12, then slot 12 is copied to slot 0.
    g = _golden("fig6_triple_buffer.txt")
    r, Q, C = (int(g[k][0][0]) for k in ("r", "Q", "C"))
    assert oracle.fifo_capacity(r, Q, C) == int(g["slots"][0][0])
    wants_w = [int(v) for v in g["write_starts"][0]]
    wants_r = [int(v) for v in g["read_starts"][0]]
    err, wp, rp = oracle.linear_fifo_replay(r, Q, C, len(wants_w))
    assert err == 0
    assert wp == wants_w
    assert rp == wants_r
    # the "otherwise" branch: Q a multiple of r
    assert oracle.fifo_capacity(4, 0, 2) == 8 and oracle.fifo_capacity(2, 8, 3) == 8
    assert oracle.fifo_capacity(1, 1, 3) == 3


@pytest.mark.parametrize("r,Q,C", [(4, 1, 3), (4, 3, 2), (3, 5, 3), (1, 0, 1), (2, 2, 2),
                                   (4, 0, 3), (5, 7, 3), (1, 1, 3), (6, 2, 2)])
def test_eq2_capacity_serves_the_linear_access_pattern(r, Q, C):
    err, _, _ = oracle.linear_fifo_replay(r, Q, C, 50)
    assert err == 0
    if Q % r != 0:
        # one slot fewer than eq. (2) and a window runs off the buffer
        err2, _, _ = oracle.linear_fifo_replay(r, Q, C, 50, cap_override=oracle.fifo_capacity(r, Q, C) - 1)
        assert err2 != 0
