"""The DPD oracle and the DPD graph pinned to the paper's model and to closed
forms: the graph satisfies the design rules and decomposes into one DC per
filter branch (Sec. IV-V); its FIFOs balance for every control value and no
interleaving deadlocks; the filter arithmetic reduces to plain convolutions
in the special cases below, and an inactive branch keeps its delay token."""
import itertools

import numpy as np
import pytest

from oracle import analysis as A
from oracle import dpd as D


def _rc(rng, *shape, scale=1.0):
    return scale * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2)


# ----------------------------------------------------------------- the graph

@pytest.mark.parametrize("K", [2, 10])
def test_dpd_graph_rules_dcs_and_consistency(K):
    g = A.dpd_graph(K)
    assert not A.check_rates(g) and not A.check_actor_types(g) and not A.design_rule_violations(g)
    dcs = A.find_dcs(g, "CONF", "POLY", "ADD")
    assert sorted(sorted(d) for d in dcs) == sorted([[f"FIR_{k}"] for k in range(K)])
    errs, elem = A.dpg_validity(g, "CONF", "POLY", "ADD")
    assert not errs and sorted(elem.values()) == list(range(1, K + 1))
    ok, _, _ = A.dpg_consistency(g, "CONF", "POLY", "ADD")
    assert ok


def test_dpd_rate_balance_for_every_control_value():
    g = A.dpd_graph(10)
    for bits in itertools.product((0, 1), repeat=10):
        assert all(b == 0 for b in A.rate_balance(g, "CONF", "POLY", "ADD", bits).values())


@pytest.mark.parametrize("L,C", [(2, 1), (2, 2), (3, 1)])
def test_dpd_graph_never_deadlocks(L, C):
    r = A.search(A.dpd_graph(2), L, C, source="SRC", config="CONF", sink="SINK")
    assert r.sequences == 4 ** L and not r.deadlocks and not r.unbalanced


# ------------------------------------------------------------- the arithmetic

def test_basis_closed_form():
    x = np.array([0.0, 1.0, -2.0, 3j, 1 + 1j])
    for k in range(1, 6):
        assert np.allclose(D.psi(x, k), x * np.abs(x) ** (k - 1), rtol=0, atol=0)
    assert np.allclose(D.psi(x, 1), x)
    assert np.allclose(D.psi(x, 3), x * (x.real ** 2 + x.imag ** 2))


def test_branch_one_always_active_is_one_fir_over_the_stream():
    # psi_1(x) = x: the DPD output is the convolution of the whole stream
    rng = np.random.default_rng(1)
    P, period, T = 5, 64, 10
    x = _rc(rng, P * period, scale=0.5)
    taps = np.zeros((3, T), complex)
    taps[0] = _rc(rng, T)
    taps[1:] = _rc(rng, 2, T)                       # inactive branches: never used
    y, h = D.run(x, [1] * P, taps, period)
    assert np.allclose(y, np.convolve(x, taps[0])[:x.size], atol=1e-12)
    assert np.allclose(h[0], x[-(T - 1):]) and np.all(h[1:] == 0)


def test_impulse_gives_scaled_taps_of_each_active_branch():
    P, period, T, K = 2, 32, 10, 4
    rng = np.random.default_rng(2)
    taps = _rc(rng, K, T)
    a = 0.6 - 0.3j
    x = np.zeros(P * period, complex)
    x[period + 5] = a
    masks = [0b1111, 0b0101]                         # period 1: branches 1 and 3
    y, _ = D.run(x, masks, taps, period)
    expect = np.zeros_like(y)
    for k in (1, 3):
        expect[period + 5:period + 5 + T] += a * abs(a) ** (k - 1) * taps[k - 1]
    assert np.allclose(y, expect, atol=1e-14)


def test_inactive_branch_keeps_its_delay_token():
    # branch 2 fires in period 0, sits out period 1, fires in period 2: its
    # first outputs in period 2 continue from the end of period 0
    rng = np.random.default_rng(3)
    period, T = 40, 10
    x = _rc(rng, 3 * period, scale=0.7)
    taps = np.zeros((2, T), complex)
    taps[1] = _rc(rng, T)
    y, h = D.run(x, [0b10, 0b00, 0b10], taps, period)
    spliced = np.concatenate([x[:period], x[2 * period:]])       # what FIR_2 consumed
    y2 = np.convolve(D.psi(spliced, 2), taps[1])[:2 * period]
    assert np.allclose(y[:period], y2[:period], atol=1e-12)
    assert np.all(y[period:2 * period] == 0)
    assert np.allclose(y[2 * period:], y2[period:], atol=1e-12)
    assert np.allclose(h[1], D.psi(x[-(T - 1):], 2))


def test_all_active_is_the_sum_of_stream_firs_and_linear_in_the_taps():
    rng = np.random.default_rng(4)
    P, period, T, K = 4, 50, 10, 10
    x = _rc(rng, P * period, scale=0.5)
    t1, t2 = _rc(rng, K, T), _rc(rng, K, T)
    hist = _rc(rng, K, T - 1, scale=0.3)
    y, _ = D.run(x, [(1 << K) - 1] * P, t1, period, hist)
    ref = sum(np.convolve(np.concatenate([hist[k], D.psi(x, k + 1)]), t1[k])[T - 1:T - 1 + x.size] for k in range(K))
    assert np.allclose(y, ref, atol=1e-10)
    masks = rng.integers(0, 1 << K, P)
    ya, _ = D.run(x, masks, t1, period, hist)
    yb, _ = D.run(x, masks, t2, period, hist)
    yab, _ = D.run(x, masks, t1 + t2, period, hist)
    assert np.allclose(yab, ya + yb, atol=1e-10)


def test_split_run_with_the_tokens_handed_over_equals_one_run():
    rng = np.random.default_rng(5)
    P, period, T, K = 6, 30, 10, 10
    x = _rc(rng, P * period, scale=0.5)
    taps = _rc(rng, K, T)
    masks = rng.integers(0, 1 << K, P)
    y, h = D.run(x, masks, taps, period)
    ya, ha = D.run(x[:3 * period], masks[:3], taps, period)
    yb, hb = D.run(x[3 * period:], masks[3:], taps, period, ha)
    assert np.allclose(np.concatenate([ya, yb]), y, atol=0) and np.allclose(hb, h, atol=0)
