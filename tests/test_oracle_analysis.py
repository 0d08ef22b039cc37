"""MoC-level oracle checks: eq. (1), design rules 1-5 with the Fig. 4
situations rebuilt from the text, the DC procedure on the Fig. 5 example,
DPG validity and consistency (Theorem of Sec. V), rate balance for every
admissible control value, and a brute-force deadlock search with negative
controls that break rule 1 and rule 2."""
import itertools
import os

import numpy as np
import pytest

import oracle
from oracle import analysis as A


def _dyn_pair_graph():
    """q controls x (output DRP px) and y (input DRP py) linked through a1."""
    g = A.Graph()
    for a, k in (("q", A.CONFIG), ("x", A.DYNAMIC), ("y", A.DYNAMIC), ("a1", A.STATIC), ("s", A.STATIC)):
        g.add_actor(a, k)
    g.add_port("s", "o", True, A.SRP, 1)
    g.add_port("q", "i", False, A.SRP, 1)
    g.add_port("q", "c", True, A.CTRL_OUT, 1)
    g.add_port("x", "c", False, A.CTRL_IN, 1)
    g.add_port("x", "px", True, A.DRP, 1)
    g.add_port("y", "c", False, A.CTRL_IN, 1)
    g.add_port("y", "py", False, A.DRP, 1)
    g.add_port("a1", "i", False, A.SRP, 1)
    g.add_port("a1", "o", True, A.SRP, 1)
    g.connect("fs", ("s", "o"), ("q", "i"), 1)
    g.connect("fcx", ("q", "c"), ("x", "c"), 1)
    g.connect("fcy", ("q", "c"), ("y", "c"), 1)
    g.connect("fx", ("x", "px"), ("a1", "i"), 1)
    g.connect("fy", ("a1", "o"), ("y", "py"), 1)
    g.table[(("q", "c"), ("x", "px"))] = 1
    g.table[(("q", "c"), ("y", "py"))] = 1
    return g


def test_eq1_fig1_dynamic_actor():
    # Fig. 1: f1, f2, f3 have rates 1, 1, 2; p1 is the control port, p2 a DRP
    # (atr 1, itr 0), p3 an SRP of rate 2.
    g = A.Graph()
    for a, k in (("q", A.CONFIG), ("x", A.DYNAMIC), ("a", A.STATIC), ("b", A.STATIC)):
        g.add_actor(a, k)
    g.add_port("q", "c", True, A.CTRL_OUT, 1)
    g.add_port("a", "o", True, A.SRP, 1)
    g.add_port("x", "p1", False, A.CTRL_IN, 1)
    g.add_port("x", "p2", False, A.DRP, 1)
    g.add_port("x", "p3", True, A.SRP, 2)
    g.add_port("b", "i", False, A.SRP, 2)
    g.connect("f1", ("q", "c"), ("x", "p1"), 1)
    g.connect("f2", ("a", "o"), ("x", "p2"), 1)
    g.connect("f3", ("x", "p3"), ("b", "i"), 2)
    g.table[(("q", "c"), ("x", "p2"))] = 1
    assert A.check_rates(g) == [] and A.check_actor_types(g) == []
    assert A.tokrate(g, ("x", "p2"), [True]) == 1
    assert A.tokrate(g, ("x", "p2"), [False]) == 0
    assert A.tokrate(g, ("x", "p3"), [False]) == 2 == A.tokrate(g, ("x", "p3"), [True])
    # a rate mismatch between a port and its FIFO is a semantic error
    g.fifos[2].rate = 3
    assert A.check_rates(g)


def test_fig4a_rule1_linked_port_control():
    g = _dyn_pair_graph()
    assert A.linked(g, ("x", "px"), ("y", "py"))
    assert A.rule1(g) == []
    g.table[(("q", "c"), ("y", "py"))] = 2
    assert A.rule1(g)


def test_fig4b_rule2_balanced_delay():
    g = _dyn_pair_graph()
    assert A.rule2(g) == []
    for f in g.fifos:
        if f.name == "fcy":
            f.delay = 1
    assert A.rule2(g)
    for f in g.fifos:
        if f.name == "fcx":
            f.delay = 1
    assert A.rule2(g) == []


def test_fig4c_rule3_shared_subchain_actor():
    # a2 is on the subchain (a1, a2) of x, y and also on a subchain of z, y.
    g = A.Graph()
    for a, k in (("q", A.CONFIG), ("x", A.DYNAMIC), ("y", A.DYNAMIC), ("z", A.DYNAMIC),
                 ("a1", A.STATIC), ("a2", A.STATIC)):
        g.add_actor(a, k)
    g.add_port("q", "c", True, A.CTRL_OUT, 1)
    for d in ("x", "y", "z"):
        g.add_port(d, "c", False, A.CTRL_IN, 1)
        g.connect(f"fc{d}", ("q", "c"), (d, "c"), 1)
    g.add_port("x", "px", True, A.DRP, 1)
    g.add_port("z", "pz", True, A.DRP, 1)
    g.add_port("y", "py", False, A.DRP, 1)
    g.add_port("a1", "i", False, A.SRP, 1)
    g.add_port("a1", "o", True, A.SRP, 1)
    g.add_port("a2", "i", False, A.SRP, 1)
    g.add_port("a2", "i2", False, A.SRP, 1)
    g.add_port("a2", "o", True, A.SRP, 1)
    g.connect("f1", ("x", "px"), ("a1", "i"), 1)
    g.connect("f2", ("a1", "o"), ("a2", "i"), 1)
    g.connect("f3", ("z", "pz"), ("a2", "i2"), 1)
    g.connect("f4", ("a2", "o"), ("y", "py"), 1)
    for p in (("x", "px"), ("z", "pz"), ("y", "py")):
        g.table[(("q", "c"), p)] = 1
    errs = A.rule3(g)
    assert any("a2" in e for e in errs)


def test_fig4d_rule4_single_sided_dynamism():
    g = _dyn_pair_graph()
    assert A.rule4(g) == []
    g.add_port("x", "pin", False, A.DRP, 1)
    assert A.rule4(g)


def test_fig4e_rule5_encapsulation():
    g = _dyn_pair_graph()
    assert A.rule5(g) == []
    g.add_actor("b", A.STATIC)
    g.add_port("b", "o", True, A.SRP, 1)
    g.add_port("a1", "i3", False, A.SRP, 1)
    g.connect("fb", ("b", "o"), ("a1", "i3"), 1)
    assert any(e.startswith("rule 5") for e in A.rule5(g))


def _fig5_graph():
    """DPG of Fig. 5: linked DRPs {px1,py1}, {px2,py1} through a1, a2, a3;
    {px3,py2} through a4; {px4,py3} on one FIFO."""
    g = A.Graph()
    for a, k in (("q", A.CONFIG), ("x", A.DYNAMIC), ("y", A.DYNAMIC)):
        g.add_actor(a, k)
    for a in ("a1", "a2", "a3", "a4"):
        g.add_actor(a, A.STATIC)
    g.add_port("q", "c", True, A.CTRL_OUT, 1)
    for d in ("x", "y"):
        g.add_port(d, "c", False, A.CTRL_IN, 1)
        g.connect(f"fc{d}", ("q", "c"), (d, "c"), 1)
    for i in range(1, 5):
        g.add_port("x", f"px{i}", True, A.DRP, 1)
    for j in range(1, 4):
        g.add_port("y", f"py{j}", False, A.DRP, 1)

    def st(a, *ports):
        for p, out in ports:
            g.add_port(a, p, out, A.SRP, 1)
    st("a1", ("i", False), ("o", True))
    st("a2", ("i", False), ("o", True))
    st("a3", ("i1", False), ("i2", False), ("o", True))
    st("a4", ("i", False), ("o", True))
    g.connect("e1", ("x", "px1"), ("a1", "i"), 1)
    g.connect("e2", ("x", "px2"), ("a2", "i"), 1)
    g.connect("e3", ("a1", "o"), ("a3", "i1"), 1)
    g.connect("e4", ("a2", "o"), ("a3", "i2"), 1)
    g.connect("e5", ("a3", "o"), ("y", "py1"), 1)
    g.connect("e6", ("x", "px3"), ("a4", "i"), 1)
    g.connect("e7", ("a4", "o"), ("y", "py2"), 1)
    g.connect("e8", ("x", "px4"), ("y", "py3"), 1)
    for p, e in ((("x", "px1"), 1), (("x", "px2"), 1), (("y", "py1"), 1), (("x", "px3"), 2),
                 (("y", "py2"), 2), (("x", "px4"), 3), (("y", "py3"), 3)):
        g.table[(("q", "c"), p)] = e
    return g


def _golden(name):
    out = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", name)) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                k, *v = line.split()
                out.setdefault(k, []).append(v)
    return out


def test_fig5_dc_procedure():
    gold = _golden("fig5_dc_example.txt")
    g = _fig5_graph()
    pairs = {(a[1], b[1]) for a, b in A.linked_drp_pairs(g)}
    assert pairs == {tuple(p.split("-")) for p in gold["linked"][0]}
    dcs = set(A.find_dcs(g, "q", "x", "y"))
    want = {frozenset(d[0].split(",")) for d in gold["dc"]}
    # the dummy actor is named after the FIFO it was inserted on (e8)
    assert {frozenset("d" if a.startswith("d:") else a for a in dc) for dc in dcs} == want
    assert len(dcs) == int(gold["M"][0][0])
    assert 1 <= len(dcs) <= min(4, 3)
    errs, elem = A.dpg_validity(g, "q", "x", "y")
    assert errs == [] and sorted(elem.values()) == [1, 2, 3]
    assert A.design_rule_violations(g) == []
    # two DCs on one control element break the bijection
    g.table[(("q", "c"), ("x", "px3"))] = 1
    g.table[(("q", "c"), ("y", "py2"))] = 1
    assert A.dpg_validity(g, "q", "x", "y")[0]


@pytest.mark.parametrize("F", [1, 2, 3, 4, 8])
def test_canonical_graph_satisfies_rules_and_is_a_valid_dpg(F):
    g = A.canonical_graph(F)
    assert A.design_rule_violations(g) == []
    dcs = A.find_dcs(g, "DET", "SEL", "SINK")
    assert sorted(map(sorted, dcs)) == [[f"HX_{b}"] for b in range(F)]   # M = F
    errs, elem = A.dpg_validity(g, "DET", "SEL", "SINK")
    assert errs == [] and sorted(elem.values()) == list(range(1, F + 1))
    ok, bounds, beta = A.dpg_consistency(g, "DET", "SEL", "SINK")
    assert ok and all(beta[f"f6_{b}"] == 1 and beta[f"f7_{b}"] == 1 for b in range(F))


@pytest.mark.parametrize("F", [1, 3, 10])
def test_rate_balance_for_every_admissible_control_value(F):
    g = A.canonical_graph(F)
    for v in itertools.product((0, 1), repeat=F):
        bal = A.rate_balance(g, "DET", "SEL", "SINK", v)
        assert all(d == 0 for d in bal.values()), (v, bal)


def test_oracle_peaks_respect_the_dpg_buffer_bound():
    rng = np.random.default_rng(11)
    F, B, T, N = 4, 8, 3, 2
    taps = (rng.standard_normal(T) + 1j * rng.standard_normal(T)).astype(np.complex64) * 0.5
    x = (rng.standard_normal((6, F, B)) + 1j * rng.standard_normal((6, F, B))).astype(np.complex64)
    x[:, 1::2] *= 4
    r = oracle.run(F, B, T, N, 30.0, taps, np.eye(N, dtype=np.complex64), x)
    _, _, beta = A.dpg_consistency(A.canonical_graph(F), "DET", "SEL", "SINK")
    assert r.stats["f6"][2] <= max(beta[f"f6_{b}"] for b in range(F))
    assert r.stats["f7"][2] <= max(beta[f"f7_{b}"] for b in range(F))


@pytest.mark.parametrize("F,L", [(1, 4), (2, 3), (3, 2)])
@pytest.mark.parametrize("C", [1, 2, 3])
def test_canonical_graph_never_deadlocks(F, L, C):
    r = A.search(A.canonical_graph(F), L, C)
    assert r.sequences == 2 ** (F * L)
    assert r.deadlocks == [] and r.unbalanced == []


def test_negative_control_rule1_broken_deadlocks():
    r = A.search(A.canonical_graph(2, swap_sink_elements=(0, 1)), 2, 3)
    assert r.deadlocks
    seq = r.deadlocks[0][0]
    assert any(v[0] != v[1] for v in seq)       # only mixed control values expose it


def test_negative_control_rule2_broken_is_caught():
    r4 = A.search(A.canonical_graph(2, delay_f4=1), 2, 3)
    assert r4.deadlocks                           # SEL one control token behind
    r5 = A.search(A.canonical_graph(2, delay_f5=1), 2, 3)
    assert r5.deadlocks or r5.unbalanced          # SINK one token ahead
