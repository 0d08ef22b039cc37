"""The native graph front end (prune_model_*, host code) against the oracle's
MoC analysis, on the canonical and DPD graphs, the Fig. 5 example, rule
breaking variants and seeded random graphs: design-rule verdicts, DPGs, DC
decompositions, validity, consistency and buffer bounds agree, and the
runtime forms are recognised."""
import random

import numpy as np

import pytest

from oracle import analysis as A
from paper_1802_06625_b300 import model as M

import test_oracle_analysis as T


def to_model(g):
    kinds = {A.STATIC: M.STATIC, A.DYNAMIC: M.DYNAMIC, A.CONFIG: M.CONFIG}
    pkinds = {A.SRP: M.SRP, A.DRP: M.DRP, A.CTRL_IN: M.CTRL_IN, A.CTRL_OUT: M.CTRL_OUT}
    m = M.Model()
    for a, k in g.actors.items():
        m.add_actor(a, kinds[k])
    for p in g.ports.values():
        m.add_port(p.actor, p.name, p.out, pkinds[p.kind], p.atr)
    for f in g.fifos:
        m.connect(f.src, f.dst, f.rate, f.delay, name=f.name)
    for (q, d), e in g.table.items():
        m.set_control(q, d, e)
    return m


def oracle_verdicts(g):
    return {"rates": bool(A.check_rates(g)), "types": bool(A.check_actor_types(g)),
            "rules": [bool(r(g)) for r in (A.rule1, A.rule2, A.rule3, A.rule4, A.rule5)]}


def model_verdicts(rep):
    return {"rates": rep["rate_errors"] > 0, "types": rep["type_errors"] > 0,
            "rules": [e > 0 for e in rep["rule_errors"]]}


def compare(g):
    m = to_model(g)
    rep = m.check()
    assert model_verdicts(rep) == oracle_verdicts(g), (rep, oracle_verdicts(g))
    for d in m.dpgs():
        q, x, y = d["q"], d["x"], d["y"]
        dcs = set(A.find_dcs(g, q, x, y))
        assert {s for s, _ in d["dcs"]} == dcs
        errs, _ = A.dpg_validity(g, q, x, y)
        assert d["valid"] == (not errs), errs
        ok, _, beta = A.dpg_consistency(g, q, x, y)
        assert d["consistent"] == (d["valid"] and ok)
        if d["consistent"]:
            for fi, fname in enumerate(m.fifos):
                assert m.buffer_bound(fi) == beta.get(fname, 0), fname
    return m, rep


@pytest.mark.parametrize("F", [1, 2, 3, 5])
def test_canonical_graph(F):
    m, rep = compare(A.canonical_graph(F))
    assert rep["n_dpgs"] == 1 and rep["consistent"] and not any(rep["rule_errors"])
    assert m.classify() == ("canonical", F)


@pytest.mark.parametrize("K", [1, 2, 4, 10])
def test_dpd_graph(K):
    m, rep = compare(A.dpd_graph(K))
    assert rep["n_dpgs"] == 1 and rep["consistent"]
    assert m.classify() == ("dpd", K)


def test_rule_breaking_canonical_variants():
    _, rep = compare(A.canonical_graph(3, swap_sink_elements=(0, 2)))
    assert rep["rule_errors"][0] > 0
    m, rep = compare(A.canonical_graph(2, delay_f4=1))
    assert rep["rule_errors"][1] > 0 and m.classify() == (None, 0)


def test_fig5_example_and_fig4_base_graph():
    compare(T._fig5_graph())
    compare(T._dyn_pair_graph())


def test_canonical_graph_at_the_bench_size():
    # 4096 DCs: the front end stays polynomial (block-cut trees, components)
    m, rep = compare_light(A.canonical_graph(4096))
    assert rep["consistent"] and m.classify() == ("canonical", 4096)


def compare_light(g):
    m = to_model(g)
    rep = m.check()
    assert not any(rep["rule_errors"]) and rep["rate_errors"] == 0 and rep["type_errors"] == 0
    return m, rep


def random_graph(seed):
    """A configuration actor q, dynamic actors x (output DRPs) and y (input
    DRPs), static actors on chains between them and a few perturbations
    that break one rule or another."""
    r = random.Random(seed)
    g = A.Graph()
    for a, k in (("S", A.STATIC), ("q", A.CONFIG), ("x", A.DYNAMIC), ("y", A.DYNAMIC), ("Z", A.STATIC)):
        g.add_actor(a, k)
    g.add_port("S", "o", True, A.SRP, 1)
    g.add_port("S", "ox", True, A.SRP, 1)
    g.add_port("q", "i", False, A.SRP, 1)
    g.add_port("q", "c", True, A.CTRL_OUT, 1)
    g.add_port("x", "c", False, A.CTRL_IN, 1)
    g.add_port("x", "i", False, A.SRP, 1)
    g.add_port("y", "c", False, A.CTRL_IN, 1)
    g.add_port("y", "o", True, A.SRP, 1)
    g.add_port("Z", "i", False, A.SRP, 1)
    g.connect("fs", ("S", "o"), ("q", "i"), 1)
    g.connect("fsx", ("S", "ox"), ("x", "i"), 1)
    g.connect("fcx", ("q", "c"), ("x", "c"), 1, delay=r.choice([0, 0, 0, 1]))
    g.connect("fcy", ("q", "c"), ("y", "c"), 1, delay=0)
    g.connect("fz", ("y", "o"), ("Z", "i"), 1)
    n = r.randint(1, 7)
    stat = [f"a{i}" for i in range(n)]
    for a in stat:
        g.add_actor(a, A.STATIC)
    nports = {}

    def port(a, out):
        k = nports.get(a, 0)
        nports[a] = k + 1
        name = f"p{k}"
        g.add_port(a, name, out, A.SRP, 1)
        return (a, name)

    K = r.randint(1, 4)
    L = r.randint(1, 4)
    fid = [0]

    def fifo(src, dst, rate=1, delay=0):
        fid[0] += 1
        g.connect(f"e{fid[0]}", src, dst, rate, delay)

    for k in range(K):
        g.add_port("x", f"o{k}", True, A.DRP, 1)
    for j in range(L):
        g.add_port("y", f"i{j}", False, A.DRP, 1)
    # DRP wiring: x's DRPs to static actors or straight to a y DRP; y's DRPs
    # from static actors (each input port one FIFO)
    y_free = [("y", f"i{j}") for j in range(L)]
    r.shuffle(y_free)
    for k in range(K):
        if y_free and r.random() < 0.2:
            fifo(("x", f"o{k}"), y_free.pop())
        else:
            fifo(("x", f"o{k}"), port(r.choice(stat), False))
    for d in y_free:
        fifo(port(r.choice(stat), True), d)
    # chains among static actors
    for _ in range(r.randint(0, n + 2)):
        a, b = r.choice(stat), r.choice(stat)
        if a == b:
            if r.random() < 0.5:
                fifo(port(a, True), port(a, False), 1, 1)     # self-loop delay
            continue
        rate = 2 if r.random() < 0.1 else 1
        src, dst = port(a, True), port(b, False)
        if rate == 2 and r.random() < 0.5:
            g.ports[src].atr = 2
            g.ports[dst].atr = 2
        fifo(src, dst, rate, r.choice([0, 0, 1]))
    # perturbations
    u = r.random()
    if u < 0.15:                                              # dangling SRP neighbour (rule 5)
        g.add_actor("b", A.STATIC)
        fifo(port(r.choice(stat), True), port("b", False))
    elif u < 0.25:                                            # a second dynamic pair sharing an actor (rule 3)
        g.add_actor("z", A.DYNAMIC)
        g.add_port("z", "c", False, A.CTRL_IN, 1)
        g.add_port("z", "d", True, A.DRP, 1)
        g.add_port("q", "c2", True, A.CTRL_OUT, 1)
        fifo(("q", "c2"), ("z", "c"))
        fifo(("z", "d"), port(r.choice(stat), False))
        g.table[(("q", "c2"), ("z", "d"))] = 1
    elif u < 0.3:                                             # two-sided dynamic actor (rule 4)
        g.add_port("x", "back", False, A.DRP, 1)
        fifo(port(r.choice(stat), True), ("x", "back"))
        g.table[(("q", "c"), ("x", "back"))] = 1
    # control elements: one per DRP of x, y's DRPs mostly the element of a
    # linked DRP of x, sometimes another
    for k in range(K):
        g.table[(("q", "c"), ("x", f"o{k}"))] = r.randint(1, K)
    for j in range(L):
        g.table[(("q", "c"), ("y", f"i{j}"))] = r.randint(0, K)
    return g


def clean_graph(seed):
    """A valid DPG: K chains x.o_k -> c_1 -> ... -> y.i_k (or a direct FIFO)
    with their own control elements, delays, self-loops and rate-2 FIFOs
    inside the chains (buffer bounds above one), sometimes an extra static
    actor given an unconnected DRP (a port-type and a connection error)."""
    r = random.Random(seed)
    g = A.Graph()
    for a, k in (("S", A.STATIC), ("q", A.CONFIG), ("x", A.DYNAMIC), ("y", A.DYNAMIC)):
        g.add_actor(a, k)
    g.add_port("S", "o", True, A.SRP, 1)
    g.add_port("q", "i", False, A.SRP, 1)
    g.add_port("q", "c", True, A.CTRL_OUT, 1)
    g.add_port("x", "c", False, A.CTRL_IN, 1)
    g.add_port("y", "c", False, A.CTRL_IN, 1)
    g.connect("fs", ("S", "o"), ("q", "i"), 1)
    g.connect("fcx", ("q", "c"), ("x", "c"), 1)
    g.connect("fcy", ("q", "c"), ("y", "c"), 1)
    K = r.randint(1, 5)
    n = [0]

    def new_actor():
        n[0] += 1
        a = f"c{n[0]}"
        g.add_actor(a, A.STATIC)
        return a

    for k in range(K):
        g.add_port("x", f"o{k}", True, A.DRP, 1)
        g.add_port("y", f"i{k}", False, A.DRP, 1)
        g.table[(("q", "c"), ("x", f"o{k}"))] = k + 1
        g.table[(("q", "c"), ("y", f"i{k}"))] = k + 1
        length = r.randint(0, 3)
        prev = ("x", f"o{k}")
        for j in range(length):
            a = new_actor()
            rate = 1 if prev[0] == "x" else r.choice([1, 1, 2])
            g.add_port(a, "i", False, A.SRP, rate)
            if prev[0] != "x":
                g.ports[prev].atr = rate
            g.connect(f"e{k}_{j}", prev, (a, "i"), rate, r.choice([0, 0, 1, 2]) if prev[0] != "x" else 0)
            g.add_port(a, "o", True, A.SRP, 1)
            if r.random() < 0.3:
                g.add_port(a, "hin", False, A.SRP, 1)
                g.add_port(a, "hout", True, A.SRP, 1)
                g.connect(f"h{k}_{j}", (a, "hout"), (a, "hin"), 1, 1)
            prev = (a, "o")
        g.connect(f"e{k}_out", prev, ("y", f"i{k}"), 1)
    if r.random() < 0.1:
        a = new_actor()
        g.add_port(a, "bad", True, A.DRP, 1)
    return g


@pytest.mark.parametrize("seed", range(300))
def test_random_graphs(seed):
    compare(random_graph(seed))


@pytest.mark.parametrize("seed", range(200))
def test_random_valid_graphs(seed):
    compare(clean_graph(seed))


# ---------------------------------------------------------------- compile

def _canonical_model(F, **kw):
    return to_model(A.canonical_graph(F, **kw))


@pytest.mark.parametrize("F", [1, 3, 64])
def test_compile_canonical_fills_the_graph_descriptor(F):
    import oracle
    m = _canonical_model(F)
    r = m.compile(B=256, T=16, N=16, C=3, tau=1024.0, taps=np.ones(16, np.complex64),
                  H=np.eye(16, dtype=np.complex64), out_frames=5)
    assert r["form"] == "canonical" and r["units"] == F
    d = r["desc"]
    assert (d.F, d.B, d.T, d.N, d.C, d.out_frames) == (F, 256, 16, 16, 3, 5)
    assert abs(d.tau - 1024.0) < 1e-6 and d.taps and d.H
    # every model FIFO has its runtime FIFO and its eq. (2) capacity
    g = A.canonical_graph(F)
    names = [f.name for f in g.fifos]
    want = {"f0": 0, "f1": 1, "f2": 2, "f3": 3, "f4": 4, "f5": 5}
    for fi, name in enumerate(names):
        role = want.get(name, 6 if name.startswith("f6_") else 7)
        assert r["roles"][fi] == role, (name, r["roles"][fi])
        assert r["capacities"][fi] == oracle.fifo_capacity(g.fifos[fi].rate, g.fifos[fi].delay, 3)


@pytest.mark.parametrize("K", [1, 4, 10])
def test_compile_dpd_fills_the_dpd_arguments(K):
    m = to_model(A.dpd_graph(K))
    r = m.compile(B=4096, T=10, C=3)
    assert (r["form"], r["units"], r["K"], r["T"], r["period"]) == ("dpd", K, K, 10, 4096)
    names = [f.name for f in A.dpd_graph(K).fifos]
    roles = dict(zip(names, r["roles"]))
    assert roles["fx"] == 0 and roles["fcfg"] == 1 and roles["fcp"] == 5 and roles["fca"] == 5 and roles["fy"] == 6
    assert all(roles[f"fp_{k}"] == 2 and roles[f"fh_{k}"] == 3 and roles[f"ff_{k}"] == 4 for k in range(K))


def _rejected(m, **kw):
    from paper_1802_06625_b300._lib import PruneError
    args = dict(B=256, T=16, N=16, C=3, tau=1.0, taps=np.ones(16, np.complex64), H=np.eye(16, dtype=np.complex64))
    args.update(kw)
    with pytest.raises(PruneError) as e:
        m.compile(**args)
    return str(e.value)


def test_compile_rejects_rule_violations_with_the_rule():
    assert "design rule 1" in _rejected(_canonical_model(3, swap_sink_elements=(0, 2)))
    assert "design rule 2" in _rejected(_canonical_model(2, delay_f4=1))


def test_compile_rejects_graphs_outside_the_runtime_forms():
    # the Fig. 5 example: a valid PRUNE graph, but not a form the runtime fires
    msg = _rejected(to_model(T._fig5_graph()))
    assert "not a runtime form" in msg or "DPG" in msg, msg
    # a canonical graph whose FIR keeps two delay tokens
    g = A.canonical_graph(3)
    for f in g.fifos:
        if f.name == "f1":
            f.delay = 2
    assert "delay line" in _rejected(to_model(g))
    # a canonical graph whose FIR has no delay line, with T > 1
    g = A.canonical_graph(3)
    g.fifos = [f for f in g.fifos if f.name != "f1"]
    g.ports = {k: p for k, p in g.ports.items() if not (p.actor == "FIR" and p.name in ("hin", "hout"))}
    assert "no self-loop" in _rejected(to_model(g), T=16)
    # DPD limits of the kernel (17 branches)
    assert "DPD kernel" in _rejected(to_model(A.dpd_graph(17)), B=4096, T=10)
    # C must be positive (eq. (2))
    assert "C must be" in _rejected(_canonical_model(2), C=0)
