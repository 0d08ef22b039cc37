"""MoC-level checks of PRUNE graphs (test infrastructure only).

A plain restatement of the paper's definitions on small graph descriptions:

* ports, FIFOs and rates (Sec. III-A): every port of a FIFO has
  ``atr(p) == fiforate(f)``; control ports have rate 1;
* actor types (Sec. III-B) and the control table ``T[j][i]`` (Sec. III-C);
* eq. (1): ``tokrate(p, phi) = BTOI(v_phi[T[q][p]]) * atr(p)``;
* adjacency, simple chains, linked ports and connecting subchains (Sec. IV);
* design rules 1-5 (Sec. IV);
* the DC-finding procedure, DPG validity (bijection between DCs and the
  elements of the control value) and DPG consistency (Sec. V, Theorem);
* eq. (2) FIFO capacities (Sec. VI-B);
* a brute-force search over all control sequences and all interleavings of
  enabled firings of a tiny graph under blocking reads/writes with eq. (2)
  capacities, reporting deadlocks and unbalanced token populations.

Nothing here is used by the CUDA path; it is pinned by the oracle tests.
"""
from __future__ import annotations

import itertools
from collections import deque
from dataclasses import dataclass, field
from fractions import Fraction

STATIC, DYNAMIC, CONFIG = "static", "dynamic", "config"
SRP, DRP, CTRL_IN, CTRL_OUT = "SRP", "DRP", "ctrl_in", "ctrl_out"


@dataclass
class Port:
    actor: str
    name: str
    out: bool            # True for an output port (p+), False for input (p-)
    kind: str            # SRP, DRP, CTRL_IN or CTRL_OUT
    atr: int = 1         # SRP fixed rate / DRP active rate; control ports: 1

    @property
    def key(self):
        return (self.actor, self.name)


@dataclass
class Fifo:
    name: str
    src: tuple           # (actor, port) of the source port p+
    dst: tuple           # (actor, port) of the sink port p-
    rate: int            # fiforate(f)
    delay: int = 0       # initial tokens


@dataclass
class Graph:
    actors: dict = field(default_factory=dict)      # name -> kind
    ports: dict = field(default_factory=dict)       # (actor, port) -> Port
    fifos: list = field(default_factory=list)
    # control table: (control output port key, DRP key) -> element index (1-based)
    table: dict = field(default_factory=dict)

    def add_actor(self, name, kind):
        self.actors[name] = kind

    def add_port(self, actor, name, out, kind, atr=1):
        self.ports[(actor, name)] = Port(actor, name, out, kind, atr)

    def connect(self, fname, src, dst, rate, delay=0):
        self.fifos.append(Fifo(fname, src, dst, rate, delay))

    # ---- derived relations -------------------------------------------------
    def fifos_of(self, pkey):
        return [f for f in self.fifos if f.src == pkey or f.dst == pkey]

    def ports_of(self, actor):
        return [p for p in self.ports.values() if p.actor == actor]

    def cport(self, actor):
        cs = [p for p in self.ports_of(actor) if p.kind == CTRL_IN]
        return cs[0].key if len(cs) == 1 else None

    def drps(self, actor):
        return [p.key for p in self.ports_of(actor) if p.kind == DRP]

    def neighbours(self, actor):
        out = set()
        for f in self.fifos:
            if f.src[0] == actor:
                out.add(f.dst[0])
            if f.dst[0] == actor:
                out.add(f.src[0])
        out.discard(actor)
        return out

    def controller(self, pkey):
        """The control output port that controls DRP ``pkey``: the source of
        the FIFO into the control port of the DRP's parent."""
        c = self.cport(pkey[0])
        if c is None:
            return None
        srcs = [f.src for f in self.fifos if f.dst == c]
        return srcs[0] if len(srcs) == 1 else None

    def element(self, pkey):
        """T[controller(p)][p] (0 if not controlled)."""
        q = self.controller(pkey)
        return self.table.get((q, pkey), 0) if q is not None else 0


# ---------------------------------------------------------------------------
# Sec. III: rates, port and actor types, eq. (1)
# ---------------------------------------------------------------------------

def check_rates(g: Graph):
    """Every FIFO's two ports have atr equal to fiforate (Sec. III-A); control
    FIFOs have rate 1.  Returns a list of violation strings."""
    errs = []
    for f in g.fifos:
        for pk in (f.src, f.dst):
            p = g.ports[pk]
            if p.kind in (CTRL_IN, CTRL_OUT):
                if f.rate != 1 or p.atr != 1:
                    errs.append(f"{f.name}: control FIFO rate must be 1")
            elif p.atr != f.rate:
                errs.append(f"{f.name}: atr({pk}) = {p.atr} != fiforate = {f.rate}")
    for pk, p in g.ports.items():
        n = len(g.fifos_of(pk))
        if not p.out and n != 1:
            errs.append(f"input port {pk} must have exactly one FIFO (has {n})")
        if p.out and n < 1:
            errs.append(f"output port {pk} is unconnected")
    return errs


def check_actor_types(g: Graph):
    """Port sets allowed per actor type (Sec. III-B)."""
    errs = []
    for a, kind in g.actors.items():
        ps = g.ports_of(a)
        kinds = [p.kind for p in ps]
        if kind == STATIC and any(k != SRP for k in kinds):
            errs.append(f"static actor {a} has a non-SRP port")
        if kind == DYNAMIC:
            if kinds.count(DRP) < 1:
                errs.append(f"dynamic actor {a} has no DRP")
            if kinds.count(CTRL_IN) != 1:
                errs.append(f"dynamic actor {a} must have exactly one control port")
            if CTRL_OUT in kinds:
                errs.append(f"dynamic actor {a} has a control output port")
        if kind == CONFIG:
            if kinds.count(CTRL_OUT) < 1:
                errs.append(f"configuration actor {a} has no control output port")
            if DRP in kinds or CTRL_IN in kinds:
                errs.append(f"configuration actor {a} has a DRP or control input")
            for p in ps:
                if p.kind == CTRL_OUT:
                    for f in g.fifos_of(p.key):
                        if g.ports[f.dst].kind != CTRL_IN:
                            errs.append(f"{p.key} feeds a non-control port")
    return errs


def tokrate(g: Graph, pkey, v):
    """Eq. (1): token rate of port ``pkey`` in a firing that consumed control
    value ``v`` (a sequence of Booleans, element 1 is v[0])."""
    p = g.ports[pkey]
    if p.kind != DRP:
        return p.atr
    e = g.element(pkey)
    if e <= 0:
        raise ValueError(f"DRP {pkey} is not controlled")
    return int(bool(v[e - 1])) * p.atr


# ---------------------------------------------------------------------------
# Sec. IV: chains, linked ports, connecting subchains, rules 1-5
# ---------------------------------------------------------------------------

def _other_ends(g, pkey):
    ends = set()
    for f in g.fifos_of(pkey):
        other = f.dst if f.src == pkey else f.src
        ends.add(other[0])
    return ends


def simple_paths(g: Graph, a, b, avoid):
    """All simple chains from actor a to actor b that avoid ``avoid``."""
    if a in avoid or b in avoid:
        return []
    out = []
    stack = [(a, (a,))]
    while stack:
        node, path = stack.pop()
        if node == b:
            out.append(path)
            continue
        for n in sorted(g.neighbours(node)):
            if n not in path and n not in avoid:
                stack.append((n, path + (n,)))
    return out


def connecting_subchains(g: Graph, px, py):
    """Connecting subchains of ports px, py (Sec. IV): sequences (a1..aN) such
    that (x, a1, ..., aN, y) is a simple chain, px is connected to a port of a1
    and py to a port of aN."""
    x, y = px[0], py[0]
    subs = []
    for a1 in _other_ends(g, px):
        for aN in _other_ends(g, py):
            for path in simple_paths(g, a1, aN, avoid={x, y}):
                subs.append(path)
    return subs


def linked(g: Graph, px, py):
    """Linked ports (Sec. IV): same FIFO, or a connecting subchain exists."""
    if px == py:
        return False
    fx = {f.name for f in g.fifos_of(px)}
    fy = {f.name for f in g.fifos_of(py)}
    return bool(fx & fy) or bool(connecting_subchains(g, px, py))


def linked_drp_pairs(g: Graph):
    drps = [k for k, p in g.ports.items() if p.kind == DRP]
    pairs = []
    for i in range(len(drps)):
        for j in range(i + 1, len(drps)):
            if drps[i][0] != drps[j][0] and linked(g, drps[i], drps[j]):
                pairs.append((drps[i], drps[j]))
    return pairs


def rule1(g: Graph):
    """Linked port control rule: T[pq][px] = T[pq][py] > 0 for linked DRPs."""
    errs = []
    for px, py in linked_drp_pairs(g):
        qx, qy = g.controller(px), g.controller(py)
        ex, ey = g.element(px), g.element(py)
        if qx is None or qx != qy or ex != ey or ex <= 0:
            errs.append(f"rule 1: linked DRPs {px}, {py} controlled by ({qx},{ex}) vs ({qy},{ey})")
    return errs


def rule2(g: Graph):
    """Balanced delay rule: all FIFOs from one control output port to control
    ports carry the same delay."""
    errs = []
    for pk, p in g.ports.items():
        if p.kind != CTRL_OUT:
            continue
        delays = {f.delay for f in g.fifos if f.src == pk and g.ports[f.dst].kind == CTRL_IN}
        if len(delays) > 1:
            errs.append(f"rule 2: control port {pk} reaches control ports with delays {sorted(delays)}")
    return errs


def _pair_subchains(g):
    """(x, y, px, py, subchain) for every linked DRP pair on distinct actors."""
    out = []
    for px, py in linked_drp_pairs(g):
        for s in connecting_subchains(g, px, py):
            out.append((px[0], py[0], px, py, s))
    return out


def rule3(g: Graph):
    """Connecting subchain rule: subchain actors are static and every subchain
    an actor belongs to is associated with the same dynamic pair {x, y}."""
    errs = []
    owner = {}
    for x, y, px, py, s in _pair_subchains(g):
        pair = frozenset((x, y))
        for a in s:
            if g.actors[a] != STATIC:
                errs.append(f"rule 3: subchain actor {a} of {px},{py} is not static")
            owner.setdefault(a, set()).add(pair)
    for a, pairs in owner.items():
        if len(pairs) > 1:
            errs.append(f"rule 3: actor {a} is on subchains of several dynamic pairs {sorted(map(sorted, pairs))}")
    return errs


def rule4(g: Graph):
    """Single-sided dynamism: a dynamic actor has DRP inputs or DRP outputs."""
    errs = []
    for a, kind in g.actors.items():
        if kind != DYNAMIC:
            continue
        dirs = {g.ports[k].out for k in g.drps(a)}
        if len(dirs) > 1:
            errs.append(f"rule 4: dynamic actor {a} has both input and output DRPs")
    return errs


def _connects(g, b, x, y):
    if b in (x, y):
        return True
    for p1 in simple_paths(g, x, b, avoid={y}):
        for p2 in simple_paths(g, b, y, avoid=set(p1[:-1])):
            if not (set(p1) & set(p2[1:])):
                return True
    return False


def rule5(g: Graph):
    """Encapsulation rule: an actor b outside a subchain S that is connected to
    an actor of S through an SRP of b must lie on a (simple) chain connecting
    x and y."""
    errs = []
    for x, y, px, py, s in _pair_subchains(g):
        for a in s:
            for f in g.fifos:
                for mine, other in ((f.src, f.dst), (f.dst, f.src)):
                    if mine[0] != a:
                        continue
                    b = other[0]
                    if b in s or g.ports[other].kind != SRP:
                        continue
                    if not _connects(g, b, x, y):
                        errs.append(f"rule 5: {b} touches subchain actor {a} of ({x},{y}) but does not connect them")
    return sorted(set(errs))


def design_rule_violations(g: Graph):
    return check_rates(g) + check_actor_types(g) + rule1(g) + rule2(g) + rule3(g) + rule4(g) + rule5(g)


# ---------------------------------------------------------------------------
# Sec. V: DPGs, the DC-finding procedure, validity, consistency
# ---------------------------------------------------------------------------

def find_dcs(g: Graph, q, x, y):
    """DC-finding procedure of Sec. V for the DPG (q, x, y).

    Step 1: a linked DRP pair sharing a FIFO gets a dummy actor on that FIFO.
    Step 2: remove q, x, y and their FIFOs; the connected components of the
    remaining DPG actors (those on connecting subchains of x's and y's linked
    DRPs, plus dummies) are the DCs.  Returns a list of frozensets; dummy
    actors are named 'd:<fifo>'.
    """
    members = set()
    edges = set()
    for px in g.drps(x):
        for py in g.drps(y):
            shared = {f.name for f in g.fifos_of(px)} & {f.name for f in g.fifos_of(py)}
            for fname in shared:
                d = f"d:{fname}"
                members.add(d)
            for s in connecting_subchains(g, px, py):
                members.update(s)
    for f in g.fifos:
        a, b = f.src[0], f.dst[0]
        if a in members and b in members and a != b:
            edges.add((a, b))
    adj = {m: set() for m in members}
    for a, b in edges:
        adj[a].add(b)
        adj[b].add(a)
    comps, seen = [], set()
    for m in sorted(members):
        if m in seen:
            continue
        comp, dq = set(), deque([m])
        while dq:
            u = dq.popleft()
            if u in comp:
                continue
            comp.add(u)
            dq.extend(adj[u] - comp)
        seen |= comp
        comps.append(frozenset(comp))
    return comps


def _dc_drps(g, dc, actor):
    """DRPs of ``actor`` connected to the DC (directly or via its dummy)."""
    out = []
    for pk in g.drps(actor):
        for f in g.fifos_of(pk):
            other = f.dst if f.src == pk else f.src
            if other[0] in dc or f"d:{f.name}" in dc:
                out.append(pk)
    return sorted(set(out))


def dpg_validity(g: Graph, q, x, y):
    """Validity of Sec. V: (a) every DC touches a DRP of x and of y; (b) the
    DRPs of one DC share one element of v and the map DC -> element is a
    bijection onto the elements used.  Returns (errors, {dc: element})."""
    errs, elem_of = [], {}
    dcs = find_dcs(g, q, x, y)
    for dc in dcs:
        dx, dy = _dc_drps(g, dc, x), _dc_drps(g, dc, y)
        if not dx or not dy:
            errs.append(f"DC {sorted(dc)} does not touch DRPs of both {x} and {y}")
        elems = {g.element(p) for p in dx + dy}
        if len(elems) != 1 or 0 in elems:
            errs.append(f"DC {sorted(dc)} DRPs use elements {sorted(elems)}")
        else:
            elem_of[dc] = elems.pop()
    if len(set(elem_of.values())) != len(elem_of):
        errs.append("two DCs share one control element (not a bijection)")
    return errs, elem_of


def repetition_vector(actors, fifos, rate_src, rate_dst):
    """Balance equations q(src) * prod = q(dst) * cons over a connected SDF
    graph (Lee and Messerschmitt); returns {actor: int} or None if
    inconsistent."""
    actors = list(actors)
    if not actors:
        return {}
    qv = {actors[0]: Fraction(1)}
    changed = True
    while changed:
        changed = False
        for f in fifos:
            a, b = f.src[0], f.dst[0]
            pa, cb = rate_src(f), rate_dst(f)
            if a in qv and b not in qv:
                qv[b] = qv[a] * pa / cb
                changed = True
            elif b in qv and a not in qv:
                qv[a] = qv[b] * cb / pa
                changed = True
    if len(qv) != len(actors):
        return None
    for f in fifos:
        if qv[f.src[0]] * rate_src(f) != qv[f.dst[0]] * rate_dst(f):
            return None
    import math
    den = 1
    for v in qv.values():
        den = den * v.denominator // math.gcd(den, v.denominator)
    ints = {a: int(v * den) for a, v in qv.items()}
    gg = 0
    for v in ints.values():
        gg = math.gcd(gg, v)
    return {a: v // gg for a, v in ints.items()}


def sdf_pass(actors, fifos, qv):
    """Simulate one period of a consistent SDF graph (a class-S schedule).
    Returns (deadlock_free, {fifo: max tokens during the period})."""
    occ = {f.name: f.delay for f in fifos}
    peak = dict(occ)
    left = dict(qv)
    progress = True
    while progress and any(left.values()):
        progress = False
        for a in actors:
            if left[a] == 0:
                continue
            ins = [f for f in fifos if f.dst[0] == a]
            if all(occ[f.name] >= f.rate for f in ins):
                for f in ins:
                    occ[f.name] -= f.rate
                for f in fifos:
                    if f.src[0] == a:
                        occ[f.name] += f.rate
                        peak[f.name] = max(peak[f.name], occ[f.name])
                left[a] -= 1
                progress = True
    return (not any(left.values())), peak


def dpg_consistency(g: Graph, q, x, y):
    """Theorem of Sec. V: the DPG is consistent iff every DC, as an SDF graph
    with its boundary FIFOs to x and y, is consistent.  Returns
    (consistent, {dc: buffer bound per FIFO}, beta) where beta[f] is the max of
    the per-DC bounds B_k(f)."""
    bounds, beta = {}, {}
    for dc in find_dcs(g, q, x, y):
        real = {a for a in dc if not a.startswith("d:")}
        sub = [f for f in g.fifos
               if (f.src[0] in real or f.dst[0] in real or f"d:{f.name}" in dc)]
        acts = set(real) | {x, y}
        qv = repetition_vector(acts, sub, lambda f: f.rate, lambda f: f.rate)
        if qv is None:
            return False, bounds, beta
        ok, peak = sdf_pass(sorted(acts), sub, qv)
        if not ok:
            return False, bounds, beta
        bounds[dc] = peak
        for fn, v in peak.items():
            beta[fn] = max(beta.get(fn, 0), v)
    return True, bounds, beta


def rate_balance(g: Graph, q, x, y, v):
    """Net token change of every DPG FIFO over one DPG iteration under control
    value v: x, y and q fire once, actors of active DCs fire once, actors of
    inactive DCs not at all; rates by eq. (1).  Returns {fifo: produced -
    consumed} (all zero for a consistent DPG)."""
    errs, elem_of = dpg_validity(g, q, x, y)
    if errs:
        raise ValueError(errs)
    fires = {x: 1, y: 1, q: 1}
    for dc, e in elem_of.items():
        for a in dc:
            if not a.startswith("d:"):
                fires[a] = int(bool(v[e - 1]))
    out = {}
    for f in g.fifos:
        a, b = f.src[0], f.dst[0]
        if a not in fires or b not in fires or g.ports[f.src].kind in (CTRL_OUT,):
            continue
        prod = fires[a] * tokrate(g, f.src, v)
        cons = fires[b] * tokrate(g, f.dst, v)
        out[f.name] = prod - cons
    return out


def fifo_capacity(r, Q, C):
    """Eq. (2) in tokens (token size factored out)."""
    if Q % r != 0:
        return r * C + Q
    return max(r * C, Q)


# ---------------------------------------------------------------------------
# The canonical graph of the hot path and its fixtures
# ---------------------------------------------------------------------------

def canonical_graph(F, swap_sink_elements=None, delay_f4=0, delay_f5=0):
    """SRC -> FIR (self-loop delay f1) -> broadcast {DET, SEL}; DET control ->
    {SEL, SINK}; SEL DRP_b -> HX_b -> SINK DRP_b.  Token unit: one block for
    data FIFOs.  ``swap_sink_elements=(b1, b2)`` breaks rule 1 by exchanging
    the control elements of SINK's DRPs b1 and b2; ``delay_f4``/``delay_f5``
    put initial control tokens on one control FIFO (breaks rule 2 if they
    differ)."""
    g = Graph()
    for a, k in (("SRC", STATIC), ("FIR", STATIC), ("DET", CONFIG), ("SEL", DYNAMIC),
                 ("SINK", DYNAMIC)):
        g.add_actor(a, k)
    g.add_port("SRC", "out", True, SRP, F)
    g.add_port("FIR", "in", False, SRP, F)
    g.add_port("FIR", "hin", False, SRP, 1)
    g.add_port("FIR", "hout", True, SRP, 1)
    g.add_port("FIR", "out", True, SRP, F)
    g.add_port("DET", "in", False, SRP, F)
    g.add_port("DET", "ctl", True, CTRL_OUT, 1)
    g.add_port("SEL", "c", False, CTRL_IN, 1)
    g.add_port("SEL", "in", False, SRP, F)
    g.add_port("SINK", "c", False, CTRL_IN, 1)
    g.connect("f0", ("SRC", "out"), ("FIR", "in"), F)
    g.connect("f1", ("FIR", "hout"), ("FIR", "hin"), 1, delay=1)
    g.connect("f2", ("FIR", "out"), ("DET", "in"), F)
    g.connect("f3", ("FIR", "out"), ("SEL", "in"), F)
    g.connect("f4", ("DET", "ctl"), ("SEL", "c"), 1, delay=delay_f4)
    g.connect("f5", ("DET", "ctl"), ("SINK", "c"), 1, delay=delay_f5)
    for b in range(F):
        hx = f"HX_{b}"
        g.add_actor(hx, STATIC)
        g.add_port("SEL", f"o{b}", True, DRP, 1)
        g.add_port(hx, "in", False, SRP, 1)
        g.add_port(hx, "out", True, SRP, 1)
        g.add_port("SINK", f"i{b}", False, DRP, 1)
        g.connect(f"f6_{b}", ("SEL", f"o{b}"), (hx, "in"), 1)
        g.connect(f"f7_{b}", (hx, "out"), ("SINK", f"i{b}"), 1)
        g.table[(("DET", "ctl"), ("SEL", f"o{b}"))] = b + 1
        g.table[(("DET", "ctl"), ("SINK", f"i{b}"))] = b + 1
    if swap_sink_elements is not None:
        b1, b2 = swap_sink_elements
        k1, k2 = (("DET", "ctl"), ("SINK", f"i{b1}")), (("DET", "ctl"), ("SINK", f"i{b2}"))
        g.table[k1], g.table[k2] = g.table[k2], g.table[k1]
    return g


def dpd_graph(K=10):
    """The Dynamic Predistortion graph of Sec. VII-A2 (figure missing from the
    source; rebuilt from the prose): SRC emits one period of input samples to
    the polynomial actor POLY and one external configuration token to the
    configuration actor CONF; CONF's control value selects which of the K
    branches fire in the period.  POLY (dynamic, output DRPs) feeds branch k
    to FIR_k (static, with a self-loop delay token: the filter's history), and
    the adder ADD (dynamic, input DRPs) sums the branches that fired into SINK.
    Token unit: one period of samples.  The DPG is (CONF, POLY, ADD) with K
    DCs {FIR_k}."""
    g = Graph()
    for a, k in (("SRC", STATIC), ("CONF", CONFIG), ("POLY", DYNAMIC), ("ADD", DYNAMIC), ("SINK", STATIC)):
        g.add_actor(a, k)
    g.add_port("SRC", "x", True, SRP, 1)
    g.add_port("SRC", "cfg", True, SRP, 1)
    g.add_port("CONF", "in", False, SRP, 1)
    g.add_port("CONF", "ctl", True, CTRL_OUT, 1)
    g.add_port("POLY", "c", False, CTRL_IN, 1)
    g.add_port("POLY", "in", False, SRP, 1)
    g.add_port("ADD", "c", False, CTRL_IN, 1)
    g.add_port("ADD", "out", True, SRP, 1)
    g.add_port("SINK", "in", False, SRP, 1)
    g.connect("fx", ("SRC", "x"), ("POLY", "in"), 1)
    g.connect("fcfg", ("SRC", "cfg"), ("CONF", "in"), 1)
    g.connect("fcp", ("CONF", "ctl"), ("POLY", "c"), 1)
    g.connect("fca", ("CONF", "ctl"), ("ADD", "c"), 1)
    g.connect("fy", ("ADD", "out"), ("SINK", "in"), 1)
    for k in range(K):
        fir = f"FIR_{k}"
        g.add_actor(fir, STATIC)
        g.add_port("POLY", f"o{k}", True, DRP, 1)
        g.add_port(fir, "in", False, SRP, 1)
        g.add_port(fir, "hin", False, SRP, 1)
        g.add_port(fir, "hout", True, SRP, 1)
        g.add_port(fir, "out", True, SRP, 1)
        g.add_port("ADD", f"i{k}", False, DRP, 1)
        g.connect(f"fp_{k}", ("POLY", f"o{k}"), (fir, "in"), 1)
        g.connect(f"fh_{k}", (fir, "hout"), (fir, "hin"), 1, delay=1)
        g.connect(f"ff_{k}", (fir, "out"), ("ADD", f"i{k}"), 1)
        g.table[(("CONF", "ctl"), ("POLY", f"o{k}"))] = k + 1
        g.table[(("CONF", "ctl"), ("ADD", f"i{k}"))] = k + 1
    return g


# ---------------------------------------------------------------------------
# Brute-force deadlock / boundedness search (token counts and control values)
# ---------------------------------------------------------------------------

@dataclass
class SearchResult:
    sequences: int = 0
    states: int = 0
    deadlocks: list = field(default_factory=list)     # (sequence, state description)
    unbalanced: list = field(default_factory=list)    # (sequence, final occupancies)


def search(g: Graph, n_frames: int, C: int, source="SRC", config="DET", sink="SINK",
           max_states=2_000_000):
    """For every control sequence (one value v per configuration-actor firing,
    2^(K * n_frames) of them for K control elements) explore every
    interleaving of enabled firings (BFS) under blocking reads/writes with
    eq. (2) capacities.  A reachable state with no enabled actor is final only
    if the source fired n_frames times and the sink n_frames times; any other
    such state is a deadlock.  A final state whose FIFO occupancies differ from
    the initial delays is unbalanced (tokens would accumulate or vanish over
    repeated iterations)."""
    names = [f.name for f in g.fifos]
    fidx = {n: i for i, n in enumerate(names)}
    cap = [fifo_capacity(f.rate, f.delay, C) for f in g.fifos]
    ctrl = [g.ports[f.dst].kind == CTRL_IN for f in g.fifos]
    actors = sorted(g.actors)
    K = max([e for e in g.table.values()] + [0])
    ins = {a: [f for f in g.fifos if f.dst[0] == a] for a in actors}
    outs = {a: [f for f in g.fifos if f.src[0] == a] for a in actors}
    res = SearchResult()

    init_occ = tuple(f.delay for f in g.fifos)
    init_ctl = tuple((tuple([0] * K),) * f.delay if ctrl[i] else () for i, f in enumerate(g.fifos))

    for seq in itertools.product(itertools.product((0, 1), repeat=K), repeat=n_frames):
        res.sequences += 1
        start = (init_occ, init_ctl, tuple(0 for _ in actors))
        seen = {start}
        dq = deque([start])
        while dq:
            occ, ctl, fired = dq.popleft()
            res.states += 1
            if res.states > max_states:
                raise RuntimeError("state budget exceeded")
            any_enabled = False
            for ai, a in enumerate(actors):
                if a == source and fired[ai] >= n_frames:
                    continue
                kind = g.actors[a]
                v = None
                if kind == DYNAMIC:
                    c = fidx[next(f.name for f in ins[a] if g.ports[f.dst].kind == CTRL_IN)]
                    if occ[c] < 1:
                        continue
                    v = ctl[c][0]
                # rates of this firing, eq. (1); a firing consumes, then produces
                cons, prod = {}, {}
                for f in ins[a]:
                    i = fidx[f.name]
                    r = 1 if ctrl[i] else (tokrate(g, f.dst, v) if v is not None else f.rate)
                    cons[i] = cons.get(i, 0) + r
                for f in outs[a]:
                    i = fidx[f.name]
                    r = 1 if ctrl[i] else (tokrate(g, f.src, v) if v is not None else f.rate)
                    prod[i] = prod.get(i, 0) + r
                ok = all(occ[i] >= r for i, r in cons.items())
                ok = ok and all(occ[i] - cons.get(i, 0) + r <= cap[i] for i, r in prod.items())
                if not ok:
                    continue
                any_enabled = True
                nocc = list(occ)
                nctl = list(ctl)
                for i, r in cons.items():
                    nocc[i] -= r
                for i, r in prod.items():
                    nocc[i] += r
                for f in ins[a]:
                    i = fidx[f.name]
                    if ctrl[i]:
                        nctl[i] = nctl[i][1:]
                if a == config:
                    val = seq[fired[ai]] if fired[ai] < n_frames else tuple([0] * K)
                    for f in outs[a]:
                        i = fidx[f.name]
                        if ctrl[i]:
                            nctl[i] = nctl[i] + (val,)
                nf = list(fired)
                nf[ai] += 1
                st = (tuple(nocc), tuple(nctl), tuple(nf))
                if st not in seen:
                    seen.add(st)
                    dq.append(st)
            if not any_enabled:
                si, ki = actors.index(source), actors.index(sink)
                final = fired[si] == n_frames and fired[ki] >= n_frames
                if not final:
                    res.deadlocks.append((seq, dict(zip(names, occ)), dict(zip(actors, fired))))
                elif occ != init_occ:
                    res.unbalanced.append((seq, dict(zip(names, occ))))
    return res
