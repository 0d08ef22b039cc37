"""Python view of the graph front end (prune_model_*): describe a PRUNE
graph, run the compile-time analysis (rates, actor types, design rules 1-5,
DPGs, DCs, validity, consistency, buffer bounds), classify it against the
forms the runtime fires and compile it into one of them.  Argument
marshalling only; host code, no device."""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import check

STATIC, DYNAMIC, CONFIG = 0, 1, 2
SRP, DRP, CTRL_IN, CTRL_OUT = 0, 1, 2, 3
FORMS = {0: None, 1: "canonical", 2: "dpd"}


class Model:
    def __init__(self):
        h = ctypes.c_void_p()
        check(_lib.lib().prune_model_create(ctypes.byref(h)))
        self.h = h
        self.actors, self.ports, self.fifos = [], [], []
        self._actor = {}
        self._port = {}

    def close(self):
        if getattr(self, "h", None):
            _lib.lib().prune_model_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _c(self, st):
        return check(st, model=self.h)

    def add_actor(self, name, kind):
        i = ctypes.c_int32()
        self._c(_lib.lib().prune_model_add_actor(self.h, name.encode(), kind, ctypes.byref(i)))
        self.actors.append(name)
        self._actor[name] = i.value
        return i.value

    def add_port(self, actor, name, out, kind, atr=1):
        i = ctypes.c_int32()
        self._c(_lib.lib().prune_model_add_port(self.h, self._actor[actor], name.encode(), int(bool(out)), kind, atr,
                                                ctypes.byref(i)))
        self.ports.append((actor, name))
        self._port[(actor, name)] = i.value
        return i.value

    def connect(self, src, dst, rate, delay=0, name=None):
        i = ctypes.c_int32()
        self._c(_lib.lib().prune_model_connect(self.h, self._port[src], self._port[dst], rate, delay, ctypes.byref(i)))
        self.fifos.append(name or f"f{i.value}")
        return i.value

    def set_control(self, ctrl_out, drp, element):
        self._c(_lib.lib().prune_model_set_control(self.h, self._port[ctrl_out], self._port[drp], element))

    def check(self):
        r = _lib.prune_model_report()
        self._c(_lib.lib().prune_model_check(self.h, ctypes.byref(r)))
        return {"rate_errors": r.rate_errors, "type_errors": r.type_errors, "rule_errors": list(r.rule_errors),
                "n_dpgs": r.n_dpgs, "consistent": bool(r.consistent),
                "first_error": r.first_error.decode(errors="replace")}

    def dpgs(self):
        out = []
        for i in range(self.check()["n_dpgs"]):
            v = [ctypes.c_int32() for _ in range(6)]
            self._c(_lib.lib().prune_model_dpg(self.h, i, *[ctypes.byref(a) for a in v]))
            q, x, y, ndc, valid, cons = (a.value for a in v)
            dcs = []
            for k in range(ndc):
                mem = (ctypes.c_int32 * 4096)()
                n, e = ctypes.c_int32(), ctypes.c_int32()
                self._c(_lib.lib().prune_model_dc(self.h, i, k, mem, 4096, ctypes.byref(n), ctypes.byref(e)))
                names = frozenset(self.actors[a] if a >= 0 else f"d:{self.fifos[-a - 1]}" for a in mem[:n.value])
                dcs.append((names, e.value))
            out.append({"q": self.actors[q], "x": self.actors[x], "y": self.actors[y], "dcs": dcs,
                        "valid": bool(valid), "consistent": bool(cons)})
        return out

    def buffer_bound(self, fifo):
        b = ctypes.c_int64()
        self._c(_lib.lib().prune_model_buffer_bound(self.h, fifo, ctypes.byref(b)))
        return b.value

    def classify(self):
        f, u = ctypes.c_int32(), ctypes.c_int32()
        self._c(_lib.lib().prune_model_classify(self.h, ctypes.byref(f), ctypes.byref(u)))
        return FORMS[f.value], u.value

    def compile(self, B, T, N=1, C=3, tau=0.0, taps=None, H=None, out_frames=0, device=-1, hbm_budget=0):
        """prune_model_compile: the runtime form of the checked model.
        Returns a dict: form ("canonical" or "dpd"), units, roles (runtime
        FIFO of every model FIFO), capacities (eq. (2) tokens) and, for the
        canonical form, desc (the prune_graph_desc, whose host arrays it
        keeps alive) or, for DPD, K, T and period.  Raises PruneError with
        the reason for any other model."""
        p = _lib.prune_compile_params(B=B, T=T, N=N, C=C, tau=float(tau), out_frames=out_frames, device=device,
                                      hbm_budget=hbm_budget)
        keep = []
        if taps is not None:
            t = np.ascontiguousarray(np.asarray(taps, np.complex64)).view(np.float32).reshape(-1)
            keep.append(t)
            p.taps = t.ctypes.data
        if H is not None:
            h = np.ascontiguousarray(np.asarray(H, np.complex64)).view(np.float32).reshape(-1)
            keep.append(h)
            p.H = h.ctypes.data
        out = _lib.prune_compiled()
        n = len(self.fifos)
        roles = (ctypes.c_int32 * max(n, 1))()
        caps = (ctypes.c_int64 * max(n, 1))()
        self._c(_lib.lib().prune_model_compile(self.h, ctypes.byref(p), ctypes.byref(out), roles, caps, n))
        r = {"form": FORMS[out.form], "units": out.units, "roles": list(roles[:n]), "capacities": list(caps[:n])}
        if out.form == 1:
            r["desc"] = out.graph
            r["_keep"] = keep
        else:
            r.update(K=out.dpd_K, T=out.dpd_T, period=out.dpd_period)
        return r
