"""Python view of the graph front end (prune_model_*): describe a PRUNE
graph, run the compile-time analysis (rates, actor types, design rules 1-5,
DPGs, DCs, validity, consistency, buffer bounds) and classify it against the
forms the runtime fires.  Argument marshalling only; host code, no device."""
from __future__ import annotations

import ctypes

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
