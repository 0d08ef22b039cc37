// Graph front end (prune_model_*): a PRUNE graph described actor by actor,
// port by port and FIFO by FIFO, checked by the paper's compile-time
// analysis and matched against the forms the runtime fires.  Host code only.
//
//   Sec. III   FIFO rates (atr of both ports = fiforate, control FIFOs rate 1),
//              port sets per actor type, eq. (2) capacities;
//   Sec. IV    linked ports and connecting subchains, design rules 1-5;
//   Sec. V     DPGs (configuration actor q, dynamic actors x and y), the
//              DC-finding procedure, validity (each DC touches DRPs of x and
//              y; DCs and control elements in bijection) and consistency (each
//              DC with its boundary FIFOs is a consistent SDF graph with a
//              deadlock-free period; beta(f) = max of its per-DC peaks).
//
// "Actor v lies on some connecting subchain of x and y" and "v lies on a
// simple chain connecting x and y" are decided with biconnected components:
// a vertex lies on some simple s-t path exactly when it belongs to a block
// on the block-cut-tree path between s and t.  Connecting subchains of the
// DRPs of x and y are the s*-t* paths of the graph without x and y, where
// the virtual s* (t*) is adjacent to the actors at the far ends of x's
// (y's) DRPs.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <map>
#include <set>
#include <string>
#include <vector>

#include "prune.h"

void prune_set_create_error(const std::string &m);  // prune_runtime.cu

namespace {

struct MPort {
  int actor;
  std::string name;
  bool out;
  int kind;
  int64_t atr;
  std::vector<int> fifos;
};
struct MFifo {
  int src, dst;  // ports
  int64_t rate, delay;
};
struct Dpg {
  int q, x, y;
  std::vector<std::vector<int>> dcs;  // actors; a dummy is -(fifo + 1)
  std::vector<int> dc_elem;           // control element of each DC (0 if none)
  bool valid = false, consistent = false;
};

}  // namespace

struct prune_model {
  std::vector<std::string> name;
  std::vector<int> kind;
  std::vector<MPort> ports;
  std::vector<MFifo> fifos;
  std::map<std::pair<int, int>, int> table;  // (control output port, DRP) -> element
  // analysis
  bool done = false;
  prune_model_report rep{};
  std::vector<Dpg> dpgs;
  std::vector<int64_t> beta;
  std::string err = "no error";

  // ---- derived relations ----------------------------------------------
  std::vector<std::set<int>> adjacency(const std::vector<char> &removed) const {
    std::vector<std::set<int>> adj(name.size());
    for (const MFifo &f : fifos) {
      const int a = ports[f.src].actor, b = ports[f.dst].actor;
      if (a == b || removed[a] || removed[b]) continue;
      adj[a].insert(b);
      adj[b].insert(a);
    }
    return adj;
  }
  int ctrl_in(int actor) const {
    int c = -1, n = 0;
    for (size_t p = 0; p < ports.size(); ++p)
      if (ports[p].actor == actor && ports[p].kind == PRUNE_PORT_CTRL_IN) {
        c = static_cast<int>(p);
        ++n;
      }
    return n == 1 ? c : -1;
  }
  int controller(int drp) const {  // control output port feeding the DRP's actor
    const int c = ctrl_in(ports[drp].actor);
    if (c < 0 || ports[c].fifos.size() != 1) return -1;
    return fifos[ports[c].fifos[0]].src;
  }
  int element(int drp) const {
    const int q = controller(drp);
    if (q < 0) return 0;
    auto it = table.find({q, drp});
    return it == table.end() ? 0 : it->second;
  }
  std::vector<int> drps(int actor) const {
    std::vector<int> v;
    for (size_t p = 0; p < ports.size(); ++p)
      if (ports[p].actor == actor && ports[p].kind == PRUNE_PORT_DRP) v.push_back(static_cast<int>(p));
    return v;
  }
  std::vector<int> far_ends(int port) const {  // actors at the other end of the port's FIFOs
    std::vector<int> v;
    for (int fi : ports[port].fifos) {
      const MFifo &f = fifos[fi];
      v.push_back(ports[f.src == port ? f.dst : f.src].actor);
    }
    return v;
  }
};

namespace {

// Vertices on some simple path between s and t in an undirected graph (adj
// over n vertices), by the block-cut tree.  Iterative Tarjan.
std::vector<char> on_simple_paths(const std::vector<std::set<int>> &adj, int s, int t) {
  const int n = static_cast<int>(adj.size());
  std::vector<char> res(n, 0);
  std::vector<int> disc(n, -1), low(n, 0);
  std::vector<std::pair<int, int>> estack;
  std::vector<std::vector<int>> blocks;  // vertex sets
  int timer = 0;
  // DFS from s only: t must be reachable from s
  struct Frame {
    int v, parent;
    std::set<int>::const_iterator it;
  };
  std::vector<Frame> st;
  disc[s] = low[s] = timer++;
  st.push_back({s, -1, adj[s].begin()});
  while (!st.empty()) {
    Frame &fr = st.back();
    if (fr.it != adj[fr.v].end()) {
      const int w = *fr.it++;
      if (w == fr.parent) continue;
      if (disc[w] < 0) {
        estack.push_back({fr.v, w});
        disc[w] = low[w] = timer++;
        st.push_back({w, fr.v, adj[w].begin()});
      } else if (disc[w] < disc[fr.v]) {
        estack.push_back({fr.v, w});
        low[fr.v] = std::min(low[fr.v], disc[w]);
      }
    } else {
      const int v = fr.v, p = fr.parent;
      st.pop_back();
      if (p >= 0) {
        low[p] = std::min(low[p], low[v]);
        if (low[v] >= disc[p]) {  // p separates the block containing edge (p, v)
          std::vector<int> blk;
          while (!estack.empty()) {
            const auto e = estack.back();
            estack.pop_back();
            blk.push_back(e.first);
            blk.push_back(e.second);
            if (e.first == p && e.second == v) break;
          }
          std::sort(blk.begin(), blk.end());
          blk.erase(std::unique(blk.begin(), blk.end()), blk.end());
          blocks.push_back(std::move(blk));
        }
      }
    }
  }
  if (disc[t] < 0 || s == t) return res;
  // block-cut tree: nodes 0..n-1 vertices, n + b blocks; BFS from s to t
  const int nb = static_cast<int>(blocks.size());
  std::vector<std::vector<int>> tree(n + nb);
  for (int b = 0; b < nb; ++b)
    for (int v : blocks[b]) {
      tree[v].push_back(n + b);
      tree[n + b].push_back(v);
    }
  std::vector<int> prev(n + nb, -2);
  std::vector<int> q{s};
  prev[s] = -1;
  for (size_t h = 0; h < q.size(); ++h) {
    const int u = q[h];
    for (int w : tree[u])
      if (prev[w] == -2) {
        prev[w] = u;
        q.push_back(w);
      }
  }
  if (prev[t] == -2) return res;
  for (int u = t; u != -1; u = prev[u])
    if (u >= n)
      for (int v : blocks[u - n]) res[v] = 1;
  return res;
}

// Actors on connecting subchains of DRPs of x and y: simple paths from an
// actor at the far end of one of x's DRPs to one at the far end of one of
// y's DRPs, avoiding x and y.
std::vector<char> subchain_actors(const prune_model &m, int x, int y) {
  const int n = static_cast<int>(m.name.size());
  std::vector<char> removed(n, 0);
  removed[x] = removed[y] = 1;
  std::vector<std::set<int>> adj = m.adjacency(removed);
  adj.resize(n + 2);
  const int s = n, t = n + 1;
  for (int p : m.drps(x))
    for (int a : m.far_ends(p))
      if (a != x && a != y) {
        adj[s].insert(a);
        adj[a].insert(s);
      }
  for (int p : m.drps(y))
    for (int a : m.far_ends(p))
      if (a != x && a != y) {
        adj[t].insert(a);
        adj[a].insert(t);
      }
  std::vector<char> on = on_simple_paths(adj, s, t);
  on.resize(n);
  return on;
}

// Components of the graph without x and y (for linked-port tests).
std::vector<int> components_without(const prune_model &m, int x, int y) {
  const int n = static_cast<int>(m.name.size());
  std::vector<char> removed(n, 0);
  removed[x] = removed[y] = 1;
  const std::vector<std::set<int>> adj = m.adjacency(removed);
  std::vector<int> comp(n, -1);
  int c = 0;
  for (int a = 0; a < n; ++a) {
    if (removed[a] || comp[a] >= 0) continue;
    std::vector<int> q{a};
    comp[a] = c;
    for (size_t h = 0; h < q.size(); ++h)
      for (int w : adj[q[h]])
        if (comp[w] < 0) {
          comp[w] = c;
          q.push_back(w);
        }
    ++c;
  }
  return comp;
}

void note(prune_model *m, const std::string &msg) {
  if (m->rep.first_error[0] == 0) {
    std::strncpy(m->rep.first_error, msg.c_str(), sizeof(m->rep.first_error) - 1);
  }
}

void analyse(prune_model *m) {
  m->rep = prune_model_report{};
  m->dpgs.clear();
  m->beta.assign(m->fifos.size(), 0);
  const int n = static_cast<int>(m->name.size());
  // ---- Sec. III: rates, connections, actor types
  for (size_t fi = 0; fi < m->fifos.size(); ++fi) {
    const MFifo &f = m->fifos[fi];
    for (int pk : {f.src, f.dst}) {
      const MPort &p = m->ports[pk];
      const bool ctl = p.kind == PRUNE_PORT_CTRL_IN || p.kind == PRUNE_PORT_CTRL_OUT;
      if ((ctl && (f.rate != 1 || p.atr != 1)) || (!ctl && p.atr != f.rate)) {
        ++m->rep.rate_errors;
        note(m, "FIFO " + std::to_string(fi) + ": port rate differs from the FIFO rate");
      }
    }
  }
  for (const MPort &p : m->ports) {
    if ((!p.out && p.fifos.size() != 1) || (p.out && p.fifos.empty())) {
      ++m->rep.rate_errors;
      note(m, "port " + m->name[p.actor] + "." + p.name + " is not connected as its direction requires");
    }
  }
  for (int a = 0; a < n; ++a) {
    int ndrp = 0, ncin = 0, ncout = 0, nother = 0;
    for (const MPort &p : m->ports) {
      if (p.actor != a) continue;
      ndrp += p.kind == PRUNE_PORT_DRP;
      ncin += p.kind == PRUNE_PORT_CTRL_IN;
      ncout += p.kind == PRUNE_PORT_CTRL_OUT;
      nother += p.kind != PRUNE_PORT_SRP;
    }
    bool bad = false;
    if (m->kind[a] == PRUNE_ACTOR_STATIC) bad = nother > 0;
    if (m->kind[a] == PRUNE_ACTOR_DYNAMIC) bad = ndrp < 1 || ncin != 1 || ncout > 0;
    if (m->kind[a] == PRUNE_ACTOR_CONFIG) bad = ncout < 1 || ndrp > 0 || ncin > 0;
    if (m->kind[a] == PRUNE_ACTOR_CONFIG)
      for (const MPort &p : m->ports)
        if (p.actor == a && p.kind == PRUNE_PORT_CTRL_OUT)
          for (int fi : p.fifos)
            if (m->ports[m->fifos[fi].dst].kind != PRUNE_PORT_CTRL_IN) bad = true;
    if (bad) {
      ++m->rep.type_errors;
      note(m, "actor " + m->name[a] + " has ports its type does not allow");
    }
  }
  std::vector<int> dyn;
  for (int a = 0; a < n; ++a)
    if (m->kind[a] == PRUNE_ACTOR_DYNAMIC) dyn.push_back(a);
  // ---- rule 1 (linked port control) over every pair of dynamic actors
  for (size_t i = 0; i < dyn.size(); ++i)
    for (size_t j = i + 1; j < dyn.size(); ++j) {
      const int x = dyn[i], y = dyn[j];
      const std::vector<int> comp = components_without(*m, x, y);
      const std::vector<int> dx = m->drps(x), dy = m->drps(y);
      auto ctrl_of = [&](int p) { return std::make_pair(m->controller(p), m->element(p)); };
      auto check = [&](int px, int py) {
        const auto cx = ctrl_of(px), cy = ctrl_of(py);
        if (cx.first < 0 || cx != cy || cx.second <= 0) {
          ++m->rep.rule_errors[0];
          note(m, "rule 1: linked DRPs " + m->name[x] + "." + m->ports[px].name + " and " + m->name[y] + "." +
                      m->ports[py].name + " are not controlled by one control element");
        }
      };
      // far-end components of every DRP, computed once per pair of actors
      auto ends_of = [&](int p) {
        std::vector<int> cs;
        for (int a : m->far_ends(p))
          if (a != x && a != y) cs.push_back(comp[a]);
        return cs;
      };
      std::vector<std::vector<int>> ex, ey;
      for (int px : dx) ex.push_back(ends_of(px));
      for (int py : dy) ey.push_back(ends_of(py));
      for (size_t u = 0; u < dx.size(); ++u)
        for (size_t v = 0; v < dy.size(); ++v) {
          const int px = dx[u], py = dy[v];
          bool linked = false;
          for (int fa : m->ports[px].fifos)
            for (int fb : m->ports[py].fifos) linked |= fa == fb;
          for (int ca : ex[u])
            for (int cb : ey[v]) linked |= ca == cb;
          if (linked) check(px, py);
        }
    }
  // ---- rule 2 (balanced delay)
  for (size_t pk = 0; pk < m->ports.size(); ++pk) {
    if (m->ports[pk].kind != PRUNE_PORT_CTRL_OUT) continue;
    std::set<int64_t> delays;
    for (int fi : m->ports[pk].fifos)
      if (m->ports[m->fifos[fi].dst].kind == PRUNE_PORT_CTRL_IN) delays.insert(m->fifos[fi].delay);
    if (delays.size() > 1) {
      ++m->rep.rule_errors[1];
      note(m, "rule 2: control port " + m->name[m->ports[pk].actor] + "." + m->ports[pk].name +
                  " reaches control ports with different delays");
    }
  }
  // ---- rules 3 and 5 (subchains) per pair of dynamic actors
  std::vector<std::set<std::pair<int, int>>> owner(n);
  for (size_t i = 0; i < dyn.size(); ++i)
    for (size_t j = i + 1; j < dyn.size(); ++j) {
      const int x = dyn[i], y = dyn[j];
      const std::vector<char> on = subchain_actors(*m, x, y);
      bool any = false;
      for (int a = 0; a < n; ++a) any |= on[a] != 0;
      if (!any) continue;
      std::vector<char> chain_xy;  // actors on a simple chain connecting x and y (full graph)
      {
        const std::vector<char> none(n, 0);
        chain_xy = on_simple_paths(m->adjacency(none), x, y);
      }
      for (int a = 0; a < n; ++a) {
        if (!on[a]) continue;
        owner[a].insert({x, y});
        if (m->kind[a] != PRUNE_ACTOR_STATIC) {
          ++m->rep.rule_errors[2];
          note(m, "rule 3: subchain actor " + m->name[a] + " is not static");
        }
        for (const MFifo &f : m->fifos) {
          for (int side = 0; side < 2; ++side) {
            const int mine = side ? f.dst : f.src, other = side ? f.src : f.dst;
            if (m->ports[mine].actor != a) continue;
            const int b = m->ports[other].actor;
            if (b == a || on[b] || m->ports[other].kind != PRUNE_PORT_SRP) continue;
            if (b != x && b != y && !chain_xy[b]) {
              ++m->rep.rule_errors[4];
              note(m, "rule 5: " + m->name[b] + " touches subchain actor " + m->name[a] + " but does not connect " +
                          m->name[x] + " and " + m->name[y]);
            }
          }
        }
      }
    }
  for (int a = 0; a < n; ++a)
    if (owner[a].size() > 1) {
      ++m->rep.rule_errors[2];
      note(m, "rule 3: actor " + m->name[a] + " is on subchains of several dynamic pairs");
    }
  // ---- rule 4 (single-sided dynamism)
  for (int a : dyn) {
    bool in = false, out = false;
    for (int p : m->drps(a)) (m->ports[p].out ? out : in) = true;
    if (in && out) {
      ++m->rep.rule_errors[3];
      note(m, "rule 4: dynamic actor " + m->name[a] + " has input and output DRPs");
    }
  }
  // ---- Sec. V: DPGs = (q, x, y) with x's output DRPs and y's input DRPs
  //      controlled from one control output port of q
  for (size_t pq = 0; pq < m->ports.size(); ++pq) {
    if (m->ports[pq].kind != PRUNE_PORT_CTRL_OUT) continue;
    std::vector<int> xs, ys;
    for (int fi : m->ports[pq].fifos) {
      const int a = m->ports[m->fifos[fi].dst].actor;
      if (m->kind[a] != PRUNE_ACTOR_DYNAMIC) continue;
      bool in = false, out = false;
      for (int p : m->drps(a)) (m->ports[p].out ? out : in) = true;
      if (out && !in) xs.push_back(a);
      if (in && !out) ys.push_back(a);
    }
    for (int x : xs)
      for (int y : ys) {
        Dpg d{m->ports[pq].actor, x, y, {}, {}};
        // members: subchain actors and one dummy per FIFO shared by DRPs of x and y
        const std::vector<char> on = subchain_actors(*m, x, y);
        std::vector<int> dummies;
        for (int px : m->drps(x))
          for (int fa : m->ports[px].fifos)
            for (int py : m->drps(y))
              for (int fb : m->ports[py].fifos)
                if (fa == fb) dummies.push_back(fa);
        std::sort(dummies.begin(), dummies.end());
        dummies.erase(std::unique(dummies.begin(), dummies.end()), dummies.end());
        bool any = !dummies.empty();
        for (int a = 0; a < n; ++a) any |= on[a] != 0;
        if (!any) continue;
        // DCs: components of the members over FIFOs between members
        std::vector<int> comp(n, -1);
        int c = 0;
        const std::vector<char> none(n, 0);
        const std::vector<std::set<int>> adj = m->adjacency(none);
        for (int a = 0; a < n; ++a) {
          if (!on[a] || comp[a] >= 0) continue;
          std::vector<int> q{a};
          comp[a] = c;
          for (size_t h = 0; h < q.size(); ++h)
            for (int w : adj[q[h]])
              if (on[w] && comp[w] < 0) {
                comp[w] = c;
                q.push_back(w);
              }
          d.dcs.push_back(q);
          ++c;
        }
        for (int fi : dummies) d.dcs.push_back({-(fi + 1)});
        // validity: each DC touches a DRP of x and of y; one element per DC; bijection
        d.valid = true;
        std::set<int> used;
        for (const std::vector<int> &dc : d.dcs) {
          std::set<int> elems;
          bool tx = false, ty = false;
          auto touch = [&](int drp, bool isx) {
            (isx ? tx : ty) = true;
            elems.insert(m->element(drp));
          };
          for (int px : m->drps(x))
            for (int fi : m->ports[px].fifos) {
              const int o = m->ports[m->fifos[fi].src == px ? m->fifos[fi].dst : m->fifos[fi].src].actor;
              for (int a : dc)
                if ((a >= 0 && a == o) || (a < 0 && -(a + 1) == fi)) touch(px, true);
            }
          for (int py : m->drps(y))
            for (int fi : m->ports[py].fifos) {
              const int o = m->ports[m->fifos[fi].src == py ? m->fifos[fi].dst : m->fifos[fi].src].actor;
              for (int a : dc)
                if ((a >= 0 && a == o) || (a < 0 && -(a + 1) == fi)) touch(py, false);
            }
          const int e = elems.size() == 1 ? *elems.begin() : 0;
          if (!tx || !ty || e <= 0 || used.count(e)) d.valid = false;
          used.insert(e);
          d.dc_elem.push_back(e);
        }
        // consistency: each DC with x, y and the FIFOs touching it as SDF
        d.consistent = d.valid;
        for (size_t k = 0; k < d.dcs.size() && d.consistent; ++k) {
          const std::vector<int> &dc = d.dcs[k];
          std::set<int> acts{x, y};
          std::vector<int> sub;
          for (int a : dc)
            if (a >= 0) acts.insert(a);
          for (size_t fi = 0; fi < m->fifos.size(); ++fi) {
            const int a = m->ports[m->fifos[fi].src].actor, b = m->ports[m->fifos[fi].dst].actor;
            bool in_dc = false;
            for (int v : dc) in_dc |= (v >= 0 && (v == a || v == b)) || (v < 0 && -(v + 1) == static_cast<int>(fi));
            if (in_dc) sub.push_back(static_cast<int>(fi));
          }
          // balance equations: both ends of a FIFO run at the FIFO's rate
          // (atr = fiforate, Sec. III-A), so a connected DC with x and y has
          // the repetition vector of all ones; it exists iff every actor is
          // reached through the DC's FIFOs
          std::set<int> seen{*acts.begin()};
          bool grown = true;
          while (grown) {
            grown = false;
            for (int fi : sub) {
              const int a = m->ports[m->fifos[fi].src].actor, b = m->ports[m->fifos[fi].dst].actor;
              if (seen.count(a) != seen.count(b)) {
                seen.insert(a);
                seen.insert(b);
                grown = true;
              }
            }
          }
          bool ok = seen.size() == acts.size();
          if (!ok) {
            d.consistent = false;
            break;
          }
          // one period (every actor fires q = 1 times here: equal production
          // and consumption rates per FIFO make the repetition vector all ones),
          // actors in name order, one firing each per round
          std::vector<int> order(acts.begin(), acts.end());
          std::sort(order.begin(), order.end(), [&](int u, int v) { return m->name[u] < m->name[v]; });
          std::map<int, int64_t> occ, peak;
          for (int fi : sub) occ[fi] = peak[fi] = m->fifos[fi].delay;
          std::map<int, int64_t> left;
          for (int a : order) left[a] = 1;
          bool progress = true;
          while (progress) {
            progress = false;
            for (int a : order) {
              if (!left[a]) continue;
              bool ready = true;
              for (int fi : sub)
                if (m->ports[m->fifos[fi].dst].actor == a && occ[fi] < m->fifos[fi].rate) ready = false;
              if (!ready) continue;
              for (int fi : sub)
                if (m->ports[m->fifos[fi].dst].actor == a) occ[fi] -= m->fifos[fi].rate;
              for (int fi : sub)
                if (m->ports[m->fifos[fi].src].actor == a) {
                  occ[fi] += m->fifos[fi].rate;
                  peak[fi] = std::max(peak[fi], occ[fi]);
                }
              left[a] = 0;
              progress = true;
            }
          }
          for (auto &l : left)
            if (l.second) ok = false;
          if (!ok) {
            d.consistent = false;
            break;
          }
          for (auto &pk : peak) m->beta[pk.first] = std::max(m->beta[pk.first], pk.second);
        }
        m->dpgs.push_back(std::move(d));
      }
  }
  m->rep.n_dpgs = static_cast<int32_t>(m->dpgs.size());
  bool cons = true;
  for (const Dpg &d : m->dpgs) cons = cons && d.valid && d.consistent;
  m->rep.consistent = cons ? 1 : 0;
  m->done = true;
}

prune_status mfail(prune_model *m, prune_status s, const std::string &msg) {
  if (m) m->err = msg;
  else prune_set_create_error(msg);
  return s;
}

}  // namespace

extern "C" {

prune_status prune_model_create(prune_model **out) {
  if (!out) return mfail(nullptr, PRUNE_EINVAL, "prune_model_create: NULL out");
  *out = new prune_model();
  return PRUNE_OK;
}

prune_status prune_model_destroy(prune_model *m) {
  delete m;
  return PRUNE_OK;
}

prune_status prune_model_add_actor(prune_model *m, const char *name, int32_t kind, int32_t *actor) {
  if (!m || !name || !actor || kind < PRUNE_ACTOR_STATIC || kind > PRUNE_ACTOR_CONFIG)
    return mfail(m, PRUNE_EINVAL, "prune_model_add_actor: bad arguments");
  for (const std::string &s : m->name)
    if (s == name) return mfail(m, PRUNE_EINVAL, std::string("prune_model_add_actor: duplicate actor ") + name);
  m->name.push_back(name);
  m->kind.push_back(kind);
  m->done = false;
  *actor = static_cast<int32_t>(m->name.size() - 1);
  return PRUNE_OK;
}

prune_status prune_model_add_port(prune_model *m, int32_t actor, const char *name, int32_t is_output, int32_t kind,
                                  int64_t atr, int32_t *port) {
  if (!m || !name || !port || actor < 0 || actor >= static_cast<int32_t>(m->name.size()) ||
      kind < PRUNE_PORT_SRP || kind > PRUNE_PORT_CTRL_OUT || atr < 1 ||
      (kind == PRUNE_PORT_CTRL_IN && is_output) || (kind == PRUNE_PORT_CTRL_OUT && !is_output))
    return mfail(m, PRUNE_EINVAL, "prune_model_add_port: bad arguments");
  m->ports.push_back(MPort{actor, name, is_output != 0, kind, atr, {}});
  m->done = false;
  *port = static_cast<int32_t>(m->ports.size() - 1);
  return PRUNE_OK;
}

prune_status prune_model_connect(prune_model *m, int32_t src, int32_t dst, int64_t rate, int64_t delay,
                                 int32_t *fifo) {
  const int32_t np = m ? static_cast<int32_t>(m->ports.size()) : 0;
  if (!m || !fifo || src < 0 || src >= np || dst < 0 || dst >= np || rate < 1 || delay < 0 || !m->ports[src].out ||
      m->ports[dst].out)
    return mfail(m, PRUNE_EINVAL, "prune_model_connect: bad arguments (output port to input port)");
  m->fifos.push_back(MFifo{src, dst, rate, delay});
  const int fi = static_cast<int>(m->fifos.size() - 1);
  m->ports[src].fifos.push_back(fi);
  m->ports[dst].fifos.push_back(fi);
  m->done = false;
  *fifo = fi;
  return PRUNE_OK;
}

prune_status prune_model_set_control(prune_model *m, int32_t ctrl_out, int32_t drp, int32_t element) {
  const int32_t np = m ? static_cast<int32_t>(m->ports.size()) : 0;
  if (!m || ctrl_out < 0 || ctrl_out >= np || drp < 0 || drp >= np || m->ports[ctrl_out].kind != PRUNE_PORT_CTRL_OUT ||
      m->ports[drp].kind != PRUNE_PORT_DRP || element < 0)
    return mfail(m, PRUNE_EINVAL, "prune_model_set_control: bad arguments");
  m->table[{ctrl_out, drp}] = element;
  m->done = false;
  return PRUNE_OK;
}

prune_status prune_model_check(prune_model *m, prune_model_report *rep) {
  if (!m || !rep) return mfail(m, PRUNE_EINVAL, "prune_model_check: NULL argument");
  if (!m->done) analyse(m);
  *rep = m->rep;
  return PRUNE_OK;
}

prune_status prune_model_dpg(prune_model *m, int32_t i, int32_t *q, int32_t *x, int32_t *y, int32_t *n_dcs,
                             int32_t *valid, int32_t *consistent) {
  if (!m) return mfail(m, PRUNE_EINVAL, "prune_model_dpg: NULL model");
  if (!m->done) analyse(m);
  if (i < 0 || i >= static_cast<int32_t>(m->dpgs.size())) return mfail(m, PRUNE_EINVAL, "prune_model_dpg: no such DPG");
  const Dpg &d = m->dpgs[i];
  if (q) *q = d.q;
  if (x) *x = d.x;
  if (y) *y = d.y;
  if (n_dcs) *n_dcs = static_cast<int32_t>(d.dcs.size());
  if (valid) *valid = d.valid;
  if (consistent) *consistent = d.consistent;
  return PRUNE_OK;
}

prune_status prune_model_dc(prune_model *m, int32_t i, int32_t k, int32_t *members, int32_t max, int32_t *n,
                            int32_t *element) {
  if (!m || !n) return mfail(m, PRUNE_EINVAL, "prune_model_dc: NULL argument");
  if (!m->done) analyse(m);
  if (i < 0 || i >= static_cast<int32_t>(m->dpgs.size()) || k < 0 ||
      k >= static_cast<int32_t>(m->dpgs[i].dcs.size()) || max < 0 || (max > 0 && !members))
    return mfail(m, PRUNE_EINVAL, "prune_model_dc: no such DC");
  const std::vector<int> &dc = m->dpgs[i].dcs[k];
  *n = static_cast<int32_t>(dc.size());
  for (int32_t j = 0; j < std::min<int32_t>(max, *n); ++j) members[j] = dc[j];
  if (element) *element = m->dpgs[i].dc_elem[k];
  return PRUNE_OK;
}

prune_status prune_model_buffer_bound(prune_model *m, int32_t fifo, int64_t *beta) {
  if (!m || !beta || fifo < 0 || fifo >= static_cast<int32_t>(m->fifos.size()))
    return mfail(m, PRUNE_EINVAL, "prune_model_buffer_bound: bad arguments");
  if (!m->done) analyse(m);
  *beta = m->beta[fifo];
  return PRUNE_OK;
}

prune_status prune_model_classify(prune_model *m, int32_t *form, int32_t *units) {
  if (!m || !form || !units) return mfail(m, PRUNE_EINVAL, "prune_model_classify: NULL argument");
  if (!m->done) analyse(m);
  *form = PRUNE_FORM_NONE;
  *units = 0;
  const prune_model_report &r = m->rep;
  int rules = r.rate_errors + r.type_errors;
  for (int e : r.rule_errors) rules += e;
  if (rules || !r.consistent || m->dpgs.size() != 1) return PRUNE_OK;
  const Dpg &d = m->dpgs[0];
  // every DC a single static actor with one input from x and one output to
  // y; with a self-loop delay FIFO on every DC actor it is the DPD form,
  // without any it is the canonical form
  int with_loop = 0;
  for (const std::vector<int> &dc : d.dcs) {
    if (dc.size() != 1 || dc[0] < 0) return PRUNE_OK;
    const int a = dc[0];
    int from_x = 0, to_y = 0, loops = 0, other = 0;
    for (const MFifo &f : m->fifos) {
      const int sa = m->ports[f.src].actor, da = m->ports[f.dst].actor;
      if (sa == a && da == a) loops += f.delay >= 1;
      else if (da == a) (sa == d.x ? from_x : other)++;
      else if (sa == a) (da == d.y ? to_y : other)++;
    }
    if (from_x != 1 || to_y != 1 || other || loops > 1) return PRUNE_OK;
    with_loop += loops;
  }
  if (with_loop == 0) *form = PRUNE_FORM_CANONICAL;
  else if (with_loop == static_cast<int>(d.dcs.size())) *form = PRUNE_FORM_DPD;
  else return PRUNE_OK;
  *units = static_cast<int32_t>(d.dcs.size());
  return PRUNE_OK;
}

namespace {

// FIFOs with an input (dst) port, or an output (src) port, on the actor.
std::vector<int> fifos_in(const prune_model *m, int a) {
  std::vector<int> v;
  for (size_t i = 0; i < m->fifos.size(); ++i)
    if (m->ports[m->fifos[i].dst].actor == a) v.push_back(static_cast<int>(i));
  return v;
}
std::vector<int> fifos_out(const prune_model *m, int a) {
  std::vector<int> v;
  for (size_t i = 0; i < m->fifos.size(); ++i)
    if (m->ports[m->fifos[i].src].actor == a) v.push_back(static_cast<int>(i));
  return v;
}
int src_actor(const prune_model *m, int f) { return m->ports[m->fifos[f].src].actor; }
int dst_actor(const prune_model *m, int f) { return m->ports[m->fifos[f].dst].actor; }
bool is_self_loop(const prune_model *m, int f) { return src_actor(m, f) == dst_actor(m, f); }
std::string fname(const prune_model *m, int f) {
  return "FIFO " + std::to_string(f) + " (" + m->name[src_actor(m, f)] + " -> " + m->name[dst_actor(m, f)] + ")";
}

// A model FIFO's role in the runtime form and whether its rate and delay are
// the ones the runtime implements.  Sets m->err and returns false otherwise.
bool need(prune_model *m, int f, int64_t rate, int64_t delay, int role, std::vector<int> &roles,
          const char *what) {
  const MFifo &x = m->fifos[f];
  if (x.rate != rate || x.delay != delay) {
    m->err = "prune_model_compile: " + fname(m, f) + " (" + what + ") has rate " + std::to_string(x.rate) +
             " and delay " + std::to_string(x.delay) + "; the runtime form needs rate " + std::to_string(rate) +
             " and delay " + std::to_string(delay);
    return false;
  }
  roles[f] = role;
  return true;
}

bool fail_form(prune_model *m, const std::string &msg) {
  m->err = "prune_model_compile: " + msg;
  return false;
}

// The canonical form: SRC -f0-> FIR (self-loop f1) -f2-> q, -f3-> x;
// q -f4-> x, -f5-> y (control); x -f6_b-> HX_b -f7_b-> y, F DCs with the
// control elements 1..F.  Token unit: one block.
bool compile_canonical(prune_model *m, const Dpg &d, int32_t T, std::vector<int> &roles) {
  const int64_t F = static_cast<int64_t>(d.dcs.size());
  // x and q: their one SRP input each comes from the same static actor (FIR),
  // F blocks per firing
  int fir = -1;
  for (int a : {d.x, d.q}) {
    int n = 0;
    for (int f : fifos_in(m, a)) {
      if (m->ports[m->fifos[f].dst].kind == PRUNE_PORT_CTRL_IN) continue;
      ++n;
      const int s = src_actor(m, f);
      if (fir < 0) fir = s;
      if (s != fir || m->kind[s] != PRUNE_ACTOR_STATIC)
        return fail_form(m, "the data inputs of " + m->name[d.q] + " and " + m->name[d.x] +
                                " must both come from one static actor (FIR)");
      if (!need(m, f, F, 0, a == d.q ? 2 : 3, roles, "FIR output")) return false;
    }
    if (n != 1) return fail_form(m, m->name[a] + " must have exactly one data input (from FIR)");
  }
  // control FIFOs: one to x, one to y, rate 1, no initial tokens
  for (int f : fifos_out(m, d.q)) {
    const int a = dst_actor(m, f);
    if (a != d.x && a != d.y) return fail_form(m, m->name[d.q] + " may only feed the control ports of x and y");
    if (!need(m, f, 1, 0, a == d.x ? 4 : 5, roles, "control")) return false;
  }
  // FIR: input f0 from a static source, the self-loop f1 (T > 1), outputs
  // only to q and x
  int src = -1, loops = 0;
  for (int f : fifos_in(m, fir)) {
    if (is_self_loop(m, f)) {
      ++loops;
      if (!need(m, f, 1, 1, 1, roles, "FIR delay line")) return false;
      continue;
    }
    if (src >= 0) return fail_form(m, m->name[fir] + " must have one data input (from the source)");
    src = src_actor(m, f);
    if (!need(m, f, F, 0, 0, roles, "source")) return false;
  }
  if (src < 0 || m->kind[src] != PRUNE_ACTOR_STATIC || !fifos_in(m, src).empty())
    return fail_form(m, "FIR's input must come from a static source actor without inputs");
  if (loops > 1) return fail_form(m, m->name[fir] + " has more than one self-loop");
  if (loops == 0 && T > 1)
    return fail_form(m, m->name[fir] + " has no self-loop delay FIFO, so it carries no delay token; only T = 1 fits");
  for (int f : fifos_out(m, fir))
    if (!is_self_loop(m, f) && dst_actor(m, f) != d.q && dst_actor(m, f) != d.x)
      return fail_form(m, m->name[fir] + " may only feed q, x and its own delay line");
  for (int f : fifos_out(m, src))
    if (dst_actor(m, f) != fir) return fail_form(m, "the source may only feed FIR");
  if (!fifos_out(m, d.y).empty())
    return fail_form(m, m->name[d.y] + " (SINK) must not feed other actors: its records go to the host");
  // the DCs: one block in from x, one block out to y; elements 1..F
  std::vector<char> seen(static_cast<size_t>(F) + 1, 0);
  for (size_t k = 0; k < d.dcs.size(); ++k) {
    const int a = d.dcs[k][0], e = d.dc_elem[k];
    if (e < 1 || e > F || seen[e]) return fail_form(m, "DC " + m->name[a] + " has no unique control element in 1..F");
    seen[e] = 1;
    for (int f : fifos_in(m, a))
      if (!need(m, f, 1, 0, 6, roles, "SEL -> HX_b")) return false;
    for (int f : fifos_out(m, a))
      if (!need(m, f, 1, 0, 7, roles, "HX_b -> SINK")) return false;
  }
  for (size_t f = 0; f < roles.size(); ++f)
    if (roles[f] < 0) return fail_form(m, fname(m, static_cast<int>(f)) + " has no place in the canonical form");
  return true;
}

// The DPD form: a static source feeds x (POLY) one period and q (CONF) one
// configuration token; q's control goes to x and y (ADD); x -> FIR_k (self
// loop) -> y for the K DCs with elements 1..K; y feeds at most one static
// sink.  Token unit: one period.
bool compile_dpd(prune_model *m, const Dpg &d, std::vector<int> &roles) {
  const int64_t K = static_cast<int64_t>(d.dcs.size());
  for (int a : {d.x, d.q}) {
    int n = 0;
    for (int f : fifos_in(m, a)) {
      if (m->ports[m->fifos[f].dst].kind == PRUNE_PORT_CTRL_IN) continue;
      ++n;
      const int s = src_actor(m, f);
      if (m->kind[s] != PRUNE_ACTOR_STATIC || !fifos_in(m, s).empty())
        return fail_form(m, m->name[a] + "'s input must come from a static source actor without inputs");
      if (!need(m, f, 1, 0, a == d.x ? 0 : 1, roles, a == d.x ? "input" : "configuration input")) return false;
    }
    if (n != 1) return fail_form(m, m->name[a] + " must have exactly one data input");
  }
  for (int f : fifos_out(m, d.q)) {
    const int a = dst_actor(m, f);
    if (a != d.x && a != d.y) return fail_form(m, m->name[d.q] + " may only feed the control ports of x and y");
    if (!need(m, f, 1, 0, 5, roles, "control")) return false;
  }
  std::vector<char> seen(static_cast<size_t>(K) + 1, 0);
  for (size_t k = 0; k < d.dcs.size(); ++k) {
    const int a = d.dcs[k][0], e = d.dc_elem[k];
    if (e < 1 || e > K || seen[e]) return fail_form(m, "DC " + m->name[a] + " has no unique control element in 1..K");
    seen[e] = 1;
    for (int f : fifos_in(m, a))
      if (!need(m, f, 1, is_self_loop(m, f) ? 1 : 0, is_self_loop(m, f) ? 3 : 2, roles,
                is_self_loop(m, f) ? "FIR_k delay line" : "POLY -> FIR_k"))
        return false;
    for (int f : fifos_out(m, a))
      if (!is_self_loop(m, f) && !need(m, f, 1, 0, 4, roles, "FIR_k -> ADD")) return false;
  }
  for (int f : fifos_out(m, d.y)) {
    const int s = dst_actor(m, f);
    if (m->kind[s] != PRUNE_ACTOR_STATIC || !fifos_out(m, s).empty())
      return fail_form(m, m->name[d.y] + " may only feed one static sink without outputs");
    if (!need(m, f, 1, 0, 6, roles, "adder output")) return false;
  }
  for (size_t f = 0; f < roles.size(); ++f)
    if (roles[f] < 0) return fail_form(m, fname(m, static_cast<int>(f)) + " has no place in the DPD form");
  return true;
}

}  // namespace

prune_status prune_model_compile(prune_model *m, const prune_compile_params *p, prune_compiled *out,
                                 int32_t *fifo_role, int64_t *fifo_capacity, int32_t n_fifos) {
  if (!m || !p || !out) return mfail(m, PRUNE_EINVAL, "prune_model_compile: NULL argument");
  if (n_fifos < 0 || (n_fifos > 0 && (!fifo_role || !fifo_capacity)))
    return mfail(m, PRUNE_EINVAL, "prune_model_compile: bad fifo_role / fifo_capacity arrays");
  if (!m->done) analyse(m);
  std::memset(out, 0, sizeof *out);
  const prune_model_report &r = m->rep;
  const std::string why = r.first_error[0] ? std::string(": ") + r.first_error : std::string();
  if (r.rate_errors) return mfail(m, PRUNE_EINVAL, "prune_model_compile: FIFO rates do not match their ports (Sec. III-A)" + why);
  if (r.type_errors) return mfail(m, PRUNE_EINVAL, "prune_model_compile: ports an actor type does not allow (Sec. III-B)" + why);
  for (int i = 0; i < 5; ++i)
    if (r.rule_errors[i])
      return mfail(m, PRUNE_EINVAL, "prune_model_compile: design rule " + std::to_string(i + 1) + " is violated (Sec. IV)" + why);
  if (m->dpgs.size() != 1)
    return mfail(m, PRUNE_EINVAL, "prune_model_compile: the runtime forms have exactly one DPG; the model has " +
                                      std::to_string(m->dpgs.size()));
  if (!r.consistent) return mfail(m, PRUNE_EINVAL, "prune_model_compile: the DPG is not valid and consistent (Sec. V)" + why);
  int32_t form = 0, units = 0;
  prune_model_classify(m, &form, &units);
  if (form == PRUNE_FORM_NONE)
    return mfail(m, PRUNE_EINVAL,
                 "prune_model_compile: not a runtime form: every DC must be one static actor fed by x and feeding y, "
                 "all with a self-loop delay (DPD) or all without (canonical)");
  if (p->C < 1) return mfail(m, PRUNE_EINVAL, "prune_model_compile: C must be >= 1 (eq. (2))");
  std::vector<int> roles(m->fifos.size(), -1);
  const Dpg &d = m->dpgs[0];
  if (form == PRUNE_FORM_CANONICAL) {
    if (!compile_canonical(m, d, p->T, roles)) return PRUNE_EINVAL;
    prune_graph_desc &g = out->graph;
    g.F = units;
    g.B = p->B;
    g.T = p->T;
    g.N = p->N;
    g.C = p->C;
    g.out_frames = p->out_frames;
    g.tau = p->tau;
    g.taps = p->taps;
    g.H = p->H;
    g.stream = p->stream;
    g.device = p->device;
    g.hbm_budget = p->hbm_budget;
  } else {
    if (!compile_dpd(m, d, roles)) return PRUNE_EINVAL;
    if (units > 16 || p->T < 1 || p->T > 16 || p->B < 8 || p->B % 8 != 0 || p->B < p->T - 1)
      return mfail(m, PRUNE_EINVAL, "prune_model_compile: the DPD kernel takes K <= 16 branches of 1..16 taps and "
                                    "periods that are multiples of 8 samples, at least T-1");
    out->dpd_K = units;
    out->dpd_T = p->T;
    out->dpd_period = p->B;
  }
  out->form = form;
  out->units = units;
  for (int32_t f = 0; f < n_fifos; ++f) {
    if (f >= static_cast<int32_t>(m->fifos.size())) {
      fifo_role[f] = -1;
      fifo_capacity[f] = 0;
      continue;
    }
    const MFifo &x = m->fifos[f];
    fifo_role[f] = roles[f];
    prune_fifo_capacity(x.rate, x.delay, p->C, &fifo_capacity[f]);
  }
  return PRUNE_OK;
}

const char *prune_model_last_error(const prune_model *m) { return m ? m->err.c_str() : "NULL model"; }

}  // extern "C"
