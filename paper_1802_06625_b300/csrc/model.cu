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

const char *prune_model_last_error(const prune_model *m) { return m ? m->err.c_str() : "NULL model"; }

}  // extern "C"
