// CPU checks of the request loop's host logic (arena, stream layout, step
// planner).  Prints one line per check, "ok <name>" or "FAIL <name>: why",
// and exits non-zero on the first failure.
#include <cstdio>
#include <cstdlib>
#include <map>
#include <random>
#include <string>
#include <vector>

#include "serve_host.hpp"

using namespace prune;

static int fails = 0;
#define CHECK(cond, name, ...)                         \
  do {                                                 \
    if (!(cond)) {                                     \
      std::printf("FAIL %s: ", name);                  \
      std::printf(__VA_ARGS__);                        \
      std::printf("\n");                               \
      std::exit(1);                                    \
    }                                                  \
  } while (0)

static void arena_random() {
  std::mt19937_64 rng(7);
  const uint64_t size = 1 << 24;
  Arena a(size, 256);
  std::map<uint64_t, uint64_t> live;  // off -> requested bytes
  for (int it = 0; it < 20000; ++it) {
    const bool do_alloc = live.empty() || (rng() % 100) < 55;
    if (do_alloc) {
      const uint64_t bytes = 1 + rng() % (size / 16);
      const uint64_t need = (bytes + 255) / 256 * 256;
      const uint64_t largest = a.largest_free();
      uint64_t off = 0;
      const bool ok = a.alloc(bytes, &off);
      CHECK(ok == (largest >= need), "arena_alloc_iff_hole", "it %d bytes %llu largest %llu ok %d", it,
            (unsigned long long)bytes, (unsigned long long)largest, ok);
      if (ok) {
        CHECK(off % 256 == 0 && off + need <= size, "arena_bounds", "off %llu", (unsigned long long)off);
        auto nx = live.lower_bound(off);
        if (nx != live.end()) CHECK(off + need <= nx->first, "arena_no_overlap_next", "it %d", it);
        if (nx != live.begin()) {
          auto pv = std::prev(nx);
          CHECK(pv->first + (pv->second + 255) / 256 * 256 <= off, "arena_no_overlap_prev", "it %d", it);
        }
        live[off] = bytes;
      }
    } else {
      auto it2 = live.begin();
      std::advance(it2, rng() % live.size());
      CHECK(a.release(it2->first), "arena_release", "off %llu", (unsigned long long)it2->first);
      live.erase(it2);
    }
    uint64_t used = 0;
    for (auto &l : live) used += (l.second + 255) / 256 * 256;
    CHECK(a.used() == used, "arena_used", "%llu vs %llu", (unsigned long long)a.used(), (unsigned long long)used);
    CHECK(a.blocks() == live.size(), "arena_blocks", "it %d", it);
  }
  CHECK(!a.release(12345), "arena_release_unknown", "accepted a bad offset");
  for (auto &l : live) a.release(l.first);
  CHECK(a.used() == 0 && a.holes() == 1 && a.largest_free() == size, "arena_coalesce", "holes %zu", a.holes());
  std::printf("ok arena_random\n");
}

static void layout() {
  for (int F : {1, 64, 2048})
    for (int T : {1, 32, 129})
      for (int N : {16, 64})
        for (int fps : {1, 4})
          for (int ring : {fps, 2 * fps + 1}) {
            const uint64_t bops = N == 64 ? 65536 : 0;
            const uint64_t fops = T <= 129 ? 16384ull * (1 + (T - 1 + 31) / 32) : 0;
            StreamLayout l = stream_layout(F, 512, T, N, fps, ring, bops, fops);
            const uint64_t L = uint64_t(F) * 512;
            const std::vector<std::pair<uint64_t, uint64_t>> parts = {
                {l.taps, 8ull * T}, {l.H, 8ull * N * N}, {l.bops, bops}, {l.fops, fops}, {l.hist, 16ull * (T > 1 ? T - 1 : 1)},
                {l.y, 8 * L * fps}, {l.energy, 4ull * F * fps}, {l.c, 4ull * ring}, {l.idx, 4ull * F * ring},
                {l.out, 8 * L * ring}};
            for (size_t i = 0; i < parts.size(); ++i) {
              CHECK(parts[i].first % 256 == 0, "layout_align", "part %zu", i);
              const uint64_t end = parts[i].first + parts[i].second;
              const uint64_t next = i + 1 < parts.size() ? parts[i + 1].first : l.total;
              CHECK(end <= next, "layout_no_overlap", "part %zu F %d T %d", i, F, T);
            }
          }
  std::printf("ok layout\n");
}

static StreamState mk(int F) {
  StreamState s;
  s.F = F;
  return s;
}

static void planner() {
  const int B = 512;
  // three streams: s0 F=4 with 5 frames in one segment of period 2, s1 F=8
  // with 3 frames, s2 nothing queued; fps 2, ring 3
  std::vector<StreamState> st = {mk(4), mk(8), mk(16)};
  alignas(16) static char buf0[4 * 512 * 8 * 2], buf1[8 * 512 * 8 * 3];
  st[0].queue.push_back(Segment{buf0, 5, 2, 0});
  st[0].queued = 5;
  st[1].queue.push_back(Segment{buf1, 3, 3, 0});
  st[1].queued = 3;
  std::vector<int32_t> order = {1, 0, 2};
  auto p = plan_step(st, order, B, 2, 3, 100);
  CHECK(p.size() == 4, "plan_size", "%zu", p.size());
  CHECK(p[0].stream == 1 && p[1].stream == 1 && p[2].stream == 0 && p[3].stream == 0, "plan_order", "");
  CHECK(p[0].x == buf1 && p[1].x == buf1 + 8 * 512 * 8 && p[0].prev == nullptr && p[1].prev == p[0].x,
        "plan_chain", "");
  CHECK(!p[0].last && p[1].last && !p[2].last && p[3].last, "plan_last", "");
  CHECK(p[2].frame == 0 && p[3].frame == 1 && st[0].fired == 2 && st[0].queued == 3, "plan_counts", "");
  // step 2: s1 has 1 left; s0 ring 3 with 2 fired and 0 pulled -> 1 more only
  p = plan_step(st, order, B, 2, 3, 100);
  CHECK(p.size() == 2 && p[0].stream == 1 && p[0].frame == 2 && p[1].stream == 0 && p[1].frame == 2,
        "plan_backpressure", "size %zu", p.size());
  CHECK(p[1].x == buf0 && p[1].prev == nullptr, "plan_period_wrap", "");  // frame 2 of period 2 -> slot 0
  CHECK(st[1].queue.empty() && st[1].queued == 0, "plan_queue_drained", "");
  // ring full for s0: nothing fires until pulls free slots
  p = plan_step(st, order, B, 2, 3, 100);
  CHECK(p.empty(), "plan_ring_full", "%zu", p.size());
  st[0].pulled = 2;
  p = plan_step(st, order, B, 2, 3, 100);
  CHECK(p.size() == 2 && p[0].frame == 3 && p[1].frame == 4 && p[0].x == buf0 + 4 * 512 * 8 && p[1].x == buf0 &&
            p[1].prev == p[0].x,
        "plan_resume", "");
  // max_entries cap, closing streams skipped
  std::vector<StreamState> st2 = {mk(4), mk(4), mk(4)};
  for (auto &s : st2) {
    s.queue.push_back(Segment{buf0, 4, 1, 0});
    s.queued = 4;
  }
  st2[1].closing = true;
  p = plan_step(st2, {0, 1, 2}, B, 4, 4, 5);
  CHECK(p.size() == 5 && p[3].stream == 0 && p[4].stream == 2 && p[4].last && st2[2].fired == 1, "plan_cap",
        "size %zu", p.size());
  CHECK(st2[1].fired == 0, "plan_closing", "");
  std::printf("ok planner\n");
}

int main() {
  arena_random();
  layout();
  planner();
  return fails;
}
