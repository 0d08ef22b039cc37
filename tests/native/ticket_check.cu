// Host check of tc_ticket_tile (the fused loops' ticket -> (frame, tile)
// mapping, frames taken W at a time round-robin): every ticket lands in
// range, tickets 0 .. frames x tiles - 1 cover every (frame, tile) pair once,
// and the mapping agrees with the window arithmetic written out with signed
// 64-bit values, also for tickets at and beyond 2^31.
#include <algorithm>
#include <cstdio>
#include <vector>

#include "firing_loop_tc.cuh"

static void mapping64(unsigned long long t, int frames, int tiles, int W, long long *k, long long *tile) {
  const unsigned long long win = static_cast<unsigned long long>(W) * tiles;
  const unsigned long long w = t / win, r = t % win;
  const long long wc = std::min<long long>(W, static_cast<long long>(frames) - static_cast<long long>(w) * W);
  *k = static_cast<long long>(w) * W + static_cast<long long>(r % static_cast<unsigned long long>(wc));
  *tile = static_cast<long long>(r / static_cast<unsigned long long>(wc));
}

int main() {
  struct Case { int frames, tiles, W; };
  const Case small[] = {{1, 1, 1}, {7, 3, 2}, {13, 17, 5}, {2, 1, 8}, {5, 2048, 1}, {336, 1024, 336},
                        {1000, 1024, 1184}, {328, 1024, 1184}, {9, 4096, 4}};
  int bad = 0;
  for (const Case &c : small) {
    const unsigned long long total = static_cast<unsigned long long>(c.frames) * c.tiles;
    std::vector<char> seen(total, 0);
    for (unsigned long long t = 0; t < total; ++t) {
      int k, tile;
      long long k64, tile64;
      prune::tc_ticket_tile(t, c.frames, c.tiles, c.W, &k, &tile);
      mapping64(t, c.frames, c.tiles, c.W, &k64, &tile64);
      if (k != k64 || tile != tile64 || k < 0 || k >= c.frames || tile < 0 || tile >= c.tiles) {
        ++bad;
        continue;
      }
      if (seen[static_cast<unsigned long long>(k) * c.tiles + tile]++) ++bad;
    }
  }
  std::printf(bad ? "FAIL small %d\n" : "ok\n", bad);
  // tickets at and beyond 2^31 (the 64-bit quotient path)
  const Case big[] = {{3000, 1 << 20, 1000}, {70000, 32768, 148 * 8}, {2100, 1 << 20, 1}};
  int bad2 = 0;
  for (const Case &c : big) {
    const unsigned long long total = static_cast<unsigned long long>(c.frames) * c.tiles;
    for (unsigned long long i = 0; i < 20000; ++i) {
      const unsigned long long t = std::min(total - 1, (1ull << 31) - 10000 + i * 104729ull);
      int k, tile;
      long long k64, tile64;
      prune::tc_ticket_tile(t, c.frames, c.tiles, c.W, &k, &tile);
      mapping64(t, c.frames, c.tiles, c.W, &k64, &tile64);
      if (k != k64 || tile != tile64) ++bad2;
    }
  }
  std::printf(bad2 ? "FAIL big %d\n" : "ok\n", bad2);
  return bad || bad2;
}
