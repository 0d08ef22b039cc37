// The batched FIR's work split on the host: per-CTA shares of the item
// order must cover every item once, in order, and each share's estimated
// cost must lie within one item's cost of the mean share.
#include <cmath>
#include <cstdio>
#include <random>
#include <vector>

#include "batch_partition.hpp"

struct It {
  int32_t x, y;
};

static int fails = 0;
#define CHECK(c)                                                 \
  do {                                                           \
    if (!(c)) {                                                  \
      std::printf("FAIL %s:%d %s\n", __FILE__, __LINE__, #c);   \
      ++fails;                                                   \
    }                                                            \
  } while (0)

int main() {
  std::mt19937 rng(7);
  const int64_t tile = 4096;
  for (int trial = 0; trial < 200; ++trial) {
    const int n = 1 + static_cast<int>(rng() % 600);
    const int B = 32 << (rng() % 5);  // 32 .. 512
    std::vector<int64_t> samples(n);
    std::vector<int> shifts(n);
    std::vector<It> map;
    for (int i = 0; i < n; ++i) {
      const int F = 1 + static_cast<int>(rng() % 3000);
      samples[i] = static_cast<int64_t>(F) * B;
      shifts[i] = 1 + static_cast<int>(rng() % 5);
      const int64_t tiles = (samples[i] + tile - 1) / tile;
      for (int64_t t = 0; t < tiles; ++t) map.push_back({i, static_cast<int32_t>(t)});
    }
    if (trial % 2) {  // some orders interleave instances: more reloads
      std::shuffle(map.begin(), map.end(), rng);
    }
    const int32_t items = static_cast<int32_t>(map.size());
    const int G = std::min<int32_t>(1 + static_cast<int>(rng() % 200), items);
    std::vector<int32_t> cta(G + 1, -1);
    auto inst = [&](int32_t i, int64_t *s, int *h) {
      *s = samples[i];
      *h = shifts[i];
    };
    prune::fir_cost_partition(map.data(), items, tile, G, inst, cta.data());
    CHECK(cta[0] == 0 && cta[G] == items);
    for (int g = 0; g < G; ++g) CHECK(cta[g] <= cta[g + 1]);
    // item costs, written out from the model's terms
    std::vector<double> w(items);
    double total = 0, wmax = 0;
    for (int32_t k = 0; k < items; ++k) {
      const int i = map[k].x;
      const int64_t nv = std::min<int64_t>(tile, samples[i] - static_cast<int64_t>(map[k].y) * tile);
      w[k] = prune::kFirCostItem + prune::kFirCostTile * static_cast<double>(nv) / tile +
             prune::kFirCostShift * std::max(0, shifts[i] - 2) +
             ((k == 0 || map[k - 1].x != i) ? prune::kFirCostReload : 0.0);
      total += w[k];
      wmax = std::max(wmax, w[k]);
    }
    for (int g = 0; g < G; ++g) {
      double c = 0;
      for (int32_t k = cta[g]; k < cta[g + 1]; ++k) c += w[k];
      CHECK(c <= total / G + wmax + 1e-9);
    }
  }
  std::printf("cover ok\n");
  // equal items (one instance, full tiles, two shifts): equal counts, to within one
  {
    std::vector<It> map;
    for (int t = 0; t < 1000; ++t) map.push_back({0, t});
    std::vector<int32_t> cta(149);
    prune::fir_cost_partition(map.data(), 1000, tile, 148,
                              [](int32_t, int64_t *s, int *h) {
                                *s = 1000 * 4096;
                                *h = 2;
                              },
                              cta.data());
    for (int g = 1; g < 148; ++g) CHECK(cta[g + 1] - cta[g] == 6 || cta[g + 1] - cta[g] == 7);
  }
  std::printf("equal ok\n");
  // costlier items get smaller shares: first half T = 128 (five shifts), second half T = 32
  {
    std::vector<It> map;
    for (int t = 0; t < 2000; ++t) map.push_back({t < 1000 ? 0 : 1, t < 1000 ? t : t - 1000});
    std::vector<int32_t> cta(11);
    prune::fir_cost_partition(map.data(), 2000, tile, 10,
                              [](int32_t i, int64_t *s, int *h) {
                                *s = 1000 * 4096;
                                *h = i == 0 ? 5 : 2;
                              },
                              cta.data());
    CHECK(cta[1] - cta[0] < cta[10] - cta[9]);
  }
  std::printf("weights ok\n");
  return fails ? 1 : 0;
}
