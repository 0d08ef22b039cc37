// Host side of the batched tensor-core FIR's work split: contiguous shares
// of its (instance, tile) items with equal estimated cost, one per
// persistent CTA.  Host-only C++ (no CUDA types), so that the split is
// checked on the CPU.
#pragma once
#include <algorithm>
#include <cstdint>
#include <vector>

namespace prune {

// Estimated cost of one FIR item in thousands of cycles of the batched
// tensor-core kernel on B300: a least-squares fit over the CTAs of clock
// probes (per item, per tile-full of samples, per GEMM shift beyond two,
// and per change of instance, whose tap operands are reloaded once the
// GEMMs before have drained).
constexpr double kFirCostItem = 2.1, kFirCostTile = 2.2, kFirCostShift = 0.14, kFirCostReload = 2.2;

// map[k] = (instance, tile) with .x and .y members, in launch order; tile
// is the samples per tile; inst(i, &samples, &shifts) gives instance i's
// frame length in samples and its GEMM shifts.  Writes cta[0..G]: CTA c
// fires items cta[c] .. cta[c + 1] - 1.  Each boundary is the prefix
// boundary nearest to its share of the total, so a share's cost is within
// one item's cost of total / G.
template <typename Item, typename InstFn>
inline void fir_cost_partition(const Item *map, int32_t items, int64_t tile, int G, InstFn inst, int32_t *cta) {
  std::vector<double> pre(static_cast<size_t>(items) + 1, 0.0);
  for (int32_t k = 0; k < items; ++k) {
    int64_t samples = 0;
    int shifts = 1;
    inst(map[k].x, &samples, &shifts);
    const int64_t nv = std::min<int64_t>(tile, samples - static_cast<int64_t>(map[k].y) * tile);
    double w = kFirCostItem + kFirCostTile * static_cast<double>(nv) / static_cast<double>(tile) +
               kFirCostShift * std::max(0, shifts - 2);
    if (k == 0 || map[k - 1].x != map[k].x) w += kFirCostReload;
    pre[k + 1] = pre[k] + w;
  }
  cta[0] = 0;
  for (int g = 1; g < G; ++g) {
    const double target = pre[items] * g / G;
    int32_t j = static_cast<int32_t>(std::lower_bound(pre.begin(), pre.end(), target) - pre.begin());
    if (j > 0 && target - pre[j - 1] < pre[j] - target) --j;  // the nearer boundary
    cta[g] = std::max(cta[g - 1], std::min(j, items));
  }
  cta[G] = items;
}

}  // namespace prune
