// Host check of RingSlot (the fused loops' ring slots from a per-launch
// base): RingSlot::of(seq0, cap).at(k) == (seq0 + k) mod cap for every
// k >= 0, including k of several times cap and seq0 beyond 2^31.
#include <cstdio>

#include "device_common.cuh"

int main() {
  const long long seq0s[] = {0, 1, 2, 335, 336, 1000, 4095, 123456789, (1ll << 31) + 7, (1ll << 40) + 12345};
  const int caps[] = {1, 2, 3, 5, 7, 48, 336, 4096, 1 << 20};
  long long bad = 0, checked = 0;
  for (long long seq0 : seq0s)
    for (int cap : caps) {
      const prune::RingSlot r = prune::RingSlot::of(seq0, cap);
      for (int k = 0; k < 3 * cap + 5 && k < 20000; ++k) {
        ++checked;
        if (r.at(k) != static_cast<int>((seq0 + k) % cap)) ++bad;
      }
    }
  std::printf(bad ? "FAIL %lld of %lld\n" : "ok %lld\n", bad, checked);
  return bad != 0;
}
