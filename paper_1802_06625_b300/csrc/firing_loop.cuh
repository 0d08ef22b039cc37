// Fused persistent firing loop (placeholder until the fused kernel lands).
#pragma once
#include "device_common.cuh"
namespace prune {
struct LoopScratch {
  uint64_t ticket;
};
__host__ inline bool loop_supported(int N) { (void)N; return false; }
}  // namespace prune
