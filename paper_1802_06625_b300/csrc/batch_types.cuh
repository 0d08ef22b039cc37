// The batch's per-instance records and launch parameters (batched firing:
// one frame of each of many independent instances per step).
#pragma once
#include <cstdint>

#include <cuda_runtime.h>

namespace prune {

struct BatchInst {
  int64_t x_off;          // offset of this instance's frame in the step's input (samples)
  const float2 *x;        // or, when not null, the frame itself (request-loop entries)
  const float2 *taps;     // T taps
  const float2 *H;        // N x N
  const uint16_t *bops;   // tensor-core HX operands (N = 64) or nullptr
  const uint16_t *fops;   // tensor-core FIR tap operands (batch_fir_tc_kernel) or nullptr
  float2 *hist;           // [2][T-1] delay token, double buffered by step parity; when null:
  const float2 *hist_in;  //   the token before the frame (null = zeros), and
  float2 *hist_out;       //   where the token after the frame goes (null = not kept)
  float2 *y;              // FIR output frame, F*B
  float *energy;          // F
  int32_t *c;             // 1: selected blocks
  int32_t *idx;           // F
  float2 *out;            // compacted HX output, F*B
  int32_t F, T, TP, fir_tile0, hx_tile0, pad;
  float tau;
  int32_t s_taps, s_h;    // exponents of the scaled tensor-core operands (TcScale, host-computed)
};

struct BatchParams {
  const BatchInst *inst;
  const int2 *fir_map;      // FIR CTA -> (instance, tile of the instance), in launch order
  const int32_t *fir_cta;   // tensor-core FIR: CTA c fires items [fir_cta[c], fir_cta[c + 1]) of fir_map,
                            // fir_ctas CTAs (nullptr: equal counts over min(SMs, fir_tiles) CTAs)
  const int32_t *hx_map;    // HX work item -> instance (an instance's items are consecutive)
  const float2 *x;          // step input, all instances back to back
  int32_t n, B, N, TS, parity, fir_tiles, hx_items, fir_ctas;
  int32_t hx_chunk;         // > 0: CTA c fires items [c * hx_chunk, (c + 1) * hx_chunk); 0: grid-stride
  int32_t fir_tc;           // 1: FIR on tensor cores (TS = 4096, every instance has fops)
  int32_t *hx_pre;          // N = 64: [n + 1] selected 128-row tiles before each instance (written by DET/SEL)
  uint32_t *hx_ctr;         //   DET/SEL CTAs done (the last one writes hx_pre and resets it)
  uint64_t timeout_ns;
  uint32_t *status;
};

}  // namespace prune
