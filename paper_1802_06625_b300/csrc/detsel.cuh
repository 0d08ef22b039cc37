// DET configuration actor and SEL dynamic actor (Sec. III-B/C, eq. (1)).
// DET: v[b] = (E_b > tau); the control token is (c, idx[0..c)) with
// c = sum_b BTOI(v[b]) and idx the ascending positions of the set elements
// (FIFO order is preserved, so the compaction is stable).  SEL consumes the
// token: its output DRP_b fires at rate BTOI(v[b]), which here means that the
// selected blocks are referenced in place by their compacted index list.
// One CTA of 1024 threads per frame: a warp ballot and popcount per 32
// blocks, a scan of the 32 warp counts, then the stable scatter of indices.
// The control token is written straight into the result record, so it never
// leaves the device.
#pragma once
#include "device_common.cuh"

namespace prune {

constexpr int kDetThreads = 1024;

struct DetSelParams {
  const float *energy;   // [slot][F]
  SlotMap eslot;
  int32_t F, frames;
  float tau;
  int32_t *c;            // [slot]
  int32_t *idx;          // [slot][F]
  int64_t *rec_frame;    // [slot] or nullptr
  SlotMap rslot;
  // graph bookkeeping (nullptr on the single-actor path)
  uint64_t *ctr;
  uint32_t *status;
  uint64_t cap_f4, cap_f5, cap_f6;
};

static __global__ void __launch_bounds__(kDetThreads) det_sel_kernel(DetSelParams p) {
  __shared__ int warp_off[32];
  __shared__ int total_s;
  const int k = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float *E = p.energy + p.eslot.slot(k) * p.F;
  const int64_t rs = p.rslot.slot(k);
  int32_t *idx = p.idx + rs * p.F;
  int running = 0;
  for (int r0 = 0; r0 < p.F; r0 += kDetThreads) {
    const int b = r0 + tid;
    const bool v = (b < p.F) && (E[b] > p.tau);
    const unsigned m = __ballot_sync(0xffffffffu, v);
    const int rank = __popc(m & ((1u << lane) - 1u));
    if (lane == 0) warp_off[warp] = __popc(m);
    __syncthreads();
    if (warp == 0) {
      const int cnt = warp_off[lane];
      int incl = cnt;
      for (int off = 1; off < 32; off <<= 1) {
        const int o = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += o;
      }
      warp_off[lane] = incl - cnt;
      if (lane == 31) total_s = incl;
    }
    __syncthreads();
    if (v) idx[running + warp_off[warp] + rank] = b;
    running += total_s;
    __syncthreads();
  }
  if (tid == 0) {
    p.c[rs] = running;
    if (p.rec_frame) p.rec_frame[rs] = p.rslot.seq0 + k;
    if (p.ctr) {
      const uint64_t frame = p.rslot.seq0 + k;
      fifo_release(p.ctr, 2, p.F, 0, p.status, kActDet, frame);          // DET reads f2
      fifo_commit(p.ctr, 4, 1, 0, p.cap_f4, p.status, kActDet, frame);   // control token
      fifo_commit(p.ctr, 5, 1, 0, p.cap_f5, p.status, kActDet, frame);   //   (broadcast)
      fifo_release(p.ctr, 4, 1, 0, p.status, kActSel, frame);            // SEL cport
      fifo_release(p.ctr, 3, p.F, 0, p.status, kActSel, frame);          // SEL SRP input
      fifo_commit(p.ctr, 6, running, 0, p.cap_f6, p.status, kActSel, frame);  // DRPs, eq. (1)
    }
  }
}

}  // namespace prune
