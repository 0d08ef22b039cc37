// FIR actor (static actor, Sec. III-B) with the DET energy reduction in its
// epilogue.  y[n] = sum_{t<T} h[t] x[n-t] over the continuous stream; the
// samples before a frame come from the previous frame of the launch or, for
// the first frame, from the delay token of the self-loop FIFO f1 (Sec. III-D).
//
// Tiling: a CTA of 256 threads fires one tile of TS samples (TS = the largest
// multiple of B not above 2048) of one frame; every thread produces 8
// consecutive outputs from a register window of 15 samples per group of 8
// taps.  The tile plus a halo of TP-1 samples (TP = T rounded up to 8; taps
// past T are zero) is staged in shared memory with float4 global loads.  The
// shared window uses one pad slot per 8 samples so that the 8-sample stride
// between threads is free of bank conflicts.
#pragma once
#include "device_common.cuh"

namespace prune {

constexpr int kFirThreads = 256;
constexpr int kSPT = 8;                         // outputs per thread
constexpr int kFirTile = kFirThreads * kSPT;    // 2048 output slots per CTA

__host__ __device__ __forceinline__ int fir_taps_padded(int T) { return (T + kSPT - 1) / kSPT * kSPT; }
__host__ __device__ __forceinline__ int pad_idx(int m) { return m + (m >> 3); }
__host__ __device__ __forceinline__ int fir_tile_samples(int B) { return (kFirTile / B) * B; }

// Output-tile layout for consumers of the FIR output in shared memory: two
// pad slots after every 8 samples, so that a thread's 8 outputs go out as
// four conflict-free float4 stores and sample pairs (2a, 2a+1) stay 16-byte
// aligned for float4 reads.
__host__ __device__ __forceinline__ int pad2_idx(int m) { return m + 2 * (m >> 3); }
constexpr int kYsSlots = kFirTile + 2 * (kFirTile / 8);  // 2560

// Complex slots of the window region (also holds the output tile).
__host__ __device__ __forceinline__ int fir_window_slots(int TP) {
  const int w = pad_idx(TP - 1 + kFirTile - 1) + 2;
  return w > kYsSlots ? w : kYsSlots;
}

// window + taps + 32 reduction slots + 256 block energies
__host__ __device__ inline size_t fir_smem_bytes(int T) {
  const int TP = fir_taps_padded(T);
  const size_t xs = static_cast<size_t>(fir_window_slots(TP)) * sizeof(float2);
  return xs + static_cast<size_t>(TP) * sizeof(float2) + (32 + 256) * sizeof(float);
}

struct FirParams {
  FrameSrc src;          // input frames (f0)
  int64_t L;             // samples per frame, F*B
  int32_t F, B, T, TP, TS, tiles, frames;
  const float2 *taps;    // T taps
  const float2 *hist;    // delay token before frame 0 (T-1 samples) or nullptr = zeros
  float2 *y;             // output frames or nullptr
  int64_t y_stride;
  SlotMap yslot;
  float *energy;         // [slot][F] block energies or nullptr
  SlotMap eslot;
  float2 *hist_out;      // delay token after the last frame, or nullptr
  // graph bookkeeping (nullptr on the single-actor path)
  uint64_t *ctr;
  uint32_t *status;
  uint64_t cap_f1, cap_f2, cap_f3;
};

// Stage the tile window: halo of TP-1 samples before s0 (previous frame of
// the launch, else the delay token, else zeros; zeros beyond T-1 where the
// padded taps are zero) and the body [s0, s0 + 2048) with float4 loads
// (zeros past the frame).
__device__ __forceinline__ void fir_stage_window(float2 *xs, const float2 *cur, const float2 *prev,
                                                 const float2 *hist, int64_t L, int T, int TP, int64_t s0,
                                                 int nv, int tid) {
  for (int m = tid; m < TP - 1; m += kFirThreads) {
    const int d = TP - 1 - m;
    const int64_t pos = s0 - d;
    float2 v = make_float2(0.f, 0.f);
    if (d <= T - 1) {
      if (pos >= 0) v = cur[pos];
      else if (prev) v = prev[L + pos];
      else if (hist) v = hist[T - 1 + pos];
    }
    xs[pad_idx(m)] = v;
  }
  const float4 *body = reinterpret_cast<const float4 *>(cur + s0);
  for (int q2 = tid; q2 < kFirTile / 2; q2 += kFirThreads) {
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (2 * q2 < nv) v = __ldg(body + q2);
    const int m = TP - 1 + 2 * q2;
    xs[pad_idx(m)] = make_float2(v.x, v.y);
    xs[pad_idx(m + 1)] = make_float2(v.z, v.w);
  }
}

// 8 consecutive outputs per thread: acc[j] = y[s0 + 8*tid + j].
__device__ __forceinline__ void fir_compute(const float2 *xs, const float2 *hs, int TP, int tid, float2 (&acc)[kSPT]) {
#pragma unroll
  for (int j = 0; j < kSPT; ++j) acc[j] = make_float2(0.f, 0.f);
  const int obase = tid * kSPT;
  for (int t0 = 0; t0 < TP; t0 += kSPT) {
    // r[m] = window[start + m], start = TP - 8 + obase - t0 (a multiple of 8)
    const int start = TP - kSPT + obase - t0;
    const int ps = pad_idx(start);
    float2 r[2 * kSPT - 1];
#pragma unroll
    for (int m = 0; m < kSPT; ++m) r[m] = xs[ps + m];
#pragma unroll
    for (int m = kSPT; m < 2 * kSPT - 1; ++m) r[m] = xs[ps + m + 1];
    float2 h[kSPT];
#pragma unroll
    for (int u = 0; u < kSPT; ++u) h[u] = hs[t0 + u];
#pragma unroll
    for (int u = 0; u < kSPT; ++u)
#pragma unroll
      for (int j = 0; j < kSPT; ++j) cmac(acc[j], h[u], r[kSPT - 1 + j - u]);
  }
}

// DET energies of the tile's blocks, E_b = sum |y|^2, into Et[nv / B]
// (shared memory), in a fixed reduction order.  Ends with a barrier.
__device__ __forceinline__ void fir_block_energies(const float2 (&acc)[kSPT], int B, int nv, int tid, float *red,
                                                   float *Et) {
  const int obase = tid * kSPT;
  float e = 0.f;
#pragma unroll
  for (int j = 0; j < kSPT; ++j)
    if (obase + j < nv) e = fmaf(acc[j].x, acc[j].x, fmaf(acc[j].y, acc[j].y, e));
  const int tpb = B / kSPT;  // threads per block
  const int seg = tpb < 32 ? tpb : 32;
  for (int off = seg >> 1; off > 0; off >>= 1) e += __shfl_xor_sync(0xffffffffu, e, off);
  if (tpb <= 32) {
    if ((tid % seg) == 0 && obase < nv) Et[obase / B] = e;
  } else {
    const int lane = tid & 31, warp = tid >> 5;
    if (lane == 0) red[warp] = e;
    __syncthreads();
    const int wpb = tpb / 32;
    if (tid < nv / B) {
      float s = 0.f;
      for (int w = 0; w < wpb; ++w) s += red[tid * wpb + w];
      Et[tid] = s;
    }
  }
  __syncthreads();
}

static __global__ void __launch_bounds__(kFirThreads) fir_energy_kernel(FirParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int TP = p.TP;
  const int win = TP - 1 + kFirTile;
  float2 *xs = reinterpret_cast<float2 *>(smem_raw);
  float2 *hs = xs + fir_window_slots(TP);
  float *red = reinterpret_cast<float *>(hs + TP);
  float *Et = red + 32;
  (void)win;

  const int tid = threadIdx.x;
  const int k = blockIdx.y;
  const int64_t s0 = static_cast<int64_t>(blockIdx.x) * p.TS;
  const int nv = static_cast<int>(min(static_cast<int64_t>(p.TS), p.L - s0));
  const float2 *cur = p.src.frame(k);
  const float2 *prev = k > 0 ? p.src.frame(k - 1) : nullptr;

  for (int t = tid; t < TP; t += kFirThreads) hs[t] = t < p.T ? p.taps[t] : make_float2(0.f, 0.f);
  fir_stage_window(xs, cur, prev, p.hist, p.L, p.T, TP, s0, nv, tid);
  __syncthreads();

  float2 acc[kSPT];
  fir_compute(xs, hs, TP, tid, acc);
  fir_block_energies(acc, p.B, nv, tid, red, Et);
  if (p.energy && tid < nv / p.B) p.energy[p.eslot.slot(k) * p.F + s0 / p.B + tid] = Et[tid];

  // next delay token (f1): the last T-1 input samples of the last frame
  if (p.hist_out && k == p.frames - 1 && s0 + nv == p.L) {
    for (int m = tid; m < p.T - 1; m += kFirThreads)
      p.hist_out[m] = xs[pad_idx(TP - 1 + nv - (p.T - 1) + m)];
  }

  // FIFO bookkeeping of the launch's firings, in frame order (the f1 token of
  // frame k+1 is the one frame k produced), by one thread.
  if (p.ctr && blockIdx.x == 0 && blockIdx.y == 0 && tid == 0) {
    for (int kk = 0; kk < p.frames; ++kk) {
      const uint64_t frame = p.yslot.seq0 + kk;
      fifo_release(p.ctr, 0, p.F, 0, p.status, kActFir, frame);
      fifo_release(p.ctr, 1, 1, 1, p.status, kActFir, frame);
      fifo_commit(p.ctr, 1, 1, 1, p.cap_f1, p.status, kActFir, frame);
      fifo_commit(p.ctr, 2, p.F, 0, p.cap_f2, p.status, kActFir, frame);
      fifo_commit(p.ctr, 3, p.F, 0, p.cap_f3, p.status, kActFir, frame);
    }
  }

  if (p.y == nullptr) return;
  // y out through shared memory (padded layout, then coalesced float4)
  __syncthreads();
  float2 *ys = xs;
  const int obase = tid * kSPT;
#pragma unroll
  for (int j = 0; j < kSPT; ++j) ys[pad_idx(obase + j)] = acc[j];
  __syncthreads();
  float4 *out = reinterpret_cast<float4 *>(p.y + p.yslot.slot(k) * p.y_stride + s0);
  for (int q2 = tid; 2 * q2 < nv; q2 += kFirThreads) {
    const float2 a = ys[pad_idx(2 * q2)], b = ys[pad_idx(2 * q2 + 1)];
    out[q2] = make_float4(a.x, a.y, b.x, b.y);
  }
}

}  // namespace prune
