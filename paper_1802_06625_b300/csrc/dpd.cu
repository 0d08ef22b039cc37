// Dynamic Predistortion workload (Sec. VII-A2): K filter branches on the
// memory-polynomial basis psi_k(x) = x |x|^(k-1), k = 1..K, each with its own
// T taps and its own delay token; a control mask per period of `period`
// samples selects the branches that fire, and the adder sums them.  A branch
// that does not fire keeps its delay token (its DC fires zero times, itr = 0),
// so the token a branch brings into period p is the tail of psi_k over the
// last earlier period in which it fired.  Because psi_k depends on the input
// alone, a scan over the control masks gives every period its branches'
// tokens up front and all periods fire in parallel.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <string>

#include "prune.h"
#include "device_common.cuh"
#include "fir.cuh"

using namespace prune;

void prune_set_create_error(const std::string &m);  // prune_runtime.cu

namespace {

constexpr int kDpdThreads = 256;
constexpr int kDpdSPT = 8;                            // outputs per thread
constexpr int kDpdTile = kDpdThreads * kDpdSPT;       // 2048 outputs per CTA
constexpr int kDpdMaxK = 16;
constexpr int kDpdMaxT = 16;

// psi_k(x) = x |x|^(k-1) in FP32: an integer power of |x|^2, times |x| when
// k-1 is odd.
__device__ __forceinline__ float2 dpd_psi(float2 x, int k) {
  const float r2 = x.x * x.x + x.y * x.y;
  float s = 1.f;
  for (int e = 2; e <= k - 1; e += 2) s *= r2;
  if ((k - 1) & 1) s *= sqrtf(r2);
  return make_float2(x.x * s, x.y * s);
}

struct DpdParams {
  const float2 *x;       // [P][period]
  int64_t period;
  int32_t P, K, T;
  const uint16_t *mask;  // [P]
  const float2 *taps;    // [K][T]
  const float2 *hist;    // [K][T-1] tokens before period 0, or nullptr (zeros)
  const int32_t *last;   // [K][P] last earlier period where branch k fired, -1 = none
  float2 *y;             // [P][period]
};

// One warp per branch: last[k][p] = the last period q < p with bit k set in
// mask[q] (or -1), 32 periods per ballot; last_all[k] = the last such period
// over all P.
__global__ void dpd_scan_kernel(const uint16_t *mask, int32_t P, int32_t K, int32_t *last, int32_t *last_all) {
  const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (k >= K) return;
  int carry = -1;
  for (int p0 = 0; p0 < P; p0 += 32) {
    const int pp = p0 + lane;
    const bool on = pp < P && ((mask[pp] >> k) & 1u);
    const unsigned bits = __ballot_sync(0xffffffffu, on);
    const unsigned before = bits & ((1u << lane) - 1u);
    if (pp < P) last[static_cast<int64_t>(k) * P + pp] = before ? p0 + 31 - __clz(before) : carry;
    if (bits) carry = p0 + 31 - __clz(bits);
  }
  if (lane == 0) last_all[k] = carry;
}

// Delay tokens after the last period: the tail of psi_k over the last period
// where branch k fired, else the incoming token.  hist_out may alias hist_in
// (each thread reads and writes the same element).
__global__ void dpd_hist_kernel(const float2 *x, int64_t period, int32_t K, int32_t T, const int32_t *last_all,
                                const float2 *hist_in, float2 *hist_out) {
  const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int H = T - 1;
  if (k >= K) return;
  const int lp = last_all[k];
  for (int m = lane; m < H; m += 32) {
    float2 v = make_float2(0.f, 0.f);
    if (lp >= 0) v = dpd_psi(x[static_cast<int64_t>(lp) * period + period - H + m], k + 1);
    else if (hist_in) v = hist_in[k * H + m];
    hist_out[k * H + m] = v;
  }
}

// One CTA per (tile of 2048 outputs, period).  The input window (NT-1 halo
// samples + the tile) is staged in shared memory once; each thread then
// reads its own window slots (its 8 outputs and the NT-1 samples before
// them) into registers and carries psi_k there across the branches,
// psi_{k+1} = psi_k |x|, so a branch needs no shared memory and no barrier.
// Only the first tile's halo differs per branch (the tail of psi_k over the
// last earlier period where branch k fired, or the incoming token): the
// threads whose window reaches it (tid 0 and 1) read it per branch.  Taps
// t >= T are zero, so NT >= T taps are computed.
template <int NT>
__global__ void __launch_bounds__(kDpdThreads, NT <= 10 ? 3 : 2) dpd_kernel(DpdParams p) {
  constexpr int HW = NT - 1;                                   // halo slots of the window
  constexpr int kWin = (HW + kDpdTile) + ((HW + kDpdTile) >> 3) + 2;
  constexpr int R = kDpdSPT + HW;                              // a thread's window slots
  __shared__ __align__(16) float2 xw[kWin];  // slot w: x at sample s0 - HW + w; at the end, the outputs
  __shared__ float2 hs[kDpdMaxK * NT];
  const int tid = threadIdx.x;
  const int pi = blockIdx.y, tile = blockIdx.x;
  const int64_t s0 = static_cast<int64_t>(tile) * kDpdTile;
  const int nv = static_cast<int>(min(static_cast<int64_t>(kDpdTile), p.period - s0));
  const float2 *base = p.x + static_cast<int64_t>(pi) * p.period;
  const int H = p.T - 1;
  const float4 *src = reinterpret_cast<const float4 *>(base + s0);
  for (int q = tid; q < kDpdTile / 2; q += kDpdThreads) {
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (2 * q < nv) v = __ldg(src + q);
    xw[pad_idx(HW + 2 * q)] = make_float2(v.x, v.y);
    xw[pad_idx(HW + 2 * q + 1)] = make_float2(v.z, v.w);
  }
  if (tid < HW) {  // halo past the first tile: the input before s0 where a tap reaches
    const int i = tid - HW;
    float2 v = make_float2(0.f, 0.f);
    if (tile > 0 && i >= -H) v = __ldg(base + s0 + i);
    xw[pad_idx(tid)] = v;
  }
  for (int q = tid; q < p.K * NT; q += kDpdThreads) {
    const int k = q / NT, t = q % NT;
    hs[q] = t < p.T ? p.taps[k * p.T + t] : make_float2(0.f, 0.f);
  }
  const uint32_t m = p.mask[pi];
  const int ob = tid * kDpdSPT;
  __syncthreads();
  float2 px[R];
  float rx[R];
#pragma unroll
  for (int q = 0; q < R; ++q) {
    px[q] = xw[pad_idx(ob + q)];
    rx[q] = sqrtf(px[q].x * px[q].x + px[q].y * px[q].y);
  }
  const bool first_halo = tile == 0 && ob < HW;  // the window reaches before the period's first sample
  float2 acc[kDpdSPT];
#pragma unroll
  for (int j = 0; j < kDpdSPT; ++j) acc[j] = make_float2(0.f, 0.f);
  for (int k = 0; k < p.K; ++k) {
    if (k > 0) {
#pragma unroll
      for (int q = 0; q < R; ++q) px[q] = make_float2(px[q].x * rx[q], px[q].y * rx[q]);
    }
    if (!((m >> k) & 1u)) continue;  // the same branch set for the whole CTA
    if (first_halo) {  // these slots hold zeros (rx = 0): set them to the branch's token
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const int i = ob + q - HW;  // sample offset from the period's start
        if (i < 0) {
          float2 v = make_float2(0.f, 0.f);
          if (i >= -H) {
            const int lp = p.last[static_cast<int64_t>(k) * p.P + pi];
            if (lp >= 0) v = dpd_psi(p.x[static_cast<int64_t>(lp) * p.period + p.period + i], k + 1);
            else if (p.hist) v = p.hist[k * H + H + i];
          }
          px[q] = v;
        }
      }
    }
    const float2 *h = hs + k * NT;
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const float2 ht = h[t];
#pragma unroll
      for (int j = 0; j < kDpdSPT; ++j) cmac(acc[j], ht, px[HW + j - t]);
    }
  }
  // coalesced store through shared memory (the window is no longer read
  // once every thread has passed this barrier)
  __syncthreads();
#pragma unroll
  for (int j = 0; j < kDpdSPT; ++j) xw[pad_idx(ob + j)] = acc[j];
  __syncthreads();
  float4 *out = reinterpret_cast<float4 *>(p.y + static_cast<int64_t>(pi) * p.period + s0);
  for (int q = tid; 2 * q < nv; q += kDpdThreads) {
    const float2 a = xw[pad_idx(2 * q)], b = xw[pad_idx(2 * q + 1)];
    out[q] = make_float4(a.x, a.y, b.x, b.y);
  }
}

prune_status dfail(prune_status s, const std::string &m) {
  prune_set_create_error(m);
  return s;
}

}  // namespace

extern "C" {

size_t prune_dpd_workspace_bytes(int32_t P, int32_t K) {
  if (P < 0 || K < 0) return 0;
  return sizeof(int32_t) * (static_cast<size_t>(K) * P + K) + 16;
}

prune_status prune_dpd_fire(const void *x, int64_t period, int32_t P, const uint16_t *mask, int32_t K, int32_t T,
                            const void *taps, const void *hist_in, void *hist_out, void *y, void *workspace,
                            size_t workspace_bytes, void *stream) {
  if (!x || !mask || !taps || !y || !workspace || P < 0 || K < 1 || K > kDpdMaxK || T < 1 || T > kDpdMaxT ||
      period < 8 || period % 8 != 0 || period < T - 1 || period > (int64_t{1} << 40))
    return dfail(PRUNE_EINVAL, "prune_dpd_fire: bad argument");
  if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) & 15u)
    return dfail(PRUNE_EINVAL, "prune_dpd_fire: x and y must be 16-byte aligned");
  if (workspace_bytes < prune_dpd_workspace_bytes(P, K))
    return dfail(PRUNE_EINVAL, "prune_dpd_fire: workspace too small");
  if (P == 0) return PRUNE_OK;
  const int64_t tiles = (period + kDpdTile - 1) / kDpdTile;
  if (tiles > (int64_t{1} << 31) - 1 || P > 65535) return dfail(PRUNE_EINVAL, "prune_dpd_fire: too many tiles or periods");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int32_t *last = static_cast<int32_t *>(workspace);
  int32_t *last_all = last + static_cast<int64_t>(K) * P;
  dpd_scan_kernel<<<1, 32 * K, 0, s>>>(mask, P, K, last, last_all);
  DpdParams dp{static_cast<const float2 *>(x), period, P, K, T, mask, static_cast<const float2 *>(taps),
               T > 1 ? static_cast<const float2 *>(hist_in) : nullptr, last, static_cast<float2 *>(y)};
  const dim3 grid(static_cast<unsigned>(tiles), static_cast<unsigned>(P));
  if (T == 10) dpd_kernel<10><<<grid, kDpdThreads, 0, s>>>(dp);
  else dpd_kernel<kDpdMaxT><<<grid, kDpdThreads, 0, s>>>(dp);
  if (T > 1 && hist_out)
    dpd_hist_kernel<<<1, 32 * K, 0, s>>>(static_cast<const float2 *>(x), period, K, T, last_all,
                                          static_cast<const float2 *>(hist_in), static_cast<float2 *>(hist_out));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return dfail(PRUNE_ECUDA, std::string("prune_dpd_fire: ") + cudaGetErrorString(e));
  return PRUNE_OK;
}

}  // extern "C"
