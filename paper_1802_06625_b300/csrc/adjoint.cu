// Adjoint (reverse-mode) kernels of the firing path over a recorded control
// trace, for training the FIR taps and H.  With the trace (c, idx) fixed the
// sink output is linear in H and in the taps; in the complex-gradient
// convention g = dL/dRe + i dL/dIm:
//   HX_b:  z = H w per selected row  ->  dL/dH += g_z w^H,  g_w = H^H g_z
//   FIR:   y[n] = sum_t h[t] x[n-t]  ->  dL/dh[t] = sum_n g_y[n] conj(x[n-t])
// with g_y = g_w on the selected blocks and 0 elsewhere (the inactive DCs
// carry no gradient, itr = 0).  The decisions themselves are piecewise
// constant and contribute nothing.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdint>
#include <string>

#include "prune.h"
#include "device_common.cuh"
#include "fir.cuh"

using namespace prune;

void prune_set_create_error(const std::string &m);  // prune_runtime.cu

namespace {

__device__ __forceinline__ float2 cmul_conj_b(float2 a, float2 b) {  // a * conj(b)
  return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}

struct AdjHxParams {
  const float2 *y;      // FIR output frames [frames][F*B] (the HX inputs)
  const int32_t *idx;   // [frames][F]
  const int32_t *c;     // [frames]
  const float2 *H;      // [N][N]
  const float2 *gout;   // [frames][F*B]: gradient of the compacted sink output (first c*B)
  float2 *gy;           // [frames][F*B]: gradient of y, written on the selected blocks
  float2 *gH;           // [N][N]: accumulated
  int32_t F, B, N, frames;
};

// Shared memory: H (N*N) | g block (B) | w block (B) | per-CTA dL/dH (N*N)
__global__ void __launch_bounds__(256) adj_hx_kernel(AdjHxParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = p.N, NN = N * N;
  float2 *Hs = reinterpret_cast<float2 *>(smem_raw);
  float2 *gs = Hs + NN;
  float2 *ws = gs + p.B;
  float2 *part = ws + p.B;
  const int tid = threadIdx.x;
  for (int q = tid; q < NN; q += 256) {
    Hs[q] = p.H[q];
    part[q] = make_float2(0.f, 0.f);
  }
  const int64_t L = static_cast<int64_t>(p.F) * p.B;
  const int64_t total = static_cast<int64_t>(p.frames) * p.F;
  for (int64_t w = blockIdx.x; w < total; w += gridDim.x) {
    const int k = static_cast<int>(w / p.F), j = static_cast<int>(w % p.F);
    const int ck = min(max(p.c[k], 0), p.F);
    if (j >= ck) continue;
    const int b = p.idx[static_cast<int64_t>(k) * p.F + j];
    if (b < 0 || b >= p.F) continue;
    __syncthreads();
    const float2 *g = p.gout + k * L + static_cast<int64_t>(j) * p.B;
    const float2 *yw = p.y + k * L + static_cast<int64_t>(b) * p.B;
    for (int q = tid; q < p.B; q += 256) {
      gs[q] = g[q];
      ws[q] = yw[q];
    }
    __syncthreads();
    // g_w = H^H g_z, row by row, written at the block's place in the frame
    float2 *gyb = p.gy + k * L + static_cast<int64_t>(b) * p.B;
    for (int q = tid; q < p.B; q += 256) {
      const int r = q / N, kk = q % N;
      float2 a = make_float2(0.f, 0.f);
      for (int i = 0; i < N; ++i) {
        const float2 h = Hs[i * N + kk], gz = gs[r * N + i];
        a.x = fmaf(h.x, gz.x, fmaf(h.y, gz.y, a.x));
        a.y = fmaf(h.x, gz.y, fmaf(-h.y, gz.x, a.y));
      }
      gyb[q] = a;
    }
    // dL/dH += sum over the block's rows of g_z w^H (entries owned by thread)
    const int R = p.B / N;
    for (int e = tid; e < NN; e += 256) {
      const int i = e / N, kk = e % N;
      float2 a = part[e];
      for (int r = 0; r < R; ++r) {
        const float2 t = cmul_conj_b(gs[r * N + i], ws[r * N + kk]);
        a.x += t.x;
        a.y += t.y;
      }
      part[e] = a;
    }
  }
  __syncthreads();
  for (int e = tid; e < NN; e += 256) {
    atomicAdd(&p.gH[e].x, part[e].x);
    atomicAdd(&p.gH[e].y, part[e].y);
  }
}

struct AdjFirParams {
  const float2 *x;      // [frames][F*B] input stream
  const float2 *hist;   // T-1 samples before frame 0 (or nullptr = zeros)
  const float2 *gy;     // [frames][F*B] gradient of the FIR output
  float2 *gtaps;        // [T] accumulated
  int64_t L;
  int32_t F, B, T, TP, TS, frames;
};

// dL/dh[t] = sum_n g_y[n] conj(x[n-t]) on one tile: thread (t, group) sums the
// group's samples for tap t; groups reduced in shared memory; one atomic per
// tap and tile.  The input window is staged as for the forward FIR.
__global__ void __launch_bounds__(kFirThreads) adj_fir_kernel(AdjFirParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int TP = p.TP;
  float2 *xs = reinterpret_cast<float2 *>(smem_raw);
  float2 *gs = xs + fir_window_slots(TP);
  float2 *red = gs + kFirTile;
  const int tid = threadIdx.x;
  const int k = blockIdx.y;
  const int64_t s0 = static_cast<int64_t>(blockIdx.x) * p.TS;
  const int nv = static_cast<int>(min(static_cast<int64_t>(p.TS), p.L - s0));
  const float2 *cur = p.x + k * p.L;
  const float2 *prev = k > 0 ? p.x + (k - 1) * p.L : nullptr;
  fir_stage_window(xs, cur, prev, p.hist, p.L, p.T, TP, s0, nv, tid);
  const float2 *g = p.gy + k * p.L + s0;
  bool any = false;
  for (int q = tid; q < kFirTile; q += kFirThreads) {
    const float2 v = q < nv ? g[q] : make_float2(0.f, 0.f);
    gs[q] = v;
    any |= (v.x != 0.f || v.y != 0.f);
  }
  if (!__syncthreads_or(any)) return;  // no selected block in this tile
  const int G = kFirThreads / TP;        // sample groups (TP divides 256: TP in {8, ..., 256}, power-of-two steps)
  const int t = tid % TP, grp = tid / TP;
  float2 a = make_float2(0.f, 0.f);
  if (grp < G) {
    for (int n = grp; n < nv; n += G) {
      // x[n - t] is window index TP - 1 + n - t
      const float2 xv = xs[pad_idx(TP - 1 + n - t)];
      const float2 gv = gs[n];
      a.x = fmaf(gv.x, xv.x, fmaf(gv.y, xv.y, a.x));
      a.y = fmaf(gv.y, xv.x, fmaf(-gv.x, xv.y, a.y));
    }
  }
  red[tid] = a;
  __syncthreads();
  if (tid < TP && tid < p.T) {
    float2 s = make_float2(0.f, 0.f);
    for (int q = 0; q < G; ++q) {
      s.x += red[q * TP + tid].x;
      s.y += red[q * TP + tid].y;
    }
    atomicAdd(&p.gtaps[tid].x, s.x);
    atomicAdd(&p.gtaps[tid].y, s.y);
  }
}

prune_status afail(prune_status s, const std::string &m) {
  prune_set_create_error(m);
  return s;
}

}  // namespace

extern "C" {

prune_status prune_hx_adjoint(const void *y, const int32_t *idx, const int32_t *c, int32_t F, int32_t B, int32_t N,
                              int32_t frames, const void *H, const void *gout, void *gy, void *gH, void *stream) {
  if (!y || !idx || !c || !H || !gout || !gy || !gH || F < 1 || B < 1 || N < 1 || N > 64 || B % N != 0 || frames < 0)
    return afail(PRUNE_EINVAL, "prune_hx_adjoint: bad argument");
  if (frames == 0) return PRUNE_OK;
  AdjHxParams p{static_cast<const float2 *>(y), idx, c, static_cast<const float2 *>(H),
                static_cast<const float2 *>(gout), static_cast<float2 *>(gy), static_cast<float2 *>(gH), F, B, N, frames};
  const size_t smem = (2 * static_cast<size_t>(N) * N + 2 * static_cast<size_t>(B)) * sizeof(float2);
  if (smem > 200 * 1024) return afail(PRUNE_EINVAL, "prune_hx_adjoint: N and B too large");
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(adj_hx_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) !=
          cudaSuccess)
    return afail(PRUNE_ECUDA, "prune_hx_adjoint: shared memory attribute");
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t work = static_cast<int64_t>(frames) * F;
  const int grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(work, sms * 4)));
  adj_hx_kernel<<<grid, 256, smem, static_cast<cudaStream_t>(stream)>>>(p);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return afail(PRUNE_ECUDA, std::string("prune_hx_adjoint: ") + cudaGetErrorString(e));
  return PRUNE_OK;
}

prune_status prune_fir_adjoint(const void *x, const void *hist, const void *gy, int32_t F, int32_t B, int32_t T,
                               int32_t frames, void *gtaps, void *stream) {
  if (!x || !gy || !gtaps || F < 1 || B < 8 || B > kFirTile || B % 8 != 0 || T < 1 || T > 256 || T - 1 > B ||
      frames < 0)
    return afail(PRUNE_EINVAL, "prune_fir_adjoint: bad argument");
  if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(gy)) & 15u)
    return afail(PRUNE_EINVAL, "prune_fir_adjoint: x and gy must be 16-byte aligned");
  if (frames == 0) return PRUNE_OK;
  AdjFirParams p{};
  p.x = static_cast<const float2 *>(x);
  p.hist = T > 1 ? static_cast<const float2 *>(hist) : nullptr;
  p.gy = static_cast<const float2 *>(gy);
  p.gtaps = static_cast<float2 *>(gtaps);
  p.L = static_cast<int64_t>(F) * B;
  p.F = F; p.B = B; p.T = T;
  // taps rounded up to a power of two >= 8 so that the sample groups divide 256
  int TPp = 8;
  while (TPp < T) TPp <<= 1;
  p.TP = TPp;
  p.TS = fir_tile_samples(B);
  p.frames = frames;
  const int tiles = static_cast<int>((p.L + p.TS - 1) / p.TS);
  const size_t smem = static_cast<size_t>(fir_window_slots(TPp)) * sizeof(float2) +
                      (static_cast<size_t>(kFirTile) + kFirThreads) * sizeof(float2);
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(adj_fir_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) !=
          cudaSuccess)
    return afail(PRUNE_ECUDA, "prune_fir_adjoint: shared memory attribute");
  adj_fir_kernel<<<dim3(tiles, frames), kFirThreads, smem, static_cast<cudaStream_t>(stream)>>>(p);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return afail(PRUNE_ECUDA, std::string("prune_fir_adjoint: ") + cudaGetErrorString(e));
  return PRUNE_OK;
}

}  // extern "C"
