// HX_b static actors (the F dynamic components of the DPG, Sec. V) on CUDA
// cores, for N < 64.  For every selected block (j < c, read on the device):
// X = reshape(block, (B/N, N)) row-major, out[r*N+i] = sum_k H[i][k] X[r][k].
// The SINK's DRP_b consumes the result in place: it is written at compacted
// position j of the frame record.
//
// Persistent grid-stride CTAs of 256 threads; thread (i, g) owns column i of
// H in registers (row i of H) and row group g; the block is staged in shared
// memory so that the X[r][k] reads are warp broadcasts.
#pragma once
#include "device_common.cuh"

namespace prune {

constexpr int kHxThreads = 256;

struct HxParams {
  const float2 *y;      // source frames (the f2/f3 tokens)
  int64_t y_stride;
  SlotMap yslot;
  const int32_t *c;     // control token: c[slot], idx[slot][F]
  const int32_t *idx;
  SlotMap rslot;
  float2 *out;          // destination frames (record payload)
  int64_t out_stride;
  SlotMap oslot;
  const float2 *H;      // [N][N]
  int32_t F, B, N, frames;
  // graph bookkeeping
  uint64_t *ctr;
  uint32_t *status;
  uint64_t cap_f7;
};

__device__ __forceinline__ void hx_bookkeeping(const HxParams &p, int k, int ck) {
  const uint64_t frame = p.rslot.seq0 + k;
  fifo_release(p.ctr, 6, ck, 0, p.status, kActHx, frame);               // HX_b read f6_b
  fifo_commit(p.ctr, 7, ck, 0, p.cap_f7, p.status, kActHx, frame);       // HX_b write f7_b
  fifo_release(p.ctr, 5, 1, 0, p.status, kActSink, frame);               // SINK cport
  fifo_release(p.ctr, 7, ck, 0, p.status, kActSink, frame);              // SINK DRPs
}

// Shared memory: max(B, N*N) complex (H is staged through it first).
template <int NT>
__global__ void __launch_bounds__(kHxThreads) hx_cuda_kernel(HxParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2 *xs = reinterpret_cast<float2 *>(smem_raw);
  const int tid = threadIdx.x;
  const int i = tid % NT, g = tid / NT;
  constexpr int RG = kHxThreads / NT;
  const int R = p.B / NT;
  for (int q = tid; q < NT * NT; q += kHxThreads) xs[q] = p.H[q];
  __syncthreads();
  float2 h[NT];
#pragma unroll
  for (int kk = 0; kk < NT; ++kk) h[kk] = xs[i * NT + kk];
  const int64_t total = static_cast<int64_t>(p.frames) * p.F;
  for (int64_t w = blockIdx.x; w < total; w += gridDim.x) {
    const int k = static_cast<int>(w / p.F), j = static_cast<int>(w % p.F);
    const int64_t rs = p.rslot.slot(k);
    const int ck = min(max(p.c[rs], 0), p.F);
    if (j == 0 && tid == 0 && p.ctr) hx_bookkeeping(p, k, ck);
    if (j >= ck) continue;  // inactive: uniform over the CTA
    const int b = p.idx[rs * p.F + j];
    if (b < 0 || b >= p.F) continue;  // malformed control token from a caller
    const float4 *src = reinterpret_cast<const float4 *>(p.y + p.yslot.slot(k) * p.y_stride +
                                                         static_cast<int64_t>(b) * p.B);
    float2 *dst = p.out + p.oslot.slot(k) * p.out_stride + static_cast<int64_t>(j) * p.B;
    __syncthreads();  // H staging / previous block done
    float4 *xs4 = reinterpret_cast<float4 *>(xs);
    for (int q2 = tid; 2 * q2 < p.B; q2 += kHxThreads) xs4[q2] = __ldg(src + q2);
    __syncthreads();
    if (NT == 1) {
      for (int r = g; r < R; r += RG) {
        float2 a = make_float2(0.f, 0.f);
        cmac(a, h[0], xs[r]);
        dst[r] = a;
      }
      continue;
    }
    // X[r][kk..kk+1] as one aligned float4 broadcast; two rows per pass
    int r = g;
    for (; r + RG < R; r += 2 * RG) {
      float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
      const float4 *x0 = reinterpret_cast<const float4 *>(xs + r * NT);
      const float4 *x1 = reinterpret_cast<const float4 *>(xs + (r + RG) * NT);
#pragma unroll
      for (int kk = 0; kk < NT; kk += 2) {
        const float4 u0 = x0[kk / 2], u1 = x1[kk / 2];
        cmac(a0, h[kk], make_float2(u0.x, u0.y));
        cmac(a1, h[kk], make_float2(u1.x, u1.y));
        cmac(a0, h[kk + 1], make_float2(u0.z, u0.w));
        cmac(a1, h[kk + 1], make_float2(u1.z, u1.w));
      }
      dst[r * NT + i] = a0;
      dst[(r + RG) * NT + i] = a1;
    }
    for (; r < R; r += RG) {
      float2 a0 = make_float2(0.f, 0.f);
      const float4 *x0 = reinterpret_cast<const float4 *>(xs + r * NT);
#pragma unroll
      for (int kk = 0; kk < NT; kk += 2) {
        const float4 u0 = x0[kk / 2];
        cmac(a0, h[kk], make_float2(u0.x, u0.y));
        cmac(a0, h[kk + 1], make_float2(u0.z, u0.w));
      }
      dst[r * NT + i] = a0;
    }
  }
}

// Any N (no register blocking): H in shared memory after the block.
static __global__ void __launch_bounds__(kHxThreads) hx_cuda_generic_kernel(HxParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2 *xs = reinterpret_cast<float2 *>(smem_raw);
  float2 *hs = xs + p.B;
  const int tid = threadIdx.x;
  const int N = p.N;
  for (int q = tid; q < N * N; q += kHxThreads) hs[q] = p.H[q];
  const int64_t total = static_cast<int64_t>(p.frames) * p.F;
  for (int64_t w = blockIdx.x; w < total; w += gridDim.x) {
    const int k = static_cast<int>(w / p.F), j = static_cast<int>(w % p.F);
    const int64_t rs = p.rslot.slot(k);
    const int ck = min(max(p.c[rs], 0), p.F);
    if (j == 0 && tid == 0 && p.ctr) hx_bookkeeping(p, k, ck);
    if (j >= ck) continue;
    const int b = p.idx[rs * p.F + j];
    if (b < 0 || b >= p.F) continue;
    const float2 *src = p.y + p.yslot.slot(k) * p.y_stride + static_cast<int64_t>(b) * p.B;
    float2 *dst = p.out + p.oslot.slot(k) * p.out_stride + static_cast<int64_t>(j) * p.B;
    __syncthreads();
    for (int q = tid; q < p.B; q += kHxThreads) xs[q] = src[q];
    __syncthreads();
    for (int q = tid; q < p.B; q += kHxThreads) {
      const int r = q / N, i = q % N;
      float2 a = make_float2(0.f, 0.f);
      for (int kk = 0; kk < N; ++kk) cmac(a, hs[i * N + kk], xs[r * N + kk]);
      dst[q] = a;
    }
  }
}

}  // namespace prune
