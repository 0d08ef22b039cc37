// Batched firing: one frame of each of many independent graph instances
// (uneven F, T, tau, taps, H; common B and N) per step, in three launches
// over all instances: FIR (+ DET energies), DET + SEL, and HX_b (+ SINK).
// Instances are independent DPGs (Sec. V), so the batch is a union of
// graphs; every instance keeps its own delay token across steps.
#pragma once
#include <algorithm>

#include "detsel.cuh"
#include "fir.cuh"
#include "hx_tc.cuh"

namespace prune {

struct BatchInst {
  int64_t x_off;          // offset of this instance's frame in the step's input (samples)
  const float2 *x;        // or, when not null, the frame itself (request-loop entries)
  const float2 *taps;     // T taps
  const float2 *H;        // N x N
  const uint16_t *bops;   // tensor-core HX operands (N = 64) or nullptr
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
};

struct BatchParams {
  const BatchInst *inst;
  const int2 *fir_map;      // FIR CTA -> (instance, tile of the instance), in launch order
  const int32_t *hx_map;    // HX work item -> instance (an instance's items are consecutive)
  const float2 *x;          // step input, all instances back to back
  int32_t n, B, N, TS, parity, fir_tiles, hx_items;
  int32_t hx_chunk;         // > 0: CTA c fires items [c * hx_chunk, (c + 1) * hx_chunk); 0: grid-stride
  uint64_t timeout_ns;
  uint32_t *status;
};

// FIR + energies: one CTA per (instance, tile).  The same device functions as
// the single-instance kernel, so both paths compute identical energies.
static __global__ void __launch_bounds__(kFirThreads) batch_fir_kernel(BatchParams bp, int32_t tp_max) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int2 tm = bp.fir_map[blockIdx.x];
  const int ii = tm.x;
  const BatchInst in = bp.inst[ii];
  const int TP = in.TP;
  float2 *xs = reinterpret_cast<float2 *>(smem_raw);
  float2 *hs = xs + fir_window_slots(tp_max);
  float *red = reinterpret_cast<float *>(hs + tp_max);
  float *Et = red + 32;
  const int tid = threadIdx.x;
  const int64_t L = static_cast<int64_t>(in.F) * bp.B;
  const int64_t s0 = static_cast<int64_t>(tm.y) * bp.TS;
  const int nv = static_cast<int>(min(static_cast<int64_t>(bp.TS), L - s0));
  const float2 *cur = in.x ? in.x : bp.x + in.x_off;
  const float2 *hist = in.T <= 1 ? nullptr : in.hist ? in.hist + bp.parity * (in.T - 1) : in.hist_in;
  float2 *hout = in.T <= 1 ? nullptr : in.hist ? in.hist + (1 - bp.parity) * (in.T - 1) : in.hist_out;
  for (int t = tid; t < TP; t += kFirThreads) hs[t] = t < in.T ? in.taps[t] : make_float2(0.f, 0.f);
  fir_stage_window(xs, cur, nullptr, hist, L, in.T, TP, s0, nv, tid);
  __syncthreads();
  float2 acc[kSPT];
  fir_compute(xs, hs, TP, tid, acc);
  fir_block_energies(acc, bp.B, nv, tid, red, Et);
  if (tid < nv / bp.B) in.energy[s0 / bp.B + tid] = Et[tid];
  if (hout && s0 + nv == L) {  // next delay token: the last T-1 input samples
    for (int m = tid; m < in.T - 1; m += kFirThreads) hout[m] = xs[pad_idx(TP - 1 + nv - (in.T - 1) + m)];
  }
  __syncthreads();
  float2 *ys = xs;
  const int obase = tid * kSPT;
#pragma unroll
  for (int j = 0; j < kSPT; ++j) ys[pad_idx(obase + j)] = acc[j];
  __syncthreads();
  float4 *out = reinterpret_cast<float4 *>(in.y + s0);
  for (int q2 = tid; 2 * q2 < nv; q2 += kFirThreads) {
    const float2 a = ys[pad_idx(2 * q2)], b = ys[pad_idx(2 * q2 + 1)];
    out[q2] = make_float4(a.x, a.y, b.x, b.y);
  }
}

// DET + SEL: one CTA per instance (ballot, warp scan, stable scatter).
static __global__ void __launch_bounds__(kDetThreads) batch_detsel_kernel(BatchParams bp) {
  __shared__ int warp_off[32];
  __shared__ int total_s;
  const BatchInst in = bp.inst[blockIdx.x];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int running = 0;
  for (int r0 = 0; r0 < in.F; r0 += kDetThreads) {
    const int b = r0 + tid;
    const bool v = (b < in.F) && (in.energy[b] > in.tau);
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
    if (v) in.idx[running + warp_off[warp] + rank] = b;
    running += total_s;
    __syncthreads();
  }
  if (tid == 0) *in.c = running;
}

// HX_b on CUDA cores for any N < 64: grid-stride over (instance, block j),
// H of the instance in shared memory, the control token read on the device.
static __global__ void __launch_bounds__(kHxThreads) batch_hx_cuda_kernel(BatchParams bp) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2 *xs = reinterpret_cast<float2 *>(smem_raw);
  float2 *hs = xs + bp.B;
  const int tid = threadIdx.x, N = bp.N;
  int loaded = -1;
  const int w0 = bp.hx_chunk > 0 ? blockIdx.x * bp.hx_chunk : blockIdx.x;
  const int w1 = bp.hx_chunk > 0 ? min(w0 + bp.hx_chunk, bp.hx_items) : bp.hx_items;
  const int ws = bp.hx_chunk > 0 ? 1 : gridDim.x;
  for (int w = w0; w < w1; w += ws) {
    const int ii = bp.hx_map[w];
    const BatchInst &in = bp.inst[ii];
    const int j = w - in.hx_tile0;
    const int ck = min(max(*in.c, 0), in.F);
    if (j >= ck) continue;
    const int b = in.idx[j];
    if (b < 0 || b >= in.F) continue;
    __syncthreads();
    if (ii != loaded) {
      for (int q = tid; q < N * N; q += kHxThreads) hs[q] = in.H[q];
      loaded = ii;
    }
    const float2 *src = in.y + static_cast<int64_t>(b) * bp.B;
    for (int q = tid; q < bp.B; q += kHxThreads) xs[q] = src[q];
    __syncthreads();
    float2 *dst = in.out + static_cast<int64_t>(j) * bp.B;
    for (int q = tid; q < bp.B; q += kHxThreads) {
      const int r = q / N, i = q % N;
      float2 a = make_float2(0.f, 0.f);
      for (int kk = 0; kk < N; ++kk) cmac(a, hs[i * N + kk], xs[r * N + kk]);
      dst[q] = a;
    }
  }
}

// HX_b on tcgen05 for N = 64: the single-instance tensor-core scheme over
// the batch's work items (instance, 128-row tile of its selected rows); an
// instance's R operands are copied into shared memory when the instance of
// the work item changes.
static __global__ void __launch_bounds__(kTcThreads, 1) batch_hx_tc_kernel(BatchParams bp) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char *base = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                          ~static_cast<uintptr_t>(1023));
  unsigned char *a_hi = base, *a_lo = base + kTcOpBytes;
  unsigned char *b_hi = base + 2 * kTcOpBytes, *b_lo = base + 3 * kTcOpBytes;
  uint64_t *mbar = reinterpret_cast<uint64_t *>(base + 4 * kTcOpBytes);
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(base + 4 * kTcOpBytes + 8);
  int32_t *s_flag = reinterpret_cast<int32_t *>(base + 4 * kTcOpBytes + 16);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int RB = bp.B / kTcNc;
  if (tid == 0) {
    mbar_init(smem_u32(mbar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *s_flag = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(128u)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  uint32_t phase = 0;
  bool pending = false;
  int loaded = -1;
  const int w0 = bp.hx_chunk > 0 ? blockIdx.x * bp.hx_chunk : blockIdx.x;
  const int w1 = bp.hx_chunk > 0 ? min(w0 + bp.hx_chunk, bp.hx_items) : bp.hx_items;
  const int ws = bp.hx_chunk > 0 ? 1 : gridDim.x;
  for (int w = w0; w < w1; w += ws) {
    const int ii = bp.hx_map[w];
    const BatchInst &in = bp.inst[ii];
    const int tau = w - in.hx_tile0;
    const int ck = min(max(*in.c, 0), in.F);
    const int rows = ck * RB;
    if (tau * kTcM >= rows) continue;  // uniform: control token read on the device
    if (ii != loaded) {                // this instance's R operands
      const uint4 *src = reinterpret_cast<const uint4 *>(in.bops);
      uint4 *dst = reinterpret_cast<uint4 *>(b_hi);
      for (int q = tid; q < static_cast<int>(2 * kTcOpBytes / 16); q += kTcThreads) dst[q] = src[q];
      loaded = ii;
    }
    for (int q = tid; q < kTcM * (kTcK / 8); q += kTcThreads) {
      const int m = q >> 4, cc = q & 15;
      const int gr = tau * kTcM + m;
      float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      if (gr < rows) {
        const int j = gr / RB, r = gr % RB;
        const int b = in.idx[j];
        if (b >= 0 && b < in.F) {
          const float4 *src =
              reinterpret_cast<const float4 *>(in.y + static_cast<int64_t>(b) * bp.B + r * kTcNc) + cc * 2;
          const float4 u0 = __ldg(src), u1 = __ldg(src + 1);
          v[0] = u0.x; v[1] = u0.y; v[2] = u0.z; v[3] = u0.w;
          v[4] = u1.x; v[5] = u1.y; v[6] = u1.z; v[7] = u1.w;
        }
      }
      const uint32_t off = sw128_off(m, cc * 8, kTcM);
      *reinterpret_cast<uint4 *>(a_hi + off) = split_pack(v, false);
      *reinterpret_cast<uint4 *>(a_lo + off) = split_pack(v, true);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t ah = smem_u32(a_hi), al = smem_u32(a_lo), bh = smem_u32(b_hi), bl = smem_u32(b_lo);
      const uint32_t pa[3] = {ah, ah, al}, pb[3] = {bh, bl, bh};
#pragma unroll
      for (int pass = 0; pass < 3; ++pass)
#pragma unroll
        for (int ks = 0; ks < kTcK / 16; ++ks) {
          const uint32_t koff = static_cast<uint32_t>((ks >> 2) * kTcM * 128 + (ks & 3) * 32);
          const uint32_t kboff = static_cast<uint32_t>((ks >> 2) * kTcNg * 128 + (ks & 3) * 32);
          umma_f16(tmem, umma_desc_sw128(pa[pass] + koff), umma_desc_sw128(pb[pass] + kboff), kTcIdesc,
                   (pass > 0 || ks > 0) ? 1u : 0u);
        }
      umma_commit(smem_u32(mbar));
    }
    pending = true;
    if (mbar_wait_bounded(smem_u32(mbar), phase, bp.timeout_ns)) {
      phase ^= 1u;
      pending = false;
    } else {
      if (tid == 0) report_error(bp.status, kDevTimeout, kActHx, 7, static_cast<uint64_t>(ii));
      *s_flag = 1;
    }
    __syncthreads();
    if (*s_flag) break;
    tc_fence_after();
    {
      const int qd = warp & 3, hf = warp >> 2;
      const int m = qd * 32 + lane;
      const int gr = tau * kTcM + m;
      float v[64];
#pragma unroll
      for (int c4 = 0; c4 < 4; ++c4) {
        float t[16];
        tmem_ld16(tmem + (static_cast<uint32_t>(qd * 32) << 16) + static_cast<uint32_t>(hf * 64 + c4 * 16), t);
#pragma unroll
        for (int e = 0; e < 16; ++e) v[c4 * 16 + e] = t[e];
      }
      tmem_ld_wait();
      if (gr < rows) {
        const int j = gr / RB, r = gr % RB;
        float4 *dst = reinterpret_cast<float4 *>(in.out + static_cast<int64_t>(j) * bp.B + r * kTcNc + hf * 32);
        const float s = 1.f / kTcBScale;
#pragma unroll
        for (int e = 0; e < 16; ++e)
          dst[e] = make_float4(v[4 * e] * s, v[4 * e + 1] * s, v[4 * e + 2] * s, v[4 * e + 3] * s);
      }
    }
    tc_fence_before();
    __syncthreads();
  }
  if (pending) mbar_wait_bounded(smem_u32(mbar), phase, bp.timeout_ns);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128u) : "memory");
  }
}

// The three launches of one step over the instances of `bp` (the batch and
// the request loop share them).  Dynamic shared memory above 48 KB must have
// been enabled on these kernels in the calling translation unit
// (batch_enable_smem).
// hx_grid: CTAs of the HX launch (0: one wave, sms for tensor cores, 8 sms
// for CUDA cores); with bp.hx_chunk > 0 the grid covers the items in chunks.
static inline cudaError_t batch_launch_step(const BatchParams &bp, int tp_max, int sms, cudaStream_t stream,
                                            int hx_grid = 0) {
  batch_fir_kernel<<<bp.fir_tiles, kFirThreads, fir_smem_bytes(tp_max), stream>>>(bp, tp_max);
  batch_detsel_kernel<<<bp.n, kDetThreads, 0, stream>>>(bp);
  const int wave = bp.N == kTcNc ? sms : sms * 8;
  const int want = bp.hx_chunk > 0 ? (bp.hx_items + bp.hx_chunk - 1) / bp.hx_chunk : (hx_grid > 0 ? hx_grid : wave);
  if (bp.N == kTcNc) {
    const int grid = std::max(1, std::min(bp.hx_items, want));
    batch_hx_tc_kernel<<<grid, kTcThreads, kTcSmemBytes, stream>>>(bp);
  } else {
    const int grid = std::max(1, std::min(bp.hx_items, want));
    const size_t smem = (static_cast<size_t>(bp.B) + static_cast<size_t>(bp.N) * bp.N) * sizeof(float2);
    batch_hx_cuda_kernel<<<grid, kHxThreads, smem, stream>>>(bp);
  }
  return cudaGetLastError();
}

// Opt the step kernels of this translation unit into the dynamic shared
// memory that taps of up to tp_max (padded) and the given B, N need.
static inline bool batch_enable_smem(int tp_max, int B, int N) {
  bool ok = true;
  if (fir_smem_bytes(tp_max) > 48 * 1024)
    ok = cudaFuncSetAttribute(batch_fir_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              static_cast<int>(fir_smem_bytes(tp_max))) == cudaSuccess;
  if (ok && N == kTcNc)
    ok = cudaFuncSetAttribute(batch_hx_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              static_cast<int>(kTcSmemBytes)) == cudaSuccess;
  if (ok && N != kTcNc) {
    const size_t smem = (static_cast<size_t>(B) + static_cast<size_t>(N) * N) * sizeof(float2);
    if (smem > 48 * 1024)
      ok = cudaFuncSetAttribute(batch_hx_cuda_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(smem)) == cudaSuccess;
  }
  return ok;
}

}  // namespace prune
