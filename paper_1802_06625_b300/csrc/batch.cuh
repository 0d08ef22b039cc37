// Batched firing: one frame of each of many independent graph instances
// (uneven F, T, tau, taps, H; common B and N) per step, in three launches
// over all instances: FIR (+ DET energies), DET + SEL, and HX_b (+ SINK).
// Instances are independent DPGs (Sec. V), so the batch is a union of
// graphs; every instance keeps its own delay token across steps.
#pragma once
#include <algorithm>

#include "batch_fir_tc.cuh"
#include "batch_types.cuh"
#include "detsel.cuh"
#include "fir.cuh"
#include "hx_tc.cuh"

namespace prune {

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

// HX_b on tcgen05 for N = 64: the single-instance tensor-core scheme (same
// split, same GEMM order, so the results are bit-identical to it) over the
// batch's work items (instance, 128-row tile of its selected rows), in a
// two-stage pipeline: the selected rows of the next item are gathered into
// the second operand buffer while the GEMMs of the current one run, and
// the current item's output leaves its tensor-memory accumulator while the
// next item's GEMMs run.  An instance's R operands are copied into shared
// memory when the instance of the work item changes (after the GEMMs that
// read the old ones have completed).
// Balanced mode (up to kBatchHxMaxInst instances): every CTA scans the
// instances' control tokens into a prefix of their selected tiles and fires
// an equal contiguous share of those tiles, so the load is even whatever
// the selections and R operands are reloaded only at instance boundaries.
// Larger batches take the work items by chunks or grid stride.
constexpr int kBatchHxMaxInst = 4096;
constexpr uint32_t kBatchHxSmemBytes = 6 * kTcOpBytes + 64 + 4 * (kBatchHxMaxInst + 1) + 1024;
// 2 x A (hi, lo), B (hi, lo), misc, tile prefix

struct BatchHxItem {
  int w, ii, tau, rows;  // w < 0: none
};

static __global__ void __launch_bounds__(kTcThreads, 1) batch_hx_tc_kernel(BatchParams bp) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char *base = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                          ~static_cast<uintptr_t>(1023));
  unsigned char *abuf = base;                                  // stage s: hi at s * 2 * kTcOpBytes, lo after
  unsigned char *b_hi = base + 4 * kTcOpBytes, *b_lo = base + 5 * kTcOpBytes;
  uint64_t *mbar = reinterpret_cast<uint64_t *>(base + 6 * kTcOpBytes);  // [2]
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(base + 6 * kTcOpBytes + 16);
  int32_t *s_flag = reinterpret_cast<int32_t *>(base + 6 * kTcOpBytes + 20);
  int32_t *wsum = reinterpret_cast<int32_t *>(base + 6 * kTcOpBytes + 24);  // [8]
  int32_t *pre = reinterpret_cast<int32_t *>(base + 6 * kTcOpBytes + 64);   // [n + 1] selected tiles before i
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int RB = bp.B / kTcNc;
  const bool balanced = bp.n <= kBatchHxMaxInst;
  if (tid == 0) {
    mbar_init(smem_u32(&mbar[0]), 1);
    mbar_init(smem_u32(&mbar[1]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *s_flag = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(256u)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  uint32_t ph[2] = {0u, 0u};
  bool pending[2] = {false, false};
  int loaded = -1;
  const int w1 = bp.hx_chunk > 0 ? min((blockIdx.x + 1) * bp.hx_chunk, bp.hx_items) : bp.hx_items;
  const int ws = bp.hx_chunk > 0 ? 1 : gridDim.x;
  int wn = bp.hx_chunk > 0 ? blockIdx.x * bp.hx_chunk : blockIdx.x;
  int64_t r_next = 0, r_end = 0;  // balanced mode: this CTA's selected tiles [r_next, r_end)
  int ib = 0;                     //   and the instance of r_next
  if (balanced) {
    // inclusive block scan of the selected tiles per instance, 256 at a time
    int carry = 0;
    for (int i0 = 0; i0 < bp.n; i0 += kTcThreads) {
      const int i = i0 + tid;
      int t = 0;
      if (i < bp.n) {
        const BatchInst &in = bp.inst[i];
        t = (min(max(*in.c, 0), in.F) * RB + kTcM - 1) / kTcM;
      }
      int x = t;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
      }
      if (lane == 31) wsum[warp] = x;
      __syncthreads();
      int before = carry, chunk = 0;
#pragma unroll
      for (int w = 0; w < kTcThreads / 32; ++w) {
        const int v = wsum[w];
        if (w < warp) before += v;
        chunk += v;
      }
      if (i < bp.n) pre[i + 1] = before + x;
      carry += chunk;
      __syncthreads();
    }
    if (tid == 0) pre[0] = 0;
    __syncthreads();
    const int64_t total = pre[bp.n];
    r_next = total * blockIdx.x / gridDim.x;
    r_end = total * (blockIdx.x + 1) / gridDim.x;
    int lo = 0, hi = bp.n;  // the instance i with pre[i] <= r_next < pre[i + 1]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (pre[mid] <= r_next) lo = mid;
      else hi = mid;
    }
    ib = lo;
  }
  // the next item with rows to fire (uniform: control tokens read on the device)
  auto next_item = [&]() -> BatchHxItem {
    if (balanced) {
      if (r_next >= r_end) return BatchHxItem{-1, 0, 0, 0};
      while (pre[ib + 1] <= r_next) ++ib;
      const BatchInst &in = bp.inst[ib];
      const BatchHxItem it{static_cast<int>(r_next), ib, static_cast<int>(r_next - pre[ib]),
                           min(max(*in.c, 0), in.F) * RB};
      ++r_next;
      return it;
    }
    for (; wn < w1; wn += ws) {
      const int ii = bp.hx_map[wn];
      const BatchInst &in = bp.inst[ii];
      const int tau = wn - in.hx_tile0;
      const int ck = min(max(*in.c, 0), in.F);
      const int rows = ck * RB;
      if (tau * kTcM < rows) {
        const BatchHxItem it{wn, ii, tau, rows};
        wn += ws;
        return it;
      }
    }
    return BatchHxItem{-1, 0, 0, 0};
  };
  // wait for the GEMMs of stage st (all threads, bounded)
  auto drain = [&](int st) -> bool {
    if (!pending[st]) return true;
    if (!mbar_wait_bounded(smem_u32(&mbar[st]), ph[st], bp.timeout_ns)) return false;
    ph[st] ^= 1u;
    pending[st] = false;
    return true;
  };
  auto load_b = [&](int ii) {
    const uint4 *src = reinterpret_cast<const uint4 *>(bp.inst[ii].bops);
    uint4 *dst = reinterpret_cast<uint4 *>(b_hi);
    for (int q = tid; q < static_cast<int>(2 * kTcOpBytes / 16); q += kTcThreads) dst[q] = src[q];
    loaded = ii;
  };
  // the selected rows of an item as the split-FP16 A operand of stage st:
  // every load of the thread is issued before the first split
  auto gather = [&](const BatchHxItem &it, int st) {
    const BatchInst &in = bp.inst[it.ii];
    unsigned char *a_hi = abuf + st * 2 * kTcOpBytes, *a_lo = a_hi + kTcOpBytes;
    constexpr int kPer = kTcM * (kTcK / 8) / kTcThreads;  // 8 pieces of 8 floats
    float4 u[kPer][2];
#pragma unroll
    for (int n = 0; n < kPer; ++n) {
      const int q = tid + n * kTcThreads;
      const int m = q >> 4, cc = q & 15;
      const int gr = it.tau * kTcM + m;
      u[n][0] = make_float4(0.f, 0.f, 0.f, 0.f);
      u[n][1] = u[n][0];
      if (gr < it.rows) {
        const int j = gr / RB, r = gr % RB;
        const int b = in.idx[j];
        if (b >= 0 && b < in.F) {
          const float4 *src =
              reinterpret_cast<const float4 *>(in.y + static_cast<int64_t>(b) * bp.B + r * kTcNc) + cc * 2;
          u[n][0] = __ldg(src);
          u[n][1] = __ldg(src + 1);
        }
      }
    }
#pragma unroll
    for (int n = 0; n < kPer; ++n) {
      const int q = tid + n * kTcThreads;
      const int m = q >> 4, cc = q & 15;
      const float v[8] = {u[n][0].x, u[n][0].y, u[n][0].z, u[n][0].w, u[n][1].x, u[n][1].y, u[n][1].z, u[n][1].w};
      const uint32_t off = sw128_off(m, cc * 8, kTcM);
      *reinterpret_cast<uint4 *>(a_hi + off) = split_pack(v, false);
      *reinterpret_cast<uint4 *>(a_lo + off) = split_pack(v, true);
    }
  };
  auto issue = [&](int st) {  // thread 0: 3 passes x 8 K steps into accumulator st
    tc_fence_after();
    const uint32_t ah = smem_u32(abuf + st * 2 * kTcOpBytes), al = ah + kTcOpBytes;
    const uint32_t bh = smem_u32(b_hi), bl = smem_u32(b_lo);
    const uint32_t pa[3] = {ah, ah, al}, pb[3] = {bh, bl, bh};
    const uint32_t d = tmem + static_cast<uint32_t>(st * 128);
#pragma unroll
    for (int pass = 0; pass < 3; ++pass)
#pragma unroll
      for (int ks = 0; ks < kTcK / 16; ++ks) {
        const uint32_t koff = static_cast<uint32_t>((ks >> 2) * kTcM * 128 + (ks & 3) * 32);
        const uint32_t kboff = static_cast<uint32_t>((ks >> 2) * kTcNg * 128 + (ks & 3) * 32);
        umma_f16(d, umma_desc_sw128(pa[pass] + koff), umma_desc_sw128(pb[pass] + kboff), kTcIdesc,
                 (pass > 0 || ks > 0) ? 1u : 0u);
      }
    umma_commit(smem_u32(&mbar[st]));
  };
  // the item's output rows are consecutive in the compacted output: stage
  // them row-major in the free operand buffer of stage st (16-byte chunks
  // XOR-swizzled by row, so the row-per-thread stores hit every bank once
  // per quarter warp), then copy the tile out with coalesced stores
  auto epilogue = [&](const BatchHxItem &it, int st) {
    const BatchInst &in = bp.inst[it.ii];
    unsigned char *stg = abuf + st * 2 * kTcOpBytes;  // 128 rows x 512 bytes
    const int qd = warp & 3, hf = warp >> 2;
    const int m = qd * 32 + lane;
    float v[64];
#pragma unroll
    for (int c4 = 0; c4 < 4; ++c4) {
      float t[16];
      tmem_ld16(tmem + (static_cast<uint32_t>(qd * 32) << 16) + static_cast<uint32_t>(st * 128 + hf * 64 + c4 * 16), t);
#pragma unroll
      for (int e = 0; e < 16; ++e) v[c4 * 16 + e] = t[e];
    }
    tmem_ld_wait();
    const float sc = 1.f / kTcBScale;
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const int c = hf * 16 + e;  // 16-byte chunk of row m
      *reinterpret_cast<float4 *>(stg + m * 512 + ((c ^ (m & 31)) << 4)) =
          make_float4(v[4 * e] * sc, v[4 * e + 1] * sc, v[4 * e + 2] * sc, v[4 * e + 3] * sc);
    }
    __syncthreads();
    const int nrows = min(kTcM, it.rows - it.tau * kTcM);
    float4 *dst = reinterpret_cast<float4 *>(in.out + static_cast<int64_t>(it.tau) * kTcM * kTcNc);
    for (int g = tid; g < nrows * 32; g += kTcThreads) {
      const int mm = g >> 5, c = g & 31;
      dst[g] = *reinterpret_cast<const float4 *>(stg + mm * 512 + ((c ^ (mm & 31)) << 4));
    }
  };

  BatchHxItem cur = next_item();
  int st = 0;
  if (cur.w >= 0) {
    load_b(cur.ii);
    gather(cur, 0);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    if (tid == 0) issue(0);
    pending[0] = true;
  }
  while (cur.w >= 0) {
    const BatchHxItem nxt = next_item();
    bool ok = true;
    if (nxt.w >= 0) {
      if (nxt.ii != loaded) {  // new R operands once the current GEMMs no longer read them
        ok = drain(st);
        __syncthreads();
        if (ok) load_b(nxt.ii);
      }
      if (ok) gather(nxt, st ^ 1);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (ok) ok = drain(st);
    if (!ok) {
      if (tid == 0) report_error(bp.status, kDevTimeout, kActHx, 7, static_cast<uint64_t>(cur.ii));
      *s_flag = 1;
    }
    tc_fence_before();
    __syncthreads();
    if (*s_flag) break;
    if (nxt.w >= 0) {
      if (tid == 0) issue(st ^ 1);
      pending[st ^ 1] = true;
    }
    tc_fence_after();
    epilogue(cur, st);  // overlaps the next item's GEMMs
    tc_fence_before();
    __syncthreads();
    cur = nxt;
    st ^= 1;
  }
  drain(0);
  drain(1);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256u) : "memory");
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
  if (bp.fir_tc)  // one persistent CTA per SM over equal shares of the tiles
    batch_fir_tc_kernel<<<std::max(1, std::min(sms, bp.fir_tiles)), kBfThreads, kBfSmemBytes, stream>>>(bp);
  else
    batch_fir_kernel<<<bp.fir_tiles, kFirThreads, fir_smem_bytes(tp_max), stream>>>(bp, tp_max);
  batch_detsel_kernel<<<bp.n, kDetThreads, 0, stream>>>(bp);
  const int wave = bp.N == kTcNc ? sms : sms * 8;
  const int want = bp.hx_chunk > 0 ? (bp.hx_items + bp.hx_chunk - 1) / bp.hx_chunk : (hx_grid > 0 ? hx_grid : wave);
  if (bp.N == kTcNc) {
    // balanced mode: one persistent CTA per SM over the selected tiles
    const int grid = bp.n <= kBatchHxMaxInst ? std::max(1, sms) : std::max(1, std::min(bp.hx_items, want));
    batch_hx_tc_kernel<<<grid, kTcThreads, kBatchHxSmemBytes, stream>>>(bp);
  } else {
    const int grid = std::max(1, std::min(bp.hx_items, want));
    const size_t smem = (static_cast<size_t>(bp.B) + static_cast<size_t>(bp.N) * bp.N) * sizeof(float2);
    batch_hx_cuda_kernel<<<grid, kHxThreads, smem, stream>>>(bp);
  }
  return cudaGetLastError();
}

// Opt the step kernels of this translation unit into the dynamic shared
// memory that taps of up to tp_max (padded), the given B, N and the
// tensor-core FIR (fir_tc) need.
static inline bool batch_enable_smem(int tp_max, int B, int N, bool fir_tc = false) {
  bool ok = true;
  if (fir_tc)
    ok = cudaFuncSetAttribute(batch_fir_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              static_cast<int>(kBfSmemBytes)) == cudaSuccess;
  if (fir_smem_bytes(tp_max) > 48 * 1024)
    ok = cudaFuncSetAttribute(batch_fir_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              static_cast<int>(fir_smem_bytes(tp_max))) == cudaSuccess;
  if (ok && N == kTcNc)
    ok = cudaFuncSetAttribute(batch_hx_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              static_cast<int>(kBatchHxSmemBytes)) == cudaSuccess;
  if (ok && N != kTcNc) {
    const size_t smem = (static_cast<size_t>(B) + static_cast<size_t>(N) * N) * sizeof(float2);
    if (smem > 48 * 1024)
      ok = cudaFuncSetAttribute(batch_hx_cuda_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(smem)) == cudaSuccess;
  }
  return ok;
}

}  // namespace prune
