// Batched firing: one frame of each of many independent graph instances
// (uneven F, T, tau, taps, H; common B and N) per step, in three launches
// over all instances: FIR (+ DET energies), DET + SEL, and HX_b (+ SINK).
// Instances are independent DPGs (Sec. V), so the batch is a union of
// graphs; every instance keeps its own delay token across steps.
#pragma once
#include <type_traits>
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
  if (!bp.hx_pre) return;
  // The last CTA to finish scans the instances' selected 128-row tiles into
  // hx_pre, the work list of the tensor-core HX launch.
  __shared__ int last;
  if (tid == 0) {
    __threadfence();
    last = atomicAdd(bp.hx_ctr, 1u) == static_cast<uint32_t>(bp.n - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  const int RB = bp.B / kTcNc;
  int carry = 0;
  for (int i0 = 0; i0 < bp.n; i0 += kDetThreads) {
    const int i = i0 + tid;
    int t = 0;
    if (i < bp.n) {
      const BatchInst &ii = bp.inst[i];
      t = (min(max(__ldcg(ii.c), 0), ii.F) * RB + kTcM - 1) / kTcM;
    }
    int x = t;
    for (int off = 1; off < 32; off <<= 1) {
      const int o = __shfl_up_sync(0xffffffffu, x, off);
      if (lane >= off) x += o;
    }
    if (lane == 31) warp_off[warp] = x;
    __syncthreads();
    int before = carry, chunk = 0;
    for (int w = 0; w < kDetThreads / 32; ++w) {
      const int v = warp_off[w];
      if (w < warp) before += v;
      chunk += v;
    }
    if (i < bp.n) bp.hx_pre[i + 1] = before + x;
    carry += chunk;
    __syncthreads();
  }
  if (tid == 0) {
    bp.hx_pre[0] = 0;
    *bp.hx_ctr = 0u;  // for the next step
  }
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
// selected 128-row tiles of the batch.  DET/SEL left the prefix of the
// instances' selected tiles in hx_pre; CTA c fires an equal contiguous
// share of them, so the load is even whatever the selections, and an
// instance's R operands are reloaded only at its boundaries.
//   warp 9      producer: per tile, the selected blocks' rows (contiguous
//               in the FIR output, B * 8 bytes a block) by bulk copies into
//               one of 2 stages of 64 KB;
//   warps 0-7   the rows, read into registers, written back over the stage
//               as the split-FP16 A operand (same size); then the previous
//               tile's accumulator is written to the compacted output;
//   warp 8      issues the 24 GEMMs of a tile into one of two 128-column
//               accumulators; their completion frees the stage.
// Every wait is bounded; warps 0-7 combine wait outcomes in a barrier with
// an AND reduction; the issuer commits once more and waits before tensor
// memory is freed.
constexpr int kBhxThreads = 320;
constexpr uint32_t kBhxStageBytes = 2 * kTcOpBytes;                      // 64 KB: 128 rows x 512 bytes
constexpr uint32_t kBhxXposeBytes = 8 * 2048;                            // 2 KB per work warp
constexpr uint32_t kBhxMiscBytes = 2048;
constexpr uint32_t kBatchHxSmemBytes = 2 * kTcOpBytes + 2 * kBhxStageBytes + kBhxMiscBytes + kBhxXposeBytes + 1024;
// B, stages, misc (barriers, records, row exponents), transpose buffers, alignment

struct BhxRec {
  float2 *out;        // the tile's first output row
  int32_t inst, nrows, s_h, pad;  // s_h: the instance's R exponent
};

static __global__ void __launch_bounds__(kBhxThreads, 1) batch_hx_tc_kernel(BatchParams bp) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char *base = smem_align1024(smem_raw);
  unsigned char *b_hi = base, *b_lo = base + kTcOpBytes;
  unsigned char *stage0 = base + 2 * kTcOpBytes;  // stage k: rows (fp32), then in place A hi | A lo
  unsigned char *misc = stage0 + 2 * kBhxStageBytes;
  uint64_t *raw_full = reinterpret_cast<uint64_t *>(misc);  // [2] rows landed (and the record)
  uint64_t *a_full = raw_full + 2;                           // [2] A operand written
  uint64_t *st_free = a_full + 2;                            // [2] the GEMMs reading the stage completed
  uint64_t *mma_done = st_free + 2;                          // [2] GEMMs into accumulator a completed
  uint64_t *acc_empty = mma_done + 2;                        // [2] accumulator a read back
  uint64_t *fin = acc_empty + 2;                             // the issuer's last commit, at exit
  uint64_t *b_full = fin + 1;                                // an instance's R operands landed
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(misc + 128);
  volatile int32_t *stop = reinterpret_cast<volatile int32_t *>(misc + 132);
  BhxRec *rec = reinterpret_cast<BhxRec *>(misc + 256);      // [2]
  int32_t *s_tile = reinterpret_cast<int32_t *>(misc + 1024); // [2] the tile's exponent per stage
  uint32_t *cred = reinterpret_cast<uint32_t *>(misc + 1088); // [2 stages][2][8] work warps' maxima
  float *xpose = reinterpret_cast<float *>(misc + kBhxMiscBytes);  // [8 warps][32 rows][16 floats]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int RB = bp.B / kTcNc;                                // rows per block
  // this CTA's selected tiles [r0, r0 + cnt) of the step
  const int total = __ldcg(&bp.hx_pre[bp.n]);
  const int r0 = static_cast<int>(static_cast<int64_t>(total) * blockIdx.x / gridDim.x);
  const int cnt = static_cast<int>(static_cast<int64_t>(total) * (blockIdx.x + 1) / gridDim.x) - r0;

  if (tid == 0) {
    for (int q = 0; q < 12; ++q) mbar_init(smem_u32(raw_full + q), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *stop = 0;
  }
  if (warp == 8) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(256u)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  auto fail = [&](uint32_t where) {
    if (!*stop) report_error(bp.status, kDevTimeout, kActHx, where, 0);
    *stop = 1;
  };

  if (warp == 9) {
    // ================================================================ producer
    int ib = 0;  // instance of tile r: hx_pre[ib] <= r < hx_pre[ib + 1]
    if (cnt > 0) {
      int lo = 0, hi = bp.n;
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldcg(&bp.hx_pre[mid]) <= r0) lo = mid;
        else hi = mid;
      }
      ib = lo;
    }
    int issued = 0;
    for (int i = 0; i < cnt; ++i) {
      const int st = i & 1;
      if (i >= 2 && !__all_sync(0xffffffffu, ws_wait(smem_u32(&st_free[st]), ((i >> 1) - 1) & 1, bp.timeout_ns, stop))) {
        if (lane == 0) fail(24);
        break;
      }
      const int r = r0 + i;
      while (ib + 1 < bp.n && __ldcg(&bp.hx_pre[ib + 1]) <= r) ++ib;
      const BatchInst &in = bp.inst[ib];
      const int tau = r - __ldcg(&bp.hx_pre[ib]);
      const int rows = min(max(__ldcg(in.c), 0), in.F) * RB;
      const int nrows = max(0, min(kTcM, rows - tau * kTcM));  // 0 only if the prefix disagrees with c
      const int nblk = nrows / RB, j0 = tau * kTcM / RB;
      unsigned char *stg = stage0 + st * kBhxStageBytes;
      if (lane == 0) {
        rec[st] = BhxRec{in.out + static_cast<int64_t>(tau) * kTcM * kTcNc, ib, nrows, in.s_h, 0};
        mbar_arrive_tx(smem_u32(&raw_full[st]), static_cast<uint32_t>(nblk) * bp.B * 8);
      }
      __syncwarp();
      for (int q = lane; q < nblk; q += 32) {  // block j0 + q: RB rows of the FIR output
        const int b = min(max(in.idx[j0 + q], 0), in.F - 1);
        bulk_g2s(smem_u32(stg + static_cast<uint32_t>(q) * bp.B * 8), in.y + static_cast<int64_t>(b) * bp.B,
                 static_cast<uint32_t>(bp.B) * 8, smem_u32(&raw_full[st]));
      }
      ++issued;
    }
    // no copy may still write a stage when the CTA leaves
    if (lane == 0)
      for (int i = max(0, issued - 2); i < issued; ++i)
        mbar_wait_bounded(smem_u32(&raw_full[i & 1]), (i >> 1) & 1, bp.timeout_ns);
    __syncwarp();
  } else if (warp == 8) {
    // ================================================================ MMA
    if (lane == 0) {
      bool any = false;
      for (int i = 0; i < cnt; ++i) {
        const int st = i & 1;
        if (!ws_wait(smem_u32(&a_full[st]), (i >> 1) & 1, bp.timeout_ns, stop)) {
          fail(25);
          break;
        }
        if (i >= 2 && !ws_wait(smem_u32(&acc_empty[st]), ((i >> 1) - 1) & 1, bp.timeout_ns, stop)) {
          fail(26);
          break;
        }
        tc_fence_after();
        const uint32_t ah = smem_u32(stage0 + st * kBhxStageBytes), al = ah + kTcOpBytes;
        const uint32_t bh = smem_u32(b_hi), bl = smem_u32(b_lo);
        const uint32_t d = tmem + static_cast<uint32_t>(st * 128);
#pragma unroll 1
        for (int pass = 0; pass < 3; ++pass) {
          const uint32_t pa = pass == 2 ? al : ah, pb = pass == 1 ? bl : bh;
#pragma unroll
          for (int ks = 0; ks < kTcK / 16; ++ks) {
            const uint32_t koff = static_cast<uint32_t>((ks >> 2) * kTcM * 128 + (ks & 3) * 32);
            const uint32_t kboff = static_cast<uint32_t>((ks >> 2) * kTcNg * 128 + (ks & 3) * 32);
            umma_f16(d, umma_desc_sw128(pa + koff), umma_desc_sw128(pb + kboff), kTcIdesc,
                     (pass > 0 || ks > 0) ? 1u : 0u);
          }
        }
        umma_commit(smem_u32(&mma_done[st]));
        umma_commit(smem_u32(&st_free[st]));
        any = true;
      }
      if (any) {  // every GEMM this thread issued has completed
        umma_commit(smem_u32(fin));
        mbar_wait_bounded(smem_u32(fin), 0u, bp.timeout_ns);
      }
    }
    __syncwarp();
  } else {
    // ================================================================ warps 0-7
    int loaded = -1;
    uint32_t b_par = 0;
    bool reload_open = false;  // an R copy issued and not yet seen to land
    int sx_pred = 0;           // scale exponent of the previous tile
    auto wait_all = [&](uint64_t *mb, uint32_t par) -> bool {
      const bool w = mbar_wait_bounded(smem_u32(mb), par, bp.timeout_ns);
      return bf_bar_and(w && !*stop);
    };
    auto epilogue = [&](int ip, const BhxRec &r) {  // accumulator of tile ip to the compacted output
      const int a = ip & 1;
      const int qd = warp & 3, hf = warp >> 2;
      float v[64];
#pragma unroll
      for (int c4 = 0; c4 < 4; ++c4) {
        float t[16];
        tmem_ld16(tmem + (static_cast<uint32_t>(qd * 32) << 16) + static_cast<uint32_t>(a * 128 + hf * 64 + c4 * 16), t);
#pragma unroll
        for (int e = 0; e < 16; ++e) v[c4 * 16 + e] = t[e];
      }
      tmem_ld_wait();
      // through a per-warp transpose, 64 bytes of each row per round: a
      // store instruction writes 8 rows x 64 contiguous bytes.  Chunk f of
      // row x sits at chunk f ^ ((x >> 1) & 3): conflict-free both ways.
      float *wx = xpose + warp * 512;
      float f1, f2;  // the tile's outputs times 2^-(s_tile + s_h)
      pow2_pair(-(s_tile[a] + r.s_h), f1, f2);
      if (f2 != 1.f) {  // a scale beyond one float factor (uniform, rare)
#pragma unroll
        for (int e = 0; e < 64; ++e) v[e] *= f2;
      }
#pragma unroll
      for (int h4 = 0; h4 < 4; ++h4) {
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          const float *vv = v + 16 * h4 + 4 * f;
          *reinterpret_cast<float4 *>(wx + lane * 16 + ((f ^ ((lane >> 1) & 3)) << 2)) =
              make_float4(vv[0] * f1, vv[1] * f1, vv[2] * f1, vv[3] * f1);
        }
        __syncwarp();
#pragma unroll
        for (int e4 = 0; e4 < 4; ++e4) {
          const int x = 8 * e4 + (lane >> 2), fq = lane & 3;  // row of the warp, 16-byte chunk
          const float4 val = *reinterpret_cast<const float4 *>(wx + x * 16 + ((fq ^ ((x >> 1) & 3)) << 2));
          const int mx = qd * 32 + x;
          if (mx < r.nrows)
            *reinterpret_cast<float4 *>(r.out + static_cast<int64_t>(mx) * kTcNc + hf * 32 + 8 * h4 + 2 * fq) = val;
        }
        __syncwarp();
      }
      tc_fence_before();
      bf_bar();
      if (tid == 0) mbar_arrive(smem_u32(&acc_empty[a]));
    };
    bool ok = true;
    BhxRec prev{};
    for (int i = 0; i < cnt; ++i) {
      const int st = i & 1;
      ok = wait_all(&raw_full[st], (i >> 1) & 1);
      if (!ok) break;
      const BhxRec r = rec[st];
      bool prev_done = i == 0;  // the GEMMs of tile i-1 have completed
      const bool reload = r.inst != loaded;
      if (reload) {  // this instance's R operands by bulk copy, once no GEMM reads the old ones
        if (!prev_done) {
          ok = wait_all(&mma_done[(i - 1) & 1], ((i - 1) >> 1) & 1);
          if (!ok) break;
          prev_done = true;
        }
        if (tid == 0) {
          const uint16_t *src = bp.inst[r.inst].bops;
          mbar_arrive_tx(smem_u32(b_full), 2 * kTcOpBytes);
          bulk_g2s(smem_u32(b_hi), src, kTcOpBytes, smem_u32(b_full));
          bulk_g2s(smem_u32(b_lo), src + kTcOpBytes / 2, kTcOpBytes, smem_u32(b_full));
        }
        reload_open = true;
        loaded = r.inst;
      }
      // the rows as the split-FP16 A operand, written over the stage once
      // every thread has read its rows; the tile scaled by the power of two
      // its largest component needs (none inside [2^0, 2^15): HX maps each
      // row on its own, so one scale per tile is exact to undo)
      unsigned char *stg = stage0 + st * kBhxStageBytes;
      constexpr int kPer = kTcM * (kTcK / 8) / kTcThreads;  // 8 pieces of 8 floats
      float4 u[kPer][2];
#pragma unroll
      for (int k = 0; k < kPer; ++k) {
        const int q = tid + k * kTcThreads;
        const int m = q >> 4, cc = q & 15;
        if (m < r.nrows) {
          // pieces 4-7 of a quarter row read their halves in the other order (bank-conflict free)
          const float4 *src = reinterpret_cast<const float4 *>(stg + m * 512 + cc * 32);
          const int sw = (cc >> 2) & 1;
          const float4 a0 = src[sw], a1 = src[sw ^ 1];
          u[k][0] = sw ? a1 : a0;
          u[k][1] = sw ? a0 : a1;
        } else {
          u[k][0] = make_float4(0.f, 0.f, 0.f, 0.f);
          u[k][1] = u[k][0];
        }
      }
      bf_bar();
      auto split_all = [&](int sxc) -> uint32_t {
        const float sc = exp2i(sxc);
        uint32_t hm = 0u;
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
          const int q = tid + k * kTcThreads;
          const int m = q >> 4, cc = q & 15;
          float v[8] = {u[k][0].x, u[k][0].y, u[k][0].z, u[k][0].w, u[k][1].x, u[k][1].y, u[k][1].z, u[k][1].w};
          // scaled by 2^sxc (a multiply by 1 for 2^0: one instantiation keeps the code small)
          const float2 s2 = make_float2(sc, sc);
          uint4 h4, l4;
          split_pair2(__fmul2_rn(make_float2(v[0], v[1]), s2), h4.x, l4.x);
          split_pair2(__fmul2_rn(make_float2(v[2], v[3]), s2), h4.y, l4.y);
          split_pair2(__fmul2_rn(make_float2(v[4], v[5]), s2), h4.z, l4.z);
          split_pair2(__fmul2_rn(make_float2(v[6], v[7]), s2), h4.w, l4.w);
          hmax_abs_acc(hm, h4.x);
          hmax_abs_acc(hm, h4.y);
          hmax_abs_acc(hm, h4.z);
          hmax_abs_acc(hm, h4.w);
          const uint32_t off = sw128_off(m, cc * 8, kTcM);
          *reinterpret_cast<uint4 *>(stg + off) = h4;
          *reinterpret_cast<uint4 *>(stg + kTcOpBytes + off) = l4;
        }
        return hm;
      };
      // the tile scaled by 2^sx, sx predicted from the previous tile (none
      // when it is 0); the largest FP16 hi part, exchanged through the
      // barrier that ends the conversion, gives the tile's own exponent, and
      // a tile whose own exponent differs is split once more from the
      // registers (uniform, rare)
      uint32_t *cr = cred + st * 16;  // [stage][hi max, FP32 max][8 warps]
      int sx = sx_pred;
      {
        const uint32_t hm = split_all(sx);
        const uint32_t wm = __reduce_max_sync(0xffffffffu, hmax_abs_bits(hm));
        if (lane == 0) cr[warp] = wm;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      if (reload) {
        ok = wait_all(b_full, b_par);
        if (!ok) break;
        b_par ^= 1u;
        reload_open = false;
      } else {
        bf_bar();
      }
      {
        uint32_t h16 = cr[0];
#pragma unroll
        for (int w = 1; w < 8; ++w) h16 = max(h16, cr[w]);
        int own = tc_shift_from_hi(h16, sx);
        if (own == -1000) {  // zero, subnormal or inf hi parts: the FP32 maximum decides
          float mx = 0.f;
#pragma unroll
          for (int k = 0; k < kPer; ++k)
#pragma unroll
            for (int h = 0; h < 2; ++h)
              mx = fmaxf(mx, fmaxf(fmaxf(fabsf(u[k][h].x), fabsf(u[k][h].y)), fmaxf(fabsf(u[k][h].z), fabsf(u[k][h].w))));
          const uint32_t fm = __reduce_max_sync(0xffffffffu, __float_as_uint(mx));
          if (lane == 0) cr[8 + warp] = fm;
          bf_bar();
          uint32_t f32 = cr[8];
#pragma unroll
          for (int w = 1; w < 8; ++w) f32 = max(f32, cr[8 + w]);
          own = tc_shift_bits(f32);
        }
        if (own != sx) {
          sx = own;
          split_all(sx);
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          bf_bar();
        }
        sx_pred = sx;
        if (tid == 0) s_tile[st] = sx;
      }
      if (tid == 0) mbar_arrive(smem_u32(&a_full[st]));
      if (i >= 1) {  // tile i-1's accumulator, read back while tile i's GEMMs run
        if (!prev_done) {
          ok = wait_all(&mma_done[(i - 1) & 1], ((i - 1) >> 1) & 1);
          if (!ok) break;
        }
        epilogue(i - 1, prev);
      }
      prev = r;
    }
    if (ok && cnt > 0) {
      ok = wait_all(&mma_done[(cnt - 1) & 1], ((cnt - 1) >> 1) & 1);
      if (ok) epilogue(cnt - 1, prev);
    }
    // an R reload whose copy was not seen to land (the warps left on a failed
    // wait): no copy may still write shared memory when the CTA leaves
    if (!ok && tid == 0) {
      fail(27);
      if (reload_open) mbar_wait_bounded(smem_u32(b_full), b_par, bp.timeout_ns);
    }
  }

  // ---- leave: every role is done (or stopped); free tensor memory
  tc_fence_before();
  __syncthreads();
  if (warp == 8) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256u) : "memory");
  }
}

// The three launches of one step over the instances of `bp` (the batch and
// the request loop share them).  Dynamic shared memory above 48 KB must have
// been enabled on these kernels in the calling translation unit
// (batch_enable_smem).
// hx_grid: CTAs of the CUDA-core HX launch (0: one wave of 8 per SM); with
// bp.hx_chunk > 0 the grid covers the items in chunks.  The tensor-core HX
// (N = 64) needs bp.hx_pre and bp.hx_ctr (zero before the first step).
static inline cudaError_t batch_launch_step(const BatchParams &bp, int tp_max, int sms, cudaStream_t stream,
                                            int hx_grid = 0) {
  if (bp.fir_tc)  // one persistent CTA per SM over equal shares of the tiles
    batch_fir_tc_kernel<<<bp.fir_cta ? bp.fir_ctas : std::max(1, std::min(sms, bp.fir_tiles)), kBfThreads,
                          kBfSmemBytes, stream>>>(bp);
  else
    batch_fir_kernel<<<bp.fir_tiles, kFirThreads, fir_smem_bytes(tp_max), stream>>>(bp, tp_max);
  batch_detsel_kernel<<<bp.n, kDetThreads, 0, stream>>>(bp);
  const int wave = bp.N == kTcNc ? sms : sms * 8;
  const int want = bp.hx_chunk > 0 ? (bp.hx_items + bp.hx_chunk - 1) / bp.hx_chunk : (hx_grid > 0 ? hx_grid : wave);
  if (bp.N == kTcNc) {
    // one persistent CTA per SM over equal shares of the selected tiles
    batch_hx_tc_kernel<<<std::max(1, sms), kBhxThreads, kBatchHxSmemBytes, stream>>>(bp);
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
