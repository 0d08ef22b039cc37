// Fused firing loop on tcgen05 tensor cores (N = 32): FIR, DET, SEL, HX_b and
// SINK per tile of 4096 outputs, with FIR and HX_b as tensor-core GEMMs.
//
// FIR as a block-Toeplitz GEMM.  A tile is 128 rows of 32 consecutive outputs;
// X_j is the j-th 32-sample chunk of the input from the tile start.  With
//   G_s[i][u] = h[i - u + 32 s]   (zero outside 0 <= i - u + 32 s < T),
// the outputs of row m are  y_m = sum_{s=0}^{S} G_s X_{m-s},  S = ceil((T-1)/32):
// this is the convolution y[n] = sum_t h[t] x[n-t] regrouped, nothing is
// approximated.  Each G_s is a 32 x 32 complex matrix used in its real form
// (64 x 64, as for HX), so a shift is one 128 x 64 x 64 real GEMM whose A
// operand holds the chunks X_{m-s}.  All shifts read one chunk array in the
// K-major 128-byte-swizzle layout, permuted so that every shift starts on an
// 8-row (1024-byte) group: GEMM row m = 8a + b carries output chunk 16b + a,
// and stored group g in [-S, 16) holds chunks 16b + g in its rows b < 8.
// Shift s then reads groups -s .. 15-s: its row 8a + b is group a - s, row b,
// i.e. chunk 16b + a - s.  The S groups below 0 repeat chunks of groups
// 16-S .. 15 one row down (plus the halo chunks before the tile).
//
// Accuracy: operands split a = a_hi + a_lo into FP16 and three products
// (hi hi, hi lo, lo hi) accumulated in FP32 in tensor memory, ~2^-22
// relative.  Every operand is scaled by a power of two first (tc_scale.cuh):
// the taps and H per graph, the input per tile (its largest component,
// halo included, in [2^14, 2^15)), the FIR output by the per-graph 2^m of
// the L1 bound; energies and outputs are scaled back exactly.
//
// HX_b (N = 32): a FIR output row is exactly one row of N samples of a
// block, so the selected blocks' FIR rows (read from TMEM) are compacted into
// the A operand of a second 128 x 64 x 64 GEMM with the real form of H.
//
// Control: block energies from the FIR accumulators, v[b] = E_b > tau, warp
// ballot compaction in the tile and the warp-parallel decoupled look-back of
// the CUDA-core firing loop across tiles (frames interleaved, see
// tc_ticket_tile); the last tile of a frame writes the SINK record and books the FIFO counters in frame order.  All waits are
// bounded; tensor memory is freed on every path.
#pragma once
#include <type_traits>

#include "firing_loop.cuh"
#include "tc_common.cuh"

namespace prune {

__host__ inline bool tc_loop_supported(int N, int B, int T) {
  return N == 32 && B % kTR == 0 && B <= kTTile && kTTile % B == 0 && T <= (kTMaxShifts - 1) * kTR + 1;
}

// Tile pipelines: NP independent pipelines of 128 threads per CTA share the
// tap and H operands; each has its own chunk array, mbarriers and 128 TMEM
// columns, so NP tiles are in flight per SM (4 when T <= 65, else 3, as far
// as shared memory allows).
constexpr int kTPipeThreads = 128;
__host__ __device__ inline int tc_pipes(int T) { return tc_shifts(T) <= 3 ? 4 : 3; }
__host__ __device__ inline size_t tc_pipe_bytes(int T) {
  return 2 * static_cast<size_t>(kTGroups + tc_shifts(T) - 1) * 1024 + 2048;
}
__host__ __device__ inline size_t tc_loop_smem_bytes(int T) {
  return 1024 + static_cast<size_t>(tc_shifts(T)) * 2 * kTOpBytes + 2 * kTOpBytes +
         static_cast<size_t>(tc_pipes(T)) * tc_pipe_bytes(T);
}

struct TcLoopParams {
  int32_t window;        // frames fired round-robin (tc_ticket_tile)
  LoopParams lp;
  const uint16_t *fir_ops;   // taps scaled by 2^s_taps
  const uint16_t *hx_ops;    // H scaled by 2^s_h
  int32_t ns;
  int32_t s_taps, m, s_h;    // TcScale of the graph
};

__device__ __forceinline__ uint4 split_pack8(const float *v, bool lo) {
  uint32_t w[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const __half h0 = __float2half_rn(v[2 * e]), h1 = __float2half_rn(v[2 * e + 1]);
    __half a = h0, b = h1;
    if (lo) {
      a = __float2half_rn(v[2 * e] - __half2float(h0));
      b = __float2half_rn(v[2 * e + 1] - __half2float(h1));
    }
    w[e] = static_cast<uint32_t>(__half_as_ushort(a)) | (static_cast<uint32_t>(__half_as_ushort(b)) << 16);
  }
  return make_uint4(w[0], w[1], w[2], w[3]);
}

// Order of the work items.  Tickets are claimed in order; ticket t maps to
// a (frame, tile) pair so that a window of up to W frames is fired
// round-robin: consecutive tickets go to different frames, and the tiles of
// one frame are claimed W tickets apart, in increasing order.  With P
// pipelines in flight a frame then has about P / W tiles in flight, so the
// look-back of a tile rarely finds an unpublished predecessor (with W = 1
// every pipeline would work on the same frame and each look-back would wait
// for the slowest of hundreds of tiles).
__host__ __device__ __forceinline__ void tc_ticket_tile(unsigned long long t, int frames, int tiles, int W, int *k,
                                                        int *tile) {
  const unsigned long long win = static_cast<unsigned long long>(W) * tiles;
  const int w = static_cast<int>(t / win);
  const int r = static_cast<int>(t % win);
  const int wc = min(W, frames - w * W);  // frames in this window
  *k = w * W + r % wc;
  *tile = r / wc;
}

template <int NP>
static __global__ void __launch_bounds__(NP * kTPipeThreads, 1) firing_loop_tc_kernel(TcLoopParams tp) {
  extern __shared__ unsigned char smem_raw[];
  const LoopParams &p = tp.lp;
  const FirParams &f = p.f;
  const int ns = tp.ns, S = ns - 1;
  unsigned char *base = smem_align1024(smem_raw);
  unsigned char *bfir = base;
  unsigned char *bhx = bfir + ns * 2 * kTOpBytes;
  const int cta_tid = threadIdx.x, cta_warp = cta_tid >> 5;
  const int pipe = cta_tid / kTPipeThreads;
  unsigned char *pipe0 = bhx + 2 * kTOpBytes;
  const size_t pbytes = tc_pipe_bytes(f.T);
  unsigned char *ahi = pipe0 + pipe * pbytes;
  unsigned char *alo = ahi + (kTGroups + S) * 1024;
  unsigned char *misc = alo + (kTGroups + S) * 1024;
  uint64_t *mbar = reinterpret_cast<uint64_t *>(misc);               // [2]
  int32_t *s_flag = reinterpret_cast<int32_t *>(misc + 16);
  int32_t *s_cnt = reinterpret_cast<int32_t *>(misc + 20);
  unsigned long long *s_ticket = reinterpret_cast<unsigned long long *>(misc + 24);
  int32_t *s_rank = reinterpret_cast<int32_t *>(misc + 64);          // [128] blocks of a tile
  float *eth = reinterpret_cast<float *>(misc + 576);                 // [128] chunk energies
  float *Et = eth + 128;                                              // [128] block energies
  float *red4 = Et + 128;                                             // [4]
  int32_t *s_rule = reinterpret_cast<int32_t *>(misc + 36);           // firing rule of the claimed tile
  long long *s_prefix = reinterpret_cast<long long *>(misc + 40);
  uint32_t *s_red = reinterpret_cast<uint32_t *>(misc + 1664);       // [3][4] warps' maxima
  uint32_t *tmem_slot0 = reinterpret_cast<uint32_t *>(pipe0 + 2 * (kTGroups + S) * 1024 + 32);

  const int tid = cta_tid % kTPipeThreads, warp = tid >> 5, lane = cta_tid & 31;  // within the pipeline
  int sx_pred = 0;  // scale exponent of this pipeline's previous tile
  // barrier of this pipeline's 128 threads (named barrier 1 + pipe)
  auto psync = [&]() { asm volatile("bar.sync %0, 128;" ::"r"(1 + pipe) : "memory"); };
  // B divides the 4096-sample tile and is a multiple of 32: a power of two,
  // so every division by B or by rows per block is a shift; ring slots take
  // one 64-bit modulo per launch and a subtraction per tile
  const int lgB = __ffs(f.B) - 1, lgR = lgB - 5;
  const RingSlot fring = RingSlot::of(f.yslot.seq0, p.C);   // frame slot of the look-back words
  const RingSlot rring = RingSlot::of(p.rslot.seq0, p.rslot.cap);
  const RingSlot ering = f.energy ? RingSlot::of(f.eslot.seq0, f.eslot.cap) : RingSlot{0, 1};
  const RingSlot sring = f.src.ring ? RingSlot::of(f.src.seq0, f.src.cap) : RingSlot{0, 1};
  auto frame_at = [&](int k) -> const float2 * {
    return f.src.ring ? f.src.ring[sring.at(k)] : f.src.base + static_cast<int64_t>(k) * f.src.stride;
  };

  // constant operands, once per CTA
  {
    const uint4 *src = reinterpret_cast<const uint4 *>(tp.fir_ops);
    uint4 *dst = reinterpret_cast<uint4 *>(bfir);
    for (int q = cta_tid; q < static_cast<int>(ns * 2 * kTOpBytes / 16); q += NP * kTPipeThreads) dst[q] = src[q];
    const uint4 *hsrc = reinterpret_cast<const uint4 *>(tp.hx_ops);
    uint4 *hdst = reinterpret_cast<uint4 *>(bhx);
    for (int q = cta_tid; q < static_cast<int>(2 * kTOpBytes / 16); q += NP * kTPipeThreads) hdst[q] = hsrc[q];
  }
  if (tid == 0) {
    mbar_init(smem_u32(&mbar[0]), 1);
    mbar_init(smem_u32(&mbar[1]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *s_flag = 0;
  }
  if (cta_warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot0)),
                 "r"(512u)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot0 + 128u * static_cast<uint32_t>(pipe);  // this pipeline's columns
  // TMEM lanes of warp `warp` (the CTA warp index mod 4 equals it)
  const uint32_t tlane = static_cast<uint32_t>(warp * 32) << 16;
  uint32_t ph0 = 0, ph1 = 0;
  bool failed = false;

  const unsigned long long total = static_cast<unsigned long long>(f.frames) * f.tiles;
  const int m = tid;                           // TMEM lane (GEMM row) owned by this thread
  const int jc = 16 * (m & 7) + (m >> 3);      // output chunk of FIR GEMM row m
  const int npieces = (kTGroups + S) * 64;     // 16-byte pieces of the chunk array
  uint64_t f0_seen = 0;                        // thread 0: last f0 counter value read
  bool fir_pending = false, hx_pending = false;
  // Tickets are claimed in order by all P = grid x NP pipelines, so the tile
  // of ticket t + P is claimed about one tile period after t.  The claiming
  // thread (thread 32 of the pipeline, while thread 0 books the previous
  // tile) checks FIR's firing rule on f0 for the claimed tile (bounded
  // wait) and, when the frame of tile t + P is already written, prefetches
  // that tile's input into L2 during the look-back, so that its loads hit in
  // L2.
  const unsigned long long P = static_cast<unsigned long long>(gridDim.x) * NP;
  const float2 *pf_src = nullptr;  // thread 32: pending L2 prefetch
  uint32_t pf_bytes = 0;
  auto claim = [&]() {
    const unsigned long long tk = atomicAdd(&p.ls->ticket, 1ull) - p.ticket_base;
    int rule = 0;
    if (tk < total) {
      int kc, tc;
      tc_ticket_tile(tk, f.frames, f.tiles, tp.window, &kc, &tc);
      const uint64_t need = (static_cast<uint64_t>(f.yslot.seq0) + kc + 1) * static_cast<uint64_t>(f.F);
      if (f0_seen < need) {
        const bool ok = bounded_wait(p, [&] {
          f0_seen = ld_acquire_u64(&p.ctr[0 * 3 + kCtrWritten]);
          return f0_seen >= need;
        }, kActFir, 0, static_cast<uint64_t>(f.yslot.seq0) + kc);
        rule = ok ? 0 : -1;
      }
      const unsigned long long u = tk + P;
      if (u < total) {
        int kn, tn;
        tc_ticket_tile(u, f.frames, f.tiles, tp.window, &kn, &tn);
        const uint64_t needn = (static_cast<uint64_t>(f.yslot.seq0) + kn + 1) * static_cast<uint64_t>(f.F);
        if (f0_seen >= needn) {  // frame written: its slot holds it
          const int64_t s0n = static_cast<int64_t>(tn) * kTTile;
          const int64_t lo = s0n >= static_cast<int64_t>(S) * kTR ? s0n - static_cast<int64_t>(S) * kTR : 0;
          const int64_t hi = min(s0n + static_cast<int64_t>(kTTile), f.L);
          pf_src = frame_at(kn) + lo;  // issued later, while warps 1-3 idle in the look-back
          pf_bytes = static_cast<uint32_t>((hi - lo) * 8);
        }
      }
    }
    *s_rule = rule;
    *s_ticket = ld_volatile_u32(&p.ls->abort) ? ~0ull : tk;
  };
  if (tid == 32) claim();
  psync();
  for (;;) {
    const unsigned long long t = *s_ticket;
    if (t >= total || *s_rule < 0) break;
    int k, tile;
    tc_ticket_tile(t, f.frames, f.tiles, tp.window, &k, &tile);
    const uint64_t seq = static_cast<uint64_t>(f.yslot.seq0) + k;
    const int64_t s0 = static_cast<int64_t>(tile) * kTTile;
    const int nv = static_cast<int>(min(static_cast<int64_t>(kTTile), f.L - s0));
    const int rows_valid = nv / kTR;

    // ---- FIR A operand: stored row R = 8 (g + S) + b holds chunk j = 16 b + g.
    // A thread's global loads are issued in batches before conversion.  The
    // tile is scaled by the pipeline's previous tile's power of two; its
    // largest component (halo included), gathered on the way, checks that
    // scale after the barrier, and a tile it does not fit is converted again.
    const float2 *cur = frame_at(k);
    const float2 *prev = k > 0 ? frame_at(k - 1) : nullptr;
    auto load_piece = [&](int q, float (&v)[8]) {
      const int row = q >> 3, pc = q & 7;
      const int j = 16 * (row & 7) + (row >> 3) - S;
      const int64_t pos0 = s0 + static_cast<int64_t>(j) * kTR + 4 * pc;
      if (j >= 0) {
        if (kTR * j + 4 * pc < nv) {
          const float4 *src = reinterpret_cast<const float4 *>(cur + pos0);
          const float4 u0 = __ldg(src), u1 = __ldg(src + 1);
          v[0] = u0.x; v[1] = u0.y; v[2] = u0.z; v[3] = u0.w;
          v[4] = u1.x; v[5] = u1.y; v[6] = u1.z; v[7] = u1.w;
        } else {
#pragma unroll
          for (int e = 0; e < 8; ++e) v[e] = 0.f;
        }
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int64_t pos = pos0 + e;
          const int64_t d = s0 - pos;
          float2 x = make_float2(0.f, 0.f);
          if (d <= f.T - 1) {
            if (pos >= 0) x = cur[pos];
            else if (prev) x = prev[f.L + pos];
            else if (f.hist) x = f.hist[f.T - 1 + pos];
          }
          v[2 * e] = x.x;
          v[2 * e + 1] = x.y;
        }
      }
    };
    if (f.hist_out && k == f.frames - 1 && s0 + nv == f.L)
      for (int i = tid; i < f.T - 1; i += kTPipeThreads) f.hist_out[i] = cur[f.L - (f.T - 1) + i];
    // the tile scaled by 2^sx, sx predicted from the pipeline's previous
    // tile (no multiply when it is 0); the largest FP16 hi part gives the
    // tile's own exponent after the barrier that ends the conversion, and a
    // tile whose own exponent differs is converted once more (uniform,
    // rare): the exponent a tile is fired with depends on the tile alone
    // loads in flight per thread: fewer with four pipelines (128 registers)
    constexpr int kPieces = NP == 4 ? 3 : kTMaxPieces;
    auto convert = [&](int sxc) -> uint32_t {
      const float xsc = exp2i(sxc);
      uint32_t hm = 0u;
      for (int q0 = 0; q0 < npieces; q0 += kPieces * kTPipeThreads) {
        float v[kPieces][8];
#pragma unroll
        for (int i = 0; i < kPieces; ++i) {
          const int q = q0 + tid + kTPipeThreads * i;
          if (q < npieces) load_piece(q, v[i]);
        }
#pragma unroll
        for (int i = 0; i < kPieces; ++i) {
          const int q = q0 + tid + kTPipeThreads * i;
          if (q >= npieces) continue;
          // scaled by 2^sxc (a multiply by 1 for 2^0: one instantiation keeps the code small)
          const float2 x2 = make_float2(xsc, xsc);
          const int row = q >> 3, pc = q & 7;
          const uint32_t off = static_cast<uint32_t>(row) * 128u + (static_cast<uint32_t>(pc ^ (row & 7)) << 4);
          uint4 h4, l4;
          split_pair2(__fmul2_rn(make_float2(v[i][0], v[i][1]), x2), h4.x, l4.x);
          split_pair2(__fmul2_rn(make_float2(v[i][2], v[i][3]), x2), h4.y, l4.y);
          split_pair2(__fmul2_rn(make_float2(v[i][4], v[i][5]), x2), h4.z, l4.z);
          split_pair2(__fmul2_rn(make_float2(v[i][6], v[i][7]), x2), h4.w, l4.w);
          hmax_abs_acc(hm, h4.x);
          hmax_abs_acc(hm, h4.y);
          hmax_abs_acc(hm, h4.z);
          hmax_abs_acc(hm, h4.w);
          *reinterpret_cast<uint4 *>(ahi + off) = h4;
          *reinterpret_cast<uint4 *>(alo + off) = l4;
        }
      }
      return hm;
    };
    int sx = sx_pred;
    for (int pass = 0;; ++pass) {
      const uint32_t hm = convert(sx);
      // s_red: [hi max of pass 0, of pass 1, FP32 max][4 warps]
      const uint32_t wm = __reduce_max_sync(0xffffffffu, hmax_abs_bits(hm));
      if (lane == 0) s_red[4 * pass + warp] = wm;
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      tc_fence_before();
      psync();
      if (pass == 1) break;
      int own = tc_shift_from_hi(max(max(s_red[0], s_red[1]), max(s_red[2], s_red[3])), sx);
      if (own == -1000) {  // zero, subnormal or inf hi parts: the FP32 maximum decides
        float mx = 0.f;
        for (int q = tid; q < npieces; q += kTPipeThreads) {
          float v[8];
          load_piece(q, v);
#pragma unroll
          for (int e = 0; e < 8; ++e) mx = fmaxf(mx, fabsf(v[e]));
        }
        const uint32_t fm = __reduce_max_sync(0xffffffffu, __float_as_uint(mx));
        if (lane == 0) s_red[8 + warp] = fm;
        psync();
        own = tc_shift_bits(max(max(s_red[8], s_red[9]), max(s_red[10], s_red[11])));
      }
      if (own == sx) break;
      sx = own;
    }
    sx_pred = sx;

    // ---- FIR GEMM: ns shifts x 3 passes x 4 K-steps of 128 x 64 x 16
    if (tid == 0) {
      tc_fence_after();
      const uint32_t ah = smem_u32(ahi), al = smem_u32(alo), b0 = smem_u32(bfir);
      for (int s = 0; s < ns; ++s) {
        const uint32_t arow = static_cast<uint32_t>(S - s) * 1024u;  // group -s
        const uint32_t pa[3] = {ah + arow, ah + arow, al + arow};
        const uint32_t bh = b0 + static_cast<uint32_t>(2 * s) * kTOpBytes, bl = bh + kTOpBytes;
        const uint32_t pb[3] = {bh, bl, bh};
#pragma unroll
        for (int pass = 0; pass < 3; ++pass)
#pragma unroll
          for (int ks = 0; ks < 4; ++ks)
            umma_f16(tmem, umma_desc_sw128(pa[pass] + ks * 32), umma_desc_sw128(pb[pass] + ks * 32), kTIdescN64,
                     (s > 0 || pass > 0 || ks > 0) ? 1u : 0u);
      }
      umma_commit(smem_u32(&mbar[0]));
    }
    fir_pending = true;
    if (mbar_wait_bounded(smem_u32(&mbar[0]), ph0, p.timeout_ns)) {
      ph0 ^= 1u;
      fir_pending = false;
    } else {
      if (tid == 0) report_error(p.status, kDevTimeout, kActFir, 2, seq);
      *s_flag = 1;
    }
    psync();
    if (*s_flag) { failed = true; break; }
    tc_fence_after();

    // ---- DET: energy of chunk jc (GEMM row m), both column halves
    {
      float2 e2 = make_float2(0.f, 0.f);  // even and odd columns' squares
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        float t16[16];
        tmem_ld16(tmem + tlane + static_cast<uint32_t>(h * 16), t16);
        tmem_ld_wait();
#pragma unroll
        for (int i = 0; i < 16; i += 2) {
          const float2 t = make_float2(t16[i], t16[i + 1]);
          e2 = __ffma2_rn(t, t, e2);
        }
      }
      eth[jc] = jc < rows_valid ? mul_pow2(e2.x + e2.y, -2 * (sx + tp.s_taps)) : 0.f;
    }
    psync();
    // block energies: eth is ordered by chunk; block b owns [rpb b, rpb (b+1));
    // a shuffle tree per segment of the warp, in a fixed order
    const int rpb = f.B / kTR;  // rows (chunks) per block
    const int nb = nv >> lgB;
    {
      float v = eth[tid];
      const int seg = rpb < 32 ? rpb : 32;
      for (int off = seg >> 1; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
      if (rpb <= 32) {
        if ((tid & (seg - 1)) == 0 && (tid >> lgR) < nb) Et[tid >> lgR] = v;
      } else {
        if (lane == 0) red4[warp] = v;
      }
      psync();
      if (rpb > 32 && tid < nb) {
        float E = 0.f;
        for (int w = 0; w < rpb / 32; ++w) E += red4[tid * (rpb / 32) + w];
        Et[tid] = E;
      }
      psync();
      if (f.energy && tid < nb) f.energy[static_cast<int64_t>(ering.at(k)) * f.F + tile * (kTTile >> lgB) + tid] = Et[tid];
    }
    // ---- SEL inside the tile: stable ballot compaction
    if (warp == 0) {
      int cnt = 0;
      for (int b0 = 0; b0 < nb; b0 += 32) {
        const int b = b0 + lane;
        const bool v = b < nb && Et[b] > p.tau;
        const unsigned msk = __ballot_sync(0xffffffffu, v);
        if (b < nb) s_rank[b] = v ? cnt + __popc(msk & ((1u << lane) - 1u)) : -1;
        cnt += __popc(msk);
      }
      if (lane == 0) *s_cnt = cnt;
    }
    psync();
    const int cnt = *s_cnt;
    // selected rows become rows of the HX A operand (the FIR operand area is
    // free): the FIR accumulators are read a second time, half a row at a
    // time, and scaled by 2^m
    {
      const float hsc = exp2i(tp.m);
      const int rk = jc < rows_valid ? s_rank[jc >> lgR] : -1;
      const int hrow = rk * rpb + (jc & (rpb - 1));
#pragma unroll
      for (int hf = 0; hf < 2; ++hf) {
        float y[32];
        {
          float t16[16];
          tmem_ld16(tmem + tlane + static_cast<uint32_t>(hf * 32), t16);
#pragma unroll
          for (int i = 0; i < 16; ++i) y[i] = t16[i] * hsc;
          tmem_ld16(tmem + tlane + static_cast<uint32_t>(hf * 32 + 16), t16);
#pragma unroll
          for (int i = 0; i < 16; ++i) y[16 + i] = t16[i] * hsc;
          tmem_ld_wait();
        }
        if (rk >= 0) {
#pragma unroll
          for (int pp = 0; pp < 4; ++pp) {
            const uint32_t off = static_cast<uint32_t>(hrow) * 128u +
                                 (static_cast<uint32_t>((4 * hf + pp) ^ (hrow & 7)) << 4);
            *reinterpret_cast<uint4 *>(ahi + off) = split_pack8(y + 8 * pp, false);
            *reinterpret_cast<uint4 *>(alo + off) = split_pack8(y + 8 * pp, true);
          }
        }
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    psync();
    // ---- HX_b GEMM on the compacted rows (needs no prefix: issued first) ...
    if (cnt > 0) {
      if (tid == 0) {
        tc_fence_after();
        const uint32_t ah = smem_u32(ahi), al = smem_u32(alo), bh = smem_u32(bhx), bl = bh + kTOpBytes;
        const uint32_t pa[3] = {ah, ah, al}, pb[3] = {bh, bl, bh};
#pragma unroll
        for (int pass = 0; pass < 3; ++pass)
#pragma unroll
          for (int ks = 0; ks < 4; ++ks)
            umma_f16(tmem + 64u, umma_desc_sw128(pa[pass] + ks * 32), umma_desc_sw128(pb[pass] + ks * 32),
                     kTIdescN64, (pass > 0 || ks > 0) ? 1u : 0u);
        umma_commit(smem_u32(&mbar[1]));
      }
      hx_pending = true;
    }
    // ... while one warp runs the look-back for the tile's offset in the frame
    const int64_t fslot = fring.at(k);
    if (warp == 0) {
      const int64_t pr = lookback_warp(p, p.look + fslot * f.tiles, tile, seq + 1, cnt, seq, lane);
      if (lane == 0) *s_prefix = pr;
    } else if (tid == 32 && pf_bytes) {
      asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(pf_src), "r"(pf_bytes) : "memory");
      pf_bytes = 0;
    }
    psync();
    const long long prefix = *s_prefix;
    if (prefix < 0) { failed = true; break; }
    if (prefix + cnt > f.F) {
      if (tid == 0) {
        report_error(p.status, kDevInvariant, kActSel, 6, seq);
        atomicExch(&p.ls->abort, 1u);
      }
      failed = true;
      break;
    }
    const int64_t rs = rring.at(k);
    if (tid < nb && s_rank[tid] >= 0) p.rec_idx[rs * f.F + prefix + s_rank[tid]] = tile * (kTTile >> lgB) + tid;

    // ---- SINK payload: HX_b outputs at their compacted positions
    if (cnt > 0) {
      if (mbar_wait_bounded(smem_u32(&mbar[1]), ph1, p.timeout_ns)) {
        ph1 ^= 1u;
        hx_pending = false;
      } else {
        if (tid == 0) report_error(p.status, kDevTimeout, kActHx, 7, seq);
        *s_flag = 1;
      }
      psync();
      if (*s_flag) { failed = true; break; }
      tc_fence_after();
      float f1, f2;  // HX outputs are H y 2^(sx + s_taps + m + s_h)
      pow2_pair(-(sx + tp.s_taps + tp.m + tp.s_h), f1, f2);
#pragma unroll
      for (int hf = 0; hf < 2; ++hf) {
        float o[32];
        {
          float t16[16];
          tmem_ld16(tmem + tlane + 64u + static_cast<uint32_t>(hf * 32), t16);
#pragma unroll
          for (int i = 0; i < 16; ++i) o[i] = t16[i];
          tmem_ld16(tmem + tlane + 64u + static_cast<uint32_t>(hf * 32 + 16), t16);
#pragma unroll
          for (int i = 0; i < 16; ++i) o[16 + i] = t16[i];
          tmem_ld_wait();
        }
        if (m < cnt * rpb) {  // 32-byte stores (whole sectors; the half-row starts 128-byte aligned)
          float *dst = reinterpret_cast<float *>(p.rec_y + rs * f.L + (prefix + (m >> lgR)) * f.B +
                                                 (m & (rpb - 1)) * kTR + hf * 16);
          if (f2 != 1.f)  // a scale beyond one float factor (uniform, rare)
            for (int i = 0; i < 32; ++i) o[i] *= f2;
#pragma unroll
          for (int i = 0; i < 4; ++i) st_global_v8(dst + 8 * i, o + 8 * i, f1);
        }
      }
    }

    // ---- frame completion: the last tile to finish writes the SINK record;
    // warp 0 then books the frames that are ready in order
    tc_fence_before();
    psync();
    if (warp == 0) {
      int last = 0;
      if (lane == 0) {
        __threadfence();
        const uint32_t old = atomicAdd(&p.done[fslot], 1u);
        if (old + 1u == static_cast<uint32_t>(f.tiles)) {
          p.done[fslot] = 0u;  // every tile of the frame has counted: reset the slot
          __threadfence();  // every tile counted: their look-back words are visible
          const uint64_t w = ld_acquire_u64(&p.look[fslot * f.tiles + f.tiles - 1]);
          p.rec_c[rs] = static_cast<int32_t>(static_cast<uint32_t>(w));
          p.rec_frame[rs] = static_cast<int64_t>(seq);
          __threadfence();
          st_release_u64(&p.ready[fslot], seq + 1);
          __threadfence();
          last = 1;
        }
      }
      if (__shfl_sync(0xffffffffu, last, 0)) drain_bookkeeping(p, static_cast<uint64_t>(f.yslot.seq0) + f.frames, lane);
    }
    if (tid == 32) claim();
    psync();
  }

  // leave: let MMAs still in flight land (bounded) before freeing tensor memory
  if (failed) {
    if (fir_pending) mbar_wait_bounded(smem_u32(&mbar[0]), ph0, p.timeout_ns);
    if (hx_pending) mbar_wait_bounded(smem_u32(&mbar[1]), ph1, p.timeout_ns);
  }
  tc_fence_before();
  __syncthreads();
  if (cta_warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(*tmem_slot0), "r"(512u) : "memory");
  }
}

}  // namespace prune
