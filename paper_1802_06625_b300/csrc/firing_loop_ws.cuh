// Warp-specialised fused firing loop on tcgen05 (N = 32, T <= 65): the same
// arithmetic as firing_loop_tc_kernel (block-Toeplitz FIR and HX_b on
// tensor cores, split FP16, look-back control), with the phases of a tile
// split over roles that run concurrently on different tiles:
//
//   warp 0          producer: claims tiles (ticket order, frame window),
//                   checks FIR's firing rule on f0 and copies the raw input
//                   tile (+ halo) into a 2-stage shared-memory ring with bulk
//                   asynchronous copies (cp.async.bulk, mbarrier tx counts);
//   warp 1          MMA: the FIR GEMMs of a tile into one of 4 TMEM slots
//                   (three split products: hi x hi, hi x lo, lo x hi);
//   warps 2-7       converter: raw FP32 -> split-FP16 chunk array (the
//                   permuted K-major 128B-swizzle operand), 2-buffer ring,
//                   with the tile scaled by the power of two of the
//                   converter's previous tile; the tile's largest component
//                   (halo included), gathered from the same registers, checks
//                   that scale after the converter's barrier, and the rare
//                   tile it does not fit is converted again with its own;
//   warps 8-19      three epilogue groups, tiles taken round-robin: block
//                   energies, DET and SEL, the HX_b operand written back into
//                   the slot's free TMEM columns (two FP16 per column), HX_b as
//                   a GEMM with its A operand in tensor memory on all 128 rows
//                   (issued by the group's last warp), the look-back
//                   (overlapping the HX GEMM), the SINK payload of the
//                   selected rows and the frame completion.
//
// A TMEM slot is 128 columns: the FIR accumulator (FP32, columns 0-63)
// whose rows are split into the HX operand (hi in 64-95, lo in 96-127), and
// the HX accumulator written over columns 0-63.  Every hand-off is an
// mbarrier whose phase flips exactly once per use, so each waiter knows the
// parity from the use count.  After the last tile the producer sends one
// sentinel item per epilogue group through the pipeline.  Every wait is
// bounded and also returns when the CTA's stop flag is set; before tensor
// memory is freed, each thread that issued GEMMs commits once more to a
// barrier of its own and waits for it (all its GEMMs have completed).
#pragma once
#include <type_traits>

#include "firing_loop_tc.cuh"

namespace prune {

// Six converter warps: the converter sets the tile period, and six measured
// faster than four (five did not); 640 threads at 90 registers fit the file.
constexpr int kWsConvWarps = 6;              // converter warps (2 .. 1 + kWsConvWarps)
constexpr int kWsConvThreads = kWsConvWarps * 32;
constexpr int kWsEpiWarp0 = 2 + kWsConvWarps; // first epilogue warp
constexpr int kWsWarps = kWsEpiWarp0 + 12;
constexpr int kWsThreads = kWsWarps * 32;
constexpr int kWsGroups = 3;                  // epilogue groups
constexpr int kWsSlots = 4;                   // TMEM slots of 128 columns
constexpr int kWsRawHalo = 64;                // halo samples staged (S <= 2)
constexpr uint32_t kWsRawBytes = ((kWsRawHalo + kTTile) * 8 + 1023) / 1024 * 1024;  // 33 KB
constexpr uint32_t kWsAOpBytes = 2u * (kTGroups + 2) * 1024;                       // 36 KB (hi | lo)
constexpr uint32_t kWsMiscBytes = 8192;
constexpr int kWsConvBatch = 3;               // converter pieces per thread in flight

__host__ __device__ inline bool ws_loop_supported(int T) { return tc_shifts(T) <= 3; }
// constants (FIR ns x hi/lo, HX hi/lo) | 2 raw stages | 2 operand buffers | misc
__host__ __device__ inline size_t ws_loop_smem_bytes(int T) {
  return 1024 + static_cast<size_t>(tc_shifts(T)) * 2 * kTOpBytes + 2 * kTOpBytes + 2 * kWsRawBytes +
         2 * kWsAOpBytes + kWsMiscBytes;
}

// Per-item record passed along the pipeline (t = ~0: sentinel); sx is the
// tile's scale exponent (set by the converter).
struct WsItem {
  unsigned long long t;
  int32_t k, tile, nv, sx;
};

// Shared scratch of one epilogue group.
struct WsGroup {
  float eth[128];
  float Et[128];
  int32_t rank[128];
  int32_t cnt;
  int32_t pad;
  long long prefix;
};

// The misc region: mbarriers [0, 256), item records [256, 448), the TMEM
// slot and stop flag [512, 520), the converter's maxima [528, 624), the
// epilogue groups' scratch from 1024.
constexpr uint32_t kWsGroupOff = 1024;
static_assert(kWsGroupOff + kWsGroups * sizeof(WsGroup) <= kWsMiscBytes, "the groups' scratch fits the misc region");
static_assert(24 * sizeof(uint64_t) <= 256, "the mbarriers fit [0, 256)");
static_assert(528 + 2 * 3 * kWsConvWarps * sizeof(uint32_t) <= kWsGroupOff, "the converter's maxima fit [528, 1024)");
static_assert(8 * sizeof(WsItem) <= 192, "the item records fit [256, 448)");

// Cold paths.  They stay inlined: as calls, the register saves around them
// cost the hot loops more than their code does.
// A wait ran out (or the CTA stops): the first reports it and the run aborts.
static __device__ __forceinline__ void ws_fail(const LoopParams &p, volatile int32_t *stop, uint32_t actor,
                                            uint32_t where, uint64_t frame) {
  if (!*stop) {
    report_error(p.status, kDevTimeout, actor, where, frame);
    atomicExch(&p.ls->abort, 1u);
  }
  *stop = 1;
}
// The frame's last tile was counted: publish its SINK record (c from the
// last look-back word) and mark the frame slot ready.
static __device__ __forceinline__ void ws_publish_frame(const LoopParams &p, int64_t fslot, int64_t rs, uint64_t seq,
                                                     int tiles) {
  p.done[fslot] = 0u;
  __threadfence();  // every tile counted: their look-back words are visible
  const uint64_t w = ld_acquire_u64(&p.look[fslot * tiles + tiles - 1]);
  p.rec_c[rs] = static_cast<int32_t>(static_cast<uint32_t>(w));
  p.rec_frame[rs] = static_cast<int64_t>(seq);
  __threadfence();
  st_release_u64(&p.ready[fslot], seq + 1);
  __threadfence();
}

// Bounded waits for the raw stages of the last two of `armed` items.
static __device__ __noinline__ void ws_drain_raw(uint64_t *raw_full, uint32_t armed, uint64_t timeout_ns) {
  for (uint32_t x = armed > 2u ? armed - 2u : 0u; x < armed; ++x)
    mbar_wait_bounded(smem_u32(&raw_full[x & 1u]), (x >> 1) & 1u, timeout_ns);
}

static __global__ void __launch_bounds__(kWsThreads, 1) firing_loop_ws_kernel(TcLoopParams tp) {
  extern __shared__ unsigned char smem_raw[];
  const LoopParams &p = tp.lp;
  const FirParams &f = p.f;
  const int ns = tp.ns, S = ns - 1;
  unsigned char *base = smem_align1024(smem_raw);
  unsigned char *bfir = base;
  unsigned char *bhx = bfir + ns * 2 * kTOpBytes;
  unsigned char *raw0 = bhx + 2 * kTOpBytes;
  unsigned char *aop0 = raw0 + 2 * kWsRawBytes;
  unsigned char *misc = aop0 + 2 * kWsAOpBytes;
  uint64_t *raw_full = reinterpret_cast<uint64_t *>(misc);          // [2]
  uint64_t *raw_empty = raw_full + 2;                               // [2]
  uint64_t *a_full = raw_empty + 2;                                 // [2]
  uint64_t *a_empty = a_full + 2;                                   // [2]
  uint64_t *fir_full = a_empty + 2;                                 // [4]
  uint64_t *slot_empty = fir_full + 4;                              // [4]
  uint64_t *hx_full = slot_empty + 4;                               // [4]
  uint64_t *fin = hx_full + 4;                                      // [4] one per issuer, at exit
  WsItem *item_raw = reinterpret_cast<WsItem *>(misc + 256);        // [2]
  WsItem *item_a = item_raw + 2;                                    // [2]
  WsItem *item_slot = item_a + 2;                                   // [4]
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(misc + 512);
  volatile int32_t *stop = reinterpret_cast<volatile int32_t *>(misc + 520);
  uint32_t *cred = reinterpret_cast<uint32_t *>(misc + 528);         // [2][3][kWsConvWarps] converter warps' maxima
  WsGroup *grp = reinterpret_cast<WsGroup *>(misc + kWsGroupOff);   // [3]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const unsigned long long total = static_cast<unsigned long long>(f.frames) * f.tiles;
  const unsigned long long kSentinel = ~0ull;

  // ---- setup: constant operands, barriers, tensor memory
  {
    const uint4 *src = reinterpret_cast<const uint4 *>(tp.fir_ops);
    uint4 *dst = reinterpret_cast<uint4 *>(bfir);
    for (int q = tid; q < static_cast<int>(ns * 2 * kTOpBytes / 16); q += kWsThreads) dst[q] = src[q];
    const uint4 *hsrc = reinterpret_cast<const uint4 *>(tp.hx_ops);
    uint4 *hdst = reinterpret_cast<uint4 *>(bhx);
    for (int q = tid; q < static_cast<int>(2 * kTOpBytes / 16); q += kWsThreads) hdst[q] = hsrc[q];
  }
  if (tid == 0) {
    for (int i = 0; i < 24; ++i) mbar_init(smem_u32(raw_full + i), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *stop = 0;
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(512u)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  auto fail = [&](uint32_t actor, uint32_t where, uint64_t frame) { ws_fail(p, stop, actor, where, frame); };

  if (warp == 0) {
    // ================================================================ producer
    uint64_t f0_seen = 0;
    int sentinels = 0;
    bool claimed_out = false;  // one failing claim per CTA
    uint32_t i = 0;            // items armed so far (a failed wait leaves before arming item i)
    for (; sentinels < kWsGroups; ++i) {
      const int s = i & 1;
      if (i >= 2 && !__all_sync(0xffffffffu, ws_wait(smem_u32(&raw_empty[s]), ((i >> 1) - 1) & 1u, p.timeout_ns, stop))) {
        if (lane == 0) fail(kActFir, 10, 0);
        break;
      }
      unsigned long long t = kSentinel;
      if (lane == 0 && !claimed_out) {
        t = atomicAdd(&p.ls->ticket, 1ull) - p.ticket_base;
        if (ld_volatile_u32(&p.ls->abort) || *stop) t = kSentinel;
      }
      t = __shfl_sync(0xffffffffu, t, 0);
      if (t >= total) {  // no more tiles: one sentinel per epilogue group
        claimed_out = true;
        if (lane == 0) {
          item_raw[s] = WsItem{kSentinel, 0, 0, 0, 0};
          mbar_arrive(smem_u32(&raw_full[s]));
        }
        ++sentinels;
        continue;
      }
      int k, tile;
      tc_ticket_tile(t, f.frames, f.tiles, tp.window, &k, &tile);
      const uint64_t seq = static_cast<uint64_t>(f.yslot.seq0) + k;
      const int64_t s0 = static_cast<int64_t>(tile) * kTTile;
      const int nv = static_cast<int>(min(static_cast<int64_t>(kTTile), f.L - s0));
      // FIR's firing rule on f0 (bounded)
      int ok = 1;
      if (lane == 0) {
        const uint64_t need = (seq + 1) * static_cast<uint64_t>(f.F);
        if (f0_seen < need)
          ok = bounded_wait(p, [&] {
            f0_seen = ld_acquire_u64(&p.ctr[0 * 3 + kCtrWritten]);
            return f0_seen >= need;
          }, kActFir, 0, seq);
      }
      if (!__shfl_sync(0xffffffffu, ok, 0)) {
        if (lane == 0) *stop = 1;
        break;
      }
      const float2 *cur = f.src.frame(k);
      unsigned char *raw = raw0 + s * kWsRawBytes;  // sample s0 - 64 at byte 0
      const uint32_t halo = static_cast<uint32_t>(S) * kTR;        // staged halo samples (<= 64)
      const uint32_t hoff = (kWsRawHalo - halo) * 8;               // halo starts here
      if (tile == 0 && k == 0) {  // delay token (or zeros) as the halo: plain stores
        for (int m = lane; m < static_cast<int>(halo); m += 32) {
          const int d = static_cast<int>(halo) - m;                // samples before s0
          float2 v = make_float2(0.f, 0.f);
          if (d <= f.T - 1 && f.hist) v = f.hist[f.T - 1 - d];
          reinterpret_cast<float2 *>(raw + hoff)[m] = v;
        }
        __syncwarp();
      }
      if (lane == 0) {
        item_raw[s] = WsItem{t, k, tile, nv, 0};
        uint32_t bytes = static_cast<uint32_t>(nv) * 8;
        if (tile > 0) bytes += halo * 8;
        else if (k > 0) bytes += halo * 8;
        mbar_arrive_tx(smem_u32(&raw_full[s]), bytes);
        if (tile > 0) {
          bulk_g2s(smem_u32(raw + hoff), cur + s0 - halo, (halo + static_cast<uint32_t>(nv)) * 8,
                   smem_u32(&raw_full[s]));
        } else {
          bulk_g2s(smem_u32(raw + kWsRawHalo * 8), cur, static_cast<uint32_t>(nv) * 8, smem_u32(&raw_full[s]));
          if (k > 0 && halo > 0)
            bulk_g2s(smem_u32(raw + hoff), f.src.frame(k - 1) + f.L - halo, halo * 8, smem_u32(&raw_full[s]));
        }
      }
      // the delay token after the run: the last T-1 input samples
      if (f.hist_out && k == f.frames - 1 && s0 + nv == f.L)
        for (int m = lane; m < f.T - 1; m += 32) f.hist_out[m] = cur[f.L - (f.T - 1) + m];
    }
    // after a failed wait the converter may not take the last two items: no
    // copy may still write a stage when the CTA leaves (on the normal path
    // both were taken and the waits return at once)
    if (lane == 0) ws_drain_raw(raw_full, i, p.timeout_ns);
  } else if (warp == 1) {
    // ================================================================ MMA
    const uint64_t dbfir = umma_desc_sw128(smem_u32(bfir));
    const uint64_t dlo = static_cast<uint64_t>((kTGroups + S) * 64);  // lo operand after hi
    int sentinels = 0;
    bool issued = false;
    for (uint32_t i = 0; sentinels < kWsGroups; ++i) {
      const int b = i & 1, j = i & 3;
      if (!__all_sync(0xffffffffu, ws_wait(smem_u32(&a_full[b]), (i >> 1) & 1u, p.timeout_ns, stop))) {
        if (lane == 0) fail(kActFir, 11, 0);
        break;
      }
      if (i >= kWsSlots &&
          !__all_sync(0xffffffffu, ws_wait(smem_u32(&slot_empty[j]), ((i >> 2) - 1) & 1u, p.timeout_ns, stop))) {
        if (lane == 0) fail(kActFir, 12, 0);
        break;
      }
      const WsItem it = item_a[b];
      if (lane == 0) {
        item_slot[j] = it;
        if (it.t == kSentinel) {
          mbar_arrive(smem_u32(&fir_full[j]));
          mbar_arrive(smem_u32(&a_empty[b]));
        } else {
          tc_fence_after();
          // Per shift and K step, hi x [B_hi | B_lo] as one N = 128 GEMM
          // (the shift's hi and lo tap operands are adjacent, one 128-row
          // operand) and lo x B_hi as an N = 64 GEMM over its first 64 rows:
          // columns 0-63 collect hi x hi + lo x hi, 64-127 hi x lo.  The
          // lo x lo product (~2^-22 of the result) is left out, as in every
          // three-pass split; the issue count is the same either way.
          // Descriptors advance by adding the byte offset / 16 (all shared
          // addresses are below 2^18 bytes).
          const uint64_t dah = umma_desc_sw128(smem_u32(aop0 + b * kWsAOpBytes));
          const uint32_t d = tmem + static_cast<uint32_t>(j * 128);
          for (int sh = 0; sh < ns; ++sh) {
            const uint64_t ds = dah + static_cast<uint64_t>((S - sh) * 64);  // row group -sh
            const uint64_t db = dbfir + static_cast<uint64_t>(sh * (2 * kTOpBytes / 16));
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
              umma_f16(d, ds + 2 * ks, db + 2 * ks, kTIdescN128, (sh > 0 || ks > 0) ? 1u : 0u);
              umma_f16(d, ds + dlo + 2 * ks, db + 2 * ks, kTIdescN64, 1u);
            }
          }
          umma_commit(smem_u32(&fir_full[j]));
          umma_commit(smem_u32(&a_empty[b]));
          issued = true;
        }
      }
      __syncwarp();
      if (it.t == kSentinel) ++sentinels;
    }
    if (lane == 0 && issued) {  // every GEMM this thread issued has completed
      umma_commit(smem_u32(&fin[0]));
      mbar_wait_bounded(smem_u32(&fin[0]), 0u, p.timeout_ns);
    }
  } else if (warp < kWsEpiWarp0) {
    // ================================================================ converter
    const int ct = tid - 64;  // 0 .. kWsConvThreads - 1
    int sentinels = 0;
    int sx_pred = 0;          // scale exponent of this converter's previous tile
    for (uint32_t i = 0; sentinels < kWsGroups; ++i) {
      const int s = i & 1, b = i & 1;
      // every converter thread waits (it reads what the copies wrote); the
      // outcomes are combined at the barrier that ends the conversion, which
      // the tile path and the sentinel path both reach once (a thread whose
      // wait gave up converts nothing), so the warpgroup leaves together
      const bool okr = ws_wait(smem_u32(&raw_full[s]), (i >> 1) & 1u, p.timeout_ns, stop);
      const bool oka = !okr || i < 2 || ws_wait(smem_u32(&a_empty[b]), ((i >> 1) - 1) & 1u, p.timeout_ns, stop);
      const bool okw = okr && oka;
      WsItem it = item_raw[s];
      const unsigned char *raw = raw0 + s * kWsRawBytes;
      unsigned char *ahi = aop0 + b * kWsAOpBytes;
      unsigned char *alo = ahi + (kTGroups + S) * 1024;
      const int npieces = (kTGroups + S) * 64;
      // cred: [item parity][hi max, FP32 max, spare][converter warp]: no thread
      // rewrites a buffer that another may still read
      uint32_t *cr = cred + (i & 1u) * (3u * kWsConvWarps);
      // kWsConvBatch pieces per thread at a time: all their loads are
      // issued before the first split, so the load latency is paid once per
      // batch.  The pieces are scaled by 2^sx (a multiply by 1 for 2^0: one
      // instantiation keeps the converter's code small, which measured
      // faster than a second, multiply-free copy); the largest FP16 hi part
      // is gathered on the way (one packed max per two components).
      auto convert = [&](int sxc) -> uint32_t {
        const float xsc = exp2i(sxc);
        uint32_t hm = 0u;
        for (int q0 = ct; q0 < npieces; q0 += kWsConvBatch * kWsConvThreads) {
          float4 u[kWsConvBatch][2];
#pragma unroll
          for (int r = 0; r < kWsConvBatch; ++r) {
            const int q = q0 + kWsConvThreads * r;
            const int row = q >> 3, pc = q & 7;
            const int j = 16 * (row & 7) + (row >> 3) - S;  // chunk from the tile start (>= -S)
            if (q < npieces && kTR * j + 4 * pc < it.nv) {
              // the 8 pieces of a row are 32 bytes apart: pieces 4-7 read
              // their halves in the other order, so each quarter-warp load
              // covers all 32 banks once
              const float4 *src = reinterpret_cast<const float4 *>(raw + (kWsRawHalo + kTR * j + 4 * pc) * 8);
              const int sw = (pc >> 2) & 1;
              const float4 a0 = src[sw], a1 = src[sw ^ 1];
              u[r][0] = sw ? a1 : a0;
              u[r][1] = sw ? a0 : a1;
            } else {
              u[r][0] = make_float4(0.f, 0.f, 0.f, 0.f);
              u[r][1] = u[r][0];
            }
          }
#pragma unroll
          for (int r = 0; r < kWsConvBatch; ++r) {
            const int q = q0 + kWsConvThreads * r;
            if (q < npieces) {
              const float2 x2 = make_float2(xsc, xsc);
              const int row = q >> 3, pc = q & 7;
              const uint32_t off = static_cast<uint32_t>(row) * 128u + (static_cast<uint32_t>(pc ^ (row & 7)) << 4);
              uint4 h4, l4;
              split_pair2(__fmul2_rn(make_float2(u[r][0].x, u[r][0].y), x2), h4.x, l4.x);
              split_pair2(__fmul2_rn(make_float2(u[r][0].z, u[r][0].w), x2), h4.y, l4.y);
              split_pair2(__fmul2_rn(make_float2(u[r][1].x, u[r][1].y), x2), h4.z, l4.z);
              split_pair2(__fmul2_rn(make_float2(u[r][1].z, u[r][1].w), x2), h4.w, l4.w);
              hmax_abs_acc(hm, h4.x);
              hmax_abs_acc(hm, h4.y);
              hmax_abs_acc(hm, h4.z);
              hmax_abs_acc(hm, h4.w);
              *reinterpret_cast<uint4 *>(ahi + off) = h4;
              *reinterpret_cast<uint4 *>(alo + off) = l4;
            }
          }
        }
        return hm;
      };
      // the tile split with the exponent predicted from the converter's
      // previous tile
      int sx = sx_pred;
      if (okw && it.t != kSentinel) {
        const uint32_t hm = convert(sx);
        const uint32_t wm = __reduce_max_sync(0xffffffffu, hmax_abs_bits(hm));
        if (lane == 0) cr[warp - 2] = wm;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      }
      if (!bar_and(1, kWsConvThreads, okw)) {
        if (ct == 0) fail(kActFir, okr ? 14 : 13, 0);
        break;
      }
      if (it.t != kSentinel) {
        // the tile's own exponent from its largest hi part; a tile whose
        // own exponent differs from the prediction is converted once more
        // (uniform, rare): the exponent a tile is fired with depends on the
        // tile alone, never on the prediction
        uint32_t hmx = cr[0];
#pragma unroll
        for (int w = 1; w < kWsConvWarps; ++w) hmx = max(hmx, cr[w]);
        int own = tc_shift_from_hi(hmx, sx);
        if (own == -1000) {  // zero, subnormal or inf hi parts: the FP32 maximum decides
          const int halo = S * kTR;
          const float4 *w4 = reinterpret_cast<const float4 *>(raw + (kWsRawHalo - halo) * 8);
          float mx = 0.f;
          for (int q = ct; q < (halo + it.nv) / 2; q += kWsConvThreads) {
            const float4 a = w4[q];
            mx = fmaxf(mx, fmaxf(fmaxf(fabsf(a.x), fabsf(a.y)), fmaxf(fabsf(a.z), fabsf(a.w))));
          }
          const uint32_t fm = __reduce_max_sync(0xffffffffu, __float_as_uint(mx));
          if (lane == 0) cr[kWsConvWarps + warp - 2] = fm;
          asm volatile("bar.sync 1, %0;" ::"n"(kWsConvThreads) : "memory");
          uint32_t fmx = cr[kWsConvWarps];
#pragma unroll
          for (int w = 1; w < kWsConvWarps; ++w) fmx = max(fmx, cr[kWsConvWarps + w]);
          own = tc_shift_bits(fmx);
        }
        if (own != sx) {
          sx = own;
          convert(sx);
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          asm volatile("bar.sync 1, %0;" ::"n"(kWsConvThreads) : "memory");
        }
        it.sx = sx;
        sx_pred = sx;
      }
      if (ct == 0) {
        item_a[b] = it;
        mbar_arrive(smem_u32(&a_full[b]));
        mbar_arrive(smem_u32(&raw_empty[s]));
      }
      if (it.t == kSentinel) ++sentinels;
    }
  } else {
    // ================================================================ epilogue
    const int e = (warp - kWsEpiWarp0) >> 2;    // group 0..2
    const int gt = tid - 32 * kWsEpiWarp0 - 128 * e;  // 0..127
    const int gw = gt >> 5;                     // warp within the group
    const int q4 = warp & 3;                    // TMEM lane quarter of this warp
    const int m = q4 * 32 + lane;               // GEMM row (TMEM lane) owned by this thread
    const int jc = 16 * (m & 7) + (m >> 3);     // output chunk of row m
    const uint32_t tlane = static_cast<uint32_t>(q4 * 32) << 16;
    WsGroup &G = grp[e];
    const int bar = 2 + e;
    auto gsync = [&]() { asm volatile("bar.sync %0, 128;" ::"r"(bar) : "memory"); };
    const int rpb = f.B / kTR;
    // B divides the 4096-sample tile and is a multiple of 32: a power of
    // two, so every division by B or by rows per block is a shift; ring
    // slots take one 64-bit modulo per launch and a subtraction per tile
    const int lgB = __ffs(f.B) - 1, lgR = lgB - 5;
    const RingSlot fring = RingSlot::of(f.yslot.seq0, p.C);   // frame slot of the look-back words
    const RingSlot rring = RingSlot::of(p.rslot.seq0, p.rslot.cap);
    const RingSlot ering = f.energy ? RingSlot::of(f.eslot.seq0, f.eslot.cap) : RingSlot{0, 1};
    constexpr int kHxIssuer = 96;               // lane 0 of the group's last warp
    bool hx_issued = false;
    for (uint32_t i = static_cast<uint32_t>(e);; i += kWsGroups) {
      const int j = i & 3;
      const uint32_t use = i >> 2;
      // every thread waits; the outcomes are combined at the barrier that
      // ends the read-back (a thread whose wait gave up touches no tensor
      // memory and its record is not used), so the group leaves together
      const bool okf = ws_wait(smem_u32(&fir_full[j]), use & 1u, p.timeout_ns, stop);
      const WsItem it = item_slot[j];
      tc_fence_after();
      const int k = it.k, tile = it.tile, nv = it.nv;
      const uint64_t seq = static_cast<uint64_t>(f.yslot.seq0) + k;
      const int rows_valid = nv / kTR;
      const uint32_t slot = tmem + static_cast<uint32_t>(j * 128);
      // ---- FIR rows = columns 0-63 + columns 64-127 (y 2^(sx + s_taps));
      //      energies; each 16-column quarter, times 2^m, split into the HX
      //      operand over the columns 64 + 16 qd .. + 15 it came from (hi in
      //      the first 8, lo in the next 8, two FP16 per column)
      if (okf && it.t != kSentinel) {
        const float hsc = exp2i(tp.m);
        const float2 hsc2 = make_float2(hsc, hsc);
        float2 en2 = make_float2(0.f, 0.f);  // even and odd columns' squares
#pragma unroll 1
        for (int qd = 0; qd < 4; ++qd) {
          float v[16], w[16];
          tmem_ld16(slot + tlane + static_cast<uint32_t>(16 * qd), v);
          tmem_ld16(slot + tlane + static_cast<uint32_t>(64 + 16 * qd), w);
          tmem_ld_wait();
          uint32_t hi[8], lo[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const float2 y = __fadd2_rn(make_float2(v[2 * q], v[2 * q + 1]), make_float2(w[2 * q], w[2 * q + 1]));
            en2 = __ffma2_rn(y, y, en2);
            split_pair2(__fmul2_rn(y, hsc2), hi[q], lo[q]);
          }
          tmem_st8(slot + tlane + static_cast<uint32_t>(64 + 16 * qd), hi);
          tmem_st8(slot + tlane + static_cast<uint32_t>(72 + 16 * qd), lo);
        }
        G.eth[jc] = jc < rows_valid ? mul_pow2(en2.x + en2.y, -2 * (it.sx + tp.s_taps)) : 0.f;
        tmem_st_wait();
      }
      tc_fence_before();
      if (!bar_and(static_cast<uint32_t>(bar), 128, okf)) {
        if (gt == 0) fail(kActFir, 15, 0);
        break;
      }
      if (it.t == kSentinel) break;
      // ---- HX_b GEMM on all 128 rows with its A operand in tensor memory,
      //      issued by the group's last warp while the first runs the block
      //      energies, SEL and the look-back (rows of unselected blocks are
      //      computed and dropped); the issue waits for the tensor pipe's queue
      if (gt == kHxIssuer) {
        tc_fence_after();
        const uint32_t bh = smem_u32(bhx), bl = bh + kTOpBytes;
#pragma unroll 1
        for (int pass = 0; pass < 3; ++pass) {
          const uint32_t pa = slot + (pass == 2 ? 72u : 64u), pb = pass == 1 ? bl : bh;
#pragma unroll
          for (int ks = 0; ks < 4; ++ks)
            umma_f16_ts(slot, pa + static_cast<uint32_t>(16 * ks), umma_desc_sw128(pb + ks * 32), kTIdescN64,
                        (pass > 0 || ks > 0) ? 1u : 0u);
        }
        umma_commit(smem_u32(&hx_full[j]));
        hx_issued = true;
      }
      // ---- block energies (fixed order), DET and SEL on the first warp: a
      //      lane sums 4 rows, the lanes of a block combine by an xor tree
      const int nb = nv >> lgB;
      int cnt_w0 = 0;  // warp 0: selected blocks, known before the look-back
      if (gw == 0) {
        const float4 e4 = reinterpret_cast<const float4 *>(G.eth)[lane];  // rows 4 lane .. 4 lane + 3
        if (rpb >= 4) {  // rpb / 4 lanes per block, nb <= 32
          const int seg = rpb >> 2;
          float sv = (e4.x + e4.y) + (e4.z + e4.w);
          for (int off = 1; off < seg; off <<= 1) sv += __shfl_xor_sync(0xffffffffu, sv, off);
          const float Eb = __shfl_sync(0xffffffffu, sv, (lane * seg) & 31);
          if (lane < nb) G.Et[lane] = Eb;
        } else if (rpb == 2) {
          G.Et[2 * lane] = e4.x + e4.y;
          G.Et[2 * lane + 1] = e4.z + e4.w;
        } else {
          reinterpret_cast<float4 *>(G.Et)[lane] = e4;
        }
        __syncwarp();
        const int64_t eb = f.energy ? static_cast<int64_t>(ering.at(k)) * f.F + tile * (kTTile >> lgB) : 0;
        for (int b0 = 0; b0 < nb; b0 += 32) {
          const int b = b0 + lane;
          const float E = b < nb ? G.Et[b] : 0.f;
          if (f.energy && b < nb) f.energy[eb + b] = E;
          const bool v = b < nb && E > p.tau;
          const unsigned msk = __ballot_sync(0xffffffffu, v);
          if (b < nb) G.rank[b] = v ? cnt_w0 + __popc(msk & ((1u << lane) - 1u)) : -1;
          cnt_w0 += __popc(msk);
        }
        if (lane == 0) G.cnt = cnt_w0;
      }
      // ---- look-back for the tile's offset in the frame (overlaps the GEMM)
      const int64_t fslot = fring.at(k);
      if (gw == 0) {
        const int64_t pr = lookback_warp(p, p.look + fslot * f.tiles, tile, seq + 1, cnt_w0, seq, lane);
        if (lane == 0) G.prefix = pr;
      }
      gsync();
      const int cnt = G.cnt;
      const long long prefix = G.prefix;
      if (prefix < 0 || prefix + cnt > f.F) {
        if (gt == 0 && prefix >= 0) {
          report_error(p.status, kDevInvariant, kActSel, 6, seq);
          atomicExch(&p.ls->abort, 1u);
        }
        if (gt == 0) *stop = 1;
        break;
      }
      const int64_t rs = rring.at(k);
      if (gt < nb && G.rank[gt] >= 0) p.rec_idx[rs * f.F + prefix + G.rank[gt]] = tile * (kTTile >> lgB) + gt;
      // ---- SINK payload: the selected rows at their compacted places (the
      //      wait outcomes are combined at the completion barrier below)
      const bool okh = ws_wait(smem_u32(&hx_full[j]), use & 1u, p.timeout_ns, stop);
      tc_fence_after();
      if (okh && cnt > 0) {
        const int rk = jc < rows_valid ? G.rank[jc >> lgR] : -1;
        float f1, f2;  // HX outputs are H y 2^(sx + s_taps + m + s_h)
        pow2_pair(-(it.sx + tp.s_taps + tp.m + tp.s_h), f1, f2);
#pragma unroll 1
        for (int hf = 0; hf < 2; ++hf) {
          float o[32];
          tmem_ld32(slot + tlane + static_cast<uint32_t>(hf * 32), o);
          tmem_ld_wait();
          if (f2 != 1.f) {  // a scale beyond one float factor (uniform, rare)
#pragma unroll
            for (int q = 0; q < 32; ++q) o[q] *= f2;
          }
          if (rk >= 0) {  // 32-byte stores (whole sectors; the half-row starts 128-byte aligned)
            float *dst = reinterpret_cast<float *>(p.rec_y + rs * f.L + (prefix + rk) * f.B + (jc & (rpb - 1)) * kTR +
                                                   hf * 16);
#pragma unroll
            for (int q = 0; q < 4; ++q) st_global_v8(dst + 8 * q, o + 8 * q, f1);
          }
        }
      }
      // ---- frame completion; the slot goes back to the MMA warp
      tc_fence_before();
      if (!bar_and(static_cast<uint32_t>(bar), 128, okh)) {
        if (gt == 0) fail(kActHx, 7, seq);
        break;
      }
      if (gw == 0) {
        int last = 0;
        if (lane == 0) {
          mbar_arrive(smem_u32(&slot_empty[j]));
          __threadfence();
          const uint32_t old = atomicAdd(&p.done[fslot], 1u);
          if (old + 1u == static_cast<uint32_t>(f.tiles)) {
            ws_publish_frame(p, fslot, rs, seq, f.tiles);
            last = 1;
          }
        }
        if (__shfl_sync(0xffffffffu, last, 0)) drain_bookkeeping(p, static_cast<uint64_t>(f.yslot.seq0) + f.frames, lane);
      }
    }
    if (gt == kHxIssuer && hx_issued) {
      umma_commit(smem_u32(&fin[1 + e]));
      mbar_wait_bounded(smem_u32(&fin[1 + e]), 0u, p.timeout_ns);
    }
  }

  // ---- leave: every role is done (or stopped); free tensor memory
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u) : "memory");
  }
}

}  // namespace prune
