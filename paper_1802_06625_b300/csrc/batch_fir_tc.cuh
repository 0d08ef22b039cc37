// Batched FIR (+ DET energies) on tcgen05: the block-Toeplitz split-FP16
// GEMM of the fused firing loops applied to the tiles of many instances,
// each with its own taps (1 <= T <= 129).  One persistent CTA per SM fires a
// contiguous share, of equal estimated cost, of the batch's (instance,
// 4096-sample tile) items, so an instance's tap operands are loaded into shared memory once per run
// of its tiles.  Four roles run concurrently on different items:
//
//   warp 17      producer: reads each item's instance record once into a
//                shared record, writes the delay token before an instance's
//                first tile, and copies the raw tile and its halo into one of
//                3 stages with bulk copies (up to 3 items ahead);
//   warps 0-7    converter: the tile is read into registers, scaled by the
//                power of two its largest component (halo included) needs
//                (none inside [2^0, 2^15)), and written back over the same
//                stage as the split-FP16 chunk array (same size per sample);
//                on a change of instance, its tap operands are copied in once
//                the GEMMs of the item before have completed;
//   warp 16      issues the FIR GEMMs (per shift and K step, hi x [B_hi|B_lo]
//                as an N = 128 GEMM and lo x B_hi as an N = 64 one: the
//                lo x lo product, ~2^-22 of the result, is left out) into
//                one of four 128-column TMEM accumulators (all 512 columns:
//                the GEMM time per item varies with T, the read-back's does
//                not), hands the item's record on
//                with the accumulator, and frees the stage by a commit once
//                the GEMMs have read it;
//   warps 8-15   read-back: y = the two column halves added, scaled back by
//                2^-(tile exponent + tap exponent), written
//                to the instance's FIR output frame through a per-warp
//                shared-memory transpose (8 rows x 64 contiguous bytes per
//                store instruction), and the block energies (fixed order).
//
// Hand-offs are mbarriers whose phase flips once per use; each wait is on a
// barrier that cannot run two phases ahead of its waiter, so the parity
// names the use.  Every wait is bounded and also returns once the CTA's stop
// flag is set; the converter and the read-back warps each combine the outcome
// of a wait in a barrier with an AND reduction, so a group leaves together.
// The issuing thread commits once more to a barrier of its own and waits
// before tensor memory is freed.
#pragma once
#include <type_traits>

#include "batch_partition.hpp"
#include "batch_types.cuh"
#include "tc_common.cuh"

namespace prune {

constexpr int kBfThreads = 576;                 // converter warps 0-7, read-back 8-15, MMA 16, producer 17
constexpr int kBfWork = 256;                    // threads of one group of 8 warps
constexpr int kBfMmaWarp = 16, kBfProdWarp = 17;
constexpr int kBfMaxShifts = 5;                 // T <= 129
constexpr int kBfRawHalo = 128;                 // samples staged before a tile (S <= 4)
constexpr int kBfStages = 3;
constexpr int kBfAccs = 4;                      // TMEM accumulators of 128 columns
constexpr uint32_t kBfRawBytes = (kBfRawHalo + kTTile) * 8;                     // 33 KB: raw tile + halo
constexpr uint32_t kBfAOpBytes = 2u * (kTGroups + kBfMaxShifts - 1) * 1024;      // 40 KB: chunk array (hi | lo)
constexpr uint32_t kBfStageBytes = kBfAOpBytes > kBfRawBytes ? kBfAOpBytes : kBfRawBytes;
constexpr uint32_t kBfBOpBytes = kBfMaxShifts * 2 * kTOpBytes;                   // 80 KB
constexpr uint32_t kBfMiscBytes = 2048;
constexpr int kBfMaxPieces = (kTGroups + kBfMaxShifts - 1) * 64 / kBfWork;       // per converter thread (5)
constexpr uint32_t kBfXposeBytes = 8 * 2048;                                      // 2 KB per read-back warp
constexpr uint32_t kBfSmemBytes = 1024 + kBfBOpBytes + kBfStages * kBfStageBytes + kBfMiscBytes + kBfXposeBytes;
static_assert(kBfStageBytes % 1024 == 0, "stages stay 1024-byte aligned");
static_assert((kTGroups + kBfMaxShifts - 1) * 64 % kBfWork == 0, "converter pieces divide evenly");

__host__ inline bool batch_fir_tc_supported(int B, int T_max) {
  return B % kTR == 0 && B <= kTTile && kTTile % B == 0 && tc_shifts(T_max) <= kBfMaxShifts;
}

// Barriers over one group of 8 warps (256 threads), named kId (the first
// also ANDs a predicate across the group).
template <int kId>
__device__ __forceinline__ bool bar256_and(bool p) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred a, b;\n setp.ne.u32 a, %1, 0;\n barrier.cta.red.and.pred b, %2, 256, a;\n selp.u32 %0, 1, 0, b;\n}"
      : "=r"(r)
      : "r"(p ? 1u : 0u), "n"(kId)
      : "memory");
  return r != 0;
}
template <int kId>
__device__ __forceinline__ void bar256() {
  asm volatile("bar.sync %0, 256;" ::"n"(kId) : "memory");
}
// The work warps (0-7) of the batched HX kernel.
__device__ __forceinline__ bool bf_bar_and(bool p) { return bar256_and<1>(p); }
__device__ __forceinline__ void bf_bar() { bar256<1>(); }

// Per-item record the producer leaves in shared memory with the stage.
struct BfRec {
  float2 *y;            // the instance's FIR output frame
  float *energy;        // its block energies
  float2 *hout;         // where its delay token after the frame goes (or null)
  const uint16_t *fops; // its tap operands
  int64_t s0, L;        // tile start, frame length (samples)
  int32_t inst, nv, S, T;
  int32_t s_taps, sx;   // the taps' exponent, the tile's (set by the converter)
};
static_assert(sizeof(BfRec) <= 80, "the misc layout holds 3 + 4 records of at most 80 bytes");

static __global__ void __launch_bounds__(kBfThreads, 1) batch_fir_tc_kernel(BatchParams bp) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char *base = smem_align1024(smem_raw);
  unsigned char *bops = base;                       // tap operands of the loaded instance (shift s: hi, lo)
  // stage k: the raw tile (sample s0 - kBfRawHalo at byte 0), then in place
  // the chunk array: hi (16 + S groups of 1024 bytes), then lo
  unsigned char *stage0 = bops + kBfBOpBytes;
  unsigned char *misc = stage0 + kBfStages * kBfStageBytes;
  uint64_t *raw_full = reinterpret_cast<uint64_t *>(misc);  // [3] raw tile landed (and its record)
  uint64_t *a_full = raw_full + kBfStages;                   // [3] chunk array written
  uint64_t *st_free = a_full + kBfStages;                    // [3] the GEMMs reading the stage completed
  uint64_t *mma_done = st_free + kBfStages;                  // [4] GEMMs into accumulator a completed
  uint64_t *acc_empty = mma_done + kBfAccs;                  // [4] accumulator a read back
  uint64_t *fin = acc_empty + kBfAccs;                       // the issuer's last commit, at exit
  uint64_t *b_full = fin + 1;                                // an instance's tap operands landed
  // misc: barriers [0, 152), tmem slot, stop flag, records [176, 416),
  // row energies [512, 1536), accumulator records [1536, 1856), converter
  // maxima [1856, 2048)
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(misc + 160);
  volatile int32_t *stop = reinterpret_cast<volatile int32_t *>(misc + 164);
  BfRec *rec = reinterpret_cast<BfRec *>(misc + 176);        // [3] per stage
  float *eth = reinterpret_cast<float *>(misc + 512);        // [2][128] row energies per column half
  BfRec *acc_rec = reinterpret_cast<BfRec *>(misc + 1536);   // [4] per accumulator
  uint32_t *cred = reinterpret_cast<uint32_t *>(misc + 1856);  // [3 stages][2][8] converter warps' maxima
  float *xpose = reinterpret_cast<float *>(misc + kBfMiscBytes);  // [8 warps][32 rows][16 floats]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int i0 = bp.fir_cta ? bp.fir_cta[blockIdx.x]
                           : static_cast<int>(static_cast<int64_t>(bp.fir_tiles) * blockIdx.x / gridDim.x);
  const int i1 = bp.fir_cta ? bp.fir_cta[blockIdx.x + 1]
                           : static_cast<int>(static_cast<int64_t>(bp.fir_tiles) * (blockIdx.x + 1) / gridDim.x);
  const int n = i1 - i0;
  const int B = bp.B, rpb = B / kTR;
  const int lgB = __ffs(B) - 1;  // B divides the 4096-sample tile and is a multiple of 32: a power of two

  if (tid == 0) {
    for (int q = 0; q < 3 * kBfStages + 2 * kBfAccs + 2; ++q) mbar_init(smem_u32(raw_full + q), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *stop = 0;
  }
  if (warp == kBfMmaWarp) {
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
  auto fail = [&](uint32_t where, uint64_t inst) {
    if (!*stop) report_error(bp.status, kDevTimeout, kActFir, where, inst);
    *stop = 1;
  };

  if (warp == kBfProdWarp) {
    // ================================================================ producer
    int issued = 0;
    for (int i = 0; i < n; ++i) {
      const int st = i % kBfStages;
      if (i >= kBfStages &&
          !__all_sync(0xffffffffu, ws_wait(smem_u32(&st_free[st]), ((i / kBfStages) - 1) & 1, bp.timeout_ns, stop))) {
        if (lane == 0) fail(23, 0);
        break;
      }
      const int2 tm = bp.fir_map[i0 + i];
      const BatchInst &in = bp.inst[tm.x];
      const int T = in.T;
      const int64_t L = static_cast<int64_t>(in.F) * B;
      const int64_t s0 = static_cast<int64_t>(tm.y) * kTTile;
      const int nv = static_cast<int>(min(static_cast<int64_t>(kTTile), L - s0));
      const int S = tc_shifts(T) - 1;
      const uint32_t halo = static_cast<uint32_t>(S) * kTR;     // staged halo samples
      const uint32_t hoff = (kBfRawHalo - halo) * 8;             // halo starts here
      const float2 *cur = in.x ? in.x : bp.x + in.x_off;
      unsigned char *raw = stage0 + st * kBfStageBytes;
      if (tm.y == 0 && halo > 0) {  // the delay token (or zeros) before the first tile
        const float2 *hist = T <= 1 ? nullptr : in.hist ? in.hist + bp.parity * (T - 1) : in.hist_in;
        for (int m = lane; m < static_cast<int>(halo); m += 32) {
          const int dd = static_cast<int>(halo) - m;  // samples before s0
          float2 v = make_float2(0.f, 0.f);
          if (dd <= T - 1 && hist) v = hist[T - 1 - dd];
          reinterpret_cast<float2 *>(raw + hoff)[m] = v;
        }
      }
      if (lane == 0) {
        BfRec r;
        r.y = in.y;
        r.energy = in.energy;
        r.hout = T <= 1 ? nullptr : in.hist ? in.hist + (1 - bp.parity) * (T - 1) : in.hist_out;
        r.fops = in.fops;
        r.s0 = s0;
        r.L = L;
        r.inst = tm.x;
        r.nv = nv;
        r.S = S;
        r.T = T;
        r.s_taps = in.s_taps;
        r.sx = 0;
        rec[st] = r;
      }
      __syncwarp();
      if (lane == 0) {
        const uint32_t bytes = static_cast<uint32_t>(nv) * 8 + (tm.y > 0 ? halo * 8 : 0u);
        mbar_arrive_tx(smem_u32(&raw_full[st]), bytes);
        if (tm.y > 0)
          bulk_g2s(smem_u32(raw + hoff), cur + s0 - halo, (halo + static_cast<uint32_t>(nv)) * 8,
                   smem_u32(&raw_full[st]));
        else
          bulk_g2s(smem_u32(raw + kBfRawHalo * 8), cur, static_cast<uint32_t>(nv) * 8, smem_u32(&raw_full[st]));
      }
      ++issued;
    }
    // no copy may still write a stage when the CTA leaves
    if (lane == 0)
      for (int i = max(0, issued - kBfStages); i < issued; ++i)
        mbar_wait_bounded(smem_u32(&raw_full[i % kBfStages]), (i / kBfStages) & 1, bp.timeout_ns);
    __syncwarp();
  } else if (warp == kBfMmaWarp) {
    // ================================================================ MMA
    if (lane == 0) {
      bool any = false;
      for (int i = 0; i < n; ++i) {
        const int st = i % kBfStages;
        if (!ws_wait(smem_u32(&a_full[st]), (i / kBfStages) & 1, bp.timeout_ns, stop)) {
          fail(20, 0);
          break;
        }
        if (i >= kBfAccs && !ws_wait(smem_u32(&acc_empty[i % kBfAccs]), ((i / kBfAccs) - 1) & 1, bp.timeout_ns, stop)) {
          fail(21, 0);
          break;
        }
        tc_fence_after();
        const BfRec r = rec[st];
        acc_rec[i % kBfAccs] = r;  // read back once the GEMMs complete
        const int S = r.S;
        const uint64_t dah = umma_desc_sw128(smem_u32(stage0 + st * kBfStageBytes));
        const uint64_t dlo = static_cast<uint64_t>((kTGroups + S) * 64);  // lo array after hi
        const uint64_t dbf = umma_desc_sw128(smem_u32(bops));
        const uint32_t d = tmem + static_cast<uint32_t>((i % kBfAccs) * 128);
        for (int sh = 0; sh <= S; ++sh) {
          const uint64_t ds = dah + static_cast<uint64_t>((S - sh) * 64);  // row group -sh
          const uint64_t db = dbf + static_cast<uint64_t>(sh * (2 * kTOpBytes / 16));
#pragma unroll
          for (int ks = 0; ks < 4; ++ks) {
            umma_f16(d, ds + 2 * ks, db + 2 * ks, kTIdescN128, (sh > 0 || ks > 0) ? 1u : 0u);
            umma_f16(d, ds + dlo + 2 * ks, db + 2 * ks, kTIdescN64, 1u);  // lo x B_hi only
          }
        }
        umma_commit(smem_u32(&mma_done[i % kBfAccs]));
        umma_commit(smem_u32(&st_free[st]));
        any = true;
      }
      if (any) {  // every GEMM this thread issued has completed
        umma_commit(smem_u32(fin));
        mbar_wait_bounded(smem_u32(fin), 0u, bp.timeout_ns);
      }
    }
    __syncwarp();
  } else if (warp < 8) {
    // ================================================================ converter
    int loaded = -1;
    uint32_t b_par = 0;
    bool reload_open = false;  // a tap copy issued and not yet seen to land
    int sx_pred = 0;           // scale exponent of the group's previous tile
    // bounded wait by every thread of the group, outcome combined
    auto wait_all = [&](uint64_t *mb, uint32_t par) -> bool {
      const bool w = ws_wait(smem_u32(mb), par, bp.timeout_ns, stop);
      return bar256_and<1>(w && !*stop);
    };
    bool ok = true;
    for (int i = 0; i < n; ++i) {
      const int st = i % kBfStages;
      ok = wait_all(&raw_full[st], (i / kBfStages) & 1);
      if (!ok) break;
      const BfRec r = rec[st];
      const int S = r.S, nv = r.nv;
      const bool reload = r.inst != loaded;
      if (reload) {  // this instance's tap operands by bulk copy, once no GEMM reads the old ones
        if (i > 0) {  // item i-1's stage freed: every GEMM up to item i-1 has completed
          const int sp = (i - 1) % kBfStages;
          ok = wait_all(&st_free[sp], ((i - 1) / kBfStages) & 1);
          if (!ok) break;
        }
        if (tid == 0) {
          mbar_arrive_tx(smem_u32(b_full), static_cast<uint32_t>(S + 1) * 2 * kTOpBytes);
          for (int sh = 0; sh <= S; ++sh)
            bulk_g2s(smem_u32(bops + sh * 2 * kTOpBytes), r.fops + static_cast<size_t>(sh) * 2 * 64 * 64,
                     2 * kTOpBytes, smem_u32(b_full));
        }
        reload_open = true;
        loaded = r.inst;
      }
      // the tile as the permuted split-FP16 chunk array (the fused loops'
      // layout), written over the raw tile once every thread has read it
      unsigned char *stg = stage0 + st * kBfStageBytes;
      const int npieces = (kTGroups + S) * 64;
      float4 u[kBfMaxPieces][2];
#pragma unroll
      for (int k = 0; k < kBfMaxPieces; ++k) {
        const int q = tid + kBfWork * k;
        const int row = q >> 3, pc = q & 7;
        const int j = 16 * (row & 7) + (row >> 3) - S;  // chunk from the tile start (>= -S)
        if (q < npieces && kTR * j + 4 * pc < nv) {
          // pieces 4-7 read their halves in the other order (bank-conflict free)
          const float4 *src = reinterpret_cast<const float4 *>(stg + (kBfRawHalo + kTR * j + 4 * pc) * 8);
          const int sw = (pc >> 2) & 1;
          const float4 a0 = src[sw], a1 = src[sw ^ 1];
          u[k][0] = sw ? a1 : a0;
          u[k][1] = sw ? a0 : a1;
        } else {
          u[k][0] = make_float4(0.f, 0.f, 0.f, 0.f);
          u[k][1] = u[k][0];
        }
      }
      // the delay token after the frame: its last T-1 input samples
      if (r.hout && r.s0 + nv == r.L)
        for (int m = tid; m < r.T - 1; m += kBfWork)
          r.hout[m] = reinterpret_cast<const float2 *>(stg)[kBfRawHalo + nv - (r.T - 1) + m];
      bar256<1>();  // every raw sample of the stage has been read
      // the tile as the split-FP16 chunk array, scaled by 2^sx, sx predicted
      // from this group's previous tile (no multiply when it is 0); the
      // largest FP16 hi part, exchanged through the barrier that ends the
      // conversion, gives the tile's own exponent, and a tile whose own
      // exponent differs is split once more from the registers (uniform,
      // rare): the exponent a tile is fired with depends on the tile alone
      unsigned char *ahi = stg, *alo = stg + (kTGroups + S) * 1024;
      auto split_all = [&](int sxc) -> uint32_t {
        const float xsc = exp2i(sxc);
        uint32_t hm = 0u;
#pragma unroll
        for (int k = 0; k < kBfMaxPieces; ++k) {
          const int q = tid + kBfWork * k;
          if (q < npieces) {
            const int row = q >> 3, pc = q & 7;
            const uint32_t off = static_cast<uint32_t>(row) * 128u + (static_cast<uint32_t>(pc ^ (row & 7)) << 4);
            const float4 a = u[k][0], c = u[k][1];
            // scaled by 2^sxc (a multiply by 1 for 2^0: one instantiation keeps the code small)
            const float2 x2 = make_float2(xsc, xsc);
            uint4 h4, l4;
            split_pair2(__fmul2_rn(make_float2(a.x, a.y), x2), h4.x, l4.x);
            split_pair2(__fmul2_rn(make_float2(a.z, a.w), x2), h4.y, l4.y);
            split_pair2(__fmul2_rn(make_float2(c.x, c.y), x2), h4.z, l4.z);
            split_pair2(__fmul2_rn(make_float2(c.z, c.w), x2), h4.w, l4.w);
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
      // cred: [stage][hi max of pass 0, FP32 max][8 warps]
      uint32_t *cr = cred + st * 16;
      int sx = sx_pred;
      {
        const uint32_t hm = split_all(sx);
        const uint32_t wm = __reduce_max_sync(0xffffffffu, hmax_abs_bits(hm));
        if (lane == 0) cr[warp] = wm;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      if (reload) {  // the tap operands (copied while the tile was converted)
        ok = wait_all(b_full, b_par);
        if (!ok) break;
        b_par ^= 1u;
        reload_open = false;
      } else {
        bar256<1>();
      }
      {
        uint32_t h16 = cr[0];
#pragma unroll
        for (int w = 1; w < 8; ++w) h16 = max(h16, cr[w]);
        int own = tc_shift_from_hi(h16, sx);
        if (own == -1000) {  // zero, subnormal or inf hi parts: the FP32 maximum decides
          float mx = 0.f;
#pragma unroll
          for (int k = 0; k < kBfMaxPieces; ++k)
#pragma unroll
            for (int h = 0; h < 2; ++h)
              mx = fmaxf(mx, fmaxf(fmaxf(fabsf(u[k][h].x), fabsf(u[k][h].y)), fmaxf(fabsf(u[k][h].z), fabsf(u[k][h].w))));
          const uint32_t fm = __reduce_max_sync(0xffffffffu, __float_as_uint(mx));
          if (lane == 0) cr[8 + warp] = fm;
          bar256<1>();
          uint32_t f32 = cr[8];
#pragma unroll
          for (int w = 1; w < 8; ++w) f32 = max(f32, cr[8 + w]);
          own = tc_shift_bits(f32);
        }
        if (own != sx) {
          sx = own;
          split_all(sx);
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          bar256<1>();
        }
        sx_pred = sx;
      }
      if (tid == 0) rec[st].sx = sx;  // read by the MMA warp after a_full
      if (tid == 0) mbar_arrive(smem_u32(&a_full[st]));
    }
    // a tap reload whose copy was not seen to land (the group left on a
    // failed wait): no copy may still write shared memory when the CTA leaves
    if (!ok && tid == 0) {
      fail(22, 0);
      if (reload_open) mbar_wait_bounded(smem_u32(b_full), b_par, bp.timeout_ns);
    }
  } else {
    // ================================================================ read-back
    const int et = tid - kBfWork, ew = warp - 8;   // 0..255, 0..7
    const int q4 = warp & 3, hf = ew >> 2;          // TMEM lane quarter, output half (16 complex)
    const int m = q4 * 32 + lane;                   // GEMM row: output chunk jc
    const int jc = 16 * (m & 7) + (m >> 3);
    float *wx = xpose + ew * 512;
    auto wait_all = [&](uint64_t *mb, uint32_t par) -> bool {
      const bool w = ws_wait(smem_u32(mb), par, bp.timeout_ns, stop);
      return bar256_and<2>(w && !*stop);
    };
    bool ok = true;
    for (int i = 0; i < n; ++i) {
      const int a = i % kBfAccs;
      ok = wait_all(&mma_done[a], (i / kBfAccs) & 1);
      if (!ok) break;
      tc_fence_after();
      // accumulator of item i: y = (hi part + lo part) 2^-(sx + s_taps) to
      // the FIR output frame, row energies, then the block energies in a
      // fixed order
      const BfRec r = acc_rec[a];
      const int rows_valid = r.nv / kTR;
      const uint32_t ta = tmem + (static_cast<uint32_t>(q4 * 32) << 16) + static_cast<uint32_t>(a * 128 + hf * 32);
      float v[32], w[32];
      tmem_ld32(ta, v);
      tmem_ld32(ta + 64u, w);
      tmem_ld_wait();
      float e = 0.f;
      float f1, f2;
      pow2_pair(-(r.sx + r.s_taps), f1, f2);
#pragma unroll
      for (int q = 0; q < 32; q += 2) {
        const float2 s = __fadd2_rn(make_float2(v[q], v[q + 1]), make_float2(w[q], w[q + 1]));
        v[q] = s.x;
        v[q + 1] = s.y;
      }
      if (f2 != 1.f) {  // a scale beyond one float factor (uniform, rare)
#pragma unroll
        for (int q = 0; q < 32; ++q) v[q] *= f2;
      }
      float2 e2 = make_float2(0.f, 0.f);  // even and odd columns' squares
#pragma unroll
      for (int q = 0; q < 32; q += 2) {
        const float2 s = __fmul2_rn(make_float2(v[q], v[q + 1]), make_float2(f1, f1));
        v[q] = s.x;
        v[q + 1] = s.y;
        e2 = __ffma2_rn(s, s, e2);
      }
      e = e2.x + e2.y;
      // the accumulator is free once every thread has its rows
      tc_fence_before();
      bar256<2>();
      if (et == 0) mbar_arrive(smem_u32(&acc_empty[a]));
      eth[hf * 128 + jc] = jc < rows_valid ? e : 0.f;
      // y through a per-warp transpose: a store instruction then writes 8
      // rows x 64 contiguous bytes instead of 32 rows x 16 bytes.  Chunk f
      // of row x sits at chunk f ^ ((x >> 1) & 3): conflict-free both ways.
#pragma unroll
      for (int h2 = 0; h2 < 2; ++h2) {
#pragma unroll
        for (int f = 0; f < 4; ++f)
          *reinterpret_cast<float4 *>(wx + lane * 16 + ((f ^ ((lane >> 1) & 3)) << 2)) =
              make_float4(v[16 * h2 + 4 * f], v[16 * h2 + 4 * f + 1], v[16 * h2 + 4 * f + 2], v[16 * h2 + 4 * f + 3]);
        __syncwarp();
#pragma unroll
        for (int e4 = 0; e4 < 4; ++e4) {
          const int x = 8 * e4 + (lane >> 2), fq = lane & 3;  // row of the warp, 16-byte chunk
          const float4 val = *reinterpret_cast<const float4 *>(wx + x * 16 + ((fq ^ ((x >> 1) & 3)) << 2));
          const int mx = q4 * 32 + x, jx = 16 * (mx & 7) + (mx >> 3);
          if (jx < rows_valid)
            *reinterpret_cast<float4 *>(r.y + r.s0 + kTR * jx + 16 * hf + 2 * (4 * h2 + fq)) = val;
        }
        __syncwarp();
      }
      bar256<2>();  // every row energy is in eth
      const int nb = r.nv >> lgB;
      if (et < nb) {
        float E = 0.f;
        for (int k = 0; k < rpb; ++k) {
          const int c = et * rpb + k;
          E += eth[c] + eth[128 + c];
        }
        r.energy[(r.s0 >> lgB) + et] = E;
      }
    }
    if (!ok && et == 0) fail(24, 0);
  }

  // ---- leave: every role is done (or stopped); free tensor memory
  tc_fence_before();
  __syncthreads();
  if (warp == kBfMmaWarp) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u) : "memory");
  }
}

}  // namespace prune
