// HX_b static actors on the 5th-generation tensor cores (tcgen05), N = 64.
//
// Each selected block is B/N rows x of N complex samples; HX_b maps every
// row to H x.  As a real GEMM over all selected rows of a frame:
//   D[m][n] = sum_k A[m][k] R[n][k],  k, n < 2N,
// where A's row m is the row x as stored (re, im interleaved: K-major, no
// transpose) and R is the real form of H:
//   R[2i][2k] = Re H[i][k],  R[2i][2k+1] = -Im H[i][k],
//   R[2i+1][2k] = Im H[i][k], R[2i+1][2k+1] = Re H[i][k],
// so D's row m is H x interleaved again.  FP32 accuracy from FP16 tensor
// cores: every operand is split a = a_hi + a_lo (a_hi = fp16(a),
// a_lo = fp16(a - a_hi)) and D = A_hi R_hi + A_hi R_lo + A_lo R_hi with FP32
// accumulation in tensor memory (the dropped A_lo R_lo term is ~2^-22
// relative).  Both operands are scaled by powers of two before the split
// (tc_scale.cuh): R once per graph by 2^s_h (its largest component in
// [2^14, 2^15)), each row of A by its own 2^s_row (likewise: HX is applied
// row by row, so a row's scale is exact to undo); the epilogue multiplies the
// row's outputs by 2^-(s_row + s_h).
//
// Tile: M = 128 rows of selected blocks (gathered through the control
// token's idx, read on the device), N = 128, K = 128; 3 x 8 MMAs of
// 128x128x16 (kind::f16) issued by one thread, completion through
// tcgen05.commit on an mbarrier.  Operands live in shared memory in the
// K-major 128-byte-swizzle layout; R is converted once per graph and copied
// into each persistent CTA once.  Accumulators: 128 TMEM columns.
#pragma once
#include <cuda_fp16.h>

#include "hx_cuda.cuh"
#include "tc_scale.cuh"

namespace prune {

constexpr int kTcThreads = 256;
constexpr int kTcNc = 64;               // complex N handled on tensor cores
constexpr int kTcM = 128;               // rows per tile
constexpr int kTcK = 2 * kTcNc;         // 128 real
constexpr int kTcNg = 2 * kTcNc;        // 128 real outputs
constexpr uint32_t kTcOpBytes = kTcM * kTcK * 2;  // 32 KB per operand half
constexpr uint32_t kTcSmemBytes = 4 * kTcOpBytes + 64 + 512 + 1024;  // operands, misc, row exponents, alignment

__host__ __device__ inline bool hx_tc_supported(int N) { return N == kTcNc; }
__host__ inline size_t hx_tc_b_elems(int N) { return 2 * static_cast<size_t>(2 * N) * (2 * N); }

// Byte offset of element (row, k) of a K-major operand with `rows` rows in
// the 128-byte swizzle layout: atoms of 64 K-elements; 128 bytes per row;
// 16-byte chunk c of row r stored at chunk c ^ (r mod 8).
__host__ __device__ __forceinline__ uint32_t sw128_off(int row, int k, int rows) {
  return static_cast<uint32_t>((k >> 6) * rows * 128 + row * 128 + ((((k & 63) >> 3) ^ (row & 7)) << 4) +
                               ((k & 7) << 1));
}

// R scaled by 2^sh (TcScale::s_h; *sh_dev when that is not null), split
// into hi / lo FP16 in the shared-memory layout.
static __global__ void hx_tc_prepare_b_kernel(const float2 *H, int sh, const int32_t *sh_dev, uint16_t *bops) {
  if (sh_dev) sh = *sh_dev;
  const int n = blockIdx.x, k = threadIdx.x;  // 128 x 128
  const int i = n >> 1, kk = k >> 1;
  const float2 h = H[i * kTcNc + kk];
  float v;
  if ((n & 1) == 0) v = (k & 1) == 0 ? h.x : -h.y;
  else v = (k & 1) == 0 ? h.y : h.x;
  v *= exp2i(sh);
  const __half hi = __float2half_rn(v);
  const __half lo = __float2half_rn(v - __half2float(hi));
  const uint32_t off = sw128_off(n, k, kTcNg) >> 1;
  bops[off] = __half_as_ushort(hi);
  bops[kTcNg * kTcK + off] = __half_as_ushort(lo);
}

__host__ inline cudaError_t hx_tc_prepare_b(const float2 *H, int N, int sh, const int32_t *sh_dev, uint16_t *bops,
                                            cudaStream_t s) {
  if (!hx_tc_supported(N)) return cudaErrorInvalidValue;
  hx_tc_prepare_b_kernel<<<kTcNg, kTcK, 0, s>>>(H, sh, sh_dev, bops);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- PTX
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
// The dynamic shared memory base rounded up to a 1024-byte boundary (the
// 128-byte-swizzle operands need it) by pointer arithmetic on the shared
// array itself: pointers derived from it stay shared-memory pointers, so
// accesses through them are shared-memory accesses, not generic ones (a
// round trip through an integer hides the address space from the compiler).
__device__ __forceinline__ unsigned char *smem_align1024(unsigned char *p) {
  return p + ((1024u - (smem_u32(p) & 1023u)) & 1023u);
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (SBO), LBO unused for this layout (1), descriptor
// version 1, base offset 0 (atoms are 1024-byte aligned).
__device__ __forceinline__ uint64_t umma_desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr >> 4) & 0x3FFFu);
  d |= static_cast<uint64_t>(1u) << 16;
  d |= static_cast<uint64_t>(1024u >> 4) << 32;
  d |= static_cast<uint64_t>(1u) << 46;
  d |= static_cast<uint64_t>(2u) << 61;
  return d;
}

// Instruction descriptor, kind::f16: D = F32, A = B = F16, both K-major,
// N = 128 (bits 17-22: N >> 3), M = 128 (bits 24-28: M >> 4).
constexpr uint32_t kTcIdesc = (1u << 4) | (static_cast<uint32_t>(kTcNg >> 3) << 17) |
                              (static_cast<uint32_t>(kTcM >> 4) << 24);

__device__ __forceinline__ void mbar_init(uint32_t addr, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(addr), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t addr, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(addr), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase with the given parity.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t addr, uint32_t parity, uint64_t timeout_ns) {
  if (mbar_try_wait(addr, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try_wait(addr, parity)) return true;
    if ((it & 127u) == 0u && globaltimer_ns() - t0 > timeout_ns) return false;
  }
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void umma_f16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

// 32 lanes x 16 consecutive 32-bit columns per warp.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ uint4 split_pack(const float (&v)[8], bool lo) {
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

struct HxTcParams {
  HxParams p;
  const uint16_t *bops;   // R hi | R lo in the swizzled layout (R scaled by 2^s_h)
  int32_t s_h;
  const int32_t *s_h_dev; // when not null, s_h is read from the device here
  int32_t tiles_per_frame;
  uint64_t timeout_ns;
};

static __global__ void __launch_bounds__(kTcThreads, 1) hx_tc_kernel(HxTcParams tp) {
  extern __shared__ unsigned char smem_raw[];
  const HxParams &p = tp.p;
  unsigned char *base = smem_align1024(smem_raw);
  unsigned char *a_hi = base, *a_lo = base + kTcOpBytes;
  unsigned char *b_hi = base + 2 * kTcOpBytes, *b_lo = base + 3 * kTcOpBytes;
  uint64_t *mbar = reinterpret_cast<uint64_t *>(base + 4 * kTcOpBytes);
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(base + 4 * kTcOpBytes + 8);
  int32_t *s_flag = reinterpret_cast<int32_t *>(base + 4 * kTcOpBytes + 16);
  int32_t *s_row = reinterpret_cast<int32_t *>(base + 4 * kTcOpBytes + 64);  // [128] row exponents

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int RB = p.B / kTcNc;  // rows per block
  const int s_h = tp.s_h_dev ? *tp.s_h_dev : tp.s_h;

  // R operands: once per CTA
  {
    const uint4 *src = reinterpret_cast<const uint4 *>(tp.bops);
    uint4 *dst = reinterpret_cast<uint4 *>(b_hi);  // b_hi and b_lo are contiguous
    for (int q = tid; q < static_cast<int>(2 * kTcOpBytes / 16); q += kTcThreads) dst[q] = src[q];
  }
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
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  uint32_t phase = 0;

  const int64_t total = static_cast<int64_t>(p.frames) * tp.tiles_per_frame;
  for (int64_t w = blockIdx.x; w < total; w += gridDim.x) {
    const int k = static_cast<int>(w / tp.tiles_per_frame);
    const int tau = static_cast<int>(w % tp.tiles_per_frame);
    const int64_t rs = p.rslot.slot(k);
    const int ck = min(max(p.c[rs], 0), p.F);
    if (tau == 0 && tid == 0 && p.ctr) hx_bookkeeping(p, k, ck);
    const int rows = ck * RB;
    if (tau * kTcM >= rows) continue;  // uniform: control token read on the device
    const float2 *yk = p.y + p.yslot.slot(k) * p.y_stride;
    const int32_t *idxk = p.idx + rs * p.F;

    // A: 128 gathered rows, each scaled by its own power of two, split hi /
    // lo, swizzled (16 chunks of 8 per row: the 16 lanes of a half-warp hold
    // one row, whose largest component they reduce by shuffles)
    for (int q = tid; q < kTcM * (kTcK / 8); q += kTcThreads) {
      const int m = q >> 4, cc = q & 15;
      const int gr = tau * kTcM + m;
      float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      if (gr < rows) {
        const int j = gr / RB, r = gr % RB;
        const int b = idxk[j];
        if (b >= 0 && b < p.F) {
          const float4 *src = reinterpret_cast<const float4 *>(yk + static_cast<int64_t>(b) * p.B + r * kTcNc) + cc * 2;
          const float4 u0 = __ldg(src), u1 = __ldg(src + 1);
          v[0] = u0.x; v[1] = u0.y; v[2] = u0.z; v[3] = u0.w;
          v[4] = u1.x; v[5] = u1.y; v[6] = u1.z; v[7] = u1.w;
        }
      }
      float mx = 0.f;
#pragma unroll
      for (int e = 0; e < 8; ++e) mx = fmaxf(mx, fabsf(v[e]));
#pragma unroll
      for (int o = 1; o < 16; o <<= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      const int sr = tc_pow2_shift(mx);
      const float sc = exp2i(sr);
#pragma unroll
      for (int e = 0; e < 8; ++e) v[e] *= sc;
      if (cc == 0) s_row[m] = sr;
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
      for (int pass = 0; pass < 3; ++pass) {
#pragma unroll
        for (int ks = 0; ks < kTcK / 16; ++ks) {
          const uint32_t koff = static_cast<uint32_t>((ks >> 2) * kTcM * 128 + (ks & 3) * 32);
          const uint32_t kboff = static_cast<uint32_t>((ks >> 2) * kTcNg * 128 + (ks & 3) * 32);
          umma_f16(tmem, umma_desc_sw128(pa[pass] + koff), umma_desc_sw128(pb[pass] + kboff), kTcIdesc,
                   (pass > 0 || ks > 0) ? 1u : 0u);
        }
      }
      umma_commit(smem_u32(mbar));
    }
    const bool ok = mbar_wait_bounded(smem_u32(mbar), phase, tp.timeout_ns);
    phase ^= 1u;
    if (!ok) {
      if (tid == 0) report_error(p.status, kDevTimeout, kActHx, 7, p.rslot.seq0 + k);
      *s_flag = 1;  // benign race: every writer stores 1
    }
    __syncthreads();
    if (*s_flag) break;
    tc_fence_after();

    // epilogue: warp quarter q reads TMEM lanes 32q..32q+31 (tile rows),
    // warp half h the 64 columns [64h, 64h+64)
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
        float4 *dst = reinterpret_cast<float4 *>(p.out + p.oslot.slot(k) * p.out_stride + static_cast<int64_t>(j) * p.B +
                                                 r * kTcNc + hf * 32);
        float f1, f2;
        pow2_pair(-(s_row[m] + s_h), f1, f2);
#pragma unroll
        for (int e = 0; e < 16; ++e)
          dst[e] = make_float4(v[4 * e] * f1 * f2, v[4 * e + 1] * f1 * f2, v[4 * e + 2] * f1 * f2,
                               v[4 * e + 3] * f1 * f2);
      }
    }
    tc_fence_before();
    __syncthreads();
  }

  // On a timeout, give the MMAs in flight one more bounded chance to land
  // before the accumulator columns are released.
  if (*s_flag) mbar_wait_bounded(smem_u32(mbar), phase ^ 1u, tp.timeout_ns);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128u) : "memory");
  }
}

__host__ inline cudaError_t launch_hx_tc(const HxParams &p, const uint16_t *bops, int s_h, const int32_t *s_h_dev,
                                         int sms, cudaStream_t s, uint64_t timeout_ns = 2000000000ull) {
  if (!hx_tc_supported(p.N)) return cudaErrorInvalidValue;
  HxTcParams tp{};
  tp.p = p;
  tp.bops = bops;
  tp.s_h = s_h;
  tp.s_h_dev = s_h_dev;
  const int64_t rows_max = static_cast<int64_t>(p.F) * (p.B / kTcNc);
  tp.tiles_per_frame = static_cast<int32_t>((rows_max + kTcM - 1) / kTcM);
  tp.timeout_ns = timeout_ns;
  cudaError_t e = cudaFuncSetAttribute(hx_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(kTcSmemBytes));
  if (e != cudaSuccess) return e;
  const int64_t work = static_cast<int64_t>(p.frames) * tp.tiles_per_frame;
  const int grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(work, sms)));
  hx_tc_kernel<<<grid, kTcThreads, kTcSmemBytes, s>>>(tp);
  return cudaGetLastError();
}

}  // namespace prune
