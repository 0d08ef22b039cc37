// Shared pieces of the tensor-core FIR kernels (the fused firing loops and
// the batched FIR): the block-Toeplitz tile geometry, the tap and H operand
// builders, and the tcgen05 / mbarrier / bulk-copy helpers.
//
// A tile is 128 GEMM rows of 32 consecutive complex outputs (4096 outputs).
// With G_s[i][u] = h[i - u + 32 s] (zero outside 0 <= i - u + 32 s < T) the
// outputs of row m are y_m = sum_{s=0}^{S} G_s X_{m-s}, S = ceil((T-1)/32),
// X_j the j-th 32-sample input chunk from the tile start: the convolution
// y[n] = sum_t h[t] x[n-t] regrouped.  Each G_s is used in its real form
// (64 x 64) split into FP16 hi and lo parts.
//
// Range.  FP16 holds magnitudes in [2^-14, 65504] at full precision, FP32
// far more, so every operand is scaled by a power of two (exact) before it
// is split (tc_scale.cuh): the taps and H once per graph, each input tile
// (with its halo) by the exponent its largest component needs, and the FIR
// output by a per-graph 2^m from the L1 bound of the taps so that the HX
// operand stays below 2^14.  Results are scaled back in the epilogues (again
// exact), so the split keeps ~2^-21 relative precision independent of the
// signal's level.
#pragma once
#include <cuda_fp16.h>

#include "hx_tc.cuh"

namespace prune {

constexpr int kTR = 32;                  // complex outputs per GEMM row
constexpr int kTRows = 128;              // GEMM rows per tile (M)
constexpr int kTTile = kTR * kTRows;     // 4096 outputs per tile
constexpr int kTMaxShifts = 5;           // T <= 4 * 32 + 1
constexpr int kTGroups = kTRows / 8;     // 8-row groups of one GEMM operand (16)
constexpr int kTMaxPieces = (kTGroups + kTMaxShifts - 1) * 64 / 256;  // per thread (5)
constexpr uint32_t kTOpBytes = 64 * 128; // one 64 x 64 FP16 operand (8 KB)
constexpr uint32_t kTIdescN64 = (1u << 4) | (static_cast<uint32_t>(64 >> 3) << 17) |
                                (static_cast<uint32_t>(kTRows >> 4) << 24);
__host__ __device__ inline int tc_shifts(int T) { return 1 + (T - 1 + kTR - 1) / kTR; }

constexpr uint32_t kTIdescN128 = (1u << 4) | (static_cast<uint32_t>(128 >> 3) << 17) |
                                 (static_cast<uint32_t>(kTRows >> 4) << 24);

// Operand elements: ns shifts x {hi, lo} x 64 x 64 for FIR, {hi, lo} x 64 x 64 for HX.
__host__ inline size_t tc_fir_ops_elems(int T) { return static_cast<size_t>(tc_shifts(T)) * 2 * 64 * 64; }
__host__ inline size_t tc_hx_ops_elems() { return 2 * 64 * 64; }

// Real form of a 32 x 32 complex matrix M (element getter) at row n, column k.
__device__ __forceinline__ float real_form(float2 g, int n, int k) {
  if ((n & 1) == 0) return (k & 1) == 0 ? g.x : -g.y;
  return (k & 1) == 0 ? g.y : g.x;
}

// v (already scaled) as FP16 hi = fp16(v) and lo = fp16(v - hi).
__device__ __forceinline__ void store_split(uint16_t *ops, uint32_t half_elems, int n, int k, float v) {
  const __half hi = __float2half_rn(v);
  const __half lo = __float2half_rn(v - __half2float(hi));
  const uint32_t off = sw128_off(n, k, 64) >> 1;
  ops[off] = __half_as_ushort(hi);
  ops[half_elems + off] = __half_as_ushort(lo);
}

// FIR operands: shift s, real row n < 64 (output 2i+a), real column k < 64,
// of the taps scaled by 2^sh (TcScale::s_taps).
static __global__ void tc_prepare_fir_kernel(const float2 *taps, int T, int sh, uint16_t *ops) {
  const int s = blockIdx.y, n = blockIdx.x, k = threadIdx.x;
  const int i = n >> 1, u = k >> 1;
  const int t = i - u + kTR * s;
  const float2 g = (t >= 0 && t < T) ? taps[t] : make_float2(0.f, 0.f);
  store_split(ops + static_cast<size_t>(s) * 2 * 64 * 64, 64 * 64, n, k, real_form(g, n, k) * exp2i(sh));
}

// HX operands: real form of H (32 x 32 complex) scaled by 2^sh (TcScale::s_h).
static __global__ void tc_prepare_hx_kernel(const float2 *H, int sh, uint16_t *ops) {
  const int n = blockIdx.x, k = threadIdx.x;
  store_split(ops, 64 * 64, n, k, real_form(H[(n >> 1) * kTR + (k >> 1)], n, k) * exp2i(sh));
}

__host__ inline cudaError_t tc_prepare_ops(const float2 *taps, int T, const float2 *H, const TcScale &sc,
                                           uint16_t *fir_ops, uint16_t *hx_ops, cudaStream_t s) {
  tc_prepare_fir_kernel<<<dim3(64, tc_shifts(T)), 64, 0, s>>>(taps, T, sc.s_taps, fir_ops);
  tc_prepare_hx_kernel<<<64, 64, 0, s>>>(H, sc.s_h, hx_ops);
  return cudaGetLastError();
}

// A named barrier over nthreads threads that also ANDs a predicate across
// them: the outcome of per-thread bounded waits becomes the group's, so no
// thread leaves a loop whose next named barrier the others still reach.
__device__ __forceinline__ bool bar_and(uint32_t id, uint32_t nthreads, bool p) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred a, b;\n setp.ne.u32 a, %1, 0;\n barrier.cta.red.and.pred b, %2, %3, a;\n selp.u32 %0, 1, 0, b;\n}"
      : "=r"(r)
      : "r"(p ? 1u : 0u), "r"(id), "r"(nthreads)
      : "memory");
  return r != 0;
}

// Bounded mbarrier wait that also gives up when the CTA's stop flag is set.
__device__ __forceinline__ bool ws_wait(uint32_t mbar, uint32_t parity, uint64_t timeout_ns,
                                        const volatile int32_t *stop) {
  if (mbar_try_wait(mbar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try_wait(mbar, parity)) return true;
    if ((it & 127u) == 0u && (*stop || globaltimer_ns() - t0 > timeout_ns)) return false;
  }
}

__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(mbar)
               : "memory");
}
// A in tensor memory, B in shared memory.
__device__ __forceinline__ void umma_f16_ts(uint32_t tmem_d, uint32_t tmem_a, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}" ::"r"(tmem_d),
      "r"(tmem_a), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&w)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
          taddr),
      "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3]), "r"(w[4]), "r"(w[5]), "r"(w[6]), "r"(w[7]), "r"(w[8]), "r"(w[9]),
      "r"(w[10]), "r"(w[11]), "r"(w[12]), "r"(w[13]), "r"(w[14]), "r"(w[15])
      : "memory");
}
// 32 lanes x 32 consecutive 32-bit columns per warp.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
      "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&w)[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), "r"(w[0]),
               "r"(w[1]), "r"(w[2]), "r"(w[3]), "r"(w[4]), "r"(w[5]), "r"(w[6]), "r"(w[7])
               : "memory");
}
__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
// Split a pair of FP32 values into FP16 hi and lo parts, packed two per
// 32-bit word (first value in the low half): hi keeps the top 10 explicit
// mantissa bits (x with its low 13 bits cleared, exact in FP16 within FP16's
// normal range), lo = x - hi (exact in FP32) rounded to FP16, so
// hi + lo = x within 2^-21 |x|.  Two paired conversions per pair.
__device__ __forceinline__ void split_pair(float a, float b, uint32_t &hi, uint32_t &lo) {
  const float ah = __uint_as_float(__float_as_uint(a) & 0xFFFFE000u);
  const float bh = __uint_as_float(__float_as_uint(b) & 0xFFFFE000u);
  const __half2 h = __floats2half2_rn(ah, bh), l = __floats2half2_rn(a - ah, b - bh);
  hi = *reinterpret_cast<const uint32_t *>(&h);
  lo = *reinterpret_cast<const uint32_t *>(&l);
}

// The same split of two components with packed FP32 arithmetic: lo = x - hi
// as one two-wide FMA (exact: x - hi is the low 13 bits of x).
__device__ __forceinline__ void split_pair2(float2 v, uint32_t &hi, uint32_t &lo) {
  const float2 h = make_float2(__uint_as_float(__float_as_uint(v.x) & 0xFFFFE000u),
                               __uint_as_float(__float_as_uint(v.y) & 0xFFFFE000u));
  const float2 l = __ffma2_rn(h, make_float2(-1.f, -1.f), v);
  const __half2 hh = __floats2half2_rn(h.x, h.y), ll = __floats2half2_rn(l.x, l.y);
  hi = *reinterpret_cast<const uint32_t *>(&hh);
  lo = *reinterpret_cast<const uint32_t *>(&ll);
}

// Eight scaled floats as one 32-byte global store (address 32-byte aligned);
// the scaling as four two-wide multiplies.
__device__ __forceinline__ void st_global_v8(float *dst, const float *v, float sc) {
  const float2 s2 = make_float2(sc, sc);
  const float2 a = __fmul2_rn(make_float2(v[0], v[1]), s2), b = __fmul2_rn(make_float2(v[2], v[3]), s2);
  const float2 c = __fmul2_rn(make_float2(v[4], v[5]), s2), d = __fmul2_rn(make_float2(v[6], v[7]), s2);
  asm volatile("st.global.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(dst), "f"(a.x), "f"(a.y), "f"(b.x),
               "f"(b.y), "f"(c.x), "f"(c.y), "f"(d.x), "f"(d.y)
               : "memory");
}

}  // namespace prune
