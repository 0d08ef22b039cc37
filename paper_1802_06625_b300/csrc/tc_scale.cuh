// Power-of-two scaling of tensor-core operands (exact in binary floating
// point).  FP16 holds magnitudes in [2^-14, 65504] at full precision; an
// operand split into FP16 hi and lo parts keeps ~2^-21 relative precision
// for its largest components when that largest magnitude M lies in
// [2^0, 2^15): nothing overflows, and the lo parts of components near M are
// normal (components far below M, whose lo parts are subnormal, carry an
// absolute error of at most 2^-25, below 2^-21 M / 16).  So an operand whose
// M is in that window is used as it is (scale 2^0, no multiply), and any
// other is scaled by 2^s, s a multiple of 8, so that M 2^s lies in
// [2^7, 2^15).  The exponent s is a function of M's exponent alone (so a
// tile gets the same scale whichever CTA fires it, and results do not depend
// on scheduling), and its steps of 8 let consecutive tiles of a signal share
// it.  Results are scaled back by 2^-s; a scaling by 2^n changes no
// rounding as long as the values stay normal floats.
//
// The constant operands (taps, H) are scaled once per graph on the host;
// their exponents travel in the kernels' parameter records.
#pragma once
#include <cmath>
#include <cstdint>
#include <cstring>

#include <cuda_runtime.h>

namespace prune {

constexpr int kTTop = 14;                // the window: largest component in [2^0, 2^(kTTop+1))
constexpr int kTMaxUp = 96;              // largest up-scaling (a tile whose largest |x| < 2^-89 keeps it)

// Exponent s for a largest magnitude M, given its biased float exponent e
// (255 for inf / NaN; e of zero = 0 with M = 0): 0 inside the window and for
// zero, inf and NaN; otherwise the multiple of 8 with e + s in [134, 141],
// at most kTMaxUp.
__host__ __device__ __forceinline__ int tc_shift_exp(int e, bool zero) {
  if (e >= 255 || zero) return 0;
  if (e >= 127 && e <= 127 + kTTop) return 0;
  const int d = 127 + kTTop - (e > 1 ? e : 1);       // > 14 or < 0
  const int s = d >= 0 ? (d / 8) * 8 : -(((-d) + 7) / 8) * 8;
  return s < kTMaxUp ? s : kTMaxUp;
}
__host__ __device__ __forceinline__ int tc_shift_bits(uint32_t b) {
  return tc_shift_exp(static_cast<int>((b >> 23) & 0xFFu), (b & 0x7FFFFFFFu) == 0u);
}
__device__ __forceinline__ int tc_pow2_shift(float mx) { return tc_shift_bits(__float_as_uint(mx)); }

// The largest |component| of FP16 hi parts, kept as a packed pair whose
// signs are meaningless (max.xorsign.abs: |result| = max(|a|, |b|); NaN
// operands are skipped).
__device__ __forceinline__ void hmax_abs_acc(uint32_t &acc, uint32_t h2) {
  asm("max.xorsign.abs.f16x2 %0, %0, %1;" : "+r"(acc) : "r"(h2));
}
__device__ __forceinline__ uint32_t hmax_abs_bits(uint32_t acc) {  // FP16 bits of the larger magnitude
  return max(acc & 0x7FFFu, (acc >> 16) & 0x7FFFu);
}
// Given the FP16 bits h of the largest hi part of a tile converted with the
// predicted exponent s (hi = the component scaled by 2^s with its low 13
// mantissa bits cleared, so its FP16 exponent is that of the scaled
// component when it is a normal FP16): the tile's own exponent, or -1000 when
// h cannot tell (zero, subnormal, inf: the caller finds the FP32 maximum).
__device__ __forceinline__ int tc_shift_from_hi(uint32_t h, int s) {
  if (h < 0x0400u || h >= 0x7C00u) return -1000;
  const int e = static_cast<int>(h >> 10) - 15 + 127 - s;       // biased FP32 exponent of M
  return tc_shift_exp(e, false);
}

// 2^n as a float for n in [-149, 127] (subnormal below -126); clamped.
__device__ __forceinline__ float exp2i(int n) {
  n = max(-149, min(127, n));
  return n >= -126 ? __uint_as_float(static_cast<uint32_t>(n + 127) << 23) : __uint_as_float(1u << (n + 149));
}
// v 2^n, exact whenever the result is a normal float (the three factors have
// the sign of n, so an intermediate under- or overflows only if the result
// does).  |n| up to 378.
__device__ __forceinline__ float mul_pow2(float v, int n) {
  n = max(-378, min(378, n));
  const int a = n / 3, b = (n - a) / 2;
  return v * exp2i(a) * exp2i(b) * exp2i(n - a - b);
}
// 2^n as f1 f2 (|n| <= 252): f2 = 1 when |n| <= 126, so one multiply by f1
// suffices then (callers test f2 != 1 once per tile).
__device__ __forceinline__ void pow2_pair(int n, float &f1, float &f2) {
  n = max(-252, min(252, n));
  if (n >= -126 && n <= 126) {
    f1 = exp2i(n);
    f2 = 1.f;
  } else {
    f1 = exp2i(n / 2);
    f2 = exp2i(n - n / 2);
  }
}

// The exponent of n complex values on the device (for operands that only
// the device holds): one block reduces their largest component.
static __global__ void tc_shift_of_kernel(const float2 *v, int64_t n, int32_t *out) {
  __shared__ uint32_t red[32];
  float mx = 0.f;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) mx = fmaxf(mx, fmaxf(fabsf(v[i].x), fabsf(v[i].y)));
  const uint32_t w = __reduce_max_sync(0xffffffffu, __float_as_uint(mx));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = w;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t r = 0;
    for (int i = 0; i < static_cast<int>(blockDim.x >> 5); ++i) r = max(r, red[i]);
    *out = tc_shift_bits(r);
  }
}
inline cudaError_t tc_shift_of(const float2 *v, int64_t n, int32_t *out, cudaStream_t s) {
  tc_shift_of_kernel<<<1, 256, 0, s>>>(v, n, out);
  return cudaGetLastError();
}

// ---- host side: exponents of the constant operands

// Largest |component| of n complex values (re, im interleaved floats).
inline uint32_t host_absmax_bits(const float *v, int64_t n) {
  float mx = 0.f;
  for (int64_t i = 0; i < 2 * n; ++i) mx = std::fmax(mx, std::fabs(v[i]));
  uint32_t b;
  std::memcpy(&b, &mx, 4);
  return b;
}

// Exponents of a graph's constant tensor-core operands: taps are used as
// h 2^s_taps, H as H 2^s_h; the FIR output (y 2^(sx + s_taps) for a tile
// scaled by 2^sx, whose largest component is then below 2^15) enters the
// HX operand times 2^m, m from the L1 bound |y_acc| <= sum_t (|Re h_t| +
// |Im h_t|) 2^s_taps 2^15, so that the HX operand stays below 2^14.
struct TcScale {
  int32_t s_taps, m, s_h, pad;
};
inline TcScale tc_scale_of(const float *taps, int T, const float *H, int N) {
  TcScale s{0, 0, 0, 0};
  if (taps) {
    s.s_taps = tc_shift_bits(host_absmax_bits(taps, T));
    double l1 = 0.0;
    for (int t = 0; t < 2 * T; ++t) l1 += std::fabs(static_cast<double>(taps[t]));
    l1 = std::ldexp(l1, s.s_taps) * (1.0 + 1.0 / 1024.0);
    if (l1 > 0.0 && std::isfinite(l1)) {
      const int cl = static_cast<int>(std::ceil(std::log2(l1)));  // l1 <= 2^cl
      s.m = kTTop - (cl + kTTop + 1);                             // 2^(cl + 15 + m) <= 2^14
    }
  }
  if (H) s.s_h = tc_shift_bits(host_absmax_bits(H, static_cast<int64_t>(N) * N));
  return s;
}

}  // namespace prune
