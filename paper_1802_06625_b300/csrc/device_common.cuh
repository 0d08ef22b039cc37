// Device-side helpers shared by the firing kernels: complex arithmetic on
// interleaved float2, memory-ordering primitives for the device FIFO
// counters, a %globaltimer based wait limit and the device status word.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace prune {

// ---------------------------------------------------------------- status
// Device status word layout (4 x uint32): code, actor, fifo, frame (low 32).
enum DevCode : uint32_t {
  kDevOk = 0,
  kDevTimeout = 1,     // a bounded wait gave up
  kDevUnderflow = 2,   // an actor found fewer tokens than its firing rule needs
  kDevOverflow = 3,    // a commit would exceed the FIFO capacity (eq. (2))
  kDevAbort = 4,       // another CTA failed first
  kDevInvariant = 5    // a compacted position fell outside the frame
};
enum DevActor : uint32_t { kActSrc = 0, kActFir = 1, kActDet = 2, kActSel = 3, kActHx = 4, kActSink = 5 };

// Counters: per FIFO {written, read, peak}.
constexpr int kNumFifos = 8;
constexpr int kCtrWritten = 0, kCtrRead = 1, kCtrPeak = 2;

__device__ __forceinline__ void report_error(uint32_t *status, uint32_t code, uint32_t actor,
                                             uint32_t fifo, uint64_t frame) {
  if (status == nullptr) return;
  if (atomicCAS(&status[0], 0u, code) == 0u) {
    status[1] = actor;
    status[2] = fifo;
    status[3] = static_cast<uint32_t>(frame);
  }
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint64_t ld_acquire_u64(const uint64_t *p) {
  uint64_t v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u64(uint64_t *p, uint64_t v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
// Relaxed GPU-scope access: coherent, but orders nothing else (for words
// that carry all the information their readers use).
__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t *p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u64(uint64_t *p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_volatile_u32(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.volatile.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// FIFO commit: bump `written` by n and track the peak occupancy
// (delay + written - read).  Reports an overflow against the eq. (2)
// capacity `cap` (in tokens).  Single thread.
__device__ __forceinline__ void fifo_commit(uint64_t *ctr, int fifo, uint64_t n, uint64_t delay,
                                            uint64_t cap, uint32_t *status, uint32_t actor,
                                            uint64_t frame) {
  uint64_t *c = ctr + fifo * 3;
  uint64_t w = atomicAdd(reinterpret_cast<unsigned long long *>(&c[kCtrWritten]),
                         static_cast<unsigned long long>(n)) + n;
  uint64_t r = ld_acquire_u64(&c[kCtrRead]);
  uint64_t occ = delay + w - r;
  atomicMax(reinterpret_cast<unsigned long long *>(&c[kCtrPeak]), static_cast<unsigned long long>(occ));
  if (occ > cap) report_error(status, kDevOverflow, actor, static_cast<uint32_t>(fifo), frame);
}
// FIFO release: bump `read` by n; reports an underflow if fewer than n
// tokens were present.
__device__ __forceinline__ void fifo_release(uint64_t *ctr, int fifo, uint64_t n, uint64_t delay,
                                             uint32_t *status, uint32_t actor, uint64_t frame) {
  uint64_t *c = ctr + fifo * 3;
  uint64_t w = ld_acquire_u64(&c[kCtrWritten]);
  uint64_t r = atomicAdd(reinterpret_cast<unsigned long long *>(&c[kCtrRead]),
                         static_cast<unsigned long long>(n));
  if (delay + w < r + n) report_error(status, kDevUnderflow, actor, static_cast<uint32_t>(fifo), frame);
}

// ------------------------------------------------------------ complex math
__device__ __forceinline__ void cmac(float2 &acc, float2 h, float2 x) {
  acc.x = fmaf(h.x, x.x, acc.x);
  acc.x = fmaf(-h.y, x.y, acc.x);
  acc.y = fmaf(h.x, x.y, acc.y);
  acc.y = fmaf(h.y, x.x, acc.y);
}

// Frame addressing: frame k (0-based within a launch) of a stream of frames
// that either sit in a descriptor ring (graph FIFO f0) or back to back.
struct FrameSrc {
  const float2 *const *ring;  // device ring of frame pointers, or nullptr
  const float2 *base;         // contiguous frames when ring == nullptr
  int64_t stride;             // samples between contiguous frames
  int64_t seq0;               // sequence number of frame 0 of the launch
  int32_t cap;                // ring capacity in frames
  __device__ __forceinline__ const float2 *frame(int64_t k) const {
    return ring ? ring[(seq0 + k) % cap] : base + k * stride;
  }
};

// Output slot addressing: frame k of a launch goes to slot (seq0 + k) % cap.
struct SlotMap {
  int64_t seq0;
  int32_t cap;
  __device__ __forceinline__ int64_t slot(int64_t k) const { return (seq0 + k) % cap; }
};

// The same slot, (seq0 + k) % cap for k >= 0, from a base taken once per
// launch: one 64-bit modulo up front, then a subtraction per frame (a run
// fires at most cap frames; the modulo stays for any larger k).
struct RingSlot {
  int32_t base, cap;
  __host__ __device__ __forceinline__ static RingSlot of(int64_t seq0, int32_t cap) {
    return RingSlot{static_cast<int32_t>(seq0 % cap), cap};
  }
  __host__ __device__ __forceinline__ int32_t at(int k) const {
    int32_t v = base + k;
    if (v >= cap) v -= cap;
    if (v >= cap) v %= cap;
    return v;
  }
};

}  // namespace prune
