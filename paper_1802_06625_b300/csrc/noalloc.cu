// prune_fire_frames_noalloc: the fused firing loop for callers that cannot
// allocate device memory.
//
// Who needs it: real-time or interrupt-driven host threads that must never
// block in the device allocator (cudaMalloc can wait on the device and on
// the driver's locks), and deployments whose device memory is budgeted and
// committed up front, where an allocation at firing time may fail or is not
// permitted at all.  Such callers hand over every input and output buffer;
// the only other device memory this entry point touches is one file-scope
// scratch array of fixed size that the library image carries.
//
// Limits and sharing:
//   - the scratch holds up to kMaxFrames frames per call and up to kMaxLook
//     look-back words (frames x tiles, tiles = ceil(F*B / TS) with TS the
//     largest multiple of B not above 2048); larger requests are rejected with
//     PRUNE_EINVAL before anything is enqueued;
//   - every GPU that loads the library holds the array until the process exits;
//   - every call uses the same array and leaves its contents behind; each
//     call clears what must start at zero (in its first kernel, stream
//     ordered), so calls ordered on one stream are safe, but calls that can
//     overlap on the GPU (different streams without ordering) race on it.
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <string>

#include "prune.h"
#include "device_common.cuh"
#include "fir.cuh"
#include "firing_loop.cuh"

using namespace prune;

void prune_set_create_error(const std::string &m);  // prune_runtime.cu

namespace {

constexpr int kMaxFrames = 256;
constexpr int kMaxLook = 65536;
constexpr int kMaxDevices = 64;

struct NoAllocScratch {
  LoopScratch ls;
  uint64_t ctr[kNumFifos * 3];     // FIFO counters of the call (not reported)
  int64_t rec_frame[kMaxFrames];   // record headers (not reported)
  uint64_t ready[kMaxFrames];
  uint32_t done[kMaxFrames];
  uint64_t look[kMaxLook];
};

// The scratch (about 527 KB).  In host code this name is only a host-side
// stand-in for the device object; its device address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

std::mutex g_setup_mu;
void *g_scratch_addr[kMaxDevices] = {};

prune_status na_fail(prune_status s, const std::string &m) {
  prune_set_create_error(m);  // read back through prune_last_error(NULL)
  return s;
}

// Clears the parts of the scratch that must start at zero and marks the
// call's frames as present in f0, so that FIR's firing rule holds.
__global__ void noalloc_init_kernel(NoAllocScratch *s, int32_t frames, int32_t tiles, int32_t F, uint32_t *status) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nthreads = gridDim.x * blockDim.x;
  for (int i = tid; i < frames * tiles; i += nthreads) s->look[i] = 0;
  for (int i = tid; i < frames; i += nthreads) {
    s->ready[i] = 0;
    s->done[i] = 0;
    s->rec_frame[i] = 0;
  }
  if (tid < kNumFifos * 3) s->ctr[tid] = 0;
  if (tid == 0) {
    s->ls.ticket = 0;
    s->ls.booked = 0;
    s->ls.abort = 0;
    s->ls.book_lock = 0;
  }
  if (tid < 4) status[tid] = 0;
  __syncthreads();
  if (tid == 0) s->ctr[0 * 3 + kCtrWritten] = static_cast<uint64_t>(frames) * static_cast<uint64_t>(F);
}

}  // namespace

extern "C" prune_status prune_fire_frames_noalloc(const void *x, const void *hist, const void *taps, const void *H,
                                                  int32_t F, int32_t B, int32_t T, int32_t N, int32_t frames,
                                                  float tau, int32_t *c, int32_t *idx, void *y, void *hist_out,
                                                  uint32_t *status, void *stream) {
  // shape rules of prune_graph_desc, the fused-loop restriction N < 64, and
  // the fixed scratch limits -- all checked before any CUDA call
  if (F < 1 || F > (1 << 20) || B < 8 || B > kFirTile || B % 8 != 0 || T < 1 || T > 256 || T - 1 > B || N < 1 ||
      N >= 64 || B % N != 0 || frames < 0)
    return na_fail(PRUNE_EINVAL, "prune_fire_frames_noalloc: bad shape (graph shape rules, and N < 64)");
  const int tpb = B / 8;
  if (!((tpb <= 32 && (tpb & (tpb - 1)) == 0) || tpb % 32 == 0))
    return na_fail(PRUNE_EINVAL, "prune_fire_frames_noalloc: B/8 must be a power of two up to 32 or a multiple of 32");
  if (!x || !taps || !H || !c || !idx || !y || !status || tau != tau)
    return na_fail(PRUNE_EINVAL, "prune_fire_frames_noalloc: NULL buffer or NaN tau");
  if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) & 15u)
    return na_fail(PRUNE_EINVAL, "prune_fire_frames_noalloc: x and y must be 16-byte aligned");
  if (T > 1 && hist && hist_out && hist == hist_out)
    return na_fail(PRUNE_EINVAL, "prune_fire_frames_noalloc: hist and hist_out must not alias");
  const int64_t L = static_cast<int64_t>(F) * B;
  const int TS = fir_tile_samples(B);
  const int64_t tiles = (L + TS - 1) / TS;
  if (frames > kMaxFrames || frames * tiles > kMaxLook)
    return na_fail(PRUNE_EINVAL, "prune_fire_frames_noalloc: " + std::to_string(frames) + " frames x " +
                                     std::to_string(tiles) + " tiles exceed the fixed scratch (at most " +
                                     std::to_string(kMaxFrames) + " frames and " + std::to_string(kMaxLook) +
                                     " look-back words per call)");
  if (frames == 0) return PRUNE_OK;

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return na_fail(PRUNE_ECUDA, std::string("prune_fire_frames_noalloc: no usable device: ") + cudaGetErrorString(e));
  // Set-up, once per device, with that device current: the device address
  // of the scratch.  It happens in the first call on a device, which should
  // come before any stream capture.
  void *scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_addr[dev]) {
      void *p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p)
        return na_fail(PRUNE_ECUDA, std::string("prune_fire_frames_noalloc: cudaGetSymbolAddress: ") +
                                        cudaGetErrorString(e));
      g_scratch_addr[dev] = p;
    }
    scratch = g_scratch_addr[dev];
  }
  NoAllocScratch *s = static_cast<NoAllocScratch *>(scratch);
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  noalloc_init_kernel<<<64, 256, 0, st>>>(s, frames, static_cast<int32_t>(tiles), F, status);
  e = cudaGetLastError();
  if (e != cudaSuccess) return na_fail(PRUNE_ECUDA, std::string("prune_fire_frames_noalloc: ") + cudaGetErrorString(e));

  LoopParams lp{};
  FirParams &fp = lp.f;
  fp.src = FrameSrc{nullptr, static_cast<const float2 *>(x), L, 0, 1};
  fp.L = L;
  fp.F = F; fp.B = B; fp.T = T; fp.TP = fir_taps_padded(T); fp.TS = TS;
  fp.tiles = static_cast<int32_t>(tiles); fp.frames = frames;
  fp.taps = static_cast<const float2 *>(taps);
  fp.hist = T > 1 ? static_cast<const float2 *>(hist) : nullptr;
  fp.hist_out = T > 1 ? static_cast<float2 *>(hist_out) : nullptr;
  fp.y = nullptr; fp.y_stride = L; fp.yslot = SlotMap{0, INT_MAX};
  fp.energy = nullptr; fp.eslot = SlotMap{0, INT_MAX};
  lp.tau = tau;
  lp.look = s->look; lp.done = s->done; lp.ready = s->ready; lp.C = frames;
  lp.rec_c = c; lp.rec_idx = idx; lp.rec_frame = s->rec_frame; lp.rec_y = static_cast<float2 *>(y);
  lp.rslot = SlotMap{0, INT_MAX};
  lp.H = static_cast<const float2 *>(H); lp.N = N;
  lp.ls = &s->ls; lp.ticket_base = 0; lp.timeout_ns = 2000000000ull;
  lp.ctr = s->ctr; lp.status = status;
  for (int i = 0; i < 8; ++i) lp.cap[i] = ~0ull;

  const unsigned long long total = static_cast<unsigned long long>(frames) * static_cast<unsigned long long>(tiles);
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = loop_smem_bytes(T, N);
  auto launch = [&](auto kern) -> cudaError_t {
    if (smem > 48 * 1024) {
      cudaError_t a = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
      if (a != cudaSuccess) return a;
    }
    int occ = 0;
    cudaError_t a = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kFirThreads, smem);
    if (a != cudaSuccess) return a;
    if (occ < 1) occ = 1;
    const unsigned long long cap = static_cast<unsigned long long>(sms) * static_cast<unsigned long long>(occ);
    const int grid = static_cast<int>(total < cap ? total : cap);
    kern<<<grid, kFirThreads, smem, st>>>(lp);
    return cudaGetLastError();
  };
  switch (N) {
    case 2: e = launch(firing_loop_kernel<2>); break;
    case 4: e = launch(firing_loop_kernel<4>); break;
    case 8: e = launch(firing_loop_kernel<8>); break;
    case 16: e = launch(firing_loop_kernel<16>); break;
    case 32: e = launch(firing_loop_kernel<32>); break;
    default: e = launch(firing_loop_kernel<0>);
  }
  if (e != cudaSuccess) return na_fail(PRUNE_ECUDA, std::string("prune_fire_frames_noalloc: ") + cudaGetErrorString(e));
  return PRUNE_OK;
}
