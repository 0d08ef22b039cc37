// Host runtime behind the C ABI of include/prune.h: the graph object, the
// FIFO layout in HBM, the firing of the actors on the device and the
// copy-in / copy-out of frames.  Every step of the dataflow runs in the
// kernels of this library; there is no host or CPU fallback.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <deque>
#include <vector>

#include "prune.h"
#include "device_common.cuh"
#include "fir.cuh"
#include "detsel.cuh"
#include "hx_cuda.cuh"
#include "firing_loop.cuh"
#include "hx_tc.cuh"
#include "firing_loop_tc.cuh"
#include "firing_loop_ws.cuh"

using namespace prune;

namespace {

thread_local std::string t_create_error = "no error";

// Eq. (2) of Sec. VI-B in tokens.
int64_t eq2_capacity(int64_t r, int64_t Q, int64_t C) {
  if (Q % r != 0) return r * C + Q;
  return std::max(r * C, Q);
}

struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (dev >= 0 && dev != prev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

bool shape_ok(int32_t F, int32_t B, int32_t T, int32_t N, std::string *why) {
  char buf[256];
  auto bad = [&](const char *m) {
    std::snprintf(buf, sizeof buf, "%s (F=%d B=%d T=%d N=%d)", m, F, B, T, N);
    *why = buf;
    return false;
  };
  if (F < 1 || F > (1 << 20)) return bad("F must be in [1, 2^20]");
  if (B < 8 || B > kFirTile || B % 8 != 0) return bad("B must be a multiple of 8 in [8, 2048]");
  const int tpb = B / 8;
  if (!((tpb <= 32 && (tpb & (tpb - 1)) == 0) || tpb % 32 == 0))
    return bad("B/8 must be a power of two up to 32 or a multiple of 32");
  if (T < 1 || T > 256) return bad("T must be in [1, 256]");
  if (T - 1 > B) return bad("the delay token (T-1 samples) must fit in one block: T-1 <= B");
  if (N < 1 || N > 128 || B % N != 0) return bad("N must divide B and be in [1, 128]");
  return true;
}

}  // namespace

// Message for prune_last_error(NULL) from entry points without a graph.
void prune_set_create_error(const std::string &m) { t_create_error = m; }

struct prune_graph {
  prune_graph_desc d{};
  int dev = 0;
  int sms = 148;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int32_t C = 3, out_cap = 3;
  int64_t L = 0;
  int32_t TP = 0, TS = 0, tiles = 0;
  uint64_t budget = 0, allocated = 0;
  std::vector<void *> allocs;
  // device state
  float2 *taps = nullptr, *H = nullptr;
  float2 *stage = nullptr;            // f0 payload slots for copied frames
  const float2 **f0_ring = nullptr;   // f0 descriptor ring [C]
  float2 *hist = nullptr;             // f1 delay token, double buffered [2][T-1]
  float2 *y_ring = nullptr;           // f2/f3 payload [C][L] (actor-per-kernel path)
  float *energy = nullptr;            // [C][F]
  int32_t *rec_c = nullptr, *rec_idx = nullptr;
  int64_t *rec_frame = nullptr;
  float2 *rec_y = nullptr;            // result ring [out_cap][L]
  uint64_t *ctr = nullptr;            // [8][3]
  uint32_t *status = nullptr;         // [4]
  LoopScratch *loop = nullptr;        // fused firing-loop scratch
  uint64_t *look = nullptr;           // [C][tiles] look-back words
  uint32_t *done = nullptr;           // [C] finished tiles per frame slot
  uint64_t *ready = nullptr;          // [C] record-final flags (frame seq + 1)
  unsigned long long ticket_base = 0;
  uint64_t timeout_ns = 2000000000ull;
  bool ws_loop = true;  // warp-specialised tensor-core loop (PRUNE_TC_KERNEL=pipes: tile pipelines)
  uint16_t *hx_b_ops = nullptr;       // tcgen05 B operands (N >= 64)
  TcScale tcs{};                      // exponents of the scaled tensor-core operands (host-computed)
  uint16_t *tc_fir_ops = nullptr;     // tensor-core firing loop: FIR tap operands
  uint16_t *tc_hx_ops = nullptr;      //   and the real form of H
  int64_t cap[PRUNE_NUM_FIFOS] = {};
  // optional per-kernel event timing
  bool profile = false;
  struct Timed { int kind; cudaEvent_t a, b; };
  std::vector<Timed> timed;
  std::vector<cudaEvent_t> event_pool;
  // Pulls copy out on their own stream after the run that fired the records
  // (an event per run), so a pull overlaps the runs and pushes enqueued
  // after it.  Pinned staging for the records' control words and status.
  cudaStream_t pull_stream = nullptr;
  std::deque<std::pair<int64_t, cudaEvent_t>> run_ends;  // (frames fired through the run, its end)
  std::vector<cudaEvent_t> run_ev_pool;
  int32_t *pull_c = nullptr;
  int64_t *pull_frame = nullptr;
  uint32_t *pull_status = nullptr;
  double kind_ms[8] = {};
  int64_t kind_n[8] = {};
  // host view of the FIFO heads/tails in frames
  int64_t pushed = 0, fired = 0, pulled = 0, runs = 0;
  bool poisoned = false;
  prune_status poison_code = PRUNE_OK;
  std::string err = "no error";
};

namespace {

prune_status fail(prune_graph *g, prune_status s, const std::string &m) {
  if (g) g->err = m;
  else t_create_error = m;
  return s;
}

#define CU(g, call)                                                                   \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return fail((g), PRUNE_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <typename T>
prune_status galloc(prune_graph *g, T **p, size_t count) {
  const size_t bytes = std::max<size_t>(count * sizeof(T), 16);
  if (g->budget && g->allocated + bytes > g->budget)
    return fail(g, PRUNE_ENOMEM, "graph would exceed its HBM budget of " + std::to_string(g->budget) + " bytes");
  void *q = nullptr;
  cudaError_t e = cudaMalloc(&q, bytes);
  if (e != cudaSuccess) return fail(g, PRUNE_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  g->allocs.push_back(q);
  g->allocated += bytes;
  *p = static_cast<T *>(q);
  return PRUNE_OK;
}

// The device status words (already copied to the host) as a status.
prune_status status_words(prune_graph *g, const uint32_t *st) {
  if (st[0] == kDevOk) return PRUNE_OK;
  static const char *actors[] = {"SRC", "FIR", "DET", "SEL", "HX", "SINK"};
  static const char *codes[] = {"ok", "bounded wait gave up", "FIFO underflow", "FIFO overflow", "aborted",
                                "compacted position out of range"};
  char buf[256];
  std::snprintf(buf, sizeof buf, "device: %s in actor %s on FIFO f%u at frame %u",
                codes[std::min<uint32_t>(st[0], 5)], actors[std::min<uint32_t>(st[1], 5)], st[2], st[3]);
  g->poisoned = true;
  g->poison_code = st[0] == kDevTimeout ? PRUNE_ETIMEOUT : PRUNE_EDEVICE;
  return fail(g, g->poison_code, buf);
}

prune_status check_device_status(prune_graph *g) {
  uint32_t st[4] = {0, 0, 0, 0};
  CU(g, cudaMemcpy(st, g->status, sizeof st, cudaMemcpyDeviceToHost));
  return status_words(g, st);
}

// Run end events whose records are all pulled go back to their pool.
void recycle_run_events(prune_graph *g) {
  while (!g->run_ends.empty() && g->run_ends.front().first <= g->pulled) {
    g->run_ev_pool.push_back(g->run_ends.front().second);
    g->run_ends.pop_front();
  }
}

prune_status sync_and_check(prune_graph *g) {
  CU(g, cudaStreamSynchronize(g->stream));
  return check_device_status(g);
}

// Event bracket around one kernel launch when profiling is on.
struct KTimer {
  prune_graph *g;
  int kind;
  cudaEvent_t a = nullptr, b = nullptr;
  cudaEvent_t take() {
    if (!g->event_pool.empty()) {
      cudaEvent_t e = g->event_pool.back();
      g->event_pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  KTimer(prune_graph *g_, int kind_) : g(g_), kind(kind_) {
    if (!g->profile) return;
    a = take();
    b = take();
    cudaEventRecord(a, g->stream);
  }
  ~KTimer() {
    if (!g->profile) return;
    cudaEventRecord(b, g->stream);
    g->timed.push_back({kind, a, b});
  }
};

void drain_timers(prune_graph *g) {
  for (auto &t : g->timed) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, t.a, t.b) == cudaSuccess) {
      g->kind_ms[t.kind] += ms;
      g->kind_n[t.kind] += 1;
    }
    g->event_pool.push_back(t.a);
    g->event_pool.push_back(t.b);
  }
  g->timed.clear();
}

struct PushPtrs {
  const float2 *p[64];
};

__global__ void f0_push_kernel(const float2 **ring, int32_t cap, int64_t seq, int32_t n, PushPtrs ptrs,
                               uint64_t *ctr, uint32_t *status, int32_t F, uint64_t cap_f0) {
  const int t = threadIdx.x;
  if (t < n) ring[(seq + t) % cap] = ptrs.p[t];
  if (t == 0) fifo_commit(ctr, 0, static_cast<uint64_t>(n) * F, 0, cap_f0, status, kActSrc, seq);
}

int hx_grid(int sms, int64_t work) {
  return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(work, static_cast<int64_t>(sms) * 8)));
}

// Launch the CUDA-core HX kernel for N < 64 (register-blocked for powers of two).
cudaError_t launch_hx_cuda(const HxParams &p, int grid, cudaStream_t s) {
  const size_t smem_blk = static_cast<size_t>(std::max(p.B, p.N * p.N)) * sizeof(float2);
  switch (p.N) {
    case 1: hx_cuda_kernel<1><<<grid, kHxThreads, smem_blk, s>>>(p); break;
    case 2: hx_cuda_kernel<2><<<grid, kHxThreads, smem_blk, s>>>(p); break;
    case 4: hx_cuda_kernel<4><<<grid, kHxThreads, smem_blk, s>>>(p); break;
    case 8: hx_cuda_kernel<8><<<grid, kHxThreads, smem_blk, s>>>(p); break;
    case 16: hx_cuda_kernel<16><<<grid, kHxThreads, smem_blk, s>>>(p); break;
    case 32: hx_cuda_kernel<32><<<grid, kHxThreads, smem_blk, s>>>(p); break;
    default: {
      const size_t smem = smem_blk + static_cast<size_t>(p.N) * p.N * sizeof(float2);
      if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(hx_cuda_generic_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(smem));
        if (e != cudaSuccess) return e;
      }
      hx_cuda_generic_kernel<<<grid, kHxThreads, smem, s>>>(p);
    }
  }
  return cudaGetLastError();
}

}  // namespace

static prune_status run_firing_loop(prune_graph *g, int64_t seq0, int32_t n, int32_t flags);

static prune_status run_actor_kernels(prune_graph *g, int64_t seq0, int32_t n) {
  const prune_graph_desc &d = g->d;
  if (!g->y_ring) {  // the first actor-path run of a graph that fires fused by default
    const prune_status s = galloc(g, &g->y_ring, static_cast<size_t>(g->C) * g->L);
    if (s != PRUNE_OK) return s;
  }
  const int64_t T1 = std::max(d.T - 1, 1);
  FirParams fp{};
  fp.src = FrameSrc{g->f0_ring, nullptr, 0, seq0, g->C};
  fp.L = g->L;
  fp.F = d.F; fp.B = d.B; fp.T = d.T; fp.TP = g->TP; fp.TS = g->TS; fp.tiles = g->tiles; fp.frames = n;
  fp.taps = g->taps;
  fp.hist = d.T > 1 ? g->hist + (g->runs & 1) * T1 : nullptr;
  fp.hist_out = d.T > 1 ? g->hist + ((g->runs + 1) & 1) * T1 : nullptr;
  fp.y = g->y_ring; fp.y_stride = g->L; fp.yslot = SlotMap{seq0, g->C};
  fp.energy = g->energy; fp.eslot = SlotMap{seq0, g->C};
  fp.ctr = g->ctr; fp.status = g->status;
  fp.cap_f1 = g->cap[1]; fp.cap_f2 = g->cap[2]; fp.cap_f3 = g->cap[3];
  {
    KTimer kt(g, 1);
    fir_energy_kernel<<<dim3(g->tiles, n), kFirThreads, fir_smem_bytes(d.T), g->stream>>>(fp);
  }
  CU(g, cudaGetLastError());

  DetSelParams dp{};
  dp.energy = g->energy; dp.eslot = SlotMap{seq0, g->C};
  dp.F = d.F; dp.frames = n; dp.tau = d.tau;
  dp.c = g->rec_c; dp.idx = g->rec_idx; dp.rec_frame = g->rec_frame; dp.rslot = SlotMap{seq0, g->out_cap};
  dp.ctr = g->ctr; dp.status = g->status;
  dp.cap_f4 = g->cap[4]; dp.cap_f5 = g->cap[5]; dp.cap_f6 = g->cap[6];
  {
    KTimer kt(g, 2);
    det_sel_kernel<<<n, kDetThreads, 0, g->stream>>>(dp);
  }
  CU(g, cudaGetLastError());

  HxParams hp{};
  hp.y = g->y_ring; hp.y_stride = g->L; hp.yslot = SlotMap{seq0, g->C};
  hp.c = g->rec_c; hp.idx = g->rec_idx; hp.rslot = SlotMap{seq0, g->out_cap};
  hp.out = g->rec_y; hp.out_stride = g->L; hp.oslot = SlotMap{seq0, g->out_cap};
  hp.H = g->H; hp.F = d.F; hp.B = d.B; hp.N = d.N; hp.frames = n;
  hp.ctr = g->ctr; hp.status = g->status; hp.cap_f7 = g->cap[7];
  if (g->hx_b_ops) {
    KTimer kt(g, 4);
    CU(g, launch_hx_tc(hp, g->hx_b_ops, g->tcs.s_h, nullptr, g->sms, g->stream));
  } else {
    KTimer kt(g, 3);
    CU(g, launch_hx_cuda(hp, hx_grid(g->sms, static_cast<int64_t>(n) * d.F), g->stream));
  }
  return PRUNE_OK;
}

static cudaError_t launch_ws_loop(const TcLoopParams &tp, int grid, size_t smem, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(firing_loop_ws_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  firing_loop_ws_kernel<<<grid, kWsThreads, smem, s>>>(tp);
  return cudaGetLastError();
}

template <int NP>
static cudaError_t launch_tc_loop(const TcLoopParams &tp, int grid, size_t smem, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(firing_loop_tc_kernel<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  firing_loop_tc_kernel<NP><<<grid, NP * kTPipeThreads, smem, s>>>(tp);
  return cudaGetLastError();
}

template <int NT>
static cudaError_t launch_loop_nt(const LoopParams &lp, int sms, size_t smem, cudaStream_t s, int *grid_out,
                                  unsigned long long total) {
  static int occ_cache[2] = {0, 0};  // per smem class is overkill: recompute when smem changes
  static size_t occ_smem = 0;
  (void)occ_cache;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(firing_loop_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
  }
  int occ = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, firing_loop_kernel<NT>, kFirThreads, smem);
  if (e != cudaSuccess) return e;
  (void)occ_smem;
  occ = std::max(occ, 1);
  const int grid = static_cast<int>(std::min<unsigned long long>(total, static_cast<unsigned long long>(sms) * occ));
  firing_loop_kernel<NT><<<grid, kFirThreads, smem, s>>>(lp);
  *grid_out = grid;
  return cudaGetLastError();
}

static prune_status run_firing_loop(prune_graph *g, int64_t seq0, int32_t n, int32_t flags) {
  const prune_graph_desc &d = g->d;
  const int64_t T1 = std::max(d.T - 1, 1);
  LoopParams lp{};
  FirParams &fp = lp.f;
  fp.src = FrameSrc{g->f0_ring, nullptr, 0, seq0, g->C};
  fp.L = g->L;
  fp.F = d.F; fp.B = d.B; fp.T = d.T; fp.TP = g->TP; fp.TS = g->TS; fp.tiles = g->tiles; fp.frames = n;
  fp.taps = g->taps;
  fp.hist = d.T > 1 ? g->hist + (g->runs & 1) * T1 : nullptr;
  fp.hist_out = d.T > 1 ? g->hist + ((g->runs + 1) & 1) * T1 : nullptr;
  fp.y = nullptr; fp.y_stride = g->L; fp.yslot = SlotMap{seq0, g->C};
  fp.energy = g->energy; fp.eslot = SlotMap{seq0, g->C};
  lp.tau = d.tau;
  lp.look = g->look; lp.done = g->done; lp.ready = g->ready; lp.C = g->C;
  lp.rec_c = g->rec_c; lp.rec_idx = g->rec_idx; lp.rec_frame = g->rec_frame; lp.rec_y = g->rec_y;
  lp.rslot = SlotMap{seq0, g->out_cap};
  lp.H = g->H; lp.N = d.N;
  lp.ls = g->loop; lp.ticket_base = g->ticket_base; lp.timeout_ns = g->timeout_ns;
  lp.ctr = g->ctr; lp.status = g->status;
  for (int i = 0; i < 8; ++i) lp.cap[i] = static_cast<uint64_t>(g->cap[i]);
  if (g->tc_fir_ops && !(flags & PRUNE_RUN_CUDA_CORES)) {
    // FIR and HX_b on tensor cores: tiles of 4096 outputs
    TcLoopParams tp{};
    tp.lp = lp;
    tp.lp.f.TS = kTTile;
    tp.lp.f.tiles = static_cast<int32_t>((g->L + kTTile - 1) / kTTile);
    tp.fir_ops = g->tc_fir_ops;
    tp.hx_ops = g->tc_hx_ops;
    tp.s_taps = g->tcs.s_taps;
    tp.m = g->tcs.m;
    tp.s_h = g->tcs.s_h;
    tp.ns = tc_shifts(d.T);
    // warp-specialised loop for T <= 65 unless PRUNE_TC_KERNEL=pipes asks
    // for the tile-pipeline loop
    if (g->ws_loop && ws_loop_supported(d.T)) {
      const size_t wsmem = ws_loop_smem_bytes(d.T);
      const unsigned long long ttotal = static_cast<unsigned long long>(n) * tp.lp.f.tiles;
      const int grid = static_cast<int>(std::max<unsigned long long>(
          1, std::min<unsigned long long>(ttotal, static_cast<unsigned long long>(g->sms))));
      // Frames fired round-robin: a CTA holds up to about 8 tiles in flight,
      // so a window of 8 x grid frames leaves about one tile of a frame in
      // flight (short look-backs); PRUNE_TC_WINDOW overrides the factor.
      int64_t wf = 8;
      if (const char *wv = std::getenv("PRUNE_TC_WINDOW")) wf = std::max<int64_t>(1, std::atoll(wv));
      tp.window = static_cast<int32_t>(std::max<int64_t>(1, std::min<int64_t>(n, wf * grid)));
      cudaError_t e;
      {
        KTimer kt(g, 6);
        e = launch_ws_loop(tp, grid, wsmem, g->stream);
      }
      if (e != cudaSuccess)
        return fail(g, PRUNE_ECUDA, std::string("tensor-core firing loop launch: ") + cudaGetErrorString(e));
      g->ticket_base += ttotal + static_cast<unsigned long long>(grid);  // one failing claim per CTA
      return PRUNE_OK;
    }
    const size_t smem = tc_loop_smem_bytes(d.T);
    const int np = tc_pipes(d.T);
    const unsigned long long ttotal = static_cast<unsigned long long>(n) * tp.lp.f.tiles;
    // one CTA per SM, np tile pipelines in each
    const int grid = static_cast<int>(std::max<unsigned long long>(
        1, std::min<unsigned long long>((ttotal + np - 1) / np, static_cast<unsigned long long>(g->sms))));
    // frames fired round-robin: about 8 tiles of one frame in flight
    tp.window = static_cast<int32_t>(std::max<int64_t>(1, std::min<int64_t>(n, (grid * np + 7) / 8)));
    cudaError_t e;
    {
      KTimer kt(g, 6);
      e = np == 4 ? launch_tc_loop<4>(tp, grid, smem, g->stream) : launch_tc_loop<3>(tp, grid, smem, g->stream);
    }
    if (e != cudaSuccess) return fail(g, PRUNE_ECUDA, std::string("tensor-core firing loop launch: ") + cudaGetErrorString(e));
    g->ticket_base += ttotal + static_cast<unsigned long long>(grid) * np;  // one failing claim per pipeline
    return PRUNE_OK;
  }
  const unsigned long long total = static_cast<unsigned long long>(n) * g->tiles;
  int grid = 0;
  cudaError_t e;
  {
    KTimer kt(g, 5);
    switch (d.N) {
      case 2: e = launch_loop_nt<2>(lp, g->sms, loop_smem_bytes(d.T, 2), g->stream, &grid, total); break;
      case 4: e = launch_loop_nt<4>(lp, g->sms, loop_smem_bytes(d.T, 4), g->stream, &grid, total); break;
      case 8: e = launch_loop_nt<8>(lp, g->sms, loop_smem_bytes(d.T, 8), g->stream, &grid, total); break;
      case 16: e = launch_loop_nt<16>(lp, g->sms, loop_smem_bytes(d.T, 16), g->stream, &grid, total); break;
      case 32: e = launch_loop_nt<32>(lp, g->sms, loop_smem_bytes(d.T, 32), g->stream, &grid, total); break;
      default: e = launch_loop_nt<0>(lp, g->sms, loop_smem_bytes(d.T, d.N), g->stream, &grid, total);
    }
  }
  if (e != cudaSuccess) return fail(g, PRUNE_ECUDA, std::string("firing loop launch: ") + cudaGetErrorString(e));
  g->ticket_base += total + static_cast<unsigned long long>(grid);
  return PRUNE_OK;
}

// ===================================================================== ABI

extern "C" {

prune_status prune_fifo_capacity(int64_t r, int64_t Q, int64_t C, int64_t *cap) {
  if (!cap || r < 1 || Q < 0 || C < 1) return fail(nullptr, PRUNE_EINVAL, "prune_fifo_capacity: need r>=1, Q>=0, C>=1");
  *cap = eq2_capacity(r, Q, C);
  return PRUNE_OK;
}

const char *prune_last_error(const prune_graph *g) {
  return g ? g->err.c_str() : t_create_error.c_str();
}

prune_status prune_graph_destroy(prune_graph *g) {
  if (!g) return PRUNE_OK;
  {
    DeviceGuard dg(g->dev);
    if (g->stream) cudaStreamSynchronize(g->stream);
    for (void *p : g->allocs) cudaFree(p);
    for (auto &t : g->timed) { cudaEventDestroy(t.a); cudaEventDestroy(t.b); }
    for (auto e : g->event_pool) cudaEventDestroy(e);
    for (auto &r : g->run_ends) cudaEventDestroy(r.second);
    for (auto e : g->run_ev_pool) cudaEventDestroy(e);
    if (g->pull_stream) {
      cudaStreamSynchronize(g->pull_stream);
      cudaStreamDestroy(g->pull_stream);
    }
    cudaFreeHost(g->pull_c);
    cudaFreeHost(g->pull_frame);
    cudaFreeHost(g->pull_status);
    if (g->own_stream && g->stream) cudaStreamDestroy(g->stream);
  }
  delete g;
  return PRUNE_OK;
}

prune_status prune_graph_create(const prune_graph_desc *desc, prune_graph **out) {
  if (out) *out = nullptr;
  if (!desc || !out) return fail(nullptr, PRUNE_EINVAL, "prune_graph_create: NULL argument");
  std::string why;
  if (!shape_ok(desc->F, desc->B, desc->T, desc->N, &why)) return fail(nullptr, PRUNE_EINVAL, why);
  if (!desc->taps || !desc->H) return fail(nullptr, PRUNE_EINVAL, "prune_graph_create: taps and H are required");
  if (std::isnan(desc->tau)) return fail(nullptr, PRUNE_EINVAL, "prune_graph_create: tau is NaN");
  if (desc->C < 0 || desc->out_frames < 0) return fail(nullptr, PRUNE_EINVAL, "prune_graph_create: C and out_frames must be >= 0");
  const int32_t C = desc->C ? desc->C : 3;
  const int32_t out_cap = desc->out_frames ? desc->out_frames : C;
  if (C > 4096 || out_cap > (1 << 20)) return fail(nullptr, PRUNE_EINVAL, "prune_graph_create: C or out_frames too large");

  // Port rates of the canonical graph against their FIFO rates (Sec. III-A):
  // {source port rate, sink port rate, fiforate} for f0..f7 (DRPs: atr).
  const int64_t F = desc->F;
  const int64_t rates[PRUNE_NUM_FIFOS][3] = {{F, F, F}, {1, 1, 1}, {F, F, F}, {F, F, F},
                                             {1, 1, 1}, {1, 1, 1}, {1, 1, 1}, {1, 1, 1}};
  for (auto &r : rates)
    if (r[0] != r[2] || r[1] != r[2]) return fail(nullptr, PRUNE_EINVAL, "port rate does not match its FIFO rate");

  int dev = desc->device;
  if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) return fail(nullptr, PRUNE_ECUDA, "no CUDA device");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0 || dev >= ndev)
    return fail(nullptr, PRUNE_ECUDA, "no CUDA device (this library has no CPU path)");
  DeviceGuard dg(dev);
  if (!dg.ok) return fail(nullptr, PRUNE_ECUDA, "cudaSetDevice failed");

  prune_graph *g = new prune_graph();
  g->d = *desc;
  g->d.taps = nullptr;
  g->d.H = nullptr;
  g->dev = dev;
  g->C = C;
  g->out_cap = out_cap;
  g->L = F * desc->B;
  g->TP = fir_taps_padded(desc->T);
  g->TS = fir_tile_samples(desc->B);
  g->tiles = static_cast<int32_t>((g->L + g->TS - 1) / g->TS);
  g->budget = desc->hbm_budget;
  cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, dev);
  g->cap[0] = eq2_capacity(F, 0, C);
  g->cap[1] = eq2_capacity(1, 1, C);
  g->cap[2] = eq2_capacity(F, 0, C);
  g->cap[3] = eq2_capacity(F, 0, C);
  g->cap[4] = eq2_capacity(1, 0, C);
  g->cap[5] = eq2_capacity(1, 0, C);
  g->cap[6] = F * eq2_capacity(1, 0, C);  // F DC FIFOs of capacity C each
  g->cap[7] = F * eq2_capacity(1, 0, C);

  auto bail = [&](prune_status s) {
    t_create_error = g->err;
    prune_graph_destroy(g);
    return s;
  };
  prune_status s;
  if (desc->stream) {
    g->stream = static_cast<cudaStream_t>(desc->stream);
  } else {
    if (cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking) != cudaSuccess) {
      g->err = "cudaStreamCreate failed";
      return bail(PRUNE_ECUDA);
    }
    g->own_stream = true;
  }
  if (cudaStreamCreateWithFlags(&g->pull_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaHostAlloc(reinterpret_cast<void **>(&g->pull_c), sizeof(int32_t) * out_cap, 0) != cudaSuccess ||
      cudaHostAlloc(reinterpret_cast<void **>(&g->pull_frame), sizeof(int64_t) * out_cap, 0) != cudaSuccess ||
      cudaHostAlloc(reinterpret_cast<void **>(&g->pull_status), sizeof(uint32_t) * 4, 0) != cudaSuccess) {
    g->err = "pull stream or staging allocation failed";
    return bail(PRUNE_ECUDA);
  }
  const int64_t L = g->L;
  const int32_t T = desc->T, N = desc->N;
  const size_t hist_len = static_cast<size_t>(std::max(T - 1, 1));
  if ((s = galloc(g, &g->taps, T)) || (s = galloc(g, &g->H, static_cast<size_t>(N) * N)) ||
      (s = galloc(g, &g->f0_ring, static_cast<size_t>(C))) || (s = galloc(g, &g->hist, 2 * hist_len)) ||
      (s = galloc(g, &g->energy, static_cast<size_t>(C) * F)) ||
      (s = galloc(g, &g->rec_c, static_cast<size_t>(out_cap))) ||
      (s = galloc(g, &g->rec_frame, static_cast<size_t>(out_cap))) ||
      (s = galloc(g, &g->rec_idx, static_cast<size_t>(out_cap) * F)) ||
      (s = galloc(g, &g->rec_y, static_cast<size_t>(out_cap) * L)) ||
      (s = galloc(g, &g->ctr, kNumFifos * 3)) || (s = galloc(g, &g->status, 4)) ||
      (s = galloc(g, &g->loop, 1)) || (s = galloc(g, &g->look, static_cast<size_t>(C) * g->tiles)) ||
      (s = galloc(g, &g->done, static_cast<size_t>(C))) || (s = galloc(g, &g->ready, static_cast<size_t>(C))))
    return bail(s);
  if (const char *kk = std::getenv("PRUNE_TC_KERNEL")) g->ws_loop = std::string(kk) != "pipes";
  if (const char *tm = std::getenv("PRUNE_TIMEOUT_MS")) {
    const long long ms = std::atoll(tm);
    if (ms > 0) g->timeout_ns = static_cast<uint64_t>(ms) * 1000000ull;
  }
  // The staging ring (copied pushes) and the FIR output ring (the
  // actor-per-kernel path) are allocated when first needed; a graph whose
  // runs all take the actor path (N >= 64) gets its FIR output ring now.
  if (!loop_supported(N) && (s = galloc(g, &g->y_ring, static_cast<size_t>(C) * L))) return bail(s);
  if (N >= 64 && hx_tc_supported(N)) {
    if ((s = galloc(g, &g->hx_b_ops, hx_tc_b_elems(N)))) return bail(s);
  }
  if (tc_loop_supported(N, desc->B, T)) {
    if ((s = galloc(g, &g->tc_fir_ops, tc_fir_ops_elems(T))) || (s = galloc(g, &g->tc_hx_ops, tc_hx_ops_elems())))
      return bail(s);
  }
  auto upload = [&](void *dst, const void *src, size_t bytes) {
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, g->stream) == cudaSuccess;
  };
  bool ok = upload(g->taps, desc->taps, sizeof(float2) * T) &&
            upload(g->H, desc->H, sizeof(float2) * N * N) &&
            cudaMemsetAsync(g->hist, 0, sizeof(float2) * 2 * hist_len, g->stream) == cudaSuccess &&
            cudaMemsetAsync(g->ctr, 0, sizeof(uint64_t) * kNumFifos * 3, g->stream) == cudaSuccess &&
            cudaMemsetAsync(g->status, 0, sizeof(uint32_t) * 4, g->stream) == cudaSuccess &&
            cudaMemsetAsync(g->loop, 0, sizeof(LoopScratch), g->stream) == cudaSuccess &&
            cudaMemsetAsync(g->f0_ring, 0, sizeof(void *) * C, g->stream) == cudaSuccess &&
            cudaMemsetAsync(g->look, 0, sizeof(uint64_t) * C * g->tiles, g->stream) == cudaSuccess &&
            cudaMemsetAsync(g->done, 0, sizeof(uint32_t) * C, g->stream) == cudaSuccess &&
            cudaMemsetAsync(g->ready, 0, sizeof(uint64_t) * C, g->stream) == cudaSuccess &&
            cudaMemsetAsync(g->rec_c, 0, sizeof(int32_t) * out_cap, g->stream) == cudaSuccess;
  g->tcs = tc_scale_of(desc->taps, T, desc->H, N);
  if (ok && g->hx_b_ops) ok = hx_tc_prepare_b(g->H, N, g->tcs.s_h, nullptr, g->hx_b_ops, g->stream) == cudaSuccess;
  if (ok && g->tc_fir_ops)
    ok = tc_prepare_ops(g->taps, T, g->H, g->tcs, g->tc_fir_ops, g->tc_hx_ops, g->stream) == cudaSuccess;
  // the initial delay token of f1 is present from the start (Q = 1)
  if (ok) {
    const uint64_t init[3] = {0, 0, 1};
    ok = cudaMemcpyAsync(g->ctr + 1 * 3, init, sizeof init, cudaMemcpyHostToDevice, g->stream) == cudaSuccess;
  }
  if (!ok || cudaStreamSynchronize(g->stream) != cudaSuccess) {
    g->err = std::string("graph upload failed: ") + cudaGetErrorString(cudaGetLastError());
    return bail(PRUNE_ECUDA);
  }
  *out = g;
  return PRUNE_OK;
}

prune_status prune_push_frames(prune_graph *g, const void *x, int32_t n, int32_t mem) {
  if (!g) return fail(nullptr, PRUNE_EINVAL, "prune_push_frames: NULL graph");
  if (g->poisoned) return fail(g, g->poison_code, "graph is poisoned by an earlier device error: " + g->err);
  if (n < 0 || (n > 0 && !x)) return fail(g, PRUNE_EINVAL, "prune_push_frames: bad x or n");
  if (mem != PRUNE_MEM_HOST && mem != PRUNE_MEM_DEVICE && mem != PRUNE_MEM_DEVICE_BORROW)
    return fail(g, PRUNE_EINVAL, "prune_push_frames: mem must be HOST, DEVICE or DEVICE_BORROW");
  if (mem != PRUNE_MEM_HOST && (reinterpret_cast<uintptr_t>(x) & 15u))
    return fail(g, PRUNE_EINVAL, "prune_push_frames: device frames must be 16-byte aligned");
  if (g->pushed - g->fired + n > g->C)
    return fail(g, PRUNE_EAGAIN, "f0 is full: " + std::to_string(g->pushed - g->fired) + " of " +
                                     std::to_string(g->C) + " frames waiting");
  DeviceGuard dg(g->dev);
  if (mem != PRUNE_MEM_DEVICE_BORROW && n > 0 && !g->stage) {  // the first copied push: the staging ring
    const prune_status s = galloc(g, &g->stage, static_cast<size_t>(g->C) * g->L);
    if (s != PRUNE_OK) return s;
  }
  const float2 *src = static_cast<const float2 *>(x);
  const size_t fbytes = static_cast<size_t>(g->L) * sizeof(float2);
  for (int32_t i0 = 0; i0 < n; i0 += 64) {
    const int32_t cnt = std::min(64, n - i0);
    PushPtrs ptrs{};
    for (int32_t i = 0; i < cnt; ++i) {
      const int64_t seq = g->pushed + i0 + i;
      const float2 *fi = src + static_cast<int64_t>(i0 + i) * g->L;
      if (mem == PRUNE_MEM_DEVICE_BORROW) {
        ptrs.p[i] = fi;
      } else {
        float2 *dst = g->stage + (seq % g->C) * g->L;
        CU(g, cudaMemcpyAsync(dst, fi, fbytes, mem == PRUNE_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                              g->stream));
        ptrs.p[i] = dst;
      }
    }
    KTimer kt(g, 0);
    f0_push_kernel<<<1, 64, 0, g->stream>>>(g->f0_ring, g->C, g->pushed + i0, cnt, ptrs, g->ctr, g->status, g->d.F,
                                            static_cast<uint64_t>(g->cap[0]));
    CU(g, cudaGetLastError());
  }
  g->pushed += n;
  return PRUNE_OK;
}

prune_status prune_run(prune_graph *g, int32_t max_frames, int32_t *n_fired, int32_t flags) {
  if (n_fired) *n_fired = 0;
  if (!g) return fail(nullptr, PRUNE_EINVAL, "prune_run: NULL graph");
  if (g->poisoned) return fail(g, g->poison_code, "graph is poisoned by an earlier device error: " + g->err);
  if (max_frames < 0) return fail(g, PRUNE_EINVAL, "prune_run: max_frames < 0");
  // Blocking rules on the host view: frames present in f0, room in the result ring.
  const bool device_rule = (flags & PRUNE_RUN_DEVICE_RULE) != 0;
  if (device_rule && ((flags & PRUNE_RUN_ACTORS) || !loop_supported(g->d.N)))
    return fail(g, PRUNE_EINVAL, "PRUNE_RUN_DEVICE_RULE needs the fused firing loop");
  const int64_t ready = device_rule ? g->C - (g->fired - std::min(g->pushed, g->fired)) : g->pushed - g->fired;
  const int64_t room = g->out_cap - (g->fired - g->pulled);
  const int32_t n = static_cast<int32_t>(std::min<int64_t>({static_cast<int64_t>(max_frames), ready, room}));
  DeviceGuard dg(g->dev);
  if (n > 0) {
    prune_status s;
    if ((flags & PRUNE_RUN_ACTORS) || !loop_supported(g->d.N)) s = run_actor_kernels(g, g->fired, n);
    else s = run_firing_loop(g, g->fired, n, flags);
    if (s != PRUNE_OK) return s;
    g->fired += n;
    g->runs++;
    cudaEvent_t ev = nullptr;
    if (!g->run_ev_pool.empty()) {
      ev = g->run_ev_pool.back();
      g->run_ev_pool.pop_back();
    } else {
      CU(g, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    }
    CU(g, cudaEventRecord(ev, g->stream));
    g->run_ends.emplace_back(g->fired, ev);
  }
  if (n_fired) *n_fired = n;
  if (flags & PRUNE_RUN_SYNC) return sync_and_check(g);
  return PRUNE_OK;
}

prune_status prune_sync(prune_graph *g) {
  if (!g) return fail(nullptr, PRUNE_EINVAL, "prune_sync: NULL graph");
  if (g->poisoned) return fail(g, g->poison_code, g->err);
  DeviceGuard dg(g->dev);
  return sync_and_check(g);
}

prune_status prune_pull(prune_graph *g, prune_frame_out *outs, int32_t max, int32_t *n, int32_t mem) {
  if (n) *n = 0;
  if (!g) return fail(nullptr, PRUNE_EINVAL, "prune_pull: NULL graph");
  if (g->poisoned) return fail(g, g->poison_code, g->err);
  if (max < 0 || (max > 0 && !outs && mem != PRUNE_MEM_DISCARD))
    return fail(g, PRUNE_EINVAL, "prune_pull: bad outs or max");
  if (mem != PRUNE_MEM_HOST && mem != PRUNE_MEM_DEVICE && mem != PRUNE_MEM_DISCARD)
    return fail(g, PRUNE_EINVAL, "prune_pull: mem must be HOST, DEVICE or DISCARD");
  const int64_t avail = g->fired - g->pulled;
  if (avail == 0) return fail(g, PRUNE_EAGAIN, "no fired frame is waiting");
  DeviceGuard dg(g->dev);
  if (mem == PRUNE_MEM_DISCARD && outs == nullptr) {
    // Stream-ordered drop: later firings reuse the slots after this work.
    const int32_t cnt = static_cast<int32_t>(std::min<int64_t>(avail, max));
    g->pulled += cnt;
    recycle_run_events(g);
    if (n) *n = cnt;
    return PRUNE_OK;
  }
  const int32_t cnt = static_cast<int32_t>(std::min<int64_t>(avail, max));
  const int64_t last = g->pulled + cnt;  // records [pulled, last)
  // after the run that fired the last record, on the pull stream
  cudaEvent_t ev = nullptr;
  for (auto &r : g->run_ends)
    if (r.first >= last) {
      ev = r.second;
      break;
    }
  if (!ev) return fail(g, PRUNE_EINVAL, "prune_pull: no run fired these records");
  cudaStream_t ps = g->pull_stream;
  CU(g, cudaStreamWaitEvent(ps, ev, 0));
  const int64_t s0 = g->pulled % g->out_cap;
  const int64_t n1 = std::min<int64_t>(cnt, g->out_cap - s0);  // the ring wraps after n1 records
  CU(g, cudaMemcpyAsync(g->pull_c, g->rec_c + s0, sizeof(int32_t) * n1, cudaMemcpyDeviceToHost, ps));
  CU(g, cudaMemcpyAsync(g->pull_frame, g->rec_frame + s0, sizeof(int64_t) * n1, cudaMemcpyDeviceToHost, ps));
  if (cnt > n1) {
    CU(g, cudaMemcpyAsync(g->pull_c + n1, g->rec_c, sizeof(int32_t) * (cnt - n1), cudaMemcpyDeviceToHost, ps));
    CU(g, cudaMemcpyAsync(g->pull_frame + n1, g->rec_frame, sizeof(int64_t) * (cnt - n1), cudaMemcpyDeviceToHost, ps));
  }
  CU(g, cudaMemcpyAsync(g->pull_status, g->status, sizeof(uint32_t) * 4, cudaMemcpyDeviceToHost, ps));
  CU(g, cudaStreamSynchronize(ps));
  {
    const uint32_t st[4] = {g->pull_status[0], g->pull_status[1], g->pull_status[2], g->pull_status[3]};
    const prune_status s = status_words(g, st);
    if (s != PRUNE_OK) return s;
  }
  const cudaMemcpyKind kind = mem == PRUNE_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  for (int32_t i = 0; i < cnt; ++i) {
    const int64_t slot = (g->pulled + i) % g->out_cap;
    const int32_t c = g->pull_c[i];
    if (outs) {
      outs[i].frame = g->pull_frame[i];
      outs[i].c = c;
      if (mem != PRUNE_MEM_DISCARD && c > 0) {
        if (!outs[i].idx || !outs[i].y) return fail(g, PRUNE_EINVAL, "prune_pull: idx and y buffers are required");
        CU(g, cudaMemcpyAsync(outs[i].idx, g->rec_idx + slot * g->d.F, sizeof(int32_t) * c, kind, ps));
        CU(g, cudaMemcpyAsync(outs[i].y, g->rec_y + slot * g->L, sizeof(float2) * static_cast<size_t>(c) * g->d.B,
                              kind, ps));
      }
    }
  }
  CU(g, cudaStreamSynchronize(ps));
  g->pulled += cnt;
  recycle_run_events(g);
  if (n) *n = cnt;
  return PRUNE_OK;
}

prune_status prune_peek(prune_graph *g, int32_t i, prune_frame_view *view) {
  if (!g || !view || i < 0) return fail(g, PRUNE_EINVAL, "prune_peek: bad argument");
  if (g->poisoned) return fail(g, g->poison_code, g->err);
  if (g->fired - g->pulled <= i) return fail(g, PRUNE_EAGAIN, "prune_peek: no such record");
  DeviceGuard dg(g->dev);
  prune_status s = sync_and_check(g);
  if (s != PRUNE_OK) return s;
  const int64_t slot = (g->pulled + i) % g->out_cap;
  CU(g, cudaMemcpy(&view->c, g->rec_c + slot, sizeof view->c, cudaMemcpyDeviceToHost));
  CU(g, cudaMemcpy(&view->frame, g->rec_frame + slot, sizeof view->frame, cudaMemcpyDeviceToHost));
  view->idx = g->rec_idx + slot * g->d.F;
  view->y = g->rec_y + slot * g->L;
  return PRUNE_OK;
}

prune_status prune_fifo_stats(prune_graph *g, int32_t fifo, uint64_t *written, uint64_t *read, uint64_t *peak) {
  if (!g || fifo < 0 || fifo >= PRUNE_NUM_FIFOS) return fail(g, PRUNE_EINVAL, "prune_fifo_stats: bad argument");
  DeviceGuard dg(g->dev);
  CU(g, cudaStreamSynchronize(g->stream));
  uint64_t c[3];
  CU(g, cudaMemcpy(c, g->ctr + fifo * 3, sizeof c, cudaMemcpyDeviceToHost));
  if (written) *written = c[0];
  if (read) *read = c[1];
  if (peak) *peak = c[2];
  return g->poisoned ? g->poison_code : PRUNE_OK;
}

prune_status prune_fifo_capacity_of(prune_graph *g, int32_t fifo, int64_t *cap) {
  if (!g || !cap || fifo < 0 || fifo >= PRUNE_NUM_FIFOS) return fail(g, PRUNE_EINVAL, "prune_fifo_capacity_of: bad argument");
  *cap = g->cap[fifo];
  return PRUNE_OK;
}

prune_status prune_profile(prune_graph *g, int32_t enable) {
  if (!g) return fail(nullptr, PRUNE_EINVAL, "prune_profile: NULL graph");
  g->profile = enable != 0;
  return PRUNE_OK;
}

prune_status prune_kernel_times(prune_graph *g, int32_t kind, double *ms, int64_t *launches, int32_t reset) {
  if (!g || kind < 0 || kind >= 8) return fail(g, PRUNE_EINVAL, "prune_kernel_times: bad argument");
  DeviceGuard dg(g->dev);
  CU(g, cudaStreamSynchronize(g->stream));
  drain_timers(g);
  if (ms) *ms = g->kind_ms[kind];
  if (launches) *launches = g->kind_n[kind];
  if (reset) {
    g->kind_ms[kind] = 0.0;
    g->kind_n[kind] = 0;
  }
  return PRUNE_OK;
}

// ------------------------------------------------------ single-actor entries

prune_status prune_fir_energy(const void *x, const void *hist, const void *taps, int32_t F, int32_t B, int32_t T,
                              int32_t frames, void *y, float *energy, void *hist_out, void *stream) {
  std::string why;
  if (!shape_ok(F, B, T, 1, &why)) return fail(nullptr, PRUNE_EINVAL, why);
  if (!x || !taps || frames < 0) return fail(nullptr, PRUNE_EINVAL, "prune_fir_energy: bad argument");
  if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) & 15u)
    return fail(nullptr, PRUNE_EINVAL, "prune_fir_energy: x and y must be 16-byte aligned");
  if (frames == 0) return PRUNE_OK;
  const int64_t L = static_cast<int64_t>(F) * B;
  FirParams fp{};
  fp.src = FrameSrc{nullptr, static_cast<const float2 *>(x), L, 0, 1};
  fp.L = L;
  fp.F = F; fp.B = B; fp.T = T; fp.TP = fir_taps_padded(T); fp.TS = fir_tile_samples(B);
  fp.tiles = static_cast<int32_t>((L + fp.TS - 1) / fp.TS); fp.frames = frames;
  fp.taps = static_cast<const float2 *>(taps);
  fp.hist = T > 1 ? static_cast<const float2 *>(hist) : nullptr;
  fp.hist_out = T > 1 ? static_cast<float2 *>(hist_out) : nullptr;
  fp.y = static_cast<float2 *>(y); fp.y_stride = L; fp.yslot = SlotMap{0, INT_MAX};
  fp.energy = energy; fp.eslot = SlotMap{0, INT_MAX};
  fir_energy_kernel<<<dim3(fp.tiles, frames), kFirThreads, fir_smem_bytes(T), static_cast<cudaStream_t>(stream)>>>(fp);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(nullptr, PRUNE_ECUDA, std::string("prune_fir_energy: ") + cudaGetErrorString(e));
  return PRUNE_OK;
}

prune_status prune_det_sel(const float *energy, int32_t F, int32_t frames, float tau, int32_t *c, int32_t *idx,
                           void *stream) {
  if (!energy || !c || !idx || F < 1 || frames < 0 || std::isnan(tau))
    return fail(nullptr, PRUNE_EINVAL, "prune_det_sel: bad argument");
  if (frames == 0) return PRUNE_OK;
  DetSelParams dp{};
  dp.energy = energy; dp.eslot = SlotMap{0, INT_MAX};
  dp.F = F; dp.frames = frames; dp.tau = tau;
  dp.c = c; dp.idx = idx; dp.rslot = SlotMap{0, INT_MAX};
  det_sel_kernel<<<frames, kDetThreads, 0, static_cast<cudaStream_t>(stream)>>>(dp);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(nullptr, PRUNE_ECUDA, std::string("prune_det_sel: ") + cudaGetErrorString(e));
  return PRUNE_OK;
}

prune_status prune_hx(const void *y, const int32_t *idx, const int32_t *c, int32_t F, int32_t B, int32_t N,
                      int32_t frames, const void *H, void *out, void *stream) {
  std::string why;
  if (!shape_ok(F, B, 1, N, &why)) return fail(nullptr, PRUNE_EINVAL, why);
  if (!y || !idx || !c || !H || !out || frames < 0) return fail(nullptr, PRUNE_EINVAL, "prune_hx: bad argument");
  if ((reinterpret_cast<uintptr_t>(y) | reinterpret_cast<uintptr_t>(out)) & 15u)
    return fail(nullptr, PRUNE_EINVAL, "prune_hx: y and out must be 16-byte aligned");
  if (frames == 0) return PRUNE_OK;
  const int64_t L = static_cast<int64_t>(F) * B;
  HxParams hp{};
  hp.y = static_cast<const float2 *>(y); hp.y_stride = L; hp.yslot = SlotMap{0, INT_MAX};
  hp.c = c; hp.idx = idx; hp.rslot = SlotMap{0, INT_MAX};
  hp.out = static_cast<float2 *>(out); hp.out_stride = L; hp.oslot = SlotMap{0, INT_MAX};
  hp.H = static_cast<const float2 *>(H); hp.F = F; hp.B = B; hp.N = N; hp.frames = frames;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e;
  if (N >= 64 && hx_tc_supported(N)) {
    // H is on the device here: its exponent is found there too (a word after
    // the operands), read by the preparation and the HX kernel
    uint16_t *bops = nullptr;
    e = cudaMallocAsync(reinterpret_cast<void **>(&bops), hx_tc_b_elems(N) * sizeof(uint16_t) + 16, s);
    int32_t *sh_dev = bops ? reinterpret_cast<int32_t *>(bops + hx_tc_b_elems(N)) : nullptr;
    if (e == cudaSuccess) e = tc_shift_of(hp.H, static_cast<int64_t>(N) * N, sh_dev, s);
    if (e == cudaSuccess) e = hx_tc_prepare_b(hp.H, N, 0, sh_dev, bops, s);
    if (e == cudaSuccess) e = launch_hx_tc(hp, bops, 0, sh_dev, sms, s);
    if (bops) cudaFreeAsync(bops, s);
  } else {
    e = launch_hx_cuda(hp, hx_grid(sms, static_cast<int64_t>(frames) * F), s);
  }
  if (e != cudaSuccess) return fail(nullptr, PRUNE_ECUDA, std::string("prune_hx: ") + cudaGetErrorString(e));
  return PRUNE_OK;
}

}  // extern "C"
