// Request loop (prune_server_*): streams admitted against a device-memory
// budget, their parameters, delay tokens and result FIFOs resident in one
// arena, and steps that fire the next frames of every ready stream in the
// batched launches (one entry per (stream, frame)).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <deque>
#include <map>
#include <cstdlib>
#include <string>
#include <vector>

#include "prune.h"
#include "batch.cuh"
#include "serve_host.hpp"

using namespace prune;

void prune_set_create_error(const std::string &m);  // prune_runtime.cu

struct prune_server {
  prune_server_desc d{};
  int dev = 0, sms = 148, tp_max = 8, TS = 0;
  bool fir_tc = false;  // FIR on tensor cores (4096-sample tiles, per-stream tap operands)
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  unsigned char *arena_base = nullptr;
  Arena arena;
  uint64_t bops_bytes = 0;
  std::vector<StreamState> streams;    // slot table
  std::vector<uint8_t> slot_used;
  std::vector<int32_t> order;          // open slots in admission order
  std::map<int64_t, int32_t> slot_of;  // stream id -> slot
  std::vector<int32_t> pending_free;   // closed slots waiting for their last step
  int64_t next_id = 1;
  // staging of the step tables, one set per step in flight
  struct Stage {
    BatchInst *inst_h = nullptr, *inst_d = nullptr;
    int2 *fir_h = nullptr, *fir_d = nullptr;
    int32_t *hx_h = nullptr, *hx_d = nullptr;
    int32_t *pre_d = nullptr;   // tensor-core HX work list (written by DET/SEL)
    uint32_t *ctr_d = nullptr;
    cudaEvent_t ev = nullptr;
  };
  std::vector<Stage> stage;
  int32_t max_entries = 0, max_fir = 0, max_hx = 0;
  struct Inflight { int64_t step; int32_t stage; std::vector<std::pair<int32_t, int32_t>> fired; };
  std::deque<Inflight> inflight;
  int64_t steps = 0, retired = -1;     // retired: last completed step
  std::vector<std::pair<int64_t, int64_t>> idle_events;  // (id, t_ns) not yet polled
  std::vector<uint8_t> idle_reported;
  float2 *param_h = nullptr;            // pinned staging of taps and H, one area per slot
  int64_t param_stride = 0;
  uint32_t *status = nullptr;
  std::string err = "no error";
};

namespace {

// Bytes of a stream's tensor-core FIR tap operands (0 when the FIR runs on
// CUDA cores).
uint64_t fops_bytes_of(const prune_server *s, int32_t T) {
  return s->fir_tc ? tc_fir_ops_elems(T) * sizeof(uint16_t) : 0;
}

prune_status sfail(prune_server *s, prune_status st, const std::string &m) {
  if (s) s->err = m;
  else prune_set_create_error(m);
  return st;
}

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

int64_t hx_items_of(int32_t F, int32_t B, int32_t N) {
  return N == kTcNc ? (static_cast<int64_t>(F) * (B / kTcNc) + kTcM - 1) / kTcM : F;
}

struct DevGuard {
  int prev = -1;
  explicit DevGuard(int dev) {
    cudaGetDevice(&prev);
    cudaSetDevice(dev);
  }
  ~DevGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

void mark_idle(prune_server *s, int32_t si) {
  StreamState &st = s->streams[si];
  if (!s->slot_used[si] || st.closing) return;
  if (st.queued == 0 && st.done == st.fired && st.fired > 0 && !s->idle_reported[si]) {
    s->idle_reported[si] = 1;
    s->idle_events.emplace_back(st.id, now_ns());
  }
}

// Apply the completion of in-flight steps (blocking on the oldest one when
// `wait_oldest`), then free the slots of closed streams whose last step is done.
prune_status retire(prune_server *s, bool wait_oldest) {
  while (!s->inflight.empty()) {
    prune_server::Inflight &f = s->inflight.front();
    cudaError_t e = wait_oldest ? cudaEventSynchronize(s->stage[f.stage].ev) : cudaEventQuery(s->stage[f.stage].ev);
    if (e == cudaErrorNotReady) break;
    if (e != cudaSuccess) return sfail(s, PRUNE_ECUDA, std::string("step completion: ") + cudaGetErrorString(e));
    wait_oldest = false;
    for (auto &p : f.fired) {
      StreamState &st = s->streams[p.first];
      st.done += p.second;
      if ((s->d.flags & PRUNE_SERVER_AUTO_RELEASE) && s->slot_used[p.first]) st.pulled = st.done;
    }
    s->retired = f.step;
    for (auto &p : f.fired) mark_idle(s, p.first);
    s->inflight.pop_front();
  }
  for (size_t i = 0; i < s->pending_free.size();) {
    const int32_t si = s->pending_free[i];
    StreamState &st = s->streams[si];
    if (st.last_step <= s->retired) {
      s->arena.release(st.mem);
      s->slot_used[si] = 0;
      st = StreamState{};
      s->pending_free.erase(s->pending_free.begin() + static_cast<std::ptrdiff_t>(i));
    } else {
      ++i;
    }
  }
  return PRUNE_OK;
}

StreamState *find(prune_server *s, int64_t id, int32_t *slot) {
  auto it = s->slot_of.find(id);
  if (it == s->slot_of.end()) return nullptr;
  if (slot) *slot = it->second;
  return &s->streams[it->second];
}

template <typename T>
T *at(prune_server *s, const StreamState &st, uint64_t off) {
  return reinterpret_cast<T *>(s->arena_base + st.mem + off);
}

}  // namespace

extern "C" {

prune_status prune_server_destroy(prune_server *s) {
  if (!s) return PRUNE_OK;
  DevGuard g(s->dev);
  if (s->stream) cudaStreamSynchronize(s->stream);
  for (auto &t : s->stage) {
    if (t.ev) cudaEventDestroy(t.ev);
    cudaFreeHost(t.inst_h);
    cudaFreeHost(t.fir_h);
    cudaFreeHost(t.hx_h);
    cudaFree(t.inst_d);
    cudaFree(t.fir_d);
    cudaFree(t.hx_d);
    cudaFree(t.pre_d);
    cudaFree(t.ctr_d);
  }
  cudaFree(s->arena_base);
  cudaFree(s->status);
  cudaFreeHost(s->param_h);
  if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
  delete s;
  return PRUNE_OK;
}

prune_status prune_server_create(const prune_server_desc *d, prune_server **out) {
  if (out) *out = nullptr;
  if (!d || !out) return sfail(nullptr, PRUNE_EINVAL, "prune_server_create: NULL argument");
  const int tpb = d->B / 8;
  if (d->B < 8 || d->B > kFirTile || d->B % 8 != 0 || !((tpb <= 32 && (tpb & (tpb - 1)) == 0) || tpb % 32 == 0) ||
      d->N < 1 || d->N > 128 || d->B % d->N != 0 || (d->N >= 64 && d->N != kTcNc) || d->F_max < 1 ||
      d->T_max < 1 || d->T_max > 256 || d->T_max - 1 > d->B || d->max_streams < 1 || d->max_streams > 65536 ||
      d->frames_per_step < 1 || d->ring < d->frames_per_step || d->max_inflight < 1 || d->max_inflight > 16 ||
      d->hbm_budget < 4096)
    return sfail(nullptr, PRUNE_EINVAL, "prune_server_create: bad descriptor");
  int dev = d->device;
  if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) return sfail(nullptr, PRUNE_ECUDA, "no CUDA device");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0 || dev >= ndev)
    return sfail(nullptr, PRUNE_ECUDA, "no CUDA device (this library has no CPU path)");
  DevGuard g(dev);
  prune_server *s = new prune_server();
  s->d = *d;
  s->dev = dev;
  {
    const char *fe = std::getenv("PRUNE_BATCH_FIR");
    s->fir_tc = batch_fir_tc_supported(d->B, d->T_max) && !(fe && std::string(fe) == "cuda_cores");
  }
  s->TS = s->fir_tc ? kTTile : fir_tile_samples(d->B);
  s->tp_max = fir_taps_padded(d->T_max);
  s->bops_bytes = d->N == kTcNc ? hx_tc_b_elems(d->N) * sizeof(uint16_t) : 0;
  cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, dev);
  auto bail = [&](prune_status st, const std::string &m) {
    prune_set_create_error(m);
    prune_server_destroy(s);
    return st;
  };
  if (d->stream) {
    s->stream = static_cast<cudaStream_t>(d->stream);
  } else if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) == cudaSuccess) {
    s->own_stream = true;
  } else {
    return bail(PRUNE_ECUDA, "prune_server_create: cudaStreamCreate failed");
  }
  if (cudaMalloc(&s->arena_base, d->hbm_budget) != cudaSuccess) {
    cudaGetLastError();
    return bail(PRUNE_ENOMEM, "prune_server_create: no device memory for the budget");
  }
  s->arena.reset(d->hbm_budget);
  if (cudaMalloc(&s->status, 16) != cudaSuccess || cudaMemsetAsync(s->status, 0, 16, s->stream) != cudaSuccess)
    return bail(PRUNE_ENOMEM, "prune_server_create: status word");
  s->param_stride = d->T_max + static_cast<int64_t>(d->N) * d->N;
  if (cudaHostAlloc(reinterpret_cast<void **>(&s->param_h), sizeof(float2) * s->param_stride * d->max_streams, 0) !=
      cudaSuccess)
    return bail(PRUNE_ENOMEM, "prune_server_create: parameter staging");
  s->streams.resize(d->max_streams);
  s->slot_used.assign(d->max_streams, 0);
  s->idle_reported.assign(d->max_streams, 0);
  s->max_entries = d->max_streams * d->frames_per_step;
  const int64_t L = static_cast<int64_t>(d->F_max) * d->B;
  const int64_t fir_per = (L + s->TS - 1) / s->TS, hx_per = hx_items_of(d->F_max, d->B, d->N);
  if (static_cast<int64_t>(s->max_entries) * std::max(fir_per, hx_per) > (int64_t{1} << 31) - 1)
    return bail(PRUNE_EINVAL, "prune_server_create: F_max x max_streams x frames_per_step too large");
  s->max_fir = static_cast<int32_t>(s->max_entries * fir_per);
  s->max_hx = static_cast<int32_t>(s->max_entries * hx_per);
  s->stage.resize(d->max_inflight);
  for (auto &t : s->stage) {
    if (cudaHostAlloc(reinterpret_cast<void **>(&t.inst_h), sizeof(BatchInst) * s->max_entries, 0) != cudaSuccess ||
        cudaHostAlloc(reinterpret_cast<void **>(&t.fir_h), sizeof(int2) * s->max_fir, 0) != cudaSuccess ||
        cudaHostAlloc(reinterpret_cast<void **>(&t.hx_h), sizeof(int32_t) * s->max_hx, 0) != cudaSuccess ||
        cudaMalloc(&t.inst_d, sizeof(BatchInst) * s->max_entries) != cudaSuccess ||
        cudaMalloc(&t.fir_d, sizeof(int2) * s->max_fir) != cudaSuccess ||
        cudaMalloc(&t.hx_d, sizeof(int32_t) * s->max_hx) != cudaSuccess ||
        cudaMalloc(&t.pre_d, sizeof(int32_t) * (s->max_entries + 1)) != cudaSuccess ||
        cudaMalloc(&t.ctr_d, sizeof(uint32_t)) != cudaSuccess ||
        cudaMemsetAsync(t.ctr_d, 0, sizeof(uint32_t), s->stream) != cudaSuccess ||
        cudaEventCreateWithFlags(&t.ev, cudaEventDisableTiming) != cudaSuccess)
      return bail(PRUNE_ENOMEM, "prune_server_create: step staging");
  }
  if (!batch_enable_smem(s->tp_max, d->B, d->N, s->fir_tc) || cudaStreamSynchronize(s->stream) != cudaSuccess)
    return bail(PRUNE_ECUDA, std::string("prune_server_create: ") + cudaGetErrorString(cudaGetLastError()));
  *out = s;
  return PRUNE_OK;
}

prune_status prune_server_open(prune_server *s, const prune_graph_desc *g, int64_t *id) {
  if (!s || !g || !id) return sfail(s, PRUNE_EINVAL, "prune_server_open: NULL argument");
  if (g->B != s->d.B || g->N != s->d.N || g->F < 1 || g->F > s->d.F_max || g->T < 1 || g->T > s->d.T_max ||
      !g->taps || !g->H || std::isnan(g->tau))
    return sfail(s, PRUNE_EINVAL, "prune_server_open: descriptor does not fit the server");
  DevGuard dg(s->dev);
  prune_status st = retire(s, false);
  if (st != PRUNE_OK) return st;
  int32_t slot = -1;
  for (int32_t i = 0; i < s->d.max_streams; ++i)
    if (!s->slot_used[i]) {
      slot = i;
      break;
    }
  if (slot < 0) return sfail(s, PRUNE_EAGAIN, "prune_server_open: every stream slot is taken");
  const int N = s->d.N;
  const StreamLayout l =
      stream_layout(g->F, s->d.B, g->T, N, s->d.frames_per_step, s->d.ring, s->bops_bytes, fops_bytes_of(s, g->T));
  uint64_t off = 0;
  if (!s->arena.alloc(l.total, &off))
    return sfail(s, PRUNE_EAGAIN, "prune_server_open: HBM budget: the stream needs " + std::to_string(l.total) +
                                      " bytes, the largest free hole holds " + std::to_string(s->arena.largest_free()));
  StreamState &ss = s->streams[slot];
  ss = StreamState{};
  ss.id = s->next_id++;
  ss.F = g->F;
  ss.T = g->T;
  ss.tau = g->tau;
  const TcScale sc = tc_scale_of(g->taps, g->T, g->H, N);
  ss.s_taps = sc.s_taps;
  ss.s_h = sc.s_h;
  ss.mem = off;
  ss.bytes = l.total;
  // through the slot's pinned staging (its previous user's copies completed
  // before that stream's memory was released), so nothing here waits for the
  // steps in flight
  float2 *ph = s->param_h + s->param_stride * slot;
  std::memcpy(ph, g->taps, sizeof(float2) * g->T);
  std::memcpy(ph + g->T, g->H, sizeof(float2) * N * N);
  bool ok = cudaMemcpyAsync(at<float2>(s, ss, l.taps), ph, sizeof(float2) * g->T, cudaMemcpyHostToDevice,
                            s->stream) == cudaSuccess &&
            cudaMemcpyAsync(at<float2>(s, ss, l.H), ph + g->T, sizeof(float2) * N * N, cudaMemcpyHostToDevice,
                            s->stream) == cudaSuccess &&
            cudaMemsetAsync(at<float2>(s, ss, l.hist), 0, sizeof(float2) * 2 * std::max(g->T - 1, 1), s->stream) ==
                cudaSuccess &&
            cudaMemsetAsync(at<int32_t>(s, ss, l.c), 0, sizeof(int32_t) * s->d.ring, s->stream) == cudaSuccess;
  if (ok && N == kTcNc)
    ok = hx_tc_prepare_b(at<float2>(s, ss, l.H), N, sc.s_h, nullptr, at<uint16_t>(s, ss, l.bops), s->stream) ==
         cudaSuccess;
  if (ok && s->fir_tc) {  // block-Toeplitz tap operands (split FP16, scaled by 2^s_taps)
    tc_prepare_fir_kernel<<<dim3(64, tc_shifts(g->T)), 64, 0, s->stream>>>(at<float2>(s, ss, l.taps), g->T,
                                                                            sc.s_taps, at<uint16_t>(s, ss, l.fops));
    ok = cudaGetLastError() == cudaSuccess;
  }
  if (!ok) {
    s->arena.release(off);
    ss = StreamState{};
    return sfail(s, PRUNE_ECUDA, std::string("prune_server_open: upload: ") + cudaGetErrorString(cudaGetLastError()));
  }
  s->slot_used[slot] = 1;
  s->idle_reported[slot] = 0;
  s->order.push_back(slot);
  s->slot_of[ss.id] = slot;
  *id = ss.id;
  return PRUNE_OK;
}

prune_status prune_server_submit(prune_server *s, int64_t id, const void *x, int64_t n, int64_t period) {
  if (!s) return sfail(nullptr, PRUNE_EINVAL, "prune_server_submit: NULL server");
  int32_t slot = -1;
  StreamState *st = find(s, id, &slot);
  if (!st || st->closing) return sfail(s, PRUNE_EINVAL, "prune_server_submit: unknown stream");
  if (!x || n < 0 || period < 1) return sfail(s, PRUNE_EINVAL, "prune_server_submit: bad arguments");
  if (reinterpret_cast<uintptr_t>(x) & 15u) return sfail(s, PRUNE_EINVAL, "prune_server_submit: x must be 16-byte aligned");
  if (n == 0) return PRUNE_OK;
  st->queue.push_back(Segment{x, n, period, 0});
  st->queued += n;
  s->idle_reported[slot] = 0;
  return PRUNE_OK;
}

prune_status prune_server_step(prune_server *s, int32_t *entries) {
  if (entries) *entries = 0;
  if (!s) return sfail(nullptr, PRUNE_EINVAL, "prune_server_step: NULL server");
  DevGuard dg(s->dev);
  prune_status st = retire(s, static_cast<int32_t>(s->inflight.size()) >= s->d.max_inflight);
  if (st != PRUNE_OK) return st;
  std::vector<PlanEntry> plan = plan_step(s->streams, s->order, s->d.B, s->d.frames_per_step, s->d.ring,
                                          s->max_entries);
  if (plan.empty()) return PRUNE_OK;
  const int32_t si = static_cast<int32_t>(s->steps % s->d.max_inflight);
  prune_server::Stage &t = s->stage[si];
  const int B = s->d.B, N = s->d.N, fps = s->d.frames_per_step;
  int32_t nfir = 0, nhx = 0, chain = 0, last_stream = -1;
  prune_server::Inflight rec{s->steps, si, {}};
  for (size_t e = 0; e < plan.size(); ++e) {
    const PlanEntry &p = plan[e];
    StreamState &ss = s->streams[p.stream];
    if (p.stream != last_stream) {
      chain = 0;
      last_stream = p.stream;
      rec.fired.emplace_back(p.stream, 0);
    }
    rec.fired.back().second++;
    const StreamLayout l = stream_layout(ss.F, B, ss.T, N, fps, s->d.ring, s->bops_bytes, fops_bytes_of(s, ss.T));
    const int64_t L = static_cast<int64_t>(ss.F) * B;
    const int64_t slot = p.frame % s->d.ring;
    BatchInst in{};
    in.x = static_cast<const float2 *>(p.x);
    in.taps = at<float2>(s, ss, l.taps);
    in.H = at<float2>(s, ss, l.H);
    in.bops = N == kTcNc ? at<uint16_t>(s, ss, l.bops) : nullptr;
    in.fops = s->fir_tc ? at<uint16_t>(s, ss, l.fops) : nullptr;
    in.hist = nullptr;
    float2 *hist = at<float2>(s, ss, l.hist);
    const int tm1 = std::max(ss.T - 1, 1);
    if (ss.T > 1) {
      in.hist_in = p.prev ? static_cast<const float2 *>(p.prev) + (L - (ss.T - 1)) : hist + ss.parity * tm1;
      in.hist_out = p.last ? hist + (1 - ss.parity) * tm1 : nullptr;
    }
    in.y = at<float2>(s, ss, l.y) + static_cast<int64_t>(chain) * L;
    in.energy = at<float>(s, ss, l.energy) + static_cast<int64_t>(chain) * ss.F;
    in.c = at<int32_t>(s, ss, l.c) + slot;
    in.idx = at<int32_t>(s, ss, l.idx) + slot * ss.F;
    in.out = at<float2>(s, ss, l.out) + slot * L;
    in.F = ss.F;
    in.T = ss.T;
    in.TP = fir_taps_padded(ss.T);
    in.tau = ss.tau;
    in.s_taps = ss.s_taps;
    in.s_h = ss.s_h;
    in.fir_tile0 = nfir;
    in.hx_tile0 = nhx;
    const int64_t tiles = (L + s->TS - 1) / s->TS, items = hx_items_of(ss.F, B, N);
    for (int64_t q = 0; q < tiles; ++q) t.fir_h[nfir++] = make_int2(static_cast<int32_t>(e), static_cast<int32_t>(q));
    for (int64_t q = 0; q < items; ++q) t.hx_h[nhx++] = static_cast<int32_t>(e);
    t.inst_h[e] = in;
    if (p.last && ss.T > 1) ss.parity ^= 1;
    ss.last_step = s->steps;
    ++chain;
  }
  const int32_t n = static_cast<int32_t>(plan.size());
  BatchParams bp{};
  bp.inst = t.inst_d;
  bp.fir_map = t.fir_d;
  bp.hx_map = t.hx_d;
  bp.fir_tc = s->fir_tc ? 1 : 0;
  bp.hx_pre = t.pre_d;
  bp.hx_ctr = t.ctr_d;
  bp.x = nullptr;
  bp.n = n;
  bp.B = B;
  bp.N = N;
  bp.TS = s->TS;
  bp.parity = 0;
  bp.fir_tiles = nfir;
  bp.hx_items = nhx;
  bp.timeout_ns = 2000000000ull;
  bp.status = s->status;
  bool ok = cudaMemcpyAsync(t.inst_d, t.inst_h, sizeof(BatchInst) * n, cudaMemcpyHostToDevice, s->stream) ==
                cudaSuccess &&
            cudaMemcpyAsync(t.fir_d, t.fir_h, sizeof(int2) * nfir, cudaMemcpyHostToDevice, s->stream) ==
                cudaSuccess &&
            cudaMemcpyAsync(t.hx_d, t.hx_h, sizeof(int32_t) * nhx, cudaMemcpyHostToDevice, s->stream) == cudaSuccess;
  cudaError_t e = ok ? batch_launch_step(bp, s->tp_max, s->sms, s->stream) : cudaGetLastError();
  if (e == cudaSuccess) e = cudaEventRecord(t.ev, s->stream);
  if (e != cudaSuccess) return sfail(s, PRUNE_ECUDA, std::string("prune_server_step: ") + cudaGetErrorString(e));
  s->inflight.push_back(std::move(rec));
  s->steps++;
  if (entries) *entries = n;
  return PRUNE_OK;
}

prune_status prune_server_progress(prune_server *s, int64_t id, int64_t *queued, int64_t *fired, int64_t *done,
                                   int64_t *pulled) {
  if (!s) return sfail(nullptr, PRUNE_EINVAL, "prune_server_progress: NULL server");
  DevGuard dg(s->dev);
  prune_status st = retire(s, false);
  if (st != PRUNE_OK) return st;
  StreamState *ss = find(s, id, nullptr);
  if (!ss) return sfail(s, PRUNE_EINVAL, "prune_server_progress: unknown stream");
  if (queued) *queued = ss->queued;
  if (fired) *fired = ss->fired;
  if (done) *done = ss->done;
  if (pulled) *pulled = ss->pulled;
  return PRUNE_OK;
}

prune_status prune_server_poll(prune_server *s, int64_t *ids, int64_t *t_ns, int32_t max, int32_t *n) {
  if (n) *n = 0;
  if (!s || !n || max < 0 || (max > 0 && !ids)) return sfail(s, PRUNE_EINVAL, "prune_server_poll: bad arguments");
  DevGuard dg(s->dev);
  prune_status st = retire(s, false);
  if (st != PRUNE_OK) return st;
  const int32_t k = std::min<int32_t>(max, static_cast<int32_t>(s->idle_events.size()));
  for (int32_t i = 0; i < k; ++i) {
    ids[i] = s->idle_events[i].first;
    if (t_ns) t_ns[i] = s->idle_events[i].second;
  }
  s->idle_events.erase(s->idle_events.begin(), s->idle_events.begin() + k);
  *n = k;
  return PRUNE_OK;
}

prune_status prune_server_pull(prune_server *s, int64_t id, prune_frame_out *out, int32_t mem) {
  if (!s) return sfail(nullptr, PRUNE_EINVAL, "prune_server_pull: NULL server");
  if (mem != PRUNE_MEM_HOST && mem != PRUNE_MEM_DEVICE && mem != PRUNE_MEM_DISCARD)
    return sfail(s, PRUNE_EINVAL, "prune_server_pull: mem");
  if (mem != PRUNE_MEM_DISCARD && !out) return sfail(s, PRUNE_EINVAL, "prune_server_pull: NULL out");
  DevGuard dg(s->dev);
  prune_status st = retire(s, false);
  if (st != PRUNE_OK) return st;
  StreamState *ss = find(s, id, nullptr);
  if (!ss) return sfail(s, PRUNE_EINVAL, "prune_server_pull: unknown stream");
  if (ss->pulled >= ss->done) return sfail(s, PRUNE_EAGAIN, "prune_server_pull: no done frame waiting");
  const int64_t f = ss->pulled;
  if (mem != PRUNE_MEM_DISCARD) {
    const StreamLayout l = stream_layout(ss->F, s->d.B, ss->T, s->d.N, s->d.frames_per_step, s->d.ring, s->bops_bytes,
                                         fops_bytes_of(s, ss->T));
    const int64_t slot = f % s->d.ring;
    int32_t c = 0;
    if (cudaMemcpy(&c, at<int32_t>(s, *ss, l.c) + slot, sizeof c, cudaMemcpyDeviceToHost) != cudaSuccess)
      return sfail(s, PRUNE_ECUDA, "prune_server_pull: copy failed");
    out->frame = f;
    out->c = c;
    if (c > 0) {
      if (!out->idx || !out->y) return sfail(s, PRUNE_EINVAL, "prune_server_pull: idx and y are required");
      const cudaMemcpyKind kind = mem == PRUNE_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
      if (cudaMemcpy(out->idx, at<int32_t>(s, *ss, l.idx) + slot * ss->F, sizeof(int32_t) * c, kind) != cudaSuccess ||
          cudaMemcpy(out->y, at<float2>(s, *ss, l.out) + slot * static_cast<int64_t>(ss->F) * s->d.B,
                     sizeof(float2) * static_cast<size_t>(c) * s->d.B, kind) != cudaSuccess)
        return sfail(s, PRUNE_ECUDA, "prune_server_pull: copy failed");
    }
  } else if (out) {
    out->frame = f;
    out->c = -1;
  }
  ss->pulled++;
  return PRUNE_OK;
}

prune_status prune_server_close(prune_server *s, int64_t id) {
  if (!s) return sfail(nullptr, PRUNE_EINVAL, "prune_server_close: NULL server");
  int32_t slot = -1;
  StreamState *ss = find(s, id, &slot);
  if (!ss) return sfail(s, PRUNE_EINVAL, "prune_server_close: unknown stream");
  ss->closing = true;
  ss->queue.clear();
  ss->queued = 0;
  s->slot_of.erase(id);
  s->order.erase(std::find(s->order.begin(), s->order.end(), slot));
  s->pending_free.push_back(slot);
  DevGuard dg(s->dev);
  return retire(s, false);
}

prune_status prune_server_sync(prune_server *s) {
  if (!s) return sfail(nullptr, PRUNE_EINVAL, "prune_server_sync: NULL server");
  DevGuard dg(s->dev);
  if (cudaStreamSynchronize(s->stream) != cudaSuccess)
    return sfail(s, PRUNE_ECUDA, std::string("prune_server_sync: ") + cudaGetErrorString(cudaGetLastError()));
  prune_status st = retire(s, false);
  if (st != PRUNE_OK) return st;
  uint32_t w[4] = {0, 0, 0, 0};
  if (cudaMemcpy(w, s->status, sizeof w, cudaMemcpyDeviceToHost) != cudaSuccess)
    return sfail(s, PRUNE_ECUDA, "prune_server_sync: status read failed");
  if (w[0] != 0)
    return sfail(s, w[0] == kDevTimeout ? PRUNE_ETIMEOUT : PRUNE_EDEVICE, "device error in a request-loop kernel");
  return PRUNE_OK;
}

prune_status prune_server_stats(prune_server *s, uint64_t *hbm_used, uint64_t *hbm_budget, int32_t *open,
                                int64_t *steps) {
  if (!s) return sfail(nullptr, PRUNE_EINVAL, "prune_server_stats: NULL server");
  if (hbm_used) *hbm_used = s->arena.used();
  if (hbm_budget) *hbm_budget = s->arena.size();
  if (open) *open = static_cast<int32_t>(s->order.size());
  if (steps) *steps = s->steps;
  return PRUNE_OK;
}

const char *prune_server_last_error(const prune_server *s) { return s ? s->err.c_str() : "NULL server"; }

}  // extern "C"
