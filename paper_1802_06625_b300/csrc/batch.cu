// Batched firing of many independent graph instances (prune_batch_*): one
// frame of every instance per step, three launches over the whole batch,
// optionally replayed as a captured CUDA graph.  The FIR runs on tensor
// cores (4096-sample tiles) when every instance has T <= 129 and B divides
// 4096 (PRUNE_BATCH_FIR=cuda_cores keeps it on CUDA cores).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "prune.h"
#include "batch.cuh"

using namespace prune;

void prune_set_create_error(const std::string &m);  // prune_runtime.cu

struct prune_batch {
  int32_t n = 0, B = 0, N = 0, TS = 0, tp_max = 8;
  bool fir_tc = false;  // FIR on tensor cores
  int dev = 0, sms = 148;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<void *> allocs;
  std::vector<int64_t> x_off, F, T;
  int64_t total_samples = 0;
  int32_t fir_tiles = 0, hx_items = 0;
  BatchInst *inst_d = nullptr;
  std::vector<BatchInst> inst_h;
  int2 *fir_map = nullptr;
  int32_t *fir_cta = nullptr;  // tensor-core FIR: per-CTA item ranges of equal estimated cost
  int32_t fir_ctas = 0;        // their count (0: equal counts)
  int32_t *hx_map = nullptr;
  int32_t *hx_pre = nullptr;   // N = 64: selected-tile prefix (written by DET/SEL each step)
  uint32_t *hx_ctr = nullptr;
  prune_batch_tuning tuning{};  // launch shape in use (prune_batch_autotune)
  uint32_t *status = nullptr;
  int64_t steps = 0;
  // captured step graphs keyed by (input pointer, parity)
  struct Cached { const void *x; int parity; cudaGraphExec_t exec; };
  std::vector<Cached> graphs;
  std::string err = "no error";
};

namespace {

prune_status bfail(prune_batch *b, prune_status s, const std::string &m) {
  if (b) b->err = m;
  else prune_set_create_error(m);
  return s;
}

template <typename T>
prune_status balloc(prune_batch *b, T **p, size_t count) {
  void *q = nullptr;
  cudaError_t e = cudaMalloc(&q, std::max<size_t>(count * sizeof(T), 16));
  if (e != cudaSuccess) return bfail(b, PRUNE_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  b->allocs.push_back(q);
  *p = static_cast<T *>(q);
  return PRUNE_OK;
}

// FIR CTAs in launch order: instance-major, or the tiles of the instances
// with the most taps first (a tile costs about 8T flop per sample, so the
// long tiles start first and the short ones fill the tail).
std::vector<int2> fir_order(const prune_batch *b, int32_t order) {
  std::vector<int32_t> inst(b->n);
  for (int32_t i = 0; i < b->n; ++i) inst[i] = i;
  if (order == 1)
    std::stable_sort(inst.begin(), inst.end(), [&](int32_t a, int32_t c) { return b->T[a] > b->T[c]; });
  std::vector<int2> m;
  m.reserve(b->fir_tiles);
  for (int32_t i : inst) {
    const int64_t tiles = (b->F[i] * b->B + b->TS - 1) / b->TS;
    for (int64_t t = 0; t < tiles; ++t) m.push_back(make_int2(i, static_cast<int32_t>(t)));
  }
  return m;
}

// The tensor-core FIR's per-CTA shares of the item order m (equal
// estimated cost), uploaded over b->fir_cta.
bool upload_fir_partition(prune_batch *b, const std::vector<int2> &m) {
  b->fir_ctas = 0;
  if (!b->fir_tc || b->fir_tiles == 0) return true;
  const int G = std::min(b->sms, b->fir_tiles);
  std::vector<int32_t> cta(static_cast<size_t>(G) + 1);
  fir_cost_partition(
      m.data(), b->fir_tiles, kTTile, G,
      [&](int32_t i, int64_t *samples, int *shifts) {
        *samples = b->F[i] * b->B;
        *shifts = tc_shifts(static_cast<int>(b->T[i]));
      },
      cta.data());
  if (cudaMemcpy(b->fir_cta, cta.data(), sizeof(int32_t) * cta.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return false;
  b->fir_ctas = G;
  return true;
}

prune_status enqueue_step(prune_batch *b, const float2 *x, int parity) {
  BatchParams bp{};
  bp.inst = b->inst_d;
  bp.fir_map = b->fir_map;
  bp.fir_cta = b->fir_ctas > 0 ? b->fir_cta : nullptr;
  bp.fir_ctas = b->fir_ctas;
  bp.hx_map = b->hx_map;
  bp.x = x;
  bp.n = b->n;
  bp.B = b->B;
  bp.N = b->N;
  bp.TS = b->TS;
  bp.parity = parity;
  bp.fir_tiles = b->fir_tiles;
  bp.hx_items = b->hx_items;
  bp.timeout_ns = 2000000000ull;
  bp.status = b->status;
  bp.hx_chunk = b->tuning.hx_chunk;
  bp.fir_tc = b->fir_tc ? 1 : 0;
  bp.hx_pre = b->hx_pre;
  bp.hx_ctr = b->hx_ctr;
  cudaError_t e = batch_launch_step(bp, b->tp_max, b->sms, b->stream, b->tuning.hx_grid);
  if (e != cudaSuccess) return bfail(b, PRUNE_ECUDA, std::string("batch launch: ") + cudaGetErrorString(e));
  return PRUNE_OK;
}

}  // namespace

extern "C" {

prune_status prune_batch_destroy(prune_batch *b) {
  if (!b) return PRUNE_OK;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(b->dev);
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (auto &c : b->graphs) cudaGraphExecDestroy(c.exec);
  for (void *p : b->allocs) cudaFree(p);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  if (prev >= 0) cudaSetDevice(prev);
  delete b;
  return PRUNE_OK;
}

prune_status prune_batch_create(const prune_graph_desc *descs, int32_t n, prune_batch **out) {
  if (out) *out = nullptr;
  if (!descs || !out || n < 1 || n > (1 << 20)) return bfail(nullptr, PRUNE_EINVAL, "prune_batch_create: bad arguments");
  const int32_t B = descs[0].B, N = descs[0].N;
  for (int32_t i = 0; i < n; ++i) {
    const prune_graph_desc &d = descs[i];
    const int tpb = d.B / 8;
    if (d.B != B || d.N != N) return bfail(nullptr, PRUNE_EINVAL, "prune_batch_create: all instances need the same B and N");
    if (d.F < 1 || d.B < 8 || d.B > kFirTile || d.B % 8 != 0 || !((tpb <= 32 && (tpb & (tpb - 1)) == 0) || tpb % 32 == 0) ||
        d.T < 1 || d.T > 256 || d.T - 1 > d.B || d.N < 1 || d.N > 128 || d.B % d.N != 0 || !d.taps || !d.H ||
        std::isnan(d.tau))
      return bfail(nullptr, PRUNE_EINVAL, "prune_batch_create: instance " + std::to_string(i) + " has a bad descriptor");
  }
  if (N >= 64 && N != kTcNc) return bfail(nullptr, PRUNE_EINVAL, "prune_batch_create: N >= 64 must be 64 (tensor cores)");
  int dev = descs[0].device;
  if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) return bfail(nullptr, PRUNE_ECUDA, "no CUDA device");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0 || dev >= ndev)
    return bfail(nullptr, PRUNE_ECUDA, "no CUDA device (this library has no CPU path)");
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(dev);
  prune_batch *b = new prune_batch();
  b->n = n;
  b->B = B;
  b->N = N;
  b->dev = dev;
  int t_max = 1;
  for (int32_t i = 0; i < n; ++i) t_max = std::max(t_max, descs[i].T);
  const char *fe = std::getenv("PRUNE_BATCH_FIR");
  b->fir_tc = batch_fir_tc_supported(B, t_max) && !(fe && std::string(fe) == "cuda_cores");
  b->TS = b->fir_tc ? kTTile : fir_tile_samples(B);
  cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
  auto bail = [&](prune_status s) {
    prune_set_create_error(b->err);
    prune_batch_destroy(b);
    if (prev >= 0) cudaSetDevice(prev);
    return s;
  };
  if (descs[0].stream) {
    b->stream = static_cast<cudaStream_t>(descs[0].stream);
  } else if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) == cudaSuccess) {
    b->own_stream = true;
  } else {
    b->err = "cudaStreamCreate failed";
    return bail(PRUNE_ECUDA);
  }
  // layout: per-instance offsets in shared buffers
  int64_t samples = 0, taps_n = 0, hist_n = 0, blocks = 0, fops_n = 0;
  std::vector<int32_t> hx_map;
  int64_t fir_count = 0;
  b->inst_h.resize(n);
  const int RB = N == kTcNc ? B / kTcNc : 0;
  for (int32_t i = 0; i < n; ++i) {
    const prune_graph_desc &d = descs[i];
    const int64_t L = static_cast<int64_t>(d.F) * B;
    BatchInst &in = b->inst_h[i];
    in.x_off = samples;
    in.F = d.F;
    in.T = d.T;
    in.TP = fir_taps_padded(d.T);
    in.tau = d.tau;
    b->tp_max = std::max(b->tp_max, in.TP);
    in.fir_tile0 = static_cast<int32_t>(fir_count);
    fir_count += (L + b->TS - 1) / b->TS;
    in.hx_tile0 = static_cast<int32_t>(hx_map.size());
    const int64_t items = N == kTcNc ? (static_cast<int64_t>(d.F) * RB + kTcM - 1) / kTcM : d.F;
    for (int64_t t = 0; t < items; ++t) hx_map.push_back(i);
    b->x_off.push_back(samples);
    b->F.push_back(d.F);
    b->T.push_back(d.T);
    samples += L;
    taps_n += d.T;
    hist_n += 2 * std::max(d.T - 1, 1);
    blocks += d.F;
    if (b->fir_tc) fops_n += static_cast<int64_t>(tc_fir_ops_elems(d.T));
  }
  b->total_samples = samples;
  if (fir_count > (int64_t{1} << 31) - 1) {
    b->err = "prune_batch_create: too many FIR tiles";
    return bail(PRUNE_EINVAL);
  }
  b->fir_tiles = static_cast<int32_t>(fir_count);
  const std::vector<int2> fir_map = fir_order(b, 0);
  b->hx_items = static_cast<int32_t>(hx_map.size());
  float2 *taps = nullptr, *H = nullptr, *hist = nullptr, *y = nullptr, *outb = nullptr;
  float *energy = nullptr;
  int32_t *c = nullptr, *idx = nullptr;
  uint16_t *bops = nullptr;
  prune_status s;
  if ((s = balloc(b, &taps, taps_n)) || (s = balloc(b, &H, static_cast<size_t>(n) * N * N)) ||
      (s = balloc(b, &hist, hist_n)) || (s = balloc(b, &y, samples)) || (s = balloc(b, &outb, samples)) ||
      (s = balloc(b, &energy, blocks)) || (s = balloc(b, &c, n)) || (s = balloc(b, &idx, blocks)) ||
      (s = balloc(b, &b->inst_d, n)) || (s = balloc(b, &b->fir_map, fir_map.size())) ||
      (s = balloc(b, &b->hx_map, hx_map.size())) || (s = balloc(b, &b->status, 4)))
    return bail(s);
  if (N == kTcNc && ((s = balloc(b, &bops, static_cast<size_t>(n) * hx_tc_b_elems(N))) ||
                     (s = balloc(b, &b->hx_pre, static_cast<size_t>(n) + 1)) || (s = balloc(b, &b->hx_ctr, 1))))
    return bail(s);
  uint16_t *fops = nullptr;
  if (b->fir_tc && ((s = balloc(b, &fops, static_cast<size_t>(fops_n))) ||
                    (s = balloc(b, &b->fir_cta, static_cast<size_t>(b->sms) + 1))))
    return bail(s);
  int64_t to = 0, ho = 0, bo = 0, fo = 0;
  bool ok = true;
  for (int32_t i = 0; i < n && ok; ++i) {
    const prune_graph_desc &d = descs[i];
    BatchInst &in = b->inst_h[i];
    in.taps = taps + to;
    in.H = H + static_cast<int64_t>(i) * N * N;
    in.bops = bops ? bops + static_cast<int64_t>(i) * hx_tc_b_elems(N) : nullptr;
    in.hist = hist + ho;
    in.y = y + in.x_off;
    in.out = outb + in.x_off;
    in.energy = energy + bo;
    in.c = c + i;
    in.idx = idx + bo;
    ok = cudaMemcpyAsync(const_cast<float2 *>(in.taps), d.taps, sizeof(float2) * d.T, cudaMemcpyHostToDevice,
                         b->stream) == cudaSuccess &&
         cudaMemcpyAsync(const_cast<float2 *>(in.H), d.H, sizeof(float2) * N * N, cudaMemcpyHostToDevice,
                         b->stream) == cudaSuccess;
    const TcScale sc = tc_scale_of(d.taps, d.T, d.H, N);
    in.s_taps = sc.s_taps;
    in.s_h = sc.s_h;
    if (ok && bops) ok = hx_tc_prepare_b(in.H, N, sc.s_h, nullptr, const_cast<uint16_t *>(in.bops), b->stream) == cudaSuccess;
    if (ok && fops) {  // block-Toeplitz tap operands (split FP16, scaled by 2^s_taps)
      in.fops = fops + fo;
      tc_prepare_fir_kernel<<<dim3(64, tc_shifts(d.T)), 64, 0, b->stream>>>(in.taps, d.T, sc.s_taps, fops + fo);
      ok = cudaGetLastError() == cudaSuccess;
      fo += static_cast<int64_t>(tc_fir_ops_elems(d.T));
    }
    to += d.T;
    ho += 2 * std::max(d.T - 1, 1);
    bo += d.F;
  }
  ok = ok && cudaMemsetAsync(hist, 0, sizeof(float2) * hist_n, b->stream) == cudaSuccess &&
       cudaMemsetAsync(c, 0, sizeof(int32_t) * n, b->stream) == cudaSuccess &&
       cudaMemsetAsync(b->status, 0, sizeof(uint32_t) * 4, b->stream) == cudaSuccess &&
       (!b->hx_ctr || cudaMemsetAsync(b->hx_ctr, 0, sizeof(uint32_t), b->stream) == cudaSuccess) &&
       cudaMemcpyAsync(b->inst_d, b->inst_h.data(), sizeof(BatchInst) * n, cudaMemcpyHostToDevice, b->stream) ==
           cudaSuccess &&
       cudaMemcpyAsync(b->fir_map, fir_map.data(), sizeof(int2) * fir_map.size(), cudaMemcpyHostToDevice,
                       b->stream) == cudaSuccess &&
       cudaMemcpyAsync(b->hx_map, hx_map.data(), sizeof(int32_t) * hx_map.size(), cudaMemcpyHostToDevice,
                       b->stream) == cudaSuccess;
  ok = ok && batch_enable_smem(b->tp_max, B, N, b->fir_tc);
  ok = ok && cudaStreamSynchronize(b->stream) == cudaSuccess && upload_fir_partition(b, fir_map);
  if (!ok || cudaStreamSynchronize(b->stream) != cudaSuccess) {
    b->err = std::string("batch upload failed: ") + cudaGetErrorString(cudaGetLastError());
    return bail(PRUNE_ECUDA);
  }
  if (prev >= 0) cudaSetDevice(prev);
  *out = b;
  return PRUNE_OK;
}

prune_status prune_batch_offset(prune_batch *b, int32_t i, int64_t *offset, int64_t *total) {
  if (!b || i < 0 || i >= b->n) return bfail(b, PRUNE_EINVAL, "prune_batch_offset: bad instance");
  if (offset) *offset = b->x_off[i];
  if (total) *total = b->total_samples;
  return PRUNE_OK;
}

prune_status prune_batch_fire(prune_batch *b, const void *x, int32_t flags) {
  if (!b || !x) return bfail(b, PRUNE_EINVAL, "prune_batch_fire: bad arguments");
  if (reinterpret_cast<uintptr_t>(x) & 15u) return bfail(b, PRUNE_EINVAL, "prune_batch_fire: x must be 16-byte aligned");
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(b->dev);
  const int parity = static_cast<int>(b->steps & 1);
  prune_status s = PRUNE_OK;
  if (flags & PRUNE_BATCH_GRAPH) {
    cudaGraphExec_t exec = nullptr;
    for (auto &c : b->graphs)
      if (c.x == x && c.parity == parity) exec = c.exec;
    if (!exec) {
      cudaGraph_t graph = nullptr;
      cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        s = enqueue_step(b, static_cast<const float2 *>(x), parity);
        e = cudaStreamEndCapture(b->stream, &graph);
      }
      if (e == cudaSuccess && s == PRUNE_OK) e = cudaGraphInstantiate(&exec, graph, 0);
      if (graph) cudaGraphDestroy(graph);
      if (e != cudaSuccess || s != PRUNE_OK) {
        if (prev >= 0) cudaSetDevice(prev);
        return s != PRUNE_OK ? s : bfail(b, PRUNE_ECUDA, std::string("batch graph capture: ") + cudaGetErrorString(e));
      }
      b->graphs.push_back({x, parity, exec});
    }
    cudaError_t e = cudaGraphLaunch(exec, b->stream);
    if (e != cudaSuccess) s = bfail(b, PRUNE_ECUDA, std::string("cudaGraphLaunch: ") + cudaGetErrorString(e));
  } else {
    s = enqueue_step(b, static_cast<const float2 *>(x), parity);
  }
  if (s == PRUNE_OK) b->steps++;
  if (prev >= 0) cudaSetDevice(prev);
  return s;
}

prune_status prune_batch_sync(prune_batch *b) {
  if (!b) return bfail(nullptr, PRUNE_EINVAL, "prune_batch_sync: NULL batch");
  if (cudaStreamSynchronize(b->stream) != cudaSuccess)
    return bfail(b, PRUNE_ECUDA, std::string("prune_batch_sync: ") + cudaGetErrorString(cudaGetLastError()));
  uint32_t st[4] = {0, 0, 0, 0};
  if (cudaMemcpy(st, b->status, sizeof st, cudaMemcpyDeviceToHost) != cudaSuccess)
    return bfail(b, PRUNE_ECUDA, "prune_batch_sync: status read failed");
  if (st[0] != 0) return bfail(b, st[0] == kDevTimeout ? PRUNE_ETIMEOUT : PRUNE_EDEVICE, "device error in a batch kernel");
  return PRUNE_OK;
}

prune_status prune_batch_pull(prune_batch *b, int32_t i, prune_frame_out *out, int32_t mem) {
  if (!b || i < 0 || i >= b->n || !out) return bfail(b, PRUNE_EINVAL, "prune_batch_pull: bad arguments");
  if (mem != PRUNE_MEM_HOST && mem != PRUNE_MEM_DEVICE) return bfail(b, PRUNE_EINVAL, "prune_batch_pull: mem");
  prune_status s = prune_batch_sync(b);
  if (s != PRUNE_OK) return s;
  const BatchInst &in = b->inst_h[i];
  int32_t c = 0;
  if (cudaMemcpy(&c, in.c, sizeof c, cudaMemcpyDeviceToHost) != cudaSuccess)
    return bfail(b, PRUNE_ECUDA, "prune_batch_pull: copy failed");
  out->frame = b->steps - 1;
  out->c = c;
  const cudaMemcpyKind kind = mem == PRUNE_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (c > 0) {
    if (!out->idx || !out->y) return bfail(b, PRUNE_EINVAL, "prune_batch_pull: idx and y are required");
    if (cudaMemcpy(out->idx, in.idx, sizeof(int32_t) * c, kind) != cudaSuccess ||
        cudaMemcpy(out->y, in.out, sizeof(float2) * static_cast<size_t>(c) * b->B, kind) != cudaSuccess)
      return bfail(b, PRUNE_ECUDA, "prune_batch_pull: copy failed");
  }
  return PRUNE_OK;
}

const char *prune_batch_last_error(const prune_batch *b) { return b ? b->err.c_str() : "NULL batch"; }

prune_status prune_batch_set_tuning(prune_batch *b, const prune_batch_tuning *t) {
  if (!b || !t || t->fir_order < 0 || t->fir_order > 1 || t->hx_chunk < 0 || t->hx_grid < 0)
    return bfail(b, PRUNE_EINVAL, "prune_batch_set_tuning: bad arguments");
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(b->dev);
  prune_status s = PRUNE_OK;
  if (t->fir_order != b->tuning.fir_order) {
    const std::vector<int2> m = fir_order(b, t->fir_order);
    if (cudaStreamSynchronize(b->stream) != cudaSuccess ||
        cudaMemcpy(b->fir_map, m.data(), sizeof(int2) * m.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        !upload_fir_partition(b, m))
      s = bfail(b, PRUNE_ECUDA, "prune_batch_set_tuning: map upload failed");
  }
  if (s == PRUNE_OK) {
    b->tuning = *t;
    for (auto &c : b->graphs) cudaGraphExecDestroy(c.exec);
    b->graphs.clear();
  }
  if (prev >= 0) cudaSetDevice(prev);
  return s;
}

prune_status prune_batch_get_tuning(const prune_batch *b, prune_batch_tuning *t) {
  if (!b || !t) return bfail(nullptr, PRUNE_EINVAL, "prune_batch_get_tuning: NULL argument");
  *t = b->tuning;
  return PRUNE_OK;
}

prune_status prune_batch_autotune(prune_batch *b, const void *x, int32_t reps, prune_batch_tuning *best,
                                  prune_batch_tuning *all, int32_t max_all, int32_t *n_all) {
  if (n_all) *n_all = 0;
  if (!b || !x || !best || reps < 1 || max_all < 0 || (max_all > 0 && !all))
    return bfail(b, PRUNE_EINVAL, "prune_batch_autotune: bad arguments");
  if (reinterpret_cast<uintptr_t>(x) & 15u) return bfail(b, PRUNE_EINVAL, "prune_batch_autotune: x must be 16-byte aligned");
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(b->dev);
  const int parity = static_cast<int>(b->steps & 1);
  const int wave = b->N == kTcNc ? b->sms : 8 * b->sms;
  std::vector<prune_batch_tuning> cand;
  for (int32_t order = 0; order < 2; ++order) {
    cand.push_back(prune_batch_tuning{order, 0, wave, 0, 0.0});
    for (int waves : {1, 2, 4}) {
      const int32_t chunk = std::max(1, (b->hx_items + waves * wave - 1) / (waves * wave));
      cand.push_back(prune_batch_tuning{order, chunk, 0, 0, 0.0});
    }
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  prune_status s = PRUNE_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    s = bfail(b, PRUNE_ECUDA, "prune_batch_autotune: event creation failed");
  int besti = -1;
  for (size_t i = 0; i < cand.size() && s == PRUNE_OK; ++i) {
    s = prune_batch_set_tuning(b, &cand[i]);
    if (s == PRUNE_OK) s = enqueue_step(b, static_cast<const float2 *>(x), parity);  // untimed
    if (s != PRUNE_OK) break;
    cudaEventRecord(e0, b->stream);
    for (int32_t r = 0; r < reps && s == PRUNE_OK; ++r) s = enqueue_step(b, static_cast<const float2 *>(x), parity);
    cudaEventRecord(e1, b->stream);
    if (s != PRUNE_OK) break;
    float ms = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      s = bfail(b, PRUNE_ECUDA, "prune_batch_autotune: timing failed");
      break;
    }
    cand[i].ms = ms / reps;
    if (besti < 0 || cand[i].ms < cand[besti].ms) besti = static_cast<int>(i);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s == PRUNE_OK) s = prune_batch_sync(b);
  if (s == PRUNE_OK) s = prune_batch_set_tuning(b, &cand[besti]);
  if (s == PRUNE_OK) {
    b->tuning.ms = cand[besti].ms;
    *best = cand[besti];
    const int32_t k = std::min<int32_t>(max_all, static_cast<int32_t>(cand.size()));
    for (int32_t i = 0; i < k; ++i) all[i] = cand[i];
    if (n_all) *n_all = k;
  }
  if (prev >= 0) cudaSetDevice(prev);
  return s;
}

}  // extern "C"
