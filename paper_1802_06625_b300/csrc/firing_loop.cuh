// Fused persistent firing loop: one launch fires FIR, DET, SEL, HX_b and SINK
// for a run of frames (actor merging, as the paper does for configuration
// actors in Sec. VII-A3; the dataflow semantics of Sec. III are unchanged).
//
// Persistent CTAs claim work items (frame k, tile t) from a ticket counter in
// order.  A work item:
//   1. checks the f0 firing rule on the device counters (bounded wait);
//   2. FIR: stages the tile window in shared memory and filters it;
//   3. DET: block energies and v[b] = (E_b > tau) for the tile's blocks;
//   4. SEL: warp ballot compaction inside the tile, then a decoupled look-back
//      over the previous tiles of the frame gives the tile's offset in the
//      frame's control token (c, idx) -- the control token never leaves the
//      device and never materialises the unselected blocks;
//   5. HX_b for every selected block straight from the tile's FIR output in
//      shared memory, written at its compacted position of the frame record;
//   6. the last tile of a frame to finish writes the record header (SINK)
//      and the FIFO counters of all actors of that frame.
// Waits are bounded by %globaltimer; a timeout sets the status word and an
// abort flag that makes every CTA leave.
#pragma once
#include "device_common.cuh"
#include "fir.cuh"

namespace prune {

struct LoopScratch {
  unsigned long long ticket;  // monotone work-item ticket counter
  unsigned long long booked;  // next frame whose FIFO counters are to be booked
  uint32_t abort;             // set by a CTA that gave up
  uint32_t book_lock;         // held by the thread that books frames in order
};

struct LoopParams {
  FirParams f;             // input frames, taps, shapes, delay token in/out, energies
  float tau;
  uint64_t *look;          // [C][tiles] look-back words: epoch:30 | flag:2 | value:32
  uint32_t *done;          // [C] finished tiles per frame slot (monotone)
  uint64_t *ready;         // [C] frame seq + 1 once the frame's record is final
  int32_t C;               // slots of look/done: frame seq % C
  int32_t *rec_c;
  int32_t *rec_idx;
  int64_t *rec_frame;
  float2 *rec_y;
  SlotMap rslot;
  const float2 *H;         // [N][N]
  int32_t N;
  LoopScratch *ls;
  unsigned long long ticket_base;
  uint64_t timeout_ns;
  uint64_t *ctr;
  uint32_t *status;
  uint64_t cap[8];
};

constexpr uint32_t kLookAgg = 1, kLookPrefix = 2;

__device__ __forceinline__ uint64_t look_pack(uint64_t epoch, uint32_t flag, uint32_t v) {
  return (epoch << 34) | (static_cast<uint64_t>(flag) << 32) | v;
}

// Spin until `pred` holds, bounded by timeout_ns; false on timeout or abort.
template <typename Pred>
__device__ __forceinline__ bool bounded_wait(const LoopParams &p, Pred pred, uint32_t actor, uint32_t fifo,
                                             uint64_t frame) {
  if (pred()) return true;
  const uint64_t t0 = globaltimer_ns();
  for (uint32_t it = 0;; ++it) {
    __nanosleep(64);
    if (pred()) return true;
    if ((it & 63u) == 63u) {
      if (ld_volatile_u32(&p.ls->abort)) return false;
      if (globaltimer_ns() - t0 > p.timeout_ns) {
        report_error(p.status, kDevTimeout, actor, fifo, frame);
        atomicExch(&p.ls->abort, 1u);
        return false;
      }
    }
  }
}

// Decoupled look-back, one warp: publish the tile's count as an aggregate,
// then read 32 predecessors per round trip, summing aggregates back to the
// nearest inclusive prefix; publish the inclusive prefix.  A look-back word
// (epoch, flag, count) carries everything its readers use, so relaxed
// GPU-scope accesses suffice: nothing else is read on the strength of it.  Waits (only when
// a predecessor has not published anything yet) are bounded.  Returns the
// exclusive prefix on every lane, or -1 on timeout / abort.
__device__ __forceinline__ int64_t lookback_warp(const LoopParams &p, uint64_t *words, int tile, uint64_t epoch,
                                                 uint32_t cnt, uint64_t frame, int lane) {
  if (tile == 0) {
    if (lane == 0) st_relaxed_u64(&words[0], look_pack(epoch, kLookPrefix, cnt));
    return 0;
  }
  if (lane == 0) st_relaxed_u64(&words[tile], look_pack(epoch, kLookAgg, cnt));
  uint64_t prefix = 0;
  int i0 = tile - 1;
  uint64_t t0 = 0;
  uint32_t polls = 0;
  for (;;) {
    const int i = i0 - lane;
    uint32_t flag = kLookPrefix, val = 0;  // i < 0: tile 0 always publishes a prefix first
    if (i >= 0) {
      const uint64_t w = ld_relaxed_u64(&words[i]);
      flag = (w >> 34) == epoch ? static_cast<uint32_t>((w >> 32) & 3u) : 0u;
      val = static_cast<uint32_t>(w);
    }
    const unsigned incl = __ballot_sync(0xffffffffu, flag == kLookPrefix);
    const unsigned none = __ballot_sync(0xffffffffu, flag == 0u);
    const int first = incl ? __ffs(incl) - 1 : 31;          // nearest inclusive prefix
    const unsigned need = first == 31 ? 0xffffffffu : ((2u << first) - 1u);
    if (none & need) {  // some predecessor up to there has published nothing yet
      if (polls == 0) t0 = globaltimer_ns();
      ++polls;
      __nanosleep(32);
      if ((polls & 63u) == 0u) {
        int stop = 0;
        if (lane == 0) {
          if (ld_volatile_u32(&p.ls->abort)) stop = 1;
          else if (globaltimer_ns() - t0 > p.timeout_ns) {
            report_error(p.status, kDevTimeout, kActSel, 3, frame);
            atomicExch(&p.ls->abort, 1u);
            stop = 1;
          }
        }
        if (__shfl_sync(0xffffffffu, stop, 0)) return -1;
      }
      continue;
    }
    uint32_t v = (static_cast<unsigned>(lane) <= static_cast<unsigned>(first)) ? val : 0u;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    prefix += v;
    if (incl) break;
    i0 -= 32;
  }
  if (lane == 0) st_relaxed_u64(&words[tile], look_pack(epoch, kLookPrefix, static_cast<uint32_t>(prefix + cnt)));
  return static_cast<int64_t>(prefix);
}

// Register copy of the FIFO counters (written, read, peak per FIFO).
struct CtrCopy {
  uint64_t w[kNumFifos], r[kNumFifos], pk[kNumFifos];
};

// The checks of fifo_release / fifo_commit, on the register copy.
__device__ __forceinline__ void book_release(CtrCopy &m, int f, uint64_t n, uint64_t delay, uint32_t *st,
                                             uint32_t actor, uint64_t frame) {
  if (st && delay + m.w[f] < m.r[f] + n) report_error(st, kDevUnderflow, actor, static_cast<uint32_t>(f), frame);
  m.r[f] += n;
}
__device__ __forceinline__ void book_commit(CtrCopy &m, int f, uint64_t n, uint64_t delay, uint64_t cap,
                                            uint32_t *st, uint32_t actor, uint64_t frame) {
  m.w[f] += n;
  const uint64_t occ = delay + m.w[f] - m.r[f];
  if (occ > m.pk[f]) m.pk[f] = occ;
  if (st && occ > cap) report_error(st, kDevOverflow, actor, static_cast<uint32_t>(f), frame);
}

// Per-frame FIFO bookkeeping of every actor's firing, in the actors' order
// (st = nullptr: counters only, no reports).
__device__ __forceinline__ void frame_bookkeeping(const LoopParams &p, CtrCopy &m, uint64_t frame, uint32_t c,
                                                  uint32_t *st) {
  const uint64_t F = p.f.F;
  book_release(m, 0, F, 0, st, kActFir, frame);
  book_release(m, 1, 1, 1, st, kActFir, frame);
  book_commit(m, 1, 1, 1, p.cap[1], st, kActFir, frame);
  book_commit(m, 2, F, 0, p.cap[2], st, kActFir, frame);
  book_commit(m, 3, F, 0, p.cap[3], st, kActFir, frame);
  book_release(m, 2, F, 0, st, kActDet, frame);
  book_commit(m, 4, 1, 0, p.cap[4], st, kActDet, frame);
  book_commit(m, 5, 1, 0, p.cap[5], st, kActDet, frame);
  book_release(m, 4, 1, 0, st, kActSel, frame);
  book_release(m, 3, F, 0, st, kActSel, frame);
  book_commit(m, 6, c, 0, p.cap[6], st, kActSel, frame);
  book_release(m, 6, c, 0, st, kActHx, frame);
  book_commit(m, 7, c, 0, p.cap[7], st, kActHx, frame);
  book_release(m, 5, 1, 0, st, kActSink, frame);
  book_release(m, 7, c, 0, st, kActSink, frame);
}

// Book finished frames in frame order, by one warp (all 32 lanes enter):
// frames finish out of order, but the f1 token of frame j+1 is the one frame
// j produced.  Lock-free: a warp that cannot take the lock leaves, and the
// holder re-checks after releasing it, so every ready frame is booked by
// someone; no thread ever waits.  The holder reads the counters once, reads
// the ready flags and SINK counts of 32 frames per round trip, replays the
// per-frame bookkeeping on a register copy (the same checks, in the same
// order) and adds each counter's change with one atomic.  f0's `written` is
// also bumped by pushes meanwhile, so it is only read (frames were pushed
// before they fired).
__device__ __forceinline__ void drain_bookkeeping(const LoopParams &p, uint64_t seq_end, int lane) {
  for (;;) {
    int got = 0;
    if (lane == 0) got = atomicCAS(&p.ls->book_lock, 0u, 1u) == 0u;
    if (!__shfl_sync(0xffffffffu, got, 0)) return;
    __threadfence();
    const uint64_t j0 = *reinterpret_cast<volatile unsigned long long *>(&p.ls->booked);
    const uint64_t cv = lane < 3 * kNumFifos ? ld_acquire_u64(&p.ctr[lane]) : 0ull;
    CtrCopy m;
#pragma unroll
    for (int f = 0; f < kNumFifos; ++f) {
      m.w[f] = __shfl_sync(0xffffffffu, cv, 3 * f + kCtrWritten);
      m.r[f] = __shfl_sync(0xffffffffu, cv, 3 * f + kCtrRead);
      m.pk[f] = __shfl_sync(0xffffffffu, cv, 3 * f + kCtrPeak);
    }
    uint64_t j = j0;
    for (;;) {
      const uint64_t jj = j + static_cast<uint64_t>(lane);
      bool rdy = false;
      uint32_t c = 0;
      if (jj < seq_end) {
        rdy = ld_acquire_u64(&p.ready[static_cast<int64_t>(jj % static_cast<uint64_t>(p.C))]) == jj + 1;
        if (rdy)
          c = static_cast<uint32_t>(
              *reinterpret_cast<volatile int32_t *>(&p.rec_c[static_cast<int64_t>(jj % static_cast<uint64_t>(p.rslot.cap))]));
      }
      const unsigned notr = __ballot_sync(0xffffffffu, !rdy);
      const int nr = notr ? __ffs(notr) - 1 : 32;  // ready frames in a row from j
      for (int i = 0; i < nr; ++i) {
        const uint32_t ci = __shfl_sync(0xffffffffu, c, i);
        frame_bookkeeping(p, m, j + static_cast<uint64_t>(i), ci, lane == 0 ? p.status : nullptr);
      }
      j += static_cast<uint64_t>(nr);
      if (nr < 32) break;
    }
    if (j > j0) {
#pragma unroll
      for (int f = 0; f < kNumFifos; ++f) {
        unsigned long long *c3 = reinterpret_cast<unsigned long long *>(p.ctr + 3 * f);
        if (f != 0 && lane == 3 * f + kCtrWritten && m.w[f] > cv) atomicAdd(&c3[kCtrWritten], m.w[f] - cv);
        if (lane == 3 * f + kCtrRead && m.r[f] > cv) atomicAdd(&c3[kCtrRead], m.r[f] - cv);
        if (lane == 3 * f + kCtrPeak && m.pk[f] > cv) atomicMax(&c3[kCtrPeak], m.pk[f]);
      }
      __threadfence();
      __syncwarp();
      if (lane == 0) *reinterpret_cast<volatile unsigned long long *>(&p.ls->booked) = j;
    }
    __threadfence();
    __syncwarp();
    if (lane == 0) atomicExch(&p.ls->book_lock, 0u);
    __threadfence();
    int again = 0;
    if (lane == 0) {
      const uint64_t jb = *reinterpret_cast<volatile unsigned long long *>(&p.ls->booked);
      again = jb < seq_end &&
              ld_acquire_u64(&p.ready[static_cast<int64_t>(jb % static_cast<uint64_t>(p.C))]) == jb + 1;
    }
    if (!__shfl_sync(0xffffffffu, again, 0)) return;
  }
}

// Shared memory: window | taps | red[32] | Et[256] | sel[256] | H [N][N]
__host__ __device__ inline size_t loop_smem_bytes(int T, int N) {
  return fir_smem_bytes(T) + 256 * sizeof(int32_t) + static_cast<size_t>(N) * N * sizeof(float2);
}

// NT > 0: H row i in registers (N == NT, a power of two <= 32); NT == 0:
// any N < 64, H read from shared memory.
template <int NT>
__global__ void __launch_bounds__(kFirThreads) firing_loop_kernel(LoopParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const FirParams &f = p.f;
  const int TP = f.TP;
  const int win = TP - 1 + kFirTile;
  float2 *xs = reinterpret_cast<float2 *>(smem_raw);
  float2 *hs = xs + fir_window_slots(TP);
  float *red = reinterpret_cast<float *>(hs + TP);
  float *Et = red + 32;
  int32_t *sel = reinterpret_cast<int32_t *>(Et + 256);
  float2 *Hs = reinterpret_cast<float2 *>(sel + 256);
  (void)win;
  __shared__ unsigned long long s_ticket;
  __shared__ int s_cnt;
  __shared__ long long s_prefix;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int N = NT > 0 ? NT : p.N;
  for (int t = tid; t < TP; t += kFirThreads) hs[t] = t < f.T ? f.taps[t] : make_float2(0.f, 0.f);
  for (int q = tid; q < N * N; q += kFirThreads) Hs[q] = p.H[q];
  __syncthreads();
  constexpr int NR = NT > 0 ? NT : 1;
  const int hi = NT > 0 ? tid % NT : 0;

  const unsigned long long total = static_cast<unsigned long long>(f.frames) * f.tiles;
  for (;;) {
    if (tid == 0) {
      const unsigned long long tk = atomicAdd(&p.ls->ticket, 1ull) - p.ticket_base;
      s_ticket = ld_volatile_u32(&p.ls->abort) ? ~0ull : tk;  // one decision per CTA
    }
    __syncthreads();  // also: the previous item is done with shared memory
    const unsigned long long t = s_ticket;
    if (t >= total) break;
    const int k = static_cast<int>(t / f.tiles);
    const int tile = static_cast<int>(t % f.tiles);
    const uint64_t seq = static_cast<uint64_t>(f.yslot.seq0) + k;
    const int64_t s0 = static_cast<int64_t>(tile) * f.TS;
    const int nv = static_cast<int>(min(static_cast<int64_t>(f.TS), f.L - s0));

    // 1. firing rule of FIR on f0: the frame's F tokens were pushed
    if (tid == 0) {
      const uint64_t need = (seq + 1) * static_cast<uint64_t>(f.F);
      const bool ok = bounded_wait(p, [&] { return ld_acquire_u64(&p.ctr[0 * 3 + kCtrWritten]) >= need; },
                                   kActFir, 0, seq);
      s_cnt = ok ? 0 : -1;
    }
    __syncthreads();
    if (s_cnt < 0) break;

    // 2. FIR
    const float2 *cur = f.src.frame(k);
    const float2 *prev = k > 0 ? f.src.frame(k - 1) : nullptr;
    fir_stage_window(xs, cur, prev, f.hist, f.L, f.T, TP, s0, nv, tid);
    __syncthreads();
    float2 acc[kSPT];
    fir_compute(xs, hs, TP, tid, acc);

    // 3. DET energies (ends with a barrier)
    fir_block_energies(acc, f.B, nv, tid, red, Et);
    const int nb = nv / f.B;
    if (f.energy && tid < nb) f.energy[f.eslot.slot(k) * f.F + s0 / f.B + tid] = Et[tid];
    if (f.hist_out && k == f.frames - 1 && s0 + nv == f.L) {
      for (int m = tid; m < f.T - 1; m += kFirThreads) f.hist_out[m] = xs[pad_idx(TP - 1 + nv - (f.T - 1) + m)];
    }
    // 4a. SEL inside the tile: stable ballot compaction of v[b] = E_b > tau
    if (warp == 0) {
      int cnt = 0;
      for (int b0 = 0; b0 < nb; b0 += 32) {
        const int b = b0 + lane;
        const bool v = b < nb && Et[b] > p.tau;
        const unsigned m = __ballot_sync(0xffffffffu, v);
        if (v) sel[cnt + __popc(m & ((1u << lane) - 1u))] = b;
        cnt += __popc(m);
      }
      if (lane == 0) s_cnt = cnt;
    }
    __syncthreads();  // everyone is done reading the window
    // FIR output tile into shared memory for HX (pad2 layout, float4 stores)
    float2 *ys = xs;
    {
      float4 *ys4 = reinterpret_cast<float4 *>(ys + pad2_idx(tid * kSPT));
#pragma unroll
      for (int j = 0; j < kSPT / 2; ++j)
        ys4[j] = make_float4(acc[2 * j].x, acc[2 * j].y, acc[2 * j + 1].x, acc[2 * j + 1].y);
    }
    // 4b. SEL across tiles: decoupled look-back for the tile's offset
    const int cnt = s_cnt;
    const int64_t fslot = static_cast<int64_t>(seq % static_cast<uint64_t>(p.C));
    if (warp == 0) {
      const int64_t pr = lookback_warp(p, p.look + fslot * f.tiles, tile, seq + 1, cnt, seq, lane);
      if (lane == 0) s_prefix = pr;
    }
    __syncthreads();
    const long long prefix = s_prefix;
    if (prefix < 0) break;
    if (prefix + cnt > f.F) {  // never expected: keep every store in bounds
      if (tid == 0) {
        report_error(p.status, kDevInvariant, kActSel, 6, seq);
        atomicExch(&p.ls->abort, 1u);
      }
      break;
    }

    // 5. HX_b of the selected blocks, written at compacted positions
    const int64_t rs = p.rslot.slot(k);
    int32_t *ridx = p.rec_idx + rs * f.F;
    float2 *ry = p.rec_y + rs * f.L;
    for (int q = tid; q < cnt; q += kFirThreads) ridx[prefix + q] = static_cast<int32_t>(s0 / f.B) + sel[q];
    const int R = f.B / N;
    float2 h[NR];  // row hi of H, loaded only for tiles with selected blocks
    if (NT >= 2 && cnt > 0) {
#pragma unroll
      for (int kk = 0; kk < NR; ++kk) h[kk] = Hs[hi * NR + kk];
    }
    for (int si = 0; si < cnt; ++si) {
      const int bo = sel[si] * f.B;
      float2 *dst = ry + (prefix + si) * f.B;
      if (NT >= 2) {
        // thread (hi, g): row hi of H in registers, rows g, g+RG, ... of X;
        // X[r][kk..kk+1] is one aligned float4 broadcast (NT is a power of 2,
        // so a pair never straddles a pad)
        constexpr int RG = kFirThreads / NR;
        const int g = tid / NR;
        int r = g;
        for (; r + RG < R; r += 2 * RG) {
          float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
          const int b0 = bo + r * NR, b1 = bo + (r + RG) * NR;
#pragma unroll
          for (int kk = 0; kk < NR; kk += 2) {
            const float4 x0 = *reinterpret_cast<const float4 *>(ys + pad2_idx(b0 + kk));
            const float4 x1 = *reinterpret_cast<const float4 *>(ys + pad2_idx(b1 + kk));
            cmac(a0, h[kk], make_float2(x0.x, x0.y));
            cmac(a1, h[kk], make_float2(x1.x, x1.y));
            cmac(a0, h[kk + 1], make_float2(x0.z, x0.w));
            cmac(a1, h[kk + 1], make_float2(x1.z, x1.w));
          }
          dst[r * NR + hi] = a0;
          dst[(r + RG) * NR + hi] = a1;
        }
        for (; r < R; r += RG) {
          float2 a0 = make_float2(0.f, 0.f);
          const int b0 = bo + r * NR;
#pragma unroll
          for (int kk = 0; kk < NR; kk += 2) {
            const float4 x0 = *reinterpret_cast<const float4 *>(ys + pad2_idx(b0 + kk));
            cmac(a0, h[kk], make_float2(x0.x, x0.y));
            cmac(a0, h[kk + 1], make_float2(x0.z, x0.w));
          }
          dst[r * NR + hi] = a0;
        }
      } else {
        for (int q = tid; q < f.B; q += kFirThreads) {
          const int r = q / N, i = q % N;
          float2 a = make_float2(0.f, 0.f);
          for (int kk = 0; kk < N; ++kk) cmac(a, Hs[i * N + kk], ys[pad2_idx(bo + r * N + kk)]);
          dst[q] = a;
        }
      }
    }

    // 6. frame completion: the last tile to finish writes the SINK record;
    //    warp 0 then books the frames that are ready in order
    __syncthreads();
    if (tid < 32) {
      int last = 0;
      if (tid == 0) {
        __threadfence();
        const uint32_t old = atomicAdd(&p.done[fslot], 1u);
        if (old + 1u == static_cast<uint32_t>(f.tiles)) {
          p.done[fslot] = 0u;  // every tile of the frame has counted: reset the slot
          __threadfence();  // every tile counted: their look-back words are visible
          const uint64_t w = ld_acquire_u64(&p.look[fslot * f.tiles + f.tiles - 1]);
          const uint32_t c = static_cast<uint32_t>(w);
          p.rec_c[rs] = static_cast<int32_t>(c);
          p.rec_frame[rs] = static_cast<int64_t>(seq);
          __threadfence();
          st_release_u64(&p.ready[fslot], seq + 1);
          __threadfence();
          last = 1;
        }
      }
      if (__shfl_sync(0xffffffffu, last, 0)) drain_bookkeeping(p, static_cast<uint64_t>(f.yslot.seq0) + f.frames, tid);
    }
  }
  // every CTA makes exactly one failing claim, unless it left early
}

__host__ inline bool loop_supported(int N) { return N < 64; }

}  // namespace prune
