/*
 * PRUNE oracle: plain sequential FP64 dataflow simulator of the canonical
 * dynamic, decidable graph.
 *
 *   TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check
 *   and the benchmark's CPU-baseline leg may load this library.  It shares no
 *   code, header, table or constant with the CUDA path and imports nothing
 *   from it.
 *
 * Graph (PRUNE MoC, Sec. III):
 *
 *   SRC --f0(F)--> FIR --f2(F)--> DET --f4(1, control)--> SEL.cport
 *                  | ^  \                 \--f5(1, control)--> SINK.cport
 *                  f1(1, delay 1)  \--f3(F)--> SEL
 *   SEL --f6_b(atr 1)--> HX_b --f7_b(atr 1)--> SINK      b = 0..F-1
 *
 * Token of f0, f2, f3, f6_b, f7_b: one block of B complex samples.
 * Token of f1: the last T-1 input samples (the FIR delay line, z^-1).
 * Token of f4, f5: one control value v[0..F) (one Boolean per DC HX_b).
 *
 * The scheduler fires, in a fixed topological round-robin order, any actor
 * whose firing rule holds (blocking reads and writes, Sec. III-A), with DRP
 * rates set from the control token by eq. (1): tokrate = BTOI(v[p]) * atr(p).
 * FIFO capacities follow eq. (2) of Sec. VI-B.  Every actor computes in FP64
 * from the FP32 inputs.
 *
 * Readings of points the paper leaves open (the same readings are listed in
 * the design notes of the repository):
 *   - FIR is the convolution y[n] = sum_t h[t] x[n-t], no tap conjugation.
 *   - The initial delay token of f1 holds T-1 zero samples.
 *   - DET energy is the sum over the block of |y|^2 of the FIR output; the
 *     decision is strict: v[b] = (E_b > tau).
 *   - SEL keeps the selected blocks in ascending block order (FIFO order).
 *   - HX_b reshapes a block row-major to (B/N, N) and multiplies each row by
 *     H: out[j*N+i] = sum_k H[i][k] X[j][k].
 *   - SINK emits a compacted record (c, idx[0..c), y[c][B]) per frame, also
 *     when c = 0.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_EINVAL 1
#define ORACLE_ENOMEM 2
#define ORACLE_EDEADLOCK 3
#define ORACLE_EOVERFLOW 4

/* FIFO indices reported in the statistics table. f6 and f7 aggregate the F
 * per-DC FIFOs f6_b / f7_b (sums of written/read; peak of the sum). */
enum { F0 = 0, F1, F2, F3, F4, F5, F6, F7, NFIFO_REPORTED };

typedef struct {
  int32_t F, B, T, N, C;
  float tau;
  const float *taps; /* 2T floats, interleaved complex */
  const float *H;    /* 2N*N floats, row-major, interleaved complex */
} oracle_graph;

typedef struct {
  long rate;      /* fiforate(f) */
  long delay;     /* Q: initial tokens */
  long cap;       /* Gamma_f in tokens, eq. (2) */
  long tok_bytes; /* bytes of one token */
  unsigned char *buf;
  long head;      /* monotone: tokens read (including initial tokens) */
  long tail;      /* monotone: tokens present ever (initial + written) */
  long written, read, peak;
} fifo_t;

/* Eq. (2) with the token size B factored out: capacity in tokens. */
long oracle_fifo_capacity(long r, long Q, long C) {
  if (r <= 0 || Q < 0 || C <= 0) return -1;
  if (Q % r != 0) return r * C + Q;
  return (r * C > Q) ? r * C : Q;
}

static int fifo_init(fifo_t *f, long rate, long delay, long C, long tok_bytes) {
  memset(f, 0, sizeof(*f));
  f->rate = rate;
  f->delay = delay;
  f->cap = oracle_fifo_capacity(rate, delay, C);
  f->tok_bytes = tok_bytes;
  f->buf = (unsigned char *)calloc((size_t)f->cap, (size_t)tok_bytes);
  if (!f->buf) return ORACLE_ENOMEM;
  /* The initial tokens are zero-valued (calloc) and already present. */
  f->tail = delay;
  f->peak = delay;
  return ORACLE_OK;
}

static void fifo_free(fifo_t *f) { free(f->buf); f->buf = NULL; }
static long fifo_count(const fifo_t *f) { return f->tail - f->head; }
static long fifo_space(const fifo_t *f) { return f->cap - fifo_count(f); }

/* Pointer to the k-th token counted from the read end (k = 0 is the oldest). */
static unsigned char *fifo_peek(fifo_t *f, long k) {
  return f->buf + (size_t)((f->head + k) % f->cap) * (size_t)f->tok_bytes;
}
/* Pointer to the slot of the k-th token to be written next. */
static unsigned char *fifo_slot(fifo_t *f, long k) {
  return f->buf + (size_t)((f->tail + k) % f->cap) * (size_t)f->tok_bytes;
}
static void fifo_commit(fifo_t *f, long n) {
  f->tail += n;
  f->written += n;
  if (fifo_count(f) > f->peak) f->peak = fifo_count(f);
}
static void fifo_release(fifo_t *f, long n) { f->head += n; f->read += n; }

typedef struct { double re, im; } cplx;

static inline cplx cmul(cplx a, cplx b) {
  cplx r = {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
  return r;
}

typedef struct {
  oracle_graph g;
  fifo_t f0, f1, f2, f3, f4, f5;
  fifo_t *f6, *f7; /* F each */
  cplx *taps, *H;
  /* input cursor of the source actor */
  const float *x;
  long n_frames, src_fired, sink_fired;
  /* outputs */
  int32_t *c_out, *idx_out;
  double *y_out, *energy_out;
  long y_cursor; /* complex samples written to y_out */
  int64_t *fires; /* per-actor firing counts: SRC, FIR, DET, SEL, HX(sum), SINK */
} sim_t;

/* ---------------- actor firing rules and firing functions ---------------- */

/* SRC: source actor, one firing = one frame of F blocks onto f0. */
static int src_can_fire(sim_t *s) {
  return s->src_fired < s->n_frames && fifo_space(&s->f0) >= s->f0.rate;
}
static void src_fire(sim_t *s) {
  const long F = s->g.F, B = s->g.B;
  const float *frame = s->x + (size_t)s->src_fired * F * B * 2;
  for (long b = 0; b < F; ++b) {
    cplx *tok = (cplx *)fifo_slot(&s->f0, b);
    for (long n = 0; n < B; ++n) {
      tok[n].re = (double)frame[(b * B + n) * 2 + 0];
      tok[n].im = (double)frame[(b * B + n) * 2 + 1];
    }
  }
  fifo_commit(&s->f0, F);
  s->src_fired++;
}

/* FIR: static actor. Reads F blocks (f0) and the delay-line token (f1);
 * writes F blocks to the broadcast port (f2 and f3) and the next delay-line
 * token (f1). */
static int fir_can_fire(sim_t *s) {
  /* f1 is a self-loop: the firing consumes its token before it produces the
   * next one, so the slot it frees counts as space. */
  return fifo_count(&s->f0) >= s->f0.rate && fifo_count(&s->f1) >= 1 &&
         fifo_space(&s->f2) >= s->f2.rate && fifo_space(&s->f3) >= s->f3.rate &&
         fifo_space(&s->f1) + 1 >= 1;
}
static void fir_fire(sim_t *s) {
  const long F = s->g.F, B = s->g.B, T = s->g.T, L = F * B;
  /* window w = [T-1 history samples | F*B frame samples] */
  cplx *w = (cplx *)malloc(sizeof(cplx) * (size_t)(T - 1 + L));
  const cplx *hist = (const cplx *)fifo_peek(&s->f1, 0);
  for (long i = 0; i < T - 1; ++i) w[i] = hist[i];
  for (long b = 0; b < F; ++b) {
    const cplx *tok = (const cplx *)fifo_peek(&s->f0, b);
    for (long n = 0; n < B; ++n) w[T - 1 + b * B + n] = tok[n];
  }
  /* y[n] = sum_{t<T} h[t] x[n-t]; x[n-t] is w[T-1+n-t]. */
  for (long b = 0; b < F; ++b) {
    cplx *o2 = (cplx *)fifo_slot(&s->f2, b);
    cplx *o3 = (cplx *)fifo_slot(&s->f3, b);
    for (long n = 0; n < B; ++n) {
      const long gn = b * B + n;
      cplx acc = {0.0, 0.0};
      for (long t = 0; t < T; ++t) {
        cplx p = cmul(s->taps[t], w[T - 1 + gn - t]);
        acc.re += p.re;
        acc.im += p.im;
      }
      o2[n] = acc; /* broadcast: the same token goes to every FIFO of the port */
      o3[n] = acc;
    }
  }
  /* next delay-line token: the last T-1 input samples of this frame */
  cplx *nh = (cplx *)fifo_slot(&s->f1, 0);
  for (long i = 0; i < T - 1; ++i) nh[i] = w[L + i];
  free(w);
  fifo_release(&s->f0, F);
  fifo_release(&s->f1, 1);
  fifo_commit(&s->f1, 1);
  fifo_commit(&s->f2, F);
  fifo_commit(&s->f3, F);
  s->fires[1]++;
}

/* DET: configuration actor. Reads F blocks (f2), writes one control token to
 * its control output port, broadcast to f4 (SEL) and f5 (SINK). */
static int det_can_fire(sim_t *s) {
  return fifo_count(&s->f2) >= s->f2.rate && fifo_space(&s->f4) >= 1 &&
         fifo_space(&s->f5) >= 1;
}
static void det_fire(sim_t *s, long frame) {
  const long F = s->g.F, B = s->g.B;
  unsigned char *v4 = fifo_slot(&s->f4, 0);
  unsigned char *v5 = fifo_slot(&s->f5, 0);
  for (long b = 0; b < F; ++b) {
    const cplx *tok = (const cplx *)fifo_peek(&s->f2, b);
    double e = 0.0;
    for (long n = 0; n < B; ++n) e += tok[n].re * tok[n].re + tok[n].im * tok[n].im;
    if (s->energy_out) s->energy_out[frame * F + b] = e;
    unsigned char v = (e > (double)s->g.tau) ? 1 : 0;
    v4[b] = v;
    v5[b] = v;
  }
  fifo_release(&s->f2, F);
  fifo_commit(&s->f4, 1);
  fifo_commit(&s->f5, 1);
  s->fires[2]++;
}

/* SEL: dynamic actor x of the DPG. Control port f4; SRP input f3 (rate F);
 * output DRP_b on f6_b with atr 1, itr 0. */
static int sel_can_fire(sim_t *s) {
  if (fifo_count(&s->f4) < 1) return 0; /* control port first */
  const unsigned char *v = fifo_peek(&s->f4, 0);
  if (fifo_count(&s->f3) < s->f3.rate) return 0;
  for (long b = 0; b < s->g.F; ++b) {
    long rate = (long)v[b] * s->f6[b].rate; /* eq. (1) */
    if (fifo_space(&s->f6[b]) < rate) return 0;
  }
  return 1;
}
static void sel_fire(sim_t *s) {
  const long F = s->g.F, B = s->g.B;
  const unsigned char *v = fifo_peek(&s->f4, 0);
  for (long b = 0; b < F; ++b) {
    long rate = (long)v[b] * s->f6[b].rate;
    if (rate) {
      memcpy(fifo_slot(&s->f6[b], 0), fifo_peek(&s->f3, b), sizeof(cplx) * (size_t)B);
      fifo_commit(&s->f6[b], rate);
    }
  }
  fifo_release(&s->f3, F);
  fifo_release(&s->f4, 1);
  s->fires[3]++;
}

/* HX_b: static actor, the single actor of dynamic component b. */
static int hx_can_fire(sim_t *s, long b) {
  return fifo_count(&s->f6[b]) >= 1 && fifo_space(&s->f7[b]) >= 1;
}
static void hx_fire(sim_t *s, long b) {
  const long B = s->g.B, N = s->g.N;
  const cplx *in = (const cplx *)fifo_peek(&s->f6[b], 0);
  cplx *out = (cplx *)fifo_slot(&s->f7[b], 0);
  for (long j = 0; j < B / N; ++j) {      /* row j of X = reshape(block, (B/N, N)) */
    for (long i = 0; i < N; ++i) {
      cplx acc = {0.0, 0.0};
      for (long k = 0; k < N; ++k) {
        cplx p = cmul(s->H[i * N + k], in[j * N + k]);
        acc.re += p.re;
        acc.im += p.im;
      }
      out[j * N + i] = acc;
    }
  }
  fifo_release(&s->f6[b], 1);
  fifo_commit(&s->f7[b], 1);
  s->fires[4]++;
}

/* SINK: dynamic actor y of the DPG. Control port f5; input DRP_b on f7_b. */
static int sink_can_fire(sim_t *s) {
  if (fifo_count(&s->f5) < 1) return 0;
  const unsigned char *v = fifo_peek(&s->f5, 0);
  for (long b = 0; b < s->g.F; ++b) {
    long rate = (long)v[b] * s->f7[b].rate; /* eq. (1) */
    if (fifo_count(&s->f7[b]) < rate) return 0;
  }
  return 1;
}
static void sink_fire(sim_t *s) {
  const long F = s->g.F, B = s->g.B;
  const long frame = s->sink_fired;
  const unsigned char *v = fifo_peek(&s->f5, 0);
  int32_t c = 0;
  for (long b = 0; b < F; ++b) {
    long rate = (long)v[b] * s->f7[b].rate;
    if (!rate) continue;
    const cplx *tok = (const cplx *)fifo_peek(&s->f7[b], 0);
    if (s->idx_out) s->idx_out[frame * F + c] = (int32_t)b;
    if (s->y_out)
      for (long n = 0; n < B; ++n) {
        s->y_out[(s->y_cursor + n) * 2 + 0] = tok[n].re;
        s->y_out[(s->y_cursor + n) * 2 + 1] = tok[n].im;
      }
    s->y_cursor += B;
    fifo_release(&s->f7[b], rate);
    ++c;
  }
  if (s->c_out) s->c_out[frame] = c;
  fifo_release(&s->f5, 1);
  s->sink_fired++;
  s->fires[5]++;
}

static void report(const fifo_t *f, int64_t *row) {
  row[0] = f->written;
  row[1] = f->read;
  row[2] = f->peak;
  row[3] = fifo_count(f);
}

/*
 * Run the canonical graph over n_frames input frames.
 *   x        [n_frames][F][B] complex FP32, interleaved
 *   hist_in  optional T-1 complex FP64 samples: initial contents of the delay
 *            token (NULL = zeros, the reading used throughout)
 *   c_out    [n_frames]              selected block count per frame
 *   idx_out  [n_frames][F]           selected block indices, ascending, first c valid
 *   y_out    [sum c * B] complex FP64 compacted sink output, frame after frame
 *   energy_out [n_frames][F]         DET block energies (optional)
 *   stats    [8][4] int64            per FIFO f0..f7: written, read, peak, final
 *                                    occupancy (f6/f7: sums over b; peak = max
 *                                    over b of the per-DC peak)
 *   fires    [6] int64               firings of SRC, FIR, DET, SEL, HX (all b), SINK
 *   hist_out optional T-1 complex FP64: the delay token left in f1
 * Returns ORACLE_OK, or ORACLE_EDEADLOCK if the scheduler stops before every
 * frame reached the sink.
 */
int oracle_run(const oracle_graph *g, const float *x, int64_t n_frames, int32_t *c_out,
               int32_t *idx_out, double *y_out, double *energy_out, int64_t *stats,
               int64_t *fires, const double *hist_in, double *hist_out) {
  if (!g || g->F < 1 || g->B < 1 || g->T < 1 || g->N < 1 || g->C < 1 || g->B % g->N != 0 ||
      n_frames < 0 || (n_frames > 0 && !x))
    return ORACLE_EINVAL;
  sim_t s;
  memset(&s, 0, sizeof(s));
  s.g = *g;
  s.x = x;
  s.n_frames = n_frames;
  s.c_out = c_out;
  s.idx_out = idx_out;
  s.y_out = y_out;
  s.energy_out = energy_out;
  int64_t local_fires[6] = {0, 0, 0, 0, 0, 0};
  s.fires = local_fires;
  const long F = g->F, B = g->B, T = g->T, N = g->N, C = g->C;
  const long hist_len = (T > 1) ? T - 1 : 1; /* keep a non-empty token for T = 1 */
  int rc = ORACLE_OK;
  s.taps = (cplx *)malloc(sizeof(cplx) * (size_t)T);
  s.H = (cplx *)malloc(sizeof(cplx) * (size_t)(N * N));
  s.f6 = (fifo_t *)calloc((size_t)F, sizeof(fifo_t));
  s.f7 = (fifo_t *)calloc((size_t)F, sizeof(fifo_t));
  if (!s.taps || !s.H || !s.f6 || !s.f7) { rc = ORACLE_ENOMEM; goto done; }
  for (long t = 0; t < T; ++t) { s.taps[t].re = g->taps[2 * t]; s.taps[t].im = g->taps[2 * t + 1]; }
  for (long i = 0; i < N * N; ++i) { s.H[i].re = g->H[2 * i]; s.H[i].im = g->H[2 * i + 1]; }

  const long blk = (long)sizeof(cplx) * B;
  if (fifo_init(&s.f0, F, 0, C, blk) || fifo_init(&s.f1, 1, 1, C, (long)sizeof(cplx) * hist_len) ||
      fifo_init(&s.f2, F, 0, C, blk) || fifo_init(&s.f3, F, 0, C, blk) ||
      fifo_init(&s.f4, 1, 0, C, F) || fifo_init(&s.f5, 1, 0, C, F)) {
    rc = ORACLE_ENOMEM;
    goto done;
  }
  for (long b = 0; b < F; ++b)
    if (fifo_init(&s.f6[b], 1, 0, C, blk) || fifo_init(&s.f7[b], 1, 0, C, blk)) {
      rc = ORACLE_ENOMEM;
      goto done;
    }
  if (hist_in && T > 1) memcpy(fifo_peek(&s.f1, 0), hist_in, sizeof(cplx) * (size_t)(T - 1));

  /* Round-robin over the actors in topological order until no actor can fire. */
  long fir_frame = 0, det_frame = 0;
  for (;;) {
    int fired = 0;
    if (src_can_fire(&s)) { src_fire(&s); local_fires[0]++; fired = 1; }
    if (fir_can_fire(&s)) { fir_fire(&s); fir_frame++; fired = 1; }
    if (det_can_fire(&s)) { det_fire(&s, det_frame); det_frame++; fired = 1; }
    if (sel_can_fire(&s)) { sel_fire(&s); fired = 1; }
    for (long b = 0; b < F; ++b)
      if (hx_can_fire(&s, b)) { hx_fire(&s, b); fired = 1; }
    if (sink_can_fire(&s)) { sink_fire(&s); fired = 1; }
    if (!fired) break;
  }
  (void)fir_frame;
  if (s.sink_fired != n_frames) rc = ORACLE_EDEADLOCK;

  if (stats) {
    report(&s.f0, stats + 0 * 4);
    report(&s.f1, stats + 1 * 4);
    report(&s.f2, stats + 2 * 4);
    report(&s.f3, stats + 3 * 4);
    report(&s.f4, stats + 4 * 4);
    report(&s.f5, stats + 5 * 4);
    for (int k = 0; k < 2; ++k) {
      fifo_t *arr = k ? s.f7 : s.f6;
      int64_t *row = stats + (6 + k) * 4;
      row[0] = row[1] = row[2] = row[3] = 0;
      for (long b = 0; b < F; ++b) {
        row[0] += arr[b].written;
        row[1] += arr[b].read;
        if (arr[b].peak > row[2]) row[2] = arr[b].peak;
        row[3] += fifo_count(&arr[b]);
      }
    }
  }
  if (fires) memcpy(fires, local_fires, sizeof(local_fires));
  if (hist_out && T > 1) memcpy(hist_out, fifo_peek(&s.f1, 0), sizeof(cplx) * (size_t)(T - 1));

done:
  fifo_free(&s.f0); fifo_free(&s.f1); fifo_free(&s.f2);
  fifo_free(&s.f3); fifo_free(&s.f4); fifo_free(&s.f5);
  if (s.f6) for (long b = 0; b < F; ++b) fifo_free(&s.f6[b]);
  if (s.f7) for (long b = 0; b < F; ++b) fifo_free(&s.f7[b]);
  free(s.f6); free(s.f7); free(s.taps); free(s.H);
  return rc;
}

/*
 * The linear buffer with copy-back of Sec. VI-B (Fig. 6), replayed on token
 * sequence numbers.  A FIFO of rate r with Q initial tokens and capacity
 * Gamma tokens (eq. (2), or cap_override > 0) is accessed through contiguous
 * windows of r slots:
 *   - Q not a multiple of r (Gamma = rC + Q): the initial tokens sit in slots
 *     [0, Q); the writer fills windows starting at Q, Q+r, ..., Q+(C-1)r; after
 *     the window that ends at slot Gamma it copies slots [Gamma-Q, Gamma) to
 *     [0, Q) and restarts at Q.  The reader takes windows starting at 0, r,
 *     ..., (C-1)r and then restarts at 0.
 *   - otherwise (Gamma = max(rC, Q)): a ring of r-slot windows; the writer
 *     starts at Q mod Gamma, the reader at 0, both wrap at Gamma.
 * Blocking semantics (Sec. III-A): a write waits until its window (and, for
 * the copy, the front slots) hold no unread token; a read waits until its
 * window holds the next tokens in order.  The replay alternates write and read
 * attempts, preferring the write, for n_iter writes and n_iter reads.
 * write_pos / read_pos (n_iter each, optional) receive the first slot of every
 * window.  Returns 0 on success, or: 1 bad arguments, 2 out of memory,
 * 3 both sides blocked (deadlock), 4 a read saw a token out of FIFO order,
 * 5 a window ran past the end of the buffer.
 */
int oracle_linear_fifo_replay(long r, long Q, long C, long cap_override, long n_iter,
                              long *write_pos, long *read_pos) {
  long cap = cap_override > 0 ? cap_override : oracle_fifo_capacity(r, Q, C);
  if (cap <= 0 || r <= 0 || Q < 0 || C <= 0 || n_iter < 0) return 1;
  const int aligned = (Q % r) == 0;
  long *seq = (long *)malloc(sizeof(long) * (size_t)cap);
  unsigned char *live = (unsigned char *)calloc((size_t)cap, 1);
  if (!seq || !live) { free(seq); free(live); return 2; }
  for (long i = 0; i < Q && i < cap; ++i) { seq[i] = i - Q; live[i] = 1; }
  long wp = aligned ? (Q % cap) : Q, rp = 0;
  long writes = 0, reads = 0, next_write = 0, next_read = -Q;
  int copy_pending = 0, err = 0;
  while ((writes < n_iter || reads < n_iter) && !err) {
    int progressed = 0;
    if (writes < n_iter || copy_pending) {
      if (copy_pending) {
        int free_front = 1;
        for (long k = 0; k < Q; ++k) if (live[k]) free_front = 0;
        if (free_front) {
          for (long k = 0; k < Q; ++k) {
            seq[k] = seq[cap - Q + k];
            live[k] = 1;
            live[cap - Q + k] = 0;
          }
          copy_pending = 0;
          wp = Q;
          progressed = 1;
        }
      } else {
        if (wp + r > cap) { err = 5; break; }
        int free_win = 1;
        for (long k = 0; k < r; ++k) if (live[wp + k]) free_win = 0;
        if (free_win) {
          for (long k = 0; k < r; ++k) { seq[wp + k] = next_write++; live[wp + k] = 1; }
          if (write_pos) write_pos[writes] = wp;
          writes++;
          wp += r;
          if (aligned) { if (wp == cap) wp = 0; }
          else if (wp == cap) copy_pending = 1;
          progressed = 1;
        }
      }
    }
    if (reads < n_iter) {
      if (rp + r > cap) { err = 5; break; }
      int ready = 1;
      for (long k = 0; k < r; ++k)
        if (!live[rp + k]) ready = 0;
        else if (seq[rp + k] != next_read + k) { err = 4; break; }
      if (err) break;
      if (ready) {
        for (long k = 0; k < r; ++k) live[rp + k] = 0;
        next_read += r;
        if (read_pos) read_pos[reads] = rp;
        reads++;
        rp += r;
        if (aligned) { if (rp == cap) rp = 0; }
        else if (rp == r * C) rp = 0;
        progressed = 1;
      }
    }
    if (!progressed) err = 3;
  }
  free(seq);
  free(live);
  return err;
}
