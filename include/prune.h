/*
 * prune.h - C ABI of the B300 firing runtime for PRUNE dynamic dataflow
 * graphs (Boutellier, Wu, Huttunen, Bhattacharyya, "PRUNE: Dynamic and
 * Decidable Dataflow for Signal Processing on Heterogeneous Platforms").
 *
 * The graph this library fires is the canonical dynamic, decidable graph
 *
 *   SRC -f0-> FIR -f2-> DET (configuration actor) -f4-> SEL.cport
 *              |  \                               -f5-> SINK.cport
 *              f1  -f3-> SEL (dynamic) -f6_b-> HX_b (static) -f7_b-> SINK (dynamic)
 *
 * with b = 0..F-1 (Sec. III: actors, ports, FIFOs; Sec. V: one DPG with
 * configuration actor DET, dynamic actors SEL and SINK and F dynamic
 * components HX_b).  Per frame:
 *   FIR  (static actor)    y[n] = sum_{t<T} h[t] x[n-t] over the continuous
 *                          stream; the last T-1 input samples are the delay
 *                          token carried on the self-loop FIFO f1 (Sec. III-D;
 *                          initial token: T-1 zeros).
 *   DET  (configuration)   E_b = sum_{n<B} |y[bB+n]|^2, v[b] = (E_b > tau);
 *                          emits one control token (Sec. III-B/C).
 *   SEL  (dynamic, x)      consumes the F blocks of y and the control token;
 *                          DRP_b fires at rate BTOI(v[b]) * 1 (eq. (1)).
 *   HX_b (static, DC b)    X = reshape(block, (B/N, N)) row-major,
 *                          out[j*N+i] = sum_k H[i][k] X[j][k].
 *   SINK (dynamic, y)      consumes the control token and c = sum_b v[b]
 *                          blocks; emits the record (frame, c, idx[c], out[c][B])
 *                          with idx ascending.
 *
 * Conventions for every entry point:
 *   - complex samples are complex64: two float32 (re, im), interleaved;
 *   - "device" pointers are CUDA device (or managed) memory of the graph's
 *     device; "host" pointers are CPU memory (pageable or pinned);
 *   - nothing is retained after return unless stated (borrowed frames);
 *   - no C++ exception crosses this interface; every function returns a
 *     prune_status and, on failure, sets a message read by prune_last_error;
 *   - a prune_graph is used by one host thread at a time;
 *   - work is enqueued on the graph's CUDA stream; functions that return data
 *     to the host (pull, peek, sync, fifo_stats) wait for it.
 * There is no CPU implementation of any step: without a usable CUDA device
 * every compute entry point returns PRUNE_ECUDA.
 */
#ifndef PRUNE_H
#define PRUNE_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define PRUNE_API __attribute__((visibility("default")))
#else
#define PRUNE_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum prune_status {
  PRUNE_OK = 0,
  PRUNE_EINVAL = 1,   /* bad argument, shape, or a rate/rule violation of the graph */
  PRUNE_ENOMEM = 2,   /* allocation failed or the graph would exceed its HBM budget */
  PRUNE_EAGAIN = 3,   /* FIFO full (push) or empty (pull): nothing was done */
  PRUNE_ETIMEOUT = 4, /* a bounded device-side wait gave up; the graph is poisoned */
  PRUNE_ECUDA = 5,    /* a CUDA call failed (no device, launch error, ...) */
  PRUNE_EBUSY = 6,    /* the request conflicts with work in flight */
  PRUNE_EDEVICE = 7   /* a device-side invariant check failed; the graph is poisoned */
} prune_status;

/* FIFO identifiers for prune_fifo_stats (see the graph above).  PRUNE_FIFO_F6
 * and PRUNE_FIFO_F7 aggregate the F per-DC FIFOs f6_b / f7_b. */
enum {
  PRUNE_FIFO_F0 = 0, /* SRC -> FIR           token: one block   rate F */
  PRUNE_FIFO_F1 = 1, /* FIR -> FIR (delay 1) token: T-1 samples rate 1 */
  PRUNE_FIFO_F2 = 2, /* FIR -> DET           token: one block   rate F */
  PRUNE_FIFO_F3 = 3, /* FIR -> SEL           token: one block   rate F */
  PRUNE_FIFO_F4 = 4, /* DET -> SEL.cport     control token      rate 1 */
  PRUNE_FIFO_F5 = 5, /* DET -> SINK.cport    control token      rate 1 */
  PRUNE_FIFO_F6 = 6, /* SEL -> HX_b          one block, atr 1 / itr 0 */
  PRUNE_FIFO_F7 = 7, /* HX_b -> SINK         one block, atr 1 / itr 0 */
  PRUNE_NUM_FIFOS = 8
};

/* Memory kinds for prune_push_frames / prune_pull. */
enum {
  PRUNE_MEM_HOST = 0,          /* host pointer: copied host -> device */
  PRUNE_MEM_DEVICE = 1,        /* device pointer: copied device -> device */
  PRUNE_MEM_DEVICE_BORROW = 2, /* device pointer, referenced in place (push only) */
  PRUNE_MEM_DISCARD = 3        /* pull only: drop the records without copying */
};

/* prune_run flags. */
enum {
  PRUNE_RUN_ASYNC = 0,   /* return once the firings are enqueued */
  PRUNE_RUN_SYNC = 1,    /* return once they completed (device status checked) */
  PRUNE_RUN_ACTORS = 2,  /* fire one kernel per actor instead of the fused firing
                            loop (same results; FIFOs f2/f3 materialised in HBM) */
  PRUNE_RUN_CUDA_CORES = 8, /* fire the fused loop with FIR and HX_b on CUDA cores even
                            where the tensor-core loop applies (N = 32, B dividing
                            4096 and a multiple of 32, T <= 129) */
  PRUNE_RUN_DEVICE_RULE = 4 /* let the device alone enforce FIR's firing rule on f0:
                            the host does not bound the run by the frames pushed,
                            so frames may be pushed later from another stream; a
                            frame that never arrives makes the bounded device wait
                            give up (PRUNE_ETIMEOUT after PRUNE_TIMEOUT_MS, default
                            2000 ms).  Fused firing loop only (N < 64). */
};

typedef struct prune_graph prune_graph;

/* Graph descriptor.  Sizes: F >= 1 blocks per frame (the rate of f0, f2, f3
 * and the number of DCs); B complex samples per block, a multiple of 8 in
 * [8, 2048] with B/8 a power of two up to 32 or a multiple of 32; T FIR taps,
 * 1 <= T <= 256, T - 1 <= B; N divides B, 1 <= N <= 128.
 * C is the buffering constant of eq. (2) (Sec. VI-B; 0 selects 3): f0 holds C
 * frames (F*C block tokens), f1 holds max(C, 1) delay tokens.  out_frames is
 * the capacity of the result ring in frames (0 selects C). */
typedef struct prune_graph_desc {
  int32_t F, B, T, N;
  int32_t C;
  int32_t out_frames;
  float tau;            /* DET threshold; v[b] = (E_b > tau) */
  const float *taps;    /* host, 2*T floats: h[t] = (taps[2t], taps[2t+1]); copied */
  const float *H;       /* host, 2*N*N floats, row-major H[i][k]; copied */
  void *stream;         /* cudaStream_t to enqueue on, or NULL for a graph-owned stream */
  int32_t device;       /* CUDA device ordinal, or -1 for the current device */
  int32_t reserved;
  uint64_t hbm_budget;  /* bytes the graph may allocate on the device; 0 = no limit */
} prune_graph_desc;

/* One frame record produced by SINK. */
typedef struct prune_frame_out {
  int64_t frame;  /* out: frame sequence number, 0 for the first frame pushed */
  int32_t c;      /* out: selected blocks (the DPG firing rate of this frame) */
  int32_t reserved;
  int32_t *idx;   /* in: caller buffer of F int32 (host or device per flags) */
  void *y;        /* in: caller buffer of F*B complex64; receives c*B samples */
} prune_frame_out;

/* Zero-copy view of a finished record that is still in the result ring. */
typedef struct prune_frame_view {
  int64_t frame;
  int32_t c;
  int32_t reserved;
  const int32_t *idx; /* device pointer, c entries */
  const void *y;      /* device pointer, c*B complex64 */
} prune_frame_view;

/* Eq. (2), Sec. VI-B: capacity in tokens of a FIFO with rate r, delay Q and
 * buffering constant C: r*C+Q if Q is not a multiple of r, else max(r*C, Q).
 * Host only.  EINVAL if r < 1, Q < 0 or C < 1. */
PRUNE_API prune_status prune_fifo_capacity(int64_t r, int64_t Q, int64_t C, int64_t *cap);

/* Validate the descriptor (shapes above; rates of every port match its FIFO,
 * Sec. III-A), size the FIFOs by eq. (2), allocate the device state (FIFO
 * rings, device-side head/tail counters, delay token = T-1 zeros, taps, H) and
 * upload it.  *out receives the graph, or NULL on error (see
 * prune_last_error(NULL)).  ENOMEM if the allocation exceeds hbm_budget.
 * Two buffers are allocated only when first needed, against the same
 * budget: the staging ring of C frames for copied pushes (at the first push
 * with PRUNE_MEM_HOST or PRUNE_MEM_DEVICE; borrowed pushes never need it),
 * and the FIR output ring of C frames of the actor-per-kernel path (at
 * creation when N >= 64, else at the first run with PRUNE_RUN_ACTORS; the
 * fused loops keep the FIR output on chip).  A call that needs one beyond
 * the budget returns ENOMEM and changes nothing. */
PRUNE_API prune_status prune_graph_create(const prune_graph_desc *desc, prune_graph **out);

/* Free every device and host resource of the graph after waiting for its
 * work.  Safe on NULL. */
PRUNE_API prune_status prune_graph_destroy(prune_graph *g);

/* Push n frames ([n][F][B] complex64) into f0 (the SRC actor's firings).
 * mem = PRUNE_MEM_HOST: x is host memory, copied asynchronously on the
 *   graph's stream (pinned memory must stay unchanged until the frames were
 *   fired, e.g. until prune_run(..., PRUNE_RUN_SYNC) or a pull of them);
 * PRUNE_MEM_DEVICE: x is device memory, copied on the stream;
 * PRUNE_MEM_DEVICE_BORROW: x is device memory that f0 references in place;
 *   it must stay valid and unchanged until the frames were fired (work that
 *   the caller orders on the graph's stream after prune_run is safe).
 * EAGAIN (and nothing pushed) if f0 lacks n*F free block slots. */
PRUNE_API prune_status prune_push_frames(prune_graph *g, const void *x, int32_t n, int32_t mem);

/* Fire the whole graph (FIR, DET, SEL, HX_b, SINK) on up to max_frames pushed
 * frames, in order, as far as the blocking rules allow (f0 tokens present and
 * room in the result ring).  The control tokens are dispatched on the device:
 * the host never reads c between DET and SINK.  *n_fired (optional) receives
 * the number of frames enqueued.  flags: PRUNE_RUN_*.  With PRUNE_RUN_SYNC a
 * device error (ETIMEOUT, EDEVICE) of these firings is returned here;
 * otherwise at the next pull, peek, sync or fifo_stats. */
PRUNE_API prune_status prune_run(prune_graph *g, int32_t max_frames, int32_t *n_fired, int32_t flags);

/* Wait for all work of the graph; report device-side errors. */
PRUNE_API prune_status prune_sync(prune_graph *g);

/* Pop up to max finished records (oldest first) into outs[0..max).  Waits for
 * the records that were fired.  mem = PRUNE_MEM_HOST or PRUNE_MEM_DEVICE
 * for the idx/y buffers, or PRUNE_MEM_DISCARD to drop the records (idx/y
 * ignored; frame and c still filled if outs is not NULL).  *n receives the
 * number popped.  EAGAIN if no fired frame is waiting.  A DISCARD with outs ==
 * NULL does not wait: the dropped slots are reused by later firings in stream
 * order. */
PRUNE_API prune_status prune_pull(prune_graph *g, prune_frame_out *outs, int32_t max, int32_t *n, int32_t mem);

/* View the i-th oldest unpulled record in place (device pointers valid until
 * it is pulled).  Waits for it.  EAGAIN if fewer than i+1 records wait. */
PRUNE_API prune_status prune_peek(prune_graph *g, int32_t i, prune_frame_view *view);

/* Cumulative token counters of one FIFO, read from the device: tokens
 * written (excluding initial tokens), tokens read, and the peak occupancy
 * observed when tokens were committed.  Waits for the graph's work. */
PRUNE_API prune_status prune_fifo_stats(prune_graph *g, int32_t fifo, uint64_t *written, uint64_t *read,
                              uint64_t *peak);

/* Capacity in tokens that the graph gave a FIFO (eq. (2)). */
PRUNE_API prune_status prune_fifo_capacity_of(prune_graph *g, int32_t fifo, int64_t *cap);

/* Per-kernel timing for measurement.  With enable != 0 the graph records a
 * CUDA event pair around every kernel it launches on its stream; kernel
 * kinds: 0 = f0 push commit, 1 = FIR(+energy), 2 = DET+SEL, 3 = HX on CUDA
 * cores, 4 = HX on tensor cores, 5 = fused firing loop on CUDA cores, 6 = fused
 * firing loop on tensor cores.  prune_kernel_times
 * waits for the graph, returns the summed device milliseconds and launch
 * count of one kind since the last reset, and resets that kind if reset != 0. */
PRUNE_API prune_status prune_profile(prune_graph *g, int32_t enable);
PRUNE_API prune_status prune_kernel_times(prune_graph *g, int32_t kind, double *ms, int64_t *launches,
                                          int32_t reset);

/* Message of the last failure on g (or of the last failed create when g is
 * NULL, per host thread).  Never NULL; valid until the next call on g. */
PRUNE_API const char *prune_last_error(const prune_graph *g);

/* ------------------------------------------------------------------------
 * Single-actor entry points on caller device buffers (stream-ordered,
 * asynchronous, no graph object).  They fire one actor (or one fused actor
 * pair) over `frames` consecutive frames of one instance and exist so that
 * each actor can be checked and timed on its own.
 * ---------------------------------------------------------------------- */

/* FIR actor with the DET energy reduction in its epilogue.
 *   x        device, [frames][F*B] complex64, the frames back to back
 *   hist     device, T-1 complex64: delay token before frame 0 (NULL = zeros)
 *   taps     device, T complex64
 *   y        device, [frames][F*B] complex64 output (may be NULL: energies only)
 *   energy   device, [frames][F] float32 block energies E_b (may be NULL)
 *   hist_out device, T-1 complex64: the delay token after the last frame (may be NULL)
 * Sizes as in prune_graph_desc. */
PRUNE_API prune_status prune_fir_energy(const void *x, const void *hist, const void *taps, int32_t F,
                              int32_t B, int32_t T, int32_t frames, void *y, float *energy,
                              void *hist_out, void *stream);

/* DET + SEL control path: v[b] = (energy[k][b] > tau); c[k] = sum_b v[b];
 * idx[k][0..c) = ascending b with v[b] (warp ballot and prefix scan).
 *   energy device [frames][F] float32; c device [frames] int32;
 *   idx device [frames][F] int32 (entries >= c[k] are left unchanged). */
PRUNE_API prune_status prune_det_sel(const float *energy, int32_t F, int32_t frames, float tau, int32_t *c,
                           int32_t *idx, void *stream);

/* HX_b over the compacted blocks (SEL's output DRPs, in place):
 *   out[k][j] = HX(y[k][idx[k][j]]) for j < c[k], where c and idx are read on
 *   the device.  y device [frames][F*B]; H device [N][N] complex64;
 *   out device [frames][F*B] (first c[k]*B samples of each frame written).
 * N < 64 runs on CUDA cores; N >= 64 on tcgen05 tensor cores (3-pass split
 * FP16 products, FP32 accumulation). */
PRUNE_API prune_status prune_hx(const void *y, const int32_t *idx, const int32_t *c, int32_t F, int32_t B,
                      int32_t N, int32_t frames, const void *H, void *out, void *stream);

/* ------------------------------------------------------------------------
 * Batched firing: many independent graph instances (Sec. V: the DPGs of
 * different instances are independent) with uneven F, T, tau, taps and H and
 * a common B and N.  One step fires one frame of every instance: FIR with the
 * instance's own delay token, DET, SEL, HX_b and SINK, in three launches over
 * the whole batch (HX_b on tcgen05 when N = 64, else CUDA cores), optionally
 * replayed as a captured CUDA graph.  Results stay on the device until pulled.
 * ---------------------------------------------------------------------- */

typedef struct prune_batch prune_batch;

enum { PRUNE_BATCH_GRAPH = 1 /* prune_batch_fire: capture the step once per (x, delay-token
                                parity) and replay it as a CUDA graph */ };

/* Create a batch of n instances from n descriptors (B and N equal in all;
 * stream, device and buffering of descs[0] apply to the batch).  The graph
 * shape rules of prune_graph_desc hold per instance; N >= 64 must be 64. */
PRUNE_API prune_status prune_batch_create(const prune_graph_desc *descs, int32_t n, prune_batch **out);
PRUNE_API prune_status prune_batch_destroy(prune_batch *b);

/* Offset (in complex samples) of instance i's frame in a step's input, and
 * the total samples of one step (the sum of F_i * B). */
PRUNE_API prune_status prune_batch_offset(prune_batch *b, int32_t i, int64_t *offset, int64_t *total);

/* Fire one frame of every instance.  x: device, complex64, 16-byte aligned,
 * all instances' frames back to back at the offsets above; referenced until
 * the step completes (stream order).  flags: PRUNE_BATCH_GRAPH.  Asynchronous. */
PRUNE_API prune_status prune_batch_fire(prune_batch *b, const void *x, int32_t flags);

/* Wait for the batch's work; report device errors. */
PRUNE_API prune_status prune_batch_sync(prune_batch *b);

/* Copy the last step's record of instance i (frame = step number, c, idx,
 * compacted y) to host (PRUNE_MEM_HOST) or device (PRUNE_MEM_DEVICE) buffers.
 * Waits for the batch. */
PRUNE_API prune_status prune_batch_pull(prune_batch *b, int32_t i, prune_frame_out *out, int32_t mem);

/* Message of the last failure on b. */
PRUNE_API const char *prune_batch_last_error(const prune_batch *b);

/* Launch shape of a batch step.  The FIR launch has one CTA per (instance,
 * tile of TS samples); the HX launch works through (instance, tile of rows)
 * items of the selected blocks. */
typedef struct prune_batch_tuning {
  int32_t fir_order;  /* 0: FIR tiles instance by instance; 1: instances with more taps first */
  int32_t hx_chunk;   /* 0: HX items spread over the grid by stride; > 0: each HX CTA fires this
                         many consecutive items (an instance's H operands load once per CTA) */
  int32_t hx_grid;    /* with hx_chunk = 0: CTAs of the HX launch (0: one wave) */
  int32_t reserved;
  double ms;          /* one step with this shape, as timed by prune_batch_autotune (else 0) */
} prune_batch_tuning;

/* Autotuner: fires the step on input x (as prune_batch_fire, without its
 * CUDA graph) with every candidate launch shape, `reps` timed steps each
 * (CUDA events on the batch's stream, after one untimed step), keeps the
 * fastest and returns it in *best; all candidates with their times go to
 * all[0..*n_all) (at most max_all; all may be NULL).  The candidates cross the
 * two FIR orders with HX grid-stride over one wave and HX chunks of one, two
 * and four waves.  The instances' state is left as it was: with the step
 * parity unchanged every trial reads the same delay tokens and overwrites
 * the same outputs.  Synchronous; cached step graphs are dropped. */
PRUNE_API prune_status prune_batch_autotune(prune_batch *b, const void *x, int32_t reps, prune_batch_tuning *best,
                                            prune_batch_tuning *all, int32_t max_all, int32_t *n_all);
/* Set / read the launch shape in use (set drops cached step graphs). */
PRUNE_API prune_status prune_batch_set_tuning(prune_batch *b, const prune_batch_tuning *t);
PRUNE_API prune_status prune_batch_get_tuning(const prune_batch *b, prune_batch_tuning *t);

/* ------------------------------------------------------------------------
 * Request loop (serving): streams of frames arrive and leave at run time.
 * Each admitted stream is one instance of the canonical graph whose
 * parameters, delay token and result FIFO stay resident in device memory
 * between requests; admission draws the stream's state from a fixed
 * device-memory budget.  A step fires the next frames of every admitted
 * stream that has queued frames and free result slots (the FIFO-space firing
 * condition, Sec. IV), all streams together in the batched launches, so that
 * streams that arrive while others are on the GPU join at the next step and
 * their work shares the device with the rest.  Up to `max_inflight` steps are
 * enqueued ahead of their completion.  One host thread per server.
 * ---------------------------------------------------------------------- */

typedef struct prune_server prune_server;

#define PRUNE_SERVER_AUTO_RELEASE 1  /* completed frames leave the result FIFO without a pull */

typedef struct prune_server_desc {
  int32_t B;               /* block size common to all streams (as prune_graph_desc) */
  int32_t N;               /* H size common to all streams; N = 64 runs HX on tensor cores */
  int32_t F_max;           /* largest F a stream may have */
  int32_t T_max;           /* largest T a stream may have */
  int32_t max_streams;     /* streams admitted at once */
  int32_t frames_per_step; /* frames one stream may advance per step (>= 1) */
  int32_t ring;            /* result FIFO of a stream, in frames (>= frames_per_step) */
  int32_t max_inflight;    /* steps enqueued ahead of completion (>= 1) */
  uint64_t hbm_budget;     /* bytes of device memory for the streams' resident state */
  void *stream;            /* cudaStream_t, or NULL for a stream owned by the server */
  int32_t device;          /* CUDA device, -1 = current */
  int32_t flags;           /* PRUNE_SERVER_* */
} prune_server_desc;

/* Allocates the budget as one device arena, the staging of max_inflight step
 * tables and the status word.  EINVAL on a bad descriptor, ENOMEM when the
 * device has no room for the budget. */
PRUNE_API prune_status prune_server_create(const prune_server_desc *d, prune_server **out);
/* Waits for the steps in flight and frees everything. */
PRUNE_API prune_status prune_server_destroy(prune_server *s);

/* Admit a stream with the parameters of g (F <= F_max, T <= T_max, B and N
 * those of the server; taps and H host pointers, copied; g->stream, C and
 * out_frames ignored).  PRUNE_EAGAIN, with nothing changed, when every slot is
 * taken or the arena has no hole for the stream's state (retry after a
 * close); the message then says which. */
PRUNE_API prune_status prune_server_open(prune_server *s, const prune_graph_desc *g, int64_t *id);

/* Queue n frames for stream id: frame q (0 <= q < n) is read at
 * x + (q % period) * F*B complex64 samples (period >= 1; period = n for n
 * distinct consecutive frames).  x device, 16-byte aligned, BORROWED: it must
 * stay valid and unchanged until those frames are done (prune_server_progress). */
PRUNE_API prune_status prune_server_submit(prune_server *s, int64_t id, const void *x, int64_t n, int64_t period);

/* Enqueue one step.  Retires completed steps first, and waits for the oldest
 * one when max_inflight are in flight.  *entries = frames fired by the step
 * (0: nothing is ready; nothing enqueued). */
PRUNE_API prune_status prune_server_step(prune_server *s, int32_t *entries);

/* Frames of stream id: submitted and not yet fired, fired, done (their step
 * completed), pulled (left the result FIFO).  Retires completed steps. */
PRUNE_API prune_status prune_server_progress(prune_server *s, int64_t id, int64_t *queued, int64_t *fired,
                                             int64_t *done, int64_t *pulled);

/* Streams that became idle (nothing queued, every fired frame done) since the
 * last call, each reported once per transition, with the host steady-clock
 * time (ns) at which the completion was observed.  Retires completed steps. */
PRUNE_API prune_status prune_server_poll(prune_server *s, int64_t *ids, int64_t *t_ns, int32_t max, int32_t *n);

/* Oldest done frame of stream id out of its result FIFO: out->frame, out->c,
 * and (mem HOST or DEVICE) c block indices into out->idx and c*B samples of
 * the compacted HX output into out->y; with PRUNE_MEM_DISCARD only the slot is
 * freed.  PRUNE_EAGAIN when no done frame is waiting. */
PRUNE_API prune_status prune_server_pull(prune_server *s, int64_t id, prune_frame_out *out, int32_t mem);

/* Leave: queued frames are dropped; the stream's memory and slot return to
 * the server once its last step has completed. */
PRUNE_API prune_status prune_server_close(prune_server *s, int64_t id);

/* Wait for every step in flight; PRUNE_ETIMEOUT / PRUNE_EDEVICE on a
 * device-side failure recorded by a kernel. */
PRUNE_API prune_status prune_server_sync(prune_server *s);

/* Arena bytes in use and in all, open streams, steps enqueued so far. */
PRUNE_API prune_status prune_server_stats(prune_server *s, uint64_t *hbm_used, uint64_t *hbm_budget,
                                          int32_t *open, int64_t *steps);

PRUNE_API const char *prune_server_last_error(const prune_server *s);

/* ------------------------------------------------------------------------
 * Graph front end: a PRUNE graph described actor by actor, port by port and
 * FIFO by FIFO (Sec. III), checked by the compile-time analysis of Sec. IV-V
 * and matched against the forms this runtime fires.  Host only; no device
 * needed.  A model is used by one host thread at a time.
 * ---------------------------------------------------------------------- */

typedef struct prune_model prune_model;

enum { PRUNE_ACTOR_STATIC = 0, PRUNE_ACTOR_DYNAMIC = 1, PRUNE_ACTOR_CONFIG = 2 };
enum { PRUNE_PORT_SRP = 0, PRUNE_PORT_DRP = 1, PRUNE_PORT_CTRL_IN = 2, PRUNE_PORT_CTRL_OUT = 3 };
enum {
  PRUNE_FORM_NONE = 0,      /* not a form the runtime fires */
  PRUNE_FORM_CANONICAL = 1, /* one DPG whose DCs are single static actors without delay
                               (HX_b): prune_graph_create with F = units */
  PRUNE_FORM_DPD = 2        /* one DPG whose DCs are single static actors each with a
                               self-loop delay (FIR_k): prune_dpd_fire with K = units */
};

typedef struct prune_model_report {
  int32_t rate_errors;    /* Sec. III-A: port atr != fiforate, control rate != 1, or a
                             port connected against its direction */
  int32_t type_errors;    /* Sec. III-B: ports an actor's type does not allow */
  int32_t rule_errors[5]; /* violations of design rules 1..5 (Sec. IV) */
  int32_t n_dpgs;         /* DPGs found: (q, x, y) with x's output DRPs and y's input
                             DRPs controlled by one control output port of q */
  int32_t consistent;     /* every DPG valid and consistent (Sec. V theorem) */
  char first_error[256];  /* the first violation found, or empty */
} prune_model_report;

PRUNE_API prune_status prune_model_create(prune_model **out);
PRUNE_API prune_status prune_model_destroy(prune_model *m);
/* Actors, ports and FIFOs get dense ids from 0 in creation order.  atr is
 * the port's active token rate (the itr of a DRP is 0, eq. (1)); control
 * ports have rate 1.  A FIFO runs from an output port to an input port with
 * `rate` tokens per firing and `delay` initial tokens. */
PRUNE_API prune_status prune_model_add_actor(prune_model *m, const char *name, int32_t kind, int32_t *actor);
PRUNE_API prune_status prune_model_add_port(prune_model *m, int32_t actor, const char *name, int32_t is_output,
                                            int32_t kind, int64_t atr, int32_t *port);
PRUNE_API prune_status prune_model_connect(prune_model *m, int32_t src_port, int32_t dst_port, int64_t rate,
                                           int64_t delay, int32_t *fifo);
/* Control table T[ctrl_out][drp] = element (1-based element of the control
 * token; 0 = not controlled). */
PRUNE_API prune_status prune_model_set_control(prune_model *m, int32_t ctrl_out_port, int32_t drp, int32_t element);
/* Run the analysis (cached until the model changes) and report. */
PRUNE_API prune_status prune_model_check(prune_model *m, prune_model_report *rep);
/* DPG i: its actors, number of DCs, validity and consistency. */
PRUNE_API prune_status prune_model_dpg(prune_model *m, int32_t i, int32_t *q, int32_t *x, int32_t *y,
                                       int32_t *n_dcs, int32_t *valid, int32_t *consistent);
/* DC k of DPG i: its members (actor ids; a dummy actor of the DC procedure's
 * step 1 is -(fifo + 1)) and its control element (0 if not unique). */
PRUNE_API prune_status prune_model_dc(prune_model *m, int32_t i, int32_t k, int32_t *members, int32_t max,
                                      int32_t *n, int32_t *element);
/* beta(f): the maximum over the DCs of the tokens on FIFO f during one period
 * of the DC's schedule (0 for FIFOs outside every DC; Sec. V proof). */
PRUNE_API prune_status prune_model_buffer_bound(prune_model *m, int32_t fifo, int64_t *beta);
/* Which runtime form the model is (PRUNE_FORM_*) and its number of DCs. */
PRUNE_API prune_status prune_model_classify(prune_model *m, int32_t *form, int32_t *units);
PRUNE_API const char *prune_model_last_error(const prune_model *m);

/* What the model does not carry: the MoC fixes token rates, not what the
 * actors compute, so the arithmetic of the runtime form's actors and the
 * size of a token come with the compile call. */
typedef struct prune_compile_params {
  int32_t B;            /* samples per data token: a block (canonical) or a period (DPD) */
  int32_t T;            /* taps of the FIR actor (of each FIR_k for DPD) */
  int32_t N;            /* canonical: H is N x N (N divides B) */
  int32_t C;            /* the buffering constant of eq. (2), >= 1 */
  float tau;            /* canonical: DET threshold, v[b] = (E_b > tau) */
  int32_t out_frames;   /* canonical: result records kept (0 = C) */
  const float *taps;    /* host; canonical: 2*T floats; DPD: the caller keeps its taps */
  const float *H;       /* host; canonical: 2*N*N floats, row-major */
  void *stream;         /* canonical: passed to prune_graph_desc */
  int32_t device;       /* canonical: passed to prune_graph_desc (-1 = current) */
  int32_t reserved;
  uint64_t hbm_budget;  /* canonical: passed to prune_graph_desc */
} prune_compile_params;

typedef struct prune_compiled {
  int32_t form;              /* PRUNE_FORM_CANONICAL or PRUNE_FORM_DPD */
  int32_t units;             /* DCs: F (canonical) or K (DPD) */
  prune_graph_desc graph;    /* canonical: the descriptor for prune_graph_create (F = units) */
  int32_t dpd_K, dpd_T;      /* DPD: K and T of prune_dpd_fire */
  int64_t dpd_period;        /* DPD: samples per period (= B) */
} prune_compiled;

/* Compile a checked model into the runtime form that fires it (Sec. IV-V:
 * the analysis must find no rate, type or design-rule violation and exactly
 * one valid, consistent DPG; Sec. VI: the compiler maps the graph onto the
 * runtime).  The canonical form is SRC -> FIR (a self-loop delay FIFO when
 * T > 1) -> {DET, SEL}, DET's control to SEL and SINK, SEL -> HX_b -> SINK
 * for the F DCs with control elements 1..F (element e = block e-1), token =
 * one block, rates F on the FIR FIFOs, 1 elsewhere, no delays besides FIR's
 * one token; it fills out->graph for prune_graph_create.  The DPD form is
 * a source feeding POLY (x) one period and CONF (q) one configuration
 * token, CONF's control to POLY and ADD (y), POLY -> FIR_k (self-loop delay
 * 1) -> ADD for K DCs with elements 1..K (element k = bit k-1 of the
 * period's mask), ADD -> at most one static sink, token = one period; it
 * fills dpd_K, dpd_T, dpd_period for prune_dpd_fire.  Any other model is
 * rejected with PRUNE_EINVAL and the rule, FIFO or actor that keeps it out
 * in prune_model_last_error(m).
 *   fifo_role[f]     (caller array of n_fifos, or NULL with n_fifos = 0): the
 *                    runtime FIFO model FIFO f becomes: canonical 0..7 = f0 (SRC
 *                    -> FIR), f1 (delay line), f2 (-> DET), f3 (-> SEL), f4, f5
 *                    (control to SEL, SINK), f6 (SEL -> HX_b), f7 (HX_b -> SINK);
 *                    DPD 0 input, 1 configuration input, 2 POLY -> FIR_k, 3 delay
 *                    line, 4 FIR_k -> ADD, 5 control, 6 adder output
 *   fifo_capacity[f] its capacity in tokens by eq. (2) with C
 * Host only; the model is not changed. */
PRUNE_API prune_status prune_model_compile(prune_model *m, const prune_compile_params *p, prune_compiled *out,
                                           int32_t *fifo_role, int64_t *fifo_capacity, int32_t n_fifos);

/* ------------------------------------------------------------------------
 * Dynamic Predistortion workload (Sec. VII-A2): a polynomial actor feeds K
 * parallel T-tap complex FIR filters (the DCs of a DPG), a configuration
 * actor selects from an external input, once per period, which filters fire,
 * and an adder sums them.  Branch k = 1..K carries psi_k(x) = x |x|^(k-1).
 * A filter that does not fire keeps its delay token (its last T-1 inputs)
 * until it fires again.  For every sample n of period p:
 *   y[n] = sum over k with bit k-1 of mask[p] set of sum_{t<T} h_k[t] psi_k[n-t]
 * where psi_k[n-t] before the period's first sample comes from branch k's
 * delay token.  All periods fire in parallel (a scan over the masks gives
 * every period its branches' tokens).
 * ---------------------------------------------------------------------- */

/* Bytes of device workspace prune_dpd_fire needs for P periods, K branches. */
PRUNE_API size_t prune_dpd_workspace_bytes(int32_t P, int32_t K);

/* Fire P periods of `period` samples (period a multiple of 8, >= T-1).
 *   x        device, [P][period] complex64, 16-byte aligned
 *   mask     device, [P] uint16: bit k-1 set = branch k fires in that period
 *            (bits >= K ignored; 0 = no branch: y is zero there)
 *   taps     device, [K][T] complex64, h_k[t] at taps[(k-1)*T + t]
 *   hist_in  device, [K][T-1] complex64 delay tokens before period 0, or NULL
 *            (zeros)
 *   hist_out device, [K][T-1] tokens after the last period, or NULL; may alias
 *            hist_in
 *   y        device, [P][period] complex64, 16-byte aligned
 *   workspace device, prune_dpd_workspace_bytes(P, K) bytes, caller-owned
 * 1 <= K <= 16, 1 <= T <= 16, P <= 65535.  Asynchronous on `stream`;
 * PRUNE_EINVAL (message in prune_last_error(NULL)) enqueues nothing. */
PRUNE_API prune_status prune_dpd_fire(const void *x, int64_t period, int32_t P, const uint16_t *mask, int32_t K,
                                      int32_t T, const void *taps, const void *hist_in, void *hist_out, void *y,
                                      void *workspace, size_t workspace_bytes, void *stream);

/* ------------------------------------------------------------------------
 * Adjoints over a recorded control trace (training the taps and H).  The
 * decisions v[b] = E_b > tau are piecewise constant in the parameters, so
 * with the trace (c, idx) of a forward firing held fixed the sink output is
 * linear in H (HX_b, Sec. V) and in the taps (FIR); the blocks of inactive
 * DCs (itr = 0) carry no gradient.  Gradients of a real loss are complex,
 * g = dL/dRe + i dL/dIm.  Both kernels ACCUMULATE into gH / gtaps (atomic
 * FP32 adds; the caller zeroes them); failures of argument checks return
 * PRUNE_EINVAL with the message in prune_last_error(NULL), enqueueing nothing.
 * ---------------------------------------------------------------------- */

/* HX_b adjoint.  For every frame k and selected slot j < c[k], block
 * b = idx[k][j], row r of B/N:  z = H w with w = y[k][b*B + r*N ...]:
 *   gH += g_z w^H  (g_z = gout[k][j*B + r*N ...], the compacted layout of
 *                   prune_hx's output)
 *   gy[k][b*B + r*N ...] = H^H g_z  (written; other blocks of gy untouched)
 *   y, gout, gy device [frames][F*B] complex64; idx, c device as from
 *   prune_det_sel; H, gH device [N][N] complex64.  N <= 64, N divides B. */
PRUNE_API prune_status prune_hx_adjoint(const void *y, const int32_t *idx, const int32_t *c, int32_t F,
                                        int32_t B, int32_t N, int32_t frames, const void *H,
                                        const void *gout, void *gy, void *gH, void *stream);

/* FIR adjoint: gtaps[t] += sum_n gy[n] conj(x[n - t]) over the frames as one
 * stream, x[n] for n < 0 taken from hist (T-1 samples, NULL = zeros).  Tiles
 * whose gy is all zero (no selected block) exit after staging.
 *   x, gy device [frames][F*B] complex64, 16-byte aligned; gtaps device [T].
 * Sizes as in prune_graph_desc. */
PRUNE_API prune_status prune_fir_adjoint(const void *x, const void *hist, const void *gy, int32_t F,
                                         int32_t B, int32_t T, int32_t frames, void *gtaps, void *stream);

/* ------------------------------------------------------------------------
 * Allocation-free firing.  The paper has no counterpart: this entry point
 * exists for callers of the library that cannot allocate device memory.
 * ---------------------------------------------------------------------- */

/* The fused firing loop (FIR, DET, SEL, HX_b, SINK; N < 64) over `frames`
 * consecutive frames of one instance, for callers that cannot call
 * cudaMalloc: real-time host threads that must not block in the device
 * allocator, and deployments whose device memory is budgeted and committed up
 * front, where an allocation at firing time may fail or is not permitted.
 * It allocates nothing: inputs and
 * outputs are the caller's, and its only scratch is a fixed array compiled
 * into the library (every GPU that loads the library holds it, about 527 KB,
 * until the process exits).  Results equal those of the graph entry points.
 *   x        device, [frames][F*B] complex64, 16-byte aligned
 *   hist     device, T-1 complex64 delay token before frame 0 (NULL = zeros)
 *   taps     device, T complex64;  H device, [N][N] complex64
 *   c        device, [frames] int32: selected blocks per frame
 *   idx      device, [frames][F] int32: ascending selected indices (first c[k])
 *   y        device, [frames][F*B] complex64, 16-byte aligned: compacted HX
 *            output (first c[k]*B samples of each frame)
 *   hist_out device, T-1 complex64 delay token after the last frame, or NULL;
 *            must not alias hist
 *   status   device, 4 uint32: zeroed by the call, then {code, actor, fifo,
 *            frame} of a device-side failure (code 0 = success)
 *   stream   cudaStream_t (NULL = legacy default stream); asynchronous
 * Limits: at most 256 frames per call and frames * tiles <= 65536, tiles =
 * ceil(F*B / TS) with TS the largest multiple of B not above 2048 (for
 * F = 4096, B = 1024: 32 frames per call).  Beyond that, for N >= 64 or for
 * a bad shape it returns PRUNE_EINVAL with a message in prune_last_error(NULL)
 * and enqueues nothing.  The first call on a device looks up the device
 * address of the scratch (once per device, with that device current); make
 * that first call before any stream capture.  Every call shares the scratch
 * and leaves its contents behind; each call clears what must start at zero,
 * in stream order, so calls ordered on one stream are safe, while calls that
 * can overlap on the GPU race on the scratch. */
PRUNE_API prune_status prune_fire_frames_noalloc(const void *x, const void *hist, const void *taps,
                                                 const void *H, int32_t F, int32_t B, int32_t T,
                                                 int32_t N, int32_t frames, float tau, int32_t *c,
                                                 int32_t *idx, void *y, void *hist_out,
                                                 uint32_t *status, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* PRUNE_H */
