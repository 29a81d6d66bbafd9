/*
 * qec.h -- C ABI of the GB300 parallel sparse-blossom decoder.
 *
 * The decoder solves the minimum-weight embedded matching problem of the
 * paper's "Decoding task" paragraph: given a detector graph G = (V, E) with
 * positive integer edge weights, boundary edges, observable masks on edges and
 * a set D of active detectors, find a minimum-weight edge set M whose degree is
 * odd exactly at the detectors in D (boundary vertices: any degree), and return
 * its weight and the XOR of the observable masks of its edges.  It runs sparse
 * blossom (SI Sec. S1: graph-fill regions, events (a)-(g), flooder events
 * ARRIVE / COLLIDE / IMPLODE) on the processing clusters of Algorithm 1 with
 * the hierarchical execution rule of Algorithm 2 (Methods).
 *
 * Every pointer is a plain host or device pointer as stated per argument; no
 * type of any framework appears here.  All calls are thread-compatible: a
 * qec_graph may be used by several threads at once for decoding; create and
 * destroy must not race with its use.
 *
 * Return codes: QEC_OK (0) or a negative QEC_E* value.  Per-shot outcomes are
 * written to status arrays as QEC_SHOT_* values.
 */
#ifndef QEC_H_
#define QEC_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- codes -- */
enum {
    QEC_OK = 0,
    QEC_EINVAL = -1,   /* bad argument: malformed graph, null pointer, size out of range */
    QEC_ENOMEM = -2,   /* host or device allocation failed */
    QEC_ECUDA = -3,    /* a CUDA runtime call failed (see qec_last_error) */
    QEC_EAGAIN = -4,   /* serving: admission is full, retry after polling */
    QEC_ERANGE = -5    /* a size exceeds a documented maximum */
};

enum {
    QEC_SHOT_OK = 0,
    QEC_SHOT_NO_SOLUTION = 1,     /* odd number of events in a part with no boundary */
    QEC_SHOT_BUDGET_EXCEEDED = 2, /* event budget hit; the kernel stopped, no hang */
    QEC_SHOT_CAPACITY = 3,        /* per-shot working set exceeds the largest slab */
    QEC_SHOT_INTERNAL = 4         /* an internal consistency check failed */
};

#define QEC_MAX_GRAPHS_PER_BATCH 32
#define QEC_MAX_OBSERVABLES 64

typedef struct qec_graph qec_graph;
typedef struct qec_stream qec_stream;
/* cudaStream_t, passed as an opaque pointer (NULL = legacy default stream). */
typedef void *qec_cuda_stream;

/* Algorithm 3 inputs (Methods, "Finite-size parameter schedule"):
 * q = q_num / q_den, phi_min = phi_num / phi_den, both in (0, 1).
 * NULL in qec_graph_desc means q = 1/10, phi_min = 1/100 (the paper's choice,
 * Methods "Numerical evaluation") and Algorithm 3's own level 1.
 * d1, b1 (internal units, twice the integer weights; 0 = Algorithm 3's) give a
 * custom level-1 processing-cluster diameter and buffer: b1 must satisfy the
 * level-1 conditions of Algorithm 3 (b1 >= d1, phi_1 = 1 > 2 d1 / b1,
 * Phi_2(b1) >= phibar_2), otherwise the schedule is rejected (QEC_EINVAL);
 * d1 alone takes the smallest such b1.  Higher levels follow from them by the
 * same recursion.  Theorem 1 makes any admissible schedule return a minimum-
 * weight matching; the parallelism it exposes differs (see QEC_DIAG_*). */
typedef struct {
    int32_t q_num, q_den;
    int32_t phi_num, phi_den;
    int32_t d1, b1;
} qec_params;

/* Detector graph (paper "Decoding task").  num_edges physical edges; edge i
 * joins detectors u[i] and v[i], or u[i] and its own boundary vertex when
 * v[i] < 0.  w[i] > 0 is the integer weight (e.g. round(16 ln((1-p)/p)));
 * obs[i] is the bit mask of logical observables the edge flips.  Parallel
 * edges are merged: the merged edge keeps the smallest weight (ties: lowest
 * input index) and that edge's mask; merged edges are ordered by
 * (min endpoint, max endpoint) with a boundary partner sorting last, and the
 * merged index decides ties between equally short boundary paths. */
typedef struct {
    int32_t num_detectors;     /* 1 .. 2^26 */
    int32_t num_edges;         /* 0 .. 2^28 */
    int32_t num_observables;   /* 0 .. 64 */
    const int32_t *u;          /* host, [num_edges] */
    const int32_t *v;          /* host, [num_edges], < 0 = boundary */
    const int32_t *w;          /* host, [num_edges], 1 .. 2^20 */
    const uint64_t *obs;       /* host, [num_edges] */
    const qec_params *params;  /* host or NULL */
} qec_graph_desc;

/* Information about a created graph. */
typedef struct {
    int32_t num_detectors;
    int32_t num_merged_edges;
    int32_t words_per_shot;    /* uint32 words of one padded syndrome row (multiple of 4) */
    int32_t wmax_internal;     /* largest merged weight x 2 */
    int32_t num_levels;        /* levels of the Alg. 3 schedule stored below */
    int64_t d_k[8];            /* Alg. 3 diameters d_k^V, internal units (level k at [k-1]) */
    int64_t b_k[8];            /* Alg. 3 buffers b_k^V, internal units */
    int32_t device;            /* CUDA device holding the graph */
    int32_t has_internal_obs;  /* some detector-detector edge carries an observable */
    int32_t components;        /* connected components of the detector graph */
    int32_t upper_single_cluster; /* 1: every detection event left after level 1
                                  * forms one processing cluster (one component
                                  * and b_2 >= distance_bound); the hierarchical
                                  * execution is then level 1 plus one top-level
                                  * cluster exactly */
    int64_t distance_bound;    /* upper bound on the distance between two connected
                                * detectors, internal units */
} qec_graph_info;

/* Algorithm 3 (Methods, "Finite-size parameter schedule") for a graph whose
 * largest internal weight (2 x the largest merged integer weight) is
 * wmax_internal: d_1 = wmax_internal + 1, phi_1 = 1; b_k is the smallest
 * integer with b_k >= d_k, phi_k > 2 d_k / b_k and Phi_{k+1}(b_k) >= phibar_{k+1};
 * phi_{k+1} = Phi_{k+1}(b_k); d_{k+1} = 3 d_k + 4 b_k + 2 wmax_internal.  Exact
 * rational arithmetic; stops early when a value would exceed 2^61.  Host only,
 * no device needed.  Writes up to max_levels entries to d_k / b_k (host
 * arrays, level k at index k-1) and returns the number of levels written
 * (>= 1), or QEC_EINVAL for bad arguments. */
int qec_schedule(int32_t wmax_internal, const qec_params *params, int64_t *d_k, int64_t *b_k,
                 int32_t max_levels);

/* Create a graph: validates and copies the host arrays, merges parallel edges,
 * computes the Alg. 3 schedule with exact rational arithmetic, and uploads a
 * CSR copy to the current CUDA device, which the library owns until
 * qec_graph_destroy.  Errors: QEC_EINVAL (endpoint out of range, self loop,
 * weight <= 0, more than 64 observables, bad params), QEC_ERANGE (size limits
 * above), QEC_ENOMEM, QEC_ECUDA.  *out is NULL on failure. */
int qec_graph_create(const qec_graph_desc *desc, qec_graph **out);
int qec_graph_destroy(qec_graph *g);
int qec_graph_get_info(const qec_graph *g, qec_graph_info *out);

/* Create the graph of one sliding window of a stream graph (the windowing rule
 * stated with qec_decode_window_batch below): the induced subgraph of `stream`
 * on its detectors [first_detector, first_detector + num_detectors), with those
 * detectors renumbered from 0 in the same order.  It holds every merged edge of
 * `stream` whose detector endpoints all lie in the range (boundary edges of
 * those detectors included) with its weight and observable mask; edges that
 * leave the range are left out.  params: host or NULL (NULL = the parameters
 * `stream` was created with).  The window is a graph of its own: on the
 * current device, owned by the library until qec_graph_destroy.  Errors:
 * QEC_EINVAL (NULL stream or out, bad params), QEC_ERANGE (range outside the
 * stream's detectors), and those of qec_graph_create.  *out is NULL on failure. */
int qec_graph_create_window(const qec_graph *stream, int32_t first_detector, int32_t num_detectors,
                            const qec_params *params, qec_graph **out);

/* Copy the merged edge list to host arrays of qec_graph_info.num_merged_edges
 * entries (u, v with -1 = boundary, internal weight = 2w, obs).  Any pointer may
 * be NULL. */
int qec_graph_merged_edges(const qec_graph *g, int32_t *u, int32_t *v, int32_t *w_internal,
                           uint64_t *obs);

/* Decode a batch of shots on the caller's stream (Alg. 1 + Alg. 2, SI S1).
 *
 * graphs            host array [num_graphs] (1 .. QEC_MAX_GRAPHS_PER_BATCH),
 *                   all created on the current device.
 * graph_of_shot     device [num_shots] int32 index into graphs, or NULL: every
 *                   shot uses graphs[0].
 * syn_offset_words  device [num_shots] int64 offset of each shot's syndrome row
 *                   in `syndromes` (in uint32 words, a multiple of 4), or NULL:
 *                   shot s starts at s * words_per_shot(graphs[0]).
 * syndromes         device uint32 rows: bit i of a row (word i/32, bit i%32,
 *                   LSB first) is detector i; words_per_shot words per row.
 * obs_out           device [num_shots] uint64 predicted observable flips.
 * weight_out        device [num_shots] int64 matching weight (original units).
 * status_out        device [num_shots] int32 QEC_SHOT_* code.
 * stream            cudaStream_t or NULL.
 *
 * The call enqueues work and returns without synchronising.  Scratch memory
 * comes from a library-owned workspace on the device, grown on first use
 * (that growth synchronises the device once, and a new workspace layout is
 * initialised by one asynchronous fill on `stream`); calls that share the
 * workspace are serialised on their streams by the library.  Errors: QEC_EINVAL (null
 * output pointers, num_graphs out of range, graphs on another device),
 * QEC_ENOMEM, QEC_ECUDA. num_shots == 0 is a no-op.
 *
 * CUDA graphs: a call on a stream that is capturing is recorded into the
 * caller's graph (kernel arguments, shot count and the current tuning are
 * fixed at capture).  It needs a call of the same shape (graphs, shot count,
 * tuning) made before outside capture, which sizes and fills the workspace;
 * otherwise it returns QEC_EINVAL.  Captured work does not take part in the
 * library's ordering of workspace users: replays of the graph must not overlap
 * other decodes on the same device.  The same holds for qec_decode_batch_ex
 * and qec_decode_window_batch. */
int qec_decode_batch(const qec_graph *const *graphs, int32_t num_graphs,
                     const int32_t *graph_of_shot, const int64_t *syn_offset_words,
                     const uint32_t *syndromes, int64_t num_shots,
                     uint64_t *obs_out, int64_t *weight_out, int32_t *status_out,
                     qec_cuda_stream stream);

/* Execution modes of qec_decode_batch_ex. */
enum {
    QEC_MODE_HIERARCHICAL = 0,   /* Alg. 1 level-1 clusters, then one top-level run (Alg. 2) */
    QEC_MODE_GLOBAL = 1          /* one sparse-blossom run over every detection event */
};

/* Per-shot diagnostics of qec_decode_batch_ex, QEC_DIAG_FIELDS int32 per shot.
 * An event is one step of the matcher: a collision of two regions (events
 * (a)-(c), (e), (g) of SI S1), a region reaching the boundary (f) or an inner
 * blossom imploding (d).  The parallel event count E_ideal and its stopping
 * time follow Methods, "Numerical evaluation": with t1 / E1 the largest
 * stopping time / event count of the level-1 clusters (0 without any), the
 * top-level run with N events, E_top(t1) of them at times <= t1, gives
 * E_ideal = max(E1, E_top(t1)) + N - E_top(t1) (E1 when no event is left after
 * level 1), which is the paper's recursion when every event above level 1
 * forms one processing cluster: qec_graph_info.upper_single_cluster = 1, true
 * for every rotated-surface-code graph here (phenomenological and circuit
 * level) under the default and the tested custom schedules.  On a graph where it
 * is 0 the hierarchical run still returns the matching of Theorem 1, but the
 * counts are those of level 1 plus one run of all remaining events.  In global
 * mode E_ideal is the run's whole event count.  Times are in internal units
 * (twice the integer weights).  Shots whose status is not QEC_SHOT_OK and
 * shots without detection events get all zeros. */
#define QEC_DIAG_FIELDS 8
enum {
    QEC_DIAG_E_IDEAL = 0,       /* parallel event count */
    QEC_DIAG_T_IDEAL = 1,       /* its critical-path stopping time */
    QEC_DIAG_EVENTS = 2,        /* events of all runs of the shot */
    QEC_DIAG_L1_CLUSTERS = 3,   /* level-1 processing clusters */
    QEC_DIAG_L1_DEFECTS = 4,    /* detection events resolved at level 1 */
    QEC_DIAG_TOP_EVENTS = 5,    /* events of the top-level (or global) run */
    QEC_DIAG_BANDS = 6,         /* flooder band extensions of the event loop (GPU work, not an event) */
    QEC_DIAG_DEFECTS = 7        /* detection events of the shot */
};

/* qec_decode_batch with an execution mode and optional diagnostics.
 * mode        QEC_MODE_HIERARCHICAL (what qec_decode_batch runs) or
 *             QEC_MODE_GLOBAL; both return a minimum-weight embedded matching
 *             (Theorem 1), and with the canonical event order the same one.
 * diag_out    device [num_shots][QEC_DIAG_FIELDS] int32, or NULL.
 * Other arguments, errors and the asynchronous behaviour are those of
 * qec_decode_batch; QEC_EINVAL also for an unknown mode. */
int qec_decode_batch_ex(const qec_graph *const *graphs, int32_t num_graphs,
                        const int32_t *graph_of_shot, const int64_t *syn_offset_words,
                        const uint32_t *syndromes, int64_t num_shots, int32_t mode,
                        uint64_t *obs_out, int64_t *weight_out, int32_t *status_out,
                        int32_t *diag_out, qec_cuda_stream stream);

/* ------------------------------------------------------ sliding windows --
 * Streaming decoding in overlapping windows (the paper's introduction: in
 * sliding-window decoding the windows are processed one after another, so the
 * time per syndrome round sets the throughput).  The caller cuts a long
 * syndrome history into windows of W detector layers every C layers; a window's
 * graph is the induced subgraph of the stream graph on its layers, and its
 * commit region is its first C layers (every layer for the last window).  The
 * window's correction -- the union of the canonical shortest paths of its
 * matching (one per matched pair, one to the boundary per boundary match) -- is
 * committed on every edge that touches the commit region: the committed
 * observable accumulates, and each committed edge whose other endpoint lies
 * outside the region flips that detector, which the next window's syndrome
 * takes over (qec_window_assemble).  Every detector lies in exactly one commit
 * region, so the committed edges of all windows together correct the whole
 * history's syndrome. */

/* Mark the detectors of g's commit region: detector_bitmap is a host array of
 * words_per_shot(g) uint32 words (bit i = detector i), copied before return;
 * NULL removes the region (and waits for the device to be idle).  Errors:
 * QEC_EINVAL, QEC_ENOMEM, QEC_ECUDA. */
int qec_graph_set_commit_region(qec_graph *g, const uint32_t *detector_bitmap);

/* Decode one window of a batch of streams (Alg. 1 + Alg. 2, as
 * qec_decode_batch).  Every graph needs a commit region (QEC_EINVAL otherwise).
 * commit_obs_inout  device [num_shots] uint64: the committed observable of
 *                   each shot is XORed into it.
 * carry_out         device uint32 rows laid out like `syndromes` (same
 *                   offsets): the detectors flipped by committed edges that
 *                   leave the commit region (all zero for a failed shot).
 * status_inout      device [num_shots] int32: set to the QEC_SHOT_* failure of
 *                   a shot that fails, left unchanged otherwise (initialise to
 *                   QEC_SHOT_OK once per stream).
 * Other arguments, errors and the asynchronous behaviour are those of
 * qec_decode_batch. */
int qec_decode_window_batch(const qec_graph *const *graphs, int32_t num_graphs,
                            const int32_t *graph_of_shot, const int64_t *syn_offset_words,
                            const uint32_t *syndromes, int64_t num_shots,
                            uint64_t *commit_obs_inout, uint32_t *carry_out, int32_t *status_inout,
                            qec_cuda_stream stream);

/* Window syndromes from stream syndromes, on the device: bit i of window row r
 * is bit (bit_begin + i) of stream row r for i < nbits (0 beyond), XOR bit
 * (carry_bit_begin + i) of carry row r for i < carry_bits when carry_rows is
 * not NULL.  Rows: stream_rows [num_rows][stream_words], carry_rows
 * [num_rows][carry_words], window_rows [num_rows][window_words] (all device
 * uint32).  Errors: QEC_EINVAL (negative sizes, NULL buffers), QEC_ERANGE
 * (nbits or carry_bits beyond the window row), QEC_ECUDA. */
int qec_window_assemble(const uint32_t *stream_rows, int64_t stream_words, int64_t bit_begin, int32_t nbits,
                        const uint32_t *carry_rows, int64_t carry_words, int64_t carry_bit_begin,
                        int32_t carry_bits, uint32_t *window_rows, int64_t window_words, int64_t num_rows,
                        qec_cuda_stream stream);

/* Same as qec_decode_batch for one shot per kernel launch: shot s is decoded
 * by its own launch of a one-warp grid (the plain per-shot GPU path). */
int qec_decode_plain(const qec_graph *g, const uint32_t *syndromes, int64_t num_shots,
                     uint64_t *obs_out, int64_t *weight_out, int32_t *status_out,
                     qec_cuda_stream stream);

/* Tuning knobs of the batched path (chosen by the autotuner in the Python
 * binding; all have safe defaults).  In qec_set_tuning a positive value sets
 * a knob, zero keeps its current value and a negative value restores the
 * default (warps_per_block 4, blocks_per_sm 0 = as many as fit, band_factor 1,
 * kcap 0 = num_detectors / 16 clamped to 64 .. 1024, or to 64 .. 4096 for graphs
 * of at least 32,768 detectors, max_events 4e6,
 * team_warps 0 = automatic, team_min_detectors 2048, team_split_events 1:
 * every shot of a block goes to the whole block; on a GB300 the autotuner's
 * split search found no threshold faster than that for single windows).
 * qec_get_tuning reports 0 for the automatic choices.
 *
 * team_warps is the number of warps that decode one shot together: 1 = one warp
 * per shot (the throughput path: as many shots in flight as warps fit), 4 or
 * 16 = one thread block of that many warps per shot (every step of the shot
 * spread over the block: the latency path for large windows).  Automatic, for
 * a batch whose largest graph has at least team_min_detectors detectors: 16
 * when the batch has at most one shot per SM, 4 when the largest graph has at
 * least 32,768 detectors or the batch has fewer shots than half the one-warp
 * teams the GPU holds at once, else 1 (and always 1 for smaller graphs).
 * Results do not depend on it.  Shots with more detection events than kcap
 * go to a second pass with one team per SM: for windows larger than the
 * default kcap holds, raise kcap to keep them in the main pass. */
typedef struct {
    int32_t warps_per_block;   /* 1 .. 32 */
    int32_t blocks_per_sm;     /* 1 .. 64 */
    int32_t band_factor;       /* flooder band width in units of the largest weight, 1 .. 64 */
    int32_t kcap;              /* detection events per shot held by a main-pass slab */
    int64_t max_events;        /* event budget per shot */
    int32_t team_warps;        /* 1, 4 or 16; 0 = automatic */
    int32_t team_min_detectors;   /* automatic team choice: smallest graph for a block per shot */
    int32_t team_split_events; /* a block decodes a shot with fewer detection events than
                                * this with its first warp alone (1: never) */
} qec_tuning;
int qec_set_tuning(const qec_tuning *t);
int qec_get_tuning(qec_tuning *t);

/* qec_decode_batch without any device allocation.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate device
 * memory while running -- a real-time decoding loop that must not stall on the
 * driver's allocator or fail half-way for lack of memory, or an application
 * that reserves all device memory at start-up.  Its scratch is one static
 * device array of QEC_STATIC_SCRATCH_BYTES that every GPU loading the library
 * holds until the process exits; it calls no cudaMalloc, cudaFree or other
 * allocating routine.
 *
 * Arguments, layouts and outputs are those of qec_decode_batch, and the band
 * width and event budget set by qec_set_tuning apply as there (the other
 * knobs do not: the launch shape and slab size are fixed).  Limits:
 * num_shots <= QEC_STATIC_MAX_SHOTS (else QEC_ERANGE, nothing launched); a
 * shot with more than QEC_STATIC_MAX_EVENTS detection events ends with status
 * QEC_SHOT_CAPACITY, and so does every shot of a graph whose rows exceed
 * QEC_STREAM_MAX_WORDS words.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current and enqueues one fill
 * of the array on `stream`; it returns QEC_EINVAL if `stream` is capturing, so
 * make that first call before any stream capture.  A first call that fails
 * leaves the device not set up, and the next call repeats the set-up.  Every call shares the array and zeroes its
 * work counters on `stream`: calls whose work overlaps on the GPU race, so the
 * caller must order them (for example by issuing them on one stream). */
#define QEC_STATIC_SCRATCH_BYTES (80LL * 1024 * 1024)
#define QEC_STATIC_WARPS 152
#define QEC_STATIC_MAX_EVENTS 128
#define QEC_STATIC_MAX_SHOTS (1 << 20)
int qec_decode_batch_static(const qec_graph *const *graphs, int32_t num_graphs,
                            const int32_t *graph_of_shot, const int64_t *syn_offset_words,
                            const uint32_t *syndromes, int64_t num_shots,
                            uint64_t *obs_out, int64_t *weight_out, int32_t *status_out,
                            qec_cuda_stream stream);

/* ------------------------------------------------------------ serving --
 * A request loop for syndrome windows that arrive one at a time (continuous
 * batching).  qec_stream_submit copies one window into the micro-batch being
 * filled; a dispatcher thread owned by the stream launches that micro-batch as
 * soon as one of the stream's in-flight slots is free, so requests that arrive
 * while others are on the GPU join the next launch and several launches
 * overlap on the device (one CUDA stream and scratch workspace per slot).
 * Graphs stay resident; results are read back into pinned memory and handed
 * out by qec_stream_poll.  Each result is the same as decoding the window
 * alone with qec_decode_batch.  Each window of a micro-batch is decoded by a
 * team of qec_tuning.team_warps warps; automatic: a thread block of 16 warps
 * per window while the micro-batch has no more windows than the GPU holds such
 * blocks at once, else one warp per window. */
#define QEC_STREAM_MAX_WORDS 2304          /* largest window: 73,728 detectors */
#define QEC_STREAM_MAX_GRAPHS QEC_MAX_GRAPHS_PER_BATCH

typedef struct {
    uint64_t request_id;
    uint64_t obs;          /* predicted observable flips */
    int64_t weight;        /* matching weight, original units */
    int32_t status;        /* QEC_SHOT_* */
    int32_t graph_index;   /* index of the graph in the stream's registry */
    int64_t t_submit_ns;   /* CLOCK_MONOTONIC time of qec_stream_submit */
    int64_t t_done_ns;     /* CLOCK_MONOTONIC time the result became available */
} qec_result;

/* Create a serving stream on the current device.  device_budget_bytes bounds
 * the device memory of the stream's in-flight slots (each slot: scratch for
 * 2 warps per SM with room for 512 detection events per window, an overflow
 * pass for larger windows, and window/result buffers); it must hold at least
 * two slots (QEC_ENOMEM otherwise) and at most eight are used.  max_inflight
 * (>= 1) bounds the windows admitted (queued or on the GPU) at once.
 * Errors: QEC_EINVAL, QEC_ENOMEM, QEC_ECUDA. */
int qec_stream_create(size_t device_budget_bytes, int32_t max_inflight, qec_stream **out);

/* Submit one window: `syndrome_host` holds words_per_shot(g) uint32 words
 * (host memory, copied before return).  Returns QEC_EAGAIN when max_inflight
 * windows are admitted or the filling micro-batch is full (poll, then retry),
 * QEC_ERANGE when the graph's rows exceed QEC_STREAM_MAX_WORDS or more than
 * QEC_STREAM_MAX_GRAPHS distinct graphs are used, QEC_EINVAL for NULL
 * arguments or a graph on another device. */
int qec_stream_submit(qec_stream *s, const qec_graph *g, const uint32_t *syndrome_host,
                      uint64_t request_id);

/* Submit n windows in order, stopping at the first one that is not admitted
 * (same rules as qec_stream_submit); *n_accepted = windows taken.  Window i
 * uses graphs[graph_of_req[i]] and starts at syn_offset_words[i] in
 * syndromes_host (host arrays). */
int qec_stream_submit_many(qec_stream *s, const qec_graph *const *graphs, int32_t num_graphs,
                           const int32_t *graph_of_req, const int64_t *syn_offset_words,
                           const uint32_t *syndromes_host, const uint64_t *request_ids, int32_t n,
                           int32_t *n_accepted);

/* Move up to max finished results to out (host array); *n_out = count.  Never blocks. */
int qec_stream_poll(qec_stream *s, qec_result *out, int32_t max, int32_t *n_out);

/* Block until every admitted window has finished (results stay pollable). */
int qec_stream_flush(qec_stream *s);

/* Stop the dispatcher, wait for in-flight work, free everything. */
int qec_stream_destroy(qec_stream *s);

/* Release the library-owned device workspace of the current device. */
int qec_release_workspace(void);

/* Text of the most recent error of the calling thread (never NULL). */
const char *qec_last_error(void);

/* Version string. */
const char *qec_version(void);

#ifdef __cplusplus
}
#endif

#endif /* QEC_H_ */
