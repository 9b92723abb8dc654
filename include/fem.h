/*
 * fem.h -- C ABI of the GB300 frequent-episode counting library (libfem.so).
 *
 * The library counts, for serial episodes with inter-event constraints, the
 * size of the largest set of non-overlapped occurrences in a time-ordered
 * event stream, and runs the level-wise (Apriori) mining procedure on top of
 * that count.  Passages of "Accelerator-Oriented Algorithm Transformation for
 * Temporal Data Mining" (Patnaik, Ponce, Cao, Ramakrishnan) are cited by
 * section name.
 *
 * Conventions shared by every entry point
 *   - Every function returns int status: FEM_OK (0) or a negative FEM_ERR_*.
 *     No function throws, aborts or prints.  fem_strerror() names a status.
 *   - Pointers marked "host or device" are device pointers when the matching
 *     *_is_device / ptr_is_device argument is non-zero, host pointers
 *     otherwise.  The library never keeps a caller pointer after it returns:
 *     it copies what it needs.
 *   - Calls are synchronous: when a call returns, its outputs (host or device)
 *     are written and every kernel it launched has finished.
 *   - A context is used by one host thread at a time (calls on one context
 *     are serialised by an internal mutex); different contexts are
 *     independent.
 *   - Times are int32 ticks in [0, 2^31 - 2] (the tick is the caller's
 *     unit); types are uint16 ids < n_types.
 *
 * Episode semantics (section "Temporal Data Mining")
 *   An N-node episode is E_1 -(lo_1,hi_1]-> E_2 ... -> E_N.  An occurrence is a
 *   choice of events j_1 < ... < j_N with type(j_k) = E_k and
 *   lo_k < t(j_{k+1}) - t(j_k) <= hi_k.  Two occurrences are non-overlapped
 *   when one ends strictly before the other starts (Algorithm 1's test
 *   prev_e < s_i).  The count is the largest number of pairwise
 *   non-overlapped occurrences.  Intervals must satisfy 0 <= lo < hi.
 */
#ifndef FEM_H
#define FEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define FEM_OK 0
#define FEM_ERR_INVAL -1       /* null pointer, negative size, type >= n_types,
                                  lo < 0, lo >= hi, episode size outside
                                  [1, FEM_MAX_NODES], bad handle */
#define FEM_ERR_UNSORTED -2    /* stream times decrease somewhere */
#define FEM_ERR_DUP -3         /* two events with the same (type, time) */
#define FEM_ERR_RANGE -4       /* a time < 0 or = 2^31 - 1 */
#define FEM_ERR_NOMEM -5       /* the context's device-memory budget (or the
                                  device) cannot hold the request */
#define FEM_ERR_TIMEOUT -6     /* a device-side wait gave up after its
                                  iteration limit; the context stays usable */
#define FEM_ERR_CUDA -7        /* a CUDA runtime call failed */
#define FEM_ERR_BUSY -8        /* serving: job queue full / job not finished */
#define FEM_ERR_NOTFOUND -9    /* serving: unknown job id */

#define FEM_MAX_NODES 16       /* largest episode size accepted */

typedef struct fem_ctx fem_ctx;
typedef struct fem_stream fem_stream;
typedef struct fem_result fem_result;

/* Candidate episodes in CSR form.
 *   n_cand           number of episodes (>= 0)
 *   offs[n_cand+1]   int64 node offsets: episode c has nodes
 *                    types[offs[c] .. offs[c+1]-1], offs[0] = 0
 *   types[offs[n]]   uint16 event type of every node
 *   lo, hi           int32 bounds of every edge: episode c's edges are at
 *                    lo/hi[offs[c]-c .. offs[c+1]-c-2] (N_c - 1 of them)
 *   ptr_is_device    non-zero: offs/types/lo/hi are device pointers         */
typedef struct {
    int64_t n_cand;
    const int64_t *offs;
    const uint16_t *types;
    const int32_t *lo;
    const int32_t *hi;
    int ptr_is_device;
} fem_cands;

/* Optional launch parameters.  Zero in a field means "choose automatically"
 * (autotuner cache, else the built-in heuristic). */
typedef struct {
    int lanes_per_cta;    /* episodes held by one CTA (multiple of 32) */
    int segments;         /* stream segments per recording (>= 1) */
    int tile_events;      /* events per shared-memory stage (multiple of 256) */
    int prepass;          /* upper-bound pre-passes of level-wise mining:
                             0 = the level-2 pair bound and, with the
                             mining graph and local tracking, the level-3
                             join bound (per candidate the number of events
                             of its middle type that end its frequent
                             2-node prefix and start its frequent 2-node
                             suffix); 1 = both and the coarse-tick bound
                             of fem_upper_bound_coarse on every level >= 3;
                             2 = the level-2 pair bound only; -1 = none.
                             Candidates whose bound is at or below the
                             threshold skip the exact count and are
                             reported as pruned, never as counted */
    int plain_path;       /* 1 = count with the one-thread-per-episode plain
                             path (comparison baseline) instead of the tiled
                             kernels */
    int autotune;         /* 1 = time a few launch configurations (lanes per
                             CTA, tile size, segment count, kernel) the first
                             time a workload signature is seen and keep the
                             fastest in the context's tuning cache */
    int kernel;           /* 0 = choose per launch (grid-wide local
                             tracking (4) for at most 256 episodes over a
                             recording of at least 2^20 events, otherwise
                             warp-per-item local tracking (7)), 1 = always the tiled
                             shared-memory broadcast kernel, 2 = the sparse
                             per-type-list kernel where it applies, 3 = the
                             sparse kernel with per-node branching instead of
                             its node-uniform variant (comparison), 4 = node-
                             by-node local tracking over the per-type lists
                             (section "Parallel Local Tracking": parallel
                             over events, for few long episodes), 5 / 6 =
                             local tracking that materialises every partial
                             occurrence, compacting each step's list with
                             atomics (5) or count, scan and write (6); an
                             episode whose list would pass 2^25 entries is
                             counted as with 4 and adds to
                             fallback_recounts; 7 = local tracking with one
                             warp per (episode, segment) work item taken
                             from an atomic queue by one persistent launch
                             for every multi-node episode of the call (with
                             0, consecutive episodes that share their first
                             N-1 nodes and edges form one item and track
                             that prefix once) */
    int level_graph;      /* mining: 0 = run the levels as one captured CUDA
                             graph where it applies (all levels when no
                             other override is set and every alphabet has at
                             least 16 types; otherwise levels >= 3 after a
                             host-driven level 2), -1 = level by level from
                             the host */
    int wait_polls;       /* 0 = default: a wait of the tiled kernel's shared-
                             memory pipeline gives up after 2^30 polls or 4 s;
                             n > 0 = after n non-blocking polls (a short limit
                             for tests of the timeout path).  A wait that gives
                             up makes the call return FEM_ERR_TIMEOUT; the
                             kernel first waits (with the default limit) for
                             its copies in flight, so the context stays
                             usable */
    int track_last;       /* last node of the warp-per-item local tracking
                             kernel: 0 = per (episode, segment), driven by
                             node N-1's events or, when they outnumber node
                             N-2's entries more than twice, by those entries
                             (one lookup in the stream's per-type time index
                             per entry, for the first end it can serve);
                             1 = always by events; 2 = always by entries */
} fem_tuning;

/* Per-call statistics filled by the counting / mining calls. */
typedef struct {
    double episode_events;      /* sum over resolved (episode, recording) of n:
                                   every candidate is resolved over its whole
                                   recording, by the exact count or, in
                                   mining, by the upper-bound pre-pass */
    double counted_episode_events; /* the part resolved by the exact count */
    double relevant_events;     /* sum over counted episodes of sum_k freq(E_k) */
    int64_t candidates_counted; /* exact counts computed */
    int64_t candidates_pruned;  /* dropped by the upper-bound pre-pass */
    int64_t fallback_recounts;  /* episodes recounted unsegmented */
    int64_t kernel_launches;    /* library kernels launched by the call */
    int64_t sparse_launches;    /* counting launches over the per-type
                                   lists (sparse or warp-per-item local
                                   tracking kernel; the rest used the tiled
                                   broadcast kernel) */
    double count_kernel_ms;     /* device time of the exact-count kernels */
    double total_ms;            /* wall time of the call */
    int levels;                 /* mining: deepest level reached */
    int graph_tails;            /* mining: 1 if levels ran as one captured
                                   CUDA graph (kernel_launches then counts its
                                   kernel nodes) */
} fem_stats;

/* ---- context ----------------------------------------------------------- */

/* Creates a context on CUDA device `device`.
 *   hbm_budget_bytes  upper bound on device memory the context may hold
 *                     (streams + scratch); 0 = 90% of the device's free memory
 *   cuda_stream       a cudaStream_t to run on, or NULL for a stream the
 *                     context creates and owns
 * On success *out owns the context; free it with fem_ctx_destroy. */
int fem_ctx_create(int device, size_t hbm_budget_bytes, void *cuda_stream, fem_ctx **out);
void fem_ctx_destroy(fem_ctx *ctx);
int fem_ctx_set_tuning(fem_ctx *ctx, const fem_tuning *t);    /* NULL resets */
int fem_ctx_last_stats(const fem_ctx *ctx, fem_stats *out);  /* of the last call */
/* Bytes currently held on the device by the context (streams + scratch). */
int fem_ctx_memory(const fem_ctx *ctx, size_t *used, size_t *budget);
/* Backs the context's autotuner cache with a JSON file: entries in `path` (if
 * it exists) are loaded now, and every new choice is written back.  The file
 * maps a workload signature ("n<size class>.r<ring class>.c<log2 episodes>.
 * e<log2 events>.m<recordings>") to [lanes_per_cta, tile_events,
 * segment multiplier, kernel (1 tiled, 2 sparse)].  NULL detaches the file (the cache stays in memory).
 * FEM_ERR_INVAL if the file exists but cannot be parsed. */
int fem_ctx_set_autotune_cache(fem_ctx *ctx, const char *path);

/* ---- streams ------------------------------------------------------------ */

/* Loads an event stream (Definition 1: time-ordered (type, time) pairs) into
 * device memory owned by the library, validates it on the device and
 * computes the level-1 counts (a 1-node episode's count is its type's
 * frequency).
 *   types[n], times[n]  host or device (ptr_is_device); caller keeps them
 *   n >= 0, n_types in [1, 65536]
 * Errors: FEM_ERR_INVAL (type >= n_types), FEM_ERR_RANGE (time < 0 or
 * time = 2^31 - 1),
 * FEM_ERR_UNSORTED, FEM_ERR_DUP (a repeated (type, time) would make two
 * events count once), FEM_ERR_NOMEM. */
int fem_load_stream(fem_ctx *ctx, const uint16_t *types, const int32_t *times, int64_t n,
                    uint32_t n_types, int ptr_is_device, fem_stream **out);
void fem_stream_free(fem_stream *s);
int fem_stream_info(const fem_stream *s, int64_t *n, uint32_t *n_types);
/* Level 1: freq[n_types] (host or device) = events of each type. */
int fem_stream_freq(fem_ctx *ctx, const fem_stream *s, uint32_t *freq, int out_is_device);

/* ---- counting (the hot path) ------------------------------------------- */

/* Exact count of every candidate episode over one stream ("Episode Counting
 * Algorithm" semantics; frequency as defined in "Temporal Data Mining").
 * counts[n_cand] (host or device) receives uint32 counts in input order.
 * Internally: segment-parallel exact counting with a boundary stitch-up
 * (section "MapConcat"), stream tiles staged in shared memory and broadcast
 * to many episode machines per CTA, and an optional upper-bound pre-pass.
 * Errors: FEM_ERR_INVAL on a malformed candidate (see above),
 * FEM_ERR_NOMEM, FEM_ERR_TIMEOUT, FEM_ERR_CUDA. */
int fem_count_episodes(fem_ctx *ctx, const fem_stream *s, const fem_cands *c, uint32_t *counts,
                       int out_is_device);

/* Same, for candidates spread over several recordings: candidate c is
 * counted on recs[rec_id[c]].  rec_id[n_cand] (host or device, like the
 * candidate arrays).  All recordings are counted in one launch. */
int fem_count_batch(fem_ctx *ctx, const fem_stream *const *recs, int n_recs, const fem_cands *c,
                    const uint32_t *rec_id, uint32_t *counts, int out_is_device);

/* Comparison path: one GPU thread per candidate, reading the stream straight
 * from global memory, the serial state machine of "Episode Counting
 * Algorithm" with its lists in global memory (the mapping the section
 * "Temporal Data Mining" calls embarrassingly parallel).  Same contract and
 * results as fem_count_episodes. */
int fem_count_episodes_plain(fem_ctx *ctx, const fem_stream *s, const fem_cands *c,
                             uint32_t *counts, int out_is_device);

/* Upper-bound pre-pass: ub[c] >= count(c) for every candidate.  It counts the
 * episode with every lower bound relaxed to 0 (a superset of occurrences, so
 * the largest non-overlapped set can only grow; anti-monotonicity, section
 * "Temporal Data Mining"). ub (host or device) is uint32[n_cand]. */
int fem_upper_bound(fem_ctx *ctx, const fem_stream *s, const fem_cands *c, uint32_t *ub,
                    int out_is_device);

/* Coarse-tick upper bound: ub[c] >= count(c), cheaper than the count on
 * long streams (a pre-pass for pruning, section "Temporal Data Mining").
 * Time is cut into ticks of w units, tick(t) = floor(t / w); an edge (lo, hi]
 * joins ticks whose difference is in [floor((lo + 1) / w),
 * floor((hi + w - 1) / w)].  With M_1 = the ticks holding an E_1 event and
 * M_{k+1} = the ticks holding an E_{k+1} event reachable from M_k, ub[c] is
 * the number of E_N events whose tick is in M_N: every event that ends an
 * occurrence is counted, and non-overlapped occurrences end at distinct
 * events.  With w = 1 it is exactly the number of events that end at least
 * one occurrence; a 1-node episode gets its frequency.
 *   tick          0 = choose: the smallest w with hi <= 31 w for every edge,
 *                 doubled while the stream's tables (2 bits per tick and
 *                 type, kept with the stream) would pass 256 MiB; else the
 *                 w to use, which must satisfy hi <= 31 w (FEM_ERR_INVAL).
 *   ub            uint32[n_cand], host or device (out_is_device).
 *   tick_used     optional: receives w.
 * Errors: FEM_ERR_INVAL on a malformed candidate or an alphabet above 8192
 * types, FEM_ERR_NOMEM, FEM_ERR_CUDA. */
int fem_upper_bound_coarse(fem_ctx *ctx, const fem_stream *s, const fem_cands *c, int32_t tick, uint32_t *ub,
                           int out_is_device, int32_t *tick_used);

/* Counting without any memory allocation.  The paper has no counterpart:
 * this entry point exists for callers that must not allocate device memory
 * when they ask for a count -- code running inside an allocator or a memory
 * pool callback, processes whose device memory is entirely reserved by
 * another framework, or latency-bound loops where a cudaMalloc (which can
 * synchronise the whole device) is not allowed.  It needs no context: every
 * pointer is a DEVICE pointer owned by the caller (stream types[n] and
 * times[n], candidate CSR as in fem_cands, counts[n_cand] output), and the
 * work runs on `cuda_stream` (NULL = the legacy default stream) of the
 * current device.  The call returns after the counts are written.
 *   Scratch: one 16 MiB array declared at file scope in the library, present
 *   on every GPU that has loaded it until the process exits.  Its device
 *   address is looked up on the first call made on each device, so make that
 *   first call before any stream capture.  All calls on a device share the
 *   array, so calls that overlap on the GPU (different host threads or
 *   streams) race and must be serialised by the caller.
 *   Limits: n_cand * (largest size - 1) * 2 <= 4,194,296 (for example
 *   139,800 episodes of up to 16 nodes, or 2,097,148 of 2 nodes); each
 *   episode's per-node ring holds min(32, 4,194,296 / (n_cand * (largest
 *   size - 1))) timestamps.  FEM_ERR_NOMEM if n_cand is too large or if a burst in the
 *   stream needs a longer ring than that (use fem_count_episodes then);
 *   FEM_ERR_INVAL on a malformed candidate or when offs[0] != 0.  It performs no stream
 *   validation: the stream must already satisfy fem_load_stream's rules.
 * The counts are those of fem_count_episodes (one thread per episode, the
 * serial state machine, rings in the static array). */
int fem_count_episodes_noalloc(const uint16_t *types, const int32_t *times, int64_t n, const int64_t *offs,
                               const uint16_t *ep_types, const int32_t *lo, const int32_t *hi, int64_t n_cand,
                               uint32_t *counts, void *cuda_stream);

/* ---- counting over a growing stream -------------------------------------- */

/* Exact counts kept while a recording grows by appends (section "Future
 * Work" names counting over arriving data; here the counts stay exact).
 * After any sequence of appends, fem_session_counts returns what
 * fem_count_episodes would return on the concatenation of every appended
 * chunk.  The session keeps, per episode, its count and the time of the
 * last occurrence kept by the greedy of Algorithm 1, plus the tail of the
 * stream that later occurrences can reach back into: the events at or after
 * t_last - S, S = the largest sum of upper bounds (hi) over the episodes.
 * Each append counts the tail followed by the new events by node-by-node
 * local tracking and keeps only occurrences that end at a new event.
 *   fem_session_create: candidates as in fem_cands (host or device, copied;
 *     FEM_ERR_INVAL on a malformed candidate or a type >= n_types); n_types in
 *     [1, 8192] is the alphabet of every chunk.
 *   fem_session_append: types[n] / times[n] (host, or device when
 *     ptr_is_device) under fem_load_stream's rules, checked together with the
 *     retained tail: the first new event may not precede the last appended
 *     one (FEM_ERR_UNSORTED) nor repeat a (type, time) pair of it
 *     (FEM_ERR_DUP); on those errors, and on FEM_ERR_INVAL / FEM_ERR_RANGE, the
 *     session is unchanged.  n = 0 is a no-op.  A FEM_ERR_NOMEM or
 *     FEM_ERR_CUDA during counting leaves the counts undefined: destroy the
 *     session.  The retained tail plus the chunk must stay below 2^30 events.
 *   fem_session_counts: uint32 counts[n_cand] (host or device) in input order.
 *   fem_session_info: events appended so far and events in the retained tail.
 * Calls on one session are serialised by its context. */
typedef struct fem_session fem_session;
int fem_session_create(fem_ctx *ctx, const fem_cands *c, uint32_t n_types, fem_session **out);
int fem_session_append(fem_session *s, const uint16_t *types, const int32_t *times, int64_t n,
                       int ptr_is_device);
int fem_session_counts(fem_session *s, uint32_t *counts, int out_is_device);
int fem_session_info(const fem_session *s, int64_t *events_seen, int64_t *tail_events);
void fem_session_destroy(fem_session *s);

/* ---- level-wise mining --------------------------------------------------- */

/* Level-wise frequent-episode discovery (section "Temporal Data Mining"):
 * level 1 = types whose frequency exceeds the threshold; level 2 = every
 * ordered pair of distinct frequent types with every interval bin; level
 * N >= 3 = joins of frequent (N-1)-episodes alpha, beta where alpha without
 * its first node equals beta without its last node (types and bins), giving
 * alpha extended by beta's last edge and node, distinct types only.  A
 * candidate is kept when count > threshold (strict).  Levels stop at
 * max_size or when a level keeps nothing.
 *   recs[n_recs]           recordings, each mined independently
 *   bin_lo/bin_hi[n_bins]  host arrays of interval bins (0 <= lo < hi)
 *   threshold[n_recs]      host array, per recording
 *   max_size               in [1, FEM_MAX_NODES]
 * All recordings' levels share one launch per step, and the levels are
 * chained in a captured CUDA graph (fem_tuning.level_graph); a flag raised
 * inside the graph (a capacity or ring-size overflow) makes the call redo the
 * mining level by level, with the same results.  *out receives a result (free with
 * fem_result_free) whose episodes are in canonical order: size, then the
 * interleaved sequence (E_1, lo_1, hi_1, E_2, ..., lo_{N-1}, hi_{N-1}, E_N). */
int fem_mine_levelwise(fem_ctx *ctx, const fem_stream *const *recs, int n_recs,
                       const int32_t *bin_lo, const int32_t *bin_hi, int n_bins,
                       const uint32_t *threshold, int max_size, fem_result **out);

/* Host views into a result (valid until fem_result_free).  For recording
 * `rec` and level `level` (1..max_size): *n_out episodes in CSR form
 * (offs[n+1], types, lo, hi as in fem_cands) with counts[n]. */
int fem_result_level(const fem_result *r, int rec, int level, int64_t *n_out,
                     const int64_t **offs, const uint16_t **types, const int32_t **lo,
                     const int32_t **hi, const uint32_t **counts);
int fem_result_stats(const fem_result *r, fem_stats *out);
void fem_result_free(fem_result *r);

/* ---- serving ------------------------------------------------------------- */

/* A serving loop that runs level-wise mining jobs with continuous batching:
 * a submitted job is admitted when its device memory (stream + candidate
 * buffers) fits the server's budget and a slot is free; the ready levels of
 * all admitted jobs are counted together in one launch; streams and
 * candidate sets stay on the device between levels; finished jobs release
 * their memory so waiting jobs can enter.  Runs on its own host thread and
 * context. */
typedef struct fem_server fem_server;

typedef struct {
    double submit_s;    /* host clock (seconds) when submitted */
    double admit_s;     /* when admitted to the device */
    double finish_s;    /* when the result was ready */
    int64_t n_events;
    int levels;
    int64_t candidates_counted;
    double episode_events;
} fem_job_info;

/*   hbm_budget_bytes  device memory the server may hold (0 = 80% of free)
 *   max_jobs          jobs resident on the device at once (>= 1) */
int fem_server_create(int device, size_t hbm_budget_bytes, int max_jobs, fem_server **out);
/* Submits one job; the stream arrays are host pointers copied before the
 * call returns.  bins / threshold / max_size as in fem_mine_levelwise.
 * *job_id receives the id.  FEM_ERR_NOMEM if the job can never fit. */
int fem_server_submit(fem_server *srv, const uint16_t *types, const int32_t *times, int64_t n,
                      uint32_t n_types, const int32_t *bin_lo, const int32_t *bin_hi, int n_bins,
                      uint32_t threshold, int max_size, uint64_t *job_id);
/* Waits up to timeout_ms (< 0: forever) for the job; on success *out
 * receives its result (owned by the caller) and *info its timings.
 * FEM_ERR_BUSY on timeout, FEM_ERR_NOTFOUND for an unknown or already
 * collected id. */
int fem_server_wait(fem_server *srv, uint64_t job_id, int timeout_ms, fem_result **out,
                    fem_job_info *info);
/* Stops the loop (jobs not yet finished are cancelled) and frees everything. */
void fem_server_destroy(fem_server *srv);

/* ---- misc ----------------------------------------------------------------- */
const char *fem_strerror(int status);
/* Library build identity: "fem <version> sm_103a". */
const char *fem_version(void);

#ifdef __cplusplus
}
#endif
#endif /* FEM_H */
