// fem_internal.cuh -- shared internals of libfem.so (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <map>
#include <unordered_map>
#include <mutex>
#include <string>
#include <vector>

#include "fem.h"

namespace fem {

// ---------------------------------------------------------------------------
// Constants of the counting kernels.
constexpr int kClasses = 6;              // entry classes kept per (episode, segment)
constexpr int kRecWords = 20;            // meta, thr[H], cnt[H], last[H], pad (80 B, int4-aligned)
constexpr int kMaxWarps = 8;             // compute warps per CTA
constexpr int kBitmapWords = 128;        // per-warp type filter: 4096 bits
constexpr int kStages = 4;               // shared-memory tile ring depth
constexpr int kTileAlign = 8;            // tiles start at multiples of 8 events (16 B)
constexpr int kMaxTile = 4096;           // largest tile (events)
constexpr int kPadEvents = kMaxTile + 64;  // device stream padding past n
constexpr int kMaxRingTiled = 64;        // larger rings go to the global-memory path
constexpr uint32_t kDensUnknown = 0xFFFFFFFFu;

// Device status bits (ctx->d_status).
constexpr int kStatusTimeout = 1;
constexpr int kStatusInval = 2;

// Record meta bits.
constexpr int kMetaRingOverflow = 1 << 8;
constexpr int kMetaClassOverflow = 1 << 9;
// The segment's classes catch every entry value that can reach it: some class
// threshold is at or after the segment's first event time, and every end
// selected in earlier segments lies before that time.
constexpr int kMetaClosed = 1 << 10;

// ---------------------------------------------------------------------------
struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
};

// One recording as seen by a counting launch.
struct RecInfo {
    const uint16_t *type;
    const int32_t *time;
    int64_t n;
    const int64_t *seg;   // P + 1 segment starts (device)
    int P;
    int slot_first;       // first launch slot of this recording in the bucket
    int64_t recbase;      // first record index of this recording
    const uint32_t *freq;
    const int64_t *toff;  // per-type event lists (sparse kernel only)
    const int32_t *ttime;
    // Optional (null elsewhere): for every type a and finest segment boundary
    // q, the index in a's list of its first event at or after the boundary,
    // tseg[a * tstride + q]; segment p of this launch starts at finest
    // boundary p * sstep (capped at tstride - 1, the end of the recording).
    const int32_t *tseg;
    int tstride;
    int sstep;
    // Optional (null elsewhere): the per-type time index of the stream (its
    // fem_stream fields d_tidx, tshift, tcells; tbase = the first event time).
    const int32_t *tidx;
    int tshift;
    int32_t tbase;
    int64_t tcells;
};

// Node-by-node local tracking with one warp per (episode, segment) work item
// (fem_track.cu).  Items are numbered like the records of the other counting
// kernels (recording-major, then episode slot, then segment) and taken from
// an atomic counter by a persistent grid.
constexpr int kTrackWarps = 8;           // warps per block
constexpr int kTrackMaxBlocksPerSm = 6;  // resident blocks per SM the grid asks for (40 registers)
constexpr int kTrackGroupMax = 64;       // episodes per prefix group (a new group every 64 slots)
constexpr int kTrackMinSeg = 8192;       // shortest segment (events) of a local-tracking item
constexpr int kTrackEntryRatio = 2;      // last node by entries when events > this x entries
constexpr int kTrackEntrySlots = 2;      // entries per lane of the entry-driven last node step
struct TrackArgs {
    const RecInfo *rinfo;
    int n_recs;
    int64_t rec_first;           // first record index of this launch
    int64_t n_items;             // items (records) of this launch ...
    const int64_t *d_n_items;    // ... or, if set, read from device memory
    const int64_t *offs;
    const uint16_t *ctypes;
    const int32_t *clo;
    const int32_t *chi;
    const int32_t *slot2cand;
    int relaxed;                 // every lower bound taken as 0 (upper bound)
    const uint8_t *skip;         // if set, candidates c with skip[c] != 0 are not counted
    unsigned long long *queue;   // work counter (zeroed by launch_track)
    int32_t *buf;                // per warp 4 * cap words (entry lists, ping-pong)
    int64_t cap;                 // at least the longest per-type list of every recording
    int32_t *rec;                // records, kRecWords each
    uint32_t *counts;            // if set: episodes of unsegmented recordings (P = 1) write their
                                 // count here instead of a record
    // Item order and prefix groups (ibase null: items numbered like the
    // records).  Recordings are taken in the order rorder (null: 0, 1, ...);
    // the i-th of them starts at item ibase[i]; recording r's first group is
    // gfirst[r]; group g holds slots [gstart[g], gstart[g+1]) (gstart null:
    // one slot per group).
    const int32_t *gstart;
    const int32_t *gfirst;
    const int64_t *ibase;
    const int32_t *rorder;
    int last_mode;               // last node: 0 by the shorter side, 1 by events, 2 by entries
};
// Inputs of track_groups: the slots (slot2cand, live count on the device or
// n_slots_cap), the candidate CSR, per-candidate recordings, the launch's
// RecInfo table (slot_first and P per recording, on the device), and
// scratch: gidx[n_slots_cap + 2], scan_tmp[(n_slots_cap + 2) / 1024 + 2],
// gstart[n_slots_cap + 2], gfirst[n_recs], ibase[n_recs + 1], n_items[1].
struct TrackGroupIn {
    const int32_t *slot2cand;
    const int32_t *d_n_slots;
    int64_t n_slots_cap;
    const int64_t *offs;
    const uint16_t *ctypes;
    const int32_t *clo;
    const int32_t *chi;
    const uint32_t *cand_rec;
    const RecInfo *rinfo;
    int n_recs;
    const int32_t *rorder;       // recordings in item order (null: 0, 1, ...)
    int32_t *gidx, *scan_tmp, *gstart, *gfirst;
    int64_t *ibase, *n_items;
    int32_t *gmax;               // if set: per recording, the largest group (track_group_starts)
    bool starts_ready;           // gidx / gstart already written by track_group_starts
};

// Results of the levels of level-wise mining run in a captured graph.
struct TailLevel {
    int N = 0;
    int64_t C = 0;                    // candidates of this level after the level-2 pruning
    std::vector<int64_t> coff;        // per-recording offsets of the counted candidates
    std::vector<int64_t> goff;        // per-recording offsets of the generated ones (level 2: before pruning)
    std::vector<int64_t> skipped;     // per recording: counted candidates a bound dropped before the count
    std::vector<uint16_t> types;      // frequent episodes, fixed stride N
    std::vector<int32_t> lo, hi;
    std::vector<uint32_t> rec, counts;
};
struct TailResult {
    std::vector<TailLevel> levels;
    float graph_ms = 0.f;             // device time of the graph launch
    float count_ms = 0.f;             // of which in the count kernels (+ stitch)
    double relevant = 0.0;            // relevant episode-events of the counted levels
    int64_t kernel_nodes = 0;         // kernel launches of one run of the graph
    int count_levels = 0;             // levels with a sparse counting launch
};
struct GraphTail;

// Autotuner choice for one workload signature.
struct TuneVal {
    int K;            // lanes (episodes) per CTA
    int T;            // events per shared-memory stage
    double seg_mult;  // multiplier on the segment-count heuristic
    int kernel;       // 1 tiled, 2 sparse, 3 local tracking (warp per item)
};
constexpr int kTuneTrack = 9;  // size-class field of the tuning key of local-tracking launches

}  // namespace fem

struct fem_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    size_t budget = 0;
    std::atomic<size_t> used{0};
    int n_sm = 0;
    int smem_optin = 0;
    int *d_status = nullptr;   // device status word
    int *h_status = nullptr;   // pinned mirror
    std::mutex mu;
    fem_tuning tuning{};
    fem_stats last{};
    std::map<int, fem::DevBuf> scratch;  // slot -> buffer (grown on demand)
    std::map<std::string, fem::TuneVal> tune;  // autotuner cache
    std::map<std::string, fem::GraphTail *> graphs;  // captured mining graphs
    std::map<std::string, int64_t> graph_cap;        // candidate capacity a graph key needed last time
    std::string tune_path;                     // JSON file backing the cache ("" = memory only)
    // Allocation cache: freed device blocks kept for reuse (all of a
    // context's work is ordered on its stream, so a block freed after its
    // last use there can serve the next allocation).  `live` maps a block
    // in use to its size; `cached` holds free blocks by size.
    std::mutex pool_mu;
    std::unordered_map<void *, size_t> live;
    std::multimap<size_t, void *> cached;
    size_t cached_bytes = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    void *pinned = nullptr;       // mapped host buffer of a destroyed mining graph, for the next one
    size_t pinned_bytes = 0;
};

// Coarse-tick tables of a stream for one tick width w (fem_bound.cu):
// bits[a * W + i] = ticks 32i..32i+31 (counted from tau0 = t_first / w)
// holding a type-a event; cum[a * (W + 1) + i] = index, in type a's time
// list, of its first event in word i or later.  W is a multiple of 32.
struct fem_coarse_tab {
    uint32_t *bits = nullptr;
    uint32_t *cum = nullptr;
    int64_t W = 0, tau0 = 0;
    size_t bytes = 0;
};

struct fem_stream {
    fem_ctx *ctx = nullptr;
    int64_t n = 0;
    uint32_t n_types = 0;
    uint16_t *d_type = nullptr;   // n + kPadEvents entries
    int32_t *d_time = nullptr;    // n + kPadEvents entries
    uint32_t *d_freq = nullptr;   // n_types
    size_t bytes = 0;
    int32_t t_first = 0, t_last = 0;  // first and last event time (n > 0)
    int64_t *d_toff = nullptr;    // per-type event lists (built on first use): offsets [n_types + 1]
    int32_t *d_ttime = nullptr;   // times grouped by type, ascending within a type [n]
    int64_t max_list = 0;         // longest per-type list (set with the lists)
    // Per-type time index (built on first use, after the lists): cells of
    // 2^tshift ticks from t_first; d_tidx[a * (tcells + 1) + c] is the
    // position in type a's list of its first event at or after
    // t_first + c * 2^tshift (cell tcells: past every event, the list's
    // length).  The cell width puts about one event of a type in a cell.
    int32_t *d_tidx = nullptr;
    int tshift = 0;
    int64_t tcells = 0;
    std::map<int32_t, uint32_t *> dens;  // lo -> per-type max events in a closed window of length lo
    std::map<int, int64_t *> segs;       // P -> segment boundaries (P + 1), cached
    std::map<int32_t, fem_coarse_tab> coarse;  // tick width -> coarse-tick tables
};

namespace fem {

// ---------------------------------------------------------------------------
// Error plumbing.
#define FEM_CUDA_TRY(expr)                         \
    do {                                           \
        cudaError_t _e = (expr);                   \
        if (_e != cudaSuccess) return FEM_ERR_CUDA; \
    } while (0)

#define FEM_TRY(expr)               \
    do {                            \
        int _s = (expr);            \
        if (_s != FEM_OK) return _s; \
    } while (0)

// Device memory accounted against the context budget.
int dev_alloc(fem_ctx *ctx, void **p, size_t bytes);
void dev_free(fem_ctx *ctx, void *p, size_t bytes);
// Scratch slot of at least `bytes` (contents undefined).
int scratch(fem_ctx *ctx, int slot, size_t bytes, void **p);
// Reads and clears the device status word (synchronises the stream).
int sync_status(fem_ctx *ctx);
// Copy helpers honouring host/device pointers.
int copy_in(fem_ctx *ctx, void *dst_dev, const void *src, size_t bytes, int src_is_device);
int copy_out(fem_ctx *ctx, void *dst, const void *src_dev, size_t bytes, int dst_is_device);
// Segment boundaries of a stream cut into P segments (cached per P).
int stream_segments(fem_ctx *ctx, fem_stream *s, int P, const int64_t **seg);
// Per-type event lists of a stream (built on first use, kept in the stream).
int stream_bytype(fem_ctx *ctx, fem_stream *s);
// Per-type time index of a stream (after its lists; built on first use).
int stream_tindex(fem_ctx *ctx, fem_stream *s);
// The stream's per-type lists and time index in a RecInfo.
inline void recinfo_lists(RecInfo &ri, const fem_stream *s) {
    ri.toff = s->d_toff;
    ri.ttime = s->d_ttime;
    ri.tidx = s->d_tidx;
    ri.tshift = s->tshift;
    ri.tbase = s->t_first;
    ri.tcells = s->tcells;
}
// Density table for one lo (computed on first use, cached in the stream).
int stream_density(fem_ctx *ctx, fem_stream *s, int32_t lo, uint32_t **d_dens);
// Densities for several lower bounds in one pass over the per-type lists
// (cached like stream_density; falls back to it when the lists cannot be
// built).
int stream_densities(fem_ctx *ctx, fem_stream *s, const std::vector<int32_t> &los);
// Returns every cached free block to the driver.
void pool_release(fem_ctx *ctx);
// Coarse-tick upper bound (fem_bound.cu) of device-resident candidates over
// one stream with tick width w (every edge's hi <= 31 w); ub is uint32 on
// the device.
int coarse_bound_dev(fem_ctx *ctx, fem_stream *s, int64_t n_cand, const int64_t *d_offs, const uint16_t *d_types,
                     const int32_t *d_lo, const int32_t *d_hi, int max_nodes, int32_t w, uint32_t *d_ub,
                     int64_t *launches);
// The tick width a bound uses for edges with upper bounds up to hi_max: the
// smallest w with hi_max <= 31 w, doubled while the stream's tables would
// pass `budget` bytes.
int32_t coarse_tick(const fem_stream *s, int64_t hi_max, size_t budget);
void coarse_free(fem_ctx *ctx, fem_stream *s);
// One recording's coarse-tick tables as the mining graph's bound kernel reads
// them (the stream cut into n_slices slices).
struct CoarseDesc {
    const uint32_t *bits, *cum;
    const int64_t *toff;
    const int32_t *ttime;
    int64_t W, tau0, n_chunks;
    int32_t w, slice_chunks;
};
int coarse_desc(fem_ctx *ctx, fem_stream *s, int32_t w, int n_slices, CoarseDesc *out);
// Captured-graph level step: bound the *d_n live level-N candidates (fixed
// stride, recordings crec) and set skip[c] when the bound is at most the
// recording's threshold (no candidate is skipped below min_cands).
int coarse_graph_level(cudaStream_t st, int n_sm, int N, const uint16_t *ct, const int32_t *cl, const int32_t *ch,
                       const uint32_t *crec, const int32_t *d_n, int64_t cap, const CoarseDesc *d_desc, int n_slices,
                       const uint32_t *thr, int64_t min_cands, uint32_t *ub, uint8_t *skip);

// Device buffers released together at scope exit (after the stream drains).
struct TmpDev {
    fem_ctx *ctx;
    std::vector<std::pair<void *, size_t>> held;
    explicit TmpDev(fem_ctx *c) : ctx(c) {}
    ~TmpDev() {
        if (held.empty()) return;
        cudaStreamSynchronize(ctx->stream);
        for (auto &h : held) dev_free(ctx, h.first, h.second);
    }
    template <typename T>
    int get(T **p, size_t n) {
        void *q = nullptr;
        const size_t b = std::max<size_t>(n, 1) * sizeof(T);
        FEM_TRY(dev_alloc(ctx, &q, b));
        held.push_back({q, b});
        *p = static_cast<T *>(q);
        return FEM_OK;
    }
};

// Counting continued over appended events: the recording is a retained
// tail of earlier events followed by the new ones; tail_cnt[a] = events of
// type a in the tail (their ends were counted before); d_prev[c] = time of
// candidate c's last kept end (INT32_MIN: none), updated.  Counts are added.
struct PltSession {
    const std::vector<int64_t> *tail_cnt;
    int32_t *d_prev;
};

// Counting by node-by-node local tracking (fem_plt.cu): the candidates
// `work` of the device CSR arrays; relaxed = every lower bound taken as 0;
// variant 0 = latest start per event, 1 / 2 = occurrence lists compacted with
// atomics / count-scan-write; sess (variant 0, one recording): continue the
// counts over appended events.
int count_plt(fem_ctx *ctx, const std::vector<fem_stream *> &recs, const int64_t *d_offs, const uint16_t *d_types,
              const int32_t *d_lo, const int32_t *d_hi, const uint32_t *d_rec, const std::vector<int32_t> &work,
              bool relaxed, uint32_t *d_counts, fem_stats *stats, float *kernel_ms, int variant,
              const PltSession *sess = nullptr);

// Persistent grid of the local-tracking kernel on this device (blocks), the
// bytes of its per-warp buffers, and its launch (queue reset + kernel).
int track_blocks(int n_sm);
// Numbers the items of a launch on the device (recordings in the order
// in.rorder, and with `grouped` the prefix groups) and sets the item fields
// and d_n_items of *a.
// Upper bound of every level-3 candidate from its two frequent 2-node
// sub-episodes (fem_joinbound.cu): per frequent 2-node episode a bitset of
// its valid ends and one of its valid starts; skip[c] = 1 where the
// popcount of their AND is at or below the threshold.
struct JoinBoundArgs {
    const RecInfo *ri;          // per recording: lists and time index
    int n_recs;
    const int32_t *stride;      // per recording: words per bitset
    const uint16_t *f2types;    // the frequent 2-node episodes (stride 2), their
    const int32_t *f2lo, *f2hi; // edges, recordings, per-recording offsets and
    const uint32_t *f2rec;      // (device) count
    const int64_t *f2foff;
    const int32_t *f2n;
    const int64_t *tab_off;     // (X, Y, bin) table: per-recording offsets,
    const uint32_t *nt;         // types per recording, the table itself
    int32_t *tab;
    int64_t tab_n;
    const int32_t *blo, *bhi;
    int nb;
    const uint16_t *ct;         // level-3 candidates (stride 3 / 2), recordings,
    const int32_t *cl, *ch;     // (device) count
    const uint32_t *crec;
    const int32_t *cn;
    const uint32_t *thr;        // per recording
    uint32_t *vbits, *sbits;    // bitsets (cap_words words each)
    int64_t cap_words;
    int nch;                    // chunks of 1024 events in the longest list
    int64_t *base;              // n_recs + 1: first word per recording, total
    uint8_t *skip;
    int or_skip;                // keep flags already set by another bound
    unsigned long long *skipc;  // per recording: skipped candidates
};
int join_bound_level3(cudaStream_t st, int n_sm, const JoinBoundArgs &a);

// Prefix groups of the slots (flags, scan, first slot of each group, and,
// if in.gmax is set, each recording's largest group) without the item
// numbering, which depends on the segmentation.
int track_group_starts(cudaStream_t st, int n_sm, const TrackGroupIn &in);
int track_groups(cudaStream_t st, int n_sm, const TrackGroupIn &in, bool grouped, TrackArgs *a);
size_t track_buf_bytes(int blocks, int64_t cap);
int launch_track(cudaStream_t st, int blocks, const TrackArgs &a);

// Scratch slot ids.
enum Slot : int {
    kSlotCandOffs = 1, kSlotCandTypes, kSlotCandLo, kSlotCandHi, kSlotCandRec,
    kSlotPrep, kSlotPerm, kSlotBucket, kSlotRecords, kSlotSeg, kSlotCounts,
    kSlotFallback, kSlotRings, kSlotDensTab, kSlotScanTmp, kSlotMisc, kSlotRecTab, kSlotDensArgs,
    kSlotTrack, kSlotTrackGrp,
    kSlotMine0 = 64,
};

double now_s();
// Autotuner cache: key of a counting launch (size class, ring class,
// log2 of episodes and of events, recordings) and lookup / store.
std::string tune_key(int nclass, int rclass, int64_t n_slots, int64_t n_events, int n_recs);
bool tune_lookup(fem_ctx *ctx, const std::string &key, TuneVal *out);
void tune_store(fem_ctx *ctx, const std::string &key, const TuneVal &v);

// Level-wise mining of one recording as a step-wise state machine (used by
// the serving loop): begin() runs level 1 and prepares level 2; the current
// candidates of many groups are counted together by mg_count_batch; advance()
// thresholds and prepares the next level.
struct MineGroup;
MineGroup *mg_create(fem_ctx *ctx, fem_stream *s, const std::vector<int32_t> &blo, const std::vector<int32_t> &bhi,
                     uint32_t thr, int max_size, fem_result *res);
int mg_begin(MineGroup *g);
int mg_advance(MineGroup *g);
bool mg_done(const MineGroup *g);
const fem_stats &mg_stats(const MineGroup *g);
void mg_destroy(MineGroup *g);
int mg_count_batch(fem_ctx *ctx, const std::vector<MineGroup *> &gs);
fem_result *result_new(int n_recs, int max_size);
void result_set_stats(fem_result *r, const fem_stats &s);
int launch_count_dev(cudaStream_t st, int nmax, int nodes, int R, const RecInfo *rinfo, int n_recs, const int64_t *d_n_threads,
                     int64_t cap_threads, const int64_t *offs, const uint16_t *ctypes, const int32_t *clo,
                     const int32_t *chi, const int32_t *slot2cand, const uint32_t *cand_rec, int32_t *rec,
                     const int32_t *d_n_slots, int64_t cap_slots, uint32_t *counts, int32_t *fb_list, int *fb_count,
                     const uint32_t *const *dens, const int32_t *lo_vals, int n_lo,
                     const uint8_t *skip = nullptr);
size_t sparse_smem_bytes(int nmax, int R);
// Both stitch kernels over the live slots (count on the device) of a launch
// whose records follow rinfo (per recording: slot_first, recbase, P).
// d_maxP (optional): the largest segment count of any recording (device);
// direct_p1: the counting kernel wrote the counts of unsegmented episodes.
int launch_stitch_dev(cudaStream_t st, int nsm, const RecInfo *rinfo, const int32_t *slot2cand,
                      const uint32_t *cand_rec, const int32_t *rec, const int32_t *d_n_slots, int64_t cap_slots,
                      uint32_t *counts, int32_t *fb_list, int *fb_count, const uint8_t *skip, const int *d_maxP,
                      int direct_p1);
// Segment boundaries (P + 1 entries) of a stream cut into P segments at time changes.
int launch_segments(cudaStream_t st, const int32_t *time, int64_t n, int P, int64_t *seg);
// Levels 1..max_size in one captured graph (streams resident; no host step
// between levels).  *used = false when it does not apply or a level raised a
// flag (capacity, ring or entry-class overflow): the caller then mines on the
// host-driven path.
int run_graph_mining(fem_ctx *ctx, const std::vector<fem_stream *> &recs, const std::vector<int32_t> &blo,
                     const std::vector<int32_t> &bhi, const std::vector<uint32_t> &thr,
                     const std::vector<int32_t> &lo_vals, int max_size, bool prepass, TailResult *out, bool *used);
int run_graph_tail(fem_ctx *ctx, const std::vector<fem_stream *> &recs, const std::vector<int32_t> &blo,
                   const std::vector<int32_t> &bhi, const std::vector<uint32_t> &thr, const std::vector<int32_t> &lo_vals,
                   int max_size, int64_t F2, const uint16_t *f2_types, const int32_t *f2_lo, const int32_t *f2_hi,
                   const uint32_t *f2_rec, const uint32_t *f2_counts, const std::vector<int64_t> &f2_off,
                   TailResult *out, bool *used);
void graph_cache_clear(fem_ctx *ctx);
void graph_cache_forget(fem_ctx *ctx, const fem_stream *s);
// Stream load without taking the context lock (caller holds it or owns the
// context exclusively).
int load_stream_unlocked(fem_ctx *ctx, const uint16_t *types, const int32_t *times, int64_t n, uint32_t n_types,
                         int ptr_is_device, fem_stream **out);
void stream_free_unlocked(fem_stream *s);
// Exclusive scan of m int32 in place; tmp holds ceil(m / 1024) entries.
int scan_exclusive(cudaStream_t st, int32_t *data, int64_t m, int32_t *tmp, int32_t *total, int64_t *launches);

}  // namespace fem

// ---------------------------------------------------------------------------
// Device helpers: shared-memory addresses, mbarriers, 1-D bulk TMA copies and
// bounded waits.
namespace fem {
namespace dev {

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Non-blocking test of the phase with the given parity.
__device__ __forceinline__ bool mbar_test_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for the phase of `bar` with the given parity to complete.  Gives up
// after `max_iter` polls or `max_ns` nanoseconds, whichever comes first, and
// returns false (the caller records a timeout and unwinds).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t max_iter,
                                          uint64_t max_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t i = 0; i < max_iter; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 255u) == 255u && globaltimer_ns() - t0 > max_ns) return false;
    }
    return false;
}

// A wait with a caller-chosen limit: polls > 0 gives up after that many
// non-blocking tests; polls == 0 is mbar_wait with the given defaults.
__device__ __forceinline__ bool mbar_wait_n(uint64_t *bar, uint32_t parity, uint32_t polls, uint32_t max_iter,
                                            uint64_t max_ns) {
    if (polls == 0) return mbar_wait(bar, parity, max_iter, max_ns);
    for (uint32_t i = 0; i < polls; ++i)
        if (mbar_test_wait(bar, parity)) return true;
    return false;
}

// 1-D bulk copy global -> shared, completing `bytes` on the mbarrier.
// Both addresses must be 16-byte aligned and bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst_smem, const void *src_gmem, uint32_t bytes,
                                         uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst_smem)),
        "l"(src_gmem), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

}  // namespace dev
}  // namespace fem
