// fem_count.cu -- exact counting of non-overlapped serial-episode occurrences.
//
// Formulation (section "Problem decomposition"): the count is the size of the
// largest set of non-overlapped occurrences, found by Algorithm 1 (greedy by
// end time) over occurrences.  For every end event it suffices to know the
// LATEST start of an occurrence ending there:
//     L_1(j) = t_j,   L_k(j) = max { L_{k-1}(i) : lo < t_j - t_i <= hi }.
// Along the stream, the partial occurrences of node k that are valid
// predecessors are the node's entries (t_i, L(i)); L is non-decreasing in t_i
// over entries, so a query only needs the newest entry that is already past
// its lower bound.  Entries younger than lo are kept in a small ring whose
// capacity R comes from the stream's window density (max events of the type
// in a window of length lo, plus one), so the ring never drops an entry a
// later query needs.  Algorithm 1 then selects an end event when its latest
// start is after the previous selected end.
//
// Segment-parallel counting (section "MapConcat"): the stream is split into
// segments; each (episode, segment) machine starts sum(hi) before its segment
// (any occurrence ending inside it starts no earlier), so its L values are
// exact.  Because the entry state -- the end of the last occurrence selected
// before the segment -- is unknown, the machine runs Algorithm 1 for every
// class of entry values that leads to a different first selection (the
// "multiple state machines ... anticipating all possible end states" of the
// Map step): class j covers entries in [thr_{j-1}, thr_j) and records
// (thr_j, count_j, last_j).  Classes stop being created once an occurrence
// starts inside the segment.  The stitch (the Concat step) walks segments in
// order, picks the class of the running end, adds its count and moves the
// end to its last selection.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <set>
#include <vector>

#include "fem_internal.cuh"
#include "fem_machine.cuh"

namespace fem {

constexpr int kBucketNode = 4;   // NMAX classes: 2, 4, 8, 16
constexpr int kBucketRing = 6;   // ring classes: R <= 2, 4, 8, 16, 32, 64
constexpr int kBucketN1 = kBucketNode * kBucketRing;      // 1-node episodes
constexpr int kBucketPlain = kBucketN1 + 1;               // global-memory path
constexpr int kBuckets = kBucketPlain + 1;

__host__ __device__ inline int nmax_of_class(int c) { return c == 0 ? 2 : c == 1 ? 4 : c == 2 ? 8 : 16; }
__host__ __device__ inline int ring_of_class(int c) { return 2 << c; }
// Largest register-ring capacity compiled for each NMAX class (0 = none).
__host__ __device__ inline int max_reg_ring(int nclass) { return nclass == 0 ? 8 : nclass == 1 ? 4 : nclass == 2 ? 2 : 0; }

struct WorkItem {
    int rec;
    int slot0;
    int nslots;
    int p;
};

struct TiledArgs {
    const RecInfo *rinfo;
    const WorkItem *items;
    const int64_t *offs;
    const uint16_t *ctypes;
    const int32_t *clo;
    const int32_t *chi;
    const int32_t *slot2cand;
    int R;                // ring capacity (shared-memory rings only)
    int K;
    int T;
    int relaxed;
    int small_alpha;      // every type < 128: the warp filter lives in registers
    uint32_t wait_polls;  // 0: default wait limits; n: pipeline waits give up after n tests
    int32_t *rec;         // records, kRecWords each
    int *status;
};

__device__ __forceinline__ int64_t lower_bound_time(const int32_t *tm, int64_t lo, int64_t hi, int64_t v) {
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if ((int64_t)tm[mid] < v)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

__device__ __forceinline__ int clampi(int64_t v, int lo, int hi) {
    return v < lo ? lo : (v > hi ? hi : (int)v);
}

// ---------------------------------------------------------------------------
// The tiled kernel.  One CTA = one work item: up to K episodes (one per lane
// of W = K/32 compute warps) of one recording, over one segment.  A producer
// warp streams the segment (plus halo) through a ring of kStages shared-memory
// stages with 1-D bulk copies; every compute warp reads each stage, filters
// events by its warp's union of episode types (bitmap + ballot), and offers
// the surviving events, in order, to its 32 machines.
template <int NMAX, int RR>
__global__ void __launch_bounds__(kMaxWarps * 32 + 32, ((NMAX == 2 && RR <= 4) ? 3 : NMAX == 2 ? 2 : 1))
    k_count_tiled(TiledArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int K = a.K, T = a.T;
    const int W = K >> 5;
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const WorkItem item = a.items[blockIdx.x];
    const RecInfo ri = a.rinfo[item.rec];

    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    uint64_t *empty = full + kStages;
    uint16_t *s_type = reinterpret_cast<uint16_t *>(smem + 128);
    int32_t *s_time = reinterpret_cast<int32_t *>(s_type + kStages * T);
    uint32_t *s_bm = reinterpret_cast<uint32_t *>(s_time + kStages * T);
    int32_t *s_rt = reinterpret_cast<int32_t *>(s_bm + W * kBitmapWords);
    int32_t *s_rl = s_rt + (RR == 0 ? (NMAX - 1) * a.R * K : 0);

    __shared__ unsigned long long s_maxsh;
    __shared__ long long s_range[4];  // i_begin, seg_b, seg_e, Tp
    __shared__ int s_abort;

    const bool compute = warp < W;
    const bool active = compute && tid < item.nslots;
    Machine<NMAX, RR> st;
    st.N = 0;
    st.ncls = 0;
    st.live = 0;
    st.M = INT32_MIN;
    st.open = 1;
    st.flags = 0;
#pragma unroll
    for (int k = 0; k < NMAX; ++k) st.E[k] = 0xFFFFFFFFu;
#pragma unroll
    for (int k = 0; k < NMAX - 1; ++k) {
        st.lo[k] = 0;
        st.hi[k] = 0;
    }
#pragma unroll
    for (int j = 0; j < kClasses; ++j) {
        st.cthr[j] = 0;
        st.cprev[j] = 0;
        st.ccnt[j] = 0;
    }
    int64_t sumhi = 0;
    int slot = 0;
    if (tid == 0) {
        s_maxsh = 0;
        s_abort = 0;
    }
    if (active) {
        slot = item.slot0 + tid;
        const int cand = a.slot2cand[slot];
        const int64_t o = a.offs[cand];
        const int N = (int)(a.offs[cand + 1] - o);
        const int64_t eo = o - cand;
        st.N = N;
#pragma unroll
        for (int k = 0; k < NMAX; ++k) {
            if (k < N) st.E[k] = a.ctypes[o + k];
            if (k < N - 1) {
                st.lo[k] = a.relaxed ? 0 : a.clo[eo + k];
                st.hi[k] = a.chi[eo + k];
                sumhi += st.hi[k];
            }
        }
    }
    if (compute) {
        st.rings.init(s_rt + tid, s_rl + tid, a.R, K);
        for (int i = lane; i < kBitmapWords; i += 32) s_bm[warp * kBitmapWords + i] = 0;
    }
    __syncthreads();
    if (active) {
#pragma unroll
        for (int k = 0; k < NMAX; ++k)
            if (k < st.N)
                atomicOr(&s_bm[warp * kBitmapWords + ((st.E[k] >> 5) & (kBitmapWords - 1))], 1u << (st.E[k] & 31));
        atomicMax(&s_maxsh, (unsigned long long)sumhi);
    }
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            dev::mbar_init(&full[s], 1);
            dev::mbar_init(&empty[s], W);
        }
        dev::fence_barrier_init();
    }
    __syncthreads();
    if (tid == 0) {
        const int64_t seg_b = ri.seg[item.p], seg_e = ri.seg[item.p + 1];
        int64_t ib = 0;
        int32_t Tp = 0;
        if (seg_b < seg_e) {
            Tp = ri.time[seg_b];
            const int64_t haloT = (int64_t)Tp - (int64_t)s_maxsh;
            ib = (item.p == 0) ? 0 : lower_bound_time(ri.time, 0, seg_b, haloT);
        } else {
            ib = seg_e;
        }
        s_range[0] = ib;
        s_range[1] = seg_b;
        s_range[2] = seg_e;
        s_range[3] = Tp;
    }
    __syncthreads();
    const int64_t i_begin = s_range[0], seg_b = s_range[1], seg_e = s_range[2];
    const int32_t Tp = (int32_t)s_range[3];
    const int64_t i_al = i_begin & ~(int64_t)(kTileAlign - 1);
    const int64_t ntiles = (seg_e > i_begin) ? (seg_e - i_al + T - 1) / T : 0;
    const uint32_t kMaxPoll = 1u << 30;
    const uint64_t kMaxNs = 4000000000ull;  // 4 s per wait

    if (warp == W) {
        // Producer warp: one lane issues the bulk copies.
        if (lane == 0) {
            int64_t issued = 0;
            for (int64_t k = 0; k < ntiles; ++k) {
                const int s = (int)(k % kStages);
                if (k >= kStages) {
                    if (!dev::mbar_wait_n(&empty[s], (uint32_t)(((k / kStages) - 1) & 1), a.wait_polls, kMaxPoll,
                                          kMaxNs)) {
                        atomicOr(a.status, kStatusTimeout);
                        s_abort = 1;
                        break;
                    }
                }
                if (*(volatile int *)&s_abort) break;
                const int64_t g = i_al + k * T;
                dev::mbar_arrive_expect_tx(&full[s], (uint32_t)T * 6u);
                dev::bulk_g2s(s_type + s * T, ri.type + g, (uint32_t)T * 2u, &full[s]);
                dev::bulk_g2s(s_time + s * T, ri.time + g, (uint32_t)T * 4u, &full[s]);
                issued = k + 1;
            }
            // Never leave with copies in flight into this CTA's shared memory.
            for (int64_t k = (issued > kStages ? issued - kStages : 0); k < issued; ++k)
                if (!dev::mbar_wait(&full[k % kStages], (uint32_t)((k / kStages) & 1), kMaxPoll, kMaxNs))
                    atomicOr(a.status, kStatusTimeout);
        }
        __syncwarp();
    } else {
        const uint32_t *bm = s_bm + warp * kBitmapWords;
        // the warp's filter in registers when every type is below 128
        const uint32_t w0 = bm[0], w1 = bm[1], w2 = bm[2], w3 = bm[3];
        const bool small = a.small_alpha != 0;
        for (int64_t k = 0; k < ntiles; ++k) {
            const int s = (int)(k % kStages);
            if (!dev::mbar_wait_n(&full[s], (uint32_t)((k / kStages) & 1), a.wait_polls, kMaxPoll, kMaxNs)) {
                atomicOr(a.status, kStatusTimeout);
                s_abort = 1;
                break;
            }
            const int64_t gbase = i_al + k * T;
            const int lo_c = clampi(i_begin - gbase, 0, T);
            const int hi_c = clampi(seg_e - gbase, 0, T);
            const int sg_c = clampi(seg_b - gbase, 0, T);
            const uint16_t *tt = s_type + s * T;
            const int32_t *tm = s_time + s * T;
            for (int c = lo_c & ~31; c < hi_c; c += 32) {
                const int idx = c + lane;
                const uint32_t ty = tt[idx];
                uint32_t word;
                if (small) {
                    const uint32_t q = ty >> 5;
                    word = q == 0 ? w0 : q == 1 ? w1 : q == 2 ? w2 : q == 3 ? w3 : 0u;
                } else {
                    word = bm[(ty >> 5) & (kBitmapWords - 1)];
                }
                const bool rel = ((word >> (ty & 31)) & 1u) && idx >= lo_c && idx < hi_c;
                uint32_t m = __ballot_sync(0xFFFFFFFFu, rel);
                while (m) {
                    const int b = __ffs(m) - 1;
                    m &= m - 1;
                    const uint32_t ety = __shfl_sync(0xFFFFFFFFu, ty, b);
                    const int32_t et = tm[c + b];
                    st.step(ety, et, (c + b) >= sg_c, Tp);
                }
            }
            __syncwarp();
            if (lane == 0) dev::mbar_arrive(&empty[s]);
        }
        if (active) {
            st.finish();
            int4 *r = reinterpret_cast<int4 *>(a.rec + (ri.recbase + (int64_t)(slot - ri.slot_first) * ri.P + item.p) *
                                                          kRecWords);
            int32_t w[kRecWords];
            w[0] = st.ncls | st.flags | (st.open ? 0 : kMetaClosed);
#pragma unroll
            for (int j = 0; j < kClasses; ++j) {
                w[1 + j] = st.cthr[j];
                w[1 + kClasses + j] = (int32_t)st.ccnt[j];
                w[1 + 2 * kClasses + j] = st.cprev[j];
            }
#pragma unroll
            for (int j = 1 + 3 * kClasses; j < kRecWords; ++j) w[j] = 0;
#pragma unroll
            for (int q = 0; q < kRecWords / 4; ++q) r[q] = make_int4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
        }
    }
}

// Concat step.  A segment's record is a map from the entry value x (end of
// the last occurrence selected before the segment, minus infinity before the
// first) to (occurrences added, exit value): the first class j with
// x < thr[j] applies, and x passes through unchanged (nothing added) when no
// class does.  Such maps compose into maps of the same form, so per episode
// (one warp) each lane composes the records of a contiguous run of segments
// into one map; a walk over the 32 lane maps then gives the count.  A lane's
// map keeps up to kChunkClasses classes; if one overflows, the warp walks all
// records in order instead (same result).
constexpr int kStitchWarps = 4;
constexpr int kChunkClasses = 8;

// Entry values are times (>= 0) or minus infinity, held as INT32_MIN.
__device__ __forceinline__ void stitch_apply(const int32_t (&r)[kRecWords], int ncls, int ncw, int32_t &x,
                                             uint32_t &total) {
    bool hit = false;
    int32_t nx = x;
    uint32_t add = 0;
#pragma unroll
    for (int j = 0; j < kClasses; ++j) {
        if (j >= ncw) break;  // warp-uniform bound
        if (!hit && j < ncls && x < r[1 + j]) {
            add = (uint32_t)r[1 + kClasses + j];
            nx = r[1 + 2 * kClasses + j];
            hit = true;
        }
    }
    x = nx;
    total += add;
}

// One lane's map: the records of segments [pa, pb) composed in order.
struct LaneMap {
    int32_t thr[kChunkClasses], last[kChunkClasses];
    uint32_t cnt[kChunkClasses];
    int m;          // classes
    int32_t top;    // last threshold (INT32_MIN without classes)
    bool through;   // entry values above top pass through unchanged
    bool bad;       // a record is flagged (ring or class overflow)
    bool ovf;       // more than kChunkClasses classes
};

// Composes this lane's records [pa, pb); every lane of the warp calls it with
// the same `per` (its trip count), so the warp-wide bounds below are safe.
__device__ __forceinline__ void stitch_compose(const int4 *__restrict__ base, int pa, int pb, int per, LaneMap &f) {
#pragma unroll
    for (int j = 0; j < kChunkClasses; ++j) f.thr[j] = f.last[j] = 0, f.cnt[j] = 0;
    f.m = 0;
    f.bad = f.ovf = false;
    f.top = INT32_MIN;
    f.through = true;
    // records are loaded one ahead of the one being composed
    int4 nx[kRecWords / 4];
#pragma unroll
    for (int q = 0; q < kRecWords / 4; ++q)
        nx[q] = pa < pb ? base[(int64_t)pa * (kRecWords / 4) + q] : make_int4(0, 0, 0, 0);
    for (int i = 0; i < per; ++i) {
        const int p = pa + i;
        int32_t r[kRecWords];
#pragma unroll
        for (int q = 0; q < kRecWords / 4; ++q) {
            const int4 v = nx[q];
            r[4 * q] = v.x, r[4 * q + 1] = v.y, r[4 * q + 2] = v.z, r[4 * q + 3] = v.w;
        }
        if (p + 1 < pb) {
#pragma unroll
            for (int q = 0; q < kRecWords / 4; ++q) nx[q] = base[(int64_t)(p + 1) * (kRecWords / 4) + q];
        }
        const int meta = p < pb ? r[0] : 0;
        if (meta & (kMetaRingOverflow | kMetaClassOverflow)) f.bad = true;
        const int ncls = meta & 0xFF;
        const int ncw = __reduce_max_sync(0xFFFFFFFFu, ncls);
        if (ncw == 0) continue;
        const int fmw = __reduce_max_sync(0xFFFFFFFFu, f.m);
        // classes already in the map have a known exit value: run it on
#pragma unroll
        for (int j = 0; j < kChunkClasses; ++j) {
            if (j >= fmw) break;
            if (j < f.m && ncls > 0) {
                int32_t x = f.last[j];
                uint32_t t = f.cnt[j];
                stitch_apply(r, ncls, ncw, x, t);
                f.last[j] = x;
                f.cnt[j] = t;
            }
        }
        if (!f.through || ncls == 0) continue;
        // entry values still passing through meet this segment's classes
        // above the map's last threshold
        const int32_t floor_thr = f.top;
#pragma unroll
        for (int c = 0; c < kClasses; ++c) {
            if (c >= ncls) break;
            if (r[1 + c] > floor_thr) {
                if (f.m == kChunkClasses) {
                    f.ovf = true;
                } else {
#pragma unroll
                    for (int j = 0; j < kChunkClasses; ++j)
                        if (j == f.m) {
                            f.thr[j] = r[1 + c];
                            f.cnt[j] = (uint32_t)r[1 + kClasses + c];
                            f.last[j] = r[1 + 2 * kClasses + c];
                        }
                    ++f.m;
                    f.top = r[1 + c];
                }
            }
        }
        if (meta & kMetaClosed) f.through = false;
    }
}

// x -> the lane map's (x', total += added): the first class with x < thr.
__device__ __forceinline__ void lanemap_apply(const LaneMap &f, int32_t &x, uint32_t &total) {
    bool hit = false;
#pragma unroll
    for (int j = 0; j < kChunkClasses; ++j)
        if (!hit && j < f.m && x < f.thr[j]) {
            total += f.cnt[j];
            x = f.last[j];
            hit = true;
        }
}

// a := a then b (the runs of a and b are adjacent, a's first).  a's classes
// have known exits, which b maps on; entry values still passing through a
// meet b's classes above a's last threshold.
__device__ __forceinline__ void lanemap_then(LaneMap &a, const LaneMap &b) {
#pragma unroll
    for (int j = 0; j < kChunkClasses; ++j)
        if (j < a.m) {
            int32_t x = a.last[j];
            uint32_t t = a.cnt[j];
            lanemap_apply(b, x, t);
            a.last[j] = x;
            a.cnt[j] = t;
        }
    if (a.through) {
#pragma unroll
        for (int c = 0; c < kChunkClasses; ++c)
            if (c < b.m && b.thr[c] > a.top) {
                if (a.m == kChunkClasses) {
                    a.ovf = true;
                } else {
#pragma unroll
                    for (int j = 0; j < kChunkClasses; ++j)
                        if (j == a.m) {
                            a.thr[j] = b.thr[c];
                            a.cnt[j] = b.cnt[c];
                            a.last[j] = b.last[c];
                        }
                    ++a.m;
                    a.top = b.thr[c];
                }
            }
        a.through = b.through;
    }
    a.bad = a.bad || b.bad;
    a.ovf = a.ovf || b.ovf;
}

// Tree composition of the warp's 32 lane maps (lane order); lane 0 ends with
// the map of the warp's whole run.
__device__ __forceinline__ void warp_compose(LaneMap &f, int lane) {
#pragma unroll 1
    for (int d = 1; d < 32; d <<= 1) {
        LaneMap o;
#pragma unroll
        for (int j = 0; j < kChunkClasses; ++j) {
            o.thr[j] = __shfl_down_sync(0xFFFFFFFFu, f.thr[j], d);
            o.last[j] = __shfl_down_sync(0xFFFFFFFFu, f.last[j], d);
            o.cnt[j] = __shfl_down_sync(0xFFFFFFFFu, f.cnt[j], d);
        }
        o.m = __shfl_down_sync(0xFFFFFFFFu, f.m, d);
        o.top = __shfl_down_sync(0xFFFFFFFFu, f.top, d);
        o.through = __shfl_down_sync(0xFFFFFFFFu, (int)f.through, d) != 0;
        o.bad = __shfl_down_sync(0xFFFFFFFFu, (int)f.bad, d) != 0;
        o.ovf = __shfl_down_sync(0xFFFFFFFFu, (int)f.ovf, d) != 0;
        if ((lane & (2 * d - 1)) == 0 && lane + d < 32) lanemap_then(f, o);
    }
}

// Every record of one episode in order (used when a lane map overflowed).
__device__ void stitch_serial(const int4 *__restrict__ base, int P, int32_t &x, uint32_t &total) {
    for (int p = 0; p < P; ++p) {
        int32_t r[kRecWords];
#pragma unroll
        for (int q = 0; q < kRecWords / 4; ++q) {
            const int4 v = base[(int64_t)p * (kRecWords / 4) + q];
            r[4 * q] = v.x, r[4 * q + 1] = v.y, r[4 * q + 2] = v.z, r[4 * q + 3] = v.w;
        }
        stitch_apply(r, r[0] & 0xFF, kClasses, x, total);
    }
}

// One warp per episode, for episodes with at most max_P segments (the others
// are left to k_stitch_block).
__global__ void __launch_bounds__(kStitchWarps * 32)
    k_stitch(const int32_t *__restrict__ rec, const RecInfo *__restrict__ rinfo,
             const int32_t *__restrict__ slot2cand, const uint32_t *__restrict__ cand_rec, int slot_begin,
             int n_slots, uint32_t *__restrict__ counts, int32_t *fb_list, int *fb_count,
             const int32_t *d_n_slots = nullptr, int max_P = INT32_MAX, const uint8_t *skip = nullptr,
             const int *d_maxP = nullptr, int direct_p1 = 0) {
    const int lane = threadIdx.x & 31;
    // direct_p1: the counting kernel wrote the counts of unsegmented
    // episodes itself (no records); nothing to do when no recording is cut
    if (direct_p1 && d_maxP && *d_maxP <= 1) return;
    const int n_live = d_n_slots ? *d_n_slots : n_slots;
    for (int wi = blockIdx.x * kStitchWarps + (threadIdx.x >> 5); wi < n_live; wi += gridDim.x * kStitchWarps) {
        const int slot = slot_begin + wi;
        const int cand = slot2cand[slot];
        const int r_id = cand_rec ? (int)cand_rec[cand] : 0;
        const RecInfo ri = rinfo[r_id];
        const int P = ri.P;
        if (P > max_P || (direct_p1 && P == 1)) continue;
        if (skip && skip[cand]) {  // pruned by a bound: count 0
            if (lane == 0) counts[cand] = 0;
            continue;
        }
        const int4 *base = reinterpret_cast<const int4 *>(
            rec + (ri.recbase + (int64_t)(slot - ri.slot_first) * P) * kRecWords);
        const int per = (P + 31) >> 5;
        const int pa = min(P, lane * per), pb = min(P, pa + per);
        LaneMap f;
        stitch_compose(base, pa, pb, per, f);
        warp_compose(f, lane);
        const bool any_bad = __shfl_sync(0xFFFFFFFFu, (int)f.bad, 0) != 0;
        const bool any_ovf = __shfl_sync(0xFFFFFFFFu, (int)f.ovf, 0) != 0;
        int32_t x = INT32_MIN;  // before the first occurrence
        uint32_t total = 0;
        if (!any_bad && !any_ovf)
            lanemap_apply(f, x, total);  // lane 0's map of the whole episode
        else if (!any_bad)
            stitch_serial(base, P, x, total);
        if (lane == 0) {
            if (any_bad) {
                const int q = atomicAdd(fb_count, 1);
                fb_list[q] = cand;
            } else {
                counts[cand] = total;
            }
        }
    }
}

// One block per episode, for episodes with more than min_P segments: 512
// lanes compose their runs, each warp composes its lanes' maps, and the
// sixteen warp maps (shared memory) are applied in order.
constexpr int kStitchBlock = 512;
constexpr int kStitchSplit = 256;  // episodes with more segments take a block

__global__ void __launch_bounds__(kStitchBlock, 1)
    k_stitch_block(const int32_t *__restrict__ rec, const RecInfo *__restrict__ rinfo,
                   const int32_t *__restrict__ slot2cand, const uint32_t *__restrict__ cand_rec, int slot_begin,
                   int n_slots, uint32_t *__restrict__ counts, int32_t *fb_list, int *fb_count,
                   const int32_t *d_n_slots, int min_P, const uint8_t *skip = nullptr, const int *d_maxP = nullptr) {
    constexpr int W = kStitchBlock / 32;
    __shared__ int32_t s_thr[W][kChunkClasses], s_last[W][kChunkClasses];
    __shared__ uint32_t s_cnt[W][kChunkClasses];
    __shared__ int s_m[W], s_flag[W];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (d_maxP && *d_maxP <= min_P) return;  // no recording is cut into that many segments
    const int n_live = d_n_slots ? *d_n_slots : n_slots;
    for (int wi = blockIdx.x; wi < n_live; wi += gridDim.x) {
        const int slot = slot_begin + wi;
        const int cand = slot2cand[slot];
        const int r_id = cand_rec ? (int)cand_rec[cand] : 0;
        const RecInfo ri = rinfo[r_id];
        const int P = ri.P;
        if (P <= min_P) continue;  // block-uniform
        if (skip && skip[cand]) {  // pruned by a bound: count 0 (block-uniform)
            if (tid == 0) counts[cand] = 0;
            continue;
        }
        const int4 *base = reinterpret_cast<const int4 *>(
            rec + (ri.recbase + (int64_t)(slot - ri.slot_first) * P) * kRecWords);
        const int per = (P + kStitchBlock - 1) / kStitchBlock;
        const int pa = min(P, tid * per), pb = min(P, pa + per);
        LaneMap f;
        stitch_compose(base, pa, pb, per, f);
        warp_compose(f, lane);
        if (lane == 0) {
#pragma unroll
            for (int j = 0; j < kChunkClasses; ++j) {
                s_thr[warp][j] = f.thr[j];
                s_last[warp][j] = f.last[j];
                s_cnt[warp][j] = f.cnt[j];
            }
            s_m[warp] = f.m;
            s_flag[warp] = (f.bad ? 1 : 0) | (f.ovf ? 2 : 0);
        }
        __syncthreads();
        if (tid == 0) {
            int fl = 0;
            for (int w = 0; w < W; ++w) fl |= s_flag[w];
            int32_t x = INT32_MIN;  // before the first occurrence
            uint32_t total = 0;
            if (fl == 0) {
                for (int w = 0; w < W; ++w) {
                    bool hit = false;
                    for (int j = 0; j < s_m[w] && !hit; ++j)
                        if (x < s_thr[w][j]) {
                            total += s_cnt[w][j];
                            x = s_last[w][j];
                            hit = true;
                        }
                }
            } else if (!(fl & 1)) {
                stitch_serial(base, P, x, total);
            }
            if (fl & 1) {
                const int q = atomicAdd(fb_count, 1);
                fb_list[q] = cand;
            } else {
                counts[cand] = total;
            }
        }
        __syncthreads();  // the maps are rewritten for the next episode
    }
}

// 1-node episodes: the count is the type's frequency (distinct times).
__global__ void k_count_n1(const int32_t *__restrict__ slot2cand, int slot_begin, int n_slots,
                           const int64_t *__restrict__ offs, const uint16_t *__restrict__ ctypes,
                           const uint32_t *__restrict__ cand_rec, const RecInfo *__restrict__ rinfo,
                           uint32_t *__restrict__ counts) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_slots) return;
    const int cand = slot2cand[slot_begin + i];
    const int r_id = cand_rec ? (int)cand_rec[cand] : 0;
    counts[cand] = rinfo[r_id].freq[ctypes[offs[cand]]];
}

// ---------------------------------------------------------------------------
// Plain comparison path: one thread per episode walks the whole stream from
// global memory running the serial state machine ("Episode Counting
// Algorithm", reset on completion), with each node's list kept as a ring of
// R timestamps in global memory.
__global__ void k_count_plain(const RecInfo *__restrict__ rinfo, const int32_t *__restrict__ slot2cand,
                              const uint32_t *__restrict__ cand_rec, int slot_begin, int n_slots,
                              const int64_t *__restrict__ offs, const uint16_t *__restrict__ ctypes,
                              const int32_t *__restrict__ clo, const int32_t *__restrict__ chi, int R,
                              int32_t *__restrict__ rings, uint32_t *__restrict__ counts, int *status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_slots) return;
    const int cand = slot2cand[slot_begin + i];
    const int r_id = cand_rec ? (int)cand_rec[cand] : 0;
    const RecInfo ri = rinfo[r_id];
    const int64_t o = offs[cand];
    const int N = (int)(offs[cand + 1] - o);
    const int64_t eo = o - cand;
    uint16_t E[FEM_MAX_NODES];
    int32_t lo[FEM_MAX_NODES], hi[FEM_MAX_NODES];
    int head[FEM_MAX_NODES];
    for (int k = 0; k < N; ++k) {
        E[k] = ctypes[o + k];
        head[k] = 0;
        if (k < N - 1) {
            lo[k] = clo[eo + k];
            hi[k] = chi[eo + k];
        }
    }
    // ring (k, r) of this thread at rings[((k * R) + r) * n_slots + i]
    const int64_t stride = n_slots;
    for (int k = 0; k < N - 1; ++k)
        for (int r = 0; r < R; ++r) rings[((int64_t)k * R + r) * stride + i] = INT32_MIN;
    int64_t prev_end = INT64_MIN;
    uint32_t count = 0;
    int ovf = 0;
    for (int64_t j = 0; j < ri.n; ++j) {
        const uint16_t ty = ri.type[j];
        const int32_t t = ri.time[j];
        for (int k = N - 1; k >= 0; --k) {
            if (E[k] != ty) continue;
            bool ok;
            if (k == 0) {
                ok = (int64_t)t > prev_end;
            } else {
                ok = false;
                int idx = head[k - 1];
                for (int q = 0; q < R; ++q) {
                    idx = (idx == 0) ? R - 1 : idx - 1;
                    const int32_t tp = rings[((int64_t)(k - 1) * R + idx) * stride + i];
                    if (tp < t - lo[k - 1]) {
                        ok = tp >= t - hi[k - 1];
                        break;
                    }
                }
            }
            if (!ok) continue;
            if (k == N - 1) {
                count++;
                prev_end = t;
                for (int q = 0; q < N - 1; ++q) {
                    head[q] = 0;
                    for (int r = 0; r < R; ++r) rings[((int64_t)q * R + r) * stride + i] = INT32_MIN;
                }
                break;
            }
            const int h = head[k];
            const int h2 = (h + 1 == R) ? 0 : h + 1;
            int32_t *slotp = &rings[((int64_t)k * R + h) * stride + i];
            const int32_t old = *slotp;
            const int32_t old2 = rings[((int64_t)k * R + h2) * stride + i];
            if (old != INT32_MIN && old >= t - hi[k] && old2 >= t - lo[k]) ovf = 1;
            *slotp = t;
            head[k] = h2;
        }
    }
    counts[cand] = count;
    if (ovf) atomicOr(status, kStatusInval);
}

// ---------------------------------------------------------------------------
// Candidate preparation: validation, ring size, bucket key.
struct PrepArgs {
    int64_t n_cand;
    const int64_t *offs;
    const uint16_t *ctypes;
    const int32_t *clo;
    const int32_t *chi;
    const uint32_t *cand_rec;
    const int32_t *subset;     // optional list of candidates to process
    const RecInfo *rinfo;
    const uint32_t *n_types;   // per recording
    const int32_t *lo_vals;    // sorted distinct lo values
    int n_lo;
    const uint32_t *const *dens;  // [rec * n_lo + j]
    int n_recs;
    int mode;                  // 0 exact, 1 plain, 2 relaxed (upper bound)
    int force_plain_ring;
    int track;                 // every multi-node episode in bucket 0 (local-tracking kernel)
    int32_t *key;              // out: bucket * n_recs + rec
    int32_t *ring;             // out: R per candidate
    int *bucket_maxR;          // out: per bucket max R
    unsigned long long *relevant;  // out: sum over candidates of sum_k freq(E_k)
    int *status;
};

__device__ __forceinline__ uint32_t dens_lookup(const PrepArgs &a, int rec, int32_t lo, uint16_t ty) {
    int lo_i = 0, hi_i = a.n_lo;
    while (lo_i < hi_i) {
        const int mid = (lo_i + hi_i) >> 1;
        if (a.lo_vals[mid] < lo)
            lo_i = mid + 1;
        else
            hi_i = mid;
    }
    if (lo_i >= a.n_lo || a.lo_vals[lo_i] != lo) return kDensUnknown;
    return a.dens[rec * a.n_lo + lo_i][ty];
}

__global__ void k_prep(PrepArgs a) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= a.n_cand) return;
    const int64_t c = a.subset ? a.subset[i] : i;
    const int rec = a.cand_rec ? (int)a.cand_rec[c] : 0;
    const int64_t o = a.offs[c];
    const int64_t N = a.offs[c + 1] - o;
    const int64_t eo = o - c;
    bool bad = (rec < 0 || rec >= a.n_recs || N < 1 || N > FEM_MAX_NODES);
    int R = 2;
    int64_t slab = 0;  // sum over nodes of the ring sizes
    int64_t sumhi = 0;
    unsigned long long relv = 0;
    if (!bad) {
        const uint32_t nt = a.n_types[rec];
        const uint32_t *freq = a.rinfo[rec].freq;
        for (int k = 0; k < N && !bad; ++k) {
            const uint16_t ty = a.ctypes[o + k];
            if (ty >= nt) {
                bad = true;
                break;
            }
            relv += freq[ty];
            if (k < N - 1) {
                const int32_t l = a.clo[eo + k], h = a.chi[eo + k];
                if (l < 0 || l >= h) {
                    bad = true;
                    break;
                }
                sumhi += h;
                const int32_t lq = (a.mode == 2) ? 0 : l;
                uint32_t d = dens_lookup(a, rec, lq, ty);
                if (d == kDensUnknown || d == 0) d = freq[ty] > 0 ? freq[ty] : 1;
                const uint32_t need = d >= 0x7FFFFFFEu ? 0x7FFFFFFFu : d + 1;
                if ((int)need > R) R = (int)need;
                slab += need < 2 ? 2 : need;
            }
        }
    }
    if (bad) {
        atomicOr(a.status, kStatusInval);
        a.key[i] = 0;
        a.ring[i] = 2;
        return;
    }
    int bucket;
    if (a.mode == 1) {
        bucket = kBucketPlain;
    } else if (N == 1) {
        bucket = kBucketN1;
    } else if (a.track) {
        bucket = 0;  // one launch for every size and ring: the kernel keeps no rings
    } else if (R > kMaxRingTiled || a.force_plain_ring) {
        bucket = kBucketPlain;
    } else {
        const int nc = N <= 2 ? 0 : N <= 4 ? 1 : N <= 8 ? 2 : 3;
        const int rc = R <= 2 ? 0 : R <= 4 ? 1 : R <= 8 ? 2 : R <= 16 ? 3 : R <= 32 ? 4 : 5;
        bucket = nc * kBucketRing + rc;
    }
    a.key[i] = bucket * a.n_recs + rec;
    a.ring[i] = R;
    atomicMax(&a.bucket_maxR[bucket], R);
    atomicMax(&a.bucket_maxR[kBuckets + bucket], (int)N);
    atomicMax(&a.bucket_maxR[2 * kBuckets + bucket], (int)(sumhi > INT32_MAX ? INT32_MAX : sumhi));
    atomicMax(&a.bucket_maxR[3 * kBuckets + bucket], (int)(slab > INT32_MAX ? INT32_MAX : slab));
    atomicAdd(a.relevant, relv);
}

// Stable partition by key: blocks of kPartBlock elements.  k_part_count
// writes blk[k * nblk + b] = elements of block b with key k; after an
// exclusive scan of that key-major table, blk[k * nblk + b] is where block b's
// first key-k element goes, and k_part_scatter (one warp per block, walking
// its elements in order) assigns stable positions.
constexpr int kPartBlock = 4096;

__global__ void k_part_count(const int32_t *__restrict__ key, int64_t n, int n_keys, int64_t nblk,
                             int32_t *__restrict__ blk) {
    extern __shared__ int32_t cnt[];
    for (int k = threadIdx.x; k < n_keys; k += blockDim.x) cnt[k] = 0;
    __syncthreads();
    const int64_t b0 = blockIdx.x * (int64_t)kPartBlock;
    const int64_t b1 = (n < b0 + kPartBlock) ? n : b0 + kPartBlock;
    for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) atomicAdd(&cnt[key[i]], 1);
    __syncthreads();
    for (int k = threadIdx.x; k < n_keys; k += blockDim.x) blk[(int64_t)k * nblk + blockIdx.x] = cnt[k];
}

__global__ void k_part_scatter(const int32_t *__restrict__ key, int64_t n, int n_keys, int64_t nblk,
                               const int32_t *__restrict__ blk, const int32_t *__restrict__ subset,
                               int32_t *__restrict__ out, int32_t *__restrict__ out_key) {
    extern __shared__ int32_t run[];
    const int lane = threadIdx.x;
    for (int k = lane; k < n_keys; k += 32) run[k] = blk[(int64_t)k * nblk + blockIdx.x];
    __syncwarp();
    const int64_t b0 = blockIdx.x * (int64_t)kPartBlock;
    const int64_t b1 = (n < b0 + kPartBlock) ? n : b0 + kPartBlock;
    for (int64_t base = b0; base < b1; base += 32) {
        const int64_t i = base + lane;
        const int k = i < b1 ? key[i] : -1;
        const uint32_t peers = __match_any_sync(0xFFFFFFFFu, k);
        const int rank = __popc(peers & ((1u << lane) - 1));
        int32_t pos = 0;
        if (k >= 0) pos = run[k] + rank;
        __syncwarp();
        if (k >= 0) {
            out[pos] = subset ? subset[i] : (int32_t)i;
            if (out_key) out_key[pos] = k;
            if (rank == 0) run[k] += __popc(peers);
        }
        __syncwarp();
    }
}

__global__ void k_gather_keyoff(const int32_t *__restrict__ blk, int n_keys, int64_t nblk,
                                int32_t *__restrict__ out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n_keys) out[k] = blk[(int64_t)k * nblk];
}

// Exclusive scan of m int32 entries in place (multi-block: per-block sums,
// a single-block scan of the sums, then add-back).
__device__ __forceinline__ int32_t block_incl_scan(int32_t v, int32_t *wsum) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int32_t x = v;
    for (int d = 1; d < 32; d <<= 1) {
        const int32_t y = __shfl_up_sync(0xFFFFFFFFu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        int32_t s = lane < nw ? wsum[lane] : 0;
        for (int d = 1; d < 32; d <<= 1) {
            const int32_t y = __shfl_up_sync(0xFFFFFFFFu, s, d);
            if (lane >= d) s += y;
        }
        if (lane < nw) wsum[lane] = s;
    }
    __syncthreads();
    const int32_t r = x + (w > 0 ? wsum[w - 1] : 0);
    __syncthreads();
    return r;
}

constexpr int kScanBlock = 1024;

__global__ void k_scan_blocks(int32_t *data, int64_t m, int32_t *bsum) {
    __shared__ int32_t wsum[32];
    const int64_t i = blockIdx.x * (int64_t)kScanBlock + threadIdx.x;
    const int32_t v = i < m ? data[i] : 0;
    const int32_t incl = block_incl_scan(v, wsum);
    if (i < m) data[i] = incl - v;
    if (threadIdx.x == kScanBlock - 1) bsum[blockIdx.x] = incl;
}

__global__ void k_scan_single(int32_t *data, int64_t m, int32_t *total) {
    __shared__ int32_t wsum[32];
    __shared__ int32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < m; base += blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const int32_t v = i < m ? data[i] : 0;
        const int32_t incl = block_incl_scan(v, wsum) + carry;
        if (i < m) data[i] = incl - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = incl;
        __syncthreads();
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void k_scan_add(int32_t *data, int64_t m, const int32_t *bsum) {
    const int64_t i = blockIdx.x * (int64_t)kScanBlock + threadIdx.x;
    if (i < m) data[i] += bsum[blockIdx.x];
}

// tmp must hold ceil(m / kScanBlock) int32.
int scan_exclusive(cudaStream_t st, int32_t *data, int64_t m, int32_t *tmp, int32_t *total, int64_t *launches) {
    if (m <= 0) return FEM_OK;
    const int64_t nb = (m + kScanBlock - 1) / kScanBlock;
    if (nb == 1) {
        k_scan_single<<<1, kScanBlock, 0, st>>>(data, m, total);
        if (launches) *launches += 1;
    } else {
        k_scan_blocks<<<(unsigned)nb, kScanBlock, 0, st>>>(data, m, tmp);
        k_scan_single<<<1, kScanBlock, 0, st>>>(tmp, nb, total);
        k_scan_add<<<(unsigned)nb, kScanBlock, 0, st>>>(data, m, tmp);
        if (launches) *launches += 3;
    }
    FEM_CUDA_TRY(cudaGetLastError());
    return FEM_OK;
}

// Segment boundaries: boundary p sits near p*n/P, at the largest gap
// between consecutive event times within +-w events of it (a quiet spot, so
// few occurrences span the boundary and few entry classes are needed); a
// boundary always falls where the time changes.
__global__ void k_segments(const int32_t *__restrict__ tm, int64_t n, int P, int64_t *__restrict__ seg) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > P) return;
    int64_t b;
    if (p == 0) {
        b = 0;
    } else if (p == P) {
        b = n;
    } else {
        const int64_t nom = (int64_t)((__int128)n * p / P);
        const int64_t seg_len = n / P;
        const int64_t w = seg_len / 4 < 4096 ? seg_len / 4 : 4096;
        const int64_t lo = nom - w > 1 ? nom - w : 1;
        const int64_t hi = nom + w < n - 1 ? nom + w : n - 1;
        b = nom;
        int64_t best = -1;
        for (int64_t i = lo; i <= hi; ++i) {
            const int64_t gap = (int64_t)tm[i] - tm[i - 1];
            if (gap > best) {
                best = gap;
                b = i;
            }
        }
        if (best <= 0)
            while (b < n && b > 0 && tm[b] == tm[b - 1]) ++b;
    }
    seg[p] = b;
}

int stream_segments(fem_ctx *ctx, fem_stream *s, int P, const int64_t **seg) {
    auto it = s->segs.find(P);
    if (it != s->segs.end()) {
        *seg = it->second;
        return FEM_OK;
    }
    if (s->segs.size() >= 64) {  // bound the cache
        cudaStreamSynchronize(ctx->stream);
        for (auto &kv : s->segs) dev_free(ctx, kv.second, sizeof(int64_t) * (kv.first + 1));
        s->segs.clear();
    }
    void *p = nullptr;
    FEM_TRY(dev_alloc(ctx, &p, sizeof(int64_t) * (P + 1)));
    k_segments<<<(P + 1 + 127) / 128, 128, 0, ctx->stream>>>(s->d_time, s->n, P, static_cast<int64_t *>(p));
    FEM_CUDA_TRY(cudaGetLastError());
    s->segs[P] = static_cast<int64_t *>(p);
    *seg = static_cast<int64_t *>(p);
    return FEM_OK;
}

int launch_segments(cudaStream_t st, const int32_t *time, int64_t n, int P, int64_t *seg) {
    k_segments<<<(P + 1 + 127) / 128, 128, 0, st>>>(time, n, P, seg);
    FEM_CUDA_TRY(cudaGetLastError());
    return FEM_OK;
}

// ---------------------------------------------------------------------------
// Host driver.
// ---------------------------------------------------------------------------
// Sparse counting kernel: one thread per (episode, segment).  Instead of
// reading every event of the segment, the thread merges, in time order, the
// per-type event lists of its episode's node types (the per-type index lists
// of section "Parallel Local Tracking"), so it touches only the events its
// episode can use.  The machine (rings, Algorithm 1 per entry class, halo)
// and the records are those of the tiled kernel; k_stitch reads both.
struct SparseArgs {
    const RecInfo *rinfo;
    int n_recs;
    int64_t rec_first;    // first record index of this plan
    int64_t n_threads;    // records of this plan = sum over recordings of c_r * P_r
    const int64_t *d_n_threads;  // if set, the thread count is read from device memory
    const int64_t *offs;
    const uint16_t *ctypes;
    const int32_t *clo;
    const int32_t *chi;
    const int32_t *slot2cand;
    int relaxed;
    int R;                // ring capacity (shared-memory rings, uniform mode)
    int32_t *rec;
    // per-node ring sizes (shared-memory rings, sized mode): window density
    // tables [rec * n_lo + j] for the distinct lower bounds lo_vals[j]; each
    // thread's rings share a slab of `slab` entries
    const uint32_t *const *dens;
    const int32_t *lo_vals;
    int n_lo;
    int slab;
    const uint8_t *skip;  // if set, candidates c with skip[c] != 0 are not counted
};

// RR > 0: register rings.  RR == 0: shared-memory rings in 64-thread blocks,
// entry e of thread i's slab at e*64 + i -- either R entries per node
// (uniform mode) or, when density tables are given, each node's ring sized
// to its own window density + 1 inside a slab of a.slab entries.
template <int NMAX, int RR>
__global__ void __launch_bounds__(RR == 0 ? 64 : 128) k_count_sparse(SparseArgs a) {
    extern __shared__ int32_t s_ring[];
    const int64_t n_thr = a.d_n_threads ? *a.d_n_threads : a.n_threads;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n_thr;
         t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t tr = a.rec_first + t;
    int lo_r = 0, hi_r = a.n_recs;  // last recording whose records start at or before tr
    while (hi_r - lo_r > 1) {
        const int mid = (lo_r + hi_r) >> 1;
        if (a.rinfo[mid].recbase <= tr) lo_r = mid; else hi_r = mid;
    }
    const RecInfo ri = a.rinfo[lo_r];
    const int64_t local = tr - ri.recbase;
    const int slot = ri.slot_first + (int)(local / ri.P);
    const int p = (int)(local % ri.P);
    const int cand = a.slot2cand[slot];
    const int64_t o = a.offs[cand];
    const int N = (int)(a.offs[cand + 1] - o);
    const int64_t eo = o - cand;

    Machine<NMAX, RR> st;
    st.N = N;
    st.ncls = 0;
    st.live = 0;
    st.M = INT32_MIN;
    st.open = 1;
    st.flags = 0;
    int64_t sumhi = 0;
#pragma unroll
    for (int k = 0; k < NMAX; ++k) st.E[k] = k < N ? (uint32_t)a.ctypes[o + k] : 0xFFFFFFFFu;
#pragma unroll
    for (int k = 0; k < NMAX - 1; ++k) {
        st.lo[k] = (k < N - 1) ? (a.relaxed ? 0 : a.clo[eo + k]) : 0;
        st.hi[k] = (k < N - 1) ? a.chi[eo + k] : 0;
        sumhi += st.hi[k];
    }
#pragma unroll
    for (int j = 0; j < kClasses; ++j) {
        st.cthr[j] = 0;
        st.cprev[j] = 0;
        st.ccnt[j] = 0;
    }
    bool slab_overflow = false;
    if constexpr (RR == 0) {
    if (a.dens) {
        int used = 0;
#pragma unroll
        for (int k = 0; k < NMAX - 1; ++k) {
            int c = 2;
            if (k < N - 1) {
                const int32_t l = a.relaxed ? 0 : st.lo[k];
                int j = 0;
                while (j < a.n_lo && a.lo_vals[j] != l) ++j;
                uint32_t d = j < a.n_lo ? a.dens[lo_r * a.n_lo + j][st.E[k]] : 0xFFFFFFFFu;
                if (d == 0xFFFFFFFFu || d == 0) d = ri.freq[st.E[k]] > 0 ? ri.freq[st.E[k]] : 1;
                c = d >= 0x7FFFFFFEu ? 0x7FFFFFFF : (int)d + 1;
            } else {
                c = 0;
            }
            st.rings.cap[k] = c < 2 && k < N - 1 ? 2 : c;
            used += st.rings.cap[k];
            if (used > a.slab) slab_overflow = true;
        }
        if (slab_overflow) {
#pragma unroll
            for (int k = 0; k < NMAX - 1; ++k) st.rings.cap[k] = 0;
        }
        st.rings.init_var(s_ring + threadIdx.x, s_ring + a.slab * blockDim.x + threadIdx.x, blockDim.x);
    } else {
        st.rings.init(s_ring + threadIdx.x, s_ring + (NMAX - 1) * a.R * blockDim.x + threadIdx.x, a.R, blockDim.x);
    }
    } else {
        st.rings.init(nullptr, nullptr, 0, 0);
    }
    if (slab_overflow) st.flags |= kMetaRingOverflow;

    const int64_t seg_b = ri.seg[p], seg_e = ri.seg[p + 1];
    int32_t Tp = 0;
    int32_t head[NMAX];
    int32_t cur[NMAX], end[NMAX];
#pragma unroll
    for (int k = 0; k < NMAX; ++k) {
        head[k] = INT32_MAX;
        cur[k] = 0;
        end[k] = 0;
    }
    if (seg_b < seg_e && !slab_overflow) {
        Tp = ri.time[seg_b];
        const int64_t haloT = (p == 0) ? INT64_MIN : (int64_t)Tp - sumhi;
        const int32_t Tend = (seg_e < ri.n) ? ri.time[seg_e] : INT32_MAX;
#pragma unroll
        for (int k = 0; k < NMAX; ++k) {
            if (k >= N) continue;
            bool first = true;  // a repeated type is merged once
#pragma unroll
            for (int j = 0; j < k; ++j)
                if (st.E[j] == st.E[k]) first = false;
            if (!first) continue;
            const int64_t b0 = ri.toff[st.E[k]], b1 = ri.toff[st.E[k] + 1];
            int64_t lo_i = b0, hi_i = b1;  // first time >= haloT
            while (lo_i < hi_i) {
                const int64_t mid = (lo_i + hi_i) >> 1;
                if ((int64_t)ri.ttime[mid] < haloT) lo_i = mid + 1; else hi_i = mid;
            }
            int64_t e_i = b1;
            if (seg_e < ri.n) {  // first time >= Tend
                int64_t l2 = lo_i, h2 = b1;
                while (l2 < h2) {
                    const int64_t mid = (l2 + h2) >> 1;
                    if (ri.ttime[mid] < Tend) l2 = mid + 1; else h2 = mid;
                }
                e_i = l2;
            }
            cur[k] = (int32_t)lo_i;
            end[k] = (int32_t)e_i;
            head[k] = lo_i < e_i ? ri.ttime[lo_i] : INT32_MAX;
        }
        for (;;) {
            int32_t best = INT32_MAX;
            int bk = -1;
#pragma unroll
            for (int k = 0; k < NMAX; ++k)
                if (head[k] < best) {
                    best = head[k];
                    bk = k;
                }
            if (bk < 0) break;
            uint32_t ety = 0;
#pragma unroll
            for (int k = 0; k < NMAX; ++k)
                if (k == bk) {
                    ety = st.E[k];
                    cur[k] += 1;
                    head[k] = cur[k] < end[k] ? ri.ttime[cur[k]] : INT32_MAX;
                }
            st.step(ety, best, best >= Tp, Tp);
        }
    }
    st.finish();
    int4 *r = reinterpret_cast<int4 *>(a.rec + tr * kRecWords);
    int32_t w[kRecWords];
    w[0] = st.ncls | st.flags | (st.open ? 0 : kMetaClosed);
#pragma unroll
    for (int j = 0; j < kClasses; ++j) {
        w[1 + j] = st.cthr[j];
        w[1 + kClasses + j] = (int32_t)st.ccnt[j];
        w[1 + 2 * kClasses + j] = st.cprev[j];
    }
#pragma unroll
    for (int j = 1 + 3 * kClasses; j < kRecWords; ++j) w[j] = 0;
#pragma unroll
    for (int q = 0; q < kRecWords / 4; ++q) r[q] = make_int4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
    }
}

// Node-uniform sparse kernel (shared-memory rings sized per node).  Every
// lane handles its next event with the same instruction sequence whatever
// node the event belongs to: the node's ring offset, size, head and bounds
// live in a small per-thread header in shared memory, so the update indexes
// them instead of branching per node (lanes of a warp are usually at
// different nodes).  Thread i's words are strided by the block size:
// header word w at w*64 + i, ring times at (H + e)*64 + i, ring starts at
// (H + slab + e)*64 + i, with H = 6*(NMAX-1).
//
// A node's ring is a queue in time order: entries from the tail up to the
// head are not yet past the node's lower bound; the entry just before the
// tail is the newest one that is.  Queries of a node come in time order, so
// the tail only moves forward and a query costs one comparison per entry
// that becomes eligible plus one.
template <int NMAX>
__global__ void __launch_bounds__(64) k_count_sparse_u(SparseArgs a) {
    extern __shared__ int32_t s_u[];
    constexpr int HW = 6 * (NMAX - 1);
    const int bd = blockDim.x;
    int32_t *hdr = s_u + threadIdx.x;                 // [w * bd]
    int32_t *rT = s_u + HW * bd + threadIdx.x;        // [e * bd]
    int32_t *rL = s_u + (HW + a.slab) * bd + threadIdx.x;
    // header fields of node k: off, cap, head, lo, hi, tail
#define H_OFF(k) hdr[(6 * (k) + 0) * bd]
#define H_CAP(k) hdr[(6 * (k) + 1) * bd]
#define H_HEAD(k) hdr[(6 * (k) + 2) * bd]
#define H_LO(k) hdr[(6 * (k) + 3) * bd]
#define H_HI(k) hdr[(6 * (k) + 4) * bd]
#define H_TAIL(k) hdr[(6 * (k) + 5) * bd]
    const int64_t n_thr = a.d_n_threads ? *a.d_n_threads : a.n_threads;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n_thr; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t tr = a.rec_first + t;
        int lo_r = 0, hi_r = a.n_recs;
        while (hi_r - lo_r > 1) {
            const int mid = (lo_r + hi_r) >> 1;
            if (a.rinfo[mid].recbase <= tr) lo_r = mid; else hi_r = mid;
        }
        const RecInfo ri = a.rinfo[lo_r];
        const int64_t local = tr - ri.recbase;
        const int slot = ri.slot_first + (int)(local / ri.P);
        const int p = (int)(local % ri.P);
        const int cand = a.slot2cand[slot];
        if (a.skip && a.skip[cand]) continue;  // the stitch writes its count (0)
        const int64_t o = a.offs[cand];
        const int N = (int)(a.offs[cand + 1] - o);
        const int64_t eo = o - cand;

        Machine<NMAX, 0> st;  // entry classes only (its rings are unused here)
        st.N = N;
        st.ncls = 0;
        st.live = 0;
        st.M = INT32_MIN;
        st.open = 1;
        st.flags = 0;
#pragma unroll
        for (int j = 0; j < kClasses; ++j) {
            st.cthr[j] = 0;
            st.cprev[j] = 0;
            st.ccnt[j] = 0;
        }
        uint32_t E[NMAX];
        int64_t sumhi = 0;
        int used = 0;
        bool slab_overflow = false;
#pragma unroll
        for (int k = 0; k < NMAX; ++k) E[k] = k < N ? (uint32_t)a.ctypes[o + k] : 0xFFFFFFFFu;
#pragma unroll
        for (int k = 0; k < NMAX - 1; ++k) {
            if (k >= N - 1) continue;
            const int32_t l = a.relaxed ? 0 : a.clo[eo + k];
            const int32_t h = a.chi[eo + k];
            sumhi += h;
            const int32_t lq = a.relaxed ? 0 : l;
            int j = 0;
            while (j < a.n_lo && a.lo_vals[j] != lq) ++j;
            uint32_t d = j < a.n_lo ? a.dens[lo_r * a.n_lo + j][E[k]] : 0xFFFFFFFFu;
            if (d == 0xFFFFFFFFu || d == 0) d = ri.freq[E[k]] > 0 ? ri.freq[E[k]] : 1;
            const int c = d >= (uint32_t)a.slab ? a.slab + 1 : (int)d + 1;
            H_OFF(k) = used;
            H_CAP(k) = c;
            H_HEAD(k) = 0;
            H_TAIL(k) = 0;
            H_LO(k) = l;
            H_HI(k) = h;
            used += c;
            if (used > a.slab) slab_overflow = true;
        }
        if (!slab_overflow)
            for (int e = 0; e < used; ++e) rT[e * bd] = INT32_MIN;
        else
            st.flags |= kMetaRingOverflow;

        const int64_t seg_b = ri.seg[p], seg_e = ri.seg[p + 1];
        int32_t Tp = 0;
        // head[k]: time at list cursor cur[k]; nxt[k]: the one after it,
        // loaded one step early so that the merge does not wait on it
        int32_t head[NMAX], nxt[NMAX];
        int32_t cur[NMAX], end[NMAX];
        uint32_t nodes[NMAX];  // nodes sharing the cursor's type (bit k = node k)
#pragma unroll
        for (int k = 0; k < NMAX; ++k) {
            head[k] = INT32_MAX;
            nxt[k] = INT32_MAX;
            cur[k] = 0;
            end[k] = 0;
            nodes[k] = 0;
        }
        if (seg_b < seg_e && !slab_overflow) {
            Tp = ri.time[seg_b];
            const int64_t haloT = (p == 0) ? INT64_MIN : (int64_t)Tp - sumhi;
            const int32_t Tend = (seg_e < ri.n) ? ri.time[seg_e] : INT32_MAX;
#pragma unroll
            for (int k = 0; k < NMAX; ++k) {
                if (k >= N) continue;
                bool first = true;
#pragma unroll
                for (int j = 0; j < k; ++j)
                    if (E[j] == E[k]) first = false;
                if (!first) continue;
                uint32_t m = 0;
#pragma unroll
                for (int j = 0; j < NMAX; ++j)
                    if (j < N && E[j] == E[k]) m |= 1u << j;
                nodes[k] = m;
                const int64_t b0 = ri.toff[E[k]], b1 = ri.toff[E[k] + 1];
                int64_t lo_i, e_i;
                if (ri.tseg) {
                    // list positions of the segment's boundaries from the
                    // table, then back over the halo's few events
                    const int32_t *tq = ri.tseg + (size_t)E[k] * ri.tstride;
                    const int qmax = ri.tstride - 1;
                    lo_i = b0 + tq[min(p * ri.sstep, qmax)];
                    e_i = b0 + tq[min((p + 1) * ri.sstep, qmax)];
                    while (lo_i > b0 && (int64_t)ri.ttime[lo_i - 1] >= haloT) --lo_i;
                } else {
                    lo_i = b0;
                    int64_t hi_i = b1;
                    while (lo_i < hi_i) {
                        const int64_t mid = (lo_i + hi_i) >> 1;
                        if ((int64_t)ri.ttime[mid] < haloT) lo_i = mid + 1; else hi_i = mid;
                    }
                    e_i = b1;
                    if (seg_e < ri.n) {
                        int64_t l2 = lo_i, h2 = b1;
                        while (l2 < h2) {
                            const int64_t mid = (l2 + h2) >> 1;
                            if (ri.ttime[mid] < Tend) l2 = mid + 1; else h2 = mid;
                        }
                        e_i = l2;
                    }
                }
                cur[k] = (int32_t)lo_i;
                end[k] = (int32_t)e_i;
                head[k] = lo_i < e_i ? ri.ttime[lo_i] : INT32_MAX;
                nxt[k] = lo_i + 1 < e_i ? ri.ttime[lo_i + 1] : INT32_MAX;
            }
            for (;;) {
                int32_t tt = INT32_MAX;
                int bk = -1;
#pragma unroll
                for (int k = 0; k < NMAX; ++k)
                    if (head[k] < tt) {
                        tt = head[k];
                        bk = k;
                    }
                if (bk < 0) break;
                uint32_t mask = 0;
#pragma unroll
                for (int k = 0; k < NMAX; ++k)
                    if (k == bk) {
                        mask = nodes[k];
                        cur[k] += 1;
                        head[k] = nxt[k];
                        nxt[k] = cur[k] + 1 < end[k] ? ri.ttime[cur[k] + 1] : INT32_MAX;
                    }
                const bool in_seg = tt >= Tp;
                // nodes of this type, last to first (one node unless the
                // episode repeats a type)
                while (mask) {
                    const int k = 31 - __clz(mask);
                    mask &= ~(1u << k);
                    bool do_push = (k == 0) && (N > 1);
                    bool do_end = false;
                    int32_t L = tt;
                    if (k > 0) {
                        const int q = k - 1;
                        const int32_t base = H_OFF(q), R = H_CAP(q), hd = H_HEAD(q);
                        const int32_t elig = tt - H_LO(q), expire = tt - H_HI(q);
                        int tl = H_TAIL(q);
                        while (tl != hd && rT[(base + tl) * bd] < elig) tl = (tl + 1 == R) ? 0 : tl + 1;
                        H_TAIL(q) = tl;
                        const int le = (tl == 0) ? R - 1 : tl - 1;  // newest eligible entry
                        const int32_t tp = rT[(base + le) * bd];
                        const bool ok = tp != INT32_MIN && tp >= expire;
                        if (ok) L = rL[(base + le) * bd];
                        if (ok) {
                            if (k == N - 1)
                                do_end = true;
                            else
                                do_push = true;
                        }
                    }
                    if (do_end && in_seg) st.greedy_end(tt, L, Tp);
                    if (do_push) {
                        // entries already past the lower bound at tt stay so
                        // for every later query: retire them first, so the
                        // queue holds only entries inside [tt - lo, tt]
                        // (at most the window density, one less than the
                        // ring) and a full ring means the density was wrong
                        const int32_t base = H_OFF(k), R = H_CAP(k), h = H_HEAD(k);
                        const int32_t eg = tt - H_LO(k);
                        int tl = H_TAIL(k);
                        while (tl != h && rT[(base + tl) * bd] < eg) tl = (tl + 1 == R) ? 0 : tl + 1;
                        const int h2 = (h + 1 == R) ? 0 : h + 1;
                        if (h2 == tl) st.flags |= kMetaRingOverflow;
                        rT[(base + h) * bd] = tt;
                        rL[(base + h) * bd] = L;
                        H_HEAD(k) = h2;
                        H_TAIL(k) = tl;
                    }
                }
            }
        }
        st.finish();
        int4 *r = reinterpret_cast<int4 *>(a.rec + tr * kRecWords);
        int32_t w[kRecWords];
        w[0] = st.ncls | st.flags | (st.open ? 0 : kMetaClosed);
#pragma unroll
        for (int j = 0; j < kClasses; ++j) {
            w[1 + j] = st.cthr[j];
            w[1 + kClasses + j] = (int32_t)st.ccnt[j];
            w[1 + 2 * kClasses + j] = st.cprev[j];
        }
#pragma unroll
        for (int j = 1 + 3 * kClasses; j < kRecWords; ++j) w[j] = 0;
#pragma unroll
        for (int q = 0; q < kRecWords / 4; ++q) r[q] = make_int4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
    }
#undef H_OFF
#undef H_CAP
#undef H_HEAD
#undef H_LO
#undef H_HI
#undef H_TAIL
}

// Shared memory of a node-uniform sparse block (64 threads, slab entries).
static size_t sparse_u_smem(int nmax, int slab) { return (size_t)(6 * (nmax - 1) + 2 * slab) * 64 * 4; }

typedef void (*SparseUFn)(SparseArgs);
static SparseUFn sparse_u_fn(int nclass) {
    switch (nclass) {
        case 0: return k_count_sparse_u<2>;
        case 1: return k_count_sparse_u<4>;
        case 2: return k_count_sparse_u<8>;
        default: return k_count_sparse_u<16>;
    }
}

// Cost inputs for choosing between the tiled and the sparse kernel, per
// bucket: for each group of 32 consecutive slots (one warp of the tiled
// kernel), the events whose type some lane uses (what the tiled warp reads),
// and the largest per-episode event count (what the slowest sparse lane reads).
__global__ void k_group_stats(const int32_t *__restrict__ perm, const int32_t *__restrict__ slot_key, int64_t n_work,
                              int n_recs, const int64_t *__restrict__ offs, const uint16_t *__restrict__ ctypes,
                              const RecInfo *__restrict__ rinfo, unsigned long long *dense_units,
                              unsigned long long *sparse_units) {
    __shared__ uint32_t bm[4][kBitmapWords];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t g = blockIdx.x * 4 + w;
    const int64_t slot = g * 32 + lane;
    for (int i = lane; i < kBitmapWords; i += 32) bm[w][i] = 0;
    __syncwarp();
    unsigned long long cov = 0, rel = 0;
    int b = -1;
    if (slot < n_work) {
        const int cand = perm[slot];
        const int key = slot_key[slot];
        b = key / n_recs;
        const uint32_t *freq = rinfo[key % n_recs].freq;
        for (int64_t q = offs[cand]; q < offs[cand + 1]; ++q) {
            const uint32_t ty = ctypes[q];
            const uint32_t f = freq[ty];
            rel += f;
            const uint32_t bit = 1u << (ty & 31);
            const uint32_t old = atomicOr(&bm[w][(ty >> 5) & (kBitmapWords - 1)], bit);
            if (!(old & bit)) cov += f;
        }
    }
    for (int d = 16; d > 0; d >>= 1) {
        cov += __shfl_down_sync(0xFFFFFFFFu, cov, d);
        const unsigned long long o = __shfl_down_sync(0xFFFFFFFFu, rel, d);
        rel = o > rel ? o : rel;
    }
    const int b0 = __shfl_sync(0xFFFFFFFFu, b, 0);
    if (lane == 0 && b0 >= 0) {
        atomicAdd(&dense_units[b0], cov);
        atomicAdd(&sparse_units[b0], rel);
    }
}

// Per-type event lists of a stream: a stable partition of the event indices
// by type, then the times gathered in that order.
__global__ void k_widen_types(const uint16_t *__restrict__ ty, int64_t n, int32_t *__restrict__ key) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        key[i] = ty[i];
}

__global__ void k_gather_ttime(const int32_t *__restrict__ perm, const int32_t *__restrict__ tm, int64_t n,
                               int32_t *__restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = tm[perm[i]];
}

__global__ void k_toff(const int32_t *__restrict__ keyoff, int n_types, int64_t n, int64_t *__restrict__ toff) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a < n_types) toff[a] = keyoff[a];
    if (a == n_types) toff[a] = n;
}

// Temporary device allocations freed together (after the stream drains).
int stream_bytype(fem_ctx *ctx, fem_stream *s) {
    if (s->d_ttime) return FEM_OK;
    if (s->n_types > 8192 || s->n > INT32_MAX / 2) return FEM_ERR_INVAL;
    const int64_t n = s->n;
    void *p1 = nullptr, *p2 = nullptr;
    FEM_TRY(dev_alloc(ctx, &p1, sizeof(int64_t) * (s->n_types + 1)));
    const int st2 = dev_alloc(ctx, &p2, sizeof(int32_t) * std::max<int64_t>(n, 1));
    if (st2 != FEM_OK) {
        dev_free(ctx, p1, sizeof(int64_t) * (s->n_types + 1));
        return st2;
    }
    int64_t *toff = static_cast<int64_t *>(p1);
    int32_t *ttime = static_cast<int32_t *>(p2);
    const int n_keys = (int)s->n_types;
    const int64_t nblk = std::max<int64_t>(1, (n + kPartBlock - 1) / kPartBlock);
    const int64_t tab_n = (int64_t)n_keys * nblk;
    TmpDev tmp(ctx);
    int32_t *key, *perm, *blk, *stmp, *koff;
    int st = tmp.get(&key, std::max<int64_t>(n, 1));
    if (st == FEM_OK) st = tmp.get(&perm, std::max<int64_t>(n, 1));
    if (st == FEM_OK) st = tmp.get(&blk, tab_n);
    if (st == FEM_OK) st = tmp.get(&stmp, tab_n / kScanBlock + 2);
    if (st == FEM_OK) st = tmp.get(&koff, n_keys + 1);
    if (st != FEM_OK) {
        dev_free(ctx, p1, sizeof(int64_t) * (s->n_types + 1));
        dev_free(ctx, p2, sizeof(int32_t) * std::max<int64_t>(n, 1));
        return st;
    }
    cudaStream_t cs = ctx->stream;
    if (n > 0) {
        const unsigned g = (unsigned)std::min<int64_t>((n + 255) / 256, 8 * ctx->n_sm);
        k_widen_types<<<g, 256, 0, cs>>>(s->d_type, n, key);
        k_part_count<<<(unsigned)nblk, 256, n_keys * 4, cs>>>(key, n, n_keys, nblk, blk);
        FEM_TRY(scan_exclusive(cs, blk, tab_n, stmp, nullptr, nullptr));
        k_part_scatter<<<(unsigned)nblk, 32, n_keys * 4, cs>>>(key, n, n_keys, nblk, blk, nullptr, perm, nullptr);
        k_gather_keyoff<<<(n_keys + 255) / 256, 256, 0, cs>>>(blk, n_keys, nblk, koff);
        k_gather_ttime<<<g, 256, 0, cs>>>(perm, s->d_time, n, ttime);
        k_toff<<<(n_keys + 1 + 255) / 256, 256, 0, cs>>>(koff, n_keys, n, toff);
    } else {
        FEM_CUDA_TRY(cudaMemsetAsync(toff, 0, sizeof(int64_t) * (s->n_types + 1), cs));
    }
    FEM_CUDA_TRY(cudaGetLastError());
    // longest per-type list (sizes the per-warp buffers of local tracking)
    std::vector<int64_t> toff_h(s->n_types + 1, 0);
    FEM_CUDA_TRY(cudaMemcpyAsync(toff_h.data(), toff, sizeof(int64_t) * (s->n_types + 1), cudaMemcpyDeviceToHost, cs));
    FEM_CUDA_TRY(cudaStreamSynchronize(cs));
    s->max_list = 0;
    for (uint32_t a = 0; a < s->n_types; ++a) s->max_list = std::max(s->max_list, toff_h[a + 1] - toff_h[a]);
    s->d_toff = toff;
    s->d_ttime = ttime;
    s->bytes += sizeof(int64_t) * (s->n_types + 1) + sizeof(int32_t) * n;
    return FEM_OK;
}

// Time index of the per-type lists (one block row per type): the event at
// list position j answers the cells after its predecessor's and up to its
// own; position len answers the cells past the type's last event.
__global__ void k_tindex(const int64_t *__restrict__ toff, const int32_t *__restrict__ ttime, int32_t tbase,
                         int shift, int64_t ncell, int32_t *__restrict__ tidx) {
    const int a = blockIdx.y;
    const int64_t b = toff[a], len = toff[a + 1] - b;
    const int32_t *t = ttime + b;
    int32_t *row = tidx + (int64_t)a * (ncell + 1);
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j <= len; j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c_lo = j == 0 ? 0 : ((int64_t)(t[j - 1] - tbase) >> shift) + 1;
        const int64_t c_hi = j == len ? ncell : ((int64_t)(t[j] - tbase) >> shift);
        for (int64_t c = c_lo; c <= c_hi; ++c) row[c] = (int32_t)j;
    }
}

int stream_tindex(fem_ctx *ctx, fem_stream *s) {
    if (s->d_tidx) return FEM_OK;
    FEM_TRY(stream_bytype(ctx, s));
    const int64_t n = s->n;
    const double span = n > 0 ? (double)s->t_last - (double)s->t_first + 1.0 : 1.0;
    // cell width: the power of two nearest the mean gap between events of
    // one type, n_types * span / n
    const double gap = n > 0 ? (double)s->n_types * span / (double)n : 1.0;
    int shift = 0;
    while (shift < 30 && (double)(2LL << shift) <= gap * 1.4142) ++shift;
    const int64_t ncell = n > 0 ? (((int64_t)s->t_last - s->t_first) >> shift) + 1 : 1;
    const size_t bytes = sizeof(int32_t) * (size_t)s->n_types * (size_t)(ncell + 1);
    void *p = nullptr;
    FEM_TRY(dev_alloc(ctx, &p, bytes));
    int32_t *tidx = static_cast<int32_t *>(p);
    if (n > 0) {
        const int64_t mean = n / std::max<uint32_t>(s->n_types, 1) + 1;
        const unsigned gx = (unsigned)std::max<int64_t>(1, std::min<int64_t>((mean + 255) / 256, 64));
        k_tindex<<<dim3(gx, s->n_types), 256, 0, ctx->stream>>>(s->d_toff, s->d_ttime, s->t_first, shift, ncell,
                                                                  tidx);
    } else if (cudaMemsetAsync(tidx, 0, bytes, ctx->stream) != cudaSuccess) {
        dev_free(ctx, p, bytes);
        return FEM_ERR_CUDA;
    }
    if (cudaGetLastError() != cudaSuccess) {
        dev_free(ctx, p, bytes);
        return FEM_ERR_CUDA;
    }
    s->d_tidx = tidx;
    s->tshift = shift;
    s->tcells = ncell;
    s->bytes += bytes;
    return FEM_OK;
}

typedef void (*SparseFn)(SparseArgs);

static SparseFn sparse_fn(int nclass, int rr) {
#define FEM_SF(NM, R_) \
    if (nmax_of_class(nclass) == NM && rr == R_) return k_count_sparse<NM, R_>;
    FEM_SF(2, 2) FEM_SF(2, 4) FEM_SF(2, 8) FEM_SF(2, 0)
    FEM_SF(4, 2) FEM_SF(4, 4) FEM_SF(4, 0)
    FEM_SF(8, 2) FEM_SF(8, 0)
    FEM_SF(16, 0)
#undef FEM_SF
    return nullptr;
}

// Device-sized counting for captured graphs: the sparse kernel with
// shared-memory rings of R entries over up to cap_threads (episode, segment)
// threads, then the stitch over up to cap_slots episodes; the live sizes are
// read from device memory.
int launch_count_dev(cudaStream_t st, int nmax, int nodes, int R, const RecInfo *rinfo, int n_recs, const int64_t *d_n_threads,
                     int64_t cap_threads, const int64_t *offs, const uint16_t *ctypes, const int32_t *clo,
                     const int32_t *chi, const int32_t *slot2cand, const uint32_t *cand_rec, int32_t *rec,
                     const int32_t *d_n_slots, int64_t cap_slots, uint32_t *counts, int32_t *fb_list, int *fb_count,
                     const uint32_t *const *dens, const int32_t *lo_vals, int n_lo, const uint8_t *skip) {
    const int nclass = nmax == 2 ? 0 : nmax == 4 ? 1 : nmax == 8 ? 2 : 3;
    SparseUFn f = sparse_u_fn(nclass);
    if (!f) return FEM_ERR_CUDA;
    SparseArgs sa{};
    sa.rinfo = rinfo;
    sa.n_recs = n_recs;
    sa.rec_first = 0;
    sa.n_threads = cap_threads;
    sa.d_n_threads = d_n_threads;
    sa.offs = offs;
    sa.ctypes = ctypes;
    sa.clo = clo;
    sa.chi = chi;
    sa.slot2cand = slot2cand;
    sa.relaxed = 0;
    sa.R = R;
    sa.rec = rec;
    sa.dens = dens;
    sa.lo_vals = lo_vals;
    sa.n_lo = n_lo;
    sa.slab = (nodes - 1) * R;  // every node's ring fits R entries (checked by the caller)
    sa.skip = skip;
    const size_t sm = sparse_u_smem(nmax, sa.slab);
    if (sm > 48 * 1024 &&
        cudaFuncSetAttribute((const void *)f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
        return FEM_ERR_CUDA;
    // grid-stride launches sized to what the GPU holds at once (the live
    // sizes are only known on the device)
    int dev = 0, nsm = 0, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, 64, sm);
    const int64_t gs = std::min<int64_t>((cap_threads + 63) / 64, (int64_t)std::max(1, nsm) * std::max(1, per_sm));
    if (cap_threads > 0) f<<<(unsigned)gs, 64, sm, st>>>(sa);
    FEM_CUDA_TRY(cudaGetLastError());
    return launch_stitch_dev(st, nsm, rinfo, slot2cand, cand_rec, rec, d_n_slots, cap_slots, counts, fb_list,
                             fb_count, skip, nullptr, 0);
}

int launch_stitch_dev(cudaStream_t st, int nsm, const RecInfo *rinfo, const int32_t *slot2cand,
                      const uint32_t *cand_rec, const int32_t *rec, const int32_t *d_n_slots, int64_t cap_slots,
                      uint32_t *counts, int32_t *fb_list, int *fb_count, const uint8_t *skip, const int *d_maxP,
                      int direct_p1) {
    // the live segment counts are only known on the device: both stitch
    // kernels run, each taking the episodes on its side of kStitchSplit
    const int64_t gst = std::min<int64_t>((cap_slots + kStitchWarps - 1) / kStitchWarps, (int64_t)std::max(1, nsm) * 8);
    const int64_t gsb = std::min<int64_t>(cap_slots, (int64_t)std::max(1, nsm) * 4);
    if (cap_slots > 0) {
        k_stitch<<<(unsigned)gst, kStitchWarps * 32, 0, st>>>(rec, rinfo, slot2cand, cand_rec, 0, (int)cap_slots,
                                                            counts, fb_list, fb_count, d_n_slots, kStitchSplit, skip,
                                                            d_maxP, direct_p1);
        k_stitch_block<<<(unsigned)gsb, kStitchBlock, 0, st>>>(rec, rinfo, slot2cand, cand_rec, 0, (int)cap_slots,
                                                               counts, fb_list, fb_count, d_n_slots, kStitchSplit,
                                                               skip, d_maxP);
    }
    FEM_CUDA_TRY(cudaGetLastError());
    return FEM_OK;
}

size_t sparse_smem_bytes(int nmax, int R) { return (size_t)2 * (nmax - 1) * R * 64 * 4; }

// Register-ring capacity compiled for (nclass, R); 0 = shared-memory rings.
static int reg_ring_for(int nclass, int R) {
    const int cap = max_reg_ring(nclass);
    for (int r = 2; r <= cap; r *= 2)
        if (R <= r) return r;
    return 0;
}

static size_t tiled_smem_rt(int nclass, int K, int R, int T) {
    const int nmax = nmax_of_class(nclass);
    const int rr = reg_ring_for(nclass, R);
    return 128 + (size_t)kStages * T * 6 + (size_t)(K / 32) * kBitmapWords * 4 +
           (rr ? 0 : (size_t)2 * (nmax - 1) * R * K * 4);
}

typedef void (*TiledFn)(TiledArgs);

static TiledFn tiled_fn(int nclass, int rr) {
#define FEM_TF(NM, R_) \
    if (nmax_of_class(nclass) == NM && rr == R_) return k_count_tiled<NM, R_>;
    FEM_TF(2, 2) FEM_TF(2, 4) FEM_TF(2, 8) FEM_TF(2, 0)
    FEM_TF(4, 2) FEM_TF(4, 4) FEM_TF(4, 0)
    FEM_TF(8, 2) FEM_TF(8, 0)
    FEM_TF(16, 0)
#undef FEM_TF
    return nullptr;
}

static int launch_tiled(fem_ctx *ctx, int nclass, int n_items, int K, int R, int T, const TiledArgs &a) {
    const size_t sm = tiled_smem_rt(nclass, K, R, T);
    TiledFn f = tiled_fn(nclass, reg_ring_for(nclass, R));
    if (!f) return FEM_ERR_CUDA;
    if (cudaFuncSetAttribute((const void *)f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
        return FEM_ERR_CUDA;
    f<<<dim3(n_items), dim3(K + 32), sm, ctx->stream>>>(a);
    FEM_CUDA_TRY(cudaGetLastError());
    return FEM_OK;
}

static int occupancy_tiled(int nclass, int K, int R, size_t sm) {
    int blocks = 0;
    TiledFn f = tiled_fn(nclass, reg_ring_for(nclass, R));
    if (f) {
        cudaFuncSetAttribute((const void *)f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, f, K + 32, sm);
    }
    cudaGetLastError();
    return std::max(blocks, 1);
}

struct CountCall {
    fem_ctx *ctx;
    std::vector<fem_stream *> recs;
    // device candidate arrays
    int64_t n_cand = 0;
    const int64_t *offs = nullptr;
    const uint16_t *types = nullptr;
    const int32_t *lo = nullptr;
    const int32_t *hi = nullptr;
    const uint32_t *cand_rec = nullptr;  // null = all recording 0
    uint32_t *counts = nullptr;          // device, n_cand
    std::vector<int32_t> lo_vals;        // distinct lo values (host)
    int mode = 0;                        // 0 exact, 1 plain, 2 relaxed
    double seg_div = 1.0;                // fallback rounds divide the segment count
    bool force_tiled = false;            // last fallback round: tiled kernel, one segment
    fem_stats stats{};
    float count_ms = 0.f;
};

static int run_count(CountCall &cc, const int32_t *subset, int64_t n_sub, int force_segments);

// Builds the per-recording RecInfo table and the density table.
static int count_core(CountCall &cc, const int32_t *subset, int64_t n_work, int force_segments) {
    fem_ctx *ctx = cc.ctx;
    const int n_recs = (int)cc.recs.size();
    // Local tracking, one warp per (episode, segment), one launch for every
    // multi-node episode: the default (kernel 0) and kernel 7; the last
    // fallback round and the explicit kernel choices 1-3 keep the
    // per-episode state machines.
    bool track = (ctx->tuning.kernel == 0 || ctx->tuning.kernel == 7) && !cc.force_tiled && cc.mode != 1;
    for (auto *r : cc.recs)
        if (r->n_types > 8192 || r->n > INT32_MAX / 2) track = false;
    if (track)
        for (auto *r : cc.recs) {
            const int sb = stream_tindex(ctx, r);
            if (sb == FEM_ERR_NOMEM) {
                track = false;
                break;
            }
            if (sb != FEM_OK) return sb;
        }
    // the launch's per-warp entry lists (4 x the longest per-type list each):
    // fewer resident warps while they would pass a quarter of the free
    // budget; without room even for one block the per-episode kernels count
    int track_nblocks = 0;
    int64_t track_cap = 1;
    if (track) {
        for (auto *r : cc.recs) track_cap = std::max(track_cap, r->max_list);
        const size_t free_b = ctx->budget > ctx->used.load() ? ctx->budget - ctx->used.load() : 0;
        track_nblocks = track_blocks(ctx->n_sm);
        while (track_nblocks > 1 && track_buf_bytes(track_nblocks, track_cap) > free_b / 4)
            track_nblocks = track_nblocks > ctx->n_sm ? track_nblocks - ctx->n_sm : track_nblocks / 2;
        if (track_buf_bytes(track_nblocks, track_cap) > free_b / 4) track = false;
    }
    const int n_keys = kBuckets * n_recs;
    // --- density tables and per-recording tables
    std::vector<int32_t> lov = cc.lo_vals;
    if (cc.mode == 2) lov = {0};
    if (lov.empty()) lov = {0};
    std::vector<const uint32_t *> dens_h((size_t)n_recs * lov.size());
    std::vector<uint32_t> nt_h(n_recs);
    for (int r = 0; r < n_recs; ++r) {
        nt_h[r] = cc.recs[r]->n_types;
        if (track) continue;  // window densities size rings; local tracking keeps none
        FEM_TRY(stream_densities(ctx, cc.recs[r], lov));
        for (size_t j = 0; j < lov.size(); ++j) {
            uint32_t *d = nullptr;
            FEM_TRY(stream_density(ctx, cc.recs[r], lov[j], &d));
            dens_h[(size_t)r * lov.size() + j] = d;
        }
    }
    // misc scratch layout: [lo_vals][n_types][dens ptrs][rinfo][bucket_maxR][relevant][fb_count]
    size_t off = 0;
    auto carve = [&](size_t bytes) {
        size_t o = off;
        off += (bytes + 255) & ~size_t(255);
        return o;
    };
    const size_t o_lo = carve(lov.size() * 4), o_nt = carve(n_recs * 4),
                 o_dp = carve(dens_h.size() * sizeof(void *)), o_ri = carve(n_recs * sizeof(RecInfo)),
                 o_bm = carve(4 * kBuckets * 4), o_rel = carve(8), o_fb = carve(8),
                 o_units = carve(2 * kBuckets * 8), o_q = carve(8);
    void *misc = nullptr;
    FEM_TRY(scratch(ctx, kSlotMisc, off, &misc));
    char *mb = static_cast<char *>(misc);
    std::vector<RecInfo> ri_h(n_recs);
    for (int r = 0; r < n_recs; ++r) {
        ri_h[r] = RecInfo{cc.recs[r]->d_type, cc.recs[r]->d_time, cc.recs[r]->n, nullptr, 1, 0, 0,
                          cc.recs[r]->d_freq, nullptr, nullptr};
    }
    FEM_CUDA_TRY(cudaMemcpyAsync(mb + o_lo, lov.data(), lov.size() * 4, cudaMemcpyHostToDevice, ctx->stream));
    FEM_CUDA_TRY(cudaMemcpyAsync(mb + o_nt, nt_h.data(), n_recs * 4, cudaMemcpyHostToDevice, ctx->stream));
    FEM_CUDA_TRY(cudaMemcpyAsync(mb + o_dp, dens_h.data(), dens_h.size() * sizeof(void *),
                                 cudaMemcpyHostToDevice, ctx->stream));
    FEM_CUDA_TRY(cudaMemcpyAsync(mb + o_ri, ri_h.data(), n_recs * sizeof(RecInfo), cudaMemcpyHostToDevice,
                                 ctx->stream));
    FEM_CUDA_TRY(cudaMemsetAsync(mb + o_bm, 0, 4 * kBuckets * 4, ctx->stream));
    FEM_CUDA_TRY(cudaMemsetAsync(mb + o_rel, 0, 8, ctx->stream));
    FEM_CUDA_TRY(cudaMemsetAsync(mb + o_fb, 0, 8, ctx->stream));
    FEM_CUDA_TRY(cudaMemsetAsync(mb + o_units, 0, 2 * kBuckets * 8, ctx->stream));

    // --- prep
    void *p_key, *p_perm, *p_blk;
    FEM_TRY(scratch(ctx, kSlotPrep, sizeof(int32_t) * std::max<int64_t>(n_work, 1) * 3, &p_key));
    int32_t *d_key = static_cast<int32_t *>(p_key);
    int32_t *d_ring = d_key + std::max<int64_t>(n_work, 1);
    int32_t *d_slotkey = d_ring + std::max<int64_t>(n_work, 1);
    FEM_TRY(scratch(ctx, kSlotPerm, sizeof(int32_t) * std::max<int64_t>(n_work, 1), &p_perm));
    int32_t *d_perm = static_cast<int32_t *>(p_perm);
    const int pb = 256;
    const int64_t nprep = (n_work + pb - 1) / pb;
    const int64_t nblk = (n_work + kPartBlock - 1) / kPartBlock;
    const int64_t tab_n = (int64_t)n_keys * std::max<int64_t>(nblk, 1);
    FEM_TRY(scratch(ctx, kSlotBucket, sizeof(int32_t) * (tab_n + (tab_n + kScanBlock - 1) / kScanBlock + n_keys + 64),
                    &p_blk));
    int32_t *d_blk = static_cast<int32_t *>(p_blk);
    int32_t *d_scan_tmp = d_blk + tab_n;
    int32_t *d_keyoff = d_scan_tmp + (tab_n + kScanBlock - 1) / kScanBlock + 1;
    PrepArgs pa{};
    pa.n_cand = n_work;
    pa.offs = cc.offs;
    pa.ctypes = cc.types;
    pa.clo = cc.lo;
    pa.chi = cc.hi;
    pa.cand_rec = cc.cand_rec;
    pa.subset = subset;
    pa.rinfo = reinterpret_cast<const RecInfo *>(mb + o_ri);
    pa.n_types = reinterpret_cast<const uint32_t *>(mb + o_nt);
    pa.lo_vals = reinterpret_cast<const int32_t *>(mb + o_lo);
    pa.n_lo = track ? 0 : (int)lov.size();  // without tables every ring is taken as unknown
    pa.dens = reinterpret_cast<const uint32_t *const *>(mb + o_dp);
    pa.n_recs = n_recs;
    pa.mode = cc.mode;
    pa.force_plain_ring = 0;
    pa.track = track ? 1 : 0;
    pa.key = d_key;
    pa.ring = d_ring;
    pa.bucket_maxR = reinterpret_cast<int *>(mb + o_bm);
    pa.relevant = reinterpret_cast<unsigned long long *>(mb + o_rel);
    pa.status = ctx->d_status;
    if (n_work > 0) {
        k_prep<<<(unsigned)nprep, pb, 0, ctx->stream>>>(pa);
        k_part_count<<<(unsigned)nblk, 256, n_keys * 4, ctx->stream>>>(d_key, n_work, n_keys, nblk, d_blk);
        FEM_TRY(scan_exclusive(ctx->stream, d_blk, tab_n, d_scan_tmp, nullptr, &cc.stats.kernel_launches));
        k_part_scatter<<<(unsigned)nblk, 32, n_keys * 4, ctx->stream>>>(d_key, n_work, n_keys, nblk, d_blk,
                                                                        subset, d_perm, d_slotkey);
        k_gather_keyoff<<<(n_keys + 255) / 256, 256, 0, ctx->stream>>>(d_blk, n_keys, nblk, d_keyoff);
        unsigned long long *units = reinterpret_cast<unsigned long long *>(mb + o_units);
        k_group_stats<<<(unsigned)((n_work + 127) / 128), 128, 0, ctx->stream>>>(
            d_perm, d_slotkey, n_work, n_recs, cc.offs, cc.types, reinterpret_cast<const RecInfo *>(mb + o_ri), units,
            units + kBuckets);
        cc.stats.kernel_launches += 5;
        FEM_CUDA_TRY(cudaGetLastError());
    }
    std::vector<int32_t> key_off(n_keys + 1, 0);
    std::vector<int32_t> bmax(4 * kBuckets, 0);
    unsigned long long relv = 0;
    if (n_work > 0)
        FEM_CUDA_TRY(cudaMemcpyAsync(key_off.data(), d_keyoff, 4 * n_keys, cudaMemcpyDeviceToHost, ctx->stream));
    FEM_CUDA_TRY(cudaMemcpyAsync(bmax.data(), mb + o_bm, 4 * kBuckets * 4, cudaMemcpyDeviceToHost, ctx->stream));
    FEM_CUDA_TRY(cudaMemcpyAsync(&relv, mb + o_rel, 8, cudaMemcpyDeviceToHost, ctx->stream));
    std::vector<unsigned long long> units_h(2 * kBuckets, 0);
    FEM_CUDA_TRY(cudaMemcpyAsync(units_h.data(), mb + o_units, 2 * kBuckets * 8, cudaMemcpyDeviceToHost, ctx->stream));
    FEM_TRY(sync_status(ctx));
    key_off[n_keys] = (int32_t)n_work;
    if (force_segments == 0)
        for (int k = 0; k < n_keys; ++k)
            cc.stats.counted_episode_events += (double)(key_off[k + 1] - key_off[k]) * (double)cc.recs[k % n_recs]->n;
    cc.stats.relevant_events += (double)relv;

    // --- launches per bucket
    const int T_def = ctx->tuning.tile_events > 0 ? ctx->tuning.tile_events : 1024;
    struct Plan {
        int bucket;
        bool sparse;
        bool track = false;   // local-tracking kernel (bucket 0 in track mode)
        int K, R, nclass, T;
        int slab;         // largest sum of per-node ring sizes in the bucket
        std::vector<RecInfo> ri;
        std::vector<WorkItem> items;
        int slot_begin, n_slots;
        int64_t records;
    };
    bool small_alpha = true;
    for (auto *rs : cc.recs)
        if (rs->n_types > 128) small_alpha = false;
    // Builds the plan of bucket b: tiled (CTA width K, tile T) or sparse, with
    // a multiplier on the segment-count heuristic; records start at recbase.
    auto make_plan = [&](int b, bool sparse, int K, int T, double seg_mult, int64_t recbase) {
        const int sb = key_off[b * n_recs], se = key_off[(b + 1) * n_recs];
        Plan pl;
        pl.bucket = b;
        pl.sparse = sparse;
        pl.track = sparse && track && b == 0;
        pl.nclass = b / kBucketRing;
        pl.R = std::max(bmax[b], 2);
        pl.slab = std::max(bmax[3 * kBuckets + b], 2);
        pl.T = T;
        if (!sparse) {
            while (K > 32 && tiled_smem_rt(pl.nclass, K, pl.R, T) > 100 * 1024) K -= 32;
            while (K > 32 && tiled_smem_rt(pl.nclass, K, pl.R, T) > (size_t)ctx->smem_optin - 2048) K -= 32;
        }
        pl.K = K;
        pl.slot_begin = sb;
        pl.n_slots = se - sb;
        const int64_t max_sumhi = bmax[2 * kBuckets + b];
        double seg_len;
        if (sparse) {
            // enough (episode, segment) threads to fill the GPU ~4 times
            // (local tracking: about four work items per resident warp)
            const double desired = pl.track ? 4.0 * track_nblocks * kTrackWarps : 4.0 * ctx->n_sm * 2048.0;
            double work = 0;
            for (int r = 0; r < n_recs; ++r) {
                const int c = key_off[b * n_recs + r + 1] - key_off[b * n_recs + r];
                work += (double)c * (double)cc.recs[r]->n;
            }
            seg_len = std::max(1.0, work / desired) / seg_mult;
        } else {
            const size_t sm = tiled_smem_rt(pl.nclass, K, pl.R, T);
            const int occ = occupancy_tiled(pl.nclass, K, pl.R, sm);
            // segments: aim for ~4 CTAs per resident slot across the bucket
            const int64_t desired = (int64_t)4 * ctx->n_sm * occ;
            double work = 0;
            for (int r = 0; r < n_recs; ++r) {
                const int c = key_off[b * n_recs + r + 1] - key_off[b * n_recs + r];
                if (c > 0) work += (double)((c + K - 1) / K) * (double)cc.recs[r]->n;
            }
            seg_len = std::max(1.0, work / (double)std::max<int64_t>(desired, 1)) / seg_mult;
        }
        pl.ri.resize(n_recs);
        int64_t rb = recbase;
        for (int r = 0; r < n_recs; ++r) {
            const int ks = key_off[b * n_recs + r], ke = key_off[b * n_recs + r + 1];
            const int c = ke - ks;
            const fem_stream *s = cc.recs[r];
            int P = 1;
            if (force_segments > 0) {
                P = force_segments;
            } else if (ctx->tuning.segments > 0) {
                // explicit request: allow short segments (down to ~16 events)
                P = std::max(1, std::min<int>((int)(ctx->tuning.segments / cc.seg_div),
                                              (int)std::max<int64_t>(1, s->n / 16)));
            } else if (c > 0) {
                // shortest useful segment: 1024 events, and at least 8 halos
                // (the halo is sum(hi) of time at the stream's mean rate)
                const double span = std::max(1.0, (double)s->t_last - (double)s->t_first);
                const double halo_ev = (double)s->n * (double)max_sumhi / span;
                const double min_seg = std::max(sparse && track ? (double)kTrackMinSeg : 1024.0, 8.0 * halo_ev);
                P = (int)std::max<double>(1.0, std::min<double>((double)s->n / seg_len, (double)s->n / min_seg) /
                                                   cc.seg_div);
                // each segment adds one record the stitch walks per episode
                if (sparse) P = std::min(P, 512);
            }
            pl.ri[r] = RecInfo{s->d_type, s->d_time, s->n, nullptr, P, ks, rb, s->d_freq, s->d_toff, s->d_ttime};
            recinfo_lists(pl.ri[r], s);
            if (c > 0) {
                if (!sparse)
                    for (int cb = 0; cb < c; cb += K)
                        for (int p = 0; p < P; ++p) pl.items.push_back(WorkItem{r, ks + cb, std::min(K, c - cb), p});
                rb += (int64_t)c * P;
            }
        }
        pl.records = rb - recbase;
        // Records take kRecWords words per (episode, segment): keep a plan's
        // records within a quarter of the context's free budget by using
        // fewer segments (never fewer than one).
        const size_t free_b = ctx->budget > ctx->used.load() ? ctx->budget - ctx->used.load() : 0;
        const double cap = std::max<double>((double)pl.n_slots, (double)free_b / 4.0 / (kRecWords * 4.0));
        if (force_segments == 0 && (double)pl.records > cap) {
            const double f = cap / (double)pl.records;
            pl.items.clear();
            rb = recbase;
            for (int r = 0; r < n_recs; ++r) {
                const int ks = key_off[b * n_recs + r], c = key_off[b * n_recs + r + 1] - ks;
                const int P = std::max(1, (int)(pl.ri[r].P * f));
                pl.ri[r].P = P;
                pl.ri[r].recbase = rb;
                if (c > 0) {
                    if (!sparse)
                        for (int cb = 0; cb < c; cb += K)
                            for (int p = 0; p < P; ++p) pl.items.push_back(WorkItem{r, ks + cb, std::min(K, c - cb), p});
                    rb += (int64_t)c * P;
                }
            }
            pl.records = rb - recbase;
        }
        return pl;
    };
    // Uploads a plan's tables and launches its counting kernel (no stitch).
    // `limit` > 0 launches only that many work items / threads (autotuner).
    int64_t segpos = 0;
    size_t tabpos = 0;
    auto launch_plan = [&](Plan &pl, int32_t *rec_base, int64_t *d_seg, char *tab, RecInfo **d_ri_out,
                           int64_t limit) -> int {
        for (int r = 0; r < n_recs; ++r) {
            const int64_t *sg = nullptr;
            FEM_TRY(stream_segments(ctx, cc.recs[r], pl.ri[r].P, &sg));
            pl.ri[r].seg = sg;
            (void)d_seg;
        }
        RecInfo *d_ri = reinterpret_cast<RecInfo *>(tab + tabpos);
        tabpos += (pl.ri.size() * sizeof(RecInfo) + 255) & ~size_t(255);
        FEM_CUDA_TRY(cudaMemcpyAsync(d_ri, pl.ri.data(), pl.ri.size() * sizeof(RecInfo), cudaMemcpyHostToDevice,
                                     ctx->stream));
        *d_ri_out = d_ri;
        if (pl.track) {
            // per-warp entry lists: 4 x (longest per-type list) words each;
            // fewer resident warps when that would pass a quarter of the
            // free budget
            const int64_t cap = track_cap;
            int blocks = track_nblocks;
            const int64_t n_items = limit > 0 ? std::min(limit, pl.records) : pl.records;
            blocks = (int)std::max<int64_t>(1, std::min<int64_t>(blocks, (n_items + kTrackWarps - 1) / kTrackWarps));
            void *pb = nullptr;
            FEM_TRY(scratch(ctx, kSlotTrack, track_buf_bytes(blocks, cap) + 256, &pb));
            TrackArgs ta{};
            ta.rinfo = d_ri;
            ta.n_recs = n_recs;
            ta.rec_first = pl.ri.empty() ? 0 : pl.ri[0].recbase;
            ta.n_items = n_items;
            ta.d_n_items = nullptr;
            if (limit == 0) {
                // items: recordings longest first; episodes sharing their
                // first N-1 nodes track that prefix once (kernel 7: one item
                // per episode and segment)
                const int64_t ns = pl.n_slots;
                const size_t gw = (size_t)(ns + 2) * 2 + (size_t)(ns + 2) / 1024 + 2 + 2 * (size_t)n_recs;
                void *pg = nullptr;
                FEM_TRY(scratch(ctx, kSlotTrackGrp, gw * 4 + (size_t)(n_recs + 2) * 8 + 1024, &pg));
                int64_t *i64 = static_cast<int64_t *>(pg);
                int32_t *i32 = reinterpret_cast<int32_t *>(i64 + n_recs + 2);
                std::vector<int32_t> ro(n_recs);
                std::iota(ro.begin(), ro.end(), 0);
                std::stable_sort(ro.begin(), ro.end(), [&](int x, int y) { return cc.recs[x]->n > cc.recs[y]->n; });
                int32_t *d_ro = i32 + 2 * (ns + 2) + n_recs + (ns + 2) / 1024 + 2;
                FEM_CUDA_TRY(cudaMemcpyAsync(d_ro, ro.data(), 4 * n_recs, cudaMemcpyHostToDevice, ctx->stream));
                TrackGroupIn gi{};
                gi.slot2cand = d_perm;
                gi.d_n_slots = nullptr;
                gi.n_slots_cap = ns;
                gi.offs = cc.offs;
                gi.ctypes = cc.types;
                gi.clo = cc.lo;
                gi.chi = cc.hi;
                gi.cand_rec = cc.cand_rec;
                gi.rinfo = d_ri;
                gi.n_recs = n_recs;
                gi.rorder = d_ro;
                gi.ibase = i64;
                gi.n_items = i64 + n_recs + 1;
                gi.gidx = i32;
                gi.gstart = i32 + (ns + 2);
                gi.gfirst = i32 + 2 * (ns + 2);
                gi.scan_tmp = i32 + 2 * (ns + 2) + n_recs;
                const bool grouped = ctx->tuning.kernel != 7;
                FEM_TRY(track_groups(ctx->stream, ctx->n_sm, gi, grouped, &ta));
                cc.stats.kernel_launches += grouped ? 4 : 1;
            }
            ta.offs = cc.offs;
            ta.ctypes = cc.types;
            ta.clo = cc.lo;
            ta.chi = cc.hi;
            ta.slot2cand = d_perm;
            ta.relaxed = cc.mode == 2;
            ta.skip = nullptr;
            ta.queue = reinterpret_cast<unsigned long long *>(mb + o_q);
            ta.buf = reinterpret_cast<int32_t *>(static_cast<char *>(pb) + 256);
            ta.cap = cap;
            ta.rec = rec_base;
            ta.counts = limit > 0 ? nullptr : cc.counts;  // unsegmented episodes: counts written directly
            ta.last_mode = ctx->tuning.track_last;
            FEM_TRY(launch_track(ctx->stream, blocks, ta));
            cc.stats.kernel_launches += 2;  // queue reset + kernel
            return FEM_OK;
        }
        if (pl.sparse) {
            SparseArgs sa{};
            sa.rinfo = d_ri;
            sa.n_recs = n_recs;
            sa.rec_first = pl.ri.empty() ? 0 : pl.ri[0].recbase;
            sa.n_threads = limit > 0 ? std::min(limit, pl.records) : pl.records;
            sa.offs = cc.offs;
            sa.ctypes = cc.types;
            sa.clo = cc.lo;
            sa.chi = cc.hi;
            sa.slot2cand = d_perm;
            sa.relaxed = cc.mode == 2;
            sa.rec = rec_base;
            sa.R = pl.R;
            const int rr = reg_ring_for(pl.nclass, pl.R);
            SparseFn f = sparse_fn(pl.nclass, rr);
            if (!f) return FEM_ERR_CUDA;
            const int bs = rr ? 128 : 64;
            // shared-memory rings sized per node inside a slab per thread;
            // episodes whose rings exceed the slab fall back (flagged)
            const int slab = std::max(2, std::min(pl.slab, 128));
            sa.dens = reinterpret_cast<const uint32_t *const *>(mb + o_dp);
            sa.lo_vals = reinterpret_cast<const int32_t *>(mb + o_lo);
            sa.n_lo = (int)lov.size();
            sa.slab = slab;
            if (!rr && ctx->tuning.kernel != 3) {
                // node-uniform variant (rings and per-node data in shared memory)
                SparseUFn fu = sparse_u_fn(pl.nclass);
                const size_t smu = sparse_u_smem(nmax_of_class(pl.nclass), slab);
                if (smu > 48 * 1024 &&
                    cudaFuncSetAttribute((const void *)fu, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smu) !=
                        cudaSuccess)
                    return FEM_ERR_CUDA;
                if (sa.n_threads > 0) fu<<<(unsigned)((sa.n_threads + 63) / 64), 64, smu, ctx->stream>>>(sa);
                FEM_CUDA_TRY(cudaGetLastError());
                cc.stats.kernel_launches++;
                return FEM_OK;
            }
            const size_t sm = rr ? 0 : (size_t)2 * slab * 64 * 4;
            if (sm > 48 * 1024 &&
                cudaFuncSetAttribute((const void *)f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
                return FEM_ERR_CUDA;
            if (sa.n_threads > 0) f<<<(unsigned)((sa.n_threads + bs - 1) / bs), bs, sm, ctx->stream>>>(sa);
            FEM_CUDA_TRY(cudaGetLastError());
            cc.stats.kernel_launches++;
            return FEM_OK;
        }
        WorkItem *d_items = reinterpret_cast<WorkItem *>(tab + tabpos);
        tabpos += (pl.items.size() * sizeof(WorkItem) + 255) & ~size_t(255);
        FEM_CUDA_TRY(cudaMemcpyAsync(d_items, pl.items.data(), pl.items.size() * sizeof(WorkItem),
                                     cudaMemcpyHostToDevice, ctx->stream));
        TiledArgs ta{};
        ta.rinfo = d_ri;
        ta.items = d_items;
        ta.offs = cc.offs;
        ta.ctypes = cc.types;
        ta.clo = cc.lo;
        ta.chi = cc.hi;
        ta.slot2cand = d_perm;
        ta.R = pl.R;
        ta.K = pl.K;
        ta.T = pl.T;
        ta.relaxed = cc.mode == 2;
        ta.small_alpha = small_alpha ? 1 : 0;
        ta.wait_polls = (uint32_t)ctx->tuning.wait_polls;
        ta.rec = rec_base;
        ta.status = ctx->d_status;
        const int64_t n_items = limit > 0 ? std::min<int64_t>(limit, pl.items.size()) : (int64_t)pl.items.size();
        FEM_TRY(launch_tiled(ctx, pl.nclass, (int)n_items, pl.K, pl.R, pl.T, ta));
        cc.stats.kernel_launches++;
        return FEM_OK;
    };
    // Per-plan scratch sizes (tables and segments) for a plan.
    auto tab_need = [&](const Plan &pl) {
        return pl.items.size() * sizeof(WorkItem) + pl.ri.size() * sizeof(RecInfo) + 512;
    };
    auto seg_need = [&](const Plan &pl) {
        int64_t t = 0;
        for (auto &r : pl.ri) t += r.P + 1;
        return t;
    };
    // Work units a plan launches (tiled: CTAs; sparse: threads) and a sample
    // of about two waves for timing trials.
    auto units_of = [&](const Plan &pl) { return pl.sparse ? pl.records : (int64_t)pl.items.size(); };
    auto sample_of = [&](const Plan &pl) -> int64_t {
        if (pl.sparse) return (int64_t)2 * ctx->n_sm * 2048;
        const size_t sm = tiled_smem_rt(pl.nclass, pl.K, pl.R, pl.T);
        return (int64_t)2 * ctx->n_sm * occupancy_tiled(pl.nclass, pl.K, pl.R, sm);
    };

    std::vector<Plan> plans;
    std::vector<int> plain_buckets, n1_buckets;
    int64_t records_needed = 0;
    for (int b = 0; b < kBuckets; ++b) {
        const int sb = key_off[b * n_recs], se = key_off[(b + 1) * n_recs];
        if (se <= sb) continue;
        if (b == kBucketN1) {
            n1_buckets.push_back(b);
            continue;
        }
        if (b == kBucketPlain) {
            plain_buckets.push_back(b);
            continue;
        }
        if (track && b == 0) {
            // local tracking: one plan, every multi-node episode; the tuner
            // chooses the segment-count multiplier
            double seg_mult = 1.0;
            const bool tunable_t = force_segments == 0 && cc.seg_div == 1.0 && ctx->tuning.segments == 0;
            if (tunable_t) {
                int64_t nmax_ev = 0;
                for (int r = 0; r < n_recs; ++r)
                    if (key_off[b * n_recs + r + 1] > key_off[b * n_recs + r]) nmax_ev = std::max(nmax_ev, cc.recs[r]->n);
                const std::string key = tune_key(kTuneTrack, 0, key_off[n_recs], nmax_ev, n_recs);
                TuneVal tv;
                if (tune_lookup(ctx, key, &tv)) {
                    seg_mult = tv.seg_mult;
                } else if (ctx->tuning.autotune == 1) {
                    float best = -1.f;
                    for (double m : {1.0, 0.25, 4.0}) {
                        Plan pl = make_plan(b, true, 32, T_def, m, 0);
                        void *pr = nullptr, *ps = nullptr, *pt = nullptr;
                        FEM_TRY(scratch(ctx, kSlotRecords, (size_t)std::max<int64_t>(pl.records, 1) * kRecWords * 4, &pr));
                        FEM_TRY(scratch(ctx, kSlotSeg, sizeof(int64_t) * seg_need(pl), &ps));
                        FEM_TRY(scratch(ctx, kSlotRecTab, tab_need(pl), &pt));
                        segpos = 0;
                        tabpos = 0;
                        RecInfo *dri = nullptr;
                        const int64_t lim = std::min<int64_t>(pl.records, (int64_t)2 * track_nblocks * kTrackWarps);
                        cudaEventRecord(ctx->ev0, ctx->stream);
                        FEM_TRY(launch_plan(pl, static_cast<int32_t *>(pr), static_cast<int64_t *>(ps),
                                            static_cast<char *>(pt), &dri, lim));
                        cudaEventRecord(ctx->ev1, ctx->stream);
                        FEM_CUDA_TRY(cudaEventSynchronize(ctx->ev1));
                        float ms = 0.f;
                        cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
                        const float cost = ms * (float)((double)pl.records / (double)std::max<int64_t>(lim, 1));
                        if (best < 0.f || cost < best) best = cost, seg_mult = m;
                    }
                    tune_store(ctx, key, TuneVal{32, 256, seg_mult, 3});
                }
            }
            Plan pl = make_plan(b, true, 32, T_def, seg_mult, records_needed);
            records_needed += pl.records;
            plans.push_back(std::move(pl));
            continue;
        }
        const int nclass = b / kBucketRing;
        const int R = std::max(bmax[b], 2);
        // the sparse kernel needs register rings and per-type lists
        bool sparse_ok = sparse_fn(nclass, reg_ring_for(nclass, R)) != nullptr && !cc.force_tiled;
        for (int r = 0; r < n_recs && sparse_ok; ++r)
            if (key_off[b * n_recs + r + 1] > key_off[b * n_recs + r] && cc.recs[r]->n_types > 8192)
                sparse_ok = false;
        // cost model: the tiled warp pays for every event whose type one of
        // its lanes uses (~64 issue slots each) plus the filter scan; a sparse
        // warp pays for the longest merged list among its lanes
        double nbar = 0;
        for (int r = 0; r < n_recs; ++r)
            if (key_off[b * n_recs + r + 1] > key_off[b * n_recs + r]) nbar = std::max(nbar, (double)cc.recs[r]->n);
        const double groups = std::ceil((se - sb) / 32.0);
        const double cost_dense = (double)units_h[b] * 64.0 + groups * nbar / 32.0 * 12.0;
        const double cost_sparse = (double)units_h[kBuckets + b] * (4.0 * nmax_of_class(nclass) + 40.0);
        bool sparse = sparse_ok && cost_sparse < cost_dense;
        if (ctx->tuning.kernel == 1) sparse = false;
        if (ctx->tuning.kernel >= 2) sparse = sparse_ok;
        // lanes per CTA: up to 256, but no wider than the bucket needs
        int K = ctx->tuning.lanes_per_cta > 0 ? ctx->tuning.lanes_per_cta : std::min(256, ((se - sb) + 31) / 32 * 32);
        int T = T_def;
        double seg_mult = 1.0;
        const bool tunable = force_segments == 0 && cc.seg_div == 1.0 && ctx->tuning.lanes_per_cta == 0 &&
                             ctx->tuning.segments == 0 && ctx->tuning.tile_events == 0 && ctx->tuning.kernel == 0;
        if (tunable) {
            int64_t nmax_ev = 0;
            for (int r = 0; r < n_recs; ++r)
                if (key_off[b * n_recs + r + 1] > key_off[b * n_recs + r]) nmax_ev = std::max(nmax_ev, cc.recs[r]->n);
            const std::string key = tune_key(nclass, b % kBucketRing, se - sb, nmax_ev, n_recs);
            TuneVal tv;
            if (tune_lookup(ctx, key, &tv)) {
                K = tv.K;
                T = tv.T;
                seg_mult = tv.seg_mult;
                sparse = (tv.kernel == 2) && sparse_ok;
            } else if (ctx->tuning.autotune == 1) {
                // Coordinate search; each trial times about two waves of the
                // bucket's work and scales to the whole launch.
                if (sparse_ok)
                    for (int r = 0; r < n_recs; ++r)
                        if (key_off[b * n_recs + r + 1] > key_off[b * n_recs + r])
                            FEM_TRY(stream_bytype(ctx, cc.recs[r]));
                auto trial = [&](bool sp, int k, int t, double m, float *cost) -> int {
                    Plan pl = make_plan(b, sp, k, t, m, 0);
                    void *pr = nullptr, *ps = nullptr, *pt = nullptr;
                    FEM_TRY(scratch(ctx, kSlotRecords, (size_t)std::max<int64_t>(pl.records, 1) * kRecWords * 4, &pr));
                    FEM_TRY(scratch(ctx, kSlotSeg, sizeof(int64_t) * seg_need(pl), &ps));
                    FEM_TRY(scratch(ctx, kSlotRecTab, tab_need(pl), &pt));
                    segpos = 0;
                    tabpos = 0;
                    RecInfo *dri = nullptr;
                    const int64_t lim = std::min(units_of(pl), sample_of(pl));
                    cudaEventRecord(ctx->ev0, ctx->stream);
                    FEM_TRY(launch_plan(pl, static_cast<int32_t *>(pr), static_cast<int64_t *>(ps),
                                        static_cast<char *>(pt), &dri, lim));
                    cudaEventRecord(ctx->ev1, ctx->stream);
                    FEM_CUDA_TRY(cudaEventSynchronize(ctx->ev1));
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
                    *cost = ms * (float)((double)units_of(pl) / (double)std::max<int64_t>(lim, 1));
                    return FEM_OK;
                };
                const int kmax = std::min(256, ((se - sb) + 31) / 32 * 32);
                float best = 0.f;
                FEM_TRY(trial(false, K, T, seg_mult, &best));
                for (int k : {32, 64, 128, 256}) {
                    if (k > kmax || k == K) continue;
                    float c;
                    FEM_TRY(trial(false, k, T, seg_mult, &c));
                    if (c < best) best = c, K = k;
                }
                for (int t : {512, 2048}) {
                    float c;
                    FEM_TRY(trial(false, K, t, seg_mult, &c));
                    if (c < best) best = c, T = t;
                }
                for (double m : {0.5, 2.0}) {
                    float c;
                    FEM_TRY(trial(false, K, T, m, &c));
                    if (c < best) best = c, seg_mult = m;
                }
                sparse = false;
                if (sparse_ok) {
                    double sm_best = 1.0;
                    float cs = 0.f;
                    FEM_TRY(trial(true, K, T, 1.0, &cs));
                    for (double m : {0.25, 4.0}) {
                        float c;
                        FEM_TRY(trial(true, K, T, m, &c));
                        if (c < cs) cs = c, sm_best = m;
                    }
                    if (cs < best) {
                        sparse = true;
                        seg_mult = sm_best;
                    }
                }
                tune_store(ctx, key, TuneVal{K, T, seg_mult, sparse ? 2 : 1});
            }
        }
        // the per-type lists cost 4 B per event (plus 8 B transient): without
        // room for them the tiled kernel does the work
        for (int r = 0; r < n_recs && sparse; ++r)
            if (key_off[b * n_recs + r + 1] > key_off[b * n_recs + r]) {
                const int sb2 = stream_bytype(ctx, cc.recs[r]);
                if (sb2 == FEM_ERR_NOMEM)
                    sparse = false;
                else if (sb2 != FEM_OK)
                    return sb2;
            }
        Plan pl = make_plan(b, sparse, K, T, seg_mult, records_needed);
        records_needed += pl.records;
        plans.push_back(std::move(pl));
    }
    // records + segments scratch
    void *p_rec = nullptr;
    if (records_needed > 0) FEM_TRY(scratch(ctx, kSlotRecords, (size_t)records_needed * kRecWords * 4, &p_rec));
    int64_t seg_total = 0;
    size_t tab_bytes = 0;
    for (auto &pl : plans) {
        seg_total += seg_need(pl);
        tab_bytes += tab_need(pl);
    }
    void *p_seg = nullptr;
    FEM_TRY(scratch(ctx, kSlotSeg, sizeof(int64_t) * std::max<int64_t>(seg_total, 1), &p_seg));
    int64_t *d_seg = static_cast<int64_t *>(p_seg);
    void *p_tab = nullptr;
    FEM_TRY(scratch(ctx, kSlotRecTab, std::max<size_t>(tab_bytes, 256), &p_tab));
    char *tab = static_cast<char *>(p_tab);
    segpos = 0;
    tabpos = 0;
    int32_t *fb_list = nullptr;
    void *p_fb = nullptr;
    FEM_TRY(scratch(ctx, kSlotFallback, sizeof(int32_t) * std::max<int64_t>(n_work, 1), &p_fb));
    fb_list = static_cast<int32_t *>(p_fb);
    int *d_fbc = reinterpret_cast<int *>(mb + o_fb);
    const RecInfo *d_ri_plain = reinterpret_cast<const RecInfo *>(mb + o_ri);

    cudaEventRecord(ctx->ev0, ctx->stream);
    for (auto &pl : plans) {
        RecInfo *d_ri = nullptr;
        FEM_TRY(launch_plan(pl, static_cast<int32_t *>(p_rec), d_seg, tab, &d_ri, 0));
        if (pl.sparse)
            cc.stats.sparse_launches++;
        int maxP = 1;
        for (auto &r : pl.ri) maxP = std::max(maxP, r.P);
        // local tracking wrote the counts of unsegmented episodes itself
        if (!(pl.track && maxP == 1)) {
            k_stitch<<<(pl.n_slots + kStitchWarps - 1) / kStitchWarps, kStitchWarps * 32, 0, ctx->stream>>>(
                static_cast<int32_t *>(p_rec), d_ri, d_perm, cc.cand_rec, pl.slot_begin, pl.n_slots, cc.counts,
                fb_list, d_fbc, nullptr, kStitchSplit, nullptr, nullptr, pl.track ? 1 : 0);
            cc.stats.kernel_launches++;
        }
        if (maxP > kStitchSplit) {
            k_stitch_block<<<(unsigned)std::min<int64_t>(pl.n_slots, (int64_t)ctx->n_sm * 4), kStitchBlock, 0,
                             ctx->stream>>>(static_cast<int32_t *>(p_rec), d_ri, d_perm, cc.cand_rec, pl.slot_begin,
                                            pl.n_slots, cc.counts, fb_list, d_fbc, nullptr, kStitchSplit);
            cc.stats.kernel_launches++;
        }
        FEM_CUDA_TRY(cudaGetLastError());
    }
    cudaEventRecord(ctx->ev1, ctx->stream);
    for (int b : n1_buckets) {
        const int sb = key_off[b * n_recs], se = key_off[(b + 1) * n_recs];
        k_count_n1<<<(se - sb + 255) / 256, 256, 0, ctx->stream>>>(d_perm, sb, se - sb, cc.offs, cc.types,
                                                                   cc.cand_rec, d_ri_plain, cc.counts);
        cc.stats.kernel_launches++;
    }
    for (int b : plain_buckets) {
        const int sb = key_off[b * n_recs], se = key_off[(b + 1) * n_recs];
        const int R = std::max(bmax[b], 2);
        void *p_rings = nullptr;
        const int maxN = std::max(bmax[kBuckets + b], 2);
        FEM_TRY(scratch(ctx, kSlotRings, (size_t)(se - sb) * (maxN - 1) * (size_t)R * 4, &p_rings));
        k_count_plain<<<(se - sb + 127) / 128, 128, 0, ctx->stream>>>(
            d_ri_plain, d_perm, cc.cand_rec, sb, se - sb, cc.offs, cc.types, cc.lo, cc.hi, R,
            static_cast<int32_t *>(p_rings), cc.counts, ctx->d_status);
        cc.stats.kernel_launches++;
        FEM_CUDA_TRY(cudaGetLastError());
    }
    int fbc = 0;
    FEM_CUDA_TRY(cudaMemcpyAsync(&fbc, d_fbc, 4, cudaMemcpyDeviceToHost, ctx->stream));
    FEM_TRY(sync_status(ctx));
    if (!plans.empty()) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
        cc.count_ms += ms;
    }
    cc.stats.candidates_counted += n_work - fbc;
    if (fbc > 0) {
        // Exact recount of the episodes whose machines ran out of entry
        // classes at some segment boundary.
        cc.stats.fallback_recounts += fbc;
        void *p_sub = nullptr;
        FEM_TRY(scratch(ctx, kSlotScanTmp, sizeof(int32_t) * fbc, &p_sub));
        FEM_CUDA_TRY(cudaMemcpyAsync(p_sub, fb_list, sizeof(int32_t) * fbc, cudaMemcpyDeviceToDevice, ctx->stream));
        // the sub-call reuses the scratch slots, so keep its subset elsewhere
        std::vector<int32_t> hsub(fbc);
        FEM_CUDA_TRY(cudaMemcpyAsync(hsub.data(), p_sub, sizeof(int32_t) * fbc, cudaMemcpyDeviceToHost, ctx->stream));
        FEM_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
        void *p_keep = nullptr;
        FEM_TRY(dev_alloc(ctx, &p_keep, sizeof(int32_t) * fbc));
        cudaMemcpyAsync(p_keep, hsub.data(), sizeof(int32_t) * fbc, cudaMemcpyHostToDevice, ctx->stream);
        // Each round divides the segment count by 8 (fewer boundaries, so
        // fewer entry classes); after a few rounds a single segment remains,
        // which never needs more than one class.
        // The last round runs the tiled kernel on one segment, where neither
        // entry classes nor rings (sized from the stream's densities) can
        // overflow.
        const double saved = cc.seg_div;
        const bool saved_ft = cc.force_tiled;
        cc.seg_div *= 8.0;
        const bool last = cc.seg_div >= 4096.0;
        if (last) cc.force_tiled = true;
        const int st = count_core(cc, static_cast<int32_t *>(p_keep), fbc, last ? 1 : 0);
        cc.seg_div = saved;
        cc.force_tiled = saved_ft;
        cudaStreamSynchronize(ctx->stream);
        dev_free(ctx, p_keep, sizeof(int32_t) * fbc);
        return st;
    }
    return FEM_OK;
}

constexpr int64_t kPltMaxCands = 256;        // automatic local tracking: at most this many episodes
constexpr int64_t kPltMinEvents = 1 << 20;   // ... over a recording of at least this many events

static int run_count(CountCall &cc, const int32_t *subset, int64_t n_sub, int force_segments) {
    // node-by-node local tracking (fem_plt.cu): when asked for, or for few
    // episodes over long recordings (its steps are parallel over the events
    // of the episodes' node types; the per-episode kernels need many
    // episodes, or many segments with their halos and records, to fill the
    // GPU)
    const int kern = cc.ctx->tuning.kernel;
    bool plt = kern >= 4;
    if (cc.ctx->tuning.kernel == 0 && n_sub <= kPltMaxCands) {
        int64_t nmax = 0;
        bool lists = true;
        for (auto *r : cc.recs) {
            nmax = std::max(nmax, r->n);
            lists = lists && r->n_types <= 8192 && r->n <= INT32_MAX / 2;
        }
        plt = lists && nmax >= kPltMinEvents;
    }
    if (cc.mode != 1 && force_segments == 0 && plt) {
        std::vector<int32_t> work(n_sub);
        if (subset) {
            FEM_CUDA_TRY(cudaMemcpyAsync(work.data(), subset, 4 * n_sub, cudaMemcpyDeviceToHost, cc.ctx->stream));
            FEM_CUDA_TRY(cudaStreamSynchronize(cc.ctx->stream));
        } else {
            for (int64_t i = 0; i < n_sub; ++i) work[i] = (int32_t)i;
        }
        FEM_TRY(count_plt(cc.ctx, cc.recs, cc.offs, cc.types, cc.lo, cc.hi, cc.cand_rec, work, cc.mode == 2,
                          cc.counts, &cc.stats, &cc.count_ms, kern >= 5 ? kern - 4 : 0));
        return sync_status(cc.ctx);
    }
    return count_core(cc, subset, n_sub, force_segments);
}

// Copies (or aliases) the candidate CSR to the device and collects the
// distinct lower bounds.
static int stage_candidates(fem_ctx *ctx, const fem_cands *c, CountCall &cc, const uint32_t *rec_id,
                            int n_recs) {
    const int64_t n = c->n_cand;
    int64_t n_nodes = 0;
    if (c->ptr_is_device) {
        FEM_CUDA_TRY(cudaMemcpyAsync(&n_nodes, c->offs + n, 8, cudaMemcpyDeviceToHost, ctx->stream));
        FEM_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    } else {
        if (c->offs[0] != 0) return FEM_ERR_INVAL;
        for (int64_t i = 0; i < n; ++i)
            if (c->offs[i + 1] <= c->offs[i] || c->offs[i + 1] - c->offs[i] > FEM_MAX_NODES) return FEM_ERR_INVAL;
        n_nodes = c->offs[n];
    }
    if (n_nodes < n || n_nodes > (int64_t)n * FEM_MAX_NODES) return FEM_ERR_INVAL;
    const int64_t n_edges = n_nodes - n;
    std::vector<int32_t> lo_h;
    if (c->ptr_is_device) {
        cc.offs = c->offs;
        cc.types = c->types;
        cc.lo = c->lo;
        cc.hi = c->hi;
        lo_h.resize(n_edges);
        if (n_edges > 0) {
            FEM_CUDA_TRY(cudaMemcpyAsync(lo_h.data(), c->lo, 4 * n_edges, cudaMemcpyDeviceToHost, ctx->stream));
            FEM_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
        }
        if (rec_id) cc.cand_rec = rec_id;
    } else {
        void *p1, *p2, *p3, *p4;
        FEM_TRY(scratch(ctx, kSlotCandOffs, 8 * (n + 1), &p1));
        FEM_TRY(scratch(ctx, kSlotCandTypes, 2 * std::max<int64_t>(n_nodes, 1), &p2));
        FEM_TRY(scratch(ctx, kSlotCandLo, 4 * std::max<int64_t>(n_edges, 1), &p3));
        FEM_TRY(scratch(ctx, kSlotCandHi, 4 * std::max<int64_t>(n_edges, 1), &p4));
        FEM_TRY(copy_in(ctx, p1, c->offs, 8 * (n + 1), 0));
        FEM_TRY(copy_in(ctx, p2, c->types, 2 * n_nodes, 0));
        FEM_TRY(copy_in(ctx, p3, c->lo, 4 * n_edges, 0));
        FEM_TRY(copy_in(ctx, p4, c->hi, 4 * n_edges, 0));
        cc.offs = static_cast<int64_t *>(p1);
        cc.types = static_cast<uint16_t *>(p2);
        cc.lo = static_cast<int32_t *>(p3);
        cc.hi = static_cast<int32_t *>(p4);
        lo_h.assign(c->lo, c->lo + n_edges);
        if (rec_id) {
            for (int64_t i = 0; i < n; ++i)
                if (rec_id[i] >= (uint32_t)n_recs) return FEM_ERR_INVAL;
            void *p5;
            FEM_TRY(scratch(ctx, kSlotCandRec, 4 * n, &p5));
            FEM_TRY(copy_in(ctx, p5, rec_id, 4 * n, 0));
            cc.cand_rec = static_cast<uint32_t *>(p5);
        }
    }
    std::set<int32_t> los(lo_h.begin(), lo_h.end());
    cc.lo_vals.assign(los.begin(), los.end());
    return FEM_OK;
}

static int count_entry(fem_ctx *ctx, const fem_stream *const *recs, int n_recs, const fem_cands *c,
                       const uint32_t *rec_id, uint32_t *counts, int out_is_device, int mode) {
    if (!ctx || !recs || n_recs < 1 || !c || c->n_cand < 0 || (c->n_cand > 0 && (!counts || !c->offs)))
        return FEM_ERR_INVAL;
    if (c->n_cand > INT32_MAX / 2) return FEM_ERR_INVAL;
    for (int r = 0; r < n_recs; ++r)
        if (!recs[r] || recs[r]->ctx != ctx) return FEM_ERR_INVAL;
    if (n_recs > 1 && !rec_id) return FEM_ERR_INVAL;
    std::lock_guard<std::mutex> g(ctx->mu);
    cudaSetDevice(ctx->device);
    const double t0 = now_s();
    CountCall cc;
    cc.ctx = ctx;
    cc.mode = mode;
    for (int r = 0; r < n_recs; ++r) cc.recs.push_back(const_cast<fem_stream *>(recs[r]));
    cc.n_cand = c->n_cand;
    if (c->n_cand == 0) {
        ctx->last = fem_stats{};
        return FEM_OK;
    }
    if (!c->types || !c->lo || !c->hi) return FEM_ERR_INVAL;
    FEM_TRY(stage_candidates(ctx, c, cc, n_recs > 1 ? rec_id : nullptr, n_recs));
    void *pc = nullptr;
    FEM_TRY(scratch(ctx, kSlotCounts, 4 * c->n_cand, &pc));
    cc.counts = static_cast<uint32_t *>(pc);
    FEM_TRY(run_count(cc, nullptr, c->n_cand, 0));
    FEM_TRY(copy_out(ctx, counts, cc.counts, 4 * c->n_cand, out_is_device));
    FEM_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    cc.stats.episode_events = cc.stats.counted_episode_events;
    cc.stats.count_kernel_ms = cc.count_ms;
    cc.stats.total_ms = (now_s() - t0) * 1e3;
    ctx->last = cc.stats;
    return FEM_OK;
}

// Counting of device-resident candidates (used by the level-wise miner).
int count_device(fem_ctx *ctx, const std::vector<fem_stream *> &recs, int64_t n_cand, const int64_t *offs,
                 const uint16_t *types, const int32_t *lo, const int32_t *hi, const uint32_t *cand_rec,
                 const std::vector<int32_t> &lo_vals, const int32_t *order, int64_t n_order, uint32_t *counts,
                 fem_stats *stats) {
    CountCall cc;
    cc.ctx = ctx;
    cc.recs = recs;
    cc.mode = ctx->tuning.plain_path == 1 ? 1 : 0;
    cc.n_cand = n_cand;
    cc.offs = offs;
    cc.types = types;
    cc.lo = lo;
    cc.hi = hi;
    cc.cand_rec = cand_rec;
    cc.counts = counts;
    cc.lo_vals = lo_vals;
    // `order` (optional) lists every candidate once, in the order the
    // counting kernels should hold them (lane neighbours share types).
    const int64_t n_work = order ? n_order : n_cand;
    if (n_work > 0) FEM_TRY(run_count(cc, order, n_work, 0));
    cc.stats.count_kernel_ms = cc.count_ms;
    *stats = cc.stats;
    return FEM_OK;
}

}  // namespace fem

using namespace fem;

extern "C" int fem_count_episodes(fem_ctx *ctx, const fem_stream *s, const fem_cands *c, uint32_t *counts,
                                  int out_is_device) {
    const fem_stream *recs[1] = {s};
    return count_entry(ctx, recs, 1, c, nullptr, counts, out_is_device, 0);
}

extern "C" int fem_count_batch(fem_ctx *ctx, const fem_stream *const *recs, int n_recs, const fem_cands *c,
                               const uint32_t *rec_id, uint32_t *counts, int out_is_device) {
    return count_entry(ctx, recs, n_recs, c, rec_id, counts, out_is_device, 0);
}

extern "C" int fem_count_episodes_plain(fem_ctx *ctx, const fem_stream *s, const fem_cands *c,
                                        uint32_t *counts, int out_is_device) {
    const fem_stream *recs[1] = {s};
    return count_entry(ctx, recs, 1, c, nullptr, counts, out_is_device, 1);
}

extern "C" int fem_upper_bound(fem_ctx *ctx, const fem_stream *s, const fem_cands *c, uint32_t *ub,
                               int out_is_device) {
    const fem_stream *recs[1] = {s};
    return count_entry(ctx, recs, 1, c, nullptr, ub, out_is_device, 2);
}
