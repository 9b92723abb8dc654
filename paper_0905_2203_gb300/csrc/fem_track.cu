// fem_track.cu -- exact counting by node-by-node local tracking, one warp per
// (episode, segment) work item, in one persistent launch fed by an atomic
// work queue.
//
// The count is the size of the largest set of non-overlapped occurrences,
// found by Algorithm 1 ("Problem decomposition") over end events, each with
// the LATEST start of an occurrence ending there:
//     L_1(j) = t_j,   L_k(j) = max { L_{k-1}(i) : lo < t_j - t_i <= hi }.
// Over the events of node k-1 that have a valid L (the node's entries), L is
// non-decreasing in time, so L_k(j) is the L of the newest entry older than
// t_j - lo, provided that entry is not older than t_j - hi.  Section
// "Parallel Local Tracking" tracks an episode node by node over the per-type
// event lists; here one warp does that for one work item:
//   * node k's events (its type's list, inside the segment and its halo) are
//     taken 32 at a time, one per lane, in time order;
//   * each lane finds its predecessor among node k-1's entries with a window
//     walk: the warp loads 32 consecutive entries, every lane ranks its own
//     query in them by a 5-step binary search over the lanes' registers, and
//     the window moves on until every lane has its rank; queries of a node
//     come in time order, so the window only moves forward;
//   * the lanes that found a valid predecessor append (t, L) to the node's
//     entry list in the warp's buffer (ballot + prefix count);
//   * at the last node the valid ends inside the segment are handed, in time
//     order, to Algorithm 1 for every entry class of the segment (the same
//     machine and record as the other counting kernels, so k_stitch composes
//     the segments; section "MapConcat").
// Every lane of the warp does the same work on the same list, so lanes stay
// converged, list reads are coalesced and no per-node ring is needed: the
// entry lists live in a per-warp global buffer of 4 x (longest list) words.
//
// The launch is persistent: each warp takes the next item index from a
// counter until the items run out, so items of very different lengths (long
// and short recordings, short and long episodes) balance across the GPU.
#include <algorithm>

#include "fem_internal.cuh"
#include "fem_machine.cuh"

namespace fem {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

// First i in [lo, hi) with v[i] >= q (hi if none), computed by the whole warp
// (every lane returns it): a 32-way search whose probes are one strided load.
__device__ __forceinline__ int64_t warp_lower_bound(const int32_t *__restrict__ v, int64_t lo, int64_t hi, int64_t q,
                                                    int lane) {
    while (hi - lo > 32) {
        const int64_t step = (hi - lo + 31) >> 5;
        const int64_t pos = lo + step * (lane + 1) - 1;
        const bool below = pos < hi && (int64_t)v[pos] < q;
        const int c = __popc(__ballot_sync(kFull, below));
        if (c == 32) return hi;
        // probe c is the first at or above q (or past hi): the answer lies
        // after probe c-1 and at or before probe c
        const int64_t pc = lo + step * (c + 1) - 1;
        lo = lo + step * c;
        hi = pc + 1 < hi ? pc + 1 : hi;
    }
    const int64_t pos = lo + lane;
    const bool below = pos < hi && (int64_t)v[pos] < q;
    return lo + __popc(__ballot_sync(kFull, below));
}

// Algorithm 1 over one chunk's valid ends (lane order = time order): the
// steady state jumps from selection to selection, otherwise every end goes
// through every entry class.
__device__ __forceinline__ void greedy_chunk(unsigned bm, int32_t t, int32_t Lv, Machine<2, 0> &st, int32_t Tp,
                                             int lane) {
    if (bm && !st.open && st.live == 1u) {
        // the next selection is the first later end whose latest start is
        // after the last selected end
        int32_t prev = st.cprev[0];
        uint32_t added = 0;
        for (;;) {
            const unsigned sel = __ballot_sync(kFull, ((bm >> lane) & 1u) && Lv > prev);
            if (!sel) break;
            const int b = __ffs(sel) - 1;
            prev = __shfl_sync(kFull, t, b);
            ++added;
            bm &= (b == 31) ? 0u : ~((2u << b) - 1u);
        }
        st.ccnt[0] += added;
        st.cprev[0] = prev;
    } else {
        while (bm) {
            const int b = __ffs(bm) - 1;
            bm &= bm - 1;
            st.greedy_end(__shfl_sync(kFull, t, b), __shfl_sync(kFull, Lv, b), Tp);
        }
    }
}

// Entries of node k-1 as one step sees them: node 0's are its type's event
// times (latest start = time); later nodes' are (time, latest start) pairs
// in the warp's buffer, so one 8-byte load brings both.
template <bool HASL>
struct Entries;
template <>
struct Entries<false> {
    const int32_t *__restrict__ t;
    __device__ __forceinline__ int2 get(int i) const {
        const int32_t v = t[i];
        return make_int2(v, v);
    }
};
template <>
struct Entries<true> {
    const int2 *__restrict__ e;
    __device__ __forceinline__ int2 get(int i) const { return e[i]; }
};

// One node step for one warp: node k's events ev[0, n_ev) (time order)
// against node k-1's entries p[0, m).  An event is valid when the newest
// entry older than t - lo exists and is not older than t - hi; its latest
// start is that entry's.  Not LAST: the valid events are appended to out as
// (t, L) and their number is returned.  LAST: the valid events at or after
// Tp are passed, in time order, to Algorithm 1 of every entry class in st.
//
// Each chunk of 32 events ranks its queries in windows of 32 entries that
// start one entry before the previous chunk's last rank and move on by 31:
// the first entry of every window is older than every query still looking,
// so a lane's predecessor is always in the window where its rank falls and
// its time and latest start are read from the window's registers by a
// shuffle.
template <bool LAST, bool HASL>
__device__ __forceinline__ int node_step(const int32_t *__restrict__ ev, int n_ev, Entries<HASL> p, int m,
                                         int32_t lo_e, int32_t hi_e, int2 *__restrict__ out, Machine<2, 0> &st,
                                         int32_t Tp, int lane) {
    // All positions fit 32 bits: a recording has fewer than 2^30 events.
    // Times are >= 0 and 0 <= lo < hi, so t - lo and t - hi stay in int32.
    int w = 0;   // entries below the previous chunk's last query
    int wc = 0;  // entries written
    int32_t t_next = lane < n_ev ? ev[lane] : INT32_MAX;
    for (int base = 0; base < n_ev; base += 32) {
        const bool in = base + lane < n_ev;
        const int32_t t = t_next;
        if (base + 32 < n_ev) t_next = (base + 32 + lane < n_ev) ? ev[base + 32 + lane] : INT32_MAX;
        const int32_t q = t - lo_e;
        const int32_t q0 = __shfl_sync(kFull, q, 0);
        int ws = w > 0 ? w - 1 : 0;
        int idx = 0;
        int32_t aT = INT32_MIN, aL = 0;
        bool done = !in;
        for (;;) {
            const int wi = ws + lane;
            const int2 v = wi < m ? p.get(wi) : make_int2(INT32_MAX, 0);
            const int32_t top = __shfl_sync(kFull, v.x, 31);
            if (top < q0 && ws + 32 < m) {  // the whole window precedes every query
                ws += 31;
                continue;
            }
            // rank of q among the window's times (ascending across lanes)
            int c = 0;
#pragma unroll
            for (int s = 16; s >= 1; s >>= 1)
                if (__shfl_sync(kFull, v.x, c + s - 1) < q) c += s;
            if (c == 31 && top < q) c = 32;
            const int src = c > 0 ? c - 1 : 0;
            const int32_t xt = __shfl_sync(kFull, v.x, src);
            const int32_t xl = HASL ? __shfl_sync(kFull, v.y, src) : xt;
            if (!done && c < 32) {
                idx = ws + c;
                aT = c > 0 ? xt : INT32_MIN;
                aL = xl;
                done = true;
            }
            if (__all_sync(kFull, done)) break;
            ws += 31;
        }
        const bool ok = in && aT != INT32_MIN && aT >= t - hi_e;
        const int32_t Lv = ok ? aL : 0;
        if (!LAST) {
            const unsigned bm = __ballot_sync(kFull, ok);
            if (ok) out[wc + __popc(bm & ((1u << lane) - 1u))] = make_int2(t, Lv);
            wc += __popc(bm);
        } else {
            greedy_chunk(__ballot_sync(kFull, ok && t >= Tp), t, Lv, st, Tp, lane);
        }
        // the next 32 queries rank at or after this chunk's last one
        w = __shfl_sync(kFull, idx, 31);
    }
    __syncwarp();
    return wc;
}

// The last node step driven by node N-2's entries instead of node N-1's
// events, for entry lists much shorter than the last node's event list.
//
// An end t of node N-1 takes the newest entry i with T_i < t - lo, so the
// ends served by entry i are those in (T_i + lo, T_{i+1} + lo]; they all
// carry L_i and are valid while t <= T_i + hi.  Within that interval only
// the first end (at or after Tp) can matter to Algorithm 1: L_i <= T_i < t,
// so once it has been offered every entry class has its last selection at or
// above L_i (it selected this end, or it could not), the largest latest start
// seen is at least L_i, and a later end with the same L_i changes no class.
// So per entry one lookup finds the first event at or after
// q = max(T_i + lo + 1, Tp), and the end is offered when it lies in the
// entry's interval and within its upper bound.
//
// The lookup uses the stream's per-type time index: the cell of q gives the
// list position of the first event at or after the cell's start, and a short
// forward scan (about one event of the type per cell) reaches the first event
// at or after q.  Lanes look up independently; the warp takes 32 x K entries
// at a time (entry base + 32 k + lane in lane k's k-th slot) and issues the
// K index loads of a lane, then its K list loads, side by side, so that each
// lane has K lookups in flight; then it offers the ends to Algorithm 1 slot
// by slot (time order).
//
// tl: the type's list; [cb, ce): the item's part of it; row: the type's
// index row (ncell + 1 cells of 2^shift ticks from tbase).
template <bool HASL, int K>
__device__ __forceinline__ void last_by_index(const int32_t *__restrict__ tl, int cb, int ce,
                                              const int32_t *__restrict__ row, int shift, uint32_t tbase,
                                              int64_t ncell, Entries<HASL> p, int m, int32_t lo_e, int32_t hi_e,
                                              Machine<2, 0> &st, int32_t Tp, int lane) {
    // Times are >= 0 and 0 <= lo < hi < 2^31, so every bound below fits an
    // unsigned 32-bit word except T_{i+1} + lo for a missing next entry.
    const uint32_t lo = (uint32_t)lo_e, hi = (uint32_t)hi_e, tp = (uint32_t)Tp;
    for (int base = 0; base < m; base += 32 * K) {
        int2 E[K];
#pragma unroll
        for (int k = 0; k < K; ++k) E[k] = base + 32 * k + lane < m ? p.get(base + 32 * k + lane) : make_int2(-1, 0);
        const int nx = base + 32 * K;
        // the first entry of the next chunk (its time bounds this chunk's
        // last interval)
        const uint32_t T_after = nx < m ? (uint32_t)p.get(nx).x : 0xFFFFFFFFu;
        // the K lookups of a lane side by side: index cell, then the first
        // event of the cell, then (rarely) a few more events
        uint32_t q[K], x[K];
        int pos[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            q[k] = (uint32_t)E[k].x + lo + 1u;
            if (q[k] < tp) q[k] = tp;
            const uint64_t c = q[k] > tbase ? (uint64_t)((q[k] - tbase) >> shift) : 0;
            pos[k] = base + 32 * k + lane < m ? row[c < (uint64_t)ncell ? c : (uint64_t)ncell] : ce;
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            if (pos[k] < cb) pos[k] = cb;
            x[k] = pos[k] < ce ? (uint32_t)tl[pos[k]] : 0xFFFFFFFFu;
        }
#pragma unroll
        for (int k = 0; k < K; ++k)
            while (x[k] < q[k]) {
                ++pos[k];
                x[k] = pos[k] < ce ? (uint32_t)tl[pos[k]] : 0xFFFFFFFFu;
            }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int i = base + 32 * k + lane;
            const uint32_t T = (uint32_t)E[k].x;
            // the next entry's time: the next lane's, the next slot's first,
            // or the next chunk's first
            uint32_t Tn = __shfl_down_sync(kFull, T, 1);
            const uint32_t Tf = k + 1 < K ? __shfl_sync(kFull, (uint32_t)E[k + 1 < K ? k + 1 : k].x, 0) : T_after;
            if (lane == 31) Tn = Tf;
            // x = the first event at or after q (none: past the item's part)
            const bool ok = i < m && pos[k] < ce && x[k] <= T + hi && (i + 1 >= m || x[k] <= Tn + lo);
            greedy_chunk(__ballot_sync(kFull, ok), (int32_t)x[k], ok ? E[k].y : 0, st, Tp, lane);
        }
    }
    __syncwarp();
}

__device__ __forceinline__ void machine_init(Machine<2, 0> &st, int N) {
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
}

// A work item is one segment p of one recording for either one episode
// (slot) or, with groups, a run of episode slots [s0, s1) that share their
// first N-1 nodes and edges: the shared prefix is tracked once, and only the
// last node step is run per episode.
__global__ void __launch_bounds__(kTrackWarps * 32, kTrackMaxBlocksPerSm) k_count_track(TrackArgs a) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    // two entry lists of (time, latest start) pairs, ping-pong
    int2 *const b0 = reinterpret_cast<int2 *>(a.buf + gw * 4 * a.cap);
    int2 *const b1 = b0 + a.cap;
    const int64_t n_items = a.d_n_items ? *a.d_n_items : a.n_items;
    for (;;) {
        unsigned long long it = 0;
        if (lane == 0) it = atomicAdd(a.queue, 1ull);
        it = __shfl_sync(kFull, it, 0);
        if ((int64_t)it >= n_items) break;
        int r = 0, P = 1, p = 0, s0 = 0, s1 = 0;
        if (a.ibase) {
            // items numbered recording by recording in the order rorder
            // (longest recordings first), each recording's groups (or
            // slots) times its segments
            int lo_r = 0, hi_r = a.n_recs;  // last position whose items start at or before it
            while (hi_r - lo_r > 1) {
                const int mid = (lo_r + hi_r) >> 1;
                if (a.ibase[mid] <= (int64_t)it) lo_r = mid; else hi_r = mid;
            }
            r = a.rorder ? a.rorder[lo_r] : lo_r;
            P = a.rinfo[r].P;
            const int64_t local = (int64_t)it - a.ibase[lo_r];
            const int64_t g = a.gfirst[r] + local / P;
            p = (int)(local % P);
            if (a.gstart) {
                s0 = a.gstart[g];
                s1 = a.gstart[g + 1];
            } else {
                s0 = (int)g;
                s1 = s0 + 1;
            }
        } else {
            const int64_t tr = a.rec_first + (int64_t)it;
            int lo_r = 0, hi_r = a.n_recs;  // last recording whose records start at or before tr
            while (hi_r - lo_r > 1) {
                const int mid = (lo_r + hi_r) >> 1;
                if (a.rinfo[mid].recbase <= tr) lo_r = mid; else hi_r = mid;
            }
            r = lo_r;
            P = a.rinfo[r].P;
            const int64_t local = tr - a.rinfo[r].recbase;
            s0 = a.rinfo[r].slot_first + (int)(local / P);
            s1 = s0 + 1;
            p = (int)(local % P);
        }
        const RecInfo &ri = a.rinfo[r];
        const int c0 = a.slot2cand[s0];
        const int64_t o0 = a.offs[c0];
        const int N = (int)(a.offs[c0 + 1] - o0);
        const int64_t eo0 = o0 - c0;
        // halo: the largest sum of upper bounds over the item's episodes
        int64_t sumhi = 0;
        for (int k = 0; k < N - 2; ++k) sumhi += a.chi[eo0 + k];
        int32_t hmax = 0;
        for (int s = s0; s < s1 && N >= 2; ++s) {
            const int c = a.slot2cand[s];
            hmax = max(hmax, a.chi[a.offs[c] - c + N - 2]);
        }
        sumhi += hmax;
        const int64_t seg_b = ri.seg[p], seg_e = ri.seg[p + 1];
        // (no prefix work when a bound dropped every episode of the item)
        bool kept = !a.skip;
        for (int s = s0 + lane; s < s1 && !kept; s += 32) kept = !a.skip[a.slot2cand[s]];
        const bool live = seg_b < seg_e && N >= 2 && __any_sync(kFull, kept);
        int32_t Tp = 0;
        int64_t haloT = INT64_MIN, Tend = INT64_MAX;
        if (live) {
            Tp = ri.time[seg_b];
            haloT = (p == 0) ? INT64_MIN : (int64_t)Tp - sumhi;
            Tend = (seg_e < ri.n) ? (int64_t)ri.time[seg_e] : INT64_MAX;
        }
        const int64_t *toff = ri.toff;
        const int32_t *ttime = ri.ttime;
        // list range of type E inside [haloT, Tend)
        auto range = [&](uint32_t E, int64_t &b, int64_t &e) {
            const int64_t b0 = toff[E], b1 = toff[E + 1];
            if (ri.tseg) {
                const int32_t *tq = ri.tseg + (size_t)E * ri.tstride;
                const int qmax = ri.tstride - 1;
                const int64_t st0 = b0 + tq[min(p * ri.sstep, qmax)];
                e = b0 + tq[min((p + 1) * ri.sstep, qmax)];
                b = (p == 0) ? st0 : warp_lower_bound(ttime, b0, st0, haloT, lane);
            } else {
                b = (p == 0) ? b0 : warp_lower_bound(ttime, b0, b1, haloT, lane);
                e = (seg_e < ri.n) ? warp_lower_bound(ttime, b, b1, Tend, lane) : b1;
            }
        };
        // shared prefix: node 0 (its type's times), then nodes 1..N-2
        // (entry lists in the warp's buffer)
        Entries<false> p0{nullptr};
        Entries<true> pe{nullptr};
        int m = 0;
        Machine<2, 0> st;
        if (live) {
            int64_t b = 0, e = 0;
            range(a.ctypes[o0], b, e);
            p0.t = ttime + b;
            m = (int)(e - b);
            for (int k = 1; k < N - 1 && m > 0; ++k) {
                int64_t cb = 0, ce = 0;
                range(a.ctypes[o0 + k], cb, ce);
                int2 *out = (k & 1) ? b1 : b0;
                const int32_t lo_k = a.relaxed ? 0 : a.clo[eo0 + k - 1], hi_k = a.chi[eo0 + k - 1];
                if (k == 1)
                    m = node_step<false>(ttime + cb, (int)(ce - cb), p0, m, lo_k, hi_k, out, st, 0, lane);
                else
                    m = node_step<false>(ttime + cb, (int)(ce - cb), pe, m, lo_k, hi_k, out, st, 0, lane);
                pe.e = out;
            }
        }
        // last node of every episode of the item
        for (int s = s0; s < s1; ++s) {
            const int c = a.slot2cand[s];
            const bool direct = P == 1 && a.counts;
            if (a.skip && a.skip[c]) {  // pruned by a bound: count 0 (else the stitch writes it)
                if (direct && lane == 0) a.counts[c] = 0;
                continue;
            }
            machine_init(st, N);
            if (live && m > 0) {
                const int64_t oc = a.offs[c], ec = oc - c;
                int64_t cb = 0, ce = 0;
                range(a.ctypes[oc + N - 1], cb, ce);
                const int n_ev = (int)(ce - cb);
                const int32_t lo_l = a.relaxed ? 0 : a.clo[ec + N - 2], hi_l = a.chi[ec + N - 2];
                // entries well short of the events: search per entry
                const bool by_entries = ri.tidx && (a.last_mode == 2 || (a.last_mode == 0 &&
                                                                         (int64_t)m * kTrackEntryRatio < (int64_t)n_ev));
                const int32_t *evl = ttime + cb;
                if (by_entries) {
                    const uint32_t E = a.ctypes[oc + N - 1];
                    const int64_t t0 = toff[E];
                    const int32_t *row = ri.tidx + (int64_t)E * (ri.tcells + 1);
                    if (N == 2)
                        last_by_index<false, kTrackEntrySlots>(ttime + t0, (int)(cb - t0), (int)(ce - t0), row,
                                                               ri.tshift, (uint32_t)ri.tbase, ri.tcells, p0, m, lo_l,
                                                               hi_l, st, Tp, lane);
                    else
                        last_by_index<true, kTrackEntrySlots>(ttime + t0, (int)(cb - t0), (int)(ce - t0), row,
                                                              ri.tshift, (uint32_t)ri.tbase, ri.tcells, pe, m, lo_l,
                                                              hi_l, st, Tp, lane);
                } else if (N == 2) {
                    node_step<true>(evl, n_ev, p0, m, lo_l, hi_l, nullptr, st, Tp, lane);
                } else {
                    node_step<true>(evl, n_ev, pe, m, lo_l, hi_l, nullptr, st, Tp, lane);
                }
            }
            st.finish();
            if (lane == 0) {
                if (direct)
                    // one segment from the recording's start: the first valid
                    // end closes the entry classes at class 0, whose count is
                    // the episode's (what the stitch would read)
                    a.counts[c] = st.ncls > 0 ? st.ccnt[0] : 0u;
                else
                    write_record(a.rec + (ri.recbase + (int64_t)(s - ri.slot_first) * P + p) * kRecWords, st);
            }
        }
    }
}

// Groups for the grouped launch: flag[s] = 1 where slot s starts a group
// (first slot, another recording or size, a different prefix of N-1 nodes
// and N-2 edges, or every kTrackGroupMax-th slot).  Episodes of one to two
// nodes share nothing and stay alone.
__global__ void k_track_group_flags(const int32_t *__restrict__ slot2cand, const int32_t *__restrict__ d_n_slots,
                                    int64_t n_slots_cap, const int64_t *__restrict__ offs,
                                    const uint16_t *__restrict__ ctypes, const int32_t *__restrict__ clo,
                                    const int32_t *__restrict__ chi, const uint32_t *__restrict__ cand_rec,
                                    int32_t *__restrict__ flag) {
    const int64_t n = d_n_slots ? (int64_t)*d_n_slots : n_slots_cap;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s <= n_slots_cap;
         s += (int64_t)gridDim.x * blockDim.x) {
        if (s >= n) {
            flag[s] = 0;
            continue;
        }
        bool f = (s == 0) || (s % kTrackGroupMax) == 0;
        if (!f) {
            const int c = slot2cand[s], b = slot2cand[s - 1];
            const int64_t oc = offs[c], ob = offs[b];
            const int N = (int)(offs[c + 1] - oc), Nb = (int)(offs[b + 1] - ob);
            f = N != Nb || N < 3 || (cand_rec && cand_rec[c] != cand_rec[b]);
            for (int k = 0; k < N - 1 && !f; ++k) f = ctypes[oc + k] != ctypes[ob + k];
            for (int k = 0; k < N - 2 && !f; ++k)
                f = clo[oc - c + k] != clo[ob - b + k] || chi[oc - c + k] != chi[ob - b + k];
        }
        flag[s] = f ? 1 : 0;
    }
}

// After an exclusive scan of the flags in place (gidx[s] = groups before
// slot s, gidx[n] = all groups): the first slot of every group, and (one
// thread) per recording its first group and its first item (groups x
// segments), and the item count.
__global__ void k_track_group_starts(const int32_t *__restrict__ gidx, const int32_t *__restrict__ d_n_slots,
                                     int64_t n_slots_cap, int32_t *__restrict__ gstart,
                                     const int32_t *__restrict__ slot2cand, const uint32_t *__restrict__ cand_rec,
                                     int32_t *__restrict__ gmax) {
    const int64_t n = d_n_slots ? (int64_t)*d_n_slots : n_slots_cap;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s <= n; s += (int64_t)gridDim.x * blockDim.x) {
        if (s == n) {
            gstart[gidx[n]] = (int32_t)n;
        } else if (gidx[s + 1] != gidx[s]) {
            gstart[gidx[s]] = (int32_t)s;
            if (gmax) {
                // the group runs to the next start (at most kTrackGroupMax slots)
                int64_t j = s + 1;
                while (j < n && gidx[j + 1] == gidx[j]) ++j;
                atomicMax(gmax + (cand_rec ? cand_rec[slot2cand[s]] : 0u), (int32_t)(j - s));
            }
        }
    }
}

// Per recording (one thread): its first group (or, without groups, its first
// slot) and, walking the recordings in the order rorder, the first item of
// each (groups x segments) and the item count.
__global__ void k_track_group_recs(const int32_t *__restrict__ gidx, const RecInfo *__restrict__ rinfo, int n_recs,
                                   const int32_t *__restrict__ rorder, const int32_t *__restrict__ d_n_slots,
                                   int64_t n_slots_cap, int32_t *__restrict__ gfirst, int64_t *__restrict__ ibase,
                                   int64_t *n_items) {
    const int64_t n = d_n_slots ? (int64_t)*d_n_slots : n_slots_cap;
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    auto first = [&](int r) -> int64_t {
        const int64_t sf = r < n_recs ? (int64_t)rinfo[r].slot_first : n;
        const int64_t c = sf < n ? sf : n;
        return gidx ? (int64_t)gidx[c] : c;
    };
    int64_t base = 0;
    for (int i = 0; i < n_recs; ++i) {
        const int r = rorder ? rorder[i] : i;
        const int64_t g0 = first(r), g1 = first(r + 1);
        gfirst[r] = (int32_t)g0;
        ibase[i] = base;
        base += (g1 - g0) * rinfo[r].P;
    }
    ibase[n_recs] = base;
    *n_items = base;
}

}  // namespace

int track_group_starts(cudaStream_t st, int n_sm, const TrackGroupIn &in) {
    const int64_t cap = in.n_slots_cap;
    const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>((cap + 256) / 256, 8 * (int64_t)n_sm));
    k_track_group_flags<<<g, 256, 0, st>>>(in.slot2cand, in.d_n_slots, cap, in.offs, in.ctypes, in.clo, in.chi,
                                           in.cand_rec, in.gidx);
    FEM_TRY(scan_exclusive(st, in.gidx, cap + 1, in.scan_tmp, nullptr, nullptr));
    if (in.gmax && cudaMemsetAsync(in.gmax, 0, sizeof(int32_t) * std::max(in.n_recs, 1), st) != cudaSuccess)
        return FEM_ERR_CUDA;
    k_track_group_starts<<<g, 256, 0, st>>>(in.gidx, in.d_n_slots, cap, in.gstart, in.slot2cand, in.cand_rec,
                                            in.gmax);
    FEM_CUDA_TRY(cudaGetLastError());
    return FEM_OK;
}

int track_groups(cudaStream_t st, int n_sm, const TrackGroupIn &in, bool grouped, TrackArgs *a) {
    const int64_t cap = in.n_slots_cap;
    if (grouped && !in.starts_ready) FEM_TRY(track_group_starts(st, n_sm, in));
    k_track_group_recs<<<1, 32, 0, st>>>(grouped ? in.gidx : nullptr, in.rinfo, in.n_recs, in.rorder, in.d_n_slots,
                                         cap, in.gfirst, in.ibase, in.n_items);
    FEM_CUDA_TRY(cudaGetLastError());
    a->gstart = grouped ? in.gstart : nullptr;
    a->gfirst = in.gfirst;
    a->ibase = in.ibase;
    a->rorder = in.rorder;
    a->d_n_items = in.n_items;
    return FEM_OK;
}

int track_blocks(int n_sm) {
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_count_track, kTrackWarps * 32, 0);
    cudaGetLastError();
    return std::max(1, n_sm) * std::max(1, std::min(per_sm, kTrackMaxBlocksPerSm));
}

size_t track_buf_bytes(int blocks, int64_t cap) {
    return (size_t)blocks * kTrackWarps * 4 * (size_t)std::max<int64_t>(cap, 1) * sizeof(int32_t);
}

int launch_track(cudaStream_t st, int blocks, const TrackArgs &a) {
    if (blocks < 1) return FEM_OK;
    if (cudaMemsetAsync(a.queue, 0, sizeof(unsigned long long), st) != cudaSuccess) return FEM_ERR_CUDA;
    k_count_track<<<(unsigned)blocks, kTrackWarps * 32, 0, st>>>(a);
    FEM_CUDA_TRY(cudaGetLastError());
    return FEM_OK;
}

}  // namespace fem
