// fem_machine.cuh -- the per-(episode, segment) counting state shared by the
// counting kernels (not part of the ABI): per-node rings of recent entries and
// Algorithm 1 ("Problem decomposition") run for every entry class of a
// segment.
#pragma once

#include "fem_internal.cuh"

namespace fem {

// ---------------------------------------------------------------------------
// Per-node rings of (time, latest start) entries, newest first.  Node 0's
// latest start is its own time, so it stores times only.
//
// Register rings: R entries per node held as a shift register (every index a
// compile-time constant after unrolling).
template <int NMAX, int R>
struct Rings {
    int32_t t[NMAX - 1][R];
    int32_t L[NMAX > 2 ? NMAX - 2 : 1][R];

    __device__ __forceinline__ void init(int32_t *, int32_t *, int, int) {
#pragma unroll
        for (int k = 0; k < NMAX - 1; ++k)
#pragma unroll
            for (int r = 0; r < R; ++r) t[k][r] = INT32_MIN;
#pragma unroll
        for (int k = 0; k < (NMAX > 2 ? NMAX - 2 : 1); ++k)
#pragma unroll
            for (int r = 0; r < R; ++r) L[k][r] = 0;
    }

    // Dropping the oldest entry is safe if it is empty, expired for every
    // query at time >= tt, or if the next-older entry is already past its
    // lower bound (so the oldest can never again be the newest eligible one).
    __device__ __forceinline__ void push(int k, int32_t tt, int32_t LL, int32_t lo, int32_t hi, int &flags) {
        const int32_t o1 = t[k][R - 1], o2 = t[k][R - 2];
        if (o1 != INT32_MIN && o1 >= tt - hi && o2 >= tt - lo) flags |= kMetaRingOverflow;
#pragma unroll
        for (int r = R - 1; r > 0; --r) {
            t[k][r] = t[k][r - 1];
            if (k > 0) L[k > 0 ? k - 1 : 0][r] = L[k > 0 ? k - 1 : 0][r - 1];
        }
        t[k][0] = tt;
        if (k > 0) L[k > 0 ? k - 1 : 0][0] = LL;
    }

    // Newest entry already past its lower bound at time tt; valid when within
    // the upper bound.  Returns its latest start through LL.
    __device__ __forceinline__ bool query(int k, int32_t tt, int32_t lo, int32_t hi, int32_t &LL) const {
        const int32_t elig = tt - lo;
        int32_t tp = INT32_MIN, lp = 0;
        bool found = false;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const bool c = !found && (t[k][r] < elig);
            if (c) {
                tp = t[k][r];
                lp = (k == 0) ? t[k][r] : L[k > 0 ? k - 1 : 0][r];
            }
            found = found || c;
        }
        LL = lp;
        return found && tp >= tt - hi;
    }
};

// Shared-memory rings (R chosen at launch): entry r of node k of this lane at
// base[(k * R + r) * K]; a per-node head index in registers.
template <int NMAX>
struct Rings<NMAX, 0> {
    int32_t *rt;
    int32_t *rl;
    int K;
    int cap[NMAX - 1];       // entries of node k's ring
    int off[NMAX - 1];       // first entry of node k's ring in this lane's slab
    int head[NMAX - 1];

    // Uniform rings: R entries per node.
    __device__ __forceinline__ void init(int32_t *rt_, int32_t *rl_, int R_, int K_) {
        rt = rt_;
        rl = rl_;
        K = K_;
#pragma unroll
        for (int k = 0; k < NMAX - 1; ++k) {
            head[k] = 0;
            cap[k] = R_;
            off[k] = k * R_;
        }
        for (int e = 0; e < (NMAX - 1) * R_; ++e) rt[e * K] = INT32_MIN;
    }

    // Rings sized per node (cap[] already set, at least 2 each); their sum
    // must fit the lane's slab.
    __device__ __forceinline__ void init_var(int32_t *rt_, int32_t *rl_, int K_) {
        rt = rt_;
        rl = rl_;
        K = K_;
        int o = 0;
#pragma unroll
        for (int k = 0; k < NMAX - 1; ++k) {
            head[k] = 0;
            off[k] = o;
            o += cap[k];
        }
        for (int e = 0; e < o; ++e) rt[e * K] = INT32_MIN;
    }

    __device__ __forceinline__ void push(int k, int32_t tt, int32_t LL, int32_t lo, int32_t hi, int &flags) {
        const int h = head[k];
        const int R = cap[k];
        int32_t *bt = rt + off[k] * K;
        int32_t *bl = rl + off[k] * K;
        const int h2 = (h + 1 == R) ? 0 : h + 1;
        const int32_t o1 = bt[h * K];
        const int32_t o2 = bt[h2 * K];
        if (o1 != INT32_MIN && o1 >= tt - hi && o2 >= tt - lo) flags |= kMetaRingOverflow;
        bt[h * K] = tt;
        bl[h * K] = LL;
        head[k] = h2;
    }

    __device__ __forceinline__ bool query(int k, int32_t tt, int32_t lo, int32_t hi, int32_t &LL) const {
        const int R = cap[k];
        const int32_t *bt = rt + off[k] * K;
        const int32_t *bl = rl + off[k] * K;
        const int32_t elig = tt - lo;
        int idx = head[k];
        for (int i = 0; i < R; ++i) {
            idx = (idx == 0) ? R - 1 : idx - 1;
            const int32_t tp = bt[idx * K];
            if (tp < elig) {
                LL = bl[idx * K];
                return tp >= tt - hi;
            }
        }
        return false;
    }
};

// Per-lane machine: the episode, its rings, and Algorithm 1 per entry class.
template <int NMAX, int RR>
struct Machine {
    int N;
    uint32_t E[NMAX];        // 0xFFFFFFFF beyond N (and for idle lanes)
    int32_t lo[NMAX - 1];
    int32_t hi[NMAX - 1];
    Rings<NMAX, RR> rings;
    int32_t cthr[kClasses];
    int32_t cprev[kClasses];
    uint32_t ccnt[kClasses];
    int ncls;
    uint32_t live;           // classes not merged into class 0 (bit 0 = class 0)
    int32_t M;
    int open;
    int flags;

    // Algorithm 1 step for an end event at time t whose latest start is Lq,
    // for every entry class of this (episode, segment) machine; a new class
    // is opened while no occurrence has started inside the segment yet.
    // A class whose last selection equals class 0's has the same future: it
    // is merged (its count kept as an offset from class 0's), so the steady
    // state is a single comparison.
    __device__ __forceinline__ void greedy_end(int32_t t, int32_t Lq, int32_t Tp) {
        if (!open && live == 1u) {
            if (Lq > cprev[0]) {
                ccnt[0] += 1;
                cprev[0] = t;
            }
            return;
        }
#pragma unroll
        for (int j = 0; j < kClasses; ++j)
            if (((live >> j) & 1u) && Lq > cprev[j]) {
                ccnt[j] += 1;
                cprev[j] = t;
            }
        if (open && Lq > M) {
            if (ncls < kClasses) {
#pragma unroll
                for (int j = 0; j < kClasses; ++j)
                    if (j == ncls) {
                        cthr[j] = Lq;
                        ccnt[j] = 1;
                        cprev[j] = t;
                    }
                live |= 1u << ncls;
                ncls += 1;
            } else {
                flags |= kMetaClassOverflow;
            }
            M = Lq;
            if (Lq >= Tp) open = 0;
        }
#pragma unroll
        for (int j = 1; j < kClasses; ++j)
            if (((live >> j) & 1u) && cprev[j] == cprev[0]) {
                ccnt[j] -= ccnt[0];  // offset from class 0 from here on
                live &= ~(1u << j);
            }
    }

    // Final per-class (count, last selection): merged classes follow class 0.
    __device__ __forceinline__ void finish() {
#pragma unroll
        for (int j = 1; j < kClasses; ++j)
            if (j < ncls && !((live >> j) & 1u)) {
                ccnt[j] += ccnt[0];
                cprev[j] = cprev[0];
            }
    }

    // One event offered to this lane's episode.  Nodes are visited last to
    // first; an entry pushed at time et never serves a query at the same time
    // (0 <= lo), so the order only mirrors the serial algorithm.
    __device__ __forceinline__ void step(uint32_t ety, int32_t et, bool in_seg, int32_t Tp) {
#pragma unroll
        for (int k = NMAX - 1; k >= 1; --k) {
            if (E[k] == ety) {
                int32_t Lq;
                if (rings.query(k - 1, et, lo[k - 1], hi[k - 1], Lq)) {
                    if (k == N - 1) {
                        if (in_seg) greedy_end(et, Lq, Tp);
                    } else {
                        rings.push(k, et, Lq, lo[k], hi[k], flags);
                    }
                }
            }
        }
        if (E[0] == ety) rings.push(0, et, et, lo[0], hi[0], flags);
    }
};

// Writes a machine's record: meta (classes, flags, closed bit) and per class
// (threshold, count, last selected end), kRecWords words, int4-aligned.
template <class M>
__device__ __forceinline__ void write_record(int32_t *dst, const M &st) {
    int4 *r = reinterpret_cast<int4 *>(dst);
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

}  // namespace fem
