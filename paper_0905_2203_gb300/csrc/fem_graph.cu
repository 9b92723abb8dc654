// fem_graph.cu -- level-wise mining chained in one captured CUDA graph.
//
// Every level runs a fixed sequence of kernels whose sizes live in device
// counters, so the levels need no host step in between:
//   level 1   frequent types: flags, scan, write ("Temporal Data Mining":
//             a 1-node count is the type's frequency);
//   level 2   every ordered pair of distinct frequent types x bins, generated
//             in canonical order; the upper-bound pre-pass (one stream pass)
//             drops pairs that cannot pass; survivors compacted;
//   level N   prefix/suffix join of level N-1 (count, scan, write);
// then, for every level >= 2: candidate index, the level's segmentation
// (chosen on the device from its candidate count), ring-capacity check,
// sparse counting + stitch, threshold (flags, scan, write) and per-recording
// offsets.  The sequence for levels `first`..max_size is captured once over
// fixed-capacity buffers and launched with a single call; a level that keeps
// nothing leaves zero counters behind and the later levels' kernels exit at
// once.  A capacity overflow, ring-capacity miss or entry-class overflow sets
// a flag; the caller then mines on the host-driven path (same results) and
// the next capture of the same workload gets the capacity that was needed.
// Graphs are cached per context for repeated calls with the same recordings
// and parameters.
#include <algorithm>
#include <cstring>
#include <memory>
#include <sstream>
#include <vector>

#include "fem_internal.cuh"

namespace fem {

namespace {

constexpr int kRingCap = 32;      // largest shared-memory ring in the graph path
constexpr int kMaxPerRec = 4096;  // finest segmentation of a recording
constexpr int64_t kFusedCap = 16384;  // largest level capacity for the single-block join / threshold

// Counters per level: [0] candidates counted C, [1] frequent F, [2] flags,
// [3] entry-class fallbacks (stitch), [4] candidates generated (level 2,
// before the pre-pass), [5] candidates needed (a capacity overflow leaves
// the true total here).
constexpr int kCtr = 6;
constexpr int kFlagCap = 1, kFlagRing = 2, kFlagFreq = 4, kFlagGen = 8;

// Largest r with pre[r] <= i (pre: n + 1 non-decreasing offsets, pre[0] = 0).
__device__ __forceinline__ int seg_of(const int64_t *pre, int n, int64_t i) {
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (pre[mid] <= i) lo = mid; else hi = mid;
    }
    return lo;
}

// For every type a of one recording and finest segment boundary q (pf + 1
// of them; the last is the recording's end): the index, relative to the
// start of a's event list, of a's first event at or after the boundary.
__global__ void k_g_tseg(const int64_t *toff, const int32_t *ttime, const int32_t *time, int64_t n,
                         const int64_t *segf, int pf, uint32_t n_types, int32_t *tseg) {
    const int64_t m = (int64_t)n_types * (pf + 1);
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < m; idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = idx / (pf + 1), q = idx % (pf + 1);
        const int64_t b0 = toff[a], b1 = toff[a + 1];
        int64_t v = b1 - b0;
        if (q < pf && segf[q] < n) {
            const int32_t T = time[segf[q]];
            int64_t lo = b0, hi = b1;
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if (ttime[mid] < T) lo = mid + 1; else hi = mid;
            }
            v = lo - b0;
        }
        tseg[idx] = (int32_t)v;
    }
}

// ---- level 1 ---------------------------------------------------------------
// Frequent types of every recording, in type order: flags over the
// concatenated type ranges (ntpre = prefix of n_types), then write.
__global__ void k_g_l1_flags(const RecInfo *ri, const uint32_t *thr, const int64_t *ntpre, int n_recs, int64_t tot,
                             int32_t *flags) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= tot; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t f = 0;
        if (i < tot) {
            const int r = seg_of(ntpre, n_recs, i);
            f = ri[r].freq[i - ntpre[r]] > thr[r] ? 1 : 0;
        }
        flags[i] = f;
    }
}

__global__ void k_g_l1_write(const int32_t *pos, const RecInfo *ri, const uint32_t *thr, const int64_t *ntpre,
                             int n_recs, int64_t tot, uint16_t *ft, uint32_t *frec, uint32_t *fcnt, int32_t *ctr) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x) {
        const int r = seg_of(ntpre, n_recs, i);
        const uint32_t a = (uint32_t)(i - ntpre[r]);
        const uint32_t f = ri[r].freq[a];
        if (f > thr[r]) {
            const int64_t o = pos[i];
            ft[o] = (uint16_t)a;
            frec[o] = (uint32_t)r;
            fcnt[o] = f;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctr[0] = (int32_t)tot;
        ctr[1] = pos[tot];
    }
}

// ---- level 2 ---------------------------------------------------------------
// Generated pairs per recording: F_r (F_r - 1) nb; offsets and total.
__global__ void k_g_gen2_off(const int64_t *foff1, int n_recs, int nb, int64_t cap2, int64_t *coff2, int32_t *ctr) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    int64_t s = 0;
    coff2[0] = 0;
    for (int r = 0; r < n_recs; ++r) {
        const int64_t F = foff1[r + 1] - foff1[r];
        s += F >= 2 ? F * (F - 1) * nb : 0;
        coff2[r + 1] = s;
    }
    ctr[4] = (int32_t)(s < INT32_MAX ? s : INT32_MAX);
    if (s > cap2) atomicOr(&ctr[2], kFlagGen);
}

// Pair c of recording r in canonical order (E1, bin, E2): the frequent types
// of the recording are in type order and the bins sorted by (lo, hi).
__global__ void k_g_gen2(const uint16_t *ft1, const int64_t *foff1, const int64_t *coff2, int n_recs,
                         const int32_t *blo, const int32_t *bhi, int nb, int64_t cap2, uint16_t *gt, int32_t *glo,
                         int32_t *ghi, uint32_t *grec) {
    const int64_t C = min(coff2[n_recs], cap2);
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < C; c += (int64_t)gridDim.x * blockDim.x) {
        const int r = seg_of(coff2, n_recs, c);
        const int64_t local = c - coff2[r];
        const int64_t F = foff1[r + 1] - foff1[r];
        const int64_t per_i = (int64_t)nb * (F - 1);
        const int64_t i = local / per_i, rem = local % per_i;
        const int k = (int)(rem / (F - 1));
        const int64_t jj = rem % (F - 1);
        const int64_t j = jj < i ? jj : jj + 1;
        gt[2 * c] = ft1[foff1[r] + i];
        gt[2 * c + 1] = ft1[foff1[r] + j];
        glo[c] = blo[k];
        ghi[c] = bhi[k];
        grec[c] = (uint32_t)r;
    }
}

// Upper-bound pre-pass over all recordings (anti-monotonicity, "Temporal Data
// Mining"): the non-overlapped occurrences of a -(lo,hi]-> b end at distinct
// b-events, each with an a-event inside its window, so
//     count(a, b, bin) <= UB = #{ b-events with an a-event in the window }.
// A block takes a tile of kUbTile consecutive events of one recording and
// stages the tile plus the events up to hi_max before it (at most kUbHalo) in
// shared memory; one thread per event scans back over its window there (in
// global memory beyond the staged halo), marks each (type, bin) once in its
// bitset and adds one to UB for it.  The bins a time difference d falls in
// come from a table of bin masks indexed by d (when hi_max < kUbLut), else
// from a loop over the bins.  Word w of thread t's bitset sits at
// bits[w * blockDim + t], so the lanes of a warp touch distinct banks.
constexpr int kUbMaxBins = 8;
constexpr int kUbLut = 65536;
constexpr int kUbTile = 1024;
constexpr int kUbHalo = 1024;

__global__ void k_g_pair_ub(const RecInfo *ri, const int64_t *tpre, int n_recs, const uint32_t *nt,
                            const int64_t *ub_off, const int32_t *blo, const int32_t *bhi, int nb, int32_t hi_max,
                            int words, const uint8_t *lut_g, uint32_t *ub) {
    extern __shared__ uint32_t sm[];
    const int bd = blockDim.x;
    const int lut_words = lut_g ? (hi_max + 4) / 4 : 0;
    uint8_t *lut = reinterpret_cast<uint8_t *>(sm);
    int32_t *s_tm = reinterpret_cast<int32_t *>(sm + lut_words);
    uint16_t *s_ty = reinterpret_cast<uint16_t *>(s_tm + kUbTile + kUbHalo);
    uint32_t *my = sm + lut_words + (kUbTile + kUbHalo) + (kUbTile + kUbHalo) / 2 + threadIdx.x;
    __shared__ int64_t s_h0;
    if (lut_g) {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(lut_g);
        for (int w = threadIdx.x; w < lut_words; w += bd) sm[w] = src[w];
    }
    const int64_t tiles = tpre[n_recs];
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int r = seg_of(tpre, n_recs, tile);
        const int64_t j0 = (tile - tpre[r]) * kUbTile;
        const int64_t n = ri[r].n;
        const int64_t j1 = min(n, j0 + kUbTile);
        const uint16_t *ty = ri[r].type;
        const int32_t *tm = ri[r].time;
        const uint32_t ntr = nt[r];
        const int wr = (int)((ntr * (uint32_t)nb + 31) / 32);
        uint32_t *u = ub + ub_off[r];
        if (threadIdx.x == 0) {
            // first event within hi_max of the tile's first event (capped)
            const int64_t lim = (int64_t)tm[j0] - hi_max;
            int64_t lo = max((int64_t)0, j0 - kUbHalo), hi = j0;
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if ((int64_t)tm[mid] < lim) lo = mid + 1; else hi = mid;
            }
            s_h0 = lo;
        }
        __syncthreads();
        const int64_t h0 = s_h0;
        for (int64_t i = h0 + threadIdx.x; i < j1; i += bd) {
            s_tm[i - h0] = tm[i];
            s_ty[i - h0] = ty[i];
        }
        __syncthreads();
        for (int64_t j = j0 + threadIdx.x; j < j1; j += bd) {
            for (int w = 0; w < wr; ++w) my[w * bd] = 0;
            const int32_t t = s_tm[j - h0];
            const uint32_t b = s_ty[j - h0];
            const int64_t lim = (int64_t)t - hi_max;
            for (int64_t i = j - 1; i >= 0; --i) {
                const bool st = i >= h0;
                const int32_t ti = st ? s_tm[i - h0] : tm[i];
                if ((int64_t)ti < lim) break;
                const int32_t d = t - ti;
                if (d <= 0) continue;
                const uint32_t a = st ? s_ty[i - h0] : ty[i];
                if (a == b) continue;
                uint32_t mask = 0;
                if (lut_g) {
                    mask = lut[d];
                } else {
                    for (int k = 0; k < nb; ++k)
                        if (blo[k] < d && d <= bhi[k]) mask |= 1u << k;
                }
                while (mask) {
                    const int k = __ffs(mask) - 1;
                    mask &= mask - 1;
                    const uint32_t bit = a * (uint32_t)nb + (uint32_t)k;
                    const uint32_t m = 1u << (bit & 31);
                    uint32_t &wd = my[(bit >> 5) * bd];
                    if (!(wd & m)) {
                        wd |= m;
                        atomicAdd(&u[((size_t)a * ntr + b) * nb + k], 1u);
                    }
                }
            }
        }
        __syncthreads();  // the staged events are replaced by the next tile's
    }
}

__device__ __forceinline__ bool g_keep2(int64_t c, const uint16_t *gt, const int32_t *glo, const int32_t *ghi,
                                        const uint32_t *grec, const uint32_t *ub, const int64_t *ub_off,
                                        const uint32_t *nt, const int32_t *blo, const int32_t *bhi, int nb,
                                        const uint32_t *thr) {
    if (!ub) return true;
    const uint32_t r = grec[c];
    int k = 0;
    while (k < nb && !(blo[k] == glo[c] && bhi[k] == ghi[c])) ++k;
    const uint32_t a = gt[2 * c], b = gt[2 * c + 1];
    return ub[ub_off[r] + ((size_t)a * nt[r] + b) * nb + k] > thr[r];
}

__global__ void k_g_prune_flags(const uint16_t *gt, const int32_t *glo, const int32_t *ghi, const uint32_t *grec,
                                const int32_t *ctr, int64_t cap2, const uint32_t *ub, const int64_t *ub_off,
                                const uint32_t *nt, const int32_t *blo, const int32_t *bhi, int nb,
                                const uint32_t *thr, int32_t *flags) {
    const int64_t C = min((int64_t)ctr[4], cap2);
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c <= cap2; c += (int64_t)gridDim.x * blockDim.x)
        flags[c] = (c < C && g_keep2(c, gt, glo, ghi, grec, ub, ub_off, nt, blo, bhi, nb, thr)) ? 1 : 0;
}

__global__ void k_g_prune_write(const int32_t *pos, const uint16_t *gt, const int32_t *glo, const int32_t *ghi,
                                const uint32_t *grec, int64_t cap2, const uint32_t *ub, const int64_t *ub_off,
                                const uint32_t *nt, const int32_t *blo, const int32_t *bhi, int nb,
                                const uint32_t *thr, int64_t cap, uint16_t *ct, int32_t *cl, int32_t *ch,
                                uint32_t *crec, int32_t *ctr) {
    const int64_t C = min((int64_t)ctr[4], cap2);
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < C; c += (int64_t)gridDim.x * blockDim.x) {
        if (!g_keep2(c, gt, glo, ghi, grec, ub, ub_off, nt, blo, bhi, nb, thr)) continue;
        const int64_t o = pos[c];
        if (o >= cap) continue;
        ct[2 * o] = gt[2 * c];
        ct[2 * o + 1] = gt[2 * c + 1];
        cl[o] = glo[c];
        ch[o] = ghi[c];
        crec[o] = grec[c];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const int64_t total = pos[cap2];
        ctr[0] = (int32_t)(total < cap ? total : cap);
        ctr[5] = (int32_t)total;
        if (total > cap) atomicOr(&ctr[2], kFlagCap);
    }
}

// ---- level N >= 3: prefix/suffix join --------------------------------------
__device__ __forceinline__ bool g_joins(const uint16_t *ft, const int32_t *fl, const int32_t *fh, int M, int64_t a,
                                        int64_t b) {
    for (int k = 1; k < M; ++k)
        if (ft[a * M + k] != ft[b * M + k - 1]) return false;
    for (int k = 1; k < M - 1; ++k)
        if (fl[a * (M - 1) + k] != fl[b * (M - 1) + k - 1] || fh[a * (M - 1) + k] != fh[b * (M - 1) + k - 1])
            return false;
    const uint16_t last = ft[b * M + M - 1];
    for (int k = 0; k < M; ++k)
        if (ft[a * M + k] == last) return false;
    return true;
}

// Partners per frequent episode a of its recording (0 beyond the live count).
__global__ void k_g_join_count(const uint16_t *ft, const int32_t *fl, const int32_t *fh, const uint32_t *frec,
                               const int64_t *foff, const int32_t *ctr_prev, int M, int64_t cap, int32_t *cnt) {
    const int64_t F = ctr_prev[1];
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a <= cap; a += (int64_t)gridDim.x * blockDim.x) {
        int32_t c = 0;
        if (a < F) {
            const uint32_t r = frec[a];
            for (int64_t b = foff[r]; b < foff[r + 1]; ++b)
                if (g_joins(ft, fl, fh, M, a, b)) ++c;
        }
        cnt[a] = c;
    }
}

__global__ void k_g_join_write(const uint16_t *ft, const int32_t *fl, const int32_t *fh, const uint32_t *frec,
                               const int64_t *foff, const int32_t *ctr_prev, int M, int64_t cap, const int32_t *pos,
                               uint16_t *ct, int32_t *cl, int32_t *ch, uint32_t *crec, int32_t *ctr) {
    const int64_t F = ctr_prev[1];
    const int N = M + 1;
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < F; a += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t r = frec[a];
        int64_t o = pos[a];
        for (int64_t b = foff[r]; b < foff[r + 1]; ++b) {
            if (!g_joins(ft, fl, fh, M, a, b)) continue;
            if (o < cap) {
                for (int k = 0; k < M; ++k) ct[o * N + k] = ft[a * M + k];
                ct[o * N + M] = ft[b * M + M - 1];
                for (int k = 0; k < M - 1; ++k) {
                    cl[o * (N - 1) + k] = fl[a * (M - 1) + k];
                    ch[o * (N - 1) + k] = fh[a * (M - 1) + k];
                }
                cl[o * (N - 1) + M - 1] = fl[b * (M - 1) + M - 2];
                ch[o * (N - 1) + M - 1] = fh[b * (M - 1) + M - 2];
                crec[o] = r;
            }
            ++o;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const int64_t total = pos[cap];
        ctr[0] = (int32_t)(total < cap ? total : cap);
        ctr[4] = ctr[0];
        ctr[5] = (int32_t)(total < INT32_MAX ? total : INT32_MAX);
        if (total > cap) atomicOr(&ctr[2], kFlagCap);
    }
}

// ---- every level >= 2 --------------------------------------------------------
// Exclusive scan of one value per thread over the block (a multiple of 32
// threads, at most 1024); *total receives the block's sum.
__device__ __forceinline__ int64_t block_excl_scan(int64_t v, int64_t *total) {
    __shared__ int64_t s_w[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int64_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_w[w] = x;
    __syncthreads();
    if (w == 0) {
        int64_t t = lane < nw ? s_w[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xFFFFFFFFu, t, o);
            if (lane >= o) t += y;
        }
        s_w[lane] = t;
    }
    __syncthreads();
    const int64_t before = (w > 0 ? s_w[w - 1] : 0) + x - v;
    *total = s_w[nw - 1];
    __syncthreads();  // s_w is reused by the next call
    return before;
}

// CSR offsets of the candidates and the identity slot order (one block or a
// grid: strided over the block's / grid's threads).
__device__ __forceinline__ void level_index(int64_t C, int N, int64_t cap, int64_t *offs, int32_t *iota, int64_t t0,
                                            int64_t stride) {
    // only the live candidates: nothing reads a slot at or past C
    for (int64_t i = t0; i <= C && i <= cap; i += stride) {
        offs[i] = i * N;
        if (i < C) iota[i] = (int32_t)i;
    }
}

// The same over the whole grid (large levels).
__global__ void k_g_level_index(const int32_t *ctr, int N, int64_t cap, int64_t *offs, int32_t *iota) {
    level_index(ctr[0], N, cap, offs, iota, blockIdx.x * (int64_t)blockDim.x + threadIdx.x,
                (int64_t)gridDim.x * blockDim.x);
}

// Per-level segmentation (one block): the level's (candidate, segment)
// threads should number about `target`, so a level with few candidates cuts
// its recordings finely and one with many coarsely: recording r gets P_r
// segments, every sstep[r]-th of its pfine[r] finest ones.  Also the
// per-recording candidate offsets and the RecInfo fields that depend on them.
//
// With prefix groups (gmax set: recording r's largest group of episodes
// that one work item counts together), an item is a whole group over one
// segment, so the work of the largest item grows with the group: such a
// recording is cut gmax[r] x 4 times finer (the 4 allows for the spread of
// per-event cost between groups), so that the largest item stays near the
// mean work of an item rather than far above the mean work per warp.  The
// factor is halved until the (candidate, segment) records fit cap_threads.
__device__ void level_info(const uint32_t *crec, int64_t C, int n_recs, int64_t *coff, RecInfo *ri,
                           int64_t *nthreads, const int32_t *pfine, int32_t *sstep, int64_t target, int *maxP,
                           const int32_t *gmax = nullptr, int64_t cap_threads = INT64_MAX) {
    for (int r = threadIdx.x; r <= n_recs; r += blockDim.x) {
        int64_t lo = 0, hi = C;  // first candidate of recording >= r
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if ((int)crec[mid] < r) lo = mid + 1; else hi = mid;
        }
        coff[r] = lo;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double W = 0;  // episode-events of the level
        for (int r = 0; r < n_recs; ++r) W += (double)(coff[r + 1] - coff[r]) * (double)ri[r].n;
        const double seg_len = fmax(1.0, W / (double)target);
        // finer cuts for grouped recordings while the records fit (the
        // plain rule, scale 0, fits by construction: at most target + C)
        double scale = gmax ? 4.0 : 0.0;
        for (;;) {
            int64_t tot = 0;
            for (int r = 0; r < n_recs; ++r) {
                const double g = scale > 0.0 ? fmax(1.0, scale * (double)gmax[r]) : 1.0;
                const int pf = pfine[r];
                const double want = fmin((double)pf, fmax(1.0, ceil(g * (double)ri[r].n / seg_len)));
                const int st = (pf + (int)want - 1) / (int)want;
                tot += (coff[r + 1] - coff[r]) * (int64_t)((pf + st - 1) / st);
            }
            if (tot <= cap_threads || scale == 0.0) break;
            scale = scale > 1.0 / 64 ? scale * 0.5 : 0.0;
        }
        int64_t base = 0;
        int pmax = 1;
        for (int r = 0; r < n_recs; ++r) {
            const double g = scale > 0.0 ? fmax(1.0, scale * (double)gmax[r]) : 1.0;
            const int pf = pfine[r];
            const double want = fmin((double)pf, fmax(1.0, ceil(g * (double)ri[r].n / seg_len)));
            const int st = (pf + (int)want - 1) / (int)want;
            const int P = (pf + st - 1) / st;
            sstep[r] = st;
            ri[r].sstep = st;
            ri[r].P = P;
            ri[r].slot_first = (int)coff[r];
            ri[r].recbase = base;
            base += (coff[r + 1] - coff[r]) * P;
            if (coff[r + 1] > coff[r] && P > pmax) pmax = P;
        }
        *nthreads = base;
        *maxP = pmax;
    }
    __syncthreads();
}

__global__ void k_g_levelinfo(const uint32_t *crec, const int32_t *ctr, int N, int64_t cap, int64_t *offs,
                              int32_t *iota, int n_recs, int64_t *coff, RecInfo *ri, int64_t *nthreads,
                              const int32_t *pfine, int32_t *sstep, int64_t target, int *maxP, const int32_t *gmax,
                              int64_t cap_threads) {
    const int64_t C = ctr[0];
    (void)offs;
    (void)iota;
    (void)N;
    (void)cap;
    level_info(crec, C, n_recs, coff, ri, nthreads, pfine, sstep, target, maxP, gmax, cap_threads);
}

// Level N = M + 1 in one block: zero the level's counters, check every
// (alpha, beta) pair of frequent (N-1)-episodes of the same recording for the
// join (pairs numbered alpha-major, each thread a contiguous run of them),
// scan, write the candidates in that order, then index and segment the level
// (for levels whose capacity keeps one block fast; at most kFusedRecs
// recordings).
constexpr int kFusedRecs = 1024;

__global__ void __launch_bounds__(1024, 1)
    k_g_join_fused(const uint16_t *ft, const int32_t *fl, const int32_t *fh, const uint32_t *frec,
                   const int64_t *foff, const int32_t *ctr_prev, int M, int64_t cap, uint16_t *ct, int32_t *cl,
                   int32_t *ch, uint32_t *crec, int32_t *ctr, unsigned long long *rel, int64_t *offs, int32_t *iota,
                   int n_recs, int64_t *coff, RecInfo *ri, int64_t *nthreads, const int32_t *pfine, int32_t *sstep,
                   int64_t target, int *maxP) {
    __shared__ int64_t s_pp[kFusedRecs + 1];  // pair offsets per recording
    const int N = M + 1;
    {
        const int64_t Fr = threadIdx.x < n_recs ? foff[threadIdx.x + 1] - foff[threadIdx.x] : 0;
        int64_t tot = 0;
        const int64_t before = block_excl_scan(Fr * Fr, &tot);
        if (threadIdx.x < n_recs) s_pp[threadIdx.x] = before;
        if (threadIdx.x == 0) s_pp[n_recs] = tot;
        __syncthreads();
    }
    const int64_t npairs = s_pp[n_recs];
    const int64_t per = (npairs + blockDim.x - 1) / blockDim.x;
    const int64_t p0 = min(npairs, (int64_t)threadIdx.x * per), p1 = min(npairs, p0 + per);
    int64_t cnt = 0;
    for (int64_t q = p0; q < p1; ++q) {
        const int r = seg_of(s_pp, n_recs, q);
        const int64_t Fr = foff[r + 1] - foff[r], loc = q - s_pp[r];
        if (g_joins(ft, fl, fh, M, foff[r] + loc / Fr, foff[r] + loc % Fr)) ++cnt;
    }
    int64_t total = 0;
    int64_t o = block_excl_scan(cnt, &total);
    for (int64_t q = p0; q < p1; ++q) {
        const int r = seg_of(s_pp, n_recs, q);
        const int64_t Fr = foff[r + 1] - foff[r], loc = q - s_pp[r];
        const int64_t a = foff[r] + loc / Fr, b = foff[r] + loc % Fr;
        if (!g_joins(ft, fl, fh, M, a, b)) continue;
        if (o < cap) {
            for (int k = 0; k < M; ++k) ct[o * N + k] = ft[a * M + k];
            ct[o * N + M] = ft[b * M + M - 1];
            for (int k = 0; k < M - 1; ++k) {
                cl[o * (N - 1) + k] = fl[a * (M - 1) + k];
                ch[o * (N - 1) + k] = fh[a * (M - 1) + k];
            }
            cl[o * (N - 1) + M - 1] = fl[b * (M - 1) + M - 2];
            ch[o * (N - 1) + M - 1] = fh[b * (M - 1) + M - 2];
            crec[o] = (uint32_t)r;
        }
        ++o;
    }
    const int64_t C = total < cap ? total : cap;
    if (threadIdx.x == 0) {
        ctr[0] = (int32_t)C;
        ctr[1] = 0;
        ctr[2] = total > cap ? kFlagCap : 0;
        ctr[3] = 0;
        ctr[4] = (int32_t)C;
        ctr[5] = (int32_t)(total < INT32_MAX ? total : INT32_MAX);
        *rel = 0ull;
    }
    level_index(C, N, cap, offs, iota, threadIdx.x, blockDim.x);
    __syncthreads();  // crec complete
    level_info(crec, C, n_recs, coff, ri, nthreads, pfine, sstep, target, maxP);
}

// The level's threshold in one block: flags, scan, write of the frequent
// episodes in candidate order, then the per-recording offsets.
__global__ void __launch_bounds__(1024, 1)
    k_g_thr_fused(const uint32_t *counts, const uint16_t *ct, const int32_t *cl, const int32_t *ch,
                  const uint32_t *crec, const uint32_t *thr, int N, int64_t cap, uint16_t *ft, int32_t *fl,
                  int32_t *fh, uint32_t *frec, uint32_t *fcnt, int32_t *ctr, int n_recs, int64_t *foff) {
    const int64_t C = ctr[0];
    const int64_t per = (C + blockDim.x - 1) / blockDim.x;
    const int64_t i0 = min(C, (int64_t)threadIdx.x * per), i1 = min(C, i0 + per);
    int64_t cnt = 0;
    for (int64_t i = i0; i < i1; ++i)
        if (counts[i] > thr[crec[i]]) ++cnt;
    int64_t total = 0;
    int64_t o = block_excl_scan(cnt, &total);
    for (int64_t i = i0; i < i1; ++i) {
        const uint32_t r = crec[i];
        if (!(counts[i] > thr[r])) continue;
        if (o < cap) {
            for (int k = 0; k < N; ++k) ft[o * N + k] = ct[i * N + k];
            for (int k = 0; k < N - 1; ++k) {
                fl[o * (N - 1) + k] = cl[i * (N - 1) + k];
                fh[o * (N - 1) + k] = ch[i * (N - 1) + k];
            }
            frec[o] = r;
            fcnt[o] = counts[i];
        }
        ++o;
    }
    const int64_t F = total < cap ? total : cap;
    if (threadIdx.x == 0) {
        ctr[1] = (int32_t)F;
        if (total > cap) atomicOr(&ctr[2], kFlagFreq);
    }
    __syncthreads();  // frec complete
    for (int r = threadIdx.x; r <= n_recs; r += blockDim.x) {
        int64_t lo = 0, hi = F;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if ((int)frec[mid] < r) lo = mid + 1; else hi = mid;
        }
        foff[r] = lo;
    }
}

// Every node's ring must fit R_cap entries (window density + 1).  Also sums
// the candidates' relevant events (sum over nodes of the node type's
// frequency in the candidate's recording) into *rel, leaving out those a
// bound dropped (skip set: they are not counted).
// It also writes the level's segment boundaries: every sstep[r]-th of the
// recording's finest ones.
__global__ void k_g_ringcheck(const uint16_t *ct, const int32_t *cl, const uint32_t *crec, const int32_t *ctr, int N,
                              const uint32_t *const *dens, const int32_t *lo_vals, int n_lo, int R_cap,
                              const RecInfo *ri, int32_t *ctr_w, unsigned long long *rel, int n_recs,
                              const int64_t *segf, const int32_t *pfine, const int32_t *sstep, int64_t *segl,
                              const uint8_t *skip) {
    const int64_t gt0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, gs = (int64_t)gridDim.x * blockDim.x;
    for (int r = 0; r < n_recs; ++r) {
        const int P = ri[r].P, st = sstep[r], pf = pfine[r];
        const int64_t *f = segf + (size_t)r * (kMaxPerRec + 1);
        int64_t *o = segl + (size_t)r * (kMaxPerRec + 1);
        for (int64_t p = gt0; p <= P; p += gs) o[p] = f[min((int)p * st, pf)];
    }
    const int64_t C = ctr[0];
    unsigned long long acc = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < C; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t r = crec[i];
        const uint32_t *fq = ri[r].freq;
        if (skip && skip[i]) continue;  // dropped by a bound: not counted
        for (int k = 0; k < N; ++k) acc += fq[ct[i * N + k]];
        for (int k = 0; k < N - 1 && dens; ++k) {  // no tables: no rings to check
            const int32_t l = cl[i * (N - 1) + k];
            int j = 0;
            while (j < n_lo && lo_vals[j] != l) ++j;
            const uint32_t d = j < n_lo ? dens[r * n_lo + j][ct[i * N + k]] : 0xFFFFFFFFu;
            if (d == 0xFFFFFFFFu || d + 1 > (uint32_t)R_cap) atomicOr(&ctr_w[2], kFlagRing);
        }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(rel, acc);
}

__global__ void k_g_thr_flags(const uint32_t *counts, const uint32_t *crec, const uint32_t *thr, const int32_t *ctr,
                              int64_t cap, int32_t *flags) {
    const int64_t C = ctr[0];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= cap; i += (int64_t)gridDim.x * blockDim.x)
        flags[i] = (i < C && counts[i] > thr[crec[i]]) ? 1 : 0;
}

__global__ void k_g_thr_write(const int32_t *pos, const uint32_t *counts, const uint16_t *ct, const int32_t *cl,
                              const int32_t *ch, const uint32_t *crec, const uint32_t *thr, int N, int64_t cap,
                              uint16_t *ft, int32_t *fl, int32_t *fh, uint32_t *frec, uint32_t *fcnt, int32_t *ctr) {
    const int64_t C = ctr[0];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < C; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t r = crec[i];
        if (!(counts[i] > thr[r])) continue;
        const int64_t o = pos[i];
        if (o >= cap) continue;
        for (int k = 0; k < N; ++k) ft[o * N + k] = ct[i * N + k];
        for (int k = 0; k < N - 1; ++k) {
            fl[o * (N - 1) + k] = cl[i * (N - 1) + k];
            fh[o * (N - 1) + k] = ch[i * (N - 1) + k];
        }
        frec[o] = r;
        fcnt[o] = counts[i];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const int64_t total = pos[cap];
        ctr[1] = (int32_t)(total < cap ? total : cap);
        if (total > cap) atomicOr(&ctr[2], kFlagFreq);
    }
}

__global__ void k_g_foff(const uint32_t *frec, const int32_t *ctr, int n_recs, int64_t *foff) {
    const int64_t F = ctr[1];
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r <= n_recs; r += gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = F;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if ((int)frec[mid] < r) lo = mid + 1; else hi = mid;
        }
        foff[r] = lo;
    }
}

// Frequent set of one level (fixed capacity).
struct FLevel {
    uint16_t *types = nullptr;
    int32_t *lo = nullptr, *hi = nullptr;
    uint32_t *rec = nullptr, *counts = nullptr;
    int64_t *foff = nullptr;
};

// Layout of the results the graph's last node writes to mapped host memory:
// the status word, the counters, the per-recording offsets, the relevant-
// event sums, then per level its frequent set (capacity-sized regions).
struct PackLayout {
    int64_t o_ctr, o_coff, o_coff2, o_rel;  // byte offsets
    int64_t o_skip3;                        // level 3: candidates per recording the join bound dropped
    int64_t o_lvl[FEM_MAX_NODES + 1];       // per level: types, then lo, hi, rec, counts
    int64_t fcap[FEM_MAX_NODES + 1];        // per level capacity
};

__device__ __forceinline__ void pack_copy(char *dst, const char *src, int64_t bytes, int64_t t0, int64_t stride) {
    // 4-byte words (every region is a multiple of 4 bytes and 8-byte aligned)
    const int64_t w = bytes / 4;
    const uint32_t *s = reinterpret_cast<const uint32_t *>(src);
    uint32_t *d = reinterpret_cast<uint32_t *>(dst);
    for (int64_t i = t0; i < w; i += stride) d[i] = s[i];
}

__global__ void k_g_pack(const int *status, const int32_t *ctr, const int64_t *coff, const int64_t *coff2,
                         const unsigned long long *rel, const unsigned long long *skip3, const FLevel *F,
                         PackLayout lay, int first, int L, int n_recs, char *out) {
    const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, gs = (int64_t)gridDim.x * blockDim.x;
    if (t0 == 0) *reinterpret_cast<int *>(out) = *status;
    pack_copy(out + lay.o_ctr, reinterpret_cast<const char *>(ctr), 4 * (int64_t)(L + 1) * kCtr, t0, gs);
    pack_copy(out + lay.o_coff, reinterpret_cast<const char *>(coff), 8 * (int64_t)(L + 1) * (n_recs + 1), t0, gs);
    pack_copy(out + lay.o_coff2, reinterpret_cast<const char *>(coff2), 8 * (int64_t)(n_recs + 1), t0, gs);
    pack_copy(out + lay.o_rel, reinterpret_cast<const char *>(rel), 8 * (int64_t)(L + 1), t0, gs);
    if (skip3) pack_copy(out + lay.o_skip3, reinterpret_cast<const char *>(skip3), 8 * (int64_t)n_recs, t0, gs);
    for (int N = first; N <= L; ++N) {
        const int64_t Fn = ctr[N * kCtr + 1], fc = lay.fcap[N];
        const FLevel f = F[N];
        char *o = out + lay.o_lvl[N];
        const int64_t tb = ((2 * fc * N) + 7) / 8 * 8, eb = 4 * fc * (N - 1);
        // types: 2-byte entries, copied as bytes pairs
        {
            const uint16_t *s = f.types;
            uint16_t *d = reinterpret_cast<uint16_t *>(o);
            for (int64_t i = t0; i < Fn * N; i += gs) d[i] = s[i];
        }
        if (N > 1) {
            pack_copy(o + tb, reinterpret_cast<const char *>(f.lo), 4 * Fn * (N - 1), t0, gs);
            pack_copy(o + tb + eb, reinterpret_cast<const char *>(f.hi), 4 * Fn * (N - 1), t0, gs);
        }
        pack_copy(o + tb + 2 * eb, reinterpret_cast<const char *>(f.rec), 4 * Fn, t0, gs);
        pack_copy(o + tb + 2 * eb + 4 * fc, reinterpret_cast<const char *>(f.counts), 4 * Fn, t0, gs);
    }
}

}  // namespace

struct GraphTail {
    fem_ctx *ctx = nullptr;
    std::string key;
    std::vector<fem_stream *> recs;
    int n_recs = 0, max_size = 0, first = 3;
    bool prepass = false;
    // coarse-tick bound of levels >= 3 (prepass = 1); a level below
    // coarse_min candidates is not bounded
    int coarse = 0;
    int64_t coarse_min = 0;
    int coarse_slices = 8;
    CoarseDesc *d_cdesc = nullptr;
    uint32_t *cub = nullptr;
    uint8_t *skip = nullptr;
    // level-3 join bound (local tracking with the pre-passes on): bitsets of
    // the frequent 2-node episodes, the (X, Y, bin) table, skipped counts
    bool jb_on = false;                    // asked for (tuning)
    bool jb = false;                       // built
    int64_t jb_cap_words = 0, jb_tab_n = 0;
    uint32_t *jb_v = nullptr, *jb_s = nullptr, *jb_nt = nullptr;
    int64_t *jb_base = nullptr, *jb_tab_off = nullptr;
    int32_t *jb_stride = nullptr, *jb_tab = nullptr;
    unsigned long long *jb_skipc = nullptr;
    int64_t cap = 0, cap2 = 0, cap_threads = 0;
    std::vector<std::pair<void *, size_t>> held;
    std::vector<FLevel> F;                 // F[N] for N = 1..max_size
    int32_t *ctr = nullptr;                // kCtr per level, indexed by N
    int64_t *coff = nullptr;               // (n_recs + 1) per level: counted candidates per recording
    int64_t *coff2 = nullptr;              // generated level-2 candidates per recording
    uint32_t *d_thr = nullptr;
    int ring_cap = kRingCap;               // ring entries per node
    // exact counts by warp-per-item local tracking (one persistent launch
    // per level, prefix groups); otherwise the node-uniform sparse kernel
    bool track = false;
    int track_nblocks = 0;
    int64_t track_cap = 0;                 // longest per-type list of any recording
    int32_t *tbuf = nullptr;
    int64_t *tqueue = nullptr;
    int32_t *tg_gidx = nullptr, *tg_gstart = nullptr, *tg_gfirst = nullptr, *tg_stmp = nullptr;
    int32_t *tg_gmax = nullptr;            // per recording: the level's largest prefix group
    int64_t *tg_ibase = nullptr, *tg_nitems = nullptr;
    int32_t *rorder = nullptr;             // recordings, longest first (item order)
    int *d_maxP = nullptr;                 // the current level's largest segment count
    int64_t *segf = nullptr, *segl = nullptr;  // finest / current level's segment starts
    int32_t *pfine = nullptr, *sstep = nullptr;
    int64_t target = 0;                    // (candidate, segment) threads per level
    unsigned long long *rel = nullptr;     // relevant events counted, per level
    std::vector<cudaEvent_t> ev;           // around each level's count kernels
    int64_t kernel_nodes = 0;              // kernel launches per run of the graph
    char *h_out = nullptr;                 // mapped host buffer the last node writes the results to
    size_t out_bytes = 0;
    PackLayout lay{};
    cudaGraphExec_t exec = nullptr;

    template <typename T>
    int get(T **p, size_t n) {
        void *q = nullptr;
        const size_t b = std::max<size_t>(n, 1) * sizeof(T);
        FEM_TRY(dev_alloc(ctx, &q, b));
        held.push_back({q, b});
        *p = static_cast<T *>(q);
        return FEM_OK;
    }
    ~GraphTail() {
        if (exec) cudaGraphExecDestroy(exec);
        cudaStreamSynchronize(ctx->stream);
        for (auto e : ev) cudaEventDestroy(e);
        for (auto &h : held) dev_free(ctx, h.first, h.second);
        if (h_out) {
            // kept by the context for the next graph (the larger buffer wins)
            if (!ctx->pinned || ctx->pinned_bytes < out_bytes) {
                if (ctx->pinned) cudaFreeHost(ctx->pinned);
                ctx->pinned = h_out;
                ctx->pinned_bytes = out_bytes;
            } else {
                cudaFreeHost(h_out);
            }
        }
    }
};

// Shared memory of the node-uniform sparse kernel for N-node episodes with
// rings of R entries (the kernel's per-thread header + slab, 64 threads).
static size_t graph_sparse_smem(int N, int R) {
    const int nmax = N <= 2 ? 2 : N <= 4 ? 4 : N <= 8 ? 8 : 16;
    return (size_t)(6 * (nmax - 1) + 2 * (N - 1) * R) * 64 * 4;
}

static int build_graph(GraphTail *g, const std::vector<int32_t> &blo, const std::vector<int32_t> &bhi,
                       const std::vector<uint32_t> &thr, const std::vector<int32_t> &lo_vals) {
    fem_ctx *ctx = g->ctx;
    cudaStream_t st = ctx->stream;
    const int n_recs = g->n_recs, L = g->max_size, first = g->first;
    const int nb = (int)blo.size();
    const int64_t cap = g->cap;
    int32_t hi_max = 0;
    for (auto h : bhi) hi_max = std::max(hi_max, h);
    // per-recording segment boundaries, per-type lists, densities
    std::vector<RecInfo> ri_h(n_recs);
    int64_t *segs = nullptr;  // finest boundaries per recording
    FEM_TRY(g->get(&segs, (size_t)n_recs * (kMaxPerRec + 1)));
    FEM_TRY(g->get(&g->segl, (size_t)n_recs * (kMaxPerRec + 1)));
    FEM_TRY(g->get(&g->pfine, n_recs));
    FEM_TRY(g->get(&g->sstep, n_recs));
    std::vector<int32_t> pfine_h(n_recs);
    const int64_t sumhi_max = (int64_t)(L - 1) * hi_max;
    // window densities size the rings of the per-episode kernels; local
    // tracking keeps no rings and does without them
    const bool need_dens = ctx->tuning.kernel != 0;
    std::vector<const uint32_t *> dens_h(need_dens ? (size_t)n_recs * lo_vals.size() : 0);
    for (int r = 0; r < n_recs; ++r) {
        fem_stream *s = g->recs[r];
        FEM_TRY(!need_dens ? stream_tindex(ctx, s) : stream_bytype(ctx, s));
        if (need_dens) {
            FEM_TRY(stream_densities(ctx, s, lo_vals));
            for (size_t j = 0; j < lo_vals.size(); ++j) {
                uint32_t *d = nullptr;
                FEM_TRY(stream_density(ctx, s, lo_vals[j], &d));
                dens_h[(size_t)r * lo_vals.size() + j] = d;
            }
        }
        // finest segments: at least 256 events and twice the halo (sum of
        // the upper bounds, in events at the recording's mean rate)
        const double span = std::max(1.0, (double)s->t_last - (double)s->t_first);
        const double halo_ev = (double)s->n * (double)sumhi_max / span;
        // (local tracking: segments of at least 8192 events, so that a warp's
        // item is long against its halo and per-item set-up)
        const double min_seg = std::max(ctx->tuning.kernel == 0 ? (double)kTrackMinSeg : 256.0, 2.0 * halo_ev);
        const int P = (int)std::max(1.0, std::min<double>(kMaxPerRec, (double)s->n / min_seg));
        pfine_h[r] = P;
        FEM_TRY(launch_segments(st, s->d_time, s->n, P, segs + (size_t)r * (kMaxPerRec + 1)));
        // list positions of the finest boundaries, per type
        int32_t *tseg = nullptr;
        FEM_TRY(g->get(&tseg, (size_t)s->n_types * (P + 1)));
        const int64_t tm = (int64_t)s->n_types * (P + 1);
        k_g_tseg<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((tm + 255) / 256, 4 * ctx->n_sm)), 256, 0, st>>>(
            s->d_toff, s->d_ttime, s->d_time, s->n, segs + (size_t)r * (kMaxPerRec + 1), P, s->n_types, tseg);
        FEM_CUDA_TRY(cudaGetLastError());
        ri_h[r] = RecInfo{s->d_type, s->d_time, s->n, g->segl + (size_t)r * (kMaxPerRec + 1), 1, 0, 0,
                          s->d_freq, s->d_toff, s->d_ttime, tseg, P + 1, 1};
        recinfo_lists(ri_h[r], s);
    }
    FEM_CUDA_TRY(cudaMemcpyAsync(g->pfine, pfine_h.data(), 4 * n_recs, cudaMemcpyHostToDevice, st));
    g->segf = segs;
    // (candidate, segment) threads per level: about two waves of the sparse
    // kernel, never more than target + live candidates (one segment each)
    g->track = ctx->tuning.kernel == 0;
    if (g->track) {
        g->track_nblocks = track_blocks(ctx->n_sm);
        for (auto *s : g->recs) g->track_cap = std::max(g->track_cap, s->max_list);
        const size_t fb = ctx->budget > ctx->used.load() ? ctx->budget - ctx->used.load() : 0;
        while (g->track_nblocks > ctx->n_sm && track_buf_bytes(g->track_nblocks, g->track_cap) > fb / 4)
            g->track_nblocks -= ctx->n_sm;
        if (track_buf_bytes(g->track_nblocks, g->track_cap) > fb / 4) return FEM_ERR_NOMEM;
        // about four work items per resident warp, segments no shorter than
        // kTrackMinSeg events (the finest segmentation above)
        g->target = (int64_t)4 * g->track_nblocks * kTrackWarps;
    } else {
        g->target = (int64_t)2 * ctx->n_sm * 512;
    }
    g->cap_threads = g->target + cap;
    // ring entries per node: the largest window density of any type + 1; the
    // graph does not apply when that exceeds kRingCap or what the deepest
    // level's shared memory holds (such streams mine on the host-driven path)
    uint32_t dmax = 1;
    for (int r = 0; r < n_recs && need_dens; ++r) {
        std::vector<uint32_t> hd(g->recs[r]->n_types);
        for (size_t j = 0; j < lo_vals.size(); ++j) {
            FEM_CUDA_TRY(cudaMemcpyAsync(hd.data(), dens_h[(size_t)r * lo_vals.size() + j], 4 * hd.size(),
                                         cudaMemcpyDeviceToHost, st));
            FEM_CUDA_TRY(cudaStreamSynchronize(st));
            for (uint32_t d : hd) dmax = std::max(dmax, d);
        }
    }
    if (g->track) {
        g->ring_cap = 1 << 30;  // local tracking keeps no rings: nothing to check
    } else {
        if (dmax + 1 > (uint32_t)kRingCap) return FEM_ERR_INVAL;
        g->ring_cap = (int)dmax + 1;
        for (int N = std::max(first, 2); N <= L; ++N)
            if (graph_sparse_smem(N, g->ring_cap) > (size_t)ctx->smem_optin - 1024) return FEM_ERR_INVAL;
    }
    // level 1 / level 2 sizes
    std::vector<int64_t> ntpre(n_recs + 1, 0), evpre(n_recs + 1, 0), ub_off(n_recs + 1, 0);
    std::vector<uint32_t> nt_h(n_recs);
    int64_t cap2 = 0;
    uint32_t nt_max = 1;
    for (int r = 0; r < n_recs; ++r) {
        const int64_t nt = g->recs[r]->n_types;
        nt_h[r] = (uint32_t)nt;
        nt_max = std::max(nt_max, (uint32_t)nt);
        ntpre[r + 1] = ntpre[r] + nt;
        evpre[r + 1] = evpre[r] + g->recs[r]->n;
        ub_off[r + 1] = ub_off[r] + nt * nt * nb;
        cap2 += nt >= 2 ? nt * (nt - 1) * nb : 0;
    }
    g->cap2 = cap2;
    const int64_t tot1 = ntpre[n_recs];
    const size_t free_b = ctx->budget > ctx->used.load() ? ctx->budget - ctx->used.load() : 0;
    // local tracking cuts grouped levels finer (records per candidate and
    // segment): room for four segments per candidate where the budget has it
    if (g->track && (size_t)(g->target + 4 * cap) * kRecWords * 4 <= free_b / 4) g->cap_threads = g->target + 4 * cap;
    if ((size_t)g->cap_threads * kRecWords * 4 > free_b / 4) return FEM_ERR_NOMEM;
    // pre-pass launch shape: the bin-mask table (when hi_max < kUbLut), the
    // staged events and a per-thread bitset of n_types x bins bits
    const int ub_words = (int)((nt_max * (uint32_t)std::max(nb, 1) + 31) / 32);
    const bool ub_lut = hi_max < kUbLut;
    const size_t ub_lut_bytes = ub_lut ? (size_t)((hi_max + 4) / 4) * 4 : 0;
    const size_t ub_stage = (size_t)(kUbTile + kUbHalo) * 4 + (size_t)(kUbTile + kUbHalo) / 2 * 4;
    const int64_t ub_room = (int64_t)ctx->smem_optin - 1024 - (int64_t)ub_lut_bytes - (int64_t)ub_stage;
    const int ub_threads =
        ub_room > 0 ? (int)std::min<int64_t>(256, ub_room / (4 * (int64_t)ub_words) / 32 * 32) : 0;
    const size_t ub_smem = ub_lut_bytes + ub_stage + (size_t)std::max(ub_threads, 0) * ub_words * 4;
    if (ub_threads < 32 || nb > kUbMaxBins) g->prepass = false;
    std::vector<int64_t> tpre(n_recs + 1, 0);
    for (int r = 0; r < n_recs; ++r) tpre[r + 1] = tpre[r] + (g->recs[r]->n + kUbTile - 1) / kUbTile;
    std::vector<uint8_t> lut_h(ub_lut ? (size_t)((hi_max + 4) / 4) * 4 : 0, 0);
    for (int32_t d = 0; ub_lut && d <= hi_max; ++d)
        for (int k = 0; k < nb; ++k)
            if (blo[k] < d && d <= bhi[k]) lut_h[d] |= (uint8_t)(1u << k);

    RecInfo *d_ri;
    const uint32_t **d_dens;
    int32_t *d_lov, *pos, *fb_list, *iota, *rec, *d_blo, *d_bhi;
    int64_t *offs, *nthreads;
    uint16_t *ct;
    int32_t *cl, *ch;
    uint32_t *crec, *counts;
    const int Nmax = L;
    const int64_t scan_m = std::max<int64_t>(std::max<int64_t>(cap, tot1), first <= 2 ? cap2 : 0);
    FEM_TRY(g->get(&d_ri, n_recs));
    FEM_TRY(g->get(&d_dens, dens_h.size()));
    FEM_TRY(g->get(&d_lov, lo_vals.size()));
    FEM_TRY(g->get(&d_blo, std::max(nb, 1)));
    FEM_TRY(g->get(&d_bhi, std::max(nb, 1)));
    FEM_TRY(g->get(&pos, scan_m + 2));
    FEM_TRY(g->get(&fb_list, cap));
    FEM_TRY(g->get(&iota, cap));
    FEM_TRY(g->get(&rec, (size_t)g->cap_threads * kRecWords));
    FEM_TRY(g->get(&g->d_maxP, 1));
    if (g->track) {
        FEM_TRY(g->get(&g->tbuf, track_buf_bytes(g->track_nblocks, g->track_cap) / sizeof(int32_t)));
        FEM_TRY(g->get(&g->tqueue, 1));
        FEM_TRY(g->get(&g->tg_gidx, cap + 2));
        FEM_TRY(g->get(&g->tg_gstart, cap + 2));
        FEM_TRY(g->get(&g->tg_gmax, std::max(n_recs, 1)));
        FEM_TRY(g->get(&g->tg_gfirst, n_recs));
        FEM_TRY(g->get(&g->tg_stmp, (cap + 2) / 1024 + 2));
        FEM_TRY(g->get(&g->tg_ibase, n_recs + 1));
        FEM_TRY(g->get(&g->tg_nitems, 1));
        FEM_TRY(g->get(&g->rorder, n_recs));
        std::vector<int32_t> ro(n_recs);
        for (int r = 0; r < n_recs; ++r) ro[r] = r;
        std::stable_sort(ro.begin(), ro.end(), [&](int x, int y) { return g->recs[x]->n > g->recs[y]->n; });
        FEM_CUDA_TRY(cudaMemcpyAsync(g->rorder, ro.data(), 4 * n_recs, cudaMemcpyHostToDevice, st));
    }
    FEM_TRY(g->get(&offs, cap + 1));
    FEM_TRY(g->get(&nthreads, 1));
    FEM_TRY(g->get(&ct, (size_t)cap * Nmax));
    FEM_TRY(g->get(&cl, (size_t)cap * std::max(Nmax - 1, 1)));
    FEM_TRY(g->get(&ch, (size_t)cap * std::max(Nmax - 1, 1)));
    FEM_TRY(g->get(&crec, cap));
    FEM_TRY(g->get(&counts, cap));
    FEM_TRY(g->get(&g->d_thr, n_recs));
    FEM_TRY(g->get(&g->ctr, (size_t)(L + 1) * kCtr));
    FEM_TRY(g->get(&g->coff, (size_t)(L + 1) * (n_recs + 1)));
    FEM_TRY(g->get(&g->coff2, n_recs + 1));
    FEM_TRY(g->get(&g->rel, (size_t)(L + 1)));
    g->ev.assign(2 * (L + 1), nullptr);
    for (auto &e : g->ev) FEM_CUDA_TRY(cudaEventCreate(&e));
    g->F.assign(L + 1, FLevel{});
    for (int N = std::max(1, first - 1); N <= L; ++N) {
        FLevel &f = g->F[N];
        const int64_t fc = N == 1 ? std::max<int64_t>(tot1, 1) : cap;
        FEM_TRY(g->get(&f.types, (size_t)fc * N));
        if (N > 1) {
            FEM_TRY(g->get(&f.lo, (size_t)fc * (N - 1)));
            FEM_TRY(g->get(&f.hi, (size_t)fc * (N - 1)));
        }
        FEM_TRY(g->get(&f.rec, fc));
        FEM_TRY(g->get(&f.counts, fc));
        FEM_TRY(g->get(&f.foff, n_recs + 1));
    }
    // level-1 / level-2 inputs
    int64_t *d_ntpre = nullptr, *d_evpre = nullptr, *d_uboff = nullptr, *d_tpre = nullptr;
    uint8_t *d_lut = nullptr;
    uint32_t *d_nt = nullptr, *ub = nullptr;
    uint16_t *gt = nullptr;
    int32_t *glo = nullptr, *ghi = nullptr;
    uint32_t *grec = nullptr;
    if (first <= 2) {
        FEM_TRY(g->get(&d_ntpre, n_recs + 1));
        FEM_TRY(g->get(&d_evpre, n_recs + 1));
        FEM_TRY(g->get(&d_uboff, n_recs + 1));
        FEM_TRY(g->get(&d_nt, n_recs));
        FEM_TRY(g->get(&d_tpre, n_recs + 1));
        if (ub_lut) FEM_TRY(g->get(&d_lut, lut_h.size()));
        FEM_TRY(g->get(&gt, (size_t)2 * std::max<int64_t>(cap2, 1)));
        FEM_TRY(g->get(&glo, std::max<int64_t>(cap2, 1)));
        FEM_TRY(g->get(&ghi, std::max<int64_t>(cap2, 1)));
        FEM_TRY(g->get(&grec, std::max<int64_t>(cap2, 1)));
        if (g->prepass) FEM_TRY(g->get(&ub, std::max<int64_t>(ub_off[n_recs], 1)));
        FEM_CUDA_TRY(cudaMemcpyAsync(d_ntpre, ntpre.data(), 8 * (n_recs + 1), cudaMemcpyHostToDevice, st));
        FEM_CUDA_TRY(cudaMemcpyAsync(d_evpre, evpre.data(), 8 * (n_recs + 1), cudaMemcpyHostToDevice, st));
        FEM_CUDA_TRY(cudaMemcpyAsync(d_uboff, ub_off.data(), 8 * (n_recs + 1), cudaMemcpyHostToDevice, st));
        FEM_CUDA_TRY(cudaMemcpyAsync(d_nt, nt_h.data(), 4 * n_recs, cudaMemcpyHostToDevice, st));
        FEM_CUDA_TRY(cudaMemcpyAsync(d_tpre, tpre.data(), 8 * (n_recs + 1), cudaMemcpyHostToDevice, st));
        if (ub_lut) FEM_CUDA_TRY(cudaMemcpyAsync(d_lut, lut_h.data(), lut_h.size(), cudaMemcpyHostToDevice, st));
    }
    FEM_CUDA_TRY(cudaMemcpyAsync(d_ri, ri_h.data(), sizeof(RecInfo) * n_recs, cudaMemcpyHostToDevice, st));
    FEM_CUDA_TRY(cudaMemcpyAsync(d_dens, dens_h.data(), sizeof(void *) * dens_h.size(), cudaMemcpyHostToDevice, st));
    FEM_CUDA_TRY(cudaMemcpyAsync(d_lov, lo_vals.data(), 4 * lo_vals.size(), cudaMemcpyHostToDevice, st));
    if (nb > 0) {
        FEM_CUDA_TRY(cudaMemcpyAsync(d_blo, blo.data(), 4 * nb, cudaMemcpyHostToDevice, st));
        FEM_CUDA_TRY(cudaMemcpyAsync(d_bhi, bhi.data(), 4 * nb, cudaMemcpyHostToDevice, st));
    }
    FEM_CUDA_TRY(cudaMemcpyAsync(g->d_thr, thr.data(), 4 * n_recs, cudaMemcpyHostToDevice, st));
    int32_t *scan_tmp;
    FEM_TRY(g->get(&scan_tmp, (scan_m + 2) / 1024 + 2));
    // results in mapped host memory (written by the graph's last node)
    {
        PackLayout &lay = g->lay;
        int64_t o = 8;
        auto take = [&](int64_t bytes) {
            const int64_t at = o;
            o += (bytes + 7) / 8 * 8;
            return at;
        };
        lay.o_ctr = take(4 * (int64_t)(L + 1) * kCtr);
        lay.o_coff = take(8 * (int64_t)(L + 1) * (n_recs + 1));
        lay.o_coff2 = take(8 * (int64_t)(n_recs + 1));
        lay.o_rel = take(8 * (int64_t)(L + 1));
        lay.o_skip3 = take(8 * (int64_t)std::max(n_recs, 1));
        for (int N = first; N <= L; ++N) {
            const int64_t fc = N == 1 ? std::max<int64_t>(tot1, 1) : cap;
            lay.fcap[N] = fc;
            const int64_t tb = ((2 * fc * N) + 7) / 8 * 8, eb = 4 * fc * (N - 1);
            lay.o_lvl[N] = take(tb + 2 * eb + 8 * fc);
        }
        g->out_bytes = (size_t)o;
        // the mapped result buffer of an earlier graph of the context, when
        // large enough (pinning a large buffer costs more than a launch)
        if (ctx->pinned && ctx->pinned_bytes >= g->out_bytes) {
            g->h_out = static_cast<char *>(ctx->pinned);
            g->out_bytes = ctx->pinned_bytes;
            ctx->pinned = nullptr;
            ctx->pinned_bytes = 0;
        } else if (cudaHostAlloc(reinterpret_cast<void **>(&g->h_out), g->out_bytes, cudaHostAllocMapped) !=
                   cudaSuccess) {
            cudaGetLastError();
            g->h_out = nullptr;
            return FEM_ERR_NOMEM;
        }
    }
    char *d_out = nullptr;
    FEM_CUDA_TRY(cudaHostGetDevicePointer(reinterpret_cast<void **>(&d_out), g->h_out, 0));
    FLevel *d_F = nullptr;
    FEM_TRY(g->get(&d_F, (size_t)L + 1));
    FEM_CUDA_TRY(cudaMemcpyAsync(d_F, g->F.data(), sizeof(FLevel) * (L + 1), cudaMemcpyHostToDevice, st));
    // coarse-tick tables of every recording (built once per stream and tick)
    if (g->coarse && L >= 3) {
        std::vector<CoarseDesc> cd(n_recs);
        for (int r = 0; r < n_recs; ++r)
            FEM_TRY(coarse_desc(ctx, g->recs[r], coarse_tick(g->recs[r], hi_max, 0), g->coarse_slices, &cd[r]));
        FEM_TRY(g->get(&g->d_cdesc, (size_t)n_recs));
        FEM_TRY(g->get(&g->cub, (size_t)cap));
        FEM_TRY(g->get(&g->skip, (size_t)cap));
        FEM_CUDA_TRY(cudaMemcpyAsync(g->d_cdesc, cd.data(), sizeof(CoarseDesc) * n_recs, cudaMemcpyHostToDevice, st));
    } else {
        g->coarse = 0;
    }
    // level-3 join bound: per frequent 2-node episode two bitsets of its
    // recording's longest list / 32 words each; capacity for every ordered
    // pair x bin of a recording being frequent, capped by the budget (a
    // level whose bitsets do not fit is not bounded)
    g->jb = g->jb_on && g->track && L >= 3 && first <= 3 && nb > 0;
    if (g->jb) {
        std::vector<int32_t> stride_h(n_recs);
        int64_t worst = 0;
        for (int r = 0; r < n_recs; ++r) {
            stride_h[r] = (int32_t)((g->recs[r]->max_list + 31) / 32);
            worst += std::min<int64_t>((int64_t)nt_h[r] * nt_h[r] * nb, cap) * stride_h[r];
        }
        const size_t fb = ctx->budget > ctx->used.load() ? ctx->budget - ctx->used.load() : 0;
        g->jb_cap_words = std::min<int64_t>(std::min<int64_t>(worst, (int64_t)1 << 28), (int64_t)(fb / 32));
        g->jb_tab_n = std::max<int64_t>(ub_off[n_recs], 1);
        if (g->jb_cap_words < 1024) {
            g->jb = false;
        } else {
            FEM_TRY(g->get(&g->jb_v, (size_t)g->jb_cap_words));
            FEM_TRY(g->get(&g->jb_s, (size_t)g->jb_cap_words));
            FEM_TRY(g->get(&g->jb_base, (size_t)n_recs + 1));
            FEM_TRY(g->get(&g->jb_stride, (size_t)n_recs));
            FEM_TRY(g->get(&g->jb_tab, (size_t)g->jb_tab_n));
            FEM_TRY(g->get(&g->jb_tab_off, (size_t)n_recs + 1));
            FEM_TRY(g->get(&g->jb_nt, (size_t)n_recs));
            FEM_TRY(g->get(&g->jb_skipc, (size_t)n_recs));
            if (!g->skip) FEM_TRY(g->get(&g->skip, (size_t)cap));
            FEM_CUDA_TRY(cudaMemcpyAsync(g->jb_stride, stride_h.data(), 4 * n_recs, cudaMemcpyHostToDevice, st));
            FEM_CUDA_TRY(cudaMemcpyAsync(g->jb_tab_off, ub_off.data(), 8 * (n_recs + 1), cudaMemcpyHostToDevice, st));
            FEM_CUDA_TRY(cudaMemcpyAsync(g->jb_nt, nt_h.data(), 4 * n_recs, cudaMemcpyHostToDevice, st));
        }
    }
    FEM_CUDA_TRY(cudaStreamSynchronize(st));

    // ---- capture levels first..L
    const unsigned gb = (unsigned)std::min<int64_t>((cap + 256) / 256, 4 * ctx->n_sm);
    const unsigned gb2 = (unsigned)std::max<int64_t>(1, std::min<int64_t>((cap2 + 256) / 256, 8 * ctx->n_sm));
    const unsigned gb1 = (unsigned)std::max<int64_t>(1, std::min<int64_t>((tot1 + 256) / 256, 4 * ctx->n_sm));
    const unsigned gbe = (unsigned)std::max<int64_t>(1, std::min<int64_t>(tpre[n_recs], 8 * ctx->n_sm));
    if (g->prepass && ub_smem > 48 * 1024) {
        if (cudaFuncSetAttribute((const void *)k_g_pair_ub, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)ub_smem) != cudaSuccess) {
            cudaGetLastError();
            g->prepass = false;
        }
    }
    cudaGraph_t graph = nullptr;
    FEM_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    int cst = FEM_OK;
    auto ok = [&](cudaError_t e) {
        if (cst == FEM_OK && e != cudaSuccess) cst = FEM_ERR_CUDA;
    };
    // levels whose candidate capacity keeps one block fast use the fused
    // single-block join and threshold kernels
    const bool fused = cap <= kFusedCap && n_recs <= kFusedRecs;
    for (int N = first; N <= L && cst == FEM_OK; ++N) {
        int32_t *cn = g->ctr + (size_t)N * kCtr;
        int64_t *coffN = g->coff + (size_t)N * (n_recs + 1);
        FLevel &nf = g->F[N];
        const bool fuse_join = fused && N >= 3;
        // the level's slots as the local-tracking group kernels see them
        auto group_in = [&]() {
            TrackGroupIn gi{};
            gi.slot2cand = iota;
            gi.d_n_slots = cn;
            gi.n_slots_cap = cap;
            gi.offs = offs;
            gi.ctypes = ct;
            gi.clo = cl;
            gi.chi = ch;
            gi.cand_rec = crec;
            gi.rinfo = d_ri;
            gi.n_recs = n_recs;
            gi.gidx = g->tg_gidx;
            gi.scan_tmp = g->tg_stmp;
            gi.gstart = g->tg_gstart;
            gi.gfirst = g->tg_gfirst;
            gi.ibase = g->tg_ibase;
            gi.n_items = g->tg_nitems;
            gi.rorder = g->rorder;
            gi.gmax = g->tg_gmax;
            return gi;
        };
        bool groups_ready = false;
        if (!fuse_join) {
            ok(cudaMemsetAsync(cn, 0, sizeof(int32_t) * kCtr, st));
            ok(cudaMemsetAsync(g->rel + N, 0, sizeof(unsigned long long), st));
        }
        if (N == 1) {
            k_g_l1_flags<<<gb1, 256, 0, st>>>(d_ri, g->d_thr, d_ntpre, n_recs, tot1, pos);
            if (cst == FEM_OK) cst = scan_exclusive(st, pos, tot1 + 1, scan_tmp, nullptr, nullptr);
            k_g_l1_write<<<gb1, 256, 0, st>>>(pos, d_ri, g->d_thr, d_ntpre, n_recs, tot1, nf.types, nf.rec, nf.counts,
                                              cn);
            k_g_foff<<<1, 256, 0, st>>>(nf.rec, cn, n_recs, nf.foff);
            ok(cudaGetLastError());
            continue;
        }
        const int nmax = N <= 2 ? 2 : N <= 4 ? 4 : N <= 8 ? 8 : 16;
        if (N == 2) {
            const FLevel &f1 = g->F[1];
            k_g_gen2_off<<<1, 32, 0, st>>>(f1.foff, n_recs, nb, cap2, g->coff2, cn);
            k_g_gen2<<<gb2, 256, 0, st>>>(f1.types, f1.foff, g->coff2, n_recs, d_blo, d_bhi, nb, cap2, gt, glo, ghi,
                                          grec);
            if (g->prepass) {
                ok(cudaMemsetAsync(ub, 0, sizeof(uint32_t) * std::max<int64_t>(ub_off[n_recs], 1), st));
                k_g_pair_ub<<<gbe, ub_threads, ub_smem, st>>>(d_ri, d_tpre, n_recs, d_nt, d_uboff, d_blo, d_bhi, nb,
                                                              hi_max, ub_words, d_lut, ub);
            }
            const uint32_t *ubp = g->prepass ? ub : nullptr;
            k_g_prune_flags<<<gb2, 256, 0, st>>>(gt, glo, ghi, grec, cn, cap2, ubp, d_uboff, d_nt, d_blo, d_bhi, nb,
                                                 g->d_thr, pos);
            if (cst == FEM_OK) cst = scan_exclusive(st, pos, cap2 + 1, scan_tmp, nullptr, nullptr);
            k_g_prune_write<<<gb2, 256, 0, st>>>(pos, gt, glo, ghi, grec, cap2, ubp, d_uboff, d_nt, d_blo, d_bhi, nb,
                                                 g->d_thr, cap, ct, cl, ch, crec, cn);
            k_g_level_index<<<gb, 256, 0, st>>>(cn, N, cap, offs, iota);
            k_g_levelinfo<<<1, 256, 0, st>>>(crec, cn, N, cap, offs, iota, n_recs, coffN, d_ri, nthreads, g->pfine,
                                             g->sstep, g->target, g->d_maxP, nullptr, g->cap_threads);
        } else {
            const int M = N - 1;
            const FLevel &pf = g->F[M];
            int32_t *cp = g->ctr + (size_t)M * kCtr;  // previous level's counters
            if (fuse_join) {
                k_g_join_fused<<<1, 1024, 0, st>>>(pf.types, pf.lo, pf.hi, pf.rec, pf.foff, cp, M, cap, ct, cl, ch,
                                                   crec, cn, g->rel + N, offs, iota, n_recs, coffN, d_ri, nthreads,
                                                   g->pfine, g->sstep, g->target, g->d_maxP);
                // local tracking: segment again, allowing for the largest
                // prefix group
                if (g->track && cst == FEM_OK) {
                    cst = track_group_starts(st, ctx->n_sm, group_in());
                    groups_ready = cst == FEM_OK;
                    k_g_levelinfo<<<1, 256, 0, st>>>(crec, cn, N, cap, offs, iota, n_recs, coffN, d_ri, nthreads,
                                                     g->pfine, g->sstep, g->target, g->d_maxP,
                                                     groups_ready ? g->tg_gmax : nullptr, g->cap_threads);
                }
            } else {
                k_g_join_count<<<gb, 256, 0, st>>>(pf.types, pf.lo, pf.hi, pf.rec, pf.foff, cp, M, cap, pos);
                if (cst == FEM_OK) cst = scan_exclusive(st, pos, cap + 1, scan_tmp, nullptr, nullptr);
                k_g_join_write<<<gb, 256, 0, st>>>(pf.types, pf.lo, pf.hi, pf.rec, pf.foff, cp, M, cap, pos, ct, cl,
                                                   ch, crec, cn);
                k_g_level_index<<<gb, 256, 0, st>>>(cn, N, cap, offs, iota);
                // local tracking: the prefix groups first, so that the
                // segmentation can allow for the largest of them
                if (g->track && cst == FEM_OK) {
                    cst = track_group_starts(st, ctx->n_sm, group_in());
                    groups_ready = cst == FEM_OK;
                }
                k_g_levelinfo<<<1, 256, 0, st>>>(crec, cn, N, cap, offs, iota, n_recs, coffN, d_ri, nthreads,
                                                 g->pfine, g->sstep, g->target, g->d_maxP,
                                                 groups_ready ? g->tg_gmax : nullptr, g->cap_threads);
            }
        }
        const bool bounded = g->coarse && N >= 3;
        if (bounded && cst == FEM_OK)
            cst = coarse_graph_level(st, ctx->n_sm, N, ct, cl, ch, crec, cn, cap, g->d_cdesc, g->coarse_slices,
                                     g->d_thr, g->coarse_min, g->cub, g->skip);
        const bool jbound = g->jb && N == 3;
        if (jbound && cst == FEM_OK) {
            const FLevel &f2 = g->F[2];
            JoinBoundArgs ja{};
            ja.ri = d_ri;
            ja.n_recs = n_recs;
            ja.stride = g->jb_stride;
            ja.f2types = f2.types;
            ja.f2lo = f2.lo;
            ja.f2hi = f2.hi;
            ja.f2rec = f2.rec;
            ja.f2foff = f2.foff;
            ja.f2n = g->ctr + 2 * kCtr + 1;
            ja.tab_off = g->jb_tab_off;
            ja.nt = g->jb_nt;
            ja.tab = g->jb_tab;
            ja.tab_n = g->jb_tab_n;
            ja.blo = d_blo;
            ja.bhi = d_bhi;
            ja.nb = nb;
            ja.ct = ct;
            ja.cl = cl;
            ja.ch = ch;
            ja.crec = crec;
            ja.cn = cn;
            ja.thr = g->d_thr;
            ja.vbits = g->jb_v;
            ja.sbits = g->jb_s;
            ja.cap_words = g->jb_cap_words;
            ja.nch = (int)std::max<int64_t>(1, (g->track_cap + 1023) / 1024);
            ja.base = g->jb_base;
            ja.skip = g->skip;
            ja.or_skip = bounded ? 1 : 0;
            ja.skipc = g->jb_skipc;
            cst = join_bound_level3(st, ctx->n_sm, ja);
        }
        const bool skipping = bounded || jbound;
        k_g_ringcheck<<<gb, 256, 0, st>>>(ct, cl, crec, cn, N, need_dens ? d_dens : nullptr, d_lov,
                                          (int)lo_vals.size(), g->ring_cap, d_ri,
                                          cn, g->rel + N, n_recs, g->segf, g->pfine, g->sstep, g->segl,
                                          skipping ? g->skip : nullptr);
        // external event nodes: their timestamps time the count kernels of
        // this level on every launch of the graph
        ok(cudaEventRecordWithFlags(g->ev[2 * N], st, cudaEventRecordExternal));
        if (cst == FEM_OK && g->track) {
            TrackArgs ta{};
            ta.rinfo = d_ri;
            ta.n_recs = n_recs;
            ta.offs = offs;
            ta.ctypes = ct;
            ta.clo = cl;
            ta.chi = ch;
            ta.slot2cand = iota;
            ta.skip = skipping ? g->skip : nullptr;
            ta.queue = reinterpret_cast<unsigned long long *>(g->tqueue);
            ta.buf = g->tbuf;
            ta.cap = g->track_cap;
            ta.rec = rec;
            ta.counts = counts;  // unsegmented recordings: counts written directly
            ta.last_mode = ctx->tuning.track_last;
            // items: recordings longest first; level 2 shares no prefix
            // work (one item per episode and segment), levels >= 3 group
            // episodes by their (N-1)-node prefix
            TrackGroupIn gi = group_in();
            gi.starts_ready = groups_ready;
            cst = track_groups(st, ctx->n_sm, gi, N >= 3, &ta);
            if (cst == FEM_OK) cst = launch_track(st, g->track_nblocks, ta);
            if (cst == FEM_OK)
                cst = launch_stitch_dev(st, ctx->n_sm, d_ri, iota, crec, rec, cn, cap, counts, fb_list, cn + 3,
                                        skipping ? g->skip : nullptr, g->d_maxP, 1);
        } else if (cst == FEM_OK) {
            cst = launch_count_dev(st, nmax, N, g->ring_cap, d_ri, n_recs, nthreads, g->cap_threads, offs, ct, cl, ch,
                                   iota, crec, rec, cn, cap, counts, fb_list, cn + 3, d_dens, d_lov,
                                   (int)lo_vals.size(), skipping ? g->skip : nullptr);
        }
        ok(cudaEventRecordWithFlags(g->ev[2 * N + 1], st, cudaEventRecordExternal));
        if (fused) {
            k_g_thr_fused<<<1, 1024, 0, st>>>(counts, ct, cl, ch, crec, g->d_thr, N, cap, nf.types, nf.lo, nf.hi,
                                              nf.rec, nf.counts, cn, n_recs, nf.foff);
        } else {
            k_g_thr_flags<<<gb, 256, 0, st>>>(counts, crec, g->d_thr, cn, cap, pos);
            if (cst == FEM_OK) cst = scan_exclusive(st, pos, cap + 1, scan_tmp, nullptr, nullptr);
            k_g_thr_write<<<gb, 256, 0, st>>>(pos, counts, ct, cl, ch, crec, g->d_thr, N, cap, nf.types, nf.lo,
                                              nf.hi, nf.rec, nf.counts, cn);
            k_g_foff<<<1, 256, 0, st>>>(nf.rec, cn, n_recs, nf.foff);
        }
        ok(cudaGetLastError());
    }
    if (cst == FEM_OK) {
        k_g_pack<<<(unsigned)(2 * ctx->n_sm), 256, 0, st>>>(ctx->d_status, g->ctr, g->coff, g->coff2, g->rel,
                                                           g->jb ? g->jb_skipc : nullptr, d_F, g->lay, first, L,
                                                           n_recs, d_out);
        ok(cudaGetLastError());
    }
    const cudaError_t ce = cudaStreamEndCapture(st, &graph);
    if (cst != FEM_OK || ce != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return cst != FEM_OK ? cst : FEM_ERR_CUDA;
    }
    // kernel nodes of the graph (reported as kernel launches per run)
    size_t n_nodes = 0;
    if (cudaGraphGetNodes(graph, nullptr, &n_nodes) == cudaSuccess && n_nodes > 0) {
        std::vector<cudaGraphNode_t> nodes(n_nodes);
        if (cudaGraphGetNodes(graph, nodes.data(), &n_nodes) == cudaSuccess)
            for (auto nd : nodes) {
                cudaGraphNodeType ty;
                if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++g->kernel_nodes;
            }
    }
    cudaGetLastError();
    const cudaError_t ie = cudaGraphInstantiate(&g->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
        cudaGetLastError();
        g->exec = nullptr;
        return FEM_ERR_CUDA;
    }
    return FEM_OK;
}

static std::string graph_key(const std::vector<fem_stream *> &recs, const std::vector<int32_t> &blo,
                             const std::vector<int32_t> &bhi, const std::vector<uint32_t> &thr, int max_size,
                             int first, bool prepass, int coarse, int kernel, int track_last) {
    std::ostringstream k;
    for (auto *s : recs) k << (const void *)s << ':' << s->n << ';';
    for (size_t i = 0; i < blo.size(); ++i) k << blo[i] << ',' << bhi[i] << ';';
    for (auto t : thr) k << t << ';';
    k << max_size << '/' << first << '/' << (prepass ? 1 : 0) << '/' << coarse << '/' << kernel << '/' << track_last;
    return k.str();
}

void graph_cache_clear(fem_ctx *ctx) {
    for (auto &kv : ctx->graphs) delete kv.second;
    ctx->graphs.clear();
}

void graph_cache_forget(fem_ctx *ctx, const fem_stream *s) {
    for (auto it = ctx->graphs.begin(); it != ctx->graphs.end();) {
        bool uses = false;
        for (auto *r : it->second->recs) uses = uses || r == s;
        if (uses) {
            ctx->graph_cap.erase(it->first);
            delete it->second;
            it = ctx->graphs.erase(it);
        } else {
            ++it;
        }
    }
}

namespace {

// Level-2 frequent set handed to a graph that starts at level 3.
struct Level2In {
    int64_t F2;
    const uint16_t *types;
    const int32_t *lo, *hi;
    const uint32_t *rec, *counts;
    const std::vector<int64_t> *off;
};

}  // namespace

// Runs levels first..max_size through the cached (or newly captured) graph.
static int run_graph(fem_ctx *ctx, const std::vector<fem_stream *> &recs, const std::vector<int32_t> &blo,
                     const std::vector<int32_t> &bhi, const std::vector<uint32_t> &thr,
                     const std::vector<int32_t> &lo_vals, int max_size, int first, bool prepass, int64_t cap_min,
                     const Level2In *in2, TailResult *out, bool *used) {
    *used = false;
    const int n_recs = (int)recs.size();
    for (auto *s : recs)
        if (s->n_types > 8192 || s->n > INT32_MAX / 2) return FEM_OK;
    // coarse-tick bound of levels >= 3: only with prepass = 1; level-3 join
    // bound: with prepass 0 (the default) or 1
    const int coarse = ctx->tuning.prepass == 1 ? 1 : 0;
    const bool jb_on = ctx->tuning.prepass == 0 || ctx->tuning.prepass == 1;
    const std::string key = graph_key(recs, blo, bhi, thr, max_size, first, prepass, coarse + 2 * (jb_on ? 1 : 0),
                                      ctx->tuning.kernel, ctx->tuning.track_last);
    int64_t cap = 4096;
    auto hint = ctx->graph_cap.find(key);
    const int64_t want = std::max<int64_t>(cap_min, hint != ctx->graph_cap.end() ? hint->second : 0);
    while (cap < want && cap < (1 << 24)) cap <<= 1;
    if (cap < want) return FEM_OK;
    GraphTail *g = nullptr;
    auto it = ctx->graphs.find(key);
    if (it != ctx->graphs.end() && it->second->cap >= cap) {
        g = it->second;
    } else {
        if (it != ctx->graphs.end()) {
            delete it->second;
            ctx->graphs.erase(it);
        }
        if (ctx->graphs.size() >= 4) graph_cache_clear(ctx);
        std::unique_ptr<GraphTail> ng(new GraphTail());
        ng->ctx = ctx;
        ng->key = key;
        ng->recs = recs;
        ng->n_recs = n_recs;
        ng->max_size = max_size;
        ng->first = first;
        ng->prepass = prepass;
        ng->jb_on = jb_on;
        ng->coarse = coarse;
        ng->coarse_min = 0;
        ng->cap = cap;
        const int st = build_graph(ng.get(), blo, bhi, thr, lo_vals);
        if (st == FEM_ERR_NOMEM || st == FEM_ERR_INVAL) return FEM_OK;  // not applicable: host path
        if (st != FEM_OK) return st;
        g = ng.release();
        ctx->graphs[key] = g;
    }
    cudaStream_t st = ctx->stream;
    if (first == 3) {
        if (!in2 || in2->F2 > g->cap) return FEM_OK;
        FLevel &f2 = g->F[2];
        const int64_t F2 = in2->F2;
        FEM_CUDA_TRY(cudaMemcpyAsync(f2.types, in2->types, 2 * 2 * F2, cudaMemcpyDeviceToDevice, st));
        FEM_CUDA_TRY(cudaMemcpyAsync(f2.lo, in2->lo, 4 * F2, cudaMemcpyDeviceToDevice, st));
        FEM_CUDA_TRY(cudaMemcpyAsync(f2.hi, in2->hi, 4 * F2, cudaMemcpyDeviceToDevice, st));
        FEM_CUDA_TRY(cudaMemcpyAsync(f2.rec, in2->rec, 4 * F2, cudaMemcpyDeviceToDevice, st));
        FEM_CUDA_TRY(cudaMemcpyAsync(f2.counts, in2->counts, 4 * F2, cudaMemcpyDeviceToDevice, st));
        FEM_CUDA_TRY(cudaMemcpyAsync(f2.foff, in2->off->data(), 8 * (n_recs + 1), cudaMemcpyHostToDevice, st));
        std::vector<int32_t> c2(kCtr, 0);
        c2[1] = (int32_t)F2;
        FEM_CUDA_TRY(cudaMemcpyAsync(g->ctr + 2 * kCtr, c2.data(), 4 * kCtr, cudaMemcpyHostToDevice, st));
    }
    cudaEventRecord(ctx->ev0, st);
    FEM_CUDA_TRY(cudaGraphLaunch(g->exec, st));
    cudaEventRecord(ctx->ev1, st);
    FEM_CUDA_TRY(cudaStreamSynchronize(st));
    const char *ho = g->h_out;
    const int status = *reinterpret_cast<const int *>(ho);
    if (status) {
        FEM_CUDA_TRY(cudaMemsetAsync(ctx->d_status, 0, sizeof(int), st));
        FEM_CUDA_TRY(cudaStreamSynchronize(st));
        if (status & kStatusTimeout) return FEM_ERR_TIMEOUT;
        return FEM_ERR_INVAL;
    }
    const int32_t *ctr = reinterpret_cast<const int32_t *>(ho + g->lay.o_ctr);
    const int64_t *coff = reinterpret_cast<const int64_t *>(ho + g->lay.o_coff);
    const int64_t *coff2 = reinterpret_cast<const int64_t *>(ho + g->lay.o_coff2);
    const unsigned long long *rel = reinterpret_cast<const unsigned long long *>(ho + g->lay.o_rel);
    bool flagged = false;
    int64_t need = 0;
    for (int N = std::max(first, 2); N <= max_size; ++N) {
        const int32_t *c = &ctr[(size_t)N * kCtr];
        if (c[2] != 0 || c[3] != 0) flagged = true;
        if (c[2] & kFlagCap) need = std::max<int64_t>(need, (int64_t)c[5] + 1);
        if (c[2] & kFlagFreq) need = std::max<int64_t>(need, 2 * g->cap);
    }
    if (flagged) {
        // redo on the host path; a capacity overflow grows the next capture
        if (need > 0) ctx->graph_cap[key] = std::max<int64_t>(need, 2 * g->cap);
        return FEM_OK;
    }
    float gms = 0.f;
    cudaEventElapsedTime(&gms, ctx->ev0, ctx->ev1);
    out->graph_ms = gms;
    out->kernel_nodes = g->kernel_nodes;
    out->count_levels = max_size - std::max(first, 2) + 1;
    // count-kernel time of the levels from the graph's event nodes (the whole
    // graph's time if the driver cannot time them)
    float cms = 0.f;
    bool timed = true;
    for (int N = std::max(first, 2); N <= max_size && timed; ++N) {
        float m = 0.f;
        if (cudaEventElapsedTime(&m, g->ev[2 * N], g->ev[2 * N + 1]) != cudaSuccess) timed = false;
        cms += m;
    }
    if (!timed) cudaGetLastError();
    out->count_ms = timed ? cms : gms;
    out->relevant = 0.0;
    for (int N = std::max(first, 2); N <= max_size; ++N) out->relevant += (double)rel[N];
    // results
    out->levels.clear();
    for (int N = first; N <= max_size; ++N) {
        const int32_t *c = &ctr[(size_t)N * kCtr];
        TailLevel tl;
        tl.N = N;
        tl.C = N == 1 ? 0 : c[0];
        if (N >= 2) {
            tl.coff.assign(coff + (size_t)N * (n_recs + 1), coff + (size_t)(N + 1) * (n_recs + 1));
            tl.goff = (N == 2 && first <= 2) ? std::vector<int64_t>(coff2, coff2 + n_recs + 1) : tl.coff;
            tl.skipped.assign(n_recs, 0);
            if (N == 3 && g->jb) {
                const int64_t *sk = reinterpret_cast<const int64_t *>(ho + g->lay.o_skip3);
                tl.skipped.assign(sk, sk + n_recs);
            }
        }
        const int64_t Fn = c[1], fc = g->lay.fcap[N];
        const char *o = ho + g->lay.o_lvl[N];
        const int64_t tb = ((2 * fc * N) + 7) / 8 * 8, eb = 4 * fc * (N - 1);
        const uint16_t *ty = reinterpret_cast<const uint16_t *>(o);
        const int32_t *lo = reinterpret_cast<const int32_t *>(o + tb);
        const int32_t *hi = reinterpret_cast<const int32_t *>(o + tb + eb);
        const uint32_t *rc = reinterpret_cast<const uint32_t *>(o + tb + 2 * eb);
        const uint32_t *ct = reinterpret_cast<const uint32_t *>(o + tb + 2 * eb + 4 * fc);
        tl.types.assign(ty, ty + Fn * N);
        tl.lo.assign(lo, lo + Fn * (N - 1));
        tl.hi.assign(hi, hi + Fn * (N - 1));
        tl.rec.assign(rc, rc + Fn);
        tl.counts.assign(ct, ct + Fn);
        out->levels.push_back(std::move(tl));
        if ((N >= 2 && c[0] == 0) || Fn == 0) break;
    }
    *used = true;
    return FEM_OK;
}

int run_graph_mining(fem_ctx *ctx, const std::vector<fem_stream *> &recs, const std::vector<int32_t> &blo,
                     const std::vector<int32_t> &bhi, const std::vector<uint32_t> &thr,
                     const std::vector<int32_t> &lo_vals, int max_size, bool prepass, TailResult *out, bool *used) {
    *used = false;
    if (max_size < 2 || blo.empty() || blo.size() > 8) return FEM_OK;
    for (auto *s : recs)
        if (s->n_types > 1024) prepass = false;
    // without the pre-pass every level-2 pair is counted: capacity for all
    int64_t cap_min = 0;
    if (!prepass)
        for (auto *s : recs) cap_min += (int64_t)s->n_types * (s->n_types - 1) * (int64_t)blo.size();
    return run_graph(ctx, recs, blo, bhi, thr, lo_vals, max_size, 1, prepass, cap_min, nullptr, out, used);
}

// Levels 3..max_size from the level-2 frequent set (device arrays +
// per-recording offsets).  Returns FEM_OK and fills `out` when every level
// completed without a flag; *used = false when the graph path did not apply
// (the caller then continues on the host-driven path).
int run_graph_tail(fem_ctx *ctx, const std::vector<fem_stream *> &recs, const std::vector<int32_t> &blo,
                   const std::vector<int32_t> &bhi, const std::vector<uint32_t> &thr, const std::vector<int32_t> &lo_vals,
                   int max_size, int64_t F2, const uint16_t *f2_types, const int32_t *f2_lo, const int32_t *f2_hi,
                   const uint32_t *f2_rec, const uint32_t *f2_counts, const std::vector<int64_t> &f2_off,
                   TailResult *out, bool *used) {
    *used = false;
    const int n_recs = (int)recs.size();
    if (max_size < 3 || F2 == 0) return FEM_OK;
    // capacity: the first join cannot exceed sum over recordings of F2_r^2
    int64_t bound = 0;
    for (int r = 0; r < n_recs; ++r) {
        const int64_t f = f2_off[r + 1] - f2_off[r];
        bound += f * f;
    }
    const Level2In in2{F2, f2_types, f2_lo, f2_hi, f2_rec, f2_counts, &f2_off};
    return run_graph(ctx, recs, blo, bhi, thr, lo_vals, max_size, 3, false, std::min<int64_t>(2 * bound, 1 << 18),
                     &in2, out, used);
}

}  // namespace fem
