// fem_plt.cu -- counting by node-by-node local tracking, for few episodes.
//
// Section "Parallel Local Tracking" (Algorithm 2) finds the occurrences of an
// episode node by node, in parallel over the events of each node's type, and
// "Problem decomposition" then removes overlaps with the greedy of
// Algorithm 1.  Here the tracking keeps, per event of node k's type, only the
// latest start of any partial occurrence of nodes 1..k ending at that event
// (the greedy needs no other start), so one step per node does:
//   for every event j of type E_{k+1} (one thread each):
//     i* = last event of E_k with t_i < t_j - lo_k   (binary search in E_k's list)
//     v  = newest E_k event at or before i* that ends a partial occurrence
//          (an inclusive max-scan of valid positions over E_k's list)
//     L_{k+1}(j) = L_k(v) when t_v >= t_j - hi_k, else none;
// the latest start is non-decreasing along a node's valid events, so v
// carries the largest start in the window.  After the last node, Algorithm 1
// walks the end events in time order and keeps an end when its latest start
// is after the previous kept end.  Work per episode is its node types' events
// (times a logarithm), spread over all events, so a single long episode on a
// long stream still fills the GPU -- the regime the section addresses.
#include <algorithm>
#include <map>
#include <tuple>
#include <vector>

#include "fem_internal.cuh"

namespace fem {

namespace {

// One episode in one step: its node-k list (A) and node-(k+1) list (B).
struct PltItem {
    int64_t a_start, b_start;  // first index of the lists in the recording's per-type times
    int32_t fa, fb;            // list lengths
    int64_t prev_base;         // first position of A's values in the previous step's arrays
    int64_t base;              // first position of B's values in this step's arrays
    const int32_t *ttime;      // the recording's per-type times
    int32_t lo, hi;
    int32_t j0;                // last step: first B position whose end may be counted
};

__device__ __forceinline__ int item_of(const PltItem *items, int n_items, int64_t g) {
    int lo = 0, hi = n_items;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (items[mid].base <= g) lo = mid; else hi = mid;
    }
    return lo;
}

// Step k -> k+1 for every (episode, event of E_{k+1}) pair; first = k is
// node 1 (every E_1 event starts a partial occurrence at its own time).
__global__ void k_plt_step(const PltItem *__restrict__ items, int n_items, int64_t total, int first,
                           const int32_t *__restrict__ Lprev, const int32_t *__restrict__ Vprev,
                           int32_t *__restrict__ Lnext, int32_t *__restrict__ flag) {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total; g += (int64_t)gridDim.x * blockDim.x) {
        const PltItem it = items[item_of(items, n_items, g)];
        const int64_t j = g - it.base;
        const int32_t *ta = it.ttime + it.a_start;
        const int64_t tj = it.ttime[it.b_start + j];
        // i* = last A event with t < tj - lo
        int64_t lo = 0, hi = it.fa;
        const int64_t lim = tj - it.lo;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if ((int64_t)ta[mid] < lim) lo = mid + 1; else hi = mid;
        }
        const int64_t istar = lo - 1;
        int32_t L = INT32_MIN;
        if (istar >= 0) {
            int64_t v;
            int32_t Lv;
            if (first) {
                v = istar;
                Lv = ta[istar];
            } else {
                const int64_t gv = Vprev[it.prev_base + istar];  // global position or -1
                v = gv >= it.prev_base ? gv - it.prev_base : -1;
                Lv = v >= 0 ? Lprev[gv] : INT32_MIN;
            }
            if (v >= 0 && (int64_t)ta[v] >= tj - it.hi) L = Lv;
        }
        Lnext[g] = L;
        flag[g] = L != INT32_MIN ? (int32_t)g : -1;
    }
}

// Inclusive max-scan of int32 (three passes: per-block scan, scan of the
// block maxima, add-back).
constexpr int kMsBlock = 1024;
// Entries an occurrence list may hold (episodes beyond it are counted by the
// latest-start steps).
constexpr int64_t kOccCap = int64_t(1) << 25;
// Largest total length of one step's arrays in a latest-start launch.
constexpr int64_t kPltMaxTotal = int64_t(1) << 28;

__global__ void k_maxscan_blocks(int32_t *d, int64_t m, int32_t *bmax) {
    __shared__ int32_t s_w[32];
    const int64_t i = blockIdx.x * (int64_t)kMsBlock + threadIdx.x;
    int32_t x = i < m ? d[i] : -1;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x = max(x, y);
    }
    if (lane == 31) s_w[w] = x;
    __syncthreads();
    if (w == 0) {
        int32_t t = s_w[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xFFFFFFFFu, t, o);
            if (lane >= o) t = max(t, y);
        }
        s_w[lane] = t;
    }
    __syncthreads();
    if (w > 0) x = max(x, s_w[w - 1]);
    if (i < m) d[i] = x;
    if (threadIdx.x == kMsBlock - 1) bmax[blockIdx.x] = x;
}

__global__ void k_maxscan_top(int32_t *bmax, int64_t nb) {
    // one block: sequential carry over chunks of kMsBlock block maxima
    __shared__ int32_t s_w[32];
    __shared__ int32_t s_carry;
    if (threadIdx.x == 0) s_carry = -1;
    __syncthreads();
    for (int64_t c0 = 0; c0 < nb; c0 += kMsBlock) {
        const int64_t i = c0 + threadIdx.x;
        int32_t x = i < nb ? bmax[i] : -1;
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
            if (lane >= o) x = max(x, y);
        }
        if (lane == 31) s_w[w] = x;
        __syncthreads();
        if (w == 0) {
            int32_t t = s_w[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t y = __shfl_up_sync(0xFFFFFFFFu, t, o);
                if (lane >= o) t = max(t, y);
            }
            s_w[lane] = t;
        }
        __syncthreads();
        if (w > 0) x = max(x, s_w[w - 1]);
        x = max(x, s_carry);
        if (i < nb) bmax[i] = x;
        __syncthreads();
        if (threadIdx.x == kMsBlock - 1) s_carry = x;
        __syncthreads();
    }
}

__global__ void k_maxscan_add(int32_t *d, int64_t m, const int32_t *bmax) {
    const int64_t i = blockIdx.x * (int64_t)kMsBlock + threadIdx.x;
    if (blockIdx.x > 0 && i < m) d[i] = max(d[i], bmax[blockIdx.x - 1]);
}

// Algorithm 1 over an episode's end events (its last node's list, in time
// order): keep an end when its latest start is after the previous kept end.
// The latest starts are non-decreasing along the valid ends, so with PM(j) =
// the latest start of the newest valid end at or before j (from the max-scan
// of valid positions), the end kept after end j is the first j' with
// PM(j') > t_j (a binary search), and the first end kept is the first valid
// one.  The count is the length of the chain from there, by pointer jumping.
__device__ __forceinline__ int32_t plt_pm(const int32_t *L, const int32_t *V, int64_t base, int64_t j) {
    const int32_t v = V[base + j];
    return v >= base ? L[v] : INT32_MIN;
}

// nxt[g] = global position of the end kept after g (or -1); cnt[g] = 1 for
// valid ends.
__global__ void k_plt_next(const PltItem *__restrict__ items, int n_items, int64_t total,
                           const int32_t *__restrict__ L, const int32_t *__restrict__ V, int32_t *__restrict__ nxt,
                           int32_t *__restrict__ cnt, int32_t *__restrict__ lst) {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total; g += (int64_t)gridDim.x * blockDim.x) {
        const PltItem it = items[item_of(items, n_items, g)];
        const int64_t j = g - it.base;
        int32_t nx = -1, c = 0;
        if (L[g] != INT32_MIN) {
            c = 1;
            const int64_t tj = it.ttime[it.b_start + j];
            int64_t lo = j + 1, hi = it.fb;  // first j' > j with PM(j') > t_j
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if ((int64_t)plt_pm(L, V, it.base, mid) > tj) hi = mid; else lo = mid + 1;
            }
            if (lo < it.fb) nx = (int32_t)(it.base + lo);
        }
        nxt[g] = nx;
        cnt[g] = c;
        if (lst) lst[g] = (int32_t)g;
    }
}

// One pointer-jumping round: cnt'[g] = cnt[g] + cnt[nxt[g]], nxt'[g] =
// nxt[nxt[g]], and (optionally) the chain's last end lst'[g] = lst[nxt[g]].
__global__ void k_plt_jump(int64_t total, const int32_t *__restrict__ nxt, const int32_t *__restrict__ cnt,
                           int32_t *__restrict__ nxt2, int32_t *__restrict__ cnt2, const int32_t *__restrict__ lst,
                           int32_t *__restrict__ lst2) {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total; g += (int64_t)gridDim.x * blockDim.x) {
        const int32_t n = nxt[g];
        cnt2[g] = cnt[g] + (n >= 0 ? cnt[n] : 0);
        nxt2[g] = n >= 0 ? nxt[n] : -1;
        if (lst) lst2[g] = n >= 0 ? lst[n] : lst[g];
    }
}

// Episode e's last-step item is items[idx[e]] (items[e] without idx).
// count = chain length from the first kept end: the first j >= j0 with
// PM(j) > prev, prev = the previous kept end (-inf without `prev`).  With
// `prev` (appended events) the count is added and prev becomes the time of
// the chain's last end; earlier ends (j < j0) have latest starts <= prev, so
// PM over them never passes prev.
__global__ void k_plt_count(const PltItem *__restrict__ items, int n_eps, const int32_t *__restrict__ idx,
                            const int32_t *__restrict__ L, const int32_t *__restrict__ V,
                            const int32_t *__restrict__ cnt, const int32_t *__restrict__ cand,
                            uint32_t *__restrict__ counts, int32_t *__restrict__ prev,
                            const int32_t *__restrict__ lst) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_eps) return;
    const PltItem it = items[idx ? idx[e] : e];
    const int32_t pv = prev ? prev[cand[e]] : INT32_MIN;
    int64_t lo = it.j0, hi = it.fb;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (plt_pm(L, V, it.base, mid) > pv) hi = mid; else lo = mid + 1;
    }
    const bool hit = lo < it.fb && plt_pm(L, V, it.base, lo) > pv;
    if (!prev) {
        counts[cand[e]] = hit ? (uint32_t)cnt[it.base + lo] : 0u;
    } else if (hit) {
        counts[cand[e]] += (uint32_t)cnt[it.base + lo];
        prev[cand[e]] = it.ttime[it.b_start + (lst[it.base + lo] - it.base)];
    }
}

// 1-node episodes: the count is the type's number of (new) events.
__global__ void k_n1_counts(const int32_t *__restrict__ cand, const uint32_t *__restrict__ val, int n,
                            uint32_t *__restrict__ counts, int accumulate) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    counts[cand[i]] = (accumulate ? counts[cand[i]] : 0u) + val[i];
}

// ---- the section's own form: every partial occurrence, node by node ------
// An occurrence list holds (start time, position in the current node's type
// list).  A step finds, for each partial occurrence ending at time t, the
// next node's events in (t + lo, t + hi] (two binary searches) and emits one
// entry per event; the output is compacted either with atomics (a block
// reserves its range with one global atomic after its threads reserved
// theirs in shared memory, "Lock-based compaction") or with count, scan,
// write ("Lock-free compaction").  After the last node the latest start per
// end event feeds the same overlap removal as above.

__device__ __forceinline__ void occ_range(const int32_t *tb, int64_t fb, int64_t t, int32_t lo, int32_t hi,
                                          int64_t &j0, int64_t &j1) {
    int64_t a = 0, b = fb;
    while (a < b) {  // first event with time > t + lo
        const int64_t mid = (a + b) >> 1;
        if ((int64_t)tb[mid] <= t + lo) a = mid + 1; else b = mid;
    }
    j0 = a;
    b = fb;
    while (a < b) {  // first event with time > t + hi
        const int64_t mid = (a + b) >> 1;
        if ((int64_t)tb[mid] <= t + hi) a = mid + 1; else b = mid;
    }
    j1 = a;
}

__global__ void k_occ_init(const int32_t *__restrict__ ta, int64_t fa, int32_t *__restrict__ s, int32_t *__restrict__ p) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < fa; i += (int64_t)gridDim.x * blockDim.x) {
        s[i] = ta[i];
        p[i] = (int32_t)i;
    }
}

// Lock-free compaction, count pass: matches per partial occurrence, and
// their exact 64-bit total (the int32 scan runs only when it fits).
__global__ void k_occ_count(const int32_t *__restrict__ p, int64_t m, const int32_t *__restrict__ ta,
                            const int32_t *__restrict__ tb, int64_t fb, int32_t lo, int32_t hi,
                            int32_t *__restrict__ cnt, unsigned long long *total) {
    for (int64_t o0 = blockIdx.x * (int64_t)blockDim.x; o0 <= m; o0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = o0 + threadIdx.x;
        int64_t c = 0;
        if (o < m) {
            int64_t j0, j1;
            occ_range(tb, fb, ta[p[o]], lo, hi, j0, j1);
            c = j1 - j0;
        }
        if (o <= m) cnt[o] = (int32_t)min(c, (int64_t)INT32_MAX);
        unsigned long long w = (unsigned long long)c;
        for (int q = 16; q > 0; q >>= 1) w += __shfl_down_sync(0xFFFFFFFFu, w, q);
        if ((threadIdx.x & 31) == 0 && w) atomicAdd(total, w);
    }
}

__global__ void k_fill_i32(int32_t *d, int64_t n, int32_t v) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        d[i] = v;
}

// Lock-free compaction, write pass at the scanned offsets.
__global__ void k_occ_write_scan(const int32_t *__restrict__ s, const int32_t *__restrict__ p, int64_t m,
                                 const int32_t *__restrict__ off, const int32_t *__restrict__ ta,
                                 const int32_t *__restrict__ tb, int64_t fb, int32_t lo, int32_t hi, int64_t cap,
                                 int32_t *__restrict__ s2, int32_t *__restrict__ p2) {
    for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < m; o += (int64_t)gridDim.x * blockDim.x) {
        int64_t j0, j1;
        occ_range(tb, fb, ta[p[o]], lo, hi, j0, j1);
        int64_t w = off[o];
        for (int64_t j = j0; j < j1 && w < cap; ++j, ++w) {
            s2[w] = s[o];
            p2[w] = (int32_t)j;
        }
    }
}

// Lock-based compaction: threads reserve in shared memory, the block once
// globally; *total counts every match (capacity overflow when > cap).
__global__ void k_occ_write_atomic(const int32_t *__restrict__ s, const int32_t *__restrict__ p, int64_t m,
                                   const int32_t *__restrict__ ta, const int32_t *__restrict__ tb, int64_t fb,
                                   int32_t lo, int32_t hi, int64_t cap, int32_t *__restrict__ s2,
                                   int32_t *__restrict__ p2, unsigned long long *total) {
    __shared__ unsigned long long s_cnt, s_base;
    for (int64_t o0 = blockIdx.x * (int64_t)blockDim.x; o0 < m; o0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = o0 + threadIdx.x;
        if (threadIdx.x == 0) s_cnt = 0;
        __syncthreads();
        int64_t j0 = 0, j1 = 0;
        if (o < m) occ_range(tb, fb, ta[p[o]], lo, hi, j0, j1);
        const unsigned long long mine = atomicAdd(&s_cnt, (unsigned long long)(j1 - j0));
        __syncthreads();
        if (threadIdx.x == 0) s_base = atomicAdd(total, (unsigned long long)s_cnt);
        __syncthreads();
        int64_t w = (int64_t)(s_base + mine);
        for (int64_t j = j0; j < j1 && w < cap; ++j, ++w) {
            s2[w] = s[o];
            p2[w] = (int32_t)j;
        }
        __syncthreads();
    }
}

// Latest start per end event (positions in the last node's list).
__global__ void k_occ_final(const int32_t *__restrict__ s, const int32_t *__restrict__ p, int64_t m,
                            int32_t *__restrict__ L) {
    for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < m; o += (int64_t)gridDim.x * blockDim.x)
        atomicMax(&L[p[o]], s[o]);
}

__global__ void k_occ_flags(const int32_t *__restrict__ L, int64_t fb, int32_t *__restrict__ V) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < fb; j += (int64_t)gridDim.x * blockDim.x)
        V[j] = L[j] != INT32_MIN ? (int32_t)j : -1;
}

}  // namespace

static int maxscan(cudaStream_t st, int32_t *d, int64_t m, int32_t *tmp) {
    if (m <= 0) return FEM_OK;
    const int64_t nb = (m + kMsBlock - 1) / kMsBlock;
    k_maxscan_blocks<<<(unsigned)nb, kMsBlock, 0, st>>>(d, m, tmp);
    if (nb > 1) {
        k_maxscan_top<<<1, kMsBlock, 0, st>>>(tmp, nb);
        k_maxscan_add<<<(unsigned)nb, kMsBlock, 0, st>>>(d, m, tmp);
    }
    FEM_CUDA_TRY(cudaGetLastError());
    return FEM_OK;
}

// One episode by occurrence lists (variant 1: atomic compaction, 2: count,
// scan, write).  *ok = false when a step's occurrences exceed `cap` (the
// caller then counts the episode with the latest-start steps).
static int count_occ_one(fem_ctx *ctx, const std::vector<PltItem> &its, int variant, int64_t cap, int32_t *s,
                         int32_t *p, int32_t *s2, int32_t *p2, int32_t *cnt, int32_t *scan_tmp,
                         unsigned long long *d_tot, int32_t *L, int32_t *V, int32_t *bm, int32_t *n1, int32_t *n2,
                         int32_t *c1, int32_t *c2, PltItem *d_item, const int32_t *d_cand, uint32_t *d_counts,
                         bool *ok, int64_t *launches) {
    cudaStream_t st = ctx->stream;
    *ok = true;
    const int N = (int)its.size() + 1;
    const unsigned g8 = (unsigned)(8 * ctx->n_sm);
    auto grid = [&](int64_t m) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((m + 255) / 256, g8)); };
    int64_t m = its[0].fa;
    const int32_t *ta0 = its[0].ttime + its[0].a_start;
    if (m > cap) {
        *ok = false;
        return FEM_OK;
    }
    k_occ_init<<<grid(m), 256, 0, st>>>(ta0, m, s, p);
    ++*launches;
    for (int k = 0; k + 1 < N && m > 0; ++k) {
        const PltItem &it = its[k];
        const int32_t *ta = it.ttime + it.a_start, *tb = it.ttime + it.b_start;
        unsigned long long tot = 0;
        FEM_CUDA_TRY(cudaMemsetAsync(d_tot, 0, 8, st));
        if (variant == 2) {
            k_occ_count<<<grid(m + 1), 256, 0, st>>>(p, m, ta, tb, it.fb, it.lo, it.hi, cnt, d_tot);
            FEM_CUDA_TRY(cudaMemcpyAsync(&tot, d_tot, 8, cudaMemcpyDeviceToHost, st));
            FEM_CUDA_TRY(cudaStreamSynchronize(st));
            if ((int64_t)tot > cap) {
                *ok = false;
                return FEM_OK;
            }
            FEM_TRY(scan_exclusive(st, cnt, m + 1, scan_tmp, nullptr, launches));
            k_occ_write_scan<<<grid(m), 256, 0, st>>>(s, p, m, cnt, ta, tb, it.fb, it.lo, it.hi, cap, s2, p2);
            *launches += 2;
        } else {
            k_occ_write_atomic<<<grid(m), 256, 0, st>>>(s, p, m, ta, tb, it.fb, it.lo, it.hi, cap, s2, p2, d_tot);
            FEM_CUDA_TRY(cudaMemcpyAsync(&tot, d_tot, 8, cudaMemcpyDeviceToHost, st));
            FEM_CUDA_TRY(cudaStreamSynchronize(st));
            if ((int64_t)tot > cap) {
                *ok = false;
                return FEM_OK;
            }
            ++*launches;
        }
        std::swap(s, s2);
        std::swap(p, p2);
        m = (int64_t)tot;
    }
    // latest start per end event, then the overlap removal of the other path
    const PltItem &last = its.back();
    const int64_t fb = last.fb;
    PltItem li = last;
    li.base = 0;
    FEM_CUDA_TRY(cudaMemcpyAsync(d_item, &li, sizeof(PltItem), cudaMemcpyHostToDevice, st));
    if (fb > 0) {
        k_fill_i32<<<grid(fb), 256, 0, st>>>(L, fb, INT32_MIN);
        if (m > 0) k_occ_final<<<grid(m), 256, 0, st>>>(s, p, m, L);
        k_occ_flags<<<grid(fb), 256, 0, st>>>(L, fb, V);
        FEM_TRY(maxscan(st, V, fb, bm));
        int rounds = 0;
        while ((int64_t(1) << rounds) < fb) ++rounds;
        k_plt_next<<<grid(fb), 256, 0, st>>>(d_item, 1, fb, L, V, n1, c1, nullptr);
        for (int q = 0; q < rounds; ++q) {
            k_plt_jump<<<grid(fb), 256, 0, st>>>(fb, n1, c1, n2, c2, nullptr, nullptr);
            std::swap(n1, n2);
            std::swap(c1, c2);
        }
        *launches += 6 + rounds;
    }
    k_plt_count<<<1, 32, 0, st>>>(d_item, 1, nullptr, L, V, c1, d_cand, d_counts, nullptr, nullptr);
    ++*launches;
    FEM_CUDA_TRY(cudaGetLastError());
    return FEM_OK;
}

// Counts the candidates `work` (indices into the CSR arrays on the device)
// by local tracking.  relaxed: every lower bound taken as 0.  variant 0:
// latest start per event; 1 / 2: occurrence lists with atomic / count-scan-
// write compaction.
int count_plt(fem_ctx *ctx, const std::vector<fem_stream *> &recs, const int64_t *d_offs, const uint16_t *d_types,
              const int32_t *d_lo, const int32_t *d_hi, const uint32_t *d_rec, const std::vector<int32_t> &work,
              bool relaxed, uint32_t *d_counts, fem_stats *stats, float *kernel_ms, int variant,
              const PltSession *sess) {
    if (sess && (variant != 0 || relaxed || recs.size() != 1)) return FEM_ERR_INVAL;
    cudaStream_t st = ctx->stream;
    const int64_t C = (int64_t)work.size();
    if (C == 0) return FEM_OK;
    // candidates to the host (few of them by construction)
    int32_t wmin = work[0], wmax = work[0];
    for (int32_t w : work) wmin = std::min(wmin, w), wmax = std::max(wmax, w);
    const int64_t span = (int64_t)wmax - wmin + 1;
    std::vector<int64_t> offs(span + 1);
    FEM_CUDA_TRY(cudaMemcpyAsync(offs.data(), d_offs + wmin, 8 * (span + 1), cudaMemcpyDeviceToHost, st));
    std::vector<uint32_t> crec(span, 0);
    if (d_rec) FEM_CUDA_TRY(cudaMemcpyAsync(crec.data(), d_rec + wmin, 4 * span, cudaMemcpyDeviceToHost, st));
    FEM_CUDA_TRY(cudaStreamSynchronize(st));
    const int64_t n0 = offs[0], n1 = offs[span];
    std::vector<uint16_t> types(n1 - n0);
    const int64_t e0 = n0 - wmin, e1 = n1 - (wmax + 1);
    std::vector<int32_t> lo(std::max<int64_t>(e1 - e0, 1)), hi(std::max<int64_t>(e1 - e0, 1));
    FEM_CUDA_TRY(cudaMemcpyAsync(types.data(), d_types + n0, 2 * (n1 - n0), cudaMemcpyDeviceToHost, st));
    if (e1 > e0) {
        FEM_CUDA_TRY(cudaMemcpyAsync(lo.data(), d_lo + e0, 4 * (e1 - e0), cudaMemcpyDeviceToHost, st));
        FEM_CUDA_TRY(cudaMemcpyAsync(hi.data(), d_hi + e0, 4 * (e1 - e0), cudaMemcpyDeviceToHost, st));
    }
    // per-type list offsets of every recording
    std::vector<std::vector<int64_t>> toff(recs.size());
    for (size_t r = 0; r < recs.size(); ++r) {
        FEM_TRY(stream_bytype(ctx, recs[r]));
        toff[r].resize(recs[r]->n_types + 1);
        FEM_CUDA_TRY(cudaMemcpyAsync(toff[r].data(), recs[r]->d_toff, 8 * toff[r].size(), cudaMemcpyDeviceToHost,
                                     st));
    }
    FEM_CUDA_TRY(cudaStreamSynchronize(st));
    // 1-node episodes: the frequency; others grouped by size
    std::vector<std::vector<int32_t>> by_n(FEM_MAX_NODES + 1);
    std::vector<uint32_t> n1_counts;
    std::vector<int32_t> n1_cand;
    double relevant = 0, counted = 0;
    for (int32_t w : work) {
        // the checks the per-episode kernels make on the device
        const int64_t o = offs[w - wmin], N = offs[w - wmin + 1] - o;
        const uint32_t r = crec[w - wmin];
        if (N < 1 || N > FEM_MAX_NODES || r >= recs.size()) return FEM_ERR_INVAL;
        for (int64_t k = 0; k < N; ++k)
            if (types[o - n0 + k] >= recs[r]->n_types) return FEM_ERR_INVAL;
        for (int64_t k = 0; k + 1 < N; ++k) {
            const int64_t eo = o - w - e0 + k;
            if (lo[eo] < 0 || lo[eo] >= hi[eo]) return FEM_ERR_INVAL;
        }
    }
    for (int32_t w : work) {
        const int64_t o = offs[w - wmin], N = offs[w - wmin + 1] - o;
        const uint32_t r = crec[w - wmin];
        counted += (double)recs[r]->n;
        const std::vector<int64_t> &tf = toff[r];
        for (int64_t k = 0; k < N; ++k) {
            const uint16_t a = types[o - n0 + k];
            relevant += (double)(tf[a + 1] - tf[a]);
        }
        if (N == 1) {
            const uint16_t a = types[o - n0];
            const int64_t old = sess ? (*sess->tail_cnt)[a] : 0;
            n1_cand.push_back(w);
            n1_counts.push_back((uint32_t)(tf[a + 1] - tf[a] - old));
        } else {
            by_n[N].push_back(w);
        }
    }
    if (!n1_cand.empty()) {
        // the count of a 1-node episode is the type's frequency (distinct
        // times); appended events add their own
        TmpDev t1(ctx);
        int32_t *dc;
        uint32_t *dv;
        const int n1n = (int)n1_cand.size();
        FEM_TRY(t1.get(&dc, n1n));
        FEM_TRY(t1.get(&dv, n1n));
        FEM_CUDA_TRY(cudaMemcpyAsync(dc, n1_cand.data(), 4 * n1n, cudaMemcpyHostToDevice, st));
        FEM_CUDA_TRY(cudaMemcpyAsync(dv, n1_counts.data(), 4 * n1n, cudaMemcpyHostToDevice, st));
        k_n1_counts<<<(n1n + 255) / 256, 256, 0, st>>>(dc, dv, n1n, d_counts, sess ? 1 : 0);
        FEM_CUDA_TRY(cudaGetLastError());
        stats->kernel_launches += 1;
    }
    float ms_total = 0.f;
    for (int N = 2; N <= FEM_MAX_NODES; ++N) {
        std::vector<int32_t> grp = by_n[N];
        if (grp.empty()) continue;
        // per step k: items and array sizes for the episodes in grp
        std::vector<std::vector<PltItem>> steps;
        std::vector<int64_t> tot;
        auto build_steps = [&]() {
            const int G = (int)grp.size();
            steps.assign(N - 1, std::vector<PltItem>(G));
            tot.assign(N - 1, 0);
            for (int k = 0; k + 1 < N; ++k) {
                int64_t base = 0;
                for (int e = 0; e < G; ++e) {
                    const int32_t w = grp[e];
                    const int64_t o = offs[w - wmin];
                    const int64_t eo = o - w;
                    const uint32_t r = crec[w - wmin];
                    const std::vector<int64_t> &tf = toff[r];
                    const uint16_t A = types[o - n0 + k], B = types[o - n0 + k + 1];
                    PltItem &it = steps[k][e];
                    it.a_start = tf[A];
                    it.fa = (int32_t)(tf[A + 1] - tf[A]);
                    it.b_start = tf[B];
                    it.fb = (int32_t)(tf[B + 1] - tf[B]);
                    it.prev_base = k > 0 ? steps[k - 1][e].base : 0;
                    it.base = base;
                    it.ttime = recs[r]->d_ttime;
                    it.lo = relaxed ? 0 : lo[eo - e0 + k];
                    it.hi = hi[eo - e0 + k];
                    it.j0 = sess && k + 2 == N ? (int32_t)(*sess->tail_cnt)[B] : 0;
                    base += it.fb;
                }
                tot[k] = base;
            }
        };
        build_steps();
        if (variant != 0) {
            // occurrence lists, one episode at a time
            const int G = (int)grp.size();
            TmpDev to(ctx);
            int64_t fmax = 1;
            for (int k = 0; k + 1 < N; ++k)
                for (const PltItem &it : steps[k]) fmax = std::max<int64_t>(fmax, std::max(it.fa, it.fb));
            const int64_t cap = kOccCap;
            int32_t *s_, *p_, *s2, *p2, *cnt, *stmp, *L, *V, *bm1, *n1o, *n2o, *c1o, *c2o, *dc;
            unsigned long long *dtot;
            PltItem *ditem;
            FEM_TRY(to.get(&s_, cap));
            FEM_TRY(to.get(&p_, cap));
            FEM_TRY(to.get(&s2, cap));
            FEM_TRY(to.get(&p2, cap));
            FEM_TRY(to.get(&cnt, cap + 1));
            FEM_TRY(to.get(&stmp, (cap + 1) / 1024 + 2));
            FEM_TRY(to.get(&L, fmax));
            FEM_TRY(to.get(&V, fmax));
            FEM_TRY(to.get(&bm1, fmax / kMsBlock + 2));
            FEM_TRY(to.get(&n1o, fmax));
            FEM_TRY(to.get(&n2o, fmax));
            FEM_TRY(to.get(&c1o, fmax));
            FEM_TRY(to.get(&c2o, fmax));
            FEM_TRY(to.get(&dtot, 1));
            FEM_TRY(to.get(&ditem, 1));
            FEM_TRY(to.get(&dc, G));
            FEM_CUDA_TRY(cudaMemcpyAsync(dc, grp.data(), 4 * G, cudaMemcpyHostToDevice, st));
            std::vector<int32_t> rest;  // episodes whose occurrence lists overflowed
            cudaEventRecord(ctx->ev0, st);
            for (int e = 0; e < G; ++e) {
                std::vector<PltItem> its(N - 1);
                for (int k = 0; k + 1 < N; ++k) its[k] = steps[k][e];
                bool ok = true;
                FEM_TRY(count_occ_one(ctx, its, variant, cap, s_, p_, s2, p2, cnt, stmp, dtot, L, V, bm1, n1o, n2o,
                                      c1o, c2o, ditem, dc + e, d_counts, &ok, &stats->kernel_launches));
                if (!ok) rest.push_back(grp[e]);
            }
            cudaEventRecord(ctx->ev1, st);
            FEM_CUDA_TRY(cudaEventSynchronize(ctx->ev1));
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
            ms_total += ms;
            if (rest.empty()) continue;
            // the latest-start steps below count the rest
            stats->fallback_recounts += (int64_t)rest.size();
            grp.swap(rest);
            build_steps();
        }
        // Batches of episodes whose per-step array totals stay within
        // kPltMaxTotal (positions in the step arrays are int32); a batch holds
        // at least one episode (a type list has fewer than 2^30 events).
        for (int b0 = 0, b1 = 0; b0 < (int)grp.size(); b0 = b1) {
            std::vector<int64_t> acc(N - 1, 0);
            for (b1 = b0; b1 < (int)grp.size(); ++b1) {
                bool fits = true;
                for (int k = 0; k + 1 < N; ++k) fits = fits && acc[k] + steps[k][b1].fb <= kPltMaxTotal;
                if (!fits && b1 > b0) break;
                for (int k = 0; k + 1 < N; ++k) acc[k] += steps[k][b1].fb;
            }
            const int G = b1 - b0;
            // Prefix sharing: episodes of one recording whose first k + 2 nodes
            // and k + 1 edges agree share the step-k item and its arrays (a trie
            // over the episode set, one level per node; level-N candidates joined
            // from one frequent (N-1)-episode share all but their last step).
            std::vector<std::vector<PltItem>> uit(N - 1);
            std::vector<int64_t> utot(N - 1, 0);
            std::vector<int32_t> leaf(G);
            {
                std::map<std::pair<uint32_t, uint16_t>, int32_t> root;
                std::map<std::tuple<int32_t, int32_t, int32_t, int64_t>, int32_t> child;
                for (int e = 0; e < G; ++e) {
                    const int32_t w = grp[b0 + e];
                    const auto key = std::make_pair(crec[w - wmin], types[offs[w - wmin] - n0]);
                    leaf[e] = root.emplace(key, (int32_t)root.size()).first->second;
                }
                for (int k = 0; k + 1 < N; ++k) {
                    child.clear();
                    for (int e = 0; e < G; ++e) {
                        const PltItem &it = steps[k][b0 + e];
                        const auto key = std::make_tuple(leaf[e], it.lo, it.hi, it.b_start);
                        const auto ins = child.emplace(key, (int32_t)uit[k].size());
                        if (ins.second) {
                            PltItem u = it;
                            u.prev_base = k > 0 ? uit[k - 1][leaf[e]].base : 0;
                            u.base = utot[k];
                            utot[k] += u.fb;
                            uit[k].push_back(u);
                        }
                        leaf[e] = ins.first->second;
                    }
                }
            }
            int64_t tmax = 1, n_items = 0;
            for (int64_t t : utot) tmax = std::max(tmax, t);
            std::vector<int64_t> ioff(N, 0);
            for (int k = 0; k + 1 < N; ++k) ioff[k + 1] = ioff[k] + (int64_t)uit[k].size();
            n_items = ioff[N - 1];
            TmpDev tmp(ctx);
            PltItem *d_items;
            int32_t *La, *Lb, *Va, *Vb, *bm, *d_cand, *d_leaf, *n1, *n2, *c1, *c2;
            FEM_TRY(tmp.get(&d_items, (size_t)n_items));
            FEM_TRY(tmp.get(&La, tmax));
            FEM_TRY(tmp.get(&Lb, tmax));
            FEM_TRY(tmp.get(&Va, tmax));
            FEM_TRY(tmp.get(&Vb, tmax));
            FEM_TRY(tmp.get(&n1, tmax));
            FEM_TRY(tmp.get(&n2, tmax));
            FEM_TRY(tmp.get(&c1, tmax));
            FEM_TRY(tmp.get(&c2, tmax));
            FEM_TRY(tmp.get(&bm, tmax / kMsBlock + 2));
            FEM_TRY(tmp.get(&d_cand, G));
            FEM_TRY(tmp.get(&d_leaf, G));
            for (int k = 0; k + 1 < N; ++k)
                FEM_CUDA_TRY(cudaMemcpyAsync(d_items + ioff[k], uit[k].data(), sizeof(PltItem) * uit[k].size(),
                                             cudaMemcpyHostToDevice, st));
            FEM_CUDA_TRY(cudaMemcpyAsync(d_cand, grp.data() + b0, 4 * G, cudaMemcpyHostToDevice, st));
            FEM_CUDA_TRY(cudaMemcpyAsync(d_leaf, leaf.data(), 4 * G, cudaMemcpyHostToDevice, st));
            cudaEventRecord(ctx->ev0, st);
            for (int k = 0; k + 1 < N; ++k) {
                const int64_t T = utot[k];
                if (T > 0) {
                    const unsigned gsz = (unsigned)std::max<int64_t>(1, std::min<int64_t>((T + 255) / 256, 8 * ctx->n_sm));
                    k_plt_step<<<gsz, 256, 0, st>>>(d_items + ioff[k], (int)uit[k].size(), T, k == 0 ? 1 : 0, La, Va, Lb,
                                                    Vb);
                    FEM_TRY(maxscan(st, Vb, T, bm));
                }
                std::swap(La, Lb);
                std::swap(Va, Vb);
            }
            // La / Va: the last node's latest starts and newest valid positions
            const PltItem *last = d_items + ioff[N - 2];
            const int n_last = (int)uit[N - 2].size();
            const int64_t T = utot[N - 2];
            int64_t fmax = 1;
            for (const PltItem &it : uit[N - 2]) fmax = std::max<int64_t>(fmax, it.fb);
            int rounds = 0;
            while ((int64_t(1) << rounds) < fmax) ++rounds;
            // appended events: also the last end of every chain
            int32_t *l1 = nullptr, *l2 = nullptr;
            if (sess) {
                FEM_TRY(tmp.get(&l1, tmax));
                FEM_TRY(tmp.get(&l2, tmax));
            }
            if (T > 0) {
                const unsigned gsz = (unsigned)std::max<int64_t>(1, std::min<int64_t>((T + 255) / 256, 8 * ctx->n_sm));
                k_plt_next<<<gsz, 256, 0, st>>>(last, n_last, T, La, Va, n1, c1, l1);
                for (int q = 0; q < rounds; ++q) {
                    k_plt_jump<<<gsz, 256, 0, st>>>(T, n1, c1, n2, c2, l1, l2);
                    std::swap(n1, n2);
                    std::swap(c1, c2);
                    std::swap(l1, l2);
                }
            }
            k_plt_count<<<(G + 127) / 128, 128, 0, st>>>(last, G, d_leaf, La, Va, c1, d_cand, d_counts,
                                                         sess ? sess->d_prev : nullptr, l1);
            cudaEventRecord(ctx->ev1, st);
            FEM_CUDA_TRY(cudaGetLastError());
            FEM_CUDA_TRY(cudaEventSynchronize(ctx->ev1));
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
            ms_total += ms;
            stats->kernel_launches += (N - 1) * 4 + 2 + rounds;
        }
    }
    stats->candidates_counted += C;
    stats->counted_episode_events += counted;
    stats->relevant_events += relevant;
    *kernel_ms += ms_total;
    return FEM_OK;
}

}  // namespace fem
