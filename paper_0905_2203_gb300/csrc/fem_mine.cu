// fem_mine.cu -- level-wise frequent-episode mining (section "Temporal Data
// Mining": N-size candidates are generated from frequent (N-1)-size episodes,
// counted in one pass over the stream, and kept when the count exceeds the
// threshold).
//
// Every level of every recording lives on the device in fixed-stride form
// (all episodes of a level have N nodes): types[i*N + k], lo/hi[i*(N-1) + k],
// rec[i].  Recordings are concatenated, each recording's episodes contiguous
// and in canonical order -- the interleaved sequence
// (E_1, lo_1, hi_1, E_2, ..., lo_{N-1}, hi_{N-1}, E_N).
//
// Candidate generation (readings of a point the paper leaves open):
//   level 2: every ordered pair (a, b) of distinct frequent types with every
//            bin, generated in canonical (a, bin, b) order and counted in a
//            tiled order (a few first types x a few second types x all bins
//            per warp) so that the episodes a warp holds share their types.
//   level N: alpha, beta frequent (N-1)-episodes of one recording with
//            alpha[2..] = beta[..N-2] (types and bins) give alpha + beta's last
//            edge and node, provided that node's type is not already in alpha.
//            Walking alpha in canonical order and beta in canonical order
//            emits candidates in canonical order.
#include <algorithm>
#include <cstring>
#include <memory>
#include <vector>

#include "fem_internal.cuh"

struct fem_result {
    struct Level {
        std::vector<int64_t> offs{0};
        std::vector<uint16_t> types;
        std::vector<int32_t> lo, hi;
        std::vector<uint32_t> counts;
    };
    int n_recs = 0;
    int max_size = 0;
    std::vector<std::vector<Level>> lv;  // [rec][level]
    fem_stats stats{};
};

namespace fem {

// Level 1: frequent types of every recording, ascending.
__global__ void k_level1_flags(const uint32_t *const *freq, const uint32_t *n_types_pre, int n_recs,
                               const uint32_t *thr, int32_t *flags, int64_t total) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= total) return;
    int r = 0;
    while (r + 1 < n_recs && (int64_t)n_types_pre[r + 1] <= g) ++r;
    const int64_t a = g - n_types_pre[r];
    flags[g] = freq[r][a] > thr[r] ? 1 : 0;
}

__global__ void k_level1_write(const int32_t *flags_scanned, const uint32_t *const *freq,
                               const uint32_t *n_types_pre, int n_recs, const uint32_t *thr, int64_t total,
                               uint16_t *ftypes, uint32_t *fcounts, uint32_t *frec) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= total) return;
    int r = 0;
    while (r + 1 < n_recs && (int64_t)n_types_pre[r + 1] <= g) ++r;
    const int64_t a = g - n_types_pre[r];
    const uint32_t f = freq[r][a];
    if (f > thr[r]) {
        const int32_t pos = flags_scanned[g];
        ftypes[pos] = (uint16_t)a;
        fcounts[pos] = f;
        frec[pos] = (uint32_t)r;
    }
}

// Level 2 candidates of recording r in canonical order: local index
// i = ((ia * nb) + bin) * (F-1) + jb, second type b = jb < ia ? jb : jb + 1.
__global__ void k_gen_level2(const uint16_t *ftypes, const int64_t *f_off, const int64_t *c_off, int n_recs,
                             const int32_t *bin_lo, const int32_t *bin_hi, int nb, int64_t total,
                             uint16_t *ctypes, int32_t *clo, int32_t *chi, uint32_t *crec, int64_t *coffs) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= total) return;
    int lo_r = 0, hi_r = n_recs;  // last r with c_off[r] <= g
    while (hi_r - lo_r > 1) {
        const int mid = (lo_r + hi_r) >> 1;
        if (c_off[mid] <= g) lo_r = mid; else hi_r = mid;
    }
    const int r = lo_r;
    const int64_t i = g - c_off[r];
    const int64_t F = f_off[r + 1] - f_off[r];
    const int64_t jb = i % (F - 1);
    const int64_t q = i / (F - 1);
    const int64_t bin = q % nb, ia = q / nb;
    const int64_t ib = jb < ia ? jb : jb + 1;
    ctypes[2 * g] = ftypes[f_off[r] + ia];
    ctypes[2 * g + 1] = ftypes[f_off[r] + ib];
    clo[g] = bin_lo[bin];
    chi[g] = bin_hi[bin];
    crec[g] = (uint32_t)r;
    coffs[g] = 2 * g;
    if (g == total - 1) coffs[total] = 2 * total;
}

// Counting order for level 2: the (first type, second type) grid is cut into
// tiles of At x Bt pairs, each tile's pairs with all their bins adjacent, so
// the 32 episodes of a warp span about At first types and Bt second types
// (a narrow per-warp type filter).  flags[g] marks grid cells that are real
// candidates (a != b, inside the grid); perm receives canonical indices.
__device__ __forceinline__ int64_t l2_cell_canon(int64_t q, int64_t F, int nb, int At, int Bt, bool &valid) {
    const int64_t TB = (F + Bt - 1) / Bt;
    const int64_t per_tile = (int64_t)At * Bt * nb;
    const int64_t tile = q / per_tile, w = q % per_tile;
    const int64_t ta = tile / TB, tb = tile % TB;
    const int64_t bin = w % nb, pr = w / nb;
    const int64_t a = ta * At + pr / Bt, b = tb * Bt + pr % Bt;
    valid = a < F && b < F && a != b;
    return (a * nb + bin) * (F - 1) + (b < a ? b : b - 1);
}

__global__ void k_perm2_flags(const int64_t *f_off, const int64_t *g_off, int n_recs, int nb, int At, int Bt,
                              int64_t total, int32_t *flags) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= total) return;
    int lo_r = 0, hi_r = n_recs;
    while (hi_r - lo_r > 1) {
        const int mid = (lo_r + hi_r) >> 1;
        if (g_off[mid] <= g) lo_r = mid; else hi_r = mid;
    }
    const int64_t F = f_off[lo_r + 1] - f_off[lo_r];
    bool valid;
    l2_cell_canon(g - g_off[lo_r], F, nb, At, Bt, valid);
    flags[g] = valid ? 1 : 0;
}

__global__ void k_perm2_write(const int32_t *pos, const int64_t *f_off, const int64_t *g_off, const int64_t *c_off,
                              int n_recs, int nb, int At, int Bt, int64_t total, int32_t *perm) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= total) return;
    int lo_r = 0, hi_r = n_recs;
    while (hi_r - lo_r > 1) {
        const int mid = (lo_r + hi_r) >> 1;
        if (g_off[mid] <= g) lo_r = mid; else hi_r = mid;
    }
    const int64_t F = f_off[lo_r + 1] - f_off[lo_r];
    bool valid;
    const int64_t canon = l2_cell_canon(g - g_off[lo_r], F, nb, At, Bt, valid);
    if (valid) perm[pos[g]] = (int32_t)(c_off[lo_r] + canon);
}

// Upper-bound pre-pass for level 2 (anti-monotonicity, section "Temporal
// Data Mining"): non-overlapped occurrences of a -(lo,hi]-> b end at distinct
// b-events, each with an a-event inside (t - hi, ... t - lo] before it, so
//     count(a, b, bin) <= UB(a, b, bin) = #{ b-events with an a-event in the
//                                            bin's window }.
// One pass over the stream: every event j looks back over the widest bin
// window and marks, per bin, which types occur (a per-thread bitset in shared
// memory dedupes repeated types; word w of thread t at bits[w * blockDim + t]
// so a warp's lanes touch distinct banks), then adds one to UB(a, type_j,
// bin) for every marked (a, bin).  The table is per recording: ub[a][b][bin].
__global__ void k_pair_ub(const uint16_t *__restrict__ ty, const int32_t *__restrict__ tm, int64_t n,
                          uint32_t n_types, const int32_t *__restrict__ blo, const int32_t *__restrict__ bhi, int nb,
                          int32_t hi_max, int words, uint32_t *__restrict__ ub) {
    extern __shared__ uint32_t bits[];
    uint32_t *my = bits + threadIdx.x;
    const int bd = blockDim.x;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        for (int w = 0; w < words; ++w) my[w * bd] = 0;
        const int32_t t = tm[j];
        const uint32_t b = ty[j];
        const int64_t lim = (int64_t)t - hi_max;
        for (int64_t i = j - 1; i >= 0 && (int64_t)tm[i] >= lim; --i) {
            const int32_t d = t - tm[i];
            if (d <= 0) continue;
            const uint32_t a = ty[i];
            if (a == b) continue;
            for (int k = 0; k < nb; ++k) {
                if (blo[k] < d && d <= bhi[k]) {
                    const uint32_t bit = a * (uint32_t)nb + (uint32_t)k;
                    const uint32_t m = 1u << (bit & 31);
                    uint32_t &wd = my[(bit >> 5) * bd];
                    if (!(wd & m)) {
                        wd |= m;
                        atomicAdd(&ub[((size_t)a * n_types + b) * nb + k], 1u);
                    }
                }
            }
        }
    }
}

// Keeps, in counting order, the level-2 candidates whose bound exceeds the
// threshold; pruned candidates get count 0 (they can never pass).
__global__ void k_prune2_flags(const int32_t *order, int64_t C, const uint16_t *ct, const int32_t *clo,
                               const int32_t *chi, const uint32_t *crec, const uint32_t *const *ub,
                               const uint32_t *n_types, const int32_t *blo, const int32_t *bhi, int nb,
                               const uint32_t *thr, int32_t *flags, uint32_t *counts) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= C) return;
    const int64_t c = order[i];
    const uint32_t r = crec[c];
    int k = 0;
    while (k < nb && !(blo[k] == clo[c] && bhi[k] == chi[c])) ++k;
    const uint32_t a = ct[2 * c], b = ct[2 * c + 1], nt = n_types[r];
    const uint32_t u = ub[r][((size_t)a * nt + b) * nb + k];
    const bool keep = u > thr[r];
    flags[i] = keep ? 1 : 0;
    if (!keep) counts[c] = 0;
}

// Levels >= 3: candidates whose coarse-tick bound is at most the threshold
// get count 0 (they can never pass) and leave the counting order.
__global__ void k_prune_ub_flags(int64_t C, const uint32_t *ub, const uint32_t *crec, const uint32_t *thr,
                                 int32_t *flags, uint32_t *counts) {
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= C) return;
    const bool keep = ub[c] > thr[crec[c]];
    flags[c] = keep ? 1 : 0;
    if (!keep) counts[c] = 0;
}

__global__ void k_prune_ub_write(const int32_t *pos, const int32_t *flags_copy, int64_t C, int32_t *kept) {
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c < C && flags_copy[c]) kept[pos[c]] = (int32_t)c;
}

__global__ void k_prune2_write(const int32_t *pos, const int32_t *flags_copy, const int32_t *order, int64_t C,
                               int32_t *kept) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= C) return;
    if (flags_copy[i]) kept[pos[i]] = order[i];
}

// Level N >= 3 join, CountScanWrite style: count partners per alpha, scan,
// then write.
__device__ __forceinline__ bool joins(const uint16_t *ft, const int32_t *fl, const int32_t *fh, int M,
                                      int64_t a, int64_t b) {
    // M = N-1 nodes per frequent episode, M-1 edges
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

__global__ void k_join_count(const uint16_t *ft, const int32_t *fl, const int32_t *fh, const uint32_t *frec,
                             const int64_t *f_off, int M, int64_t F, int32_t *cnt) {
    const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (a >= F) return;
    const uint32_t r = frec[a];
    int32_t c = 0;
    for (int64_t b = f_off[r]; b < f_off[r + 1]; ++b)
        if (joins(ft, fl, fh, M, a, b)) ++c;
    cnt[a] = c;
}

__global__ void k_join_write(const uint16_t *ft, const int32_t *fl, const int32_t *fh, const uint32_t *frec,
                             const int64_t *f_off, int M, int64_t F, const int32_t *pos, uint16_t *ct,
                             int32_t *cl, int32_t *ch, uint32_t *crec, int64_t *coffs, int64_t total) {
    const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (a >= F) return;
    const uint32_t r = frec[a];
    int64_t o = pos[a];
    const int N = M + 1;
    for (int64_t b = f_off[r]; b < f_off[r + 1]; ++b) {
        if (!joins(ft, fl, fh, M, a, b)) continue;
        for (int k = 0; k < M; ++k) ct[o * N + k] = ft[a * M + k];
        ct[o * N + M] = ft[b * M + M - 1];
        for (int k = 0; k < M - 1; ++k) {
            cl[o * (N - 1) + k] = fl[a * (M - 1) + k];
            ch[o * (N - 1) + k] = fh[a * (M - 1) + k];
        }
        cl[o * (N - 1) + M - 1] = fl[b * (M - 1) + M - 2];
        ch[o * (N - 1) + M - 1] = fh[b * (M - 1) + M - 2];
        crec[o] = r;
        coffs[o] = o * N;
        ++o;
    }
    if (a == F - 1) coffs[total] = total * N;
}

// Threshold: flags in canonical order (count > threshold, strict).
__global__ void k_thr_flags(const uint32_t *counts, const uint32_t *crec, const uint32_t *thr, int64_t total,
                            int32_t *flags) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= total) return;
    flags[i] = counts[i] > thr[crec[i]] ? 1 : 0;
}

__global__ void k_thr_write(const int32_t *pos, const uint32_t *counts, const uint16_t *ct, const int32_t *cl,
                            const int32_t *ch, const uint32_t *crec, const uint32_t *thr, int N, int64_t total,
                            uint16_t *ft, int32_t *fl, int32_t *fh, uint32_t *frec, uint32_t *fcnt) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= total) return;
    const uint32_t r = crec[i];
    if (!(counts[i] > thr[r])) return;
    const int64_t o = pos[i];
    for (int k = 0; k < N; ++k) ft[o * N + k] = ct[i * N + k];
    for (int k = 0; k < N - 1; ++k) {
        fl[o * (N - 1) + k] = cl[i * (N - 1) + k];
        fh[o * (N - 1) + k] = ch[i * (N - 1) + k];
    }
    frec[o] = r;
    fcnt[o] = counts[i];
}

// Per-recording offsets of a rec-sorted array.
__global__ void k_rec_offsets(const uint32_t *rec, int64_t n, int n_recs, int64_t *off) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r > n_recs) return;
    int64_t lo = 0, hi = n;  // first index with rec >= r
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if ((int)rec[mid] < r) lo = mid + 1; else hi = mid;
    }
    off[r] = lo;
}

// Counting entry shared with fem_count.cu (mode 0, device candidate arrays).
int count_device(fem_ctx *ctx, const std::vector<fem_stream *> &recs, int64_t n_cand, const int64_t *offs,
                 const uint16_t *types, const int32_t *lo, const int32_t *hi, const uint32_t *cand_rec,
                 const std::vector<int32_t> &lo_vals, const int32_t *order, int64_t n_order, uint32_t *counts,
                 fem_stats *stats);

namespace {

struct DevLevel {
    int N = 0;
    int64_t n = 0;
    uint16_t *types = nullptr;
    int32_t *lo = nullptr, *hi = nullptr;
    uint32_t *rec = nullptr, *counts = nullptr;
    int64_t *off = nullptr;  // per-recording offsets (n_recs + 1)
    std::vector<int64_t> h_off;
};

// Device allocations released together (one level's arrays, or the group's
// constants); freed after the stream has drained.
struct Pool {
    fem_ctx *ctx;
    std::vector<std::pair<void *, size_t>> held;
    explicit Pool(fem_ctx *c) : ctx(c) {}
    Pool(const Pool &) = delete;
    ~Pool() { release(); }
    void release() {
        if (held.empty()) return;
        cudaStreamSynchronize(ctx->stream);
        for (auto &h : held) dev_free(ctx, h.first, h.second);
        held.clear();
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

int copy_level_to_host(fem_ctx *ctx, const DevLevel &L, fem_result *res, const std::vector<int> &out_rec,
                       int level) {
    const int N = L.N;
    std::vector<uint16_t> t(L.n * N);
    std::vector<int32_t> lo(L.n * (N - 1)), hi(L.n * (N - 1));
    std::vector<uint32_t> c(L.n);
    if (L.n > 0) {
        FEM_CUDA_TRY(cudaMemcpyAsync(t.data(), L.types, 2 * t.size(), cudaMemcpyDeviceToHost, ctx->stream));
        if (N > 1) {
            FEM_CUDA_TRY(cudaMemcpyAsync(lo.data(), L.lo, 4 * lo.size(), cudaMemcpyDeviceToHost, ctx->stream));
            FEM_CUDA_TRY(cudaMemcpyAsync(hi.data(), L.hi, 4 * hi.size(), cudaMemcpyDeviceToHost, ctx->stream));
        }
        FEM_CUDA_TRY(cudaMemcpyAsync(c.data(), L.counts, 4 * c.size(), cudaMemcpyDeviceToHost, ctx->stream));
        FEM_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    }
    for (size_t r = 0; r + 1 < L.h_off.size(); ++r) {
        fem_result::Level &out = res->lv[out_rec[r]][level];
        const int64_t b = L.h_off[r], e = L.h_off[r + 1];
        out.offs.assign(1, 0);
        out.types.clear();
        out.lo.clear();
        out.hi.clear();
        out.counts.clear();
        for (int64_t i = b; i < e; ++i) {
            out.types.insert(out.types.end(), t.begin() + i * N, t.begin() + (i + 1) * N);
            if (N > 1) {
                out.lo.insert(out.lo.end(), lo.begin() + i * (N - 1), lo.begin() + (i + 1) * (N - 1));
                out.hi.insert(out.hi.end(), hi.begin() + i * (N - 1), hi.begin() + (i + 1) * (N - 1));
            }
            out.counts.push_back(c[i]);
            out.offs.push_back((int64_t)out.types.size());
        }
    }
    return FEM_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// One set of recordings mined in lock-step: every recording of the group is
// at the same level.  begin() runs level 1 and prepares the level-2
// candidates; after the candidates have been counted (by anyone: a counting
// call of its own, or a launch shared with other groups), advance() applies
// the threshold and prepares the next level's candidates.
struct MineGroup {
    fem_ctx *ctx = nullptr;
    std::vector<fem_stream *> recs;
    std::vector<int> out_rec;           // result slot of each recording
    fem_result *res = nullptr;
    std::vector<int32_t> blo, bhi, lo_vals;
    std::vector<uint32_t> thr;
    int max_size = 0;
    int level = 0;                      // level of the current candidates; 0 when done
    bool done = false;
    fem_stats S{};

    std::unique_ptr<Pool> pconst, pprev, pcand;
    uint32_t *d_thr = nullptr;
    int32_t *d_blo = nullptr, *d_bhi = nullptr;
    DevLevel prev, cand;
    int64_t *d_coffs = nullptr;         // CSR node offsets of the candidates
    int64_t *d_coff_rec = nullptr;      // per-recording candidate offsets
    int32_t *d_order = nullptr;         // counting order (level 2) or null
    int64_t n_order = 0;                // candidates left for the exact count
    std::vector<int64_t> c_off;         // host copy of d_coff_rec

    int nrec() const { return (int)recs.size(); }

    int begin();
    int advance();
    int graph_tail();

  private:
    int gen_level2();
    int gen_join();
    int coarse_prune();
    int finish_candidates();
};

int MineGroup::begin() {
    const int n_recs = nrec();
    const int nb = (int)blo.size();
    cudaStream_t st = ctx->stream;
    const int B = 256;
    pconst.reset(new Pool(ctx));
    pprev.reset(new Pool(ctx));
    FEM_TRY(pconst->get(&d_thr, n_recs));
    FEM_TRY(pconst->get(&d_blo, std::max(nb, 1)));
    FEM_TRY(pconst->get(&d_bhi, std::max(nb, 1)));
    FEM_CUDA_TRY(cudaMemcpyAsync(d_thr, thr.data(), 4 * n_recs, cudaMemcpyHostToDevice, st));
    if (nb > 0) {
        FEM_CUDA_TRY(cudaMemcpyAsync(d_blo, blo.data(), 4 * nb, cudaMemcpyHostToDevice, st));
        FEM_CUDA_TRY(cudaMemcpyAsync(d_bhi, bhi.data(), 4 * nb, cudaMemcpyHostToDevice, st));
    }
    lo_vals = blo;
    std::sort(lo_vals.begin(), lo_vals.end());
    lo_vals.erase(std::unique(lo_vals.begin(), lo_vals.end()), lo_vals.end());

    // ---- level 1: frequent types
    std::vector<uint32_t> nt_pre(n_recs + 1, 0);
    std::vector<const uint32_t *> freq_p(n_recs);
    for (int r = 0; r < n_recs; ++r) {
        nt_pre[r + 1] = nt_pre[r] + recs[r]->n_types;
        freq_p[r] = recs[r]->d_freq;
    }
    const int64_t tot1 = nt_pre[n_recs];
    Pool tmp(ctx);
    uint32_t *d_ntpre;
    const uint32_t **d_freqp;
    int32_t *d_flags, *d_scan, *d_total;
    FEM_TRY(tmp.get(&d_ntpre, n_recs + 1));
    FEM_TRY(tmp.get(&d_freqp, n_recs));
    FEM_TRY(tmp.get(&d_flags, tot1 + 1));
    FEM_TRY(tmp.get(&d_scan, tot1 / 1024 + 2));
    FEM_TRY(tmp.get(&d_total, 2));
    FEM_CUDA_TRY(cudaMemcpyAsync(d_ntpre, nt_pre.data(), 4 * (n_recs + 1), cudaMemcpyHostToDevice, st));
    FEM_CUDA_TRY(cudaMemcpyAsync(d_freqp, freq_p.data(), sizeof(void *) * n_recs, cudaMemcpyHostToDevice, st));
    k_level1_flags<<<(unsigned)((tot1 + B - 1) / B), B, 0, st>>>(d_freqp, d_ntpre, n_recs, d_thr, d_flags, tot1);
    FEM_TRY(scan_exclusive(st, d_flags, tot1, d_scan, d_total, &S.kernel_launches));
    int32_t F1 = 0;
    FEM_CUDA_TRY(cudaMemcpyAsync(&F1, d_total, 4, cudaMemcpyDeviceToHost, st));
    FEM_CUDA_TRY(cudaStreamSynchronize(st));
    prev = DevLevel{};
    prev.N = 1;
    prev.n = F1;
    FEM_TRY(pprev->get(&prev.types, F1));
    FEM_TRY(pprev->get(&prev.counts, F1));
    FEM_TRY(pprev->get(&prev.rec, F1));
    FEM_TRY(pprev->get(&prev.off, n_recs + 1));
    k_level1_write<<<(unsigned)((tot1 + B - 1) / B), B, 0, st>>>(d_flags, d_freqp, d_ntpre, n_recs, d_thr, tot1,
                                                                prev.types, prev.counts, prev.rec);
    k_rec_offsets<<<(n_recs + 1 + 127) / 128, 128, 0, st>>>(prev.rec, prev.n, n_recs, prev.off);
    S.kernel_launches += 3;
    prev.h_off.resize(n_recs + 1);
    FEM_CUDA_TRY(cudaMemcpyAsync(prev.h_off.data(), prev.off, 8 * (n_recs + 1), cudaMemcpyDeviceToHost, st));
    FEM_CUDA_TRY(cudaStreamSynchronize(st));
    FEM_TRY(copy_level_to_host(ctx, prev, res, out_rec, 1));
    S.levels = 1;
    if (max_size < 2 || F1 < 2 || nb == 0) {
        done = true;
        level = 0;
        return FEM_OK;
    }
    level = 2;
    FEM_TRY(gen_level2());
    return finish_candidates();
}

int MineGroup::gen_level2() {
    const int n_recs = nrec();
    const int nb = (int)blo.size();
    cudaStream_t st = ctx->stream;
    const int B = 256;
    pcand.reset(new Pool(ctx));
    c_off.assign(n_recs + 1, 0);
    for (int r = 0; r < n_recs; ++r) {
        const int64_t F = prev.h_off[r + 1] - prev.h_off[r];
        c_off[r + 1] = c_off[r] + (F >= 2 ? F * (F - 1) * nb : 0);
    }
    const int64_t C = c_off[n_recs];
    cand = DevLevel{};
    cand.N = 2;
    cand.n = C;
    d_order = nullptr;
    n_order = C;
    FEM_TRY(pcand->get(&d_coff_rec, n_recs + 1));
    FEM_CUDA_TRY(cudaMemcpyAsync(d_coff_rec, c_off.data(), 8 * (n_recs + 1), cudaMemcpyHostToDevice, st));
    if (C == 0) return FEM_OK;
    FEM_TRY(pcand->get(&cand.types, 2 * C));
    FEM_TRY(pcand->get(&cand.lo, C));
    FEM_TRY(pcand->get(&cand.hi, C));
    FEM_TRY(pcand->get(&cand.rec, C));
    FEM_TRY(pcand->get(&cand.counts, C));
    FEM_TRY(pcand->get(&d_coffs, C + 1));
    k_gen_level2<<<(unsigned)((C + B - 1) / B), B, 0, st>>>(prev.types, prev.off, d_coff_rec, n_recs, d_blo, d_bhi,
                                                           nb, C, cand.types, cand.lo, cand.hi, cand.rec, d_coffs);
    S.kernel_launches++;
    // counting order: tiles of At x Bt type pairs with all bins
    const int pairs = std::max(1, 32 / std::max(1, nb));
    const int At = pairs >= 32 ? 8 : pairs >= 8 ? 4 : pairs >= 2 ? 2 : 1;
    const int Bt = std::max(1, pairs / At);
    std::vector<int64_t> g_off(n_recs + 1, 0);
    for (int r = 0; r < n_recs; ++r) {
        const int64_t F = prev.h_off[r + 1] - prev.h_off[r];
        const int64_t cells = (F >= 2) ? ((F + At - 1) / At) * ((F + Bt - 1) / Bt) * (int64_t)At * Bt * nb : 0;
        g_off[r + 1] = g_off[r] + cells;
    }
    const int64_t G = g_off[n_recs];
    Pool tmp(ctx);
    int64_t *d_goff;
    int32_t *d_gfl, *d_gtmp;
    FEM_TRY(tmp.get(&d_goff, n_recs + 1));
    FEM_TRY(tmp.get(&d_gfl, G + 1));
    FEM_TRY(tmp.get(&d_gtmp, G / 1024 + 2));
    FEM_TRY(pcand->get(&d_order, C));
    FEM_CUDA_TRY(cudaMemcpyAsync(d_goff, g_off.data(), 8 * (n_recs + 1), cudaMemcpyHostToDevice, st));
    k_perm2_flags<<<(unsigned)((G + B - 1) / B), B, 0, st>>>(prev.off, d_goff, n_recs, nb, At, Bt, G, d_gfl);
    FEM_TRY(scan_exclusive(st, d_gfl, G, d_gtmp, nullptr, &S.kernel_launches));
    k_perm2_write<<<(unsigned)((G + B - 1) / B), B, 0, st>>>(d_gfl, prev.off, d_goff, d_coff_rec, n_recs, nb, At, Bt,
                                                            G, d_order);
    S.kernel_launches += 2;

    // ---- upper-bound pre-pass
    if (ctx->tuning.prepass == -1 || nb > 8) return FEM_OK;
    for (int r = 0; r < n_recs; ++r)
        if (recs[r]->n_types > 1024) return FEM_OK;
    int32_t hi_max = 0;
    for (int k = 0; k < nb; ++k) hi_max = std::max(hi_max, bhi[k]);
    std::vector<const uint32_t *> ubp(n_recs);
    for (int r = 0; r < n_recs; ++r) {
        const uint32_t nt = recs[r]->n_types;
        uint32_t *u;
        FEM_TRY(tmp.get(&u, (size_t)nt * nt * nb));
        FEM_CUDA_TRY(cudaMemsetAsync(u, 0, sizeof(uint32_t) * (size_t)nt * nt * nb, st));
        const int words = (int)((nt * (uint32_t)nb + 31) / 32);
        int threads = std::min(256, (int)(48 * 1024 / (4 * words)) / 32 * 32);
        threads = std::max(threads, 32);
        if (recs[r]->n > 0 && (prev.h_off[r + 1] - prev.h_off[r]) >= 2) {
            const int64_t blocks = std::min<int64_t>((recs[r]->n + threads - 1) / threads, 8 * ctx->n_sm);
            k_pair_ub<<<(unsigned)blocks, threads, (size_t)threads * words * 4, st>>>(
                recs[r]->d_type, recs[r]->d_time, recs[r]->n, nt, d_blo, d_bhi, nb, hi_max, words, u);
            S.kernel_launches++;
        }
        ubp[r] = u;
    }
    const uint32_t **d_ubp;
    uint32_t *d_nt;
    int32_t *d_pf, *d_pf2, *d_ptmp, *d_ptot, *d_kept;
    FEM_TRY(tmp.get(&d_ubp, n_recs));
    FEM_TRY(tmp.get(&d_nt, n_recs));
    FEM_TRY(tmp.get(&d_pf, C + 1));
    FEM_TRY(tmp.get(&d_pf2, C + 1));
    FEM_TRY(tmp.get(&d_ptmp, C / 1024 + 2));
    FEM_TRY(tmp.get(&d_ptot, 2));
    FEM_TRY(pcand->get(&d_kept, C));
    std::vector<uint32_t> nth(n_recs);
    for (int r = 0; r < n_recs; ++r) nth[r] = recs[r]->n_types;
    FEM_CUDA_TRY(cudaMemcpyAsync(d_ubp, ubp.data(), sizeof(void *) * n_recs, cudaMemcpyHostToDevice, st));
    FEM_CUDA_TRY(cudaMemcpyAsync(d_nt, nth.data(), 4 * n_recs, cudaMemcpyHostToDevice, st));
    k_prune2_flags<<<(unsigned)((C + B - 1) / B), B, 0, st>>>(d_order, C, cand.types, cand.lo, cand.hi, cand.rec, d_ubp,
                                                             d_nt, d_blo, d_bhi, nb, d_thr, d_pf, cand.counts);
    FEM_CUDA_TRY(cudaMemcpyAsync(d_pf2, d_pf, 4 * C, cudaMemcpyDeviceToDevice, st));
    FEM_TRY(scan_exclusive(st, d_pf, C, d_ptmp, d_ptot, &S.kernel_launches));
    k_prune2_write<<<(unsigned)((C + B - 1) / B), B, 0, st>>>(d_pf, d_pf2, d_order, C, d_kept);
    S.kernel_launches += 2;
    int32_t kept = 0;
    FEM_CUDA_TRY(cudaMemcpyAsync(&kept, d_ptot, 4, cudaMemcpyDeviceToHost, st));
    FEM_CUDA_TRY(cudaStreamSynchronize(st));
    n_order = kept;
    d_order = d_kept;
    S.candidates_pruned += C - kept;
    return FEM_OK;
}

int MineGroup::gen_join() {
    const int n_recs = nrec();
    const int N = level;
    const int M = N - 1;
    cudaStream_t st = ctx->stream;
    const int B = 256;
    const int64_t F = prev.n;
    pcand.reset(new Pool(ctx));
    cand = DevLevel{};
    cand.N = N;
    d_order = nullptr;
    c_off.assign(n_recs + 1, 0);
    FEM_TRY(pcand->get(&d_coff_rec, n_recs + 1));
    if (F == 0) {
        cand.n = 0;
        n_order = 0;
        return FEM_OK;
    }
    Pool tmp(ctx);
    int32_t *d_cnt, *d_tmp, *d_tot;
    FEM_TRY(tmp.get(&d_cnt, F + 1));
    FEM_TRY(tmp.get(&d_tmp, F / 1024 + 2));
    FEM_TRY(tmp.get(&d_tot, 2));
    k_join_count<<<(unsigned)((F + B - 1) / B), B, 0, st>>>(prev.types, prev.lo, prev.hi, prev.rec, prev.off, M, F,
                                                           d_cnt);
    FEM_TRY(scan_exclusive(st, d_cnt, F, d_tmp, d_tot, &S.kernel_launches));
    int32_t Ct = 0;
    FEM_CUDA_TRY(cudaMemcpyAsync(&Ct, d_tot, 4, cudaMemcpyDeviceToHost, st));
    FEM_CUDA_TRY(cudaStreamSynchronize(st));
    S.kernel_launches++;
    const int64_t C = Ct;
    cand.n = C;
    n_order = C;
    if (C == 0) return FEM_OK;
    FEM_TRY(pcand->get(&cand.types, (size_t)C * N));
    FEM_TRY(pcand->get(&cand.lo, (size_t)C * (N - 1)));
    FEM_TRY(pcand->get(&cand.hi, (size_t)C * (N - 1)));
    FEM_TRY(pcand->get(&cand.rec, C));
    FEM_TRY(pcand->get(&cand.counts, C));
    FEM_TRY(pcand->get(&d_coffs, C + 1));
    k_join_write<<<(unsigned)((F + B - 1) / B), B, 0, st>>>(prev.types, prev.lo, prev.hi, prev.rec, prev.off, M, F,
                                                           d_cnt, cand.types, cand.lo, cand.hi, cand.rec, d_coffs, C);
    k_rec_offsets<<<(n_recs + 1 + 127) / 128, 128, 0, st>>>(cand.rec, C, n_recs, d_coff_rec);
    FEM_CUDA_TRY(cudaMemcpyAsync(c_off.data(), d_coff_rec, 8 * (n_recs + 1), cudaMemcpyDeviceToHost, st));
    FEM_CUDA_TRY(cudaStreamSynchronize(st));
    S.kernel_launches += 2;
    return coarse_prune();
}

// Coarse-tick bound of the level's candidates (fem_bound.cu), one launch per
// recording; candidates at or below their threshold are dropped before the
// exact count.  Only with prepass = 1: on the many-recordings workload the
// bound costs about half of the count it replaces, and the candidates it
// keeps (frequent types) are the expensive ones, so it does not pay by
// default.
int MineGroup::coarse_prune() {
    const int n_recs = nrec();
    const int N = level;
    const int64_t C = cand.n;
    const int pp = ctx->tuning.prepass;
    if (C == 0 || N < 3 || pp != 1) return FEM_OK;
    cudaStream_t st = ctx->stream;
    const int B = 256;
    int32_t hi_max = 1;
    for (int32_t h : bhi) hi_max = std::max(hi_max, h);
    Pool tmp(ctx);
    uint32_t *d_ub;
    int32_t *d_pf, *d_pf2, *d_ptmp, *d_ptot, *d_kept;
    FEM_TRY(tmp.get(&d_ub, C));
    for (int r = 0; r < n_recs; ++r) {
        const int64_t c0 = c_off[r], n = c_off[r + 1] - c0;
        if (n == 0) continue;
        if (recs[r]->n_types > 8192 || recs[r]->n > INT32_MAX / 2) {
            FEM_CUDA_TRY(cudaMemsetAsync(d_ub + c0, 0xFF, 4 * n, st));  // no bound: keep all
            continue;
        }
        const int32_t w = coarse_tick(recs[r], hi_max, 0);
        // dense layout: the first n + 1 entries of d_coffs are 0, N, ..., nN
        FEM_TRY(coarse_bound_dev(ctx, recs[r], n, d_coffs, cand.types + c0 * N, cand.lo + c0 * (N - 1),
                                 cand.hi + c0 * (N - 1), N, w, d_ub + c0, &S.kernel_launches));
    }
    FEM_TRY(tmp.get(&d_pf, C + 1));
    FEM_TRY(tmp.get(&d_pf2, C + 1));
    FEM_TRY(tmp.get(&d_ptmp, C / 1024 + 2));
    FEM_TRY(tmp.get(&d_ptot, 2));
    FEM_TRY(pcand->get(&d_kept, C));
    k_prune_ub_flags<<<(unsigned)((C + B - 1) / B), B, 0, st>>>(C, d_ub, cand.rec, d_thr, d_pf, cand.counts);
    FEM_CUDA_TRY(cudaMemcpyAsync(d_pf2, d_pf, 4 * C, cudaMemcpyDeviceToDevice, st));
    FEM_TRY(scan_exclusive(st, d_pf, C, d_ptmp, d_ptot, &S.kernel_launches));
    k_prune_ub_write<<<(unsigned)((C + B - 1) / B), B, 0, st>>>(d_pf, d_pf2, C, d_kept);
    S.kernel_launches += 2;
    int32_t kept = 0;
    FEM_CUDA_TRY(cudaMemcpyAsync(&kept, d_ptot, 4, cudaMemcpyDeviceToHost, st));
    FEM_CUDA_TRY(cudaStreamSynchronize(st));
    S.candidates_pruned += C - kept;
    n_order = kept;
    d_order = d_kept;
    return FEM_OK;
}

// Statistics of the candidates about to be counted; an empty candidate set
// ends the group.
int MineGroup::finish_candidates() {
    if (cand.n == 0) {
        done = true;
        level = 0;
        pcand.reset();
        return FEM_OK;
    }
    for (int r = 0; r < nrec(); ++r) S.episode_events += (double)(c_off[r + 1] - c_off[r]) * (double)recs[r]->n;
    return FEM_OK;
}

int MineGroup::advance() {
    const int n_recs = nrec();
    const int N = level;
    cudaStream_t st = ctx->stream;
    const int B = 256;
    const int64_t C = cand.n;
    std::unique_ptr<Pool> pnext(new Pool(ctx));
    Pool tmp(ctx);
    int32_t *d_fl, *d_tmp2, *d_tot2;
    FEM_TRY(tmp.get(&d_fl, C + 1));
    FEM_TRY(tmp.get(&d_tmp2, C / 1024 + 2));
    FEM_TRY(tmp.get(&d_tot2, 2));
    k_thr_flags<<<(unsigned)((C + B - 1) / B), B, 0, st>>>(cand.counts, cand.rec, d_thr, C, d_fl);
    FEM_TRY(scan_exclusive(st, d_fl, C, d_tmp2, d_tot2, &S.kernel_launches));
    int32_t Fn = 0;
    FEM_CUDA_TRY(cudaMemcpyAsync(&Fn, d_tot2, 4, cudaMemcpyDeviceToHost, st));
    FEM_CUDA_TRY(cudaStreamSynchronize(st));
    DevLevel next;
    next.N = N;
    next.n = Fn;
    FEM_TRY(pnext->get(&next.types, (size_t)Fn * N));
    FEM_TRY(pnext->get(&next.lo, (size_t)Fn * (N - 1)));
    FEM_TRY(pnext->get(&next.hi, (size_t)Fn * (N - 1)));
    FEM_TRY(pnext->get(&next.rec, Fn));
    FEM_TRY(pnext->get(&next.counts, Fn));
    FEM_TRY(pnext->get(&next.off, n_recs + 1));
    k_thr_write<<<(unsigned)((C + B - 1) / B), B, 0, st>>>(d_fl, cand.counts, cand.types, cand.lo, cand.hi, cand.rec,
                                                          d_thr, N, C, next.types, next.lo, next.hi, next.rec,
                                                          next.counts);
    k_rec_offsets<<<(n_recs + 1 + 127) / 128, 128, 0, st>>>(next.rec, next.n, n_recs, next.off);
    S.kernel_launches += 3;
    next.h_off.resize(n_recs + 1);
    FEM_CUDA_TRY(cudaMemcpyAsync(next.h_off.data(), next.off, 8 * (n_recs + 1), cudaMemcpyDeviceToHost, st));
    FEM_CUDA_TRY(cudaStreamSynchronize(st));
    FEM_TRY(copy_level_to_host(ctx, next, res, out_rec, N));
    S.levels = N;
    prev = next;
    pprev = std::move(pnext);
    pcand.reset();
    if (Fn == 0 || N >= max_size) {
        done = true;
        level = 0;
        return FEM_OK;
    }
    level = N + 1;
    FEM_TRY(gen_join());
    return finish_candidates();
}

// Copies the levels a captured graph produced into the result and the
// statistics (the candidates the level-2 pre-pass and the level-3 join bound
// dropped count as pruned).
static void fill_graph_levels(MineGroup &g, const TailResult &tr) {
    const int n_recs = g.nrec();
    for (const TailLevel &tl : tr.levels) {
        const int N = tl.N;
        if (N >= 2) {
            if (tl.C == 0) break;
            g.S.candidates_counted += tl.C;
            for (int r = 0; r < n_recs; ++r) {
                // a bound's dropped candidates count as pruned, not counted
                const int64_t sk = r < (int)tl.skipped.size() ? tl.skipped[r] : 0;
                g.S.candidates_counted -= sk;
                const double gr = (double)(tl.goff[r + 1] - tl.goff[r]);
                const double cr = (double)(tl.coff[r + 1] - tl.coff[r] - sk);
                g.S.episode_events += gr * (double)g.recs[r]->n;
                g.S.counted_episode_events += cr * (double)g.recs[r]->n;
                g.S.candidates_pruned += (int64_t)(gr - cr);
            }
        }
        g.S.levels = N;
        std::vector<int64_t> off(n_recs + 1, 0);
        for (uint32_t r : tl.rec) off[r + 1]++;
        for (int r = 0; r < n_recs; ++r) off[r + 1] += off[r];
        for (int r = 0; r < n_recs; ++r) {
            fem_result::Level &out = g.res->lv[g.out_rec[r]][N];
            out.offs.assign(1, 0);
            out.types.clear();
            out.lo.clear();
            out.hi.clear();
            out.counts.clear();
            for (int64_t i = off[r]; i < off[r + 1]; ++i) {
                out.types.insert(out.types.end(), tl.types.begin() + i * N, tl.types.begin() + (i + 1) * N);
                if (N > 1) {
                    out.lo.insert(out.lo.end(), tl.lo.begin() + i * (N - 1), tl.lo.begin() + (i + 1) * (N - 1));
                    out.hi.insert(out.hi.end(), tl.hi.begin() + i * (N - 1), tl.hi.begin() + (i + 1) * (N - 1));
                }
                out.counts.push_back(tl.counts[i]);
                out.offs.push_back((int64_t)out.types.size());
            }
        }
    }
    g.S.graph_tails += 1;
    g.S.kernel_launches += tr.kernel_nodes;
    g.S.sparse_launches += tr.count_levels;
    g.S.count_kernel_ms += tr.count_ms;
    g.S.relevant_events += tr.relevant;
}

// Levels 3..max_size through the captured graph (fem_graph.cu), starting
// from the level-2 frequent set; when it does not apply or reports a flag the
// group simply continues level by level.
int MineGroup::graph_tail() {
    TailResult tr;
    bool used = false;
    FEM_TRY(run_graph_tail(ctx, recs, blo, bhi, thr, lo_vals, max_size, prev.n, prev.types, prev.lo, prev.hi, prev.rec,
                           prev.counts, prev.h_off, &tr, &used));
    if (!used) return FEM_OK;
    // the level-3 candidates the host path had prepared are superseded: the
    // graph accounts for them itself
    for (int r = 0; r < nrec(); ++r) S.episode_events -= (double)(c_off[r + 1] - c_off[r]) * (double)recs[r]->n;
    fill_graph_levels(*this, tr);
    done = true;
    level = 0;
    pcand.reset();
    return FEM_OK;
}

// Counting of the candidates of one group with the library's counting path.
static int count_group(MineGroup &g) {
    fem_stats cs{};
    FEM_TRY(count_device(g.ctx, g.recs, g.cand.n, g.d_coffs, g.cand.types, g.cand.lo, g.cand.hi, g.cand.rec, g.lo_vals,
                         g.d_order, g.n_order, g.cand.counts, &cs));
    g.S.kernel_launches += cs.kernel_launches;
    g.S.sparse_launches += cs.sparse_launches;
    g.S.candidates_counted += cs.candidates_counted;
    g.S.fallback_recounts += cs.fallback_recounts;
    g.S.relevant_events += cs.relevant_events;
    g.S.count_kernel_ms += cs.count_kernel_ms;
    g.S.counted_episode_events += cs.counted_episode_events;
    return FEM_OK;
}

// ---------------------------------------------------------------------------
// Continuous batching: the current candidates of several groups (each at its
// own level) are concatenated and counted in one counting call, then the
// counts are handed back to each group.
__global__ void k_fill_group(int64_t C, int N, int64_t cbase, int64_t nbase, int rbase, const uint32_t *grec,
                             const int32_t *gorder, int64_t n_order, int64_t obase, int64_t *offs, uint32_t *rec,
                             int32_t *order) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < C) {
        offs[cbase + i] = nbase + i * N;
        rec[cbase + i] = (uint32_t)rbase + grec[i];
    }
    if (i < n_order) order[obase + i] = (int32_t)(cbase + (gorder ? gorder[i] : i));
}

__global__ void k_set_last_offs(int64_t *offs, int64_t C, int64_t nodes) { offs[C] = nodes; }

int mg_count_batch(fem_ctx *ctx, const std::vector<MineGroup *> &gs) {
    cudaStream_t st = ctx->stream;
    std::vector<fem_stream *> recs;
    std::vector<int32_t> lo_vals;
    int64_t C = 0, nodes = 0, edges = 0, norder = 0;
    for (MineGroup *g : gs) {
        if (g->done || g->cand.n == 0) continue;
        recs.insert(recs.end(), g->recs.begin(), g->recs.end());
        lo_vals.insert(lo_vals.end(), g->lo_vals.begin(), g->lo_vals.end());
        C += g->cand.n;
        nodes += g->cand.n * g->cand.N;
        edges += g->cand.n * (g->cand.N - 1);
        norder += g->n_order;
    }
    if (C == 0) return FEM_OK;
    std::sort(lo_vals.begin(), lo_vals.end());
    lo_vals.erase(std::unique(lo_vals.begin(), lo_vals.end()), lo_vals.end());
    void *p[7];
    FEM_TRY(scratch(ctx, kSlotMine0 + 0, 8 * (C + 1), &p[0]));
    FEM_TRY(scratch(ctx, kSlotMine0 + 1, 2 * nodes, &p[1]));
    FEM_TRY(scratch(ctx, kSlotMine0 + 2, 4 * std::max<int64_t>(edges, 1), &p[2]));
    FEM_TRY(scratch(ctx, kSlotMine0 + 3, 4 * std::max<int64_t>(edges, 1), &p[3]));
    FEM_TRY(scratch(ctx, kSlotMine0 + 4, 4 * C, &p[4]));
    FEM_TRY(scratch(ctx, kSlotMine0 + 5, 4 * std::max<int64_t>(norder, 1), &p[5]));
    FEM_TRY(scratch(ctx, kSlotMine0 + 6, 4 * C, &p[6]));
    int64_t *offs = static_cast<int64_t *>(p[0]);
    uint16_t *types = static_cast<uint16_t *>(p[1]);
    int32_t *lo = static_cast<int32_t *>(p[2]), *hi = static_cast<int32_t *>(p[3]);
    uint32_t *rec = static_cast<uint32_t *>(p[4]);
    int32_t *order = static_cast<int32_t *>(p[5]);
    uint32_t *counts = static_cast<uint32_t *>(p[6]);
    int64_t cb = 0, nbse = 0, ebse = 0, ob = 0;
    int rb = 0;
    for (MineGroup *g : gs) {
        if (g->done || g->cand.n == 0) continue;
        const int64_t c = g->cand.n;
        const int N = g->cand.N;
        FEM_CUDA_TRY(cudaMemcpyAsync(types + nbse, g->cand.types, 2 * c * N, cudaMemcpyDeviceToDevice, st));
        if (N > 1) {
            FEM_CUDA_TRY(cudaMemcpyAsync(lo + ebse, g->cand.lo, 4 * c * (N - 1), cudaMemcpyDeviceToDevice, st));
            FEM_CUDA_TRY(cudaMemcpyAsync(hi + ebse, g->cand.hi, 4 * c * (N - 1), cudaMemcpyDeviceToDevice, st));
        }
        // pruned candidates already hold their final count (0)
        FEM_CUDA_TRY(cudaMemcpyAsync(counts + cb, g->cand.counts, 4 * c, cudaMemcpyDeviceToDevice, st));
        const int64_t m = std::max(c, g->n_order);
        k_fill_group<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(c, N, cb, nbse, rb, g->cand.rec, g->d_order,
                                                                  g->n_order, ob, offs, rec, order);
        cb += c;
        nbse += c * N;
        ebse += c * (N - 1);
        ob += g->n_order;
        rb += g->nrec();
    }
    k_set_last_offs<<<1, 1, 0, st>>>(offs, C, nodes);
    FEM_CUDA_TRY(cudaGetLastError());
    fem_stats cs{};
    FEM_TRY(count_device(ctx, recs, C, offs, types, lo, hi, rec, lo_vals, order, norder, counts, &cs));
    cb = 0;
    for (MineGroup *g : gs) {
        if (g->done || g->cand.n == 0) continue;
        FEM_CUDA_TRY(cudaMemcpyAsync(g->cand.counts, counts + cb, 4 * g->cand.n, cudaMemcpyDeviceToDevice, st));
        g->S.kernel_launches += 2;
        cb += g->cand.n;
    }
    // shared launch statistics are attributed to the first group
    gs[0]->S.kernel_launches += cs.kernel_launches;
    gs[0]->S.sparse_launches += cs.sparse_launches;
    gs[0]->S.count_kernel_ms += cs.count_kernel_ms;
    for (MineGroup *g : gs) {
        if (g->done) continue;
        g->S.candidates_counted += g->n_order;
        // every counted candidate of a group is counted over its own recording
        g->S.counted_episode_events += (double)g->n_order * (double)g->recs[0]->n;
    }
    return sync_status(ctx);
}

MineGroup *mg_create(fem_ctx *ctx, fem_stream *s, const std::vector<int32_t> &blo, const std::vector<int32_t> &bhi,
                     uint32_t thr, int max_size, fem_result *res) {
    MineGroup *g = new (std::nothrow) MineGroup();
    if (!g) return nullptr;
    g->ctx = ctx;
    g->recs = {s};
    g->out_rec = {0};
    g->res = res;
    g->blo = blo;
    g->bhi = bhi;
    g->thr = {thr};
    g->max_size = max_size;
    return g;
}
int mg_begin(MineGroup *g) { return g->begin(); }
int mg_advance(MineGroup *g) { return g->advance(); }
bool mg_done(const MineGroup *g) { return g->done; }
const fem_stats &mg_stats(const MineGroup *g) { return g->S; }
void mg_destroy(MineGroup *g) { delete g; }

fem_result *result_new(int n_recs, int max_size) {
    fem_result *res = new (std::nothrow) fem_result();
    if (!res) return nullptr;
    res->n_recs = n_recs;
    res->max_size = max_size;
    res->lv.assign(n_recs, std::vector<fem_result::Level>(max_size + 1));
    return res;
}
void result_set_stats(fem_result *r, const fem_stats &s) { r->stats = s; }

static int mine_impl(fem_ctx *ctx, const std::vector<fem_stream *> &recs, const std::vector<int32_t> &blo,
                     const std::vector<int32_t> &bhi, const std::vector<uint32_t> &thr, int max_size,
                     fem_result *res) {
    MineGroup g;
    g.ctx = ctx;
    g.recs = recs;
    for (int r = 0; r < (int)recs.size(); ++r) g.out_rec.push_back(r);
    g.res = res;
    g.blo = blo;
    g.bhi = bhi;
    g.thr = thr;
    g.max_size = max_size;
    // The whole pass as one captured graph (sparse counting kernel, device-
    // chosen segmentation) unless a tuning override asks for the host-driven
    // path or an alphabet is small enough for the tiled kernel to be the
    // better choice at level 2.
    const fem_tuning &tu = ctx->tuning;
    bool whole = tu.level_graph != -1 && tu.plain_path != 1 && tu.kernel == 0 && tu.segments == 0 &&
                 tu.lanes_per_cta == 0 && tu.tile_events == 0 && max_size >= 2;
    for (auto *s : recs)
        if (s->n_types < 16) whole = false;
    if (whole) {
        std::vector<int32_t> lo_vals = blo;
        std::sort(lo_vals.begin(), lo_vals.end());
        lo_vals.erase(std::unique(lo_vals.begin(), lo_vals.end()), lo_vals.end());
        TailResult tr;
        bool used = false;
        FEM_TRY(run_graph_mining(ctx, recs, blo, bhi, thr, lo_vals, max_size, tu.prepass != -1, &tr, &used));
        if (used) {
            fill_graph_levels(g, tr);
            res->stats = g.S;
            return FEM_OK;
        }
    }
    int st = g.begin();
    while (st == FEM_OK && !g.done) {
        st = count_group(g);
        if (st == FEM_OK) st = sync_status(ctx);
        if (st == FEM_OK) st = g.advance();
        // after level 2, the remaining levels run as one captured graph
        if (st == FEM_OK && !g.done && g.level == 3 && ctx->tuning.level_graph != -1 && ctx->tuning.plain_path != 1)
            st = g.graph_tail();
    }
    res->stats = g.S;
    return st;
}

}  // namespace fem

using namespace fem;

extern "C" int fem_mine_levelwise(fem_ctx *ctx, const fem_stream *const *recs, int n_recs, const int32_t *bin_lo,
                                  const int32_t *bin_hi, int n_bins, const uint32_t *threshold, int max_size,
                                  fem_result **out) {
    if (!ctx || !recs || n_recs < 1 || !out || max_size < 1 || max_size > FEM_MAX_NODES || !threshold)
        return FEM_ERR_INVAL;
    if (n_bins < 0 || (n_bins > 0 && (!bin_lo || !bin_hi)) || (max_size > 1 && n_bins < 1)) return FEM_ERR_INVAL;
    *out = nullptr;
    std::vector<std::pair<int32_t, int32_t>> bins;
    for (int b = 0; b < n_bins; ++b) {
        if (bin_lo[b] < 0 || bin_lo[b] >= bin_hi[b]) return FEM_ERR_INVAL;
        bins.push_back({bin_lo[b], bin_hi[b]});
    }
    std::sort(bins.begin(), bins.end());
    bins.erase(std::unique(bins.begin(), bins.end()), bins.end());
    std::vector<int32_t> blo, bhi;
    for (auto &b : bins) {
        blo.push_back(b.first);
        bhi.push_back(b.second);
    }
    std::vector<fem_stream *> rv;
    std::vector<uint32_t> thr(threshold, threshold + n_recs);
    for (int r = 0; r < n_recs; ++r) {
        if (!recs[r] || recs[r]->ctx != ctx) return FEM_ERR_INVAL;
        rv.push_back(const_cast<fem_stream *>(recs[r]));
    }
    fem_result *res = new (std::nothrow) fem_result();
    if (!res) return FEM_ERR_NOMEM;
    res->n_recs = n_recs;
    res->max_size = max_size;
    res->lv.assign(n_recs, std::vector<fem_result::Level>(max_size + 1));
    int st;
    const double t0 = now_s();
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        cudaSetDevice(ctx->device);
        st = mine_impl(ctx, rv, blo, bhi, thr, max_size, res);
        if (st == FEM_OK) st = sync_status(ctx);
    }
    if (st != FEM_OK) {
        delete res;
        return st;
    }
    res->stats.total_ms = (now_s() - t0) * 1e3;
    ctx->last = res->stats;
    *out = res;
    return FEM_OK;
}

extern "C" int fem_result_level(const fem_result *r, int rec, int level, int64_t *n_out, const int64_t **offs,
                                const uint16_t **types, const int32_t **lo, const int32_t **hi,
                                const uint32_t **counts) {
    if (!r || rec < 0 || rec >= r->n_recs || level < 1 || level > r->max_size || !n_out) return FEM_ERR_INVAL;
    const fem_result::Level &L = r->lv[rec][level];
    *n_out = (int64_t)L.counts.size();
    if (offs) *offs = L.offs.data();
    if (types) *types = L.types.data();
    if (lo) *lo = L.lo.data();
    if (hi) *hi = L.hi.data();
    if (counts) *counts = L.counts.data();
    return FEM_OK;
}

extern "C" int fem_result_stats(const fem_result *r, fem_stats *out) {
    if (!r || !out) return FEM_ERR_INVAL;
    *out = r->stats;
    return FEM_OK;
}

extern "C" void fem_result_free(fem_result *r) { delete r; }
