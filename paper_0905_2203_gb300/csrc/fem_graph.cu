// fem_graph.cu -- levels 3..max of level-wise mining chained in one captured
// CUDA graph.
//
// After level 2 (which is host-driven: upper-bound pre-pass, choice of
// counting kernel), every later level runs the same fixed sequence --
// join (count, scan, write), candidate index, ring-capacity check, sparse
// counting + stitch, threshold (flags, scan, write), per-recording offsets --
// whose sizes live in device counters.  The sequence for all remaining
// levels is captured once into a graph over fixed-capacity buffers and
// launched with a single call; a level that keeps nothing leaves zero
// counters behind, so the later levels' kernels exit at once.  Any capacity
// overflow, ring-capacity miss or entry-class overflow sets a flag; the
// caller then runs the host-driven path instead (same results).
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

constexpr int kRingCap = 16;      // shared-memory ring entries in the graph path
constexpr int kMaxPerRec = 4096;  // finest segmentation of a recording

// Counters per level: [0] candidates C, [1] frequent F, [2] flags, [3]
// entry-class fallbacks (stitch), [4..5] padding.
constexpr int kCtr = 6;

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
        if (total > cap) atomicOr(&ctr[2], 1);
    }
}

// CSR offsets of the candidates, identity slot order, per-recording
// candidate offsets, and the RecInfo fields that depend on them.
__global__ void k_g_index(const uint32_t *crec, const int32_t *ctr, int N, int64_t cap, int64_t *offs, int32_t *iota) {
    const int64_t C = ctr[0];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= cap; i += (int64_t)gridDim.x * blockDim.x) {
        if (i <= C) offs[i] = i * N;
        if (i < cap) iota[i] = (int32_t)i;
    }
}

// Per-level segmentation: the level's (candidate, segment) threads should
// number about `target`, so a level with few candidates cuts its recordings
// finely and one with many coarsely.  Segment boundaries are taken from the
// recording's finest boundaries (pfine[r] segments, in segf) every s-th one.
__global__ void k_g_recinfo(const uint32_t *crec, const int32_t *ctr, int n_recs, int64_t *coff, RecInfo *ri,
                            int64_t *nthreads, const int64_t *segf, const int32_t *pfine, int32_t *sstep,
                            int64_t *segl, int64_t target) {
    const int64_t C = ctr[0];
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
        int64_t base = 0;
        for (int r = 0; r < n_recs; ++r) {
            const int pf = pfine[r];
            const double want = fmin((double)pf, fmax(1.0, ceil((double)ri[r].n / seg_len)));
            const int st = (pf + (int)want - 1) / (int)want;
            const int P = (pf + st - 1) / st;
            sstep[r] = st;
            ri[r].P = P;
            ri[r].slot_first = (int)coff[r];
            ri[r].recbase = base;
            base += (coff[r + 1] - coff[r]) * P;
        }
        *nthreads = base;
    }
    __syncthreads();
    for (int r = 0; r < n_recs; ++r) {
        const int P = ri[r].P, st = sstep[r], pf = pfine[r];
        const int64_t *f = segf + (size_t)r * (kMaxPerRec + 1);
        int64_t *o = segl + (size_t)r * (kMaxPerRec + 1);
        for (int p = threadIdx.x; p <= P; p += blockDim.x) o[p] = f[min(p * st, pf)];
    }
}

// Every node's ring must fit kRingCap entries (window density + 1).  Also
// sums the candidates' relevant events (sum over nodes of the node type's
// frequency in the candidate's recording) into *rel.
__global__ void k_g_ringcheck(const uint16_t *ct, const int32_t *cl, const uint32_t *crec, const int32_t *ctr, int N,
                              const uint32_t *const *dens, const int32_t *lo_vals, int n_lo, int R_cap,
                              const RecInfo *ri, int32_t *ctr_w, unsigned long long *rel) {
    const int64_t C = ctr[0];
    unsigned long long acc = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < C; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t r = crec[i];
        const uint32_t *fq = ri[r].freq;
        for (int k = 0; k < N; ++k) acc += fq[ct[i * N + k]];
        for (int k = 0; k < N - 1; ++k) {
            const int32_t l = cl[i * (N - 1) + k];
            int j = 0;
            while (j < n_lo && lo_vals[j] != l) ++j;
            const uint32_t d = j < n_lo ? dens[r * n_lo + j][ct[i * N + k]] : 0xFFFFFFFFu;
            if (d == 0xFFFFFFFFu || d + 1 > (uint32_t)R_cap) atomicOr(&ctr_w[2], 2);
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
        if (total > cap) atomicOr(&ctr[2], 4);
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

}  // namespace

struct GraphTail {
    fem_ctx *ctx = nullptr;
    std::string key;
    std::vector<fem_stream *> recs;
    int n_recs = 0, max_size = 0;
    int64_t cap = 0, cap_threads = 0;
    std::vector<std::pair<void *, size_t>> held;
    std::vector<FLevel> F;                 // F[N] for N = 2..max_size
    int32_t *ctr = nullptr;                // kCtr per level, indexed by N
    int64_t *coff = nullptr;               // (n_recs + 1) per level
    uint32_t *d_thr = nullptr;
    int ring_cap = kRingCap;               // ring entries per node
    int64_t *segf = nullptr, *segl = nullptr;  // finest / current level's segment starts
    int32_t *pfine = nullptr, *sstep = nullptr;
    int64_t target = 0;                    // (candidate, segment) threads per level
    unsigned long long *rel = nullptr;    // relevant events counted, per level
    std::vector<cudaEvent_t> ev;           // around each level's count kernels
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
    }
};

static int build_tail(GraphTail *g, const std::vector<int32_t> &blo, const std::vector<int32_t> &bhi,
                      const std::vector<uint32_t> &thr, const std::vector<int32_t> &lo_vals) {
    fem_ctx *ctx = g->ctx;
    cudaStream_t st = ctx->stream;
    const int n_recs = g->n_recs, L = g->max_size;
    const int64_t cap = g->cap;
    int32_t hi_max = 0;
    for (auto h : bhi) hi_max = std::max(hi_max, h);
    // per-recording segment counts and boundaries, per-type lists, densities
    std::vector<RecInfo> ri_h(n_recs);
    int64_t *segs = nullptr;  // finest boundaries per recording
    FEM_TRY(g->get(&segs, (size_t)n_recs * (kMaxPerRec + 1)));
    FEM_TRY(g->get(&g->segl, (size_t)n_recs * (kMaxPerRec + 1)));
    FEM_TRY(g->get(&g->pfine, n_recs));
    FEM_TRY(g->get(&g->sstep, n_recs));
    std::vector<int32_t> pfine_h(n_recs);
    const int64_t sumhi_max = (int64_t)(L - 1) * hi_max;
    std::vector<const uint32_t *> dens_h((size_t)n_recs * lo_vals.size());
    for (int r = 0; r < n_recs; ++r) {
        fem_stream *s = g->recs[r];
        FEM_TRY(stream_bytype(ctx, s));
        for (size_t j = 0; j < lo_vals.size(); ++j) {
            uint32_t *d = nullptr;
            FEM_TRY(stream_density(ctx, s, lo_vals[j], &d));
            dens_h[(size_t)r * lo_vals.size() + j] = d;
        }
        // finest segments: at least 256 events and twice the halo (sum of
        // the upper bounds, in events at the recording's mean rate)
        const double span = std::max(1.0, (double)s->t_last - (double)s->t_first);
        const double halo_ev = (double)s->n * (double)sumhi_max / span;
        const double min_seg = std::max(256.0, 2.0 * halo_ev);
        const int P = (int)std::max(1.0, std::min<double>(kMaxPerRec, (double)s->n / min_seg));
        pfine_h[r] = P;
        FEM_TRY(launch_segments(st, s->d_time, s->n, P, segs + (size_t)r * (kMaxPerRec + 1)));
        ri_h[r] = RecInfo{s->d_type, s->d_time, s->n, g->segl + (size_t)r * (kMaxPerRec + 1), 1, 0, 0,
                          s->d_freq, s->d_toff, s->d_ttime};
    }
    FEM_CUDA_TRY(cudaMemcpyAsync(g->pfine, pfine_h.data(), 4 * n_recs, cudaMemcpyHostToDevice, st));
    g->segf = segs;
    // (candidate, segment) threads per level: about two waves of the sparse
    // kernel, never more than target + live candidates (one segment each)
    g->target = (int64_t)2 * ctx->n_sm * 512;
    g->cap_threads = g->target + cap;
    const size_t free_b = ctx->budget > ctx->used.load() ? ctx->budget - ctx->used.load() : 0;
    if ((size_t)g->cap_threads * kRecWords * 4 > free_b / 4) return FEM_ERR_NOMEM;
    // ring entries per node: the largest window density of any type + 1
    // (capped at kRingCap; nodes needing more are flagged by the ring check)
    uint32_t dmax = 1;
    for (int r = 0; r < n_recs; ++r) {
        std::vector<uint32_t> hd(g->recs[r]->n_types);
        for (size_t j = 0; j < lo_vals.size(); ++j) {
            FEM_CUDA_TRY(cudaMemcpyAsync(hd.data(), dens_h[(size_t)r * lo_vals.size() + j], 4 * hd.size(),
                                         cudaMemcpyDeviceToHost, st));
            FEM_CUDA_TRY(cudaStreamSynchronize(st));
            for (uint32_t d : hd) dmax = std::max(dmax, d);
        }
    }
    g->ring_cap = (int)std::min<uint32_t>(kRingCap, dmax + 1);
    RecInfo *d_ri;
    const uint32_t **d_dens;
    int32_t *d_lov, *pos, *fb_list, *iota, *rec;
    int64_t *offs, *nthreads;
    uint16_t *ct;
    int32_t *cl, *ch;
    uint32_t *crec, *counts;
    const int Nmax = L;
    FEM_TRY(g->get(&d_ri, n_recs));
    FEM_TRY(g->get(&d_dens, dens_h.size()));
    FEM_TRY(g->get(&d_lov, lo_vals.size()));
    FEM_TRY(g->get(&pos, cap + 2));
    FEM_TRY(g->get(&fb_list, cap));
    FEM_TRY(g->get(&iota, cap));
    FEM_TRY(g->get(&rec, (size_t)g->cap_threads * kRecWords));
    FEM_TRY(g->get(&offs, cap + 1));
    FEM_TRY(g->get(&nthreads, 1));
    FEM_TRY(g->get(&ct, (size_t)cap * Nmax));
    FEM_TRY(g->get(&cl, (size_t)cap * (Nmax - 1)));
    FEM_TRY(g->get(&ch, (size_t)cap * (Nmax - 1)));
    FEM_TRY(g->get(&crec, cap));
    FEM_TRY(g->get(&counts, cap));
    FEM_TRY(g->get(&g->d_thr, n_recs));
    FEM_TRY(g->get(&g->ctr, (size_t)(L + 1) * kCtr));
    FEM_TRY(g->get(&g->coff, (size_t)(L + 1) * (n_recs + 1)));
    FEM_TRY(g->get(&g->rel, (size_t)(L + 1)));
    g->ev.assign(2 * (L + 1), nullptr);
    for (auto &e : g->ev) FEM_CUDA_TRY(cudaEventCreate(&e));
    g->F.assign(L + 1, FLevel{});
    for (int N = 2; N <= L; ++N) {
        FLevel &f = g->F[N];
        FEM_TRY(g->get(&f.types, (size_t)cap * N));
        FEM_TRY(g->get(&f.lo, (size_t)cap * (N - 1)));
        FEM_TRY(g->get(&f.hi, (size_t)cap * (N - 1)));
        FEM_TRY(g->get(&f.rec, cap));
        FEM_TRY(g->get(&f.counts, cap));
        FEM_TRY(g->get(&f.foff, n_recs + 1));
    }
    FEM_CUDA_TRY(cudaMemcpyAsync(d_ri, ri_h.data(), sizeof(RecInfo) * n_recs, cudaMemcpyHostToDevice, st));
    FEM_CUDA_TRY(cudaMemcpyAsync(d_dens, dens_h.data(), sizeof(void *) * dens_h.size(), cudaMemcpyHostToDevice, st));
    FEM_CUDA_TRY(cudaMemcpyAsync(d_lov, lo_vals.data(), 4 * lo_vals.size(), cudaMemcpyHostToDevice, st));
    FEM_CUDA_TRY(cudaMemcpyAsync(g->d_thr, thr.data(), 4 * n_recs, cudaMemcpyHostToDevice, st));
    int32_t *scan_tmp;
    FEM_TRY(g->get(&scan_tmp, (cap + 2) / 1024 + 2));
    FEM_CUDA_TRY(cudaStreamSynchronize(st));
    // smem attribute for the sparse kernels before capture
    for (int N = 3; N <= L; ++N) {
        const int nmax = N <= 2 ? 2 : N <= 4 ? 4 : N <= 8 ? 8 : 16;
        if ((size_t)(6 * (nmax - 1) + 2 * (N - 1) * g->ring_cap) * 64 * 4 > (size_t)ctx->smem_optin - 1024)
            return FEM_ERR_INVAL;
    }

    // ---- capture levels 3..L
    const unsigned gb = (unsigned)std::min<int64_t>((cap + 256) / 256, 4 * ctx->n_sm);
    cudaGraph_t graph = nullptr;
    FEM_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    int cst = FEM_OK;
    for (int N = 3; N <= L && cst == FEM_OK; ++N) {
        const int M = N - 1;
        const FLevel &pf = g->F[M];
        FLevel &nf = g->F[N];
        int32_t *cp = g->ctr + (size_t)M * kCtr;  // previous level's counters
        int32_t *cn = g->ctr + (size_t)N * kCtr;
        int64_t *coffN = g->coff + (size_t)N * (n_recs + 1);
        const int nmax = N <= 4 ? 4 : N <= 8 ? 8 : 16;
        if (cudaMemsetAsync(cn, 0, sizeof(int32_t) * kCtr, st) != cudaSuccess ||
            cudaMemsetAsync(g->rel + N, 0, sizeof(unsigned long long), st) != cudaSuccess)
            cst = FEM_ERR_CUDA;
        k_g_join_count<<<gb, 256, 0, st>>>(pf.types, pf.lo, pf.hi, pf.rec, pf.foff, cp, M, cap, pos);
        if (cst == FEM_OK) cst = scan_exclusive(st, pos, cap + 1, scan_tmp, nullptr, nullptr);
        k_g_join_write<<<gb, 256, 0, st>>>(pf.types, pf.lo, pf.hi, pf.rec, pf.foff, cp, M, cap, pos, ct, cl, ch, crec, cn);
        k_g_index<<<gb, 256, 0, st>>>(crec, cn, N, cap, offs, iota);
        k_g_recinfo<<<1, 256, 0, st>>>(crec, cn, n_recs, coffN, d_ri, nthreads, g->segf, g->pfine, g->sstep,
                                       g->segl, g->target);
        k_g_ringcheck<<<gb, 256, 0, st>>>(ct, cl, crec, cn, N, d_dens, d_lov, (int)lo_vals.size(), g->ring_cap, d_ri, cn,
                                          g->rel + N);
        // external event nodes: their timestamps time the count kernels of
        // this level on every launch of the graph
        if (cst == FEM_OK && cudaEventRecordWithFlags(g->ev[2 * N], st, cudaEventRecordExternal) != cudaSuccess)
            cst = FEM_ERR_CUDA;
        if (cst == FEM_OK)
            cst = launch_count_dev(st, nmax, N, g->ring_cap, d_ri, n_recs, nthreads, g->cap_threads, offs, ct, cl, ch, iota,
                                   crec, rec, cn, cap, counts, fb_list, cn + 3, d_dens, d_lov, (int)lo_vals.size());
        if (cst == FEM_OK && cudaEventRecordWithFlags(g->ev[2 * N + 1], st, cudaEventRecordExternal) != cudaSuccess)
            cst = FEM_ERR_CUDA;
        k_g_thr_flags<<<gb, 256, 0, st>>>(counts, crec, g->d_thr, cn, cap, pos);
        if (cst == FEM_OK) cst = scan_exclusive(st, pos, cap + 1, scan_tmp, nullptr, nullptr);
        k_g_thr_write<<<gb, 256, 0, st>>>(pos, counts, ct, cl, ch, crec, g->d_thr, N, cap, nf.types, nf.lo, nf.hi,
                                          nf.rec, nf.counts, cn);
        k_g_foff<<<1, 256, 0, st>>>(nf.rec, cn, n_recs, nf.foff);
        if (cst == FEM_OK && cudaGetLastError() != cudaSuccess) cst = FEM_ERR_CUDA;
    }
    const cudaError_t ce = cudaStreamEndCapture(st, &graph);
    if (cst != FEM_OK || ce != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return cst != FEM_OK ? cst : FEM_ERR_CUDA;
    }
    const cudaError_t ie = cudaGraphInstantiate(&g->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
        cudaGetLastError();
        g->exec = nullptr;
        return FEM_ERR_CUDA;
    }
    return FEM_OK;
}

static std::string tail_key(const std::vector<fem_stream *> &recs, const std::vector<int32_t> &blo,
                            const std::vector<int32_t> &bhi, const std::vector<uint32_t> &thr, int max_size,
                            int64_t cap) {
    std::ostringstream k;
    for (auto *s : recs) k << (const void *)s << ':' << s->n << ';';
    for (size_t i = 0; i < blo.size(); ++i) k << blo[i] << ',' << bhi[i] << ';';
    for (auto t : thr) k << t << ';';
    k << max_size << '/' << cap;
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
            delete it->second;
            it = ctx->graphs.erase(it);
        } else {
            ++it;
        }
    }
}

// Runs levels 3..max_size through the cached (or newly captured) graph,
// starting from the level-2 frequent set (device arrays + per-recording
// offsets).  Returns FEM_OK and fills `out` when every level completed
// without a flag; *used = false when the graph path did not apply (the
// caller then continues on the host-driven path).
int run_graph_tail(fem_ctx *ctx, const std::vector<fem_stream *> &recs, const std::vector<int32_t> &blo,
                   const std::vector<int32_t> &bhi, const std::vector<uint32_t> &thr, const std::vector<int32_t> &lo_vals,
                   int max_size, int64_t F2, const uint16_t *f2_types, const int32_t *f2_lo, const int32_t *f2_hi,
                   const uint32_t *f2_rec, const uint32_t *f2_counts, const std::vector<int64_t> &f2_off,
                   TailResult *out, bool *used) {
    *used = false;
    const int n_recs = (int)recs.size();
    if (max_size < 3 || F2 == 0) return FEM_OK;
    for (auto *s : recs)
        if (s->n_types > 8192 || s->n > INT32_MAX / 2) return FEM_OK;
    // capacity: the first join cannot exceed sum over recordings of F2_r^2
    int64_t bound = 0;
    for (int r = 0; r < n_recs; ++r) {
        const int64_t f = f2_off[r + 1] - f2_off[r];
        bound += f * f;
    }
    int64_t cap = 4096;
    while (cap < 2 * bound && cap < (1 << 18)) cap <<= 1;
    const std::string key = tail_key(recs, blo, bhi, thr, max_size, cap);
    GraphTail *g = nullptr;
    auto it = ctx->graphs.find(key);
    if (it != ctx->graphs.end()) {
        g = it->second;
    } else {
        if (ctx->graphs.size() >= 4) graph_cache_clear(ctx);
        std::unique_ptr<GraphTail> ng(new GraphTail());
        ng->ctx = ctx;
        ng->key = key;
        ng->recs = recs;
        ng->n_recs = n_recs;
        ng->max_size = max_size;
        ng->cap = cap;
        const int st = build_tail(ng.get(), blo, bhi, thr, lo_vals);
        if (st == FEM_ERR_NOMEM || st == FEM_ERR_INVAL) return FEM_OK;  // not applicable: host path
        if (st != FEM_OK) return st;
        g = ng.release();
        ctx->graphs[key] = g;
    }
    if (F2 > g->cap) return FEM_OK;
    // level-2 frequent set into the graph's input buffers
    cudaStream_t st = ctx->stream;
    FLevel &f2 = g->F[2];
    FEM_CUDA_TRY(cudaMemcpyAsync(f2.types, f2_types, 2 * 2 * F2, cudaMemcpyDeviceToDevice, st));
    FEM_CUDA_TRY(cudaMemcpyAsync(f2.lo, f2_lo, 4 * F2, cudaMemcpyDeviceToDevice, st));
    FEM_CUDA_TRY(cudaMemcpyAsync(f2.hi, f2_hi, 4 * F2, cudaMemcpyDeviceToDevice, st));
    FEM_CUDA_TRY(cudaMemcpyAsync(f2.rec, f2_rec, 4 * F2, cudaMemcpyDeviceToDevice, st));
    FEM_CUDA_TRY(cudaMemcpyAsync(f2.counts, f2_counts, 4 * F2, cudaMemcpyDeviceToDevice, st));
    FEM_CUDA_TRY(cudaMemcpyAsync(f2.foff, f2_off.data(), 8 * (n_recs + 1), cudaMemcpyHostToDevice, st));
    std::vector<int32_t> c2(kCtr, 0);
    c2[1] = (int32_t)F2;
    FEM_CUDA_TRY(cudaMemcpyAsync(g->ctr + 2 * kCtr, c2.data(), 4 * kCtr, cudaMemcpyHostToDevice, st));
    cudaEventRecord(ctx->ev0, st);
    FEM_CUDA_TRY(cudaGraphLaunch(g->exec, st));
    cudaEventRecord(ctx->ev1, st);
    std::vector<int32_t> ctr((size_t)(max_size + 1) * kCtr);
    std::vector<int64_t> coff((size_t)(max_size + 1) * (n_recs + 1));
    FEM_CUDA_TRY(cudaMemcpyAsync(ctr.data(), g->ctr, 4 * ctr.size(), cudaMemcpyDeviceToHost, st));
    FEM_CUDA_TRY(cudaMemcpyAsync(coff.data(), g->coff, 8 * coff.size(), cudaMemcpyDeviceToHost, st));
    std::vector<unsigned long long> rel((size_t)max_size + 1, 0ull);
    FEM_CUDA_TRY(cudaMemcpyAsync(rel.data(), g->rel, 8 * rel.size(), cudaMemcpyDeviceToHost, st));
    FEM_TRY(sync_status(ctx));
    for (int N = 3; N <= max_size; ++N) {
        const int32_t *c = &ctr[(size_t)N * kCtr];
        if (c[2] != 0 || c[3] != 0) return FEM_OK;  // flagged: redo on the host path
    }
    float gms = 0.f;
    cudaEventElapsedTime(&gms, ctx->ev0, ctx->ev1);
    out->graph_ms = gms;
    // count-kernel time of the levels from the graph's event nodes (the whole
    // graph's time if the driver cannot time them)
    float cms = 0.f;
    bool timed = true;
    for (int N = 3; N <= max_size && timed; ++N) {
        float m = 0.f;
        if (cudaEventElapsedTime(&m, g->ev[2 * N], g->ev[2 * N + 1]) != cudaSuccess) timed = false;
        cms += m;
    }
    if (!timed) cudaGetLastError();
    out->count_ms = timed ? cms : gms;
    out->relevant = 0.0;
    for (int N = 3; N <= max_size; ++N) out->relevant += (double)rel[N];
    // results
    out->levels.clear();
    for (int N = 3; N <= max_size; ++N) {
        const int32_t *c = &ctr[(size_t)N * kCtr];
        TailLevel tl;
        tl.N = N;
        tl.C = c[0];
        tl.coff.assign(coff.begin() + (size_t)N * (n_recs + 1), coff.begin() + (size_t)(N + 1) * (n_recs + 1));
        const int64_t Fn = c[1];
        tl.types.resize((size_t)Fn * N);
        tl.lo.resize((size_t)Fn * (N - 1));
        tl.hi.resize((size_t)Fn * (N - 1));
        tl.rec.resize(Fn);
        tl.counts.resize(Fn);
        if (Fn > 0) {
            const FLevel &f = g->F[N];
            FEM_CUDA_TRY(cudaMemcpyAsync(tl.types.data(), f.types, 2 * tl.types.size(), cudaMemcpyDeviceToHost, st));
            FEM_CUDA_TRY(cudaMemcpyAsync(tl.lo.data(), f.lo, 4 * tl.lo.size(), cudaMemcpyDeviceToHost, st));
            FEM_CUDA_TRY(cudaMemcpyAsync(tl.hi.data(), f.hi, 4 * tl.hi.size(), cudaMemcpyDeviceToHost, st));
            FEM_CUDA_TRY(cudaMemcpyAsync(tl.rec.data(), f.rec, 4 * tl.rec.size(), cudaMemcpyDeviceToHost, st));
            FEM_CUDA_TRY(cudaMemcpyAsync(tl.counts.data(), f.counts, 4 * tl.counts.size(), cudaMemcpyDeviceToHost, st));
        }
        out->levels.push_back(std::move(tl));
        if (c[0] == 0 || Fn == 0) break;
    }
    FEM_CUDA_TRY(cudaStreamSynchronize(st));
    *used = true;
    return FEM_OK;
}

}  // namespace fem
